// internal.h -- declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>
#include "sweep.cuh"

namespace oais {

// A target in the device layout the kernels read: X zero-padded to D columns
// (D = the compiled width), rows padded to a multiple of 4, fp64 for the
// Gaussian family and fp32 otherwise.
struct DevTarget {
    int kind = 0;
    int d = 0, D = 0, n = 0, n_pad = 0;
    double ref_scale = 1.0, p0 = 1.0;
    void* X = nullptr;   // GAUSS: double[D]; GMM: float[n][D]; rows: float[n_pad][D]
    void* y = nullptr;   // rows: float[n_pad]
    bool tc = false;     // tensor-core form: BF16 image of X and label bits below
    void* tc_img = nullptr;
    uint32_t* tc_ybits = nullptr;
    int* tc_handed = nullptr;    // [tiles] hand-off flags of the persistent schedules (resident and streamed forms)
    bool tcs = false;    // streamed tensor-core form: chunk images of X~ (and y), particle state
    void* tcs_img = nullptr;
    float* tcs_state = nullptr;
    bool tcs_q8 = false; // the streamed form's X is stored as FP8 e4m3 with per-row scales
    int tcs_dp = 0;      // padded width of the streamed form's chunk images
    const float* fsched = nullptr;   // fp32 roundings of the running schedule (GmmTarget::fsched)
    bool wide = false;   // plain FP32 form for 32 < d <= 256 (D = 64, 128 or 256): X [n_pad][D]
    float* wide_state = nullptr;   // positions, gradients, momenta [3][D][tiles * 64]
};

// Plain FP32 CUDA-core form for the row families at 32 < d <= 256 (sweep_wide.cu): tiles of 64
// particles, one CTA each; the state width D = wide_width(d)
int wide_width(int d);
int wide_tiles(int64_t N);
size_t wide_state_bytes(int D, int64_t N);
cudaError_t launch_sweep_wide(const DevTarget& t, int move, const SweepParams& sp, cudaStream_t s);
cudaError_t launch_potential_wide(const DevTarget& t, const float* x, int64_t N, double* ell, float* grad,
                                  cudaStream_t s);

// Streamed tensor-core sweep (sweep_tcs.cu): sizes of one configuration.  dp = d padded to
// 16, 32 or a multiple of 64 (at most 256); X~ is cut into nch chunks of `chunk` rows, each
// a stage image of stage_bytes (X~ lines in the swizzled K-major layout, then y for linear
// regression); shared memory holds the A operand (two terms) and `stages` chunk buffers;
// TMEM holds two forward accumulators, two per-row factor buffers and the gradient sum.
struct TcsPlan {
    int dp = 0, chunk = 0, nch = 0, stages = 0, tmem_cols = 0;
    uint32_t y_off = 0, stage_bytes = 0, off_x = 0, off_misc = 0, smem = 0;
    bool q8 = false;                     // FP8 e4m3 storage of X with per-row scales
    int h = 2;                           // column groups per lane quarter (particle warps / 4)
    int stages8 = 0;
    uint32_t off_x8 = 0, stage8_bytes = 0;
    size_t img_bytes = 0;
    bool ok = false;
};
// dp > 0 forces the padded width (a context keeps the width its chunk images were made for)
TcsPlan tcs_plan(int kind, int n, int d, int chunk, int stages, bool q8 = false, int h = 0, int dp = 0);
// grid of a per-step kernel that usually returns at once (the resampling kernels): at most
// per_sm CTAs per SM, the work taken grid-stride
int capped_grid(int64_t want, int per_sm);
// chunk rows a plan may take (the single-problem kernels: the default only; the batched kernel
// also 32 and 128 for logistic problems with d_pad <= 64)
bool tcs_chunk_ok(int kind, int dp, int chunk, bool q8);
// bytes of a context's chunk images: the plan's, padded with zero rows to a multiple of 128
// rows where the problem may run 128-row chunks
size_t tcs_image_bytes(const TcsPlan& L, int kind, int n);
void tcs_prepare(const TcsPlan& L, int kind, const float* X, const float* y, int n, int d,
                 std::vector<unsigned char>& img);
void tcs_prepare_q8(const TcsPlan& L, const float* X, const float* y, int n, int d, std::vector<unsigned char>& img);
int tcs_tiles(int64_t N);
// state: 5 arrays [dp][tiles * 128] fp32 (accepted x, its gradient, proposal, momentum,
// drained gradient sum)
// handed: [tiles] hand-off flags (nullable): with more tiles than CTAs resident at once the
// sweep runs as a persistent grid with the wrap-around schedule over tiles x steps
cudaError_t launch_sweep_tcs(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state,
                             int move, int leapfrog, double p0, int n, int d, cudaStream_t s,
                             int* handed = nullptr);
// batched persistent form: per-problem parameter blocks (opaque, tcs_params_bytes each) whose
// Misc region sits at the common offset off_misc, a queue of (problem, tile) items, a head
// counter (zero before the launch), one CTA per SM
size_t tcs_params_bytes();
uint32_t tcs_misc_bytes();
void tcs_batch_params(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state, int move,
                      int leapfrog, double p0, int n, int d, uint32_t off_misc, void* out);
cudaError_t launch_sweep_tcs_batch(int kind, int h, const void* d_params, const void* d_items, uint32_t n_items,
                                   uint32_t* d_head, uint32_t off_misc, uint32_t smem, int grid, cudaStream_t s,
                                   bool alt_chunks = false);
// ASMC on the streamed form: step t (t = 0: the draw from eta) of the whole population, with
// the tiles' (log w, 2 log w) records in ess_parts; then the resampling test, scan and CDF of
// asmc.cu (decide/scan/cdf, no gather) and launch_gather_tcs for the particle state
cudaError_t launch_step_tcs(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state,
                            int move, int leapfrog, double p0, int n, int d, int t, StepPartial* ess_parts,
                            cudaStream_t s);
cudaError_t launch_gather_tcs(const TcsPlan& L, const AsmcState* st, const double* cdf, int64_t N, float* state,
                              double* ell, double* ell_scratch, double* logw, int64_t* ancestors, cudaStream_t s);
// the ESS pieces' buffer (StepParams::ess_parts) holds nparts pieces and then
// asmc_ess_groups(nparts) group records of the two-level merge
int asmc_ess_groups(int nparts);
cudaError_t launch_asmc_decide_scan(AsmcState* st, const StepParams& P, int nparts, double ess_frac, double* bsum,
                                    double* boff, double* cdf, double* ess_trace, int* resampled, cudaStream_t s);
// one evaluation of log L and grad log L (grad may be null) at states x [d][N] with the
// streamed tensor-core contraction
cudaError_t launch_potential_tcs(const TcsPlan& L, int kind, const void* img, const float* x, int64_t N,
                                 double* ell, float* grad, double p0, int n, int d, unsigned* status,
                                 float* state, int64_t state_particles, cudaStream_t s);

// tensor-core logistic sweep (sweep_tc.cu)
int tc_grid(int64_t N);
int tc_records(int64_t N);
// Online conditional-ESS schedule (zja.cu): line-search state of the current step
struct ZjaState {
    double lo, hi;       // bracket of delta = beta_t - beta_{t-1}
    double beta_prev;    // beta_{t-1}
    int done;            // 1: beta_t fixed (the pass and narrow kernels return at once)
    int skip;            // 1: beta reached 1 at an earlier step (this step does nothing)
};
int zja_grid(int64_t N);
size_t zja_part_bytes(int64_t N);
cudaError_t launch_zja_search(ZjaState* zs, const AsmcState* st, const StepParams& P, float2* fg, double2* anchor,
                              float2* part, double cess_frac, int t, int T_max, double* beta, double* eps,
                              const double* beta_ref, const double* eps_ref, int T_ref, cudaStream_t s);

cudaError_t launch_sweep_tc(const SweepParams& sp, const void* Ximg, const uint32_t* ybits, int n, int d,
                            float* grad_state, int* handed, cudaStream_t s);

// log w += ell_x - ell, ell = ell_x (the final reweighting from X~ to X of the tensor-core forms)
cudaError_t launch_reweight_to_data(double* logw, double* ell, const double* ell_x, int64_t N, unsigned* status,
                                    cudaStream_t s);

// records m as the calling thread's error text for calls without a context
// (oais_last_error(NULL)) and returns s; the status is an oais_status value
int fail_call(int s, const char* m);

// smallest compiled width >= d for the family, 0 if none
int padded_width(int kind, int d);

// launch the sweep for one family; grid = oais_sweep_blocks(P.N)
cudaError_t launch_sweep_gauss(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_unid(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_logreg(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_gmm(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);
cudaError_t launch_sweep_linreg(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s);

// ASMC: init (t = 0) or one annealing step, per family
cudaError_t launch_asmc_gauss(const DevTarget& t, int move, bool init, const StepParams& P, cudaStream_t s);
cudaError_t launch_asmc_unid(const DevTarget& t, int move, bool init, const StepParams& P, cudaStream_t s);
cudaError_t launch_asmc_logreg(const DevTarget& t, int move, bool init, const StepParams& P, cudaStream_t s);
cudaError_t launch_asmc_gmm(const DevTarget& t, int move, bool init, const StepParams& P, cudaStream_t s);
cudaError_t launch_asmc_linreg(const DevTarget& t, int move, bool init, const StepParams& P, cudaStream_t s);

// log L and grad log L for a batch of states, per family
cudaError_t launch_potential_gauss(const DevTarget& t, const PotentialParams& P, cudaStream_t s);
cudaError_t launch_potential_unid(const DevTarget& t, const PotentialParams& P, cudaStream_t s);
cudaError_t launch_potential_logreg(const DevTarget& t, const PotentialParams& P, cudaStream_t s);
cudaError_t launch_potential_gmm(const DevTarget& t, const PotentialParams& P, cudaStream_t s);
cudaError_t launch_potential_linreg(const DevTarget& t, const PotentialParams& P, cudaStream_t s);

inline int sweep_grid(int64_t N) { return (int)((N + kSweepThreads - 1) / kSweepThreads); }

template <class Kern, class Params, class Tgt>
cudaError_t launch_kernel(Kern* k, const Tgt& tg, size_t smem, const Params& P, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<sweep_grid(P.N), kSweepThreads, smem, s>>>(P, tg);
    return cudaGetLastError();
}

// generic launchers used by the per-family translation units
template <class Tgt, int MOVE, int D, typename R>
cudaError_t launch_one(const Tgt& tg, size_t smem, const SweepParams& P, cudaStream_t s)
{
    return launch_kernel(&oais_sweep_kernel<Tgt, MOVE, D, R>, tg, smem, P, s);
}

template <class Tgt, int MOVE, int D, typename R>
cudaError_t launch_one(const Tgt& tg, size_t smem, const StepParams& P, bool init, cudaStream_t s)
{
    if (init) return launch_kernel(&asmc_init_kernel<Tgt, MOVE, D, R>, tg, smem, P, s);
    return launch_kernel(&asmc_step_kernel<Tgt, MOVE, D, R>, tg, smem, P, s);
}

// the potential kernel does not depend on the move: every MOVE maps to one instantiation
template <class Tgt, int MOVE, int D, typename R>
cudaError_t launch_one(const Tgt& tg, size_t smem, const PotentialParams& P, cudaStream_t s)
{
    return launch_kernel(&potential_kernel<Tgt, D, R>, tg, smem, P, s);
}

// one family's dispatch over (move, width) for both kernel kinds
// targets that carry the launch's random-number generator take it from the move configuration
template <class TG, class P> inline void bind_rng(TG&, const P&) {}
template <typename R, int D> inline void bind_rng(GmmTarget<R, D>& tg, const SweepParams& p) { tg.rks.set(p.mv.rng); }
template <typename R, int D> inline void bind_rng(GmmTarget<R, D>& tg, const StepParams& p) { tg.rks.set(p.mv.rng); }

#define OAIS_FAMILY_DISPATCH(FAM, MAKE, R, ...)                                                  \
    template <int D, class P, class... A>                                                        \
    static cudaError_t go(const DevTarget& t, int move, const P& prm, cudaStream_t s, A... a)   \
    {                                                                                            \
        size_t smem = 0;                                                                         \
        auto tg = MAKE<D>(t, &smem);                                                             \
        bind_rng(tg, prm);                                                                       \
        using TG = decltype(tg);                                                                 \
        switch (move) {                                                                          \
        case kRwmh: return launch_one<TG, kRwmh, D, R>(tg, smem, prm, a..., s);                  \
        case kMala: return launch_one<TG, kMala, D, R>(tg, smem, prm, a..., s);                  \
        case kHmc:  return launch_one<TG, kHmc, D, R>(tg, smem, prm, a..., s);                   \
        }                                                                                        \
        return cudaErrorInvalidValue;                                                            \
    }                                                                                            \
    template <class P, class... A>                                                               \
    static cudaError_t by_width(const DevTarget& t, int move, const P& prm, cudaStream_t s, A... a) \
    {                                                                                            \
        switch (t.D) {                                                                           \
        __VA_ARGS__                                                                              \
        }                                                                                        \
        return cudaErrorInvalidValue;                                                            \
    }                                                                                            \
    cudaError_t launch_sweep_##FAM(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s) \
    {                                                                                            \
        return by_width(t, move, P, s);                                                          \
    }                                                                                            \
    cudaError_t launch_asmc_##FAM(const DevTarget& t, int move, bool init, const StepParams& P,  \
                                  cudaStream_t s)                                                \
    {                                                                                            \
        return by_width(t, move, P, s, init);                                                    \
    }                                                                                            \
    cudaError_t launch_potential_##FAM(const DevTarget& t, const PotentialParams& P, cudaStream_t s) \
    {                                                                                            \
        return by_width(t, (int)kRwmh, P, s);                                                    \
    }

#define OAIS_WIDTH(W) case W: return go<W>(t, move, prm, s, a...);

} // namespace oais
