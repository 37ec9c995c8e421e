// sweep_tcs.cu -- the loop-swapped OAIS sweep (Sec. 5.1.2) with the likelihood contraction on
// the tensor cores and the data streamed from global memory: any number of rows n, state
// dimension up to 256, logistic regression and Bayesian linear regression, MALA or HMC moves
// (Sec. 2.1.1 kernel family, identity mass).
//
// A CTA owns a tile of 128 particles (the tcgen05 M = 128 lane layout).  For each evaluation
// of log L and grad log L at the tile's current positions P it streams X in chunks of CHUNK
// rows:
//   forward   Z   = P X_c^T          (M = 128, N = CHUNK, K = d)        into TMEM D1[c % 2]
//   epilogue  per element: linear regression r = y - z, sum r^2;
//             logistic (label sign folded into X) u = s z, log sigmoid(u), sigmoid(-u)
//   backward  G  += R X_c            (M = 128, N = d,     K = CHUNK)    into TMEM D2
// Operands are f16: the data X~ (X rounded to bf16, then stored exactly as f16; values below
// 2^-17 in magnitude take the nearest f16) and the two-term split v = hi + lo of the
// positions and of the per-row factors R (hi = f16(v), lo = f16(v - hi): relative error about
// 2^-22, far below the posterior scale even at n = 50 000).  Accumulation is fp32 in TMEM;
// sums over rows of the epilogue terms are fp32 per chunk and fp64 across chunks.
//
// Roles (352 threads):
//   warps 0-7  particle warps: thread (warp w, lane l) owns particle 32 (w % 4) + l (its TMEM
//              lane) and the coordinate half w / 4 and column half w / 4 of every chunk
//   warp 8     one thread issues the forward MMAs, warp 10 one thread the backward MMAs
//   warp 9     one thread streams the chunk images (X~ in the swizzled shared-memory layout and
//              y) with bulk copies into a ring of STAGES buffers
// Synchronisation is by mbarriers; every wait is bounded (2 s), after which the CTA sets
// status bit 2, stops issuing work and runs to its end without blocking.
//
// Particle state between evaluations lives in global memory (L2): accepted position and
// gradient, proposal position and momentum, [d_pad][N_pad] fp32 each, read and written only
// by the thread that owns the (particle, coordinate) pair.
#include <algorithm>

#include "sweep_tcs.cuh"

namespace oais {

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
namespace {
int padded_dim(int d)
{
    if (d <= 16) return 16;
    if (d <= 32) return 32;
    return (d + 63) / 64 * 64;
}
uint32_t align1024(uint32_t v) { return (v + 1023u) & ~1023u; }
} // namespace

TcsPlan tcs_plan(int kind, int n, int d, int chunk, int stages, bool q8, int h, int dp)
{
    TcsPlan L{};
    L.q8 = q8;
    L.dp = dp > 0 ? dp : padded_dim(d);
    // column split: two column groups per lane quarter (8 particle warps).  Four groups (16
    // warps, a quarter of each chunk's columns per thread) were measured slower on the logistic
    // workload: the per-chunk synchronisation is paid for half the work and the register cap
    // drops to 96; the split stays a template parameter of the kernel.
    L.h = h > 0 ? h : 2;
    L.chunk = chunk > 0 ? chunk : tcs::chunk_rows(L.dp);
    L.nch = (n + L.chunk - 1) / L.chunk;
    L.y_off = (uint32_t)L.chunk * L.dp * 2;
    // f16 stage: lines, y (linear regression), and with FP8 storage the row scales
    const uint32_t tail = (kind == kLinreg ? (uint32_t)L.chunk * 4 : 0u) * (q8 ? 2u : 1u);
    L.stage_bytes = align1024(L.y_off + tail);
    const uint32_t a_bytes = (uint32_t)tcs::kTile * L.dp * 2;   // hi term of the positions
    L.off_x = a_bytes;
    const uint32_t limit = 227u * 1024u;
    const uint32_t misc = (uint32_t)((sizeof(tcs::Misc) + 1023) & ~(size_t)1023);
    if (q8) {
        // FP8 chunk image (q rows, y, s) ring: three buffers, the rest to the f16 ring
        L.stage8_bytes = align1024((uint32_t)L.chunk * L.dp + 2u * (uint32_t)L.chunk * 4u);
        L.stages8 = 3;
    }
    const uint32_t ring8 = (uint32_t)L.stages8 * L.stage8_bytes;
    int S = stages > 0 ? stages : 8;
    while (S > 2 && L.off_x + (uint32_t)S * L.stage_bytes + ring8 + misc > limit) --S;
    L.stages = S;
    L.off_x8 = L.off_x + (uint32_t)S * L.stage_bytes;
    L.off_misc = L.off_x8 + ring8;
    L.smem = L.off_misc + (uint32_t)sizeof(tcs::Misc);
    L.tmem_cols = 512;
    // 512 TMEM columns leave room for one CTA per SM: make the shared memory say so too
    if (L.tmem_cols == 512 && L.smem < 120u * 1024u) L.smem = 120u * 1024u;
    L.img_bytes = (size_t)L.nch * (q8 ? L.stage8_bytes : L.stage_bytes);
    L.ok = L.dp <= 256 && tcs_chunk_ok(kind, L.dp, L.chunk, q8) && L.smem <= limit && L.stages >= 2 &&
           L.stages <= 8 && L.h == 2;
    return L;
}

size_t tcs_image_bytes(const TcsPlan& L, int kind, int n)
{
    // room for the chunk images at every chunk size the batched launch may give the problem:
    // 128-row chunks read up to 64 zero rows past a 64-row plan's last chunk
    if (!tcs_chunk_ok(kind, L.dp, 128, L.q8)) return L.img_bytes;
    const size_t rows128 = (size_t)(n + 127) / 128 * 128;
    return std::max(L.img_bytes, rows128 * (size_t)L.dp * 2);
}

bool tcs_chunk_ok(int kind, int dp, int chunk, bool q8)
{
    // 64 rows (32 at d_pad = 256 if so compiled); the batched launch also takes 128-row chunks
    // for logistic problems with d_pad <= 64: their chunk images are the rows of X~ in order
    // (one K slab, no y lines), so the same image serves both chunk sizes.  (32-row chunks for
    // the same problems were built and measured slower than 64 in every width class.)
    return chunk == tcs::chunk_rows(dp) || (!q8 && kind == kLogreg && dp <= 64 && chunk == 128);
}

// X~ = f16(bf16(X)) in the stage layout (logistic: rows multiplied by the label sign), and y
static uint16_t f16_of_bf16(float v)
{
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even bf16 (finite inputs)
    u &= 0xFFFF0000u;
    float b;
    std::memcpy(&b, &u, 4);
    const __half h = __float2half_rn(b);
    uint16_t r;
    std::memcpy(&r, &h, 2);
    return r;
}

void tcs_prepare(const TcsPlan& L, int kind, const float* X, const float* y, int n, int d,
                 std::vector<unsigned char>& img)
{
    img.assign(L.img_bytes, 0);
    const tcs::KLayout K = tcs::klayout(L.dp);
    for (int r = 0; r < n; ++r) {
        const int c = r / L.chunk, rr = r % L.chunk;
        unsigned char* st = img.data() + (size_t)c * L.stage_bytes;
        const bool neg = kind == kLogreg && !(y[r] > 0.5f);
        for (int i = 0; i < d; ++i) {
            uint16_t hbits = f16_of_bf16(X[(size_t)r * d + i]);
            if (neg) hbits ^= 0x8000u;
            const uint32_t off = tcs::kmaj_off(rr, i & ~7, L.chunk, K) + (uint32_t)(i & 7) * 2;
            std::memcpy(st + off, &hbits, 2);
        }
        if (kind == kLinreg) std::memcpy(st + L.y_off + (size_t)rr * 4, &y[r], 4);
    }
}

// e4m3 (bias 7, three mantissa bits, subnormal quantum 2^-9, largest 448) nearest to a finite
// |v| <= 448, ties to even
static uint8_t e4m3_rn(float v)
{
    const uint8_t sign = std::signbit(v) ? 0x80u : 0u;
    const double a = std::fabs((double)v);
    if (a == 0.0) return sign;
    int e = 0;
    std::frexp(a, &e);                         // a in [2^(e-1), 2^e)
    int E = std::max(e - 1, -6);               // below 2^-6: the subnormal quantum 2^-9
    double r = std::nearbyint(std::ldexp(a, -(E - 3)));   // a / quantum, ties to even
    if (r >= 16.0) { ++E; r = 8.0; }
    if (r < 8.0) return sign | (uint8_t)r;     // subnormal (E == -6)
    uint32_t ex = (uint32_t)(E + 7), mant = (uint32_t)r - 8u;
    if (ex > 15u || (ex == 15u && mant > 6u)) { ex = 15u; mant = 6u; }
    return sign | (uint8_t)(ex << 3) | (uint8_t)mant;
}

// FP8 chunk images: per row r the scale s_r = max_j |X_rj| / 448 (1 for a zero row, fp32) and
// q_rj = e4m3(X_rj / s_r); per chunk [q rows (d_pad bytes each) | y | s]
void tcs_prepare_q8(const TcsPlan& L, const float* X, const float* y, int n, int d, std::vector<unsigned char>& img)
{
    img.assign(L.img_bytes, 0);
    for (int r = 0; r < n; ++r) {
        const int c = r / L.chunk, rr = r % L.chunk;
        unsigned char* st = img.data() + (size_t)c * L.stage8_bytes;
        float mx = 0.0f;
        for (int i = 0; i < d; ++i) mx = std::max(mx, std::fabs(X[(size_t)r * d + i]));
        const float sc = mx > 0.0f ? mx / 448.0f : 1.0f;
        for (int i = 0; i < d; ++i) st[(size_t)rr * L.dp + i] = e4m3_rn(X[(size_t)r * d + i] / sc);
        std::memcpy(st + (size_t)L.chunk * L.dp + (size_t)rr * 4, &y[r], 4);
        std::memcpy(st + (size_t)L.chunk * L.dp + (size_t)(L.chunk + rr) * 4, &sc, 4);
    }
}

int tcs_tiles(int64_t N) { return (int)((N + tcs::kTile - 1) / tcs::kTile); }

static void fill_params(tcs::Params& P, const TcsPlan& L, int kind, const SweepParams& sp, const void* img,
                        float* state, int move, int leapfrog, double p0, int n, int d, const float* x_in,
                        double* ell_pot, float* grad_pot, int64_t pstride, int64_t state_particles)
{
    P.sp = sp;
    P.t_begin = 1;          // the OAIS sweep: x_0 ~ eta, then steps 1..T
    P.t_end = sp.T;
    P.resume = 0;
    P.ess_parts = nullptr;
    P.span = 0;
    P.tiles = tcs_tiles(sp.N);
    P.handed = nullptr;
    P.x_in = x_in;
    P.ell_pot = ell_pot;
    P.grad_pot = grad_pot;
    P.pstride = pstride;
    P.seg = tcs::kSegMmas / (L.chunk / 8);
    P.chunk = L.chunk;
    P.img = static_cast<const unsigned char*>(img);
    const int tiles = tcs_tiles(sp.N);
    P.Np = state_particles > 0 ? state_particles : (int64_t)tiles * tcs::kTile;
    // state: [xa | ga | xp | mom | gs], each [dp][Np]; the potential uses only gs
    P.xa = state;
    P.ga = state + (size_t)L.dp * P.Np;
    P.xp = state + (size_t)2 * L.dp * P.Np;
    P.mom = state + (size_t)3 * L.dp * P.Np;
    P.gs = state + (size_t)4 * L.dp * P.Np;
    P.n = n;
    P.d = d;
    P.dp = L.dp;
    P.nch = L.nch;
    P.stages = L.stages;
    P.stage_bytes = L.stage_bytes;
    P.y_off = L.y_off;
    P.off_x8 = L.off_x8;
    P.stage8_bytes = L.stage8_bytes;
    P.stages8 = L.stages8;
    P.off_x = L.off_x;
    P.off_misc = L.off_misc;
    P.tmem_cols = (uint32_t)L.tmem_cols;
    P.move = move;
    P.leapfrog = leapfrog;
    P.log_norm = kind == kLinreg ? (double)n * (std::log(p0) + 0.5 * std::log(2.0 * 3.14159265358979323846)) : 0.0;
    P.gscale = kind == kLinreg ? (float)(1.0 / (p0 * p0)) : 1.0f;
    P.half_inv_var = kind == kLinreg ? (float)(0.5 / (p0 * p0)) : 0.0f;
}

static cudaError_t launch_tcs(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state,
                              int move, int leapfrog, double p0, int n, int d, const float* x_in, double* ell_pot,
                              float* grad_pot, int64_t pstride, cudaStream_t s, int64_t state_particles = 0,
                              int t_begin = 1, int t_end = -1, int resume = 0, StepPartial* ess_parts = nullptr,
                              int* handed = nullptr)
{
    tcs::Params P;
    fill_params(P, L, kind, sp, img, state, move, leapfrog, p0, n, d, x_in, ell_pot, grad_pot, pstride,
                state_particles);
    if (t_end >= 0) {
        P.t_begin = t_begin;
        P.t_end = t_end;
        P.resume = resume;
        P.ess_parts = ess_parts;
    }
    const int tiles = tcs_tiles(sp.N);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        if (e != cudaSuccess) return e;
        const int threads = tcs::Roles<2>::threads(L.q8 ? 1 : 0);
        // the OAIS sweep with more tiles than CTAs resident at once: a persistent grid with the
        // wrap-around schedule (every CTA resident: a cooperative launch, since a CTA may wait
        // for another's hand-off)
        int per_sm = 0, dev = 0, sms = 0;
        if (handed && !x_in && t_end < 0) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, L.smem);
            if (e == cudaSuccess) e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
        }
        const int resident = per_sm * sms;
        if (resident > 0 && tiles > resident && sp.T > 0) {
            P.span = std::max<int64_t>(sp.T, ((int64_t)tiles * sp.T + resident - 1) / resident);
            P.handed = handed;
            e = cudaMemsetAsync(handed, 0, sizeof(int) * (size_t)tiles, s);
            if (e != cudaSuccess) return e;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(resident);
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = L.smem;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, kern, P);
            if (e != cudaSuccess) return e;
            return cudaGetLastError();
        }
        kern<<<tiles, threads, L.smem, s>>>(P);
        return cudaGetLastError();
    };
    if (L.chunk != tcs::chunk_rows(L.dp)) return cudaErrorInvalidValue;
    if (L.q8) {
        if (kind != kLinreg || L.h != 2) return cudaErrorInvalidValue;
        switch (L.dp) {
        case 16: return go(tcs::oais_sweep_tcs_kernel<kLinreg, 16, 1, 2>);
        case 32: return go(tcs::oais_sweep_tcs_kernel<kLinreg, 32, 1, 2>);
        case 64: return go(tcs::oais_sweep_tcs_kernel<kLinreg, 64, 1, 2>);
        case 128: return go(tcs::oais_sweep_tcs_kernel<kLinreg, 128, 1, 2>);
        case 256: return go(tcs::oais_sweep_tcs_kernel<kLinreg, 256, 1, 2>);
        }
        return cudaErrorInvalidValue;
    }
    if (L.h != 2) return cudaErrorInvalidValue;
#define OAIS_TCS_DP(FAMK, DPV) case DPV: return go(tcs::oais_sweep_tcs_kernel<FAMK, DPV, 0, 2>);
    if (kind == kLinreg) {
        switch (L.dp) {
        OAIS_TCS_DP(kLinreg, 16) OAIS_TCS_DP(kLinreg, 32) OAIS_TCS_DP(kLinreg, 64)
        OAIS_TCS_DP(kLinreg, 128) OAIS_TCS_DP(kLinreg, 256)
        }
    } else {
        switch (L.dp) {
        OAIS_TCS_DP(kLogreg, 16) OAIS_TCS_DP(kLogreg, 32) OAIS_TCS_DP(kLogreg, 64)
        OAIS_TCS_DP(kLogreg, 128) OAIS_TCS_DP(kLogreg, 256)
        }
    }
#undef OAIS_TCS_DP
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_tcs(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state,
                             int move, int leapfrog, double p0, int n, int d, cudaStream_t s, int* handed)
{
    return launch_tcs(L, kind, sp, img, state, move, leapfrog, p0, n, d, nullptr, nullptr, nullptr, 0, s, 0, 1, -1,
                      0, nullptr, handed);
}

cudaError_t launch_step_tcs(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state,
                            int move, int leapfrog, double p0, int n, int d, int t, StepPartial* ess_parts,
                            cudaStream_t s)
{
    // t = 0: x_0 ~ eta and its evaluation; t >= 1: step t from the stored state
    return launch_tcs(L, kind, sp, img, state, move, leapfrog, p0, n, d, nullptr, nullptr, nullptr, 0, s, 0,
                      t == 0 ? 1 : t, t == 0 ? 0 : t, t == 0 ? 0 : 1, t == 0 ? nullptr : ess_parts);
}

// systematic resampling of the streamed form's particles (after asmc_decide / scan / cdf):
// the ancestor rows of position and gradient go to the scratch arrays, then back
__global__ void __launch_bounds__(256)
tcs_gather_kernel(const AsmcState* st, const double* __restrict__ cdf, int64_t N, int64_t Np, int dp,
                  const float* __restrict__ xa, const float* __restrict__ ga, float* xs, float* gs,
                  const double* __restrict__ ell, double* ell_s, double* logw, int64_t* ancestors)
{
    if (!st->pend) return;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const double thr = ((double)n + st->U) / (double)N;
        int64_t lo = 0, hi = N - 1;   // a = min{m : C_m > thr}, clamped to N - 1
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > thr) hi = mid; else lo = mid + 1;
        }
        for (int i = 0; i < dp; ++i) {
            xs[(int64_t)i * Np + n] = xa[(int64_t)i * Np + lo];
            gs[(int64_t)i * Np + n] = ga[(int64_t)i * Np + lo];
        }
        ell_s[n] = ell[lo];
        logw[n] = 0.0;
        if (ancestors) ancestors[n] = lo;
    }
}

__global__ void __launch_bounds__(256)
tcs_copyback_kernel(const AsmcState* st, int64_t N, int64_t Np, int dp, float* xa, float* ga,
                    const float* __restrict__ xs, const float* __restrict__ gs, double* ell,
                    const double* __restrict__ ell_s)
{
    if (!st->pend) return;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < dp; ++i) {
            xa[(int64_t)i * Np + n] = xs[(int64_t)i * Np + n];
            ga[(int64_t)i * Np + n] = gs[(int64_t)i * Np + n];
        }
        ell[n] = ell_s[n];
    }
}

cudaError_t launch_gather_tcs(const TcsPlan& L, const AsmcState* st, const double* cdf, int64_t N, float* state,
                              double* ell, double* ell_scratch, double* logw, int64_t* ancestors, cudaStream_t s)
{
    const int64_t Np = (int64_t)tcs_tiles(N) * tcs::kTile;
    float* xa = state;
    float* ga = state + (size_t)L.dp * Np;
    float* xs = state + (size_t)2 * L.dp * Np;
    float* gs = state + (size_t)3 * L.dp * Np;
    const int gb = capped_grid((N + 255) / 256, 4);   // usually returns at once
    tcs_gather_kernel<<<gb, 256, 0, s>>>(st, cdf, N, Np, L.dp, xa, ga, xs, gs, ell, ell_scratch, logw, ancestors);
    tcs_copyback_kernel<<<gb, 256, 0, s>>>(st, N, Np, L.dp, xa, ga, xs, gs, ell, ell_scratch);
    return cudaGetLastError();
}

cudaError_t launch_potential_tcs(const TcsPlan& L, int kind, const void* img, const float* x, int64_t N,
                                 double* ell, float* grad, double p0, int n, int d, unsigned* status,
                                 float* state, int64_t state_particles, cudaStream_t s)
{
    // batches of at most state_particles (the scratch the state buffer holds)
    const int64_t cap = state_particles / tcs::kTile * tcs::kTile;
    if (cap < tcs::kTile) return cudaErrorInvalidValue;
    for (int64_t b0 = 0; b0 < N; b0 += cap) {
        SweepParams sp{};
        sp.N = std::min(cap, N - b0);
        sp.T = 0;
        sp.status = status;
        sp.mv.K = 1;
        // the state buffer is laid out for state_particles: keep its stride
        cudaError_t e = launch_tcs(L, kind, sp, img, state, kMala, 1, p0, n, d, x + b0, ell + b0,
                                   grad ? grad + b0 : nullptr, N, s, state_particles);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t tcs_params_bytes() { return sizeof(tcs::Params); }
uint32_t tcs_misc_bytes() { return (uint32_t)sizeof(tcs::Misc); }

void tcs_batch_params(const TcsPlan& L, int kind, const SweepParams& sp, const void* img, float* state, int move,
                      int leapfrog, double p0, int n, int d, uint32_t off_misc, void* out)
{
    tcs::Params P;
    fill_params(P, L, kind, sp, img, state, move, leapfrog, p0, n, d, nullptr, nullptr, nullptr, 0, 0);
    P.off_misc = off_misc;
    std::memcpy(out, &P, sizeof(P));
}

} // namespace oais
