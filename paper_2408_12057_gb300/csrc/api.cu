// api.cu -- host side of the C ABI: context lifetime, the OAIS round driver (Alg. 2),
// OptimiseSchedule (Alg. 3) and step-size carry-over between rounds.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "../../include/oais.h"

namespace oais {
cudaError_t launch_asmc_resample(AsmcState* st, const StepParams& P, int nparts, double ess_frac, int d,
                                 bool grad, bool fp64, double* bsum, double* boff, double* cdf,
                                 double* ess_trace, int* resampled, int64_t* ancestors, cudaStream_t s);
int scan_blocks(int64_t N);
int tc_image_bytes();
int tc_max_rows();
void tc_prepare_logreg(const float* X, const float* y, int n, int d, std::vector<uint16_t>& img,
                       std::vector<uint32_t>& ybits);
cudaError_t launch_merge_stats(const StepPartial*, int, int, double, double*, double*, double*, cudaStream_t);
cudaError_t launch_fisher(const double* logw, const double* ell, const void* x, bool fp64, int64_t N, int d,
                          const double* lse, double ref_scale, int kind, int nrows, double p0, void* scratch,
                          double* out, cudaStream_t s);
cudaError_t launch_logsumexp(const double*, int64_t, double*, void*, cudaStream_t);
size_t logsumexp_scratch_bytes(int64_t n);

// the families whose particles and arithmetic are fp64 (the others run in fp32)
static bool f64_kind(int kind) { return kind == kGauss || kind == kUnid; }

int padded_width(int kind, int d)
{
    static const int gauss[] = {1, 2, 4, 8, 16}, rows[] = {2, 4, 8, 16, 32}, gmm[] = {2, 4, 8, 16};
    if (kind == kUnid) return d == 2 ? 2 : 0;
    const int* w = rows; int nw = 5;
    if (kind == kGauss) { w = gauss; nw = 5; }
    else if (kind == kGmm) { w = gmm; nw = 4; }
    for (int i = 0; i < nw; ++i) if (d <= w[i]) return w[i];
    return 0;
}

// ---------------------------------------------------------------------------
// Monotone piecewise-cubic Hermite interpolant (Fritsch & Carlson 1980; interior slopes
// by the weighted harmonic mean of Fritsch & Butland 1984; shape-preserving three-point
// end slopes).  This is the reading of Alg. 3's "monotone spline".
// ---------------------------------------------------------------------------
class MonotoneCubic {
public:
    MonotoneCubic(std::vector<double> xs, std::vector<double> ys) : x_(std::move(xs)), y_(std::move(ys)) {
        const size_t K = x_.size();
        slope_.assign(K, 0.0);
        std::vector<double> h(K - 1), sec(K - 1);
        for (size_t i = 0; i + 1 < K; ++i) { h[i] = x_[i + 1] - x_[i]; sec[i] = (y_[i + 1] - y_[i]) / h[i]; }
        if (K == 2) { slope_[0] = slope_[1] = sec[0]; return; }
        for (size_t k = 1; k + 1 < K; ++k) {
            if (sec[k - 1] * sec[k] > 0.0) {
                const double a = 2.0 * h[k] + h[k - 1], b = h[k] + 2.0 * h[k - 1];
                slope_[k] = (a + b) / (a / sec[k - 1] + b / sec[k]);
            }
        }
        slope_[0] = end(h[0], h[1], sec[0], sec[1]);
        slope_[K - 1] = end(h[K - 2], h[K - 3], sec[K - 2], sec[K - 3]);
    }
    double operator()(double v) const {
        const size_t K = x_.size();
        size_t i = std::upper_bound(x_.begin(), x_.end(), v) - x_.begin();
        i = (i == 0) ? 0 : std::min(i - 1, K - 2);
        const double h = x_[i + 1] - x_[i], u = (v - x_[i]) / h, w = 1.0 - u;
        return y_[i] * w * w * (1.0 + 2.0 * u) + y_[i + 1] * u * u * (3.0 - 2.0 * u)
             + h * (slope_[i] * u * w * w - slope_[i + 1] * u * u * w);
    }
private:
    static int sgn(double v) { return (v > 0.0) - (v < 0.0); }
    static double end(double h0, double h1, double s0, double s1) {
        const double e = ((2.0 * h0 + h1) * s0 - h0 * s1) / (h0 + h1);
        if (sgn(e) != sgn(s0)) return 0.0;
        if (sgn(s0) != sgn(s1) && std::fabs(e) > 3.0 * std::fabs(s0)) return 3.0 * s0;
        return e;
    }
    std::vector<double> x_, y_, slope_;
};

static void optimise_schedule(int T, const double* beta, const double* lg, int Tn, double* out,
                              double* D_out, double* Lam_out)
{
    std::vector<double> Lam(T + 1, 0.0);
    for (int t = 1; t <= T; ++t) {
        double D = lg[3 * (t - 1) + 2] - 2.0 * lg[3 * (t - 1) + 1] + lg[3 * (t - 1)];
        D = (D > 0.0) ? D : 0.0;   // NaN and rounding negatives count as zero
        if (D_out) D_out[t - 1] = D;
        Lam[t] = Lam[t - 1] + std::sqrt(D);
    }
    if (Lam_out) std::copy(Lam.begin(), Lam.end(), Lam_out);
    std::vector<double> kx, ky;
    for (int t = 0; t <= T; ++t) {
        if (!kx.empty() && !(Lam[t] > kx.back())) continue;
        kx.push_back(Lam[t]);
        ky.push_back(beta[t]);
    }
    if (kx.size() < 2) {
        for (int i = 0; i <= Tn; ++i) out[i] = (double)i / Tn;
    } else {
        ky.back() = beta[T];
        MonotoneCubic f(kx, ky);
        for (int i = 0; i <= Tn; ++i) out[i] = f(Lam[T] * ((double)i / Tn));
    }
    out[0] = 0.0;
    out[Tn] = 1.0;
}

// Diagonal curvature estimate kappa of -log L (per unit beta) behind the starting step-size rule
// and the carry-over of step sizes between rounds: the Gaussian 1 / p0^2; logistic
// sum X^2 / (4 d) (the sigmoid's largest slope); linear regression sum X^2 / (d p0^2); mixture
// 1 / p0 (a component's precision); Unid m q (1 - q)^-1 q^2, q = k / m (the binomial ridge's
// width in the probit coordinates).  Xh: the data as doubles (rows of X, or (m, k) for Unid).
static double curvature(int kind, int d, double p0, const std::vector<double>& Xh)
{
    if (kind == kGauss) return 1.0 / (p0 * p0);
    if (kind == kGmm) return 1.0 / p0;
    if (kind == kUnid) {
        const double q = Xh[1] / Xh[0];
        return Xh[0] / (q * (1.0 - q)) * q * q;
    }
    double ss = 0.0;
    for (double v : Xh) ss += v * v;
    return kind == kLogreg ? 0.25 * ss / d : ss / d / (p0 * p0);
}

static bool valid_schedule(const double* beta, int T)
{
    if (T < 1 || !beta || beta[0] != 0.0 || beta[T] != 1.0) return false;
    for (int t = 1; t <= T; ++t) if (!(beta[t] > beta[t - 1]) || !std::isfinite(beta[t])) return false;
    return true;
}

} // namespace oais

using namespace oais;

static thread_local std::string g_err;

struct oais_ctx {
    oais_target tg_in{};
    oais_move mv{};
    DevTarget dt;
    int64_t N = 0;
    int64_t N_cap = 0;                   // the particle count the workspace was laid out for
    int T_max = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    // device workspace
    void* ws = nullptr;
    bool own_ws = false;
    double *d_beta = nullptr, *d_eps = nullptr, *d_logw = nullptr, *d_ell = nullptr;
    float* d_fsched = nullptr;           // fp32 roundings of the schedule (GmmTarget::fsched)
    std::vector<float> h_fsched;
    void* d_x = nullptr;
    StepPartial* d_parts = nullptr;
    double *d_log_ghat = nullptr, *d_accept = nullptr, *d_lse = nullptr;
    double* d_elbo = nullptr;            // [T_max] ELBO terms sum_n W_{t-1}^n log g_t^n
    // online conditional-ESS rounds
    float2* d_zfg = nullptr;
    double2* d_zanchor = nullptr;
    float2* d_zpart = nullptr;
    ZjaState* d_zstate = nullptr;
    double *d_zbeta = nullptr, *d_zeps = nullptr;
    void* d_lse_scratch = nullptr;
    unsigned* d_status = nullptr;
    // ASMC: second particle buffer, gradient buffers, resampling scratch and traces
    void* d_x1 = nullptr;
    void *d_g0 = nullptr, *d_g1 = nullptr;
    double* d_ell1 = nullptr;
    StepPartial* d_ess_parts = nullptr;
    AsmcState* d_st = nullptr;
    double *d_bsum = nullptr, *d_boff = nullptr, *d_cdf = nullptr, *d_ess_trace = nullptr;
    int* d_resampled = nullptr;
    int64_t* d_anc = nullptr;
    bool last_asmc = false;
    int l_n_resample = 0;
    // sharding: this context's particles are [n_offset, n_offset + N) of N_total
    int64_t n_offset = 0, N_total = 0;
    int pend_T = 0;                      // > 0 after oais_round_local, until the commit
    float pend_ms = 0.0f;
    std::vector<double> pend_lg, pend_acc;
    double pend_lse[2] = {0.0, 0.0};
    std::vector<double> cur_elbo;        // the running round's ELBO terms (empty: not available)
    std::vector<double> l_ess_trace;
    std::vector<int> l_resampled;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // schedule of the next round
    std::vector<double> beta, eps;
    int round = 0;
    int problem = 0;                     // problem index in the random-number tag
    double kappa = 0.0;                  // curvature estimate of -log L (step-size carry-over)
    bool exact_data = false;             // tensor-core forms: reweight the final particles from X~ to X
    // test support (oais_arm_fault): a fault armed for the next round
    int fault_kind = 0;
    uint64_t fault_wait_ns = 0;
    // last completed round
    bool have_last = false;
    std::vector<double> l_beta, l_eps, l_log_ghat, l_D, l_accept, l_elbo;
    double l_logZ = 0, l_se = 0, l_Lambda = 0, l_ess = 0;
    std::string err;
};

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            set_err(ctx, std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return OAIS_ECUDA;                                                       \
        }                                                                            \
    } while (0)

static void set_err(oais_ctx* ctx, const std::string& m)
{
    if (ctx) ctx->err = m; else g_err = m;
}

static oais_status fail(oais_ctx* ctx, oais_status s, const std::string& m)
{
    set_err(ctx, m);
    return s;
}

// the calling thread's error text for calls without a context (oais_last_error(NULL)), for
// the library's other translation units
namespace oais {
int fail_call(int s, const char* m)
{
    g_err = m;
    return s;
}
} // namespace oais

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static size_t elt_bytes(int kind) { return f64_kind(kind) ? sizeof(double) : sizeof(float); }

struct Layout {
    size_t X, y, beta, eps, logw, ell, x, parts, lg, acc, elbo, lse, lse_scr, status;
    size_t x1, g0, g1, ell1, ess_parts, st, bsum, boff, cdf, ess_trace, resampled, anc, tc_img, tc_y;
    size_t tcs_img, tcs_state, tc_handed, zja_fg, zja_anchor, zja_part, zja_state, zja_beta, zja_eps, wide_state, fsched,
        total;
};

// which sweep form a target runs: 0 CUDA cores, 1 resident tensor-core, 2 streamed tensor-core
static int sweep_form(const oais_target* tg, const oais_move* mv)
{
    if (tg->contraction == OAIS_CONTRACT_BF16_TC_STREAM || tg->contraction == OAIS_CONTRACT_FP8_TC_STREAM) return 2;
    if (tg->contraction != OAIS_CONTRACT_BF16_TC) return 0;
    if (tg->kind == kLogreg && tg->d <= 32 && tg->n <= tc_max_rows() && mv->kind == OAIS_MALA) return 1;
    return 2;
}

static int records_per_step(int64_t N)
{
    return std::max(std::max(sweep_grid(N), tc_records(N)), std::max(tcs_tiles(N), wide_tiles(N)));
}

static Layout layout(const oais_target* tg, const oais_move* mv, int D, int64_t N, int T_max)
{
    Layout L{};
    const int n_pad = (tg->n + 3) & ~3;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes ? bytes : 1); return o; };
    size_t xb;
    if (tg->kind == kGauss) xb = sizeof(double) * D;
    else if (tg->kind == kUnid) xb = sizeof(double) * 4;   // m, k, b, c0
    else if (tg->kind == kGmm) xb = sizeof(float) * (size_t)tg->n * D;
    else xb = sizeof(float) * (size_t)n_pad * D;
    L.X = take(xb);
    L.y = take((tg->kind == kLogreg || tg->kind == kLinreg) ? sizeof(float) * n_pad : 0);
    L.beta = take(sizeof(double) * (T_max + 1));
    L.eps = take(sizeof(double) * T_max);
    L.logw = take(sizeof(double) * N);
    L.ell = take(sizeof(double) * N);
    L.x = take(elt_bytes(tg->kind) * (size_t)tg->d * N);
    L.parts = take(sizeof(StepPartial) * (size_t)T_max * records_per_step(N));
    L.lg = take(sizeof(double) * 3 * T_max);
    L.acc = take(sizeof(double) * T_max);
    L.elbo = take(sizeof(double) * T_max);
    L.lse = take(sizeof(double) * 2);
    L.lse_scr = take(logsumexp_scratch_bytes(N));
    L.status = take(sizeof(unsigned));
    const size_t xbytes = elt_bytes(tg->kind) * (size_t)tg->d * N;
    L.x1 = take(xbytes);
    L.g0 = take(xbytes);
    L.g1 = take(xbytes);
    L.ell1 = take(sizeof(double) * N);
    L.ess_parts = take(sizeof(StepPartial) * (size_t)(sweep_grid(N) + asmc_ess_groups(sweep_grid(N))));
    L.st = take(sizeof(AsmcState));
    L.bsum = take(sizeof(double) * scan_blocks(N));
    L.boff = take(sizeof(double) * (scan_blocks(N) + 1));
    L.cdf = take(sizeof(double) * N);
    L.ess_trace = take(sizeof(double) * T_max);
    L.resampled = take(sizeof(int) * T_max);
    L.anc = take(sizeof(int64_t) * N);
    const int form = sweep_form(tg, mv);
    L.tc_img = take(form == 1 ? (size_t)tc_image_bytes() : 0);
    L.tc_y = take(form == 1 ? (size_t)tc_max_rows() / 8 : 0);
    L.tc_handed = take(form >= 1 ? sizeof(int) * (size_t)std::max(tc_records(N), tcs_tiles(N)) : 0);
    // online conditional-ESS rounds (CUDA-core form): offsets, anchors, candidate sums, state,
    // the schedule found online and its step sizes
    L.zja_fg = take(sizeof(float2) * (size_t)N);
    L.zja_anchor = take((sizeof(double2) + sizeof(float2)) * (size_t)zja_grid(N));   // anchors, then their fp32 offsets
    L.zja_part = take(zja_part_bytes(N));
    L.zja_state = take(sizeof(ZjaState));
    L.zja_beta = take(sizeof(double) * (T_max + 1));
    L.zja_eps = take(sizeof(double) * T_max);
    TcsPlan tp;
    // the streamed form's image and state: its own sweeps, and the resampling rounds and the
    // potential of a resident-form context (whose kernel is a whole-sweep kernel)
    if (form >= 1) tp = tcs_plan(tg->kind, tg->n, tg->d, 0, 0, tg->contraction == OAIS_CONTRACT_FP8_TC_STREAM);
    L.tcs_img = take(form >= 1 ? tcs_image_bytes(tp, tg->kind, tg->n) : 0);
    L.tcs_state = take(form >= 1 ? sizeof(float) * 5 * (size_t)tp.dp * tcs_tiles(N) * 128 : 0);
    // the tiled fp32 form (32 < d <= 256): positions, gradients, momenta of every tile
    L.wide_state = take(D > 32 ? wide_state_bytes(D, N) : 0);
    L.fsched = take(sizeof(float) * (3 * (size_t)T_max + 1));
    L.total = off;
    return L;
}

static oais_status check_target(oais_ctx* ctx, const oais_target* tg, const oais_move* mv, int64_t N,
                                int T_max, int* D)
{
    if (!tg || !mv) return fail(ctx, OAIS_EINVAL, "null target or move");
    if (tg->kind < 0 || tg->kind > 4) return fail(ctx, OAIS_EINVAL, "unknown target kind");
    if (tg->d < 1 || !tg->X) return fail(ctx, OAIS_EINVAL, "bad dimension or missing X");
    if (!(tg->ref_scale > 0) || !(tg->p0 > 0)) return fail(ctx, OAIS_EINVAL, "ref_scale and p0 must be > 0");
    if (!f64_kind(tg->kind) && tg->n < 1) return fail(ctx, OAIS_EINVAL, "n must be >= 1");
    if (tg->kind == kUnid) {
        if (tg->d != 2 || tg->ref_scale != 1.0 || tg->dtype != OAIS_DT_F64)
            return fail(ctx, OAIS_EINVAL, "UNID: d = 2, ref_scale = 1 and float64 (m, k)");
        if (tg->contraction != OAIS_CONTRACT_FP32)
            return fail(ctx, OAIS_EUNSUPPORTED, "UNID runs on the CUDA-core form");
        if (!tg->on_device) {
            const double* mk = static_cast<const double*>(tg->X);
            if (!(mk[0] >= 1.0 && mk[1] > 0.0 && mk[1] < mk[0]))
                return fail(ctx, OAIS_EINVAL, "UNID: trials m >= 1 and successes 0 < k < m");
        }
    }
    if ((tg->kind == kLogreg || tg->kind == kLinreg) && !tg->y) return fail(ctx, OAIS_EINVAL, "missing y");
    if (tg->kind == kGmm && tg->n > GmmTarget<float, 16>::kMaxK)
        return fail(ctx, OAIS_EUNSUPPORTED, "at most 16 mixture components");
    if (tg->dtype != OAIS_DT_F64 && tg->dtype != OAIS_DT_F32) return fail(ctx, OAIS_EINVAL, "bad dtype");
    if (tg->contraction < OAIS_CONTRACT_FP32 || tg->contraction > OAIS_CONTRACT_FP8_TC_STREAM)
        return fail(ctx, OAIS_EINVAL, "bad contraction");
    if (tg->contraction == OAIS_CONTRACT_FP8_TC_STREAM && tg->kind != kLinreg)
        return fail(ctx, OAIS_EUNSUPPORTED, "FP8 storage of X is built for LINREG");
    if (tg->contraction != OAIS_CONTRACT_FP32) {
        const bool fam = (tg->kind == kLogreg && mv->kind == OAIS_MALA) ||
                         (tg->kind == kLinreg && (mv->kind == OAIS_MALA || mv->kind == OAIS_HMC));
        if (!fam || tg->d > 256)
            return fail(ctx, OAIS_EUNSUPPORTED,
                        "the tensor-core contraction is built for LOGREG (MALA) and LINREG (MALA, HMC), d <= 256");
        if (sweep_form(tg, mv) >= 1) {
            const TcsPlan tp = tcs_plan(tg->kind, tg->n, tg->d, 0, 0, tg->contraction == OAIS_CONTRACT_FP8_TC_STREAM);
            const int Le = mv->kind == OAIS_HMC ? mv->leapfrog : 1;
            const double chunks = (1.0 + (double)T_max * mv->moves * Le) * tp.nch;
            if (!tp.ok || chunks >= 4294967295.0)
                return fail(ctx, OAIS_EUNSUPPORTED, "streamed tensor-core form: size out of range");
        }
    }
    if (tg->kind == kGauss && tg->dtype != OAIS_DT_F64)
        return fail(ctx, OAIS_EINVAL, "the Gaussian family takes float64 mu");
    if (mv->kind < 0 || mv->kind > 2 || mv->moves < 1 || (mv->kind == OAIS_HMC && mv->leapfrog < 1))
        return fail(ctx, OAIS_EINVAL, "bad move");
    if (N < 1 || N > 0x7FFFFFFFLL) return fail(ctx, OAIS_EINVAL, "N out of range");
    if (T_max < 1 || T_max > (1 << 24)) return fail(ctx, OAIS_EINVAL, "T_max out of range");
    *D = padded_width(tg->kind, tg->d);
    // the row families above d = 32 in fp32: the tiled CUDA-core form, width 64, 128 or 256
    if (*D == 0 && (tg->kind == kLogreg || tg->kind == kLinreg) && tg->contraction == OAIS_CONTRACT_FP32)
        *D = wide_width(tg->d);
    // the streamed tensor-core form needs no CUDA-core width (D = 0: no CUDA-core copy of X)
    if (*D == 0 && sweep_form(tg, mv) != 2) return fail(ctx, OAIS_EUNSUPPORTED, "dimension not built for this family");
    return OAIS_OK;
}

// host copy of an input array as doubles (input host or device, f32 or f64)
static oais_status fetch(oais_ctx* ctx, const void* src, size_t count, int dtype, int on_device,
                         std::vector<double>& out)
{
    out.resize(count);
    const size_t eb = dtype == OAIS_DT_F64 ? 8 : 4;
    std::vector<unsigned char> raw(count * eb);
    if (on_device) CK(cudaMemcpy(raw.data(), src, count * eb, cudaMemcpyDeviceToHost));
    else std::memcpy(raw.data(), src, count * eb);
    for (size_t i = 0; i < count; ++i) {
        if (dtype == OAIS_DT_F64) { double v; std::memcpy(&v, &raw[i * 8], 8); out[i] = v; }
        else { float v; std::memcpy(&v, &raw[i * 4], 4); out[i] = v; }
    }
    return OAIS_OK;
}

extern "C" {

const char* oais_status_string(oais_status s)
{
    switch (s) {
    case OAIS_OK: return "ok";
    case OAIS_EINVAL: return "invalid argument";
    case OAIS_ENOMEM: return "out of device memory";
    case OAIS_ECUDA: return "CUDA error";
    case OAIS_ENONFINITE: return "non-finite log-weight or log-likelihood";
    case OAIS_ETIMEOUT: return "device wait timed out";
    case OAIS_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* oais_last_error(const oais_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int32_t oais_sweep_blocks(int64_t N) { return sweep_grid(N); }
int32_t oais_step_partial_bytes(void) { return (int32_t)sizeof(StepPartial); }

oais_status oais_workspace_bytes(const oais_target* tg, const oais_move* mv, int64_t N, int32_t T_max,
                                 size_t* bytes)
{
    int D = 0;
    oais_status st = check_target(nullptr, tg, mv, N, T_max, &D);
    if (st != OAIS_OK) return st;
    if (!bytes) return fail(nullptr, OAIS_EINVAL, "null bytes");
    *bytes = layout(tg, mv, D, N, T_max).total;
    return OAIS_OK;
}

oais_status oais_optimise_schedule(int32_t T, const double* beta, const double* log_ghat, int32_t T_next,
                                   double* beta_next, double* D_hat, double* Lambda)
{
    if (T < 1 || T_next < 1 || !beta || !log_ghat || !beta_next)
        return fail(nullptr, OAIS_EINVAL, "bad arguments to oais_optimise_schedule");
    optimise_schedule(T, beta, log_ghat, T_next, beta_next, D_hat, Lambda);
    return OAIS_OK;
}

oais_status oais_init(oais_ctx** out, const oais_target* tg, const oais_move* mv, int64_t N,
                      const double* beta, int32_t T, int32_t T_max, const double* eps, uint64_t seed,
                      void* workspace, size_t ws_bytes, void* stream)
{
    if (!out) return fail(nullptr, OAIS_EINVAL, "null ctx pointer");
    *out = nullptr;
    int D = 0;
    oais_status st = check_target(nullptr, tg, mv, N, T_max, &D);
    if (st != OAIS_OK) return st;
    if (T > T_max) return fail(nullptr, OAIS_EINVAL, "T > T_max");
    if (!valid_schedule(beta, T)) return fail(nullptr, OAIS_EINVAL, "schedule must be 0 = beta_0 < ... < beta_T = 1");
    if (eps) for (int t = 0; t < T; ++t) if (!(eps[t] > 0)) return fail(nullptr, OAIS_EINVAL, "step sizes must be > 0");

    oais_ctx* ctx = new oais_ctx();
    ctx->tg_in = *tg;
    ctx->mv = *mv;
    ctx->N = N;
    ctx->N_cap = N;
    ctx->N_total = N;
    ctx->T_max = T_max;
    ctx->seed = seed;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->beta.assign(beta, beta + T + 1);
    if (eps) ctx->eps.assign(eps, eps + T);
    else ctx->eps.assign(T, 0.5 / std::sqrt((double)tg->d));

    Layout L = layout(tg, mv, D, N, T_max);
    if (workspace) {
        if (ws_bytes < L.total) { delete ctx; return fail(nullptr, OAIS_ENOMEM, "workspace too small"); }
        ctx->ws = workspace;
    } else {
        cudaError_t e = cudaMalloc(&ctx->ws, L.total);
        if (e != cudaSuccess) { delete ctx; return fail(nullptr, OAIS_ENOMEM, cudaGetErrorString(e)); }
        ctx->own_ws = true;
    }
    char* b = static_cast<char*>(ctx->ws);
    DevTarget& dt = ctx->dt;
    dt.kind = tg->kind; dt.d = tg->d; dt.D = D; dt.n = f64_kind(tg->kind) ? 0 : tg->n;
    dt.n_pad = (dt.n + 3) & ~3;
    dt.ref_scale = tg->ref_scale; dt.p0 = tg->p0;
    dt.X = b + L.X;
    dt.y = (tg->kind == kLogreg || tg->kind == kLinreg) ? b + L.y : nullptr;
    dt.wide = D > 32;
    dt.wide_state = dt.wide ? reinterpret_cast<float*>(b + L.wide_state) : nullptr;
    ctx->d_beta = reinterpret_cast<double*>(b + L.beta);
    ctx->d_fsched = reinterpret_cast<float*>(b + L.fsched);
    ctx->d_eps = reinterpret_cast<double*>(b + L.eps);
    ctx->d_logw = reinterpret_cast<double*>(b + L.logw);
    ctx->d_ell = reinterpret_cast<double*>(b + L.ell);
    ctx->d_x = b + L.x;
    ctx->d_parts = reinterpret_cast<StepPartial*>(b + L.parts);
    ctx->d_log_ghat = reinterpret_cast<double*>(b + L.lg);
    ctx->d_elbo = reinterpret_cast<double*>(b + L.elbo);
    ctx->d_zfg = reinterpret_cast<float2*>(b + L.zja_fg);
    ctx->d_zanchor = reinterpret_cast<double2*>(b + L.zja_anchor);
    ctx->d_zpart = reinterpret_cast<float2*>(b + L.zja_part);
    ctx->d_zstate = reinterpret_cast<ZjaState*>(b + L.zja_state);
    ctx->d_zbeta = reinterpret_cast<double*>(b + L.zja_beta);
    ctx->d_zeps = reinterpret_cast<double*>(b + L.zja_eps);
    ctx->d_accept = reinterpret_cast<double*>(b + L.acc);
    ctx->d_lse = reinterpret_cast<double*>(b + L.lse);
    ctx->d_lse_scratch = b + L.lse_scr;
    ctx->d_status = reinterpret_cast<unsigned*>(b + L.status);
    ctx->d_x1 = b + L.x1;
    ctx->d_g0 = b + L.g0;
    ctx->d_g1 = b + L.g1;
    ctx->d_ell1 = reinterpret_cast<double*>(b + L.ell1);
    ctx->d_ess_parts = reinterpret_cast<StepPartial*>(b + L.ess_parts);
    ctx->d_st = reinterpret_cast<AsmcState*>(b + L.st);
    ctx->d_bsum = reinterpret_cast<double*>(b + L.bsum);
    ctx->d_boff = reinterpret_cast<double*>(b + L.boff);
    ctx->d_cdf = reinterpret_cast<double*>(b + L.cdf);
    ctx->d_ess_trace = reinterpret_cast<double*>(b + L.ess_trace);
    ctx->d_resampled = reinterpret_cast<int*>(b + L.resampled);
    ctx->d_anc = reinterpret_cast<int64_t*>(b + L.anc);

    // data in the padded device layout
    const int rows = f64_kind(tg->kind) ? 1 : tg->n;
    std::vector<double> Xh, yh;
    st = fetch(ctx, tg->X, (size_t)rows * tg->d, tg->dtype, tg->on_device, Xh);
    if (st == OAIS_OK && dt.y) st = fetch(ctx, tg->y, (size_t)tg->n, tg->dtype, tg->on_device, yh);
    if (st != OAIS_OK) { g_err = ctx->err; oais_destroy(ctx); return st; }
    ctx->kappa = curvature(tg->kind, tg->d, tg->p0, Xh);
    cudaError_t e = cudaSuccess;
    if (tg->kind == kGauss) {
        std::vector<double> mu(D, 0.0);
        for (int i = 0; i < tg->d; ++i) mu[i] = Xh[i];
        e = cudaMemcpy(dt.X, mu.data(), sizeof(double) * D, cudaMemcpyHostToDevice);
    } else if (tg->kind == kUnid) {
        // (m, k, b, c0) with c0 = log Binom(k; m, k/m): Stirling's series for large counts
        // (-1/2 log(2 pi m q (1 - q)) + 1/(12 m) - 1/(12 k) - 1/(12 (m - k))), log-gamma below
        const double m = Xh[0], k = Xh[1], q = k / m;
        double c0;
        if (std::min(k, m - k) >= 1e6)
            c0 = -0.5 * std::log(6.283185307179586 * m * q * (1.0 - q)) + 1.0 / (12.0 * m) - 1.0 / (12.0 * k) -
                 1.0 / (12.0 * (m - k));
        else
            c0 = std::lgamma(m + 1.0) - std::lgamma(k + 1.0) - std::lgamma(m - k + 1.0) + k * std::log(q) +
                 (m - k) * std::log1p(-q);
        const double par[4] = {m, k, tg->p0, c0};
        if (!(m >= 1.0 && k > 0.0 && k < m)) { fail(ctx, OAIS_EINVAL, "UNID: trials m >= 1 and successes 0 < k < m");
                                               g_err = ctx->err; oais_destroy(ctx); return OAIS_EINVAL; }
        e = cudaMemcpy(dt.X, par, sizeof(par), cudaMemcpyHostToDevice);
    } else {
        const int nr = tg->kind == kGmm ? tg->n : dt.n_pad;
        std::vector<float> Xp((size_t)nr * D, 0.0f), yp(dt.n_pad, 0.0f);
        if (D > 0) {   // the CUDA-core copy of X (absent when only the streamed form exists)
            for (int r = 0; r < tg->n; ++r)
                for (int i = 0; i < tg->d; ++i) Xp[(size_t)r * D + i] = (float)Xh[(size_t)r * tg->d + i];
            e = cudaMemcpy(dt.X, Xp.data(), sizeof(float) * Xp.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && dt.y) {
            for (int r = 0; r < tg->n; ++r) yp[r] = (float)yh[r];
            e = cudaMemcpy(dt.y, yp.data(), sizeof(float) * yp.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && sweep_form(tg, mv) >= 1) {
            std::vector<float> Xf((size_t)tg->n * tg->d), yf(tg->n);
            for (size_t i = 0; i < Xf.size(); ++i) Xf[i] = (float)Xh[i];
            for (int r = 0; r < tg->n; ++r) yf[r] = (float)yh[r];
            const bool q8 = tg->contraction == OAIS_CONTRACT_FP8_TC_STREAM;
            const TcsPlan tp = tcs_plan(tg->kind, tg->n, tg->d, 0, 0, q8);
            std::vector<unsigned char> img;
            if (q8) tcs_prepare_q8(tp, Xf.data(), yf.data(), tg->n, tg->d, img);
            else tcs_prepare(tp, tg->kind, Xf.data(), yf.data(), tg->n, tg->d, img);
            img.resize(tcs_image_bytes(tp, tg->kind, tg->n), 0);   // zero rows past the last chunk
            dt.tcs = true;
            dt.tcs_q8 = q8;
            dt.tcs_dp = tp.dp;
            dt.tcs_img = b + L.tcs_img;
            dt.tcs_state = reinterpret_cast<float*>(b + L.tcs_state);
            dt.tc_handed = reinterpret_cast<int*>(b + L.tc_handed);
            e = cudaMemcpy(dt.tcs_img, img.data(), img.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && sweep_form(tg, mv) == 1) {
            std::vector<float> Xf((size_t)tg->n * tg->d), yf(tg->n);
            for (size_t i = 0; i < Xf.size(); ++i) Xf[i] = (float)Xh[i];
            for (int r = 0; r < tg->n; ++r) yf[r] = (float)yh[r];
            std::vector<uint16_t> img;
            std::vector<uint32_t> yb;
            tc_prepare_logreg(Xf.data(), yf.data(), tg->n, tg->d, img, yb);
            dt.tc = true;
            dt.tc_img = b + L.tc_img;
            dt.tc_ybits = reinterpret_cast<uint32_t*>(b + L.tc_y);
            dt.tc_handed = reinterpret_cast<int*>(b + L.tc_handed);
            e = cudaMemcpy(dt.tc_img, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(dt.tc_ybits, yb.data(), yb.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e != cudaSuccess) { g_err = cudaGetErrorString(e); oais_destroy(ctx); return OAIS_ECUDA; }
    *out = ctx;
    return OAIS_OK;
}

void oais_destroy(oais_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
    delete ctx;
}

static cudaError_t launch_sweep(const DevTarget& dt, int move, const SweepParams& P, cudaStream_t s)
{
    switch (dt.kind) {
    case kGauss: return launch_sweep_gauss(dt, move, P, s);
    case kUnid: return launch_sweep_unid(dt, move, P, s);
    case kLogreg: return launch_sweep_logreg(dt, move, P, s);
    case kGmm: return launch_sweep_gmm(dt, move, P, s);
    case kLinreg: return launch_sweep_linreg(dt, move, P, s);
    }
    return cudaErrorInvalidValue;
}

static SweepParams make_params(const oais_ctx* ctx, int T, const double* d_beta, const double* d_eps,
                               uint64_t seed, uint32_t tag, int64_t n_offset, int64_t N, double* logw,
                               double* ell, void* x, void* parts, unsigned* status)
{
    SweepParams P{};
    P.N = N; P.n_offset = n_offset; P.T = T; P.beta = d_beta; P.eps = d_eps;
    P.ref_scale = ctx->dt.ref_scale; P.mv.K = ctx->mv.moves; P.mv.leapfrog = ctx->mv.leapfrog;
    P.mv.cycle = ctx->mv.cycle;
    P.mv.rng.k0 = (uint32_t)(seed & 0xFFFFFFFFu); P.mv.rng.k1 = (uint32_t)(seed >> 32); P.mv.rng.tag = tag;
    P.logw = logw; P.x_out = x; P.ell_out = ell; P.partials = static_cast<StepPartial*>(parts);
    P.status = status;
    if (ctx->fault_kind == OAIS_FAULT_WITHHOLD_HANDOFF) {
        P.withhold = 1;
        P.handoff_wait_ns = ctx->fault_wait_ns;
    }
    return P;
}

oais_status oais_ctx_sweep(oais_ctx* ctx, int32_t T, const double* d_beta, const double* d_eps, uint64_t seed,
                           uint32_t tag, int64_t n_offset, int64_t N, double* d_logw, double* d_ell, void* d_x,
                           void* d_partials, uint32_t* d_status, void* stream)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (T < 1 || N < 1 || !d_beta || !d_eps || !d_logw || !d_ell || !d_x || !d_partials || !d_status)
        return fail(ctx, OAIS_EINVAL, "bad arguments to oais_ctx_sweep");
    if (n_offset < 0 || n_offset + N > 0xFFFFFFFFLL) return fail(ctx, OAIS_EINVAL, "particle index out of range");
    if (ctx->dt.D == 0 || ctx->dt.wide)
        return fail(ctx, OAIS_EUNSUPPORTED, "no one-thread-per-particle CUDA-core form for this dimension");
    SweepParams P = make_params(ctx, T, d_beta, d_eps, seed, tag, n_offset, N, d_logw, d_ell, d_x, d_partials,
                                d_status);
    CK(launch_sweep(ctx->dt, ctx->mv.kind, P, static_cast<cudaStream_t>(stream)));
    return OAIS_OK;
}

oais_status oais_merge_stats(const void* d_partials, int32_t nblocks, int32_t T, int64_t N, int32_t moves,
                             double* d_log_ghat, double* d_accept, void* stream)
{
    oais_ctx* ctx = nullptr;
    if (!d_partials || nblocks < 1 || T < 1 || N < 1 || moves < 1 || !d_log_ghat || !d_accept)
        return fail(nullptr, OAIS_EINVAL, "bad arguments to oais_merge_stats");
    CK(launch_merge_stats(static_cast<const StepPartial*>(d_partials), nblocks, T, 1.0 / ((double)N * moves),
                          d_log_ghat, d_accept, nullptr, static_cast<cudaStream_t>(stream)));
    return OAIS_OK;
}

size_t oais_logsumexp_scratch_bytes(int64_t n) { return logsumexp_scratch_bytes(n); }

oais_status oais_logsumexp(const double* d_a, int64_t n, double* d_out, void* d_scratch, void* stream)
{
    oais_ctx* ctx = nullptr;
    if (!d_a || n < 1 || !d_out || !d_scratch) return fail(nullptr, OAIS_EINVAL, "bad arguments to oais_logsumexp");
    CK(launch_logsumexp(d_a, n, d_out, d_scratch, static_cast<cudaStream_t>(stream)));
    return OAIS_OK;
}

// Carry step sizes to a new schedule (reading r9).  A step size is held as its ratio to the
// shape of the starting rule, h(beta) = 1 / sqrt(1/s^2 + beta kappa) (the scale of pi_beta under
// a Gaussian approximation of the likelihood's curvature): log(eps / h) is interpolated linearly
// in beta between the old steps and held constant beyond them, and the new step size is that
// ratio times h at the new beta.  A new schedule that puts steps at betas far below the old first
// step (the optimised schedule of a steep start) so gets steps that widen with the flatter
// tempered targets there, instead of the old first step's size.  When adapting, a
// multiplicative nudge moves each step toward the move's target acceptance.
static std::vector<double> next_step_sizes(const oais_ctx* ctx, const std::vector<double>& beta_old,
                                           const std::vector<double>& eps_old,
                                           const std::vector<double>& acc, const std::vector<double>& beta_new)
{
    const int T = (int)eps_old.size(), Tn = (int)beta_new.size() - 1;
    std::vector<double> out(Tn);
    const double target = ctx->mv.kind == OAIS_RWMH ? 0.3 : (ctx->mv.kind == OAIS_MALA ? 0.574 : 0.7);
    const double inv_s2 = 1.0 / (ctx->dt.ref_scale * ctx->dt.ref_scale);
    auto log_h = [&](double b) { return -0.5 * std::log(inv_s2 + b * ctx->kappa); };
    for (int i = 1; i <= Tn; ++i) {
        const double b = beta_new[i];
        // locate b among beta_old[1..T]
        int j = (int)(std::lower_bound(beta_old.begin() + 1, beta_old.end(), b) - beta_old.begin());
        j = std::max(1, std::min(j, T));
        double lr, a;
        if (j == 1 || T == 1) { lr = std::log(eps_old[0]) - log_h(beta_old[1]); a = acc[0]; }
        else {
            const double b0 = beta_old[j - 1], b1 = beta_old[j], w = (b - b0) / (b1 - b0);
            lr = (1 - w) * (std::log(eps_old[j - 2]) - log_h(b0)) + w * (std::log(eps_old[j - 1]) - log_h(b1));
            a = (1 - w) * acc[j - 2] + w * acc[j - 1];
        }
        double le = lr + log_h(b);
        if (ctx->mv.adapt && !(ctx->mv.kind == OAIS_RWMH && ctx->mv.cycle))
            le += std::max(-0.7, std::min(0.7, 1.5 * (a - target)));
        out[i - 1] = std::exp(le);
    }
    return out;
}

static StepParams make_step_params(const oais_ctx* ctx, int T, uint32_t tag)
{
    StepParams P{};
    P.N = ctx->N; P.t = 0; P.T = T; P.beta = ctx->d_beta; P.eps = ctx->d_eps;
    P.ref_scale = ctx->dt.ref_scale; P.mv.K = ctx->mv.moves; P.mv.leapfrog = ctx->mv.leapfrog;
    P.mv.cycle = ctx->mv.cycle;
    P.mv.rng.k0 = (uint32_t)(ctx->seed & 0xFFFFFFFFu); P.mv.rng.k1 = (uint32_t)(ctx->seed >> 32);
    P.mv.rng.tag = tag;
    P.x[0] = ctx->d_x; P.x[1] = ctx->d_x1; P.gl[0] = ctx->d_g0; P.gl[1] = ctx->d_g1;
    P.ell[0] = ctx->d_ell; P.ell[1] = ctx->d_ell1; P.logw = ctx->d_logw;
    P.st = ctx->d_st; P.partials = ctx->d_parts; P.ess_parts = ctx->d_ess_parts; P.status = ctx->d_status;
    return P;
}

static cudaError_t launch_asmc(const DevTarget& dt, int move, bool init, const StepParams& P, cudaStream_t s)
{
    switch (dt.kind) {
    case kGauss: return launch_asmc_gauss(dt, move, init, P, s);
    case kUnid: return launch_asmc_unid(dt, move, init, P, s);
    case kLogreg: return launch_asmc_logreg(dt, move, init, P, s);
    case kGmm: return launch_asmc_gmm(dt, move, init, P, s);
    case kLinreg: return launch_asmc_linreg(dt, move, init, P, s);
    }
    return cudaErrorInvalidValue;
}

// One round of Alg. 2: ASMC(N, B_T) on the current schedule, then Budget is the caller's
// T_next and OptimiseSchedule(T_next, B_T, g_hat) becomes the next schedule.
// asmc = false: AIS with the particle and time loops swapped (Sec. 5.1.2);
// asmc = true: lock-step particles with adaptive resampling at threshold ess_frac.
static oais_status commit_round(oais_ctx* ctx, int T, int32_t T_next, const std::vector<double>& lg,
                                const std::vector<double>& acc, double logZ, double ess, double se, float ms,
                                bool asmc, int n_res, const std::vector<double>& ess_tr,
                                const std::vector<int>& rs, oais_round_result* out);

static oais_status run_round_impl(oais_ctx* ctx, int32_t T_next, bool asmc, double ess_frac, oais_round_result* out,
                                  bool local_only)
{
    if (T_next < 1 || T_next > ctx->T_max) return fail(ctx, OAIS_EINVAL, "T_next out of range");
    if (asmc && !(ess_frac >= 0.0 && ess_frac <= 1.0 + 1e-12))
        return fail(ctx, OAIS_EINVAL, "ess_frac must be in [0, 1]");
    if (ctx->N_total != ctx->N && !local_only)
        return fail(ctx, OAIS_EINVAL, "a shard's round needs the global statistics: use oais_round_local/commit");
    const int T = (int)ctx->beta.size() - 1;
    cudaStream_t s = ctx->stream;
    CK(cudaMemcpyAsync(ctx->d_beta, ctx->beta.data(), sizeof(double) * (T + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_eps, ctx->eps.data(), sizeof(double) * T, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s));
    const uint32_t tag = (uint32_t)(ctx->round & 0xFFFF) | ((uint32_t)ctx->problem << 16);
    const int grid = sweep_grid(ctx->N);
    const double logN = std::log((double)ctx->N);
    // the fp32 roundings of the schedule for the fp32 forms of the CUDA-core sweep
    ctx->h_fsched.assign(3 * (size_t)T + 1, 0.0f);
    for (int t = 0; t <= T; ++t) ctx->h_fsched[t] = (float)ctx->beta[t];
    for (int t = 1; t <= T; ++t) {
        ctx->h_fsched[T + t] = (float)(ctx->beta[t] - ctx->beta[t - 1]);
        ctx->h_fsched[2 * T + t] = (float)ctx->eps[t - 1];
    }
    CK(cudaMemcpyAsync(ctx->d_fsched, ctx->h_fsched.data(), sizeof(float) * ctx->h_fsched.size(),
                       cudaMemcpyHostToDevice, s));
    std::vector<double> lg(3 * T), acc(T), elbo(T), ess_tr;
    std::vector<int> rs;
    unsigned status = 0;
    double logZ, ess, se;
    int n_res = 0;
    if (!asmc) {
        SweepParams P = make_params(ctx, T, ctx->d_beta, ctx->d_eps, ctx->seed, tag, ctx->n_offset, ctx->N,
                                    ctx->d_logw, ctx->d_ell, ctx->d_x, ctx->d_parts, ctx->d_status);
        CK(cudaEventRecord(ctx->ev0, s));
        // the resident form hands a split tile's gradient over in the ASMC gradient buffer
        if (ctx->dt.tc) CK(launch_sweep_tc(P, ctx->dt.tc_img, ctx->dt.tc_ybits, ctx->dt.n, ctx->dt.d,
                                           static_cast<float*>(ctx->d_g0), ctx->dt.tc_handed, s));
        else if (ctx->dt.tcs)
            CK(launch_sweep_tcs(tcs_plan(ctx->dt.kind, ctx->dt.n, ctx->dt.d, 0, 0, ctx->dt.tcs_q8), ctx->dt.kind, P, ctx->dt.tcs_img,
                                ctx->dt.tcs_state, ctx->mv.kind, ctx->mv.leapfrog, ctx->dt.p0, ctx->dt.n,
                                ctx->dt.d, s, ctx->dt.tc_handed));
        else if (ctx->dt.wide) CK(launch_sweep_wide(ctx->dt, ctx->mv.kind, P, s));
        else {
            DevTarget dt = ctx->dt;
            dt.fsched = ctx->d_fsched;
            CK(launch_sweep(dt, ctx->mv.kind, P, s));
        }
        CK(cudaEventRecord(ctx->ev1, s));
        if (ctx->exact_data) {
            // the last target of the sequence: gamma(.; X) instead of gamma(.; X~), reached from
            // x_T with the incremental weight L(x_T; X) / L(x_T; X~) (fp32 CUDA-core evaluation of X)
            PotentialParams pp{ctx->N, ctx->d_x, ctx->d_ell1, nullptr};
            CK(ctx->dt.kind == kLogreg ? launch_potential_logreg(ctx->dt, pp, s) : launch_potential_linreg(ctx->dt, pp, s));
            CK(launch_reweight_to_data(ctx->d_logw, ctx->d_ell, ctx->d_ell1, ctx->N, ctx->d_status, s));
        }
        const int records = ctx->dt.tc ? tc_records(ctx->N)
                          : (ctx->dt.tcs ? tcs_tiles(ctx->N) : (ctx->dt.wide ? wide_tiles(ctx->N) : grid));
        CK(launch_merge_stats(ctx->d_parts, records, T,
                              1.0 / ((double)ctx->N * ctx->mv.moves), ctx->d_log_ghat, ctx->d_accept, ctx->d_elbo, s));
        CK(launch_logsumexp(ctx->d_logw, ctx->N, ctx->d_lse, ctx->d_lse_scratch, s));
        double lse[2];
        CK(cudaMemcpyAsync(lg.data(), ctx->d_log_ghat, sizeof(double) * 3 * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(acc.data(), ctx->d_accept, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(elbo.data(), ctx->d_elbo, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(lse, ctx->d_lse, sizeof(lse), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (local_only) {
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
            if (status & 2u) return fail(ctx, OAIS_ETIMEOUT, "a tensor-core completion wait gave up");
            if (status & 4u) return fail(ctx, OAIS_ECUDA, "shared memory base not 1024-byte aligned");
            if (status & 1u) return fail(ctx, OAIS_ENONFINITE, "non-finite log-weight or log-likelihood");
            ctx->pend_T = T;
            ctx->pend_ms = ms;
            ctx->pend_lg = lg;
            ctx->pend_acc.resize(T);
            for (int t = 0; t < T; ++t) ctx->pend_acc[t] = std::round(acc[t] * (double)ctx->N * ctx->mv.moves);
            ctx->pend_lse[0] = lse[0];
            ctx->pend_lse[1] = lse[1];
            return OAIS_OK;
        }
        logZ = lse[0] - logN;
        ess = std::exp(2.0 * lse[0] - lse[1]);
        se = std::sqrt(std::max(0.0, 1.0 / ess - 1.0 / (double)ctx->N));
    } else {
        if (ctx->N_total != ctx->N) return fail(ctx, OAIS_EUNSUPPORTED, "ASMC resamples globally: no shards");
        if ((ctx->dt.D == 0 || ctx->dt.wide) && !ctx->dt.tcs)
            return fail(ctx, OAIS_EUNSUPPORTED,
                        "resampling rounds need the one-thread-per-particle CUDA-core form (d <= 32) or the streamed form");
        CK(cudaMemsetAsync(ctx->d_st, 0, sizeof(AsmcState), s));
        StepParams P = make_step_params(ctx, T, tag);
        const bool grad = ctx->mv.kind != OAIS_RWMH;
        int records = grid;
        CK(cudaEventRecord(ctx->ev0, s));
        if (ctx->dt.tcs) {
            // the streamed tensor-core form: one launch per step over the stored particle state
            const TcsPlan tp = tcs_plan(ctx->dt.kind, ctx->dt.n, ctx->dt.d, 0, 0, ctx->dt.tcs_q8);
            SweepParams S = make_params(ctx, T, ctx->d_beta, ctx->d_eps, ctx->seed, tag, 0, ctx->N, ctx->d_logw,
                                        ctx->d_ell, ctx->d_x, ctx->d_parts, ctx->d_status);
            records = tcs_tiles(ctx->N);
            for (int t = 0; t <= T; ++t) {
                CK(launch_step_tcs(tp, ctx->dt.kind, S, ctx->dt.tcs_img, ctx->dt.tcs_state, ctx->mv.kind,
                                   ctx->mv.leapfrog, ctx->dt.p0, ctx->dt.n, ctx->dt.d, t, ctx->d_ess_parts, s));
                if (t == 0) continue;
                P.t = t;
                CK(launch_asmc_decide_scan(ctx->d_st, P, records, ess_frac, ctx->d_bsum, ctx->d_boff, ctx->d_cdf,
                                           ctx->d_ess_trace, ctx->d_resampled, s));
                CK(launch_gather_tcs(tp, ctx->d_st, ctx->d_cdf, ctx->N, ctx->dt.tcs_state, ctx->d_ell, ctx->d_ell1,
                                     ctx->d_logw, ctx->d_anc, s));
            }
        } else {
            CK(launch_asmc(ctx->dt, ctx->mv.kind, true, P, s));
            for (int t = 1; t <= T; ++t) {
                P.t = t;
                CK(launch_asmc(ctx->dt, ctx->mv.kind, false, P, s));
                CK(launch_asmc_resample(ctx->d_st, P, grid, ess_frac, ctx->dt.d, grad, f64_kind(ctx->dt.kind),
                                        ctx->d_bsum, ctx->d_boff, ctx->d_cdf, ctx->d_ess_trace, ctx->d_resampled,
                                        ctx->d_anc, s));
            }
        }
        CK(cudaEventRecord(ctx->ev1, s));
        CK(launch_merge_stats(ctx->d_parts, records, T, 1.0 / ((double)ctx->N * ctx->mv.moves),
                              ctx->d_log_ghat, ctx->d_accept, ctx->d_elbo, s));
        AsmcState st;
        ess_tr.resize(T);
        rs.resize(T);
        CK(cudaMemcpyAsync(lg.data(), ctx->d_log_ghat, sizeof(double) * 3 * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(acc.data(), ctx->d_accept, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(elbo.data(), ctx->d_elbo, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&st, ctx->d_st, sizeof(st), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(ess_tr.data(), ctx->d_ess_trace, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(rs.data(), ctx->d_resampled, sizeof(int) * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // the particles of the last step live in buffer cur (no resampling is pending at t = T)
        if (!ctx->dt.tcs && (st.cur ^ st.pend) == 1) {
            const size_t xb = elt_bytes(ctx->dt.kind) * (size_t)ctx->dt.d * ctx->N;
            CK(cudaMemcpyAsync(ctx->d_x, ctx->d_x1, xb, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(ctx->d_ell, ctx->d_ell1, sizeof(double) * ctx->N, cudaMemcpyDeviceToDevice, s));
            CK(cudaStreamSynchronize(s));
        }
        logZ = st.logZ;
        n_res = st.n_resample;
        ess = ess_tr[T - 1];
        // delta-method variance of a product of independent segment means
        double v = 0.0;
        for (int t = 0; t < T; ++t) if (rs[t]) v += std::max(0.0, 1.0 / ess_tr[t] - 1.0 / (double)ctx->N);
        se = std::sqrt(v);
    }
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (status & 2u) return fail(ctx, OAIS_ETIMEOUT, "a tensor-core completion wait gave up");
    if (status & 4u) return fail(ctx, OAIS_ECUDA, "shared memory base not 1024-byte aligned");
    if (status & 1u) return fail(ctx, OAIS_ENONFINITE, "non-finite log-weight or log-likelihood");
    ctx->cur_elbo = elbo;
    return commit_round(ctx, T, T_next, lg, acc, logZ, ess, se, ms, asmc, n_res, ess_tr, rs, out);
}

// Test support: the device copies of the data whose first element an armed NaN-data fault
// overwrites (the CUDA-core layout, the resident tensor-core image, the streamed f16 image),
// with the width of that element
struct FaultSite { void* p; size_t bytes; };
static std::vector<FaultSite> fault_sites(const oais_ctx* ctx)
{
    std::vector<FaultSite> v;
    if (ctx->dt.D > 0 && ctx->dt.X) v.push_back({ctx->dt.X, f64_kind(ctx->dt.kind) ? sizeof(double) : sizeof(float)});
    if (ctx->dt.tc && ctx->dt.tc_img) v.push_back({ctx->dt.tc_img, 2});
    if (ctx->dt.tcs && ctx->dt.tcs_img && !ctx->dt.tcs_q8) v.push_back({ctx->dt.tcs_img, 2});
    return v;
}

static oais_status run_round(oais_ctx* ctx, int32_t T_next, bool asmc, double ess_frac, oais_round_result* out,
                             bool local_only = false)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (ctx->fault_kind != OAIS_FAULT_NAN_DATA) {
        const oais_status st = run_round_impl(ctx, T_next, asmc, ess_frac, out, local_only);
        ctx->fault_kind = OAIS_FAULT_NONE;        // a fault is armed for one round
        return st;
    }
    // NaN data: element 0 of every device copy of X becomes a quiet NaN for this round and gets
    // its value back afterwards (whatever the round's outcome)
    const std::vector<FaultSite> sites = fault_sites(ctx);
    std::vector<uint64_t> saved(sites.size(), 0);
    ctx->fault_kind = OAIS_FAULT_NONE;
    CK(cudaStreamSynchronize(ctx->stream));   // no earlier work of the context still reads X
    for (size_t i = 0; i < sites.size(); ++i) {
        const double qd = NAN;
        const float qf = NAN;
        const uint16_t qh = sites[i].p == ctx->dt.tc_img ? 0x7FC0u : 0x7E00u;   // bf16 / f16 quiet NaN
        const void* q = sites[i].bytes == 8 ? (const void*)&qd : sites[i].bytes == 4 ? (const void*)&qf
                                                                                       : (const void*)&qh;
        CK(cudaMemcpy(&saved[i], sites[i].p, sites[i].bytes, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(sites[i].p, q, sites[i].bytes, cudaMemcpyHostToDevice));
    }
    const oais_status st = run_round_impl(ctx, T_next, asmc, ess_frac, out, local_only);
    const std::string msg = ctx->err;
    cudaStreamSynchronize(ctx->stream);
    for (size_t i = 0; i < sites.size(); ++i)
        CK(cudaMemcpy(sites[i].p, &saved[i], sites[i].bytes, cudaMemcpyHostToDevice));
    ctx->err = msg;
    return st;
}

// Alg. 3 and the carry-over of step sizes from the round's (global) statistics
static oais_status commit_round(oais_ctx* ctx, int T, int32_t T_next, const std::vector<double>& lg,
                                const std::vector<double>& acc, double logZ, double ess, double se, float ms,
                                bool asmc, int n_res, const std::vector<double>& ess_tr,
                                const std::vector<int>& rs, oais_round_result* out)
{
    std::vector<double> beta_next(T_next + 1), D(T), Lam(T + 1);
    optimise_schedule(T, ctx->beta.data(), lg.data(), T_next, beta_next.data(), D.data(), Lam.data());
    std::vector<double> eps_next = next_step_sizes(ctx, ctx->beta, ctx->eps, acc, beta_next);

    ctx->have_last = true;
    ctx->last_asmc = asmc;
    ctx->l_beta = ctx->beta;
    ctx->l_eps = ctx->eps;
    ctx->l_log_ghat = lg;
    ctx->l_D = D;
    ctx->l_accept = acc;
    ctx->l_logZ = logZ;
    ctx->l_ess = ess;
    ctx->l_se = se;
    ctx->l_Lambda = Lam[T];
    ctx->l_n_resample = n_res;
    ctx->l_ess_trace = ess_tr;
    ctx->l_resampled = rs;
    // ELBO = sum_t sum_n W_{t-1}^n log g_t^n and KL = log Z_hat - ELBO (log Z = ELBO + KL);
    // not formed for a sharded round (its terms are per shard)
    double elbo = NAN;
    if ((int)ctx->cur_elbo.size() == T) {
        elbo = 0.0;
        for (int t = 0; t < T; ++t) elbo += ctx->cur_elbo[t];
    }
    ctx->l_elbo = ctx->cur_elbo;
    ctx->cur_elbo.clear();
    if (out) {
        out->logZ = logZ;
        out->se = se;
        out->Lambda_hat = Lam[T];
        out->ess = ess;
        out->sweep_ms = ms;
        out->T = T;
        out->round = ctx->round;
        out->n_resample = n_res;
        out->pad = 0;
        out->elbo = elbo;
        out->kl = logZ - elbo;
    }
    ctx->beta = beta_next;
    ctx->eps = eps_next;
    ++ctx->round;
    return OAIS_OK;
}

oais_status oais_round(oais_ctx* ctx, int32_t T_next, oais_round_result* out)
{
    return run_round(ctx, T_next, false, 0.0, out);
}

// The online conditional-ESS comparator (Zhou, Johansen & Aston 2016; the paper's section on
// the connection to online CESS optimisation): lock-step particles as in oasmc_round, but
// beta_t is found on the device before step t (zja.cu) so that CESS_t / N = cess_frac; the
// run ends at beta = 1 (at most T_max steps, the last one forced to beta = 1).  The host
// reads beta once every kZjaCheck steps; steps launched after the one that reached beta = 1
// find the device flag set and do nothing.
constexpr int kZjaCheck = 8;

oais_status oais_zja_round(oais_ctx* ctx, double cess_frac, double ess_frac, int32_t T_next, oais_round_result* out)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (!(cess_frac > 0.0 && cess_frac < 1.0)) return fail(ctx, OAIS_EINVAL, "cess_frac must be in (0, 1)");
    if (!(ess_frac >= 0.0 && ess_frac <= 1.0 + 1e-12)) return fail(ctx, OAIS_EINVAL, "ess_frac must be in [0, 1]");
    if (T_next < 1 || T_next > ctx->T_max) return fail(ctx, OAIS_EINVAL, "T_next out of range");
    if (ctx->N_total != ctx->N) return fail(ctx, OAIS_EUNSUPPORTED, "the online schedule needs every particle: no shards");
    if (ctx->dt.D == 0 || ctx->dt.wide)
        return fail(ctx, OAIS_EUNSUPPORTED, "online-CESS rounds run on the one-thread-per-particle CUDA-core form");
    cudaStream_t s = ctx->stream;
    const int T_ref = (int)ctx->beta.size() - 1;
    const int T_max = ctx->T_max;
    // the current schedule is the step-size reference (log eps interpolated in beta)
    CK(cudaMemcpyAsync(ctx->d_beta, ctx->beta.data(), sizeof(double) * (T_ref + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_eps, ctx->eps.data(), sizeof(double) * T_ref, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s));
    CK(cudaMemsetAsync(ctx->d_st, 0, sizeof(AsmcState), s));
    const ZjaState z0{0.0, 1.0, 0.0, 0, 0};
    const double b0 = 0.0;
    CK(cudaMemcpyAsync(ctx->d_zstate, &z0, sizeof(z0), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_zbeta, &b0, sizeof(double), cudaMemcpyHostToDevice, s));
    const uint32_t tag = (uint32_t)(ctx->round & 0xFFFF) | ((uint32_t)ctx->problem << 16);
    StepParams P = make_step_params(ctx, T_max, tag);
    P.beta = ctx->d_zbeta;
    P.eps = ctx->d_zeps;
    P.skip = &ctx->d_zstate->skip;
    const int grid = sweep_grid(ctx->N);
    const bool grad = ctx->mv.kind != OAIS_RWMH;
    CK(cudaEventRecord(ctx->ev0, s));
    CK(launch_asmc(ctx->dt, ctx->mv.kind, true, P, s));
    int T = 0;
    for (int t = 1; t <= T_max; ++t) {
        CK(launch_zja_search(ctx->d_zstate, ctx->d_st, P, ctx->d_zfg, ctx->d_zanchor, ctx->d_zpart, cess_frac, t,
                             T_max, ctx->d_zbeta, ctx->d_zeps, ctx->d_beta, ctx->d_eps, T_ref, s));
        P.t = t;
        CK(launch_asmc(ctx->dt, ctx->mv.kind, false, P, s));
        CK(launch_asmc_resample(ctx->d_st, P, grid, ess_frac, ctx->dt.d, grad, f64_kind(ctx->dt.kind), ctx->d_bsum,
                                ctx->d_boff, ctx->d_cdf, ctx->d_ess_trace, ctx->d_resampled, ctx->d_anc, s));
        if (t % kZjaCheck == 0 || t == T_max) {
            double bp = 0.0;
            CK(cudaMemcpyAsync(&bp, &ctx->d_zstate->beta_prev, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (bp >= 1.0 || t == T_max) {
                // the step that reached beta = 1: the first one since this round began
                std::vector<double> zb_head(t + 1);
                CK(cudaMemcpyAsync(zb_head.data(), ctx->d_zbeta, sizeof(double) * (t + 1), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                T = t;
                for (int u = 1; u <= t; ++u)
                    if (zb_head[u] >= 1.0) { T = u; break; }
                break;
            }
        }
    }
    CK(cudaEventRecord(ctx->ev1, s));
    std::vector<double> lg(3 * T), acc(T), elbo(T), ess_tr(T), zb(T + 1), ze(T);
    std::vector<int> rs(T);
    CK(launch_merge_stats(ctx->d_parts, grid, T, 1.0 / ((double)ctx->N * ctx->mv.moves), ctx->d_log_ghat,
                          ctx->d_accept, ctx->d_elbo, s));
    AsmcState st;
    unsigned status = 0;
    CK(cudaMemcpyAsync(lg.data(), ctx->d_log_ghat, sizeof(double) * 3 * T, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(acc.data(), ctx->d_accept, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(elbo.data(), ctx->d_elbo, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&st, ctx->d_st, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ess_tr.data(), ctx->d_ess_trace, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rs.data(), ctx->d_resampled, sizeof(int) * T, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(zb.data(), ctx->d_zbeta, sizeof(double) * (T + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ze.data(), ctx->d_zeps, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // the particles of the last step live in buffer cur (no resampling is pending at beta = 1)
    if ((st.cur ^ st.pend) == 1) {
        const size_t xb = elt_bytes(ctx->dt.kind) * (size_t)ctx->dt.d * ctx->N;
        CK(cudaMemcpyAsync(ctx->d_x, ctx->d_x1, xb, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->d_ell, ctx->d_ell1, sizeof(double) * ctx->N, cudaMemcpyDeviceToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (status & 1u) return fail(ctx, OAIS_ENONFINITE, "non-finite log-weight or log-likelihood");
    double v = 0.0;
    for (int t = 0; t < T; ++t) if (rs[t]) v += std::max(0.0, 1.0 / ess_tr[t] - 1.0 / (double)ctx->N);
    // the schedule that ran is the round's (its moments give D_hat and the next schedule)
    ctx->beta = zb;
    ctx->eps = ze;
    ctx->cur_elbo = elbo;
    return commit_round(ctx, T, T_next, lg, acc, st.logZ, ess_tr[T - 1], std::sqrt(v), ms, true, st.n_resample,
                        ess_tr, rs, out);
}

oais_status oasmc_round(oais_ctx* ctx, int32_t T_next, double ess_frac, oais_round_result* out)
{
    return run_round(ctx, T_next, true, ess_frac, out);
}

// ---- checkpoint / resume of the round state (Alg. 2 between rounds) ----
static const uint64_t kStateMagic = 0x4F41495353543031ull;   // "OAISST01"

struct StateHeader {
    uint64_t magic;
    int64_t N, N_total, n_offset;
    uint64_t seed;
    int32_t round, T, kind, d, move, moves;
};

size_t state_bytes_for(const oais_ctx* ctx)
{
    return sizeof(StateHeader) + sizeof(double) * (2 * ctx->beta.size() - 1);
}

oais_status oais_state_bytes(const oais_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return fail(nullptr, OAIS_EINVAL, "null argument");
    *bytes = state_bytes_for(ctx);
    return OAIS_OK;
}

oais_status oais_save_state(const oais_ctx* ctx, void* buf, size_t bytes)
{
    if (!ctx || !buf) return fail(nullptr, OAIS_EINVAL, "null argument");
    if (bytes < state_bytes_for(ctx)) return fail(nullptr, OAIS_EINVAL, "state buffer too small");
    StateHeader h{kStateMagic, ctx->N, ctx->N_total, ctx->n_offset, ctx->seed, ctx->round,
                  (int32_t)ctx->beta.size() - 1, ctx->dt.kind, ctx->dt.d, ctx->mv.kind, ctx->mv.moves};
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &h, sizeof(h));
    std::memcpy(p + sizeof(h), ctx->beta.data(), sizeof(double) * ctx->beta.size());
    std::memcpy(p + sizeof(h) + sizeof(double) * ctx->beta.size(), ctx->eps.data(), sizeof(double) * ctx->eps.size());
    return OAIS_OK;
}

oais_status oais_load_state(oais_ctx* ctx, const void* buf, size_t bytes)
{
    if (!ctx || !buf) return fail(nullptr, OAIS_EINVAL, "null argument");
    if (bytes < sizeof(StateHeader)) return fail(ctx, OAIS_EINVAL, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kStateMagic) return fail(ctx, OAIS_EINVAL, "not an OAIS state");
    if (h.N != ctx->N || h.kind != ctx->dt.kind || h.d != ctx->dt.d || h.move != ctx->mv.kind ||
        h.moves != ctx->mv.moves)
        return fail(ctx, OAIS_EINVAL, "state belongs to a different problem or move");
    if (h.T < 1 || h.T > ctx->T_max || bytes < sizeof(h) + sizeof(double) * (2 * (size_t)h.T + 1))
        return fail(ctx, OAIS_EINVAL, "bad schedule size in state");
    const double* b = reinterpret_cast<const double*>(static_cast<const char*>(buf) + sizeof(h));
    if (!valid_schedule(b, h.T)) return fail(ctx, OAIS_EINVAL, "bad schedule in state");
    // the same checks as oais_set_schedule (step sizes) and oais_set_shard (particle block)
    for (int t = 0; t < h.T; ++t)
        if (!(b[h.T + 1 + t] > 0.0) || !std::isfinite(b[h.T + 1 + t]))
            return fail(ctx, OAIS_EINVAL, "bad step sizes in state");
    if (h.n_offset < 0 || h.N_total < ctx->N || h.n_offset + ctx->N > h.N_total || h.N_total > 0xFFFFFFFFLL)
        return fail(ctx, OAIS_EINVAL, "bad shard block in state");
    if (h.round < 0) return fail(ctx, OAIS_EINVAL, "bad round index in state");
    ctx->beta.assign(b, b + h.T + 1);
    ctx->eps.assign(b + h.T + 1, b + 2 * h.T + 1);
    ctx->seed = h.seed;
    ctx->round = h.round;
    ctx->n_offset = h.n_offset;
    ctx->N_total = h.N_total;
    ctx->pend_T = 0;
    // the results of a round run before the load belong to another state
    ctx->have_last = false;
    return OAIS_OK;
}

oais_status oais_set_shard(oais_ctx* ctx, int64_t n_offset, int64_t N_total)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (n_offset < 0 || N_total < ctx->N || n_offset + ctx->N > N_total || N_total > 0xFFFFFFFFLL)
        return fail(ctx, OAIS_EINVAL, "shard [n_offset, n_offset + N) must lie in [0, N_total)");
    ctx->n_offset = n_offset;
    ctx->N_total = N_total;
    return OAIS_OK;
}

oais_status oais_round_local(oais_ctx* ctx, double* log_ghat, double* accepted, double* lse, int32_t* T)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    oais_status st = run_round(ctx, ctx->T_max, false, 0.0, nullptr, true);
    if (st != OAIS_OK) return st;
    const int t = ctx->pend_T;
    if (T) *T = t;
    if (log_ghat) std::copy(ctx->pend_lg.begin(), ctx->pend_lg.end(), log_ghat);
    if (accepted) std::copy(ctx->pend_acc.begin(), ctx->pend_acc.end(), accepted);
    if (lse) { lse[0] = ctx->pend_lse[0]; lse[1] = ctx->pend_lse[1]; }
    return OAIS_OK;
}

oais_status oais_round_commit(oais_ctx* ctx, int32_t T_next, const double* log_ghat, const double* accepted,
                              const double* lse, oais_round_result* out)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (ctx->pend_T <= 0) return fail(ctx, OAIS_EINVAL, "no local round to commit");
    if (T_next < 1 || T_next > ctx->T_max) return fail(ctx, OAIS_EINVAL, "T_next out of range");
    if (!log_ghat || !accepted || !lse) return fail(ctx, OAIS_EINVAL, "null global statistics");
    const int T = ctx->pend_T;
    const double Nt = (double)ctx->N_total;
    std::vector<double> lg(log_ghat, log_ghat + 3 * T), acc(T);
    for (int t = 0; t < T; ++t) acc[t] = accepted[t] / (Nt * ctx->mv.moves);
    const double logZ = lse[0] - std::log(Nt);
    const double ess = std::exp(2.0 * lse[0] - lse[1]);
    const double se = std::sqrt(std::max(0.0, 1.0 / ess - 1.0 / Nt));
    ctx->pend_T = 0;
    return commit_round(ctx, T, T_next, lg, acc, logZ, ess, se, ctx->pend_ms, false, 0, {}, {}, out);
}

oais_status oais_get_resampling(const oais_ctx* ctx, double* ess, int32_t* resampled, int64_t* ancestors)
{
    if (!ctx || !ctx->have_last) return fail(nullptr, OAIS_EINVAL, "no completed round");
    if (!ctx->last_asmc) return fail(nullptr, OAIS_EINVAL, "the last round did not resample (OAIS)");
    if (ess) std::copy(ctx->l_ess_trace.begin(), ctx->l_ess_trace.end(), ess);
    if (resampled) std::copy(ctx->l_resampled.begin(), ctx->l_resampled.end(), resampled);
    if (ancestors) {
        cudaError_t e = cudaMemcpy(ancestors, ctx->d_anc, sizeof(int64_t) * ctx->N, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(nullptr, OAIS_ECUDA, cudaGetErrorString(e));
    }
    return OAIS_OK;
}

oais_status asmc_run(const oais_target* target, const oais_move* move, int64_t N, const double* beta,
                     int32_t T, const double* eps, double ess_frac, uint64_t seed, void* stream,
                     oais_round_result* out, double* log_ghat, double* ess_trace, int32_t* resampled)
{
    oais_ctx* ctx = nullptr;
    oais_status st = oais_init(&ctx, target, move, N, beta, T, T, eps, seed, nullptr, 0, stream);
    if (st != OAIS_OK) return st;
    st = oasmc_round(ctx, T, ess_frac, out);
    if (st == OAIS_OK && log_ghat) std::copy(ctx->l_log_ghat.begin(), ctx->l_log_ghat.end(), log_ghat);
    if (st == OAIS_OK) st = oais_get_resampling(ctx, ess_trace, resampled, nullptr);
    if (st != OAIS_OK) g_err = ctx->err.empty() ? g_err : ctx->err;
    oais_destroy(ctx);
    return st;
}

oais_status oais_logZ(const oais_ctx* ctx, double* logZ, double* se)
{
    if (!ctx || !ctx->have_last) return fail(nullptr, OAIS_EINVAL, "no completed round");
    if (logZ) *logZ = ctx->l_logZ;
    if (se) *se = ctx->l_se;
    return OAIS_OK;
}

oais_status oais_get_stats(const oais_ctx* ctx, double* log_ghat, double* D_hat, double* beta, double* accept,
                           int32_t* T)
{
    if (!ctx || !ctx->have_last) return fail(nullptr, OAIS_EINVAL, "no completed round");
    const int t = (int)ctx->l_D.size();
    if (T) *T = t;
    if (log_ghat) std::copy(ctx->l_log_ghat.begin(), ctx->l_log_ghat.end(), log_ghat);
    if (D_hat) std::copy(ctx->l_D.begin(), ctx->l_D.end(), D_hat);
    if (beta) std::copy(ctx->l_beta.begin(), ctx->l_beta.end(), beta);
    if (accept) std::copy(ctx->l_accept.begin(), ctx->l_accept.end(), accept);
    return OAIS_OK;
}

oais_status oais_get_elbo(const oais_ctx* ctx, double* elbo_terms, int32_t* T)
{
    if (!ctx || !ctx->have_last) return fail(nullptr, OAIS_EINVAL, "no completed round");
    if ((int)ctx->l_elbo.size() != (int)ctx->l_D.size())
        return fail(nullptr, OAIS_EINVAL, "the last round was a sharded round: no ELBO terms");
    if (T) *T = (int32_t)ctx->l_elbo.size();
    if (elbo_terms) std::copy(ctx->l_elbo.begin(), ctx->l_elbo.end(), elbo_terms);
    return OAIS_OK;
}

oais_status oais_get_schedule(const oais_ctx* ctx, double* beta, double* eps, int32_t* T)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (T) *T = (int32_t)ctx->beta.size() - 1;
    if (beta) std::copy(ctx->beta.begin(), ctx->beta.end(), beta);
    if (eps) std::copy(ctx->eps.begin(), ctx->eps.end(), eps);
    return OAIS_OK;
}

oais_status oais_set_schedule(oais_ctx* ctx, const double* beta, const double* eps, int32_t T)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (T > ctx->T_max || !valid_schedule(beta, T))
        return fail(ctx, OAIS_EINVAL, "schedule must be 0 = beta_0 < ... < beta_T = 1 with T <= T_max");
    if (eps) for (int t = 0; t < T; ++t) if (!(eps[t] > 0)) return fail(ctx, OAIS_EINVAL, "step sizes must be > 0");
    ctx->beta.assign(beta, beta + T + 1);
    if (eps) ctx->eps.assign(eps, eps + T);
    else ctx->eps.assign(T, 0.5 / std::sqrt((double)ctx->dt.d));
    return OAIS_OK;
}

oais_status oais_particles(const oais_ctx* ctx, const double** logw, const double** ell, const void** x)
{
    if (!ctx || !ctx->have_last) return fail(nullptr, OAIS_EINVAL, "no completed round");
    if (logw) *logw = ctx->d_logw;
    if (ell) *ell = ctx->d_ell;
    if (x) *x = ctx->d_x;
    return OAIS_OK;
}

oais_status oais_grad_logZ(oais_ctx* ctx, double* grad)
{
    if (!ctx || !ctx->have_last) return fail(nullptr, OAIS_EINVAL, "no completed round");
    if (!grad) return fail(ctx, OAIS_EINVAL, "null grad");
    cudaStream_t s = ctx->stream;
    // log-sum-exp of the final weights, then the weighted sums of grad_theta log gamma
    CK(launch_logsumexp(ctx->d_logw, ctx->N, ctx->d_lse, ctx->d_lse_scratch, s));
    CK(launch_fisher(ctx->d_logw, ctx->d_ell, ctx->d_x, f64_kind(ctx->dt.kind), ctx->N, ctx->dt.d, ctx->d_lse,
                     ctx->dt.ref_scale, ctx->dt.kind, ctx->dt.n, ctx->dt.p0, ctx->d_lse_scratch,
                     ctx->d_lse, s));
    double g[2];
    CK(cudaMemcpyAsync(g, ctx->d_lse, sizeof(g), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // UNID: the reference is fixed (it makes X and Y uniform), no scale to differentiate
    grad[0] = ctx->dt.kind == kUnid ? NAN : g[0];
    grad[1] = (ctx->dt.kind == kGauss || ctx->dt.kind == kLinreg) ? g[1] : NAN;
    return OAIS_OK;
}

oais_status oais_potential(oais_ctx* ctx, const void* d_x, int64_t N, double* d_ell, void* d_grad, void* stream)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (!d_x || !d_ell || N < 1) return fail(ctx, OAIS_EINVAL, "bad arguments to oais_potential");
    if (ctx->dt.tcs) {
        if (N > 0xFFFFFFFFLL) return fail(ctx, OAIS_EINVAL, "N out of range");
        CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), static_cast<cudaStream_t>(stream)));
        CK(launch_potential_tcs(tcs_plan(ctx->dt.kind, ctx->dt.n, ctx->dt.d, 0, 0, ctx->dt.tcs_q8), ctx->dt.kind, ctx->dt.tcs_img,
                                static_cast<const float*>(d_x), N, d_ell, static_cast<float*>(d_grad), ctx->dt.p0,
                                ctx->dt.n, ctx->dt.d, ctx->d_status, ctx->dt.tcs_state,
                                (int64_t)tcs_tiles(ctx->N) * 128, static_cast<cudaStream_t>(stream)));
        unsigned status = 0;
        CK(cudaMemcpyAsync(&status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           static_cast<cudaStream_t>(stream)));
        CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        if (status & 2u) return fail(ctx, OAIS_ETIMEOUT, "a tensor-core completion wait gave up");
        if (status & 4u) return fail(ctx, OAIS_ECUDA, "shared memory base not 1024-byte aligned");
        return OAIS_OK;
    }
    if (ctx->dt.wide) {
        CK(launch_potential_wide(ctx->dt, static_cast<const float*>(d_x), N, d_ell, static_cast<float*>(d_grad),
                                 static_cast<cudaStream_t>(stream)));
        return OAIS_OK;
    }
    if (ctx->dt.D == 0) return fail(ctx, OAIS_EUNSUPPORTED, "no CUDA-core form for this dimension");
    PotentialParams P{N, d_x, d_ell, d_grad};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (ctx->dt.kind) {
    case kGauss: CK(launch_potential_gauss(ctx->dt, P, s)); break;
    case kUnid: CK(launch_potential_unid(ctx->dt, P, s)); break;
    case kLogreg: CK(launch_potential_logreg(ctx->dt, P, s)); break;
    case kGmm: CK(launch_potential_gmm(ctx->dt, P, s)); break;
    case kLinreg: CK(launch_potential_linreg(ctx->dt, P, s)); break;
    }
    return OAIS_OK;
}

} // extern "C"

// ---------------------------------------------------------------------------------------
// Batched problems: P independent OAIS runs (Alg. 2 each) whose sweeps share one persistent
// launch of the streamed tensor-core kernel.  Each problem keeps its own context (data,
// particles, statistics, schedule; problem index p in the random-number tag), so every
// problem's round is the same computation as a single run with that index.
// ---------------------------------------------------------------------------------------
struct oais_batch {
    int P = 0, kind = 0, T_max = 0;
    int64_t N = 0;
    std::vector<oais_ctx*> ctx;
    cudaStream_t stream = nullptr;        // the caller's stream
    cudaStream_t work = nullptr;          // the batch's own stream (captured; the default stream cannot be)
    cudaEvent_t ready = nullptr;
    int stages_class[4] = {0, 0, 0, 0};   // ring depth per d_pad class 16/32/64/128 (0: largest that fits)
    int chunk_class[4] = {0, 0, 0, 0};    // rows per X chunk per class (0: the default, 64)
    int h = 2;                            // column split of the batched kernel
    std::vector<TcsPlan> plan;
    uint32_t off_misc = 0, smem = 0;
    size_t pbytes = 0, sched_stride = 0, out_stride = 0;
    unsigned char* d_params = nullptr;
    uint2* d_items = nullptr;
    uint32_t n_items = 0;
    uint32_t* d_head = nullptr;
    double* d_sched = nullptr;
    unsigned* d_status = nullptr;
    unsigned char* h_params = nullptr;
    double* h_sched = nullptr;
    double* h_out = nullptr;
    unsigned* h_status = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_T = -1;
    int grid = 0;
    std::string err;
};

static int dp_class(int dp) { return dp <= 16 ? 0 : dp <= 32 ? 1 : dp <= 64 ? 2 : 3; }

static oais_status batch_fail(oais_batch* b, oais_status s, const std::string& m)
{
    if (b) b->err = m; else g_err = m;
    return s;
}

#define BK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return batch_fail(b, OAIS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// shared-memory plans of every problem and the common Misc offset; drops the captured graph
static void batch_plan(oais_batch* b)
{
    b->plan.resize(b->P);
    uint32_t top = 0;
    // one launch, one column split: the problems' own (default) split if they all agree, else 2
    int h = 0;
    for (int p = 0; p < b->P; ++p) {
        const DevTarget& dt = b->ctx[p]->dt;
        const int hp = tcs_plan(dt.kind, dt.n, dt.d, 0, 0, false, 0, dt.tcs_dp).h;
        h = (p == 0 || h == hp) ? hp : 2;
    }
    b->h = h;
    for (int p = 0; p < b->P; ++p) {
        const DevTarget& dt = b->ctx[p]->dt;
        const int ch = b->chunk_class[dp_class(dt.tcs_dp)];
        TcsPlan L = tcs_plan(dt.kind, dt.n, dt.d, ch, 0, false, h, dt.tcs_dp);
        const int want = b->stages_class[dp_class(L.dp)];
        if (want > 0 && want < L.stages) L = tcs_plan(dt.kind, dt.n, dt.d, ch, want, false, h, dt.tcs_dp);
        b->plan[p] = L;
        top = std::max(top, L.off_x + (uint32_t)L.stages * L.stage_bytes);
    }
    b->off_misc = (top + 1023u) & ~1023u;
    b->smem = b->off_misc + tcs_misc_bytes();
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->graph_T = -1;
}

// (problem, tile) items, longest first: a tile of problem p costs ~ chunks x (d_pad + 64)
static void batch_items(oais_batch* b, std::vector<uint2>& items)
{
    items.clear();
    std::vector<std::pair<double, uint2>> c;
    const uint32_t tiles = (uint32_t)tcs_tiles(b->N);
    for (int p = 0; p < b->P; ++p) {
        const double cost = (double)b->plan[p].nch * (b->plan[p].dp + 64);
        for (uint32_t t = 0; t < tiles; ++t) c.push_back({cost, make_uint2((uint32_t)p, t)});
    }
    std::stable_sort(c.begin(), c.end(), [](const auto& a, const auto& z) { return a.first > z.first; });
    for (auto& e : c) items.push_back(e.second);
}

// every problem's parameter block for a round at schedule length T
static void batch_fill(oais_batch* b, int T)
{
    for (int p = 0; p < b->P; ++p) {
        oais_ctx* c = b->ctx[p];
        double* sb = b->h_sched + (size_t)p * b->sched_stride;
        std::copy(c->beta.begin(), c->beta.end(), sb);
        std::copy(c->eps.begin(), c->eps.end(), sb + b->T_max + 1);
        const double* db = b->d_sched + (size_t)p * b->sched_stride;
        const uint32_t tag = (uint32_t)(c->round & 0xFFFF) | ((uint32_t)c->problem << 16);
        SweepParams sp = make_params(c, T, db, db + b->T_max + 1, c->seed, tag, c->n_offset, c->N, c->d_logw, c->d_ell,
                                     c->d_x, c->d_parts, b->d_status + p);
        tcs_batch_params(b->plan[p], c->dt.kind, sp, c->dt.tcs_img, c->dt.tcs_state, c->mv.kind, c->mv.leapfrog,
                         c->dt.p0, c->dt.n, c->dt.d, b->off_misc, b->h_params + (size_t)p * b->pbytes);
    }
}

// the round's device work: schedules and parameter blocks in, the persistent sweep, then per
// problem the merge of the moment records, the log-sum-exp of the final weights and the
// copies of the statistics out (captured once per schedule length as a CUDA graph)
static oais_status batch_enqueue(oais_batch* b, int T)
{
    cudaStream_t s = b->work;
    BK(cudaMemcpyAsync(b->d_sched, b->h_sched, sizeof(double) * b->sched_stride * b->P, cudaMemcpyHostToDevice, s));
    BK(cudaMemcpyAsync(b->d_params, b->h_params, b->pbytes * b->P, cudaMemcpyHostToDevice, s));
    BK(cudaMemsetAsync(b->d_status, 0, sizeof(unsigned) * b->P, s));
    BK(cudaMemsetAsync(b->d_head, 0, sizeof(uint32_t), s));
    // external records: inside a captured graph a plain record only orders the capture
    BK(cudaEventRecordWithFlags(b->ev0, s, cudaEventRecordExternal));
    bool alt = false;   // some class runs chunks of other than 64 rows
    for (const TcsPlan& L : b->plan) alt = alt || L.chunk != 64;
    BK(launch_sweep_tcs_batch(b->kind, b->h, b->d_params, b->d_items, b->n_items, b->d_head, b->off_misc, b->smem,
                              b->grid, s, alt));
    BK(cudaEventRecordWithFlags(b->ev1, s, cudaEventRecordExternal));
    for (int p = 0; p < b->P; ++p) {
        oais_ctx* c = b->ctx[p];
        BK(launch_merge_stats(c->d_parts, tcs_tiles(c->N), T, 1.0 / ((double)c->N * c->mv.moves), c->d_log_ghat,
                              c->d_accept, c->d_elbo, s));
        BK(launch_logsumexp(c->d_logw, c->N, c->d_lse, c->d_lse_scratch, s));
        double* o = b->h_out + (size_t)p * b->out_stride;
        BK(cudaMemcpyAsync(o, c->d_log_ghat, sizeof(double) * 3 * T, cudaMemcpyDeviceToHost, s));
        BK(cudaMemcpyAsync(o + 3 * b->T_max, c->d_accept, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
        BK(cudaMemcpyAsync(o + 4 * b->T_max, c->d_lse, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        BK(cudaMemcpyAsync(o + 4 * b->T_max + 2, c->d_elbo, sizeof(double) * T, cudaMemcpyDeviceToHost, s));
    }
    BK(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(unsigned) * b->P, cudaMemcpyDeviceToHost, s));
    return OAIS_OK;
}

extern "C" {

oais_status oais_batch_init(oais_batch** out, int32_t P, const oais_target* targets, const oais_move* move,
                            int64_t N, const double* beta, int32_t T, int32_t T_max, const double* eps,
                            uint64_t seed, void* const* workspaces, const size_t* ws_bytes, void* stream)
{
    oais_batch* b = nullptr;
    if (!out) return batch_fail(nullptr, OAIS_EINVAL, "null batch pointer");
    *out = nullptr;
    if (P < 1 || P > 0xFFFF || !targets || !move) return batch_fail(nullptr, OAIS_EINVAL, "bad problem list");
    for (int p = 0; p < P; ++p) {
        if (targets[p].kind != targets[0].kind || (targets[0].kind != kLogreg && targets[0].kind != kLinreg))
            return batch_fail(nullptr, OAIS_EUNSUPPORTED, "a batch holds LOGREG or LINREG problems of one family");
        if (targets[p].d > 128) return batch_fail(nullptr, OAIS_EUNSUPPORTED, "batched problems take d <= 128");
    }
    b = new oais_batch();
    b->P = P;
    b->kind = targets[0].kind;
    b->N = N;
    b->T_max = T_max;
    b->stream = static_cast<cudaStream_t>(stream);
    for (int p = 0; p < P; ++p) {
        oais_target t = targets[p];
        t.contraction = OAIS_CONTRACT_BF16_TC_STREAM;
        oais_ctx* c = nullptr;
        oais_status st = oais_init(&c, &t, move, N, beta, T, T_max, eps ? eps + (size_t)p * T : nullptr, seed,
                                   workspaces ? workspaces[p] : nullptr, ws_bytes ? ws_bytes[p] : 0, stream);
        if (st != OAIS_OK) {
            std::string m = "problem " + std::to_string(p) + ": " + g_err;
            oais_batch_destroy(b);
            return batch_fail(nullptr, st, m);
        }
        c->problem = p;
        b->ctx.push_back(c);
    }
    batch_plan(b);
    std::vector<uint2> items;
    batch_items(b, items);
    b->n_items = (uint32_t)items.size();
    b->pbytes = tcs_params_bytes();   // the kernel indexes the blocks as an array: no padding
    b->sched_stride = 2 * (size_t)T_max + 1;
    b->out_stride = 5 * (size_t)T_max + 2;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, std::min(sms, (int)b->n_items));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_params, b->pbytes * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(uint2) * items.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_head, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sched, sizeof(double) * b->sched_stride * P);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(unsigned) * P);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_params, b->pbytes * P);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_sched, sizeof(double) * b->sched_stride * P);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, sizeof(double) * b->out_stride * P);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(unsigned) * P);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        std::string m = cudaGetErrorString(e);
        oais_batch_destroy(b);
        return batch_fail(nullptr, OAIS_ENOMEM, m);
    }
    *out = b;
    return OAIS_OK;
}

oais_status oais_batch_round(oais_batch* b, int32_t T_next, oais_round_result* results)
{
    if (!b) return batch_fail(nullptr, OAIS_EINVAL, "null batch");
    if (T_next < 1 || T_next > b->T_max) return batch_fail(b, OAIS_EINVAL, "T_next out of range");
    const int T = (int)b->ctx[0]->beta.size() - 1;
    for (oais_ctx* c : b->ctx)
        if ((int)c->beta.size() - 1 != T) return batch_fail(b, OAIS_EINVAL, "problems hold schedules of different lengths");
    batch_fill(b, T);
    // the round follows the caller's earlier work on its stream
    BK(cudaEventRecord(b->ready, b->stream));
    BK(cudaStreamWaitEvent(b->work, b->ready, 0));
    if (!b->gexec || b->graph_T != T) {
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        BK(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal));
        oais_status st = batch_enqueue(b, T);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->work, &g);
        if (st != OAIS_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return batch_fail(b, OAIS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        b->graph = g;
        BK(cudaGraphInstantiate(&b->gexec, b->graph, 0));
        b->graph_T = T;
    }
    BK(cudaGraphLaunch(b->gexec, b->work));
    BK(cudaStreamSynchronize(b->work));
    float ms = 0.0f;
    BK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    oais_status worst = OAIS_OK;
    for (int p = 0; p < b->P; ++p) {
        oais_ctx* c = b->ctx[p];
        const unsigned status = b->h_status[p];
        oais_status st = OAIS_OK;
        if (status & 2u) st = fail(c, OAIS_ETIMEOUT, "a tensor-core completion wait gave up");
        else if (status & 12u) st = fail(c, OAIS_ECUDA, "batched sweep: bad shared-memory base or width");
        else if (status & 1u) st = fail(c, OAIS_ENONFINITE, "non-finite log-weight or log-likelihood");
        if (st == OAIS_OK) {
            const double* o = b->h_out + (size_t)p * b->out_stride;
            std::vector<double> lg(o, o + 3 * T), acc(o + 3 * b->T_max, o + 3 * b->T_max + T);
            const double lse0 = o[4 * b->T_max], lse1 = o[4 * b->T_max + 1];
            const double logZ = lse0 - std::log((double)c->N);
            const double ess = std::exp(2.0 * lse0 - lse1);
            const double se = std::sqrt(std::max(0.0, 1.0 / ess - 1.0 / (double)c->N));
            c->cur_elbo.assign(o + 4 * b->T_max + 2, o + 4 * b->T_max + 2 + T);
            st = commit_round(c, T, T_next, lg, acc, logZ, ess, se, ms, false, 0, {}, {},
                              results ? results + p : nullptr);
        }
        if (st != OAIS_OK && worst == OAIS_OK) {
            worst = st;
            b->err = "problem " + std::to_string(p) + ": " + c->err;
        }
    }
    return worst;
}

// Tile shape per width class, chosen by timing: for each class present, the largest problem
// of the class sweeps T_probe steps (its own data, a linear schedule, the first tiles of its
// particles filling every SM once) through the batched kernel itself, for every candidate
// (rows per X chunk, ring depth): chunks of 64 rows and, where the class's chunk images allow
// it, of 128; ring depths 2, 3, 4, 6, 8 as far as shared memory holds them.  The fastest pair
// is kept.  The probe runs on the problem's own particle buffers (the next round redraws them).
oais_status oais_batch_autotune(oais_batch* b, int32_t T_probe, int32_t* chosen)
{
    if (!b) return batch_fail(nullptr, OAIS_EINVAL, "null batch");
    if (T_probe < 1 || T_probe > b->T_max) return batch_fail(b, OAIS_EINVAL, "T_probe out of range");
    cudaStream_t s = b->work;
    BK(cudaEventRecord(b->ready, b->stream));
    BK(cudaStreamWaitEvent(s, b->ready, 0));
    struct Scratch {
        void* items = nullptr;
        void* params = nullptr;
        ~Scratch() { cudaFree(items); cudaFree(params); }
    } tmp;
    BK(cudaMalloc(&tmp.items, sizeof(uint2) * (size_t)b->grid));
    BK(cudaMalloc(&tmp.params, b->pbytes));
    std::vector<unsigned char> hp(b->pbytes);
    std::vector<double> sched(2 * (size_t)T_probe + 1);
    for (int t = 0; t <= T_probe; ++t) sched[t] = (double)t / T_probe;
    for (int c = 0; c < 4; ++c) {
        int best_p = -1;
        for (int p = 0; p < b->P; ++p)
            if (dp_class(b->plan[p].dp) == c && (best_p < 0 || b->ctx[p]->dt.n > b->ctx[best_p]->dt.n)) best_p = p;
        if (chosen) chosen[c] = 0;
        if (best_p < 0) continue;
        oais_ctx* x = b->ctx[best_p];
        const DevTarget& dt = x->dt;
        for (int t = 0; t < T_probe; ++t) sched[T_probe + 1 + t] = x->eps.empty() ? 0.01 : x->eps[0];
        BK(cudaMemcpyAsync(b->d_sched, sched.data(), sizeof(double) * sched.size(), cudaMemcpyHostToDevice, s));
        const int64_t Nprobe = std::min<int64_t>(x->N, (int64_t)b->grid * 128);
        const int ptiles = tcs_tiles(Nprobe);
        std::vector<uint2> items(ptiles);
        for (int t = 0; t < ptiles; ++t) items[t] = make_uint2(0u, (uint32_t)t);   // the one parameter block
        BK(cudaMemcpyAsync(tmp.items, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice, s));
        // every problem of the class must take the chunk size
        std::vector<int> chunks = {64};
        for (int ch : {128}) {
            bool all = true;
            for (int p = 0; p < b->P; ++p)
                if (dp_class(b->plan[p].dp) == c) all = all && tcs_chunk_ok(b->ctx[p]->dt.kind, b->plan[p].dp, ch, false);
            if (all) chunks.push_back(ch);
        }
        float best_ms = 0.0f;
        int best_S = 0, best_ch = 0;
        for (int ch : chunks) {
            const TcsPlan full = tcs_plan(dt.kind, dt.n, dt.d, ch, 0, false, b->h, dt.tcs_dp);
            for (int S : {2, 3, 4, 6, 8}) {
                if (S > full.stages) break;
                const TcsPlan L = tcs_plan(dt.kind, dt.n, dt.d, ch, S, false, b->h, dt.tcs_dp);
                if (!L.ok) continue;
                const uint32_t off_misc = (L.off_x + (uint32_t)S * L.stage_bytes + 1023u) & ~1023u;
                const uint32_t smem = off_misc + tcs_misc_bytes();
                SweepParams sp = make_params(x, T_probe, b->d_sched, b->d_sched + T_probe + 1, x->seed, 0xFFFFu, 0,
                                             Nprobe, x->d_logw, x->d_ell, x->d_x, x->d_parts, b->d_status);
                tcs_batch_params(L, dt.kind, sp, dt.tcs_img, dt.tcs_state, x->mv.kind, x->mv.leapfrog, dt.p0, dt.n,
                                 dt.d, off_misc, hp.data());
                BK(cudaMemcpyAsync(tmp.params, hp.data(), b->pbytes, cudaMemcpyHostToDevice, s));
                float ms = 0.0f;
                for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
                    BK(cudaMemsetAsync(b->d_head, 0, sizeof(uint32_t), s));
                    BK(cudaEventRecord(b->ev0, s));
                    BK(launch_sweep_tcs_batch(b->kind, b->h, tmp.params, tmp.items, (uint32_t)ptiles, b->d_head,
                                              off_misc, smem, std::min(b->grid, ptiles), s, ch != 64));
                    BK(cudaEventRecord(b->ev1, s));
                    BK(cudaEventSynchronize(b->ev1));
                    BK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
                }
                if (best_S == 0 || ms < best_ms) { best_ms = ms; best_S = S; best_ch = ch; }
            }
        }
        b->stages_class[c] = best_S;
        b->chunk_class[c] = best_ch == 64 ? 0 : best_ch;
        if (chosen) chosen[c] = best_S;
    }
    batch_plan(b);
    return OAIS_OK;
}

oais_status oais_batch_tile_shape(const oais_batch* b, int32_t width_class, int32_t* chunk_rows, int32_t* stages)
{
    if (!b || width_class < 0 || width_class > 3 || !chunk_rows || !stages)
        return batch_fail(nullptr, OAIS_EINVAL, "bad batch, width class or output");
    *chunk_rows = 0;
    *stages = 0;
    for (int p = 0; p < b->P; ++p)
        if (dp_class(b->plan[p].dp) == width_class) {
            *chunk_rows = b->plan[p].chunk;
            *stages = b->plan[p].stages;
            break;
        }
    return OAIS_OK;
}

oais_status oais_batch_set_tile_shape(oais_batch* b, int32_t width_class, int32_t chunk_rows, int32_t stages)
{
    if (!b) return batch_fail(nullptr, OAIS_EINVAL, "null batch");
    if (width_class < 0 || width_class > 3) return batch_fail(b, OAIS_EINVAL, "width class out of range");
    if (stages != 0 && (stages < 2 || stages > 8)) return batch_fail(b, OAIS_EINVAL, "ring depth out of range");
    if (chunk_rows != 0 && chunk_rows != 64 && chunk_rows != 128)
        return batch_fail(b, OAIS_EINVAL, "chunk rows not 64 or 128");
    for (int p = 0; p < b->P; ++p) {
        if (dp_class(b->plan[p].dp) != width_class) continue;
        const int ch = chunk_rows == 0 ? 64 : chunk_rows;
        if (!tcs_chunk_ok(b->ctx[p]->dt.kind, b->plan[p].dp, ch, false))
            return batch_fail(b, OAIS_EUNSUPPORTED, "problem " + std::to_string(p) + " cannot take that chunk size");
    }
    b->chunk_class[width_class] = chunk_rows == 64 ? 0 : chunk_rows;
    b->stages_class[width_class] = stages;
    batch_plan(b);
    return OAIS_OK;
}

oais_status oais_batch_context(oais_batch* b, int32_t p, oais_ctx** ctx)
{
    if (!b || !ctx || p < 0 || p >= b->P) return batch_fail(b, OAIS_EINVAL, "bad problem index");
    *ctx = b->ctx[p];
    return OAIS_OK;
}

const char* oais_batch_last_error(const oais_batch* b) { return b ? b->err.c_str() : g_err.c_str(); }

void oais_batch_destroy(oais_batch* b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->work) cudaStreamDestroy(b->work);
    cudaFree(b->d_params);
    cudaFree(b->d_items);
    cudaFree(b->d_head);
    cudaFree(b->d_sched);
    cudaFree(b->d_status);
    cudaFreeHost(b->h_params);
    cudaFreeHost(b->h_sched);
    cudaFreeHost(b->h_out);
    cudaFreeHost(b->h_status);
    for (oais_ctx* c : b->ctx) oais_destroy(c);
    delete b;
}

// Merge of per-shard round statistics (Sec. 5.1.2: the particles of a round are independent,
// so a sum over all particles is the sum of the shards' sums).  Each moment log g_hat_{t,i} and
// each final-weight sum is a logarithm of a sum over particles: the merge is the log-sum-exp
// over shards, the plain definition (maximum, then the sum of exp(a_p - max) in shard order);
// acceptance counts add.  Every rank calling it on the same inputs gets the same bits.
static double lse_over_shards(const double* a, int P, size_t stride)
{
    double m = -INFINITY;
    for (int p = 0; p < P; ++p) {
        const double v = a[(size_t)p * stride];
        if (std::isnan(v)) return v;
        if (v > m) m = v;
    }
    if (m == -INFINITY || m == INFINITY) return m;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += std::exp(a[(size_t)p * stride] - m);
    return m + std::log(s);
}

oais_status oais_merge_shard_stats(int32_t P, int32_t T, const double* log_ghat, const double* accepted,
                                   const double* lse, double* log_ghat_out, double* accepted_out, double* lse_out)
{
    if (P < 1 || T < 1 || !log_ghat || !accepted || !lse || !log_ghat_out || !accepted_out || !lse_out)
        return fail(nullptr, OAIS_EINVAL, "bad arguments to oais_merge_shard_stats");
    for (int j = 0; j < 3 * T; ++j) log_ghat_out[j] = lse_over_shards(log_ghat + j, P, (size_t)3 * T);
    for (int t = 0; t < T; ++t) {
        double a = 0.0;
        for (int p = 0; p < P; ++p) a += accepted[(size_t)p * T + t];
        accepted_out[t] = a;
    }
    for (int i = 0; i < 2; ++i) lse_out[i] = lse_over_shards(lse + i, P, 2);
    return OAIS_OK;
}

// The starting rule for per-step sizes (a reading: the paper fixes no step sizes): the scale of
// pi_beta along a typical direction, approximated by a Gaussian whose precision is the
// reference's plus beta times a diagonal curvature estimate of -log L, times the usual
// dimension scaling of each kernel (random walk 2.38 / sqrt(d); MALA 1.2 d^(-1/6); HMC
// d^(-1/4)).  Curvature per family: Gaussian 1 / p0^2; logistic (1/4) sum X^2 / d (the
// sigmoid's largest slope); linear regression sum X^2 / (d p0^2); mixture 1 / p0 (a
// component's precision); Unid m q (1 - q)^-1 q^2 with q = k / m (the binomial ridge's
// width in the probit coordinates).
oais_status oais_default_step_sizes(const oais_target* tg, int32_t move_kind, const double* beta, int32_t T,
                                    double* eps)
{
    if (!tg || !beta || !eps || T < 1) return fail(nullptr, OAIS_EINVAL, "bad arguments to oais_default_step_sizes");
    if (move_kind < OAIS_RWMH || move_kind > OAIS_HMC) return fail(nullptr, OAIS_EINVAL, "bad move kind");
    if (tg->d < 1 || !tg->X || !(tg->ref_scale > 0) || !(tg->p0 > 0))
        return fail(nullptr, OAIS_EINVAL, "bad target");
    if (tg->dtype != OAIS_DT_F64 && tg->dtype != OAIS_DT_F32) return fail(nullptr, OAIS_EINVAL, "bad dtype");
    const double d = (double)tg->d;
    if (tg->kind < kGauss || tg->kind > kUnid) return fail(nullptr, OAIS_EINVAL, "unknown target kind");
    std::vector<double> Xh;
    if (tg->kind == kLogreg || tg->kind == kLinreg) {
        if (tg->n < 1) return fail(nullptr, OAIS_EINVAL, "n must be >= 1");
        oais_status st = fetch(nullptr, tg->X, (size_t)tg->n * tg->d, tg->dtype, tg->on_device, Xh);
        if (st != OAIS_OK) return st;
    } else if (tg->kind == kUnid) {
        oais_status st = fetch(nullptr, tg->X, 2, OAIS_DT_F64, tg->on_device, Xh);
        if (st != OAIS_OK) return st;
        const double q = Xh[1] / Xh[0];
        if (!(q > 0.0 && q < 1.0)) return fail(nullptr, OAIS_EINVAL, "UNID: successes 0 < k < m");
    }
    const double curv = curvature(tg->kind, tg->d, tg->p0, Xh);
    const double c = move_kind == OAIS_RWMH ? 2.38 / std::sqrt(d)
                   : move_kind == OAIS_MALA ? 1.2 * std::pow(d, -1.0 / 6.0) : std::pow(d, -0.25);
    const double s2 = tg->ref_scale * tg->ref_scale;
    for (int t = 1; t <= T; ++t) eps[t - 1] = c / std::sqrt(1.0 / s2 + beta[t] * curv);
    return OAIS_OK;
}

oais_status oais_budget(int64_t N, int32_t T, int64_t N_cap, int32_t T_cap, int64_t* N_next, int32_t* T_next)
{
    if (N < 1 || T < 1 || N_cap < N || T_cap < T || !N_next || !T_next)
        return fail(nullptr, OAIS_EINVAL, "bad arguments to oais_budget");
    const double r2 = std::sqrt(2.0);
    int64_t n = (int64_t)std::llround((double)N * r2 / 128.0) * 128;
    n = std::max<int64_t>(128, n);
    int64_t t;
    if (N < N_cap) {    // grow both; the last growth step stops at the cap
        n = std::min(std::max(n, N + 1), N_cap);
        t = std::llround((double)T * r2);
    } else {            // memory exhausted: keep N, double T
        n = N;
        t = 2 * (int64_t)T;
    }
    t = std::max<int64_t>(t, (int64_t)T + 1);
    *N_next = std::min(n, N_cap);
    *T_next = (int32_t)std::min<int64_t>(t, T_cap);
    return OAIS_OK;
}

oais_status oais_set_particles(oais_ctx* ctx, int64_t N)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (ctx->N_total != ctx->N) return fail(ctx, OAIS_EINVAL, "sharded contexts keep their particle block");
    if (N < 1 || N > ctx->N_cap) return fail(ctx, OAIS_EINVAL, "N outside [1, the count the context was created with]");
    ctx->N = N;
    ctx->N_total = N;
    return OAIS_OK;
}

oais_status oais_set_exact_data(oais_ctx* ctx, int32_t on)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (on && !(ctx->dt.tc || ctx->dt.tcs))
        return fail(ctx, OAIS_EUNSUPPORTED, "the final reweighting applies to the tensor-core forms");
    if (on && !(ctx->dt.D > 0 && ctx->dt.D <= 32 && (ctx->dt.kind == kLogreg || ctx->dt.kind == kLinreg)))
        return fail(ctx, OAIS_EUNSUPPORTED, "the final reweighting needs the fp32 copy of X (d <= 32)");
    ctx->exact_data = on != 0;
    return OAIS_OK;
}

oais_status oais_arm_fault(oais_ctx* ctx, int32_t kind, double wait_seconds)
{
    if (!ctx) return fail(nullptr, OAIS_EINVAL, "null ctx");
    if (!(wait_seconds >= 0.0 && wait_seconds <= 60.0)) return fail(ctx, OAIS_EINVAL, "wait_seconds in [0, 60]");
    switch (kind) {
    case OAIS_FAULT_NONE:
        break;
    case OAIS_FAULT_NAN_DATA:
        if (ctx->dt.tcs_q8) return fail(ctx, OAIS_EUNSUPPORTED, "NaN data: not for FP8 storage");
        if (fault_sites(ctx).empty()) return fail(ctx, OAIS_EUNSUPPORTED, "NaN data: no device copy of X");
        break;
    case OAIS_FAULT_WITHHOLD_HANDOFF:
        if (!ctx->dt.tc && !ctx->dt.tcs)
            return fail(ctx, OAIS_EUNSUPPORTED, "withheld hand-off: only the tensor-core forms hand tiles over");
        break;
    default:
        return fail(ctx, OAIS_EINVAL, "unknown fault kind");
    }
    ctx->fault_kind = kind;
    ctx->fault_wait_ns = (uint64_t)(wait_seconds * 1e9);
    return OAIS_OK;
}

oais_status oais_set_problem(oais_ctx* ctx, int32_t p)
{
    if (!ctx || p < 0 || p > 0xFFFF) return fail(ctx, OAIS_EINVAL, "problem index out of range");
    ctx->problem = p;
    return OAIS_OK;
}

} // extern "C"
