// zja.cu -- the online conditional-ESS schedule of Zhou, Johansen & Aston (2016), the
// comparator of the paper's section on the connection to online CESS optimisation and of its
// GPU experiments ("ZJA").  Before step t the next annealing parameter is chosen so that
//   CESS_t / N = (sum_n W_n g_n)^2 / (sum_n W_n g_n^2) = c,   g_n = L(X_{t-1}^n)^delta,
// delta = beta_t - beta_{t-1}, W the normalised weights since the last resampling, c a target
// fraction (the paper sets it from D ~ Lambda^2 / T^2, i.e. c = exp(-Lambda^2 / T^2)).
// CESS is 1 at delta = 0 and decreases in delta; where weighted particles lie outside the
// likelihood's support (log L = -inf), CESS drops at once to their complement's share A of the
// weight, which no step can avoid, so the target is taken relative to it: CESS / N >= c A.
// The line search first scans the geometric
// candidates hi 4^-(32-j), j = 1..32 (hi = 1 - beta_{t-1}: eighteen decades, for targets whose
// likelihood spread asks for steps of 1e-10 and less), keeping the last one that meets the
// target, then refines the bracket it ends in over five passes of 32 equally spaced candidates
// lo + (hi - lo) j / 32; the step is the final lower end.  The whole interval is taken when its
// end meets the target, and the smallest geometric candidate when none does (every step
// advances).
//
// Per pass: zja_pass_kernel writes, per CTA, the shifted sums of the three weighted powers of
// g at each candidate; zja_narrow_kernel (one CTA) merges them, evaluates the candidates and
// narrows the bracket.  The particles' (log w, log L) enter as fp32 offsets from a per-CTA
// anchor (zja_prep_kernel, once per step), so the candidate sums need no fp64 exponentials.
#include "internal.h"

namespace oais {

constexpr int kZjaThreads = 256;
constexpr int kZjaCand = 32;                  // candidates per pass
constexpr int kZjaSums = 2 + 2 * kZjaCand;    // S0; S_alive; S1 at each candidate; S2 at each
constexpr int kZjaPasses = 6;                 // one geometric scan, five linear refinements

int zja_grid(int64_t N) { return (int)((N + kZjaThreads - 1) / kZjaThreads); }
size_t zja_part_bytes(int64_t N) { return sizeof(float2) * kZjaSums * (size_t)zja_grid(N); }

// offsets of each particle from its CTA's anchor: f = log w - log w_a, g = log L - log L_a
// (the anchor: the CTA's first particle with finite log w and log L; -inf offsets mark a zero
// weight, g = -inf a state outside the likelihood's support)
__global__ void __launch_bounds__(kZjaThreads)
zja_prep_kernel(const AsmcState* st, const StepParams P, float2* __restrict__ fg, double2* __restrict__ anchor)
{
    __shared__ int first;
    if (threadIdx.x == 0) first = kZjaThreads;
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * kZjaThreads + threadIdx.x;
    const int b = st->cur ^ st->pend;
    const double lw = n < P.N ? P.logw[n] : -INFINITY;
    const double ell = n < P.N ? P.ell[b][n] : -INFINITY;
    const bool ok = lw > -INFINITY && ell > -INFINITY;
    if (ok) atomicMin(&first, (int)threadIdx.x);
    __syncthreads();
    __shared__ double a_lw, a_ell;
    if ((int)threadIdx.x == first) { a_lw = lw; a_ell = ell; }
    __syncthreads();
    if (first == kZjaThreads) {
        if (n < P.N) fg[n] = make_float2(-INFINITY, 0.0f);
        if (threadIdx.x == 0) anchor[blockIdx.x] = make_double2(-INFINITY, 0.0);
        return;
    }
    if (n < P.N) fg[n] = make_float2(lw > -INFINITY ? (float)(lw - a_lw) : -INFINITY,
                                     ell > -INFINITY ? (float)(ell - a_ell) : -INFINITY);
    if (threadIdx.x == 0) anchor[blockIdx.x] = make_double2(a_lw, a_ell);
}

// per CTA and candidate: (max, sum exp(e - max)) of e = f + k delta g: k = 0 (S0); the weight
// inside the support (S_alive: e = f where g is finite); k = 1, 2 at each candidate
// candidate j (1..32) of a pass: geometric in pass 0, equally spaced after
__device__ __forceinline__ float zja_candidate(int pass, float lo, float hi, int j)
{
    return pass == 0 ? hi * exp2f(-2.0f * (float)(kZjaCand - j)) : lo + (hi - lo) * (float)j / (float)kZjaCand;
}

__global__ void __launch_bounds__(kZjaThreads)
zja_pass_kernel(const ZjaState* zs, int pass, int64_t N, const float2* __restrict__ fg, float2* __restrict__ part)
{
    if (zs->done) return;
    __shared__ float wmax[kZjaThreads / 32][kZjaSums], wsum[kZjaThreads / 32][kZjaSums];
    const int64_t n = (int64_t)blockIdx.x * kZjaThreads + threadIdx.x;
    const float2 v = n < N ? fg[n] : make_float2(-INFINITY, 0.0f);
    const float lo = (float)zs->lo, hi = (float)zs->hi;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < kZjaSums; ++c) {
        const int j = c < 2 ? 0 : (c - 2) % kZjaCand + 1;      // candidate 1..32 (0: S0, S_alive)
        const float k = c < 2 ? 0.0f : (c < 2 + kZjaCand ? 1.0f : 2.0f);
        const float delta = j == 0 ? 0.0f : zja_candidate(pass, lo, hi, j);
        // f + k delta g: a zero weight (f = -inf) or, for c >= 1, a state outside the support
        // (g = -inf) gives -inf; never 0 * inf
        const float e = (v.x == -INFINITY || (c >= 1 && v.y == -INFINITY)) ? -INFINITY
                                                                           : (k > 0.0f ? v.x + k * delta * v.y : v.x);
        float m = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        float s = m == -INFINITY ? 0.0f : __expf(e - m);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) { wmax[warp][c] = m; wsum[warp][c] = s; }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kZjaSums; c += kZjaThreads) {
        float M = -INFINITY;
        for (int w = 0; w < kZjaThreads / 32; ++w) M = fmaxf(M, wmax[w][c]);
        float S = 0.0f;
        if (M > -INFINITY)
            for (int w = 0; w < kZjaThreads / 32; ++w)
                if (wmax[w][c] > -INFINITY) S += wsum[w][c] * __expf(wmax[w][c] - M);
        part[(size_t)blockIdx.x * kZjaSums + c] = make_float2(M, S);
    }
}

// The step size at beta: the reference schedule runs step t at beta_ref[t] with eps_ref[t-1];
// log eps is interpolated linearly in beta between those points, constant beyond the ends.
__device__ double zja_step_size(double b, const double* beta_ref, const double* eps_ref, int T_ref)
{
    if (T_ref <= 1 || b <= beta_ref[1]) return eps_ref[0];
    if (b >= beta_ref[T_ref]) return eps_ref[T_ref - 1];
    int t = 1;
    while (t + 1 < T_ref && beta_ref[t + 1] <= b) ++t;
    const double u = (b - beta_ref[t]) / (beta_ref[t + 1] - beta_ref[t]);
    return exp(log(eps_ref[t - 1]) + u * (log(eps_ref[t]) - log(eps_ref[t - 1])));
}

// Merge the CTAs' sums, evaluate CESS / N at the candidates and narrow the bracket; after the
// last pass (or when the whole remaining interval meets the target) fix beta_t, its step size
// (linear interpolation of the reference schedule's in beta) and the next step's bracket.
__global__ void __launch_bounds__(128)
zja_narrow_kernel(ZjaState* zs, const double2* __restrict__ anchor, const float2* __restrict__ part, int nblk,
                  double log_target, int pass, int t, int T_max, double* beta, double* eps,
                  const double* __restrict__ beta_ref, const double* __restrict__ eps_ref, int T_ref)
{
    if (zs->done) return;
    __shared__ double logS[kZjaSums];
    const double lo = zs->lo, hi = zs->hi;
    for (int c = threadIdx.x; c < kZjaSums; c += blockDim.x) {
        const int j = c < 2 ? 0 : (c - 2) % kZjaCand + 1;
        const double k = c < 2 ? 0.0 : (c < 2 + kZjaCand ? 1.0 : 2.0);
        // the same fp32 candidate the pass kernel used
        const double delta = j == 0 ? 0.0 : (double)zja_candidate(pass, (float)lo, (float)hi, j);
        double M = -INFINITY;
        for (int b = 0; b < nblk; ++b) {
            const float2 q = part[(size_t)b * kZjaSums + c];
            const double2 a = anchor[b];
            if (q.x == -INFINITY || a.x == -INFINITY) continue;
            M = fmax(M, a.x + k * delta * a.y + (double)q.x);
        }
        double S = 0.0;
        if (M > -INFINITY)
            for (int b = 0; b < nblk; ++b) {
                const float2 q = part[(size_t)b * kZjaSums + c];
                const double2 a = anchor[b];
                if (q.x == -INFINITY || a.x == -INFINITY) continue;
                S += (double)q.y * (double)__expf((float)(a.x + k * delta * a.y + (double)q.x - M));
            }
        logS[c] = M > -INFINITY ? M + log(S) : -INFINITY;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // the last candidate whose CESS / N = S1^2 / (S0 S2) still meets c A, A = S_alive / S0
    const double lt = log_target + logS[1] - logS[0];
    int best = 0;
    for (int j = 1; j <= kZjaCand; ++j) {
        const double lr = 2.0 * logS[1 + j] - logS[0] - logS[1 + kZjaCand + j];
        if (lr >= lt) best = j;
    }
    auto cand = [&](int j) { return (double)zja_candidate(pass, (float)lo, (float)hi, j); };
    bool fix = false;
    double delta = 0.0, nlo = lo, nhi = hi;
    if (best == kZjaCand) {            // the whole remaining interval meets the target
        fix = true;
        delta = hi;
    } else if (best == 0 && pass == 0) {   // not even the smallest step does: take it
        fix = true;
        delta = cand(1);
    } else {
        nlo = best > 0 ? cand(best) : lo;
        nhi = cand(best + 1);
        if (pass == kZjaPasses - 1) {
            fix = true;
            delta = nlo;
        }
    }
    zs->lo = nlo;
    zs->hi = nhi;
    if (!fix) return;
    if (delta < 1e-14 && hi > 1e-14) delta = 1e-14;   // every step advances beta
    double bt = zs->beta_prev + delta;
    if (bt >= 1.0 - 1e-12 || t >= T_max) bt = 1.0;
    beta[t] = bt;
    eps[t - 1] = zja_step_size(bt, beta_ref, eps_ref, T_ref);
    zs->beta_prev = bt;
    zs->lo = 0.0;
    zs->hi = 1.0 - bt;
    zs->done = 1;
}

// open the search for step t (the pass and narrow kernels return at once while done == 1)
__global__ void zja_open_kernel(ZjaState* zs) { zs->done = zs->beta_prev >= 1.0 ? 1 : 0; }

cudaError_t launch_zja_search(ZjaState* zs, const AsmcState* st, const StepParams& P, float2* fg, double2* anchor,
                              float2* part, double cess_frac, int t, int T_max, double* beta, double* eps,
                              const double* beta_ref, const double* eps_ref, int T_ref, cudaStream_t s)
{
    const int grid = zja_grid(P.N);
    zja_open_kernel<<<1, 1, 0, s>>>(zs);
    zja_prep_kernel<<<grid, kZjaThreads, 0, s>>>(st, P, fg, anchor);
    for (int pass = 0; pass < kZjaPasses; ++pass) {
        zja_pass_kernel<<<grid, kZjaThreads, 0, s>>>(zs, pass, P.N, fg, part);
        zja_narrow_kernel<<<1, 128, 0, s>>>(zs, anchor, part, grid, log(cess_frac), pass, t, T_max, beta, eps,
                                            beta_ref, eps_ref, T_ref);
    }
    return cudaGetLastError();
}

} // namespace oais
