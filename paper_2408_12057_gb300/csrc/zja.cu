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
// g at each candidate; zja_narrow_kernel (one CTA, a warp per sum) merges them, evaluates the
// candidates and narrows the bracket.  The particles' (log w, log L) enter as fp32 offsets
// from a per-CTA anchor, the CTA's particle of largest log w (zja_prep_kernel, once per step),
// and the anchors as fp32 offsets from the largest of them (zja_anchor_kernel), so neither the
// candidate sums nor their merge need fp64 arithmetic; the reference anchor cancels from the
// ratios the search compares.  (The merge had taken fp64 offsets per CTA and sum in a few
// threads, 30 us per pass on this part's slow fp64 pipe.)
#include "internal.h"

namespace oais {

constexpr int kZjaThreads = 256;
constexpr int kZjaCand = 32;                  // candidates per pass
constexpr int kZjaSums = 2 + 2 * kZjaCand;    // S0; S_alive; S1 at each candidate; S2 at each
constexpr int kZjaPasses = 6;                 // one geometric scan, five linear refinements

int zja_grid(int64_t N) { return (int)((N + kZjaThreads - 1) / kZjaThreads); }
size_t zja_part_bytes(int64_t N) { return sizeof(float2) * kZjaSums * (size_t)zja_grid(N); }

// offsets of each particle from its CTA's anchor: f = log w - log w_a, g = log L - log L_a.
// The anchor is the CTA's particle of largest log w among those with finite log w and log L
// (or, if none has both, of largest finite log w, with log L_a = 0: then every g is -inf);
// -inf offsets mark a zero weight, g = -inf a state outside the likelihood's support.
__device__ __forceinline__ unsigned long long zja_order_key(double v)
{
    // a 64-bit key ordered like v (for the block maximum by an integer atomic)
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__global__ void __launch_bounds__(kZjaThreads)
zja_prep_kernel(const AsmcState* st, const StepParams P, float2* __restrict__ fg, double2* __restrict__ anchor)
{
    __shared__ unsigned long long best_both, best_w;
    __shared__ int who_both, who_w;
    __shared__ double a_lw, a_ell;
    if (threadIdx.x == 0) { best_both = 0ull; best_w = 0ull; who_both = kZjaThreads; who_w = kZjaThreads; }
    __syncthreads();
    const int64_t n = (int64_t)blockIdx.x * kZjaThreads + threadIdx.x;
    const int b = st->cur ^ st->pend;
    const double lw = n < P.N ? P.logw[n] : -INFINITY;
    const double ell = n < P.N ? P.ell[b][n] : -INFINITY;
    const bool fw = lw > -INFINITY, both = fw && ell > -INFINITY;
    const unsigned long long key = zja_order_key(lw);
    if (both) atomicMax(&best_both, key);
    if (fw) atomicMax(&best_w, key);
    __syncthreads();
    if (both && key == best_both) atomicMin(&who_both, (int)threadIdx.x);
    if (fw && key == best_w) atomicMin(&who_w, (int)threadIdx.x);
    __syncthreads();
    const bool any_both = who_both < kZjaThreads;
    if ((int)threadIdx.x == (any_both ? who_both : who_w)) { a_lw = lw; a_ell = any_both ? ell : 0.0; }
    __syncthreads();
    if (who_w == kZjaThreads) {               // no finite weight in this CTA
        if (n < P.N) fg[n] = make_float2(-INFINITY, 0.0f);
        if (threadIdx.x == 0) anchor[blockIdx.x] = make_double2(-INFINITY, 0.0);
        return;
    }
    if (n < P.N) fg[n] = make_float2(fw ? (float)(lw - a_lw) : -INFINITY,
                                     ell > -INFINITY ? (float)(ell - a_ell) : -INFINITY);
    if (threadIdx.x == 0) anchor[blockIdx.x] = make_double2(a_lw, a_ell);
}

// the CTA anchors as fp32 offsets from the one of largest log w (-inf: a CTA without weight)
__global__ void __launch_bounds__(kZjaThreads)
zja_anchor_kernel(const ZjaState* zs, const double2* __restrict__ anchor, int nblk, float2* __restrict__ adiff)
{
    if (zs->done) return;
    __shared__ unsigned long long best;
    __shared__ int who;
    __shared__ double2 ref;
    if (threadIdx.x == 0) { best = 0ull; who = nblk; }
    __syncthreads();
    for (int b = threadIdx.x; b < nblk; b += kZjaThreads)
        if (anchor[b].x > -INFINITY) atomicMax(&best, zja_order_key(anchor[b].x));
    __syncthreads();
    for (int b = threadIdx.x; b < nblk; b += kZjaThreads)
        if (anchor[b].x > -INFINITY && zja_order_key(anchor[b].x) == best) atomicMin(&who, b);
    __syncthreads();
    if (threadIdx.x == 0) ref = who < nblk ? anchor[who] : make_double2(0.0, 0.0);
    __syncthreads();
    for (int b = threadIdx.x; b < nblk; b += kZjaThreads) {
        const double2 a = anchor[b];
        adiff[b] = a.x > -INFINITY ? make_float2((float)(a.x - ref.x), (float)(a.y - ref.y))
                                   : make_float2(-INFINITY, 0.0f);
    }
}

// per CTA and candidate: (max, sum exp(e - max)) of e = f + k delta g: k = 0 (S0); the weight
// inside the support (S_alive: e = f where g is finite); k = 1, 2 at each candidate
// Candidate j (1..32) of a pass, defined in fp64 arithmetic with every operation rounded to
// nearest (no contraction), so that the grid is one set of values whatever evaluates CESS on
// it: geometric in pass 0, hi 4^-(32 - j) (an exact power-of-two scaling), equally spaced
// after, lo + ((hi - lo) j) / 32.
__device__ __forceinline__ double zja_candidate(int pass, double lo, double hi, int j)
{
    if (pass == 0) return ldexp(hi, -2 * (kZjaCand - j));
    return __dadd_rn(lo, __dmul_rn(__dmul_rn(__dsub_rn(hi, lo), (double)j), 1.0 / kZjaCand));
}

__global__ void __launch_bounds__(kZjaThreads)
zja_pass_kernel(const ZjaState* zs, int pass, int64_t N, const float2* __restrict__ fg, float2* __restrict__ part)
{
    if (zs->done) return;
    __shared__ float wmax[kZjaThreads / 32][kZjaSums], wsum[kZjaThreads / 32][kZjaSums];
    __shared__ float cand[kZjaCand + 1];
    const int64_t n = (int64_t)blockIdx.x * kZjaThreads + threadIdx.x;
    const float2 v = n < N ? fg[n] : make_float2(-INFINITY, 0.0f);
    // the pass's candidates (fp64 grid), rounded once to the fp32 of the per-particle sums
    if (threadIdx.x <= kZjaCand)
        cand[threadIdx.x] = threadIdx.x == 0 ? 0.0f : (float)zja_candidate(pass, zs->lo, zs->hi, threadIdx.x);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < kZjaSums; ++c) {
        const int j = c < 2 ? 0 : (c - 2) % kZjaCand + 1;      // candidate 1..32 (0: S0, S_alive)
        const float k = c < 2 ? 0.0f : (c < 2 + kZjaCand ? 1.0f : 2.0f);
        const float delta = cand[j];
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
constexpr int kZjaNarrowThreads = 1024;
__global__ void __launch_bounds__(kZjaNarrowThreads)
zja_narrow_kernel(ZjaState* zs, const float2* __restrict__ adiff, const float2* __restrict__ part, int nblk,
                  double log_target, int pass, int t, int T_max, double* beta, double* eps,
                  const double* __restrict__ beta_ref, const double* __restrict__ eps_ref, int T_ref)
{
    if (zs->done) return;
    __shared__ float logS[kZjaSums];
    const double lo = zs->lo, hi = zs->hi;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warp w merges sums w, w + 32, ...: lane l the CTAs l, l + 32, ...; each CTA's sum enters on
    // its anchor's offset from the reference anchor, v = a_f + k delta a_g + m_CTA
    for (int c = warp; c < kZjaSums; c += kZjaNarrowThreads / 32) {
        const int j = c < 2 ? 0 : (c - 2) % kZjaCand + 1;
        const float k = c < 2 ? 0.0f : (c < 2 + kZjaCand ? 1.0f : 2.0f);
        // the candidate as the pass kernel's sums used it
        const float delta = j == 0 ? 0.0f : (float)zja_candidate(pass, lo, hi, j);
        float M = -INFINITY;
        for (int b = lane; b < nblk; b += 32) {
            const float2 q = part[(size_t)b * kZjaSums + c];
            const float2 a = adiff[b];
            if (q.x == -INFINITY || a.x == -INFINITY) continue;
            M = fmaxf(M, (k > 0.0f ? a.x + k * delta * a.y : a.x) + q.x);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xFFFFFFFFu, M, o));
        float S = 0.0f;
        if (M > -INFINITY)
            for (int b = lane; b < nblk; b += 32) {
                const float2 q = part[(size_t)b * kZjaSums + c];
                const float2 a = adiff[b];
                if (q.x == -INFINITY || a.x == -INFINITY) continue;
                S += q.y * __expf((k > 0.0f ? a.x + k * delta * a.y : a.x) + q.x - M);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xFFFFFFFFu, S, o);
        if (lane == 0) logS[c] = M > -INFINITY ? M + logf(S) : -INFINITY;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    // the last candidate whose CESS / N = S1^2 / (S0 S2) still meets c A, A = S_alive / S0
    const double lt = log_target + (double)logS[1] - (double)logS[0];
    int best = 0;
    for (int j = 1; j <= kZjaCand; ++j) {
        const double lr = 2.0 * (double)logS[1 + j] - (double)logS[0] - (double)logS[1 + kZjaCand + j];
        if (lr >= lt) best = j;
    }
    auto cand = [&](int j) { return zja_candidate(pass, lo, hi, j); };
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

// open the search for step t (the pass and narrow kernels return at once while done == 1); a
// step after the one that reached beta = 1 is skipped altogether (the host looks only every
// few steps)
__global__ void zja_open_kernel(ZjaState* zs)
{
    zs->skip = zs->beta_prev >= 1.0 ? 1 : 0;
    zs->done = zs->skip;
}

cudaError_t launch_zja_search(ZjaState* zs, const AsmcState* st, const StepParams& P, float2* fg, double2* anchor,
                              float2* part, double cess_frac, int t, int T_max, double* beta, double* eps,
                              const double* beta_ref, const double* eps_ref, int T_ref, cudaStream_t s)
{
    const int grid = zja_grid(P.N);
    float2* adiff = reinterpret_cast<float2*>(anchor + grid);   // the buffer's second part
    zja_open_kernel<<<1, 1, 0, s>>>(zs);
    zja_prep_kernel<<<grid, kZjaThreads, 0, s>>>(st, P, fg, anchor);
    zja_anchor_kernel<<<1, kZjaThreads, 0, s>>>(zs, anchor, grid, adiff);
    for (int pass = 0; pass < kZjaPasses; ++pass) {
        zja_pass_kernel<<<grid, kZjaThreads, 0, s>>>(zs, pass, P.N, fg, part);
        zja_narrow_kernel<<<1, kZjaNarrowThreads, 0, s>>>(zs, adiff, part, grid, log(cess_frac), pass, t, T_max,
                                                          beta, eps, beta_ref, eps_ref, T_ref);
    }
    return cudaGetLastError();
}

} // namespace oais
