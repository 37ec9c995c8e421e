// asmc.cu -- the resampling half of ASMC (Alg. 1, resample step; Sec. 2.1.3):
//   decide:   ESS of w_{t^-} = (sum w)^2 / sum w^2 (eq. sample_size_IS); resample when
//             ESS < nu N, and always close the last segment (t = T, or beta_t = 1); on a resampling
//             time Z_hat *= mean(w) (eq. estimator_Z), kept as log Z_hat += LSE(log w) - log N;
//   scan:     weights exp(log w_m - LSE~) and their inclusive cumulative sums P_m in fp64
//             (block sums, block offsets, in-block scan: a fixed order), normalised by
//             their own fp64 total, C_m = P_m / P_{N-1}, so C does not inherit the
//             rounding of the shift LSE~ (which comes from the fp32-summed ESS pieces);
//   gather:   systematic resampling, a^n = min{m : C_m > (n + U)/N} by binary search,
//             particles copied to the other buffer, w = 1.
// Every kernel after `decide` reads the device flag `pend` and returns at once when the
// step does not resample, so a whole schedule is launched without host round-trips.
#include <algorithm>

#include "internal.h"

namespace oais {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;   // particles per scan block

int scan_blocks(int64_t N) { return (int)((N + kScanTile - 1) / kScanTile); }

// The ESS test merges the per-CTA pieces (m_j, s_j) of log w and 2 log w into
// LSE = M + log sum_j s_j exp(m_j - M), in two levels within one launch: groups of kEssGroup
// pieces on as many CTAs, then the groups in the CTA that completes the last one (the
// decision).  Each merge takes two passes, the largest shift M and then the rescaled sum, whose
// factors exp(m_j - M) take the fp64 difference (<= 0) rounded once to fp32 and an fp32
// exponential (relative effect on a sum below a few 1e-8, the pieces themselves being fp32
// sums).  One CTA merging every piece through a chain of fp64 exponentials (each waiting for
// the last) took 70 us for 2 048 pieces on this part's slow fp64 pipe; one CTA doing the two
// passes over them, 21 us; the two levels in two launches, 13 us.
constexpr int kEssGroup = 64;
int asmc_ess_groups(int nparts) { return (nparts + kEssGroup - 1) / kEssGroup; }

template <int NT>
__device__ __forceinline__ double block_reduce_max(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = lane < NT / 32 ? sh[lane] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;                                     // in every thread
}
template <int NT>
__device__ __forceinline__ double block_reduce_sum(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
// (M_i, S_i), i = 0, 1, of the pieces [0, n) (all threads of the CTA call it; thread t takes
// pieces t, t + NT, ...)
// kL2: read the pieces at L2 (written by other CTAs of the same launch)
template <int NT, bool kL2 = false>
__device__ __forceinline__ void merge_ess_pieces(const StepPartial* __restrict__ parts, int n, double (&M)[2],
                                                 double (&S)[2], double* sh)
{
    auto ld = [](const double* p) { return kL2 ? __ldcg(p) : *p; };
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        double mx = -INFINITY;
        for (int j = threadIdx.x; j < n; j += NT) mx = fmax(mx, ld(&parts[j].m[i]));
        M[i] = block_reduce_max<NT>(mx, sh);
        double sum = 0.0;
        if (M[i] > -INFINITY) {
            for (int j = threadIdx.x; j < n; j += NT) {
                const double m = ld(&parts[j].m[i]);
                if (m > -INFINITY) sum += ld(&parts[j].s[i]) * (double)expf((float)(m - M[i]));
            }
        }
        S[i] = block_reduce_sum<NT>(sum, sh);
    }
}

// the decision of step t from the merged shifts and sums (one thread)
__device__ __forceinline__ void asmc_decide(AsmcState* st, const double (&M)[2], const double (&S)[2], int t, int T,
                                        const double* __restrict__ beta, double ess_frac, int64_t N, Rng rng,
                                        double* ess_trace, int* resampled)
{
    // ESS = exp(2 LSE(log w) - LSE(2 log w)) = S_0^2 / S_1 exp(2 M_0 - M_1); the shift of the
    // doubled weights is exactly twice the other (doubling commutes with rounding), so the
    // exponential is 1 but for empty sums, and the logarithms (fp64, slow here) are taken
    // only when the segment closes
    const double d2 = 2.0 * M[0] - M[1];
    const double ess = S[0] * S[0] / S[1] * (d2 == 0.0 ? 1.0 : exp(d2));
    st->cur ^= st->pend;             // the previous step's gather is now the live buffer
    // the last step (t = T, or beta_t = 1 for a schedule found online) closes the segment
    const bool last = (t == T) || beta[t] >= 1.0;
    const bool fire = last || (ess_frac > 0.0 && ess < ess_frac * (double)N);
    int pend = 0;
    if (fire) {
        const double lse1 = M[0] + log(S[0]);
        st->logZ += lse1 - log((double)N);
        if (!last) {
            pend = 1;
            st->n_resample += 1;
            st->lse = lse1;
            const Philox4 r = philox4x32_10(0xFFFFFFFFu, (uint32_t)t, 0u, rng.tag, rng.k0, rng.k1);
            st->U = u01d(r.v[0]);
        }
    }
    st->pend = pend;
    if (ess_trace) ess_trace[t - 1] = ess;
    if (resampled) resampled[t - 1] = fire ? 1 : 0;
}

// One launch per step: CTA g merges the pieces [64 g, 64 g + 64) into group record g; the CTA
// that completes the last group (a ticket in the ASMC state, no waiting) merges the groups and
// takes the decision, then resets the ticket for the next step.
__global__ void __launch_bounds__(kEssGroup)
asmc_ess_decide_kernel(const StepPartial* __restrict__ parts, int nparts, StepPartial* __restrict__ groups,
                       AsmcState* st, int t, int T, const double* __restrict__ beta, double ess_frac, int64_t N,
                       Rng rng, double* ess_trace, int* resampled, const int* skip)
{
    if (skip && *skip) return;           // the step was skipped: st (pend = 0) stays as it is
    __shared__ double sh[kEssGroup / 32];
    __shared__ int last;
    const int j0 = blockIdx.x * kEssGroup;
    double M[2], S[2];
    merge_ess_pieces<kEssGroup>(parts + j0, min(kEssGroup, nparts - j0), M, S, sh);
    if (threadIdx.x == 0) {
        StepPartial g{};
        g.m[0] = M[0]; g.s[0] = S[0];
        g.m[1] = M[1]; g.s[1] = S[1];
        g.m[2] = -INFINITY;
        groups[blockIdx.x] = g;
        __threadfence();                 // the record before the ticket
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();                     // every group record before reading them
    merge_ess_pieces<kEssGroup, true>(groups, gridDim.x, M, S, sh);
    if (threadIdx.x == 0) {
        st->ticket = 0u;
        asmc_decide(st, M, S, t, T, beta, ess_frac, N, rng, ess_trace, resampled);
    }
}

// block-level inclusive scan of kScanTile doubles held kScanItems per thread
__device__ __forceinline__ double block_scan_inclusive(double (&v)[kScanItems], double* sh,
                                                       double* thread_prefix = nullptr)
{
    // thread-local inclusive scan
#pragma unroll
    for (int i = 1; i < kScanItems; ++i) v[i] += v[i - 1];
    const int tid = threadIdx.x;
    sh[tid] = v[kScanItems - 1];
    __syncthreads();
    // Hillis-Steele over the thread totals (fixed order)
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const double add = tid >= off ? sh[tid - off] : 0.0;
        __syncthreads();
        sh[tid] += add;
        __syncthreads();
    }
    const double prefix = tid > 0 ? sh[tid - 1] : 0.0;
    if (thread_prefix) *thread_prefix = prefix;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] += prefix;
    return sh[kScanThreads - 1];
}

// The block-sum, CDF and gather kernels run on every step and return at once unless the step
// resamples: their grids are capped at a few CTAs per SM (tiles and particles taken
// grid-stride), so that a step without resampling does not schedule thousands of empty CTAs.
__global__ void __launch_bounds__(kScanThreads)
asmc_blocksum_kernel(const AsmcState* st, const double* __restrict__ logw, int64_t N, int nb, double* bsum)
{
    if (!st->pend) return;
    __shared__ double sh[kScanThreads];
    const double lse = st->lse;
    for (int tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
        double v[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) v[i] = base + i < N ? exp(logw[base + i] - lse) : 0.0;
        const double tot = block_scan_inclusive(v, sh);
        if (threadIdx.x == 0) bsum[tile] = tot;
        __syncthreads();                 // sh is reused by the next tile's scan
    }
}

// exclusive scan of the block sums by one CTA, in chunks of kScanTile; boff[nb] = total
__global__ void __launch_bounds__(kScanThreads)
asmc_offsets_kernel(const AsmcState* st, const double* __restrict__ bsum, int nb, double* boff)
{
    if (!st->pend) return;
    __shared__ double sh[kScanThreads];
    double carry = 0.0;
    for (int c0 = 0; c0 < nb; c0 += kScanTile) {
        const int base = c0 + threadIdx.x * kScanItems;
        double v[kScanItems], pre = 0.0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) v[i] = base + i < nb ? bsum[base + i] : 0.0;
        const double tot = block_scan_inclusive(v, sh, &pre);
#pragma unroll
        for (int i = 0; i < kScanItems; ++i)
            if (base + i < nb) boff[base + i] = carry + (i == 0 ? pre : v[i - 1]);
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) boff[nb] = carry;
}

__global__ void __launch_bounds__(kScanThreads)
asmc_cdf_kernel(const AsmcState* st, const double* __restrict__ logw, int64_t N, int nb,
                const double* __restrict__ boff, double* cdf)
{
    if (!st->pend) return;
    __shared__ double sh[kScanThreads];
    const double lse = st->lse, total = boff[nb];
    for (int tile = blockIdx.x; tile < nb; tile += gridDim.x) {
        const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
        double v[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) v[i] = base + i < N ? exp(logw[base + i] - lse) : 0.0;
        block_scan_inclusive(v, sh);
        const double off = boff[tile];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) if (base + i < N) cdf[base + i] = (off + v[i]) / total;
        __syncthreads();                 // sh is reused by the next tile's scan
    }
}

// Systematic resampling: particle n takes ancestor a^n = min{m : C_m > (n + U)/N}, clamped to
// N - 1 (binary search over the CDF), and copies that ancestor's state.  The copy loads eight
// coordinates before storing them (the source and destination buffers are distinct, which the
// compiler cannot see), so that a particle's loads are in flight together.
template <typename R>
__device__ __forceinline__ void copy_rows(const R* __restrict__ src, R* __restrict__ dst, int d, int64_t N,
                                          int64_t from, int64_t to)
{
    for (int i0 = 0; i0 < d; i0 += 8) {
        R v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = i0 + j < d ? src[(size_t)(i0 + j) * N + from] : R(0);
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (i0 + j < d) dst[(size_t)(i0 + j) * N + to] = v[j];
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
asmc_gather_kernel(const AsmcState* st, StepParams P, int d, int grad, const double* __restrict__ cdf,
                   int64_t* ancestors)
{
    if (!st->pend) return;
    const double U = st->U, Nd = (double)P.N;
    const int src = st->cur, dst = src ^ 1;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < P.N; n += (int64_t)gridDim.x * blockDim.x) {
        const double thr = ((double)n + U) / Nd;
        int64_t lo = 0, hi = P.N - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > thr) hi = mid; else lo = mid + 1;
        }
        const int64_t a = lo;
        copy_rows<R>(reinterpret_cast<const R*>(P.x[src]), reinterpret_cast<R*>(P.x[dst]), d, P.N, a, n);
        if (grad) copy_rows<R>(reinterpret_cast<const R*>(P.gl[src]), reinterpret_cast<R*>(P.gl[dst]), d, P.N, a, n);
        P.ell[dst][n] = P.ell[src][a];
        P.logw[n] = 0.0;
        if (ancestors) ancestors[n] = a;
    }
}

int capped_grid(int64_t want, int per_sm)
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms <= 0)
            sms = 152;
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
}

cudaError_t launch_asmc_decide_scan(AsmcState* st, const StepParams& P, int nparts, double ess_frac, double* bsum,
                                    double* boff, double* cdf, double* ess_trace, int* resampled, cudaStream_t s)
{
    const int ng = asmc_ess_groups(nparts);
    StepPartial* groups = P.ess_parts + nparts;   // the buffer holds nparts pieces, then the groups
    asmc_ess_decide_kernel<<<ng, kEssGroup, 0, s>>>(P.ess_parts, nparts, groups, st, P.t, P.T, P.beta, ess_frac,
                                                    P.N, P.mv.rng, ess_trace, resampled, P.skip);
    const int nb = scan_blocks(P.N), gs = capped_grid(nb, 2);
    asmc_blocksum_kernel<<<gs, kScanThreads, 0, s>>>(st, P.logw, P.N, nb, bsum);
    asmc_offsets_kernel<<<1, kScanThreads, 0, s>>>(st, bsum, nb, boff);
    asmc_cdf_kernel<<<gs, kScanThreads, 0, s>>>(st, P.logw, P.N, nb, boff, cdf);
    return cudaGetLastError();
}

cudaError_t launch_asmc_resample(AsmcState* st, const StepParams& P, int nparts, double ess_frac, int d,
                                 bool grad, bool fp64, double* bsum, double* boff, double* cdf,
                                 double* ess_trace, int* resampled, int64_t* ancestors, cudaStream_t s)
{
    const int ng = asmc_ess_groups(nparts);
    StepPartial* groups = P.ess_parts + nparts;   // the buffer holds nparts pieces, then the groups
    asmc_ess_decide_kernel<<<ng, kEssGroup, 0, s>>>(P.ess_parts, nparts, groups, st, P.t, P.T, P.beta, ess_frac,
                                                    P.N, P.mv.rng, ess_trace, resampled, P.skip);
    const int nb = scan_blocks(P.N), gs = capped_grid(nb, 2);
    asmc_blocksum_kernel<<<gs, kScanThreads, 0, s>>>(st, P.logw, P.N, nb, bsum);
    asmc_offsets_kernel<<<1, kScanThreads, 0, s>>>(st, bsum, nb, boff);
    asmc_cdf_kernel<<<gs, kScanThreads, 0, s>>>(st, P.logw, P.N, nb, boff, cdf);
    const int gb = capped_grid((P.N + 255) / 256, 8);
    if (fp64) asmc_gather_kernel<double><<<gb, 256, 0, s>>>(st, P, d, grad ? 1 : 0, cdf, ancestors);
    else      asmc_gather_kernel<float><<<gb, 256, 0, s>>>(st, P, d, grad ? 1 : 0, cdf, ancestors);
    return cudaGetLastError();
}

} // namespace oais
