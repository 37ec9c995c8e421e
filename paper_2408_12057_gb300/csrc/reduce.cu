// reduce.cu -- deterministic cross-CTA reductions of the sweep:
//   * per-step moments g_hat_{t,0:2} (Alg. 1) from the per-CTA StepPartial records;
//   * log-sum-exp of the final log-weights, which gives log Z_hat (eq. estimator_Z)
//     and the ESS (eq. sample_size_IS).
// Every reduction visits its inputs in a fixed order, so results are bit-identical
// from run to run (no floating-point atomics).
#include "internal.h"
#include "../../include/oais.h"

namespace oais {

constexpr int kMergeThreads = 256;

// merge of (m, s, u): exp(m) s + exp(m') s' with u carried on the same shift as s (a part
// whose factor underflows to 0 adds nothing to u, even a -inf one)
__device__ __forceinline__ double scaled(double u, double f) { return f > 0.0 ? u * f : 0.0; }
__device__ __forceinline__ void lse_merge_u(double& m, double& s, double& u, double m2, double s2, double u2)
{
    if (m2 == -INFINITY) return;
    if (m == -INFINITY) { m = m2; s = s2; u = u2; return; }
    if (m2 > m) { const double f = exp(m - m2); s = s * f + s2; u = scaled(u, f) + u2; m = m2; }
    else        { const double f = exp(m2 - m); s = s + s2 * f; u = u + scaled(u2, f); }
}

// one CTA per step t: log g_hat_{t,i}, the acceptance rate and (elbo != null) the ELBO term
// sum_n W_{t-1}^n log g_t^n = u / s_0
__global__ void __launch_bounds__(kMergeThreads)
merge_stats_kernel(const StepPartial* __restrict__ parts, int nblocks, double inv_count,
                   double* __restrict__ log_ghat, double* __restrict__ accept, double* __restrict__ elbo)
{
    __shared__ double sm[3][kMergeThreads], ss[3][kMergeThreads], su[kMergeThreads];
    __shared__ unsigned long long sa[kMergeThreads];
    const int t = blockIdx.x, tid = threadIdx.x;
    const StepPartial* p = parts + (size_t)t * nblocks;
    double m[3] = {-INFINITY, -INFINITY, -INFINITY}, s[3] = {0.0, 0.0, 0.0}, u = 0.0;
    unsigned long long a = 0;
    for (int j = tid; j < nblocks; j += kMergeThreads) {
        const StepPartial q = p[j];
        lse_merge_u(m[0], s[0], u, q.m[0], q.s[0], q.u);
#pragma unroll
        for (int i = 1; i < 3; ++i) lse_merge(m[i], s[i], q.m[i], q.s[i]);
        a += q.accepted;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) { sm[i][tid] = m[i]; ss[i][tid] = s[i]; }
    su[tid] = u;
    sa[tid] = a;
    __syncthreads();
    for (int stride = kMergeThreads / 2; stride > 0; stride >>= 1) {
        if (tid < stride) {
            double mm = sm[0][tid], s0 = ss[0][tid], u0 = su[tid];
            lse_merge_u(mm, s0, u0, sm[0][tid + stride], ss[0][tid + stride], su[tid + stride]);
            sm[0][tid] = mm; ss[0][tid] = s0; su[tid] = u0;
#pragma unroll
            for (int i = 1; i < 3; ++i) {
                mm = sm[i][tid]; s0 = ss[i][tid];
                lse_merge(mm, s0, sm[i][tid + stride], ss[i][tid + stride]);
                sm[i][tid] = mm; ss[i][tid] = s0;
            }
            sa[tid] += sa[tid + stride];
        }
        __syncthreads();
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) log_ghat[3 * t + i] = sm[i][0] + log(ss[i][0]);
        accept[t] = (double)sa[0] * inv_count;
        if (elbo) elbo[t] = su[0] / ss[0][0];
    }
}

// ---- log-sum-exp of a[0..n) and of 2 a[0..n) ----
constexpr int kLseThreads = 256;
constexpr int kLseMaxBlocks = 1024;

struct LsePair { double m1, s1, m2, s2; };

__device__ __forceinline__ void lse_push(double& m, double& s, double v)
{
    if (v == -INFINITY) return;
    if (v > m) { s = s * exp(m - v) + 1.0; m = v; }
    else       { s += exp(v - m); }
}

__global__ void __launch_bounds__(kLseThreads)
lse_partial_kernel(const double* __restrict__ a, int64_t n, LsePair* __restrict__ out)
{
    __shared__ double s_m1[kLseThreads], s_s1[kLseThreads], s_m2[kLseThreads], s_s2[kLseThreads];
    double m1 = -INFINITY, s1 = 0.0, m2 = -INFINITY, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a[i];
        lse_push(m1, s1, v);
        lse_push(m2, s2, 2.0 * v);
    }
    const int tid = threadIdx.x;
    s_m1[tid] = m1; s_s1[tid] = s1; s_m2[tid] = m2; s_s2[tid] = s2;
    __syncthreads();
    for (int stride = kLseThreads / 2; stride > 0; stride >>= 1) {
        if (tid < stride) {
            double mm = s_m1[tid], ss = s_s1[tid];
            lse_merge(mm, ss, s_m1[tid + stride], s_s1[tid + stride]);
            s_m1[tid] = mm; s_s1[tid] = ss;
            mm = s_m2[tid]; ss = s_s2[tid];
            lse_merge(mm, ss, s_m2[tid + stride], s_s2[tid + stride]);
            s_m2[tid] = mm; s_s2[tid] = ss;
        }
        __syncthreads();
    }
    if (tid == 0) out[blockIdx.x] = LsePair{s_m1[0], s_s1[0], s_m2[0], s_s2[0]};
}

__global__ void __launch_bounds__(kLseThreads)
lse_final_kernel(const LsePair* __restrict__ parts, int nparts, double* __restrict__ out)
{
    __shared__ double s_m1[kLseThreads], s_s1[kLseThreads], s_m2[kLseThreads], s_s2[kLseThreads];
    double m1 = -INFINITY, s1 = 0.0, m2 = -INFINITY, s2 = 0.0;
    for (int j = threadIdx.x; j < nparts; j += kLseThreads) {
        lse_merge(m1, s1, parts[j].m1, parts[j].s1);
        lse_merge(m2, s2, parts[j].m2, parts[j].s2);
    }
    const int tid = threadIdx.x;
    s_m1[tid] = m1; s_s1[tid] = s1; s_m2[tid] = m2; s_s2[tid] = s2;
    __syncthreads();
    for (int stride = kLseThreads / 2; stride > 0; stride >>= 1) {
        if (tid < stride) {
            double mm = s_m1[tid], ss = s_s1[tid];
            lse_merge(mm, ss, s_m1[tid + stride], s_s1[tid + stride]);
            s_m1[tid] = mm; s_s1[tid] = ss;
            mm = s_m2[tid]; ss = s_s2[tid];
            lse_merge(mm, ss, s_m2[tid + stride], s_s2[tid + stride]);
            s_m2[tid] = mm; s_s2[tid] = ss;
        }
        __syncthreads();
    }
    if (tid == 0) {
        out[0] = s_m1[0] + log(s_s1[0]);
        out[1] = s_m2[0] + log(s_s2[0]);
    }
}

int lse_blocks(int64_t n)
{
    int64_t b = (n + kLseThreads * 4 - 1) / (kLseThreads * 4);
    return (int)(b < 1 ? 1 : (b > kLseMaxBlocks ? kLseMaxBlocks : b));
}

cudaError_t launch_merge_stats(const StepPartial* parts, int nblocks, int T, double inv_count,
                               double* log_ghat, double* accept, double* elbo, cudaStream_t s)
{
    if (T <= 0) return cudaSuccess;
    merge_stats_kernel<<<T, kMergeThreads, 0, s>>>(parts, nblocks, inv_count, log_ghat, accept, elbo);
    return cudaGetLastError();
}

cudaError_t launch_logsumexp(const double* a, int64_t n, double* out, void* scratch, cudaStream_t s)
{
    const int nb = lse_blocks(n);
    LsePair* parts = static_cast<LsePair*>(scratch);
    lse_partial_kernel<<<nb, kLseThreads, 0, s>>>(a, n, parts);
    lse_final_kernel<<<1, kLseThreads, 0, s>>>(parts, nb, out);
    return cudaGetLastError();
}

size_t logsumexp_scratch_bytes(int64_t n) { return sizeof(LsePair) * (size_t)lse_blocks(n); }

// ---- Fisher identity: grad_theta log Z = E_pi[grad_theta log gamma(x; theta)] ----
// estimated with the normalised final weights W_n = exp(log w_n - LSE) (eq. estimator_pi_t)
// for theta = (log s, log p0): d/dlog s log N(x; 0, s^2 I) = |x|^2 / s^2 - d, and
// d/dlog p0 log L from the cached log L: Gaussian -2 log L; linear regression
// -n - 2 log L - n log(2 pi p0^2); other families: not defined (0).
struct FisherPair { double a, b; };

template <typename R>
__global__ void __launch_bounds__(kLseThreads)
fisher_partial_kernel(const double* __restrict__ logw, const double* __restrict__ ell,
                      const R* __restrict__ x, int64_t N, int d, const double* __restrict__ lse,
                      double inv_s2, int kind, double nrows, double lin_c, FisherPair* __restrict__ out)
{
    __shared__ double sa[kLseThreads], sb[kLseThreads];
    const double L = lse[0];
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double W = exp(logw[i] - L);
        double xx = 0.0;
        for (int j = 0; j < d; ++j) { const double v = (double)x[(size_t)j * N + i]; xx += v * v; }
        a += W * (xx * inv_s2 - d);
        double db = 0.0;
        if (kind == kGauss) db = -2.0 * ell[i];
        else if (kind == kLinreg) db = -nrows - 2.0 * ell[i] - nrows * lin_c;
        b += W * db;
    }
    const int tid = threadIdx.x;
    sa[tid] = a; sb[tid] = b;
    __syncthreads();
    for (int stride = kLseThreads / 2; stride > 0; stride >>= 1) {
        if (tid < stride) { sa[tid] += sa[tid + stride]; sb[tid] += sb[tid + stride]; }
        __syncthreads();
    }
    if (tid == 0) out[blockIdx.x] = FisherPair{sa[0], sb[0]};
}

__global__ void fisher_final_kernel(const FisherPair* __restrict__ parts, int nparts, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int j = 0; j < nparts; ++j) { a += parts[j].a; b += parts[j].b; }
    out[0] = a;
    out[1] = b;
}

size_t fisher_scratch_bytes(int64_t n) { return sizeof(FisherPair) * (size_t)lse_blocks(n); }

cudaError_t launch_fisher(const double* logw, const double* ell, const void* x, bool fp64, int64_t N, int d,
                          const double* lse, double ref_scale, int kind, int nrows, double p0, void* scratch,
                          double* out, cudaStream_t s)
{
    const int nb = lse_blocks(N);
    FisherPair* parts = static_cast<FisherPair*>(scratch);
    const double inv_s2 = 1.0 / (ref_scale * ref_scale);
    const double lin_c = log(6.283185307179586 * p0 * p0);
    if (fp64)
        fisher_partial_kernel<double><<<nb, kLseThreads, 0, s>>>(logw, ell, static_cast<const double*>(x), N, d,
                                                                 lse, inv_s2, kind, (double)nrows, lin_c, parts);
    else
        fisher_partial_kernel<float><<<nb, kLseThreads, 0, s>>>(logw, ell, static_cast<const float*>(x), N, d,
                                                                lse, inv_s2, kind, (double)nrows, lin_c, parts);
    fisher_final_kernel<<<1, 32, 0, s>>>(parts, nb, out);
    return cudaGetLastError();
}


// The final reweighting of the tensor-core forms from the rounded data X~ to the data X (one more
// target in the annealing sequence, the step from gamma(.; X~) to gamma(.; X) at beta = 1 with no
// move, whose incremental weight is L(x_T; X) / L(x_T; X~)): log w_n += ell_x[n] - ell_n, then
// ell_n = ell_x[n]; status bit 0 for a non-finite result.
__global__ void reweight_to_data_kernel(double* __restrict__ logw, double* __restrict__ ell,
                                        const double* __restrict__ ell_x, int64_t N, unsigned* status)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double lx = ell_x[n];
    const double lw = logw[n] + (lx - ell[n]);
    logw[n] = lw;
    ell[n] = lx;
    if (isnan(lw) || lw == INFINITY || isnan(lx) || lx == INFINITY) atomicOr(status, 1u);
}

cudaError_t launch_reweight_to_data(double* logw, double* ell, const double* ell_x, int64_t N, unsigned* status,
                                    cudaStream_t s)
{
    reweight_to_data_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(logw, ell, ell_x, N, status);
    return cudaGetLastError();
}

} // namespace oais
