// targets.cuh -- target families on the geometric path gamma_beta = eta * L^beta (Sec. 2),
// eta = N(0, s^2 I).  Each family evaluates log L(x) and, when asked, grad_x log L(x)
// for one particle per thread.  Families that read a data matrix stream it through
// shared memory in chunks, so every thread of the CTA must call eval() together.
#pragma once
#include "oais_device.cuh"

namespace oais {

enum TargetKind { kGauss = 0, kLogreg = 1, kGmm = 2, kLinreg = 3, kUnid = 4 };

// -------------------------------------------------------------------------
// Conjugate Gaussian likelihood L(x) = exp(-|x - mu|^2 / (2 sigma^2)).
// -------------------------------------------------------------------------
template <typename R, int D>
struct GaussTarget {
    static constexpr int kind = kGauss;
    const R* mu;      // [d] in global memory
    int d;
    R inv_sig2;
    R mu_r[D];

    __device__ void setup(unsigned char*) {
#pragma unroll
        for (int i = 0; i < D; ++i) mu_r[i] = (i < d) ? mu[i] : R(0);
    }
    static constexpr size_t smem_bytes(int) { return 0; }

    template <bool GRAD>
    __device__ R eval(const R (&x)[D], R (&g)[D]) const {
        R acc = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const R r = x[i] - mu_r[i];
            acc += r * r;
            if (GRAD) g[i] = -r * inv_sig2;
        }
        return R(-0.5) * acc * inv_sig2;
    }
};

// -------------------------------------------------------------------------
// Unidentifiable product parameterisation (the paper's GPU workload "Unid", its model
// appendix): X, Y ~ Uniform(0, b), K | X, Y ~ Binomial(m, X Y).  The state is z in R^2 under
// the reference N(0, I): X = b Phi(z_1), Y = b Phi(z_2) are then Uniform(0, b), so the path
// eta L^beta has the model's Z.  log L = log Binom(k; m, p) with p = X Y, -inf where p is
// not in (0, 1).  It is evaluated as c0 - m D(p^ || p), p^ = k / m, c0 = log Binom(k; m, p^)
// (precomputed on the host), D the Bernoulli KL divergence in log1p form: with m = 10^11
// the terms are ~10^10 and their differences O(1), which fp64 keeps.
// -------------------------------------------------------------------------
template <typename R, int D>
struct UnidTarget {
    static constexpr int kind = kUnid;
    const double* par;   // [4] in global memory: m, k, b, c0
    int d;
    double m, k, b, c0, ph;

    __device__ void setup(unsigned char*) {
        m = par[0]; k = par[1]; b = par[2]; c0 = par[3];
        ph = k / m;
    }
    static constexpr size_t smem_bytes(int) { return 0; }

    template <bool GRAD>
    __device__ R eval(const R (&x)[D], R (&g)[D]) const {
        static_assert(D == 2, "the Unid state is two-dimensional");
        const double u1 = normcdf((double)x[0]), u2 = normcdf((double)x[1]);
        const double p = b * b * u1 * u2;
        if (GRAD) { g[0] = R(0); g[1] = R(0); }
        if (!(p > 0.0 && p < 1.0)) return R(-INFINITY);
        const double dkl = -ph * log1p((p - ph) / ph) - (1.0 - ph) * log1p((ph - p) / (1.0 - ph));
        if (GRAD) {
            // d log L / dp = (k - m p) / (p (1 - p)); dp/dz_i = b^2 phi(z_i) u_j
            const double dldp = (k - m * p) / (p * (1.0 - p));
            const double c = 0.39894228040143268 * b * b;   // b^2 / sqrt(2 pi)
            g[0] = R(dldp * c * u2 * exp(-0.5 * (double)x[0] * (double)x[0]));
            g[1] = R(dldp * c * u1 * exp(-0.5 * (double)x[1] * (double)x[1]));
        }
        return R(c0 - m * dkl);
    }
};

// -------------------------------------------------------------------------
// Gaussian mixture p = (1/K) sum_k N(mu_k, v I); L = p / eta so that Z = 1.
// Means live in shared memory.
// -------------------------------------------------------------------------
template <typename R, int D>
struct GmmTarget {
    static constexpr int kind = kGmm;
    static constexpr int kMaxK = 16;
    const R* means;   // [K][D] (padded to D columns)
    int d, K;
    R inv_v;          // 1 / v
    R inv_s2;         // 1 / s^2
    R log_const;      // -(d/2) log(2 pi v) - log K + (d/2) log(2 pi s^2)
    const R* sm;      // shared copy
    // fp32 roundings of the running schedule (nullable), 3 T + 1 floats: beta_t at [t]
    // (t = 0..T), beta_t - beta_{t-1} (rounded from its fp64 difference) at [T + t] and eps_t at
    // [2 T + t] (t = 1..T); the sweep reads them instead of converting the fp64 schedule per step
    const float* fsched;
    // fp32 forms: -log2(e) / (2 v), the exponent factor of a component in base-2 units
    float c2;
    // the launch's random-number generator with its round keys precomputed (set per launch
    // from the move configuration; the random-walk moves of the fp32 forms draw from it)
    RngKS rks;

    // fp32 forms take the components in groups of eight (K > 4) or four (one test of K per
    // group, and the group's instructions can interleave: on the mixture workload, K = 8,
    // 1.32e10 particle-steps/s one by one, 1.445e10 in pairs, 1.484e10 in fours, 1.503e10 in
    // eights); K is padded to a multiple of the group with dummy components whose means lie so
    // far away (1e18 in every coordinate) that their weights are exactly 0: the exponent is
    // about -1e37, whose ex2 is +0, so sums, maxima and the gradient are unchanged bit for bit
    static constexpr int kGroupMax = (sizeof(R) == 4 && D % 2 == 0) ? 8 : 1;
    static constexpr size_t smem_bytes(int K) { return sizeof(R) * (size_t)((K + kGroupMax - 1) / kGroupMax * kGroupMax) * D; }
    __device__ void setup(unsigned char* smem) {
        R* s = reinterpret_cast<R*>(smem);
        const int Kg = (K + kGroupMax - 1) / kGroupMax * kGroupMax;
        for (int i = threadIdx.x; i < Kg * D; i += blockDim.x) s[i] = i < K * D ? means[i] : R(1e18);
        sm = s;
        __syncthreads();
    }

    template <bool GRAD>
    __device__ R eval(const R (&x)[D], R (&g)[D]) const {
        if constexpr (kGroupMax == 8) {
            if (K > 4) return eval_g<GRAD, 8>(x, g);
            return eval_g<GRAD, 4>(x, g);
        } else {
            return eval_g<GRAD, 1>(x, g);
        }
    }

    template <bool GRAD, int G>
    __device__ R eval_g(const R (&x)[D], R (&g)[D]) const {
        // fp32: the squared distances, |x|^2 and the gradient's mixture sums two coordinates
        // per packed instruction (even and odd coordinates summed apart, then added)
        constexpr bool kPair = sizeof(R) == 4 && D % 2 == 0;
        const int Kg = (K + G - 1) / G * G;
        R q[kMaxK];
        R mx = R(-INFINITY);
#pragma unroll
        for (int k0 = 0; k0 < kMaxK; k0 += G) {
            if (k0 < Kg) {
#pragma unroll
            for (int k = k0; k < k0 + G; ++k) {
                R acc = 0;
                if constexpr (kPair) {
                    // two accumulator pairs (even and odd coordinate pairs): half the
                    // dependent chain of multiply-adds
                    const float2* m2 = reinterpret_cast<const float2*>(sm + k * D);
                    float2 a2 = make_float2(0.0f, 0.0f), b2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int i = 0; i < D / 2; ++i) {
                        const float2 r = sub_f32x2(make_float2(x[2 * i], x[2 * i + 1]), m2[i]);
                        if (i & 1) b2 = fma_f32x2(r, r, b2);
                        else a2 = fma_f32x2(r, r, a2);
                    }
                    if constexpr (D >= 4) a2 = add_f32x2(a2, b2);
                    acc = a2.x + a2.y;
                    q[k] = acc * c2;                  // base-2 units
                } else {
#pragma unroll
                    for (int i = 0; i < D; ++i) { const R r = x[i] - sm[k * D + i]; acc += r * r; }
                    q[k] = R(-0.5) * acc * inv_v;
                }
                mx = q[k] > mx ? q[k] : mx;
            }
            }
        }
        R sum = 0, xx = 0;
#pragma unroll
        for (int k0 = 0; k0 < kMaxK; k0 += G)
            if (k0 < Kg) {
#pragma unroll
                for (int k = k0; k < k0 + G; ++k) {
                    if constexpr (kPair) q[k] = ex2_(q[k] - mx);
                    else q[k] = exp_(q[k] - mx);
                    sum += q[k];
                }
            }
        if constexpr (kPair) {
            float2 a2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < D / 2; ++i) {
                const float2 v = make_float2(x[2 * i], x[2 * i + 1]);
                a2 = fma_f32x2(v, v, a2);
            }
            xx = a2.x + a2.y;
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) xx += x[i] * x[i];
        }
        if (GRAD) {
            const R inv = R(1) / sum;
            if constexpr (kPair) {
#pragma unroll
                for (int i = 0; i < D / 2; ++i) {
                    float2 a2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int k = 0; k < kMaxK; ++k)
                        if (k < Kg) a2 = fma_f32x2(make_float2(q[k], q[k]), reinterpret_cast<const float2*>(sm + k * D)[i], a2);
                    g[2 * i] = (a2.x * inv - x[2 * i]) * inv_v + x[2 * i] * inv_s2;
                    g[2 * i + 1] = (a2.y * inv - x[2 * i + 1]) * inv_v + x[2 * i + 1] * inv_s2;
                }
            } else {
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    R acc = 0;
#pragma unroll
                    for (int k = 0; k < kMaxK; ++k) if (k < K) acc += q[k] * sm[k * D + i];
                    g[i] = (acc * inv - x[i]) * inv_v + x[i] * inv_s2;
                }
            }
        }
        if constexpr (kPair) return 0.69314718055994531f * (mx + lg2_(sum)) + log_const + R(0.5) * xx * inv_s2;
        else return mx + log_(sum) + log_const + R(0.5) * xx * inv_s2;
    }
    __device__ static float ex2_(float v) { float y; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v)); return y; }
    __device__ static float lg2_(float v) { float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v)); return y; }
    __device__ static float exp_(float v) { return __expf(v); }
    __device__ static double exp_(double v) { return exp(v); }
    __device__ static float log_(float v) { return __logf(v); }
    __device__ static double log_(double v) { return log(v); }
};

// -------------------------------------------------------------------------
// Row-structured likelihoods, log L = sum_r f(y_r, X_r . x):
//   logistic: f = y z - softplus(z),       df/dz = y - sigmoid(z)
//   linear:   f = -(y - z)^2 / (2 sig^2),  df/dz = (y - z) / sig^2  (+ constant)
// X [n][D] fp32 (zero-padded columns), y [n] fp32, streamed through shared
// memory in chunks of kChunkFloats with cp.async double buffering.
// -------------------------------------------------------------------------
constexpr int kChunkFloats = 8192;   // 32 KB of X per buffer

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int D, bool LOGISTIC>
struct RowsTarget {
    static constexpr int kind = LOGISTIC ? kLogreg : kLinreg;
    static constexpr int kRows = kChunkFloats / D;
    const float* X;     // [n_pad][D], n_pad a multiple of 4
    const float* y;     // [n_pad]
    int d, n;
    float inv_sig2;     // linear only
    float lin_const;    // linear only: -(n/2) log(2 pi sig^2)
    float* xs;          // [2][kRows * D]
    float* ys;          // [2][kRows]

    static constexpr size_t smem_bytes(int) { return sizeof(float) * 2 * (size_t)(kRows * D + kRows); }
    __device__ void setup(unsigned char* smem) {
        xs = reinterpret_cast<float*>(smem);
        ys = xs + 2 * kRows * D;
    }

    __device__ void load_chunk(int c, int buf) const {
        const int r0 = c * kRows;
        int rows = n - r0; rows = rows < kRows ? rows : kRows;
        rows = (rows + 3) & ~3;                        // n_pad keeps this in bounds
        const float* srcX = X + (size_t)r0 * D;
        float* dstX = xs + buf * kRows * D;
        const int nx = rows * D / 4;                   // 16-byte pieces
        for (int i = threadIdx.x; i < nx; i += blockDim.x) cp_async16(dstX + 4 * i, srcX + 4 * i);
        const float* srcy = y + r0;
        float* dsty = ys + buf * kRows;
        for (int i = threadIdx.x; i < rows / 4; i += blockDim.x) cp_async16(dsty + 4 * i, srcy + 4 * i);
        cp_async_commit();
    }

    // X_r . x with 4 independent partial sums (shorter FMA dependency chain)
    __device__ __forceinline__ static float row_dot(const float* xr, const float (&x)[D]) {
        float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
        for (int i = 0; i < D; i += 4) {
            if (D % 4 == 0) {
                const float4 v = *reinterpret_cast<const float4*>(xr + i);
                z0 = fmaf(v.x, x[i], z0); z1 = fmaf(v.y, x[i + 1], z1);
                z2 = fmaf(v.z, x[i + 2], z2); z3 = fmaf(v.w, x[i + 3], z3);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) if (i + q < D) z0 = fmaf(xr[i + q], x[i + q], z0);
            }
        }
        return (z0 + z1) + (z2 + z3);
    }

    // per-row term f(y, z) into `part`; returns df/dz
    __device__ __forceinline__ float row_term(float z, float yv, float& part) const {
        if (LOGISTIC) {
            // softplus(z) = max(z, 0) + log(1 + e^-|z|); sigmoid from the same exponential
            const float e = __expf(-fabsf(z));
            const float inv = __frcp_rn(1.0f + e);
            part = yv * z - (fmaxf(z, 0.0f) + __logf(1.0f + e));
            return yv - (z >= 0.0f ? inv : e * inv);
        } else {
            const float r = yv - z;
            part = r * r;
            return r * inv_sig2;
        }
    }

    template <bool GRAD>
    __device__ float eval(const float (&x)[D], float (&g)[D]) const {
        float ell = 0.0f;
        if (GRAD) {
#pragma unroll
            for (int i = 0; i < D; ++i) g[i] = 0.0f;
        }
        const int nch = (n + kRows - 1) / kRows;
        load_chunk(0, 0);
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) { load_chunk(c + 1, (c + 1) & 1); cp_async_wait<1>(); }
            else             { cp_async_wait<0>(); }
            __syncthreads();
            const float* Xc = xs + (c & 1) * kRows * D;
            const float* yc = ys + (c & 1) * kRows;
            int rows = n - c * kRows; rows = rows < kRows ? rows : kRows;
            float part = 0.0f;
            int r = 0;
            // two rows per iteration: independent dot products and epilogues overlap
            for (; r + 1 < rows; r += 2) {
                const float* xa = Xc + r * D;
                const float* xb = xa + D;
                const float za = row_dot(xa, x), zb = row_dot(xb, x);
                float pa, pb;
                const float ra = row_term(za, yc[r], pa), rb = row_term(zb, yc[r + 1], pb);
                part += pa + pb;
                if (GRAD) {
#pragma unroll
                    for (int i = 0; i < D; ++i) g[i] = fmaf(ra, xa[i], fmaf(rb, xb[i], g[i]));
                }
            }
            if (r < rows) {
                const float* xa = Xc + r * D;
                float pa;
                const float ra = row_term(row_dot(xa, x), yc[r], pa);
                part += pa;
                if (GRAD) {
#pragma unroll
                    for (int i = 0; i < D; ++i) g[i] = fmaf(ra, xa[i], g[i]);
                }
            }
            ell += part;
            __syncthreads();
        }
        return LOGISTIC ? ell : (-0.5f * ell * inv_sig2 + lin_const);
    }
};

} // namespace oais
