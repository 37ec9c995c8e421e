// oais_device.cuh -- device building blocks of the OAIS particle sweep (sm_103a).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), one call per
// (particle, step, move, block) counter, so every particle's stream is fixed by its
// index alone (the split-stream "strong parallelism invariance" of App. E.3).
//   counter = (n, t, (k << 16) | j, tag),  key = (seed_lo, seed_hi),
//   tag = round | (problem << 16); t = 0 is the draw from the reference.
//   uniform u = ((r >> 9) + 0.5) * 2^-23  (exact in fp32, never 0 or 1)
//   normals by Box-Muller on the pairs (w0, w1) and (w2, w3);
//   the MH uniform of move k at step t is word 0 of block j = 0xFFFF;
//   the systematic-resampling uniform of step t is word 0 of counter (~0, t, 0, tag).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace oais {

// packed fp32 pairs (one instruction for both lanes of a pair, round to nearest even)
__device__ __forceinline__ float2 add_f32x2(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub_f32x2(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul_f32x2(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 fma_f32x2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

struct Philox4 { uint32_t v[4]; };

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // each 32 x 32 -> 64-bit product is one wide multiply (both halves at once)
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    Philox4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

struct Rng {
    uint32_t k0, k1, tag;
    __device__ __forceinline__ Philox4 block(uint32_t n, uint32_t t, uint32_t k, uint32_t j) const {
        return philox4x32_10(n, t, (k << 16) | (j & 0xFFFFu), tag, k0, k1);
    }
};

// The same generator with its ten round keys precomputed on the host (k + r * W for the Weyl
// constants W above): held in a kernel parameter, each round's key is a constant-bank operand
// of the round's XOR instead of two additions per round and call.
struct RngKS {
    uint32_t k0[10], k1[10], tag;
    __host__ __device__ void set(const Rng& r) {
        for (int i = 0; i < 10; ++i) {
            k0[i] = r.k0 + (uint32_t)i * 0x9E3779B9u;
            k1[i] = r.k1 + (uint32_t)i * 0xBB67AE85u;
        }
        tag = r.tag;
    }
    __device__ __forceinline__ Philox4 block(uint32_t n, uint32_t t, uint32_t k, uint32_t j) const {
        uint32_t c0 = n, c1 = t, c2 = (k << 16) | (j & 0xFFFFu), c3 = tag;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
            const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0[r], n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1[r];
            c1 = (uint32_t)p1;
            c3 = (uint32_t)p0;
            c0 = n0;
            c2 = n2;
        }
        Philox4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
        return o;
    }
};

// u = ((r >> 9) + 1/2) 2^-23: the 23 bits as the mantissa of a float in [1, 2), minus
// 1 - 2^-24 (an exact subtraction by Sterbenz's lemma), the same value as the conversion of
// the integer, without an integer-to-float conversion
__device__ __forceinline__ float u01f(uint32_t r)
{
    return __uint_as_float((r >> 9) | 0x3F800000u) - 0.99999994039535522461f;
}
__device__ __forceinline__ double u01d(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

// four standard normals from one Philox block
__device__ __forceinline__ void box_muller4(const Philox4& b, float z[4])
{
    float s0, c0, s1, c1;
    const float r0 = sqrtf(-2.0f * logf(u01f(b.v[0])));
    const float r1 = sqrtf(-2.0f * logf(u01f(b.v[2])));
    sincospif(2.0f * u01f(b.v[1]), &s0, &c0);
    sincospif(2.0f * u01f(b.v[3]), &s1, &c1);
    z[0] = r0 * c0; z[1] = r0 * s0; z[2] = r1 * c1; z[3] = r1 * s1;
}
// the same four normals with the special-function-unit forms of log2, sqrt, sin and cos
// (documented PTX approximations, absolute error of order 1e-6 in z): the tensor-core kernels,
// whose particle arithmetic is fp32.  The angle 2 pi u is taken as pi (2u - 1) + pi so that
// the sine and cosine arguments lie in (-pi, pi).
__device__ __forceinline__ float sfu_lg2(float x) { float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sfu_sqrt(float x) { float y; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sfu_sin(float x) { float y; asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sfu_cos(float x) { float y; asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ void box_muller4_sfu(const Philox4& b, float z[4])
{
    const float m2ln2 = -1.3862943611198906f;                  // -2 ln 2
    const float pi = 3.14159265358979f;
    const float r0 = sfu_sqrt(m2ln2 * sfu_lg2(u01f(b.v[0])));
    const float r1 = sfu_sqrt(m2ln2 * sfu_lg2(u01f(b.v[2])));
    const float a0 = pi * (2.0f * u01f(b.v[1]) - 1.0f), a1 = pi * (2.0f * u01f(b.v[3]) - 1.0f);
    // cos(a + pi) = -cos a, sin(a + pi) = -sin a
    z[0] = -r0 * sfu_cos(a0); z[1] = -r0 * sfu_sin(a0); z[2] = -r1 * sfu_cos(a1); z[3] = -r1 * sfu_sin(a1);
}
__device__ __forceinline__ void box_muller4(const Philox4& b, double z[4])
{
    double s0, c0, s1, c1;
    const double r0 = sqrt(-2.0 * log(u01d(b.v[0])));
    const double r1 = sqrt(-2.0 * log(u01d(b.v[2])));
    sincospi(2.0 * u01d(b.v[1]), &s0, &c0);
    sincospi(2.0 * u01d(b.v[3]), &s1, &c1);
    z[0] = r0 * c0; z[1] = r0 * s0; z[2] = r1 * c1; z[3] = r1 * s1;
}

// z[0..D) for (n, t, k); only the first d are meaningful, the rest are zero
template <int D, typename R>
__device__ __forceinline__ void normals(const Rng& rng, uint32_t n, uint32_t t, uint32_t k, int d, R (&z)[D])
{
#pragma unroll
    for (int j = 0; j < (D + 3) / 4; ++j) {
        R v[4];
        if (4 * j < d) box_muller4(rng.block(n, t, k, (uint32_t)j), v);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * j + q < D) z[4 * j + q] = (4 * j + q < d) ? v[q] : R(0);
    }
}

template <int D, class G>
__device__ __forceinline__ void normals_sfu(const G& rng, uint32_t n, uint32_t t, uint32_t k, int d, float (&z)[D])
{
#pragma unroll
    for (int j = 0; j < (D + 3) / 4; ++j) {
        float v[4];
        if (4 * j < d) box_muller4_sfu(rng.block(n, t, k, (uint32_t)j), v);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * j + q < D) z[4 * j + q] = (4 * j + q < d) ? v[q] : 0.0f;
    }
}

__device__ __forceinline__ float mh_log_uniform(const Rng& rng, uint32_t n, uint32_t t, uint32_t k, float)
{
    return logf(u01f(rng.block(n, t, k, 0xFFFFu).v[0]));
}
// the same with the special-function logarithm (relative error of order 1e-7; a decision can
// differ from the exact form's only at a near tie): the random-walk moves of the fp32 forms
template <class G>
__device__ __forceinline__ float mh_log_uniform_sfu(const G& rng, uint32_t n, uint32_t t, uint32_t k)
{
    return __logf(u01f(rng.block(n, t, k, 0xFFFFu).v[0]));
}
__device__ __forceinline__ double mh_log_uniform(const Rng& rng, uint32_t n, uint32_t t, uint32_t k, double)
{
    return log(u01d(rng.block(n, t, k, 0xFFFFu).v[0]));
}

// ---------------------------------------------------------------------------
// Per-step moment statistics (Alg. 1, "compute moments"; Sec. 5.1.1):
//   g_hat_{t,i} = sum_n w_{t-1}^n (g_t^n)^i,  i = 0, 1, 2,
// kept as a shifted sum: g_hat = exp(m) * s, and with it the weighted sum of log g_t on
// moment 0's shift, u = sum_n exp(log w - m[0]) log g, so that u / s[0] is the term
// sum_n W_{t-1}^n log g_t^n of the ELBO estimator (Sec. on the KL divergence of a schedule).
// One record per (t, CTA or tile); the records are merged in a fixed order by
// merge_stats_kernel.
// ---------------------------------------------------------------------------
struct StepPartial {
    double m[3];    // shift (an upper estimate of max_n log w + i log g)
    double s[3];    // sum_n exp(log w + i log g - m)
    double u;       // sum_n exp(log w - m[0]) log g
    uint32_t accepted;
    uint32_t pad;
};
static_assert(sizeof(StepPartial) == 64, "StepPartial layout");

constexpr int kMaxWarps = 32;

// log g_t = (beta_t - beta_{t-1}) log L(X_{t-1}); a state outside the likelihood's support
// (log L = -inf) gets weight 0 for any positive increment and keeps its weight for a zero one
__device__ __forceinline__ double log_increment(double dbeta, double ell)
{
    return dbeta == 0.0 ? 0.0 : dbeta * ell;
}
// a log-weight or log-likelihood is admissible unless NaN or +inf (-inf: zero weight or a
// state outside the support)
__device__ __forceinline__ bool admissible(double v) { return !isnan(v) && v != INFINITY; }

// Warp part: v_i = lw + i * lg for the lane's particle (or -inf if inactive).
// Writes the warp's (m_i, s_i) for i = 0..2 and u (ws[3], on m_0) through lane 0.  By default the offsets from the
// anchor particle and from the warp maximum are fp64 differences rounded once.  kFast (the
// forms whose particle arithmetic is fp32; the fp64 pipe of this part is slow): the offsets
// come from two fp64 differences per particle, lw - lw_a and lg - lg_a, rounded to fp32,
// which adds about 2^-24 (|lw - lw_a| + i |lg - lg_a|) to exponent i.  The anchor a is the
// warp's largest v_1 (found from a first pass over the fp32 roundings of log w and log g),
// so that the error is small where the weight is: with an arbitrary
// anchor, spreads of 10^4 in log w (a large first step of a likelihood over hundreds of
// rows) moved D_hat by ~1e-3.  Both paths let log w = -inf (a zero weight) and log g = -inf
// (a state outside the likelihood's support) drop out of the moments they zero.
__device__ __forceinline__ bool finite_bits(double v)
{
    return (__double2hiint(v) & 0x7FF00000) != 0x7FF00000;   // exponent field not all ones
}
// With kFast the lead lane leaves the anchors (wm[0] = log w_a, wm[1] = log g_a) and the fp32
// maxima (ws[4 + i]) instead of forming m_i = log w_a + i log g_a + max_i in fp64, which the CTA
// merge then does for its W pieces only (merge_deferred_pieces; ws holds 8 floats).
template <bool kFast = false>
__device__ __forceinline__ void warp_moment_partial(double lw, double lg, bool active,
                                                    double* wm /*3*/, float* ws /*4, or 8 with kFast*/)
{
    const unsigned full = 0xFFFFFFFFu;
    const bool lead = (threadIdx.x & 31) == 0;
    if (kFast) {
        const bool fw = active && finite_bits(lw), fg = active && finite_bits(lg);
        const unsigned bw = __ballot_sync(full, fw);
        if (bw == 0) {
            if (lead) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    wm[i] = 0.0;
                    ws[i] = 0.0f;
                    ws[4 + i] = -INFINITY;
                }
                ws[3] = 0.0f;
            }
            return;
        }
        const unsigned bg = __ballot_sync(full, fg);
        double a0 = __shfl_sync(full, lw, __ffs(bw) - 1);
        double b0 = bg ? __shfl_sync(full, lg, __ffs(bg) - 1) : 0.0;
        if (__ballot_sync(full, fw && fg)) {
            // re-anchor at the lane with the largest v_1 (a first-pass estimate from the fp32
            // roundings of log w and log g: the anchor need only be near the maximum)
            const float f1 = (fw && fg) ? (float)lw + (float)lg : -INFINITY;
            float m1 = f1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m1 = fmaxf(m1, __shfl_xor_sync(full, m1, o));
            const int src = __ffs(__ballot_sync(full, f1 == m1)) - 1;
            a0 = __shfl_sync(full, lw, src);
            b0 = __shfl_sync(full, lg, src);
        }
        const float dw = (float)(lw - a0), dg = (float)(lg - b0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float f = !active ? -INFINITY : (i == 0 ? dw : dw + (float)i * dg);
            float mx = f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(full, mx, o));
            float e = f > -INFINITY ? __expf(f - mx) : 0.0f;
            float u = (i == 0 && e > 0.0f) ? e * (float)lg : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(full, e, o);
            if (i == 0) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(full, u, o);
            }
            if (lead) {
                ws[4 + i] = mx;
                if (i == 0) { wm[0] = a0; wm[1] = b0; }
                ws[i] = e;
                if (i == 0) ws[3] = u;
            }
        }
        return;
    }
    // per moment, the particles with v_i = lw + i lg > -inf take part (log w or log g may be
    // -inf: zero weight, or a state outside the likelihood's support); the anchor of moment i
    // is the first such particle, and an offset is the fp64 difference rounded once
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double v = i == 0 ? lw : lw + i * lg;
        const bool on = active && v > -INFINITY;
        const unsigned act = __ballot_sync(full, on);
        if (act == 0) {
            if (lead) { wm[i] = -INFINITY; ws[i] = 0.0f; if (i == 0) ws[3] = 0.0f; }
            continue;
        }
        const double anchor = __shfl_sync(full, v, __ffs(act) - 1);
        const float f = on ? (float)(v - anchor) : -INFINITY;
        float mx = f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(full, mx, o));
        const double M = anchor + (double)mx;
        float e = on ? __expf((float)(v - M)) : 0.0f;
        // the ELBO sum: a weighted particle outside the support (log g = -inf) makes it -inf;
        // a weight that underflowed to 0 adds nothing
        float u = (i == 0 && e > 0.0f) ? e * (float)lg : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(full, e, o);
        if (i == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(full, u, o);
        }
        if (lead) {
            wm[i] = M;
            ws[i] = e;
            if (i == 0) ws[3] = u;
        }
    }
}

// Merge of W warps' (m, s) pieces (lane j of the calling warp reads warp j's) in a fixed
// order into one record: M = max_j m_j, S = sum_j s_j exp(m_j - M).  The shifts stay in
// fp64.  kFast: the rescaling takes d_j = m_j - M (exact in fp64) rounded to fp32 and an fp32
// exponential, and the sum is fp32 (|d| e^d <= 1/e bounds the effect of the rounding of d on S
// by 2^-24 / e of S; the pieces s_j are fp32 sums already), a handful of fp64 instructions
// instead of an fp64 exponential per moment: the forms with fp32 particle arithmetic use it,
// the fp64 pipe being slow on this part.  Lanes < W take part (every lane of the warp calls it); W is a
// power of two <= 32.
// kFast = false keeps the rescaling and the sum in fp64 (the fp64 forms).  Lane j < W
// passes piece j's shifts m[3], sums s[3] and count acc; lane 0 writes the record.
template <int W, bool kFast>
__device__ __forceinline__ void merge_lane_pieces(int lane, const double (&mj)[3], const float (&sj)[4],
                                                  unsigned accj, StepPartial* out)
{
    static_assert(W >= 1 && W <= 32 && (W & (W - 1)) == 0, "W: a power of two");
    StepPartial rec;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double m = lane < W ? mj[i] : -INFINITY;
        double M = m;
        if (kFast) {
#pragma unroll
            for (int o = 1; o < W; o <<= 1) M = fmax(M, __shfl_xor_sync(0xFFFFFFFFu, M, o));
        } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) M = fmax(M, __shfl_xor_sync(0xFFFFFFFFu, M, o));
        }
        if (kFast) {
            const float dj = (float)(m - M);      // -inf for an empty piece; NaN when every piece is
            const float fj = (lane < W && !isnan(dj)) ? expf(dj) : 0.0f;
            float v = sj[i] * fj, uu = (i == 0 && fj > 0.0f) ? sj[3] * fj : 0.0f;
#pragma unroll
            for (int o = 1; o < W; o <<= 1) {
                v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                uu += __shfl_xor_sync(0xFFFFFFFFu, uu, o);
            }
            rec.s[i] = (double)v;
            if (i == 0) rec.u = (double)uu;
        } else {
            const double fj = (lane < W && m != -INFINITY) ? exp(m - M) : 0.0;
            double v = (double)sj[i] * fj, uu = (i == 0 && fj > 0.0) ? (double)sj[3] * fj : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                uu += __shfl_xor_sync(0xFFFFFFFFu, uu, o);
            }
            rec.s[i] = v;
            if (i == 0) rec.u = uu;
        }
        rec.m[i] = M;
    }
    unsigned a = lane < W ? accj : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    if (lane == 0) {
        rec.accepted = a;
        rec.pad = 0;
        *out = rec;
    }
}
template <int W, bool kFast>
__device__ __forceinline__ void merge_warp_pieces(int lane, const double (*wm)[3], const float (*ws)[4],
                                                  const unsigned* wacc, StepPartial* out)
{
    double m[3];
    float sv[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) m[i] = lane < W ? wm[lane][i] : -INFINITY;
#pragma unroll
    for (int i = 0; i < 4; ++i) sv[i] = lane < W ? ws[lane][i] : 0.0f;
    merge_lane_pieces<W, kFast>(lane, m, sv, (wacc && lane < W) ? wacc[lane] : 0u, out);
}

// The merge of W pieces written with kFast: lane j < W forms piece j's shifts
// m_i = log w_a + i log g_a + max_i in fp64 (-inf for an empty moment), then as merge_warp_pieces
// with the fp32 rescaling.
template <int W>
__device__ __forceinline__ void merge_deferred_pieces(int lane, const double (*wm)[3], const float (*ws)[8],
                                                      const unsigned* wacc, StepPartial* out)
{
    const bool on = lane < W;
    const double a = on ? wm[lane][0] : 0.0, b = on ? wm[lane][1] : 0.0;
    double m[3];
    float sv[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float mx = on ? ws[lane][4 + i] : -INFINITY;
        m[i] = mx > -INFINITY ? a + i * b + (double)mx : -INFINITY;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) sv[i] = on ? ws[lane][i] : 0.0f;
    merge_lane_pieces<W, true>(lane, m, sv, (wacc && on) ? wacc[lane] : 0u, out);
}

// One record from a CTA's values in shared memory, computed by one half-warp, for the fp32
// forms' lock-step ASMC kernel whose log w is fp64: lane l of the half takes particles l,
// l + 16, ... (NP per lane) with v_i = lw + i lg, lw = lwp[p] + (ess ? lgp[p] : 0) and lg =
// (ess ? lw : lgp[p]), acc[p] the accepted moves (-1: inactive).  ess = false gives the moment
// record of (w_{t-1}, g_t); ess = true the (log w, 2 log w) pieces of w_t for the ESS test.  The
// semantics are warp_moment_partial<true>'s and merge_deferred_pieces' for the whole CTA at
// once: the anchor at the largest fp32 rounding of v_1 (else a particle with a finite log w), the
// offsets fp64 differences rounded once to fp32, the fp64 shift formed once per record.  Both
// halves of the warp call it together (the shuffles span the warp).
template <int NP>
__device__ __forceinline__ void half_record_fp64w(int lane, const double* lwp, const float* lgp, const float* accp,
                                                  bool ess, bool on, StepPartial* out)
{
    const unsigned full = 0xFFFFFFFFu;
    const int half = lane >> 4, l = lane & 15;
    double lw[NP], lg[NP];
    bool act[NP];
    float bk = -INFINITY;
    int bj = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int p = l + 16 * j;
        act[j] = accp[p] >= 0.0f;
        const double g = (double)lgp[p];
        lw[j] = ess ? lwp[p] + g : lwp[p];
        lg[j] = ess ? lw[j] : g;
        const bool fw = act[j] && finite_bits(lw[j]), fg = act[j] && finite_bits(lg[j]);
        const float key = fw ? (fg ? (float)lw[j] + (float)lg[j] : -3.0e38f) : -INFINITY;
        if (key > bk) { bk = key; bj = j; }
    }
    double ca = 0.0, cb = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j)
        if (j == bj) { ca = lw[j]; cb = finite_bits(lg[j]) && act[j] ? lg[j] : 0.0; }
    float mk = bk;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mk = fmaxf(mk, __shfl_xor_sync(full, mk, o));
    const unsigned hb = (__ballot_sync(full, bk == mk && mk > -INFINITY) >> (16 * half)) & 0xFFFFu;
    const int src = hb ? 16 * half + __ffs(hb) - 1 : lane;
    const double a0 = __shfl_sync(full, ca, src), b0 = __shfl_sync(full, cb, src);
    float dw[NP], dg[NP];
    float mx[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        dw[j] = (float)(lw[j] - a0);
        dg[j] = (float)(lg[j] - b0);
        if (act[j]) {
            mx[0] = fmaxf(mx[0], dw[j]);
            mx[1] = fmaxf(mx[1], dw[j] + dg[j]);
            mx[2] = fmaxf(mx[2], dw[j] + 2.0f * dg[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) mx[i] = fmaxf(mx[i], __shfl_xor_sync(full, mx[i], o));
    float e[3] = {0.0f, 0.0f, 0.0f}, u = 0.0f;
    unsigned acc = 0u;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        if (!act[j]) continue;
        const float f[3] = {dw[j], dw[j] + dg[j], dw[j] + 2.0f * dg[j]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float ei = f[i] > -INFINITY ? __expf(f[i] - mx[i]) : 0.0f;
            e[i] += ei;
            if (i == 0 && ei > 0.0f) u += ei * (float)lg[j];
        }
        acc += (unsigned)accp[l + 16 * j];
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) e[i] += __shfl_xor_sync(full, e[i], o);
        u += __shfl_xor_sync(full, u, o);
        acc += __shfl_xor_sync(full, acc, o);
    }
    if (on && l == 0) {
        StepPartial rec;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            rec.m[i] = mx[i] > -INFINITY ? a0 + i * b0 + (double)mx[i] : -INFINITY;
            rec.s[i] = (double)e[i];
        }
        rec.u = (double)u;
        rec.accepted = ess ? 0u : acc;
        rec.pad = 0;
        *out = rec;
    }
}

// ---------------------------------------------------------------------------------------
// fp32-only bookkeeping of the one-thread-per-particle fp32 forms.  GB300's fp64 pipe runs at a
// small fraction of its fp32 rate, so the per-step fp64 additions and conversions of the moment
// bookkeeping occupied it for a third of the mixture sweep.  Instead:
//   log w is held as an unevaluated sum hi + lo of two fp32 values, each step's log g (an fp32
//   value) added by Knuth's TwoSum (hi the rounded sum, lo += the exact rounding error), so that
//   hi + lo carries about 48 bits; a zero weight (-inf) or a non-finite value stays in hi;
//   a step's record takes an anchor particle (a_hi, a_lo, log g_a) and the offsets
//   (hi - a_hi) + (lo - a_lo) + i (log g - log g_a) in fp32 (hi - a_hi is exact where it matters,
//   within a factor of two of the anchor, by Sterbenz's lemma), and forms the fp64 shift
//   a_hi + a_lo + i log g_a + max_i once per record.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void df_add(float& hi, float& lo, float v)
{
    const float s = hi + v;
    if (!isfinite(s)) { hi = s; lo = 0.0f; return; }
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

// One step's record from the CTA's per-particle values, computed by one half-warp: v holds, for
// every particle of the CTA, (log w_{t-1} as the pair hi, lo; log g_t; the step's accepted moves,
// or -1 for an inactive lane), and lane l of the half takes particles l, l + 16, l + 32, ...
// (NP = particles / 16).  The anchor is the particle of largest log w + log g among those with
// both finite (else one with a finite log w); the offsets (hi - a_hi) + (lo - a_lo) +
// i (log g - log g_a) are fp32, and the record's shift is the fp64 a_hi + a_lo + i log g_a +
// max of the offsets.
// Both halves of the warp must call it together (the shuffles span the warp); `on` says whether
// this half's step exists.
template <int NP>
__device__ __forceinline__ void half_step_record_df(int lane, const float4* v, bool on, StepPartial* out)
{
    const unsigned full = 0xFFFFFFFFu;
    const int half = lane >> 4, l = lane & 15;
    float bk = -INFINITY, bh = 0.0f, bl = 0.0f, bg = 0.0f;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float4 r = v[l + 16 * j];
        const bool act = r.w >= 0.0f, fw = act && isfinite(r.x), fg = act && isfinite(r.z);
        const float key = fw ? (fg ? r.x + r.z : -3.0e38f) : -INFINITY;
        if (key > bk) { bk = key; bh = r.x; bl = r.y; bg = fg ? r.z : 0.0f; }
    }
    float mk = bk;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mk = fmaxf(mk, __shfl_xor_sync(full, mk, o));
    const unsigned hb = (__ballot_sync(full, bk == mk && mk > -INFINITY) >> (16 * half)) & 0xFFFFu;
    const int src = hb ? 16 * half + __ffs(hb) - 1 : lane;
    const float ah = __shfl_sync(full, bh, src), al = __shfl_sync(full, bl, src), b0 = __shfl_sync(full, bg, src);
    float mx[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float4 r = v[l + 16 * j];
        if (r.w >= 0.0f) {
            const float dw = (r.x - ah) + (r.y - al), dg = r.z - b0;
            mx[0] = fmaxf(mx[0], dw);
            mx[1] = fmaxf(mx[1], dw + dg);
            mx[2] = fmaxf(mx[2], dw + 2.0f * dg);
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) mx[i] = fmaxf(mx[i], __shfl_xor_sync(full, mx[i], o));
    float e[3] = {0.0f, 0.0f, 0.0f}, u = 0.0f;
    unsigned acc = 0u;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float4 r = v[l + 16 * j];
        if (r.w >= 0.0f) {
            const float dw = (r.x - ah) + (r.y - al), dg = r.z - b0;
            const float f[3] = {dw, dw + dg, dw + 2.0f * dg};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float ei = f[i] > -INFINITY ? __expf(f[i] - mx[i]) : 0.0f;
                e[i] += ei;
                if (i == 0 && ei > 0.0f) u += ei * r.z;
            }
            acc += (unsigned)r.w;
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) e[i] += __shfl_xor_sync(full, e[i], o);
        u += __shfl_xor_sync(full, u, o);
        acc += __shfl_xor_sync(full, acc, o);
    }
    if (on && l == 0) {
        StepPartial rec;
        const double a = (double)ah + (double)al;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            rec.m[i] = mx[i] > -INFINITY ? a + i * (double)b0 + (double)mx[i] : -INFINITY;
            rec.s[i] = (double)e[i];
        }
        rec.u = (double)u;
        rec.accepted = acc;
        rec.pad = 0;
        *out = rec;
    }
}


// CTA part: warp 0 merges the W warps' pieces and writes one record.  Call after a
// __syncthreads that follows warp_moment_partial.
template <int W, bool kFast = false>
__device__ __forceinline__ void cta_moment_record(const double (*wm)[3], const float (*ws)[4],
                                                  const unsigned* wacc, StepPartial* out)
{
    if ((threadIdx.x >> 5) != 0) return;
    merge_warp_pieces<W, kFast>(threadIdx.x & 31, wm, ws, wacc, out);
}

// merge (m, s) pairs: exp(m) s + exp(m') s'
__device__ __forceinline__ void lse_merge(double& m, double& s, double m2, double s2)
{
    if (m2 == -INFINITY) return;
    if (m == -INFINITY) { m = m2; s = s2; return; }
    if (m2 > m) { s = s * exp(m - m2) + s2; m = m2; }
    else        { s = s + s2 * exp(m2 - m); }
}

} // namespace oais
