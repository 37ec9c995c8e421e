// sweep_wide.cu -- the plain FP32 CUDA-core form of the loop-swapped sweep (Sec. 5.1.2) for the
// row families (logistic and linear regression) at state dimensions 32 < d <= 256, where a
// particle's state no longer fits in one thread's registers.
//
// A CTA owns a tile of 64 particles for the whole sweep and runs Alg. 1 on it in lock-step:
// every evaluation of log L and grad log L at the tile's 64 states is two fp32 contractions
// on the CUDA cores over the data X, streamed through shared memory in chunks of 64 rows
// (cp.async, double-buffered):
//   forward   Z[r][p] = sum_k X[r][k] Y[k][p]      (Y: the tile's states, in shared memory)
//   epilogue  f = per-row log-likelihood term, R[r][p] = df/dz
//   backward  G[k][p] += sum_r X[r][k] R[r][p]     (G: the gradients, in registers)
// Each thread computes a 4 x 4 block of Z and an (DP/32) x 8 block of G, so both contractions
// run at 8-16 fused multiply-adds per 16-byte shared-memory load, and loads the next step's
// operands while the current step's multiply-adds run (at d = 256 into a second register set,
// the two sets alternating, so no copies between prefetched and current operands).  Particle vectors (positions,
// gradients, momenta) live in device memory between evaluations, each thread touching only
// its own elements; the per-particle sums of the Metropolis-Hastings ratios are warp
// reductions; one moment record per (step, tile) as in the other forms.
//
// Thread layout ("coordinate layout"): warp w owns particles 8w .. 8w + 7 of the tile, lane l
// the coordinates coord(a), a < KB = DP / 32: for KB >= 4, 128 (a / 4) + 4 l + a % 4 (whole
// Philox blocks of four normals, and 16-byte shared-memory loads that are contiguous across
// the warp); for KB = 2, 2 l + a.  The per-particle scalars (log w, log L, the MH decision) of
// particle 8w + b are held by lane b < 8 of warp w.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace oais {
namespace wide {

constexpr int kP = 64;               // particles per tile (one CTA)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kPW = kP / kWarps;     // particles per warp in the coordinate layout (8)
constexpr int kTS = kP + 4;          // row stride (floats) of the particle-minor tiles Y and R
static_assert(kPW == 8, "coordinate layout: 8 particles per warp");

template <int DP>
struct Lay {
    static constexpr int KB = DP / 32;                       // coordinates per lane
    // data rows per chunk (each thread's forward block is kRPT rows x 4 particles): 64 rows,
    // 4 x 4 blocks, measured faster than 32 rows and 2 x 4 blocks at every width, although the
    // larger buffers leave room for fewer tiles per SM at d <= 128
    static constexpr int kRows = 64;
    static constexpr int kRPT = kRows / 16;
    static constexpr int kXS = DP + 4;                       // X chunk row stride (floats)
    static constexpr int kOffX = 0;                          // [2][kRows][kXS]
    static constexpr int kOffYv = kOffX + 2 * kRows * kXS;   // [2][kRows] responses / labels
    static constexpr int kOffY = kOffYv + 2 * kRows;         // [DP][kTS] evaluation point
    static constexpr int kOffR = kOffY + DP * kTS;           // [kRows][kTS] df/dz
    static constexpr int kOffRed = kOffR + kRows * kTS;      // [kWarps][kP] log L partial sums
    static constexpr int kOffEll = kOffRed + kWarps * kP;    // [kP] log L of the evaluation
    static constexpr int kFloats = kOffEll + kP;
    static constexpr size_t kBytes = sizeof(float) * (size_t)kFloats;
    static_assert(DP == 64 || DP == 128 || DP == 256, "wide widths");
    static_assert(kBytes <= 227 * 1024, "shared memory budget");
    __device__ static int coord(int a, int lane) { return KB >= 4 ? 128 * (a / 4) + 4 * lane + (a % 4) : 2 * lane + a; }
};

struct Args {
    SweepParams sp;
    const float* X;          // [n_pad][DP] zero-padded columns
    const float* yv;         // [n_pad]
    int n, d, tiles;
    int64_t Np;              // tiles * 64: the row length of the state arrays
    float* xs;               // [DP][Np] positions
    float* gs;               // [DP][Np] grad log L at xs
    float* ms;               // [DP][Np] MALA w / HMC momentum
    float inv_sig2, lin_const;   // linear regression
    // potential mode: one evaluation at given states (sweep skipped)
    const float* x_in;       // [d][pstride]
    double* ell_pot;         // [N]
    float* grad_pot;         // [d][pstride] or null
    int64_t pstride, N;
};

template <int DP, bool LOGISTIC>
struct Eval {
    using L = Lay<DP>;
    static constexpr int KB = L::KB;

    __device__ static void load_chunk(const Args& A, float* sm, int c, int buf)
    {
        const int r0 = c * L::kRows;
        const int rows = min(L::kRows, A.n - r0);
        const float* src = A.X + (size_t)r0 * DP;
        float* dst = sm + L::kOffX + buf * L::kRows * L::kXS;
        constexpr int kPieces = DP / 4;                 // 16-byte pieces per row
        for (int i = threadIdx.x; i < rows * kPieces; i += kThreads) {
            const int r = i / kPieces, q = i % kPieces;
            cp_async16(dst + r * L::kXS + 4 * q, src + (size_t)r * DP + 4 * q);
        }
        const float* sy = A.yv + r0;
        float* dy = sm + L::kOffYv + buf * L::kRows;
        for (int i = threadIdx.x; i < (rows + 3) / 4; i += kThreads) cp_async16(dy + 4 * i, sy + 4 * i);
        cp_async_commit();
    }

    // per-row term f(y, z) into part; returns df/dz (the same arithmetic as the register form)
    __device__ __forceinline__ static float row_term(const Args& A, float z, float yr, float& part)
    {
        if (LOGISTIC) {
            const float e = __expf(-fabsf(z));
            const float inv = __frcp_rn(1.0f + e);
            part = yr * z - (fmaxf(z, 0.0f) + __logf(1.0f + e));
            return yr - (z >= 0.0f ? inv : e * inv);
        } else {
            const float r = yr - z;
            part = r * r;
            return r * A.inv_sig2;
        }
    }

    // log L at the tile's states (shared-memory tile Y) into sm[kOffEll + p]; with GRAD the
    // gradient in G (the coordinate layout).  Every thread of the CTA calls it; it starts and
    // ends on a barrier.
    template <bool GRAD>
    __device__ static void run(const Args& A, float* sm, float (&G)[KB][kPW])
    {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const int rb = tid / 16, pb = tid % 16;        // forward block: rows 2 rb, 2 rb + 1; particles 4 pb ..
        const float* Y = sm + L::kOffY;
        float* R = sm + L::kOffR;
#pragma unroll
        for (int a = 0; a < KB; ++a)
#pragma unroll
            for (int b = 0; b < kPW; ++b) G[a][b] = 0.0f;
        float part[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int nch = (A.n + L::kRows - 1) / L::kRows;
        load_chunk(A, sm, 0, 0);
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) { load_chunk(A, sm, c + 1, (c + 1) & 1); cp_async_wait<1>(); }
            else             { cp_async_wait<0>(); }
            __syncthreads();
            const float* Xc = sm + L::kOffX + (c & 1) * L::kRows * L::kXS;
            const float* yc = sm + L::kOffYv + (c & 1) * L::kRows;
            const int rows = min(L::kRows, A.n - c * L::kRows);
            // forward: a kRPT x 4 block of Z (rows kRPT rb ..; particles 4 pb ..); the next k step's
            // operands are loaded while this one's multiply-adds run
            constexpr int RPT = L::kRPT;
            float z[RPT][4];
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) z[i][j] = 0.0f;
            const float* xrow = Xc + (RPT * rb) * L::kXS;
            float4 xa[RPT], ya[4];
            auto load_k = [&](int k, float4 (&xv)[RPT], float4 (&yv)[4]) {
#pragma unroll
                for (int i = 0; i < RPT; ++i) xv[i] = *reinterpret_cast<const float4*>(xrow + i * L::kXS + k);
#pragma unroll
                for (int q = 0; q < 4; ++q) yv[q] = *reinterpret_cast<const float4*>(Y + (k + q) * kTS + 4 * pb);
            };
            auto fma_k = [&](const float4 (&xv)[RPT], const float4 (&yv)[4]) {
#pragma unroll
                for (int i = 0; i < RPT; ++i) {
                    const float fx[4] = {xv[i].x, xv[i].y, xv[i].z, xv[i].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        z[i][0] = fmaf(fx[q], yv[q].x, z[i][0]); z[i][1] = fmaf(fx[q], yv[q].y, z[i][1]);
                        z[i][2] = fmaf(fx[q], yv[q].z, z[i][2]); z[i][3] = fmaf(fx[q], yv[q].w, z[i][3]);
                    }
                }
            };
            load_k(0, xa, ya);
            if constexpr (DP >= 256) {
                // one tile per SM and the full register budget: two register sets of operands,
                // used alternately (no copies between them)
                float4 xb[RPT], yb[4];
#pragma unroll 1
                for (int k = 0; k < DP; k += 8) {
                    load_k(k + 4, xb, yb);                 // DP is a multiple of 8
                    fma_k(xa, ya);
                    if (k + 8 < DP) load_k(k + 8, xa, ya);
                    fma_k(xb, yb);
                }
            } else {
                // two or three tiles per SM: one set, the next step's operands loaded ahead
#pragma unroll 2
                for (int k = 0; k < DP; k += 4) {
                    float4 xn[RPT], yn[4];
                    load_k(k + 4 < DP ? k + 4 : k, xn, yn);
                    fma_k(xa, ya);
#pragma unroll
                    for (int i = 0; i < RPT; ++i) xa[i] = xn[i];
#pragma unroll
                    for (int q = 0; q < 4; ++q) ya[q] = yn[q];
                }
            }
            // epilogue: rows past the data (stale buffer contents) are masked by selects
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int r = RPT * rb + i;
                const bool valid = r < rows;
                const float yr = valid ? yc[r] : 0.0f;
                float rv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float f;
                    const float dz = row_term(A, z[i][j], yr, f);
                    part[j] += valid ? f : 0.0f;
                    rv[j] = valid ? dz : 0.0f;
                }
                if (GRAD) *reinterpret_cast<float4*>(R + r * kTS + 4 * pb) = make_float4(rv[0], rv[1], rv[2], rv[3]);
            }
            if (GRAD) {
                __syncthreads();
                // backward: G[coord(a)][8 warp + b] += sum_r X[r][coord(a)] R[r][8 warp + b], the next
                // row's operands loaded while this row's multiply-adds run
                auto load_row = [&](int r, float (&xv)[KB], float (&rr)[kPW]) {
                    const float* xr = Xc + r * L::kXS;
                    if (KB >= 4) {
#pragma unroll
                        for (int g4 = 0; g4 < KB / 4; ++g4) {
                            const float4 v = *reinterpret_cast<const float4*>(xr + 128 * g4 + 4 * lane);
                            xv[4 * g4] = v.x; xv[4 * g4 + 1] = v.y; xv[4 * g4 + 2] = v.z; xv[4 * g4 + 3] = v.w;
                        }
                    } else {
                        const float2 v = *reinterpret_cast<const float2*>(xr + 2 * lane);
                        xv[0] = v.x; xv[KB - 1] = v.y;
                    }
                    const float4 r0 = *reinterpret_cast<const float4*>(R + r * kTS + kPW * warp);
                    const float4 r1 = *reinterpret_cast<const float4*>(R + r * kTS + kPW * warp + 4);
                    rr[0] = r0.x; rr[1] = r0.y; rr[2] = r0.z; rr[3] = r0.w;
                    rr[4] = r1.x; rr[5] = r1.y; rr[6] = r1.z; rr[7] = r1.w;
                };
                auto fma_row = [&](const float (&xv)[KB], const float (&rr)[kPW]) {
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) G[a][b] = fmaf(xv[a], rr[b], G[a][b]);
                };
                if (DP >= 256 && rows > 0) {
                    // one tile per SM and the full register budget: two register sets of operands,
                    // used alternately (no copies between them)
                    float xa[KB], ra[kPW], xb[KB], rb2[kPW];
                    load_row(0, xa, ra);
                    int r = 0;
#pragma unroll 1
                    for (; r + 1 < rows; r += 2) {
                        load_row(r + 1, xb, rb2);
                        fma_row(xa, ra);
                        if (r + 2 < rows) load_row(r + 2, xa, ra);
                        fma_row(xb, rb2);
                    }
                    if (r < rows) fma_row(xa, ra);   // an odd last row
                } else if (rows > 0) {
                    // two or three tiles per SM: one set, the next row's operands loaded ahead
                    float xv[KB], rr[kPW];
                    load_row(0, xv, rr);
                    for (int r = 0; r < rows; ++r) {
                        float xn[KB], rn[kPW];
                        load_row(r + 1 < rows ? r + 1 : r, xn, rn);
                        fma_row(xv, rr);
#pragma unroll
                        for (int a = 0; a < KB; ++a) xv[a] = xn[a];
#pragma unroll
                        for (int b = 0; b < kPW; ++b) rr[b] = rn[b];
                    }
                }
            }
            __syncthreads();   // the chunk's buffers and R are free for the next chunk
        }
        // log L per particle: lanes l and l ^ 16 share particles 4 pb .. 4 pb + 3; then the warps
        float* red = sm + L::kOffRed;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            part[j] += __shfl_xor_sync(0xFFFFFFFFu, part[j], 16);
            if (lane < 16) red[warp * kP + 4 * pb + j] = part[j];
        }
        __syncthreads();
        if (tid < kP) {
            float s = 0.0f;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += red[w * kP + tid];
            sm[L::kOffEll + tid] = LOGISTIC ? s : (-0.5f * s * A.inv_sig2 + A.lin_const);
        }
        __syncthreads();
    }
};

// the 8 per-particle sums of a warp (one per particle 8 w + b, partial over this lane's
// coordinates) reduced over the warp's 32 lanes; every lane gets the 8 totals
__device__ __forceinline__ void warp_sum8(float (&v)[kPW])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int b = 0; b < kPW; ++b) v[b] += __shfl_xor_sync(0xFFFFFFFFu, v[b], o);
}
__device__ __forceinline__ float pick8(const float (&v)[kPW], int b)
{
    float r = v[0];
#pragma unroll
    for (int i = 1; i < kPW; ++i) r = b == i ? v[i] : r;
    return r;
}

// the standard normals of the thread's elements for counter (n_b, t, k): particle b's
// coordinates coord(a) (zero past d)
template <int DP>
__device__ __forceinline__ void draw_normals(const Rng& rng, const uint32_t (&nb)[kPW], uint32_t t, uint32_t k,
                                             int d, int lane, float (&z)[Lay<DP>::KB][kPW])
{
    constexpr int KB = Lay<DP>::KB;
#pragma unroll
    for (int b = 0; b < kPW; ++b) {
        if (KB >= 4) {
#pragma unroll
            for (int g4 = 0; g4 < KB / 4; ++g4) {
                const int j = 32 * g4 + lane;          // Philox block of coordinates 4 j .. 4 j + 3
                float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (4 * j < d) box_muller4(rng.block(nb[b], t, k, (uint32_t)j), v);
#pragma unroll
                for (int q = 0; q < 4; ++q) z[4 * g4 + q][b] = (4 * j + q < d) ? v[q] : 0.0f;
            }
        } else {
            const int j = lane / 2;                    // the pair 2 l, 2 l + 1 is half of block l / 2
            float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (4 * j < d) box_muller4(rng.block(nb[b], t, k, (uint32_t)j), v);
#pragma unroll
            for (int a = 0; a < KB; ++a) {
                const int c = 2 * lane + a;
                z[a][b] = c < d ? v[2 * (lane & 1) + a] : 0.0f;
            }
        }
    }
}

// element (a, b) of a state array [DP][Np]: row coord(a), column tile * 64 + 8 warp + b
template <int DP>
__device__ __forceinline__ void load_vec(const float* base, int64_t Np, int64_t col0, int lane, float (&v)[Lay<DP>::KB][kPW])
{
#pragma unroll
    for (int a = 0; a < Lay<DP>::KB; ++a) {
        const float* p = base + (size_t)Lay<DP>::coord(a, lane) * Np + col0;
        const float4 u0 = *reinterpret_cast<const float4*>(p), u1 = *reinterpret_cast<const float4*>(p + 4);
        v[a][0] = u0.x; v[a][1] = u0.y; v[a][2] = u0.z; v[a][3] = u0.w;
        v[a][4] = u1.x; v[a][5] = u1.y; v[a][6] = u1.z; v[a][7] = u1.w;
    }
}
template <int DP>
__device__ __forceinline__ void store_vec(float* base, int64_t Np, int64_t col0, int lane, const float (&v)[Lay<DP>::KB][kPW])
{
#pragma unroll
    for (int a = 0; a < Lay<DP>::KB; ++a) {
        float* p = base + (size_t)Lay<DP>::coord(a, lane) * Np + col0;
        *reinterpret_cast<float4*>(p) = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
        *reinterpret_cast<float4*>(p + 4) = make_float4(v[a][4], v[a][5], v[a][6], v[a][7]);
    }
}
// the same elements of the shared evaluation tile Y [DP][kTS]
template <int DP>
__device__ __forceinline__ void store_tile(float* Y, int warp, int lane, const float (&v)[Lay<DP>::KB][kPW])
{
#pragma unroll
    for (int a = 0; a < Lay<DP>::KB; ++a) {
        float* p = Y + Lay<DP>::coord(a, lane) * kTS + kPW * warp;
        *reinterpret_cast<float4*>(p) = make_float4(v[a][0], v[a][1], v[a][2], v[a][3]);
        *reinterpret_cast<float4*>(p + 4) = make_float4(v[a][4], v[a][5], v[a][6], v[a][7]);
    }
}
template <int DP>
__device__ __forceinline__ void load_tile(const float* Y, int warp, int lane, float (&v)[Lay<DP>::KB][kPW])
{
#pragma unroll
    for (int a = 0; a < Lay<DP>::KB; ++a) {
        const float* p = Y + Lay<DP>::coord(a, lane) * kTS + kPW * warp;
        const float4 u0 = *reinterpret_cast<const float4*>(p), u1 = *reinterpret_cast<const float4*>(p + 4);
        v[a][0] = u0.x; v[a][1] = u0.y; v[a][2] = u0.z; v[a][3] = u0.w;
        v[a][4] = u1.x; v[a][5] = u1.y; v[a][6] = u1.z; v[a][7] = u1.w;
    }
}

// CTAs per SM the register allocation must allow: two tiles per SM at d <= 64 (128 registers,
// measured faster than three at 85 registers, which spill), one above
template <int DP> struct WideMinBlocks { static constexpr int value = DP <= 64 ? 2 : 1; };

template <int DP, bool LOGISTIC, int MOVE>
__global__ void __launch_bounds__(kThreads, WideMinBlocks<DP>::value)
wide_sweep_kernel(const Args A)
{
    extern __shared__ __align__(16) float sm[];
    using L = Lay<DP>;
    using E = Eval<DP, LOGISTIC>;
    constexpr int KB = L::KB;
    constexpr bool GRAD = MOVE != kRwmh;
    __shared__ double s_m[2][kWarps][3];
    __shared__ float s_s[2][kWarps][8];
    __shared__ unsigned s_acc[2][kWarps];

    const SweepParams& P = A.sp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t col0 = tile * kP + kPW * warp;        // this warp's first particle (state column)
    float* Y = sm + L::kOffY;
    // particle counters of the thread's 8 particles (inactive ones shadow the last particle, so
    // that the tile always evaluates finite states; their results are never written)
    uint32_t nb[kPW];
#pragma unroll
    for (int b = 0; b < kPW; ++b) {
        const int64_t q = col0 + b;
        nb[b] = (uint32_t)(P.n_offset + (q < P.N ? q : P.N - 1));
    }
    // lane b < 8 holds particle col0 + b's scalars
    const int64_t qs = col0 + (lane < kPW ? lane : 0);
    const bool owner = lane < kPW;
    const bool act = owner && qs < P.N;
    const float s = (float)P.ref_scale, inv_s2 = 1.0f / (s * s);

    float G[KB][kPW];
    {
        float x0[KB][kPW];
        draw_normals<DP>(P.mv.rng, nb, 0u, 0u, A.d, lane, x0);
#pragma unroll
        for (int a = 0; a < KB; ++a)
#pragma unroll
            for (int b = 0; b < kPW; ++b) x0[a][b] *= s;
        store_vec<DP>(A.xs, A.Np, col0, lane, x0);
        store_tile<DP>(Y, warp, lane, x0);
    }
    E::template run<GRAD>(A, sm, G);
    if (GRAD) store_vec<DP>(A.gs, A.Np, col0, lane, G);
    float ell = sm[L::kOffEll + kPW * warp + (owner ? lane : 0)];
    double logw = 0.0;

    double beta_prev = P.beta[0];
    for (int t = 1; t <= P.T; ++t) {
        const double beta_t = __ldg(P.beta + t);
        const double eps_t = __ldg(P.eps + t - 1);
        const double lg = step_log_increment<float>(beta_t - beta_prev, ell);
        beta_prev = beta_t;
        const float beta = (float)beta_t, e = (float)eps_t, h = 0.5f * e;
        const int slot = t & 1;
        warp_moment_partial<true>(logw, lg, act, s_m[slot][warp], s_s[slot][warp]);
        logw += lg;
        unsigned acc = 0;
        for (int k = 0; k < P.mv.K; ++k) {
            float zz[kPW], dxx[kPW], rev[kPW];
#pragma unroll
            for (int b = 0; b < kPW; ++b) { zz[b] = 0.0f; dxx[b] = 0.0f; rev[b] = 0.0f; }
            {
                float z[KB][kPW], x[KB][kPW], g[KB][kPW];
                draw_normals<DP>(P.mv.rng, nb, (uint32_t)t, (uint32_t)k, A.d, lane, z);
                load_vec<DP>(A.xs, A.Np, col0, lane, x);
                if (MOVE == kRwmh) {
                    float sd = e;
                    if (P.mv.cycle) {
                        const int c = ((t - 1) * P.mv.K + k) % 3;
                        sd = c == 0 ? 0.1f : (c == 1 ? 1.0f : 10.0f);
                    }
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) {
                            const float xp = x[a][b] + sd * z[a][b];
                            dxx[b] += (xp - x[a][b]) * (xp + x[a][b]);
                            z[a][b] = xp;
                        }
                    store_tile<DP>(Y, warp, lane, z);
                } else if (MOVE == kMala) {
                    load_vec<DP>(A.gs, A.Np, col0, lane, g);
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) {
                            const float gpi = -x[a][b] * inv_s2 + beta * g[a][b];
                            const float xp = x[a][b] + e * (h * gpi + z[a][b]);
                            zz[b] += z[a][b] * z[a][b];
                            z[a][b] = z[a][b] + h * gpi;                  // w
                            dxx[b] += (xp - x[a][b]) * (xp + x[a][b]);
                            x[a][b] = xp;
                        }
                    store_vec<DP>(A.ms, A.Np, col0, lane, z);
                    store_tile<DP>(Y, warp, lane, x);
                } else {
                    // HMC, identity mass: momentum p (kept in ms), position x' in the tile
                    load_vec<DP>(A.gs, A.Np, col0, lane, g);
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) {
                            zz[b] += z[a][b] * z[a][b];                   // 2 x kinetic energy at the start
                            z[a][b] += 0.5f * e * (-x[a][b] * inv_s2 + beta * g[a][b]);
                        }
                    store_vec<DP>(A.ms, A.Np, col0, lane, z);
                    store_tile<DP>(Y, warp, lane, x);
                }
            }
            float ellp;
            if (MOVE == kHmc) {
                for (int l = 0; l < P.mv.leapfrog; ++l) {
                    {
                        float p[KB][kPW], xp[KB][kPW];
                        load_vec<DP>(A.ms, A.Np, col0, lane, p);
                        load_tile<DP>(Y, warp, lane, xp);
#pragma unroll
                        for (int a = 0; a < KB; ++a)
#pragma unroll
                            for (int b = 0; b < kPW; ++b) xp[a][b] += e * p[a][b];
                        store_tile<DP>(Y, warp, lane, xp);
                    }
                    E::template run<true>(A, sm, G);
                    float p[KB][kPW], xp[KB][kPW];
                    load_vec<DP>(A.ms, A.Np, col0, lane, p);
                    load_tile<DP>(Y, warp, lane, xp);
                    const float f = (l + 1 < P.mv.leapfrog) ? e : 0.5f * e;
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) p[a][b] += f * (-xp[a][b] * inv_s2 + beta * G[a][b]);
                    store_vec<DP>(A.ms, A.Np, col0, lane, p);
                }
                float p[KB][kPW], xp[KB][kPW], x[KB][kPW];
                load_vec<DP>(A.ms, A.Np, col0, lane, p);
                load_tile<DP>(Y, warp, lane, xp);
                load_vec<DP>(A.xs, A.Np, col0, lane, x);
#pragma unroll
                for (int a = 0; a < KB; ++a)
#pragma unroll
                    for (int b = 0; b < kPW; ++b) {
                        rev[b] += p[a][b] * p[a][b];                       // 2 x kinetic energy at the end
                        dxx[b] += (xp[a][b] - x[a][b]) * (xp[a][b] + x[a][b]);
                    }
                ellp = sm[L::kOffEll + kPW * warp + (owner ? lane : 0)];
            } else {
                E::template run<GRAD>(A, sm, G);
                ellp = sm[L::kOffEll + kPW * warp + (owner ? lane : 0)];
                if (MOVE == kMala) {
                    float w[KB][kPW], xp[KB][kPW];
                    load_vec<DP>(A.ms, A.Np, col0, lane, w);
                    load_tile<DP>(Y, warp, lane, xp);
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) {
                            const float q = w[a][b] + h * (-xp[a][b] * inv_s2 + beta * G[a][b]);
                            rev[b] += q * q;
                        }
                }
            }
            warp_sum8(zz);
            warp_sum8(dxx);
            warp_sum8(rev);
            const int me = owner ? lane : 0;
            float log_alpha = -0.5f * pick8(dxx, me) * inv_s2 + beta * (ellp - ell);
            if (MOVE != kRwmh) log_alpha -= 0.5f * (pick8(rev, me) - pick8(zz, me));
            const float logu = mh_log_uniform(P.mv.rng, nb[me], (uint32_t)t, (uint32_t)k, 0.0f);
            const bool accept = owner && logu < log_alpha;
            if (accept) ell = ellp;
            acc += (accept && act) ? 1u : 0u;
            const unsigned mask = __ballot_sync(0xFFFFFFFFu, accept);
            if (mask) {
                float x[KB][kPW], xp[KB][kPW];
                load_vec<DP>(A.xs, A.Np, col0, lane, x);
                load_tile<DP>(Y, warp, lane, xp);
#pragma unroll
                for (int a = 0; a < KB; ++a)
#pragma unroll
                    for (int b = 0; b < kPW; ++b) x[a][b] = ((mask >> b) & 1u) ? xp[a][b] : x[a][b];
                store_vec<DP>(A.xs, A.Np, col0, lane, x);
                if (GRAD) {
                    float g[KB][kPW];
                    load_vec<DP>(A.gs, A.Np, col0, lane, g);
#pragma unroll
                    for (int a = 0; a < KB; ++a)
#pragma unroll
                        for (int b = 0; b < kPW; ++b) g[a][b] = ((mask >> b) & 1u) ? G[a][b] : g[a][b];
                    store_vec<DP>(A.gs, A.Np, col0, lane, g);
                }
            }
        }
        unsigned wa = acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wa += __shfl_xor_sync(0xFFFFFFFFu, wa, o);
        if (lane == 0) s_acc[slot][warp] = wa;
        __syncthreads();
        if (warp == 0)
            merge_deferred_pieces<kWarps>(lane, s_m[slot], s_s[slot], s_acc[slot],
                                          P.partials + (size_t)(t - 1) * A.tiles + tile);
    }
    // final particles: log w, log L and the positions [d][N] of the active particles
    if (act) {
        P.logw[qs] = logw;
        P.ell_out[qs] = (double)ell;
        if (!admissible(logw) || !admissible((double)ell)) atomicOr(P.status, 1u);
    }
    {
        float x[KB][kPW];
        load_vec<DP>(A.xs, A.Np, col0, lane, x);
        float* xo = reinterpret_cast<float*>(P.x_out);
#pragma unroll
        for (int a = 0; a < KB; ++a) {
            const int c = L::coord(a, lane);
            if (c < A.d)
#pragma unroll
                for (int b = 0; b < kPW; ++b)
                    if (col0 + b < P.N) xo[(size_t)c * P.N + col0 + b] = x[a][b];
        }
    }
}

// one evaluation (log L and, if grad_pot, grad log L) at the states x_in [d][pstride]
template <int DP, bool LOGISTIC>
__global__ void __launch_bounds__(kThreads, WideMinBlocks<DP>::value)
wide_potential_kernel(const Args A)
{
    extern __shared__ __align__(16) float sm[];
    using L = Lay<DP>;
    constexpr int KB = L::KB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t col0 = (int64_t)blockIdx.x * kP + kPW * warp;
    float v[KB][kPW];
#pragma unroll
    for (int a = 0; a < KB; ++a) {
        const int c = L::coord(a, lane);
#pragma unroll
        for (int b = 0; b < kPW; ++b) {
            const int64_t q = col0 + b < A.N ? col0 + b : A.N - 1;
            v[a][b] = c < A.d ? A.x_in[(size_t)c * A.pstride + q] : 0.0f;
        }
    }
    store_tile<DP>(sm + L::kOffY, warp, lane, v);
    float G[KB][kPW];
    if (A.grad_pot) Eval<DP, LOGISTIC>::template run<true>(A, sm, G);
    else Eval<DP, LOGISTIC>::template run<false>(A, sm, G);
    if (tid < kP && (int64_t)blockIdx.x * kP + tid < A.N)
        A.ell_pot[(int64_t)blockIdx.x * kP + tid] = (double)sm[L::kOffEll + tid];
    if (A.grad_pot) {
#pragma unroll
        for (int a = 0; a < KB; ++a) {
            const int c = L::coord(a, lane);
            if (c < A.d)
#pragma unroll
                for (int b = 0; b < kPW; ++b)
                    if (col0 + b < A.N) A.grad_pot[(size_t)c * A.pstride + col0 + b] = G[a][b];
        }
    }
}

template <int DP, bool LOGISTIC, int MOVE>
static cudaError_t launch3(const Args& A, bool potential, cudaStream_t s)
{
    const size_t smem = Lay<DP>::kBytes;
    if (potential) {
        auto* k = &wide_potential_kernel<DP, LOGISTIC>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)((A.N + kP - 1) / kP), kThreads, smem, s>>>(A);
    } else {
        auto* k = &wide_sweep_kernel<DP, LOGISTIC, MOVE>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<A.tiles, kThreads, smem, s>>>(A);
    }
    return cudaGetLastError();
}

template <int DP>
static cudaError_t launch2(const Args& A, bool logistic, int move, bool potential, cudaStream_t s)
{
    if (logistic) {
        switch (move) {
        case kRwmh: return launch3<DP, true, kRwmh>(A, potential, s);
        case kMala: return launch3<DP, true, kMala>(A, potential, s);
        case kHmc:  return launch3<DP, true, kHmc>(A, potential, s);
        }
    } else {
        switch (move) {
        case kRwmh: return launch3<DP, false, kRwmh>(A, potential, s);
        case kMala: return launch3<DP, false, kMala>(A, potential, s);
        case kHmc:  return launch3<DP, false, kHmc>(A, potential, s);
        }
    }
    return cudaErrorInvalidValue;
}

static Args make_args(const DevTarget& t)
{
    Args A{};
    A.X = static_cast<const float*>(t.X);
    A.yv = static_cast<const float*>(t.y);
    A.n = t.n;
    A.d = t.d;
    const double sig2 = t.p0 * t.p0;
    A.inv_sig2 = (float)(1.0 / sig2);
    A.lin_const = (float)(-0.5 * t.n * std::log(6.283185307179586 * sig2));
    return A;
}

static cudaError_t dispatch(const Args& A, int D, bool logistic, int move, bool potential, cudaStream_t s)
{
    switch (D) {
    case 64: return launch2<64>(A, logistic, move, potential, s);
    case 128: return launch2<128>(A, logistic, move, potential, s);
    case 256: return launch2<256>(A, logistic, move, potential, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace wide

int wide_width(int d) { return d <= 64 ? 64 : (d <= 128 ? 128 : (d <= 256 ? 256 : 0)); }
int wide_tiles(int64_t N) { return (int)((N + wide::kP - 1) / wide::kP); }
size_t wide_state_bytes(int D, int64_t N) { return sizeof(float) * 3 * (size_t)D * (size_t)wide_tiles(N) * wide::kP; }

cudaError_t launch_sweep_wide(const DevTarget& t, int move, const SweepParams& sp, cudaStream_t s)
{
    wide::Args A = wide::make_args(t);
    A.sp = sp;
    A.tiles = wide_tiles(sp.N);
    A.Np = (int64_t)A.tiles * wide::kP;
    A.xs = t.wide_state;
    A.gs = A.xs + (size_t)t.D * A.Np;
    A.ms = A.gs + (size_t)t.D * A.Np;
    A.N = sp.N;
    return wide::dispatch(A, t.D, t.kind == kLogreg, move, false, s);
}

cudaError_t launch_potential_wide(const DevTarget& t, const float* x, int64_t N, double* ell, float* grad,
                                  cudaStream_t s)
{
    wide::Args A = wide::make_args(t);
    A.x_in = x;
    A.ell_pot = ell;
    A.grad_pot = grad;
    A.pstride = N;
    A.N = N;
    return wide::dispatch(A, t.D, t.kind == kLogreg, kRwmh, true, s);
}

} // namespace oais
