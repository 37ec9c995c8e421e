// sweep_tcs.cuh -- device code of the streamed tensor-core sweep (see sweep_tcs.cu for the
// design); shared by the single-problem kernels (sweep_tcs.cu) and the batched kernel
// (sweep_tcs_batch.cu), compiled as two translation units.
#pragma once
#include <cuda_fp16.h>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tcgen05.cuh"
#include "../../include/oais.h"

namespace oais {
namespace tcs {
using namespace oais::tc;

constexpr int kTile = 128;
// Role layout for a column split H (2 or 4): 4 H particle warps (four lane quarters times H
// column groups), then the forward issuer, the producer, the backward issuer and (FP8
// storage) the converter warp.
template <int H>
struct Roles {
    static constexpr int kEpiWarps = 4 * H;
    static constexpr int kEpiThreads = 32 * kEpiWarps;
    static constexpr int kFwdWarp = kEpiWarps, kLoadWarp = kEpiWarps + 1, kBwdWarp = kEpiWarps + 2;
    static constexpr int kCvtWarp0 = kEpiWarps + 3;
    static constexpr int threads(int q8) { return kEpiThreads + 96 + (q8 ? 32 : 0); }
};
constexpr int kMaxH = 4;
// FP8 storage of X (e4m3 values q with a per-row scale s, X~ = s q): two warps expand each
// chunk from the FP8 ring into the f16 stage the MMAs read, one row per thread: the producer
// warp (whose lane 0 also issues the copies) and one more warp (a 12-warp block keeps the
// register budget of the other roles)
constexpr int kCvtArrivals = 2;
constexpr int kSlice = 8;   // coordinates per state-update step (one 16-byte f16 chunk)
// The tensor core rounds each accumulation toward zero, so a long running sum in one TMEM
// accumulator drifts toward zero by about half an ulp per MMA (a relative shrink of ~1e-4
// after the ~6000 backward MMAs of a 50 000-row evaluation).  The gradient sum is therefore
// cut into segments of kSegMmas MMAs (relative drift ~1e-5): at the end of a segment the
// particle threads add D2 into an fp32 sum in memory (round to nearest) and the next
// segment restarts D2.
constexpr int kSegMmas = 512;

// ---------------------------------------------------------------------------------------
// K-major operand layout in shared memory: rows of `kw` 16-bit elements (kw = 64 with the
// 128-byte swizzle when the K extent is a multiple of 64, else 32 / 16 with the 64 / 32-byte
// swizzle); K beyond 64 is split into slabs of `rows` lines each.  The swizzle permutes the
// 16-byte chunks of a line by the line index (bits 4-6 of the address XOR bits 7-9 for
// 128B, bits 4-5 XOR 7-8 for 64B, bit 4 XOR bit 7 for 32B).  The same bytes read as an
// MN-major operand (N along the line) give the backward's B.
// ---------------------------------------------------------------------------------------
struct KLayout {
    int kw;      // elements per line
    int lb;      // bytes per line
    int mode;    // 0: 128B, 1: 64B, 2: 32B swizzle
};
__host__ __device__ constexpr KLayout klayout(int k_extent)
{
    return KLayout{k_extent >= 64 ? 64 : k_extent, 2 * (k_extent >= 64 ? 64 : k_extent),
                   k_extent >= 64 ? 0 : (k_extent == 32 ? 1 : 2)};
}
// rows per chunk: 64, or 32 when d_pad = 256 (shared memory)
#ifndef OAIS_TCS_CHUNK256
#define OAIS_TCS_CHUNK256 64
#endif
__host__ __device__ constexpr int chunk_rows(int dp) { return dp >= 256 ? OAIS_TCS_CHUNK256 : 64; }
// TMEM columns: NB forward accumulators D1 (one chunk each), NB per-row factor buffers R
// (hi | lo, f16 pairs), A_lo (the lo term of the positions, f16 pairs: the forward's A
// operand for that term), D2 (gradient accumulator, d_pad columns).  The hi term of the
// positions is the shared-memory A operand.  Two buffers (the forward of the next chunk runs
// while the particle warps work on this one) wherever the 512 columns allow: 64-row chunks up
// to d_pad = 128, 32-row chunks at 256; 128-row chunks take one.
template <int DP, int CHR = chunk_rows(DP)>
struct Cols {
    // two buffers of D1 and R wherever the 512 columns hold them with A_lo and D2
    static constexpr int NB = ((4 * CHR + DP / 2 + 31) / 32 * 32 + DP <= 512) ? 2 : 1;
    static constexpr int CH = CHR;
    static constexpr int D1 = 0, R = NB * CH, ALO = 2 * NB * CH;
    static constexpr int D2 = (ALO + DP / 2 + 31) / 32 * 32;
    static_assert(D2 + DP <= 512, "TMEM columns");
};
// byte offset of the 16-byte chunk holding elements [k0, k0 + 8) of `row`
__host__ __device__ inline uint32_t kmaj_off(int row, int k0, int rows, const KLayout& L)
{
    const int slab = k0 / L.kw;
    const int line = slab * rows + row;
    const int c = (k0 % L.kw) >> 3;
    const int sw = L.mode == 0 ? (line & 7) : (L.mode == 1 ? ((line >> 1) & 3) : ((line >> 2) & 1));
    return (uint32_t)line * (uint32_t)L.lb + (uint32_t)((c ^ sw) << 4);
}
__host__ __device__ constexpr uint64_t layout_code(const KLayout& L)
{
    return L.mode == 0 ? kSW128 : (L.mode == 1 ? kSW64 : kSW32);
}

struct Params {
    SweepParams sp;
    const unsigned char* img;   // [nch][stage_bytes] chunk images
    float* xa;                  // accepted positions    [dp][Np]
    float* ga;                  // grad log L at xa      [dp][Np]
    float* xp;                  // proposal / trajectory [dp][Np]
    float* mom;                 // HMC momentum; MALA: z + (eps/2) grad log pi(x)  [dp][Np]
    float* gs;                  // drained part of the running gradient sum G      [dp][Np]
    int64_t Np;
    int seg;                    // chunks per gradient segment (see kSegMmas)
    int n, d, dp, nch, stages;
    int chunk;                  // rows per chunk (the batched launch dispatches on it)
    uint32_t stage_bytes, y_off;   // f16 stage: lines, then y [64] and (FP8 storage) s [64]
    uint32_t off_x8, stage8_bytes; // FP8 storage: ring of chunk images (q rows, y, s)
    int stages8;
    uint32_t off_x, off_misc;   // shared-memory regions (A starts at 0)
    uint32_t tmem_cols;
    int move, leapfrog;
    // potential mode (one evaluation at given states, no sweep): x_in [d][N], outputs
    // ell_pot [N] and grad_pot [d][N] (may be null)
    const float* x_in;
    double* ell_pot;
    float* grad_pot;
    int64_t pstride;            // row stride of x_in and grad_pot
    // step range: steps t_begin..t_end of the schedule; resume = 0 starts from x_0 ~ eta (the
    // OAIS sweep: 1..T), resume = 1 continues from the stored state, log w and log L (one ASMC
    // step) and writes each tile's (log w, 2 log w) moment record to ess_parts
    int t_begin, t_end, resume;
    StepPartial* ess_parts;
    // persistent wrap-around schedule of the OAIS sweep (span > 0): CTA b runs the positions
    // [b span, (b + 1) span) of the tiles x steps sequence; handed[tile] flags a split tile's
    // first part done (0: one tile per CTA, the whole sweep)
    int64_t span;
    int tiles;
    int* handed;
    double log_norm;            // linear regression: n (log sigma + log(2 pi) / 2)
    float gscale;               // grad log L = gscale * G (1 / sigma^2 or 1)
    float half_inv_var;         // linear regression: 1 / (2 sigma^2)
};

// misc region: barriers, TMEM address, abort flag, exchange buffers, moment scratch
struct Misc {
    uint64_t xfull[8], xempty[8];
    uint64_t x8full[4], x8empty[4];
    uint64_t d1full[2], d1empty[2], rfull[2], rempty[2];
    uint64_t afull, d2full, done, d2seg, d2drained;
    uint32_t tmem;
    volatile int abort;
    double xl[kMaxH][kTile];    // per column group: partial log-likelihood
    float4 xm[kMaxH][kTile];    // per coordinate group: partial sums of the MH ratio
    double s_m[2][4][3];
    float s_s[2][4][8];                // warp pieces with deferred shifts (warp_moment_partial<true>)
    unsigned s_acc[2][4];
    Params prm;                 // batched launch: the current item's problem
    uint32_t item;              // batched launch: the current item
};

// f16 two-term split of a pair: hi = f16(v), lo = f16(v - hi) (one packed subtraction)
__device__ __forceinline__ void split_pair_h(float a, float b, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(a, b);
    const float2 d = sub_f32x2(make_float2(a, b), __half22float2(h));
    const __half2 l = __floats2half2_rn(d.x, d.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void normals8(const Rng& rng, uint32_t n, uint32_t t, uint32_t k, int d, int i0,
                                         float (&z)[kSlice])
{
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int j = i0 / 4 + b;
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (4 * j < d) box_muller4_sfu(rng.block(n, t, k, (uint32_t)j), v);
#pragma unroll
        for (int q = 0; q < 4; ++q) z[4 * b + q] = (4 * j + q < d) ? v[q] : 0.0f;
    }
}

template <int DP, int H, int CHR = chunk_rows(DP)>
struct Thread {
    static constexpr int CHUNK = CHR;
    using C = Cols<DP, CHR>;
    static constexpr int HC = CHUNK / H;   // columns of a chunk per thread
    static constexpr int DH = DP / H;      // coordinates per thread
    static constexpr int kEpi = Roles<H>::kEpiThreads;
    static_assert(DH >= 8 && HC >= 16, "a thread owns at least one 8-coordinate slice and 16 columns");
    unsigned char* smem;
    Misc* M;
    const Params* P;
    int p, h, q, lane;
    uint32_t lane_off;
    uint32_t tmem;  // TMEM base (lane 0, column 0)
    uint32_t d2;
    uint32_t g;     // chunks consumed
    uint32_t e;     // evaluations done
    int xs;         // stage of chunk g
    uint32_t xph;   // phase of that stage
    uint32_t sph;   // phase of the segment barrier
    bool drained;   // the last evaluation drained D2 at least once
    float* GS;      // this particle's drained gradient sum (stride Np)

    __device__ bool wait(uint64_t* bar, uint32_t parity)
    {
        if (M->abort) return false;
        if (mbar_wait(saddr(bar), parity, &M->abort)) return true;
        M->abort = 1;
        atomicOr(P->sp.status, 2u);
        return false;
    }

    // one 8-coordinate slice of the tile's positions, times `scale`, into the A operand (both
    // terms); the logistic family passes log2(e), so that the forward gives the margins in
    // base-2 units
    __device__ void write_a(int i0, const float (&v)[kSlice], float scale)
    {
        constexpr KLayout L = klayout(DP);
        const uint32_t off = kmaj_off(p, i0, kTile, L);
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split_pair_h(scale * v[2 * j], scale * v[2 * j + 1], hi[j], lo[j]);
        *reinterpret_cast<uint4*>(smem + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        tmem_st4(tmem + (uint32_t)(C::ALO + i0 / 2) + lane_off, lo);
    }

    __device__ void load_grad(int i0, float (&gv)[kSlice])
    {
        uint32_t v[8];
        tmem_ld8(d2 + lane_off + (uint32_t)i0, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < kSlice; ++j) {
            float gsum = __uint_as_float(v[j]);
            if (drained) gsum += GS[(int64_t)(i0 + j) * P->Np];
            gv[j] = P->gscale * gsum;
        }
    }

    // end of a gradient segment: add D2 (this thread's lanes and coordinate half) into GS,
    // W columns at a time with all W memory reads in flight together
    __device__ void drain(bool first)
    {
        wait(&M->d2seg, sph);
        sph ^= 1u;
        __syncwarp();
        tc_after_sync();
        constexpr int W = DH < 32 ? DH : 32;
        for (int i0 = h * DH; i0 < (h + 1) * DH; i0 += W) {
            uint32_t v[W];
            if constexpr (W == 32) tmem_ld32(d2 + lane_off + (uint32_t)i0, v);
            else if constexpr (W == 16) tmem_ld16(d2 + lane_off + (uint32_t)i0, v);
            else tmem_ld8(d2 + lane_off + (uint32_t)i0, v);
            float old[W];
#pragma unroll
            for (int j = 0; j < W; ++j) old[j] = first ? 0.0f : GS[(int64_t)(i0 + j) * P->Np];
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < W; ++j) GS[(int64_t)(i0 + j) * P->Np] = old[j] + __uint_as_float(v[j]);
        }
        tc_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(saddr(&M->d2drained));
    }

    // log L at the positions just written to A (this thread's half of the rows' terms summed
    // with the other half's), leaving grad log L / gscale in D2.
    template <int FAM, int Q8>
    __device__ double eval()
    {
        tmem_wait_st();   // A_lo in TMEM
        fence_proxy_async();   // A_hi in shared memory, visible to the tensor core
        tc_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(saddr(&M->afull));
        const int nch = P->nch;
        double acc0 = 0.0, acc1 = 0.0;   // linear: sum r^2; logistic: sum (u - |u|), sum log2 q
        float mid0 = 0.0f, mid1 = 0.0f;
        const int seg = P->seg;
        drained = false;
        for (int c = 0; c < nch; ++c, ++g) {
            constexpr int NB = C::NB;
            const int b = NB == 2 ? (int)(g & 1u) : 0;
            const uint32_t ph = NB == 2 ? (g >> 1) & 1u : g & 1u;   // use count of buffer b
            wait(&M->d1full[b], ph);
            __syncwarp();
            tc_after_sync();
            uint32_t v[HC];
            const uint32_t src = tmem + (uint32_t)(C::D1 + b * CHUNK + h * HC) + lane_off;
            if constexpr (HC == 16) {
                tmem_ld16(src, v);
            } else if constexpr (HC == 32) {
                tmem_ld32(src, v);
            } else {
                static_assert(HC == 64, "columns per thread");
                tmem_ld32(src, *reinterpret_cast<uint32_t(*)[32]>(v));
                tmem_ld32(src + 32, *reinterpret_cast<uint32_t(*)[32]>(v + 32));
            }
            tmem_wait_ld();
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&M->d1empty[b]));
            uint32_t hi[HC / 2], lo[HC / 2];
            float part0 = 0.0f, part1 = 0.0f;
            if constexpr (FAM == kLinreg) {
                wait(&M->xfull[xs], xph);   // y of this chunk is in the stage
                const float* ys = reinterpret_cast<const float*>(smem + P->off_x + (uint32_t)xs * P->stage_bytes +
                                                                 P->y_off) + h * HC;
                if constexpr (Q8) {
                    // X~_r = s_r q_r: z = s_r (q_r . x), and the backward's factor is r s_r
                    const float* ss = ys + CHUNK;
#pragma unroll
                    for (int j = 0; j < HC; j += 2) {
                        const float r0 = fmaf(-ss[j], __uint_as_float(v[j]), ys[j]);
                        const float r1 = fmaf(-ss[j + 1], __uint_as_float(v[j + 1]), ys[j + 1]);
                        part0 = fmaf(r0, r0, part0);
                        part0 = fmaf(r1, r1, part0);
                        split_pair_h(r0 * ss[j], r1 * ss[j + 1], hi[j / 2], lo[j / 2]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < HC; j += 2) {
                        const float r0 = ys[j] - __uint_as_float(v[j]);
                        const float r1 = ys[j + 1] - __uint_as_float(v[j + 1]);
                        part0 = fmaf(r0, r0, part0);
                        part0 = fmaf(r1, r1, part0);
                        split_pair_h(r0, r1, hi[j / 2], lo[j / 2]);
                    }
                }
            } else {
                // X'_r = s_r X~_r with s_r = 2 y_r - 1 and the A operand log2(e) x, so u is the
                // margin s z in base-2 units: log sigmoid(s z) = ln 2 (min(u, 0) + log2 q) with
                // q = 1 / (1 + 2^-|u|), d/dz = s sigmoid(-s z) = s (u >= 0 ? 2^-|u| q : q).  The rows
                // of a pair go through the packed fp32 pair instructions; the product of q is kept
                // per lane of the pair (HC / 2 <= 32 values in [1/2, 1] each), one log per chunk.
                const float2 one2 = make_float2(1.0f, 1.0f);
                float2 prod = one2, mn = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int j = 0; j < HC; j += 2) {
                    const float ua = __uint_as_float(v[j]), ub = __uint_as_float(v[j + 1]);
                    const float2 ee = make_float2(ex2_approx(-fabsf(ua)), ex2_approx(-fabsf(ub)));
                    const float2 dq = add_f32x2(ee, one2);
                    const float2 q = make_float2(rcp_approx(dq.x), rcp_approx(dq.y));
                    const float2 eq = mul_f32x2(ee, q);
                    mn = add_f32x2(mn, make_float2(fminf(ua, 0.0f), fminf(ub, 0.0f)));
                    prod = mul_f32x2(prod, q);
                    split_pair_h(ua >= 0.0f ? eq.x : q.x, ub >= 0.0f ? eq.y : q.y, hi[j / 2], lo[j / 2]);
                }
                part0 = mn.x + mn.y;
                part1 = lg2_approx(prod.x * prod.y);
            }
            if (++xs == P->stages) { xs = 0; xph ^= 1u; }
            // R (two f16 terms) into TMEM, the A operand of the backward
            wait(&M->rempty[b], ph ^ 1u);
            __syncwarp();
            tc_after_sync();
            const uint32_t rcol = tmem + (uint32_t)(C::R + b * CHUNK + h * (HC / 2)) + lane_off;
            if constexpr (HC == 64) {
                tmem_st16(rcol, *reinterpret_cast<const uint32_t(*)[16]>(hi));
                tmem_st16(rcol + 16, *reinterpret_cast<const uint32_t(*)[16]>(hi + 16));
                tmem_st16(rcol + CHUNK / 2, *reinterpret_cast<const uint32_t(*)[16]>(lo));
                tmem_st16(rcol + CHUNK / 2 + 16, *reinterpret_cast<const uint32_t(*)[16]>(lo + 16));
            } else if constexpr (HC == 32) {
                tmem_st16(rcol, hi);
                tmem_st16(rcol + CHUNK / 2, lo);
            } else {
                tmem_st8(rcol, hi);
                tmem_st8(rcol + CHUNK / 2, lo);
            }
            tmem_wait_st();
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(saddr(&M->rfull[b]));
            // chunk c - 1 closed a gradient segment: its backward is the last of the segment
            if (c >= 1 && (c - 1) % seg == seg - 1) {
                drain(!drained);
                drained = true;
            }
            mid0 += part0;
            mid1 += part1;
            if ((c & 15) == 15) { acc0 += mid0; acc1 += mid1; mid0 = 0.0f; mid1 = 0.0f; }
        }
        acc0 += mid0;
        acc1 += mid1;
        wait(&M->d2full, e & 1u);
        __syncwarp();
        tc_after_sync();
        ++e;
        double part;
        if constexpr (FAM == kLinreg) part = -P->half_inv_var * acc0;
        else part = 0.69314718055994531 * ((double)acc0 + (double)acc1);
        M->xl[h][p] = part;
        named_sync(1, kEpi);
        double tot = M->xl[0][p];
#pragma unroll
        for (int k = 1; k < H; ++k) tot += M->xl[k][p];
        named_sync(1, kEpi);
        if constexpr (FAM == kLinreg) return tot - P->log_norm;
        else return tot + (double)(nch * CHUNK - P->n) * 0.69314718055994531;
    }

    // sum of this particle's four partial sums over the two coordinate halves
    __device__ float4 combine(float4 mine)
    {
        M->xm[h][p] = mine;
        named_sync(1, kEpi);
        float4 a = M->xm[0][p];
#pragma unroll
        for (int k = 1; k < H; ++k) {
            const float4 b = M->xm[k][p];
            a = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
        }
        named_sync(1, kEpi);
        return a;
    }
};

__device__ __forceinline__ void mbar_inval(uint32_t bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// (thread 0) fresh barriers for one tile; prev_stages > 0: the previous tile's barriers (with
// that many stage pairs) are invalidated first
__device__ __forceinline__ void init_barriers(Misc* M, int stages, int prev_stages, int stages8, int epi_warps)
{
    uint64_t* all[] = {&M->d1full[0], &M->d1empty[0], &M->rfull[0], &M->rempty[0], &M->d1full[1], &M->d1empty[1],
                       &M->rfull[1], &M->rempty[1], &M->afull, &M->d2full, &M->done, &M->d2seg, &M->d2drained};
    if (prev_stages > 0) {
        for (int s = 0; s < prev_stages; ++s) { mbar_inval(saddr(&M->xfull[s])); mbar_inval(saddr(&M->xempty[s])); }
        for (int s = 0; s < stages8; ++s) { mbar_inval(saddr(&M->x8full[s])); mbar_inval(saddr(&M->x8empty[s])); }
        for (uint64_t* b : all) mbar_inval(saddr(b));
    }
    // f16 stages are filled by the bulk copy (one arrival + bytes) or, with FP8 storage, by
    // the two converter warps
    for (int s = 0; s < stages; ++s) {
        mbar_init(saddr(&M->xfull[s]), stages8 > 0 ? kCvtArrivals : 1);
        mbar_init(saddr(&M->xempty[s]), 1);
    }
    for (int s = 0; s < stages8; ++s) {
        mbar_init(saddr(&M->x8full[s]), 1);
        mbar_init(saddr(&M->x8empty[s]), kCvtArrivals);
    }
    for (int b = 0; b < 2; ++b) {
        mbar_init(saddr(&M->d1full[b]), 1);
        mbar_init(saddr(&M->d1empty[b]), epi_warps);
        mbar_init(saddr(&M->rfull[b]), epi_warps);
        mbar_init(saddr(&M->rempty[b]), 1);
    }
    mbar_init(saddr(&M->afull), epi_warps);
    mbar_init(saddr(&M->d2full), 1);
    mbar_init(saddr(&M->done), 2);
    mbar_init(saddr(&M->d2seg), 1);
    mbar_init(saddr(&M->d2drained), epi_warps);
    M->abort = 0;
    fence_mbar_init();
}

// One tile (128 particles) of one problem for a whole sweep, by all 352 threads of the CTA;
// the barriers are fresh and TMEM (512 columns at `tmem`) is held by the caller.
// FP8 -> f16 stage: row `row` of a chunk (q bytes to the swizzled f16 lines), its y and s
template <int DP, int CHR = chunk_rows(DP)>
__device__ __forceinline__ void convert_row(const unsigned char* src, unsigned char* dst, int row, uint32_t y_off)
{
    constexpr int CHUNK = CHR;
    constexpr KLayout LA = klayout(DP);
    const unsigned char* qrow = src + (uint32_t)row * DP;
#pragma unroll 4
    for (int k0 = 0; k0 < DP; k0 += 16) {
        const uint4 raw = *reinterpret_cast<const uint4*>(qrow + k0);
        const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
        uint32_t hv[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            hv[2 * i] = cvt_f16x2_e4m3x2((uint16_t)(w[i] & 0xFFFFu));
            hv[2 * i + 1] = cvt_f16x2_e4m3x2((uint16_t)(w[i] >> 16));
        }
        *reinterpret_cast<uint4*>(dst + kmaj_off(row, k0, CHUNK, LA)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(dst + kmaj_off(row, k0 + 8, CHUNK, LA)) = make_uint4(hv[4], hv[5], hv[6], hv[7]);
    }
    const float* yq = reinterpret_cast<const float*>(src + (uint32_t)CHUNK * DP);
    float* yd = reinterpret_cast<float*>(dst + y_off);
    yd[row] = yq[row];
    yd[CHUNK + row] = yq[CHUNK + row];
}

template <int FAM, int DP, int Q8, int H, int CHR = chunk_rows(DP)>
__device__ __forceinline__ void run_tile(const Params& P, uint32_t tile, uint32_t tiles, unsigned char* smem,
                                         uint32_t tmem)
{
    constexpr int CHUNK = CHR;
    using C = Cols<DP, CHR>;
    constexpr float kAScale = FAM == kLogreg ? 1.4426950408889634f : 1.0f;   // A operand scale
    const SweepParams& S = P.sp;
    Misc* M = reinterpret_cast<Misc*>(smem + P.off_misc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Le = P.move == kHmc ? P.leapfrog : 1;
    const uint32_t nsteps = P.t_end >= P.t_begin ? (uint32_t)(P.t_end - P.t_begin + 1) : 0u;
    const uint32_t evals = P.x_in ? 1u : (P.resume ? 0u : 1u) + nsteps * (uint32_t)S.mv.K * (uint32_t)Le;
    const uint32_t total = evals * (uint32_t)P.nch;
    const uint32_t D2 = tmem + (uint32_t)C::D2;
    constexpr int NB = C::NB;
    constexpr KLayout LA = klayout(DP);
    constexpr int kFwdWarp = Roles<H>::kFwdWarp, kLoadWarp = Roles<H>::kLoadWarp, kBwdWarp = Roles<H>::kBwdWarp;
    constexpr int kCvtWarp0 = Roles<H>::kCvtWarp0;

    if (Q8 && warp == kLoadWarp) {
        // ---------------- producer + converter (rows 0-31) ----------------
        // lane 0 keeps the FP8 ring full: it issues every copy whose ring slot is free, from
        // inside the warp's waits, so the warp never blocks on a copy nobody has issued
        uint32_t issued = 0, c = 0, pph = 0;
        int ps = 0;
        const uint32_t bytes8 = P.stage8_bytes;
        const uint32_t base8 = saddr(smem + P.off_x8);
        auto try_issue = [&]() {
            while (issued < total && mbar_try_wait(saddr(&M->x8empty[ps]), pph ^ 1u)) {
                mbar_arrive_expect_tx(saddr(&M->x8full[ps]), bytes8);
                bulk_g2s(base8 + (uint32_t)ps * bytes8, P.img + (size_t)c * bytes8, bytes8, saddr(&M->x8full[ps]));
                ++issued;
                if (++c == (uint32_t)P.nch) c = 0;
                if (++ps == P.stages8) { ps = 0; pph ^= 1u; }
            }
        };
        auto wait_issuing = [&](uint32_t bar, uint32_t parity) -> bool {
            const uint64_t t0 = globaltimer();
            for (;;) {
                if (lane == 0) try_issue();
                if (mbar_try_wait(bar, parity)) return true;
                if (M->abort || globaltimer() - t0 > kWaitLimitNs) return false;
            }
        };
        int s8 = 0, s = 0;
        uint32_t ph8 = 0, ph = 0;
        for (uint32_t g = 0; g < total; ++g) {
            if (!wait_issuing(saddr(&M->x8full[s8]), ph8) || !wait_issuing(saddr(&M->xempty[s]), ph ^ 1u)) {
                M->abort = 1;
                atomicOr(S.status, 2u);
                break;
            }
            if (lane < CHUNK)
                convert_row<DP, CHR>(smem + P.off_x8 + (uint32_t)s8 * P.stage8_bytes,
                                     smem + P.off_x + (uint32_t)s * P.stage_bytes, lane, P.y_off);
            fence_proxy_async();   // the f16 stage, visible to the tensor core
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(saddr(&M->xfull[s]));
                mbar_arrive(saddr(&M->x8empty[s8]));
                try_issue();
            }
            if (++s8 == P.stages8) { s8 = 0; ph8 ^= 1u; }
            if (++s == P.stages) { s = 0; ph ^= 1u; }
        }
        // copies still in flight land before the CTA ends (bounded)
        if (lane == 0) {
            const uint32_t first = issued > (uint32_t)P.stages8 ? issued - P.stages8 : 0u;
            for (uint32_t g = first; g < issued; ++g)
                mbar_wait(saddr(&M->x8full[g % P.stages8]), (g / P.stages8) & 1u);
        }
    } else if (warp == kLoadWarp) {
        // ---------------- producer: chunk images into the stage ring ----------------
        if (lane == 0) {
            const int ring = P.stages;
            const uint32_t bytes = P.stage_bytes;
            uint64_t* full = M->xfull;
            uint64_t* empty = M->xempty;
            int s = 0;
            uint32_t ph = 0, issued = 0;
            const uint32_t sbase = saddr(smem + P.off_x);
            for (uint32_t g = 0, c = 0; g < total; ++g) {
                if (M->abort) break;
                if (!mbar_wait(saddr(&empty[s]), ph ^ 1u, &M->abort)) {
                    M->abort = 1;
                    atomicOr(S.status, 2u);
                    break;
                }
                mbar_arrive_expect_tx(saddr(&full[s]), bytes);
                bulk_g2s(sbase + (uint32_t)s * bytes, P.img + (size_t)c * bytes, bytes, saddr(&full[s]));
                ++issued;
                if (++c == (uint32_t)P.nch) c = 0;
                if (++s == ring) { s = 0; ph ^= 1u; }
            }
            // copies still in flight land before the CTA ends (bounded)
            const uint32_t first = issued > (uint32_t)ring ? issued - ring : 0u;
            for (uint32_t g = first; g < issued; ++g) mbar_wait(saddr(&full[g % ring]), (g / ring) & 1u);
        }
    } else if (Q8 && warp >= kCvtWarp0) {
        // ---------------- converter: FP8 chunk -> f16 stage (rows 32-63) ----------------
        int s8 = 0, s = 0;
        uint32_t ph8 = 0, ph = 0;
        for (uint32_t g = 0; g < total; ++g) {
            if (!mbar_wait(saddr(&M->x8full[s8]), ph8, &M->abort) ||
                !mbar_wait(saddr(&M->xempty[s]), ph ^ 1u, &M->abort)) {
                M->abort = 1;
                atomicOr(S.status, 2u);
                break;
            }
            if (32 + lane < CHUNK)   // chunks of 32 rows: the producer warp converts them all
                convert_row<DP, CHR>(smem + P.off_x8 + (uint32_t)s8 * P.stage8_bytes,
                                     smem + P.off_x + (uint32_t)s * P.stage_bytes, 32 + lane, P.y_off);
            fence_proxy_async();   // the f16 stage, visible to the tensor core
            __syncwarp();
            if ((threadIdx.x & 31) == 0) {
                mbar_arrive(saddr(&M->xfull[s]));
                mbar_arrive(saddr(&M->x8empty[s8]));
            }
            if (++s8 == P.stages8) { s8 = 0; ph8 ^= 1u; }
            if (++s == P.stages) { s = 0; ph ^= 1u; }
        }
    } else if (warp == kFwdWarp || warp == kBwdWarp) {
        // ---------------- MMA issue: forwards and backwards from two threads ----------------
        // Each stream is issued in chunk order as soon as its inputs are ready; a commit
        // tracks only its own thread's MMAs, and every buffer the two streams share is
        // ordered through the particle warps' barriers (a backward of chunk g follows the
        // particle warps' read of that chunk's forward result).
        if (lane == 0) {
            constexpr uint32_t idf = idesc_kind_f16(kTile, CHUNK, false, false);
            constexpr uint32_t idb = idesc_kind_f16(kTile, DP, false, true);
            constexpr uint64_t ca = layout_code(LA);
            const uint32_t xbase = saddr(smem + P.off_x);
            const int nch = P.nch, seg = P.seg, S_ = P.stages;
            bool ok = true;
            int s = 0;
            uint32_t ph = 0;
            if (warp == kFwdWarp) {
                // forward g: its X stage loaded, its D1 buffer read by the particle warps and,
                // for the first chunk of an evaluation, the new positions in A.  The
                // descriptors of the A bases take constant offsets (16-byte units) per K step.
                const uint64_t adesc = sdesc(saddr(smem), 16, 8 * LA.lb, ca);
                const uint32_t alo = tmem + (uint32_t)C::ALO;
                for (uint32_t g = 0, c = 0, e = 0; g < total; ++g) {
                    if ((c == 0 && !mbar_wait(saddr(&M->afull), e & 1u, &M->abort)) ||
                        !mbar_wait(saddr(&M->xfull[s]), ph, &M->abort) ||
                        !mbar_wait(saddr(&M->d1empty[NB == 2 ? g & 1u : 0u]), (NB == 2 ? (g >> 1) & 1u : g & 1u) ^ 1u,
                                   &M->abort)) { ok = false; break; }
                    const int b = NB == 2 ? (int)(g & 1u) : 0;
                    const uint32_t d1 = tmem + (uint32_t)(C::D1 + b * CHUNK);
                    tc_after_sync();
                    const uint64_t xd = sdesc(xbase + (uint32_t)s * P.stage_bytes, 16, 8 * LA.lb, ca);
                    // the small (lo) term first, from TMEM: the running sum is small while it
                    // accumulates, so only the hi term's steps round a large sum toward zero
#pragma unroll
                    for (int kk = 0; kk < DP / 16; ++kk) {
                        constexpr int kw = LA.kw;
                        const int slab = 16 * kk / kw, within = (16 * kk % kw) * 2;
                        mma_f16_ts(d1, alo + (uint32_t)(kk * 8), xd + (uint64_t)((slab * CHUNK * LA.lb + within) / 16),
                                   idf, kk == 0 ? 0u : 1u);
                    }
#pragma unroll
                    for (int kk = 0; kk < DP / 16; ++kk) {
                        constexpr int kw = LA.kw;
                        const int slab = 16 * kk / kw, within = (16 * kk % kw) * 2;
                        mma_f16(d1, adesc + (uint64_t)((slab * kTile * LA.lb + within) / 16),
                                xd + (uint64_t)((slab * CHUNK * LA.lb + within) / 16), idf, 1u);
                    }
                    mma_commit(saddr(&M->d1full[b]));
                    if (++s == S_) { s = 0; ph ^= 1u; }
                    if (++c == (uint32_t)nch) { c = 0; ++e; }
                }
            } else {
                // backward g: R of chunk g in TMEM and, for the first chunk of a gradient
                // segment, the previous segment drained
                uint32_t dph = 0;
                for (uint32_t g = 0, c = 0; g < total; ++g) {
                    const bool first = c % (uint32_t)seg == 0;
                    const int b = NB == 2 ? (int)(g & 1u) : 0;
                    if (!mbar_wait(saddr(&M->rfull[b]), NB == 2 ? (g >> 1) & 1u : g & 1u, &M->abort) ||
                        !mbar_wait(saddr(&M->xfull[s]), ph, &M->abort) ||
                        (first && c != 0 && !mbar_wait(saddr(&M->d2drained), dph, &M->abort))) { ok = false; break; }
                    if (first && c != 0) dph ^= 1u;
                    tc_after_sync();
                    const uint64_t xd = sdesc(xbase + (uint32_t)s * P.stage_bytes, CHUNK * LA.lb, 8 * LA.lb, ca);
                    const uint32_t ra = tmem + (uint32_t)(C::R + b * CHUNK);
#pragma unroll
                    for (int term = 0; term < 2; ++term) {
#pragma unroll
                        for (int kk = 0; kk < CHUNK / 16; ++kk)
                            mma_f16_ts(D2, ra + (uint32_t)(term * (CHUNK / 2) + kk * 8),
                                       xd + (uint64_t)(kk * 16 * LA.lb / 16), idb,
                                       (first && term == 0 && kk == 0) ? 0u : 1u);
                    }
                    mma_commit(saddr(&M->rempty[b]));
                    mma_commit(saddr(&M->xempty[s]));
                    if (c % (uint32_t)seg == (uint32_t)seg - 1 && c < (uint32_t)nch - 1) mma_commit(saddr(&M->d2seg));
                    if (c == (uint32_t)nch - 1) mma_commit(saddr(&M->d2full));
                    if (++s == S_) { s = 0; ph ^= 1u; }
                    if (++c == (uint32_t)nch) c = 0;
                }
            }
            if (!ok) { M->abort = 1; atomicOr(S.status, 2u); }
            // every MMA issued by either thread has completed before TMEM is released (bounded)
            mma_commit(saddr(&M->done));
            mbar_wait(saddr(&M->done), 0u);
        }
    } else {
        // ---------------- particle warps ----------------
        Thread<DP, H, CHR> Th;
        Th.smem = smem;
        Th.M = M;
        Th.P = &P;
        Th.q = warp & 3;
        Th.h = warp >> 2;
        Th.lane = lane;
        Th.p = 32 * Th.q + lane;
        Th.lane_off = (uint32_t)(Th.q * 32) << 16;
        Th.tmem = tmem;
        Th.d2 = D2;
        Th.g = 0;
        Th.e = 0;
        Th.xs = 0;
        Th.xph = 0;
        Th.sph = 0;
        Th.drained = false;
        const int p = Th.p, h = Th.h;
        const int64_t n64 = (int64_t)tile * kTile + p;
        const bool active = n64 < S.N;
        Th.GS = P.gs + n64;
        const uint32_t n = (uint32_t)(S.n_offset + (active ? n64 : S.N - 1));
        constexpr int dh = DP / H;
        const int c0 = h * dh;
        const int64_t Np = P.Np;
        const float sref = (float)S.ref_scale;
        const float inv_s2 = 1.0f / (sref * sref);
        float* XA = P.xa + n64;
        float* GA = P.ga + n64;
        float* XP = P.xp + n64;
        float* MO = P.mom + n64;

        if (P.x_in) {
            // potential mode: log L and grad log L at the given states
            const int64_t src = active ? n64 : S.N - 1;
            for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                float xv[kSlice];
#pragma unroll
                for (int j = 0; j < kSlice; ++j)
                    xv[j] = i0 + j < P.d ? P.x_in[(int64_t)(i0 + j) * P.pstride + src] : 0.0f;
                Th.write_a(i0, xv, kAScale);
            }
            const double ellv = Th.template eval<FAM, Q8>();
            for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                float gv[kSlice];
                Th.load_grad(i0, gv);
                if (active && P.grad_pot) {
#pragma unroll
                    for (int j = 0; j < kSlice; ++j)
                        if (i0 + j < P.d) P.grad_pot[(int64_t)(i0 + j) * P.pstride + n64] = gv[j];
                }
            }
            if (active && h == 0) P.ell_pot[n64] = ellv;
        } else {
        double ell, logw;
        if (!P.resume) {
            // x_0 ~ eta, its log L and gradient
            for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                float z[kSlice];
                normals8(S.mv.rng, n, 0u, 0u, P.d, i0, z);
#pragma unroll
                for (int j = 0; j < kSlice; ++j) {
                    z[j] *= sref;
                    XA[(int64_t)(i0 + j) * Np] = z[j];
                }
                Th.write_a(i0, z, kAScale);
            }
            ell = Th.template eval<FAM, Q8>();
            for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                float gv[kSlice];
                Th.load_grad(i0, gv);
#pragma unroll
                for (int j = 0; j < kSlice; ++j) GA[(int64_t)(i0 + j) * Np] = gv[j];
            }
            logw = 0.0;
        } else {
            // an ASMC step continues from the stored state (gathered after a resampling)
            const int64_t src = active ? n64 : S.N - 1;
            ell = S.ell_out[src];
            logw = S.logw[src];
        }
        double beta_prev = S.beta[P.t_begin - 1];
        for (int t = P.t_begin; t <= P.t_end; ++t) {
            const double beta_t = __ldg(S.beta + t);
            const double eps_t = __ldg(S.eps + t - 1);
            const double lg = (beta_t - beta_prev) * ell;
            beta_prev = beta_t;
            const int slot = t & 1;
            if (h == 0) warp_moment_partial<true>(logw, lg, active, M->s_m[slot][Th.q], M->s_s[slot][Th.q]);
            logw += lg;
            unsigned acc = 0;
            const float beta = (float)beta_t, eps = (float)eps_t, he = 0.5f * eps;
            for (int k = 0; k < S.mv.K; ++k) {
                // proposal start: MALA x' = x + eps (z + (eps/2) grad log pi(x));
                // HMC m = z + (eps/2) grad log pi(x), x' = x + eps m
                float zz = 0.0f, dxx = 0.0f;
                for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                    float z[kSlice], xpv[kSlice];
                    normals8(S.mv.rng, n, (uint32_t)t, (uint32_t)k, P.d, i0, z);
#pragma unroll
                    for (int j = 0; j < kSlice; ++j) {
                        const int64_t o = (int64_t)(i0 + j) * Np;
                        const float xv = XA[o], gv = GA[o];
                        const float gpi = -xv * inv_s2 + beta * gv;
                        const float m = z[j] + he * gpi;
                        xpv[j] = xv + eps * m;
                        zz += z[j] * z[j];
                        dxx += (xpv[j] - xv) * (xpv[j] + xv);
                        XP[o] = xpv[j];
                        MO[o] = m;
                    }
                    Th.write_a(i0, xpv, kAScale);
                }
                double ellp = 0.0;
                float tail = 0.0f;   // MALA: |reverse noise|^2; HMC: |final momentum|^2
                for (int l = 0; l < Le; ++l) {
                    ellp = Th.template eval<FAM, Q8>();
                    const bool last = l + 1 == Le;
                    if (P.move == kHmc) {
                        const float f = last ? he : eps;
                        dxx = last ? 0.0f : dxx;
                        for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                            float gv[kSlice], xpv[kSlice];
                            Th.load_grad(i0, gv);
#pragma unroll
                            for (int j = 0; j < kSlice; ++j) {
                                const int64_t o = (int64_t)(i0 + j) * Np;
                                const float xq = XP[o];
                                float m = MO[o] + f * (-xq * inv_s2 + beta * gv[j]);
                                if (!last) {
                                    xpv[j] = xq + eps * m;
                                    XP[o] = xpv[j];
                                    MO[o] = m;
                                } else {
                                    const float xv = XA[o];
                                    tail += m * m;
                                    dxx += (xq - xv) * (xq + xv);
                                    xpv[j] = xq;
                                }
                            }
                            if (!last) Th.write_a(i0, xpv, kAScale);
                        }
                    } else {
                        for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                            float gv[kSlice];
                            Th.load_grad(i0, gv);
#pragma unroll
                            for (int j = 0; j < kSlice; ++j) {
                                const int64_t o = (int64_t)(i0 + j) * Np;
                                const float qv = MO[o] + he * (-XP[o] * inv_s2 + beta * gv[j]);
                                tail += qv * qv;
                            }
                        }
                    }
                }
                const float4 tot = Th.combine(make_float4(zz, dxx, tail, 0.0f));
                // HMC: log alpha = [log pi(x') - |m'|^2/2] - [log pi(x) - |z|^2/2];
                // MALA: log alpha = log pi(x') - log pi(x) - (|q|^2 - |z|^2) / 2
                const float log_alpha =
                    -0.5f * tot.y * inv_s2 + beta * (float)(ellp - ell) - 0.5f * (tot.z - tot.x);
                const float logu = mh_log_uniform(S.mv.rng, n, (uint32_t)t, (uint32_t)k, 0.0f);
                const bool accept = logu < log_alpha;
                for (int i0 = c0; i0 < c0 + dh; i0 += kSlice) {
                    float gv[kSlice];
                    Th.load_grad(i0, gv);   // warp-collective: outside the branch
                    if (accept) {
#pragma unroll
                        for (int j = 0; j < kSlice; ++j) {
                            const int64_t o = (int64_t)(i0 + j) * Np;
                            XA[o] = XP[o];
                            GA[o] = gv[j];
                        }
                    }
                }
                if (accept) { ell = ellp; ++acc; }
            }
            if (h == 0) {
                acc = active ? acc : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
                if (lane == 0) M->s_acc[slot][Th.q] = acc;
                named_sync(2, 128);
                if (warp == 0)
                    merge_deferred_pieces<4>(lane, M->s_m[slot], M->s_s[slot], M->s_acc[slot],
                                         S.partials + (size_t)(t - 1) * tiles + tile);
            }
        }
        if (P.ess_parts && h == 0) {
            // (log w, 2 log w) moments of the tile for the ESS of the resampling test
            const int slot = (P.t_end + 1) & 1;
            warp_moment_partial<true>(logw, logw, active, M->s_m[slot][Th.q], M->s_s[slot][Th.q]);
            if (lane == 0) M->s_acc[slot][Th.q] = 0u;
            named_sync(2, 128);
            if (warp == 0) merge_deferred_pieces<4>(lane, M->s_m[slot], M->s_s[slot], M->s_acc[slot], P.ess_parts + tile);
        }
        if (active) {
            if (P.t_end == S.T) {
                float* xo = reinterpret_cast<float*>(S.x_out);
                for (int i = c0; i < c0 + dh && i < P.d; ++i) xo[(size_t)i * S.N + n64] = XA[(int64_t)i * Np];
            }
            if (h == 0) {
                S.logw[n64] = logw;
                S.ell_out[n64] = ell;
                if (!isfinite(logw) || !isfinite(ell)) atomicOr(S.status, 1u);
            }
        }
        }   // sweep
    }
}

template <int FAM, int DP, int Q8, int H>
__global__ void __launch_bounds__(Roles<H>::threads(Q8), 1)
oais_sweep_tcs_kernel(const Params P)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    if (saddr(smem) & 1023u) {
        if (threadIdx.x == 0) atomicOr(P.sp.status, 4u);
        return;
    }
    Misc* M = reinterpret_cast<Misc*>(smem + P.off_misc);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) init_barriers(M, P.stages, 0, Q8 ? P.stages8 : 0, Roles<H>::kEpiWarps);
    if (warp == 0) {
        tmem_alloc(saddr(&M->tmem), P.tmem_cols);
        tmem_relinquish();
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(&M->tmem);
    if (P.span == 0) {
        run_tile<FAM, DP, Q8, H>(P, blockIdx.x, gridDim.x, smem, tmem);
    } else {
        // Persistent grid, wrap-around schedule (McNaughton's rule for preemptive scheduling
        // of independent jobs): tile i is the job of T steps at positions [i T, (i + 1) T) of
        // the concatenated sequence, CTA b covers [b L, (b + 1) L) with L = span >= T.  A tile
        // split between CTAs b and b + 1 runs its first steps at the start of CTA b + 1 and its
        // last steps at the end of CTA b, which cannot overlap in time because L >= T; the
        // first part leaves the state where the resumed part reads it (positions, gradients,
        // log w, log L) and sets handed[tile], the last part waits for the flag (bounded).
        // Every piece starts on fresh barriers (TMEM stays allocated).
        Params& sP = M->prm;
        const int T = P.sp.T;
        const int64_t total = (int64_t)P.tiles * T;
        const int64_t pos1 = min(((int64_t)blockIdx.x + 1) * P.span, total);
        bool first = true;
        for (int64_t pos = (int64_t)blockIdx.x * P.span; pos < pos1 && T > 0;) {
            const int64_t tile = pos / T;
            const int off = (int)(pos % T);
            int t0, t1;
            if (off != 0) {                       // head: the first T - off steps of a split tile
                t0 = 1;
                t1 = T - off;
                pos = (tile + 1) * T;
            } else if (pos + T <= pos1) {         // a whole tile
                t0 = 1;
                t1 = T;
                pos += T;
            } else {                              // tail: the last pos1 - pos steps of a split tile
                t0 = T - (int)(pos1 - pos) + 1;
                t1 = T;
                pos = pos1;
            }
            if (threadIdx.x == 0) {
                if (!first) init_barriers(M, P.stages, P.stages, Q8 ? P.stages8 : 0, Roles<H>::kEpiWarps);
                sP = P;
                sP.t_begin = t0;
                sP.t_end = t1;
                sP.resume = t0 > 1 ? 1 : 0;
                if (t0 > 1) {
                    const uint64_t w0 = globaltimer();
                    const uint64_t limit = P.sp.handoff_wait_ns ? P.sp.handoff_wait_ns : kWaitLimitNs;
                    while (ld_acquire_gpu(P.handed + tile) == 0) {
                        if (globaltimer() - w0 > limit) {
                            M->abort = 1;
                            atomicOr(P.sp.status, 2u);
                            break;
                        }
                        __nanosleep(256);
                    }
                }
            }
            tc_before_sync();
            __syncthreads();
            tc_after_sync();
            if (M->abort) break;
            run_tile<FAM, DP, Q8, H>(sP, (uint32_t)tile, (uint32_t)P.tiles, smem, tmem);
            // every role has finished the piece (its copies and MMAs complete) before the
            // barriers are reused; the piece's state is written before the flag is raised
            tc_before_sync();
            __syncthreads();
            tc_after_sync();
            if (M->abort) break;
            if (t1 < T && threadIdx.x == 0 && !P.sp.withhold) {
                __threadfence();
                st_release_gpu(P.handed + tile, 1);
            }
            first = false;
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, P.tmem_cols);
}

} // namespace tcs
} // namespace oais
