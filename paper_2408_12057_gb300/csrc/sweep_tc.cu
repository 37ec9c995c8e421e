// sweep_tc.cu -- the loop-swapped OAIS sweep (Sec. 5.1.2) for the logistic-regression
// family with the likelihood contraction on the tensor cores (tcgen05, BF16 operands,
// FP32 accumulation in tensor memory).
//
// For a tile of 128 particles P (rows) and a chunk of 64 data rows X_c:
//   forward   Z   = P X_c^T          (M = 128 particles, N = 64 rows,  K = d = 32)
//   epilogue  f   = y z - softplus(z),  r = y - sigmoid(z)      (CUDA cores, per element)
//   backward  G  += R X_c            (M = 128 particles, N = d = 32, K = 64 rows)
// so log L(x) = sum f (kept in fp32 registers) and grad log L(x) = G (kept in TMEM)
// for every particle of the tile in one pass over X.  To keep the products at fp32
// accuracy the particle states and the residuals are split into two BF16 terms,
// v = hi + lo with hi a bf16 and lo = bf16(v - hi) (relative error below 2^-16), and each
// contraction is issued once per term.  The data X is rounded to BF16 once (X~); the
// sampler targets the posterior of X~.
//
// CTA = 2 independent groups of 8 particle warps plus one MMA warp each; group g owns 128
// particles, two threads per particle (each takes half the columns of every chunk and half
// the coordinates; they exchange partial sums through TMEM), its own TMEM columns, operand
// tiles and barriers, and shares the BF16 image of X (resident in shared memory for the whole
// sweep).  The group's MMA warp issues its tcgen05.mma instructions (one lane issues, the warp
// runs the loop), so the particle warps never wait on the issue of a contraction.
//
// Shared memory (dynamic, 1024-byte aligned base):
//   R tiles  [group][hi|lo]  128 x 64 bf16, K-major, 128B swizzle    4 x 16 KB
//   A tiles  [group][hi|lo]  128 x 32 bf16, K-major, 64B swizzle     4 x  8 KB
//   X image  2048 x 32 bf16, rows of 64 B, 64B swizzle              128 KB
//            (read as the K-major B of the forward and the MN-major B of the backward)
//   y bits   2048 labels as a bitmask                                256 B
//   6 mbarriers per group, the TMEM base address, the abort flag, per-group moment scratch
#include <cuda_bf16.h>
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tcgen05.cuh"
#include "../../include/oais.h"

namespace oais {
namespace tc {

constexpr int kGroups = 2;
constexpr int kTile = 128;                   // particles per group (the tcgen05 M = 128 lanes)
constexpr int kHalves = 2;                   // threads per particle: each takes half the columns
                                             // of a chunk and half the coordinates
constexpr int kGroupThreads = kTile * kHalves;
constexpr int kGroupWarps = kGroupThreads / 32;
constexpr int kMmaWarp0 = kGroups * kGroupWarps;         // group g's MMA warp: kMmaWarp0 + g
constexpr int kParticlesPerCta = kGroups * kTile;
constexpr int kThreads = kGroups * kGroupThreads + 32 * kGroups;
constexpr int kBarsPerGroup = 6;             // forward into D1[0], D1[1]; backward; R written; A written; end
constexpr int kD = 32;                       // padded state dimension
constexpr int kChunk = 64;                   // data rows per contraction chunk
constexpr int kHalfD = kD / kHalves;         // coordinates per thread
constexpr int kHalfCols = kChunk / kHalves;  // columns of a chunk per thread
constexpr int kMaxRows = 2048;
constexpr int kRTile = 128 * kChunk * 2;     // 16 KB
constexpr int kATile = 128 * kD * 2;         // 8 KB
constexpr int kOffR = 0;
constexpr int kOffA = kOffR + kGroups * 2 * kRTile;          // 64 KB
constexpr int kOffX = kOffA + kGroups * 2 * kATile;          // 96 KB
constexpr int kOffY = kOffX + kMaxRows * kD * 2;             // 224 KB
constexpr int kOffBar = kOffY + kMaxRows / 8;                // + 256 B
constexpr int kOffTmem = kOffBar + 8 * kBarsPerGroup * kGroups;
constexpr int kOffAbort = kOffTmem + 4;
constexpr int kOffStat = kOffTmem + 16;
constexpr int kStatBytes = 2 * 4 * 48;       // [slot][warp] WarpPiece
constexpr int kOffDesc = kOffStat + kGroups * kStatBytes;  // [group] EvalDesc
constexpr int kSmemBytes = kOffDesc + kGroups * 16;
constexpr int kTmemCols = 512;               // group g: D1[0], D1[1] at 256 g + {0, 64}, D2 at 256 g + 128,
                                             // parked x and grad at + 160, the halves' exchange at + 224
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");

constexpr float kLog2e = 1.4426950408889634f;
constexpr uint32_t kIdescFwd = idesc_bf16(128, kChunk, false);
constexpr uint32_t kIdescBwd = idesc_bf16(128, kD, true);

__device__ __forceinline__ void group_sync(int g) { named_sync(1 + g, kGroupThreads); }

// two-column TMEM store and load (the halves of a particle exchange partial sums through them)
__device__ __forceinline__ void tmem_st2f(uint32_t taddr, float a, float b)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ float2 tmem_ld2f(uint32_t taddr)
{
    uint32_t a, b;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr));
    tmem_wait_ld();
    return make_float2(__uint_as_float(a), __uint_as_float(b));
}
__device__ __forceinline__ void tmem_st16f(uint32_t taddr, const float (&f)[16])
{
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __float_as_uint(f[i]);
    tmem_st16(taddr, v);
}
__device__ __forceinline__ void tmem_ld16f(uint32_t taddr, float (&f)[16])
{
    uint32_t v[16];
    tmem_ld16(taddr, v);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
}

// Two-term bf16 split of a pair of floats, v = hi + lo: hi = v with the low 16 bits of its
// fp32 word cleared (a bf16 value, |v - hi| < 2^-7 |v|, exact in fp32), lo = v - hi rounded
// to the nearest bf16 (error at most 2^-9 |v - hi|, no sign bias), so hi + lo is within
// 2^-16 |v|.  The hi pair is the top halves of the two fp32 words (one byte permute); the
// two differences take one packed subtraction and the lo pair one conversion.
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo)
{
    const float ha = __uint_as_float(__float_as_uint(a) & 0xFFFF0000u);
    const float hb = __uint_as_float(__float_as_uint(b) & 0xFFFF0000u);
    const float2 l = sub_f32x2(make_float2(a, b), make_float2(ha, hb));
    hi = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
    lo = bf16x2_rn(l.x, l.y);
}

struct TcParams {
    SweepParams sp;
    const uint4* Ximg;       // [kMaxRows * 64 B / 16] BF16 image of X in the smem layout
    const uint32_t* ybits;   // [kMaxRows / 32]
    int n;                   // data rows
    int d;                   // true dimension (<= 32; padded columns of X are zero)
    int tiles;               // tiles of 128 particles (moment records per step)
    int64_t span;            // annealing steps per slot (group) of the persistent grid
    float* grad_state;       // [d][N]: grad log L of a tile handed between two slots
    int* handed;             // [tiles]: 1 once a tile's first part has stored its state
};

// the shared-memory and TMEM addresses of group g's barriers and accumulators
struct GroupAddr {
    uint32_t barF[2], barB;  // mbarriers: forward into D1[i] done, backward done
    uint32_t barR;           // mbarrier: the group's warps have written their R rows
    uint32_t barA;           // mbarrier: the group's warps have written their A rows
    uint32_t barEnd;         // mbarrier: every MMA of the group has completed (end of the sweep)
    uint32_t d1[2], d2;      // TMEM addresses
    uint32_t smem;           // shared-memory base address
    int g;
};
__device__ __forceinline__ GroupAddr group_addr(unsigned char* smem, uint32_t tmem, int g)
{
    GroupAddr A;
    const uint32_t bars = saddr(smem + kOffBar) + 8u * (uint32_t)(kBarsPerGroup * g);
    A.barF[0] = bars;
    A.barF[1] = bars + 8;
    A.barB = bars + 16;
    A.barR = bars + 24;
    A.barA = bars + 32;
    A.barEnd = bars + 40;
    A.d1[0] = tmem + (uint32_t)(g * 256);
    A.d1[1] = tmem + (uint32_t)(g * 256 + 64);
    A.d2 = tmem + (uint32_t)(g * 256 + 128);
    A.smem = saddr(smem);
    A.g = g;
    return A;
}

// One warp's share of a step's moment record (Alg. 1 moments, Sec. 5.1.1): the anchor (the
// first active particle's log w and log g), per moment i the maximum fp32 offset
// (log w - a0) + i (log g - b0) over the warp and the sum of exp(offset - maximum), and the
// warp's acceptance count, and u = sum exp(offset_0 - mx_0) log g (the ELBO term on moment
// 0's shift).  The shift m_i = a0 + i b0 + mx_i is formed in fp64 by the merge.
struct WarpPiece {
    double a0;               // -inf: no active particle in the warp
    float b0, mx[3], s[3], u;
    unsigned acc;
    unsigned pad;
};
static_assert(sizeof(WarpPiece) == 48, "WarpPiece layout");

__device__ __forceinline__ void warp_piece(double lw, float lg, bool active, WarpPiece* out)
{
    const unsigned full = 0xFFFFFFFFu;
    const unsigned act = __ballot_sync(full, active);
    const bool lead = (threadIdx.x & 31) == 0;
    if (act == 0) {
        if (lead) {
            out->a0 = -INFINITY;
            out->b0 = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; ++i) { out->mx[i] = 0.0f; out->s[i] = 0.0f; }
            out->u = 0.0f;
        }
        return;
    }
    const int src = __ffs(act) - 1;
    const double a0 = __shfl_sync(full, lw, src);
    const float b0 = __shfl_sync(full, lg, src);
    const float dw = (float)(lw - a0), dg = lg - b0;
    if (lead) { out->a0 = a0; out->b0 = b0; }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float f = active ? dw + (float)i * dg : -INFINITY;
        float mx = f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(full, mx, o));
        float e = active ? __expf(f - mx) : 0.0f;
        float u = i == 0 ? e * lg : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(full, e, o);
        if (i == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(full, u, o);
        }
        if (lead) {
            out->mx[i] = mx;
            out->s[i] = e;
            if (i == 0) out->u = u;
        }
    }
}

// the group's 4 pieces of a step into one record (every lane of the calling warp takes part)
__device__ __forceinline__ void merge_pieces(int lane, const WarpPiece* pc, StepPartial* out)
{
    const WarpPiece& q = pc[lane & 3];         // lanes >= 4 read a valid piece and ignore it
    double m[3];
    float sv[4];
    const bool has = lane < 4 && q.a0 != -INFINITY;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        m[i] = has ? q.a0 + i * (double)q.b0 + (double)q.mx[i] : -INFINITY;
        sv[i] = has ? q.s[i] : 0.0f;
    }
    sv[3] = has ? q.u : 0.0f;
    merge_lane_pieces<4, true>(lane, m, sv, lane < 4 ? q.acc : 0u, out);
}

// What the MMA warp does at the start of an evaluation (written by the group's thread 0
// before it arrives on barA): stop, or issue the evaluation and, at the first evaluation of
// step t + 1 of a piece, merge step t's record into rec.
struct EvalDesc {
    StepPartial* rec;        // null: no record to merge
    int slot;                // pieces slot of that step (t & 1)
    int stop;                // 1: no more evaluations
};
static_assert(sizeof(EvalDesc) <= 16, "EvalDesc fits its slot");

struct Group {
    GroupAddr a;
    int g;                   // group
    int h;                   // half: columns [32 h, 32 h + 32) of a chunk, coordinates [16 h, 16 h + 16)
    int q;                   // lane quarter of the warp (TMEM lanes 32 q .. 32 q + 31)
    int p;                   // particle of the tile: 32 q + lane
    int gt;                  // thread index within the group
    uint32_t lane_off;       // TMEM lane offset of the warp
    uint32_t stash;          // TMEM columns parking the particle state during an evaluation
    uint32_t xch;            // TMEM columns where the two halves exchange partial sums
    uint32_t phF, phB;       // expected phase of barF[i] (bit i), barB
    bool dead;               // a barrier wait timed out or the MMA warp gave up
    volatile int* abort;     // set by whichever role times out first
    unsigned char* smem;
};

// write this thread's 16 coordinates of its particle's row, scaled by log2(e) and split hi/lo,
// into the group's A tiles (the forward contraction then gives the margins in base-2 units)
__device__ __forceinline__ void write_state_tile(const Group& G, const float (&v)[kHalfD])
{
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split_pair(kLog2e * v[2 * j], kLog2e * v[2 * j + 1], hi[j], lo[j]);
    unsigned char* ah = G.smem + kOffA + (G.g * 2 + 0) * kATile;
    unsigned char* al = G.smem + kOffA + (G.g * 2 + 1) * kATile;
    const int p = G.p;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
        const int c = 2 * G.h + cc;            // 16-byte chunk of the 64-byte row: coordinates 8c .. 8c + 7
        const int off = p * 64 + ((c ^ ((p >> 1) & 3)) << 4);
        *reinterpret_cast<uint4*>(ah + off) = make_uint4(hi[4 * cc], hi[4 * cc + 1], hi[4 * cc + 2], hi[4 * cc + 3]);
        *reinterpret_cast<uint4*>(al + off) = make_uint4(lo[4 * cc], lo[4 * cc + 1], lo[4 * cc + 2], lo[4 * cc + 3]);
    }
}

// forward contraction of chunk c into D1[buf]: Z = (P_hi + P_lo) X'_c^T
__device__ __forceinline__ void issue_fwd(const GroupAddr& G, int c, int buf, uint32_t leader)
{
    const uint32_t base = G.smem;
    const uint32_t xb = base + kOffX;
#pragma unroll
    for (int hl = 0; hl < 2; ++hl) {
        const uint32_t aa = base + kOffA + (G.g * 2 + hl) * kATile;
#pragma unroll
        for (int kk = 0; kk < kD / 16; ++kk) {
            const uint64_t a = sdesc(aa + kk * 32, 16, 512, kSW64);
            const uint64_t b = sdesc(xb + c * kChunk * 64 + kk * 32, 16, 512, kSW64);
            mma_f16_by(leader, G.d1[buf], a, b, kIdescFwd, (hl == 0 && kk == 0) ? 0u : 1u);
        }
    }
    mma_commit_by(leader, G.barF[buf]);
}

// backward contraction of chunk c into D2: G += (R_hi + R_lo) X'_c (first starts the sum)
__device__ __forceinline__ void issue_bwd(const GroupAddr& G, int c, bool first, uint32_t leader)
{
    const uint32_t base = G.smem;
    const uint32_t xb = base + kOffX;
#pragma unroll
    for (int hl = 0; hl < 2; ++hl) {
        const uint32_t ra = base + kOffR + (G.g * 2 + hl) * kRTile;
#pragma unroll
        for (int kk = 0; kk < kChunk / 16; ++kk) {
            const uint64_t a = sdesc(ra + kk * 32, 16, 1024, kSW128);
            const uint64_t b = sdesc(xb + (c * kChunk + kk * 16) * 64, 8192, 512, kSW64);
            mma_f16_by(leader, G.d2, a, b, kIdescBwd, (first && hl == 0 && kk == 0) ? 0u : 1u);
        }
    }
    mma_commit_by(leader, G.barB);
}

__device__ __forceinline__ void wait_fwd(Group& G, int buf)
{
    if (!G.dead && !mbar_wait(G.a.barF[buf], (G.phF >> buf) & 1u, G.abort)) {
        G.dead = true;
        *G.abort = 1;
    }
    G.phF ^= 1u << buf;
}
__device__ __forceinline__ void wait_bwd(Group& G)
{
    if (!G.dead && !mbar_wait(G.a.barB, G.phB, G.abort)) {
        G.dead = true;
        *G.abort = 1;
    }
    G.phB ^= 1u;
}

// Group g's MMA warp (lane 0 issues): per evaluation it waits for the A tile, reads the
// evaluation's descriptor and issues the forwards of chunks 0 and 1, then per chunk c waits
// for the R tile and issues the backward of chunk c and the forward of chunk c + 2 into the D1
// buffer just read.  Between the forwards and the first backward it merges the moment record
// the descriptor names (a finished step's; off the particle warps' path: that step's pieces
// slot is next written two steps later, after this evaluation's contractions).  A wait that
// times out (or another role's) sets the abort flag and ends the loop; before returning the
// warp waits for every MMA it issued, so tensor memory is never released under a running
// contraction.
__device__ void mma_issuer(unsigned char* smem, uint32_t tmem, int g, int nch, volatile int* abort)
{
    const GroupAddr A = group_addr(smem, tmem, g);
    const WarpPiece (*pieces)[4] = reinterpret_cast<const WarpPiece (*)[4]>(smem + kOffStat + g * kStatBytes);
    const volatile EvalDesc* desc = reinterpret_cast<const volatile EvalDesc*>(smem + kOffDesc + 16 * g);
    const uint32_t leader = (threadIdx.x & 31) == 0;
    uint32_t phA = 0, phR = 0;
    bool ok = true;
    for (;;) {
        ok = mbar_wait(A.barA, phA, abort);
        phA ^= 1u;
        if (!ok || desc->stop) break;
        StepPartial* rec = desc->rec;
        const int slot = desc->slot;
        tc_after_sync();
        issue_fwd(A, 0, 0, leader);
        if (nch > 1) issue_fwd(A, 1, 1, leader);
        if (rec) merge_pieces(threadIdx.x & 31, pieces[slot], rec);
        for (int c = 0; c < nch; ++c) {
            ok = mbar_wait(A.barR, phR, abort);
            phR ^= 1u;
            if (!ok) break;
            tc_after_sync();
            issue_bwd(A, c, c == 0, leader);
            if (c + 2 < nch) issue_fwd(A, c + 2, c & 1, leader);
        }
        if (!ok) break;
    }
    if (!ok) *abort = 1;
    mma_commit_by(leader, A.barEnd);
    if (!mbar_wait(A.barEnd, 0)) *abort = 1;
}

// log L(x) and grad log L(x) for the group's 128 particles; every thread of the group calls it,
// the two threads of a particle each taking half the columns of every chunk.
// Pipeline per chunk c: the forward of chunk c+1 runs into the other D1 buffer while the
// epilogue of chunk c reads D1[c%2].  Each warp arrives on barA once its rows of the A tile
// are written and on barR once its rows of the R tile are written (and its reads of D1 are
// done); the MMA warp then issues the backward of chunk c (it runs while the next chunk's
// epilogue is computed; the R tile is waited for before the next write) and the forward of
// chunk c+2 into the D1 buffer just read.
// tc_eval_begin writes the state tile; tc_eval_run does the chunks and returns this half's
// part of log L (the halves' parts add up to log L) and its half of grad log L.
__device__ __forceinline__ void tc_eval_begin(Group& G, const float (&x)[kHalfD])
{
    write_state_tile(G, x);
    fence_proxy_async();
    tc_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(G.a.barA);
}
__device__ float tc_eval_run(Group& G, const TcParams& P, float (&grad)[kHalfD])
{
    const int nch = (P.n + kChunk - 1) / kChunk;
    const int p = G.p;
    unsigned char* rh = G.smem + kOffR + (G.g * 2 + 0) * kRTile;
    unsigned char* rl = G.smem + kOffR + (G.g * 2 + 1) * kRTile;
    // The image holds X'_r = s_r X~_r with s_r = 2 y_r - 1 and the state tile holds log2(e) x,
    // so the forward contraction gives u = log2(e) s z (the margin in base-2 units).  Per row:
    // log sigmoid(s z) = ln 2 (min(u, 0) + log2 q), q = 1 / (1 + 2^-|u|), and d/dz = s sigmoid(-s z),
    // so grad = sum_r sigmoid(-s_r z_r) X'_r with sigmoid(-s z) = 2^-|u| q for u >= 0, q for u < 0.
    // The rows of a pair go through the packed fp32 pair instructions; the sum of min(u, 0)
    // and the product of q are kept per lane of the pair and per chunk (32 rows of this half:
    // each product of 16 values in [1/2, 1], no underflow), with one log per chunk.  Padded
    // rows (X' = 0) give u = 0: log2 q = -1 each, corrected below, and nothing to the gradient.
    float sum_min = 0.0f, logs2 = 0.0f;
    const float2 one2 = make_float2(1.0f, 1.0f);
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        wait_fwd(G, b);
        __syncwarp();                             // tcgen05.ld below is warp-aligned
        tc_after_sync();
        float2 prod = one2, mn = make_float2(0.0f, 0.0f);
        // this half's 32 columns in one load (one wait per chunk; 1.6 % faster than two
        // 16-column loads at the same 96 registers), then two 16-column passes
        uint32_t vv[32];
        tmem_ld32(G.a.d1[b] + G.lane_off + G.h * kHalfCols, vv);
        tmem_wait_ld();
#pragma unroll
        for (int sub = 0; sub < 2; ++sub) {
            const uint32_t* v = vv + sub * 16;
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const float ua = __uint_as_float(v[j]), ub = __uint_as_float(v[j + 1]);
                const float2 e = make_float2(ex2_approx(-fabsf(ua)), ex2_approx(-fabsf(ub)));
                const float2 dq = add_f32x2(e, one2);
                const float2 q = make_float2(rcp_approx(dq.x), rcp_approx(dq.y));
                // with h = [u >= 0] and 1 - h (each 0 or 1, so the products below are exact):
                // sigmoid(-u) = q (h 2^-|u| + (1 - h)), min(u, 0) = u (1 - h)
                const float2 hge = make_float2(step_ge0(ua), step_ge0(ub));
                const float2 omh = sub_f32x2(one2, hge);
                const float2 r = mul_f32x2(q, fma_f32x2(hge, e, omh));
                mn = fma_f32x2(make_float2(ua, ub), omh, mn);
                prod = mul_f32x2(prod, q);
                split_pair(r.x, r.y, hi[j / 2], lo[j / 2]);
            }
            if (sub == 0 && c > 0) wait_bwd(G);   // the backward of chunk c-1 has read R
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int chunk = G.h * 4 + sub * 2 + cc;   // 16-byte chunk of the 128-byte R row
                const int off = p * 128 + ((chunk ^ (p & 7)) << 4);
                *reinterpret_cast<uint4*>(rh + off) =
                    make_uint4(hi[4 * cc], hi[4 * cc + 1], hi[4 * cc + 2], hi[4 * cc + 3]);
                *reinterpret_cast<uint4*>(rl + off) =
                    make_uint4(lo[4 * cc], lo[4 * cc + 1], lo[4 * cc + 2], lo[4 * cc + 3]);
            }
        }
        sum_min += mn.x + mn.y;
        logs2 += lg2_approx(prod.x * prod.y);
        fence_proxy_async();                      // my R rows, visible to the tensor core
        tc_before_sync();                         // my reads of D1[b] before its next forward
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(G.a.barR);
    }
    wait_bwd(G);                                  // the backward of the last chunk
    __syncwarp();
    tc_after_sync();
    uint32_t v[kHalfD];
    tmem_ld16(G.a.d2 + G.lane_off + G.h * kHalfD, v);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < kHalfD; ++i) grad[i] = __uint_as_float(v[i]);
    tc_before_sync();
    const float ln2 = 0.69314718055994531f;
    return ln2 * (sum_min + logs2 + (G.h == 0 ? (float)(nch * kChunk - P.n) : 0.0f));
}

// The two threads of a particle swap a pair of partial sums through TMEM; both return
// (half 0's, half 1's) so that both form the same totals in the same order.
__device__ __forceinline__ void exchange(Group& G, float a, float b, float2& h0, float2& h1)
{
    tmem_st2f(G.xch + G.lane_off + 2 * G.h, a, b);
    tmem_wait_st();
    tc_before_sync();
    group_sync(G.g);
    tc_after_sync();
    const float2 other = tmem_ld2f(G.xch + G.lane_off + 2 * (1 - G.h));
    const float2 mine = make_float2(a, b);
    h0 = G.h == 0 ? mine : other;
    h1 = G.h == 0 ? other : mine;
}

// log L of the particle (both halves) and this half's gradient
__device__ __forceinline__ float tc_eval(Group& G, const TcParams& P, const float (&x)[kHalfD],
                                         float (&grad)[kHalfD])
{
    tc_eval_begin(G, x);
    const float part = tc_eval_run(G, P, grad);
    float2 a, b;
    exchange(G, part, 0.0f, a, b);
    return a.x + b.x;
}

// this half's 16 normals of block (n, t, k): blocks 4 h .. 4 h + 3 of the particle's draw
__device__ __forceinline__ void half_normals(const Group& G, const Rng& rng, uint32_t n, uint32_t t, uint32_t k,
                                             int d, float (&z)[kHalfD])
{
#pragma unroll
    for (int jj = 0; jj < kHalfD / 4; ++jj) {
        const int j = G.h * (kHalfD / 4) + jj;
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (4 * j < d) box_muller4_sfu(rng.block(n, t, k, (uint32_t)j), v);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) z[4 * jj + qq] = (4 * j + qq < d) ? v[qq] : 0.0f;
    }
}

__global__ void __launch_bounds__(kThreads, 1)
oais_sweep_tc_kernel(const TcParams P)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const SweepParams& S = P.sp;
    // the 128B-swizzled tiles need a 1024-byte aligned base
    if (saddr(smem) & 1023u) {
        if (threadIdx.x == 0) atomicOr(S.status, 4u);
        return;
    }
    // stage the BF16 image of the label-signed data X' (kept for the whole sweep)
    {
        const uint4* src = P.Ximg;
        for (int i = threadIdx.x; i < kMaxRows * kD * 2 / 16; i += kThreads) cp_async16(smem + kOffX + 16 * i, src + i);
        cp_async_commit();
        cp_async_wait<0>();
    }
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOffBar);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffAbort);
    if (threadIdx.x == 0) {
        for (int g = 0; g < kGroups; ++g) {
            for (int i = 0; i < 3; ++i) mbar_init(saddr(&bars[kBarsPerGroup * g + i]), 1);
            mbar_init(saddr(&bars[kBarsPerGroup * g + 3]), kGroupWarps);   // one arrival per warp
            mbar_init(saddr(&bars[kBarsPerGroup * g + 4]), kGroupWarps);
            mbar_init(saddr(&bars[kBarsPerGroup * g + 5]), 1);
        }
        *abort = 0;
        fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tmem_alloc(saddr(smem + kOffTmem), kTmemCols);
        tmem_relinquish();
    }
    fence_proxy_async();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + kOffTmem);

    if (threadIdx.x / 32 >= kMmaWarp0) {
        mma_issuer(smem, tmem, threadIdx.x / 32 - kMmaWarp0, (P.n + kChunk - 1) / kChunk, abort);
        if (threadIdx.x % 32 == 0 && *abort) atomicOr(S.status, 2u);
        tc_before_sync();
        __syncthreads();
        return;
    }

    Group G;
    G.g = threadIdx.x / kGroupThreads;
    G.gt = threadIdx.x % kGroupThreads;
    {
        const int wg = G.gt / 32;
        G.h = wg / 4;
        G.q = wg % 4;                                  // = (CTA warp index) % 4: the warp's TMEM lane quarter
        G.p = G.q * 32 + (threadIdx.x & 31);
    }
    G.a = group_addr(smem, tmem, G.g);
    G.lane_off = (uint32_t)(G.q * 32) << 16;
    G.stash = tmem + (uint32_t)(G.g * 256 + 160);  // x at + 16 h, grad at + 32 + 16 h
    G.xch = tmem + (uint32_t)(G.g * 256 + 224);
    G.phF = 0;
    G.phB = 0;
    G.dead = false;
    G.abort = abort;
    G.smem = smem;
    WarpPiece (*pieces)[4] = reinterpret_cast<WarpPiece (*)[4]>(smem + kOffStat + G.g * kStatBytes);

    volatile EvalDesc* desc = reinterpret_cast<volatile EvalDesc*>(smem + kOffDesc + 16 * G.g);
    const int d = P.d;
    const int i0 = G.h * kHalfD;                   // this thread's coordinates: i0 .. i0 + 15
    const float sref = (float)S.ref_scale;
    const float inv_s2 = 1.0f / (sref * sref);
    const int lane = threadIdx.x & 31;
    const uint32_t sx = G.stash + G.lane_off + (uint32_t)(G.h * kHalfD);
    const uint32_t sg = sx + (uint32_t)kD;
    // thread 0 says what the MMA warp does at the next evaluation, before the group's barA
    auto announce = [&](StepPartial* rec, int slot) {
        if (G.gt == 0) {
            desc->rec = rec;
            desc->slot = slot;
            desc->stop = 0;
        }
    };

    // Persistent grid, wrap-around schedule (McNaughton's rule for preemptive scheduling of
    // independent jobs): tile i is the job of T steps at positions [i T, (i + 1) T) of the
    // concatenated sequence, slot s (group g of CTA b, s = 2 b + g) covers the positions
    // [s L, (s + 1) L) with L = span >= T.  A tile split between slots s and s + 1 runs its
    // first steps at the start of slot s + 1 and its last steps at the end of slot s, which
    // cannot overlap in time because L >= T; the first part stores the tile's state and sets
    // handed[tile], the last part waits for the flag (bounded) and loads the state.  So the
    // slot's work is: the head (a split tile's first steps), whole tiles, the tail (a split
    // tile's last steps).  With at most one tile per slot (L = T) this is one tile per group.
    const int T = S.T;
    const int64_t total = (int64_t)P.tiles * T;
    const int64_t slot_id = (int64_t)blockIdx.x * kGroups + G.g;
    const int64_t pos0 = slot_id * P.span, pos1 = min(pos0 + P.span, total);
    float* xo = reinterpret_cast<float*>(S.x_out);
    for (int64_t pos = pos0; pos < pos1 && T > 0;) {
        // the piece at position pos: tile, first and last step
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
        const int64_t n64 = tile * kTile + G.p;
        const bool active = n64 < S.N;
        const uint32_t n = (uint32_t)(S.n_offset + (active ? n64 : S.N - 1));
        float x[kHalfD], gl[kHalfD], ell;
        double logw;
        if (t0 == 1) {
            half_normals(G, S.mv.rng, n, 0u, 0u, d, x);
#pragma unroll
            for (int i = 0; i < kHalfD; ++i) x[i] *= sref;
            announce(nullptr, 0);
            ell = tc_eval(G, P, x, gl);
            logw = 0.0;
        } else {
            // the tile's first part ran at the start of the next slot: wait for its state
            if (G.gt == 0 && !G.dead) {
                const uint64_t w0 = globaltimer();
                const uint64_t limit = S.handoff_wait_ns ? S.handoff_wait_ns : kWaitLimitNs;
                while (ld_acquire_gpu(P.handed + tile) == 0) {
                    if (*G.abort || globaltimer() - w0 > limit) { G.dead = true; *G.abort = 1; break; }
                    __nanosleep(256);
                }
            }
            group_sync(G.g);
            (void)ld_acquire_gpu(P.handed + tile);
#pragma unroll
            for (int i = 0; i < kHalfD; ++i) {
                x[i] = (active && i0 + i < d) ? xo[(size_t)(i0 + i) * S.N + n64] : 0.0f;
                gl[i] = (active && i0 + i < d) ? P.grad_state[(size_t)(i0 + i) * S.N + n64] : 0.0f;
            }
            ell = active ? (float)S.ell_out[n64] : 0.0f;
            logw = active ? S.logw[n64] : 0.0;
        }
        double beta_prev = S.beta[t0 - 1];
        for (int t = t0; t <= t1; ++t) {
            const double beta_t = __ldg(S.beta + t);
            const double eps_t = __ldg(S.eps + t - 1);
            // log g_t = (beta_t - beta_{t-1}) log L(x) in fp32 (log L is an fp32 value); log w in fp64
            const float lg = (float)(beta_t - beta_prev) * ell;
            beta_prev = beta_t;
            const int slot = t & 1;
            if (G.h == 0) warp_piece(logw, lg, active, &pieces[slot][G.q]);
            logw += (double)lg;
            unsigned acc = 0;
            const float beta = (float)beta_t, e = (float)eps_t, hh = 0.5f * e;
            for (int k = 0; k < S.mv.K; ++k) {
                // MALA (Sec. 2.1.1 kernel family): x' = x + e w with w = z + (e/2) grad log pi(x);
                // each half proposes its 16 coordinates, the sums over coordinates add up
                float zz = 0.0f, dxx = 0.0f;
                {
                    float w[kHalfD], xp[kHalfD];
                    half_normals(G, S.mv.rng, n, (uint32_t)t, (uint32_t)k, d, w);
#pragma unroll
                    for (int i = 0; i < kHalfD; ++i) {
                        const float gpi = -x[i] * inv_s2 + beta * gl[i];
                        zz += w[i] * w[i];
                        w[i] = __fmaf_rn(hh, gpi, w[i]);
                        xp[i] = __fmaf_rn(e, w[i], x[i]);
                        dxx += (xp[i] - x[i]) * (xp[i] + x[i]);
                    }
                    // park x and grad in the group's free TMEM columns while the evaluation runs
                    // (registers go to the epilogue); w is drawn again afterwards and x'
                    // rebuilt from them with the same rounding
                    tmem_st16f(sx, x);
                    tmem_st16f(sg, gl);
                    tmem_wait_st();
                    // the first evaluation of step t: step t - 1's record is complete
                    const bool merge = k == 0 && t > t0;
                    announce(merge ? S.partials + (int64_t)(t - 2) * P.tiles + tile : nullptr, (t - 1) & 1);
                    tc_eval_begin(G, xp);
                }
                float glp[kHalfD];
                const float part = tc_eval_run(G, P, glp);
                __syncwarp();
                tmem_ld16f(sx, x);
                tmem_ld16f(sg, gl);
                float w[kHalfD];
                half_normals(G, S.mv.rng, n, (uint32_t)t, (uint32_t)k, d, w);
                float rev = 0.0f;
#pragma unroll
                for (int i = 0; i < kHalfD; ++i) {
                    const float gpi = -x[i] * inv_s2 + beta * gl[i];
                    w[i] = __fmaf_rn(hh, gpi, w[i]);
                    const float xp = __fmaf_rn(e, w[i], x[i]);
                    const float qv = w[i] + hh * (-xp * inv_s2 + beta * glp[i]);
                    rev += qv * qv;
                }
                // the halves' parts: log L(x') and -(1/2)(|x'|^2 - |x|^2)/s^2 - (1/2)(|w'|^2 - |z|^2)
                float2 a0, a1;
                exchange(G, part, -0.5f * dxx * inv_s2 - 0.5f * (rev - zz), a0, a1);
                const float ellp = a0.x + a1.x;
                const float log_alpha = (a0.y + a1.y) + beta * (ellp - ell);
                const float logu = mh_log_uniform(S.mv.rng, n, (uint32_t)t, (uint32_t)k, 0.0f);
                if (logu < log_alpha) {
#pragma unroll
                    for (int i = 0; i < kHalfD; ++i) { x[i] = __fmaf_rn(e, w[i], x[i]); gl[i] = glp[i]; }
                    ell = ellp;
                    ++acc;
                }
            }
            acc = active ? acc : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (G.h == 0 && lane == 0) pieces[slot][G.q].acc = acc;
        }
        // the piece's last step's record (the MMA warp merged the others)
        group_sync(G.g);
        if (G.gt < 32) merge_pieces(lane, pieces[t1 & 1], S.partials + (int64_t)(t1 - 1) * P.tiles + tile);
        if (active) {
            if (G.h == 0) {
                S.logw[n64] = logw;
                S.ell_out[n64] = (double)ell;
            }
#pragma unroll
            for (int i = 0; i < kHalfD; ++i) if (i0 + i < d) xo[(size_t)(i0 + i) * S.N + n64] = x[i];
            if (t1 < T) {
#pragma unroll
                for (int i = 0; i < kHalfD; ++i) if (i0 + i < d) P.grad_state[(size_t)(i0 + i) * S.N + n64] = gl[i];
            } else if (G.h == 0 && (!isfinite(logw) || !isfinite(ell))) {
                atomicOr(S.status, 1u);
            }
        }
        if (t1 < T) __threadfence();
        group_sync(G.g);                      // pieces slots free; the state is stored
        if (t1 < T && G.gt == 0 && !S.withhold) st_release_gpu(P.handed + tile, 1);
    }
    // no more evaluations: release the MMA warp
    if (G.gt == 0) desc->stop = 1;
    __syncwarp();
    if (lane == 0) mbar_arrive(G.a.barA);
    if (G.dead && G.gt == 0) atomicOr(S.status, 2u);
    tc_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(tmem, kTmemCols);
}

} // namespace tc

int tc_grid(int64_t N) { return (int)((N + tc::kParticlesPerCta - 1) / tc::kParticlesPerCta); }
int tc_records(int64_t N) { return tc_grid(N) * tc::kGroups; }

// BF16 image of X in the kernel's shared-memory layout (rows of 64 B, 64B swizzle) and the
// label bitmask; X is [n][d] row-major fp32 on the host.
int tc_image_bytes() { return tc::kMaxRows * tc::kD * 2; }
int tc_max_rows() { return tc::kMaxRows; }
void tc_prepare_logreg(const float* X, const float* y, int n, int d, std::vector<uint16_t>& img,
                       std::vector<uint32_t>& ybits)
{
    img.assign((size_t)tc::kMaxRows * tc::kD, 0);
    ybits.assign(tc::kMaxRows / 32, 0u);
    auto bf16 = [](float v) -> uint16_t {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even (finite inputs)
        return (uint16_t)(u >> 16);
    };
    for (int r = 0; r < n; ++r) {
        // label sign folded into the row: X'_r = (2 y_r - 1) X_r (exact in bf16)
        const bool pos = y[r] > 0.5f;
        for (int i = 0; i < d; ++i) {
            const int c = i / 8, q = i % 8;
            const int phys = (c ^ ((r >> 1) & 3));
            const uint16_t b = bf16(X[(size_t)r * d + i]);
            img[(size_t)r * tc::kD + phys * 8 + q] = pos ? b : (uint16_t)(b ^ 0x8000u);
        }
        if (pos) ybits[r / 32] |= 1u << (r % 32);
    }
}

// Persistent grid: one tile per group when the tiles fit in one wave of groups, else one CTA
// per SM and the wrap-around schedule over tiles x steps (span = steps per group >= T).
cudaError_t launch_sweep_tc(const SweepParams& sp, const void* Ximg, const uint32_t* ybits, int n, int d,
                            float* grad_state, int* handed, cudaStream_t s)
{
    tc::TcParams P;
    P.sp = sp;
    P.Ximg = static_cast<const uint4*>(Ximg);
    P.ybits = ybits;
    P.n = n;
    P.d = d;
    P.tiles = tc_records(sp.N);
    P.grad_state = grad_state;
    P.handed = handed;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int grid = (P.tiles + tc::kGroups - 1) / tc::kGroups;
    P.span = sp.T;
    if (grid > sms) {
        grid = sms;
        const int64_t slots = (int64_t)grid * tc::kGroups, total = (int64_t)P.tiles * sp.T;
        P.span = std::max<int64_t>(sp.T, (total + slots - 1) / slots);
        e = cudaMemsetAsync(handed, 0, sizeof(int) * P.tiles, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(tc::oais_sweep_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    if (e != cudaSuccess) return e;
    // a group may wait for another CTA's hand-off: every CTA resident at once (cooperative)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tc::kThreads);
    cfg.dynamicSmemBytes = tc::kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, tc::oais_sweep_tc_kernel, P);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

} // namespace oais
