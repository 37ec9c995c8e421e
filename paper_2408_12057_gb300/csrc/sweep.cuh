// sweep.cuh -- the loop-swapped OAIS particle sweep (Sec. 5.1.2): each thread owns one
// particle for all T annealing steps, so the particle's state never leaves registers;
// the only cross-particle work per step is the moment reduction of Alg. 1, done per CTA
// and written as one StepPartial record per (step, CTA).
//
// Step t of Alg. 1 for one particle, in the order the kernel runs it:
//   log g_t = (beta_t - beta_{t-1}) * log L(X_{t-1})   (incremental weight at the
//             pre-move state, quasi-reversal backward kernel, Sec. 2.1.2)
//   moments of (w_{t-1}, g_t)                           (Alg. 1 / eq. CESS)
//   log w_t = log w_{t-1} + log g_t                     (reweight)
//   K moves of a pi_{beta_t}-invariant MH kernel        (propagate)
#pragma once
#include "targets.cuh"

namespace oais {

enum MoveKind { kRwmh = 0, kMala = 1, kHmc = 2 };

constexpr int kSweepThreads = 128;

// what an MH move needs besides the particle
struct MoveCfg {
    Rng rng;
    int K;                // moves per step
    int leapfrog;
    int cycle;            // RWMH std cycles 0.1, 1, 10 by global move index
};

struct SweepParams {
    int64_t N;            // particles in this launch
    int64_t n_offset;     // global index of particle 0 (counter word 0)
    int T;
    const double* beta;   // [T+1]
    const double* eps;    // [T] step size per annealing step
    double ref_scale;     // s
    MoveCfg mv;
    // outputs
    double* logw;         // [N]
    void* x_out;          // [d][N] SoA, element type R
    double* ell_out;      // [N]
    StepPartial* partials;// [T][gridDim.x]
    unsigned* status;     // bit 0: non-finite value seen
    // test support (oais_arm_fault): with withhold != 0 the persistent tensor-core schedules
    // raise no hand-off flag, and a resumed tile waits for its flag at most handoff_wait_ns
    // (0: the default limit of every bounded wait)
    int withhold;
    uint64_t handoff_wait_ns;
};

template <typename R> __device__ __forceinline__ R rsq(R a) { return a * a; }

// Forms with fp32 particle arithmetic take the moment partials with fp32 offsets and
// rescaling (warp_moment_partial / merge_lane_pieces, kFast), and their random-walk moves the
// special-function-unit Box-Muller (absolute error of order 1e-6 in z, like the tensor-core
// kernels): the fp64 pipe of this part is slow, and with a cheap target (the mixture: two
// moves of a few hundred operations a step) the per-step fp64 bookkeeping and the exact
// Box-Muller took half of the step.  MALA and HMC keep the exact Box-Muller: their gradient
// evaluations dominate the step, and an HMC trajectory amplifies an error in its momentum.
// The fp64 forms keep both exact.
template <typename R> constexpr bool kFp32 = sizeof(R) == 4;

// log g_t = (beta_t - beta_{t-1}) log L(X_{t-1}): in fp64 for the fp64 forms; for the fp32 forms
// (log L an fp32 value) the product in fp32, log w accumulated in fp64 by the caller
template <typename R>
__device__ __forceinline__ double step_log_increment(double dbeta, R ell)
{
    if constexpr (kFp32<R>) {
        const float db = (float)dbeta;
        return db == 0.0f ? 0.0 : (double)(db * ell);
    } else {
        return log_increment(dbeta, (double)ell);
    }
}

// beta and eps: beta_t and the step size of step t in the particle precision
template <class Tgt, int MOVE, int D, typename R>
__device__ __forceinline__ bool mh_move(const Tgt& tg, const MoveCfg& P, R (&x)[D], R& ell,
                                        R (&gl)[D], R beta, R eps, uint32_t n,
                                        uint32_t t, uint32_t k, int d, R inv_s2)
{
    constexpr bool GRAD = (MOVE != kRwmh);
    R z[D];
    if constexpr (kFp32<R> && MOVE == kRwmh && Tgt::kind == kGmm) {
        // the mixture target carries the generator's precomputed round keys; at d = D the
        // padding tests fold away
        if (d == D) normals_sfu<D>(tg.rks, n, t, k, D, z);
        else normals_sfu<D>(tg.rks, n, t, k, d, z);
    } else if constexpr (kFp32<R> && MOVE == kRwmh) {
        normals_sfu<D>(P.rng, n, t, k, d, z);
    } else {
        normals<D>(P.rng, n, t, k, d, z);
    }
    R xp[D], glp[D];
    R log_alpha;
    R ellp;
    if (MOVE == kRwmh) {
        R sd = eps;
        if (P.cycle) {
            const int gm = ((int)t - 1) * P.K + (int)k;
            const int c = gm % 3;
            sd = c == 0 ? R(0.1) : (c == 1 ? R(1) : R(10));
        }
        R dxx = 0;                                    // |xp|^2 - |x|^2
        if constexpr (kFp32<R> && D % 2 == 0) {
            // two coordinates per packed instruction
            const float2 sd2 = make_float2(sd, sd);
            float2 a2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < D; i += 2) {
                const float2 x2 = make_float2(x[i], x[i + 1]);
                const float2 p2 = fma_f32x2(sd2, make_float2(z[i], z[i + 1]), x2);
                xp[i] = p2.x;
                xp[i + 1] = p2.y;
                a2 = fma_f32x2(sub_f32x2(p2, x2), add_f32x2(p2, x2), a2);
            }
            dxx = a2.x + a2.y;
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) {
                xp[i] = x[i] + sd * z[i];
                dxx += (xp[i] - x[i]) * (xp[i] + x[i]);
            }
        }
        ellp = tg.template eval<false>(xp, glp);
        log_alpha = -R(0.5) * dxx * inv_s2 + beta * (ellp - ell);
    } else if (MOVE == kMala) {
        // x' = x + (e^2/2) grad log pi(x) + e z;  with w = z + (e/2) grad log pi(x) the
        // reverse-proposal term is |w + (e/2) grad log pi(x')|^2 / 2 and the forward one |z|^2 / 2
        const R e = eps, h = R(0.5) * e;
        R zz = 0, dxx = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const R gpi = -x[i] * inv_s2 + beta * gl[i];
            xp[i] = x[i] + e * (h * gpi + z[i]);
            zz += z[i] * z[i];
            z[i] = z[i] + h * gpi;                     // w
            dxx += (xp[i] - x[i]) * (xp[i] + x[i]);
        }
        ellp = tg.template eval<true>(xp, glp);
        R rev = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) rev += rsq(z[i] + h * (-xp[i] * inv_s2 + beta * glp[i]));
        log_alpha = -R(0.5) * dxx * inv_s2 + beta * (ellp - ell) - R(0.5) * (rev - zz);
    } else {
        // HMC, identity mass: leapfrog with momentum p (kept in z)
        const R e = eps;
        R ke0 = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            ke0 += z[i] * z[i];
            z[i] += R(0.5) * e * (-x[i] * inv_s2 + beta * gl[i]);
            xp[i] = x[i];
        }
        ellp = ell;
        for (int l = 0; l < P.leapfrog; ++l) {
#pragma unroll
            for (int i = 0; i < D; ++i) xp[i] += e * z[i];
            ellp = tg.template eval<true>(xp, glp);
            const R f = (l + 1 < P.leapfrog) ? e : R(0.5) * e;
#pragma unroll
            for (int i = 0; i < D; ++i) z[i] += f * (-xp[i] * inv_s2 + beta * glp[i]);
        }
        R ke1 = 0, dxx = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) { ke1 += z[i] * z[i]; dxx += (xp[i] - x[i]) * (xp[i] + x[i]); }
        log_alpha = -R(0.5) * dxx * inv_s2 + beta * (ellp - ell) - R(0.5) * (ke1 - ke0);
    }
    R logu;
    if constexpr (kFp32<R> && MOVE == kRwmh && Tgt::kind == kGmm) logu = mh_log_uniform_sfu(tg.rks, n, t, k);
    else if constexpr (kFp32<R> && MOVE == kRwmh) logu = mh_log_uniform_sfu(P.rng, n, t, k);
    else logu = mh_log_uniform(P.rng, n, t, k, R(0));
    const bool acc = logu < log_alpha;
    if (acc) {
#pragma unroll
        for (int i = 0; i < D; ++i) { x[i] = xp[i]; if (GRAD) gl[i] = glp[i]; }
        ell = ellp;
    }
    return acc;
}

// CTAs per SM that the register allocation must allow (0: the compiler's choice).  The
// random-walk step of the mixture is cheap and latency-bound: the sweep runs fastest at 5 CTAs
// (96 registers: 1.445e10 particle-steps/s on the mixture workload, 1.398e10 at 6 CTAs and 80
// registers, 1.401e10 at 8 and 64; an explicit 1 gave 122 registers and 30 % less), the
// lock-step ASMC kernel of the same step at 8 (a T = 256 round in 44.1 ms; 46.1 at 6, 53.0
// with the compiler's 92 registers).
template <class Tgt, int MOVE> struct SweepMinBlocks { static constexpr int value = 0; };
template <typename R, int D> struct SweepMinBlocks<GmmTarget<R, D>, kRwmh> { static constexpr int value = 5; };
template <class Tgt, int MOVE> struct StepMinBlocks { static constexpr int value = 0; };
template <typename R, int D> struct StepMinBlocks<GmmTarget<R, D>, kRwmh> { static constexpr int value = 8; };

template <class Tgt, int MOVE, int D, typename R>
__global__ void __launch_bounds__(kSweepThreads, (SweepMinBlocks<Tgt, MOVE>::value))
oais_sweep_kernel(const SweepParams P, Tgt tg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kSS = kFp32<R> ? 8 : 4;   // floats per warp piece (fp32 forms: deferred shifts)
    __shared__ double s_m[2][kSweepThreads / 32][3];
    __shared__ float s_s[2][kSweepThreads / 32][kSS];
    __shared__ unsigned s_acc[2][kSweepThreads / 32];

    tg.setup(smem);
    const int d = tg.d;
    const int64_t n64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = n64 < P.N;
    // inactive lanes shadow the last particle so that every thread of the CTA joins
    // the cooperative target evaluations; their results are never written
    const uint32_t n = (uint32_t)(P.n_offset + (active ? n64 : P.N - 1));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R s = (R)P.ref_scale;
    const R inv_s2 = R(1) / (s * s);
    constexpr bool GRAD = (MOVE != kRwmh);

    R x[D], gl[D];
    normals<D>(P.mv.rng, n, 0u, 0u, d, x);
#pragma unroll
    for (int i = 0; i < D; ++i) { x[i] *= s; gl[i] = R(0); }
    R ell = tg.template eval<GRAD>(x, gl);
    double logw = 0.0;
    unsigned bad = 0;
    (void)lane;

    if constexpr (kFp32<R> && Tgt::kind == kGmm) {
        // fp32 bookkeeping (see df_add): log w = lwh + lwl, the step's schedule values from the
        // fp32 roundings the host prepared (the same values the conversions of the fp64 schedule
        // give), and the moment records of kMergeSteps steps at once: every thread leaves its
        // (log w_{t-1}, log g_t, accepted moves) of each step in shared memory (double-buffered,
        // so the warps run on into the next steps), and after the batch's barrier each half-warp
        // forms one step's record from the CTA's 128 values (half_step_record_df).  For the
        // mixture, whose evaluations are a few hundred instructions without barriers, the
        // per-step fp64 bookkeeping and barrier were a large share of the step (1.06e10 ->
        // 1.19e10 particle-steps/s), and the per-step warp reductions of the moments some 90
        // instructions per particle-step; the row families' evaluations synchronise the CTA
        // every data chunk anyway and keep the per-step form below.
        constexpr int kMergeSteps = 2 * (kSweepThreads / 32);   // one step per half-warp
        static_assert(kSweepThreads == 128, "16 lanes x 8 particles per step record");
        __shared__ float4 s_v[2][kMergeSteps][kSweepThreads];
        float lwh = 0.0f, lwl = 0.0f;
        double beta_prev = P.beta[0];
        for (int t = 1; t <= P.T; ++t) {
            float db, beta_r, eps_r;
            if (tg.fsched) {
                beta_r = tg.fsched[t];
                db = tg.fsched[P.T + t];
                eps_r = tg.fsched[2 * P.T + t];
            } else {
                const double beta_t = __ldg(P.beta + t);
                db = (float)(beta_t - beta_prev);
                beta_prev = beta_t;
                beta_r = (float)beta_t;
                eps_r = (float)__ldg(P.eps + t - 1);
            }
            const float lg = db == 0.0f ? 0.0f : db * (float)ell;
            const int buf = ((t - 1) / kMergeSteps) & 1, st = (t - 1) % kMergeSteps;
            const float pwh = lwh, pwl = lwl;   // log w_{t-1}
            df_add(lwh, lwl, lg);
            unsigned acc = 0;
            for (int k = 0; k < P.mv.K; ++k)
                acc += mh_move<Tgt, MOVE, D, R>(tg, P.mv, x, ell, gl, (R)beta_r, (R)eps_r, n, (uint32_t)t,
                                                (uint32_t)k, d, inv_s2) ? 1u : 0u;
            s_v[buf][st][threadIdx.x] = make_float4(pwh, pwl, lg, active ? (float)acc : -1.0f);
            if (st == kMergeSteps - 1 || t == P.T) {
                __syncthreads();
                const int t0 = t - st, s = 2 * warp + (lane >> 4);   // the batch's first step; this half's
                const bool on = s <= st;
                half_step_record_df<kSweepThreads / 16>(lane, s_v[buf][on ? s : 0], on,
                                                        P.partials + (size_t)(t0 - 1 + (on ? s : 0)) * gridDim.x +
                                                            blockIdx.x);
            }
        }
        logw = (double)lwh + (double)lwl;
    } else {
        double beta_prev = P.beta[0];
        for (int t = 1; t <= P.T; ++t) {
            const double beta_t = __ldg(P.beta + t);
            const double eps_t = __ldg(P.eps + t - 1);
            const double lg = step_log_increment<R>(beta_t - beta_prev, ell);
            beta_prev = beta_t;
            const R beta_r = (R)beta_t, eps_r = (R)eps_t;
            const int slot = t & 1;
            warp_moment_partial<kFp32<R>>(logw, lg, active, s_m[slot][warp], s_s[slot][warp]);
            logw += lg;
            unsigned acc = 0;
            for (int k = 0; k < P.mv.K; ++k)
                acc += mh_move<Tgt, MOVE, D, R>(tg, P.mv, x, ell, gl, beta_r, eps_r, n, (uint32_t)t,
                                                (uint32_t)k, d, inv_s2) ? 1u : 0u;
            acc = active ? acc : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (lane == 0) s_acc[slot][warp] = acc;
            __syncthreads();
            if constexpr (kFp32<R>) {
                if (warp == 0)
                    merge_deferred_pieces<kSweepThreads / 32>(lane, s_m[slot], s_s[slot], s_acc[slot],
                                                              P.partials + (size_t)(t - 1) * gridDim.x + blockIdx.x);
            } else {
                cta_moment_record<kSweepThreads / 32, false>(s_m[slot], s_s[slot], s_acc[slot],
                                                             P.partials + (size_t)(t - 1) * gridDim.x + blockIdx.x);
            }
        }
    }
    if (!admissible(logw) || !admissible((double)ell)) bad = 1;
    if (active) {
        P.logw[n64] = logw;
        P.ell_out[n64] = (double)ell;
        R* xo = reinterpret_cast<R*>(P.x_out);
#pragma unroll
        for (int i = 0; i < D; ++i) if (i < d) xo[(size_t)i * P.N + n64] = x[i];
    }
    if (active && bad) atomicOr(P.status, 1u);
}

// ---------------------------------------------------------------------------
// ASMC (Alg. 1 with adaptive resampling): particles advance in lock-step, one launch per
// annealing step, because the resampling test needs every particle's weight.  The
// particle store is double-buffered structure-of-arrays; the buffer in use is
// cur ^ pend (pend = "the previous step resampled into the other buffer"), both read
// from device memory, so a whole schedule can be launched without host round-trips.
// ---------------------------------------------------------------------------
struct AsmcState {
    int cur;            // buffer holding the particles at the start of the last decision
    int pend;           // 1: the last step resampled into buffer cur ^ 1
    int n_resample;     // intermediate resampling events so far
    unsigned ticket;    // CTAs of the ESS merge done this step (the last one decides, then resets it)
    double logZ;        // accumulated sum_r (LSE(log w_{tau_r^-}) - log N)
    double lse;         // LSE of the weights of the pending resampling event
    double U;           // its systematic-resampling uniform
};

struct StepParams {
    int64_t N;
    int t, T;
    const double* beta;
    const double* eps;
    double ref_scale;
    MoveCfg mv;
    void* x[2];           // [d][N] element type R
    void* gl[2];          // [d][N] grad log L (MALA/HMC), else unused
    double* ell[2];       // [N]
    double* logw;         // [N]
    const AsmcState* st;
    StepPartial* partials;  // [T][gridDim.x]
    StepPartial* ess_parts; // [gridDim.x]: m/s[0] for log w, m/s[1] for 2 log w
    unsigned* status;
    const int* skip;        // nullable device flag: when set, the step and its decision do nothing
                            // (a schedule found online that has already reached beta = 1)
};

template <class Tgt, int MOVE, int D, typename R>
__global__ void __launch_bounds__(kSweepThreads, (StepMinBlocks<Tgt, MOVE>::value))
asmc_step_kernel(const StepParams P, Tgt tg)
{
    if (P.skip && *P.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kSS = kFp32<R> ? 8 : 4;   // floats per warp piece (fp32 forms: deferred shifts)
    __shared__ double s_m[kSweepThreads / 32][3];
    __shared__ float s_s[kSweepThreads / 32][kSS];
    __shared__ unsigned s_acc[kSweepThreads / 32];
    constexpr bool GRAD = (MOVE != kRwmh);

    tg.setup(smem);
    const int d = tg.d;
    const int64_t n64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = n64 < P.N;
    const int64_t idx = active ? n64 : P.N - 1;
    const uint32_t n = (uint32_t)idx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R s = (R)P.ref_scale;
    const R inv_s2 = R(1) / (s * s);
    const int b = P.st->cur ^ P.st->pend;
    const R* xb = reinterpret_cast<const R*>(P.x[b]);
    const R* gb = reinterpret_cast<const R*>(P.gl[b]);

    R x[D], gl[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        x[i] = i < d ? xb[(size_t)i * P.N + idx] : R(0);
        gl[i] = (GRAD && i < d) ? gb[(size_t)i * P.N + idx] : R(0);
    }
    R ell = (R)P.ell[b][idx];
    double logw = P.logw[idx];

    const double beta_t = P.beta[P.t], eps_t = P.eps[P.t - 1];
    const double lg = step_log_increment<R>(beta_t - P.beta[P.t - 1], ell);
    const R beta_r = (R)beta_t, eps_r = (R)eps_t;
    if constexpr (kFp32<R>) {
        // the fp32 forms: the two records of the step (the moments of (w_{t-1}, g_t), the ESS
        // pieces of w_t) from the CTA's values in shared memory, one per half of warp 0, after
        // one barrier (instead of warp shuffle trees and a CTA merge for each)
        __shared__ double s_lw[kSweepThreads];
        __shared__ float s_lg[kSweepThreads], s_ac[kSweepThreads];
        const double lw_prev = logw;
        logw += lg;
        unsigned acc = 0;
        for (int k = 0; k < P.mv.K; ++k)
            acc += mh_move<Tgt, MOVE, D, R>(tg, P.mv, x, ell, gl, beta_r, eps_r, n, (uint32_t)P.t,
                                            (uint32_t)k, d, inv_s2) ? 1u : 0u;
        s_lw[threadIdx.x] = lw_prev;
        s_lg[threadIdx.x] = (float)lg;
        s_ac[threadIdx.x] = active ? (float)acc : -1.0f;
        __syncthreads();
        if (warp == 0) {
            const bool ess = lane >= 16;
            half_record_fp64w<kSweepThreads / 16>(lane, s_lw, s_lg, s_ac, ess, true,
                                                  ess ? P.ess_parts + blockIdx.x
                                                      : P.partials + (size_t)(P.t - 1) * gridDim.x + blockIdx.x);
        }
    } else {
    warp_moment_partial<kFp32<R>>(logw, lg, active, s_m[warp], s_s[warp]);
    logw += lg;
    unsigned acc = 0;
    for (int k = 0; k < P.mv.K; ++k)
        acc += mh_move<Tgt, MOVE, D, R>(tg, P.mv, x, ell, gl, beta_r, eps_r, n, (uint32_t)P.t,
                                        (uint32_t)k, d, inv_s2) ? 1u : 0u;
    acc = active ? acc : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    cta_moment_record<kSweepThreads / 32, false>(s_m, s_s, s_acc,
                                                 P.partials + (size_t)(P.t - 1) * gridDim.x + blockIdx.x);
    __syncthreads();
    // ESS pieces of w_{t^-}: LSE of log w (slot 0) and of 2 log w (slot 1)
    warp_moment_partial<kFp32<R>>(logw, logw, active, s_m[warp], s_s[warp]);
    __syncthreads();
    cta_moment_record<kSweepThreads / 32, false>(s_m, s_s, nullptr, P.ess_parts + blockIdx.x);
    }
    if (active) {
        R* xw = reinterpret_cast<R*>(P.x[b]);
        R* gw = reinterpret_cast<R*>(P.gl[b]);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if (i < d) {
                xw[(size_t)i * P.N + n64] = x[i];
                if (GRAD) gw[(size_t)i * P.N + n64] = gl[i];
            }
        }
        P.ell[b][n64] = (double)ell;
        P.logw[n64] = logw;
        if (!admissible(logw) || !admissible((double)ell)) atomicOr(P.status, 1u);
    }
}

// The potential on its own: log L(x_n) and, if asked, grad_x log L(x_n) for a batch of
// states x [d][N] (the forward and backward of the likelihood used by MALA and HMC).
struct PotentialParams {
    int64_t N;
    const void* x;        // [d][N] element type R
    double* ell;          // [N]
    void* grad;           // [d][N] element type R, or nullptr
};

template <class Tgt, int D, typename R>
__global__ void __launch_bounds__(kSweepThreads)
potential_kernel(const PotentialParams P, Tgt tg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    tg.setup(smem);
    const int d = tg.d;
    const int64_t n64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = n64 < P.N;
    const int64_t idx = active ? n64 : P.N - 1;
    const R* xs = reinterpret_cast<const R*>(P.x);
    R x[D], g[D];
#pragma unroll
    for (int i = 0; i < D; ++i) { x[i] = i < d ? xs[(size_t)i * P.N + idx] : R(0); g[i] = R(0); }
    // all threads take the same branch (cooperative evaluation)
    const R ell = P.grad ? tg.template eval<true>(x, g) : tg.template eval<false>(x, g);
    if (active) {
        P.ell[n64] = (double)ell;
        if (P.grad) {
            R* gw = reinterpret_cast<R*>(P.grad);
#pragma unroll
            for (int i = 0; i < D; ++i) if (i < d) gw[(size_t)i * P.N + n64] = g[i];
        }
    }
}

// t = 0 of Alg. 1: X_0 ~ eta, w_0 = 1, cached log L and its gradient, into buffer 0.
template <class Tgt, int MOVE, int D, typename R>
__global__ void __launch_bounds__(kSweepThreads)
asmc_init_kernel(const StepParams P, Tgt tg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool GRAD = (MOVE != kRwmh);
    tg.setup(smem);
    const int d = tg.d;
    const int64_t n64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = n64 < P.N;
    const uint32_t n = (uint32_t)(active ? n64 : P.N - 1);
    const R s = (R)P.ref_scale;
    R x[D], gl[D];
    normals<D>(P.mv.rng, n, 0u, 0u, d, x);
#pragma unroll
    for (int i = 0; i < D; ++i) { x[i] *= s; gl[i] = R(0); }
    const R ell = tg.template eval<GRAD>(x, gl);
    if (active) {
        R* xw = reinterpret_cast<R*>(P.x[0]);
        R* gw = reinterpret_cast<R*>(P.gl[0]);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if (i < d) {
                xw[(size_t)i * P.N + n64] = x[i];
                if (GRAD) gw[(size_t)i * P.N + n64] = gl[i];
            }
        }
        P.ell[0][n64] = (double)ell;
        P.logw[n64] = 0.0;
    }
}

} // namespace oais
