/*
 * oais_oracle.c -- plain FP64 CPU oracle for annealed SMC / AIS and the
 * round-based schedule optimisation of Syed, Bouchard-Cote, Chern and Doucet,
 * "Optimised Annealed Sequential Monte Carlo Samplers" (arXiv 2408.12057).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker for the CUDA
 * path: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA library; its random numbers come from its own
 * Philox4x32-10 written from the published definition (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *
 * Everything is double precision and written to be read against the paper:
 *   - Alg. 1 (ASMC) in its printed order, time loop outside, particles inside;
 *   - incremental weight of an MCMC forward kernel, g = gamma_b'(x)/gamma_b(x)
 *     evaluated at the pre-move state (Sec. 2.1.2, quasi-reversal backward kernel);
 *   - moments g_hat_{t,i} = sum_n w_{t-1}^n (g_t^n)^i, i = 0,1,2 (Alg. 1, Sec. 5.1.1),
 *     kept as logarithms: log g_hat_{t,i} = LSE_n(log w_{t-1}^n + i log g_t^n);
 *   - Z_hat = prod_r (1/N) sum_n w^n_{tau_r^-} (eq. estimator_Z), as a log;
 *   - ESS = (sum w)^2 / sum w^2 (eq. sample_size_IS) and adaptive resampling;
 *   - systematic resampling (Sec. 2.1.3);
 *   - OptimiseSchedule (Alg. 3): D_hat, Lambda_hat, monotone interpolation.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - Counter layout of the random numbers, the uniform map u = ((r>>9)+0.5)2^-23
 *     and Box-Muller normals;
 *   - MH acceptance iff log u < log alpha (strict);
 *   - systematic resampling a^n = min{m : C_m > (n+U)/N}, C the inclusive
 *     cumulative normalised weights;
 *   - "monotone spline" = piecewise cubic Hermite with Fritsch-Carlson
 *     (harmonic-mean) slopes and three-point one-sided end slopes;
 *   - D_hat clamped at 0, knots with equal Lambda_hat dropped (first kept).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 3; known-answer vectors in the tests)     */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u;   /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Counter layout: (particle n, step t, (move k << 16) | block j, tag).
 * tag = round | (problem << 16).  Key = the two halves of the 64-bit seed. */
static void rng_block(uint64_t seed, uint32_t n, uint32_t t, uint32_t k, uint32_t j,
                      uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4] = {n, t, (k << 16) | (j & 0xFFFFu), tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

double orc_u01(uint32_t r) { return ((double)(r >> 9) + 0.5) * (1.0 / 8388608.0); }

/* d standard normals for (n, t, k): block j gives z[4j..4j+3] by two Box-Muller pairs. */
void orc_normals(uint64_t seed, uint32_t n, uint32_t t, uint32_t k, uint32_t tag, int d, double* z)
{
    for (int j = 0; 4 * j < d; ++j) {
        uint32_t r[4];
        rng_block(seed, n, t, k, (uint32_t)j, tag, r);
        double rad0 = sqrt(-2.0 * log(orc_u01(r[0])));
        double ang0 = 2.0 * ORC_PI * orc_u01(r[1]);
        double rad1 = sqrt(-2.0 * log(orc_u01(r[2])));
        double ang1 = 2.0 * ORC_PI * orc_u01(r[3]);
        double v[4] = {rad0 * cos(ang0), rad0 * sin(ang0), rad1 * cos(ang1), rad1 * sin(ang1)};
        for (int q = 0; q < 4 && 4 * j + q < d; ++q) z[4 * j + q] = v[q];
    }
}

/* the uniform of the Metropolis-Hastings test of move k at step t */
double orc_mh_uniform(uint64_t seed, uint32_t n, uint32_t t, uint32_t k, uint32_t tag)
{
    uint32_t r[4];
    rng_block(seed, n, t, k, 0xFFFFu, tag, r);
    return orc_u01(r[0]);
}

/* the uniform of a systematic resampling event at step t */
double orc_resample_uniform(uint64_t seed, uint32_t t, uint32_t tag)
{
    uint32_t r[4];
    uint32_t ctr[4] = {0xFFFFFFFFu, t, 0u, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, r);
    return orc_u01(r[0]);
}

/* ------------------------------------------------------------------ */
/* Targets: path gamma_beta = eta^(1-beta) gamma^beta = eta * L^beta     */
/* (Sec. 2, geometric path), with eta = N(0, s^2 I) and gamma = eta * L. */
/* ------------------------------------------------------------------ */
enum { ORC_GAUSS = 0, ORC_LOGREG = 1, ORC_GMM = 2, ORC_LINREG = 3, ORC_UNID = 4 };

typedef struct {
    int kind;
    int d;            /* state dimension */
    int n;            /* data rows (LOGREG, LINREG) or mixture components (GMM) */
    const double* X;  /* LOGREG/LINREG: n x d row-major; GMM: n x d means; GAUSS: mu (d);
                         UNID: (m, k) trials and successes */
    const double* y;  /* LOGREG: labels in {0,1}; LINREG: responses */
    double ref_scale; /* s: eta = N(0, s^2 I) */
    double p0;        /* GAUSS: sigma of the likelihood; GMM: component variance; LINREG: noise sigma;
                         UNID: upper end b of the uniform priors */
} orc_target;

/* log of the binomial probability of k successes in m trials at the success rate k/m:
 * log C(m, k) + k log(k/m) + (m - k) log(1 - k/m).  Log-gamma for moderate counts; for
 * counts of a million and more Stirling's series (each log-gamma expanded to its 1/(12x)
 * term, the rest O(1/min(k, m-k)^3)), which keeps the O(1) result free of the cancellation
 * of terms of size m log m. */
double orc_binom_mode_logpmf(double m, double k)
{
    const double q = k / m;
    if (k < 1e6 || m - k < 1e6)
        return lgamma(m + 1.0) - lgamma(k + 1.0) - lgamma(m - k + 1.0) + k * log(q) + (m - k) * log1p(-q);
    return -0.5 * log(2.0 * ORC_PI * m * q * (1.0 - q)) + 1.0 / (12.0 * m) - 1.0 / (12.0 * k) -
           1.0 / (12.0 * (m - k));
}

static double std_normal_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

static double dot(const double* a, const double* b, int d)
{
    double acc = 0.0;
    for (int i = 0; i < d; ++i) acc += a[i] * b[i];
    return acc;
}

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigmoid(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

double orc_log_ref(const orc_target* tg, const double* x)
{
    double s2 = tg->ref_scale * tg->ref_scale;
    return -0.5 * tg->d * log(2.0 * ORC_PI * s2) - 0.5 * dot(x, x, tg->d) / s2;
}

/* log L(x); if grad != NULL also grad_x log L(x) */
double orc_log_lik(const orc_target* tg, const double* x, double* grad)
{
    const int d = tg->d, n = tg->n;
    if (grad) for (int i = 0; i < d; ++i) grad[i] = 0.0;
    switch (tg->kind) {
    case ORC_GAUSS: {
        double sig2 = tg->p0 * tg->p0, acc = 0.0;
        for (int i = 0; i < d; ++i) {
            double r = x[i] - tg->X[i];
            acc += r * r;
            if (grad) grad[i] = -r / sig2;
        }
        return -0.5 * acc / sig2;
    }
    case ORC_LOGREG: {
        double acc = 0.0;
        for (int r = 0; r < n; ++r) {
            const double* xr = tg->X + (size_t)r * d;
            double z = dot(xr, x, d);
            acc += tg->y[r] * z - softplus(z);
            if (grad) {
                double res = tg->y[r] - sigmoid(z);
                for (int i = 0; i < d; ++i) grad[i] += res * xr[i];
            }
        }
        return acc;
    }
    case ORC_GMM: {
        /* log p(x) with p = (1/K) sum_k N(x; mu_k, v I); L = p / eta */
        double v = tg->p0;
        double* lk = (double*)malloc(sizeof(double) * n);
        double mx = -INFINITY;
        for (int k = 0; k < n; ++k) {
            const double* mu = tg->X + (size_t)k * d;
            double q = 0.0;
            for (int i = 0; i < d; ++i) { double r = x[i] - mu[i]; q += r * r; }
            lk[k] = -0.5 * d * log(2.0 * ORC_PI * v) - 0.5 * q / v;
            if (lk[k] > mx) mx = lk[k];
        }
        double sum = 0.0;
        for (int k = 0; k < n; ++k) sum += exp(lk[k] - mx);
        double logp = mx + log(sum) - log((double)n);
        if (grad) {
            for (int k = 0; k < n; ++k) {
                double resp = exp(lk[k] - mx) / sum;
                const double* mu = tg->X + (size_t)k * d;
                for (int i = 0; i < d; ++i) grad[i] += resp * (mu[i] - x[i]) / v;
            }
            double s2 = tg->ref_scale * tg->ref_scale;
            for (int i = 0; i < d; ++i) grad[i] += x[i] / s2;
        }
        free(lk);
        return logp - orc_log_ref(tg, x);
    }
    case ORC_LINREG: {
        double sig2 = tg->p0 * tg->p0, acc = 0.0;
        for (int r = 0; r < n; ++r) {
            const double* xr = tg->X + (size_t)r * d;
            double res = tg->y[r] - dot(xr, x, d);
            acc += res * res;
            if (grad) for (int i = 0; i < d; ++i) grad[i] += res * xr[i] / sig2;
        }
        return -0.5 * n * log(2.0 * ORC_PI * sig2) - 0.5 * acc / sig2;
    }
    case ORC_UNID: {
        /* the unidentifiable product model (the paper's model appendix, its GPU workload
         * "Unid"): X, Y ~ Uniform(0, b), K ~ Binomial(m, X Y).  State z in R^2 under N(0, I),
         * X = b Phi(z_1), Y = b Phi(z_2).  log L = log Binom(k; m, p), p = X Y, -inf outside
         * (0, 1); by the identity log Binom(k; m, p) = log Binom(k; m, q) - m D(q || p), q = k/m,
         * D(q || p) = q log(q/p) + (1 - q) log((1 - q)/(1 - p)) the Bernoulli KL divergence
         * (written with log1p of the relative differences). */
        const double m = tg->X[0], k = tg->X[1], b = tg->p0, q = k / m;
        const double u1 = std_normal_cdf(x[0]), u2 = std_normal_cdf(x[1]);
        const double p = b * b * u1 * u2;
        if (!(p > 0.0 && p < 1.0)) return -INFINITY;
        const double D = -q * log1p((p - q) / q) - (1.0 - q) * log1p((q - p) / (1.0 - q));
        if (grad) {
            const double dldp = k / p - (m - k) / (1.0 - p);
            const double phi1 = exp(-0.5 * x[0] * x[0]) / sqrt(2.0 * ORC_PI);
            const double phi2 = exp(-0.5 * x[1] * x[1]) / sqrt(2.0 * ORC_PI);
            grad[0] = dldp * b * b * phi1 * u2;
            grad[1] = dldp * b * b * u1 * phi2;
        }
        return orc_binom_mode_logpmf(m, k) - m * D;
    }
    }
    return NAN;
}

/* log pi_beta up to its normaliser, and its gradient: log eta + beta log L */
static double log_tempered(const orc_target* tg, double beta, const double* x, double ell,
                           const double* gell, double* g_out)
{
    double s2 = tg->ref_scale * tg->ref_scale;
    if (g_out) for (int i = 0; i < tg->d; ++i) g_out[i] = -x[i] / s2 + beta * gell[i];
    return orc_log_ref(tg, x) + beta * ell;
}

/* ------------------------------------------------------------------ */
/* MCMC forward kernels K_beta targeting pi_beta (Sec. 2.1.1)            */
/* ------------------------------------------------------------------ */
enum { ORC_RWMH = 0, ORC_MALA = 1, ORC_HMC = 2, ORC_EXACT = 3 };

typedef struct {
    int kind;
    int moves;      /* K moves per annealing step */
    int leapfrog;   /* HMC leapfrog steps */
    int cycle;      /* RWMH only: cycle proposal std over {0.1, 1, 10} by global move index */
} orc_move;

typedef struct {
    double* x;      /* d */
    double ell;     /* log L(x) */
    double* gell;   /* grad log L(x), d (MALA/HMC) */
} particle_ref;

/* one MH move; returns 1 if accepted. margin = |log u - log alpha|. */
static int mh_move(const orc_target* tg, const orc_move* mv, double beta, double eps,
                   uint64_t seed, uint32_t n, uint32_t t, uint32_t k, uint32_t tag,
                   int global_move, particle_ref* p, double* margin, double* work)
{
    const int d = tg->d;
    double* z = work;            /* d */
    double* xp = work + d;       /* d */
    double* gp = work + 2 * d;   /* d: grad log L at proposal */
    double* gpi = work + 3 * d;  /* d: grad log pi at current */
    double* gpip = work + 4 * d; /* d: grad log pi at proposal */
    double* mom = work + 5 * d;  /* d: HMC momentum */
    double log_alpha, ellp;
    int need_grad = (mv->kind == ORC_MALA || mv->kind == ORC_HMC);

    orc_normals(seed, n, t, k, tag, d, z);
    if (mv->kind == ORC_EXACT) {
        /* GAUSS family only: pi_beta is N(m, v I) with precision 1/s^2 + beta/sigma^2;
         * an exact draw makes Assumptions 2-4 (temporal and particle independence,
         * efficient local exploration) hold exactly. */
        double prec = 1.0 / (tg->ref_scale * tg->ref_scale) + beta / (tg->p0 * tg->p0);
        for (int i = 0; i < d; ++i)
            p->x[i] = (beta / (tg->p0 * tg->p0)) * tg->X[i] / prec + z[i] / sqrt(prec);
        p->ell = orc_log_lik(tg, p->x, p->gell);
        return 1;
    }
    if (mv->kind == ORC_RWMH) {
        double sd = eps;
        if (mv->cycle) {
            static const double cyc[3] = {0.1, 1.0, 10.0};
            sd = cyc[global_move % 3];
        }
        for (int i = 0; i < d; ++i) xp[i] = p->x[i] + sd * z[i];
        ellp = orc_log_lik(tg, xp, NULL);
        log_alpha = log_tempered(tg, beta, xp, ellp, NULL, NULL)
                  - log_tempered(tg, beta, p->x, p->ell, NULL, NULL);
    } else if (mv->kind == ORC_MALA) {
        /* x' = x + (eps^2/2) grad log pi(x) + eps z;  q(a|b) = N(a; b + (eps^2/2) grad log pi(b), eps^2 I) */
        double h = 0.5 * eps * eps;
        log_tempered(tg, beta, p->x, p->ell, p->gell, gpi);
        for (int i = 0; i < d; ++i) xp[i] = p->x[i] + h * gpi[i] + eps * z[i];
        ellp = orc_log_lik(tg, xp, gp);
        double lp_new = log_tempered(tg, beta, xp, ellp, gp, gpip);
        double lp_old = log_tempered(tg, beta, p->x, p->ell, NULL, NULL);
        double fwd = 0.0, rev = 0.0;
        for (int i = 0; i < d; ++i) {
            double a = xp[i] - p->x[i] - h * gpi[i];
            double b = p->x[i] - xp[i] - h * gpip[i];
            fwd += a * a;
            rev += b * b;
        }
        log_alpha = lp_new - lp_old - (rev - fwd) / (2.0 * eps * eps);
    } else {
        /* HMC, identity mass, leapfrog of `leapfrog` steps of size eps */
        for (int i = 0; i < d; ++i) { mom[i] = z[i]; xp[i] = p->x[i]; }
        double ke0 = 0.5 * dot(mom, mom, d);
        double lp_old = log_tempered(tg, beta, p->x, p->ell, p->gell, gpi);
        for (int i = 0; i < d; ++i) mom[i] += 0.5 * eps * gpi[i];
        ellp = p->ell;
        for (int l = 0; l < mv->leapfrog; ++l) {
            for (int i = 0; i < d; ++i) xp[i] += eps * mom[i];
            ellp = orc_log_lik(tg, xp, gp);
            log_tempered(tg, beta, xp, ellp, gp, gpip);
            double f = (l + 1 < mv->leapfrog) ? eps : 0.5 * eps;
            for (int i = 0; i < d; ++i) mom[i] += f * gpip[i];
        }
        double lp_new = log_tempered(tg, beta, xp, ellp, NULL, NULL);
        double ke1 = 0.5 * dot(mom, mom, d);
        log_alpha = (lp_new - ke1) - (lp_old - ke0);
    }
    double logu = log(orc_mh_uniform(seed, n, t, k, tag));
    double m = fabs(logu - log_alpha);
    if (!isnan(*margin) && !(m >= *margin)) *margin = m;   /* a NaN margin sticks */
    if (logu < log_alpha) {
        memcpy(p->x, xp, sizeof(double) * d);
        p->ell = ellp;
        if (need_grad) memcpy(p->gell, gp, sizeof(double) * d);
        return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* log-sum-exp of a[0..n): the plain definition with a max shift         */
/* ------------------------------------------------------------------ */
double orc_logsumexp(const double* a, long n)
{
    double mx = -INFINITY;
    for (long i = 0; i < n; ++i) if (a[i] > mx) mx = a[i];
    if (!isfinite(mx)) return mx;
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += exp(a[i] - mx);
    return mx + log(s);
}

/* Systematic resampling (Sec. 2.1.3): normalised weights W from log w,
 * inclusive cumulative sums C, ancestor a^n = min{m : C_m > (n + U)/N}. */
void orc_systematic_resample(long N, const double* logw, double U, int64_t* anc)
{
    double lse = orc_logsumexp(logw, N);
    double* C = (double*)malloc(sizeof(double) * N);
    double acc = 0.0;
    for (long m = 0; m < N; ++m) { acc += exp(logw[m] - lse); C[m] = acc; }
    long m = 0;
    for (long n = 0; n < N; ++n) {
        double thr = ((double)n + U) / (double)N;
        while (m < N - 1 && !(C[m] > thr)) ++m;
        anc[n] = m;
    }
    free(C);
}

/* ------------------------------------------------------------------ */
/* Alg. 1: ASMC(N, B_T).  ess_frac = 0 gives AIS (one resampling time at   */
/* T, i.e. no intermediate resampling); ess_frac in (0,1] gives adaptive  */
/* resampling with threshold nu = ess_frac (eq. sample_size_IS).            */
/* ------------------------------------------------------------------ */
typedef struct {
    double logZ;
    int n_resample;
} orc_result;

int orc_asmc(const orc_target* tg, const orc_move* mv, long N, int T, const double* beta,
             const double* eps /* T per-step sizes */, uint64_t seed, uint32_t tag,
             long n_offset /* particle n uses counter n_offset + n */, double ess_frac,
             /* outputs (any may be NULL except res) */
             orc_result* res, double* log_ghat /* T x 3 */, double* accept /* T */,
             double* ess_trace /* T */, double* logw_out /* N */, double* x_out /* N x d */,
             double* ell_out /* N */, double* margin_out /* N */, int64_t* resample_steps /* T */,
             double* elbo_t /* T */, int64_t* anc_out /* N: ancestors of the last intermediate event */)
{
    const int d = tg->d;
    int need_grad = (mv->kind != ORC_RWMH);   /* EXACT keeps the gradient too (cheap) */
    double* X = (double*)malloc(sizeof(double) * N * d);
    double* G = (double*)malloc(sizeof(double) * N * d);
    double* ell = (double*)malloc(sizeof(double) * N);
    double* logw = (double*)malloc(sizeof(double) * N);
    double* logg = (double*)malloc(sizeof(double) * N);
    double* tmp = (double*)malloc(sizeof(double) * N);
    double* margin = (double*)malloc(sizeof(double) * N);
    int* acc_count = (int*)malloc(sizeof(int) * N);
    if (!X || !G || !ell || !logw || !logg || !tmp || !margin || !acc_count) return -1;

    /* t = 0: X_0^n ~ eta, w_0^n = 1 */
    for (long n = 0; n < N; ++n) {
        orc_normals(seed, (uint32_t)(n_offset + n), 0u, 0u, tag, d, X + n * d);
        for (int i = 0; i < d; ++i) X[n * d + i] *= tg->ref_scale;
        ell[n] = orc_log_lik(tg, X + n * d, need_grad ? G + n * d : NULL);
        logw[n] = 0.0;
        margin[n] = INFINITY;
    }
    double logZ = 0.0;
    int n_res = 0;

    for (int t = 1; t <= T; ++t) {
        double db = beta[t] - beta[t - 1];
        /* g_t^n = gamma_{beta_t}(X_{t-1}^n) / gamma_{beta_{t-1}}(X_{t-1}^n) = L(X_{t-1}^n)^(db) */
        /* L^0 = 1, also where L = 0 (a state outside the support) */
        for (long n = 0; n < N; ++n) logg[n] = db == 0.0 ? 0.0 : db * ell[n];
        /* moments g_hat_{t,i} = sum_n w_{t-1}^n (g_t^n)^i, as logarithms */
        if (log_ghat) {
            for (int i = 0; i < 3; ++i) {
                for (long n = 0; n < N; ++n) tmp[n] = i == 0 ? logw[n] : logw[n] + i * logg[n];
                log_ghat[(size_t)(t - 1) * 3 + i] = orc_logsumexp(tmp, N);
            }
        }
        /* ELBO term of step t (the estimator of the section on the KL divergence of a schedule):
           sum_n W_{t-1}^n log g_t^n, W_{t-1}^n = w_{t-1}^n / sum_m w_{t-1}^m the normalised
           weights (since the last resampling) */
        if (elbo_t) {
            const double lse = orc_logsumexp(logw, N);
            double e = 0.0;
            for (long n = 0; n < N; ++n) {
                const double W = exp(logw[n] - lse);
                if (W > 0.0) e += W * logg[n];   /* a zero weight adds nothing, even with g = 0 */
            }
            elbo_t[t - 1] = e;
        }
        /* reweight: w_{t^-} = w_{t-1} g_t */
        for (long n = 0; n < N; ++n) logw[n] += logg[n];
        /* propagate: K moves of the pi_{beta_t}-invariant kernel */
        #pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            double work[6 * 512];
            double* wk = (d <= 512) ? work : (double*)malloc(sizeof(double) * 6 * d);
            particle_ref p = {X + n * d, ell[n], G + n * d};
            int a = 0;
            for (int k = 0; k < mv->moves; ++k)
                a += mh_move(tg, mv, beta[t], eps[t - 1], seed, (uint32_t)(n_offset + n), (uint32_t)t,
                             (uint32_t)k, tag, (t - 1) * mv->moves + k, &p, &margin[n], wk);
            ell[n] = p.ell;
            acc_count[n] = a;
            if (wk != work) free(wk);
        }
        if (accept) {
            double s = 0.0;
            for (long n = 0; n < N; ++n) s += acc_count[n];
            accept[t - 1] = s / ((double)N * mv->moves);
        }
        /* ESS of w_{t^-} */
        double lse1 = orc_logsumexp(logw, N);
        for (long n = 0; n < N; ++n) tmp[n] = 2.0 * logw[n];
        double lse2 = orc_logsumexp(tmp, N);
        double ess = exp(2.0 * lse1 - lse2);
        if (ess_trace) ess_trace[t - 1] = ess;
        int resample = (t == T) || (ess_frac > 0.0 && ess < ess_frac * (double)N);
        if (resample) {
            /* Z_hat <- Z_hat * (1/N) sum_n w_{t^-}^n */
            logZ += lse1 - log((double)N);
            if (resample_steps) resample_steps[t - 1] = 1;
            if (t < T) {
                ++n_res;
                int64_t* anc = (int64_t*)malloc(sizeof(int64_t) * N);
                orc_systematic_resample(N, logw, orc_resample_uniform(seed, (uint32_t)t, tag), anc);
                double* X2 = (double*)malloc(sizeof(double) * N * d);
                double* G2 = (double*)malloc(sizeof(double) * N * d);
                double* e2 = (double*)malloc(sizeof(double) * N);
                double* m2 = (double*)malloc(sizeof(double) * N);
                for (long n = 0; n < N; ++n) {
                    memcpy(X2 + n * d, X + anc[n] * d, sizeof(double) * d);
                    memcpy(G2 + n * d, G + anc[n] * d, sizeof(double) * d);
                    e2[n] = ell[anc[n]];
                    m2[n] = margin[anc[n]];
                }
                memcpy(X, X2, sizeof(double) * N * d);
                memcpy(G, G2, sizeof(double) * N * d);
                memcpy(ell, e2, sizeof(double) * N);
                memcpy(margin, m2, sizeof(double) * N);
                for (long n = 0; n < N; ++n) logw[n] = 0.0;   /* w_t^n = 1 */
                if (anc_out) memcpy(anc_out, anc, sizeof(int64_t) * N);
                free(anc); free(X2); free(G2); free(e2); free(m2);
            }
        } else if (resample_steps) {
            resample_steps[t - 1] = 0;
        }
    }
    res->logZ = logZ;
    res->n_resample = n_res;
    if (logw_out) memcpy(logw_out, logw, sizeof(double) * N);
    if (x_out) memcpy(x_out, X, sizeof(double) * N * d);
    if (ell_out) memcpy(ell_out, ell, sizeof(double) * N);
    if (margin_out) memcpy(margin_out, margin, sizeof(double) * N);
    free(X); free(G); free(ell); free(logw); free(logg); free(tmp); free(margin); free(acc_count);
    return 0;
}

/* ------------------------------------------------------------------ */
/* The online conditional-ESS schedule of Zhou, Johansen & Aston (2016), */
/* the comparator of the section on the connection to online CESS        */
/* optimisation: before step t, beta_t is chosen so that                  */
/* CESS_t / N = (sum W g)^2 / (sum W g^2) = cess_frac, g = L^(beta_t -    */
/* beta_{t-1}), W the normalised weights since the last resampling.       */
/* Line search (a reading): the geometric candidates hi 4^-(32-j),       */
/* j = 1..32, hi = 1 - beta_{t-1}, keeping the last one that meets the    */
/* target, then five passes over 32 equally spaced candidates of the      */
/* bracket it ends in; the step is the final lower end, the whole interval */
/* when its end meets the target, the smallest geometric candidate when   */
/* none does (steps of at least 1e-14).  The target is relative to the   */
/* weight share A inside the likelihood's support: CESS/N >= c A (A = 1   */
/* unless weighted states have L = 0).  The candidates are fp64 values.   */
/* Step sizes: log eps interpolated linearly in beta                      */
/* through the points (beta_ref[t], eps_ref[t-1]), constant beyond.        */
/* Then the ASMC step of orc_asmc; the step with beta_t = 1 (forced at     */
/* t = T_max) closes the last segment.                                    */
/* ------------------------------------------------------------------ */
static double lse_shift(const double* lw, const double* ell, double k, double delta, long N)
{
    /* log sum_n exp(lw_n + k delta ell_n), zero weights and (k > 0) zero likelihoods skipped */
    double mx = -INFINITY;
    for (long n = 0; n < N; ++n) {
        if (lw[n] == -INFINITY || (k > 0.0 && ell[n] == -INFINITY)) continue;
        const double v = k > 0.0 ? lw[n] + k * delta * ell[n] : lw[n];
        if (v > mx) mx = v;
    }
    if (mx == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (long n = 0; n < N; ++n) {
        if (lw[n] == -INFINITY || (k > 0.0 && ell[n] == -INFINITY)) continue;
        s += exp((k > 0.0 ? lw[n] + k * delta * ell[n] : lw[n]) - mx);
    }
    return mx + log(s);
}

static double zja_step_size(double b, const double* beta_ref, const double* eps_ref, int T_ref)
{
    if (T_ref <= 1 || b <= beta_ref[1]) return eps_ref[0];
    if (b >= beta_ref[T_ref]) return eps_ref[T_ref - 1];
    int t = 1;
    while (t + 1 < T_ref && beta_ref[t + 1] <= b) ++t;
    const double u = (b - beta_ref[t]) / (beta_ref[t + 1] - beta_ref[t]);
    return exp(log(eps_ref[t - 1]) + u * (log(eps_ref[t]) - log(eps_ref[t - 1])));
}

/* Candidate j (1..32) of a pass of the line search (a reading; the paper fixes only the CESS
 * target): geometric in pass 0, hi 4^-(32 - j); equally spaced in the bracket after,
 * lo + ((hi - lo) j) / 32.  Plain fp64 arithmetic, rounded to nearest at every operation
 * (the oracle is built without contraction), so the grid is defined exactly. */
static double zja_candidate(int pass, double lo, double hi, int j)
{
    return pass == 0 ? ldexp(hi, -2 * (32 - j)) : lo + ((hi - lo) * (double)j) * (1.0 / 32.0);
}

/* the next annealing parameter from the particles' log-weights and log-likelihoods */

double orc_zja_next_beta(long N, const double* logw, const double* ell, double beta_prev, double cess_frac,
                         int t, int T_max)
{
    double lo = 0.0, hi = 1.0 - beta_prev, delta = 0.0;
    /* the target relative to the weight share A inside the support (CESS -> A as the step
       -> 0+: weighted states with L = 0 are lost at any positive step) */
    const double l0 = lse_shift(logw, ell, 0.0, 0.0, N);
    const double la = lse_shift(logw, ell, 1.0, 0.0, N);
    const double lt = log(cess_frac) + la - l0;
    for (int pass = 0; pass < 6; ++pass) {
        int best = 0;
        for (int j = 1; j <= 32; ++j) {
            const double dj = zja_candidate(pass, lo, hi, j);
            const double ratio = 2.0 * lse_shift(logw, ell, 1.0, dj, N) - l0 - lse_shift(logw, ell, 2.0, dj, N);
            if (ratio >= lt) best = j;
        }
        if (best == 32) { delta = hi; break; }
        if (best == 0 && pass == 0) { delta = zja_candidate(0, lo, hi, 1); break; }
        const double nlo = best > 0 ? zja_candidate(pass, lo, hi, best) : lo;
        const double nhi = zja_candidate(pass, lo, hi, best + 1);
        if (pass == 5) { delta = nlo; break; }
        lo = nlo;
        hi = nhi;
    }
    if (delta < 1e-14 && hi > 1e-14) delta = 1e-14;   /* every step advances beta */
    double bt = beta_prev + delta;
    if (bt >= 1.0 - 1e-12 || t >= T_max) bt = 1.0;
    return bt;
}

int orc_zja(const orc_target* tg, const orc_move* mv, long N, int T_max, const double* beta_ref,
            const double* eps_ref, int T_ref, double cess_frac, double ess_frac, uint64_t seed, uint32_t tag,
            /* outputs */
            orc_result* res, int* T_out, double* beta /* T_max + 1 */, double* eps /* T_max */,
            double* log_ghat /* T_max x 3 */, double* logw_out /* N */, double* x_out /* N x d */,
            double* ell_out /* N */, double* margin_out /* N */, double* elbo_t /* T_max */)
{
    const int d = tg->d;
    int need_grad = (mv->kind != ORC_RWMH);
    double* X = (double*)malloc(sizeof(double) * N * d);
    double* G = (double*)malloc(sizeof(double) * N * d);
    double* ell = (double*)malloc(sizeof(double) * N);
    double* logw = (double*)malloc(sizeof(double) * N);
    double* logg = (double*)malloc(sizeof(double) * N);
    double* tmp = (double*)malloc(sizeof(double) * N);
    double* margin = (double*)malloc(sizeof(double) * N);
    if (!X || !G || !ell || !logw || !logg || !tmp || !margin) return -1;
    for (long n = 0; n < N; ++n) {
        orc_normals(seed, (uint32_t)n, 0u, 0u, tag, d, X + n * d);
        for (int i = 0; i < d; ++i) X[n * d + i] *= tg->ref_scale;
        ell[n] = orc_log_lik(tg, X + n * d, need_grad ? G + n * d : NULL);
        logw[n] = 0.0;
        margin[n] = INFINITY;
    }
    double logZ = 0.0;
    int n_res = 0, T = 0;
    beta[0] = 0.0;
    for (int t = 1; t <= T_max; ++t) {
        beta[t] = orc_zja_next_beta(N, logw, ell, beta[t - 1], cess_frac, t, T_max);
        eps[t - 1] = zja_step_size(beta[t], beta_ref, eps_ref, T_ref);
        const double db = beta[t] - beta[t - 1];
        for (long n = 0; n < N; ++n) logg[n] = db == 0.0 ? 0.0 : db * ell[n];
        if (log_ghat) {
            for (int i = 0; i < 3; ++i) {
                for (long n = 0; n < N; ++n) tmp[n] = i == 0 ? logw[n] : logw[n] + i * logg[n];
                log_ghat[(size_t)(t - 1) * 3 + i] = orc_logsumexp(tmp, N);
            }
        }
        if (elbo_t) {
            const double lse = orc_logsumexp(logw, N);
            double e = 0.0;
            for (long n = 0; n < N; ++n) {
                const double W = exp(logw[n] - lse);
                if (W > 0.0) e += W * logg[n];
            }
            elbo_t[t - 1] = e;
        }
        for (long n = 0; n < N; ++n) logw[n] += logg[n];
        #pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            double work[6 * 512];
            double* wk = (d <= 512) ? work : (double*)malloc(sizeof(double) * 6 * d);
            particle_ref p = {X + n * d, ell[n], G + n * d};
            for (int k = 0; k < mv->moves; ++k)
                mh_move(tg, mv, beta[t], eps[t - 1], seed, (uint32_t)n, (uint32_t)t, (uint32_t)k, tag,
                        (t - 1) * mv->moves + k, &p, &margin[n], wk);
            ell[n] = p.ell;
            if (wk != work) free(wk);
        }
        const double lse1 = orc_logsumexp(logw, N);
        for (long n = 0; n < N; ++n) tmp[n] = 2.0 * logw[n];
        const double ess = exp(2.0 * lse1 - orc_logsumexp(tmp, N));
        const int last = beta[t] >= 1.0;
        T = t;
        if (last || (ess_frac > 0.0 && ess < ess_frac * (double)N)) {
            logZ += lse1 - log((double)N);
            if (!last) {
                ++n_res;
                int64_t* anc = (int64_t*)malloc(sizeof(int64_t) * N);
                orc_systematic_resample(N, logw, orc_resample_uniform(seed, (uint32_t)t, tag), anc);
                double* X2 = (double*)malloc(sizeof(double) * N * d);
                double* G2 = (double*)malloc(sizeof(double) * N * d);
                double* e2 = (double*)malloc(sizeof(double) * N);
                double* m2 = (double*)malloc(sizeof(double) * N);
                for (long n = 0; n < N; ++n) {
                    memcpy(X2 + n * d, X + anc[n] * d, sizeof(double) * d);
                    memcpy(G2 + n * d, G + anc[n] * d, sizeof(double) * d);
                    e2[n] = ell[anc[n]];
                    m2[n] = margin[anc[n]];
                }
                memcpy(X, X2, sizeof(double) * N * d);
                memcpy(G, G2, sizeof(double) * N * d);
                memcpy(ell, e2, sizeof(double) * N);
                memcpy(margin, m2, sizeof(double) * N);
                for (long n = 0; n < N; ++n) logw[n] = 0.0;
                free(anc); free(X2); free(G2); free(e2); free(m2);
            }
        }
        if (last) break;
    }
    res->logZ = logZ;
    res->n_resample = n_res;
    *T_out = T;
    if (logw_out) memcpy(logw_out, logw, sizeof(double) * N);
    if (x_out) memcpy(x_out, X, sizeof(double) * N * d);
    if (ell_out) memcpy(ell_out, ell, sizeof(double) * N);
    if (margin_out) memcpy(margin_out, margin, sizeof(double) * N);
    free(X); free(G); free(ell); free(logw); free(logg); free(tmp); free(margin);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Monotone piecewise cubic Hermite interpolation (Fritsch & Carlson,    */
/* SIAM J. Numer. Anal. 1980, with the harmonic-mean interior slopes of  */
/* Fritsch & Butland 1984 and three-point one-sided end slopes).          */
/* ------------------------------------------------------------------ */
static int sgn(double v) { return (v > 0) - (v < 0); }

static double end_slope(double h0, double h1, double m0, double m1)
{
    double s = ((2.0 * h0 + h1) * m0 - h0 * m1) / (h0 + h1);
    if (sgn(s) != sgn(m0)) return 0.0;
    if (sgn(m0) != sgn(m1) && fabs(s) > fabs(3.0 * m0)) return 3.0 * m0;
    return s;
}

void orc_pchip_slopes(int K, const double* xk, const double* yk, double* dk)
{
    if (K == 2) {
        double m = (yk[1] - yk[0]) / (xk[1] - xk[0]);
        dk[0] = dk[1] = m;
        return;
    }
    double* h = (double*)malloc(sizeof(double) * (K - 1));
    double* m = (double*)malloc(sizeof(double) * (K - 1));
    for (int i = 0; i < K - 1; ++i) { h[i] = xk[i + 1] - xk[i]; m[i] = (yk[i + 1] - yk[i]) / h[i]; }
    for (int i = 1; i < K - 1; ++i) {
        if (m[i - 1] == 0.0 || m[i] == 0.0 || sgn(m[i - 1]) != sgn(m[i])) {
            dk[i] = 0.0;
        } else {
            double w1 = 2.0 * h[i] + h[i - 1], w2 = h[i] + 2.0 * h[i - 1];
            dk[i] = (w1 + w2) / (w1 / m[i - 1] + w2 / m[i]);
        }
    }
    dk[0] = end_slope(h[0], h[1], m[0], m[1]);
    dk[K - 1] = end_slope(h[K - 2], h[K - 3], m[K - 2], m[K - 3]);
    free(h); free(m);
}

double orc_pchip_eval(int K, const double* xk, const double* yk, const double* dk, double x)
{
    int i = 0;
    if (x <= xk[0]) i = 0;
    else if (x >= xk[K - 1]) i = K - 2;
    else { int lo = 0, hi = K - 1; while (hi - lo > 1) { int mid = (lo + hi) / 2; if (xk[mid] <= x) lo = mid; else hi = mid; } i = lo; }
    double h = xk[i + 1] - xk[i];
    double s = (x - xk[i]) / h;
    double h00 = (1 + 2 * s) * (1 - s) * (1 - s), h10 = s * (1 - s) * (1 - s);
    double h01 = s * s * (3 - 2 * s), h11 = s * s * (s - 1);
    return h00 * yk[i] + h10 * h * dk[i] + h01 * yk[i + 1] + h11 * h * dk[i + 1];
}

/* Alg. 3 OptimiseSchedule(T', B_T, g_hat).  Outputs the new schedule (T'+1)
 * and, if requested, D_hat (T) and Lambda_hat (T+1). */
int orc_optimise_schedule(int T, const double* beta, const double* log_ghat, int Tn,
                          double* beta_new, double* D_hat_out, double* Lambda_out)
{
    double* Lam = (double*)malloc(sizeof(double) * (T + 1));
    double* kx = (double*)malloc(sizeof(double) * (T + 1));
    double* ky = (double*)malloc(sizeof(double) * (T + 1));
    double* kd = (double*)malloc(sizeof(double) * (T + 1));
    Lam[0] = 0.0;
    for (int t = 1; t <= T; ++t) {
        const double* g = log_ghat + (size_t)(t - 1) * 3;
        double D = g[2] - 2.0 * g[1] + g[0];      /* D_hat_t (eq. CESS) */
        if (!(D > 0.0)) D = 0.0;                  /* reading: clamp rounding negatives */
        if (D_hat_out) D_hat_out[t - 1] = D;
        Lam[t] = Lam[t - 1] + sqrt(D);            /* Lambda_hat_t */
    }
    if (Lambda_out) memcpy(Lambda_out, Lam, sizeof(double) * (T + 1));
    /* knots (Lambda_hat_t, beta_t), strictly increasing in Lambda_hat */
    int K = 0;
    for (int t = 0; t <= T; ++t) {
        if (K > 0 && !(Lam[t] > kx[K - 1])) continue;
        kx[K] = Lam[t]; ky[K] = beta[t]; ++K;
    }
    if (K >= 2) {
        /* the last knot must carry beta_T = 1 */
        ky[K - 1] = beta[T];
        orc_pchip_slopes(K, kx, ky, kd);
    }
    for (int tp = 0; tp <= Tn; ++tp) {
        double u = (double)tp / (double)Tn;
        if (K < 2) beta_new[tp] = u;             /* Lambda_hat_T = 0: uniform schedule */
        else beta_new[tp] = orc_pchip_eval(K, kx, ky, kd, Lam[T] * u);
    }
    beta_new[0] = 0.0;
    beta_new[Tn] = 1.0;
    free(Lam); free(kx); free(ky); free(kd);
    return 0;
}

/* Weighted expectation sum_n W^n f(X^n) of grad_theta log gamma(x; theta),
 * theta = (log s, log sigma) for LINREG (eta = N(0, s^2 I), noise sigma) and
 * theta = (log s, log sigma_L) for GAUSS -- the identity
 * grad log Z = E_pi[grad_theta log gamma] with the estimator of
 * eq. estimator_pi_t (final weights, final states). */
int orc_fisher_grad(const orc_target* tg, long N, const double* logw, const double* X,
                    double* grad /* 2 */)
{
    const int d = tg->d;
    double lse = orc_logsumexp(logw, N);
    double g0 = 0.0, g1 = 0.0;
    double s2 = tg->ref_scale * tg->ref_scale;
    for (long n = 0; n < N; ++n) {
        double W = exp(logw[n] - lse);
        const double* x = X + n * d;
        /* d/dlog s of log N(x; 0, s^2 I) = -d + |x|^2 / s^2 */
        double a = -d + dot(x, x, d) / s2;
        double b = 0.0;
        if (tg->kind == ORC_LINREG) {
            double sig2 = tg->p0 * tg->p0, acc = 0.0;
            for (int r = 0; r < tg->n; ++r) {
                double res = tg->y[r] - dot(tg->X + (size_t)r * d, x, d);
                acc += res * res;
            }
            b = -tg->n + acc / sig2;
        } else if (tg->kind == ORC_GAUSS) {
            double sig2 = tg->p0 * tg->p0, acc = 0.0;
            for (int i = 0; i < d; ++i) { double r = x[i] - tg->X[i]; acc += r * r; }
            b = acc / sig2;   /* d/dlog sigma_L of -|x-mu|^2/(2 sigma_L^2) */
        }
        g0 += W * a;
        g1 += W * b;
    }
    grad[0] = g0;
    grad[1] = g1;
    return 0;
}
