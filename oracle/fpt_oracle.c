/*
 * FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (see fpt_oracle.h).
 *
 * A plain transcription of the method of arXiv:2206.11234, §2: biased
 * Euler–Maruyama runs of a 1-D Langevin equation until first passage, with the
 * importance weight w = p_T / p_S accumulated step by step, and the binned
 * estimators of the first-passage-time density.  Nothing here is blocked,
 * fused or reordered; each function cites the passage it follows.
 *
 * Build: cc -O2 -fPIC -shared -ffp-contract=off -o liboracle.so fpt_oracle.c -lm
 * (contraction off so that every expression is rounded as written, on x86
 * and on Arm alike).
 */
#include "fpt_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdint.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11, §4: a 4-word counter is mixed with a 2-word key  */
/* by 10 rounds; each round multiplies words 0 and 2 by two fixed odd        */
/* constants (keeping both halves of the 64-bit products), XORs the high     */
/* halves into the other two words together with the round key, and         */
/* permutes; the round key is bumped by two Weyl constants between rounds.  */
/* (The RNG is a choice of this implementation: the paper only says each    */
/* xi_m is drawn from a unit normal, §2.1 below Eq. (8).)                     */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u /* golden ratio */
#define PHILOX_W1 0xBB67AE85u /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Box–Muller: two uniforms in (0, 1) give two independent unit normals,
 * r = sqrt(-2 ln u0), (r cos 2 pi u1, r sin 2 pi u1).  A 32-bit word w maps
 * to u = (w + 1/2) 2^-32 and a 16-bit field h to u = (h + 1/2) 2^-16; both are
 * exact in binary64 and never 0 or 1. */
static double uniform_open(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
static double uniform_open16(uint32_t h) { return ((double)h + 0.5) * 0x1p-16; }

/* Which Philox words feed which normals (the paper names no generator, §2.1
 * below Eq. (8); this assignment is a choice of the project, made the same way
 * on both sides).  Steps come in groups of sixteen: group G = k div 4 uses the
 * twelve words of the Philox counters (3G, id_lo, id_hi, set_id),
 * (3G + 1, ...), (3G + 2, ...), taken in that order.  The four steps of block
 * k (steps 4k .. 4k+3) use words 3j, 3j + 1 and 3j + 2 of the twelve, with
 * j = k mod 4: the first two are the radius words of the block's two
 * Box–Muller pairs, the third holds their angles, the first pair's in its
 * high 16 bits and the second pair's in its low 16 bits.  A pair thus takes
 * 48 bits.  Angles at the 2^16 midpoints of equal arcs reproduce every
 * trigonometric moment of degree below 2^16 exactly, so the normals keep
 * their law; the radius keeps all 32 bits. */
void oracle_normals4(uint64_t seed, uint64_t traj, uint32_t set_id, uint32_t k, double xi[4]) {
    const uint32_t G = k / 4, j = k % 4;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t words[12];
    for (uint32_t c = 0; c < 3; ++c) {
        const uint32_t ctr[4] = {3 * G + c, (uint32_t)traj, (uint32_t)(traj >> 32), set_id};
        oracle_philox4x32_10(ctr, key, words + 4 * c);
    }
    const uint32_t radius[2] = {words[3 * j], words[3 * j + 1]};
    const uint32_t angle[2] = {words[3 * j + 2] >> 16, words[3 * j + 2] & 0xFFFFu};
    const double two_pi = 6.283185307179586; /* 2 pi rounded to binary64 */
    for (int p = 0; p < 2; ++p) {
        double u0 = uniform_open(radius[p]);
        double u1 = uniform_open16(angle[p]);
        double r = sqrt(-2.0 * log(u0));
        double a = two_pi * u1;
        xi[2 * p] = r * cos(a);
        xi[2 * p + 1] = r * sin(a);
    }
}

/* ------------------------------------------------------------------------ */
/* Model: drift D and noise amplitude S of the slow-roll Langevin equation  */
/* (§1 Eqs. (3)-(4), §2.3 Eq. (17)) for V = m^2 phi^2 / 2 (§3 Eq. (25)),     */
/* M_Pl = 1:  H^2 = V/3,  D = -V'/(3 H^2),  S = H / (2 pi).                  */
/* ------------------------------------------------------------------------ */
/* V(phi) and dV/dphi of the polynomial model, by Horner's rule from the top term. */
static double poly_V(const oracle_run* r, double phi) {
    double v = 0.0;
    for (int k = ORACLE_POLY_TERMS - 1; k >= 0; --k) v = v * phi + r->poly[k];
    return v;
}
static double poly_dV(const oracle_run* r, double phi) {
    double v = 0.0;
    for (int k = ORACLE_POLY_TERMS - 1; k >= 1; --k) v = v * phi + (double)k * r->poly[k];
    return v;
}

static double drift(const oracle_run* r, double phi) {
    if (r->model == ORACLE_MODEL_CONSTANT) return r->a0;
    double V, dV;
    if (r->model == ORACLE_MODEL_POLYNOMIAL) {
        V = poly_V(r, phi);
        dV = poly_dV(r, phi);
    } else {
        V = 0.5 * r->m * r->m * phi * phi;
        dV = r->m * r->m * phi;
    }
    double H2 = V / 3.0;
    return -dV / (3.0 * H2);
}

static double noise(const oracle_run* r, double phi) {
    if (r->model == ORACLE_MODEL_CONSTANT) return r->s0;
    double V = r->model == ORACLE_MODEL_POLYNOMIAL ? poly_V(r, phi) : 0.5 * r->m * r->m * phi * phi;
    double H = sqrt(V / 3.0);
    return H / (2.0 * M_PI);
}

/* ------------------------------------------------------------------------ */
/* MLP bias b(phi, N): 2 -> 64 tanh -> 64 tanh -> 1.                         */
/* ------------------------------------------------------------------------ */
#define HID ORACLE_MLP_HIDDEN
#define P_W1 0
#define P_B1 (P_W1 + HID * 2)
#define P_W2 (P_B1 + HID)
#define P_B2 (P_W2 + HID * HID)
#define P_W3 (P_B2 + HID)
#define P_B3 (P_W3 + HID)

double oracle_mlp_forward(const double* p, const double norm[4], double phi, double N, double* h1o,
                          double* h2o) {
    double x0 = (phi - norm[0]) * norm[1];
    double x1 = (N - norm[2]) * norm[3];
    double h1[HID], h2[HID];
    for (int j = 0; j < HID; ++j)
        h1[j] = tanh(p[P_W1 + 2 * j] * x0 + p[P_W1 + 2 * j + 1] * x1 + p[P_B1 + j]);
    for (int n = 0; n < HID; ++n) {
        double acc = p[P_B2 + n];
        for (int k = 0; k < HID; ++k) acc += p[P_W2 + HID * n + k] * h1[k];
        h2[n] = tanh(acc);
    }
    double out = p[P_B3];
    for (int n = 0; n < HID; ++n) out += p[P_W3 + n] * h2[n];
    if (h1o)
        for (int j = 0; j < HID; ++j) h1o[j] = h1[j];
    if (h2o)
        for (int j = 0; j < HID; ++j) h2o[j] = h2[j];
    return out;
}

void oracle_mlp_backward(const double* p, const double norm[4], double phi, double N, double g,
                         double* grad) {
    double h1[HID], h2[HID], d2[HID];
    oracle_mlp_forward(p, norm, phi, N, h1, h2);
    double x0 = (phi - norm[0]) * norm[1];
    double x1 = (N - norm[2]) * norm[3];
    grad[P_B3] += g;
    for (int n = 0; n < HID; ++n) {
        grad[P_W3 + n] += g * h2[n];
        d2[n] = g * p[P_W3 + n] * (1.0 - h2[n] * h2[n]);
        grad[P_B2 + n] += d2[n];
        for (int k = 0; k < HID; ++k) grad[P_W2 + HID * n + k] += d2[n] * h1[k];
    }
    for (int k = 0; k < HID; ++k) {
        double dh = 0.0;
        for (int n = 0; n < HID; ++n) dh += d2[n] * p[P_W2 + HID * n + k];
        double d1 = dh * (1.0 - h1[k] * h1[k]);
        grad[P_B1 + k] += d1;
        grad[P_W1 + 2 * k] += d1 * x0;
        grad[P_W1 + 2 * k + 1] += d1 * x1;
    }
}

/* ------------------------------------------------------------------------ */
/* One run of the biased Euler–Maruyama scheme until first passage.          */
/* ------------------------------------------------------------------------ */
static int run_valid(const oracle_run* r) {
    if (!(r->dN > 0.0) || !isfinite(r->dN)) return 0;
    if (!(r->n_max > 0.0) || !isfinite(r->n_max)) return 0;
    if (!isfinite(r->phi_in) || !isfinite(r->phi_end) || isnan(r->phi_uv)) return 0;
    if (r->phi_in > r->phi_uv) return 0;
    if (r->model == ORACLE_MODEL_QUADRATIC) {
        if (!(r->m > 0.0) || !(r->phi_end > 0.0)) return 0;
    } else if (r->model == ORACLE_MODEL_CONSTANT) {
        if (!(r->s0 > 0.0)) return 0;
    } else if (r->model == ORACLE_MODEL_POLYNOMIAL) {
        /* the potential must be positive where runs start and end */
        if (!(poly_V(r, r->phi_in) > 0.0) || !(poly_V(r, r->phi_end) > 0.0)) return 0;
    } else {
        return 0;
    }
    if (r->bias_kind == ORACLE_BIAS_MLP) {
        if (r->mlp == NULL || r->k_eval < 1) return 0;
    } else if (r->bias_kind == ORACLE_BIAS_POWER) {
        if (r->model != ORACLE_MODEL_QUADRATIC || !isfinite(r->bias_p)) return 0;
    } else if (r->bias_kind != ORACLE_BIAS_CONST) {
        return 0;
    }
    return 1;
}

/* Optional per-run recording; all pointers may be NULL. */
typedef struct {
    double* phi;    /* phi[0..M] */
    double* xi;     /* xi[0..M-1] */
    double* b_used; /* b[0..M-1] */
    int64_t max_steps;
    /* gradient pass: coefficient and accumulator (coef == 0: off) */
    double coef;
    double* grad;
} recorder;

static int64_t run_one(const oracle_run* r, uint64_t traj, double* N_out, double* lw_out,
                       recorder* rec) {
    const double dN = r->dN;
    const double sq = sqrt(dN);
    const int64_t m_max = (int64_t)ceil(r->n_max / dN);
    double phi = r->phi_in;
    double lw = 0.0;
    int64_t m = 0;
    double xi4[4];
    double b_cur = r->b;
    /* gradient pass: inputs of the current bias block and its sum of normals */
    double blk_phi = 0.0, blk_N = 0.0, blk_xisum = 0.0;

    if (rec && rec->phi) rec->phi[0] = phi;
    /* Absorbing end: a run that starts at or below phi_end has N = 0 (the
     * absorbing boundary condition at phi_end of Appendix A). */
    if (phi <= r->phi_end) {
        *N_out = 0.0;
        *lw_out = 0.0;
        return 0;
    }
    for (;;) {
        if (rec && rec->max_steps >= 0 && m >= rec->max_steps) return -1;
        if (m % 4 == 0) oracle_normals4(r->seed, traj, r->set_id, (uint32_t)(m / 4), xi4);
        const double xi = xi4[m % 4];
        if (r->bias_kind == ORACLE_BIAS_MLP && m % r->k_eval == 0) {
            const double N_el = (double)m * dN;
            if (rec && rec->coef != 0.0 && m > 0)
                oracle_mlp_backward(r->mlp, r->mlp_norm, blk_phi, blk_N, rec->coef * (-sq * blk_xisum),
                                    rec->grad);
            b_cur = oracle_mlp_forward(r->mlp, r->mlp_norm, phi, N_el, NULL, NULL);
            blk_phi = phi;
            blk_N = N_el;
            blk_xisum = 0.0;
        }
        blk_xisum += xi;
        const double D = drift(r, phi);
        const double S = noise(r, phi);
        /* §2.3 Eq. (18) with f = S, or the power law of §3.4 Eq. (26) */
        const double B = r->bias_kind == ORACLE_BIAS_POWER ? r->b * pow(phi, r->bias_p) : b_cur * S;
        /* §2.2 Eq. (11): x_{m+1} - x_m = [D + B] dt + S xi sqrt(dt) */
        double phi_new = phi + (D + B) * dN + S * xi * sq;
        /* log of §2.2 Eq. (12) with the step densities of Eqs. (13)-(14):
         * ln w = -sum (B/S^2) [B dt / 2 + S xi sqrt(dt)].  (Eq. (15) prints
         * the opposite overall sign; expanding (13)/(14) gives this one.) */
        lw -= (B / (S * S)) * (0.5 * B * dN + S * xi * sq);
        if (rec && rec->xi) rec->xi[m] = xi;
        if (rec && rec->b_used) rec->b_used[m] = r->bias_kind == ORACLE_BIAS_POWER ? B / S : b_cur;
        /* Reflecting wall at phi_UV (§2.3 below Eq. (19), §3): mirror once. */
        if (phi_new > r->phi_uv) phi_new = 2.0 * r->phi_uv - phi_new;
        if (rec && rec->phi) rec->phi[m + 1] = phi_new;
        /* First passage through phi_end (§2.1 below Eq. (8)); the crossing
         * time is interpolated linearly between the last two points. */
        if (phi_new <= r->phi_end) {
            const double theta = (phi - r->phi_end) / (phi - phi_new);
            *N_out = ((double)m + theta) * dN;
            *lw_out = lw;
            if (rec && rec->coef != 0.0 && r->bias_kind == ORACLE_BIAS_MLP)
                oracle_mlp_backward(r->mlp, r->mlp_norm, blk_phi, blk_N, rec->coef * (-sq * blk_xisum),
                                    rec->grad);
            return m + 1;
        }
        phi = phi_new;
        m += 1;
        /* Censoring: still inflating after m_max steps. */
        if (m >= m_max) {
            *N_out = INFINITY;
            *lw_out = lw;
            if (rec && rec->coef != 0.0 && r->bias_kind == ORACLE_BIAS_MLP)
                oracle_mlp_backward(r->mlp, r->mlp_norm, blk_phi, blk_N, rec->coef * (-sq * blk_xisum),
                                    rec->grad);
            return m;
        }
    }
}

int oracle_simulate(const oracle_run* run, int64_t n, double* out_N, double* out_logw,
                    int64_t* out_steps) {
    if (!run || n < 0 || !run_valid(run)) return -1;
    if (n > 0 && (!out_N || !out_logw)) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t M = run_one(run, run->traj_offset + (uint64_t)i, &out_N[i], &out_logw[i], NULL);
        if (out_steps) out_steps[i] = M;
    }
    return 0;
}

int64_t oracle_path(const oracle_run* run, int64_t index, int64_t max_steps, double* phi,
                    double* xi, double* b_used, double* out_N, double* out_logw) {
    if (!run || !run_valid(run) || index < 0 || max_steps < 0) return -1;
    recorder rec = {phi, xi, b_used, max_steps, 0.0, NULL};
    return run_one(run, run->traj_offset + (uint64_t)index, out_N, out_logw, &rec);
}

int oracle_grad_pass(const oracle_run* run, int64_t n, const double* coef, double* grad) {
    if (!run || n < 0 || !run_valid(run) || run->bias_kind != ORACLE_BIAS_MLP || !coef || !grad)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (coef[i] == 0.0) continue;
        recorder rec = {NULL, NULL, NULL, -1, coef[i], grad};
        double N, lw;
        run_one(run, run->traj_offset + (uint64_t)i, &N, &lw, &rec);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Weighted histogram (§2.1 Eq. (9), §2.2 Eq. (16)).  Bins are right-closed: */
/* bin j holds lo + j d < N <= lo + (j+1) d.                                 */
/* ------------------------------------------------------------------------ */
int oracle_histogram(const double* N, const double* logw, int64_t n, int32_t n_bins, double lo,
                     double hi, int32_t n_sub, uint64_t id_offset, double* bins, int64_t* counts) {
    if (n < 0 || n_bins < 1 || n_sub < 1 || !(lo < hi) || !isfinite(lo) || !isfinite(hi) || !bins ||
        !counts || (n > 0 && (!N || !logw)))
        return -1;
    const double d = (hi - lo) / (double)n_bins;
    const int64_t nb = (int64_t)n_bins * n_sub;
    for (int64_t b = 0; b < nb; ++b) {
        bins[8 * b + 0] = -INFINITY;
        for (int f = 1; f < 8; ++f) bins[8 * b + f] = 0.0;
    }
    counts[0] = counts[1] = counts[2] = 0;
    counts[3] = n;
    /* pass 1: classify and find the largest log-weight of each bin */
    for (int64_t i = 0; i < n; ++i) {
        if (!(N[i] < INFINITY)) { counts[2]++; continue; }
        if (N[i] <= lo) { counts[0]++; continue; }
        if (N[i] > hi) { counts[1]++; continue; }
        int64_t j = (int64_t)ceil((N[i] - lo) / d) - 1;
        if (j < 0) j = 0;
        if (j > n_bins - 1) j = n_bins - 1;
        int64_t s = (int64_t)((id_offset + (uint64_t)i) % (uint64_t)n_sub);
        int64_t b = s * n_bins + j;
        if (logw[i] > bins[8 * b + 0]) bins[8 * b + 0] = logw[i];
    }
    /* pass 2: sums of powers of the shifted log-weight x = lw - max_lw <= 0 */
    for (int64_t i = 0; i < n; ++i) {
        if (!(N[i] < INFINITY) || N[i] <= lo || N[i] > hi) continue;
        int64_t j = (int64_t)ceil((N[i] - lo) / d) - 1;
        if (j < 0) j = 0;
        if (j > n_bins - 1) j = n_bins - 1;
        int64_t s = (int64_t)((id_offset + (uint64_t)i) % (uint64_t)n_sub);
        int64_t b = s * n_bins + j;
        double x = logw[i] - bins[8 * b + 0];
        bins[8 * b + 1] += exp(x);
        bins[8 * b + 2] += exp(2.0 * x);
        bins[8 * b + 3] += x;
        bins[8 * b + 4] += x * x;
        bins[8 * b + 5] += x * x * x;
        bins[8 * b + 6] += x * x * x * x;
        bins[8 * b + 7] += 1.0;
    }
    return 0;
}
