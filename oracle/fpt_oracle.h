/*
 * FP64 CPU oracle for importance-sampled first-passage times
 * (Jackson, Assadullahi, Koyama, Vennin, Wands — "Numerical simulations of
 * stochastic inflation using importance sampling", arXiv:2206.11234).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, scalar definition
 * that the GPU library is checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * source, header, table or helper with the CUDA library; the only thing both
 * sides have in common is the published definition of each step.
 *
 * Everything is IEEE binary64, compiled without floating-point contraction
 * (-ffp-contract=off), so each arithmetic expression below is rounded
 * exactly as written.
 */
#ifndef FPT_ORACLE_H
#define FPT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Models (drift D and noise amplitude S of the Langevin equation, §2.1 Eq. (7)). */
#define ORACLE_MODEL_QUADRATIC 0 /* §3 Eq. (25) with §2.3 Eq. (17): D = -2/phi, S = m phi / (2 pi sqrt 6) */
#define ORACLE_MODEL_CONSTANT 1  /* test model: D = a0, S = s0 (constant drift and noise) */
#define ORACLE_MODEL_POLYNOMIAL 2 /* V = sum_k poly[k] phi^k, D = -V'/(3 H^2), H^2 = V/3, S = H/(2 pi) (§2.3 Eq. (17)) */
#define ORACLE_POLY_TERMS 8

/* Bias kinds (§2.3 Eq. (18): B = A f(phi)). */
#define ORACLE_BIAS_CONST 0 /* B = b S(phi): f = S, A = b */
#define ORACLE_BIAS_POWER 1 /* B = b phi^p (§3.4 Eq. (26)): A_p = b, p = bias_p */
#define ORACLE_BIAS_MLP 2   /* B = b(phi, N_elapsed) S(phi), b an MLP re-evaluated every k_eval steps */

#define ORACLE_MLP_HIDDEN 64
/* Parameter vector layout: W1[64][2], b1[64], W2[64][64], b2[64], w3[64], b3[1]. */
#define ORACLE_MLP_NPARAM (64 * 2 + 64 + 64 * 64 + 64 + 64 + 1)

typedef struct {
    int32_t model;      /* ORACLE_MODEL_* */
    int32_t bias_kind;  /* ORACLE_BIAS_* */
    double m;           /* inflaton mass (M_Pl = 1), quadratic model */
    double a0, s0;      /* constant model: drift and noise amplitude */
    double phi_in, phi_end, phi_uv; /* phi_uv = +inf: no reflecting wall */
    double dN;          /* Euler–Maruyama time step (e-folds) */
    double b;           /* constant bias amplitude in noise units */
    double n_max;       /* censoring time: a run still going after ceil(n_max/dN) steps is censored */
    uint64_t seed;      /* Philox key */
    uint32_t set_id;    /* Philox counter word 3 */
    uint64_t traj_offset; /* global id of trajectory 0 */
    /* MLP bias only */
    const double* mlp;  /* ORACLE_MLP_NPARAM parameters */
    double mlp_norm[4]; /* inputs: x0 = (phi - c0) * s0, x1 = (N - c1) * s1 as {c0, s0, c1, s1} */
    int32_t k_eval;     /* bias is re-evaluated at steps m = 0, k_eval, 2 k_eval, ... */
    /* power-law bias only */
    double bias_p;      /* exponent p of B = b phi^p */
    /* polynomial model only */
    double poly[ORACLE_POLY_TERMS]; /* V(phi) = sum_k poly[k] phi^k */
} oracle_run;

/* Philox4x32-10 block function: out = Philox(ctr, key), 10 rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The four standard normals used by steps 4k .. 4k+3 of trajectory `traj`:
 * Box–Muller on three of the twelve words of the Philox counters
 * (3G + c, traj_lo, traj_hi, set_id), c = 0, 1, 2, G = k div 4 (the word
 * assignment is spelled out in fpt_oracle.c). */
void oracle_normals4(uint64_t seed, uint64_t traj, uint32_t set_id, uint32_t k, double xi[4]);

/* Simulate n runs with global ids traj_offset + i.  Writes the first-passage
 * time out_N[i] (+inf when censored), the log-weight out_logw[i] and, if
 * out_steps is non-NULL, the number of steps taken.  Returns 0, or -1 on an
 * invalid argument. */
int oracle_simulate(const oracle_run* run, int64_t n, double* out_N, double* out_logw,
                    int64_t* out_steps);

/* One run, recording the path: phi[0..M] (M+1 values, at most max_steps+1),
 * the normals xi[0..M-1] and the bias amplitude b_used[0..M-1] = B/S of each step.
 * Returns M, or -1 if the run needs more than max_steps steps. */
int64_t oracle_path(const oracle_run* run, int64_t index, int64_t max_steps, double* phi,
                    double* xi, double* b_used, double* out_N, double* out_logw);

/* Weighted histogram of first-passage times (§2.1 Eq. (9), §2.2 Eq. (16)).
 * bins: (lo + j d, lo + (j+1) d], d = (hi - lo)/n_bins.  Run i (global id
 * id_offset + i) goes to subset (id_offset + i) mod n_sub.  For each
 * (subset, bin) the output holds 8 doubles:
 *   {max_lw, s1 = sum exp(x), s2 = sum exp(2 x), l1 = sum x, l2 = sum x^2, l3 = sum x^3,
 *    l4 = sum x^4, count} with x = lw - max_lw (the moments feed the lognormal estimator and
 *   the normality test of §2.3, Eqs. (27)-(29)).
 * counts[4] = {under (N <= lo), over (lo < ... N > hi, finite), censored (N not finite), total}. */
int oracle_histogram(const double* N, const double* logw, int64_t n, int32_t n_bins, double lo,
                     double hi, int32_t n_sub, uint64_t id_offset, double* bins, int64_t* counts);

/* MLP bias b(phi, N): 2 -> 64 tanh -> 64 tanh -> 1.  h1, h2 may be NULL. */
double oracle_mlp_forward(const double* params, const double norm[4], double phi, double N,
                          double* h1, double* h2);

/* grad += g * d b(phi, N) / d params. */
void oracle_mlp_backward(const double* params, const double norm[4], double phi, double N,
                         double g, double* grad);

/* Gradient pass of the tail-variance objective.  For every run i with
 * coef[i] != 0, re-simulate it and add coef[i] * d(log w)/d(params) at fixed
 * path to grad, where d(log w)/d(b_k) = -sqrt(dN) * (sum of the normals of
 * bias block k).  Returns 0, or -1 on an invalid argument. */
int oracle_grad_pass(const oracle_run* run, int64_t n, const double* coef, double* grad);

#ifdef __cplusplus
}
#endif
#endif
