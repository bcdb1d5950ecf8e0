/*
 * fpt.h — C ABI of the GB300 (sm_103a) importance-sampled first-passage-time
 * library.
 *
 * The method is that of Jackson, Assadullahi, Koyama, Vennin, Wands,
 * "Numerical simulations of stochastic inflation using importance sampling"
 * (arXiv:2206.11234), §2:
 *   - runs of the 1-D Langevin equation dphi/dN = D(phi) + S(phi) xi
 *     (§2.1 Eq. (7)) with the drift shifted by a bias B (§2.2 Eq. (10)),
 *     integrated by Euler–Maruyama (§2.2 Eq. (11)) until phi first reaches
 *     phi_end (§2.1, below Eq. (8));
 *   - for slow-roll inflation D = -V'/(3H^2), S = H/(2 pi) (§2.3 Eq. (17))
 *     with V = m^2 phi^2 / 2 (§3 Eq. (25)) and M_Pl = 1, so D = -2/phi and
 *     S = m phi / (2 pi sqrt 6); the bias is B = b S (§2.3 Eq. (18), f = S);
 *   - each run records its first-passage time N and its log importance weight
 *     ln w = ln(p_T/p_S) = -sum_m (B/S^2)[B dN/2 + S xi_m sqrt(dN)]
 *     (§2.2 Eqs. (12)-(14); Eq. (15) is printed with the opposite overall sign,
 *     which contradicts Eqs. (13)-(14));
 *   - an optional reflecting wall at phi_uv (§2.3 below Eq. (19), §3);
 *   - the records are binned into a weighted histogram (§2.1 Eq. (9),
 *     §2.2 Eq. (16)).
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller unless the
 *     name ends in _host.  Outputs are indexed by trajectory, whatever order
 *     the GPU finishes them in, so the records (N, ln w) are deterministic for
 *     a given k_steps and independent of block_dim and of the grid.  Histogram
 *     counts and maxima are exact; the FP64 bin sums are accumulated with
 *     atomics, so their last bits can vary from call to call.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; the call then reads back a device status word, which
 *     synchronises that stream only.
 *   - Return value: FPT_OK (0) or a negative FPT_E* code.  Argument errors are
 *     detected on the host before any GPU work is enqueued.  fpt_strerror()
 *     names a code; fpt_last_error() describes the last failure of the calling
 *     thread.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with counter
 *     (c, i_lo, i_hi, set_id) and key (seed_lo, seed_hi), mapped to normals by
 *     Box–Muller with 48 bits per pair of normals.  Steps 16G .. 16G + 15 of
 *     trajectory i use the twelve words of counters c = 3G, 3G + 1, 3G + 2;
 *     steps 16G + 4j .. 16G + 4j + 3 take words 3j and 3j + 1 (radius words
 *     of their two pairs) and 3j + 2 (the two 16-bit angles, first pair in
 *     the high half).  Any run can be reproduced from (seed, set_id, i)
 *     alone, so an id range can be split across calls or GPUs (traj_offset)
 *     with bit-identical results.
 *   - A run still inflating after ceil(n_max/dN) steps is censored: N = +inf,
 *     ln w = its weight at that step (E[w] = 1 still holds).
 */
#ifndef FPT_H
#define FPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FPT_ABI_VERSION 3 /* 2: fpt_bin carries four moments of ln w; fpt_estimate; 3: bias terms of the lognormal estimate */

/* return codes */
#define FPT_OK 0
#define FPT_EINVAL (-1)          /* invalid argument (checked on the host) */
#define FPT_ECUDA (-2)           /* a CUDA runtime call failed */
#define FPT_ENOMEM (-3)          /* device allocation failed */
#define FPT_EUNSUPPORTED (-4)    /* valid but not provided (e.g. FP64 with the MLP bias) */
#define FPT_EDEVICE_STATUS (-5)  /* a kernel reported an internal error (bounded wait expired) */

/* drift/noise model */
#define FPT_MODEL_QUADRATIC 0 /* D = -2/phi, S = m phi/(2 pi sqrt 6): §2.3 Eq. (17) + §3 Eq. (25) */
#define FPT_MODEL_CONSTANT 1  /* D = a0, S = s0: constant drift and noise (inverse-Gaussian test model) */
#define FPT_MODEL_POLYNOMIAL 2 /* V(phi) = sum_k poly[k] phi^k (M_Pl = 1): D = -V'/(3 H^2), H^2 = V/3,
                                  S = H/(2 pi) (§2.3 Eq. (17)); V must be positive wherever runs go */
#define FPT_POLY_TERMS 8

/* arithmetic of the stepper */
#define FPT_PREC_F64 0        /* everything binary64 (reference mode, per-run parity with the FP64 oracle) */
#define FPT_PREC_F32_KAHAN 1  /* binary32 state; ln w from binary32 block sums + compensated (Kahan) running sum */
#define FPT_PREC_F32_F64ACC 2 /* binary32 state; ln w running sum and crossing interpolation in binary64 */

/* bias of the sample process (§2.3 Eq. (18)) */
#define FPT_BIAS_CONST 0 /* B = b S(phi), b constant (the set's bias) */
#define FPT_BIAS_POWER 1 /* B = A_p phi^p (§3.4 Eq. (26)), A_p = the set's bias, p = bias_p; quadratic model */
#define FPT_BIAS_MLP 2   /* B = b S, b = MLP(phi, N_elapsed), held for k_eval steps (see fpt_mlp_params) */

#define FPT_MAX_SETS 64       /* parameter sets per batched launch */
#define FPT_MAX_HIST_BINS 4096 /* n_sub * n_bins per histogram */

typedef struct fpt_params {
    int32_t abi_version; /* must be FPT_ABI_VERSION */
    int32_t model;       /* FPT_MODEL_* */
    int32_t precision;   /* FPT_PREC_* */
    int32_t bias_kind;   /* FPT_BIAS_* */
    double m;            /* inflaton mass (quadratic model), > 0 */
    double a0, s0;       /* constant model: drift and noise amplitude (s0 > 0) */
    double n_max;        /* censoring time, finite and > 0 */
    double bias_p;       /* FPT_BIAS_POWER: exponent p (finite; integers 0..4 have specialised kernels) */
    double poly[FPT_POLY_TERMS]; /* FPT_MODEL_POLYNOMIAL: coefficients of V (the sets' m is ignored) */
    const void* mlp;     /* FPT_BIAS_MLP: device pointer to an fpt_mlp_params */
    int32_t k_eval;      /* FPT_BIAS_MLP: steps between bias evaluations (0 = 32) */
    int32_t block_dim;   /* threads per block of the stepper (0 = autotuned or default) */
    int32_t k_steps;     /* steps per scheduling block of the stepper (0 = autotuned or default) */
    uint32_t set_id;     /* Philox counter word 3 (fpt_simulate only) */
    uint64_t traj_offset; /* global id of the first trajectory (fpt_simulate only) */
    void* stream;        /* cudaStream_t */
    uint64_t* steps_out; /* optional device counter: the number of Euler–Maruyama steps taken is ADDED to it */
} fpt_params;

/* Learned bias (FPT_BIAS_MLP): b(phi, N) = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3,
 * x = ((phi - norm[0]) norm[1], (N_elapsed - norm[2]) norm[3]), 64 hidden units
 * per layer.  The bias of the EM step is B = b(phi, N) S(phi) (§2.3 Eq. (18)
 * with a state-dependent amplitude); b is evaluated at the start of every
 * k_eval-step block of a run and held for the block, so the importance weight
 * of §2.2 Eqs. (12)-(14) stays exact.  Parameters are BF16 (the bit pattern of
 * the upper half of an IEEE float) in the order W1[64][2] (row-major), b1[64],
 * W2[64][64] (row-major, out x in), b2[64], w3[64], b3; the vector is padded to
 * FPT_MLP_NPARAM_PAD entries (the padding is ignored).  Device memory. */
#define FPT_MLP_HIDDEN 64
#define FPT_MLP_NPARAM 4417
#define FPT_MLP_NPARAM_PAD 4424
typedef struct fpt_mlp_params {
    float norm[4];
    uint16_t w[FPT_MLP_NPARAM_PAD];
} fpt_mlp_params;

/* Simulate n_traj runs of one parameter set (§2.2 Eqs. (10)-(15)).
 *   phi_in, phi_end : start and end of inflation; phi_in <= phi_end gives N = 0, ln w = 0
 *   phi_uv          : reflecting wall, >= phi_in, or +INFINITY for none
 *   dN              : time step (e-folds), > 0
 *   bias            : b (FPT_BIAS_CONST), A_p (FPT_BIAS_POWER), ignored for FPT_BIAS_MLP
 *   out_N, out_logw : device double[n_traj]; out_N[i] = +inf when censored.
 * n_traj = 0 is a no-op.  Errors: FPT_EINVAL, FPT_EUNSUPPORTED, FPT_ECUDA,
 * FPT_ENOMEM, FPT_EDEVICE_STATUS. */
int fpt_simulate(const fpt_params* p, int64_t n_traj, double phi_in, double phi_end, double phi_uv,
                 double dN, double bias, uint64_t seed, double* out_N, double* out_logw);

/* One parameter set of a batched launch (host memory). */
typedef struct fpt_set {
    double phi_in, phi_end, phi_uv; /* as in fpt_simulate */
    double m;                        /* mass (quadratic model; the constant model uses p->a0, p->s0) */
    double b;                        /* bias amplitude */
    double dN;                       /* time step */
    double n_max;                    /* censoring time */
    int64_t n_traj;                  /* runs in this set (>= 0) */
    uint64_t traj_offset;            /* global id of this set's first run */
    uint32_t set_id;                 /* Philox counter word 3 */
    int32_t n_bins;                  /* histogram bins for this set (fpt_simulate_batch with bins) */
    double hist_lo, hist_hi;         /* histogram range (lo, hi] */
} fpt_set;

/* Weighted-histogram bin (§2.1 Eq. (9), §2.2 Eq. (16)) with max-shifted sums so
 * that weights spanning hundreds of e-folds stay representable.  With
 * x_i = ln w_i - max_lw <= 0 over the runs i of the bin:
 *   sum_i w_i   = exp(max_lw) * s1,   sum_i w_i^2 = exp(2 max_lw) * s2,
 *   l_k = sum_i x_i^k (k = 1..4: the moments of ln w behind the lognormal
 *   estimator and the normality test of §2.4), count = n_j.
 * Empty bin: max_lw = -inf, sums 0.  64 bytes. */
typedef struct fpt_bin {
    double max_lw, s1, s2, l1, l2, l3, l4;
    int64_t count;
} fpt_bin;

/* Counters of a histogram: runs with N <= lo, finite N > hi, N not finite
 * (censored), and all runs. */
typedef struct fpt_hist_counts {
    int64_t under, over, censored, total;
} fpt_hist_counts;

/* Simulate n_sets parameter sets in ONE persistent launch (finished lanes
 * refill from a global ticket counter across all sets).  Set s writes
 * out_N/out_logw[off_s .. off_s + n_traj_s), off_s = sum_{t<s} n_traj_t.
 * If out_bins is non-NULL the per-set histograms are built in the same call:
 * set s fills out_bins[boff_s .. boff_s + n_bins_s), boff_s = sum_{t<s} n_bins_t,
 * and out_counts[s] (device).
 * sets: host array, 1 <= n_sets <= FPT_MAX_SETS; p->set_id and p->traj_offset
 * are ignored (each set carries its own).
 * Device memory: the call takes a stream-ordered workspace from the library's
 * pool (the set table and scratch, and with bins 4 bytes per run for the bin
 * index of the histogram's first pass) and returns it before returning; the
 * pool keeps it mapped for the next call.  FPT_ENOMEM if it cannot be had. */
int fpt_simulate_batch(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                       double* out_N, double* out_logw, fpt_bin* out_bins,
                       fpt_hist_counts* out_counts);

/* Reusable, graph-captured batched launch.  fpt_plan_create validates the
 * sets once, uploads their constants to a plan-owned device workspace and
 * captures [scratch reset, persistent stepper, histogram kernels (if out_bins),
 * status copy] into one CUDA graph writing to the given device outputs (laid
 * out as in fpt_simulate_batch); the stepper's launch shape is fixed at
 * creation (p->block_dim / k_steps, or the autotuned shape).
 * fpt_plan_launch(plan, seed, stream) sets the seed and replays the graph on
 * `stream` (the device current at creation), then synchronises it and checks
 * the device status; results equal fpt_simulate_batch's with the same seed.
 * fpt_plan_destroy frees the plan.  A plan is not safe for concurrent launches. */
typedef struct fpt_plan fpt_plan;
int fpt_plan_create(const fpt_params* p, const fpt_set* sets, int32_t n_sets, double* out_N,
                    double* out_logw, fpt_bin* out_bins, fpt_hist_counts* out_counts,
                    fpt_plan** plan_out);
int fpt_plan_launch(fpt_plan* plan, uint64_t seed, void* stream);
int fpt_plan_destroy(fpt_plan* plan);

/* Weighted histogram of n records.  Bins (lo + j d, lo + (j+1) d],
 * d = (hi - lo)/n_bins, j = ceil((N - lo)/d) - 1 clamped to [0, n_bins).
 * Record i (global id id_offset + i) goes to subset (id_offset + i) mod n_sub
 * (jackknife subsets, §2.1); bins[s * n_bins + j].  The outputs are
 * overwritten.  1 <= n_bins, 1 <= n_sub, n_sub * n_bins <= FPT_MAX_HIST_BINS,
 * lo < hi finite.  Device memory: a workspace of 4 bytes per record (the bin
 * index of the first pass) and a few hundred bytes from the library's pool,
 * returned before the call returns; FPT_ENOMEM if it cannot be had. */
int fpt_histogram(const double* N, const double* logw, int64_t n, int32_t n_bins, double lo,
                  double hi, int32_t n_sub, uint64_t id_offset, fpt_bin* bins,
                  fpt_hist_counts* counts, void* stream);

/* Merge of weighted histograms of disjoint sets of runs (shards of one
 * workload on several GPUs, or calls over split id ranges: runs are
 * independent, §2.1) into the histogram of their union, in binary64 on the
 * host.  parts: host array of n_parts x n_bins bins, part p's bins at
 * parts + p * n_bins, all with the same bin edges; out: n_bins host bins
 * (may not alias parts).  Each part is moved to the common max_lw M of its
 * bin, d = max_lw - M <= 0: s1 e^d, s2 e^(2d), l_k -> sum_i C(k,i) d^(k-i) l_i
 * (l_0 = count), then summed; empty parts (max_lw = -inf) add nothing.
 * part_counts / out_counts (nullable together): the counters, summed.
 * Bins with max_lw NaN or a negative count are rejected (FPT_EINVAL).  No GPU
 * work; callable without a device. */
int fpt_hist_merge(const fpt_bin* parts, int32_t n_parts, int64_t n_bins, const fpt_hist_counts* part_counts,
                   fpt_bin* out, fpt_hist_counts* out_counts);

/* Per-bin estimates of the first-passage-time density from a histogram
 * (fpt_estimate).  d = bin width, n_total = runs of the histogram (all of
 * them: in range, out of range and censored).
 *   p_direct, se_direct : sum w / (d n_total) (§2.1 Eq. (9), §2.2 Eq. (16)) and
 *                         sqrt((sum w^2/n_total - (sum w/n_total)^2)/n_total)/d
 *   p_lognormal         : n_j exp(mean_lw + var_lw/2) / (d n_total) (§2.4 Eqs. (22), (23))
 *   eps_lo, eps_hi      : p_lognormal |exp(-+a) - 1|, a = sqrt(var/n_j + var^2/(2 n_j - 2)) (Eq. (24))
 *   mean_lw, var_lw     : sample mean and unbiased sample variance of ln w in the bin
 *   skew, kurt          : sample skewness sqrt(b1) = m3/m2^1.5 and kurtosis b2 = m4/m2^2
 *   z_skew, z_kurt      : their normal deviates (D'Agostino 1970; Anscombe and Glynn 1983)
 *   k2, p_normal        : D'Agostino-Pearson K^2 = z_skew^2 + z_kurt^2 and its chi^2(2)
 *                         p-value exp(-K^2/2) (the normality test of ln w in §2.4)
 *   jk_direct, jk_lognormal : jackknife errors (§2.1): the unbiased spread of the
 *                         n_sub subset estimates (each with its own n_total) / sqrt(n_sub)
 *   bias_ln, bias_se    : the next terms of ln <w> beyond Eq. (22)'s mean + var/2,
 *                         ln <w> = k1 + k2/2 + k3/6 + k4/24 + ... (cumulants of ln w),
 *                         estimated by the unbiased k-statistics of ln w in the bin as
 *                         k3/6 + k4/24, and its standard error under normality
 *                         sqrt(var k3 / 36 + var k4 / 576), var k3 = 6 n k2^3/((n-1)(n-2)),
 *                         var k4 = 24 n (n+1) k2^4/((n-1)(n-2)(n-3)).  p_lognormal
 *                         exp(bias_ln) is the cumulant-corrected estimate; a skewness
 *                         of ln w too small for the normality test still shifts the
 *                         lognormal estimate by about bias_ln.
 * Empty bin: both estimates 0, eps 0.  The lognormal estimate needs n_j >= 2,
 * the bias terms n_j >= 4, the normality test n_j >= 8 (both var_lw > 0), the
 * jackknife n_sub >= 2 and every subset's estimate defined; otherwise NaN.
 * 144 bytes. */
typedef struct fpt_estimate_bin {
    double count, p_direct, se_direct, p_lognormal, eps_lo, eps_hi, mean_lw, var_lw;
    double skew, kurt, z_skew, z_kurt, k2, p_normal, jk_direct, jk_lognormal;
    double bias_ln, bias_se;
} fpt_estimate_bin;

/* Estimates of one histogram made by fpt_histogram (or one set's histogram of
 * fpt_simulate_batch, with n_sub = 1): bins[s * n_bins + j] (device, as
 * written), n_total runs with global ids id_offset .. id_offset + n_total - 1
 * (run id i belongs to subset i mod n_sub).  Writes out[j], j < n_bins
 * (device).  Asynchronous on `stream`; argument errors are reported
 * synchronously (1 <= n_bins, 1 <= n_sub, n_sub * n_bins <= FPT_MAX_HIST_BINS,
 * lo < hi finite, n_total >= 1). */
int fpt_estimate(const fpt_bin* bins, int32_t n_bins, int32_t n_sub, double lo, double hi,
                 int64_t n_total, uint64_t id_offset, fpt_estimate_bin* out, void* stream);

/* Multi-bias reconstruction (§3.2: simulations with different bias amplitudes
 * probe different ranges of N and are combined where they overlap).  est:
 * device fpt_estimate_bin[n_runs][n_bins], the estimates of the SAME bins from
 * n_runs independent simulations (fpt_estimate).  For each bin, a run
 * contributes if its bin holds >= min_count runs, its estimate (estimator:
 * FPT_ESTIMATOR_DIRECT or FPT_ESTIMATOR_LOGNORMAL) is defined and > 0, and,
 * for the lognormal estimator, p_normal >= p_threshold or var_lw = 0 (w = 1
 * in the bin: a degenerate normal; p_threshold = 0 disables the test; §2.4
 * uses 0.005).  Contributions are combined in log space with inverse-
 * variance weights, ln p = sum_k ln p_k / a_k^2 / sum_k 1/a_k^2 with a_k the
 * relative error of run k (lognormal: sqrt(a^2 + 1/n_j), Eq. (24)'s a with the
 * relative fluctuation of the bin count added; direct: se/p), and
 * a = 1/sqrt(sum_k 1/a_k^2).  out[j] (device): {p, eps_lo = p (1 - e^-a),
 * eps_hi = p (e^a - 1), a, n_used, best = index of the run with the smallest
 * a_k}; bins without a contribution: p = NaN, n_used = 0, best = -1.
 * Asynchronous on `stream`; argument errors are synchronous. */
#define FPT_ESTIMATOR_DIRECT 0
#define FPT_ESTIMATOR_LOGNORMAL 1
typedef struct fpt_stitch_bin {
    double p, eps_lo, eps_hi, log_err, n_used, best;
} fpt_stitch_bin;
int fpt_stitch(const fpt_estimate_bin* est, int32_t n_runs, int32_t n_bins, int32_t estimator, int64_t min_count,
               double p_threshold, fpt_stitch_bin* out, void* stream);

/* Pearson's correlation coefficient of (N_i, ln w_i) over the runs with finite
 * N_i (§3.4: |r| of log10 w with N measures how tightly the (N, w) cloud is
 * squeezed and guides the choice of the bias; log10 w and ln w differ by a
 * constant factor, which r does not see).  N, logw: device double[n].  Two
 * passes in binary64: means, then centred sums.  out: device double[8] =
 * {r, count, mean_N, mean_lw, var_N, var_lw, cov, 0} with unbiased variances
 * and covariance; r = NaN when fewer than 2 runs or a variance is zero; the
 * 8 doubles are also the reduction's work area.  Asynchronous on `stream`. */
int fpt_pearson(const double* N, const double* logw, int64_t n, double* out, void* stream);

/* One training record of the learned-bias stepper: the MLP inputs at the start
 * of a k_eval-step block of run `run` (its record index in the call's outputs)
 * and the sum of the normals drawn in that block (up to the run's last step).
 * d ln w / d b of the block is -sqrt(dN) * xi_sum. */
typedef struct fpt_mlp_record {
    float phi, N, xi_sum;
    uint32_t run;
} fpt_mlp_record;

/* Simulate with the learned bias (p->bias_kind = FPT_BIAS_MLP, p->mlp = device
 * fpt_mlp_params, p->precision = FPT_PREC_F32_F64ACC, quadratic model): as
 * fpt_simulate_batch (no histograms; fpt_set.b is ignored) with b(phi, N)
 * evaluated on the tensor cores for 128 runs at a time at the start of every
 * k_eval-step block (p->k_eval in {16, 32, 64, 128}, 0 = 32; runs start on a block
 * boundary, so a run's evaluations are at steps 0, k_eval, 2 k_eval, ...).
 * If records is non-NULL, one fpt_mlp_record per simulated block is appended
 * (in no particular order) up to record_capacity; *n_records_out (host, may be
 * NULL) receives the number of blocks simulated, and the call fails with
 * FPT_ENOMEM if that exceeds the capacity.  Total runs must be < 2^32. */
int fpt_simulate_mlp(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                     double* out_N, double* out_logw, fpt_mlp_record* records, int64_t record_capacity,
                     int64_t* n_records_out);

/* Device buffers of the learned-bias training loop (owned by the caller). */
typedef struct fpt_mlp_train_state {
    float* master;            /* FPT_MLP_NPARAM FP32 parameters, updated in place */
    float* adam_m;            /* FPT_MLP_NPARAM first moments (start at 0) */
    float* adam_v;            /* FPT_MLP_NPARAM second moments (start at 0) */
    float* grad;              /* FPT_MLP_NPARAM scratch */
    fpt_mlp_params* w;        /* BF16 parameters the simulation uses; rewritten from master */
    fpt_mlp_record* records;  /* record_capacity records of the step's simulation */
    int64_t record_capacity;
    double* out_N;            /* n_traj first-passage times of the step's runs */
    double* out_logw;         /* n_traj log-weights */
    double* coef;             /* n_traj scratch */
    float* rows;              /* 3 * record_capacity scratch */
    int32_t step;             /* Adam step counter (host; incremented by each call) */
} fpt_mlp_train_state;

typedef struct fpt_mlp_train_stats {
    double log_second_moment; /* log of the estimate of E_S[w^2 1{N > tail_N}] before the update */
    double p_hat;             /* estimate of P(N > tail_N) from the step's runs (§2.2 Eq. (16)) */
    double n_eff;             /* p_hat^2 / its variance estimate */
    double frac_in_tail;      /* fraction of sample runs with N > tail_N */
    int64_t n_records;        /* blocks simulated */
} fpt_mlp_train_stats;

/* One Adam step on log E_S[w^2 1{N > tail_N}], the second moment of the
 * weighted tail estimator (minimising it minimises the estimator's variance):
 * simulate set->n_traj runs with the current BF16 parameters (p as for
 * fpt_simulate_mlp, p->mlp == state->w) recording every block, weight run i by
 * w_i^2 1{N_i > tail_N} / sum_j w_j^2 1{N_j > tail_N} (max-shifted), back-propagate
 * -sqrt(dN) * xi_sum of every block through the MLP on the tensor cores and
 * update master / w with Adam (beta 0.9, 0.999, learning rate lr).  All of it
 * runs on the device; the call synchronises p->stream once at the end. */
int fpt_mlp_train_step(const fpt_params* p, const fpt_set* set, uint64_t seed, double tail_N, double lr,
                       fpt_mlp_train_state* state, fpt_mlp_train_stats* stats_out);

/* Batched MLP forward: out_b[i] = b(phi[i], N[i]) for i < n (device arrays,
 * float).  The hidden 64 x 64 layer runs on the tensor cores (BF16 inputs,
 * FP32 accumulation); the others on the CUDA cores with tanh.approx. */
int fpt_mlp_forward(const fpt_mlp_params* w, const float* phi, const float* N, int64_t n, float* out_b,
                    void* stream);

/* Batched MLP backward: grad[j] += sum_i g[i] * d b(phi[i], N[i]) / d param_j for
 * the FPT_MLP_NPARAM parameters in the packed order (device float array,
 * accumulated, not cleared).  The products delta2 W2 and delta2^T h1 run on the
 * tensor cores; the sums of the vector gradients on the CUDA cores. */
int fpt_mlp_backward(const fpt_mlp_params* w, const float* phi, const float* N, const float* g, int64_t n,
                     float* grad, void* stream);

/* Autotuner of the stepper's launch shape (threads per block in {128, 256, 512}
 * and steps per scheduling block k_steps in {16, 32, 64}, binary64: {4, 8};
 * the binary32 power-law bias kernels exist for 32 only).
 * Runs pilot launches over the given sets with each n_traj scaled by
 * `fraction` in (0, 1] (raised if needed so the pilot fills the GPU), times
 * each shape with CUDA events on p->stream and keeps the fastest in EM steps
 * per second.  The result is cached per (device, precision, model, wall) and
 * used by every later call whose block_dim or k_steps is 0.  Outputs (host,
 * each may be NULL): the chosen shape and its pilot steps/s.  Records do not
 * depend on block_dim; k_steps only changes the rounding of the ln w sum. */
int fpt_autotune(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                 double fraction, int32_t* block_dim_out, int32_t* k_steps_out,
                 double* steps_per_s_out);
/* Forget every autotuned shape (later calls use the defaults until re-tuned). */
void fpt_autotune_reset(void);

/* End-to-end call with HOST buffers: copies nothing in but the parameters,
 * runs fpt_simulate_batch with bins on a private device workspace and copies
 * (N, ln w) and the histograms back to host_N/host_logw (may be NULL to skip)
 * and host_bins/host_counts.  The device buffers are taken from and returned
 * to a library-owned stream-ordered pool (one per device), which keeps the
 * memory for later calls until the process exits. */
int fpt_simulate_batch_host(const fpt_params* p, const fpt_set* sets, int32_t n_sets, uint64_t seed,
                            double* host_N, double* host_logw, fpt_bin* host_bins,
                            fpt_hist_counts* host_counts);

/* No-allocation variant of fpt_simulate_batch (records only, no histograms).
 * The paper has no counterpart: this entry exists for callers that must not
 * allocate device memory while they run — for example a process whose device
 * memory is entirely reserved by its own pool allocator or a fixed budget, or a
 * latency-bound loop that cannot afford an allocation failing mid-run or the
 * device synchronisation that freeing memory implies.  The caller passes the
 * inputs (host sets array) and the device outputs exactly as for
 * fpt_simulate_batch; the stepper's scratch (ticket counter, step total and
 * status word in a 256-byte header, then up to FPT_NOALLOC_MAX_SETS per-set
 * constant blocks: 15,232 bytes in all) is a fixed array inside the library
 * that every GPU loading the library keeps until the process exits.  No device
 * memory is allocated or freed.
 *   - n_sets must be in [1, FPT_NOALLOC_MAX_SETS]; more is rejected with
 *     FPT_EINVAL (fpt_last_error() says why).
 *   - Set-up: the first call on a device looks up the array's device address
 *     with that device current and caches it (again for a new CUDA context on
 *     the same device); make that first call before any stream capture.
 *   - All calls share the one array: each call re-initialises what it uses,
 *     but calls whose GPU work overlaps (other streams or host threads) race
 *     on it and must be serialised by the caller.
 *   - The call uploads the scratch image from host memory, launches the
 *     stepper and reads the status word back: it synchronises `stream`
 *     before returning.
 *   - Results equal those of fpt_simulate_batch with the same arguments. */
#define FPT_NOALLOC_MAX_SETS 48
int fpt_simulate_batch_noalloc(const fpt_params* p, const fpt_set* sets, int32_t n_sets,
                               uint64_t seed, double* out_N, double* out_logw);

/* Diagnostic: the unit normals xi_{4k} .. xi_{4k+3} for k = k0 .. k0 + n_blocks - 1
 * of run `traj` of set `set_id` (exactly what the stepper draws; §2.1 below
 * Eq. (8)), written to the device array out as double (FPT_PREC_F64) or float
 * (the binary32 precisions), 4 * n_blocks values.  precision =
 * FPT_NORMALS_RAW_BITS writes instead the 4 Philox words of each counter
 * c = k0 .. k0 + n_blocks - 1 (counter (c, traj_lo, traj_hi, set_id)) as
 * uint32.  Synchronises `stream`. */
#define FPT_NORMALS_RAW_BITS 3
int fpt_normals(uint64_t seed, uint64_t traj, uint32_t set_id, uint32_t k0, int64_t n_blocks,
                int32_t precision, void* out, void* stream);

/* Self-test of the bounded waits (no paper counterpart).  The tensor-core
 * kernels wait for their matrix operations on an mbarrier; each wait gives up
 * after 2^18 attempts (about 1 s on GB300), records the expiry in a status
 * word and lets the kernel finish, and the call then fails with
 * FPT_EDEVICE_STATUS instead of hanging the GPU.  This entry runs that same
 * wait, in one warp, on an mbarrier that nothing arrives at, so it must
 * expire.  It writes *expired_out = 1 when it did, 0 otherwise, and the
 * kernel's duration in seconds to *seconds_out (may be NULL).  The context
 * stays usable.  Synchronises `stream`. */
int fpt_wait_selftest(int32_t* expired_out, double* seconds_out, void* stream);

/* Failure injection on the host (no paper counterpart; for tests of the error
 * paths without faulting a GPU).
 * fpt_inject_alloc_failures(count): the next `count` device allocations of
 * the library's scratch (any entry point) fail as if the device were full:
 * no memory is requested, the call returns FPT_ENOMEM, and later calls run
 * normally.  count = 0 cancels pending failures; count < 0 is FPT_EINVAL.
 * fpt_inject_status(bits): the next fpt_simulate, fpt_simulate_batch or
 * fpt_simulate_batch_host call starts its device status word at `bits`
 * instead of 0; the kernels run normally and the call returns
 * FPT_EDEVICE_STATUS when bits != 0 (the path a device-side check takes).
 * Both settings are process-wide. */
int fpt_inject_alloc_failures(int32_t count);
int fpt_inject_status(uint32_t bits);

/* Measured throughput of the execution pipes the kernels are bound by, on the
 * current device (no paper counterpart: the denominators of the kernels'
 * rooflines).  Each figure is thread operations per second of a loop of one
 * instruction kind over independent dependency chains on every SM (32 warps
 * per SM), timed with CUDA events after a warm-up launch, at the clock the GPU
 * runs at during the call:
 *   fp64_fma_per_s   binary64 fused multiply-adds (the FP64 pipe),
 *   xu_lg2_per_s     lg2.approx.f32 (the XU / MUFU pipe),
 *   wide_mul_per_s   mul.wide.u32, the 32 x 32 -> 64-bit multiply of a
 *                    Philox round (the fma-heavy pipe),
 *   fp32_fma_per_s   binary32 fused multiply-adds.
 * Takes about 0.1 s; synchronises `stream`. */
typedef struct {
    double fp64_fma_per_s;
    double xu_lg2_per_s;
    double wide_mul_per_s;
    double fp32_fma_per_s;
} fpt_pipe_rates_out;
int fpt_pipe_rates(fpt_pipe_rates_out* out, void* stream);

/* Human-readable name of a return code (static string). */
const char* fpt_strerror(int code);
/* Description of the last failure in the calling thread ("" if none). */
const char* fpt_last_error(void);
/* Library ABI version (FPT_ABI_VERSION of the build). */
int fpt_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FPT_H */
