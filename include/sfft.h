/*
 * sfft.h — C ABI of the GB300 multidimensional phase-shift sparse FFT.
 *
 * The library recovers the k integer frequency vectors w_j in a box of side N
 * and the complex coefficients a_j of a d-variate black-box signal
 *     f(t) = sum_j a_j exp(2 pi i w_j . t)                 (Sec. 2.2, Eq. 9; Eq. 32)
 * by Algorithm 2 (MultiPhaseshift) in its general form.  Each round samples
 * f - g along a line t = x u / p (u an integer direction, p prime, x = 0..p-1)
 * and along its copies shifted by e_n / N, n = 1..d (Eq. 41), takes the length-p
 * DFTs of the d + 1 sample sets (Eq. 3), keeps the bins that pass the ratio test
 * for every n (Eq. 42), reads each coordinate off the phase of Y_n / Y_0 and the
 * coefficient off Y_0 / p (Eq. 41), and merges the result into the registry R
 * whose model g is subtracted in the next round.
 *
 * Conventions for every call:
 *  - Arguments named *_dev are device pointers (any allocator); the caller owns
 *    them and keeps them valid until the call returns.  Other pointers are host.
 *  - Complex numbers are interleaved (re, im).  "complex128" is two doubles,
 *    "complex64" two floats.  Frequencies are int32, row-major [count x d].
 *  - Every call returns an sfft_status; no call throws or aborts.  After
 *    SFFT_ERR_CUDA, sfft_last_cuda_error() returns the cudaError_t value.
 *  - All work is issued on the plan's stream; calls that return host-visible
 *    results (counts, stats) synchronise that stream before returning.
 *  - A plan is not thread-safe: one call at a time per plan.
 */
#ifndef SFFT_H_
#define SFFT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFFT_OK = 0,
  SFFT_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range            */
  SFFT_ERR_NOT_CONVERGED = 2, /* max_rounds reached with bins still occupied           */
  SFFT_ERR_CAPACITY = 3,      /* an output, registry or scratch capacity was exceeded   */
  SFFT_ERR_PRECISION = 4,     /* the requested N is beyond the policy's phase resolution */
  SFFT_ERR_INCONSISTENT = 5,  /* converged with more than k modes in the registry       */
  SFFT_ERR_CUDA = 6,          /* a CUDA runtime call failed (see sfft_last_cuda_error)  */
  SFFT_ERR_TIMEOUT = 7        /* a bounded device-side wait ran out                     */
} sfft_status;

/* Arithmetic of the hot path.  AUTO: sampling and DFT in float; the phase
 * ratio, frequency read-out and coefficient estimate in double when N > 2^14
 * (where float's phase resolution starts to matter against pi / N), else in
 * float.  FP32_FP64RATIO: the same with the ratio step always in double.
 * FP32: every step in float.  FP64: every step in double.
 * FP32_BF16DFT: as AUTO, except that a round whose prime is at most 8191 takes
 * its DFT (Eq. 3) as a dense contraction with the DFT matrix on the tensor
 * cores: operands split into two BF16 terms each (hi = bf16(v), lo = bf16(v -
 * hi)), three products per pair, FP32 accumulation; longer rounds use the float
 * Bluestein DFT, and no round is fused.  Its DFT carries about 2^-16 of each
 * operand's size instead of float's 2^-24 (at most 64 sample sets).
 * FP32_THEN_FP64: sfft_execute runs the rounds in float (as AUTO) until a round accepts fewer
 * than k* / 64 of the bins (k* the modes left: float's rounding no longer reads them), then
 * continues in double from the float registry, the round counter and the empty-bin reference
 * carried over: the double rounds read the modes float could not read and cancel its false
 * positives.  They keep the float rounds' empty-bin level (rho), below which the float
 * coefficients' own errors stay: coefficients of the modes found in float keep float's error
 * (the float policies' tolerance), the others double's.  opts.tau and delta apply to the float
 * rounds, the double rounds take the FP64 ones.  Plain form only: a batch of such plans is
 * INVALID_ARG.
 * DF64: as FP64, except that sampling (Alg. 2's black-box evaluation, the bulk of the work) runs
 * in double-float on the FP32 pipe: each value a pair of floats hi + lo (about 48 significant
 * bits), products exact through FMA and sums through two-sum, the samples written in double; the
 * DFT, ratio test, read-out and coefficients stay in double.  On GPUs whose FP64 rate is a small
 * fraction of FP32 this is the faster way to double-like accuracy.  Batches of DF64 plans count
 * as FP64 (they may share a batch only with each other). */
typedef enum {
  SFFT_PREC_AUTO = 0,
  SFFT_PREC_FP32_FP64RATIO = 1,
  SFFT_PREC_FP32 = 2,
  SFFT_PREC_FP64 = 3,
  SFFT_PREC_FP32_BF16DFT = 4,
  SFFT_PREC_FP32_THEN_FP64 = 5,
  SFFT_PREC_DF64 = 6
} sfft_precision;

typedef struct sfft_plan_s* sfft_plan;
typedef struct sfft_signal_s* sfft_signal;
typedef struct sfft_batch_s* sfft_batch;

/* Prime schedule (Alg. 1 and Alg. 2: p = i-th prime >= c k*, c = 5 in Sec. 5).
 * c is an input of both algorithms; c_eighths > 0 gives it in eighths (c = c_eighths / 8, so
 * 2.5 is 20), overriding c_prime, and the rule takes the i-th prime >= ceil(c k*).  A smaller c
 * samples fewer points per round (about c k* per set) at the price of more collisions (a mode
 * is alone in its bin with probability about e^{-1/c}) and so more rounds.
 * primes != NULL overrides the rule: round i uses primes[(i-1) mod n_primes].
 * p_min > 0 floors the rule: round i uses the i-th prime >= max(ceil(c k*), p_min).
 * With noisy samples the phase read-out w_n = N Arg(Y_n / Y_0) / (2 pi) of a
 * mode a varies by about N sigma / (2 pi sqrt(p) |a|), so reading modes down
 * to |a| reliably needs p of order (4 N sigma / (2 pi delta |a|))^2, which the
 * noiseless rule c k* does not give once k* is small.  The same holds for the
 * float policies' own rounding when a read-out resolves many values from one
 * phase (the tilted form's Q = (base + height) N): a floor keeps late rounds'
 * bins p |a| large against it (N = 512, Q = 5.9e5: the slowest of 256 signals
 * needs 39 rounds without a floor, 7 with p_min = 1024). */
typedef struct {
  int c_prime;            /* c; 0 means 5 (1 .. 4096) */
  int n_primes;
  const int64_t* primes;  /* host, n_primes entries, each prime and >= 5 */
  int64_t p_min;          /* 0: no floor */
  int c_eighths;          /* 0: c = c_prime; else c = c_eighths / 8 (1 .. 32768) */
} sfft_pschedule;

/* Line directions (Sec. 3.2, 3.3, 4.1).  Either n_dirs explicit integer
 * directions (tilted lines), row-major [n_dirs x d], or partial unwrapping:
 * n_blocks blocks of the coordinates, block q covering block_sizes[q]
 * consecutive coordinates, whose direction has N^r on the block's r-th
 * coordinate (Eq. 35-38).  Round i uses direction / block (i mod count), the
 * paper's m = (i mod d2) + 1 in 1-based numbering.  Both empty means one block
 * per the default rule: the smallest b with N^b >= 4 c k, d / b blocks; with
 * opts.shift = TILT, both empty means Alg. 3's two rotated axes. */
typedef struct {
  int n_dirs;
  const int64_t* dirs;      /* host */
  int n_blocks;
  const int* block_sizes;   /* host */
} sfft_tilts;

typedef struct {
  int precision;     /* sfft_precision */
  int box_lo;        /* 0: frequencies in [0, N); -N/2: the paper's [-N/2, N/2) */
  double tau;        /* ratio-test tolerance (Eq. 8, 42); 0 = policy default      */
  double rho;        /* empty-bin level / (p * first-round largest bin / p); 0 = default */
  double delta;      /* max distance of N Arg/(2 pi) from an integer; 0 = default */
  double noise_sigma;/* known noise level of the samples; adds 6 sigma sqrt(p)   */
  int max_rounds;    /* 0 = 64 + 4 ceil(log2 k)                                   */
  int profile;       /* 1: time each kernel class with CUDA events into sfft_stats */
  int graph;         /* 1: run the round loop as one CUDA graph whose while-loop the device ends */
  int coef_set0;     /* 1: coefficient a = Y_0[h] / p as printed in Eq. 41; 0 (default): the mean
                        over the d + 1 sets of Y_n[h] e^{-2 pi i w_n / N} / p, equal to it for a
                        single-mode bin and less affected by rounding */
  int residual;      /* sfft_residual: where g, built from the registry, leaves f each round */
  int shift;         /* sfft_shift: which shifted copies of the line are sampled */
  int unfused;       /* FP32 policies run each signal's rounds of Bluestein length <= 2048 in one
                        fused kernel, one block per signal; 1: every round through the batched
                        kernels (same arithmetic, other summation order of the samples) */
  int tilt_base;     /* shift = TILT: the rotation of Sec. 3.3, sin = tilt_height / tilt_hypo,  */
  int tilt_height;   /* cos = tilt_base / tilt_hypo (Eq. 25): a primitive Pythagorean triple,   */
  int tilt_hypo;     /* both legs >= 1 and <= 2^20; Theorem 1 wants tilt_base > 2 N (see below) */
  int fuse_max_len;  /* FP32 policies: rounds whose Bluestein length is at most this (and at most the
                        fused kernel's limit for the slot's set count) run fused; 0: that limit */
  int empty_rounds;  /* rounds in a row with no bin of any set above the empty-bin level that end the
                        recovery; 0: the number of line directions under the float policies, 1
                        under FP64 (see the stop rule below) */
} sfft_opts;

/* Stop rule.  The recovery ends when empty_rounds rounds in a row, on successive line directions,
 * find no bin of any set above the empty-bin level (the residual is empty).  A read-out that is
 * wrong in a coordinate outside its round's block passes the own-bin check (w . u) mod p = h,
 * since u is zero there, and one wrong by a multiple of p inside the block passes it too (a
 * collision that slipped through the ratio test reads such values).  The registry then holds w'
 * instead of w, and the pair shares a bin on every line that does not separate them, where set
 * 0 cancels and the shifted sets differ by a phase of only 2 pi |w_n - w'_n| / N, below the level
 * at large N.  A later line of the block where they differ, with another prime, separates them:
 * so the float policies wait for an empty round on every direction.  The FP64 policy's ratio
 * test (tau = 1e-7) lets a collision through with negligible probability, and its read-outs do
 * not slip, so one empty round ends it. */

/* The shifted sample sets (Alg. 2).  COORD (default): one set per coordinate, shifted by e_n / N,
 * reads w_n = N Arg(Y_n / Y_0) / (2 pi); d + 1 sets.  BLOCK (Alg. 2 as printed): one set per
 * block of the partial unwrapping (tilts.block_sizes, or the default rule), shifted by
 * v_n / (2 N^{d1}) along the block's unwrap vector (N^r on its r-th coordinate, Eq. 35); it reads
 * the block's unwrapped frequency 2 N^{d1} Arg(Y_n / Y_0) / (2 pi) and splits it into d1 base-N
 * digits; 1 + (number of blocks) sets.  With BLOCK the precision policy follows N^{d1}: AUTO
 * reads phases in double above 2^14, and the float policies return PRECISION above 2^20.
 *
 * TILT (Alg. 3, Sec. 3.3; d = 2 only): the lines run along the rotated axes in turn, axis
 * (i mod 2) + 1 in round i, which are the integer directions (base, -height) and (height, base)
 * (Eq. 27 after the factor hypo) unless tilts.dirs gives others; set n = 1, 2 is shifted by
 * eps = 1 / Q along rotated axis n, Q = (base + height) N.  A mode w is seen with the rotated
 * frequencies w~ = (base w_1 - height w_2, height w_1 + base w_2), each read as
 * Q Arg(Y_n / Y_0) / (2 pi) within the box's window; the pair is turned back (Alg. 3, last step)
 * to hypo^2 w and accepted only when it divides exactly and lands in the box.  With
 * base > 2 N and gcd(base, height) = 1 no two modes of the box share a rotated coordinate
 * (Theorem 1), which resolves configurations no parallel projection separates (the corners of
 * axis-aligned rectangles).  Precision follows Q: AUTO reads phases in double above 2^15, the
 * float policies return PRECISION above 2^21, and Q may not exceed 2^40.  INVALID_ARG for
 * d != 2 or a triple that is not primitive Pythagorean. */
typedef enum { SFFT_SHIFT_COORD = 0, SFFT_SHIFT_BLOCK = 1, SFFT_SHIFT_TILT = 2 } sfft_shift;

/* Alg. 2 removes g (the function of the registry's modes) from f before each round's
 * test (Sec. 5, "Algorithm").  SAMPLES evaluates f - g at every sample point, as the
 * algorithm writes it: the sampling kernel sums k + |R| modes.  BINS (default) samples
 * f alone and, by the linearity of the DFT, subtracts g's transform bin by bin: mode
 * (w, a) of the registry removes p a e^{2 pi i w_n / N} from bin (w . u) mod p of set n,
 * O(|R| (d + 1)) work instead of O(p |R| (d + 1)).  Both give the same sets; the
 * coefficients agree to the policy's rounding. */
typedef enum { SFFT_RESIDUAL_BINS = 0, SFFT_RESIDUAL_SAMPLES = 1 } sfft_residual;

#define SFFT_STATS_MAX_ROUNDS 256
/* kernel classes of sfft_stats.kernel_ms / kernel_launches: round setup and
 * per-prime tables, mode projection, sampling, DFT, classification, registry
 * merge + prune + output, and the fused kernel that runs whole rounds on short lines */
#define SFFT_NKCLASS 7
typedef struct {
  int rounds;                     /* rounds run, including the final empty one  */
  int converged;                  /* 1 when the last round found no occupied bin */
  int64_t samples;                /* black-box samples, sum over rounds of (d+1) p */
  int64_t terms;                  /* sample terms, sum over rounds of (d+1) p K  */
  int64_t terms_fused;            /* of these, the terms of rounds run by the fused kernel */
  int64_t p[SFFT_STATS_MAX_ROUNDS];
  int32_t K[SFFT_STATS_MAX_ROUNDS];        /* modes summed per sample: k, or k + |R| under SAMPLES */
  int32_t accepted[SFFT_STATS_MAX_ROUNDS]; /* bins accepted in the round */
  int32_t registry[SFFT_STATS_MAX_ROUNDS]; /* live registry entries after the round */
  int64_t kernel_launches[SFFT_NKCLASS];   /* kernels launched, per class */
  double kernel_ms[SFFT_NKCLASS];          /* CUDA-event time per class (opts.profile) */
} sfft_stats;

/* Create a plan for signals of dimension d, box side N and sparsity k.
 * Allocates every device buffer the hot path needs for any round (sized by k,
 * d and the largest prime the schedule can reach); nothing is allocated
 * during execute.  stream: a cudaStream_t, or NULL for the default stream.
 * pschedule, tilts, opts may be NULL (defaults).  Errors: INVALID_ARG for
 * d < 1, N < 2, k < 0, a direction that overflows int64, a largest prime at or
 * above 2^22 under a float policy, or bad options (including a tilted form that
 * is not two-dimensional or whose triple is not primitive Pythagorean);
 * PRECISION when N exceeds 2^23 under a float policy, or when the block or
 * tilted read-out resolves more values than the policy's phase precision;
 * CUDA when an allocation fails. */
sfft_status sfft_plan_create(int d, int64_t N, int64_t k, const sfft_pschedule* pschedule,
                             const sfft_tilts* tilts, const sfft_opts* opts, void* stream,
                             sfft_plan* plan_out);
void sfft_plan_destroy(sfft_plan plan);

/* A synthetic black box f(t) = sum_j coeffs_j exp(2 pi i freqs_j . t) with k
 * modes.  freqs_dev: int32 [k x d] device; coeffs_dev: complex128 [k] device.
 * Both are copied; the handle owns its copy until sfft_signal_destroy.
 * noise_sigma >= 0: every sample the method takes carries complex Gaussian
 * noise, Re and Im each N(0, sigma^2 / 2).  Sample (set n, point x) of round i
 * draws Philox4x32-10 (Salmon et al., SC 2011) of the counter (x, n, i, 0)
 * under the key (noise_seed mod 2^32, noise_seed div 2^32), and its first two
 * words w0, w1 give sqrt(-2 ln((w0 + 1/2) / 2^32)) e^{2 pi i w1 / 2^32}
 * sigma / sqrt(2) (Box-Muller).  The plan's opts.noise_sigma is the level the
 * thresholds assume.  INVALID_ARG for a negative or non-finite noise_sigma. */
sfft_status sfft_signal_synthetic(int d, int64_t N, int64_t k, const int32_t* freqs_dev,
                                  const double* coeffs_dev, double noise_sigma,
                                  uint64_t noise_seed, sfft_signal* signal_out);
void sfft_signal_destroy(sfft_signal signal);

/* Replace the modes of an existing black box with k new ones (k at most the
 * count it was created with; same d and N).  freqs_dev / coeffs_dev as in
 * sfft_signal_synthetic.  Allocates nothing; the copy runs on the legacy
 * default stream and has finished when the call returns. */
sfft_status sfft_signal_assign(sfft_signal signal, int64_t k, const int32_t* freqs_dev,
                               const double* coeffs_dev);

/* Refill n black boxes at once, each as sfft_signal_assign would, from one packed
 * pair of device arrays: signal s takes ks[s] modes (ks: host), its frequency rows
 * (d_s int32 each) following those of signals 0..s-1 in freqs_dev and its
 * coefficients (complex128) following theirs in coeffs_dev.  The copies are
 * enqueued on `stream` (a cudaStream_t, NULL for the legacy default stream) and
 * nothing waits for them: work enqueued later on the same stream sees the new
 * modes.  Allocates nothing.  INVALID_ARG, with nothing changed, if n < 0, a
 * handle is NULL or some ks[s] is negative or above the handle's capacity. */
sfft_status sfft_signal_assign_many(int n, const sfft_signal* signals, const int64_t* ks,
                                    const int32_t* freqs_dev, const double* coeffs_dev, void* stream);

/* Run Algorithm 2 on the signal until a round finds no occupied bin.
 * Writes the live registry (unordered) to freqs_out_dev (int32 [capacity x d])
 * and coeffs_out_dev (complex128 [capacity]); *n_found = number of entries.
 * stats may be NULL.  Returns NOT_CONVERGED after max_rounds (outputs still
 * written), CAPACITY if more than capacity entries are live (nothing written
 * beyond capacity), INCONSISTENT if more than k entries are live at the end. */
sfft_status sfft_execute(sfft_plan plan, sfft_signal signal, int64_t capacity,
                         int32_t* freqs_out_dev, double* coeffs_out_dev, int64_t* n_found,
                         sfft_stats* stats);

/* ---- batches: many independent signals in every launch -------------------- */

/* A batch of n signal slots; slot s takes d, N, k, schedule, directions and
 * thresholds from plans[s] (the same plan may appear many times).  All plans
 * must share the float-or-double choice of their precision.  The batch owns
 * its own device buffers; the plans may be destroyed afterwards.  graph is a
 * set of flags: SFFT_BATCH_GRAPH runs the rounds as one CUDA graph with a
 * device-ended while-loop; SFFT_BATCH_PROFILE (also on when some plan has
 * opts.profile) enqueues the rounds from the host with CUDA events between
 * the kernel classes and fills sfft_stats.kernel_ms.  INVALID_ARG for other
 * bits. */
#define SFFT_BATCH_GRAPH 1
#define SFFT_BATCH_PROFILE 2
sfft_status sfft_batch_create(int n, const sfft_plan* plans, void* stream, int graph, sfft_batch* batch_out);
void sfft_batch_destroy(sfft_batch batch);
int64_t sfft_batch_device_bytes(sfft_batch batch);

/* Recover all n signals (signals[s] must match slot s's d and N, with at most
 * its k modes).  Outputs are packed: slot s writes up to capacities[s] rows
 * starting at row sum_{t<s} capacities[t] of coeffs_out_dev (complex128) and
 * at element sum_{t<s} capacities[t] d_t of freqs_out_dev (int32).
 * n_found[s] and status[s] (an sfft_status) are host arrays of n entries.
 * Returns the first non-OK slot status, else OK.  stats (nullable) sums the
 * work over slots and records the per-round history of slot 0. */
sfft_status sfft_batch_execute(sfft_batch batch, const sfft_signal* signals, const int64_t* capacities,
                               int32_t* freqs_out_dev, double* coeffs_out_dev, int64_t* n_found,
                               int32_t* status, sfft_stats* stats);

/* ---- the steps of one round, callable on their own ------------------------ */

/* Kernel (a), sample-and-residual (Alg. 2 sampling; Eq. 41): for the K modes
 * (freqs_dev int32 [K x d], coeffs_dev complex128 [K]) writes
 *     y[n][x] = sum_j coeffs_j exp(2 pi i w_j . (x u / p + s_n)),
 * s_0 = 0, s_n the plan's shifted sets (e_n / N unless opts.shift says otherwise),
 * x < p, n <= d, to y_out_dev, row-major [(d+1) x p],
 * complex64 for float plans and complex128 for FP64 plans.  u: host int64 [d].
 * Requires 2 <= p <= the plan's largest prime; CAPACITY when K exceeds the
 * plan's k. */
sfft_status sfft_sample(sfft_plan plan, int64_t p, const int64_t* u, int64_t K,
                        const int32_t* freqs_dev, const double* coeffs_dev, void* y_out_dev);

/* Kernel (b), batched prime-length DFT (Eq. 3): Y[r][h] = sum_x y[r][x]
 * exp(-2 pi i h x / p) for rows r < n_rows, h < p.  y_dev and Y_out_dev are
 * [n_rows x p] in the plan's complex type; n_rows <= d + 1. */
sfft_status sfft_dft(sfft_plan plan, int64_t p, int n_rows, const void* y_dev, void* Y_out_dev);

/* Kernel (c), bin classification and read-out (Eq. 41-42): for the
 * sfft_plan_sets(plan) x p transforms Y_dev (plan's complex type; d + 1 rows in
 * the coordinate and tilted forms) of the line with direction u (host int64 [d])
 * returns every bin h with |Y_0[h]| > eta_bin that passes the ratio test for all
 * n, whose read-out (the plan's shift form) rounds to integers within delta and
 * lands in its own bin.  Outputs (device): h_out int32 [capacity], freqs_out
 * int32 [capacity x d], coeffs_out complex128 [capacity] (the plan's coefficient
 * estimator: Y_0[h] / p with opts.coef_set0, else the mean over the sets);
 * *n_out = count (order unspecified).  CAPACITY if more bins pass than fit. */
sfft_status sfft_classify(sfft_plan plan, int64_t p, const int64_t* u, const void* Y_dev,
                          double eta_bin, int64_t capacity, int32_t* h_out_dev,
                          int32_t* freqs_out_dev, double* coeffs_out_dev, int64_t* n_out);

/* Allocation-free sampling (kernel (a) without a plan).  The paper has no
 * counterpart: this serves callers that may not allocate device memory at the
 * point where they need samples (a fixed memory pool that must not grow, a
 * process that forbids cudaMalloc after start-up, code that cannot own a plan).
 * Writes the same samples as sfft_sample,
 *     y[n][x] = sum_j coeffs_j exp(2 pi i w_j . (x u / p + s_n)),  s_0 = 0, s_n = e_n / N,
 * complex64 [(d+1) x p] to y_out_dev, for K modes (freqs_dev int32 [K x d],
 * coeffs_dev complex128 [K], frequencies in [box_lo, box_lo + N)), u host int64 [d].
 * Work is enqueued on `stream` (a cudaStream_t, NULL = default) and the call
 * returns without waiting; y_out_dev is complete when the stream reaches it.
 * Scratch: one 8 MiB device array inside the library, present on every GPU
 * that loads it until the process exits; it must hold p complex64 entries, two
 * int32 arrays and (d+1) complex64 arrays of K rounded up to 32, each padded to
 * 256 bytes (for d = 5: p + 7 K' complex64-sized entries up to 8 MiB).  Larger
 * requests return SFFT_ERR_CAPACITY; d > 32, N > 2^23 or p >= 2^22 return
 * SFFT_ERR_INVALID_ARG.  The first call on each device looks the array's
 * device address up (cudaGetSymbolAddress) with that device current, so make
 * that first call before any stream capture.  All calls share the array, and
 * each overwrites every scratch entry it reads, so nothing needs clearing; calls
 * whose work overlaps on the GPU (other streams, other threads) race on it and
 * must be serialised by the caller.  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
sfft_status sfft_sample_noalloc(int d, int64_t N, int64_t p, const int64_t* u, int64_t K,
                                const int32_t* freqs_dev, const double* coeffs_dev, void* y_out_dev,
                                int box_lo, void* stream);

/* Plan facts: largest prime any round can use, mode capacity (k + registry),
 * bytes of device memory the plan holds. */
int64_t sfft_plan_max_prime(sfft_plan plan);
int64_t sfft_plan_mode_capacity(sfft_plan plan);
/* Sample sets per round: d + 1 (coordinate shifts) or 1 + blocks (block shifts); -1 for NULL. */
int sfft_plan_sets(sfft_plan plan);
int64_t sfft_plan_device_bytes(sfft_plan plan);

/* The last cudaError_t seen by any call of this thread (0 if none). */
int sfft_last_cuda_error(void);
const char* sfft_status_string(sfft_status s);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_H_ */
