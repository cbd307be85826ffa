/*
 * QoZ oracle: plain, slow, single-threaded CPU restatement of the QoZ method
 * (arXiv 2310.14133, "Dynamic Quality Metric Oriented Error-bounded Lossy
 * Compression for Scientific Datasets").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code with the CUDA library.
 *
 * Conventions
 *   - dims are slowest-first: 2D (ny, nx), 3D (nz, ny, nx); x is contiguous.
 *   - all floating-point arithmetic on field values is IEEE binary32 with
 *     contraction disabled (-ffp-contract=off) and a fixed evaluation order.
 *   - interpolator type: 0 = linear, 1 = cubic.
 *   - dimension order: index into the lexicographic list of permutations of
 *     the axes (3D: 012,021,102,120,201,210; 2D: 01,10), Sec. 5.2.2.
 *   - quant code 0 marks an unpredictable (or anchor) point; otherwise
 *     code = q + 32768 with |q| <= 32767.
 */
#ifndef QOZ_ORACLE_H
#define QOZ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LEVELS 8
#define ORC_RADIUS 32768

typedef struct {
  int32_t anchor_stride;               /* power of two; levels L = log2(stride) */
  uint8_t interp[ORC_MAX_LEVELS];      /* interp[l-1] for level l */
  uint8_t order[ORC_MAX_LEVELS];       /* order[l-1] for level l */
  double alpha, beta;                  /* Eq. (ebl) */
} orc_params;

/* Per-level statistics of one predictor run (used by Algorithm 1). */
typedef struct {
  double l1[ORC_MAX_LEVELS];           /* sum over level-l points of |x - pred| */
  int64_t cnt[ORC_MAX_LEVELS];         /* number of level-l points */
} orc_level_stats;

/* Value range over the finite values of x (Sec. 7.1.4: e = eps * vrange).
 * Returns the number of finite values; min = max = 0 when there is none. */
int64_t orc_value_range(const float* x, int64_t n, float* out_min, float* out_max);

/* Level-wise error bounds, Eq. (ebl): e_l = e / min(alpha^(l-1), beta),
 * l = 1..L, written to el[l-1].  alpha^(l-1) by repeated multiplication. */
void orc_level_bounds(double e, double alpha, double beta, int L, double* el);

/* Permutation table entry: axes of order index `ord` for ndims axes (the
 * dimension orders of Sec. 5.2, enumerated lexicographically). */
void orc_order_axes(int ndims, int ord, int* axes);

/* Multi-level interpolation predictor + linear-scale quantizer (Sec. 5).
 * x[N] input; codes[N], recon[N] outputs (recon may be NULL); anchors gets
 * the losslessly stored anchor values in array order (may be NULL).
 * Unpredictable points are returned sorted by linear index; at most `cap` are
 * written, the full count is returned in *n_unpred.
 * stop_level: levels below it are not processed (1 = whole field).
 * stats may be NULL.  Returns 0 on success, nonzero on invalid arguments. */
int orc_compress(const float* x, int ndims, const int64_t* dims, double e,
                 const orc_params* p, int stop_level,
                 uint16_t* codes, float* recon, float* anchors, int64_t* n_anchors,
                 int64_t* unpred_idx, float* unpred_val, int64_t cap, int64_t* n_unpred,
                 orc_level_stats* stats);

/* Mirror of orc_compress (decompression, Sec. 5.1): rebuilds the field from
 * codes, anchors and the sorted unpredictable list. */
int orc_decompress(const uint16_t* codes, int ndims, const int64_t* dims, double e,
                   const orc_params* p, const float* anchors,
                   const int64_t* unpred_idx, const float* unpred_val, int64_t n_unpred,
                   float* out);

/* Number of anchor points (Sec. 5.2.1: all coordinates multiples of the
 * stride). */
int64_t orc_anchor_count(int ndims, const int64_t* dims, int anchor_stride);

/* 65536-bin histogram of the quant codes of non-anchor points: the counts
 * the rate estimate of Sec. 6.1 is computed from. */
void orc_histogram(const uint16_t* codes, int ndims, const int64_t* dims,
                   int anchor_stride, uint64_t* hist);

/* Total length in bits of an optimal (Huffman) prefix code for the symbol
 * counts hist[0..K-1]; a single used symbol costs 1 bit per occurrence. */
uint64_t orc_huffman_bits(const uint64_t* hist, int K);

/* Entropy stage (qoz_oracle_entropy.cpp), the Huffman coding whose size the
 * rate estimate of Sec. 6.1 stands for: Huffman code lengths of
 * hist[0..K-1] with the stated tie rule (returns the longest length, 0 if no
 * symbol is used); canonical codes from the lengths (RFC 1951 Sec. 3.2.2);
 * chunked MSB-first encoding (returns the total 32-bit words, < 0 on error);
 * decoding (0 on success). */
int orc_huffman_lengths(const uint64_t* hist, int K, uint8_t* len);
void orc_canonical_codes(const uint8_t* len, int K, uint64_t* code);
int64_t orc_huffman_encode(const uint16_t* sym, int64_t n, int chunk, const uint8_t* len,
                           const uint64_t* code, uint64_t* offs, uint32_t* words,
                           int64_t cap_words);
int orc_huffman_decode(const uint32_t* words, const uint64_t* offs, int64_t n, int chunk,
                       const uint8_t* len, const uint64_t* code, int K, uint16_t* out);
/* Sub-run table of the chunked stream: a chunk of `chunk` >= 1024 codes is
 * cut into S = chunk / 512 runs of 512 codes, and the table holds, per chunk
 * in order, the coded length in bits of its first S - 1 runs (runs past the
 * end of the codes count 0); chunks of fewer than 1024 codes have none.
 * Writes n_chunks * (S - 1) entries to sub (none when S == 1); returns S, or
 * -1 for a symbol without a code. */
int orc_huffman_subruns(const uint16_t* sym, int64_t n, int chunk, const uint8_t* len,
                        uint16_t* sub);

/* Rate estimate: Huffman bits of the codes + 32 bits per unpredictable value
 * + 32 bits per anchor. */
double orc_estimate_bits(const uint64_t* hist, int64_t n_unpred, int64_t n_anchors);

/* Metrics, Sec. 3: maximum absolute error; mean squared error (the MSE of
 * Eq. (psnr)). */
double orc_max_abs_err(const float* a, const float* b, int64_t n);
double orc_mse(const float* a, const float* b, int64_t n);
/* Eq. (ac): autocorrelation at lag k of the errors e_i = b_i - a_i over the
 * flattened arrays: the mean over the n - k pairs of (e_i - mu)(e_{i+k} - mu)
 * divided by sigma^2, mu and sigma^2 the population mean and variance of all
 * n errors; 0 when sigma^2 = 0 or n <= k. */
double orc_autocorr(const float* a, const float* b, int64_t n, int64_t k);
/* Eq. (ac) over errors cut into blocks (block j = e[starts[j] ..
 * starts[j+1])), as the tuner scores its sampled blocks (Sec. 6.1): pairs
 * stay inside a block, mu and sigma^2 are over all errors. */
double orc_autocorr_blocks(const double* e, const int64_t* starts, int64_t nblocks, int64_t k);
/* Eq. (psnr): 20 log10(vrange / sqrt(MSE)), +inf when the MSE is 0. */
double orc_psnr(const float* a, const float* b, int64_t n, double vrange);
/* Eq. (ssim): mean SSIM over all box windows of edge `win` placed every `step` points
 * that lie fully inside the array; c1 = (0.01 vrange)^2, c2 = (0.03 vrange)^2.
 * Returns the number of windows in *n_windows and the SUM of window SSIMs in
 * *sum (either may be NULL); the return value is the mean (NaN if none). */
double orc_ssim(const float* a, const float* b, int ndims, const int64_t* dims,
                int win, int step, double vrange, int64_t* n_windows, double* sum);


/* ------------------------------------------------------------------------
 * Online tuning, Sec. 6
 * ---------------------------------------------------------------------- */

#define ORC_METRIC_MAXERR 0
#define ORC_METRIC_PSNR 1
#define ORC_METRIC_SSIM 2
#define ORC_METRIC_AC 3   /* lag-1 autocorrelation of the errors, lower is better */

typedef struct {
  int32_t block;          /* sample block size b (power of two); blocks hold b+1 points per axis */
  double rate;            /* sampling rate r; stride S = round(b * r^(-1/d)) */
  int32_t n_orders;       /* 2: increasing/decreasing axis order only; 6: all (3D) */
  int32_t n_alpha;
  double alphas[8];
  int32_t n_beta;
  double betas[8];
  int32_t ssim_win, ssim_step;
  int32_t anchor_stride;  /* of the full field */
} orc_tune_opts;

/* Result of one trial compression of all sampled blocks. */
typedef struct {
  double bits;            /* Huffman bits of the aggregated codes + 32 U + 32 A */
  double B;               /* bits per sampled point */
  int64_t npts, n_unpred, n_anchors;
  double max_err, sse;    /* over the sampled points */
  double ssim_sum;
  int64_t ssim_n;
  orc_level_stats stats;  /* summed over blocks */
  double ac;              /* lag-1 error autocorrelation, pooled over the blocks */
} orc_trial;

typedef struct {
  orc_params params;
  double e;               /* absolute bound to compress with */
  double B, M;            /* sampled bit rate and metric of the chosen setting */
  int32_t n_trials;
  int32_t n_blocks;
  int64_t n_sampled_points;
  double alg1_score[ORC_MAX_LEVELS];
} orc_tune_result;

/* Uniform block sampling, Sec. 6.1.  Writes block origins (3 per block,
 * slowest-first, unused axes 0) and the common block extent; returns the
 * number of blocks (at most cap are written). */
int64_t orc_sample_blocks(int ndims, const int64_t* dims, int b, double rate,
                          int64_t* origins, int64_t cap, int64_t* block_dims, int64_t* stride);

/* Trial compression of the sampled blocks (Sec. 6.1) with params p (anchor
 * stride of the blocks = p->anchor_stride) at absolute bound e, down to
 * stop_level. */
int orc_block_trial(const float* x, int ndims, const int64_t* dims,
                    const int64_t* origins, int64_t nblocks, const int64_t* block_dims,
                    const orc_params* p, double e, int stop_level, int ssim_win, int ssim_step,
                    double vrange, orc_trial* out);

/* Metric value of a trial, higher is better (the M of Sec. 6.3): PSNR (dB),
 * SSIM, -AC (lag 1, pooled over the blocks) or -max error. */
double orc_trial_metric(const orc_trial* t, int metric, double vrange);

/* Table I comparison of the incumbent I = (b1, m1) with the challenger
 * II = (b2, m2), both at bound e (metric m higher-is-better).
 * Returns 0 (keep I), 1 (II replaces I), or -1 when the case needs one more
 * trial of II: then *second_scale is set to 0.8 (case 3) or 1.2 (case 4) and
 * the caller runs II at second_scale * e and calls again with (b2p, m2p).
 * On the first call pass b2p = m2p = NaN. */
int orc_table1(double b1, double m1, double b2, double m2, double b2p, double m2p,
               double* second_scale);

/* Sec. 6.3.2 keep-best over n candidates taken in order (alpha ascending,
 * then beta), from each one's rate B[k] and metric M[k] at the user's bound.
 * The incumbent is solution I, the new candidate solution II; when Table I
 * needs II's second point (0.8 e in case 3, 1.2 e in case 4) retrial(ctx, k,
 * scale, &B', &M') supplies it (nonzero return: failure).  maxerr_mode
 * compares B alone (strictly lower replaces).  Returns the kept index, or -1
 * on failure. */
/* Candidate k (0 .. n_alpha n_beta - 1) of the (alpha, beta) search: alpha
 * ascending in the outer loop, beta in the inner one. */
void orc_ab_candidate(const orc_tune_opts* o, int k, double* alpha, double* beta);
typedef int (*orc_retrial_fn)(void* ctx, int k, double scale, double* b, double* m);
int orc_select_fixed(int n, const double* B, const double* M, int maxerr_mode,
                     orc_retrial_fn retrial, void* ctx);

/* Target mode (this project's reading of a target PSNR / SSIM): scale of a
 * candidate's second point (1.2 if M meets the target, else 0.8); the rate
 * at the target on the line through the two points; one secant step on
 * (log e, M) clamped to [e0/16, e_user] (returns 0: no step); the final
 * pick: the largest tried bound <= e_user that met the target, else the
 * smallest tried bound. */
double orc_target_scale(double M, double target);
double orc_target_rate(double B, double M, double B2, double M2, double target);
int orc_secant_step(double ea, double ma, double eb, double mb, double target, double e0,
                    double e_user, double* e_next);
int orc_target_pick(int n, const double* e, const double* M, double target, double e_user);

/* Whole tuner.  metric: ORC_METRIC_*; target NaN selects the paper's
 * fixed-bound mode (max-error metric: maximise compression ratio; PSNR / SSIM:
 * Table I comparisons at e); a finite target selects the target mode. */
int orc_tune(const float* x, int ndims, const int64_t* dims, double e_user, double vrange,
             int metric, double target, const orc_tune_opts* o, orc_tune_result* out);

/* ---------------------------------------------------------- learned tuner
 * (qoz_oracle_learn.cpp: definitions in its header comment) */
#define ORC_NFEAT 64
#define ORC_H 128
#define ORC_NOUT 16
#define ORC_NPARAM (ORC_H * ORC_NFEAT + ORC_H + ORC_H * ORC_H + ORC_H + ORC_NOUT * ORC_H + ORC_NOUT)

/* Learned tuner (this project's definition; the paper's concluding section
 * leaves it to future work): the 64 features of the sampled blocks
 * (origins / block_dims as written by orc_sample_blocks). */
int orc_features(const float* x, int ndims, const int64_t* dims, double rel_eb, double vrange,
                 const int64_t* origins, int64_t nblocks, const int64_t* block_dims,
                 double* out);
/* logits[B][16] of raw features X[B][64]. */
void orc_mlp_forward(const double* params, const double* mean, const double* sd,
                     const double* X, int64_t B, double* logits);
/* Mean over the batch of the summed per-head cross-entropies; grad (may be
 * NULL) receives its gradient (ORC_NPARAM values, packed like params). */
double orc_mlp_loss_grad(const double* params, const double* mean, const double* sd,
                         const double* X, const int32_t* labels, int64_t B, double* grad);
/* One Adam step (Kingma and Ba, bias-corrected moments; t = 1 for the first
 * step). */
void orc_adam_step(double* params, const double* grad, double* m, double* v, int64_t n,
                   int64_t t, double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif
