/*
 * qoz.h -- C ABI of the GB300 (sm_103a) QoZ library.
 *
 * QoZ is the quality-metric-oriented, error-bounded lossy compressor of
 * arXiv 2310.14133.  This library implements its data path on one GPU:
 *   - the multi-level interpolation predictor with anchor points and
 *     level-adapted interpolators (Sec. 5.1, Sec. 5.2.1, Sec. 5.2.2),
 *   - level-wise error bounds e_l = e / min(alpha^(l-1), beta) (Eq. ebl),
 *   - linear-scale quantization and its mirror on decompression (Sec. 5.1),
 *   - the quality metrics max error, PSNR (Eq. psnr) and SSIM (Eq. ssim,
 *     Eq. ssim2), and the Huffman rate estimate of the quantization bins
 *     (Sec. 6.1),
 *   - the sampled online tuner (Sec. 6.1 sampling, Algorithm 1, Sec. 6.3
 *     candidates and Table I comparisons),
 *   - the lag-k error autocorrelation (Eq. ac) and its tuning mode,
 *   - a learned tuner (features, a small network and its training), which
 *     the paper's conclusion leaves to future work,
 *   - batched compression of many fields in one plan,
 *   - serialization with canonical Huffman coding of the codes (the entropy
 *     stage the rate estimate of Sec. 6.1 stands for).
 *
 * General conventions
 *   - Field dims are slowest-first: 2D {ny, nx}, 3D {nz, ny, nx}; the last
 *     axis is contiguous.  Values are IEEE binary32.
 *   - Pointers named d_* are device pointers of the current CUDA device;
 *     h_* are host pointers.  Inputs are never modified.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls return after the host-visible
 *     results they document (counts, sizes) are known, which synchronises the
 *     stream where stated.
 *   - Every entry point returns a qoz_status; on failure qoz_last_error()
 *     gives a message (thread-local).  No call throws across the ABI.
 *   - Quant codes are uint16 in array order: 0 marks an anchor or an
 *     unpredictable point, otherwise code = q + 32768 with |q| <= 32767.
 *   - Interpolator per level: 0 linear, 1 cubic.  Dimension order per level:
 *     index into the lexicographic permutations of the axes (3D: 012 021 102
 *     120 201 210; 2D: 01 10); the first axis of the order is interpolated
 *     first (Sec. 5.2.2).
 */
#ifndef QOZ_H
#define QOZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QOZ_MAX_LEVELS 8

typedef enum {
  QOZ_OK = 0,
  QOZ_EINVAL = 1,        /* invalid argument (shape, bound, parameters) */
  QOZ_ENOMEM = 2,        /* device or host allocation failed */
  QOZ_ECUDA = 3,         /* a CUDA call or kernel launch failed */
  QOZ_ECORRUPT = 4,      /* serialized stream damaged (magic, size, checksum) */
  QOZ_ETIMEOUT = 5,      /* a bounded device wait gave up */
  QOZ_EUNSUPPORTED = 6   /* valid request that this compiled library does not handle */
} qoz_status;

typedef enum {
  QOZ_METRIC_MAXERR = 0,
  QOZ_METRIC_PSNR = 1,
  QOZ_METRIC_SSIM = 2,
  QOZ_METRIC_AC = 3  /* lag-1 error autocorrelation (Eq. ac), lower is better; no target mode */
} qoz_metric;

typedef struct {
  int32_t ndims;         /* 2 or 3 */
  int64_t dims[3];       /* slowest-first; entries past ndims ignored */
} qoz_shape;

/* The tuned parameter set theta (Sec. 3 problem statement, Eq. ebl). */
typedef struct {
  int32_t anchor_stride;               /* power of two; 0 = default (3D 32, 2D 64, Sec. 7.1.4) */
  uint8_t interp[QOZ_MAX_LEVELS];      /* interp[l-1]: interpolator of level l */
  uint8_t order[QOZ_MAX_LEVELS];       /* order[l-1]: dimension order of level l */
  double alpha;                        /* >= 1 */
  double beta;                         /* >= 1 */
} qoz_params;

typedef struct qoz_blob qoz_blob;      /* opaque compressed field; owns device memory */

typedef struct {
  qoz_shape shape;
  qoz_params params;
  double abs_eb;                       /* absolute error bound e used */
  double rel_eb;                       /* e / value range (NaN if given absolutely) */
  float vmin, vmax;                    /* value range of the finite input values */
  int64_t n_points;
  int64_t n_anchors;
  int64_t n_unpredictable;
  double est_bits;                     /* Huffman bits of the codes + 32 per unpredictable and anchor */
  double est_ratio;                    /* 32 * n_points / est_bits */
} qoz_blob_info;

/* ---------------------------------------------------------------- field ops */

/* Value range of the finite values of d_x[0..n) (Sec. 7.1.4: the
 * value-range-relative bound e = eps * (max - min)).  Synchronises `stream`.
 * h_count receives the number of finite values (may be NULL); min = max = 0
 * when there is none. */
qoz_status qoz_value_range(const float* d_x, int64_t n, float* h_min, float* h_max,
                           int64_t* h_count, void* stream);

/* Value range without any allocation, for callers that cannot allocate
 * device memory: code running where cudaMalloc is unavailable or forbidden
 * (inside a host-side memory budget, a pre-planned arena, or a capture that
 * must not add allocations).  The per-CTA partial results live in a
 * library-owned static device array, about 10 KB, that every GPU which
 * loads the library holds until the process exits; the caller passes only
 * the input and the outputs.
 *   d_minmax: device, 2 floats: min and max of the finite values of
 *             d_x[0..n) (both 0 when there is none);
 *   d_count:  device, 1 int64: number of finite values (may be NULL).
 * n must not exceed QOZ_NOALLOC_MAX_VALUES (QOZ_EUNSUPPORTED otherwise).
 * Asynchronous on `stream`; calls no cudaMalloc, cudaFree or other
 * allocating routine.  The first call on a device looks up the scratch
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is kept per device context: after
 * cudaDeviceReset the next call looks it up again (make that call before
 * any capture too).  All calls share the one array, which keeps the
 * last call's contents: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race and must be serialised by the
 * caller.  The paper has no counterpart to this entry point. */
#define QOZ_NOALLOC_MAX_VALUES ((int64_t)1 << 40)
qoz_status qoz_value_range_noalloc(const float* d_x, int64_t n, float* d_minmax, int64_t* d_count,
                                   void* stream);

/* Compress (Sec. 5): value range, anchors (Sec. 5.2.1), then levels L..1 of
 * the interpolation predictor with level-wise bounds (Eq. ebl), each level's
 * dimension passes predicting from reconstructed values and quantizing
 * linearly; then the 65536-bin code histogram.  rel_eb > 0 and finite;
 * p = NULL selects cubic, order 0, alpha = beta = 1 on every level.  The blob
 * is allocated stream-ordered on `stream`; the call synchronises `stream`
 * once, at the end, to learn the number of unpredictable points.
 * d_recon, if not NULL, receives the reconstruction the decompressor will
 * produce (N floats, caller-owned). */
qoz_status qoz_compress(const float* d_field, qoz_shape shape, double rel_eb,
                        const qoz_params* p, float* d_recon, void* stream, qoz_blob** out);

/* Same with an absolute bound e >= 0, the error bound of Sec. 3 given
 * directly instead of relative to the value range (Sec. 7.1.4): no
 * value-range pass, and the blob's vmin/vmax are then 0. */
qoz_status qoz_compress_abs(const float* d_field, qoz_shape shape, double abs_eb,
                            const qoz_params* p, float* d_recon, void* stream, qoz_blob** out);

/* Decompress (mirror of Sec. 5.1): anchors, then the same passes with
 * recon = pred + 2 e_l (code - 32768), or the stored value where code = 0.
 * d_out: caller-owned N floats.  Asynchronous on `stream`, so problems the
 * kernels find in the blob are not in the returned status: a code-0 point
 * whose index is missing from the unpredictable list (a corrupt blob whose
 * checksum still matched) is written as 0.0f and flagged in the blob;
 * qoz_blob_check reads the flag. */
qoz_status qoz_decompress(const qoz_blob* b, float* d_out, void* stream);

/* Status of the blob's last decompression (this library's check; the paper
 * has no counterpart): synchronises `stream` (NULL: the blob's stream) and
 * returns QOZ_ECORRUPT when a code-0 point had no unpredictable-list entry
 * or its coded stream did not decode, QOZ_OK otherwise.  The flags are
 * cleared at the start of every qoz_decompress. */
qoz_status qoz_blob_check(const qoz_blob* b, void* stream);

/* The blob's shape, parameters, bounds and counts, and the rate estimate of
 * Sec. 6.1 (est_bits, est_ratio: the optimal prefix-code cost of the code
 * histogram plus 32 bits per unpredictable value and per anchor), into *info
 * (host).  Reads the histogram back: synchronises the blob's stream. */
qoz_status qoz_blob_get_info(const qoz_blob* b, qoz_blob_info* info);

/* Device views of the blob's arrays (owned by the blob; valid until
 * qoz_blob_free): the quantization codes of Sec. 5.2.2 (q + 32768 per point
 * in array order, 0 for an unpredictable point or an anchor), the
 * unpredictable points (d_unpred_idx linear indices sorted ascending,
 * d_unpred_val their exact values) and the anchors of Sec. 5.2.1 (compact
 * grid, float32).  Any output pointer may be NULL. */
qoz_status qoz_blob_arrays(const qoz_blob* b, const uint16_t** d_codes,
                           const int64_t** d_unpred_idx, const float** d_unpred_val,
                           int64_t* n_unpred, const float** d_anchors, int64_t* n_anchors);

/* Copies the blob's arrays into caller-owned device buffers (any may be
 * NULL): codes N uint16, unpredictable indices / values n_unpredictable each,
 * anchors n_anchors floats.  Asynchronous on `stream`. */
qoz_status qoz_blob_copy_arrays(const qoz_blob* b, uint16_t* d_codes, int64_t* d_unpred_idx,
                                float* d_unpred_val, float* d_anchors, void* stream);

/* Copy the 65536-bin histogram of the non-anchor codes, the counts the rate
 * estimate of Sec. 6.1 is computed from, to h_hist (host, 65536 uint32), on
 * `stream` (NULL: the blob's stream), which it then synchronises. */
qoz_status qoz_blob_histogram(const qoz_blob* b, uint32_t* h_hist, void* stream);

/* Serialized form (format 3): a 160-byte header (magic, version, shape,
 * bound, params, counts, checksum), the anchors (float32), the unpredictable
 * indices (int64) and values (float32), then the code section: the codes of
 * all N points (anchors carry code 0) in canonical Huffman code, the entropy
 * stage the rate estimate of Sec. 6.1 stands for.  The code section holds a
 * 288-byte fixed part (used symbols, longest code, chunk size, chunk and
 * word counts, number of codes per length 0..63), the used symbols in
 * (length, symbol) order, the n_chunks + 1 word offsets (uint64), for chunks
 * of 1024 codes or more the run table (per chunk, the coded length in bits
 * of each 512-code run but the last, uint16, padded to 8 bytes) and the
 * stream (uint32 words; each chunk starts on a word, codes most significant
 * bit first from each word's most significant bit).  Code lengths follow
 * Huffman's construction with ties going to the leaf queue; codes are
 * RFC 1951's canonical assignment.  The writer takes the largest chunk size
 * of 256, 512, 1024, 2048 and 4096 codes that gives at least 8192 chunks
 * (else 256); a reader accepts any multiple of 8 up to 4096.  Every part is padded
 * to 8 bytes.  The checksum is a 64-bit sum of splitmix64-mixed 8-byte words.
 *
 * The stream's length depends on the code table, which is built on the
 * device: serialization synchronises `stream` once to learn it.  With
 * h_buf = NULL only *used is set (the required size).  Synchronises. */
qoz_status qoz_blob_serialize(const qoz_blob* b, void* h_buf, size_t cap, size_t* used,
                              void* stream);
/* Same stream: after the one synchronisation that sizes the stream (*used is
 * set on return), the coding, the payload copies and a host callback that
 * writes the header are enqueued on `stream` without waiting.  h_buf must be
 * pinned host memory (or the copies become synchronous) and must stay valid
 * until the stream has passed the call; the stream is complete once the
 * stream (or an event recorded after the call) is synchronized.  The blob
 * must not be freed before then, except by stream-ordered qoz_blob_free on
 * the same stream. */
qoz_status qoz_blob_serialize_async(const qoz_blob* b, void* h_buf, size_t cap, size_t* used,
                                    void* stream);
/* An upper bound on the serialized size, from the counts alone (no device
 * work): an optimal prefix code averages under 17 bits per symbol on a
 * 65536-symbol alphabet, and each chunk adds at most one partial word. */
qoz_status qoz_blob_serialize_bound(const qoz_blob* b, size_t* bound);
/* Parses a serialized stream (format 3) onto the device: checks the header,
 * the code section (a complete canonical code, consistent chunk offsets) and
 * the unpredictable list on the host, decodes the codes on the device and
 * verifies the checksum.  QOZ_ECORRUPT for any inconsistency.  Synchronises. */
qoz_status qoz_blob_deserialize(const void* h_buf, size_t size, void* stream, qoz_blob** out);

/* Releases the blob's device memory, stream-ordered on the stream the blob
 * was created on (that stream must still exist). */
void qoz_blob_free(qoz_blob* b);

/* The message of the calling thread's last failed call (thread-local; an
 * empty string if none).  Owned by the library, valid until the thread's next
 * call. */
const char* qoz_last_error(void);

/* ---------------------------------------------------------------- batches
 * Compression of many fields together (the same method as qoz_compress on
 * each field: Sec. 5.1 predictor, Sec. 5.2.1 anchors, Eq. ebl bounds).  A
 * plan fixes the fields' shapes and parameters; every run then issues each
 * level of all fields as one launch per kernel instance (fields sharing a
 * level's order and dimensionality share the launch), so the small coarse
 * levels of many fields fill the GPU together, and after the first run the
 * whole device sequence replays as one CUDA graph.  Each field's blob holds
 * exactly what qoz_compress / qoz_compress_abs would produce for it. */
typedef struct qoz_batch qoz_batch;     /* opaque plan; owns device scratch */

#define QOZ_BATCH_AUTOTUNE 1u   /* time the variants of the level-1 launches on the first run
                                   (otherwise level 1 takes bulk tensor copies where the arrays allow) */
#define QOZ_BATCH_NO_GRAPH 2u   /* issue the launches directly on every run (no CUDA graph) */

/* shapes: nfields entries; params: nfields entries or NULL (defaults as in
 * qoz_compress).  Allocates the plan's device scratch on the current device
 * (synchronous).  Errors: QOZ_EINVAL for a bad shape, parameter or count
 * (1 <= nfields <= 4096), QOZ_ENOMEM. */
qoz_status qoz_batch_create(const qoz_shape* shapes, int32_t nfields, const qoz_params* params,
                            uint32_t flags, qoz_batch** out);

/* Compresses d_fields[i] (device, 4-byte aligned, the plan's shape i) with
 * bound eb[i]: relative to the field's value range when eb_relative != 0
 * (eb > 0), absolute otherwise (eb >= 0).  outs[i] receive blobs allocated
 * stream-ordered on `stream` (free each with qoz_blob_free).  Synchronises
 * `stream` after the run and again once the unpredictable lists are copied
 * out (the plan reuses its list buffers).  A plan serves one run at a time:
 * calls on one plan must not overlap.  A field whose unpredictable points
 * overflow the plan's list is compressed again alone (qoz_compress_abs's
 * path, same result).  Errors: QOZ_EINVAL (a NULL array, a misaligned field
 * or a bad bound), QOZ_ENOMEM, QOZ_ECUDA, and QOZ_ETIMEOUT when a bounded
 * wait for a tile's bulk copy gave up in any field, after which the plan
 * serves the next call as before; on any failure no blob is returned
 * (every outs[i] = NULL). */
qoz_status qoz_batch_compress(qoz_batch* plan, const float* const* d_fields, const double* eb,
                              int32_t eb_relative, void* stream, qoz_blob** outs);

typedef struct {
  int32_t nfields;
  int32_t n_groups;            /* batched level launches per run */
  int32_t launches_per_run;    /* kernel launches per run (all kernels of the sequence) */
  int32_t graph;               /* 1 once the run sequence is a CUDA graph */
  int32_t autotuned;           /* 1 once the tile variants were timed */
  int32_t level1_groups;       /* number of level-1 launches */
  int32_t level1_variant[16];  /* variant chosen for each (first 16): 0, 1 row-copy tiles, 2 bulk
                                  copies one tile per CTA, 3 persistent bulk-copy CTAs (3-D) */
  double level1_ms[16][4];     /* timed duration of each variant (autotune; 1e30: not possible), else 0 */
  int64_t ctas_per_run;        /* CTAs of all batched level launches */
} qoz_batch_info;
qoz_status qoz_batch_get_info(const qoz_batch* plan, qoz_batch_info* info);

/* Releases the plan (synchronises the device first). */
void qoz_batch_free(qoz_batch* plan);

/* One-shot convenience: plan, run with the same relative bound for every
 * field, release. */
qoz_status qoz_compress_batch(const float* const* d_fields, const qoz_shape* shapes,
                              int32_t nfields, double rel_eb, const qoz_params* params,
                              void* stream, qoz_blob** outs);

/* ---------------------------------------------------------------- metrics */

typedef struct {
  double max_abs_err;    /* max |a - b|, exact: the difference of the maximising pair in double */
  double mse;            /* mean of (a - b)^2 over all points: compensated binary32 sums per
                            thread, double across threads (1e-6 relative of the double sum) */
  double psnr;           /* Eq. psnr: 20 log10(vrange / sqrt(mse)); +inf if mse = 0 */
  double ssim;           /* Eq. ssim: mean over windows (NaN if not requested / none) */
  int64_t ssim_windows;
  double ac;             /* Eq. ac at lag 1 of the errors b - a, flattened (row-major) order */
} qoz_metrics;

/* Quality metrics of Sec. 3 between the original d_a and the reconstruction
 * d_b.  ssim_win > 0 requests SSIM over box windows of edge ssim_win placed
 * every ssim_step points, fully inside the array, with c1 = (0.01 vrange)^2
 * and c2 = (0.03 vrange)^2 (Eq. ssim2).  Synchronises `stream`. */
qoz_status qoz_compute_metrics(const float* d_a, const float* d_b, qoz_shape shape,
                               double vrange, int32_t ssim_win, int32_t ssim_step,
                               qoz_metrics* out, void* stream);

/* Eq. (ac): autocorrelation at lag >= 1 of the errors e_i = d_b[i] - d_a[i]
 * over n values in the given (flattened) order: the mean over the n - lag
 * pairs of (e_i - mu)(e_{i+lag} - mu), divided by sigma^2, with mu and
 * sigma^2 the population mean and variance of all n errors.  One pass of
 * compensated binary32 sums per thread, double across threads and on the
 * host.  *ac = 0 when n <= lag or the variance vanishes (below 1e-6 of the
 * mean square).  Synchronises `stream`. */
qoz_status qoz_error_autocorr(const float* d_a, const float* d_b, int64_t n, int64_t lag,
                              double* ac, void* stream);

/* ---------------------------------------------------------------- tuning */

/* Options of the sampled online tuner (Sec. 6).  Zero / empty fields take
 * the paper's defaults (Sec. 7.1.4, Sec. 6.3.1): 3D block 16, rate 0.5 %;
 * 2D block 64, rate 1 %; alpha {1, 1.25, 1.5, 1.75, 2}; beta {1.5, 2, 3, 4};
 * two dimension orders (increasing and decreasing); SSIM windows 7, step 2. */
typedef struct {
  int32_t block;          /* sample block size b (power of two); blocks hold b+1 points per axis */
  double rate;            /* sampling rate r: block stride S = round(b r^(-1/d)) */
  int32_t n_orders;       /* 2: increasing/decreasing axis order; 6: all six (3D) */
  int32_t n_alpha;
  double alphas[8];
  int32_t n_beta;
  double betas[8];
  int32_t ssim_win, ssim_step;
  int32_t anchor_stride;  /* of the full field (0: 3D 32, 2D 64) */
} qoz_tune_opts;

typedef struct {
  qoz_params params;      /* chosen interpolators / orders per level, alpha, beta */
  double abs_eb;          /* bound to compress with (target mode may lower it) */
  double vmin, vmax;      /* value range of the field */
  double B;               /* sampled bit rate of the chosen setting (bits per point) */
  double M;               /* sampled metric (PSNR dB, SSIM, or -max error) */
  int32_t n_trials;       /* trial compressions of the sampled blocks that ran */
  int32_t n_blocks;
  int64_t n_sampled_points;
  double alg1_score[QOZ_MAX_LEVELS];  /* mean |x - pred| of the chosen interpolator per level */
} qoz_tune_report;

/* Sampled online tuning, Sec. 6: uniform block sampling (Sec. 6.1),
 * level-adapted interpolator selection (Algorithm 1, greedy from the top
 * level down, each level scored by the mean absolute prediction error at
 * bound e), then the (alpha, beta) candidates (Sec. 6.3.1) compared by the
 * sampled bit rate (Huffman cost of the pooled codes, Sec. 6.1) and metric:
 *   metric MAXERR, target NaN: minimum bit rate under the bound (the
 *     maximise-compression-ratio mode);
 *   metric PSNR / SSIM, target NaN: Table I comparisons at the bound e;
 *   finite target (PSNR dB or SSIM): each (alpha, beta) is scored by the bit
 *     rate interpolated at the target between two sampled bounds, then a
 *     short secant on log e picks the bound (capped at rel_eb * vrange).
 * Synchronises `stream` several times. */
qoz_status qoz_tune(const float* d_field, qoz_shape shape, double rel_eb, qoz_metric metric,
                    double target, const qoz_tune_opts* opts, void* stream,
                    qoz_tune_report* out);

/* ---------------------------------------------------------- learned tuner
 * A network that proposes the tuner's choices from features of the sampled
 * blocks, in place of the sampled trials.  The paper's concluding section
 * leaves better selection policies and hyper-parameter auto-tuning to future
 * work; the features and the network are this library's definitions:
 *
 * Features (64), over the sampled blocks of Sec. 6.1 (each block on its own)
 * with e = rel_eb * vrange (1 if 0) and L(v) = log2(1 + v / e):
 *   [0] log10(rel_eb); [1] log10(vrange / sigma), sigma the deviation of the
 *   sampled values (0 if either is 0); [2] ndims / 3; [3] log2(points) / 30;
 *   [4..6] L(mean |first difference|) per axis; [7..9] L(mean |second
 *   difference|) per axis (2-D: third slot 0); [10..33] fractions of points
 *   in 24 bins of floor(log2(|forward gradient| / e)) + 12, clamped (0 in
 *   bin 0); [34..57] the same for |x - first-order Lorenzo prediction| / e;
 *   [58..60] L(mean |x - linear interpolation|), [61..63] L(mean |x - cubic
 *   interpolation|), at half-strides 1, 2, 4 along every axis with the
 *   predictor's stencils (Sec. 5.1), targets with all four neighbours in
 *   their block.
 * Network: z = (f - mean) / std; h1 = relu(W1 z + b1) (128);
 *   h2 = relu(W2 h1 + b2) (128); logits = W3 h2 + b3 (16): heads [0:2]
 *   interpolator (linear, cubic), [2:8] dimension order (2-D: first two
 *   used), [8:13] alpha, [13:16] beta, indices into the tuner's candidate
 *   sets.  Loss: batch mean of the summed per-head softmax cross-entropies.
 *   Parameters are packed W1 (128 x 64, row-major), b1, W2 (128 x 128), b2,
 *   W3 (16 x 128), b3 (QOZ_MLP_PARAMS floats). */
#define QOZ_NFEATURES 64
#define QOZ_MLP_PARAMS 26896
typedef struct qoz_model qoz_model;    /* opaque; weights, normalisation, Adam state on the device */

/* Features of d_field (value range pass, sampling with opts as in qoz_tune)
 * into h_features (host, 64 doubles) and/or d_features (device, 64 floats);
 * either may be NULL.  Synchronises `stream`. */
qoz_status qoz_features(const float* d_field, qoz_shape shape, double rel_eb,
                        const qoz_tune_opts* opts, double* h_features, float* d_features,
                        void* stream);

/* A model on the current device: He-uniform weights from a splitmix64
 * sequence seeded by `seed`, zero biases, mean 0 / std 1 normalisation. */
qoz_status qoz_model_create(uint64_t seed, qoz_model** out);
/* Replace parameters (QOZ_MLP_PARAMS floats; resets the Adam state) and/or
 * the 64-entry normalisation; any pointer may be NULL.  Synchronous. */
qoz_status qoz_model_set(qoz_model* m, const float* h_params, const float* h_mean,
                         const float* h_sd);
qoz_status qoz_model_get(const qoz_model* m, float* h_params, float* h_mean, float* h_sd);
/* Logits (n x 16, device) of n feature rows (n x 64, device). */
qoz_status qoz_model_forward(const qoz_model* m, const float* d_features, int64_t n,
                             float* d_logits, void* stream);
/* Gradient of the loss (device, QOZ_MLP_PARAMS floats; may be NULL) for n
 * rows with labels (n x 4 int32, device: interpolator, order, alpha index,
 * beta index, each within its head); h_loss (may be NULL) receives the loss
 * and then the call synchronises.  A label outside its head makes the loss
 * NaN (it is never used as an index). */
qoz_status qoz_model_gradient(qoz_model* m, const float* d_features, const int32_t* d_labels,
                              int64_t n, float* d_grad, float* h_loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * gradient of the batch. */
qoz_status qoz_model_train_step(qoz_model* m, const float* d_features, const int32_t* d_labels,
                                int64_t n, float lr, float* h_loss, void* stream);
void qoz_model_free(qoz_model* m);

/* Tuning by the network: features, one forward pass, the argmax of each
 * head (one interpolator and order for every level, alpha and beta from
 * opts' candidate sets, which must hold 5 and 3 values).  The bound is
 * rel_eb * vrange, or with a PSNR target the uniform-error estimate
 * vrange sqrt(3) 10^(-target / 20) when that is smaller (an SSIM target
 * keeps rel_eb * vrange: qoz_tune_learned_verified sets the bound).  The
 * report's B and M are NaN (no trial ran).  Synchronises `stream`. */
qoz_status qoz_tune_learned(const float* d_field, qoz_shape shape, double rel_eb,
                            qoz_metric metric, double target, const qoz_tune_opts* opts,
                            const qoz_model* model, void* stream, qoz_tune_report* out);

/* Sampled verification of a given setting (the trials of Sec. 6.1 on the
 * sampled blocks): with target NaN one trial at rel_eb * vrange reports B and
 * M; with a PSNR or SSIM target, trials at e0 (PSNR: the uniform-error
 * estimate, SSIM: rel_eb * vrange) and at 0.8 e0 / 1.2 e0, then the target
 * mode's secant (at most four more trials) picks the bound, capped at
 * rel_eb * vrange.  The report's params are the given ones.  Synchronises. */
qoz_status qoz_tune_verify(const float* d_field, qoz_shape shape, double rel_eb,
                           qoz_metric metric, double target, const qoz_tune_opts* opts,
                           const qoz_params* params, void* stream, qoz_tune_report* out);

/* The network proposes (qoz_tune_learned), the sampled trials verify and set
 * the bound (qoz_tune_verify). */
qoz_status qoz_tune_learned_verified(const float* d_field, qoz_shape shape, double rel_eb,
                                     qoz_metric metric, double target,
                                     const qoz_tune_opts* opts, const qoz_model* model,
                                     void* stream, qoz_tune_report* out);

/* ---------------------------------------------------------------- profiling
 * Tooling with no counterpart in the paper: per-stage device timers, a
 * launch counter and the bounds-checking build's record. */

/* Stage ids of the per-stage timers. */
#define QOZ_PROF_STAGES 32
#define QOZ_STAGE_RANGE 0      /* value range pass */
#define QOZ_STAGE_SETUP 1      /* bound table + anchor gather */
#define QOZ_STAGE_LEVEL 2      /* + l (l = 1..8): compress, level l */
#define QOZ_STAGE_HIST 11      /* code histogram */
#define QOZ_STAGE_FINAL 12     /* count read-back and unpredictable ordering */
#define QOZ_STAGE_DLEVEL 12    /* + l (l = 1..8): decompress, level l */
#define QOZ_STAGE_METRICS 21
#define QOZ_STAGE_TUNE 22      /* sampled-block trials of the tuner */
#define QOZ_STAGE_FEATURES 23  /* learned tuner: the features of the sampled blocks */
#define QOZ_STAGE_FORWARD 24   /* learned tuner: the network's forward pass and read-back */

typedef struct {
  double ms[QOZ_PROF_STAGES];      /* accumulated device time per stage (CUDA events) */
  int64_t calls[QOZ_PROF_STAGES];  /* timed occurrences per stage */
  int64_t launches;                /* kernels launched by the library */
} qoz_stage_times;

/* Turns per-stage event timing on or off (process-wide; off by default).
 * The launch counter always runs. */
qoz_status qoz_profile_enable(int32_t enable);
/* Index checks of the bounds-checking build (built with QOZ_DEBUG_BOUNDS):
 * every checked shared- or global-memory index that falls outside its array
 * is skipped instead of accessed, and the first one is recorded as
 * (1 << 63) | (source line << 40) | (index & (2^40 - 1)).  *first_bad
 * receives the record of the kernels that ran since the last reset (0: none);
 * reset != 0 clears it.  Synchronises the device.  A product build returns
 * QOZ_EUNSUPPORTED. */
qoz_status qoz_debug_bounds(uint64_t* first_bad, int32_t reset);
/* Selects the stages that record events while timing is on: bit i of mask
 * enables stage i (process-wide; all stages by default).  Each timed stage
 * adds two event records to its stream, so a caller timing a whole pipeline
 * selects only the stages it reads. */
qoz_status qoz_profile_stages(uint32_t mask);
/* Folds in all recorded stages (synchronising on their events) and copies
 * the totals; reset != 0 clears them and the launch counter afterwards. */
qoz_status qoz_profile_read(qoz_stage_times* out, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* QOZ_H */
