// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/qoz.h"
#include "qoz_device.cuh"

namespace qoz {

// Adds n to the library's kernel-launch counter (qoz_profile.cu).
void note_launch(int n);

// One level launch.  The level-l points of the field are the points of the
// grid G = field subsampled by 2^(l-1) (all coordinates multiples of
// 2^(l-1)) that have an odd coordinate in G; their neighbours at +-h, +-3h
// are at +-1, +-3 in G, and the points of G with all coordinates even (the
// coarse grid) were reconstructed by the levels above.  A launch therefore
// always works at half-stride 1 on G, whatever the level.  Per-axis arrays
// are physical (0 = slowest z, 2 = contiguous x).
struct LevelLaunch {
  bool decompress;
  bool is2d;          // field embedded as (1, ny, nx)
  int order3;         // 3D order index (2D: 0 = (y, x), 1 = (x, y))
  int level;          // 1-based, index into the bound table
  int interp;         // 0 linear, 1 cubic
  long long g[3];     // extent of G
  long long xs[3];    // strides of G inside the full-resolution arrays (field, codes)
  long long cs[3];    // strides of the compact coarse arrays (G subsampled by 2)
  long long os[3];    // strides of the compact arrays of G (outputs)
  const float* x;     // compress: the field
  const uint16_t* cin;  // compress: compact coarse codes (NULL: all 0); decompress: codes
  const float* rc;    // compact coarse reconstruction
  float* rout;        // compact reconstruction of G (optional)
  uint16_t* cout;     // compress: compact codes of G
  const BoundTable* bt;
  UnpredList ul;      // compress: unpredictable points of this level
  const long long* uidx;  // decompress: sorted unpredictable list
  const float* uval;
  long long nu;
  int* err;           // decompress: set to 1 if a code-0 point has no list entry
  unsigned* hist;     // compress, level 1: 65536-bin code histogram (optional)
  // bulk-copy tiles: bytes the tile's mbarrier expects beyond its copies (0;
  // a positive value is the host fault injection that makes the wait run
  // out) and the wait's poll limit (0: the default)
  int extra_tx;
  int wait_polls;
};

// Launch wrappers (qoz_level.cu)
cudaError_t launch_level(const LevelLaunch& L, cudaStream_t s);
// Sets the opt-in dynamic shared-memory size of a kernel once per device.
cudaError_t ensure_smem_attr(const void* fn, unsigned long long* done_mask, size_t bytes);

// Batched level launches (qoz_level_batch.cu).  One launch runs the same
// level of many fields that share a kernel instance: the items are those
// fields' LevelLaunch descriptors in device memory, and a per-CTA map names
// the item each CTA works on; the CTA's tile is its index minus the item's
// first CTA.  Only compression is batched.
struct LevelItem {
  LevelLaunch L;
  int nt1, nt2;         // tiles along y and x
  int vec;              // 16-byte row copies allowed (set per call: depends on x)
  unsigned tile_begin;  // first CTA of this item in its launch
};
// Kernel instance of a batched launch: 2-D or 3-D, the level's order, whether
// the launch accumulates the histogram (level 1), the level's interpolator
// and the tile variant (0, 1: row copies; 2: bulk tensor copies, one tile per
// CTA; 3: the persistent bulk-copy kernel of 3-D level 1, its CTAs walking
// the tiles of all the launch's items; 2 and 3 are level 1 only and need the
// tensor maps of each item; a 2-D key takes 2 for 3).
struct LevelKey {
  bool is2d;
  int order3;
  bool hist;
  int interp;
  int variant;
};
constexpr int kLevelVariants = 4;
constexpr int kLevelVariantBulk = 2;
constexpr int kLevelVariantPersist = 3;
// Tensor maps of one item of a bulk-copy launch (device memory).
struct alignas(64) LevelTmaMaps {
  CUtensorMap x, rc, cc, out;
  int use_out;
};
// A rank-3 tiled tensor map (dims and box innermost first, strides in bytes
// of dims 1 and 2, zero fill outside the array); false when the driver's
// encoder is unavailable or rejects the map.
bool encode_tensor_map_3d(CUtensorMap* m, CUtensorMapDataType type, const void* base,
                          const unsigned long long dims[3], const unsigned long long strides[2],
                          const unsigned box[3]);
// Encodes an item's tensor maps for the key's bulk-copy tiles; false when
// the item's arrays do not meet the bulk-copy alignment rules.
bool level_tma_maps(const LevelKey& k, const LevelLaunch& L, LevelTmaMaps* m);
// Tile extent (z, y, x) of a key's kernel instance.
void level_tile_shape(const LevelKey& k, int t[3]);
// Tiles of one item under the key's tile shape (nt[0] * nt[1] * nt[2]).
long long level_item_tiles(const LevelKey& k, const LevelLaunch& L, long long nt[3]);
// Prepares the kernel instance (shared-memory attribute); call before any
// stream capture.
cudaError_t level_batch_prepare(const LevelKey& k);
cudaError_t launch_level_batch(const LevelKey& k, const LevelItem* d_items,
                               const uint16_t* d_map, const LevelTmaMaps* d_maps,
                               unsigned nblocks, cudaStream_t s);
cudaError_t launch_anchor_gather(const float* x, float* anchors, const long long na[3],
                                 const long long fst[3], long long stride, cudaStream_t s);

// Value range and bound table (qoz_range.cu)
int range_partial_blocks();
cudaError_t launch_range(const float* x, long long n, float* pmin, float* pmax,
                         unsigned long long* pcnt, cudaStream_t s);
cudaError_t launch_bound_table(const float* pmin, const float* pmax,
                               const unsigned long long* pcnt, int nparts, int use_range,
                               double eb, double alpha, double beta, int L, BoundTable* bt,
                               cudaStream_t s);

// Per-field descriptor of a batched compression (device memory, rewritten
// before each run because the field pointers and outputs change per call).
struct BatchFieldDesc {
  const float* x;
  long long n;             // points
  int chunk_begin, nchunks;  // this field's value-range chunks
  int use_range, L;
  double eb, alpha, beta;  // bound (relative when use_range), Eq. (ebl) parameters
  BoundTable* bt;
  float* anchors;
  long long na[3];
  long long fst0, fst1, stride;
  unsigned* hist;
  UnpredList ul;
  int* err;
  int* host_sort;          // out: 1 when the list was left for a host-driven sort
};
// A contiguous piece [begin, end) of one field for the value range.
struct RangeChunk {
  int field;
  int pad;
  long long begin, end;
};
constexpr long long kRangeChunk = 1LL << 20;

// Batched value range (qoz_range.cu): one CTA per chunk, then one CTA per
// field folds its chunks into the field's bound table (Eq. ebl).
cudaError_t launch_range_batch(const BatchFieldDesc* d, const RangeChunk* chunks, int nchunks,
                               float* pmin, float* pmax, unsigned long long* pcnt,
                               cudaStream_t s);
cudaError_t launch_bound_batch(const BatchFieldDesc* d, int nfields, const float* pmin,
                               const float* pmax, const unsigned long long* pcnt, cudaStream_t s);
// Batched setup and finish (qoz_hist.cu): zero each field's histogram,
// counter and flags; afterwards take the anchors out of bin 0 and sort each
// short unpredictable list by index on the device.
cudaError_t launch_batch_init(const BatchFieldDesc* d, int nfields, cudaStream_t s);
cudaError_t launch_batch_finish(const BatchFieldDesc* d, int nfields, cudaStream_t s);
// Batched anchor gather (qoz_level.cu).
cudaError_t launch_anchor_batch(const BatchFieldDesc* d, int nfields, cudaStream_t s);

// Histogram and unpredictable ordering (qoz_hist.cu)
cudaError_t launch_histogram(const uint16_t* codes, long long n, unsigned* hist,
                             long long n_anchors, cudaStream_t s);
cudaError_t launch_hist_remove_anchors(unsigned* hist, long long n_anchors, cudaStream_t s);
cudaError_t launch_sort_pairs(long long* idx, float* val, long long n, long long* tmp_idx,
                              float* tmp_val, cudaStream_t s);
size_t sort_pairs_scratch(long long n);

// Metrics (qoz_metrics.cu)
// One pass: err_metric_blocks() partials each of the squared-error sum and
// the max |a - b|, and ac_parts() doubles of lag-1 autocorrelation sums (the
// layout autocorr_from_parts reads).
cudaError_t launch_err_metrics(const float* a, const float* b, long long n, double* part_sse,
                               double* part_max, double* part_ac, cudaStream_t s);
int err_metric_blocks();
// SSIM partial sums of (1 - SSIM_w), one per part; ssim_parts() gives the count.
cudaError_t launch_ssim(const float* a, const float* b, const long long dims[3], bool is3d,
                        int win, int step, double c1, double c2, double* part_diss,
                        cudaStream_t s);
int ssim_parts(const long long dims[3], bool is3d, int win, int step);
// Eq. (ac) at lag k over the flattened arrays: ac_parts() doubles of per-CTA
// sums, combined by autocorr_from_parts on the host.
int ac_parts();
cudaError_t launch_autocorr(const float* a, const float* b, long long n, long long k,
                            double* part, cudaStream_t s);
double autocorr_from_parts(const double* h, long long n, long long k);

// Entropy stage (qoz_entropy.cu): canonical Huffman coding of the codes.
constexpr int kEntropyChunk = 4096;     // largest chunk: symbols per independently coded chunk
constexpr int kEntropyChunkMin = 256;   // smallest chunk a stream is written with
// Chunk size for N codes: the largest power of two from 256 to 4096 that
// still gives at least 8192 chunks (one decoding thread per chunk), else
// 256; a reader accepts any multiple of 8 up to 4096.
inline int entropy_chunk(long long N) {
  int c = kEntropyChunk;
  while (c > kEntropyChunkMin && (N + c - 1) / c < 8192) c >>= 1;
  return c;
}
// Runs of a chunk: a chunk of 1024 codes or more is cut into runs of
// kEntropyRun codes, and the section records the coded length of each run
// but the last (n_chunks * (runs - 1) uint16 after the chunk offsets), so
// that the decoder starts a thread at every run.
constexpr int kEntropyRun = 512;
__host__ __device__ inline int entropy_runs(int chunk) {
  return chunk >= 2 * kEntropyRun ? chunk / kEntropyRun : 1;
}
inline size_t entropy_sub_bytes(long long n_chunks, int chunk) {
  return ((size_t)2 * (size_t)n_chunks * (size_t)(entropy_runs(chunk) - 1) + 7) & ~(size_t)7;
}
constexpr int kMaxCodeLen = 58;      // longest code the coder handles

// Fixed part of the serialized code section (288 bytes): counts, then the
// number of codes of each length 0..63.
struct HuffFixed {
  uint32_t n_sym, max_len, chunk, flags;
  uint64_t n_chunks, n_words;
  uint32_t bl_count[64];
};
static_assert(sizeof(HuffFixed) == 288, "code section header layout");

inline size_t pad8_bytes(size_t v) { return (v + 7) & ~(size_t)7; }

// A blob's coded stream on the device: d_section holds the fixed part, room
// for 65536 symbols (sym_bytes) and the n_chunks + 1 word offsets; d_words
// the n_words stream words.
struct HuffEncoded {
  HuffFixed fixed;
  int chunk;  // symbols per chunk
  long long n_chunks, n_words;
  size_t sym_bytes;
  size_t sub_bytes;  // the run table after the chunk offsets (padded to 8)
  void* d_work;
  void* d_section;
  uint32_t* d_words;
};

// Builds the code table from the blob's histogram (anchors added back to
// symbol 0), counts, scans and (unless sizes_only) writes the chunks;
// synchronises once on s to learn the stream's length.  huff_free releases
// (stream-ordered).
qoz_status huff_encode(const qoz_blob* b, cudaStream_t s, HuffEncoded* h, bool sizes_only);
void huff_free(HuffEncoded* h, cudaStream_t s);
// Decodes nchunks chunks into d_codes (N symbols) from a device section laid
// out as huff_encode's; bit 2 of *d_err reports a stream that does not
// decode.
cudaError_t huff_decode(const void* d_section, const uint32_t* d_words, long long nchunks,
                        int chunk, unsigned n_sym, long long N, uint16_t* d_codes, int* d_err,
                        cudaStream_t s);

#ifdef QOZ_DEBUG_BOUNDS
// Records of failed index checks, one per translation unit that checks.
unsigned long long bounds_take_level(bool reset);
unsigned long long bounds_take_level_batch(bool reset);
unsigned long long bounds_take_tune(bool reset);
unsigned long long bounds_take_entropy(bool reset);
#endif

}  // namespace qoz
