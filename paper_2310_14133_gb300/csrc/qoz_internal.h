// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

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
};

// Launch wrappers (qoz_level.cu)
cudaError_t launch_level(const LevelLaunch& L, cudaStream_t s);
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

// Histogram and unpredictable ordering (qoz_hist.cu)
cudaError_t launch_histogram(const uint16_t* codes, long long n, unsigned* hist,
                             long long n_anchors, cudaStream_t s);
cudaError_t launch_hist_remove_anchors(unsigned* hist, long long n_anchors, cudaStream_t s);
cudaError_t launch_sort_pairs(long long* idx, float* val, long long n, long long* tmp_idx,
                              float* tmp_val, cudaStream_t s);
size_t sort_pairs_scratch(long long n);

// Metrics (qoz_metrics.cu)
cudaError_t launch_err_metrics(const float* a, const float* b, long long n, double* part_sse,
                               double* part_max, int nparts, cudaStream_t s);
int err_metric_blocks();
cudaError_t launch_ssim(const float* a, const float* b, const long long dims[3], bool is3d,
                        int win, int step, double c1, double c2, double* part_sum, int nparts,
                        cudaStream_t s);
int ssim_blocks();

}  // namespace qoz
