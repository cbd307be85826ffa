// Host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qoz_device.cuh"

namespace qoz {

// Adds n to the library's kernel-launch counter (qoz_profile.cu).
void note_launch(int n);

// Geometry of one level launch.  The level-l targets of the full field are
// exactly the finest-level targets of the grid G = the full field subsampled
// by f = 2^(l-1) (its points whose coordinates are all multiples of f):
// along each axis a target has an odd G coordinate, its neighbours at
// +-h, +-3h are at +-1, +-3 in G, and the points with all G coordinates even
// (the coarse grid) were reconstructed by the levels above.  A launch
// therefore always works at half-stride 1 on G, whatever the level.
//
// All per-axis arrays are in ORDER space: index 0 is the axis interpolated
// first in this level (u), 1 the second (v), 2 the third (w).
struct LevelGeom {
  long long g[3];    // extent of G
  long long xs[3];   // element stride of the full-resolution arrays (x, codes)
  long long cs[3];   // stride of the compact coarse reconstruction (G subsampled by 2)
  long long os[3];   // stride of the compact reconstruction of G (output)
  int T[3];          // tile extent (even; T[0] may be 1 when g[0] == 1)
  int phys_of[3];    // physical axis (0 slowest .. 2 contiguous) of order axis k
  int ord_of[3];     // order axis of physical axis p
  long long nt[3];   // number of tiles per PHYSICAL axis
  int level;         // 1-based level, index into the bound table
  int interp;        // 0 linear, 1 cubic
};

// Launch wrappers (qoz_level.cu)
cudaError_t launch_level(bool decompress, const LevelGeom& G, const float* x, uint16_t* codes,
                         const float* rc, float* rout, const BoundTable* bt, UnpredList ul,
                         const long long* uidx, const float* uval, long long nu, int* err,
                         cudaStream_t s);
cudaError_t launch_anchor_gather(const float* x, uint16_t* codes, float* anchors,
                                 const long long na[3], const long long fst[3], long long stride,
                                 cudaStream_t s);
size_t level_smem_bytes(const LevelGeom& G);

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
