// Host-side helpers shared by the library's C-ABI translation units.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qoz.h"

// The compressed field behind the opaque qoz_blob handle.
struct qoz_blob {
  qoz_shape shape;
  long long n[3];        // dims embedded in 3D, 2D as (1, ny, nx)
  long long N;
  int L;
  qoz_params params;     // as given (2D orders are 2D indices)
  double abs_eb, rel_eb;
  float vmin, vmax;
  uint16_t* d_codes;
  long long* d_uidx;
  float* d_uval;
  long long nu;
  float* d_anchors;
  long long na;
  unsigned* d_hist;
  int* d_err;            // decode status written by decompression kernels
  cudaStream_t stream;
  int device;
};

namespace qoz {

// A validated request: dims embedded in 3D (2D as (1, ny, nx)), parameters
// with defaults filled in, and each level's dimension order as 3D axes.
struct Resolved {
  int ndims;
  long long n[3];
  long long N;
  qoz_params p;
  int L;
  int axes[QOZ_MAX_LEVELS][3];
};

qoz_status fail(qoz_status st, const char* fmt, ...);
qoz_status cuda_fail(cudaError_t e, const char* what);
qoz_status resolve(const qoz_shape& shape, const qoz_params* p, Resolved* r);
bool fault_injected(const char* step);
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);
cudaError_t launch_check(cudaError_t e);
void configure_pool_once();

struct LevelLaunch;

// Compact per-grid scratch of the hierarchy: for k = 1..L-1 the
// reconstruction (float) and, when compressing, the codes (uint16) of the
// field subsampled by 2^k.
struct Coarse {
  size_t roff[QOZ_MAX_LEVELS + 1];
  size_t coff[QOZ_MAX_LEVELS + 1];
  size_t bytes;
};

// Geometry helpers of the level hierarchy (qoz_api.cu).
void grid_dims(const Resolved& r, int k, long long g[3]);
Coarse coarse_layout(const Resolved& r, bool with_codes);
long long anchor_dims(const Resolved& r, long long na[3]);
void level_geometry(const Resolved& r, int l, LevelLaunch* L);
// Single-field compression behind qoz_compress / qoz_compress_abs.
qoz_status compress_impl(const float* d_field, const qoz_shape& shape, bool rel, double eb,
                         const qoz_params* p, float* d_recon, cudaStream_t s, qoz_blob** out);

// Sampled blocks of the tuners (Sec. 6.1), in the embedded 3-D layout.
struct Sampling {
  std::vector<int> origins;  // 3 per block (embedded)
  int nb = 0;
  int bd[3] = {1, 1, 1};
  long long npts = 0;
  int Ls = 0;
  long long anchors = 0;     // anchors over all blocks
};
Sampling sample_blocks(const Resolved& r, int b, double rate, int s);
// Tuner options with the defaults filled in and checked (qoz_tune.cu).
qoz_status resolve_tune_opts(const qoz_shape& shape, const Resolved& r,
                             const qoz_tune_opts* opts_in, qoz_tune_opts* out);

// Adds n to the library's kernel-launch counter.
void note_launch(int n);

// Records the device time of a stage between construction and destruction
// (only while profiling is enabled).
class ProfScope {
 public:
  ProfScope(int stage, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int stage_;
  cudaStream_t s_;
  cudaEvent_t a_;
};

// Total bits of an optimal prefix code for the counts (Huffman): sort the
// non-zero counts, then merge with two FIFO queues (leaves, and merged nodes,
// which come out in non-decreasing order); every merge adds its weight.  A
// single used symbol costs one bit per occurrence.
inline uint64_t huffman_bits_u32(const unsigned* h, int K) {
  std::vector<uint64_t> leaf;
  for (int i = 0; i < K; ++i)
    if (h[i]) leaf.push_back(h[i]);
  if (leaf.empty()) return 0;
  if (leaf.size() == 1) return leaf[0];
  std::sort(leaf.begin(), leaf.end());
  std::vector<uint64_t> node;
  node.reserve(leaf.size());
  size_t li = 0, ni = 0;
  uint64_t total = 0;
  auto take = [&]() -> uint64_t {
    if (ni < node.size() && (li >= leaf.size() || node[ni] < leaf[li])) return node[ni++];
    return leaf[li++];
  };
  for (size_t m = 1; m < leaf.size(); ++m) {
    const uint64_t a = take();
    const uint64_t b = take();
    total += a + b;
    node.push_back(a + b);
  }
  return total;
}

}  // namespace qoz
