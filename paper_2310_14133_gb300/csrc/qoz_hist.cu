// Quant-code histogram (the input of the Huffman rate estimate, Sec. 6.1)
// and ordering of the unpredictable list by index.
#include <cuda_runtime.h>

#include <climits>

#include "qoz_internal.h"

namespace qoz {
namespace {

// Codes concentrate around the zero bin 32768; a shared-memory window covers
// the bins near it, the rare far bins go straight to global memory.  One
// atomic per code: merging a warp's equal codes with a match first measured
// slower in the tuner's trials.
constexpr int kWinLo = kRadius - 2048;
constexpr int kWin = 4096;
constexpr int kHistThreads = 512;
constexpr int kHistBlocks = 152 * 2;

// Adds one code per lane; all 32 lanes of the warp call it together, lanes
// without a code pass kNoCode.
constexpr unsigned kNoCode = 0xffffffffu;
__device__ __forceinline__ void hist_add(unsigned* sh, unsigned* gh, unsigned code) {
  if (code == kNoCode) return;
  const unsigned k = code - (unsigned)kWinLo;
  if (k < (unsigned)kWin)
    atomicAdd(&sh[k], 1u);
  else
    atomicAdd(&gh[code], 1u);
}

__global__ void __launch_bounds__(kHistThreads) hist_kernel(const uint16_t* __restrict__ codes,
                                                            long long n, unsigned* hist) {
  __shared__ unsigned sh[kWin];
  for (int i = threadIdx.x; i < kWin; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long n8 = n / 8;
  const uint4* c8 = reinterpret_cast<const uint4*>(codes);
  // warp-uniform trip counts: every lane of a warp runs every iteration
  const long long wbase = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31);
  const int lane = threadIdx.x & 31;
  for (long long i0 = wbase; i0 < n8; i0 += nth) {
    const long long i = i0 + lane;
    const bool ok = i < n8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (ok) v = c8[i];
    const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      hist_add(sh, hist, ok ? (w[k] & 0xffffu) : kNoCode);
      hist_add(sh, hist, ok ? (w[k] >> 16) : kNoCode);
    }
  }
  for (long long i0 = 8 * n8 + wbase; i0 < n; i0 += nth) {
    const long long i = i0 + lane;
    hist_add(sh, hist, i < n ? (unsigned)codes[i] : kNoCode);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kWin; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[kWinLo + i], sh[i]);
}

// Anchors carry code 0 but are not coded symbols: take them out of bin 0.
__global__ void hist_remove_anchors(unsigned* hist, long long n_anchors) {
  if (threadIdx.x == 0 && blockIdx.x == 0) hist[0] -= (unsigned)n_anchors;
}

// ---- ordering of (index, value) pairs by index

constexpr int kSmemSort = 2048;

// Bitonic sort of n <= kSmemSort pairs by one block of 1024 threads, in
// shared memory (padding keys are the largest index).
__device__ __forceinline__ void sort_small_block(long long* idx, float* val, long long n) {
  __shared__ long long k[kSmemSort];
  __shared__ float v[kSmemSort];
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    k[i] = i < n ? idx[i] : LLONG_MAX;
    v[i] = i < n ? val[i] : 0.0f;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          if ((k[i] > k[j]) == up) {
            const long long tk = k[i];
            k[i] = k[j];
            k[j] = tk;
            const float tv = v[i];
            v[i] = v[j];
            v[j] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    idx[i] = k[i];
    val[i] = v[i];
  }
}

__global__ void __launch_bounds__(1024) sort_small_kernel(long long* idx, float* val,
                                                          long long n) {
  sort_small_block(idx, val, n);
}

// Batched compression, before the levels: zero each field's histogram (grid
// y = field), list counter and flags.
__global__ void __launch_bounds__(1024) batch_init_kernel(const BatchFieldDesc* __restrict__ d) {
  const BatchFieldDesc& f = d[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 65536; i += gridDim.x * blockDim.x)
    f.hist[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *f.ul.count = 0ull;
    *f.err = 0;
    *f.host_sort = 0;
  }
}

// Batched compression, after the levels: one block per field takes the
// anchors out of bin 0 and sorts a list of at most kSmemSort entries; longer
// lists are flagged for a sort driven from the host.
__global__ void __launch_bounds__(1024) batch_finish_kernel(const BatchFieldDesc* __restrict__ d) {
  const BatchFieldDesc& f = d[blockIdx.x];
  if (threadIdx.x == 0) f.hist[0] -= (unsigned)(f.na[0] * f.na[1] * f.na[2]);
  const long long cnt = (long long)*f.ul.count;  // same value in every thread
  if (cnt <= 1) return;
  if (cnt > f.ul.cap || cnt > kSmemSort) {
    if (threadIdx.x == 0) *f.host_sort = 1;
    return;
  }
  sort_small_block(f.ul.idx, f.ul.val, cnt);
}

__global__ void sort_fill_kernel(const long long* idx, const float* val, long long n,
                                 long long P, long long* k, float* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    k[i] = i < n ? idx[i] : LLONG_MAX;
    v[i] = i < n ? val[i] : 0.0f;
  }
}

__global__ void sort_step_kernel(long long* k, float* v, long long P, long long size,
                                 long long stride) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    const long long j = i ^ stride;
    if (j > i) {
      const bool up = (i & size) == 0;
      if ((k[i] > k[j]) == up) {
        const long long tk = k[i];
        k[i] = k[j];
        k[j] = tk;
        const float tv = v[i];
        v[i] = v[j];
        v[j] = tv;
      }
    }
  }
}

__global__ void sort_back_kernel(const long long* k, const float* v, long long n, long long* idx,
                                 float* val) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    idx[i] = k[i];
    val[i] = v[i];
  }
}

long long pow2_at_least(long long n) {
  long long P = 1;
  while (P < n) P <<= 1;
  return P;
}

}  // namespace

cudaError_t launch_histogram(const uint16_t* codes, long long n, unsigned* hist,
                             long long n_anchors, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * 65536, s);
  if (e != cudaSuccess) return e;
  if (reinterpret_cast<uintptr_t>(codes) & 15) return cudaErrorMisalignedAddress;
  long long want = (n / 8 + kHistThreads - 1) / kHistThreads;
  const int blocks = (int)(want < 1 ? 1 : (want < kHistBlocks ? want : kHistBlocks));
  hist_kernel<<<blocks, kHistThreads, 0, s>>>(codes, n, hist); note_launch(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_hist_remove_anchors(hist, n_anchors, s);
}

cudaError_t launch_hist_remove_anchors(unsigned* hist, long long n_anchors, cudaStream_t s) {
  hist_remove_anchors<<<1, 32, 0, s>>>(hist, n_anchors); note_launch(1);
  return cudaGetLastError();
}

size_t sort_pairs_scratch(long long n) {
  if (n <= kSmemSort) return 0;
  const long long P = pow2_at_least(n);
  return (size_t)P * (sizeof(long long) + sizeof(float));
}

cudaError_t launch_sort_pairs(long long* idx, float* val, long long n, long long* tmp_idx,
                              float* tmp_val, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  if (n <= kSmemSort) {
    sort_small_kernel<<<1, 1024, 0, s>>>(idx, val, n); note_launch(1);
    return cudaGetLastError();
  }
  const long long P = pow2_at_least(n);
  const int threads = 256;
  long long want = (P + threads - 1) / threads;
  const int blocks = (int)(want < 152 * 8 ? want : 152 * 8);
  sort_fill_kernel<<<blocks, threads, 0, s>>>(idx, val, n, P, tmp_idx, tmp_val); note_launch(1);
  for (long long size = 2; size <= P; size <<= 1) {
    for (long long stride = size >> 1; stride > 0; stride >>= 1) {
      sort_step_kernel<<<blocks, threads, 0, s>>>(tmp_idx, tmp_val, P, size, stride); note_launch(1);
    }
  }
  sort_back_kernel<<<blocks, threads, 0, s>>>(tmp_idx, tmp_val, n, idx, val); note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchFieldDesc* d, int nfields, cudaStream_t s) {
  if (nfields <= 0) return cudaSuccess;
  batch_init_kernel<<<dim3(16, nfields), 1024, 0, s>>>(d);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchFieldDesc* d, int nfields, cudaStream_t s) {
  if (nfields <= 0) return cudaSuccess;
  batch_finish_kernel<<<nfields, 1024, 0, s>>>(d);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace qoz
