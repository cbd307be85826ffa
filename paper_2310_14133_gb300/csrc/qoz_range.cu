// Value range of the finite values (Sec. 7.1.4: e = eps * vrange) and the
// level-wise bound table of Eq. (ebl), both on the device.
//
// range_kernel streams the field once with 16-byte loads (a pure HBM read,
// 4 bytes per point) and leaves one (min, max, count) triple per CTA;
// bound_table_kernel folds the triples and evaluates e and e_l in double,
// rounding each table entry to binary32 once, so the predictor's launches
// can follow without a host round trip.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>
#include <utility>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"

namespace qoz {
namespace {

constexpr int kRangeThreads = 512;
constexpr int kRangeBlocks = 152 * 4;  // 4 resident CTAs on each of the 152 SMs

template <typename C>
__device__ __forceinline__ void fold(float v, float& mn, float& mx, C& c) {
  if (isfinite(v)) {
    mn = fminf(mn, v);
    mx = fmaxf(mx, v);
    ++c;
  }
}
__device__ __forceinline__ void fold4(const float4& v, float& mn, float& mx, unsigned& c) {
  fold(v.x, mn, mx, c);
  fold(v.y, mn, mx, c);
  fold(v.z, mn, mx, c);
  fold(v.w, mn, mx, c);
}

__global__ void __launch_bounds__(kRangeThreads) range_kernel(const float* __restrict__ x,
                                                              long long n, float* pmin,
                                                              float* pmax,
                                                              unsigned long long* pcnt) {
  float mn = FLT_MAX, mx = -FLT_MAX;
  // per-thread count: at most 4 ceil(n / 4 / threads) + 1 values, far below
  // 2^32 for any field that fits in device memory
  unsigned ct = 0;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  // 16-byte aligned body (the caller passes the aligned start), four
  // independent loads in flight per thread, then a scalar tail
  const long long n4 = n / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  long long i = tid;
  for (; i + 3 * nth < n4; i += 4 * nth) {
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __ldcs(x4 + i + k * nth);
#pragma unroll
    for (int k = 0; k < 4; ++k) fold4(v[k], mn, mx, ct);
  }
  for (; i < n4; i += nth) fold4(__ldcs(x4 + i), mn, mx, ct);
  for (long long j = 4 * n4 + tid; j < n; j += nth) fold(x[j], mn, mx, ct);
  unsigned long long c = ct;

  for (int off = 16; off > 0; off >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  __shared__ float smn[32], smx[32];
  __shared__ unsigned long long sc[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    smn[w] = mn;
    smx[w] = mx;
    sc[w] = c;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    mn = l < nw ? smn[l] : FLT_MAX;
    mx = l < nw ? smx[l] : -FLT_MAX;
    c = l < nw ? sc[l] : 0;
    for (int off = 16; off > 0; off >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    if (l == 0) {
      pmin[blockIdx.x] = mn;
      pmax[blockIdx.x] = mx;
      pcnt[blockIdx.x] = c;
    }
  }
}

// Scalar head for a field pointer that is not 16-byte aligned: folded into
// the first partial afterwards by the table kernel.
__global__ void range_head_kernel(const float* __restrict__ x, int nhead, float* pmin,
                                  float* pmax, unsigned long long* pcnt) {
  if (threadIdx.x != 0) return;
  float mn = FLT_MAX, mx = -FLT_MAX;
  unsigned long long c = 0;
  for (int i = 0; i < nhead; ++i) fold(x[i], mn, mx, c);
  *pmin = mn;
  *pmax = mx;
  *pcnt = c;
}

// The bound table from the folded range: e = eb * vrange (relative) or eb,
// then Eq. (ebl): e_l = e / min(alpha^(l-1), beta), alpha^(l-1) by repeated
// multiplication in double; each entry rounded to binary32 once.
__device__ void fill_bound_table(float mn, float mx, unsigned long long c, int use_range,
                                 double eb, double alpha, double beta, int L, BoundTable* bt) {
  if (c == 0) {
    mn = 0.0f;
    mx = 0.0f;
  }
  BoundTable t;
  t.vmin = mn;
  t.vmax = mx;
  t.n_finite = (long long)c;
  t.vrange = (double)mx - (double)mn;
  t.e = use_range ? eb * t.vrange : eb;
  double a = 1.0;
  for (int l = 0; l < kMaxLevels; ++l) {
    if (l < L) {
      const double den = a < beta ? a : beta;
      const double el = t.e / den;
      t.el[l] = (float)el;
      t.two_e[l] = (float)(2.0 * el);
      t.inv[l] = (float)(1.0 / (2.0 * el));
      a = a * alpha;
    } else {
      t.el[l] = t.two_e[l] = t.inv[l] = 0.0f;
    }
  }
  *bt = t;
}

// One block folds the per-CTA partials (a tree over the threads), then one
// thread evaluates Eq. (ebl).
constexpr int kTableThreads = 1024;

__global__ void __launch_bounds__(kTableThreads)
    bound_table_kernel(const float* pmin, const float* pmax, const unsigned long long* pcnt,
                       int nparts, int use_range, double eb, double alpha, double beta, int L,
                       BoundTable* bt) {
  float mn = FLT_MAX, mx = -FLT_MAX;
  unsigned long long c = 0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    if (pcnt[i] == 0) continue;
    mn = fminf(mn, pmin[i]);
    mx = fmaxf(mx, pmax[i]);
    c += pcnt[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  __shared__ float smn[32], smx[32];
  __shared__ unsigned long long sc[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    smn[w] = mn;
    smx[w] = mx;
    sc[w] = c;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  mn = FLT_MAX;
  mx = -FLT_MAX;
  c = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    mn = fminf(mn, smn[i]);
    mx = fmaxf(mx, smx[i]);
    c += sc[i];
  }
  fill_bound_table(mn, mx, c, use_range, eb, alpha, beta, L, bt);
}

// Min / max / count across a block (warp shuffles, then the first warp);
// the result is valid in thread 0.
__device__ __forceinline__ void block_fold(float& mn, float& mx, unsigned long long& c) {
  for (int off = 16; off > 0; off >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  __shared__ float smn[32], smx[32];
  __shared__ unsigned long long sc[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    smn[w] = mn;
    smx[w] = mx;
    sc[w] = c;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    mn = l < nw ? smn[l] : FLT_MAX;
    mx = l < nw ? smx[l] : -FLT_MAX;
    c = l < nw ? sc[l] : 0;
    for (int off = 16; off > 0; off >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      c += __shfl_xor_sync(0xffffffffu, c, off);
    }
  }
}

// One CTA per chunk of one field: 16-byte loads over the chunk's aligned
// body, scalar head and tail.
__global__ void __launch_bounds__(kRangeThreads) range_batch_kernel(
    const BatchFieldDesc* __restrict__ d, const RangeChunk* __restrict__ chunks, float* pmin,
    float* pmax, unsigned long long* pcnt) {
  const RangeChunk ch = chunks[blockIdx.x];
  const float* x = d[ch.field].x;
  float mn = FLT_MAX, mx = -FLT_MAX;
  unsigned long long c = 0;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(x + ch.begin);
  long long head = (long long)(((16 - (a0 & 15)) & 15) / 4);
  if (head > ch.end - ch.begin) head = ch.end - ch.begin;
  const long long b4 = ch.begin + head;
  const long long n4 = (ch.end - b4) / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x + b4);
  for (long long i = threadIdx.x; i < n4; i += blockDim.x) {
    const float4 v = __ldcs(x4 + i);
    fold(v.x, mn, mx, c);
    fold(v.y, mn, mx, c);
    fold(v.z, mn, mx, c);
    fold(v.w, mn, mx, c);
  }
  if ((long long)threadIdx.x < head) fold(x[ch.begin + threadIdx.x], mn, mx, c);
  for (long long i = b4 + 4 * n4 + threadIdx.x; i < ch.end; i += blockDim.x)
    fold(x[i], mn, mx, c);
  block_fold(mn, mx, c);
  if (threadIdx.x == 0) {
    pmin[blockIdx.x] = mn;
    pmax[blockIdx.x] = mx;
    pcnt[blockIdx.x] = c;
  }
}

// One CTA per field: fold the field's chunk partials, evaluate Eq. (ebl).
__global__ void __launch_bounds__(256) bound_batch_kernel(const BatchFieldDesc* __restrict__ d,
                                                          const float* pmin, const float* pmax,
                                                          const unsigned long long* pcnt) {
  const BatchFieldDesc& f = d[blockIdx.x];
  float mn = FLT_MAX, mx = -FLT_MAX;
  unsigned long long c = 0;
  if (f.use_range)
    for (int i = threadIdx.x; i < f.nchunks; i += blockDim.x) {
      const int k = f.chunk_begin + i;
      if (pcnt[k] == 0) continue;
      mn = fminf(mn, pmin[k]);
      mx = fmaxf(mx, pmax[k]);
      c += pcnt[k];
    }
  block_fold(mn, mx, c);
  if (threadIdx.x == 0)
    fill_bound_table(mn, mx, c, f.use_range, f.eb, f.alpha, f.beta, f.L, f.bt);
}

}  // namespace

int range_partial_blocks() { return kRangeBlocks + 1; }

cudaError_t launch_range(const float* x, long long n, float* pmin, float* pmax,
                         unsigned long long* pcnt, cudaStream_t s) {
  // partial 0 holds the unaligned head (possibly empty), 1.. the main pass
  const uintptr_t addr = reinterpret_cast<uintptr_t>(x);
  int head = (int)(((16 - (addr & 15)) & 15) / 4);
  if ((addr & 3) != 0) return cudaErrorMisalignedAddress;
  if (head > n) head = (int)n;
  range_head_kernel<<<1, 32, 0, s>>>(x, head, pmin, pmax, pcnt); note_launch(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long rest = n - head;
  long long want = (rest / 4 + kRangeThreads - 1) / kRangeThreads;
  int blocks = (int)(want < kRangeBlocks ? (want < 1 ? 1 : want) : kRangeBlocks);
  range_kernel<<<blocks, kRangeThreads, 0, s>>>(x + head, rest, pmin + 1, pmax + 1, pcnt + 1); note_launch(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // unused partial slots must not contribute
  if (blocks < kRangeBlocks)
    e = cudaMemsetAsync(pcnt + 1 + blocks, 0,
                        sizeof(unsigned long long) * (kRangeBlocks - blocks), s);
  return e;
}

cudaError_t launch_bound_table(const float* pmin, const float* pmax,
                               const unsigned long long* pcnt, int nparts, int use_range,
                               double eb, double alpha, double beta, int L, BoundTable* bt,
                               cudaStream_t s) {
  bound_table_kernel<<<1, kTableThreads, 0, s>>>(pmin, pmax, pcnt, nparts, use_range, eb, alpha,
                                                  beta, L, bt);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_range_batch(const BatchFieldDesc* d, const RangeChunk* chunks, int nchunks,
                               float* pmin, float* pmax, unsigned long long* pcnt,
                               cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  range_batch_kernel<<<nchunks, kRangeThreads, 0, s>>>(d, chunks, pmin, pmax, pcnt);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_bound_batch(const BatchFieldDesc* d, int nfields, const float* pmin,
                               const float* pmax, const unsigned long long* pcnt, cudaStream_t s) {
  if (nfields <= 0) return cudaSuccess;
  bound_batch_kernel<<<nfields, 256, 0, s>>>(d, pmin, pmax, pcnt);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace qoz

// ---------------------------------------------------------------------------
// Value range with library-owned scratch in a static device array, for
// callers that must not allocate device memory themselves (see
// qoz_value_range_noalloc in qoz.h).

namespace qoz {
namespace {

constexpr int kNoAllocParts = kRangeBlocks + 1;

// Partial (min, max, count) of every CTA of one call; shared by all calls on
// a device, so calls whose work overlaps on the GPU race.
struct RangeScratch {
  float pmin[kNoAllocParts];
  float pmax[kNoAllocParts];
  unsigned long long pcnt[kNoAllocParts];
};
__device__ __align__(256) RangeScratch g_range_scratch;

// Folds the partials into the caller's outputs: {min, max} and the count of
// finite values (0, 0 and 0 when there is none).
__global__ void __launch_bounds__(kTableThreads)
    range_fold_kernel(const RangeScratch* sc, int nparts, float* out_minmax,
                      long long* out_count) {
  float mn = FLT_MAX, mx = -FLT_MAX;
  unsigned long long c = 0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    if (sc->pcnt[i] == 0) continue;
    mn = fminf(mn, sc->pmin[i]);
    mx = fmaxf(mx, sc->pmax[i]);
    c += sc->pcnt[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  __shared__ float smn[32], smx[32];
  __shared__ unsigned long long sc_[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    smn[w] = mn;
    smx[w] = mx;
    sc_[w] = c;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  mn = FLT_MAX;
  mx = -FLT_MAX;
  c = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    mn = fminf(mn, smn[i]);
    mx = fmaxf(mx, smx[i]);
    c += sc_[i];
  }
  if (c == 0) {
    mn = 0.0f;
    mx = 0.0f;
  }
  out_minmax[0] = mn;
  out_minmax[1] = mx;
  if (out_count) *out_count = (long long)c;
}

std::mutex g_scratch_mu;
// The scratch's device address per device, with the id of the context it was
// taken in: a device reset destroys the context (and the module with the
// array), and the context created next has another id, so the address is
// looked up again.
struct ScratchSlot {
  RangeScratch* ptr;
  unsigned long long ctx_id;
};
ScratchSlot g_scratch_slot[64] = {};

// Id of the calling thread's current context (0 when the driver entry points
// are unavailable), through the runtime's driver entry-point lookup so that
// the library does not link the driver library.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static const std::pair<GetCurrent, GetId> fns = [] {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    const bool ok =
        cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess;
    if (!ok) {
      cudaGetLastError();
      return std::pair<GetCurrent, GetId>(nullptr, nullptr);
    }
    return std::pair<GetCurrent, GetId>(reinterpret_cast<GetCurrent>(a),
                                        reinterpret_cast<GetId>(b));
  }();
  if (!fns.first || !fns.second) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (fns.first(&ctx) != CUDA_SUCCESS || !ctx || fns.second(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace
}  // namespace qoz

extern "C" qoz_status qoz_value_range_noalloc(const float* d_x, int64_t n, float* d_minmax,
                                              int64_t* d_count, void* stream) {
  using namespace qoz;
  if (!d_x || !d_minmax || n < 0) return fail(QOZ_EINVAL, "invalid argument");
  if (n > QOZ_NOALLOC_MAX_VALUES)
    return fail(QOZ_EUNSUPPORTED, "qoz_value_range_noalloc: %lld values exceed the maximum of "
                "%lld", (long long)n, (long long)QOZ_NOALLOC_MAX_VALUES);
  if (reinterpret_cast<uintptr_t>(d_x) & 3) return fail(QOZ_EINVAL, "d_x must be 4-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(QOZ_EUNSUPPORTED, "device ordinal %d", dev);
  RangeScratch* sc;
  {
    // once per device context, with that device current: the device address
    // of the static scratch (its host-side name is not a device address);
    // the lookup itself sets the context up when none is current yet, so
    // the context's id is taken after it
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchSlot& slot = g_scratch_slot[dev];
    if (!slot.ptr || slot.ctx_id == 0 || slot.ctx_id != current_context_id()) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_range_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
      slot.ptr = static_cast<RangeScratch*>(p);
      slot.ctx_id = current_context_id();
    }
    sc = slot.ptr;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every partial slot the fold reads is written by this call (the range
  // pass zeroes the counts of the CTAs it does not launch)
  e = launch_check(launch_range(d_x, n, sc->pmin, sc->pmax, sc->pcnt, s));
  if (e == cudaErrorMisalignedAddress) return fail(QOZ_EINVAL, "misaligned input");
  if (e == cudaSuccess) {
    range_fold_kernel<<<1, kTableThreads, 0, s>>>(sc, kNoAllocParts, d_minmax,
                                                  reinterpret_cast<long long*>(d_count));
    note_launch(1);
    e = launch_check(cudaGetLastError());
  }
  if (e != cudaSuccess) return cuda_fail(e, "value range (no allocation)");
  return QOZ_OK;
}
