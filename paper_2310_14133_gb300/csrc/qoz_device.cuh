// Device building blocks of the QoZ data path (sm_103a).
//
// Every floating-point step on field values uses an explicit round-to-nearest
// intrinsic (__fadd_rn, __fmul_rn, ...) in a fixed order and the library is
// compiled with --fmad=false, so no contraction changes a result: the
// reconstruction is a pure function of the inputs.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qoz {

// Index checks of the bounds-checking build.  QOZ_IN(i, n) is true when
// 0 <= i < n; with QOZ_DEBUG_BOUNDS defined a failing check also records
// its source line and index (the first failure since the last reset, in
// this translation unit's bounds_word) and the caller skips the access.  In
// the product build it is the constant true and costs nothing.
#ifdef QOZ_DEBUG_BOUNDS
static __device__ unsigned long long bounds_word;
__device__ __forceinline__ bool bounds_ok(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&bounds_word, 0ull,
            (1ull << 63) | ((unsigned long long)(line & 0x7fffff) << 40) |
                ((unsigned long long)i & 0xffffffffffull));
  return false;
}
// Reads and optionally clears this translation unit's record (host).
static inline unsigned long long bounds_take(bool reset) {
  unsigned long long v = 0ull, z = 0ull;
  cudaMemcpyFromSymbol(&v, bounds_word, sizeof(v));
  if (reset) cudaMemcpyToSymbol(bounds_word, &z, sizeof(z));
  return v;
}
#define QOZ_IN(i, n) ::qoz::bounds_ok((long long)(i), (long long)(n), __LINE__)
#else
#define QOZ_IN(i, n) true
#endif

constexpr int kMaxLevels = 8;
constexpr int kRadius = 32768;
constexpr int kHalo = 3;  // stencil reach at the finest level of a grid

// Level-wise bound table, Eq. (ebl), computed once on the device from the
// value range so that no host round trip sits between the range pass and
// the predictor.
struct BoundTable {
  double e;                     // absolute bound
  double vrange;                // (double)max - (double)min of finite values
  float vmin, vmax;
  long long n_finite;
  float el[kMaxLevels];         // (float) e_l
  float two_e[kMaxLevels];      // (float) (2 e_l)
  float inv[kMaxLevels];        // (float) (1 / (2 e_l))
};

// Interpolation along one axis at half-stride 1 of the current grid
// (Sec. 5.1; level-adapted type, Sec. 5.2.2).  a3, a1, b1, b3 are the
// reconstructed values at -3, -1, +1, +3.  Weights are the Lagrange weights
// of the nodes that exist: cubic (-1, 9, 9, -1)/16; quadratic (-1, 6, 3)/8
// or (3, 6, -1)/8; linear (1, 1)/2; without a right neighbour linear
// extrapolation (3 a1 - a3)/2, or a1 alone.
__device__ __forceinline__ float predict(float a3, float a1, float b1, float b3, bool has_a3,
                                         bool has_b1, bool has_b3, int interp) {
  if (!has_b1) {
    if (has_a3) return __fsub_rn(__fmul_rn(a1, 1.5f), __fmul_rn(a3, 0.5f));
    return a1;
  }
  if (interp == 1) {
    if (has_a3 && has_b3)
      return __fmul_rn(__fsub_rn(__fmul_rn(9.0f, __fadd_rn(a1, b1)), __fadd_rn(a3, b3)),
                       0.0625f);
    if (has_a3)
      return __fmul_rn(__fsub_rn(__fadd_rn(__fmul_rn(6.0f, a1), __fmul_rn(3.0f, b1)), a3),
                       0.125f);
    if (has_b3)
      return __fmul_rn(__fsub_rn(__fadd_rn(__fmul_rn(3.0f, a1), __fmul_rn(6.0f, b1)), b3),
                       0.125f);
  }
  return __fmul_rn(__fadd_rn(a1, b1), 0.5f);
}

// Linear-scale quantization (Sec. 5.1): bin width 2 e_l, index rounded half
// away from zero; a point whose index leaves [-32767, 32767] or whose
// reconstruction misses the bound is unpredictable (returns false).
// Rounding half away from zero of d / (2 e_l) is trunc(d inv + sign(d) 0.5):
// binary32 rounding is symmetric in sign, so this equals sign(d) times
// floor(|d| inv + 0.5) bit for bit; d = 0 maps to bin 0 without the product
// (which is NaN for e = 0), and adding 0 turns a -0 index into +0.
__device__ __forceinline__ bool quantize(float x, float pred, float el, float two_e, float inv,
                                         uint16_t* code, float* rec) {
  const float d = __fsub_rn(x, pred);
  const float t = d == 0.0f ? 0.0f : __fmul_rn(d, inv);
  const float qf = __fadd_rn(truncf(__fadd_rn(t, copysignf(0.5f, t))), 0.0f);
  if (!(fabsf(qf) < 32768.0f)) return false;
  const float r = __fadd_rn(pred, __fmul_rn(qf, two_e));
  if (!(fabsf(__fsub_rn(x, r)) <= el)) return false;
  *code = (uint16_t)(int)__fadd_rn(qf, 32768.0f);
  *rec = r;
  return true;
}

__device__ __forceinline__ float dequantize(float pred, int code, float two_e) {
  return __fadd_rn(pred, __fmul_rn((float)(code - kRadius), two_e));
}

// Unpredictable points of one compression: appended with an atomic counter,
// ordered by index afterwards.
struct UnpredList {
  long long* idx;
  float* val;
  unsigned long long* count;
  long long cap;
};

__device__ __forceinline__ void unpred_append(const UnpredList& u, long long i, float v) {
  const unsigned long long k = atomicAdd(u.count, 1ull);
  if ((long long)k < u.cap) {
    u.idx[k] = i;
    u.val[k] = v;
  }
}

// Sorted-list lookup of an unpredictable value (decompression).  Returns
// false if the index is missing (corrupt input).
__device__ __forceinline__ bool unpred_lookup(const long long* idx, const float* val, long long n,
                                              long long key, float* out) {
  long long lo = 0, hi = n;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (idx[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < n && idx[lo] == key) {
    *out = val[lo];
    return true;
  }
  return false;
}

}  // namespace qoz
