// Sampled online tuner (Sec. 6): uniform block sampling (Sec. 6.1),
// Algorithm 1 (level-adapted interpolator selection, Sec. 6.2) and the
// alpha / beta search with the Table I comparisons (Sec. 6.3).
//
// Every trial compression of the sampled blocks runs on the GPU: one CTA per
// (candidate, block) copies its block into shared memory and runs the whole
// multi-level predictor on it as an independent small field (anchors at the
// block corners, log2 min(b, s) levels), accumulating the mean absolute
// prediction error of the scored level, the code histogram (pooled over the
// candidate's blocks), the unpredictable count, the squared and maximum
// error and the SSIM window sums.  The host mirrors the method's sequential
// decisions; trials whose outcome does not depend on an earlier decision are
// batched into one launch (all candidates of an Algorithm 1 level; all
// (alpha, beta) at e and at the 0.8 e / 1.2 e that Table I may ask for).
// Every (1, beta) gives e_l = e on all levels (beta >= 1), so of those only
// the first setting runs and the others take its results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"
#include "qoz_tma.cuh"

namespace qoz {
namespace {

// Threads per trial CTA: the full-resolution block (stop level 1, up to
// 33^3 values in shared memory, one CTA per SM) gets 512; the subsampled
// blocks of the coarser Algorithm 1 levels (17^3 values and fewer) get 128,
// so that several CTAs share an SM and the grid fits in one wave.
constexpr int kTrialThreads = 512;
constexpr int kTrialThreadsCoarse = 128;
constexpr int kTHistLo = kRadius - 2048;
constexpr int kTHistWin = 4096;
// per (candidate, block): l1, l1_cnt, unpred, sse, maxerr, ssim_sum, ssim_n,
// copy-timeout flag, then the lag-1 error sums of Eq. (ac) in block order
// (sum e, sum e^2, sum e_i e_{i+1}) and the block's first and last error
constexpr int kOutStride = 16;

struct TrialCand {
  unsigned char interp[kMaxLevels];
  unsigned char axes[kMaxLevels][3];  // physical axes of each level's order
  float el[kMaxLevels], two_e[kMaxLevels], inv[kMaxLevels];
};

struct TrialArgs {
  const float* x;
  long long st0, st1;      // element strides of the embedded field (z, y)
  const int* origins;      // 3 per block (embedded z, y, x)
  int nblocks;
  int bd[3];               // block extent (embedded)
  int Ls;                  // levels of the block predictor
  int stop_level;          // lowest level run
  int score_level;         // level whose |x - pred| is summed (0: none)
  const TrialCand* cands;
  unsigned* hist;          // [ncand][65536] or null
  double* out;             // [ncand][nblocks][kOutStride]
  int metrics;             // accumulate sse / max error / SSIM after the last level
  int ssim_win, ssim_step, is3d;
  double c1, c2;           // SSIM constants (used when bt is null)
  int ac;                  // accumulate the lag-1 error sums of Eq. (ac) after the last level
  const BoundTable* bt;    // value range on the device: SSIM constants from its range
  int use_tma;             // full-resolution block by one bulk tensor copy (tensor map given)
  int pitch;               // row pitch of the block in shared memory (values)
};

// Compensated (Kahan) binary32 accumulator for per-target sums: double
// arithmetic runs at a small fraction of the binary32 rate on this part, so
// per-point work stays in binary32 and only per-thread totals widen.
struct KSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Merges another compensated sum (s2 - c2) into k: the rounding error of
// s + s2 is recovered exactly (Knuth's two-sum, symmetric in its operands,
// so every lane of a butterfly ends with the same value) and moved into the
// compensation.  Binary32 only: double arithmetic issues at a small fraction
// of the binary32 rate on this part and dominated the short trials.
__device__ __forceinline__ void ksum_merge(KSum& k, float s2, float c2) {
  const float t = __fadd_rn(k.s, s2);
  const float bb = __fsub_rn(t, k.s);
  const float err = __fadd_rn(__fsub_rn(k.s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
  k.c = __fsub_rn(__fadd_rn(k.c, c2), err);
  k.s = t;
}
__device__ __forceinline__ void warp_ksum(KSum& k) {
  for (int off = 16; off > 0; off >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, k.s, off);
    const float c2 = __shfl_xor_sync(0xffffffffu, k.c, off);
    ksum_merge(k, s2, c2);
  }
}
// Maximum that keeps a NaN once one is seen.
__device__ __forceinline__ float nan_max(float m, float v) { return (v != v || v > m) ? v : m; }
__device__ __forceinline__ float warp_nan_max(float v) {
  for (int off = 16; off > 0; off >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// The block is held in shared memory subsampled by f = 2^(stop_level - 1):
// the levels that run (stop_level and above) only ever touch those points,
// and level l of the block is level l - stop_level + 1 of the subsampled
// grid (half-stride 2^(l - stop_level)).  x becomes the reconstruction in
// place, target by target.
// Polls of the block copy's mbarrier before the CTA gives up (the out slot's
// flag then reports it).
constexpr unsigned kTrialWaitPolls = 1u << 24;

// One pass of a trial, its geometry fixed at compile time: Bk is physical
// axis k's role in the pass (0: an axis the level's order visits before the
// pass axis, every h; 1: the pass axis, targets at h mod 2h; 2: an axis
// visited after it, every 2h), IP the interpolator.  Every target of the
// pass, flattened (x fastest) so that all lanes work; the quotients come
// from a binary32 reciprocal, which is exact for dividends below 70000 and
// divisors below 4100 (checked exhaustively), else from integer division.
struct TrialPass {
  float* S;
  int nS;
  int m0, m1, m2, st0, st1, h;
  float el, two_e, inv;
  bool score, metrics, hist;
  unsigned* SH;     // histogram window
  unsigned* ghist;  // the candidate's global histogram (codes outside the window)
};

struct TrialAcc {
  KSum l1, sse;
  float mx = 0.0f;
  int l1n = 0, unp = 0;
};

constexpr float kQTwo23 = 8388608.0f;     // 2^23
constexpr float kQCodeBias = 8421376.0f;  // 2^23 + 32768

template <int THREADS, bool kFull, int B0, int B1, int B2, int IP>
__device__ __forceinline__ void trial_pass(const TrialPass& t, TrialAcc& acc) {
  static_assert((B0 == 1) + (B1 == 1) + (B2 == 1) == 1, "one pass axis");
  constexpr int AX = B0 == 1 ? 0 : (B1 == 1 ? 1 : 2);
  const int h = t.h, h2 = 2 * h;
  const int s0 = B0 == 1 ? h : 0, s1 = B1 == 1 ? h : 0, s2 = B2 == 1 ? h : 0;
  const int d0 = B0 == 0 ? h : h2, d1 = B1 == 0 ? h : h2, d2 = B2 == 0 ? h : h2;
  const int c0n = t.m0 - 1 >= s0 ? (t.m0 - 1 - s0) / d0 + 1 : 0;
  const int c1n = t.m1 - 1 >= s1 ? (t.m1 - 1 - s1) / d1 + 1 : 0;
  const int c2n = t.m2 - 1 >= s2 ? (t.m2 - 1 - s2) / d2 + 1 : 0;
  const int sa = AX == 0 ? t.st0 : (AX == 1 ? t.st1 : 1);
  const int na = AX == 0 ? t.m0 : (AX == 1 ? t.m1 : t.m2);
  const int hs = h * sa;
  const int nrow = c0n * c1n;
  const int items = nrow * c2n;
  const bool fdiv = items < 70000 && c2n < 4100 && c1n < 4100;
  const float rc2 = 1.0f / (float)(c2n > 0 ? c2n : 1);
  const float rc1 = 1.0f / (float)(c1n > 0 ? c1n : 1);
  float* S = t.S;
  const int nS = t.nS;
  (void)nS;
  // a target's position, its field value and its prediction
  struct Tgt {
    int li;
    float xv, pred;
    bool ok;
  };
  auto fetch = [&](int it) -> Tgt {
    const int row =
        fdiv ? __float2int_rz(__fmul_rn(__fadd_rn(__int2float_rn(it), 0.5f), rc2)) : it / c2n;
    const int i2 = it - row * c2n;
    const int i0 =
        fdiv ? __float2int_rz(__fmul_rn(__fadd_rn(__int2float_rn(row), 0.5f), rc1)) : row / c1n;
    const int i1 = row - i0 * c1n;
    const int z = s0 + i0 * d0, y = s1 + i1 * d1, xx = s2 + i2 * d2;
    Tgt g;
    g.li = z * t.st0 + y * t.st1 + xx;
    const int ca = AX == 0 ? z : (AX == 1 ? y : xx);
    const bool hb1 = ca + h < na, ha3 = ca >= 3 * h, hb3 = ca + 3 * h < na;
    g.ok = QOZ_IN(g.li, nS) && QOZ_IN(g.li - hs, nS) && (!hb1 || QOZ_IN(g.li + hs, nS)) &&
           (!ha3 || QOZ_IN(g.li - 3 * hs, nS)) && (!hb3 || QOZ_IN(g.li + 3 * hs, nS));
    if (!g.ok) {
      g.xv = g.pred = 0.0f;
      return g;
    }
    const float a1 = S[g.li - hs];
    const float b1 = hb1 ? S[g.li + hs] : 0.0f;
    const float a3 = ha3 ? S[g.li - 3 * hs] : 0.0f;
    const float b3 = hb3 ? S[g.li + 3 * hs] : 0.0f;
    g.pred = predict(a3, a1, b1, b3, ha3, hb1, hb3, IP);
    g.xv = S[g.li];  // not yet predicted: still the field value
    return g;
  };
  auto finish = [&](const Tgt& g) {
    const float xv = g.xv, pred = g.pred;
    if (t.score) {
      const float ad = fabsf(__fsub_rn(xv, pred));
      if (isfinite(ad)) {
        acc.l1.add(ad);
        ++acc.l1n;
      }
    }
    // the quantizer's fast path: m = floor(|d| inv + 0.5) from a
    // round-toward-minus-infinity add of 2^23, the code from the bits of
    // q + 2^23 + 32768; whenever it accepts a point its result is the
    // reference quantizer's, which decides every other point
    const float d = __fsub_rn(xv, pred);
    const float u = __fadd_rn(__fmul_rn(fabsf(d), t.inv), 0.5f);
    const float m = __fsub_rn(__fadd_rd(u, kQTwo23), kQTwo23);
    const float cf = __fadd_rn(copysignf(m, d), kQCodeBias);
    float rec = __fadd_rn(pred, __fmul_rn(__fsub_rn(cf, kQCodeBias), t.two_e));
    unsigned code = __float_as_uint(cf) & 0xffffu;
    if (!((u < 32768.0f) & (fabsf(__fsub_rn(xv, rec)) <= t.el))) {
      uint16_t c16;
      float rr;
      if (quantize(xv, pred, t.el, t.two_e, t.inv, &c16, &rr)) {
        code = c16;
        rec = rr;
      } else {
        code = 0;
        rec = xv;
        ++acc.unp;
      }
    }
    S[g.li] = rec;
    if (kFull && t.metrics) {  // every non-anchor point is a target once
      const float e = __fsub_rn(xv, rec);
      acc.sse.add(__fmul_rn(e, e));
      const float ae = fabsf(e);
      if (ae != ae || ae > acc.mx) acc.mx = ae;
    }
    if (kFull && t.hist) {
      // one shared atomic per code (the window around the zero bin), global
      // beyond it
      const unsigned kk = code - (unsigned)kTHistLo;
      if (kk < (unsigned)kTHistWin)
        atomicAdd(&t.SH[kk], 1u);
      else
        atomicAdd(&t.ghist[code], 1u);
    }
  };
  for (int it = threadIdx.x; it < items; it += THREADS) {
    const Tgt g = fetch(it);
    if (g.ok) finish(g);
  }
}

// The pass for role code b0 * 9 + b1 * 3 + b2 and interpolator ip (uniform
// over the CTA).
template <int THREADS, bool kFull>
__device__ __forceinline__ void trial_pass_dispatch(int roles, int ip, const TrialPass& t,
                                                    TrialAcc& acc) {
#define QOZ_TRIAL_PASS(B0, B1, B2)                                 \
  case B0 * 9 + B1 * 3 + B2:                                       \
    if (ip == 1)                                                   \
      trial_pass<THREADS, kFull, B0, B1, B2, 1>(t, acc);           \
    else                                                           \
      trial_pass<THREADS, kFull, B0, B1, B2, 0>(t, acc);           \
    break;
  switch (roles) {
    QOZ_TRIAL_PASS(1, 0, 0)
    QOZ_TRIAL_PASS(1, 0, 2)
    QOZ_TRIAL_PASS(1, 2, 0)
    QOZ_TRIAL_PASS(1, 2, 2)
    QOZ_TRIAL_PASS(0, 1, 0)
    QOZ_TRIAL_PASS(0, 1, 2)
    QOZ_TRIAL_PASS(2, 1, 0)
    QOZ_TRIAL_PASS(2, 1, 2)
    QOZ_TRIAL_PASS(0, 0, 1)
    QOZ_TRIAL_PASS(0, 2, 1)
    QOZ_TRIAL_PASS(2, 0, 1)
    QOZ_TRIAL_PASS(2, 2, 1)
    default:
      break;
  }
#undef QOZ_TRIAL_PASS
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS >= 512 ? 1 : 4)
    trial_kernel(const TrialArgs a, const __grid_constant__ CUtensorMap tmap) {
  // the coarse variant runs only levels above the finest (no histogram, no
  // metrics): that code is compiled out of it
  constexpr bool kFull = THREADS >= kTrialThreads;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  const int f = 1 << (a.stop_level - 1);
  const int m0 = (a.bd[0] - 1) / f + 1, m1 = (a.bd[1] - 1) / f + 1, m2 = (a.bd[2] - 1) / f + 1;
  const int P = a.pitch;  // >= m2 (+ the bulk copy's 16-byte shift)
  // 128-byte aligned block buffer; the histogram window after it
  unsigned char* base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
  unsigned* SH = reinterpret_cast<unsigned*>(
      base + (((size_t)sizeof(float) * m0 * m1 * P + 15) & ~size_t(15)));
  __shared__ float redf[THREADS / 32][11];    // l1, sse, ac sums (s, c each), max error
  __shared__ unsigned redu[THREADS / 32][2];  // l1 count, unpredictable count
  __shared__ double redd[THREADS / 32][2];    // SSIM sum, window count

  const int cand = blockIdx.x / a.nblocks;
  const int blk = blockIdx.x % a.nblocks;
  const TrialCand& C = a.cands[cand];
  const int oz = a.origins[3 * blk + 0], oy = a.origins[3 * blk + 1], ox = a.origins[3 * blk + 2];
  const float* xb = a.x + (long long)oz * a.st0 + (long long)oy * a.st1 + ox;
  const long long fs0 = (long long)f * a.st0, fs1 = (long long)f * a.st1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // the bulk copy starts at the 16-byte boundary at or below the block's x
  // origin; the block itself then starts ox mod 4 values into the buffer
  float* S = reinterpret_cast<float*>(base) + (a.use_tma ? (ox & 3) : 0);
  // values of the block buffer reachable from S (checked by the
  // bounds-checking build)
  const int nS = m0 * m1 * P - (a.use_tma ? (ox & 3) : 0);
  (void)nS;

  if (a.use_tma) {
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_expect_tx(&mbar, (unsigned)(sizeof(float) * m0 * m1 * P));
      tma_load_3d(base, &tmap, ox & ~3, oy, oz, &mbar);
    }
  } else {
    for (int row = warp; row < m0 * m1; row += nw) {
      const int z = row / m1, y = row - (row / m1) * m1;
      const float* src = xb + z * fs0 + y * fs1;
      float* dst = S + row * P;
      for (int xx = lane; xx < m2; xx += 32) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst + xx);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + xx * f)
                     : "memory");
      }
    }
  }
  if (a.hist)
    for (int i = threadIdx.x; i < kTHistWin; i += blockDim.x) SH[i] = 0;
  if (a.use_tma) {
    bool landed = false;
    for (unsigned it = 0; it < kTrialWaitPolls; ++it)
      if (mbar_try_wait(&mbar, 0)) {
        landed = true;
        break;
      }
    if (!__syncthreads_and(landed)) {
      if (threadIdx.x == 0) a.out[((size_t)cand * a.nblocks + blk) * kOutStride + 7] = 1.0;
      return;
    }
  } else {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
  }

  KSum sse0;         // the anchors' squared errors
  float mx0 = 0.0f;  // and their maximum
  const int st1 = P, st0 = m1 * P;
  if (kFull && a.metrics) {
    // the block's anchors (never targets) reconstruct exactly: they add to
    // the squared and maximum error only through non-finite values
    const int as = 1 << (a.Ls - a.stop_level + 1);
    const int n0 = (m0 - 1) / as + 1, n1a = (m1 - 1) / as + 1, n2a = (m2 - 1) / as + 1;
    for (int i = threadIdx.x; i < n0 * n1a * n2a; i += THREADS) {
      const int i2 = i % n2a, r = i / n2a;
      const int si = (r / n1a) * as * st0 + (r % n1a) * as * st1 + i2 * as;
      const float v = QOZ_IN(si, nS) ? S[si] : 0.0f;
      const float d = __fsub_rn(v, v);
      sse0.add(__fmul_rn(d, d));
      const float ad = fabsf(d);
      if (ad != ad || ad > mx0) mx0 = ad;
    }
  }
  TrialAcc acc;
  for (int l = a.Ls; l >= a.stop_level; --l) {
    const int h = 1 << (l - a.stop_level);
    const int interp = C.interp[l - 1];
    const int ax0 = C.axes[l - 1][0], ax1 = C.axes[l - 1][1];
    TrialPass tp;
    tp.S = S;
    tp.nS = nS;
    tp.m0 = m0;
    tp.m1 = m1;
    tp.m2 = m2;
    tp.st0 = st0;
    tp.st1 = st1;
    tp.h = h;
    tp.el = C.el[l - 1];
    tp.two_e = C.two_e[l - 1];
    tp.inv = C.inv[l - 1];
    tp.score = l == a.score_level;
    tp.metrics = kFull && a.metrics;
    tp.hist = kFull && a.hist != nullptr;
    tp.SH = SH;
    tp.ghist = a.hist ? a.hist + (size_t)cand * 65536 : nullptr;
    for (int k = 0; k < 3; ++k) {
      // position of each physical axis in the order: before the pass axis
      // (0), the pass axis (1), after it (2)
      const int j0 = ax0 == 0 ? 0 : (ax1 == 0 ? 1 : 2);
      const int j1 = ax0 == 1 ? 0 : (ax1 == 1 ? 1 : 2);
      const int j2 = ax0 == 2 ? 0 : (ax1 == 2 ? 1 : 2);
      const int b0 = j0 == k ? 1 : (j0 < k ? 0 : 2);
      const int b1 = j1 == k ? 1 : (j1 < k ? 0 : 2);
      const int b2 = j2 == k ? 1 : (j2 < k ? 0 : 2);
      trial_pass_dispatch<THREADS, kFull>(b0 * 9 + b1 * 3 + b2, interp, tp, acc);
      __syncthreads();
    }
  }
  KSum& l1 = acc.l1;
  KSum& sse = acc.sse;
  ksum_merge(sse, sse0.s, sse0.c);  // the anchors' terms (zero unless non-finite)
  float mx = nan_max(acc.mx, mx0);
  const int l1n = acc.l1n, unp = acc.unp;

  double ss = 0.0, sn = 0.0;
  if (kFull && a.metrics) {  // stop_level == 1: S is the whole block
    const int n1 = a.bd[1], n2 = a.bd[2];
    if (a.ssim_win > 0) {
      double c1 = a.c1, c2 = a.c2;
      if (a.bt) {
        const double vr = a.bt->vrange;
        c1 = __dmul_rn(__dmul_rn(0.01, vr), __dmul_rn(0.01, vr));
        c2 = __dmul_rn(__dmul_rn(0.03, vr), __dmul_rn(0.03, vr));
      }
      const int n0 = a.bd[0];
      const int w = a.ssim_win, sp = a.ssim_step;
      const int wz = a.is3d ? w : 1;
      auto cntw = [&](int n) { return n >= w ? (n - w) / sp + 1 : 0; };
      const int c0 = a.is3d ? cntw(n0) : 1, c1n = cntw(n1), c2n = cntw(n2);
      const int nwin = c0 * c1n * c2n;
      const double np = (double)w * w * wz;
      for (int wi = threadIdx.x; wi < nwin; wi += blockDim.x) {
        const int w2 = wi % c2n;
        const int r = wi / c2n;
        const int w1 = r % c1n;
        const int w0 = r / c1n;
        if (!QOZ_IN((w0 * sp + wz - 1) * n1 * P + (w1 * sp + w - 1) * P + w2 * sp + w - 1, nS))
          continue;
        // window moments in binary32, centred on the window means to keep the
        // variances well conditioned; the SSIM formula itself in double
        float sx = 0.0f, sy = 0.0f;
        for (int i = 0; i < wz; ++i)
          for (int j = 0; j < w; ++j) {
            const int z = w0 * sp + i, y = w1 * sp + j;
            const float* src = xb + z * a.st0 + y * a.st1 + w2 * sp;
            const float* rec = S + (z * n1 + y) * P + w2 * sp;
            for (int k = 0; k < w; ++k) {
              sx = __fadd_rn(sx, src[k]);
              sy = __fadd_rn(sy, rec[k]);
            }
          }
        const float fx = sx / (float)np, fy = sy / (float)np;
        float vxx = 0.0f, vyy = 0.0f, vxy = 0.0f, rx = 0.0f, ry = 0.0f;
        for (int i = 0; i < wz; ++i)
          for (int j = 0; j < w; ++j) {
            const int z = w0 * sp + i, y = w1 * sp + j;
            const float* src = xb + z * a.st0 + y * a.st1 + w2 * sp;
            const float* rec = S + (z * n1 + y) * P + w2 * sp;
            for (int k = 0; k < w; ++k) {
              const float dx = __fsub_rn(src[k], fx), dy = __fsub_rn(rec[k], fy);
              rx = __fadd_rn(rx, dx);
              ry = __fadd_rn(ry, dy);
              vxx = __fadd_rn(vxx, __fmul_rn(dx, dx));
              vyy = __fadd_rn(vyy, __fmul_rn(dy, dy));
              vxy = __fadd_rn(vxy, __fmul_rn(dx, dy));
            }
          }
        // exact-in-exact-arithmetic corrections for the rounded means
        const double mxx = (double)fx + (double)rx / np, myy = (double)fy + (double)ry / np;
        const double ex = (double)rx / np, ey = (double)ry / np;
        const double vx = (double)vxx / np - ex * ex, vy = (double)vyy / np - ey * ey;
        const double cxy = (double)vxy / np - ex * ey;
        ss += ((2.0 * mxx * myy + c1) * (2.0 * cxy + c2)) /
              ((mxx * mxx + myy * myy + c1) * (vx + vy + c2));
        sn += 1.0;
      }
    }
  }
  // Eq. (ac) sums over the block in its row-major order (stop_level == 1:
  // S holds the whole reconstruction): e = reconstruction - original
  KSum as1, as2, ask;
  if (kFull && a.ac && a.metrics) {
    const int n0 = a.bd[0], n1 = a.bd[1], n2 = a.bd[2];
    const int nbp = n0 * n1 * n2;
    double* o = a.out + ((size_t)cand * a.nblocks + blk) * kOutStride;
    auto err_at = [&](int z, int y, int x) {
      const int si = (z * n1 + y) * P + x;
      return QOZ_IN(si, nS) ? __fsub_rn(S[si], xb[z * a.st0 + y * a.st1 + x]) : 0.0f;
    };
    for (int i = threadIdx.x; i < nbp; i += THREADS) {
      const int x = i % n2, r = i / n2, y = r % n1, z = r / n1;
      const float e = err_at(z, y, x);
      as1.add(e);
      as2.add(__fmul_rn(e, e));
      if (i + 1 < nbp) {
        int x2 = x + 1, y2 = y, z2 = z;
        if (x2 == n2) {
          x2 = 0;
          if (++y2 == n1) {
            y2 = 0;
            ++z2;
          }
        }
        ask.add(__fmul_rn(e, err_at(z2, y2, x2)));
      }
      if (i == 0) o[11] = (double)e;
      if (i == nbp - 1) o[12] = (double)e;
    }
  }
  if (kFull && a.hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTHistWin; i += blockDim.x)
      if (SH[i]) atomicAdd(&a.hist[(size_t)cand * 65536 + kTHistLo + i], SH[i]);
  }
  // fixed-order block reduction: warps, then warp 0 over the warps' partials
  warp_ksum(l1);
  warp_ksum(sse);
  if (kFull && a.ac) {
    warp_ksum(as1);
    warp_ksum(as2);
    warp_ksum(ask);
  }
  mx = warp_nan_max(mx);
  const unsigned l1c = __reduce_add_sync(0xffffffffu, (unsigned)l1n);
  const unsigned unc = __reduce_add_sync(0xffffffffu, (unsigned)unp);
  if (kFull && a.ssim_win > 0) {
    ss = warp_sum(ss);
    sn = warp_sum(sn);
  }
  if (lane == 0) {
    redf[warp][0] = l1.s;
    redf[warp][1] = l1.c;
    redf[warp][2] = sse.s;
    redf[warp][3] = sse.c;
    redf[warp][4] = mx;
    redf[warp][5] = as1.s;
    redf[warp][6] = as1.c;
    redf[warp][7] = as2.s;
    redf[warp][8] = as2.c;
    redf[warp][9] = ask.s;
    redf[warp][10] = ask.c;
    redu[warp][0] = l1c;
    redu[warp][1] = unc;
    redd[warp][0] = ss;
    redd[warp][1] = sn;
  }
  __syncthreads();
  if (warp == 0) {
    const bool on = lane < nw;
    KSum t1, t3;
    t1.s = on ? redf[lane][0] : 0.0f;
    t1.c = on ? redf[lane][1] : 0.0f;
    t3.s = on ? redf[lane][2] : 0.0f;
    t3.c = on ? redf[lane][3] : 0.0f;
    warp_ksum(t1);
    warp_ksum(t3);
    const float m = warp_nan_max(on ? redf[lane][4] : 0.0f);
    const unsigned c1 = __reduce_add_sync(0xffffffffu, on ? redu[lane][0] : 0u);
    const unsigned c2 = __reduce_add_sync(0xffffffffu, on ? redu[lane][1] : 0u);
    KSum t8, t9, t10;
    if (kFull && a.ac) {
      t8.s = on ? redf[lane][5] : 0.0f;
      t8.c = on ? redf[lane][6] : 0.0f;
      t9.s = on ? redf[lane][7] : 0.0f;
      t9.c = on ? redf[lane][8] : 0.0f;
      t10.s = on ? redf[lane][9] : 0.0f;
      t10.c = on ? redf[lane][10] : 0.0f;
      warp_ksum(t8);
      warp_ksum(t9);
      warp_ksum(t10);
    }
    double s5 = 0.0, s6 = 0.0;
    if (kFull && a.ssim_win > 0) {
      s5 = warp_sum(on ? redd[lane][0] : 0.0);
      s6 = warp_sum(on ? redd[lane][1] : 0.0);
    }
    if (lane == 0) {
      double* o = a.out + ((size_t)cand * a.nblocks + blk) * kOutStride;
      o[0] = t1.value();
      o[1] = (double)c1;
      o[2] = (double)c2;
      o[3] = t3.value();
      o[4] = (double)m;
      o[5] = s5;
      o[6] = s6;
      o[7] = 0.0;
      if (kFull && a.ac) {
        o[8] = t8.value();
        o[9] = t9.value();
        o[10] = t10.value();
      }
    }
  }
}

// Optimal prefix-code cost of one candidate's pooled histogram (the rate
// estimate of Sec. 6.1): one CTA per candidate.  The cost is the sum of the
// weights of the merged nodes of Huffman's construction, run as the
// two-queue merge (leaves and merged nodes both come out in non-decreasing
// order).  Up to kHuffSmall used codes, the counts are sorted and merged one
// by one with the queue heads in registers.  With more, the leaves come
// sorted without a sort (counts up to kHuffSmall bucketed by value, the few
// larger ones sorted) and the merge runs over runs of equal weight: while
// the smallest item's run holds two or more items, pairing them is what the
// merge would do step by step, so all pairs of the run are merged at once.
// Integer arithmetic: the same total as the host computation.  More than
// kHuffBig large counts or kHuffNodes live node runs are left to the host
// (flag 1).
constexpr int kHuffThreads = 1024;
constexpr int kHuffSmall = 4096;
constexpr int kHuffBig = 2048;
constexpr int kHuffNodes = 4096;  // node runs alive at once (a ring)

struct HuffCostSmem {
  unsigned small[kHuffSmall + 1];        // multiplicity of each count 1..kHuffSmall
  union {
    struct {                             // up to kHuffSmall used codes: the counts
      unsigned cnt[kHuffSmall];          // (sorted in place) and the merged weights
      unsigned node[kHuffSmall];         // (at most the sampled points, < 2^32)
    } sorted;
    struct {                             // more used codes: the non-empty buckets
      unsigned rc[kHuffSmall], rm[kHuffSmall];  // in count order
    } runs;
  } u;
  unsigned big[kHuffBig];                // counts above kHuffSmall (sorted in place)
  unsigned long long nw[kHuffNodes];     // node runs: weight
  unsigned nm[kHuffNodes];               // node runs: multiplicity
};

__global__ void __launch_bounds__(kHuffThreads)
    huffman_cost_kernel(const unsigned* __restrict__ hist, unsigned long long* bits, int* flag) {
  extern __shared__ __align__(16) unsigned char hsm[];
  HuffCostSmem& S = *reinterpret_cast<HuffCostSmem*>(hsm);
  __shared__ int nbig, nruns;
  __shared__ unsigned long long nsym;
  __shared__ int wsum[32];
  const uint4* h4 = reinterpret_cast<const uint4*>(hist + (size_t)blockIdx.x * 65536);
  const int t = threadIdx.x;
  for (int i = t; i <= kHuffSmall; i += kHuffThreads) S.small[i] = 0u;
  if (t == 0) {
    nbig = 0;
    nsym = 0ull;
  }
  __syncthreads();
  // coalesced 16-byte scan, kBatch loads in flight per thread: each warp
  // appends its non-zero counts (any order: they are sorted next) and the
  // total of used codes
  constexpr int kVec = 65536 / 4 / kHuffThreads, kBatch = 4;
  const int lane = t & 31;
  for (int j0 = 0; j0 < kVec; j0 += kBatch) {
    uint4 v[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) v[j] = h4[(j0 + j) * kHuffThreads + t];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const unsigned q[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
      const int nz = (q[0] != 0u) + (q[1] != 0u) + (q[2] != 0u) + (q[3] != 0u);
      if (__ballot_sync(0xffffffffu, nz != 0) == 0u) continue;
      int inc = nz;  // inclusive prefix over the warp
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
      }
      unsigned long long base = 0ull;
      if (lane == 31) base = atomicAdd(&nsym, (unsigned long long)inc);
      unsigned long long k = __shfl_sync(0xffffffffu, base, 31) + (unsigned long long)(inc - nz);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (q[e] != 0u) {
          if (k < (unsigned long long)kHuffSmall) S.u.sorted.cnt[k] = q[e];
          ++k;
        }
    }
  }
  __syncthreads();
  if (nsym <= (unsigned long long)kHuffSmall) {
    // few used codes: sort the counts and run the two-queue merge with the
    // queue heads in registers and the next leaf prefetched (the sorted
    // leaves are padded with 0xffffffff)
    unsigned* cnt = S.u.sorted.cnt;
    unsigned* node = S.u.sorted.node;
    const int n = (int)nsym;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + t; i < P; i += kHuffThreads) cnt[i] = 0xffffffffu;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = t; i < P; i += kHuffThreads) {
          const int j = i ^ stride;
          if (j > i) {
            const bool up = (i & size) == 0;
            const unsigned a = cnt[i], b = cnt[j];
            if ((a > b) == up) {
              cnt[i] = b;
              cnt[j] = a;
            }
          }
        }
        __syncthreads();
      }
    if (t != 0) return;
    unsigned long long total = 0ull;
    if (n == 1) {
      total = cnt[0];
    } else if (n > 1) {
      int li = 0, ni = 0, nn = 0;
      unsigned hl = cnt[0], hl2 = cnt[1], hn = 0u;
      for (int m = 1; m < n; ++m) {
        unsigned ab[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (ni < nn && (li >= n || hn < hl)) {
            ab[k] = hn;
            ++ni;
            hn = ni < nn ? node[ni] : 0u;
          } else {
            ab[k] = hl;
            ++li;
            hl = hl2;
            hl2 = li + 1 < P ? cnt[li + 1] : 0xffffffffu;
          }
        }
        const unsigned sum = ab[0] + ab[1];
        total += sum;
        node[nn] = sum;
        if (ni == nn) hn = sum;
        ++nn;
      }
    }
    bits[blockIdx.x] = total;
    flag[blockIdx.x] = 0;
    return;
  }
  // many used codes: a second scan buckets the counts by value
  for (int j0 = 0; j0 < kVec; j0 += kBatch) {
    uint4 v[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) v[j] = h4[(j0 + j) * kHuffThreads + t];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const unsigned q[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const unsigned c = q[e];
        if (c == 0u) continue;
        if (c <= (unsigned)kHuffSmall) {
          atomicAdd(&S.small[c], 1u);
        } else {
          const int kb = atomicAdd(&nbig, 1);
          if (kb < kHuffBig) S.big[kb] = c;
        }
      }
    }
  }
  __syncthreads();
  const int nb = nbig;
  if (nb > kHuffBig) {
    if (t == 0) {
      flag[blockIdx.x] = 1;
      bits[blockIdx.x] = 0ull;
    }
    return;
  }
  // the non-empty buckets, compacted in count order (a block-wide scan over
  // four consecutive buckets per thread)
  {
    static_assert(kHuffSmall == 4 * kHuffThreads, "four buckets per thread");
    const int c0 = 4 * t + 1;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) cnt += S.small[c0 + k] != 0u ? 1 : 0;
    const int lane = t & 31, w = t >> 5;
    int inc = cnt;
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
      const int x = wsum[lane];
      int wi = x;
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += y;
      }
      wsum[lane] = wi - x;
      if (lane == 31) nruns = wi;
    }
    __syncthreads();
    int pos = wsum[w] + inc - cnt;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned m = S.small[c0 + k];
      if (m != 0u) {
        S.u.runs.rc[pos] = (unsigned)(c0 + k);
        S.u.runs.rm[pos] = m;
        ++pos;
      }
    }
  }
  int P = 1;
  while (P < nb) P <<= 1;
  for (int i = nb + t; i < P; i += kHuffThreads) S.big[i] = 0xffffffffu;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = t; i < P; i += kHuffThreads) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned a = S.big[i], b = S.big[j];
          if ((a > b) == up) {
            S.big[i] = b;
            S.big[j] = a;
          }
        }
      }
      __syncthreads();
    }
  if (t != 0) return;
  // leaf runs in order: the bucketed counts, then the sorted large ones
  const int nr = nruns;
  int ri = 0, bi = 0;                    // next bucket run / big index
  unsigned long long lw = 0ull;          // current leaf run (weight, items left)
  unsigned long long lm = 0ull;
  auto next_leaf_run = [&]() {
    lm = 0ull;
    if (ri < nr) {
      lw = (unsigned long long)S.u.runs.rc[ri];
      lm = S.u.runs.rm[ri];
      ++ri;
      return;
    }
    if (bi < nb) {
      lw = S.big[bi];
      lm = 0ull;
      while (bi < nb && S.big[bi] == lw) {
        ++lm;
        ++bi;
      }
    }
  };
  next_leaf_run();
  unsigned long long items = nsym;
  unsigned long long total = 0ull;
  int bad = 0;
  if (items == 1ull) {
    total = lw;  // a lone symbol: one bit per occurrence
  } else {
    unsigned nh = 0u, nt = 0u;  // node-run ring [nh, nt), indices taken mod kHuffNodes
    constexpr unsigned kMask = kHuffNodes - 1;
    static_assert((kHuffNodes & (kHuffNodes - 1)) == 0, "ring size is a power of two");
    auto push_node = [&](unsigned long long w, unsigned long long m) {
      if (nt > nh && S.nw[(nt - 1u) & kMask] == w) {
        S.nm[(nt - 1u) & kMask] += (unsigned)m;
      } else if (nt - nh < (unsigned)kHuffNodes) {
        S.nw[nt & kMask] = w;
        S.nm[nt & kMask] = (unsigned)m;
        ++nt;
      } else {
        bad = 1;
      }
    };
    // takes one item of the smallest front; returns its weight
    auto take_one = [&]() -> unsigned long long {
      const bool node = nt > nh && (lm == 0ull || S.nw[nh & kMask] < lw);
      unsigned long long w;
      if (node) {
        w = S.nw[nh & kMask];
        if (--S.nm[nh & kMask] == 0u) ++nh;
      } else {
        w = lw;
        if (--lm == 0ull) next_leaf_run();
      }
      return w;
    };
    while (items > 1ull && !bad) {
      const bool node = nt > nh && (lm == 0ull || S.nw[nh & kMask] < lw);
      const unsigned long long w = node ? S.nw[nh & kMask] : lw;
      const unsigned long long m = node ? (unsigned long long)S.nm[nh & kMask] : lm;
      if (m >= 2ull) {
        // every pair of this run is among the two smallest items in turn
        const unsigned long long k = m / 2ull;
        total += 2ull * w * k;
        if (node) {
          S.nm[nh & kMask] -= (unsigned)(2ull * k);
          if (S.nm[nh & kMask] == 0u) ++nh;
        } else {
          lm -= 2ull * k;
          if (lm == 0ull) next_leaf_run();
        }
        push_node(2ull * w, k);
        items -= k;
      } else {
        const unsigned long long a = take_one();
        const unsigned long long b = take_one();
        total += a + b;
        push_node(a + b, 1ull);
        items -= 1ull;
      }
    }
  }
  bits[blockIdx.x] = bad ? 0ull : total;
  flag[blockIdx.x] = bad;
}

// Algorithm 1 on the device, one level at a time: the level's candidates
// (interpolator, order) are scored by the mean |x - pred| of their trial
// (one warp per candidate sums its blocks in double, lane-strided with a
// fixed butterfly); the first candidate within 1e-12 relative of the best
// wins; the choice is recorded and the next level's candidates are built
// (levels above keep the choices made), so the levels run back to back
// without the host.
struct Alg1Ctl {
  unsigned char ci[16], co[16];  // candidate interpolators and orders
  unsigned char chi[kMaxLevels], cho[kMaxLevels];  // choices per level
  double score[kMaxLevels];
};

__constant__ int kPermDev[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ void set_axes_dev(TrialCand* c, int level, int ndims, int order) {
  const int o3 = ndims == 3 ? order : (order == 0 ? 0 : 1);
  for (int k = 0; k < 3; ++k) c->axes[level - 1][k] = (unsigned char)kPermDev[o3][k];
}

constexpr int kAlg1MaxCand = 16;

// Level bounds of Eq. (ebl) for one candidate: e_l = e / min(alpha^(l-1),
// beta) in double, each entry rounded to binary32 once (the same operations,
// in the same order, as the host's fill_bounds).
__device__ void fill_bounds_dev(TrialCand* c, double e, double alpha, double beta, int L) {
  double a = 1.0;
  for (int l = 0; l < kMaxLevels; ++l) {
    if (l < L) {
      const double den = a < beta ? a : beta;
      const double el = __ddiv_rn(e, den);
      const double two = __dmul_rn(2.0, el);
      c->el[l] = __double2float_rn(el);
      c->two_e[l] = __double2float_rn(two);
      c->inv[l] = __double2float_rn(__ddiv_rn(1.0, two));
      a = __dmul_rn(a, alpha);
    } else {
      c->el[l] = c->two_e[l] = c->inv[l] = 0.0f;
    }
  }
}

// The tuner's starting bound e0 from the device value range: the user's
// bound rel * range, or, for a PSNR target (Sec. 6.3.2), the smaller of that
// and range * sqrt(3) * 10^(-P / 20) (both factors evaluated on the host).
struct E0Spec {
  int psnr_target;
  double sqrt3, p10;
};
__device__ double e0_dev(const BoundTable& bt, const E0Spec& sp) {
  double e0 = bt.e;  // rel * range (the bound table was filled with eb = rel)
  if (sp.psnr_target) {
    const double t = __dmul_rn(__dmul_rn(bt.vrange, sp.sqrt3), sp.p10);
    e0 = t > e0 ? e0 : t;
  }
  return e0;
}

// The (alpha, beta) candidates of Sec. 6.3, built on the device once
// Algorithm 1 has chosen every level: candidate k = (si * na + ia) * nb + ib
// at bound scales[si] * e0.
// The (alpha, beta) candidates of a tune: n_pairs distinct settings (index
// pairs into alphas / betas) at n_scales bounds.  With alpha = 1 every level
// bound is e (min(1, beta) = 1 for beta >= 1), so the pairs (1, beta) after
// the first give the same trial and are not run; the host copies its result.
struct AbSpec {
  int n_alpha, n_beta, n_scales, n_pairs;
  double alphas[8], betas[8], scales[3];
  unsigned char pa[64], pb[64];
};

// Bounds of the top-level Algorithm 1 candidates (alpha = beta = 1, every
// level at e0) and e0 itself, from the device value range.
__global__ void alg1_setup_kernel(TrialCand* cands, int nc, const BoundTable* bt,
                                  const E0Spec sp, int Ls, double* e0_out) {
  const double e0 = e0_dev(*bt, sp);
  if (threadIdx.x == 0) *e0_out = e0;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) fill_bounds_dev(&cands[c], e0, 1.0, 1.0, Ls);
}

__global__ void __launch_bounds__(32 * kAlg1MaxCand)
    alg1_select_kernel(const double* __restrict__ out, int nc, int nb, int l, int Ls,
                       const TrialCand base, int ndims, Alg1Ctl* ctl, TrialCand* cands,
                       const AbSpec ab, const double* e0p) {
  __shared__ double mean[kAlg1MaxCand];
  __shared__ Alg1Ctl h;
  __shared__ int pick;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) h = *ctl;
  if (warp < nc) {
    double l1 = 0.0, l1n = 0.0;
    for (int b = lane; b < nb; b += 32) {
      l1 += out[((size_t)warp * nb + b) * kOutStride + 0];
      l1n += out[((size_t)warp * nb + b) * kOutStride + 1];
    }
    l1 = warp_sum(l1);
    l1n = warp_sum(l1n);
    if (lane == 0) mean[warp] = l1n > 0 ? l1 / l1n : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double best = 0.0;
    int bi = 0;
    for (int k = 0; k < nc; ++k) {
      const double cur = mean[k];
      if (k == 0 || cur < best - 1e-12 * best) {
        best = cur;
        bi = k;
      }
    }
    h.chi[l - 1] = h.ci[bi];
    h.cho[l - 1] = h.co[bi];
    h.score[l - 1] = best;
    ctl->chi[l - 1] = h.ci[bi];
    ctl->cho[l - 1] = h.co[bi];
    ctl->score[l - 1] = best;
    pick = bi;
  }
  __syncthreads();
  if (l == 1) {
    // every level chosen: the (alpha, beta) candidates, when asked for
    const int np = ab.n_pairs;
    if (np == 0) return;
    const double e0 = *e0p;
    for (int k = threadIdx.x; k < ab.n_scales * np; k += blockDim.x) {
      TrialCand t = base;
      for (int ll = 1; ll <= Ls; ++ll) {
        t.interp[ll - 1] = h.chi[ll - 1];
        set_axes_dev(&t, ll, ndims, h.cho[ll - 1]);
      }
      const int si = k / np, kk = k - si * np;
      fill_bounds_dev(&t, __dmul_rn(ab.scales[si], e0), ab.alphas[ab.pa[kk]], ab.betas[ab.pb[kk]],
                      Ls);
      cands[k] = t;
    }
    return;
  }
  const int c = threadIdx.x;
  if (c >= nc) return;
  // candidate c of level l - 1: its current entry (levels above l already
  // chosen, the bounds filled on the device) with level l set to the pick
  TrialCand t = cands[c];
  t.interp[l - 1] = h.ci[pick];
  set_axes_dev(&t, l, ndims, h.co[pick]);
  t.interp[l - 2] = h.ci[c];
  set_axes_dev(&t, l - 1, ndims, h.co[c]);
  cands[c] = t;
}

// ------------------------------------------------------------- host side


int floor_log2(long long v) {
  int l = 0;
  while ((2LL << l) <= v) ++l;
  return l;
}

}  // namespace

// Uniform block sampling, Sec. 6.1: blocks of b+1 points per axis placed
// every S = round(b r^(-1/d)) points while they fit; an axis shorter than a
// block is taken whole.
Sampling sample_blocks(const Resolved& r, int b, double rate, int s) {
  Sampling sm;
  const int d = r.ndims;
  long long S = std::llround((double)b * std::pow(rate, -1.0 / (double)d));
  if (S < 1) S = 1;
  std::vector<long long> starts[3];
  for (int p = 0; p < 3; ++p) {
    const bool active = !(d == 2 && p == 0);
    if (!active) {
      starts[p].push_back(0);
      sm.bd[p] = 1;
      continue;
    }
    for (long long o = 0; o + b <= r.n[p] - 1; o += S) starts[p].push_back(o);
    if (starts[p].empty()) {
      starts[p].push_back(0);
      sm.bd[p] = (int)r.n[p];
    } else {
      sm.bd[p] = b + 1;
    }
  }
  for (long long o0 : starts[0])
    for (long long o1 : starts[1])
      for (long long o2 : starts[2]) {
        sm.origins.push_back((int)o0);
        sm.origins.push_back((int)o1);
        sm.origins.push_back((int)o2);
      }
  sm.nb = (int)(sm.origins.size() / 3);
  sm.npts = (long long)sm.nb * sm.bd[0] * sm.bd[1] * sm.bd[2];
  sm.Ls = floor_log2(b < s ? b : s);
  const long long sb = 1LL << sm.Ls;
  long long apb = 1;
  for (int p = 0; p < 3; ++p) apb *= (sm.bd[p] + sb - 1) / sb;
  sm.anchors = apb * sm.nb;
  return sm;
}

namespace {

// Level bounds of Eq. (ebl) in double, each rounded to binary32 once.
void fill_bounds(TrialCand* c, double e, double alpha, double beta, int L) {
  double a = 1.0;
  for (int l = 0; l < kMaxLevels; ++l) {
    if (l < L) {
      const double den = a < beta ? a : beta;
      const double el = e / den;
      c->el[l] = (float)el;
      c->two_e[l] = (float)(2.0 * el);
      c->inv[l] = (float)(1.0 / (2.0 * el));
      a = a * alpha;
    } else {
      c->el[l] = c->two_e[l] = c->inv[l] = 0.0f;
    }
  }
}

const int kPerm3T[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

void set_axes(TrialCand* c, int level, int ndims, int order) {
  const int o3 = ndims == 3 ? order : (order == 0 ? 0 : 1);
  for (int k = 0; k < 3; ++k) c->axes[level - 1][k] = (unsigned char)kPerm3T[o3][k];
}

struct TrialResult {
  double B, M;             // bit rate, metric (higher is better)
  double l1_mean;
};

// Pinned host staging for the tuner's read-backs, one per host thread (a
// tuner call synchronises before it returns, so one call uses it at a
// time); grows on demand.
void* pinned_stage(size_t bytes) {
  static thread_local void* p = nullptr;
  static thread_local size_t cap = 0;
  if (bytes > cap) {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
      p = nullptr;
      return nullptr;
    }
    cap = bytes;
  }
  return p;
}

static_assert(sizeof(BoundTable) <= 256 && sizeof(Alg1Ctl) <= 256,
              "tuner range scratch layout");

class Tuner {
 public:
  Tuner(const float* x, const Resolved& r, const Sampling& sm, cudaStream_t s, int metric,
        int ssim_win, int ssim_step, double vrange)
      : x_(x), r_(r), sm_(sm), s_(s), metric_(metric), win_(ssim_win), step_(ssim_step),
        vr_(vrange) {}
  ~Tuner() {
    dev_free(d_orig_, s_);
    dev_free(d_cands_, s_);
    dev_free(d_out_, s_);
    dev_free(d_hist_, s_);
    dev_free(d_bits_, s_);
    dev_free(d_range_, s_);
  }

  qoz_status init() {
    if (dev_alloc((void**)&d_orig_, sizeof(int) * sm_.origins.size(), s_) != cudaSuccess)
      return fail(QOZ_ENOMEM, "tuner allocation");
    cudaMemcpyAsync(d_orig_, sm_.origins.data(), sizeof(int) * sm_.origins.size(),
                    cudaMemcpyHostToDevice, s_);
    // full-resolution blocks arrive by one bulk tensor copy when the field's
    // rows start on 16-byte boundaries: the copy starts at the boundary at or
    // below each block's x origin, so rows hold up to 3 more values
    memset(&tmap_, 0, sizeof(tmap_));
    tma_pitch_ = (sm_.bd[2] + 3 + 3) & ~3;
    const long long st1 = r_.n[2], st0 = r_.n[1] * r_.n[2];
    if ((reinterpret_cast<uintptr_t>(x_) & 15) == 0 && st1 % 4 == 0 && st0 % 4 == 0 &&
        tma_pitch_ <= 256 && sm_.bd[1] <= 256 && sm_.bd[0] <= 256) {
      const unsigned long long d[3] = {(unsigned long long)r_.n[2], (unsigned long long)r_.n[1],
                                       (unsigned long long)r_.n[0]};
      const unsigned long long st[2] = {4ull * st1, 4ull * st0};
      const unsigned bx[3] = {(unsigned)tma_pitch_, (unsigned)sm_.bd[1], (unsigned)sm_.bd[0]};
      tma_ok_ = encode_tensor_map_3d(&tmap_, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, x_, d, st, bx);
    }
    return QOZ_OK;
  }

  // Value range of the field on the device (per-CTA partials, then the
  // bound table with eb = rel, so its e is rel * range): the trial bounds and
  // the SSIM constants follow from it without a host round trip.  Also holds
  // the Algorithm 1 control block and e0.
  qoz_status start_range(double rel) {
    const int np = range_partial_blocks();
    if (!d_range_ && dev_alloc(&d_range_, kRangeOff + np * (sizeof(float) * 2 + 8) + 64, s_) !=
                         cudaSuccess)
      return fail(QOZ_ENOMEM, "tuner allocation");
    char* base = static_cast<char*>(d_range_);
    d_bt_ = reinterpret_cast<BoundTable*>(base);
    d_ctl_ = reinterpret_cast<Alg1Ctl*>(base + kCtlOff);
    d_e0_ = reinterpret_cast<double*>(base + kE0Off);
    float* pmin = reinterpret_cast<float*>(base + kRangeOff);
    float* pmax = pmin + np;
    unsigned long long* pcnt =
        reinterpret_cast<unsigned long long*>(((uintptr_t)(pmax + np) + 15) & ~(uintptr_t)15);
    cudaError_t e = launch_check(launch_range(x_, r_.N, pmin, pmax, pcnt, s_));
    if (e == cudaSuccess)
      e = launch_check(launch_bound_table(pmin, pmax, pcnt, np, 1, rel, 1.0, 1.0, 1, d_bt_, s_));
    if (e != cudaSuccess) return cuda_fail(e, "tuner value range");
    return QOZ_OK;
  }

  // Algorithm 1 over levels Ls..1 on the device, enqueued only: the
  // top-level candidates get their bounds from the device value range
  // (alg1_setup_kernel), each level's trials are followed by
  // alg1_select_kernel (choice + next level's candidates) and the last one
  // builds the (alpha, beta) candidates of `ab` in d_cands_.  The choices
  // are read back by collect().  Needs start_range() first.
  qoz_status alg1_enqueue(const TrialCand& base, const std::vector<std::pair<int, int>>& cl,
                          int ndims, const E0Spec& sp, const AbSpec& ab) {
    const int nc = (int)cl.size();
    if (nc == 0 || nc > kAlg1MaxCand) return fail(QOZ_EINVAL, "1..16 Algorithm 1 candidates");
    if (!d_range_) return fail(QOZ_EINVAL, "tuner value range not started");
    const int nab = ab.n_pairs * ab.n_scales;
    qoz_status st = ensure(nc > nab ? nc : nab);
    if (st != QOZ_OK) return st;
    Alg1Ctl h;
    memset(&h, 0, sizeof(h));
    for (int c = 0; c < nc; ++c) {
      h.ci[c] = (unsigned char)cl[c].first;
      h.co[c] = (unsigned char)cl[c].second;
    }
    std::vector<TrialCand> top;
    for (int c = 0; c < nc; ++c) {
      TrialCand t = base;
      t.interp[sm_.Ls - 1] = h.ci[c];
      set_axes(&t, sm_.Ls, ndims, h.co[c]);
      top.push_back(t);
    }
    cudaError_t e = cudaMemcpyAsync(d_ctl_, &h, sizeof(h), cudaMemcpyHostToDevice, s_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_cands_, top.data(), sizeof(TrialCand) * nc, cudaMemcpyHostToDevice,
                          s_);
    if (e == cudaSuccess) {
      alg1_setup_kernel<<<1, 32, 0, s_>>>(d_cands_, nc, d_bt_, sp, sm_.Ls, d_e0_);
      note_launch(1);
      e = launch_check(cudaGetLastError());
    }
    for (int l = sm_.Ls; l >= 1 && e == cudaSuccess; --l) {
      if ((st = launch(nc, l, l, false)) != QOZ_OK) return st;
      alg1_select_kernel<<<1, 32 * nc, 0, s_>>>(d_out_, nc, sm_.nb, l, sm_.Ls, base, ndims,
                                                 d_ctl_, d_cands_, ab, d_e0_);
      note_launch(1);
      e = launch_check(cudaGetLastError());
    }
    if (e != cudaSuccess) return cuda_fail(e, "Algorithm 1");
    return QOZ_OK;
  }

  qoz_status ensure(int nc) {
    if (nc > cap_c_) {
      dev_free(d_cands_, s_);
      dev_free(d_out_, s_);
      dev_free(d_hist_, s_);
      dev_free(d_bits_, s_);
      cap_c_ = nc;
      if (dev_alloc((void**)&d_cands_, sizeof(TrialCand) * nc, s_) != cudaSuccess ||
          dev_alloc((void**)&d_out_, sizeof(double) * kOutStride * nc * sm_.nb, s_) !=
              cudaSuccess ||
          dev_alloc((void**)&d_hist_, sizeof(unsigned) * 65536 * (size_t)nc, s_) != cudaSuccess ||
          dev_alloc((void**)&d_bits_, (sizeof(unsigned long long) + sizeof(int)) * nc, s_) !=
              cudaSuccess)
        return fail(QOZ_ENOMEM, "tuner allocation");
    }
    return QOZ_OK;
  }

  // Launches the trials of the nc candidates already in d_cands_ (and, with
  // `full`, their prefix-code costs); no read-back.
  qoz_status launch(int nc, int stop_level, int score_level, bool full) {
    cudaError_t e = cudaSuccess;
    if (full) e = cudaMemsetAsync(d_hist_, 0, sizeof(unsigned) * 65536 * (size_t)nc, s_);
    TrialArgs a;
    memset(&a, 0, sizeof(a));
    a.x = x_;
    a.st0 = r_.n[1] * r_.n[2];
    a.st1 = r_.n[2];
    a.origins = d_orig_;
    a.nblocks = sm_.nb;
    for (int p = 0; p < 3; ++p) a.bd[p] = sm_.bd[p];
    a.Ls = sm_.Ls;
    a.stop_level = stop_level;
    a.score_level = score_level;
    a.cands = d_cands_;
    a.hist = full ? d_hist_ : nullptr;
    a.out = d_out_;
    a.metrics = full ? 1 : 0;
    a.ssim_win = (full && metric_ == QOZ_METRIC_SSIM) ? win_ : 0;
    a.ssim_step = step_;
    a.ac = (full && metric_ == QOZ_METRIC_AC) ? 1 : 0;
    a.is3d = r_.ndims == 3;
    a.c1 = (0.01 * vr_) * (0.01 * vr_);
    a.c2 = (0.03 * vr_) * (0.03 * vr_);
    a.bt = d_bt_;
    const int f = 1 << (stop_level - 1);
    const int m2 = (sm_.bd[2] - 1) / f + 1;
    const long long rows = (long long)((sm_.bd[0] - 1) / f + 1) * ((sm_.bd[1] - 1) / f + 1);
    auto smem_for = [&](int pitch) {
      return (size_t)128 + ((sizeof(float) * rows * pitch + 15) & ~size_t(15)) +
             (full ? sizeof(unsigned) * kTHistWin : 0);
    };
    a.use_tma = (tma_ok_ && f == 1 && smem_for(tma_pitch_) <= 220 * 1024) ? 1 : 0;
    a.pitch = a.use_tma ? tma_pitch_ : m2;
    const long long npb = rows * a.pitch;
    const size_t smem = smem_for(a.pitch);
    if (smem > 220 * 1024)
      return fail(QOZ_EUNSUPPORTED, "sample block too large (%lld points)", npb);
    const bool coarse = stop_level > 1;
    const void* fn = coarse ? (const void*)trial_kernel<kTrialThreadsCoarse>
                            : (const void*)trial_kernel<kTrialThreads>;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      ProfScope ps(QOZ_STAGE_TUNE, s_);
      const unsigned grid = (unsigned)(nc * sm_.nb);
      if (coarse)
        trial_kernel<kTrialThreadsCoarse><<<grid, kTrialThreadsCoarse, smem, s_>>>(a, tmap_);
      else
        trial_kernel<kTrialThreads><<<grid, kTrialThreads, smem, s_>>>(a, tmap_);
      note_launch(1);
      e = launch_check(cudaGetLastError());
    }
    trials_ += nc;
    unsigned long long* d_bits = reinterpret_cast<unsigned long long*>(d_bits_);
    int* d_flag = reinterpret_cast<int*>(d_bits + nc);
    if (e == cudaSuccess && full) {
      static unsigned long long attr_done = 0;
      e = ensure_smem_attr((const void*)huffman_cost_kernel, &attr_done, sizeof(HuffCostSmem));
      if (e == cudaSuccess)
        huffman_cost_kernel<<<nc, kHuffThreads, sizeof(HuffCostSmem), s_>>>(d_hist_, d_bits,
                                                                            d_flag);
      note_launch(1);
      e = launch_check(cudaGetLastError());
    }
    if (e != cudaSuccess) return cuda_fail(e, "tuner trial");
    return QOZ_OK;
  }

  // Runs the given candidates; fills per-candidate results.  hist/metrics
  // only when stop_level == 1.
  qoz_status run(const std::vector<TrialCand>& cands, int stop_level, int score_level,
                 bool full, std::vector<TrialResult>* res) {
    const int nc = (int)cands.size();
    if (nc == 0) return QOZ_OK;
    qoz_status st = ensure(nc);
    if (st != QOZ_OK) return st;
    cudaError_t e = cudaMemcpyAsync(d_cands_, cands.data(), sizeof(TrialCand) * nc,
                                    cudaMemcpyHostToDevice, s_);
    if (e != cudaSuccess) return cuda_fail(e, "tuner trial");
    if ((st = launch(nc, stop_level, score_level, full)) != QOZ_OK) return st;
    return collect(nc, full, res, nullptr, nullptr);
  }

  // Reads back the results of the last launch (nc candidates), and, when
  // asked, the Algorithm 1 control block and the device value range (which
  // then sets the range used for PSNR), with one synchronisation through a
  // pinned staging buffer; folds the blocks of each candidate.
  qoz_status collect(int nc, bool full, std::vector<TrialResult>* res, Alg1Ctl* ctl,
                     BoundTable* bt) {
    unsigned long long* d_bits = reinterpret_cast<unsigned long long*>(d_bits_);
    int* d_flag = reinterpret_cast<int*>(d_bits + nc);
    const size_t n_out = (size_t)kOutStride * nc * sm_.nb;
    auto up16 = [](size_t v) { return (v + 15) & ~size_t(15); };
    const size_t o_bits = up16(sizeof(double) * n_out);
    const size_t o_flag = o_bits + up16(sizeof(unsigned long long) * nc);
    const size_t o_ctl = o_flag + up16(sizeof(int) * nc);
    const size_t o_bt = o_ctl + up16(sizeof(Alg1Ctl));
    char* hs = static_cast<char*>(pinned_stage(o_bt + sizeof(BoundTable)));
    if (!hs) return fail(QOZ_ENOMEM, "pinned staging buffer");
    const double* out = reinterpret_cast<const double*>(hs);
    unsigned long long* hbits = reinterpret_cast<unsigned long long*>(hs + o_bits);
    int* hflag = reinterpret_cast<int*>(hs + o_flag);
    cudaError_t e =
        cudaMemcpyAsync(hs, d_out_, sizeof(double) * n_out, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess && full)
      e = cudaMemcpyAsync(hbits, d_bits, sizeof(unsigned long long) * nc, cudaMemcpyDeviceToHost,
                          s_);
    if (e == cudaSuccess && full)
      e = cudaMemcpyAsync(hflag, d_flag, sizeof(int) * nc, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess && ctl)
      e = cudaMemcpyAsync(hs + o_ctl, d_ctl_, sizeof(Alg1Ctl), cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess && bt)
      e = cudaMemcpyAsync(hs + o_bt, d_bt_, sizeof(BoundTable), cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) return cuda_fail(e, "tuner trial");
    if (ctl) memcpy(ctl, hs + o_ctl, sizeof(Alg1Ctl));
    if (bt) {
      memcpy(bt, hs + o_bt, sizeof(BoundTable));
      vr_ = bt->vrange;
    }
    std::vector<unsigned long long> bits(nc, 0ull);
    for (int c = 0; c < nc && full; ++c) bits[c] = hbits[c];
    // histograms with too many distinct codes for the device sort: host
    std::vector<unsigned> hist;
    for (int c = 0; c < nc && full; ++c) {
      if (!hflag[c]) continue;
      hist.resize(65536);
      e = cudaMemcpyAsync(hist.data(), d_hist_ + (size_t)c * 65536, sizeof(unsigned) * 65536,
                          cudaMemcpyDeviceToHost, s_);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
      if (e != cudaSuccess) return cuda_fail(e, "tuner histogram");
      bits[c] = huffman_bits_u32(hist.data(), 65536);
    }
    for (size_t i = 7; i < n_out; i += kOutStride)
      if (out[i] != 0.0) return fail(QOZ_ETIMEOUT, "a sample block's bulk copy did not complete");
    res->assign(nc, TrialResult{0, 0, 0});
    for (int c = 0; c < nc; ++c) {
      double l1 = 0, l1n = 0, unp = 0, sse = 0, mx = 0, ss = 0, sn = 0;
      for (int b = 0; b < sm_.nb; ++b) {
        const double* o = &out[((size_t)c * sm_.nb + b) * kOutStride];
        l1 += o[0];
        l1n += o[1];
        unp += o[2];
        sse += o[3];
        if (o[4] != o[4] || o[4] > mx) mx = o[4];
        ss += o[5];
        sn += o[6];
      }
      TrialResult& t = (*res)[c];
      t.l1_mean = l1n > 0 ? l1 / l1n : 0.0;
      if (full) {
        const double nbits = (double)bits[c] + 32.0 * unp + 32.0 * (double)sm_.anchors;
        t.B = nbits / (double)sm_.npts;
        if (metric_ == QOZ_METRIC_PSNR) {
          const double mse = sse / (double)sm_.npts;
          t.M = mse == 0.0 ? INFINITY : 20.0 * std::log10(vr_ / std::sqrt(mse));
        } else if (metric_ == QOZ_METRIC_SSIM) {
          t.M = sn > 0 ? ss / sn : NAN;
        } else if (metric_ == QOZ_METRIC_AC) {
          t.M = -pooled_ac(&out[(size_t)c * sm_.nb * kOutStride]);
        } else {
          t.M = -mx;
        }
      }
    }
    return QOZ_OK;
  }

  // Eq. (ac) at lag 1 pooled over the blocks of one candidate: pairs inside
  // each block (in its row-major order), mean and variance over all sampled
  // points; 0 when the variance vanishes (below 1e-6 of the mean square).
  double pooled_ac(const double* o) const {
    double s1 = 0.0, s2 = 0.0, sk = 0.0, hd = 0.0, tl = 0.0;
    for (int b = 0; b < sm_.nb; ++b) {
      const double* q = o + (size_t)b * kOutStride;
      s1 += q[8];
      s2 += q[9];
      sk += q[10];
      hd += q[8] - q[12];
      tl += q[8] - q[11];
    }
    const double n = (double)sm_.npts, P = (double)(sm_.npts - sm_.nb);
    if (!(n > 0.0) || !(P > 0.0)) return 0.0;
    const double mu = s1 / n, ms = s2 / n, var = ms - mu * mu;
    if (!(var > 1e-6 * ms)) return 0.0;
    return ((sk - mu * (hd + tl)) / P + mu * mu) / var;
  }

  int trials() const { return trials_; }

 private:
  const float* x_;
  const Resolved& r_;
  const Sampling& sm_;
  cudaStream_t s_;
  int metric_, win_, step_;
  double vr_;
  int* d_orig_ = nullptr;
  TrialCand* d_cands_ = nullptr;
  double* d_out_ = nullptr;
  unsigned* d_hist_ = nullptr;
  void* d_bits_ = nullptr;  // per candidate: prefix-code bits (u64), then host-fallback flags (int)
  // device value range scratch: bound table, Algorithm 1 control, e0, then
  // the range partials
  static constexpr size_t kCtlOff = 256, kE0Off = 512, kRangeOff = 1024;
  void* d_range_ = nullptr;
  BoundTable* d_bt_ = nullptr;
  Alg1Ctl* d_ctl_ = nullptr;
  double* d_e0_ = nullptr;
  CUtensorMap tmap_;        // the field, boxes of one full-resolution sample block
  bool tma_ok_ = false;
  int tma_pitch_ = 0;
  int cap_c_ = 0;
  int trials_ = 0;
};

// Table I: 0 keeps the incumbent I, 1 takes II, -1 asks for II at
// *scale * e (0.8 in case 3, 1.2 in case 4); pass b2p = NaN first.
int table1(double b1, double m1, double b2, double m2, double b2p, double m2p, double* scale) {
  if (b1 <= b2 && m1 >= m2) return 0;
  if (b1 >= b2 && m1 <= m2) return 1;
  const bool case3 = b1 > b2 && m1 > m2;
  if (std::isnan(b2p)) {
    *scale = case3 ? 0.8 : 1.2;
    return -1;
  }
  double m_line;
  if (b2p == b2)
    m_line = m2 > m2p ? m2 : m2p;
  else
    m_line = m2 + (m2p - m2) * (b1 - b2) / (b2p - b2);
  return m1 >= m_line ? 0 : 1;
}

}  // namespace

// Tuner options with the paper's defaults filled in (Sec. 7.1.4, Sec. 6.3.1)
// and checked.
qoz_status resolve_tune_opts(const qoz_shape& shape, const Resolved& r,
                             const qoz_tune_opts* opts_in, qoz_tune_opts* out) {
  qoz_tune_opts o;
  memset(&o, 0, sizeof(o));
  if (opts_in) o = *opts_in;
  const int d = r.ndims;
  if (o.block == 0) o.block = d == 3 ? 16 : 64;
  if (!(o.rate > 0.0)) o.rate = d == 3 ? 0.005 : 0.01;
  if (o.n_orders == 0) o.n_orders = 2;
  if (o.n_alpha == 0) {
    const double al[5] = {1.0, 1.25, 1.5, 1.75, 2.0};
    o.n_alpha = 5;
    for (int i = 0; i < 5; ++i) o.alphas[i] = al[i];
  }
  if (o.n_beta == 0) {
    const double be[4] = {1.5, 2.0, 3.0, 4.0};
    o.n_beta = 4;
    for (int i = 0; i < 4; ++i) o.betas[i] = be[i];
  }
  if (o.ssim_win == 0) o.ssim_win = 7;
  if (o.ssim_step == 0) o.ssim_step = 2;
  if (o.anchor_stride == 0) o.anchor_stride = d == 3 ? 32 : 64;
  if (o.block < 2 || (o.block & (o.block - 1)) != 0)
    return fail(QOZ_EINVAL, "block must be a power of two >= 2");
  if (o.n_alpha < 1 || o.n_alpha > 8 || o.n_beta < 1 || o.n_beta > 8)
    return fail(QOZ_EINVAL, "1..8 alpha and beta candidates");
  for (int i = 0; i < o.n_alpha; ++i)
    if (!(o.alphas[i] >= 1.0)) return fail(QOZ_EINVAL, "alpha < 1");
  for (int i = 0; i < o.n_beta; ++i)
    if (!(o.betas[i] >= 1.0)) return fail(QOZ_EINVAL, "beta < 1");
  {
    qoz_params chk;
    memset(&chk, 0, sizeof(chk));
    chk.anchor_stride = o.anchor_stride;
    chk.alpha = chk.beta = 1.0;
    Resolved rr;
    if (resolve(shape, &chk, &rr) != QOZ_OK) return fail(QOZ_EINVAL, "invalid anchor stride");
  }
  *out = o;
  return QOZ_OK;
}

// A sampled (bound, bit rate, metric) point of the target mode.
struct TargetPoint {
  double e, B, M;
};

// Secant on (log e, M) for one setting from the last two points of *pts, at
// most four more trials (bound capped at e_user, floored at e0 / 16); the
// pick is the largest bound whose sampled metric meets the target, else the
// smallest bound tried (capped at e_user).
qoz_status target_secant(Tuner& T, const TrialCand& setting, double alpha, double beta, int Ls,
                         double target, double e0, double e_user,
                         std::vector<TargetPoint>* pts, TargetPoint* pick_out) {
  for (int it = 0; it < 4; ++it) {
    const TargetPoint pa = (*pts)[pts->size() - 2];
    const TargetPoint pb = (*pts)[pts->size() - 1];
    if (pa.M == pb.M) break;
    const double le =
        std::log(pb.e) + (target - pb.M) * (std::log(pa.e) - std::log(pb.e)) / (pa.M - pb.M);
    double en = std::exp(le);
    if (en > e_user) en = e_user;
    if (en < e0 / 16.0) en = e0 / 16.0;
    if (en == pb.e) break;
    TrialCand c = setting;
    fill_bounds(&c, en, alpha, beta, Ls);
    std::vector<TrialResult> r1;
    const qoz_status st = T.run({c}, 1, 0, true, &r1);
    if (st != QOZ_OK) return st;
    pts->push_back({en, r1[0].B, r1[0].M});
  }
  int pick = -1;
  for (size_t k = 0; k < pts->size(); ++k)
    if ((*pts)[k].M >= target && (*pts)[k].e <= e_user &&
        (pick < 0 || (*pts)[k].e > (*pts)[pick].e))
      pick = (int)k;
  if (pick < 0) {
    pick = 0;
    for (size_t k = 1; k < pts->size(); ++k)
      if ((*pts)[k].e < (*pts)[pick].e) pick = (int)k;
  }
  *pick_out = (*pts)[pick];
  if (pick_out->e > e_user) pick_out->e = e_user;
  return QOZ_OK;
}

qoz_status tune_impl(const float* d_field, const qoz_shape& shape, double rel_eb, int metric,
                     double target, const qoz_tune_opts* opts_in, cudaStream_t s,
                     qoz_tune_report* out) {
  if (!d_field || !out) return fail(QOZ_EINVAL, "NULL argument");
  if (!(rel_eb > 0.0 && std::isfinite(rel_eb))) return fail(QOZ_EINVAL, "rel_eb must be > 0");
  if (metric < QOZ_METRIC_MAXERR || metric > QOZ_METRIC_AC)
    return fail(QOZ_EINVAL, "unknown metric %d", metric);
  const bool target_mode = !std::isnan(target);
  if (target_mode && (metric == QOZ_METRIC_MAXERR || metric == QOZ_METRIC_AC))
    return fail(QOZ_EINVAL, "a target needs the PSNR or SSIM metric");
  Resolved r;
  qoz_status st = resolve(shape, nullptr, &r);
  if (st != QOZ_OK) return st;
  qoz_tune_opts o;
  if ((st = resolve_tune_opts(shape, r, opts_in, &o)) != QOZ_OK) return st;
  const int d = r.ndims;
  int L = 0;
  while ((1 << L) < o.anchor_stride) ++L;

  // the value range stays on the device until the single read-back below:
  // Algorithm 1 and the (alpha, beta) trials take their bounds from it there
  Sampling sm = sample_blocks(r, o.block, o.rate, o.anchor_stride);
  Tuner T(d_field, r, sm, s, metric, o.ssim_win, o.ssim_step, NAN);
  if ((st = T.init()) != QOZ_OK) return st;
  if ((st = T.start_range(rel_eb)) != QOZ_OK) return st;
  E0Spec sp;
  sp.psnr_target = target_mode && metric == QOZ_METRIC_PSNR;
  sp.sqrt3 = std::sqrt(3.0);
  sp.p10 = sp.psnr_target ? std::pow(10.0, -target / 20.0) : 0.0;

  // candidate interpolators: linear before cubic, then the orders
  std::vector<std::pair<int, int>> cands;
  {
    std::vector<int> orders;
    if (d == 2)
      orders = {0, 1};
    else if (o.n_orders >= 6)
      orders = {0, 1, 2, 3, 4, 5};
    else
      orders = {0, 5};
    for (int t = 0; t < 2; ++t)
      for (int od : orders) cands.push_back({t, od});
  }

  memset(out, 0, sizeof(*out));
  TrialCand base;  // bounds are filled on the device
  memset(&base, 0, sizeof(base));
  for (int l = 1; l <= kMaxLevels; ++l) set_axes(&base, l, d, 0);
  unsigned char ch_interp[kMaxLevels] = {0}, ch_order[kMaxLevels] = {0};

  // ---- Algorithm 1, from the top sampled level down (choices on the
  // device), then the alpha / beta candidates at e0 and, batched, at 0.8 e0
  // and 1.2 e0 (built on the device from the choices); one read-back
  const int nab = o.n_alpha * o.n_beta;
  const bool need_scaled = metric != QOZ_METRIC_MAXERR;
  AbSpec ab;
  memset(&ab, 0, sizeof(ab));
  ab.n_alpha = o.n_alpha;
  ab.n_beta = o.n_beta;
  ab.n_scales = need_scaled ? 3 : 1;
  for (int i = 0; i < o.n_alpha; ++i) ab.alphas[i] = o.alphas[i];
  for (int i = 0; i < o.n_beta; ++i) ab.betas[i] = o.betas[i];
  ab.scales[0] = 1.0;
  ab.scales[1] = 0.8;
  ab.scales[2] = 1.2;
  // distinct settings: every (1, beta) after the first repeats its trial
  std::vector<int> pair_of(nab);
  int first_unit = -1;
  ab.n_pairs = 0;
  for (int k = 0; k < nab; ++k) {
    const int ai = k / o.n_beta, bi = k % o.n_beta;
    if (o.alphas[ai] == 1.0 && first_unit >= 0) {
      pair_of[k] = first_unit;
      continue;
    }
    if (o.alphas[ai] == 1.0) first_unit = ab.n_pairs;
    ab.pa[ab.n_pairs] = (unsigned char)ai;
    ab.pb[ab.n_pairs] = (unsigned char)bi;
    pair_of[k] = ab.n_pairs++;
  }
  std::vector<TrialResult> ures, res;
  Alg1Ctl ctl;
  BoundTable bt;
  if ((st = T.alg1_enqueue(base, cands, d, sp, ab)) != QOZ_OK) return st;
  if ((st = T.launch(ab.n_scales * ab.n_pairs, 1, 0, true)) != QOZ_OK) return st;
  if ((st = T.collect(ab.n_scales * ab.n_pairs, true, &ures, &ctl, &bt)) != QOZ_OK) return st;
  res.resize((size_t)ab.n_scales * nab);
  for (int si = 0; si < ab.n_scales; ++si)
    for (int k = 0; k < nab; ++k)
      res[(size_t)si * nab + k] = ures[(size_t)si * ab.n_pairs + pair_of[k]];
  for (int l = 1; l <= sm.Ls; ++l) {
    ch_interp[l - 1] = ctl.chi[l - 1];
    ch_order[l - 1] = ctl.cho[l - 1];
    out->alg1_score[l - 1] = ctl.score[l - 1];
  }
  const float vmin = bt.vmin, vmax = bt.vmax;
  const double vr = (double)vmax - (double)vmin;
  const double e_user = rel_eb * vr;
  // the same e0 as the device's (the same operations on the same range)
  double e0 = e_user;
  if (sp.psnr_target) {
    e0 = vr * sp.sqrt3 * sp.p10;
    if (e0 > e_user) e0 = e_user;
  }
  qoz_params fp;
  memset(&fp, 0, sizeof(fp));
  fp.anchor_stride = o.anchor_stride;
  for (int l = 1; l <= L; ++l) {
    const int src = l <= sm.Ls ? l : sm.Ls;
    fp.interp[l - 1] = ch_interp[src - 1];
    fp.order[l - 1] = ch_order[src - 1];
  }

  // ---- alpha / beta selection (Table I) over the batched results
  TrialCand chosen = base;
  for (int l = 1; l <= sm.Ls; ++l) {
    chosen.interp[l - 1] = ch_interp[l - 1];
    set_axes(&chosen, l, d, ch_order[l - 1]);
  }
  auto at = [&](int si, int k) -> const TrialResult& { return res[(size_t)si * nab + k]; };

  int best_k = 0;
  double best_B = 0, best_M = 0, best_score = INFINITY, best_e = e0;
  bool have = false;
  std::vector<TargetPoint> pts;
  for (int k = 0; k < nab; ++k) {
    const TrialResult& t = at(0, k);
    if (!target_mode) {
      bool replace;
      if (!have) {
        replace = true;
      } else if (metric == QOZ_METRIC_MAXERR) {
        replace = t.B < best_B;
      } else {
        double scale = 0.0;
        int dec = table1(best_B, best_M, t.B, t.M, NAN, NAN, &scale);
        if (dec < 0) {
          const TrialResult& t2 = at(scale < 1.0 ? 1 : 2, k);
          dec = table1(best_B, best_M, t.B, t.M, t2.B, t2.M, &scale);
        }
        replace = dec == 1;
      }
      if (replace) {
        have = true;
        best_k = k;
        best_B = t.B;
        best_M = t.M;
      }
    } else {
      const double sc = t.M >= target ? 1.2 : 0.8;
      const TrialResult& t2 = at(sc > 1.0 ? 2 : 1, k);
      double Bstar;
      if (t2.M == t.M)
        Bstar = t.M >= target ? (t.B < t2.B ? t.B : t2.B) : INFINITY;
      else
        Bstar = t.B + (target - t.M) * (t2.B - t.B) / (t2.M - t.M);
      if (!have || Bstar < best_score) {
        have = true;
        best_score = Bstar;
        best_k = k;
        pts = {{e0, t.B, t.M}, {sc * e0, t2.B, t2.M}};
      }
    }
  }
  fp.alpha = o.alphas[best_k / o.n_beta];
  fp.beta = o.betas[best_k % o.n_beta];

  if (target_mode) {
    TargetPoint pk;
    if ((st = target_secant(T, chosen, fp.alpha, fp.beta, sm.Ls, target, e0, e_user, &pts, &pk)) !=
        QOZ_OK)
      return st;
    best_e = pk.e;
    best_B = pk.B;
    best_M = pk.M;
  } else {
    best_e = e_user;
  }

  out->params = fp;
  out->abs_eb = best_e;
  out->vmin = vmin;
  out->vmax = vmax;
  out->B = best_B;
  out->M = best_M;
  out->n_trials = T.trials();
  out->n_blocks = sm.nb;
  out->n_sampled_points = sm.npts;
  return QOZ_OK;
}

// Sampled verification of one given setting (Sec. 6.1 trials): in the
// fixed-bound mode one trial at the bound; with a target, trials at e0 and
// at 0.8 e0 / 1.2 e0, then the target mode's secant on the bound.
qoz_status verify_impl(const float* d_field, const qoz_shape& shape, double rel_eb, int metric,
                       double target, const qoz_tune_opts* opts_in, const qoz_params* p_in,
                       cudaStream_t s, qoz_tune_report* out) {
  if (!d_field || !out || !p_in) return fail(QOZ_EINVAL, "NULL argument");
  if (!(rel_eb > 0.0 && std::isfinite(rel_eb))) return fail(QOZ_EINVAL, "rel_eb must be > 0");
  if (metric < QOZ_METRIC_MAXERR || metric > QOZ_METRIC_AC)
    return fail(QOZ_EINVAL, "unknown metric %d", metric);
  const bool target_mode = !std::isnan(target);
  if (target_mode && (metric == QOZ_METRIC_MAXERR || metric == QOZ_METRIC_AC))
    return fail(QOZ_EINVAL, "a target needs the PSNR or SSIM metric");
  Resolved r;
  qoz_status st = resolve(shape, p_in, &r);
  if (st != QOZ_OK) return st;
  qoz_tune_opts o;
  if ((st = resolve_tune_opts(shape, r, opts_in, &o)) != QOZ_OK) return st;
  o.anchor_stride = r.p.anchor_stride;
  const int d = r.ndims;
  float vmin, vmax;
  int64_t cnt;
  st = qoz_value_range(d_field, r.N, &vmin, &vmax, &cnt, s);
  if (st != QOZ_OK) return st;
  const double vr = (double)vmax - (double)vmin;
  const double e_user = rel_eb * vr;
  Sampling sm = sample_blocks(r, o.block, o.rate, o.anchor_stride);
  Tuner T(d_field, r, sm, s, metric, o.ssim_win, o.ssim_step, vr);
  if ((st = T.init()) != QOZ_OK) return st;
  TrialCand c;
  memset(&c, 0, sizeof(c));
  for (int l = 1; l <= kMaxLevels; ++l) set_axes(&c, l, d, 0);
  for (int l = 1; l <= sm.Ls; ++l) {
    c.interp[l - 1] = r.p.interp[l - 1];
    set_axes(&c, l, d, r.p.order[l - 1]);
  }
  const double alpha = r.p.alpha, beta = r.p.beta;
  double e0 = e_user;
  if (target_mode && metric == QOZ_METRIC_PSNR) {
    e0 = vr * std::sqrt(3.0) * std::pow(10.0, -target / 20.0);
    if (e0 > e_user) e0 = e_user;
  }
  memset(out, 0, sizeof(*out));
  std::vector<TrialResult> res;
  if (!target_mode) {
    TrialCand t = c;
    fill_bounds(&t, e_user, alpha, beta, sm.Ls);
    if ((st = T.run({t}, 1, 0, true, &res)) != QOZ_OK) return st;
    out->abs_eb = e_user;
    out->B = res[0].B;
    out->M = res[0].M;
  } else {
    std::vector<TrialCand> tc;
    const double scales[3] = {1.0, 0.8, 1.2};
    for (double sc : scales) {
      TrialCand t = c;
      fill_bounds(&t, sc * e0, alpha, beta, sm.Ls);
      tc.push_back(t);
    }
    if ((st = T.run(tc, 1, 0, true, &res)) != QOZ_OK) return st;
    const TrialResult& t1 = res[0];
    const double sc = t1.M >= target ? 1.2 : 0.8;
    const TrialResult& t2 = res[sc > 1.0 ? 2 : 1];
    std::vector<TargetPoint> pts = {{e0, t1.B, t1.M}, {sc * e0, t2.B, t2.M}};
    TargetPoint pk;
    if ((st = target_secant(T, c, alpha, beta, sm.Ls, target, e0, e_user, &pts, &pk)) != QOZ_OK)
      return st;
    out->abs_eb = pk.e;
    out->B = pk.B;
    out->M = pk.M;
  }
  out->params = r.p;
  out->vmin = vmin;
  out->vmax = vmax;
  out->n_trials = T.trials();
  out->n_blocks = sm.nb;
  out->n_sampled_points = sm.npts;
  return QOZ_OK;
}

}  // namespace qoz

extern "C" qoz_status qoz_tune(const float* d_field, qoz_shape shape, double rel_eb,
                               qoz_metric metric, double target, const qoz_tune_opts* opts,
                               void* stream, qoz_tune_report* out) {
  return qoz::tune_impl(d_field, shape, rel_eb, (int)metric, target, opts, (cudaStream_t)stream,
                        out);
}

extern "C" qoz_status qoz_tune_verify(const float* d_field, qoz_shape shape, double rel_eb,
                                      qoz_metric metric, double target,
                                      const qoz_tune_opts* opts, const qoz_params* params,
                                      void* stream, qoz_tune_report* out) {
  return qoz::verify_impl(d_field, shape, rel_eb, (int)metric, target, opts, params,
                          (cudaStream_t)stream, out);
}

#ifdef QOZ_DEBUG_BOUNDS
namespace qoz {
// This translation unit's record of failed index checks (bounds-checking build).
unsigned long long bounds_take_tune(bool reset) { return bounds_take(reset); }
}  // namespace qoz
#endif
