// Learned tuner: features of the sampled blocks, a 64-128-128-16 ReLU
// network trained on the GPU (forward, backward, Adam), and the tuning call
// that replaces the sampled trials by one network evaluation.
//
// The paper leaves better selection policies and hyper-parameter
// auto-tuning to future work (its concluding section); the features and the
// network are this library's own definitions:
//
// Features, over the blocks of the sampled tuner (Sec. 6.1), each block on
// its own, e = rel_eb * vrange (1 if 0), L(v) = log2(1 + v / e):
//   [0] log10(rel_eb)  [1] log10(vrange / sigma) of the sampled values
//   [2] ndims / 3      [3] log2(N) / 30
//   [4..6] L(mean |first difference|) per axis, [7..9] the same for second
//   differences (2-D: third slot 0);
//   [10..33] fractions in 24 bins of floor(log2(|gradient| / e)) + 12;
//   [34..57] the same for |x - Lorenzo prediction| / e;
//   [58..60] / [61..63] L(mean |x - linear| / |x - cubic| interpolation) at
//   half-strides 1, 2, 4 along every axis (Sec. 5.1 stencils, targets with
//   all four neighbours in the block).
// Differences, predictions, products and bin arguments are binary32
// operations in one fixed order (so the integer bins, decided by frexp,
// are the same on every implementation); 1/e and 1/e^2 are rounded to
// binary32 once; sums over points are compensated binary32 per thread and
// double across threads.  The gradient bin is floor(floor(log2 t) / 2) + 12
// with t = |gradient|^2 / e^2 (no square root).
//
// Network: z = (f - mean) / std; h1 = relu(W1 z + b1); h2 = relu(W2 h1 + b2);
// o = W3 h2 + b3; heads o[0:2] interpolator, o[2:8] dimension order,
// o[8:13] alpha, o[13:16] beta; loss = mean over samples of the summed
// per-head softmax cross-entropies.  Training kernels are deterministic:
// per-CTA gradient partials are summed in a fixed order before Adam
// (Kingma and Ba, bias-corrected moments).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"

using namespace qoz;

namespace {

constexpr int NF = 64, NH = 128, NO = 16;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH,
              NPARAM = OFF_B3 + NO;
static_assert(NPARAM == QOZ_MLP_PARAMS, "packed parameter count");
__constant__ int kHeadOff[4] = {0, 2, 8, 13};
__constant__ int kHeadLen[4] = {2, 6, 5, 3};

// ------------------------------------------------------------- features
constexpr int kFeatThreads = 256;
constexpr int kNSum = 14;            // s1, s2, d1[3], d2[3], lin[3], cub[3]
constexpr int kNCnt = 12 + 48;       // n, n1[3], n2[3], nint[3], ng, nl, gh[24], lh[24]

struct FeatPart {
  double sum[kNSum];
  unsigned long long cnt[kNCnt];
};

struct FeatArgs {
  const float* x;
  long long n1, n2;        // embedded dims (n0 implied)
  const int* origins;      // 3 per block (embedded)
  int bd0, bd1, bd2;
  int is2d;
  int chunk;               // block points per CTA (a multiple of kFeatThreads)
  int chunks;              // CTAs per block
  float inv_e, inv_e2;     // (float)(1 / e), (float)(1 / e^2)
  long long c_index;       // the value that shifts the second moment
  FeatPart* parts;
};

__device__ __forceinline__ int clamp_bin(int b) { return b < 0 ? 0 : (b > 23 ? 23 : b); }

__device__ __forceinline__ int res_bin(float r) {
  if (!(r > 0.0f)) return 0;
  if (isinf(r)) return 23;
  int ex = 0;
  frexpf(r, &ex);
  return clamp_bin(ex - 1 + 12);
}

__device__ __forceinline__ int grad_bin(float t) {
  if (!(t > 0.0f)) return 0;
  if (isinf(t)) return 23;
  int ex = 0;
  frexpf(t, &ex);
  const int k = ex - 1;
  const int half = k >= 0 ? k / 2 : -((-k + 1) / 2);
  return clamp_bin(half + 12);
}

// Compensated binary32 sum (Kahan); the value is s - c.
struct KSumF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
};

// A binary32 pair hi + lo (about 48 significant bits) for combining the
// per-thread compensated sums without binary64 arithmetic (1/64 of the
// binary32 rate on this part): Knuth's TwoSum on the leading parts, the
// trailing parts added to its error, then Fast2Sum renormalisation.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  const float hi = __fadd_rn(s, lo);
  return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

__device__ __forceinline__ DF df_shfl_xor(DF v, int off) {
  return DF{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

// One bin increment per distinct bin of the warp (bin < 0: no increment);
// every lane of the warp calls it.
__device__ __forceinline__ void warp_bin_add(unsigned* h, int bin) {
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  if (bin >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[bin], __popc(peers));
}

// Each CTA walks `chunk` points of one sampled block (the points of a block
// in row-major order, kFeatThreads apart per thread, coordinates carried
// from one point to the next by a mixed-radix add), accumulates the moment,
// difference and interpolation-error sums as compensated binary32 sums and
// the two histograms in shared memory, and writes one partial.
template <bool is2d>
__global__ void __launch_bounds__(kFeatThreads, 4) feature_kernel(const FeatArgs a) {
  __shared__ unsigned sc[kNCnt];
  __shared__ DF sred[kFeatThreads / 32][kNSum];
  for (int i = threadIdx.x; i < kNCnt; i += blockDim.x) sc[i] = 0u;
  __syncthreads();
  const int blk = blockIdx.y;
  const int bd0 = a.bd0, bd1 = a.bd1, bd2 = a.bd2;
  const int st0 = (int)(a.n1 * a.n2), st1 = (int)a.n2;  // field < 2^32 points: fits int
  const float* blk_base = a.x + (long long)a.origins[3 * blk] * a.n1 * a.n2 +
                          (long long)a.origins[3 * blk + 1] * a.n2 + a.origins[3 * blk + 2];
  const float cshift = __ldg(a.x + a.c_index);
  const int bpts = bd0 * bd1 * bd2;
  const int p0 = blockIdx.x * a.chunk;
  const int p1 = min(bpts, p0 + a.chunk);
  const int iters = (p1 - p0 + kFeatThreads - 1) / kFeatThreads;
  const int bdv[3] = {bd0, bd1, bd2};
  const int stv[3] = {st0, st1, 1};
  KSumF m1, m2, d1[3], d2[3], lin[3], cub[3];
  unsigned n = 0, n1[3] = {0, 0, 0}, n2[3] = {0, 0, 0}, nint[3] = {0, 0, 0}, ng = 0, nl = 0;
  int p = p0 + threadIdx.x;
  int c[3];
  c[2] = p % bd2;
  c[1] = (p / bd2) % bd1;
  c[0] = (p / bd2) / bd1;
  // kFeatThreads in the block's mixed radix (each digit below its radix)
  const int k2 = kFeatThreads % bd2, k1 = (kFeatThreads / bd2) % bd1,
            k0 = (kFeatThreads / bd2) / bd1;
  for (int it = 0; it < iters; ++it, p += kFeatThreads) {
    const bool valid = p < p1;
    int gbin = -1, lbin = -1;
    if (valid) {
      const float* pt = blk_base + (long long)c[0] * st0 + (long long)c[1] * st1 + c[2];
      const float v = pt[0];
      const float u = __fsub_rn(v, cshift);
      m1.add(u);
      m2.add(__fmul_rn(u, u));
      ++n;
      bool fwd = true, bwd = true;
      float gs = 0.0f;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        if (is2d && ax == 0) continue;
        const int k = is2d ? ax - 1 : ax;
        const int sa = stv[ax], ca = c[ax], ba = bdv[ax];
        const bool hasf = ca + 1 < ba, hasb = ca >= 1;
        fwd = fwd && hasf;
        bwd = bwd && hasb;
        if (hasf) {
          const float xf = pt[sa];
          const float df = __fsub_rn(xf, v);
          d1[k].add(fabsf(df));
          ++n1[k];
          gs = __fadd_rn(gs, __fmul_rn(df, df));
          if (hasb) {
            d2[k].add(fabsf(__fsub_rn(__fadd_rn(xf, pt[-sa]), __fmul_rn(2.0f, v))));
            ++n2[k];
          }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int h = 1 << j;
          if ((ca & (2 * h - 1)) != h || ca - 3 * h < 0 || ca + 3 * h > ba - 1) continue;
          const float a3 = pt[-3 * h * sa], a1 = pt[-h * sa], b1 = pt[h * sa],
                      b3 = pt[3 * h * sa];
          const float s1 = __fadd_rn(a1, b1);
          lin[j].add(fabsf(__fsub_rn(v, __fmul_rn(s1, 0.5f))));
          cub[j].add(fabsf(__fsub_rn(
              v, __fmul_rn(__fsub_rn(__fmul_rn(9.0f, s1), __fadd_rn(a3, b3)), 0.0625f))));
          ++nint[j];
        }
      }
      if (fwd) {
        gbin = grad_bin(__fmul_rn(gs, a.inv_e2));
        ++ng;
      }
      if (bwd) {
        float pred;
        if (!is2d) {
          const float sa = __fadd_rn(__fadd_rn(pt[-st0], pt[-st1]), pt[-1]);
          const float sb = __fadd_rn(__fadd_rn(pt[-st0 - st1], pt[-st0 - 1]), pt[-st1 - 1]);
          pred = __fadd_rn(__fsub_rn(sa, sb), pt[-st0 - st1 - 1]);
        } else {
          pred = __fsub_rn(__fadd_rn(pt[-st1], pt[-1]), pt[-st1 - 1]);
        }
        lbin = res_bin(__fmul_rn(fabsf(__fsub_rn(v, pred)), a.inv_e));
        ++nl;
      }
    }
    warp_bin_add(sc + 12, gbin);
    warp_bin_add(sc + 36, lbin);
    c[2] += k2;
    int cy = c[2] >= bd2;
    c[2] -= cy ? bd2 : 0;
    c[1] += k1 + cy;
    cy = c[1] >= bd1;
    c[1] -= cy ? bd1 : 0;
    c[0] += k0 + cy;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  // counts (exact): warp sums, then one atomic per warp
  unsigned cnt[12] = {n, n1[0], n1[1], n1[2], n2[0], n2[1], n2[2], nint[0], nint[1], nint[2],
                      ng, nl};
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const unsigned v = __reduce_add_sync(0xffffffffu, cnt[i]);
    if (l == 0) atomicAdd(&sc[i], v);
  }
  // sums: warp trees, then warps in order
  const KSumF ks[kNSum] = {m1,     m2,     d1[0],  d1[1],  d1[2],  d2[0],  d2[1],
                           d2[2],  lin[0], lin[1], lin[2], cub[0], cub[1], cub[2]};
#pragma unroll
  for (int i = 0; i < kNSum; ++i) {
    DF v{ks[i].s, -ks[i].c};
    for (int off = 16; off > 0; off >>= 1) v = df_add(v, df_shfl_xor(v, off));
    if (l == 0) sred[w][i] = v;
  }
  __syncthreads();
  FeatPart* out = a.parts + (long long)blockIdx.y * a.chunks + blockIdx.x;
  if (threadIdx.x < kNSum) {
    DF v = sred[0][threadIdx.x];
    for (int k = 1; k < kFeatThreads / 32; ++k) v = df_add(v, sred[k][threadIdx.x]);
    out->sum[threadIdx.x] = (double)v.hi + (double)v.lo;
  }
  for (int i = threadIdx.x; i < kNCnt; i += blockDim.x) out->cnt[i] = sc[i];
}

// Fold the partials: one warp per accumulated quantity, its lanes striding
// over the partials, combined by a fixed shuffle tree (a fixed order for the
// double sums; the counts are exact); then one thread per feature.
constexpr int kFinalThreads = 1024;
constexpr int kFinalWarps = kFinalThreads / 32;
static_assert(NF <= kFinalThreads, "one thread per feature");

__global__ void __launch_bounds__(kFinalThreads)
    feature_final_kernel(const FeatPart* parts, int nparts, double rel_eb, double vrange,
                         double e, double npoints, int ndims, double* fd, float* ff) {
  __shared__ double s[kNSum];
  __shared__ unsigned long long c[kNCnt];
  const int t = threadIdx.x, w = t >> 5, l = t & 31;
  for (int q = w; q < kNSum + kNCnt; q += kFinalWarps) {
    if (q < kNSum) {
      double v = 0.0;
      for (int p = l; p < nparts; p += 32) v += parts[p].sum[q];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (l == 0) s[q] = v;
    } else {
      unsigned long long v = 0ull;
      for (int p = l; p < nparts; p += 32) v += parts[p].cnt[q - kNSum];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (l == 0) c[q - kNSum] = v;
    }
  }
  __syncthreads();
  if (t >= NF) return;
  const int i = t;
  double f = 0.0;
  if (i == 0) {
    f = log10(rel_eb);
  } else if (i == 1) {
    double var = 0.0;
    if (c[0]) {
      const double n = (double)c[0];
      const double m = s[0] / n;
      var = s[1] / n - m * m;
      if (var < 0.0) var = 0.0;
    }
    const double sigma = sqrt(var);
    f = (sigma > 0.0 && vrange > 0.0) ? log10(vrange / sigma) : 0.0;
  } else if (i == 2) {
    f = ndims / 3.0;
  } else if (i == 3) {
    f = log2(npoints) / 30.0;
  } else if (i < 7) {  // mean |first difference| per axis
    const int k = i - 4;
    if (k < ndims && c[1 + k]) f = log2(1.0 + (s[2 + k] / (double)c[1 + k]) / e);
  } else if (i < 10) {  // mean |second difference| per axis
    const int k = i - 7;
    if (k < ndims && c[4 + k]) f = log2(1.0 + (s[5 + k] / (double)c[4 + k]) / e);
  } else if (i < 34) {  // gradient-magnitude histogram
    if (c[10]) f = (double)c[12 + (i - 10)] / (double)c[10];
  } else if (i < 58) {  // Lorenzo-residual histogram
    if (c[11]) f = (double)c[36 + (i - 34)] / (double)c[11];
  } else if (i < 61) {  // linear interpolation error per stride
    const int j = i - 58;
    if (c[7 + j]) f = log2(1.0 + (s[8 + j] / (double)c[7 + j]) / e);
  } else {  // cubic interpolation error per stride
    const int j = i - 61;
    if (c[7 + j]) f = log2(1.0 + (s[11 + j] / (double)c[7 + j]) / e);
  }
  if (fd) fd[i] = f;
  if (ff) ff[i] = (float)f;
}

// ------------------------------------------------------------- network
constexpr int kMlpThreads = 256;
constexpr int kMlpS = 16;  // samples per CTA

struct MlpSmem {
  float z[kMlpS][NF];
  float h1[kMlpS][NH];
  float h2[kMlpS][NH];
  float o[kMlpS][NO];
  float dout[kMlpS][NO];
  float dh2[kMlpS][NH];
  float dh1[kMlpS][NH];
  float loss[kMlpS];
};

// Forward for kMlpS samples per CTA; TRAIN adds the loss, the backward pass
// and this CTA's gradient partial (NPARAM floats at gpart + cta * NPARAM).
template <bool TRAIN>
__global__ void __launch_bounds__(kMlpThreads) mlp_kernel(
    const float* __restrict__ P, const float* __restrict__ mean, const float* __restrict__ sd,
    const float* __restrict__ X, const int* __restrict__ labels, long long B, float invB,
    float* __restrict__ logits, float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smraw[];
  MlpSmem& sm = *reinterpret_cast<MlpSmem*>(smraw);
  const int t = threadIdx.x;
  const long long s0 = (long long)blockIdx.x * kMlpS;
  const float* W1 = P + OFF_W1;
  const float* b1 = P + OFF_B1;
  const float* W2 = P + OFF_W2;
  const float* b2 = P + OFF_B2;
  const float* W3 = P + OFF_W3;
  const float* b3 = P + OFF_B3;
  for (int i = t; i < kMlpS * NF; i += kMlpThreads) {
    const int s = i / NF, f = i % NF;
    const float d = sd[f] != 0.0f ? sd[f] : 1.0f;
    sm.z[s][f] = s0 + s < B ? __fdiv_rn(__fsub_rn(X[(s0 + s) * NF + f], mean[f]), d) : 0.0f;
  }
  __syncthreads();
  // dense layers: one warp per output row, the row's weights read once
  // (coalesced) and applied to every sample of the CTA; lane partial sums
  // are combined by a fixed shuffle tree
  const int warp = t >> 5, lane = t & 31;
  constexpr int kWarps = kMlpThreads / 32;
  // inference walks only the CTA's valid samples (one for a single field);
  // training keeps every slot, the padded ones computed from z = 0, so the
  // gradient sums below read no unwritten shared memory
  const int ns = TRAIN ? kMlpS : (int)(B - s0 < kMlpS ? B - s0 : kMlpS);
  for (int o = warp; o < NH; o += kWarps) {
    const float w0 = W1[o * NF + lane], w1 = W1[o * NF + 32 + lane];
    for (int s = 0; s < ns; ++s) {
      float v = __fadd_rn(__fmul_rn(w0, sm.z[s][lane]), __fmul_rn(w1, sm.z[s][32 + lane]));
      for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
      if (lane == 0) {
        const float acc = __fadd_rn(b1[o], v);
        sm.h1[s][o] = acc > 0.0f ? acc : 0.0f;
      }
    }
  }
  __syncthreads();
  for (int o = warp; o < NH; o += kWarps) {
    float w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = W2[o * NH + 32 * j + lane];
    for (int s = 0; s < ns; ++s) {
      float v = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) v = __fadd_rn(v, __fmul_rn(w[j], sm.h1[s][32 * j + lane]));
      for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
      if (lane == 0) {
        const float acc = __fadd_rn(b2[o], v);
        sm.h2[s][o] = acc > 0.0f ? acc : 0.0f;
      }
    }
  }
  __syncthreads();
  for (int o = warp; o < NO; o += kWarps) {
    float w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = W3[o * NH + 32 * j + lane];
    for (int s = 0; s < ns; ++s) {
      float v = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) v = __fadd_rn(v, __fmul_rn(w[j], sm.h2[s][32 * j + lane]));
      for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, off));
      if (lane == 0) {
        const float acc = __fadd_rn(b3[o], v);
        sm.o[s][o] = acc;
        if (!TRAIN && s0 + s < B) logits[(s0 + s) * NO + o] = acc;
      }
    }
  }
  if (!TRAIN) return;
  __syncthreads();
  // loss and d loss / d logits, one (sample, head) per thread
  if (t < kMlpS * 4) {
    const int s = t / 4, hd = t % 4;
    const int off = kHeadOff[hd], len = kHeadLen[hd];
    float l = 0.0f;
    if (s0 + s < B) {
      const int lab = labels[(s0 + s) * 4 + hd];
      // a label outside its head is not read through: the loss becomes NaN
      // (the batch is invalid) and the head's gradient lacks the label term
      const bool lab_ok = lab >= 0 && lab < len;
      float mx = sm.o[s][off];
      for (int j = 1; j < len; ++j) mx = fmaxf(mx, sm.o[s][off + j]);
      float se = 0.0f;
      for (int j = 0; j < len; ++j) se += expf(sm.o[s][off + j] - mx);
      l = (logf(se) + mx) - (lab_ok ? sm.o[s][off + lab] : __int_as_float(0x7fc00000));
      for (int j = 0; j < len; ++j)
        sm.dout[s][off + j] = (expf(sm.o[s][off + j] - mx) / se - (j == lab ? 1.0f : 0.0f)) * invB;
    } else {
      for (int j = 0; j < len; ++j) sm.dout[s][off + j] = 0.0f;
    }
    // per-sample loss: heads summed in order by lane hd == 0 after a shuffle
    const float l1 = __shfl_down_sync(0xffffffffu, l, 1, 4);
    const float l2 = __shfl_down_sync(0xffffffffu, l, 2, 4);
    const float l3 = __shfl_down_sync(0xffffffffu, l, 3, 4);
    if (hd == 0) sm.loss[s] = ((l + l1) + l2) + l3;
  }
  __syncthreads();
  for (int i = t; i < kMlpS * NH; i += kMlpThreads) {
    const int s = i / NH, k = i % NH;
    float acc = 0.0f;
    for (int o = 0; o < NO; ++o) acc += W3[o * NH + k] * sm.dout[s][o];
    sm.dh2[s][k] = sm.h2[s][k] > 0.0f ? acc : 0.0f;
  }
  __syncthreads();
  for (int i = t; i < kMlpS * NH; i += kMlpThreads) {
    const int s = i / NH, k = i % NH;
    float acc = 0.0f;
    for (int o = 0; o < NH; ++o) acc += W2[o * NH + k] * sm.dh2[s][o];
    sm.dh1[s][k] = sm.h1[s][k] > 0.0f ? acc : 0.0f;
  }
  __syncthreads();
  float* g = gpart + (long long)blockIdx.x * NPARAM;
  for (int p = t; p < NPARAM; p += kMlpThreads) {
    float acc = 0.0f;
    if (p < OFF_B1) {
      const int o = p / NF, k = p % NF;
      for (int s = 0; s < kMlpS; ++s) acc += sm.dh1[s][o] * sm.z[s][k];
    } else if (p < OFF_W2) {
      const int o = p - OFF_B1;
      for (int s = 0; s < kMlpS; ++s) acc += sm.dh1[s][o];
    } else if (p < OFF_B2) {
      const int q = p - OFF_W2, o = q / NH, k = q % NH;
      for (int s = 0; s < kMlpS; ++s) acc += sm.dh2[s][o] * sm.h1[s][k];
    } else if (p < OFF_W3) {
      const int o = p - OFF_B2;
      for (int s = 0; s < kMlpS; ++s) acc += sm.dh2[s][o];
    } else if (p < OFF_B3) {
      const int q = p - OFF_W3, o = q / NH, k = q % NH;
      for (int s = 0; s < kMlpS; ++s) acc += sm.dout[s][o] * sm.h2[s][k];
    } else {
      const int o = p - OFF_B3;
      for (int s = 0; s < kMlpS; ++s) acc += sm.dout[s][o];
    }
    g[p] = acc;
  }
  if (t == 0) {
    float l = 0.0f;
    for (int s = 0; s < kMlpS; ++s) l += sm.loss[s];
    lpart[blockIdx.x] = l;
  }
}

// Sum of the CTA partials (fixed order), then Adam on each parameter.
__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ gpart, const float* __restrict__ lpart,
                            int nparts, float invB, int update, float lr, float beta1,
                            float beta2, float c1, float c2, float eps, float* grad_out,
                            float* loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    float l = 0.0f;
    for (int c = 0; c < nparts; ++c) l += lpart[c];
    *loss_out = l * invB;
  }
  if (p >= NPARAM) return;
  float g = 0.0f;
  for (int c = 0; c < nparts; ++c) g += gpart[(long long)c * NPARAM + p];
  if (grad_out) grad_out[p] = g;
  if (!update) return;
  const float mm = beta1 * m[p] + (1.0f - beta1) * g;
  const float vv = beta2 * v[p] + (1.0f - beta2) * g * g;
  m[p] = mm;
  v[p] = vv;
  P[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace

struct qoz_model {
  float* d_params = nullptr;
  float* d_mean = nullptr;
  float* d_sd = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_gpart = nullptr;
  float* d_lpart = nullptr;
  float* d_loss = nullptr;
  long long gpart_ctas = 0;
  long long t = 0;
};

namespace {

// splitmix64: deterministic initial weights from the seed
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

qoz_status ensure_partials(qoz_model* m, long long ctas) {
  if (ctas <= m->gpart_ctas) return QOZ_OK;
  cudaFree(m->d_gpart);
  cudaFree(m->d_lpart);
  m->d_gpart = nullptr;
  m->d_lpart = nullptr;
  m->gpart_ctas = 0;
  if (cudaMalloc((void**)&m->d_gpart, sizeof(float) * NPARAM * ctas) != cudaSuccess ||
      cudaMalloc((void**)&m->d_lpart, sizeof(float) * ctas) != cudaSuccess) {
    cudaGetLastError();
    return fail(QOZ_ENOMEM, "model gradient partials");
  }
  m->gpart_ctas = ctas;
  return QOZ_OK;
}

constexpr size_t kMlpSmem = sizeof(MlpSmem);

template <bool TRAIN>
cudaError_t launch_mlp(const qoz_model* m, const float* X, const int* labels, long long B,
                       float* logits, cudaStream_t s) {
  static unsigned long long done = 0;
  cudaError_t e = ensure_smem_attr((const void*)mlp_kernel<TRAIN>, &done, kMlpSmem);
  if (e != cudaSuccess) return e;
  const long long ctas = (B + kMlpS - 1) / kMlpS;
  mlp_kernel<TRAIN><<<(unsigned)ctas, kMlpThreads, kMlpSmem, s>>>(
      m->d_params, m->d_mean, m->d_sd, X, labels, B, 1.0f / (float)B, logits, m->d_gpart,
      m->d_lpart);
  note_launch(1);
  return cudaGetLastError();
}

// Gradient (and optionally one Adam step) on a batch.
qoz_status grad_step(qoz_model* m, const float* X, const int* labels, long long B, int update,
                     float lr, float* d_grad, float* h_loss, cudaStream_t s) {
  if (!m || !X || !labels || B < 1) return fail(QOZ_EINVAL, "invalid argument");
  const long long ctas = (B + kMlpS - 1) / kMlpS;
  qoz_status st = ensure_partials(m, ctas);
  if (st != QOZ_OK) return st;
  cudaError_t e = launch_mlp<true>(m, X, labels, B, nullptr, s);
  const double b1 = 0.9, b2 = 0.999;
  const long long t = update ? m->t + 1 : m->t;
  const float c1 = update ? (float)(1.0 - std::pow(b1, (double)t)) : 1.0f;
  const float c2 = update ? (float)(1.0 - std::pow(b2, (double)t)) : 1.0f;
  if (e == cudaSuccess) {
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(
        m->d_params, m->d_m, m->d_v, m->d_gpart, m->d_lpart, (int)ctas, 1.0f / (float)B,
        update, lr, (float)b1, (float)b2, c1, c2, 1e-8f, d_grad, m->d_loss);
    note_launch(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && h_loss) {
    e = cudaMemcpyAsync(h_loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "model step");
  if (update) m->t = t;
  return QOZ_OK;
}

// Features of the sampled blocks into device buffers fd (double, may be
// NULL) / ff (float, may be NULL); returns the value range through vr.
qoz_status features_impl(const float* d_field, const qoz_shape& shape, double rel_eb,
                         const qoz_tune_opts* opts_in, double* fd, float* ff, cudaStream_t s,
                         double* vr_out, double* vmin_out, double* vmax_out, Sampling* sm_out) {
  if (!d_field) return fail(QOZ_EINVAL, "d_field is NULL");
  if (!(rel_eb > 0.0 && std::isfinite(rel_eb))) return fail(QOZ_EINVAL, "rel_eb must be > 0");
  Resolved r;
  qoz_status st = resolve(shape, nullptr, &r);
  if (st != QOZ_OK) return st;
  qoz_tune_opts o;
  if ((st = resolve_tune_opts(shape, r, opts_in, &o)) != QOZ_OK) return st;
  float vmin, vmax;
  int64_t cnt;
  st = qoz_value_range(d_field, r.N, &vmin, &vmax, &cnt, s);
  if (st != QOZ_OK) return st;
  const double vr = (double)vmax - (double)vmin;
  const double e0 = rel_eb * vr;
  const double e = e0 > 0.0 ? e0 : 1.0;
  Sampling sm = sample_blocks(r, o.block, o.rate, o.anchor_stride);
  const long long bpts = (long long)sm.bd[0] * sm.bd[1] * sm.bd[2];
  // points per CTA: enough CTAs for about two waves at four CTAs per SM,
  // at least eight points per thread
  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    nsm = 1;
  const long long want = 8LL * nsm;
  const long long per_block = std::max(1LL, (want + sm.nb - 1) / sm.nb);
  long long chunk = (bpts + per_block - 1) / per_block;
  chunk = std::max<long long>(8LL * kFeatThreads, (chunk + kFeatThreads - 1) / kFeatThreads *
                                                      kFeatThreads);
  const int chunks = (int)((bpts + chunk - 1) / chunk);
  const long long nparts = (long long)chunks * sm.nb;
  if (sm.nb > 65535) return fail(QOZ_EUNSUPPORTED, "too many sampled blocks");
  if (bpts > 0x7fff0000LL) return fail(QOZ_EUNSUPPORTED, "sampled block too large");
  void* scratch = nullptr;
  const size_t ob = ((size_t)sm.origins.size() * sizeof(int) + 255) & ~(size_t)255;
  cudaError_t ce = dev_alloc(&scratch, ob + sizeof(FeatPart) * nparts, s);
  if (ce != cudaSuccess) return fail(QOZ_ENOMEM, "feature scratch");
  int* d_org = (int*)scratch;
  FeatPart* parts = (FeatPart*)((char*)scratch + ob);
  ce = cudaMemcpyAsync(d_org, sm.origins.data(), sizeof(int) * sm.origins.size(),
                       cudaMemcpyHostToDevice, s);
  ProfScope ps(QOZ_STAGE_FEATURES, s);
  if (ce == cudaSuccess) {
    FeatArgs a;
    a.x = d_field;
    a.n1 = r.n[1];
    a.n2 = r.n[2];
    a.origins = d_org;
    a.bd0 = sm.bd[0];
    a.bd1 = sm.bd[1];
    a.bd2 = sm.bd[2];
    a.is2d = r.ndims == 2;
    a.chunk = (int)chunk;
    a.chunks = chunks;
    a.inv_e = (float)(1.0 / e);
    a.inv_e2 = (float)(1.0 / (e * e));
    // the second moment is shifted by the first sampled value
    a.c_index = ((long long)sm.origins[0] * r.n[1] + sm.origins[1]) * r.n[2] + sm.origins[2];
    a.parts = parts;
    if (a.is2d)
      feature_kernel<true><<<dim3(chunks, sm.nb), kFeatThreads, 0, s>>>(a);
    else
      feature_kernel<false><<<dim3(chunks, sm.nb), kFeatThreads, 0, s>>>(a);
    note_launch(1);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) {
    feature_final_kernel<<<1, kFinalThreads, 0, s>>>(parts, (int)nparts, rel_eb, vr, e,
                                                     (double)r.N, r.ndims, fd, ff);
    note_launch(1);
    ce = cudaGetLastError();
  }
  dev_free(scratch, s);
  if (ce != cudaSuccess) return cuda_fail(ce, "features");
  if (vr_out) *vr_out = vr;
  if (vmin_out) *vmin_out = vmin;
  if (vmax_out) *vmax_out = vmax;
  if (sm_out) *sm_out = sm;
  return QOZ_OK;
}

}  // namespace

extern "C" {

qoz_status qoz_features(const float* d_field, qoz_shape shape, double rel_eb,
                        const qoz_tune_opts* opts, double* h_features, float* d_features,
                        void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  configure_pool_once();
  double* d_tmp = nullptr;
  if (h_features && dev_alloc((void**)&d_tmp, sizeof(double) * NF, s) != cudaSuccess)
    return fail(QOZ_ENOMEM, "feature output");
  qoz_status st = features_impl(d_field, shape, rel_eb, opts, d_tmp, d_features, s, nullptr,
                                nullptr, nullptr, nullptr);
  if (st == QOZ_OK && h_features) {
    cudaError_t e = cudaMemcpyAsync(h_features, d_tmp, sizeof(double) * NF,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "features read-back");
  }
  dev_free(d_tmp, s);
  return st;
}

qoz_status qoz_model_create(uint64_t seed, qoz_model** out) {
  if (!out) return fail(QOZ_EINVAL, "out is NULL");
  *out = nullptr;
  qoz_model* m = new qoz_model();
  const size_t pb = sizeof(float) * NPARAM;
  if (cudaMalloc((void**)&m->d_params, pb) != cudaSuccess ||
      cudaMalloc((void**)&m->d_m, pb) != cudaSuccess ||
      cudaMalloc((void**)&m->d_v, pb) != cudaSuccess ||
      cudaMalloc((void**)&m->d_mean, sizeof(float) * NF) != cudaSuccess ||
      cudaMalloc((void**)&m->d_sd, sizeof(float) * NF) != cudaSuccess ||
      cudaMalloc((void**)&m->d_loss, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    qoz_model_free(m);
    return fail(QOZ_ENOMEM, "model allocation");
  }
  // He-uniform weights (bound sqrt(6 / fan_in)), zero biases, identity
  // normalisation
  std::vector<float> P(NPARAM, 0.0f), mean(NF, 0.0f), sd(NF, 1.0f);
  uint64_t st = seed;
  auto fill = [&](int off, int n, int fan_in) {
    const double bound = std::sqrt(6.0 / fan_in);
    for (int i = 0; i < n; ++i) {
      const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      P[off + i] = (float)((2.0 * u - 1.0) * bound);
    }
  };
  fill(OFF_W1, NH * NF, NF);
  fill(OFF_W2, NH * NH, NH);
  fill(OFF_W3, NO * NH, NH);
  const qoz_status s2 = qoz_model_set(m, P.data(), mean.data(), sd.data());
  if (s2 != QOZ_OK) {
    qoz_model_free(m);
    return s2;
  }
  *out = m;
  return QOZ_OK;
}

qoz_status qoz_model_set(qoz_model* m, const float* h_params, const float* h_mean,
                         const float* h_sd) {
  if (!m) return fail(QOZ_EINVAL, "model is NULL");
  cudaError_t e = cudaSuccess;
  if (h_params) {
    e = cudaMemcpy(m->d_params, h_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, sizeof(float) * NPARAM);
    if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, sizeof(float) * NPARAM);
    m->t = 0;
  }
  if (e == cudaSuccess && h_mean)
    e = cudaMemcpy(m->d_mean, h_mean, sizeof(float) * NF, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && h_sd)
    e = cudaMemcpy(m->d_sd, h_sd, sizeof(float) * NF, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "model upload");
  return QOZ_OK;
}

qoz_status qoz_model_get(const qoz_model* m, float* h_params, float* h_mean, float* h_sd) {
  if (!m) return fail(QOZ_EINVAL, "model is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && h_params)
    e = cudaMemcpy(h_params, m->d_params, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_mean)
    e = cudaMemcpy(h_mean, m->d_mean, sizeof(float) * NF, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && h_sd)
    e = cudaMemcpy(h_sd, m->d_sd, sizeof(float) * NF, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "model download");
  return QOZ_OK;
}

qoz_status qoz_model_forward(const qoz_model* m, const float* d_features, int64_t n,
                             float* d_logits, void* stream) {
  if (!m || !d_features || !d_logits || n < 1) return fail(QOZ_EINVAL, "invalid argument");
  cudaError_t e = launch_mlp<false>(m, d_features, nullptr, n, d_logits, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "model forward");
  return QOZ_OK;
}

qoz_status qoz_model_gradient(qoz_model* m, const float* d_features, const int32_t* d_labels,
                              int64_t n, float* d_grad, float* h_loss, void* stream) {
  return grad_step(m, d_features, d_labels, n, 0, 0.0f, d_grad, h_loss, (cudaStream_t)stream);
}

qoz_status qoz_model_train_step(qoz_model* m, const float* d_features, const int32_t* d_labels,
                                int64_t n, float lr, float* h_loss, void* stream) {
  if (!(lr > 0.0f)) return fail(QOZ_EINVAL, "lr must be > 0");
  return grad_step(m, d_features, d_labels, n, 1, lr, nullptr, h_loss, (cudaStream_t)stream);
}

void qoz_model_free(qoz_model* m) {
  if (!m) return;
  cudaFree(m->d_params);
  cudaFree(m->d_m);
  cudaFree(m->d_v);
  cudaFree(m->d_mean);
  cudaFree(m->d_sd);
  cudaFree(m->d_gpart);
  cudaFree(m->d_lpart);
  cudaFree(m->d_loss);
  delete m;
}

qoz_status qoz_tune_learned(const float* d_field, qoz_shape shape, double rel_eb,
                            qoz_metric metric, double target, const qoz_tune_opts* opts,
                            const qoz_model* model, void* stream, qoz_tune_report* out) {
  if (!model || !out) return fail(QOZ_EINVAL, "NULL argument");
  if (metric < QOZ_METRIC_MAXERR || metric > QOZ_METRIC_AC)
    return fail(QOZ_EINVAL, "unknown metric %d", metric);
  const bool target_mode = !std::isnan(target);
  if (target_mode && (metric == QOZ_METRIC_MAXERR || metric == QOZ_METRIC_AC))
    return fail(QOZ_EINVAL, "a target needs the PSNR or SSIM metric");
  cudaStream_t s = (cudaStream_t)stream;
  configure_pool_once();
  Resolved r;
  qoz_status st = resolve(shape, nullptr, &r);
  if (st != QOZ_OK) return st;
  qoz_tune_opts o;
  if ((st = resolve_tune_opts(shape, r, opts, &o)) != QOZ_OK) return st;
  if (o.n_alpha != 5 || o.n_beta != 3)
    return fail(QOZ_EINVAL, "the network's heads need 5 alpha and 3 beta candidates");
  float* d_buf = nullptr;
  if (dev_alloc((void**)&d_buf, sizeof(float) * (NF + NO), s) != cudaSuccess)
    return fail(QOZ_ENOMEM, "tuner scratch");
  double vr = 0.0, vmin = 0.0, vmax = 0.0;
  Sampling sm;
  st = features_impl(d_field, shape, rel_eb, &o, nullptr, d_buf, s, &vr, &vmin, &vmax, &sm);
  float logits[NO];
  if (st == QOZ_OK) {
    ProfScope ps(QOZ_STAGE_FORWARD, s);
    cudaError_t e = launch_mlp<false>(model, d_buf, nullptr, 1, d_buf + NF, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(logits, d_buf + NF, sizeof(logits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "learned tuner");
  }
  dev_free(d_buf, s);
  if (st != QOZ_OK) return st;
  auto argmax = [&](int off, int len) {
    int b = 0;
    for (int j = 1; j < len; ++j)
      if (logits[off + j] > logits[off + b]) b = j;
    return b;
  };
  const int interp = argmax(0, 2);
  const int order = argmax(2, r.ndims == 3 ? 6 : 2);
  const int ia = argmax(8, 5), ib = argmax(13, 3);
  memset(out, 0, sizeof(*out));
  for (int l = 0; l < QOZ_MAX_LEVELS; ++l) {
    out->params.interp[l] = (uint8_t)interp;
    out->params.order[l] = (uint8_t)order;
  }
  out->params.alpha = o.alphas[ia];
  out->params.beta = o.betas[ib];
  out->params.anchor_stride = o.anchor_stride;
  double e = rel_eb * vr;
  if (target_mode && metric == QOZ_METRIC_PSNR) {
    // uniform-error estimate of the bound that meets the PSNR target
    const double e0 = vr * std::sqrt(3.0) * std::pow(10.0, -target / 20.0);
    if (e0 < e) e = e0;
  }
  out->abs_eb = e;
  out->vmin = vmin;
  out->vmax = vmax;
  out->B = NAN;
  out->M = NAN;
  out->n_trials = 0;
  out->n_blocks = sm.nb;
  out->n_sampled_points = sm.npts;
  return QOZ_OK;
}

qoz_status qoz_tune_learned_verified(const float* d_field, qoz_shape shape, double rel_eb,
                                     qoz_metric metric, double target,
                                     const qoz_tune_opts* opts, const qoz_model* model,
                                     void* stream, qoz_tune_report* out) {
  qoz_tune_report proposal;
  qoz_status st =
      qoz_tune_learned(d_field, shape, rel_eb, metric, target, opts, model, stream, &proposal);
  if (st != QOZ_OK) return st;
  return qoz_tune_verify(d_field, shape, rel_eb, metric, target, opts, &proposal.params, stream,
                         out);
}

}  // extern "C"
