// Quality metrics of Sec. 3: max abs error, MSE / PSNR (Eq. psnr) and SSIM
// (Eq. ssim, Eq. ssim2).  Per-CTA partial sums are combined on the host in a
// fixed order, so every result is deterministic.
//
// Arithmetic.  The maximum error is exact: the binary32 difference |a - b| is
// a monotone rounding of the exact one, so each thread keeps the element that
// leads by its rounded difference and, among ties, by the subtraction's
// rounding error; the leader's difference is taken in double at the end.
// The squared errors and the autocorrelation terms are summed in binary32
// with compensation (Kahan), per thread, then in double across threads.
//
// SSIM.  For windows of edge 7 the moments are box sums taken separably:
// along x in registers, along y in shared memory, along z through a ring of
// per-plane sums while the CTA marches through its z-range.  The sums are
// kept in binary32 on the rewritten form of each window's index:
//   with d = b - a,  SSIM_w = (1 - md^2 / D1) (1 - vd / D2),
//   D1 = mx^2 + my^2 + c1,  D2 = vx + vy + c2,
// which is Eq. (ssim) with (2 mx my + c1) = D1 - md^2 and
// (2 cxy + c2) = D2 - vd.  The small quantities md and vd come from the
// moments of d itself, so the cancellation that makes 1 - SSIM inaccurate
// in the plain form never happens; each CTA also shifts a by one of its own
// values before forming second moments.  Each thread accumulates 1 - SSIM_w.
#include <cuda_runtime.h>

#include "qoz_internal.h"

namespace qoz {
namespace {

constexpr int kErrThreads = 512;
constexpr int kErrBlocks = 152 * 2;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = l < nw ? sh[l] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  return v;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = l < nw ? sh[l] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  }
  return v;
}

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
};

// Max and NaN bookkeeping of one error e = fl(b - a) (|e| = |fl(a - b)|).
// fl is monotone, so the exact maximum of |b - a| has the largest |e|; among
// equal |e| it has the largest t, the rounding error of the subtraction
// (Knuth's TwoSum, exact in binary32) signed towards |e|, since the exact
// |b - a| is |e| + t.  The leader's inputs are kept and its difference is
// taken in binary64 at the end, as the definition does.  Only a new or tied
// leader (rare after a thread's first few elements) takes the branch; start
// with mxf = -1 so that the first element leads.  (Differences beyond the
// binary32 range all round to infinity; the first of them leads.)
struct ErrMax {
  float mxf = -1.0f, mxt = 0.0f, ma = 0.0f, mb = 0.0f;
  __device__ __forceinline__ void add(float av, float bv, float e) {
    const float ad = fabsf(e);  // NaN never leads
    if (ad >= mxf) {
      const float bp = __fsub_rn(e, bv);
      const float ap = __fsub_rn(e, bp);
      const float t = __fadd_rn(__fsub_rn(bv, ap), __fsub_rn(-av, bp));
      const float tt = e < 0.0f ? -t : t;
      if (ad > mxf || tt > mxt) {
        mxf = ad;
        mxt = tt;
        ma = av;
        mb = bv;
      }
    }
  }
  __device__ __forceinline__ double value() const {
    return mxf < 0.0f ? 0.0 : fabs((double)mb - (double)ma);
  }
};

constexpr int kAcParts = 5;

// One pass over a and b for the metrics call: the exact max |a - b|, the sum
// of squared errors and the lag-1 autocorrelation sums of e = b - a (sum e,
// sum e^2, sum e_i e_{i+1}, and sum e without its last / first element).
// With 16-byte aligned inputs a thread takes four consecutive errors per
// step, adds their terms pairwise and each of the three partials to a
// compensated binary32 sum; the error after its fourth comes from the next
// lane by a shuffle, or by a load for the warp's last lane.  Part layout:
// part_sse[g], part_max[g], part_ac[j * g + cta].
struct ErrAcc {
  ErrMax mx;
  Kahan s1, s2, sk;
  int nans = 0;
  // four consecutive errors of (u, v); nx the one after them (has_next)
  __device__ __forceinline__ void step4(const float4& u, const float4& v, float e0, float nx,
                                        bool has_next) {
    const float e1 = __fsub_rn(v.y, u.y), e2 = __fsub_rn(v.z, u.z), e3 = __fsub_rn(v.w, u.w);
    const float q = __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)),
                              __fadd_rn(__fmul_rn(e2, e2), __fmul_rn(e3, e3)));
    if (q != q) ++nans;  // a square is NaN only for a NaN error
    const float am = fmaxf(fmaxf(fabsf(e0), fabsf(e1)), fmaxf(fabsf(e2), fabsf(e3)));
    if (am >= mx.mxf) {
      mx.add(u.x, v.x, e0);
      mx.add(u.y, v.y, e1);
      mx.add(u.z, v.z, e2);
      mx.add(u.w, v.w, e3);
    }
    s1.add(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, e3)));
    s2.add(q);
    const float k3 = has_next ? __fmul_rn(e3, nx) : 0.0f;
    sk.add(__fadd_rn(__fadd_rn(__fmul_rn(e0, e1), __fmul_rn(e1, e2)),
                     __fadd_rn(__fmul_rn(e2, e3), k3)));
  }
  __device__ __forceinline__ void step1(float av, float bv, float e) {
    if (e != e) ++nans;
    mx.add(av, bv, e);
    s1.add(e);
    s2.add(__fmul_rn(e, e));
  }
};

__global__ void __launch_bounds__(kErrThreads, 2) err_kernel(const float* __restrict__ a,
                                                             const float* __restrict__ b,
                                                             long long n, double* part_sse,
                                                             double* part_max, double* part_ac) {
  __shared__ double sh[32];
  ErrAcc acc;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const bool vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
  long long i0 = 0;
  if (vec) {
    const long long n4 = n >> 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    // i - lane is the warp's first vector, so the trip counts are
    // warp-uniform. Full steps (all 32 lanes in range) load the next step's
    // vectors before this step's arithmetic; at most one partial step per
    // warp follows.
    long long i = tid;
    float4 un = make_float4(0.f, 0.f, 0.f, 0.f), vn = un;
    if (i - lane < n4 - 31) {
      un = __ldcs(a4 + i);
      vn = __ldcs(b4 + i);
    }
    for (; i - lane < n4 - 31; i += nthr) {
      const float4 u = un, v = vn;
      if (i + nthr - lane < n4 - 31) {
        un = __ldcs(a4 + i + nthr);
        vn = __ldcs(b4 + i + nthr);
      }
      const float e0 = __fsub_rn(v.x, u.x);
      float nx = __shfl_down_sync(0xffffffffu, e0, 1);
      bool has_next = true;
      if (lane == 31) {
        const long long j = 4 * i + 4;
        has_next = j < n;
        nx = has_next ? __fsub_rn(b[j], a[j]) : 0.0f;
      }
      acc.step4(u, v, e0, nx, has_next);
    }
    if (i - lane < n4) {
      const bool ok = i < n4;
      float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
      if (ok) {
        u = __ldcs(a4 + i);
        v = __ldcs(b4 + i);
      }
      const float e0 = __fsub_rn(v.x, u.x);
      float nx = __shfl_down_sync(0xffffffffu, e0, 1);
      if (ok) {
        const long long j = 4 * i + 4;
        const bool has_next = j < n;
        if (has_next && (lane == 31 || i + 1 >= n4)) nx = __fsub_rn(b[j], a[j]);
        acc.step4(u, v, e0, nx, has_next);
      }
    }
    i0 = n4 << 2;
  }
  for (long long i = i0 + tid; i < n; i += nthr) {
    const float av = a[i], bv = b[i];
    const float e = __fsub_rn(bv, av);
    acc.step1(av, bv, e);
    if (i + 1 < n) acc.sk.add(__fmul_rn(e, __fsub_rn(b[i + 1], a[i + 1])));
  }
  // the pair sums' members: all errors but the last (head), all but the first (tail)
  Kahan head = acc.s1, tail = acc.s1;
  if (tid == 0 && n > 0) {
    tail.add(-__fsub_rn(b[0], a[0]));
    head.add(-__fsub_rn(b[n - 1], a[n - 1]));
  }
  const double ss = block_sum((double)acc.s2.s - (double)acc.s2.c, sh);
  const double m = block_max(acc.mx.value(), sh);
  const double nn = block_sum((double)acc.nans, sh);  // a NaN difference makes the max NaN
  if (threadIdx.x == 0) {
    part_sse[blockIdx.x] = ss;
    part_max[blockIdx.x] = nn > 0.0 ? __longlong_as_double(0x7ff8000000000000LL) : m;
    part_ac[1 * gridDim.x + blockIdx.x] = ss;
  }
  const Kahan* ks[4] = {&acc.s1, &acc.sk, &head, &tail};
  const int slot[4] = {0, 2, 3, 4};
  for (int j = 0; j < 4; ++j) {
    const double v = block_sum((double)ks[j]->s - (double)ks[j]->c, sh);
    if (threadIdx.x == 0) part_ac[(size_t)slot[j] * gridDim.x + blockIdx.x] = v;
  }
}

// ---------------------------------------------------------------- Eq. (ac)
// Lag-k autocorrelation of the errors e_i = b_i - a_i over the flattened
// arrays: one pass accumulating sum e, sum e^2, sum e_i e_{i+k} over the
// n - k pairs and the sums of the pairs' first and second members, each in
// compensated binary32 per thread and double across threads; the host forms
// the mean, the variance and the lag covariance from them.

__global__ void __launch_bounds__(kErrThreads) ac_kernel(const float* __restrict__ a,
                                                         const float* __restrict__ b,
                                                         long long n, long long k,
                                                         double* part) {
  __shared__ double sh[32];
  Kahan s1, s2, sk, head, tail;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < n; i += nthr) {
    const float e = __fsub_rn(__ldcs(b + i), __ldcs(a + i));
    s1.add(e);
    s2.add(__fmul_rn(e, e));
    if (i + k < n) {
      const float f = __fsub_rn(b[i + k], a[i + k]);
      sk.add(__fmul_rn(e, f));
      head.add(e);
    }
    if (i >= k) tail.add(e);
  }
  Kahan* acc[kAcParts] = {&s1, &s2, &sk, &head, &tail};
  for (int j = 0; j < kAcParts; ++j) {
    const double v = block_sum((double)acc[j]->s - (double)acc[j]->c, sh);
    if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = v;
  }
}

// ---------------------------------------------------------------- SSIM, tiled
constexpr int kTileThreads = 256;
constexpr int kWX = 32;   // windows per CTA along x
constexpr int kWY = 8;    // windows per CTA along y (kWX * kWY == kTileThreads)
constexpr int kG = 4;     // windows per thread in the x pass
constexpr int kZC = 32;   // windows per CTA along z (3-D)

template <int WIN, int STEP>
struct SsimGeo {
  static constexpr int EX = STEP * (kWX - 1) + WIN;   // input columns per plane tile
  static constexpr int EY = STEP * (kWY - 1) + WIN;   // input rows per plane tile
  static constexpr int EX4 = (EX + 3) / 4;            // 16-byte chunks per input row
  static constexpr int EXP = (4 * EX4) | 1;           // odd row pitch holding whole chunks
  static constexpr int NCH = EY * EX4;                // chunks per plane tile
  static constexpr int LPT = (NCH + kTileThreads - 1) / kTileThreads;
  static constexpr int SPAN = STEP * (kG - 1) + WIN;  // points one x task reads
  static constexpr int NXT = EY * (kWX / kG);         // x tasks per plane
  static_assert(kWX * kWY == kTileThreads, "one thread per (wy, wx) window column");
  static_assert(NXT <= kTileThreads, "x tasks fit one pass");
};

template <int WIN, int STEP, bool IS3D>
struct SsimSmem {
  using G = SsimGeo<WIN, STEP>;
  float xs[G::EY * G::EXP];
  float ys[G::EY * G::EXP];
  float h[5][G::EY][kWX + 1];   // padded: the x pass's lanes write down a column
  // z sums: per-plane sums of the last WIN planes, or with step 2 the last
  // three sums of plane pairs (2k, 2k + 1)
  static constexpr int kRing = !IS3D ? 1 : (STEP == 2 && WIN == 7 ? 3 : WIN);
  float ring[kRing][5][kTileThreads];
};

template <int WIN, int STEP, bool IS3D>
__global__ void __launch_bounds__(kTileThreads, 4) ssim_tile_kernel(
    const float* __restrict__ a, const float* __restrict__ b, long long n1, long long n2,
    long long c0, long long c1n, long long c2n, float k1, float k2, double* part) {
  using G = SsimGeo<WIN, STEP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  auto& sm = *reinterpret_cast<SsimSmem<WIN, STEP, IS3D>*>(smraw);
  __shared__ double red[32];
  const int t = threadIdx.x;
  const long long plane = n1 * n2;
  const long long y0 = (long long)blockIdx.y * (STEP * kWY);
  const long long x0 = (long long)blockIdx.x * (STEP * kWX);
  const long long wz0 = IS3D ? (long long)blockIdx.z * kZC : 0;
  const long long wz1 = IS3D ? min(wz0 + kZC, c0) : 1;
  const int nplanes = IS3D ? (int)(STEP * (wz1 - wz0 - 1) + WIN) : 1;
  const long long z0 = STEP * wz0;
  const float c = __ldg(a + z0 * plane + y0 * n2 + x0);   // shift for the moments of a
  constexpr float kInvN = 1.0f / (float)(WIN * WIN * (IS3D ? WIN : 1));

  // this thread's window column
  const int wyl = t / kWX, wxl = t % kWX;
  const bool col_ok = (y0 / STEP + wyl) < c1n && (x0 / STEP + wxl) < c2n;

  // The plane tile moves in 16-byte chunks: a chunk inside the field (rows
  // on 16-byte boundaries) is one vector load per array, one crossing the
  // field's last column takes scalar loads, the rest is zero.
  const bool vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0 &&
                   (n2 & 3) == 0;
  float4 px[G::LPT], py[G::LPT];
  auto load_plane = [&](int p) {
    const long long zb = (z0 + p) * plane;
#pragma unroll
    for (int i = 0; i < G::LPT; ++i) {
      const int e = t + i * kTileThreads;
      const int r = e / G::EX4, c4 = e - (e / G::EX4) * G::EX4;
      const long long y = y0 + r, x = x0 + 4 * c4;
      px[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      py[i] = px[i];
      if (e < G::NCH && y < n1 && x < n2) {
        const long long idx = zb + y * n2 + x;
        if (vec && x + 3 < n2) {
          px[i] = __ldg(reinterpret_cast<const float4*>(a + idx));
          py[i] = __ldg(reinterpret_cast<const float4*>(b + idx));
        } else {
          px[i].x = __ldg(a + idx);
          py[i].x = __ldg(b + idx);
          if (x + 1 < n2) px[i].y = __ldg(a + idx + 1), py[i].y = __ldg(b + idx + 1);
          if (x + 2 < n2) px[i].z = __ldg(a + idx + 2), py[i].z = __ldg(b + idx + 2);
          if (x + 3 < n2) px[i].w = __ldg(a + idx + 3), py[i].w = __ldg(b + idx + 3);
        }
      }
    }
  };

  float diss = 0.f;
  float prev[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // the last even plane's sums (step 2)
  load_plane(0);
  for (int p = 0; p < nplanes; ++p) {
#pragma unroll
    for (int i = 0; i < G::LPT; ++i) {
      const int e = t + i * kTileThreads;
      if (e < G::NCH) {
        const int r = e / G::EX4, c4 = e - (e / G::EX4) * G::EX4;
        float* xd = sm.xs + r * G::EXP + 4 * c4;
        float* yd = sm.ys + r * G::EXP + 4 * c4;
        xd[0] = px[i].x, xd[1] = px[i].y, xd[2] = px[i].z, xd[3] = px[i].w;
        yd[0] = py[i].x, yd[1] = py[i].y, yd[2] = py[i].z, yd[3] = py[i].w;
      }
    }
    __syncthreads();
    if (p + 1 < nplanes) load_plane(p + 1);   // in flight during this plane's sums

    // x pass: kG windows of one input row per task, five moments each
    if (t < G::NXT) {
      const int r = t % G::EY, g = t / G::EY;
      const float* xr = sm.xs + r * G::EXP + g * (kG * STEP);
      const float* yr = sm.ys + r * G::EXP + g * (kG * STEP);
      auto moments = [&](int j, float mo[5]) {
        const float xv = xr[j], yv = yr[j];
        const float u = __fsub_rn(xv, c);
        const float d = __fsub_rn(yv, xv);
        mo[0] = u;
        mo[1] = d;
        mo[2] = __fmul_rn(u, u);
        mo[3] = __fmul_rn(d, d);
        mo[4] = __fmul_rn(u, d);
      };
      if constexpr (STEP == 2 && WIN == 7) {
        // window k = the pairs (2k, 2k+1), (2k+2, 2k+3), (2k+4, 2k+5) and
        // point 2k+6; each pair is formed once and serves up to three windows
        float pr[3][5];  // the last three pairs, oldest first
        float ev[5];
#pragma unroll
        for (int j = 0; j < G::SPAN; ++j) {
          float mo[5];
          moments(j, mo);
          if (j % 2 == 0) {
            if (j >= 6) {
              const int k = (j - 6) / 2;
#pragma unroll
              for (int m = 0; m < 5; ++m)
                sm.h[m][r][g * kG + k] =
                    __fadd_rn(__fadd_rn(__fadd_rn(pr[0][m], pr[1][m]), pr[2][m]), mo[m]);
            }
#pragma unroll
            for (int m = 0; m < 5; ++m) ev[m] = mo[m];
          } else {
#pragma unroll
            for (int m = 0; m < 5; ++m) {
              pr[0][m] = pr[1][m];
              pr[1][m] = pr[2][m];
              pr[2][m] = __fadd_rn(ev[m], mo[m]);
            }
          }
        }
      } else {
        float acc[kG][5];
#pragma unroll
        for (int k = 0; k < kG; ++k)
#pragma unroll
          for (int m = 0; m < 5; ++m) acc[k][m] = 0.f;
#pragma unroll
        for (int j = 0; j < G::SPAN; ++j) {
          float mo[5];
          moments(j, mo);
#pragma unroll
          for (int k = 0; k < kG; ++k)
            if (j >= STEP * k && j < STEP * k + WIN)
#pragma unroll
              for (int m = 0; m < 5; ++m) acc[k][m] = __fadd_rn(acc[k][m], mo[m]);
        }
#pragma unroll
        for (int k = 0; k < kG; ++k)
#pragma unroll
          for (int m = 0; m < 5; ++m) sm.h[m][r][g * kG + k] = acc[k][m];
      }
    }
    __syncthreads();

    // y pass: one window column per thread
    float s[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      float v = sm.h[m][STEP * wyl][wxl];
#pragma unroll
      for (int j = 1; j < WIN; ++j) v = __fadd_rn(v, sm.h[m][STEP * wyl + j][wxl]);
      s[m] = v;
    }
    bool window = true;
    if constexpr (IS3D && STEP == 2 && WIN == 7) {
      // window k spans planes 2k .. 2k + 6: the pairs formed at planes
      // 2k + 1, 2k + 3, 2k + 5 and plane 2k + 6 itself
      if (p & 1) {
        const int slot = (p >> 1) % 3;
#pragma unroll
        for (int m = 0; m < 5; ++m) sm.ring[slot][m][t] = __fadd_rn(prev[m], s[m]);
        window = false;
      } else {
        window = p >= 6;
        const int h0 = (p >> 1) % 3, h1 = (h0 + 1) % 3, h2 = (h0 + 2) % 3;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          prev[m] = s[m];
          if (window)
            s[m] = __fadd_rn(
                __fadd_rn(__fadd_rn(sm.ring[h0][m][t], sm.ring[h1][m][t]), sm.ring[h2][m][t]),
                s[m]);
        }
      }
    } else if constexpr (IS3D) {
      const int slot = p % WIN;
#pragma unroll
      for (int m = 0; m < 5; ++m) sm.ring[slot][m][t] = s[m];
      window = p >= WIN - 1 && (p - (WIN - 1)) % STEP == 0;
      if (window) {
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          float v = 0.f;
#pragma unroll
          for (int j = 0; j < WIN; ++j) v = __fadd_rn(v, sm.ring[j][m][t]);
          s[m] = v;
        }
      }
    }
    if (window && col_ok) {
      const float mu = s[0] * kInvN, md = s[1] * kInvN;
      const float vx = s[2] * kInvN - mu * mu;
      const float vd = s[3] * kInvN - md * md;
      const float cxd = s[4] * kInvN - mu * md;
      const float mx = c + mu, my = mx + md;
      const float vy = vx + 2.f * cxd + vd;
      const float A = md * md / (mx * mx + my * my + k1);
      const float B = vd / (vx + vy + k2);
      diss += A + B - A * B;
    }
  }
  const double tot = block_sum((double)diss, red);
  if (t == 0)
    part[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot;
}

// Any other window edge / step: one window per thread iteration, moments in
// double, 1 - SSIM_w accumulated.
constexpr int kSsimThreads = 256;
constexpr int kSsimBlocks = 152 * 8;

__global__ void __launch_bounds__(kSsimThreads) ssim_direct_kernel(
    const float* __restrict__ a, const float* __restrict__ b, long long n0, long long n1,
    long long n2, int win, int wz, int step, long long c0, long long c1n, long long c2n,
    double k1, double k2, double* part) {
  __shared__ double sh[32];
  const long long nwin = c0 * c1n * c2n;
  const double npts = (double)win * (double)win * (double)wz;
  double acc = 0.0;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nwin;
       w += (long long)gridDim.x * blockDim.x) {
    const long long w2 = w % c2n;
    const long long r = w / c2n;
    const long long w1 = r % c1n;
    const long long w0 = r / c1n;
    double sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
    for (int i = 0; i < wz; ++i)
      for (int j = 0; j < win; ++j) {
        const long long base = ((w0 * step + i) * n1 + (w1 * step + j)) * n2 + w2 * step;
        for (int k = 0; k < win; ++k) {
          const double xv = a[base + k], yv = b[base + k];
          sx += xv;
          sy += yv;
          sxx += xv * xv;
          syy += yv * yv;
          sxy += xv * yv;
        }
      }
    const double mx = sx / npts, my = sy / npts;
    const double vx = sxx / npts - mx * mx;
    const double vy = syy / npts - my * my;
    const double cxy = sxy / npts - mx * my;
    acc += 1.0 - ((2.0 * mx * my + k1) * (2.0 * cxy + k2)) /
                     ((mx * mx + my * my + k1) * (vx + vy + k2));
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

struct SsimPlan {
  long long c0, c1, c2;
  bool tiled;
  dim3 grid;
  int parts;
};

SsimPlan plan_ssim(const long long dims[3], bool is3d, int win, int step) {
  SsimPlan p;
  auto cnt = [&](long long n) { return n >= win ? (n - win) / step + 1 : 0; };
  p.c0 = is3d ? cnt(dims[0]) : 1;
  p.c1 = cnt(dims[1]);
  p.c2 = cnt(dims[2]);
  p.tiled = win == 7 && (step == 1 || step == 2);
  if (p.tiled) {
    p.grid = dim3((unsigned)((p.c2 + kWX - 1) / kWX), (unsigned)((p.c1 + kWY - 1) / kWY),
                  (unsigned)(is3d ? (p.c0 + kZC - 1) / kZC : 1));
    p.parts = (p.c0 * p.c1 * p.c2 == 0) ? 0 : (int)(p.grid.x * p.grid.y * p.grid.z);
  } else {
    p.grid = dim3(kSsimBlocks);
    p.parts = kSsimBlocks;
  }
  return p;
}

template <int WIN, int STEP, bool IS3D>
cudaError_t launch_tile(const float* a, const float* b, const long long dims[3],
                        const SsimPlan& p, float k1, float k2, double* part, cudaStream_t s) {
  const size_t smem = sizeof(SsimSmem<WIN, STEP, IS3D>);
  auto kern = ssim_tile_kernel<WIN, STEP, IS3D>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<p.grid, kTileThreads, smem, s>>>(a, b, dims[1], dims[2], p.c0, p.c1, p.c2, k1, k2,
                                           part);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace

int err_metric_blocks() { return kErrBlocks; }

int ssim_parts(const long long dims[3], bool is3d, int win, int step) {
  return plan_ssim(dims, is3d, win, step).parts;
}

cudaError_t launch_err_metrics(const float* a, const float* b, long long n, double* part_sse,
                               double* part_max, double* part_ac, cudaStream_t s) {
  err_kernel<<<kErrBlocks, kErrThreads, 0, s>>>(a, b, n, part_sse, part_max, part_ac);
  note_launch(1);
  return cudaGetLastError();
}

int ac_parts() { return kAcParts * kErrBlocks; }

cudaError_t launch_autocorr(const float* a, const float* b, long long n, long long k,
                            double* part, cudaStream_t s) {
  ac_kernel<<<kErrBlocks, kErrThreads, 0, s>>>(a, b, n, k, part);
  note_launch(1);
  return cudaGetLastError();
}

// Eq. (ac) from the per-CTA sums (host, double): mu = S1 / n,
// sigma^2 = S2 / n - mu^2, covariance = (Sk - mu (head + tail)) / P + mu^2
// over the P = n - k pairs.  A variance below 1e-6 of the mean square (all
// errors equal up to rounding) gives 0, as an exact zero variance does.
double autocorr_from_parts(const double* h, long long n, long long k) {
  double v[kAcParts] = {0, 0, 0, 0, 0};
  for (int j = 0; j < kAcParts; ++j)
    for (int i = 0; i < kErrBlocks; ++i) v[j] += h[(size_t)j * kErrBlocks + i];
  const long long P = n - k;
  if (n <= 0 || P <= 0) return 0.0;
  const double mu = v[0] / (double)n, ms = v[1] / (double)n;
  const double var = ms - mu * mu;
  if (!(var > 1e-6 * ms)) return 0.0;
  const double cov = (v[2] - mu * (v[3] + v[4])) / (double)P + mu * mu;
  return cov / var;
}

cudaError_t launch_ssim(const float* a, const float* b, const long long dims[3], bool is3d,
                        int win, int step, double c1, double c2, double* part_diss,
                        cudaStream_t s) {
  const SsimPlan p = plan_ssim(dims, is3d, win, step);
  if (p.parts == 0) return cudaSuccess;
  if (p.tiled) {
    const float k1 = (float)c1, k2 = (float)c2;
    if (step == 2)
      return is3d ? launch_tile<7, 2, true>(a, b, dims, p, k1, k2, part_diss, s)
                  : launch_tile<7, 2, false>(a, b, dims, p, k1, k2, part_diss, s);
    return is3d ? launch_tile<7, 1, true>(a, b, dims, p, k1, k2, part_diss, s)
                : launch_tile<7, 1, false>(a, b, dims, p, k1, k2, part_diss, s);
  }
  const int wz = is3d ? win : 1;
  ssim_direct_kernel<<<p.parts, kSsimThreads, 0, s>>>(a, b, dims[0], dims[1], dims[2], win, wz,
                                                      step, p.c0, p.c1, p.c2, c1, c2,
                                                      part_diss);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace qoz
