// Quality metrics of Sec. 3: max abs error, MSE / PSNR (Eq. psnr) and SSIM
// (Eq. ssim, Eq. ssim2).  Per-CTA partial sums are combined on the host in a
// fixed order, so every result is deterministic.
//
// Arithmetic.  The maximum error is exact: the binary32 difference |a - b| is
// a monotone rounding of the exact one, so only elements whose rounded
// difference reaches the running maximum are re-evaluated in double.  The
// squared errors are summed in binary32 with compensation (Kahan), per
// thread, then in double across threads.
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
constexpr int kErrBlocks = 152 * 4;

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

__device__ __forceinline__ void err_point(float av, float bv, float& mxf, double& mxd,
                                          int& nans, Kahan& sse) {
  const float d = __fsub_rn(av, bv);
  const float ad = fabsf(d);
  if (ad != ad) {
    ++nans;
  } else if (ad >= mxf) {  // candidate: the exact maximum always passes this test
    mxf = ad;
    mxd = fmax(mxd, fabs((double)av - (double)bv));
  }
  sse.add(__fmul_rn(d, d));
}

__global__ void __launch_bounds__(kErrThreads) err_kernel(const float* __restrict__ a,
                                                          const float* __restrict__ b,
                                                          long long n, double* part_sse,
                                                          double* part_max) {
  __shared__ double sh[32];
  float mxf = 0.f;
  double mxd = 0.0;
  int nans = 0;
  Kahan sse;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
  long long i0 = 0;
  if (vec) {
    const long long n4 = n >> 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    for (long long i = tid; i < n4; i += nthr) {
      const float4 u = __ldcs(a4 + i), v = __ldcs(b4 + i);
      err_point(u.x, v.x, mxf, mxd, nans, sse);
      err_point(u.y, v.y, mxf, mxd, nans, sse);
      err_point(u.z, v.z, mxf, mxd, nans, sse);
      err_point(u.w, v.w, mxf, mxd, nans, sse);
    }
    i0 = n4 << 2;
  }
  for (long long i = i0 + tid; i < n; i += nthr) err_point(a[i], b[i], mxf, mxd, nans, sse);
  const double s = block_sum((double)sse.s - (double)sse.c, sh);
  const double m = block_max(mxd, sh);
  const double nn = block_sum((double)nans, sh);  // a NaN difference makes the max NaN
  if (threadIdx.x == 0) {
    part_sse[blockIdx.x] = s;
    part_max[blockIdx.x] = nn > 0.0 ? __longlong_as_double(0x7ff8000000000000LL) : m;
  }
}

// ---------------------------------------------------------------- Eq. (ac)
// Lag-k autocorrelation of the errors e_i = b_i - a_i over the flattened
// arrays: one pass accumulating sum e, sum e^2, sum e_i e_{i+k} over the
// n - k pairs and the sums of the pairs' first and second members, each in
// compensated binary32 per thread and double across threads; the host forms
// the mean, the variance and the lag covariance from them.
constexpr int kAcParts = 5;

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
  static constexpr int EXP = EX | 1;                  // odd row pitch
  static constexpr int NIN = EY * EX;
  static constexpr int LPT = (NIN + kTileThreads - 1) / kTileThreads;
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
  float h[5][G::EY][kWX];
  float ring[IS3D ? WIN : 1][5][kTileThreads];
};

template <int WIN, int STEP, bool IS3D>
__global__ void __launch_bounds__(kTileThreads) ssim_tile_kernel(
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

  float px[G::LPT], py[G::LPT];
  auto load_plane = [&](int p) {
    const long long zb = (z0 + p) * plane;
#pragma unroll
    for (int i = 0; i < G::LPT; ++i) {
      const int e = t + i * kTileThreads;
      const int r = e / G::EX, cc = e - (e / G::EX) * G::EX;
      const long long y = y0 + r, x = x0 + cc;
      px[i] = 0.f;
      py[i] = 0.f;
      if (e < G::NIN && y < n1 && x < n2) {
        const long long idx = zb + y * n2 + x;
        px[i] = __ldg(a + idx);
        py[i] = __ldg(b + idx);
      }
    }
  };

  float diss = 0.f;
  load_plane(0);
  for (int p = 0; p < nplanes; ++p) {
#pragma unroll
    for (int i = 0; i < G::LPT; ++i) {
      const int e = t + i * kTileThreads;
      if (e < G::NIN) {
        const int r = e / G::EX, cc = e - (e / G::EX) * G::EX;
        sm.xs[r * G::EXP + cc] = px[i];
        sm.ys[r * G::EXP + cc] = py[i];
      }
    }
    __syncthreads();
    if (p + 1 < nplanes) load_plane(p + 1);   // in flight during this plane's sums

    // x pass: kG windows of one input row per task, five moments each
    if (t < G::NXT) {
      const int r = t % G::EY, g = t / G::EY;
      const float* xr = sm.xs + r * G::EXP + g * (kG * STEP);
      const float* yr = sm.ys + r * G::EXP + g * (kG * STEP);
      float acc[kG][5];
#pragma unroll
      for (int k = 0; k < kG; ++k)
#pragma unroll
        for (int m = 0; m < 5; ++m) acc[k][m] = 0.f;
#pragma unroll
      for (int j = 0; j < G::SPAN; ++j) {
        const float xv = xr[j], yv = yr[j];
        const float u = __fsub_rn(xv, c);
        const float d = __fsub_rn(yv, xv);
        const float mo[5] = {u, d, __fmul_rn(u, u), __fmul_rn(d, d), __fmul_rn(u, d)};
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
    __syncthreads();

    // y pass: one window column per thread
    float s[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      float v = 0.f;
#pragma unroll
      for (int j = 0; j < WIN; ++j) v = __fadd_rn(v, sm.h[m][STEP * wyl + j][wxl]);
      s[m] = v;
    }
    bool window = true;
    if constexpr (IS3D) {
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
                               double* part_max, int nparts, cudaStream_t s) {
  err_kernel<<<nparts, kErrThreads, 0, s>>>(a, b, n, part_sse, part_max); note_launch(1);
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
