// Quality metrics of Sec. 3: max abs error, MSE / PSNR (Eq. psnr) and SSIM
// (Eq. ssim, Eq. ssim2).  Differences and products are formed in double
// (exact for binary32 inputs); per-CTA partial sums are combined on the host
// in a fixed order.
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

__global__ void __launch_bounds__(kErrThreads) err_kernel(const float* __restrict__ a,
                                                          const float* __restrict__ b,
                                                          long long n, double* part_sse,
                                                          double* part_max) {
  __shared__ double sh[32];
  double sse = 0.0, mx = 0.0, nans = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double d = (double)a[i] - (double)b[i];
    sse += d * d;
    const double ad = fabs(d);
    if (ad != ad)
      nans += 1.0;
    else
      mx = fmax(mx, ad);
  }
  const double s = block_sum(sse, sh);
  const double m = block_max(mx, sh);
  const double nn = block_sum(nans, sh);  // a NaN difference makes the max NaN
  if (threadIdx.x == 0) {
    part_sse[blockIdx.x] = s;
    part_max[blockIdx.x] = nn > 0.0 ? __longlong_as_double(0x7ff8000000000000LL) : m;
  }
}

constexpr int kSsimThreads = 256;
constexpr int kSsimBlocks = 152 * 8;

// One window per thread iteration: the five moments over the win^d box.
__global__ void __launch_bounds__(kSsimThreads) ssim_kernel(
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
    acc += ((2.0 * mx * my + k1) * (2.0 * cxy + k2)) /
           ((mx * mx + my * my + k1) * (vx + vy + k2));
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

}  // namespace

int err_metric_blocks() { return kErrBlocks; }
int ssim_blocks() { return kSsimBlocks; }

cudaError_t launch_err_metrics(const float* a, const float* b, long long n, double* part_sse,
                               double* part_max, int nparts, cudaStream_t s) {
  err_kernel<<<nparts, kErrThreads, 0, s>>>(a, b, n, part_sse, part_max); note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_ssim(const float* a, const float* b, const long long dims[3], bool is3d,
                        int win, int step, double c1, double c2, double* part_sum, int nparts,
                        cudaStream_t s) {
  const int wz = is3d ? win : 1;
  auto cnt = [&](long long n) { return n >= win ? (n - win) / step + 1 : 0; };
  const long long c0 = is3d ? cnt(dims[0]) : 1;
  const long long cy = cnt(dims[1]), cx = cnt(dims[2]);
  ssim_kernel<<<nparts, kSsimThreads, 0, s>>>(a, b, dims[0], dims[1], dims[2], win, wz, step, c0,
                                              cy, cx, c1, c2, part_sum); note_launch(1);
  return cudaGetLastError();
}

}  // namespace qoz
