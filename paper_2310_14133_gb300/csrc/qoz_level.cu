// One level of the QoZ interpolation predictor (Sec. 5.1, Sec. 5.2.2) as a
// shared-memory tile kernel, for compression and its mirror.
//
// A launch handles the finest level of a grid G (see LevelGeom).  Each CTA
// owns a tile of G and computes the level's three dimension passes for it:
//   pass 1 (axis u): targets with u odd, v and w even; neighbours are coarse
//                    points, read from the compact coarse reconstruction;
//   pass 2 (axis v): targets with v odd, w even, any u; neighbours are
//                    coarse or pass-1 points in the same u-plane;
//   pass 3 (axis w): targets with w odd; neighbours are even-w points of the
//                    same (u, v) line.
// Pass 2 reads +-3 along v and pass 3 +-3 along w, so the shared tile carries
// a 3-point halo along v and w; the halo's pass-1/pass-2 points are computed
// again by each tile that needs them.  That recomputation is bit-identical:
// same inputs, same operations, same order.  Along u nothing beyond the tile
// is needed except coarse values, which pass 1 reads from global memory.
#include <cuda_runtime.h>

#include "qoz_internal.h"

namespace qoz {
namespace {

template <bool DECOMP>
__global__ void __launch_bounds__(512) level_kernel(
    const LevelGeom G, const float* __restrict__ x, uint16_t* __restrict__ codes,
    const float* __restrict__ rc, float* __restrict__ rout, const BoundTable* __restrict__ bt,
    const UnpredList ul, const long long* __restrict__ uidx, const float* __restrict__ uval,
    const long long nu, int* __restrict__ err) {
  extern __shared__ float S[];
  const int T0 = G.T[0], T1 = G.T[1], T2 = G.T[2];
  const int E1 = T1 + 2 * kHalo, E2 = T2 + 2 * kHalo;
  const long long g0 = G.g[0], g1 = G.g[1], g2 = G.g[2];

  long long b = blockIdx.x;
  long long tp[3];
  tp[2] = b % G.nt[2];
  b /= G.nt[2];
  tp[1] = b % G.nt[1];
  tp[0] = b / G.nt[1];
  const long long o0 = tp[G.phys_of[0]] * T0;
  const long long o1 = tp[G.phys_of[1]] * T1;
  const long long o2 = tp[G.phys_of[2]] * T2;

  const int lvl = G.level - 1;
  const float el = bt->el[lvl];
  const float two_e = bt->two_e[lvl];
  const float inv = bt->inv[lvl];
  const int interp = G.interp;

  // ---- load: coarse values from the compact coarse grid, field values (or
  // codes) at the targets this tile computes.  Physical-x-fastest order keeps
  // the global reads coalesced whatever the dimension order.
  {
    int lo[3], ext[3];
    lo[0] = 0;
    ext[0] = T0;
    lo[1] = lo[2] = -kHalo;
    ext[1] = E1;
    ext[2] = E2;
    const int pe0 = ext[G.ord_of[0]], pe1 = ext[G.ord_of[1]], pe2 = ext[G.ord_of[2]];
    const int pl0 = lo[G.ord_of[0]], pl1 = lo[G.ord_of[1]], pl2 = lo[G.ord_of[2]];
    const int total = pe0 * pe1 * pe2;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int q2 = i % pe2;
      const int r = i / pe2;
      const int q1 = r % pe1;
      const int q0 = r / pe1;
      int lp[3];
      lp[0] = q0 + pl0;
      lp[1] = q1 + pl1;
      lp[2] = q2 + pl2;
      const int lu = lp[G.phys_of[0]], lv = lp[G.phys_of[1]], lw = lp[G.phys_of[2]];
      const long long cu = o0 + lu, cv = o1 + lv, cw = o2 + lw;
      if (cu < 0 || cu >= g0 || cv < 0 || cv >= g1 || cw < 0 || cw >= g2) continue;
      const int si = (lu * E1 + (lv + kHalo)) * E2 + (lw + kHalo);
      const bool ev = !(cv & 1), ew = !(cw & 1);
      if (!(cu & 1) && ev && ew) {
        S[si] = rc[(cu >> 1) * G.cs[0] + (cv >> 1) * G.cs[1] + (cw >> 1) * G.cs[2]];
        continue;
      }
      const bool in_v = lv >= 0 && lv < T1, in_w = lw >= 0 && lw < T2;
      bool need;
      if (ev && ew)
        need = true;          // pass-1 target, needed over the whole halo
      else if (ew)
        need = in_v;          // pass-2 target, needed over the w halo
      else
        need = in_v && in_w;  // pass-3 target, tile proper only
      if (!need) continue;
      const long long xi = cu * G.xs[0] + cv * G.xs[1] + cw * G.xs[2];
      if (DECOMP)
        S[si] = (float)codes[xi];
      else
        S[si] = x[xi];
    }
  }
  __syncthreads();

  // Final value of a target given its prediction: quantize (compress) or
  // dequantize (decompress).  emit: the target belongs to this tile.
  auto finish = [&](int si, float pred, long long xi, bool emit) {
    if (DECOMP) {
      const int code = (int)S[si];
      float v;
      if (code == 0) {
        if (!unpred_lookup(uidx, uval, nu, xi, &v)) {
          v = 0.0f;
          atomicOr(err, 1);
        }
      } else {
        v = dequantize(pred, code, two_e);
      }
      S[si] = v;
    } else {
      const float xv = S[si];
      uint16_t code;
      float rec;
      if (quantize(xv, pred, el, two_e, inv, &code, &rec)) {
        S[si] = rec;
      } else {
        code = 0;
        if (emit) unpred_append(ul, xi, xv);
      }
      if (emit) codes[xi] = code;
    }
  };

  // ---- pass 1 (along u): u odd, v and w even over the whole v/w halo
  {
    const int nu_ = T0 / 2, nv = T1 / 2 + 3, nw = T2 / 2 + 3;
    const int total = nu_ * nv * nw;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int wi = i % nw;
      const int r = i / nw;
      const int vi = r % nv;
      const int ui = r / nv;
      const int lu = 2 * ui + 1, lv = 2 * vi - 2, lw = 2 * wi - 2;
      const long long cu = o0 + lu, cv = o1 + lv, cw = o2 + lw;
      if (cu >= g0 || cv < 0 || cv >= g1 || cw < 0 || cw >= g2) continue;
      const long long cb = (cv >> 1) * G.cs[1] + (cw >> 1) * G.cs[2];
      const long long ca = (cu - 1) >> 1;
      const bool hb1 = cu + 1 < g0, ha3 = cu >= 3, hb3 = cu + 3 < g0;
      const float a1 = rc[cb + ca * G.cs[0]];
      const float b1 = hb1 ? rc[cb + (ca + 1) * G.cs[0]] : 0.0f;
      const float a3 = ha3 ? rc[cb + (ca - 1) * G.cs[0]] : 0.0f;
      const float b3 = hb3 ? rc[cb + (ca + 2) * G.cs[0]] : 0.0f;
      const float pred = predict(a3, a1, b1, b3, ha3, hb1, hb3, interp);
      const int si = (lu * E1 + (lv + kHalo)) * E2 + (lw + kHalo);
      const long long xi = cu * G.xs[0] + cv * G.xs[1] + cw * G.xs[2];
      finish(si, pred, xi, lv >= 0 && lv < T1 && lw >= 0 && lw < T2);
    }
  }
  __syncthreads();

  // ---- pass 2 (along v): v odd inside the tile, w even over the w halo
  {
    const int nv = T1 / 2, nw = T2 / 2 + 3;
    const int total = T0 * nv * nw;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int wi = i % nw;
      const int r = i / nw;
      const int vi = r % nv;
      const int lu = r / nv;
      const int lv = 2 * vi + 1, lw = 2 * wi - 2;
      const long long cu = o0 + lu, cv = o1 + lv, cw = o2 + lw;
      if (cu >= g0 || cv >= g1 || cw < 0 || cw >= g2) continue;
      const int si = (lu * E1 + (lv + kHalo)) * E2 + (lw + kHalo);
      const bool hb1 = cv + 1 < g1, ha3 = cv >= 3, hb3 = cv + 3 < g1;
      const float a1 = S[si - E2];
      const float b1 = hb1 ? S[si + E2] : 0.0f;
      const float a3 = ha3 ? S[si - 3 * E2] : 0.0f;
      const float b3 = hb3 ? S[si + 3 * E2] : 0.0f;
      const float pred = predict(a3, a1, b1, b3, ha3, hb1, hb3, interp);
      const long long xi = cu * G.xs[0] + cv * G.xs[1] + cw * G.xs[2];
      finish(si, pred, xi, lw >= 0 && lw < T2);
    }
  }
  __syncthreads();

  // ---- pass 3 (along w): w odd inside the tile
  {
    const int nw = T2 / 2;
    const int total = T0 * T1 * nw;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int wi = i % nw;
      const int r = i / nw;
      const int lv = r % T1;
      const int lu = r / T1;
      const int lw = 2 * wi + 1;
      const long long cu = o0 + lu, cv = o1 + lv, cw = o2 + lw;
      if (cu >= g0 || cv >= g1 || cw >= g2) continue;
      const int si = (lu * E1 + (lv + kHalo)) * E2 + (lw + kHalo);
      const bool hb1 = cw + 1 < g2, ha3 = cw >= 3, hb3 = cw + 3 < g2;
      const float a1 = S[si - 1];
      const float b1 = hb1 ? S[si + 1] : 0.0f;
      const float a3 = ha3 ? S[si - 3] : 0.0f;
      const float b3 = hb3 ? S[si + 3] : 0.0f;
      const float pred = predict(a3, a1, b1, b3, ha3, hb1, hb3, interp);
      const long long xi = cu * G.xs[0] + cv * G.xs[1] + cw * G.xs[2];
      finish(si, pred, xi, true);
    }
  }

  // ---- reconstruction of the tile (coarse points included) to the compact
  // output grid, physical-x fastest for coalesced stores
  if (rout != nullptr) {
    __syncthreads();
    int ext[3] = {T0, T1, T2};
    const int pe0 = ext[G.ord_of[0]], pe1 = ext[G.ord_of[1]], pe2 = ext[G.ord_of[2]];
    const int total = pe0 * pe1 * pe2;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int q2 = i % pe2;
      const int r = i / pe2;
      const int q1 = r % pe1;
      const int q0 = r / pe1;
      int lp[3] = {q0, q1, q2};
      const int lu = lp[G.phys_of[0]], lv = lp[G.phys_of[1]], lw = lp[G.phys_of[2]];
      const long long cu = o0 + lu, cv = o1 + lv, cw = o2 + lw;
      if (cu >= g0 || cv >= g1 || cw >= g2) continue;
      const int si = (lu * E1 + (lv + kHalo)) * E2 + (lw + kHalo);
      rout[cu * G.os[0] + cv * G.os[1] + cw * G.os[2]] = S[si];
    }
  }
}

__global__ void anchor_gather_kernel(const float* __restrict__ x, uint16_t* __restrict__ codes,
                                     float* __restrict__ anchors, long long na0, long long na1,
                                     long long na2, long long fst0, long long fst1,
                                     long long stride) {
  const long long n = na0 * na1 * na2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long i2 = i % na2;
    const long long r = i / na2;
    const long long i1 = r % na1;
    const long long i0 = r / na1;
    const long long full = stride * (i0 * fst0 + i1 * fst1 + i2);
    anchors[i] = x[full];
    codes[full] = 0;
  }
}

// The opt-in dynamic shared memory limit is a per-device function attribute:
// set it once per (device, kernel).
constexpr size_t kMaxLevelSmem = 200 * 1024;

cudaError_t ensure_smem_attr(const void* fn, int which) {
  static unsigned long long done[2] = {0, 0};  // bit per device ordinal
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done[which], __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxLevelSmem);
  if (e == cudaSuccess) __atomic_fetch_or(&done[which], bit, __ATOMIC_ACQ_REL);
  return e;
}

}  // namespace

size_t level_smem_bytes(const LevelGeom& G) {
  return sizeof(float) * (size_t)G.T[0] * (G.T[1] + 2 * kHalo) * (G.T[2] + 2 * kHalo);
}

cudaError_t launch_level(bool decompress, const LevelGeom& G, const float* x, uint16_t* codes,
                         const float* rc, float* rout, const BoundTable* bt, UnpredList ul,
                         const long long* uidx, const float* uval, long long nu, int* err,
                         cudaStream_t s) {
  const long long nblocks = G.nt[0] * G.nt[1] * G.nt[2];
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const size_t smem = level_smem_bytes(G);
  if (smem > kMaxLevelSmem) return cudaErrorInvalidConfiguration;
  const void* fn = decompress ? (const void*)level_kernel<true> : (const void*)level_kernel<false>;
  cudaError_t e = ensure_smem_attr(fn, decompress ? 1 : 0);
  if (e != cudaSuccess) return e;
  const int threads = 512;
  if (decompress)
    level_kernel<true><<<(unsigned)nblocks, threads, smem, s>>>(G, x, codes, rc, rout, bt, ul,
                                                                uidx, uval, nu, err);
  else
    level_kernel<false><<<(unsigned)nblocks, threads, smem, s>>>(G, x, codes, rc, rout, bt, ul,
                                                                 uidx, uval, nu, err);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_anchor_gather(const float* x, uint16_t* codes, float* anchors,
                                 const long long na[3], const long long fst[3], long long stride,
                                 cudaStream_t s) {
  const long long n = na[0] * na[1] * na[2];
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  anchor_gather_kernel<<<(unsigned)blocks, threads, 0, s>>>(x, codes, anchors, na[0], na[1],
                                                            na[2], fst[0], fst[1], stride); note_launch(1);
  return cudaGetLastError();
}

}  // namespace qoz
