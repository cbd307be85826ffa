// Level 1 of the interpolation predictor on a 3-D field (Sec. 5.1, Sec. 5.2.2)
// as a persistent kernel fed by bulk tensor copies.
//
// Level 1 predicts 7/8 of all points, so it carries most of the cost of a
// compression.  Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x,
// ... of the field.  A tile's input (the field over the tile and its halo,
// the coarse reconstruction box, the tile's coarse codes) arrives by three
// cp.async.bulk.tensor copies on the CTA's mbarrier; the next tile's copies
// are issued as soon as the passes are done with the input, so they land
// while the CTA counts the codes and while the SM's other CTAs (four per SM)
// predict theirs.  The tile's codes leave by one bulk tensor store.
//
// Geometry (axes physical: 0 = z, 1 = y, 2 = x; A0, A1, A2 = the level's
// dimension order):
//   pass 1 along A0: targets odd on A0, even on A1 and A2 (over the halo);
//                    neighbours are coarse points, read from the coarse box,
//                    which pass 1 also copies into the even positions of the
//                    field box (the coarse patch) on its way;
//   pass 2 along A1: targets odd on A1, any on A0, even on A2 (over the halo);
//   pass 3 along A2: targets odd on A2, any on A0 and A1.
// A1 and A2 carry a 3-point halo (the field box spans [-3, T + 3) on a halo
// axis that is z or y and [-4, TX + 4) on x, so that every row starts on a 16-
// byte boundary); halo targets are recomputed bit for bit by every tile that
// needs them.  A pass along z or y gives each work item a segment of a line
// and four consecutive x (or the even x of four), with the line's even
// positions in a register window; a pass along x gives each item four odd x
// of one row.  Every binary32 operation is a separately rounded scalar one
// (the packed f32x2 forms were measured to come out fused with their
// neighbours, which changes the last bit of a reconstruction).
//
// Quantizer fast path: m = floor(|d| inv + 0.5) is formed without a
// conversion (adding 2^23 with rounding toward -inf leaves m in the low
// mantissa bits), and the code q + 32768 is read from the bits of
// q + 2^23 + 32768.  Whenever it accepts a point its result equals
// qoz::quantize bit for bit; when it declines (out of range, bound missed,
// non-finite values, or an infinite 1/(2 e_l)), the point goes through
// qoz::quantize itself.
#pragma once

#include <cuda_runtime.h>

#include "qoz_internal.h"
#include "qoz_tma.cuh"

namespace qoz {
namespace l1 {

constexpr int kThr = 256;
#ifndef QOZ_L1_CTAS
#define QOZ_L1_CTAS 4
#endif
constexpr int kCtasPerSm = QOZ_L1_CTAS;  // resident CTAs per SM (a build-time choice)
// Decompression keeps fewer values per target live and runs faster with the
// registers of three CTAs per SM (measured: 925 against 861 GB/s at 512^3).
#ifndef QOZ_L1_DEC_CTAS
#define QOZ_L1_DEC_CTAS 3
#endif
constexpr int kDecCtasPerSm = QOZ_L1_DEC_CTAS;
constexpr int kHistLo = kRadius - 512;  // shared histogram window [32768 - 512, 32768 + 512)
constexpr int kHistWin = 1024;
constexpr unsigned kPolls = 1u << 24;   // mbarrier polls before a tile gives up

enum Role { kOdd, kAny, kEvenH };

template <int A0_, int A1_, int A2_, int TZ_, int TY_, int TX_>
struct Geo {
  static constexpr int A0 = A0_, A1 = A1_, A2 = A2_;
  static constexpr int TZ = TZ_, TY = TY_, TX = TX_;
  __host__ __device__ static constexpr int T(int p) { return p == 0 ? TZ : (p == 1 ? TY : TX); }
  // halo: none on the first axis; 3 on z / y, 4 on x (16-byte rows)
  static constexpr int HZ = A0 == 0 ? 0 : 3;
  static constexpr int HY = A0 == 1 ? 0 : 3;
  static constexpr int XL = A0 == 2 ? 0 : 4;
  static constexpr int EZ = TZ + 2 * HZ, EY = TY + 2 * HY, EX = TX + 2 * XL;
  static constexpr unsigned a128(unsigned v) { return (v + 127u) & ~127u; }
  static constexpr int kS = EZ * EY * EX;
  __host__ __device__ static constexpr int sidx(int z, int y, int x) {
    return ((z + HZ) * EY + (y + HY)) * EX + x + XL;
  }
  // coarse reconstruction box: coarse coordinates -1 .. T/2 + 1 on z and y,
  // -4 .. TX/2 + 3 on x (its first column on a 16-byte boundary); indexed by
  // even tile-local fine coordinates
  static constexpr int CBZ = TZ / 2 + 3, CBY = TY / 2 + 3, CBX = TX / 2 + 8;
  static constexpr int kCB = CBZ * CBY * CBX;
  __host__ __device__ static constexpr int cbidx(int fz, int fy, int fx) {
    return ((fz / 2 + 1) * CBY + (fy / 2 + 1)) * CBX + fx / 2 + 4;
  }
  // the tile's own coarse codes
  static constexpr int CCZ = TZ / 2, CCY = TY / 2, CCX = TX / 2;
  static constexpr int kCC = CCZ * CCY * CCX;
  __host__ __device__ static constexpr int ccidx(int fz, int fy, int fx) {
    return ((fz / 2) * CCY + fy / 2) * CCX + fx / 2;
  }
  static constexpr int kC = TZ * TY * TX;
  __host__ __device__ static constexpr int cidx(int z, int y, int x) { return (z * TY + y) * TX + x; }
  // decompression's code box: the codes over the field box's extent, its x
  // range widened to [-8, TX + 8) (16-byte rows of 16-bit codes) where x has
  // a halo
  static constexpr int XC = XL ? 8 : 0;
  static constexpr int ECX = TX + 2 * XC;
  static constexpr int kCode = EZ * EY * ECX;
  __host__ __device__ static constexpr int xidx(int z, int y, int x) {
    return ((z + HZ) * EY + (y + HY)) * ECX + x + XC;
  }
  // decompression's shared memory: field box | code box | coarse box
  static constexpr unsigned dCode = a128(4u * kS);
  static constexpr unsigned dCB = dCode + a128(2u * kCode);
  static constexpr unsigned kDecTxBytes = 2u * kCode + 4u * kCB;
  static constexpr unsigned kDecSmem = 128u + dCB + a128(4u * kCB);
  // role of physical axis P in pass PASS
  template <int PASS, int P>
  __host__ __device__ static constexpr int role() {
    return PASS == 1 ? (P == A0 ? kOdd : kEvenH)
                     : (PASS == 2 ? (P == A0 ? kAny : (P == A1 ? kOdd : kEvenH))
                                  : (P == A2 ? kOdd : kAny));
  }
  // shared memory: the tile's input (field box | coarse box | coarse
  // codes), its code buffer, the histogram window
  static constexpr unsigned oCB = a128(4u * kS);
  static constexpr unsigned oCC = oCB + a128(4u * kCB);
  static constexpr unsigned kStage = oCC + a128(2u * kCC);
  static constexpr unsigned kTxBytes = 4u * kS + 4u * kCB + 2u * kCC;
  static constexpr unsigned oC16 = kStage;
  static constexpr unsigned kC16 = a128(2u * kC);
  static constexpr unsigned oHist = oC16 + kC16;
  static constexpr unsigned kSmem = 128u + oHist + 4u * kHistWin;
  static_assert(TX % 16 == 0 && TY % 2 == 0 && TZ % 2 == 0, "tile extents");
};

// Tile of the level-1 launch by the axis the order takes first: the first
// axis carries no halo and gets the short extent.
struct Tile3 {
  int tz, ty, tx;
};
__host__ __device__ constexpr Tile3 tile_for(int a0) {
  return a0 == 0 ? Tile3{8, 16, 32} : (a0 == 1 ? Tile3{16, 8, 32} : Tile3{8, 8, 32});
}

struct Ctx {
  int oz, oy, ox;
  int g0, g1, g2;
  float el, two_e, inv;
  bool full;     // compression: every point of the tile lies inside the field
  unsigned* SH;  // compression: the shared histogram window
};

// ---- arithmetic

// Interpolation with every neighbour present: cubic (-1, 9, 9, -1)/16 or
// linear (1, 1)/2 (the same operations, in the same order, as
// qoz::predict).
template <int IP>
__device__ __forceinline__ float pfull(float a3, float a1, float b1, float b3) {
  if (IP == 1)
    return __fmul_rn(__fsub_rn(__fmul_rn(9.0f, __fadd_rn(a1, b1)), __fadd_rn(a3, b3)), 0.0625f);
  return __fmul_rn(__fadd_rn(a1, b1), 0.5f);
}
// Prediction of a target at coordinate c along the pass axis of extent g:
// the full stencil inside, qoz::predict's border stencils near the edges.
template <int IP, bool BORDER>
__device__ __forceinline__ float pred1(float a3, float a1, float b1, float b3, int c, int g) {
  if (!BORDER) return pfull<IP>(a3, a1, b1, b3);
  return predict(a3, a1, b1, b3, c >= 3, c + 1 < g, c + 3 < g, IP);
}

constexpr float kTwo23 = 8388608.0f;       // 2^23
constexpr float kCodeBias = 8421376.0f;    // 2^23 + 32768

// Fast path of the quantizer (see the file comment).  cbits: the low 16 bits
// are the code.
__device__ __forceinline__ bool qfast(float x, float p, const Ctx& c, float& r, unsigned& cbits) {
  const float d = __fsub_rn(x, p);
  const float u = __fadd_rn(__fmul_rn(fabsf(d), c.inv), 0.5f);
  const float m = __fsub_rn(__fadd_rd(u, kTwo23), kTwo23);
  const float cf = __fadd_rn(copysignf(m, d), kCodeBias);
  const float q = __fsub_rn(cf, kCodeBias);  // q, with +0 for a zero bin
  r = __fadd_rn(p, __fmul_rn(q, c.two_e));
  cbits = __float_as_uint(cf);
  // both checks without a branch between them (the values above are only
  // used when both hold)
  return (u < 32768.0f) & (fabsf(__fsub_rn(x, r)) <= c.el);
}

// Adds one code to the histogram: the shared window around the zero bin,
// the global histogram outside it.
__device__ __forceinline__ void hist_add(const LevelLaunch& a, unsigned* SH, unsigned code) {
  const unsigned kk = code - (unsigned)kHistLo;
  if (kk < (unsigned)kHistWin)
    atomicAdd(&SH[kk], 1u);
  else
    atomicAdd(&a.hist[code], 1u);
}

// Slow path of one point: the reference quantizer; an unpredictable point
// keeps its value, gets code 0 and, when it is a valid point of this tile
// (store), joins the list at its field index (cz, cy, cx).  Returns (bits of
// the reconstruction, code).  The bound and the extents are read again from
// the launch: the rare call holds few of the caller's registers.
static __device__ __noinline__ uint2 qslow(const LevelLaunch& a, float x, float p, bool store, int cz,
                                    int cy, int cx) {
  uint16_t cd;
  float rr;
  if (quantize(x, p, a.bt->el[0], a.bt->two_e[0], a.bt->inv[0], &cd, &rr))
    return make_uint2(__float_as_uint(rr), cd);
  if (store && cz >= 0 && cz < a.g[0] && cy >= 0 && cy < a.g[1] && cx >= 0 && cx < a.g[2]) {
    const long long xi = (long long)((unsigned long long)cz * a.xs[0] +
                                     (unsigned long long)cy * a.xs[1] +
                                     (unsigned long long)cx * a.xs[2]);
    unpred_append(a.ul, xi, x);
  }
  return make_uint2(__float_as_uint(x), 0u);
}

// One point: fast path, else the slow one.
__device__ __forceinline__ void quant1(const LevelLaunch& a, const Ctx& c, float x, float p,
                                       bool store, int lz, int ly, int lx, float& r,
                                       unsigned& code) {
  unsigned cb;
  float rf;
  const bool ok = qfast(x, p, c, rf, cb);
  r = rf;
  code = cb & 0xffffu;
  // the code of a point of this tile joins the histogram here when the
  // tile lies inside the field (other tiles count theirs after the passes):
  // the common case is one predicated shared atomic, and a single rarely
  // taken branch covers the slow quantizer and codes outside the window
  const bool cnt = store & c.full;
  const unsigned kk = code - (unsigned)kHistLo;
  const bool common = ok & (!cnt | (kk < (unsigned)kHistWin));
  if (cnt & common) atomicAdd(&c.SH[kk], 1u);
  if (__builtin_expect(!common, 0)) {
    if (!ok) {
      const uint2 v = qslow(a, x, p, store, c.oz + lz, c.oy + ly, c.ox + lx);
      r = __uint_as_float(v.x);
      code = v.y;
    }
    if (cnt) hist_add(a, c.SH, code);
  }
}

// Two neighbouring points along x (lx, lx + 1); code2 packs their codes.
__device__ __forceinline__ void quant2(const LevelLaunch& a, const Ctx& c, float2 x, float2 p,
                                       bool store, int lz, int ly, int lx, float2& r,
                                       unsigned& code2) {
  unsigned k0, k1;
  quant1(a, c, x.x, p.x, store, lz, ly, lx, r.x, k0);
  quant1(a, c, x.y, p.y, store, lz, ly, lx + 1, r.y, k1);
  code2 = k0 | (k1 << 16);
}

// Decompression of one point whose code is 0: the stored value from the
// sorted unpredictable list (0 and a flag when it is missing; 0 for a halo
// position outside the field, which no valid point reads).
static __device__ __noinline__ float dslow(const LevelLaunch& a, int cz, int cy, int cx) {
  if (cz < 0 || cz >= a.g[0] || cy < 0 || cy >= a.g[1] || cx < 0 || cx >= a.g[2]) return 0.0f;
  const long long xi = (long long)((unsigned long long)cz * a.xs[0] +
                                   (unsigned long long)cy * a.xs[1] +
                                   (unsigned long long)cx * a.xs[2]);
  float v;
  if (!unpred_lookup(a.uidx, a.uval, a.nu, xi, &v)) {
    v = 0.0f;
    if (a.err) atomicOr(a.err, 1);
  }
  return v;
}

// Reconstruction from a code (Sec. 5.1 mirrored): p + (code - 32768) 2 e_l,
// the same operations as qoz::dequantize; (float)(code - 32768) is read from
// the bits of 2^23 + code.
__device__ __forceinline__ float deq1(const LevelLaunch& a, const Ctx& c, unsigned code, float p,
                                      int lz, int ly, int lx) {
  if (code == 0u) return dslow(a, c.oz + lz, c.oy + ly, c.ox + lx);
  const float q = __fsub_rn(__uint_as_float(0x4B000000u | code), kCodeBias);
  return __fadd_rn(p, __fmul_rn(q, c.two_e));
}

// ---- segment length of a line pass: minimises rounds x per-item work
__host__ __device__ constexpr int seg_for(int NT, int lanes) {
  int best = 1;
  long long best_cost = -1;
  for (int s = 1; s <= NT && s <= 4; s *= 2) {
    if (NT % s) continue;
    const long long items = (long long)(NT / s) * lanes;
    const long long rounds = (items + kThr - 1) / kThr;
    const long long cost = rounds * (21LL * s + 3);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = s;
    }
  }
  return best;
}

// ---- a pass along z or y.  R is the other of z and y.  Compression
// (DEC false): CC / C16 are the tile's coarse codes and its code buffer.
// Decompression: CC is the code box and C16 is unused.
template <class G, int PASS, int IP, bool BORDER, bool WREC, bool DEC>
__device__ __forceinline__ void line_pass(const LevelLaunch& a, const Ctx& c, float* S,
                                          const float* CB, const uint16_t* CC, uint16_t* C16) {
  constexpr int P = PASS == 1 ? G::A0 : (PASS == 2 ? G::A1 : G::A2);
  static_assert(P != 2, "x passes use x_pass");
  constexpr int R = 1 - P;
  constexpr int XK = G::template role<PASS, 2>();
  constexpr int RK = G::template role<PASS, R>();
  constexpr bool FROM_CB = PASS == 1;
  static_assert(!FROM_CB || (XK == kEvenH && RK == kEvenH), "pass 1 reads even x and R");
  constexpr int TP = G::T(P), TR = G::T(R);
  constexpr int NT = TP / 2;
  constexpr int NR = RK == kAny ? TR : TR / 2 + 3;
  constexpr int NXC = XK == kAny ? G::TX / 4 : (G::TX + 8) / 4;
  constexpr int SEG = seg_for(NT, NR * NXC);
  constexpr int NSEG = NT / SEG;
  constexpr int items = NSEG * NR * NXC;
  constexpr int SP = P == 0 ? G::EY * G::EX : G::EX;    // field box stride along P
  constexpr int XP = P == 0 ? G::EY * G::ECX : G::ECX;  // code box stride along P
  const int gP = P == 0 ? c.g0 : c.g1;
  const int oP = P == 0 ? c.oz : c.oy;

  for (int it = threadIdx.x; it < items; it += kThr) {
    const int xc = it % NXC;
    const int rest = it / NXC;
    const int ri = rest % NR;
    const int seg = rest / NR;
    const int lr = RK == kAny ? ri : 2 * ri - 2;
    const int lx = XK == kAny ? 4 * xc : 4 * xc - 4;
    const int p0 = seg * 2 * SEG;
    const int sb = P == 0 ? G::sidx(0, lr, lx) : G::sidx(lr, 0, lx);
    const int xb = P == 0 ? G::xidx(0, lr, lx) : G::xidx(lr, 0, lx);
    const int lz_of = P == 0 ? 0 : lr, ly_of = P == 0 ? lr : 0;  // R's contribution
    const bool r_in = lr >= 0 && lr < TR;
    const bool x_in = XK == kAny || (lx >= 0 && lx < G::TX);
    const bool inside = r_in && x_in;
    // bounds-checking build: the item's first and last index in every buffer
    // it touches (the constant true otherwise)
    {
      const int lzf = P == 0 ? p0 : lz_of, lyf = P == 0 ? ly_of : p0;
      const int lzl = P == 0 ? p0 + 2 * SEG - 1 : lz_of, lyl = P == 0 ? ly_of : p0 + 2 * SEG - 1;
      // pass 1 reads its window from the coarse box and touches the field box
      // only at this segment's own positions; later passes read a window of
      // field-box positions two beyond the segment on each side
      const int slo = FROM_CB ? p0 : p0 - 2, shi = FROM_CB ? p0 + 2 * SEG - 1 : p0 + 2 * SEG + 2;
      if (!QOZ_IN(sb + slo * SP, G::kS) || !QOZ_IN(sb + shi * SP + 3, G::kS)) continue;
      if (DEC && (!QOZ_IN(xb + (p0 + 1) * XP, G::kCode) ||
                  !QOZ_IN(xb + (p0 + 2 * SEG - 1) * XP + 3, G::kCode)))
        continue;
      if (FROM_CB &&
          (!QOZ_IN(P == 0 ? G::cbidx(p0 - 2, lr, lx) : G::cbidx(lr, p0 - 2, lx), G::kCB) ||
           !QOZ_IN((P == 0 ? G::cbidx(p0 + 2 * SEG + 2, lr, lx)
                           : G::cbidx(lr, p0 + 2 * SEG + 2, lx)) + 1, G::kCB)))
        continue;
      if (!DEC && inside &&
          (!QOZ_IN(G::cidx(lzf, lyf, lx), G::kC) ||
           !QOZ_IN(G::cidx(lzl, lyl, lx) + 3, G::kC) ||
           (FROM_CB && (!QOZ_IN(G::ccidx(lzf, lyf, lx), G::kCC) ||
                        !QOZ_IN(G::ccidx(lzl, lyl, lx) + 1, G::kCC)))))
        continue;
    }
    if constexpr (XK == kAny) {
      // four targets per position
      float4 w[SEG + 3];
#pragma unroll
      for (int k = 0; k < SEG + 3; ++k)
        w[k] = *reinterpret_cast<const float4*>(S + sb + (p0 - 2 + 2 * k) * SP);
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        const int pos = p0 + 2 * j + 1;
        float4* tp = reinterpret_cast<float4*>(S + sb + pos * SP);
        const int cP = oP + pos;
        float2 plo, phi;
        plo.x = pred1<IP, BORDER>(w[j].x, w[j + 1].x, w[j + 2].x, w[j + 3].x, cP, gP);
        plo.y = pred1<IP, BORDER>(w[j].y, w[j + 1].y, w[j + 2].y, w[j + 3].y, cP, gP);
        phi.x = pred1<IP, BORDER>(w[j].z, w[j + 1].z, w[j + 2].z, w[j + 3].z, cP, gP);
        phi.y = pred1<IP, BORDER>(w[j].w, w[j + 1].w, w[j + 2].w, w[j + 3].w, cP, gP);
        const int lz = P == 0 ? pos : lz_of, ly = P == 0 ? ly_of : pos;
        if constexpr (DEC) {
          const uint2 cw = *reinterpret_cast<const uint2*>(CC + xb + pos * XP);
          *tp = make_float4(deq1(a, c, cw.x & 0xffffu, plo.x, lz, ly, lx),
                            deq1(a, c, cw.x >> 16, plo.y, lz, ly, lx + 1),
                            deq1(a, c, cw.y & 0xffffu, phi.x, lz, ly, lx + 2),
                            deq1(a, c, cw.y >> 16, phi.y, lz, ly, lx + 3));
        } else {
          const float4 xv = *tp;
          float2 rlo, rhi;
          unsigned clo, chi;
          quant2(a, c, make_float2(xv.x, xv.y), plo, inside, lz, ly, lx, rlo, clo);
          quant2(a, c, make_float2(xv.z, xv.w), phi, inside, lz, ly, lx + 2, rhi, chi);
          if (WREC) *tp = make_float4(rlo.x, rlo.y, rhi.x, rhi.y);
          if (inside)
            *reinterpret_cast<uint2*>(C16 + G::cidx(lz, ly, lx)) = make_uint2(clo, chi);
        }
      }
    } else {
      // two targets per position (x = lx and lx + 2)
      float2 w[SEG + 3];
#pragma unroll
      for (int k = 0; k < SEG + 3; ++k) {
        const int pos = p0 - 2 + 2 * k;
        if (FROM_CB) {
          const int cbi = P == 0 ? G::cbidx(pos, lr, lx) : G::cbidx(lr, pos, lx);
          w[k] = *reinterpret_cast<const float2*>(CB + cbi);
        } else {
          const float4 v = *reinterpret_cast<const float4*>(S + sb + pos * SP);
          w[k] = make_float2(v.x, v.z);
        }
      }
      if (FROM_CB) {
        // coarse patch: this segment's even positions [p0, p0 + 2 SEG)
#pragma unroll
        for (int k = 1; k <= SEG; ++k) {
          const int pos = p0 - 2 + 2 * k;
          float* sp = S + sb + pos * SP;
          sp[0] = w[k].x;
          sp[2] = w[k].y;
          if (!DEC && inside) {
            const int lz = P == 0 ? pos : lz_of, ly = P == 0 ? ly_of : pos;
            const unsigned cc = *reinterpret_cast<const unsigned*>(CC + G::ccidx(lz, ly, lx));
            uint16_t* cp = C16 + G::cidx(lz, ly, lx);
            cp[0] = (uint16_t)(cc & 0xffffu);
            cp[2] = (uint16_t)(cc >> 16);
            if (c.full) {
              hist_add(a, c.SH, cc & 0xffffu);
              hist_add(a, c.SH, cc >> 16);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < SEG; ++j) {
        const int pos = p0 + 2 * j + 1;
        float* sp = S + sb + pos * SP;
        const int cP = oP + pos;
        const float p0v = pred1<IP, BORDER>(w[j].x, w[j + 1].x, w[j + 2].x, w[j + 3].x, cP, gP);
        const float p1v = pred1<IP, BORDER>(w[j].y, w[j + 1].y, w[j + 2].y, w[j + 3].y, cP, gP);
        const int lz = P == 0 ? pos : lz_of, ly = P == 0 ? ly_of : pos;
        if constexpr (DEC) {
          const uint2 cw = *reinterpret_cast<const uint2*>(CC + xb + pos * XP);
          sp[0] = deq1(a, c, cw.x & 0xffffu, p0v, lz, ly, lx);
          sp[2] = deq1(a, c, cw.y & 0xffffu, p1v, lz, ly, lx + 2);
        } else {
          const float4 xv = *reinterpret_cast<const float4*>(sp);
          float r0, r1;
          unsigned k0, k1;
          quant1(a, c, xv.x, p0v, inside, lz, ly, lx, r0, k0);
          quant1(a, c, xv.z, p1v, inside, lz, ly, lx + 2, r1, k1);
          if (WREC) *reinterpret_cast<float4*>(sp) = make_float4(r0, xv.y, r1, xv.w);
          if (inside) {
            uint16_t* cp = C16 + G::cidx(lz, ly, lx);
            cp[0] = (uint16_t)k0;
            cp[2] = (uint16_t)k1;
          }
        }
      }
    }
  }
}

// ---- a pass along x: each item takes the odd x 8c + 1, + 3, + 5, + 7 of one row.
template <class G, int PASS, int IP, bool BORDER, bool WREC, bool DEC>
__device__ __forceinline__ void x_pass(const LevelLaunch& a, const Ctx& c, float* S,
                                       const float* CB, const uint16_t* CC, uint16_t* C16) {
  constexpr bool FROM_CB = PASS == 1;  // the order takes x first
  constexpr int ZK = G::template role<PASS, 0>();
  constexpr int YK = G::template role<PASS, 1>();
  constexpr int NZ = ZK == kAny ? G::TZ : G::TZ / 2 + 3;
  constexpr int NY = YK == kAny ? G::TY : G::TY / 2 + 3;
  constexpr int NXC = G::TX / 8;
  constexpr int items = NZ * NY * NXC;
  static_assert(FROM_CB || G::XL == 4, "x halo");

  for (int it = threadIdx.x; it < items; it += kThr) {
    const int xc = it % NXC;
    const int rest = it / NXC;
    const int yi = rest % NY;
    const int zi = rest / NY;
    const int lz = ZK == kAny ? zi : 2 * zi - 2;
    const int ly = YK == kAny ? yi : 2 * yi - 2;
    const int lx0 = 8 * xc;
    const int base = G::sidx(lz, ly, lx0);
    const bool inside = lz >= 0 && lz < G::TZ && ly >= 0 && ly < G::TY;
    // bounds-checking build: the item's first and last index in each buffer
    if (!QOZ_IN(base - (FROM_CB ? 0 : 4), G::kS) || !QOZ_IN(base + (FROM_CB ? 7 : 11), G::kS))
      continue;
    if (FROM_CB && (!QOZ_IN(G::cbidx(lz, ly, lx0) - 1, G::kCB) ||
                    !QOZ_IN(G::cbidx(lz, ly, lx0) + 5, G::kCB)))
      continue;
    if (DEC && !QOZ_IN(G::xidx(lz, ly, lx0) + 7, G::kCode)) continue;
    if (!DEC && inside &&
        (!QOZ_IN(G::cidx(lz, ly, lx0) + 7, G::kC) ||
         (FROM_CB && !QOZ_IN(G::ccidx(lz, ly, lx0) + 3, G::kCC))))
      continue;
    float4* t4 = reinterpret_cast<float4*>(S + base);
    float e[7];  // even x at lx0 - 2, lx0, ..., lx0 + 10
    float4 v0, v1;
    if (FROM_CB) {
      const int cbi = G::cbidx(lz, ly, lx0);
      const float4 cm = *reinterpret_cast<const float4*>(CB + cbi);
      const float2 cn = *reinterpret_cast<const float2*>(CB + cbi + 4);
      e[0] = CB[cbi - 1];
      e[1] = cm.x;
      e[2] = cm.y;
      e[3] = cm.z;
      e[4] = cm.w;
      e[5] = cn.x;
      e[6] = cn.y;
      if (!DEC) {
        v0 = t4[0];
        v1 = t4[1];
      }
    } else {
      const float4 vm = t4[-1], v2 = t4[2];
      v0 = t4[0];
      v1 = t4[1];
      e[0] = vm.z;
      e[1] = v0.x;
      e[2] = v0.z;
      e[3] = v1.x;
      e[4] = v1.z;
      e[5] = v2.x;
      e[6] = v2.z;
    }
    float r[4];
    if constexpr (DEC) {
      const uint4 cw = *reinterpret_cast<const uint4*>(CC + G::xidx(lz, ly, lx0));
      const unsigned cd[4] = {cw.x >> 16, cw.y >> 16, cw.z >> 16, cw.w >> 16};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int lx = lx0 + 2 * q + 1;
        const float p = pred1<IP, BORDER>(e[q], e[q + 1], e[q + 2], e[q + 3], c.ox + lx, c.g2);
        r[q] = deq1(a, c, cd[q], p, lz, ly, lx);
      }
    } else {
      const float tv[4] = {v0.y, v0.w, v1.y, v1.w};
      unsigned k[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int lx = lx0 + 2 * q + 1;
        const float p = pred1<IP, BORDER>(e[q], e[q + 1], e[q + 2], e[q + 3], c.ox + lx, c.g2);
        quant1(a, c, tv[q], p, inside, lz, ly, lx, r[q], k[q]);
      }
      if (inside) {
        uint16_t* cp = C16 + G::cidx(lz, ly, lx0);
        if (FROM_CB) {
          const uint2 cc = *reinterpret_cast<const uint2*>(CC + G::ccidx(lz, ly, lx0));
          if (c.full) {
            hist_add(a, c.SH, cc.x & 0xffffu);
            hist_add(a, c.SH, cc.x >> 16);
            hist_add(a, c.SH, cc.y & 0xffffu);
            hist_add(a, c.SH, cc.y >> 16);
          }
          uint4 o;
          o.x = __byte_perm(cc.x, k[0], 0x5410);
          o.y = __byte_perm(cc.x, k[1], 0x5432);
          o.z = __byte_perm(cc.y, k[2], 0x5410);
          o.w = __byte_perm(cc.y, k[3], 0x5432);
          *reinterpret_cast<uint4*>(cp) = o;
        } else {
          cp[1] = (uint16_t)k[0];
          cp[3] = (uint16_t)k[1];
          cp[5] = (uint16_t)k[2];
          cp[7] = (uint16_t)k[3];
        }
      }
    }
    if (WREC || FROM_CB || DEC) {
      t4[0] = make_float4(e[1], r[0], e[2], r[1]);
      t4[1] = make_float4(e[3], r[2], e[4], r[3]);
    }
  }
}

template <class G, int PASS, int IP, bool BORDER, bool WREC, bool DEC>
__device__ __forceinline__ void run_pass_b(const LevelLaunch& a, const Ctx& c, float* S,
                                           const float* CB, const uint16_t* CC, uint16_t* C16) {
  constexpr int P = PASS == 1 ? G::A0 : (PASS == 2 ? G::A1 : G::A2);
  if constexpr (P == 2)
    x_pass<G, PASS, IP, BORDER, WREC, DEC>(a, c, S, CB, CC, C16);
  else
    line_pass<G, PASS, IP, BORDER, WREC, DEC>(a, c, S, CB, CC, C16);
}

// A pass needs the border stencils only when the tile comes within 4 points
// of the grid's edge along the pass axis; elsewhere every target's four
// neighbours exist.
template <class G, int PASS, int IP, bool WREC, bool DEC>
__device__ __forceinline__ void run_pass(const LevelLaunch& a, const Ctx& c, float* S,
                                         const float* CB, const uint16_t* CC, uint16_t* C16) {
  constexpr int P = PASS == 1 ? G::A0 : (PASS == 2 ? G::A1 : G::A2);
  const int o = P == 0 ? c.oz : (P == 1 ? c.oy : c.ox);
  const int g = P == 0 ? c.g0 : (P == 1 ? c.g1 : c.g2);
  if (o >= 4 && o + G::T(P) + 4 <= g)
    run_pass_b<G, PASS, IP, false, WREC, DEC>(a, c, S, CB, CC, C16);
  else
    run_pass_b<G, PASS, IP, true, WREC, DEC>(a, c, S, CB, CC, C16);
}

template <class G, int IP, bool DEC>
__device__ __forceinline__ void run_tile(const LevelLaunch& a, const Ctx& c, float* S,
                                         const float* CB, const uint16_t* CC, uint16_t* C16,
                                         bool want_rec) {
  run_pass<G, 1, IP, true, DEC>(a, c, S, CB, CC, C16);
  __syncthreads();
  run_pass<G, 2, IP, true, DEC>(a, c, S, CB, CC, C16);
  __syncthreads();
  if (want_rec || DEC)
    run_pass<G, 3, IP, true, DEC>(a, c, S, CB, CC, C16);
  else
    run_pass<G, 3, IP, false, DEC>(a, c, S, CB, CC, C16);
}

// The tile's reconstruction (field box interior) into the compact output
// rows of the level's grid, four x per item.
template <class G>
__device__ __forceinline__ void store_tile(const LevelLaunch& a, const Ctx& c, const float* S) {
  const unsigned os0 = (unsigned)a.os[0], os1 = (unsigned)a.os[1];
  const bool vec = (a.os[1] % 4) == 0 && (a.os[0] % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(a.rout) & 15) == 0;
  for (int g = threadIdx.x; g < G::kC / 4; g += kThr) {
    const int lx = (g % (G::TX / 4)) * 4;
    const int t = g / (G::TX / 4);
    const int ly = t % G::TY, lz = t / G::TY;
    const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
    if (cz >= c.g0 || cy >= c.g1 || cx >= c.g2) continue;
    if (!QOZ_IN(G::sidx(lz, ly, lx) + 3, G::kS)) continue;
    const float4 v = *reinterpret_cast<const float4*>(S + G::sidx(lz, ly, lx));
    const unsigned oi = (unsigned)cz * os0 + (unsigned)cy * os1 + (unsigned)cx;
    if (vec && cx + 4 <= c.g2) {
      *reinterpret_cast<float4*>(a.rout + oi) = v;
    } else {
      a.rout[oi] = v.x;
      if (cx + 1 < c.g2) a.rout[oi + 1] = v.y;
      if (cx + 2 < c.g2) a.rout[oi + 2] = v.z;
      if (cx + 3 < c.g2) a.rout[oi + 3] = v.w;
    }
  }
}

// Issues the three bulk copies of a tile into a stage (one thread).
template <class G>
__device__ __forceinline__ void issue_tile(unsigned char* stage, uint64_t* mbar, int tile,
                                           int nt1, int nt2, const CUtensorMap* mx,
                                           const CUtensorMap* mrc, const CUtensorMap* mcc) {
  const int tx = tile % nt2;
  const int r = tile / nt2;
  const int ty = r % nt1;
  const int tz = r / nt1;
  const int ox = tx * G::TX, oy = ty * G::TY, oz = tz * G::TZ;
  mbar_expect_tx(mbar, G::kTxBytes);
  tma_load_3d(stage, mx, ox - G::XL, oy - G::HY, oz - G::HZ, mbar);
  tma_load_3d(stage + G::oCB, mrc, ox / 2 - 4, oy / 2 - 1, oz / 2 - 1, mbar);
  tma_load_3d(stage + G::oCC, mcc, ox / 2, oy / 2, oz / 2, mbar);
}

__device__ __forceinline__ bool wait_polls(uint64_t* m, unsigned parity, unsigned polls) {
  for (unsigned k = 0; k < polls; ++k)
    if (mbar_try_wait(m, parity)) return true;
  return false;
}

// The level-1 compression of a 3-D field (the grid G is the field itself).
template <class G, int IP>
__device__ __forceinline__ void compress_tiles(const LevelLaunch& a, unsigned char* smem_raw,
                                               uint64_t* mbar, int nt1, int nt2, int ntiles,
                                               const CUtensorMap* mx, const CUtensorMap* mrc,
                                               const CUtensorMap* mcc, const CUtensorMap* mout) {
  unsigned char* sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned* SH = reinterpret_cast<unsigned*>(sm + G::oHist);
  Ctx c;
  c.g0 = (int)a.g[0];
  c.g1 = (int)a.g[1];
  c.g2 = (int)a.g[2];
  c.el = a.bt->el[0];
  c.two_e = a.bt->two_e[0];
  c.inv = a.bt->inv[0];
  c.SH = SH;
  c.full = false;
  const bool want_rec = a.rout != nullptr;

  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&mbar[2], 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kHistWin; i += kThr) SH[i] = 0;
  __syncthreads();

  if (a.extra_tx > 0) {
    // host fault injection: a barrier that expects bytes no copy brings; the
    // bounded wait runs out and the launch reports it (no copy is in flight)
    if (threadIdx.x == 0) mbar_expect_tx(&mbar[2], (unsigned)a.extra_tx);
    const bool ok = wait_polls(&mbar[2], 0, a.wait_polls > 0 ? (unsigned)a.wait_polls : kPolls);
    if (!__syncthreads_and(ok) && threadIdx.x == 0 && a.err) atomicOr(a.err, 2);
    return;
  }

  if (threadIdx.x == 0) issue_tile<G>(sm, &mbar[0], blockIdx.x, nt1, nt2, mx, mrc, mcc);
  float* S = reinterpret_cast<float*>(sm);
  const float* CB = reinterpret_cast<const float*>(sm + G::oCB);
  const uint16_t* CC = reinterpret_cast<const uint16_t*>(sm + G::oCC);
  uint16_t* C16 = reinterpret_cast<uint16_t*>(sm + G::oC16);
  int i = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const bool landed = wait_polls(&mbar[0], (unsigned)i & 1u, kPolls);
    if (threadIdx.x == 0 && i >= 1) bulk_wait_read0();  // the last code store has read its buffer
    if (!__syncthreads_and(landed)) {
      // a copy never completed: report it and leave (after the code store)
      if (threadIdx.x == 0) {
        if (a.err) atomicOr(a.err, 2);
        bulk_wait_read0();
      }
      return;
    }
    {
      const int tx = tile % nt2;
      const int r = tile / nt2;
      c.ox = tx * G::TX;
      c.oy = (r % nt1) * G::TY;
      c.oz = (r / nt1) * G::TZ;
    }
    // every point of the tile lies inside the field
    const bool full = c.oz + G::TZ <= c.g0 && c.oy + G::TY <= c.g1 && c.ox + G::TX <= c.g2;
    c.full = full;
    run_tile<G, IP, false>(a, c, S, CB, CC, C16, want_rec);
    fence_proxy_async_smem();  // code tile written: visible to the bulk store
    __syncthreads();
    if (want_rec) {
      store_tile<G>(a, c, S);  // the caller asked for the reconstruction
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // the code tile leaves; the next tile's input loads while this CTA
      // counts the codes (the passes are done with the input buffers)
      tma_store_3d(mout, c.ox, c.oy, c.oz, C16);
      bulk_commit();
      const int nt = tile + (int)gridDim.x;
      if (nt < ntiles) issue_tile<G>(sm, &mbar[0], nt, nt1, nt2, mx, mrc, mcc);
    }
    // a tile that reaches past the field counts the codes of its points
    // inside the field here (full tiles counted theirs in the passes)
    if (!full) {
      for (int g = threadIdx.x; g < G::kC / 8; g += kThr) {
        const uint4 v = reinterpret_cast<const uint4*>(C16)[g];
        const int lx = (g % (G::TX / 8)) * 8;
        const int t = g / (G::TX / 8);
        const int ly = t % G::TY, lz = t / G::TY;
        const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
        const int nval = (cz < c.g0 && cy < c.g1) ? min(8, max(0, c.g2 - cx)) : 0;
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k < nval) hist_add(a, SH, (wv[k >> 1] >> (16 * (k & 1))) & 0xffffu);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kHistWin; k += kThr)
    if (SH[k]) atomicAdd(&a.hist[kHistLo + k], SH[k]);
  if (threadIdx.x == 0) bulk_wait_read0();
}

// Level 1 of several 3-D fields in one launch (a batched plan): tile t of
// the launch belongs to item map[t], as that item's tile t - tile_begin.
// The CTAs walk the launch's tiles as above; a CTA whose next tile starts a
// new item flushes its histogram window into the old item's histogram and
// takes the new item's descriptor into shared memory.  The items' tensor
// maps sit in device memory; the next tile's copies are issued with its own
// item's maps.
template <class G, int IP>
__device__ __forceinline__ void compress_tiles_batch(const LevelItem* __restrict__ items,
                                                     const uint16_t* __restrict__ map,
                                                     const LevelTmaMaps* __restrict__ maps,
                                                     int ntiles, unsigned char* smem_raw,
                                                     uint64_t* mbar, LevelItem& it) {
  unsigned char* sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned* SH = reinterpret_cast<unsigned*>(sm + G::oHist);
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[2], 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kHistWin; i += kThr) SH[i] = 0;
  __syncthreads();
  if ((int)blockIdx.x >= ntiles) return;
  {
    // host fault injection (every level-1 item carries it): a barrier that
    // expects bytes no copy brings, before any copy is issued
    const LevelLaunch& f = items[map[blockIdx.x]].L;
    if (f.extra_tx > 0) {
      if (threadIdx.x == 0) mbar_expect_tx(&mbar[2], (unsigned)f.extra_tx);
      const bool ok = wait_polls(&mbar[2], 0, f.wait_polls > 0 ? (unsigned)f.wait_polls : kPolls);
      if (!__syncthreads_and(ok) && threadIdx.x == 0 && f.err) atomicOr(f.err, 2);
      return;
    }
  }
  auto issue = [&](int tile) {  // one thread
    const int k = map[tile];
    const LevelItem& q = items[k];
    issue_tile<G>(sm, &mbar[0], tile - (int)q.tile_begin, q.nt1, q.nt2, &maps[k].x, &maps[k].rc,
                  &maps[k].cc);
  };
  if (threadIdx.x == 0) issue((int)blockIdx.x);
  float* S = reinterpret_cast<float*>(sm);
  const float* CB = reinterpret_cast<const float*>(sm + G::oCB);
  const uint16_t* CC = reinterpret_cast<const uint16_t*>(sm + G::oCC);
  uint16_t* C16 = reinterpret_cast<uint16_t*>(sm + G::oC16);
  Ctx c;
  c.SH = SH;
  c.full = false;
  int cur = -1;
  bool counting = false;
  int i = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int k = map[tile];
    if (k != cur) {
      __syncthreads();  // the CTA is done with the old item and its window
      if (cur >= 0 && counting)
        for (int j = threadIdx.x; j < kHistWin; j += kThr)
          if (SH[j]) {
            atomicAdd(&it.L.hist[kHistLo + j], SH[j]);
            SH[j] = 0;
          }
      __syncthreads();
      static_assert(sizeof(LevelItem) % 4 == 0 && sizeof(LevelItem) / 4 <= kThr, "item copy");
      if (threadIdx.x < sizeof(LevelItem) / 4)
        reinterpret_cast<unsigned*>(&it)[threadIdx.x] =
            reinterpret_cast<const unsigned*>(items + k)[threadIdx.x];
      __syncthreads();
      cur = k;
      c.g0 = (int)it.L.g[0];
      c.g1 = (int)it.L.g[1];
      c.g2 = (int)it.L.g[2];
      c.el = it.L.bt->el[0];
      c.two_e = it.L.bt->two_e[0];
      c.inv = it.L.bt->inv[0];
      counting = it.L.hist != nullptr;
    }
    const bool landed = wait_polls(&mbar[0], (unsigned)i & 1u, kPolls);
    if (threadIdx.x == 0 && i >= 1) bulk_wait_read0();  // the last code store has read its buffer
    if (!__syncthreads_and(landed)) {
      // a copy never completed: report it and leave (after the code store)
      if (threadIdx.x == 0) {
        if (it.L.err) atomicOr(it.L.err, 2);
        bulk_wait_read0();
      }
      return;
    }
    {
      const int lt = tile - (int)it.tile_begin;
      const int r = lt / it.nt2;
      c.ox = (lt % it.nt2) * G::TX;
      c.oy = (r % it.nt1) * G::TY;
      c.oz = (r / it.nt1) * G::TZ;
    }
    const bool full = c.oz + G::TZ <= c.g0 && c.oy + G::TY <= c.g1 && c.ox + G::TX <= c.g2;
    c.full = full && counting;
    const bool want_rec = it.L.rout != nullptr;
    run_tile<G, IP, false>(it.L, c, S, CB, CC, C16, want_rec);
    fence_proxy_async_smem();  // code tile written: visible to the bulk store
    __syncthreads();
    if (want_rec) {
      store_tile<G>(it.L, c, S);
      __syncthreads();
    }
    if (maps[k].use_out) {
      if (threadIdx.x == 0) {
        tma_store_3d(&maps[k].out, c.ox, c.oy, c.oz, C16);
        bulk_commit();
      }
    } else {
      // the code array's rows are not on 16-byte boundaries: plain stores
      for (int g = threadIdx.x; g < G::kC; g += kThr) {
        const int lx = g % G::TX, t = g / G::TX;
        const int cz = c.oz + t / G::TY, cy = c.oy + t % G::TY, cx = c.ox + lx;
        if (cz < c.g0 && cy < c.g1 && cx < c.g2)
          it.L.cout[(long long)cz * it.L.os[0] + (long long)cy * it.L.os[1] + cx] = C16[g];
      }
    }
    if (threadIdx.x == 0) {
      const int nt = tile + (int)gridDim.x;
      if (nt < ntiles) issue(nt);
    }
    if (!full && counting) {
      for (int g = threadIdx.x; g < G::kC / 8; g += kThr) {
        const uint4 v = reinterpret_cast<const uint4*>(C16)[g];
        const int lx = (g % (G::TX / 8)) * 8;
        const int t = g / (G::TX / 8);
        const int ly = t % G::TY, lz = t / G::TY;
        const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
        const int nval = (cz < c.g0 && cy < c.g1) ? min(8, max(0, c.g2 - cx)) : 0;
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nval) hist_add(it.L, SH, (wv[q >> 1] >> (16 * (q & 1))) & 0xffffu);
      }
    }
  }
  __syncthreads();
  if (cur >= 0 && counting)
    for (int j = threadIdx.x; j < kHistWin; j += kThr)
      if (SH[j]) atomicAdd(&it.L.hist[kHistLo + j], SH[j]);
  if (threadIdx.x == 0) bulk_wait_read0();
}

// The level-1 decompression of a 3-D field: per tile, the codes over the
// tile and its halo and the coarse box arrive by bulk copies (the field box
// is filled by the passes themselves); the next tile's copies are issued
// once the passes are done, while the CTA writes the tile's reconstruction.
template <class G, int IP>
__device__ __forceinline__ void decompress_tiles(const LevelLaunch& a, unsigned char* smem_raw,
                                                 uint64_t* mbar, int nt1, int nt2, int ntiles,
                                                 const CUtensorMap* mcode,
                                                 const CUtensorMap* mrc) {
  unsigned char* sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float* S = reinterpret_cast<float*>(sm);
  const uint16_t* CODE = reinterpret_cast<const uint16_t*>(sm + G::dCode);
  const float* CB = reinterpret_cast<const float*>(sm + G::dCB);
  Ctx c;
  c.g0 = (int)a.g[0];
  c.g1 = (int)a.g[1];
  c.g2 = (int)a.g[2];
  c.el = a.bt->el[0];
  c.two_e = a.bt->two_e[0];
  c.inv = a.bt->inv[0];
  c.full = false;
  c.SH = nullptr;
  auto issue = [&](int tile) {
    const int tx = tile % nt2;
    const int r = tile / nt2;
    const int ox = tx * G::TX, oy = (r % nt1) * G::TY, oz = (r / nt1) * G::TZ;
    mbar_expect_tx(&mbar[0], G::kDecTxBytes);
    tma_load_3d(sm + G::dCode, mcode, ox - G::XC, oy - G::HY, oz - G::HZ, &mbar[0]);
    tma_load_3d(sm + G::dCB, mrc, ox / 2 - 4, oy / 2 - 1, oz / 2 - 1, &mbar[0]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) issue(blockIdx.x);
  int i = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const bool landed = wait_polls(&mbar[0], (unsigned)i & 1u, kPolls);
    if (!__syncthreads_and(landed)) {
      if (threadIdx.x == 0 && a.err) atomicOr(a.err, 2);
      return;
    }
    const int tx = tile % nt2;
    const int r = tile / nt2;
    c.ox = tx * G::TX;
    c.oy = (r % nt1) * G::TY;
    c.oz = (r / nt1) * G::TZ;
    run_tile<G, IP, true>(a, c, S, CB, CODE, nullptr, true);
    __syncthreads();  // the passes are done with the code box and the coarse box
    if (threadIdx.x == 0 && tile + (int)gridDim.x < ntiles) issue(tile + (int)gridDim.x);
    store_tile<G>(a, c, S);
  }
}

}  // namespace l1
}  // namespace qoz
