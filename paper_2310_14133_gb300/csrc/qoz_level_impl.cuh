// Templates of one level of the QoZ interpolation predictor (Sec. 5.1, Sec. 5.2.2) as a
// shared-memory tile kernel, for compression and its mirror.
//
// A launch handles the finest level of a grid G (see LevelLaunch).  Each CTA
// owns a TZ x TY x TX tile of G and runs the level's three dimension passes
// on it (A0, A1, A2 = physical axes in the level's order):
//   pass 1 (along A0): targets odd on A0, even on A1 and A2; neighbours are
//                      coarse points;
//   pass 2 (along A1): targets odd on A1, even on A2;
//   pass 3 (along A2): targets odd on A2.
// Pass 2 reaches +-3 along A1 and pass 3 +-3 along A2, so the tile carries a
// 3-point halo on A1 and A2 and the halo's pass-1 / pass-2 points are
// computed again by every tile that needs them (bit-identical: same inputs,
// same operations, same order).  Pass 1 also reads coarse values at local
// A0 positions -2, T0 and T0+2 ("side" rows).
//
// Shared layout.  The tile is stored as rows along x covering local
// x in [-4, TX+4).  At level 1 each row arrives as 16-byte cp.async copies
// (every copy of the tile in flight at once); coarse values come from the
// compact coarse reconstruction into a small staging area and are patched
// into the even positions of coarse rows after the copies land.  Passes map
// consecutive lanes to consecutive x: a pass along x gives each lane one
// odd-x target; a pass along z or y gives each lane an x position and a
// segment of the line along the pass axis, whose even (reconstructed)
// positions sit in a register window, so each target costs one shared load
// of its own value.  Tiles whose halo lies inside the grid take an interior
// path with no bounds or border-stencil tests.
//
// Compression writes the grid's codes compactly: its targets' codes plus the
// coarse points' codes copied from the coarse grid's compact code array,
// staged in shared memory and stored eight at a time.  At level 1 that
// compact grid is the field itself, so the output array is written exactly
// once; the level-1 launch also accumulates the code histogram.
#pragma once

#include <cuda_runtime.h>

#include "qoz_internal.h"
#include "qoz_tma.cuh"


namespace qoz {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kHistLo = kRadius - 2048;  // shared histogram window [32768-2048, 32768+2048)
constexpr int kHistWin = 4096;
// the bulk-copy kernel's smaller window [32768-512, 32768+512)
constexpr int kTmaHistLo = kRadius - 512;
constexpr int kTmaHistWin = 1024;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Role of an axis in a pass:
//   kOdd  : odd positions inside the tile (the pass axis)
//   kAny  : every position inside the tile
//   kEvenH: even positions over the tile and its 3-point halo (-2 .. T+2)
enum Role { kOdd, kAny, kEvenH };

template <int A0, int A1, int A2, int PASS, int P>
struct RoleOf {
  static constexpr int value =
      PASS == 1 ? (P == A0 ? kOdd : kEvenH)
                : (PASS == 2 ? (P == A0 ? kAny : (P == A1 ? kOdd : kEvenH))
                             : (P == A2 ? kOdd : kAny));
};

template <int ROLE, int T>
struct Span {
  static constexpr int start = ROLE == kOdd ? 1 : (ROLE == kAny ? 0 : -2);
  static constexpr int step = ROLE == kAny ? 1 : 2;
  static constexpr int count = ROLE == kOdd ? T / 2 : (ROLE == kAny ? T : T / 2 + 3);
};

// Targets per work item along a line of NT targets with `lines` lines: at
// most 16 (register window), halved while the items would still fill no more
// than half the block.
__host__ __device__ constexpr int pick_seg(int NT, int lines, int threads = kThreads) {
  int seg = NT < 16 ? NT : 16;
  while (seg > 4 && NT % (seg / 2) == 0 && (NT / seg) * lines * 2 <= threads) seg /= 2;
  return seg;
}

// Halo of a tile along z and y: the axis interpolated first (A0) needs none.
__host__ __device__ constexpr int halo_z(int a0) { return a0 == 0 ? 0 : kHalo; }
__host__ __device__ constexpr int halo_y(int a0) { return a0 == 1 ? 0 : kHalo; }

template <int A0_, int A1_, int A2_, int TZ_, int TY_, int TX_, int THR_ = kThreads,
          int IP_ = -1>
struct Geo {
  static constexpr int A0 = A0_, A1 = A1_, A2 = A2_;
  static constexpr int TZ = TZ_, TY = TY_, TX = TX_;
  static constexpr int kThr = THR_;    // threads of the CTA that owns the tile
  static constexpr int kInterp = IP_;  // interpolator fixed at compile time (-1: runtime)
  __host__ __device__ static constexpr int T(int p) { return p == 0 ? TZ : (p == 1 ? TY : TX); }
  static constexpr int HZ = halo_z(A0);
  static constexpr int HY = halo_y(A0);
  static constexpr int EZ = TZ + 2 * HZ, EY = TY + 2 * HY;
  static constexpr int EX = TX + 8;  // local x in [-4, TX + 4), stored at x + 4
  static constexpr int HX = EX / 2;  // even x of a row: -4, -2, ..., TX + 2
  static constexpr int T0 = T(A0);
  static constexpr int NMAIN = EZ * EY;
  // coarse rows of the main box: even z and even y (lowest even local
  // coordinate -2 with a halo, 0 without)
  static constexpr int ZLO = HZ ? -2 : 0, YLO = HY ? -2 : 0;
  static constexpr int NCZ = HZ ? TZ / 2 + 3 : (TZ + 1) / 2;
  static constexpr int NCY = HY ? TY / 2 + 3 : (TY + 1) / 2;
  static constexpr int NCMAIN = NCZ * NCY;
  // side rows (A0 = z or y): A0 at -2, T0, T0 + 2; the other of z, y even
  // over its halo (-2 .. T + 2)
  static constexpr int NOS = (A0 == 0 ? TY : TZ) / 2 + 3;
  static constexpr int NSIDE = (A0 == 2 || T0 < 2) ? 0 : 3 * NOS;
  static constexpr int kS = NMAIN * EX;                 // floats
  static constexpr int kCR = (NCMAIN + NSIDE) * HX;     // floats (coarse staging)
  static constexpr int kC = TZ * TY * TX;               // codes
  static constexpr size_t kSBytes = sizeof(float) * kS;             // multiple of 16
  static constexpr size_t kCRBytes = (sizeof(float) * kCR + 15) & ~size_t(15);
  static constexpr size_t kCodeBytes = (sizeof(uint16_t) * kC + 15) & ~size_t(15);
  static constexpr size_t kInBytes = (sizeof(uint16_t) * kS + 15) & ~size_t(15);  // staged codes
  static constexpr size_t kHistBytes = sizeof(unsigned) * kHistWin;
  __host__ __device__ static constexpr size_t smem_bytes(bool decomp, bool hist) {
    return kSBytes + kCRBytes + (decomp ? kInBytes : kCodeBytes + (hist ? kHistBytes : 0));
  }
  __device__ static constexpr int row(int z, int y) { return (z + HZ) * EY + (y + HY); }
  __device__ static constexpr int crow(int z, int y) {
    return ((z - ZLO) >> 1) * NCY + ((y - YLO) >> 1);
  }
  __device__ static constexpr int side_row(int k, int other) {
    return NCMAIN + k * NOS + ((other + 2) >> 1);
  }
  __device__ static constexpr int cidx(int z, int y, int x) { return (z * TY + y) * TX + x; }
  // Bulk-copy layout (level 1): the coarse reconstruction box covers even
  // local coordinates -4 .. T + 2 (z, y) and -8 .. TX + 6 (x, so that its
  // first column sits on a 16-byte boundary); the coarse code box covers the
  // tile's own coarse points.
  static constexpr int CBZ = TZ / 2 + 4, CBY = TY / 2 + 4, CBX = TX / 2 + 8;
  static constexpr int kCB = CBZ * CBY * CBX;
  static constexpr int CCZ = (TZ + 1) / 2, CCY = (TY + 1) / 2, CCX = TX / 2;
  static constexpr int kCC = CCZ * CCY * CCX;
  __device__ static constexpr int cbidx(int z, int y, int x) {
    return ((z / 2 + 2) * CBY + (y / 2 + 2)) * CBX + (x / 2 + 4);
  }
  static constexpr size_t align128(size_t v) { return (v + 127) & ~size_t(127); }
  static constexpr size_t kTmaS = align128(sizeof(float) * kS);
  static constexpr size_t kTmaCB = align128(sizeof(float) * kCB);
  static constexpr size_t kTmaC16 = align128(sizeof(uint16_t) * kC);
  static constexpr size_t kTmaCC = align128(sizeof(uint16_t) * kCC);
  __host__ __device__ static constexpr size_t tma_smem_bytes(bool hist) {
    return 128 + kTmaS + kTmaCB + kTmaC16 + kTmaCC + (hist ? sizeof(unsigned) * kTmaHistWin : 0);
  }
  // true when every position the tile touches lies inside the grid
  __device__ static bool interior(int oz, int oy, int ox, int g0, int g1, int g2) {
    return oz >= 4 && oz + TZ + 4 <= g0 && oy >= 4 && oy + TY + 4 <= g1 && ox >= 4 &&
           ox + TX + 4 <= g2;
  }
};

struct Ctx {
  int oz, oy, ox;  // tile origin in G
  int g0, g1, g2;  // grid extent
  float el, two_e, inv;
  int interp;
};

template <int P>
__device__ __forceinline__ int gsel(const Ctx& c) {
  return P == 0 ? c.g0 : (P == 1 ? c.g1 : c.g2);
}
template <int P>
__device__ __forceinline__ int osel(const Ctx& c) {
  return P == 0 ? c.oz : (P == 1 ? c.oy : c.ox);
}

// The level's interpolator: the compile-time one when the instance fixes it.
template <class G>
__device__ __forceinline__ int interp_of(const Ctx& c) {
  return G::kInterp >= 0 ? G::kInterp : c.interp;
}

// Interpolation with every neighbour present (interior tiles).
__device__ __forceinline__ float predict_full(float a3, float a1, float b1, float b3, int interp) {
  if (interp == 1)
    return __fmul_rn(__fsub_rn(__fmul_rn(9.0f, __fadd_rn(a1, b1)), __fadd_rn(a3, b3)), 0.0625f);
  return __fmul_rn(__fadd_rn(a1, b1), 0.5f);
}

// Final value of one target from its prediction: quantize (compress) or
// dequantize (decompress, code read from the staged codes).  `inside`: the
// target belongs to this tile.
template <bool DECOMP>
__device__ __forceinline__ void finish(const LevelLaunch& a, const Ctx& c, float* S,
                                       const uint16_t* IN16, int si, float pred, bool inside,
                                       uint16_t* code_slot, int cz, int cy, int cx) {
  if (DECOMP) {
    const int code = IN16[si];
    float v;
    if (code == 0) {
      const long long xi = (long long)((unsigned long long)cz * a.xs[0] +
                                       (unsigned long long)cy * a.xs[1] +
                                       (unsigned long long)cx * a.xs[2]);
      if (!unpred_lookup(a.uidx, a.uval, a.nu, xi, &v)) {
        v = 0.0f;
        atomicOr(a.err, 1);
      }
    } else {
      v = dequantize(pred, code, c.two_e);
    }
    S[si] = v;
  } else {
    const float xv = S[si];
    uint16_t code;
    float rec;
    if (quantize(xv, pred, c.el, c.two_e, c.inv, &code, &rec)) {
      S[si] = rec;
    } else {
      code = 0;
      if (inside) {
        const long long xi = (long long)((unsigned long long)cz * a.xs[0] +
                                         (unsigned long long)cy * a.xs[1] +
                                         (unsigned long long)cx * a.xs[2]);
        unpred_append(a.ul, xi, xv);
      }
    }
    if (inside) *code_slot = code;
  }
}

// ---- a pass along z or y: lines along P, lanes on consecutive x, R = the
// other of z and y.
template <class G, int PASS, bool DECOMP, bool INTERIOR, bool CBOX = false>
__device__ __forceinline__ void pass_line(const LevelLaunch& a, const Ctx& c, float* S,
                                          const float* CR, const uint16_t* IN16,
                                          uint16_t* C16) {
  constexpr int A0 = G::A0, A1 = G::A1, A2 = G::A2;
  constexpr int P = PASS == 1 ? A0 : (PASS == 2 ? A1 : A2);
  static_assert(P != 2, "x passes use pass_x");
  constexpr int R = 1 - P;
  constexpr int XR = RoleOf<A0, A1, A2, PASS, 2>::value;
  constexpr int RR = RoleOf<A0, A1, A2, PASS, R>::value;
  using SR = Span<RR, G::T(R)>;
  using SX = Span<XR, G::TX>;
  constexpr int TP = G::T(P);
  constexpr int NT = TP / 2;
  if (NT == 0) return;
  constexpr int SEG = NT == 0 ? 1 : (PASS == 1 ? NT : pick_seg(NT, SX::count * SR::count, G::kThr));
  constexpr int NSEG = NT / SEG;
  static_assert(NT == 0 || NT % SEG == 0, "segments must tile the line");
  static_assert(PASS != 1 || NSEG == 1 || NT == 0, "the first pass walks whole lines");
  static_assert(PASS != 1 || NT <= 16, "first-pass lines hold at most 16 targets");
  constexpr int SP = (P == 1 ? 1 : G::EY) * G::EX;  // shared stride along P
  constexpr int items = NSEG * SR::count * SX::count;
  const int gP = gsel<P>(c), gR = gsel<R>(c);
  const int oP = osel<P>(c), oR = osel<R>(c);

  for (int it = threadIdx.x; it < items; it += G::kThr) {
    const int m = it % SX::count;
    const int t = it / SX::count;
    const int ri = t % SR::count;
    const int seg = t / SR::count;
    const int lx = SX::start + m * SX::step;
    const int lr = SR::start + ri * SR::step;
    const int cx = c.ox + lx, cr = oR + lr;
    if (!INTERIOR && (cx < 0 || cx >= c.g2 || cr < 0 || cr >= gR)) continue;
    const int p0 = seg * 2 * SEG;
    if (!INTERIOR && oP + p0 >= gP) continue;
    const bool inside = lx >= 0 && lx < G::TX && lr >= 0 && lr < G::T(R);
    const int rbase = (P == 1 ? G::row(lr, 0) : G::row(0, lr)) * G::EX + lx + 4;
    float w[SEG + 3];
#pragma unroll
    for (int k = 0; k < SEG + 3; ++k) {
      const int pos = p0 - 2 + 2 * k;
      if (PASS == 1 && (pos < 0 || pos >= TP)) {
        if constexpr (CBOX) {
          const int ci = G::cbidx(P == 0 ? pos : lr, P == 1 ? pos : lr, lx);
          w[k] = QOZ_IN(ci, G::kCB) ? CR[ci] : 0.0f;
        } else {
          const int kk = pos < 0 ? 0 : (pos == TP ? 1 : 2);
          const int ci = G::side_row(kk, lr) * G::HX + ((lx + 4) >> 1);
          w[k] = QOZ_IN(ci, G::kCR) ? CR[ci] : 0.0f;
        }
      } else {
        const int si = rbase + pos * SP;
        w[k] = QOZ_IN(si, G::kS) ? S[si] : 0.0f;
      }
    }
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      const int pos = p0 + 2 * j + 1;
      const int cP = oP + pos;
      if (!INTERIOR && cP >= gP) break;
      float pred;
      if (INTERIOR) {
        pred = predict_full(w[j], w[j + 1], w[j + 2], w[j + 3], interp_of<G>(c));
      } else {
        const bool hb1 = cP + 1 < gP, ha3 = cP >= 3, hb3 = cP + 3 < gP;
        pred = predict(w[j], w[j + 1], w[j + 2], w[j + 3], ha3, hb1, hb3, interp_of<G>(c));
      }
      const int lz = P == 0 ? pos : lr, ly = P == 1 ? pos : lr;
      if (!QOZ_IN(rbase + pos * SP, G::kS) || (inside && !QOZ_IN(G::cidx(lz, ly, lx), G::kC)))
        continue;
      finish<DECOMP>(a, c, S, IN16, rbase + pos * SP, pred, inside, C16 + G::cidx(lz, ly, lx),
                     c.oz + lz, c.oy + ly, cx);
    }
  }
}

// ---- a pass along x on an interior tile: one odd-x target per lane in U
// rows that share an item (consecutive rows along a no-halo axis, so the
// whole item is inside the tile or outside it together).
template <class G, int PASS, bool DECOMP, int U, bool ALONG_Y>
__device__ __forceinline__ void pass_x_rows(const LevelLaunch& a, const Ctx& c, float* S,
                                            const uint16_t* IN16, uint16_t* C16) {
  constexpr int A0 = G::A0, A1 = G::A1, A2 = G::A2;
  using SZ = Span<RoleOf<A0, A1, A2, PASS, 0>::value, G::TZ>;
  using SY = Span<RoleOf<A0, A1, A2, PASS, 1>::value, G::TY>;
  constexpr int NTX = G::TX / 2;
  constexpr int NY = ALONG_Y ? SY::count / U : SY::count;
  constexpr int NZ = ALONG_Y ? SZ::count : SZ::count / U;
  constexpr int items = NZ * NY * NTX;
  // shared-memory and code-tile distance between the rows of one item
  constexpr int DS = ALONG_Y ? SY::step * G::EX : SZ::step * G::EY * G::EX;
  constexpr int DC = ALONG_Y ? SY::step * G::TX : SZ::step * G::TY * G::TX;
  for (int it = threadIdx.x; it < items; it += G::kThr) {
    const int mm = it % NTX;
    const int t = it / NTX;
    const int yi = t % NY;
    const int zi = t / NY;
    const int lz = SZ::start + (ALONG_Y ? zi : zi * U) * SZ::step;
    const int ly = SY::start + (ALONG_Y ? yi * U : yi) * SY::step;
    const int lx = 2 * mm + 1;
    const bool inside = ALONG_Y ? (lz >= 0 && lz < G::TZ) : (ly >= 0 && ly < G::TY);
    const int si0 = G::row(lz, ly) * G::EX + lx + 4;
    const int ci0 = G::cidx(lz, ly, lx);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int si = si0 + u * DS;
      if (!QOZ_IN(si - 3, G::kS) || !QOZ_IN(si + 3, G::kS) ||
          (inside && !QOZ_IN(ci0 + u * DC, G::kC)))
        continue;
      const float pred = predict_full(S[si - 3], S[si - 1], S[si + 1], S[si + 3], interp_of<G>(c));
      const int uz = ALONG_Y ? lz : lz + u * SZ::step, uy = ALONG_Y ? ly + u * SY::step : ly;
      finish<DECOMP>(a, c, S, IN16, si, pred, inside, C16 + ci0 + u * DC, c.oz + uz, c.oy + uy,
                     c.ox + lx);
    }
  }
}

// ---- a pass along x: one odd-x target per lane.
template <class G, int PASS, bool DECOMP, bool INTERIOR>
__device__ __forceinline__ void pass_x(const LevelLaunch& a, const Ctx& c, float* S,
                                       const uint16_t* IN16, uint16_t* C16) {
  constexpr int A0 = G::A0, A1 = G::A1, A2 = G::A2;
  using SZ = Span<RoleOf<A0, A1, A2, PASS, 0>::value, G::TZ>;
  using SY = Span<RoleOf<A0, A1, A2, PASS, 1>::value, G::TY>;
  constexpr int NTX = G::TX / 2;
  if constexpr (INTERIOR && RoleOf<A0, A1, A2, PASS, 1>::value == kAny && SY::count % 4 == 0) {
    pass_x_rows<G, PASS, DECOMP, 4, true>(a, c, S, IN16, C16);
    return;
  } else if constexpr (INTERIOR && RoleOf<A0, A1, A2, PASS, 0>::value == kAny &&
                       SZ::count % 4 == 0) {
    pass_x_rows<G, PASS, DECOMP, 4, false>(a, c, S, IN16, C16);
    return;
  }
  constexpr int items = SZ::count * SY::count * NTX;
  for (int it = threadIdx.x; it < items; it += G::kThr) {
    const int mm = it % NTX;
    const int t = it / NTX;
    const int yi = t % SY::count;
    const int zi = t / SY::count;
    const int lz = SZ::start + zi * SZ::step, ly = SY::start + yi * SY::step;
    const int lx = 2 * mm + 1;
    const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
    if (!INTERIOR && (cz < 0 || cz >= c.g0 || cy < 0 || cy >= c.g1 || cx >= c.g2)) continue;
    const int si = G::row(lz, ly) * G::EX + lx + 4;
    const bool inside = lz >= 0 && lz < G::TZ && ly >= 0 && ly < G::TY;
    if (!QOZ_IN(si - 3, G::kS) || !QOZ_IN(si + 3, G::kS) ||
        (inside && !QOZ_IN(G::cidx(lz, ly, lx), G::kC)))
      continue;
    const float a3 = S[si - 3], a1 = S[si - 1], b1 = S[si + 1], b3 = S[si + 3];
    float pred;
    if (INTERIOR) {
      pred = predict_full(a3, a1, b1, b3, interp_of<G>(c));
    } else {
      const bool hb1 = cx + 1 < c.g2, ha3 = cx >= 3, hb3 = cx + 3 < c.g2;
      pred = predict(a3, a1, b1, b3, ha3, hb1, hb3, interp_of<G>(c));
    }
    finish<DECOMP>(a, c, S, IN16, si, pred, inside, C16 + G::cidx(lz, ly, lx), cz, cy, cx);
  }
}

template <class G, int PASS, bool DECOMP, bool INTERIOR, bool CBOX = false>
__device__ __forceinline__ void run_pass(const LevelLaunch& a, const Ctx& c, float* S,
                                         const float* CR, const uint16_t* IN16, uint16_t* C16) {
  constexpr int P = PASS == 1 ? G::A0 : (PASS == 2 ? G::A1 : G::A2);
  if constexpr (P == 2)
    pass_x<G, PASS, DECOMP, INTERIOR>(a, c, S, IN16, C16);
  else
    pass_line<G, PASS, DECOMP, INTERIOR, CBOX>(a, c, S, CR, IN16, C16);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// One CTA's tile: tile index b (x fastest) of the launch described by a.
template <int A0, int A1, int A2, int TZ, int TY, int TX, bool DECOMP, bool HIST>
__device__ __forceinline__ void level_tile(const LevelLaunch& a, unsigned char* smem, int b,
                                           int nt1, int nt2, int vec_rows) {
  using G = Geo<A0, A1, A2, TZ, TY, TX>;
  float* S = reinterpret_cast<float*>(smem);
  float* CR = reinterpret_cast<float*>(smem + G::kSBytes);
  unsigned char* tail = smem + G::kSBytes + G::kCRBytes;
  uint16_t* IN16 = reinterpret_cast<uint16_t*>(tail);  // decompress: staged codes
  uint16_t* C16 = reinterpret_cast<uint16_t*>(tail);   // compress: tile codes
  unsigned* SH = reinterpret_cast<unsigned*>(tail + G::kCodeBytes);

  Ctx c;
  {
    const int tx = b % nt2;
    b /= nt2;
    const int ty = b % nt1;
    const int tz = b / nt1;
    c.oz = tz * TZ;
    c.oy = ty * TY;
    c.ox = tx * TX;
  }
  c.g0 = (int)a.g[0];
  c.g1 = (int)a.g[1];
  c.g2 = (int)a.g[2];
  const int lvl = a.level - 1;
  c.el = a.bt->el[lvl];
  c.two_e = a.bt->two_e[lvl];
  c.inv = a.bt->inv[lvl];
  c.interp = a.interp;
  const unsigned xs0 = (unsigned)a.xs[0], xs1 = (unsigned)a.xs[1], xs2 = (unsigned)a.xs[2];
  const unsigned cs0 = (unsigned)a.cs[0], cs1 = (unsigned)a.cs[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (HIST)
    for (int i = threadIdx.x; i < kHistWin; i += kThreads) SH[i] = 0;

  // ---- codes of the tile's coarse points (compress): plain loads issued
  // before the copies so that their latency overlaps them; stored into the
  // code tile once the copies have been issued
  constexpr int NCCZ = (TZ + 1) / 2, NCCY = (TY + 1) / 2, NCCX = TX / 2;
  constexpr int NCC = NCCZ * NCCY * NCCX;
  constexpr int kCCPer = (NCC + kThreads - 1) / kThreads;
  uint16_t cc_val[kCCPer];
  int cc_slot[kCCPer];
#pragma unroll
  for (int k = 0; k < kCCPer; ++k) {
    cc_slot[k] = -1;
    cc_val[k] = 0;
    const int i = threadIdx.x + k * kThreads;
    if (DECOMP || i >= NCC) continue;
    const int ix = i % NCCX;
    const int t = i / NCCX;
    const int iy = t % NCCY;
    const int iz = t / NCCY;
    const int lz = 2 * iz, ly = 2 * iy, lx = 2 * ix;
    const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
    if (cz >= c.g0 || cy >= c.g1 || cx >= c.g2) continue;
    cc_slot[k] = G::cidx(lz, ly, lx);
    if (a.cin)
      cc_val[k] = a.cin[(unsigned)(cz >> 1) * cs0 + (unsigned)(cy >> 1) * cs1 + (unsigned)(cx >> 1)];
  }

  // ---- main rows: the field (or the codes) over x in [-4, TX + 4).  Halo
  // rows at odd coordinates hold nothing any pass reads and are skipped.
  for (int r = warp; r < G::NMAIN; r += kWarps) {
    const int lz = r / G::EY - G::HZ;
    const int ly = r % G::EY - G::HY;
    const int cz = c.oz + lz, cy = c.oy + ly;
    if (cz < 0 || cz >= c.g0 || cy < 0 || cy >= c.g1) continue;
    const bool hz = lz < 0 || lz >= TZ, hy = ly < 0 || ly >= TY;
    if ((hz && (cz & 1)) || (hy && (cy & 1))) continue;
    if (!QOZ_IN(r * G::EX + G::EX - 1, G::kS)) continue;
    const unsigned rbase = (unsigned)cz * xs0 + (unsigned)cy * xs1;
    if (vec_rows) {
      // groups of four x: 16-byte copies of the field (8 bytes of codes)
      for (int i = lane; i < G::EX / 4; i += 32) {
        const int gx = c.ox - 4 + 4 * i;
        if (gx >= 0 && gx + 4 <= c.g2) {
          if (DECOMP)
            cp_async8(IN16 + r * G::EX + 4 * i, a.cin + rbase + (unsigned)gx);
          else
            cp_async16(S + r * G::EX + 4 * i, a.x + rbase + (unsigned)gx);
        } else {
          for (int k = 0; k < 4; ++k) {
            const int xx = gx + k;
            if (xx < 0 || xx >= c.g2) continue;
            if (DECOMP)
              IN16[r * G::EX + 4 * i + k] = a.cin[rbase + (unsigned)xx];
            else
              cp_async4(S + r * G::EX + 4 * i + k, a.x + rbase + (unsigned)xx);
          }
        }
      }
    } else {
      for (int lx = lane - 4; lx < TX + 4; lx += 32) {
        const int cx = c.ox + lx;
        if (cx < 0 || cx >= c.g2) continue;
        const unsigned xi = rbase + (unsigned)cx * xs2;
        if (DECOMP)
          IN16[r * G::EX + lx + 4] = a.cin[xi];
        else
          cp_async4(S + r * G::EX + lx + 4, a.x + xi);
      }
    }
  }
  // ---- coarse reconstruction into the staging rows: the main box's coarse
  // rows, then the side rows (A0 = -2, T0, T0 + 2)
  for (int r = warp; r < G::NCMAIN + G::NSIDE; r += kWarps) {
    int lz, ly;
    if (r < G::NCMAIN) {
      lz = G::ZLO + 2 * (r / G::NCY);
      ly = G::YLO + 2 * (r % G::NCY);
    } else {
      const int k = (r - G::NCMAIN) / G::NOS;
      const int other = 2 * ((r - G::NCMAIN) % G::NOS) - 2;
      const int a0pos = k == 0 ? -2 : G::T0 + 2 * (k - 1);
      lz = A0 == 0 ? a0pos : other;
      ly = A0 == 0 ? other : a0pos;
    }
    const int cz = c.oz + lz, cy = c.oy + ly;
    if (cz < 0 || cz >= c.g0 || cy < 0 || cy >= c.g1) continue;
    const unsigned cb = (unsigned)(cz >> 1) * cs0 + (unsigned)(cy >> 1) * cs1;
    if (!QOZ_IN(r * G::HX + G::HX - 1, G::kCR)) continue;
    for (int j = lane; j < G::HX; j += 32) {
      const int cx = c.ox - 4 + 2 * j;
      if (cx < 0 || cx >= c.g2) continue;
      cp_async4(CR + r * G::HX + j, a.rc + cb + (unsigned)(cx >> 1));
    }
  }
  if (!DECOMP) {
    // the coarse codes fetched first now land in the code tile
#pragma unroll
    for (int k = 0; k < kCCPer; ++k)
      if (cc_slot[k] >= 0 && QOZ_IN(cc_slot[k], G::kC)) C16[cc_slot[k]] = cc_val[k];
  }
  cp_async_wait_all();
  __syncthreads();
  // ---- coarse values into the even positions of the main box's coarse rows
  for (int i = threadIdx.x; i < G::NCMAIN * G::HX; i += kThreads) {
    const int j = i % G::HX;
    const int r = i / G::HX;
    const int lz = G::ZLO + 2 * (r / G::NCY), ly = G::YLO + 2 * (r % G::NCY);
    const int si = G::row(lz, ly) * G::EX + 2 * j;
    if (QOZ_IN(si, G::kS) && QOZ_IN(i, G::kCR)) S[si] = CR[i];
  }
  __syncthreads();

  if (G::interior(c.oz, c.oy, c.ox, c.g0, c.g1, c.g2)) {
    run_pass<G, 1, DECOMP, true>(a, c, S, CR, IN16, C16);
    __syncthreads();
    run_pass<G, 2, DECOMP, true>(a, c, S, CR, IN16, C16);
    __syncthreads();
    run_pass<G, 3, DECOMP, true>(a, c, S, CR, IN16, C16);
  } else {
    run_pass<G, 1, DECOMP, false>(a, c, S, CR, IN16, C16);
    __syncthreads();
    run_pass<G, 2, DECOMP, false>(a, c, S, CR, IN16, C16);
    __syncthreads();
    run_pass<G, 3, DECOMP, false>(a, c, S, CR, IN16, C16);
  }
  __syncthreads();

  // ---- outputs, eight points per thread along x: compact codes
  // (compress), compact reconstruction, histogram
  static_assert(TX % 8 == 0, "tile rows hold whole groups of eight");
  constexpr int NG = TZ * TY * (TX / 8);
  const unsigned os0 = (unsigned)a.os[0], os1 = (unsigned)a.os[1];
  const bool rows8 = (a.os[1] % 8) == 0 && (a.os[0] % 8) == 0;
  const bool vec_codes = rows8 && (reinterpret_cast<uintptr_t>(a.cout) & 15) == 0;
  const bool vec_rec = rows8 && (reinterpret_cast<uintptr_t>(a.rout) & 15) == 0;
  for (int i = threadIdx.x; i < NG; i += kThreads) {
    const int gx = i % (TX / 8);
    const int t = i / (TX / 8);
    const int ly = t % TY;
    const int lz = t / TY;
    const int lx = gx * 8;
    const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
    if (cz >= c.g0 || cy >= c.g1 || cx >= c.g2) continue;
    const unsigned oi = (unsigned)cz * os0 + (unsigned)cy * os1 + (unsigned)cx;
    const bool full = cx + 8 <= c.g2;
    if (!QOZ_IN(G::cidx(lz, ly, lx) + 7, G::kC) ||
        !QOZ_IN(G::row(lz, ly) * G::EX + lx + 11, G::kS) ||
        !QOZ_IN((long long)oi + (full ? 7 : c.g2 - 1 - cx), (long long)c.g0 * os0))
      continue;
    if (!DECOMP) {
      const uint4 v = *reinterpret_cast<const uint4*>(C16 + G::cidx(lz, ly, lx));
      if (full && vec_codes) {
        *reinterpret_cast<uint4*>(a.cout + oi) = v;
      } else {
        const uint16_t* cv = reinterpret_cast<const uint16_t*>(&v);
        for (int k = 0; k < 8 && cx + k < c.g2; ++k) a.cout[oi + k] = cv[k];
      }
      if (HIST) {
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (cx + k >= c.g2) break;
          const unsigned cd = (wv[k >> 1] >> (16 * (k & 1))) & 0xffffu;
          const unsigned kk = cd - (unsigned)kHistLo;
          if (kk < (unsigned)kHistWin)
            atomicAdd(&SH[kk], 1u);
          else
            atomicAdd(&a.hist[cd], 1u);
        }
      }
    }
    if (a.rout) {
      const float* srow = S + G::row(lz, ly) * G::EX + lx + 4;
      const float4 v0 = *reinterpret_cast<const float4*>(srow);
      const float4 v1 = *reinterpret_cast<const float4*>(srow + 4);
      if (full && vec_rec) {
        float4* o4 = reinterpret_cast<float4*>(a.rout + oi);
        o4[0] = v0;
        o4[1] = v1;
      } else {
        const float r8[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        for (int k = 0; k < 8 && cx + k < c.g2; ++k) a.rout[oi + k] = r8[k];
      }
    }
  }
  if (HIST) {
    __syncthreads();
    for (int i = threadIdx.x; i < kHistWin; i += kThreads)
      if (SH[i]) atomicAdd(&a.hist[kHistLo + i], SH[i]);
  }
}


// ---- level 1 with bulk tensor copies (TMA) ---------------------------------
// The tile's input box (field over the main box, coarse reconstruction box,
// coarse code box) arrives as three cp.async.bulk.tensor copies issued by
// one thread and tracked by one mbarrier; the tile's codes leave as one
// bulk tensor store.  The passes are the same as in level_tile (pass 1 reads
// the coarse values beyond the tile along A0 from the coarse box).

// Tile (z, y, x extents and threads) of the bulk-copy level-1 launches, by
// the axis the level's order takes first: the first axis carries no halo and
// gets the short extent; 256-thread CTAs, four per SM.  2-D fields (z extent
// 1) take 32 x 128 tiles with 512 threads.
struct TmaTile {
  int tz, ty, tx, thr;
};
__host__ __device__ constexpr TmaTile tma_tile_for(bool is2d, int a0) {
  return is2d ? TmaTile{1, 32, 128, 512}
              : (a0 == 0 ? TmaTile{8, 16, 32, 256}
                         : (a0 == 1 ? TmaTile{16, 8, 32, 256} : TmaTile{8, 8, 32, 256}));
}
// The first axis of each 3-D order (orders enumerate the axis permutations
// lexicographically).
constexpr int kOrderAxis0[6] = {0, 0, 1, 1, 2, 2};

// Polls of the tile's mbarrier before the CTA gives up (a copy that has not
// landed after this many polls is reported through a.err, bit 2).
constexpr unsigned kTmaWaitPolls = 1u << 24;

// map_x: the field (f32, dims x, y, z); map_rc: coarse reconstruction (f32);
// map_cc: coarse codes (u16); map_out: the codes (u16), or nullptr to store
// them with plain stores.
template <int A0, int A1, int A2, int TZ, int TY, int TX, int THR, int IP, bool HIST>
__device__ __forceinline__ void level_tile_tma(const LevelLaunch& a, unsigned char* smem_raw,
                                               uint64_t* mbar, int b, int nt1, int nt2,
                                               const void* map_x, const void* map_rc,
                                               const void* map_cc, const void* map_out) {
  using G = Geo<A0, A1, A2, TZ, TY, TX, THR, IP>;
  // 128-byte aligned sub-buffers (bulk tensor copies need it)
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float* S = reinterpret_cast<float*>(smem);
  float* CB = reinterpret_cast<float*>(smem + G::kTmaS);
  uint16_t* C16 = reinterpret_cast<uint16_t*>(smem + G::kTmaS + G::kTmaCB);
  uint16_t* CC = reinterpret_cast<uint16_t*>(smem + G::kTmaS + G::kTmaCB + G::kTmaC16);
  unsigned* SH =
      reinterpret_cast<unsigned*>(smem + G::kTmaS + G::kTmaCB + G::kTmaC16 + G::kTmaCC);

  Ctx c;
  {
    const int tx = b % nt2;
    b /= nt2;
    const int ty = b % nt1;
    const int tz = b / nt1;
    c.oz = tz * TZ;
    c.oy = ty * TY;
    c.ox = tx * TX;
  }
  c.g0 = (int)a.g[0];
  c.g1 = (int)a.g[1];
  c.g2 = (int)a.g[2];
  const int lvl = a.level - 1;
  c.el = a.bt->el[lvl];
  c.two_e = a.bt->two_e[lvl];
  c.inv = a.bt->inv[lvl];
  c.interp = a.interp;

  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    constexpr unsigned kBytes = (unsigned)(sizeof(float) * (G::kS + G::kCB) +
                                           sizeof(uint16_t) * G::kCC);
    mbar_expect_tx(mbar, kBytes);
    tma_load_3d(S, map_x, c.ox - 4, c.oy - G::HY, c.oz - G::HZ, mbar);
    tma_load_3d(CB, map_rc, c.ox / 2 - 4, c.oy / 2 - 2, c.oz / 2 - 2, mbar);
    tma_load_3d(CC, map_cc, c.ox / 2, c.oy / 2, c.oz / 2, mbar);
  }
  if (HIST)
    for (int i = threadIdx.x; i < kTmaHistWin; i += THR) SH[i] = 0;
  bool landed = false;
  for (unsigned it = 0; it < kTmaWaitPolls; ++it)
    if (mbar_try_wait(mbar, 0)) {
      landed = true;
      break;
    }
  landed = __syncthreads_and(landed) != 0;
  if (landed && a.extra_tx > 0) {
    // host fault injection: once the copies have landed, the barrier's next
    // phase expects bytes that never come, and its bounded wait runs out
    // with no copy in flight
    if (threadIdx.x == 0) mbar_expect_tx(mbar, (unsigned)a.extra_tx);
    const unsigned polls = a.wait_polls > 0 ? (unsigned)a.wait_polls : kTmaWaitPolls;
    bool done = false;
    for (unsigned it = 0; it < polls; ++it)
      if (mbar_try_wait(mbar, 1)) {
        done = true;
        break;
      }
    landed = __syncthreads_and(done) != 0;
  }
  if (!landed) {
    if (threadIdx.x == 0 && a.err) atomicOr(a.err, 2);
    return;
  }

  // coarse values into the even positions of the main box's coarse rows
  for (int i = threadIdx.x; i < G::NCMAIN * G::HX; i += THR) {
    const int j = i % G::HX;
    const int r = i / G::HX;
    const int lz = G::ZLO + 2 * (r / G::NCY), ly = G::YLO + 2 * (r % G::NCY);
    const int si = G::row(lz, ly) * G::EX + 2 * j, bi = G::cbidx(lz, ly, 2 * j - 4);
    if (QOZ_IN(si, G::kS) && QOZ_IN(bi, G::kCB)) S[si] = CB[bi];
  }
  // the tile's coarse codes into the code tile
  for (int i = threadIdx.x; i < G::kCC; i += THR) {
    const int ix = i % G::CCX;
    const int t = i / G::CCX;
    const int iy = t % G::CCY;
    const int iz = t / G::CCY;
    const int ci = G::cidx(2 * iz, 2 * iy, 2 * ix);
    if (QOZ_IN(ci, G::kC)) C16[ci] = CC[i];
  }
  __syncthreads();

  if (G::interior(c.oz, c.oy, c.ox, c.g0, c.g1, c.g2)) {
    run_pass<G, 1, false, true, true>(a, c, S, CB, nullptr, C16);
    __syncthreads();
    run_pass<G, 2, false, true, true>(a, c, S, CB, nullptr, C16);
    __syncthreads();
    run_pass<G, 3, false, true, true>(a, c, S, CB, nullptr, C16);
  } else {
    run_pass<G, 1, false, false, true>(a, c, S, CB, nullptr, C16);
    __syncthreads();
    run_pass<G, 2, false, false, true>(a, c, S, CB, nullptr, C16);
    __syncthreads();
    run_pass<G, 3, false, false, true>(a, c, S, CB, nullptr, C16);
  }
  if (map_out) fence_proxy_async_smem();  // code tile written: visible to the bulk store
  __syncthreads();
  if (map_out && threadIdx.x == 0) {
    tma_store_3d(map_out, c.ox, c.oy, c.oz, C16);
    bulk_commit();
  }

  // histogram, reconstruction output and (without a store map) the codes,
  // eight points per thread along x
  static_assert(TX % 8 == 0, "tile rows hold whole groups of eight");
  constexpr int NG = TZ * TY * (TX / 8);
  const bool need_loop = HIST || a.rout || !map_out;
  if (need_loop) {
    const unsigned os0 = (unsigned)a.os[0], os1 = (unsigned)a.os[1];
    const bool rows8 = (a.os[1] % 8) == 0 && (a.os[0] % 8) == 0;
    const bool vec_codes = rows8 && (reinterpret_cast<uintptr_t>(a.cout) & 15) == 0;
    const bool vec_rec = rows8 && (reinterpret_cast<uintptr_t>(a.rout) & 15) == 0;
    for (int i = threadIdx.x; i < NG; i += THR) {
      const int gx = i % (TX / 8);
      const int t = i / (TX / 8);
      const int ly = t % TY;
      const int lz = t / TY;
      const int lx = gx * 8;
      const int cz = c.oz + lz, cy = c.oy + ly, cx = c.ox + lx;
      if (cz >= c.g0 || cy >= c.g1 || cx >= c.g2) continue;
      const unsigned oi = (unsigned)cz * os0 + (unsigned)cy * os1 + (unsigned)cx;
      const bool full = cx + 8 <= c.g2;
      if (!QOZ_IN(G::cidx(lz, ly, lx) + 7, G::kC) ||
          !QOZ_IN(G::row(lz, ly) * G::EX + lx + 11, G::kS) ||
          !QOZ_IN((long long)oi + (full ? 7 : c.g2 - 1 - cx), (long long)c.g0 * os0))
        continue;
      const uint4 v = *reinterpret_cast<const uint4*>(C16 + G::cidx(lz, ly, lx));
      if (!map_out) {
        if (full && vec_codes) {
          *reinterpret_cast<uint4*>(a.cout + oi) = v;
        } else {
          const uint16_t* cv = reinterpret_cast<const uint16_t*>(&v);
          for (int k = 0; k < 8 && cx + k < c.g2; ++k) a.cout[oi + k] = cv[k];
        }
      }
      if (HIST) {
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (cx + k >= c.g2) break;
          const unsigned cd = (wv[k >> 1] >> (16 * (k & 1))) & 0xffffu;
          const unsigned kk = cd - (unsigned)kTmaHistLo;
          if (kk < (unsigned)kTmaHistWin)
            atomicAdd(&SH[kk], 1u);
          else
            atomicAdd(&a.hist[cd], 1u);
        }
      }
      if (a.rout) {
        const float* srow = S + G::row(lz, ly) * G::EX + lx + 4;
        const float4 v0 = *reinterpret_cast<const float4*>(srow);
        const float4 v1 = *reinterpret_cast<const float4*>(srow + 4);
        if (full && vec_rec) {
          float4* o4 = reinterpret_cast<float4*>(a.rout + oi);
          o4[0] = v0;
          o4[1] = v1;
        } else {
          const float r8[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
          for (int k = 0; k < 8 && cx + k < c.g2; ++k) a.rout[oi + k] = r8[k];
        }
      }
    }
  }
  if (HIST) {
    __syncthreads();
    for (int i = threadIdx.x; i < kTmaHistWin; i += THR)
      if (SH[i]) atomicAdd(&a.hist[kTmaHistLo + i], SH[i]);
  }
  // the code tile must stay in shared memory until the store has read it
  if (map_out && threadIdx.x == 0) bulk_wait_read0();
}

}  // namespace
}  // namespace qoz
