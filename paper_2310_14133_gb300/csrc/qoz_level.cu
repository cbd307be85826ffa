// Single-field launches of the level kernel (templates in qoz_level_impl.cuh),
// the anchor gather, and the kernel-attribute helper shared with the batched
// launches.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>

#include "qoz_level1.cuh"
#include "qoz_level_impl.cuh"

namespace qoz {

// The driver's tensor-map encoder, looked up through the runtime (the
// library does not link the driver library itself, so that it loads on
// hosts without a GPU driver); null when unavailable.
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// A rank-3 tiled tensor map (dims and box innermost first; strides in bytes
// of dims 1 and 2); false when the driver rejects it.
bool encode_tensor_map_3d(CUtensorMap* m, CUtensorMapDataType type, const void* base,
                const unsigned long long dims[3], const unsigned long long strides[2],
                const unsigned box[3]) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  const cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
  const cuuint64_t st[2] = {strides[0], strides[1]};
  const cuuint32_t bx[3] = {box[0], box[1], box[2]};
  return enc(m, type, 3, const_cast<void*>(base), d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// Level-1 compression with bulk tensor copies (see level_tile_tma).
template <int A0, int A1, int A2, int TZ, int TY, int TX, int THR, int IP, bool HIST>
__global__ void __launch_bounds__(THR, 1024 / THR)
    level_tma_kernel(const LevelLaunch a, int nt1, int nt2, const __grid_constant__ CUtensorMap mx,
                     const __grid_constant__ CUtensorMap mrc,
                     const __grid_constant__ CUtensorMap mcc,
                     const __grid_constant__ CUtensorMap mout, int use_out) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  level_tile_tma<A0, A1, A2, TZ, TY, TX, THR, IP, HIST>(a, smem, &mbar, blockIdx.x, nt1, nt2,
                                                        &mx, &mrc, &mcc,
                                                        use_out ? &mout : nullptr);
}

bool tma_enabled() {
  static const int on = [] {
    const char* e = getenv("QOZ_LEVEL_TMA");
    return (e && e[0] == '0') ? 0 : 1;
  }();
  return on != 0;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Runs the level-1 launch with bulk tensor copies when the grid is the field
// itself and every array's rows start on 16-byte boundaries; returns false
// (nothing launched) otherwise.
// Tensor maps of a level-1 launch for tiles TZ x TY x TX with halos HZ, HY:
// the field box, the coarse reconstruction box, the coarse code box and (when
// the code array's rows allow) the code tile store; false when an array
// does not meet the bulk-copy alignment rules.
bool encode_level_maps(const LevelLaunch& a, int TZ, int TY, int TX, int HZ, int HY,
                       LevelTmaMaps* m) {
  if (!tma_enabled() || a.decompress || a.xs[2] != 1 || !a.cin || !a.rc) return false;
  if (!aligned16(a.x) || !aligned16(a.rc) || !aligned16(a.cin)) return false;
  if (a.xs[1] % 4 || a.xs[0] % 4 || a.cs[1] % 8 || a.cs[0] % 8) return false;
  const unsigned long long g2 = a.g[2], g1 = a.g[1], g0 = a.g[0];
  const unsigned long long c2 = (g2 + 1) / 2, c1 = (g1 + 1) / 2, c0 = (g0 + 1) / 2;
  memset(m, 0, sizeof(*m));
  {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {4ull * a.xs[1], 4ull * a.xs[0]};
    const unsigned bx[3] = {(unsigned)(TX + 8), (unsigned)(TY + 2 * HY), (unsigned)(TZ + 2 * HZ)};
    if (!encode_tensor_map_3d(&m->x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.x, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {4ull * a.cs[1], 4ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)(TX / 2 + 8), (unsigned)(TY / 2 + 4), (unsigned)(TZ / 2 + 4)};
    if (!encode_tensor_map_3d(&m->rc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.rc, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {2ull * a.cs[1], 2ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)(TX / 2), (unsigned)((TY + 1) / 2), (unsigned)((TZ + 1) / 2)};
    if (!encode_tensor_map_3d(&m->cc, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cin, d, st, bx)) return false;
  }
  m->use_out = 0;
  if (aligned16(a.cout) && a.os[1] % 8 == 0 && a.os[0] % 8 == 0) {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {2ull * a.os[1], 2ull * a.os[0]};
    const unsigned bx[3] = {(unsigned)TX, (unsigned)TY, (unsigned)TZ};
    m->use_out = encode_tensor_map_3d(&m->out, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cout, d, st, bx) ? 1 : 0;
  }
  return true;
}

// Runs the level-1 launch with bulk tensor copies when the grid is the field
// itself and every array's rows start on 16-byte boundaries; returns false
// (nothing launched) otherwise.
template <int A0, int A1, int A2, int TZ, int TY, int TX, int THR, int IP, bool HIST>
bool try_launch_tma(const LevelLaunch& a, cudaStream_t s, cudaError_t* err) {
  using G = Geo<A0, A1, A2, TZ, TY, TX, THR, IP>;
  if (a.interp != IP) return false;
  LevelTmaMaps m;
  if (!encode_level_maps(a, TZ, TY, TX, G::HZ, G::HY, &m)) return false;
  static unsigned long long done = 0;
  constexpr size_t smem = G::tma_smem_bytes(HIST);
  static_assert((smem + 1088) * (1024 / THR) <= 228 * 1024, "tiles must fit the CTAs per SM");
  const void* fn = (const void*)level_tma_kernel<A0, A1, A2, TZ, TY, TX, THR, IP, HIST>;
  cudaError_t e = ensure_smem_attr(fn, &done, smem);
  if (e != cudaSuccess) {
    *err = e;
    return true;
  }
  const long long nt0 = (a.g[0] + TZ - 1) / TZ;
  const long long nt1 = (a.g[1] + TY - 1) / TY;
  const long long nt2 = (a.g[2] + TX - 1) / TX;
  const long long nb = nt0 * nt1 * nt2;
  if (nb > 0x7fffffffLL) {
    *err = cudaErrorInvalidConfiguration;
    return true;
  }
  level_tma_kernel<A0, A1, A2, TZ, TY, TX, THR, IP, HIST><<<(unsigned)nb, THR, smem, s>>>(
      a, (int)nt1, (int)nt2, m.x, m.rc, m.cc, m.out, m.use_out);
  note_launch(1);
  *err = cudaGetLastError();
  return true;
}

// ---- level 1 of a 3-D compression: the persistent bulk-copy kernel
// (qoz_level1.cuh)

template <int A0, int A1, int A2, int IP>
using L1Geo = l1::Geo<A0, A1, A2, l1::tile_for(A0).tz, l1::tile_for(A0).ty, l1::tile_for(A0).tx>;

template <int A0, int A1, int A2, int IP>
__global__ void __launch_bounds__(l1::kThr, l1::kCtasPerSm)
    level1_kernel(const __grid_constant__ LevelLaunch a, int nt1, int nt2, int ntiles,
                  const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mrc,
                  const __grid_constant__ CUtensorMap mcc,
                  const __grid_constant__ CUtensorMap mout) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[3];
  l1::compress_tiles<L1Geo<A0, A1, A2, IP>, IP>(a, smem, mbar, nt1, nt2, ntiles, &mx, &mrc,
                                                &mcc, &mout);
}

bool l1_enabled() {
  static const int on = [] {
    const char* e = getenv("QOZ_L1");
    return (e && e[0] == '0') ? 0 : 1;
  }();
  return on != 0;
}

// Streaming multiprocessors of the current device (cached per device).
int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  int& v = cache[dev & 63];
  if (v == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    v = n;
  }
  return v;
}

// Launches level 1 of a 3-D compression on the persistent kernel when the
// field, the coarse arrays and the code array meet the bulk-copy rules;
// returns false (nothing launched) otherwise.
template <int A0, int A1, int A2, int IP>
bool try_launch_l1(const LevelLaunch& a, cudaStream_t s, cudaError_t* err) {
  using G = L1Geo<A0, A1, A2, IP>;
  if (!l1_enabled() || !tma_enabled() || a.decompress || a.is2d || a.level != 1 ||
      a.xs[2] != 1 || !a.cin || !a.rc || !a.cout || !a.hist)
    return false;
  if (!aligned16(a.x) || !aligned16(a.rc) || !aligned16(a.cin) || !aligned16(a.cout))
    return false;
  if (a.xs[1] % 4 || a.xs[0] % 4 || a.cs[1] % 8 || a.cs[0] % 8 || a.os[1] % 8 || a.os[0] % 8)
    return false;
  const unsigned long long g2 = a.g[2], g1 = a.g[1], g0 = a.g[0];
  const unsigned long long c2 = (g2 + 1) / 2, c1 = (g1 + 1) / 2, c0 = (g0 + 1) / 2;
  CUtensorMap mx, mrc, mcc, mout;
  {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {4ull * a.xs[1], 4ull * a.xs[0]};
    const unsigned bx[3] = {(unsigned)G::EX, (unsigned)G::EY, (unsigned)G::EZ};
    if (!encode_tensor_map_3d(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.x, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {4ull * a.cs[1], 4ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)G::CBX, (unsigned)G::CBY, (unsigned)G::CBZ};
    if (!encode_tensor_map_3d(&mrc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.rc, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {2ull * a.cs[1], 2ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)G::CCX, (unsigned)G::CCY, (unsigned)G::CCZ};
    if (!encode_tensor_map_3d(&mcc, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cin, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {2ull * a.os[1], 2ull * a.os[0]};
    const unsigned bx[3] = {(unsigned)G::TX, (unsigned)G::TY, (unsigned)G::TZ};
    if (!encode_tensor_map_3d(&mout, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cout, d, st, bx))
      return false;
  }
  static unsigned long long done = 0;
  constexpr size_t smem = G::kSmem;
  static_assert((smem + 1024 + 64) * l1::kCtasPerSm <= 228 * 1024, "CTAs per SM");
  const void* fn = (const void*)level1_kernel<A0, A1, A2, IP>;
  cudaError_t e = ensure_smem_attr(fn, &done, smem);
  if (e != cudaSuccess) {
    *err = e;
    return true;
  }
  const long long nt0 = (a.g[0] + G::TZ - 1) / G::TZ;
  const long long nt1 = (a.g[1] + G::TY - 1) / G::TY;
  const long long nt2 = (a.g[2] + G::TX - 1) / G::TX;
  const long long nt = nt0 * nt1 * nt2;
  if (nt > 0x7fffffffLL) {
    *err = cudaErrorInvalidConfiguration;
    return true;
  }
  const long long slots = (long long)l1::kCtasPerSm * sm_count();
  const unsigned grid = (unsigned)(nt < slots ? nt : (slots > 0 ? slots : 1));
  level1_kernel<A0, A1, A2, IP><<<grid, l1::kThr, smem, s>>>(a, (int)nt1, (int)nt2, (int)nt, mx,
                                                             mrc, mcc, mout);
  note_launch(1);
  *err = cudaGetLastError();
  return true;
}

template <int A0, int A1, int A2, int IP>
__global__ void __launch_bounds__(l1::kThr, l1::kDecCtasPerSm)
    level1_dec_kernel(const __grid_constant__ LevelLaunch a, int nt1, int nt2, int ntiles,
                      const __grid_constant__ CUtensorMap mcode,
                      const __grid_constant__ CUtensorMap mrc) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[1];
  l1::decompress_tiles<L1Geo<A0, A1, A2, IP>, IP>(a, smem, mbar, nt1, nt2, ntiles, &mcode, &mrc);
}

// Level 1 of a 3-D decompression on the persistent kernel, under the same
// bulk-copy rules (16-byte rows of the code array: x extent a multiple of 8);
// false (nothing launched) otherwise.
template <int A0, int A1, int A2, int IP>
bool try_launch_l1_dec(const LevelLaunch& a, cudaStream_t s, cudaError_t* err) {
  using G = L1Geo<A0, A1, A2, IP>;
  if (!l1_enabled() || !tma_enabled() || !a.decompress || a.is2d || a.level != 1 ||
      a.xs[2] != 1 || !a.cin || !a.rc || !a.rout)
    return false;
  if (!aligned16(a.cin) || !aligned16(a.rc)) return false;
  if (a.xs[1] % 8 || a.xs[0] % 8 || a.cs[1] % 8 || a.cs[0] % 8) return false;
  const unsigned long long g2 = a.g[2], g1 = a.g[1], g0 = a.g[0];
  const unsigned long long c2 = (g2 + 1) / 2, c1 = (g1 + 1) / 2, c0 = (g0 + 1) / 2;
  CUtensorMap mcode, mrc;
  {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {2ull * a.xs[1], 2ull * a.xs[0]};
    const unsigned bx[3] = {(unsigned)G::ECX, (unsigned)G::EY, (unsigned)G::EZ};
    if (!encode_tensor_map_3d(&mcode, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cin, d, st, bx))
      return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {4ull * a.cs[1], 4ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)G::CBX, (unsigned)G::CBY, (unsigned)G::CBZ};
    if (!encode_tensor_map_3d(&mrc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.rc, d, st, bx)) return false;
  }
  static unsigned long long done = 0;
  constexpr size_t smem = G::kDecSmem;
  static_assert((smem + 1024 + 64) * l1::kDecCtasPerSm <= 228 * 1024, "CTAs per SM");
  const void* fn = (const void*)level1_dec_kernel<A0, A1, A2, IP>;
  cudaError_t e = ensure_smem_attr(fn, &done, smem);
  if (e != cudaSuccess) {
    *err = e;
    return true;
  }
  const long long nt0 = (a.g[0] + G::TZ - 1) / G::TZ;
  const long long nt1 = (a.g[1] + G::TY - 1) / G::TY;
  const long long nt2 = (a.g[2] + G::TX - 1) / G::TX;
  const long long nt = nt0 * nt1 * nt2;
  if (nt > 0x7fffffffLL) {
    *err = cudaErrorInvalidConfiguration;
    return true;
  }
  const long long slots = (long long)l1::kDecCtasPerSm * sm_count();
  const unsigned grid = (unsigned)(nt < slots ? nt : (slots > 0 ? slots : 1));
  level1_dec_kernel<A0, A1, A2, IP><<<grid, l1::kThr, smem, s>>>(a, (int)nt1, (int)nt2, (int)nt,
                                                                 mcode, mrc);
  note_launch(1);
  *err = cudaGetLastError();
  return true;
}

template <int A0, int A1, int A2>
bool try_l1_order(const LevelLaunch& a, cudaStream_t s, cudaError_t* err) {
  if (a.decompress)
    return a.interp == 1 ? try_launch_l1_dec<A0, A1, A2, 1>(a, s, err)
                         : try_launch_l1_dec<A0, A1, A2, 0>(a, s, err);
  return a.interp == 1 ? try_launch_l1<A0, A1, A2, 1>(a, s, err)
                       : try_launch_l1<A0, A1, A2, 0>(a, s, err);
}

template <int A0, int A1, int A2, int TZ, int TY, int TX, bool DECOMP, bool HIST>
__global__ void __launch_bounds__(kThreads, 2) level_kernel(const LevelLaunch a, int nt1, int nt2,
                                                            int vec_rows) {
  extern __shared__ __align__(16) unsigned char smem[];
  level_tile<A0, A1, A2, TZ, TY, TX, DECOMP, HIST>(a, smem, blockIdx.x, nt1, nt2, vec_rows);
}

__global__ void anchor_gather_kernel(const float* __restrict__ x, float* __restrict__ anchors,
                                     long long na0, long long na1, long long na2, long long fst0,
                                     long long fst1, long long stride) {
  const long long n = na0 * na1 * na2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long i2 = i % na2;
    const long long r = i / na2;
    const long long i1 = r % na1;
    const long long i0 = r / na1;
    anchors[i] = x[stride * (i0 * fst0 + i1 * fst1 + i2)];
  }
}

template <int A0, int A1, int A2, int IP, bool HIST>
bool try_tma_order_ip(const LevelLaunch& a, cudaStream_t s, cudaError_t* err) {
  constexpr TmaTile t = tma_tile_for(false, A0);
  return try_launch_tma<A0, A1, A2, t.tz, t.ty, t.tx, t.thr, IP, HIST>(a, s, err);
}

// One instance per interpolator (the level's interpolator is a compile-time
// constant inside the tile code).
template <int A0, int A1, int A2, bool HIST>
bool try_tma_order(const LevelLaunch& a, cudaStream_t s, cudaError_t* err) {
  return a.interp == 1 ? try_tma_order_ip<A0, A1, A2, 1, HIST>(a, s, err)
                       : try_tma_order_ip<A0, A1, A2, 0, HIST>(a, s, err);
}

template <int A0, int A1, int A2, int TZ, int TY, int TX, bool DECOMP, bool HIST>
cudaError_t launch_one(const LevelLaunch& a, cudaStream_t s) {
  using G = Geo<A0, A1, A2, TZ, TY, TX>;
  if constexpr (DECOMP && TZ > 1) {  // level 1 of a 3-D decompression
    cudaError_t te = cudaSuccess;
    if (try_l1_order<A0, A1, A2>(a, s, &te)) return te;
  }
  if constexpr (!DECOMP && HIST) {  // level 1 of a compression (the histogram launch)
    cudaError_t te = cudaSuccess;
    if constexpr (TZ > 1) {
      if (try_l1_order<A0, A1, A2>(a, s, &te)) return te;
      if (try_tma_order<A0, A1, A2, HIST>(a, s, &te)) return te;
    } else {
      constexpr TmaTile t = tma_tile_for(true, A0);
      const bool done =
          a.interp == 1 ? try_launch_tma<A0, A1, A2, t.tz, t.ty, t.tx, t.thr, 1, HIST>(a, s, &te)
                        : try_launch_tma<A0, A1, A2, t.tz, t.ty, t.tx, t.thr, 0, HIST>(a, s, &te);
      if (done) return te;
    }
  }
  static unsigned long long done = 0;
  constexpr size_t smem = G::smem_bytes(DECOMP, HIST);
  static_assert(smem <= 112 * 1024, "tile must leave room for two CTAs per SM");
  const void* fn = (const void*)level_kernel<A0, A1, A2, TZ, TY, TX, DECOMP, HIST>;
  cudaError_t e = ensure_smem_attr(fn, &done, smem);
  if (e != cudaSuccess) return e;
  const long long nt0 = (a.g[0] + TZ - 1) / TZ;
  const long long nt1 = (a.g[1] + TY - 1) / TY;
  const long long nt2 = (a.g[2] + TX - 1) / TX;
  const long long nb = nt0 * nt1 * nt2;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  // rows of the input can be read four values at a time when the grid is the
  // field itself, its rows start on four-value boundaries and the base
  // pointer is aligned for the vector width (16 bytes field, 8 bytes codes)
  const void* in = DECOMP ? (const void*)a.cin : (const void*)a.x;
  const int vec = a.xs[2] == 1 && (a.xs[1] % 4) == 0 && (a.xs[0] % 4) == 0 &&
                  (reinterpret_cast<uintptr_t>(in) & (DECOMP ? 7 : 15)) == 0;
  level_kernel<A0, A1, A2, TZ, TY, TX, DECOMP, HIST>
      <<<(unsigned)nb, kThreads, smem, s>>>(a, (int)nt1, (int)nt2, vec);
  note_launch(1);
  return cudaGetLastError();
}

// Tile shape per dimension order: the axis interpolated first carries no
// halo and gets the short extent.
template <bool DECOMP, bool HIST>
cudaError_t dispatch3(const LevelLaunch& a, cudaStream_t s) {
  switch (a.order3) {
    case 0: return launch_one<0, 1, 2, 8, 16, 64, DECOMP, HIST>(a, s);
    case 1: return launch_one<0, 2, 1, 8, 16, 64, DECOMP, HIST>(a, s);
    case 2: return launch_one<1, 0, 2, 16, 8, 64, DECOMP, HIST>(a, s);
    case 3: return launch_one<1, 2, 0, 16, 8, 64, DECOMP, HIST>(a, s);
    case 4: return launch_one<2, 0, 1, 12, 16, 32, DECOMP, HIST>(a, s);
    case 5: return launch_one<2, 1, 0, 12, 16, 32, DECOMP, HIST>(a, s);
  }
  return cudaErrorInvalidValue;
}

// 2D fields (z extent 1): order 0 = (y, x), order 1 = (x, y)
template <bool DECOMP, bool HIST>
cudaError_t dispatch2(const LevelLaunch& a, cudaStream_t s) {
  if (a.order3 == 0) return launch_one<0, 1, 2, 1, 32, 128, DECOMP, HIST>(a, s);
  return launch_one<0, 2, 1, 1, 32, 128, DECOMP, HIST>(a, s);
}

// Batched anchor gather: grid y = field.
__global__ void anchor_batch_kernel(const BatchFieldDesc* __restrict__ d) {
  const BatchFieldDesc& f = d[blockIdx.y];
  const long long na1 = f.na[1], na2 = f.na[2];
  const long long n = f.na[0] * na1 * na2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long i2 = i % na2;
    const long long r = i / na2;
    const long long i1 = r % na1;
    const long long i0 = r / na1;
    f.anchors[i] = f.x[f.stride * (i0 * f.fst0 + i1 * f.fst1 + i2)];
  }
}

}  // namespace

// The opt-in dynamic shared memory limit is a per-device function attribute:
// set it once per (device, kernel instance).
cudaError_t ensure_smem_attr(const void* fn, unsigned long long* done_mask, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) __atomic_fetch_or(done_mask, bit, __ATOMIC_ACQ_REL);
  return e;
}

cudaError_t launch_level(const LevelLaunch& L, cudaStream_t s) {
  if (L.g[0] <= 0 || L.g[1] <= 0 || L.g[2] <= 0) return cudaSuccess;
  const bool hist = !L.decompress && L.hist != nullptr;
  if (L.is2d) {
    if (L.decompress) return dispatch2<true, false>(L, s);
    return hist ? dispatch2<false, true>(L, s) : dispatch2<false, false>(L, s);
  }
  if (L.decompress) return dispatch3<true, false>(L, s);
  return hist ? dispatch3<false, true>(L, s) : dispatch3<false, false>(L, s);
}

cudaError_t launch_anchor_gather(const float* x, float* anchors, const long long na[3],
                                 const long long fst[3], long long stride, cudaStream_t s) {
  const long long n = na[0] * na[1] * na[2];
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  anchor_gather_kernel<<<(unsigned)blocks, threads, 0, s>>>(x, anchors, na[0], na[1], na[2],
                                                            fst[0], fst[1], stride);
  note_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_anchor_batch(const BatchFieldDesc* d, int nfields, cudaStream_t s) {
  if (nfields <= 0) return cudaSuccess;
  anchor_batch_kernel<<<dim3(8, nfields), 256, 0, s>>>(d);
  note_launch(1);
  return cudaGetLastError();
}

// Tensor maps of the persistent level-1 kernel's tiles (the single-field
// launch's boxes, l1::Geo) for a 3-D order whose first axis is a0; false when
// an input array does not meet the bulk-copy rules.
static bool encode_l1_maps(const LevelLaunch& a, int a0, LevelTmaMaps* m) {
  if (!tma_enabled() || a.decompress || a.is2d || a.level != 1 || a.xs[2] != 1 || !a.cin ||
      !a.rc || !a.cout)
    return false;
  if (!aligned16(a.x) || !aligned16(a.rc) || !aligned16(a.cin)) return false;
  if (a.xs[1] % 4 || a.xs[0] % 4 || a.cs[1] % 8 || a.cs[0] % 8) return false;
  const l1::Tile3 t = l1::tile_for(a0);
  const unsigned hz = a0 == 0 ? 0 : 3, hy = a0 == 1 ? 0 : 3, xl = a0 == 2 ? 0 : 4;
  const unsigned long long g2 = a.g[2], g1 = a.g[1], g0 = a.g[0];
  const unsigned long long c2 = (g2 + 1) / 2, c1 = (g1 + 1) / 2, c0 = (g0 + 1) / 2;
  memset(m, 0, sizeof(*m));
  {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {4ull * a.xs[1], 4ull * a.xs[0]};
    const unsigned bx[3] = {t.tx + 2 * xl, t.ty + 2 * hy, t.tz + 2 * hz};
    if (!encode_tensor_map_3d(&m->x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.x, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {4ull * a.cs[1], 4ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)t.tx / 2 + 8, (unsigned)t.ty / 2 + 3, (unsigned)t.tz / 2 + 3};
    if (!encode_tensor_map_3d(&m->rc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a.rc, d, st, bx)) return false;
  }
  {
    const unsigned long long d[3] = {c2, c1, c0};
    const unsigned long long st[2] = {2ull * a.cs[1], 2ull * a.cs[0]};
    const unsigned bx[3] = {(unsigned)t.tx / 2, (unsigned)t.ty / 2, (unsigned)t.tz / 2};
    if (!encode_tensor_map_3d(&m->cc, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cin, d, st, bx)) return false;
  }
  // the code tile's bulk store when the code array's rows start on 16 bytes
  // (else the kernel stores the codes itself)
  m->use_out = 0;
  if (aligned16(a.cout) && a.os[1] % 8 == 0 && a.os[0] % 8 == 0) {
    const unsigned long long d[3] = {g2, g1, g0};
    const unsigned long long st[2] = {2ull * a.os[1], 2ull * a.os[0]};
    const unsigned bx[3] = {(unsigned)t.tx, (unsigned)t.ty, (unsigned)t.tz};
    m->use_out =
        encode_tensor_map_3d(&m->out, CU_TENSOR_MAP_DATA_TYPE_UINT16, a.cout, d, st, bx) ? 1 : 0;
  }
  return true;
}

bool level_tma_maps(const LevelKey& k, const LevelLaunch& L, LevelTmaMaps* m) {
  if (k.variant == kLevelVariantPersist && !k.is2d)
    return encode_l1_maps(L, kOrderAxis0[k.order3], m);
  const int a0 = k.is2d ? 0 : kOrderAxis0[k.order3];
  const TmaTile t = tma_tile_for(k.is2d, a0);
  return encode_level_maps(L, t.tz, t.ty, t.tx, halo_z(a0), halo_y(a0), m);
}

}  // namespace qoz

#ifdef QOZ_DEBUG_BOUNDS
namespace qoz {
// This translation unit's record of failed index checks (bounds-checking build).
unsigned long long bounds_take_level(bool reset) { return bounds_take(reset); }
}  // namespace qoz
#endif
