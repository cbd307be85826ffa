// Batched level launches: one launch runs one level of many fields (Sec. 5.1
// predictor, Sec. 5.2.2 level-wise bounds) whose kernel instance is the same.
// Each CTA reads its item from the per-CTA map, copies the item's descriptor
// into shared memory and runs the same tile code as the single-field launch,
// so every field's codes, reconstruction, list and histogram are those of a
// single-field compression.  Two row-copy tile shapes per instance are
// compiled, and for level 1 the bulk-copy kernel (one tile per CTA) and, for
// 3-D fields, the persistent bulk-copy kernel of qoz_level1.cuh, whose CTAs
// walk the tiles of all the launch's fields; the batch plan can time them
// on its first run and keep the fastest.
#include "qoz_level1.cuh"
#include "qoz_level_impl.cuh"

namespace qoz {
namespace {

template <int A0, int A1, int A2, int TZ, int TY, int TX, bool HIST>
__global__ void __launch_bounds__(kThreads, 2)
    level_batch_kernel(const LevelItem* __restrict__ items, const uint16_t* __restrict__ map) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) LevelItem it;
  static_assert(sizeof(LevelItem) % 4 == 0 && sizeof(LevelItem) / 4 <= kThreads, "item copy");
  if (threadIdx.x < sizeof(LevelItem) / 4) {
    const unsigned k = map[blockIdx.x];
    reinterpret_cast<unsigned*>(&it)[threadIdx.x] =
        reinterpret_cast<const unsigned*>(items + k)[threadIdx.x];
  }
  __syncthreads();
  level_tile<A0, A1, A2, TZ, TY, TX, false, HIST>(it.L, smem, (int)(blockIdx.x - it.tile_begin),
                                                  it.nt1, it.nt2, it.vec);
}

// Level 1 with bulk tensor copies: the item's tensor maps sit in device
// memory next to the item table.
template <int A0, int A1, int A2, int TZ, int TY, int TX, int THR, int IP>
__global__ void __launch_bounds__(THR, 1024 / THR)
    level_tma_batch_kernel(const LevelItem* __restrict__ items, const uint16_t* __restrict__ map,
                           const LevelTmaMaps* __restrict__ maps) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(16) LevelItem it;
  __shared__ __align__(8) uint64_t mbar;
  const unsigned k = map[blockIdx.x];
  if (threadIdx.x < sizeof(LevelItem) / 4)
    reinterpret_cast<unsigned*>(&it)[threadIdx.x] =
        reinterpret_cast<const unsigned*>(items + k)[threadIdx.x];
  __syncthreads();
  const LevelTmaMaps* mp = maps + k;
  level_tile_tma<A0, A1, A2, TZ, TY, TX, THR, IP, true>(
      it.L, smem, &mbar, (int)(blockIdx.x - it.tile_begin), it.nt1, it.nt2, &mp->x, &mp->rc,
      &mp->cc, mp->use_out ? &mp->out : nullptr);
}

// Level 1 of 3-D fields on the persistent bulk-copy kernel: grid-stride CTAs
// over all the launch's tiles (ntiles), each tile's item from the map.  The
// per-item state costs registers: three CTAs per SM (85 registers) keep the
// kernel free of spills, where four (64) spilled.
constexpr int kBatchL1CtasPerSm = 4;
template <int A0, int A1, int A2, int IP>
__global__ void __launch_bounds__(l1::kThr, kBatchL1CtasPerSm)
    level1_batch_kernel(const LevelItem* __restrict__ items, const uint16_t* __restrict__ map,
                        const LevelTmaMaps* __restrict__ maps, int ntiles) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[3];
  __shared__ __align__(16) LevelItem it;
  constexpr l1::Tile3 t = l1::tile_for(A0);
  l1::compress_tiles_batch<l1::Geo<A0, A1, A2, t.tz, t.ty, t.tx>, IP>(items, map, maps, ntiles,
                                                                       smem, mbar, it);
}

struct Info {
  const void* fn;
  size_t smem;
  int t[3];
  int threads;
  unsigned long long* done;
  bool persistent;  // grid-stride CTAs (one per resident slot) over the tiles
};

template <int A0, int A1, int A2, int TZ, int TY, int TX, bool HIST>
Info info_of() {
  using G = Geo<A0, A1, A2, TZ, TY, TX>;
  static unsigned long long done = 0;
  constexpr size_t smem = G::smem_bytes(false, HIST);
  static_assert(smem + sizeof(LevelItem) <= 112 * 1024, "two CTAs per SM");
  return Info{(const void*)level_batch_kernel<A0, A1, A2, TZ, TY, TX, HIST>, smem, {TZ, TY, TX},
              kThreads, &done, false};
}

template <int A0, int A1, int A2, bool IS2D, int IP>
Info info_tma() {
  constexpr TmaTile t = tma_tile_for(IS2D, A0);
  using G = Geo<A0, A1, A2, t.tz, t.ty, t.tx, t.thr, IP>;
  static unsigned long long done = 0;
  constexpr size_t smem = G::tma_smem_bytes(true);
  static_assert((smem + sizeof(LevelItem) + 1088) * (1024 / t.thr) <= 228 * 1024,
                "tiles must fit the CTAs per SM");
  return Info{(const void*)level_tma_batch_kernel<A0, A1, A2, t.tz, t.ty, t.tx, t.thr, IP>, smem,
              {t.tz, t.ty, t.tx}, t.thr, &done, false};
}

template <int A0, int A1, int A2, int IP>
Info info_l1() {
  constexpr l1::Tile3 t = l1::tile_for(A0);
  using G = l1::Geo<A0, A1, A2, t.tz, t.ty, t.tx>;
  static unsigned long long done = 0;
  constexpr size_t smem = G::kSmem;
  static_assert((smem + sizeof(LevelItem) + 1024 + 64) * kBatchL1CtasPerSm <= 228 * 1024,
                "CTAs per SM");
  return Info{(const void*)level1_batch_kernel<A0, A1, A2, IP>, smem, {t.tz, t.ty, t.tx},
              l1::kThr, &done, true};
}

template <int IP>
Info info_l1_ip(int order3) {
  switch (order3) {
    case 0: return info_l1<0, 1, 2, IP>();
    case 1: return info_l1<0, 2, 1, IP>();
    case 2: return info_l1<1, 0, 2, IP>();
    case 3: return info_l1<1, 2, 0, IP>();
    case 4: return info_l1<2, 0, 1, IP>();
    default: return info_l1<2, 1, 0, IP>();
  }
}

template <int IP>
Info info_tma_ip(int is2d, int order3) {
  if (is2d) return order3 == 0 ? info_tma<0, 1, 2, true, IP>() : info_tma<0, 2, 1, true, IP>();
  switch (order3) {
    case 0: return info_tma<0, 1, 2, false, IP>();
    case 1: return info_tma<0, 2, 1, false, IP>();
    case 2: return info_tma<1, 0, 2, false, IP>();
    case 3: return info_tma<1, 2, 0, false, IP>();
    case 4: return info_tma<2, 0, 1, false, IP>();
    default: return info_tma<2, 1, 0, false, IP>();
  }
}

// Tile shapes: variant 0 is the single-field launch's shape; variant 1
// trades halo along one axis for extent along another.
template <bool HIST>
Info info_h(int is2d, int order3, int v) {
  if (is2d) {
    if (order3 == 0)
      return v ? info_of<0, 1, 2, 1, 64, 128, HIST>() : info_of<0, 1, 2, 1, 32, 128, HIST>();
    return v ? info_of<0, 2, 1, 1, 64, 128, HIST>() : info_of<0, 2, 1, 1, 32, 128, HIST>();
  }
  switch (order3) {
    case 0: return v ? info_of<0, 1, 2, 4, 32, 64, HIST>() : info_of<0, 1, 2, 8, 16, 64, HIST>();
    case 1: return v ? info_of<0, 2, 1, 4, 32, 64, HIST>() : info_of<0, 2, 1, 8, 16, 64, HIST>();
    case 2: return v ? info_of<1, 0, 2, 32, 4, 64, HIST>() : info_of<1, 0, 2, 16, 8, 64, HIST>();
    case 3: return v ? info_of<1, 2, 0, 32, 4, 64, HIST>() : info_of<1, 2, 0, 16, 8, 64, HIST>();
    // x first: no 48-wide tile (its instances spilled 116-136 bytes at the
    // 64-register cap of two 512-thread CTAs per SM)
    case 4: return v ? info_of<2, 0, 1, 16, 12, 32, HIST>() : info_of<2, 0, 1, 12, 16, 32, HIST>();
    default:
      return v ? info_of<2, 1, 0, 16, 12, 32, HIST>() : info_of<2, 1, 0, 12, 16, 32, HIST>();
  }
}

Info get_info(const LevelKey& k) {
  if (k.variant == kLevelVariantPersist && !k.is2d)
    return k.interp == 1 ? info_l1_ip<1>(k.order3) : info_l1_ip<0>(k.order3);
  if (k.variant == kLevelVariantBulk || k.variant == kLevelVariantPersist)
    return k.interp == 1 ? info_tma_ip<1>(k.is2d, k.order3) : info_tma_ip<0>(k.is2d, k.order3);
  const int v = k.variant ? 1 : 0;
  return k.hist ? info_h<true>(k.is2d, k.order3, v) : info_h<false>(k.is2d, k.order3, v);
}

}  // namespace

void level_tile_shape(const LevelKey& k, int t[3]) {
  const Info in = get_info(k);
  for (int i = 0; i < 3; ++i) t[i] = in.t[i];
}

long long level_item_tiles(const LevelKey& k, const LevelLaunch& L, long long nt[3]) {
  int t[3];
  level_tile_shape(k, t);
  for (int i = 0; i < 3; ++i) nt[i] = L.g[i] > 0 ? (L.g[i] + t[i] - 1) / t[i] : 0;
  return nt[0] * nt[1] * nt[2];
}

cudaError_t level_batch_prepare(const LevelKey& k) {
  const Info in = get_info(k);
  return ensure_smem_attr(in.fn, in.done, in.smem);
}

cudaError_t launch_level_batch(const LevelKey& k, const LevelItem* d_items, const uint16_t* d_map,
                               const LevelTmaMaps* d_maps, unsigned nblocks, cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  const Info in = get_info(k);
  if (in.persistent) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      nsm = 1;
    const unsigned slots = (unsigned)(kBatchL1CtasPerSm * (nsm > 0 ? nsm : 1));
    int ntiles = (int)nblocks;
    void* args[] = {(void*)&d_items, (void*)&d_map, (void*)&d_maps, (void*)&ntiles};
    cudaError_t e = cudaLaunchKernel(in.fn, dim3(nblocks < slots ? nblocks : slots),
                                     dim3(in.threads), args, in.smem, s);
    note_launch(1);
    return e;
  }
  void* args[] = {(void*)&d_items, (void*)&d_map, (void*)&d_maps};
  cudaError_t e = cudaLaunchKernel(in.fn, dim3(nblocks), dim3(in.threads), args, in.smem, s);
  note_launch(1);
  return e;
}

}  // namespace qoz

#ifdef QOZ_DEBUG_BOUNDS
namespace qoz {
// This translation unit's record of failed index checks (bounds-checking build).
unsigned long long bounds_take_level_batch(bool reset) { return bounds_take(reset); }
}  // namespace qoz
#endif
