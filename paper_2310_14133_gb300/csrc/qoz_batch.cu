// Batched compression plans (qoz_batch_* in include/qoz.h): the single-field
// method (Sec. 5.1, 5.2, Eq. (ebl)) applied to many fields at once.
//
// A plan fixes the shapes and parameters of nfields fields.  A run issues
//   table uploads -> init -> value range -> bound tables -> anchors ->
//   levels Lmax..1 (one launch per level and kernel instance) -> finish
//   (anchors out of bin 0, short lists sorted) -> read-back of the counts
// for all fields at once.  Every kernel finds its field through descriptor
// tables in device memory that the run rewrites from pinned host memory as
// its first step, so the same sequence, captured once as a CUDA graph, serves
// every later run whatever the field and output pointers are.  Each field's
// kernels are those of the single-field path (same tile code, same bound
// table arithmetic), so each blob equals the single-field result.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"

using namespace qoz;

namespace {

constexpr int kMaxFields = 4096;
constexpr size_t kAlign = 256;
size_t up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

struct Group {
  int level;
  LevelKey key;
  int item_begin, nitems;   // items of this launch in the item table
  size_t map_begin;         // first entry of its CTA map
  unsigned nblocks;
  double ms[kLevelVariants];  // autotune timings (level 1)
};

// One (field, level) launch inside a group, before pointers are filled.
struct ItemRef {
  int field, level;
  LevelKey key;  // the group's kernel instance
};

}  // namespace

struct qoz_batch {
  int nf = 0;
  int device = 0;
  uint32_t flags = 0;
  std::vector<qoz_shape> shapes;
  std::vector<Resolved> r;
  std::vector<long long> na;
  std::vector<long long> cap;
  std::vector<Coarse> cl;
  // scratch: [bt | cnt | hs] per field (one read-back), lists, coarse grids
  size_t off_bt = 0, off_cnt = 0, off_hs = 0, off_err = 0;
  std::vector<size_t> off_uidx, off_uval, off_coarse;
  size_t scratch_bytes = 0;
  char* d_scratch = nullptr;
  // value range
  std::vector<RangeChunk> chunks;
  std::vector<int> chunk_begin;
  RangeChunk* d_chunks = nullptr;
  float* d_pmin = nullptr;
  float* d_pmax = nullptr;
  unsigned long long* d_pcnt = nullptr;
  // level launches
  std::vector<Group> groups;
  std::vector<ItemRef> refs;      // parallel to the item table
  std::vector<LevelItem> items;   // geometry part (pointers filled per run)
  std::vector<uint16_t> map;
  LevelItem* d_items = nullptr;
  LevelTmaMaps* d_maps = nullptr;  // per item; written for bulk-copy items only
  uint16_t* d_map = nullptr;
  size_t map_cap = 0;
  BatchFieldDesc* d_desc = nullptr;
  // pinned host
  BatchFieldDesc* h_desc = nullptr;
  LevelItem* h_items = nullptr;
  LevelTmaMaps* h_maps = nullptr;
  char* h_back = nullptr;  // read-back of [bt | cnt | hs | err]
  size_t back_bytes = 0;
  // graph
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_rel = -1;  // eb_relative the graph was captured with
  bool autotuned = false;
  bool no_bulk = false;  // a run's arrays did not allow bulk copies: row copies from then on
  bool any_bulk = false;  // the current layout has bulk-copy launches
  int launches = 0;
};

namespace {

BoundTable* bt_of(qoz_batch* p, int f) {
  return reinterpret_cast<BoundTable*>(p->d_scratch + p->off_bt) + f;
}
unsigned long long* cnt_of(qoz_batch* p, int f) {
  return reinterpret_cast<unsigned long long*>(p->d_scratch + p->off_cnt) + f;
}
int* hs_of(qoz_batch* p, int f) { return reinterpret_cast<int*>(p->d_scratch + p->off_hs) + f; }
// Per-field status of a run: bit 2 = a level tile's bulk copy did not
// complete (zeroed by the run's init kernel, read back with the counts).
int* err_of(qoz_batch* p, int f) { return reinterpret_cast<int*>(p->d_scratch + p->off_err) + f; }

// The level launch of (field f, level l) with the plan-owned pointers
// (coarse grids, bound table, list); the per-run pointers (field, anchors,
// codes, histogram) are filled by fill_tables.
LevelLaunch plan_launch(qoz_batch* p, int f, int l) {
  const Resolved& r = p->r[f];
  LevelLaunch L;
  memset(&L, 0, sizeof(L));
  level_geometry(r, l, &L);
  char* coarse = p->d_scratch + p->off_coarse[f];
  const Coarse& cl = p->cl[f];
  L.decompress = false;
  L.rc = l == r.L ? nullptr : (const float*)(coarse + cl.roff[l]);
  L.rout = l > 1 ? (float*)(coarse + cl.roff[l - 1]) : nullptr;
  L.cin = l == r.L ? nullptr : (const uint16_t*)(coarse + cl.coff[l]);
  L.cout = l > 1 ? (uint16_t*)(coarse + cl.coff[l - 1]) : nullptr;
  L.bt = bt_of(p, f);
  L.ul = UnpredList{(long long*)(p->d_scratch + p->off_uidx[f]),
                    (float*)(p->d_scratch + p->off_uval[f]), cnt_of(p, f), p->cap[f]};
  return L;
}

LevelKey key_of(const Resolved& r, int l, int variant) {
  LevelKey k;
  k.is2d = r.ndims == 2;
  k.order3 = r.ndims == 3 ? r.p.order[l - 1] : (r.p.order[l - 1] == 0 ? 0 : 1);
  k.hist = l == 1;
  k.interp = r.p.interp[l - 1];
  k.variant = variant;
  return k;
}

// Level-1 launches are also split by interpolator (the bulk-copy kernel
// fixes it at compile time).
bool same_instance(const LevelKey& a, const LevelKey& b) {
  return a.is2d == b.is2d && a.order3 == b.order3 && a.hist == b.hist &&
         (!a.hist || a.interp == b.interp);
}

// Builds the groups, items and CTA maps for the given level-1 variants
// (variant of every other level: 0).
qoz_status build_launches(qoz_batch* p, const std::vector<int>& l1_variant) {
  p->groups.clear();
  p->refs.clear();
  p->items.clear();
  p->map.clear();
  p->any_bulk = false;
  int Lmax = 0;
  for (int f = 0; f < p->nf; ++f) Lmax = std::max(Lmax, p->r[f].L);
  int l1_index = 0;
  for (int l = Lmax; l >= 1; --l) {
    // distinct kernel instances at this level, in field order of first use
    std::vector<LevelKey> keys;
    for (int f = 0; f < p->nf; ++f) {
      if (p->r[f].L < l) continue;
      const LevelKey k = key_of(p->r[f], l, 0);
      bool seen = false;
      for (const LevelKey& q : keys) seen = seen || same_instance(q, k);
      if (!seen) keys.push_back(k);
    }
    for (LevelKey k : keys) {
      if (l == 1) {
        // default: the persistent bulk-copy kernel for 3-D fields, the
        // one-tile-per-CTA bulk copies for 2-D ones (which have no
        // persistent kernel: 3 falls back to 2)
        k.variant = l1_index < (int)l1_variant.size()
                        ? l1_variant[l1_index]
                        : (p->no_bulk ? 0 : kLevelVariantPersist);
        if (k.variant == kLevelVariantPersist && k.is2d) k.variant = kLevelVariantBulk;
        if ((k.variant == kLevelVariantBulk || k.variant == kLevelVariantPersist) && p->no_bulk)
          k.variant = 0;
        if (k.variant == kLevelVariantBulk || k.variant == kLevelVariantPersist)
          p->any_bulk = true;
        ++l1_index;
      }
      Group g;
      memset(&g, 0, sizeof(g));
      g.level = l;
      g.key = k;
      g.item_begin = (int)p->items.size();
      g.map_begin = p->map.size();
      unsigned long long blocks = 0;
      for (int f = 0; f < p->nf; ++f) {
        if (p->r[f].L < l || !same_instance(key_of(p->r[f], l, 0), k)) continue;
        LevelItem it;
        memset(&it, 0, sizeof(it));
        it.L = plan_launch(p, f, l);
        long long nt[3];
        const long long tiles = level_item_tiles(k, it.L, nt);
        if (tiles <= 0) continue;
        if (p->items.size() >= 65535) return fail(QOZ_EINVAL, "batch has too many launches");
        it.nt1 = (int)nt[1];
        it.nt2 = (int)nt[2];
        it.tile_begin = (unsigned)blocks;
        const uint16_t idx = (uint16_t)p->items.size();
        blocks += (unsigned long long)tiles;
        if (blocks > 0x7fffffffULL) return fail(QOZ_EUNSUPPORTED, "batched launch too large");
        p->map.insert(p->map.end(), (size_t)tiles, idx);
        p->items.push_back(it);
        p->refs.push_back(ItemRef{f, l, k});
      }
      g.nitems = (int)p->items.size() - g.item_begin;
      g.nblocks = (unsigned)blocks;
      if (g.nitems > 0) p->groups.push_back(g);
    }
  }
  return QOZ_OK;
}

// Uploads the CTA maps (synchronously: not part of a run).
qoz_status upload_maps(qoz_batch* p) {
  if (p->map.size() > p->map_cap) {
    if (p->d_map) cudaFree(p->d_map);
    p->d_map = nullptr;
    p->map_cap = 0;
    if (cudaMalloc((void**)&p->d_map, sizeof(uint16_t) * std::max<size_t>(p->map.size(), 1)) !=
        cudaSuccess)
      return fail(QOZ_ENOMEM, "batch CTA map");
    p->map_cap = p->map.size();
  }
  if (!p->map.empty() && cudaMemcpy(p->d_map, p->map.data(), sizeof(uint16_t) * p->map.size(),
                                    cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(QOZ_ECUDA, "batch CTA map upload");
  return QOZ_OK;
}

// Item table sized for the largest layout the plan can have.
qoz_status alloc_items(qoz_batch* p) {
  if (p->h_items) return QOZ_OK;
  size_t n = 0;
  for (int f = 0; f < p->nf; ++f) n += (size_t)p->r[f].L;
  n = std::max<size_t>(n, 1);
  if (cudaMalloc((void**)&p->d_items, sizeof(LevelItem) * n) != cudaSuccess ||
      cudaMallocHost((void**)&p->h_items, sizeof(LevelItem) * n) != cudaSuccess ||
      cudaMalloc((void**)&p->d_maps, sizeof(LevelTmaMaps) * n) != cudaSuccess ||
      cudaMallocHost((void**)&p->h_maps, sizeof(LevelTmaMaps) * n) != cudaSuccess)
    return fail(QOZ_ENOMEM, "batch item table");
  return QOZ_OK;
}

// Per-run pointers into the pinned tables; false when a bulk-copy item's
// arrays do not allow its tensor maps (nothing else is affected).
bool fill_tables(qoz_batch* p, const float* const* x, const double* eb, int rel,
                 qoz_blob* const* outs) {
  bool maps_ok = true;
  for (int f = 0; f < p->nf; ++f) {
    const Resolved& r = p->r[f];
    BatchFieldDesc& d = p->h_desc[f];
    memset(&d, 0, sizeof(d));
    d.x = x[f];
    d.n = r.N;
    d.chunk_begin = p->chunk_begin[f];
    d.nchunks = p->chunk_begin[f + 1] - p->chunk_begin[f];
    d.use_range = rel ? 1 : 0;
    d.L = r.L;
    d.eb = eb[f];
    d.alpha = r.p.alpha;
    d.beta = r.p.beta;
    d.bt = bt_of(p, f);
    d.anchors = outs[f]->d_anchors;
    long long na3[3];
    anchor_dims(r, na3);
    for (int i = 0; i < 3; ++i) d.na[i] = na3[i];
    d.fst0 = r.n[1] * r.n[2];
    d.fst1 = r.n[2];
    d.stride = r.p.anchor_stride;
    d.hist = outs[f]->d_hist;
    d.ul = UnpredList{(long long*)(p->d_scratch + p->off_uidx[f]),
                      (float*)(p->d_scratch + p->off_uval[f]), cnt_of(p, f), p->cap[f]};
    d.err = err_of(p, f);
    d.host_sort = hs_of(p, f);
  }
  const bool inject_wait = fault_injected("tma_wait");
  for (size_t i = 0; i < p->items.size(); ++i) {
    LevelItem it = p->items[i];
    const int f = p->refs[i].field, l = p->refs[i].level;
    const Resolved& r = p->r[f];
    it.L.x = x[f];
    it.L.err = err_of(p, f);
    if (l == 1 && inject_wait) {
      // host fault injection: a barrier phase that expects bytes no copy
      // brings, so the tile's bounded wait runs out after 4096 polls
      it.L.extra_tx = 16;
      it.L.wait_polls = 4096;
    }
    if (l == r.L) it.L.rc = outs[f]->d_anchors;
    if (l == 1) {
      it.L.cout = outs[f]->d_codes;
      it.L.hist = outs[f]->d_hist;
    }
    // 16-byte row copies: the same rule as the single-field launch
    it.vec = it.L.xs[2] == 1 && (it.L.xs[1] % 4) == 0 && (it.L.xs[0] % 4) == 0 &&
             (reinterpret_cast<uintptr_t>(it.L.x) & 15) == 0;
    p->h_items[i] = it;
    if (p->refs[i].key.variant == kLevelVariantBulk ||
        p->refs[i].key.variant == kLevelVariantPersist)
      maps_ok = maps_ok && level_tma_maps(p->refs[i].key, it.L, &p->h_maps[i]);
  }
  return maps_ok;
}

// The run's device sequence on stream s (captured or issued directly).
cudaError_t enqueue(qoz_batch* p, int rel, cudaStream_t s) {
  int launches = 0;
  cudaError_t e = cudaMemcpyAsync(p->d_desc, p->h_desc, sizeof(BatchFieldDesc) * p->nf,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !p->items.empty())
    e = cudaMemcpyAsync(p->d_items, p->h_items, sizeof(LevelItem) * p->items.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && p->any_bulk)
    e = cudaMemcpyAsync(p->d_maps, p->h_maps, sizeof(LevelTmaMaps) * p->items.size(),
                        cudaMemcpyHostToDevice, s);
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) {
      e = r;
      ++launches;
    }
  };
  if (e == cudaSuccess) step(launch_batch_init(p->d_desc, p->nf, s));
  if (e == cudaSuccess && rel)
    step(launch_range_batch(p->d_desc, p->d_chunks, (int)p->chunks.size(), p->d_pmin, p->d_pmax,
                            p->d_pcnt, s));
  if (e == cudaSuccess)
    step(launch_bound_batch(p->d_desc, p->nf, p->d_pmin, p->d_pmax, p->d_pcnt, s));
  if (e == cudaSuccess) step(launch_anchor_batch(p->d_desc, p->nf, s));
  for (const Group& g : p->groups)
    if (e == cudaSuccess)
      step(launch_level_batch(g.key, p->d_items, p->d_map + g.map_begin, p->d_maps, g.nblocks,
                              s));
  if (e == cudaSuccess) step(launch_batch_finish(p->d_desc, p->nf, s));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->h_back, p->d_scratch + p->off_bt, p->back_bytes,
                        cudaMemcpyDeviceToHost, s);
  p->launches = launches;
  return e;
}

qoz_status prepare_kernels(qoz_batch* p) {
  for (const Group& g : p->groups)
    if (level_batch_prepare(g.key) != cudaSuccess) return fail(QOZ_ECUDA, "kernel attributes");
  return QOZ_OK;
}

void drop_graph(qoz_batch* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
  p->graph_rel = -1;
}

qoz_status capture(qoz_batch* p, int rel) {
  drop_graph(p);
  if (!p->cap_stream &&
      cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(QOZ_ECUDA, "capture stream");
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  cudaError_t e2 = enqueue(p, rel, p->cap_stream);
  e = cudaStreamEndCapture(p->cap_stream, &g);
  if (e2 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return cuda_fail(e2 != cudaSuccess ? e2 : e, "capture of the batch sequence");
  }
  e = cudaGraphInstantiate(&p->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p->exec = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  p->graph_rel = rel;
  return QOZ_OK;
}

// Times each tile variant of every level-1 launch on the run just issued
// (inputs in place); the timed launches only add to histograms and lists
// that the next run clears.
qoz_status autotune(qoz_batch* p, int rel, const float* const* x, const double* eb,
                    qoz_blob* const* outs, cudaStream_t s) {
  std::vector<int> l1;
  for (const Group& g : p->groups)
    if (g.level == 1) l1.push_back(0);
  const int n1 = (int)l1.size();
  std::vector<std::vector<double>> ms(n1, std::vector<double>(kLevelVariants, 0.0));
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return fail(QOZ_ECUDA, "events");
  qoz_status st = QOZ_OK;
  for (int v = 0; v < kLevelVariants && st == QOZ_OK; ++v) {
    std::vector<int> vv(n1, v);
    st = build_launches(p, vv);
    if (st == QOZ_OK) st = upload_maps(p);
    if (st == QOZ_OK) st = prepare_kernels(p);
    if (st != QOZ_OK) break;
    if (!fill_tables(p, x, eb, rel, outs)) {
      for (int k = 0; k < n1; ++k) ms[k][v] = 1e30;  // bulk copies not possible here
      continue;
    }
    cudaError_t e = enqueue(p, rel, s);  // coarse levels in place for this layout
    int k = 0;
    for (const Group& g : p->groups) {
      if (g.level != 1 || e != cudaSuccess) continue;
      float best = 1e30f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a, s);
        e = launch_level_batch(g.key, p->d_items, p->d_map + g.map_begin, p->d_maps, g.nblocks,
                               s);
        cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
        best = std::min(best, t);
      }
      ms[k++][v] = best;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "autotune");
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != QOZ_OK) return st;
  for (int k = 0; k < n1; ++k) {
    int best = 0;
    for (int v = 1; v < kLevelVariants; ++v)
      if (ms[k][v] < ms[k][best]) best = v;
    l1[k] = best;
  }
  st = build_launches(p, l1);
  if (st == QOZ_OK) st = upload_maps(p);
  if (st == QOZ_OK) st = prepare_kernels(p);
  if (st != QOZ_OK) return st;
  int k = 0;
  for (Group& g : p->groups)
    if (g.level == 1) {
      for (int v = 0; v < kLevelVariants; ++v) g.ms[v] = ms[k][v];
      ++k;
    }
  p->autotuned = true;
  return QOZ_OK;
}

void free_plan(qoz_batch* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  drop_graph(p);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->d_scratch);
  cudaFree(p->d_chunks);
  cudaFree(p->d_pmin);
  cudaFree(p->d_pmax);
  cudaFree(p->d_pcnt);
  cudaFree(p->d_items);
  cudaFree(p->d_maps);
  cudaFree(p->d_map);
  cudaFree(p->d_desc);
  cudaFreeHost(p->h_desc);
  cudaFreeHost(p->h_items);
  cudaFreeHost(p->h_maps);
  cudaFreeHost(p->h_back);
  delete p;
}

void free_blobs(qoz_blob** outs, int n) {
  for (int i = 0; i < n; ++i) {
    qoz_blob_free(outs[i]);
    outs[i] = nullptr;
  }
}

}  // namespace

extern "C" {

qoz_status qoz_batch_create(const qoz_shape* shapes, int32_t nfields, const qoz_params* params,
                            uint32_t flags, qoz_batch** out) {
  if (!out) return fail(QOZ_EINVAL, "out is NULL");
  *out = nullptr;
  if (!shapes || nfields < 1 || nfields > kMaxFields)
    return fail(QOZ_EINVAL, "nfields must be in [1, %d]", kMaxFields);
  configure_pool_once();
  qoz_batch* p = new qoz_batch();
  p->nf = nfields;
  p->flags = flags;
  cudaGetDevice(&p->device);
  p->shapes.assign(shapes, shapes + nfields);
  p->r.resize(nfields);
  p->na.resize(nfields);
  p->cap.resize(nfields);
  p->cl.resize(nfields);
  for (int f = 0; f < nfields; ++f) {
    const qoz_status st = resolve(shapes[f], params ? &params[f] : nullptr, &p->r[f]);
    if (st != QOZ_OK) {
      free_plan(p);
      return st;
    }
    long long na3[3];
    p->na[f] = anchor_dims(p->r[f], na3);
    const long long N = p->r[f].N;
    long long cap = N / 1024;
    if (cap < 65536) cap = 65536;
    if (cap > N) cap = N > 0 ? N : 1;
    p->cap[f] = cap;
    p->cl[f] = coarse_layout(p->r[f], true);
  }
  // scratch layout
  size_t o = 0;
  p->off_bt = o;
  o += up(sizeof(BoundTable) * nfields);
  p->off_cnt = o;
  o += up(sizeof(unsigned long long) * nfields);
  p->off_hs = o;
  o += up(sizeof(int) * nfields);
  p->off_err = o;
  o += up(sizeof(int) * nfields);
  p->back_bytes = o - p->off_bt;
  p->off_uidx.resize(nfields);
  p->off_uval.resize(nfields);
  p->off_coarse.resize(nfields);
  for (int f = 0; f < nfields; ++f) {
    p->off_uidx[f] = o;
    o += up(sizeof(long long) * p->cap[f]);
    p->off_uval[f] = o;
    o += up(sizeof(float) * p->cap[f]);
    p->off_coarse[f] = o;
    o += up(p->cl[f].bytes);
  }
  p->scratch_bytes = o;
  // value-range chunks
  p->chunk_begin.resize(nfields + 1);
  for (int f = 0; f < nfields; ++f) {
    p->chunk_begin[f] = (int)p->chunks.size();
    for (long long b = 0; b < p->r[f].N; b += kRangeChunk)
      p->chunks.push_back(RangeChunk{f, 0, b, std::min(p->r[f].N, b + kRangeChunk)});
  }
  p->chunk_begin[nfields] = (int)p->chunks.size();
  const size_t nc = std::max<size_t>(p->chunks.size(), 1);
  if (cudaMalloc((void**)&p->d_scratch, p->scratch_bytes) != cudaSuccess ||
      cudaMalloc((void**)&p->d_chunks, sizeof(RangeChunk) * nc) != cudaSuccess ||
      cudaMalloc((void**)&p->d_pmin, sizeof(float) * nc) != cudaSuccess ||
      cudaMalloc((void**)&p->d_pmax, sizeof(float) * nc) != cudaSuccess ||
      cudaMalloc((void**)&p->d_pcnt, sizeof(unsigned long long) * nc) != cudaSuccess ||
      cudaMalloc((void**)&p->d_desc, sizeof(BatchFieldDesc) * nfields) != cudaSuccess ||
      cudaMallocHost((void**)&p->h_desc, sizeof(BatchFieldDesc) * nfields) != cudaSuccess ||
      cudaMallocHost((void**)&p->h_back, p->back_bytes) != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return fail(QOZ_ENOMEM, "batch plan allocation (%zu bytes of scratch)", p->scratch_bytes);
  }
  if (!p->chunks.empty() &&
      cudaMemcpy(p->d_chunks, p->chunks.data(), sizeof(RangeChunk) * p->chunks.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    free_plan(p);
    return fail(QOZ_ECUDA, "batch chunk upload");
  }
  qoz_status st = alloc_items(p);
  if (st == QOZ_OK) st = build_launches(p, std::vector<int>());
  if (st == QOZ_OK) st = upload_maps(p);
  if (st == QOZ_OK) st = prepare_kernels(p);
  if (st != QOZ_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return QOZ_OK;
}

qoz_status qoz_batch_compress(qoz_batch* p, const float* const* d_fields, const double* eb,
                              int32_t eb_relative, void* stream, qoz_blob** outs) {
  if (!p || !d_fields || !eb || !outs) return fail(QOZ_EINVAL, "NULL argument");
  const int rel = eb_relative ? 1 : 0;
  for (int f = 0; f < p->nf; ++f) {
    outs[f] = nullptr;
    if (!d_fields[f]) return fail(QOZ_EINVAL, "d_fields[%d] is NULL", f);
    if (reinterpret_cast<uintptr_t>(d_fields[f]) & 3)
      return fail(QOZ_EINVAL, "d_fields[%d] must be 4-byte aligned", f);
    if (rel && !(eb[f] > 0.0 && std::isfinite(eb[f])))
      return fail(QOZ_EINVAL, "eb[%d] must be finite and > 0", f);
    if (!rel && !(eb[f] >= 0.0 && std::isfinite(eb[f])))
      return fail(QOZ_EINVAL, "eb[%d] must be finite and >= 0", f);
  }
  cudaStream_t s = (cudaStream_t)stream;
  // blobs: codes, anchors, histogram, decode flag (lists after the run)
  for (int f = 0; f < p->nf; ++f) {
    const Resolved& r = p->r[f];
    qoz_blob* b = new qoz_blob();
    memset(b, 0, sizeof(*b));
    b->shape = p->shapes[f];
    for (int i = 0; i < 3; ++i) b->n[i] = r.n[i];
    b->N = r.N;
    b->L = r.L;
    b->params = r.p;
    b->stream = s;
    b->device = p->device;
    b->na = p->na[f];
    outs[f] = b;
    cudaError_t e;
    if ((e = dev_alloc((void**)&b->d_codes, sizeof(uint16_t) * r.N, s)) != cudaSuccess ||
        (e = dev_alloc((void**)&b->d_anchors, sizeof(float) * b->na, s)) != cudaSuccess ||
        (e = dev_alloc((void**)&b->d_hist, sizeof(unsigned) * 65536, s)) != cudaSuccess ||
        (e = dev_alloc((void**)&b->d_err, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_err, 0, sizeof(int), s)) != cudaSuccess) {
      free_blobs(outs, p->nf);
      return fail(QOZ_ENOMEM, "blob allocation: %s", cudaGetErrorString(e));
    }
  }
  qoz_status st = QOZ_OK;
  if ((p->flags & QOZ_BATCH_AUTOTUNE) && !p->autotuned) {
    st = autotune(p, rel, d_fields, eb, outs, s);
    if (st == QOZ_OK) drop_graph(p);
  }
  if (st == QOZ_OK && !fill_tables(p, d_fields, eb, rel, outs)) {
    // this run's arrays rule out bulk copies: row copies from now on
    p->no_bulk = true;
    std::vector<int> l1;
    for (const Group& g : p->groups)
      if (g.level == 1)
        l1.push_back(g.key.variant == kLevelVariantBulk || g.key.variant == kLevelVariantPersist
                         ? 0
                         : g.key.variant);
    st = build_launches(p, l1);
    if (st == QOZ_OK) st = upload_maps(p);
    if (st == QOZ_OK) st = prepare_kernels(p);
    drop_graph(p);
    if (st == QOZ_OK) fill_tables(p, d_fields, eb, rel, outs);
  }
  if (st == QOZ_OK) {
    const bool use_graph = !(p->flags & QOZ_BATCH_NO_GRAPH);
    if (use_graph && (!p->exec || p->graph_rel != rel)) st = capture(p, rel);
    if (st == QOZ_OK) {
      cudaError_t e = use_graph ? cudaGraphLaunch(p->exec, s) : enqueue(p, rel, s);
      if (e == cudaSuccess && use_graph) note_launch(p->launches);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_fail(e, "batch run");
    }
  }
  if (st != QOZ_OK) {
    free_blobs(outs, p->nf);
    return st;
  }
  // per-field results: bound, count, list
  const BoundTable* bt = reinterpret_cast<const BoundTable*>(p->h_back);
  const unsigned long long* cnt =
      reinterpret_cast<const unsigned long long*>(p->h_back + (p->off_cnt - p->off_bt));
  const int* hs = reinterpret_cast<const int*>(p->h_back + (p->off_hs - p->off_bt));
  const int* errs = reinterpret_cast<const int*>(p->h_back + (p->off_err - p->off_bt));
  for (int f = 0; f < p->nf; ++f)
    if (errs[f] & 2) {
      free_blobs(outs, p->nf);
      return fail(QOZ_ETIMEOUT, "field %d: a tile's bulk copy did not complete (flag %d)", f,
                  errs[f]);
    }
  for (int f = 0; f < p->nf && st == QOZ_OK; ++f) {
    qoz_blob* b = outs[f];
    const long long count = (long long)cnt[f];
    if (count > p->cap[f]) {
      // more unpredictable points than the plan's list holds: this field
      // again through the single-field path, which sizes its list itself
      qoz_blob* nb = nullptr;
      st = compress_impl(d_fields[f], p->shapes[f], rel != 0, eb[f], &p->r[f].p, nullptr, s,
                         &nb);
      if (st == QOZ_OK) {
        qoz_blob_free(b);
        outs[f] = nb;
      }
      continue;
    }
    b->nu = count;
    b->abs_eb = bt[f].e;
    b->rel_eb = rel ? eb[f] : NAN;
    b->vmin = rel ? bt[f].vmin : 0.0f;
    b->vmax = rel ? bt[f].vmax : 0.0f;
    long long* uidx = (long long*)(p->d_scratch + p->off_uidx[f]);
    float* uval = (float*)(p->d_scratch + p->off_uval[f]);
    cudaError_t e = cudaSuccess;
    if (hs[f]) {
      void* tmp = nullptr;
      const size_t tb = sort_pairs_scratch(count);
      e = dev_alloc(&tmp, tb, s);
      if (e == cudaSuccess)
        e = launch_sort_pairs(uidx, uval, count, (long long*)tmp,
                              (float*)((char*)tmp + tb / 12 * 8), s);
      dev_free(tmp, s);
    }
    if (e == cudaSuccess &&
        (e = dev_alloc((void**)&b->d_uidx, sizeof(long long) * count, s)) == cudaSuccess)
      e = dev_alloc((void**)&b->d_uval, sizeof(float) * count, s);
    if (e == cudaSuccess && count > 0)
      e = cudaMemcpyAsync(b->d_uidx, uidx, sizeof(long long) * count, cudaMemcpyDeviceToDevice,
                          s);
    if (e == cudaSuccess && count > 0)
      e = cudaMemcpyAsync(b->d_uval, uval, sizeof(float) * count, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "batch unpredictable lists");
  }
  if (st == QOZ_OK) {
    // the plan's lists are reused by the next run
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "batch finish");
  }
  if (st != QOZ_OK) free_blobs(outs, p->nf);
  return st;
}

qoz_status qoz_batch_get_info(const qoz_batch* p, qoz_batch_info* info) {
  if (!p || !info) return fail(QOZ_EINVAL, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->nfields = p->nf;
  info->n_groups = (int32_t)p->groups.size();
  info->launches_per_run = p->launches;
  info->graph = p->exec != nullptr;
  info->autotuned = p->autotuned;
  int k = 0;
  for (const Group& g : p->groups) {
    info->ctas_per_run += g.nblocks;
    if (g.level != 1) continue;
    if (k < 16) {
      info->level1_variant[k] = g.key.variant;
      for (int v = 0; v < kLevelVariants; ++v) info->level1_ms[k][v] = g.ms[v];
    }
    ++k;
  }
  info->level1_groups = k;
  return QOZ_OK;
}

void qoz_batch_free(qoz_batch* p) { free_plan(p); }

qoz_status qoz_compress_batch(const float* const* d_fields, const qoz_shape* shapes,
                              int32_t nfields, double rel_eb, const qoz_params* params,
                              void* stream, qoz_blob** outs) {
  qoz_batch* p = nullptr;
  qoz_status st = qoz_batch_create(shapes, nfields, params, QOZ_BATCH_NO_GRAPH, &p);
  if (st != QOZ_OK) return st;
  std::vector<double> eb(nfields, rel_eb);
  st = qoz_batch_compress(p, d_fields, eb.data(), 1, stream, outs);
  free_plan(p);
  return st;
}

}  // extern "C"
