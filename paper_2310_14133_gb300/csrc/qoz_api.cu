// C ABI of the library (include/qoz.h): argument checks, device memory,
// stream-ordered orchestration of the kernels, the compressed-blob format.
//
// A compression runs the steps of the paper in order: the value range and
// the bound e = eps * vrange (Sec. 7.1.4), the level-wise bounds (Eq. (ebl)),
// the anchor points (Sec. 5.2.1), then the interpolation levels from the
// coarsest to the finest with the linear-scale quantizer (Sec. 5.1, 5.2),
// and the code histogram of the rate estimate (Sec. 6.1).  Decompression
// mirrors it; the metrics follow Sec. 3.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"

using namespace qoz;


namespace qoz {

// ------------------------------------------------------------- errors

static thread_local std::string g_err;

qoz_status fail(qoz_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

qoz_status cuda_fail(cudaError_t e, const char* what) {
  return fail(QOZ_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Host-side fault injection for the failure-path tests: QOZ_FAULT is a
// comma-separated list of steps to fail ("alloc", "launch", "header",
// "tma_wait").
bool fault_injected(const char* step) {
  const char* env = getenv("QOZ_FAULT");
  if (!env || !*env) return false;
  const size_t n = strlen(step);
  for (const char* p = env; *p;) {
    const char* q = strchr(p, ',');
    const size_t len = q ? (size_t)(q - p) : strlen(p);
    if (len == n && strncmp(p, step, n) == 0) return true;
    if (!q) break;
    p = q + 1;
  }
  return false;
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (fault_injected("alloc")) return cudaErrorMemoryAllocation;
  if (bytes == 0) bytes = 16;
  return cudaMallocAsync(p, bytes, s);
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

cudaError_t launch_check(cudaError_t e) {
  if (e == cudaSuccess && fault_injected("launch")) return cudaErrorLaunchFailure;
  return e;
}

// Keep freed blocks in the stream-ordered pool: repeated calls then reuse
// device memory instead of returning it to the driver.
void configure_pool_once() {
  static unsigned long long done = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  __atomic_fetch_or(&done, bit, __ATOMIC_ACQ_REL);
}

// ------------------------------------------------------------- geometry

int log2_exact(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return (1LL << l) == v ? l : -1;
}

static const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

qoz_status resolve(const qoz_shape& shape, const qoz_params* p, Resolved* r) {
  if (shape.ndims != 2 && shape.ndims != 3)
    return fail(QOZ_EINVAL, "ndims must be 2 or 3 (got %d)", shape.ndims);
  for (int i = 0; i < shape.ndims; ++i)
    if (shape.dims[i] < 1) return fail(QOZ_EINVAL, "dims[%d] = %lld < 1", i, (long long)shape.dims[i]);
  r->ndims = shape.ndims;
  if (shape.ndims == 2) {
    r->n[0] = 1;
    r->n[1] = shape.dims[0];
    r->n[2] = shape.dims[1];
  } else {
    for (int i = 0; i < 3; ++i) r->n[i] = shape.dims[i];
  }
  // the product is formed with a bound check per factor, so that extents whose
  // product wraps around 64 bits (a corrupt header, say) are refused too
  constexpr long long kMaxPoints = (1LL << 32) - 1;
  r->N = 1;
  for (int i = 0; i < 3; ++i) {
    if (r->n[i] > kMaxPoints / r->N)
      return fail(QOZ_EUNSUPPORTED, "fields of 2^32 points or more are not supported");
    r->N *= r->n[i];
  }
  qoz_params d;
  memset(&d, 0, sizeof(d));
  if (p) {
    d = *p;
  } else {
    for (int l = 0; l < QOZ_MAX_LEVELS; ++l) d.interp[l] = 1;
    d.alpha = 1.0;
    d.beta = 1.0;
  }
  if (d.anchor_stride == 0) d.anchor_stride = shape.ndims == 3 ? 32 : 64;
  const int L = log2_exact(d.anchor_stride);
  if (L < 1 || L > QOZ_MAX_LEVELS)
    return fail(QOZ_EINVAL, "anchor_stride %d is not a power of two in [2, 256]",
                d.anchor_stride);
  const int nperm = shape.ndims == 3 ? 6 : 2;
  for (int l = 0; l < L; ++l) {
    if (d.interp[l] > 1) return fail(QOZ_EINVAL, "interp[%d] = %d is not 0 or 1", l, d.interp[l]);
    if (d.order[l] >= nperm)
      return fail(QOZ_EINVAL, "order[%d] = %d out of range", l, d.order[l]);
  }
  if (!(d.alpha >= 1.0) || !std::isfinite(d.alpha) || !(d.beta >= 1.0) || !std::isfinite(d.beta))
    return fail(QOZ_EINVAL, "alpha and beta must be finite and >= 1");
  r->p = d;
  r->L = L;
  for (int l = 0; l < L; ++l) {
    // a 2D order (y,x) or (x,y) is the 3D order with z first and no z targets
    const int o3 = shape.ndims == 3 ? d.order[l] : (d.order[l] == 0 ? 0 : 1);
    for (int k = 0; k < 3; ++k) r->axes[l][k] = kPerm3[o3][k];
  }
  return QOZ_OK;
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

void grid_dims(const Resolved& r, int k, long long g[3]) {
  // grid subsampled by 2^k
  for (int p = 0; p < 3; ++p) g[p] = ceil_div(r.n[p], 1LL << k);
}

// Row pitch of the compact array of the grid subsampled by 2^k: the field's
// own rows at k = 0 and the anchor grid's at k = L (both dense); rounded up to
// 8 values in between, so that every row of a coarse reconstruction (float)
// or code (uint16) array starts on a 16-byte boundary (the tile kernel's
// bulk tensor copies need that).
long long grid_pitch(const Resolved& r, int k) {
  long long g[3];
  grid_dims(r, k, g);
  return (k == 0 || k >= r.L) ? g[2] : (g[2] + 7) & ~7LL;
}

Coarse coarse_layout(const Resolved& r, bool with_codes) {
  Coarse c;
  memset(&c, 0, sizeof(c));
  size_t tot = 0;
  for (int k = 1; k < r.L; ++k) {
    long long g[3];
    grid_dims(r, k, g);
    const size_t n = (size_t)(g[0] * g[1] * grid_pitch(r, k));
    c.roff[k] = tot;
    tot += (n * sizeof(float) + 255) & ~(size_t)255;
    if (with_codes) {
      c.coff[k] = tot;
      tot += (n * sizeof(uint16_t) + 255) & ~(size_t)255;
    }
  }
  c.bytes = tot;
  return c;
}

long long anchor_dims(const Resolved& r, long long na[3]) {
  for (int p = 0; p < 3; ++p) na[p] = ceil_div(r.n[p], r.p.anchor_stride);
  return na[0] * na[1] * na[2];
}

// Geometry of level l: G = field subsampled by 2^(l-1), coarse = by 2^l.
void level_geometry(const Resolved& r, int l, LevelLaunch* L) {
  long long g[3], gc[3];
  grid_dims(r, l - 1, g);
  grid_dims(r, l, gc);
  const long long f = 1LL << (l - 1);
  const long long fst[3] = {r.n[1] * r.n[2], r.n[2], 1};
  for (int p = 0; p < 3; ++p) {
    L->g[p] = g[p];
    L->xs[p] = f * fst[p];
  }
  const long long pc = grid_pitch(r, l), pg = grid_pitch(r, l - 1);
  L->cs[0] = gc[1] * pc;
  L->cs[1] = pc;
  L->cs[2] = 1;
  L->os[0] = g[1] * pg;
  L->os[1] = pg;
  L->os[2] = 1;
  L->is2d = r.ndims == 2;
  L->order3 = r.ndims == 3 ? r.p.order[l - 1] : (r.p.order[l - 1] == 0 ? 0 : 1);
  L->level = l;
  L->interp = r.p.interp[l - 1];
}

// Runs levels L..1 (compress or decompress) over the grid hierarchy.
cudaError_t run_levels(bool decompress, const Resolved& r, const float* x, uint16_t* codes,
                       const float* anchors, char* coarse_base, const Coarse& cl,
                       float* final_out, const BoundTable* bt, UnpredList ul,
                       const long long* uidx, const float* uval, long long nu, int* err,
                       unsigned* hist, cudaStream_t s) {
  for (int l = r.L; l >= 1; --l) {
    LevelLaunch L;
    memset(&L, 0, sizeof(L));
    level_geometry(r, l, &L);
    L.decompress = decompress;
    L.rc = l == r.L ? anchors : (const float*)(coarse_base + cl.roff[l]);
    L.rout = l > 1 ? (float*)(coarse_base + cl.roff[l - 1]) : final_out;
    L.bt = bt;
    if (decompress) {
      L.cin = codes;
      L.uidx = uidx;
      L.uval = uval;
      L.nu = nu;
      L.err = err;
    } else {
      L.x = x;
      L.err = err;  // compress: bit 2 reports a tile copy that never landed
      if (l == 1 && fault_injected("tma_wait")) {
        // host fault injection: the tile barrier expects 16 bytes that never
        // come, so every bounded wait runs out after 4096 polls
        L.extra_tx = 16;
        L.wait_polls = 4096;
      }
      L.cin = l == r.L ? nullptr : (const uint16_t*)(coarse_base + cl.coff[l]);
      L.cout = l > 1 ? (uint16_t*)(coarse_base + cl.coff[l - 1]) : codes;
      L.ul = ul;
      L.hist = l == 1 ? hist : nullptr;
    }
    ProfScope ps(decompress ? QOZ_STAGE_DLEVEL + l : QOZ_STAGE_LEVEL + l, s);
    cudaError_t e = launch_check(launch_level(L, s));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Pinned host staging for the few values read back per call.
struct HostStage {
  BoundTable bt;
  unsigned long long count;
  int err;
};
HostStage* host_stage() {
  static thread_local HostStage* h = nullptr;
  if (!h) {
    if (cudaMallocHost((void**)&h, sizeof(HostStage)) != cudaSuccess) h = nullptr;
  }
  return h;
}

qoz_status compress_impl(const float* d_field, const qoz_shape& shape, bool rel, double eb,
                         const qoz_params* p, float* d_recon, cudaStream_t s, qoz_blob** out) {
  if (!out) return fail(QOZ_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d_field) return fail(QOZ_EINVAL, "d_field is NULL");
  if (rel && !(eb > 0.0 && std::isfinite(eb)))
    return fail(QOZ_EINVAL, "rel_eb must be finite and > 0");
  if (!rel && !(eb >= 0.0 && std::isfinite(eb)))
    return fail(QOZ_EINVAL, "abs_eb must be finite and >= 0");
  if (reinterpret_cast<uintptr_t>(d_field) & 3)
    return fail(QOZ_EINVAL, "d_field must be 4-byte aligned");
  Resolved r;
  qoz_status st = resolve(shape, p, &r);
  if (st != QOZ_OK) return st;
  configure_pool_once();
  HostStage* hs = host_stage();
  if (!hs) return fail(QOZ_ENOMEM, "pinned staging buffer");

  qoz_blob* b = new qoz_blob();
  memset(b, 0, sizeof(*b));
  b->shape = shape;
  for (int i = 0; i < 3; ++i) b->n[i] = r.n[i];
  b->N = r.N;
  b->L = r.L;
  b->params = r.p;
  b->stream = s;
  cudaGetDevice(&b->device);
  long long na3[3];
  b->na = anchor_dims(r, na3);

  cudaError_t e;
  void* scratch = nullptr;
  const Coarse cl = coarse_layout(r, true);
  const size_t cb = cl.bytes;
  const int nparts = range_partial_blocks();
  long long cap = r.N / 1024;
  if (cap < 65536) cap = 65536;
  if (cap > r.N) cap = r.N > 0 ? r.N : 1;

  auto cleanup = [&](qoz_status code) {
    dev_free(scratch, s);
    dev_free(b->d_codes, s);
    dev_free(b->d_anchors, s);
    dev_free(b->d_hist, s);
    dev_free(b->d_uidx, s);
    dev_free(b->d_uval, s);
    dev_free(b->d_err, s);
    delete b;
    return code;
  };

  if ((e = dev_alloc((void**)&b->d_codes, sizeof(uint16_t) * r.N, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_anchors, sizeof(float) * b->na, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_hist, sizeof(unsigned) * 65536, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_err, sizeof(int), s)) != cudaSuccess)
    return cleanup(fail(QOZ_ENOMEM, "device allocation: %s", cudaGetErrorString(e)));
  cudaMemsetAsync(b->d_err, 0, sizeof(int), s);

  for (int attempt = 0; attempt < 2; ++attempt) {
    // scratch: bound table | range partials | unpredictable list | coarse grids
    const size_t sort_tmp = sort_pairs_scratch(cap);
    size_t o_bt = 0;
    size_t o_pmin = 256;
    size_t o_pmax = o_pmin + ((nparts * sizeof(float) + 255) & ~(size_t)255);
    size_t o_pcnt = o_pmax + ((nparts * sizeof(float) + 255) & ~(size_t)255);
    size_t o_cnt = o_pcnt + ((nparts * sizeof(unsigned long long) + 255) & ~(size_t)255);
    size_t o_uidx = o_cnt + 256;
    size_t o_uval = o_uidx + ((cap * sizeof(long long) + 255) & ~(size_t)255);
    size_t o_sort = o_uval + ((cap * sizeof(float) + 255) & ~(size_t)255);
    size_t o_coarse = o_sort + ((sort_tmp + 255) & ~(size_t)255);
    const size_t total = o_coarse + cb;
    if ((e = dev_alloc(&scratch, total, s)) != cudaSuccess)
      return cleanup(fail(QOZ_ENOMEM, "scratch allocation (%zu bytes): %s", total,
                          cudaGetErrorString(e)));
    char* base = (char*)scratch;
    BoundTable* d_bt = (BoundTable*)(base + o_bt);
    float* pmin = (float*)(base + o_pmin);
    float* pmax = (float*)(base + o_pmax);
    unsigned long long* pcnt = (unsigned long long*)(base + o_pcnt);
    unsigned long long* d_count = (unsigned long long*)(base + o_cnt);
    long long* uidx = (long long*)(base + o_uidx);
    float* uval = (float*)(base + o_uval);
    char* coarse = base + o_coarse;

    e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_hist, 0, sizeof(unsigned) * 65536, s);
    if (e == cudaSuccess && rel) {
      ProfScope ps(QOZ_STAGE_RANGE, s);
      e = launch_check(launch_range(d_field, r.N, pmin, pmax, pcnt, s));
    }
    const long long fst[3] = {r.n[1] * r.n[2], r.n[2], 1};
    if (e == cudaSuccess) {
      ProfScope ps(QOZ_STAGE_SETUP, s);
      e = launch_check(launch_bound_table(pmin, pmax, pcnt, rel ? nparts : 0, rel ? 1 : 0, eb,
                                          r.p.alpha, r.p.beta, r.L, d_bt, s));
      if (e == cudaSuccess)
        e = launch_check(
            launch_anchor_gather(d_field, b->d_anchors, na3, fst, r.p.anchor_stride, s));
    }
    UnpredList ul{uidx, uval, d_count, cap};
    if (e == cudaSuccess)
      e = run_levels(false, r, d_field, b->d_codes, b->d_anchors, coarse, cl, d_recon, d_bt, ul,
                     nullptr, nullptr, 0, b->d_err, b->d_hist, s);
    if (e == cudaSuccess) {
      ProfScope ps(QOZ_STAGE_HIST, s);
      e = launch_check(launch_hist_remove_anchors(b->d_hist, b->na, s));
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&hs->count, d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&hs->bt, d_bt, sizeof(BoundTable), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&hs->err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "compress"));
    if (hs->err != 0)
      return cleanup(fail(QOZ_ETIMEOUT, "a tile's bulk copy did not complete (flag %d)", hs->err));

    const long long count = (long long)hs->count;
    if (count > cap) {
      // more unpredictable points than the list holds: redo with room for all
      dev_free(scratch, s);
      scratch = nullptr;
      cap = count;
      continue;
    }
    b->nu = count;
    b->abs_eb = hs->bt.e;
    b->rel_eb = rel ? eb : NAN;
    b->vmin = rel ? hs->bt.vmin : 0.0f;
    b->vmax = rel ? hs->bt.vmax : 0.0f;
    if ((e = dev_alloc((void**)&b->d_uidx, sizeof(long long) * count, s)) != cudaSuccess ||
        (e = dev_alloc((void**)&b->d_uval, sizeof(float) * count, s)) != cudaSuccess)
      return cleanup(fail(QOZ_ENOMEM, "unpredictable list allocation"));
    if (count > 1)
      e = launch_check(launch_sort_pairs(uidx, uval, count, (long long*)(base + o_sort),
                                         (float*)(base + o_sort + sort_tmp / 12 * 8), s));
    if (e == cudaSuccess && count > 0)
      e = cudaMemcpyAsync(b->d_uidx, uidx, sizeof(long long) * count, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && count > 0)
      e = cudaMemcpyAsync(b->d_uval, uval, sizeof(float) * count, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "unpredictable list"));
    dev_free(scratch, s);
    scratch = nullptr;
    *out = b;
    return QOZ_OK;
  }
  return cleanup(fail(QOZ_ECUDA, "unpredictable list did not converge"));
}

qoz_status decompress_impl(const qoz_blob* b, float* d_out, cudaStream_t s) {
  if (!b || !d_out) return fail(QOZ_EINVAL, "NULL argument");
  Resolved r;
  qoz_status st = resolve(b->shape, &b->params, &r);
  if (st != QOZ_OK) return st;
  configure_pool_once();
  const Coarse cl = coarse_layout(r, false);
  void* scratch = nullptr;
  cudaError_t e = dev_alloc(&scratch, 256 + cl.bytes, s);
  if (e != cudaSuccess) return fail(QOZ_ENOMEM, "decompress scratch: %s", cudaGetErrorString(e));
  BoundTable* d_bt = (BoundTable*)scratch;
  char* coarse = (char*)scratch + 256;
  // the decode flags start clean for every decompression (qoz_blob_check)
  e = cudaMemsetAsync(b->d_err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = launch_check(launch_bound_table(nullptr, nullptr, nullptr, 0, 0, b->abs_eb, r.p.alpha,
                                        r.p.beta, r.L, d_bt, s));
  UnpredList ul{nullptr, nullptr, nullptr, 0};
  if (e == cudaSuccess)
    e = run_levels(true, r, nullptr, b->d_codes, b->d_anchors, coarse, cl, d_out, d_bt, ul,
                   b->d_uidx, b->d_uval, b->nu, b->d_err, nullptr, s);
  dev_free(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "decompress");
  return QOZ_OK;
}

}  // namespace qoz

// =============================================================== C ABI

extern "C" {

const char* qoz_last_error(void) { return g_err.c_str(); }

qoz_status qoz_value_range(const float* d_x, int64_t n, float* h_min, float* h_max,
                           int64_t* h_count, void* stream) {
  if (!d_x || !h_min || !h_max || n < 0) return fail(QOZ_EINVAL, "invalid argument");
  if (reinterpret_cast<uintptr_t>(d_x) & 3) return fail(QOZ_EINVAL, "d_x must be 4-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  configure_pool_once();
  HostStage* hs = host_stage();
  if (!hs) return fail(QOZ_ENOMEM, "pinned staging buffer");
  const int nparts = range_partial_blocks();
  void* scratch = nullptr;
  cudaError_t e = dev_alloc(&scratch, 256 + nparts * (sizeof(float) * 2 + 8) + 1024, s);
  if (e != cudaSuccess) return fail(QOZ_ENOMEM, "scratch: %s", cudaGetErrorString(e));
  char* base = (char*)scratch;
  BoundTable* d_bt = (BoundTable*)base;
  float* pmin = (float*)(base + 256);
  float* pmax = pmin + nparts;
  unsigned long long* pcnt = (unsigned long long*)(((uintptr_t)(pmax + nparts) + 15) & ~(uintptr_t)15);
  e = launch_check(launch_range(d_x, n, pmin, pmax, pcnt, s));
  if (e == cudaSuccess)
    e = launch_check(launch_bound_table(pmin, pmax, pcnt, nparts, 1, 1.0, 1.0, 1.0, 1, d_bt, s));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hs->bt, d_bt, sizeof(BoundTable), cudaMemcpyDeviceToHost, s);
  dev_free(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "value range");
  *h_min = hs->bt.vmin;
  *h_max = hs->bt.vmax;
  if (h_count) *h_count = hs->bt.n_finite;
  return QOZ_OK;
}

qoz_status qoz_compress(const float* d_field, qoz_shape shape, double rel_eb, const qoz_params* p,
                        float* d_recon, void* stream, qoz_blob** out) {
  return compress_impl(d_field, shape, true, rel_eb, p, d_recon, (cudaStream_t)stream, out);
}

qoz_status qoz_compress_abs(const float* d_field, qoz_shape shape, double abs_eb,
                            const qoz_params* p, float* d_recon, void* stream, qoz_blob** out) {
  return compress_impl(d_field, shape, false, abs_eb, p, d_recon, (cudaStream_t)stream, out);
}

qoz_status qoz_decompress(const qoz_blob* b, float* d_out, void* stream) {
  return decompress_impl(b, d_out, (cudaStream_t)stream);
}

qoz_status qoz_blob_get_info(const qoz_blob* b, qoz_blob_info* info) {
  if (!b || !info) return fail(QOZ_EINVAL, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->shape = b->shape;
  info->params = b->params;
  info->abs_eb = b->abs_eb;
  info->rel_eb = b->rel_eb;
  info->vmin = b->vmin;
  info->vmax = b->vmax;
  info->n_points = b->N;
  info->n_anchors = b->na;
  info->n_unpredictable = b->nu;
  std::vector<unsigned> h(65536);
  cudaError_t e = cudaMemcpyAsync(h.data(), b->d_hist, sizeof(unsigned) * 65536,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "histogram read-back");
  const double bits = (double)huffman_bits_u32(h.data(), 65536) + 32.0 * (double)b->nu +
                      32.0 * (double)b->na;
  info->est_bits = bits;
  info->est_ratio = bits > 0 ? 32.0 * (double)b->N / bits : INFINITY;
  return QOZ_OK;
}

qoz_status qoz_blob_arrays(const qoz_blob* b, const uint16_t** d_codes,
                           const int64_t** d_unpred_idx, const float** d_unpred_val,
                           int64_t* n_unpred, const float** d_anchors, int64_t* n_anchors) {
  if (!b) return fail(QOZ_EINVAL, "NULL blob");
  if (d_codes) *d_codes = b->d_codes;
  if (d_unpred_idx) *d_unpred_idx = (const int64_t*)b->d_uidx;
  if (d_unpred_val) *d_unpred_val = b->d_uval;
  if (n_unpred) *n_unpred = b->nu;
  if (d_anchors) *d_anchors = b->d_anchors;
  if (n_anchors) *n_anchors = b->na;
  return QOZ_OK;
}

qoz_status qoz_blob_check(const qoz_blob* b, void* stream) {
  if (!b) return fail(QOZ_EINVAL, "NULL blob");
  HostStage* hs = host_stage();
  if (!hs) return fail(QOZ_ENOMEM, "pinned staging buffer");
  cudaStream_t s = stream ? (cudaStream_t)stream : b->stream;
  cudaError_t e = cudaMemcpyAsync(&hs->err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "blob status read-back");
  if (hs->err & 1)
    return fail(QOZ_ECORRUPT, "a code-0 point has no entry in the unpredictable list");
  if (hs->err & 4) return fail(QOZ_ECORRUPT, "the coded stream does not decode");
  if (hs->err & 2) return fail(QOZ_ETIMEOUT, "a tile's bulk copy did not complete");
  return QOZ_OK;
}

qoz_status qoz_blob_histogram(const qoz_blob* b, uint32_t* h_hist, void* stream) {
  if (!b || !h_hist) return fail(QOZ_EINVAL, "NULL argument");
  cudaStream_t s = stream ? (cudaStream_t)stream : b->stream;
  cudaError_t e =
      cudaMemcpyAsync(h_hist, b->d_hist, sizeof(unsigned) * 65536, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "histogram read-back");
  return QOZ_OK;
}

void qoz_blob_free(qoz_blob* b) {
  if (!b) return;
  dev_free(b->d_codes, b->stream);
  dev_free(b->d_anchors, b->stream);
  dev_free(b->d_hist, b->stream);
  dev_free(b->d_uidx, b->stream);
  dev_free(b->d_uval, b->stream);
  dev_free(b->d_err, b->stream);
  delete b;
}

qoz_status qoz_compute_metrics(const float* d_a, const float* d_b, qoz_shape shape, double vrange,
                               int32_t ssim_win, int32_t ssim_step, qoz_metrics* out,
                               void* stream) {
  if (!d_a || !d_b || !out) return fail(QOZ_EINVAL, "NULL argument");
  Resolved r;
  qoz_status st = resolve(shape, nullptr, &r);
  if (st != QOZ_OK) return st;
  if (ssim_win > 0 && ssim_step < 1) return fail(QOZ_EINVAL, "ssim_step must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  configure_pool_once();
  const int ne = err_metric_blocks();
  const int ns = ssim_win > 0 ? ssim_parts(r.n, r.ndims == 3, ssim_win, ssim_step) : 0;
  const int na = ac_parts();
  void* scratch = nullptr;
  cudaError_t e = dev_alloc(&scratch, sizeof(double) * (2 * ne + ns + na), s);
  if (e != cudaSuccess) return fail(QOZ_ENOMEM, "metrics scratch: %s", cudaGetErrorString(e));
  double* psse = (double*)scratch;
  double* pmax = psse + ne;
  double* pss = pmax + ne;
  double* pac = pss + ns;
  e = launch_check(launch_err_metrics(d_a, d_b, r.N, psse, pmax, pac, s));
  const double c1 = (0.01 * vrange) * (0.01 * vrange);
  const double c2 = (0.03 * vrange) * (0.03 * vrange);
  if (e == cudaSuccess && ssim_win > 0)
    e = launch_check(launch_ssim(d_a, d_b, r.n, r.ndims == 3, ssim_win, ssim_step, c1, c2, pss,
                                 s));
  std::vector<double> h(2 * ne + ns + na, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), scratch, sizeof(double) * (2 * ne + ns + na),
                        cudaMemcpyDeviceToHost, s);
  dev_free(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "metrics");
  double sse = 0.0, mx = 0.0;
  for (int i = 0; i < ne; ++i) sse += h[i];
  for (int i = 0; i < ne; ++i) {
    const double v = h[ne + i];
    if (v != v || v > mx) mx = v;
    if (mx != mx) break;
  }
  out->max_abs_err = mx;
  out->mse = r.N > 0 ? sse / (double)r.N : 0.0;
  out->psnr = out->mse == 0.0 ? INFINITY : 20.0 * std::log10(vrange / std::sqrt(out->mse));
  out->ssim = NAN;
  out->ssim_windows = 0;
  out->ac = autocorr_from_parts(h.data() + 2 * ne + ns, r.N, 1);
  if (ssim_win > 0) {
    auto cnt = [&](long long n) { return n >= ssim_win ? (n - ssim_win) / ssim_step + 1 : 0; };
    const long long nw = (r.ndims == 3 ? cnt(r.n[0]) : 1) * cnt(r.n[1]) * cnt(r.n[2]);
    double ss = 0.0;
    for (int i = 0; i < ns; ++i) ss += h[2 * ne + i];
    out->ssim_windows = nw;
    out->ssim = nw > 0 ? 1.0 - ss / (double)nw : NAN;  // parts hold sums of 1 - SSIM_w
  }
  return QOZ_OK;
}

qoz_status qoz_error_autocorr(const float* d_a, const float* d_b, int64_t n, int64_t lag,
                              double* ac, void* stream) {
  if (!d_a || !d_b || !ac) return fail(QOZ_EINVAL, "NULL argument");
  if (n < 0 || lag < 1) return fail(QOZ_EINVAL, "n >= 0 and lag >= 1 required");
  cudaStream_t s = (cudaStream_t)stream;
  configure_pool_once();
  const int na = ac_parts();
  void* scratch = nullptr;
  cudaError_t e = dev_alloc(&scratch, sizeof(double) * na, s);
  if (e != cudaSuccess) return fail(QOZ_ENOMEM, "autocorrelation scratch");
  {
    ProfScope ps(QOZ_STAGE_METRICS, s);
    e = launch_check(launch_autocorr(d_a, d_b, n, lag, (double*)scratch, s));
  }
  std::vector<double> h(na, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), scratch, sizeof(double) * na, cudaMemcpyDeviceToHost, s);
  dev_free(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "autocorrelation");
  *ac = autocorr_from_parts(h.data(), n, lag);
  return QOZ_OK;
}

}  // extern "C"
