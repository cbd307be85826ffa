// Serialized blob format and array export.  The code section holds the
// Huffman coding of the quantization codes whose size the rate estimate of
// Sec. 6.1 stands for (canonical codes as in RFC 1951 Sec. 3.2.2).
//
// Layout (little-endian): a 160-byte header, then the anchors (float32), the
// unpredictable indices (int64) and values (float32), and the code section,
// each part padded to 8 bytes.  The code section is the entropy stage's
// output: its 288-byte fixed part (symbol count, longest code, chunk size,
// chunk and word counts, number of codes per length), the used symbols in
// (length, symbol) order, the n_chunks + 1 word offsets (uint64), for chunks
// of 1024 codes or more the run table (the coded bits of each 512-code run
// but a chunk's last, uint16) and the stream words (uint32).  The header's
// checksum field holds a 64-bit sum over
// every 8-byte word w_i of header and payload of mix(w_i ^ mix(i)), taken
// with the field itself zero; being a sum, it is computed on the device for
// the device-resident parts, in parallel, and on the host for the header.
// mix is the splitmix64 finalizer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"


namespace qoz {

namespace {

constexpr char kMagic[8] = {'Q', 'O', 'Z', 'G', 'B', '3', '0', '0'};
constexpr uint32_t kVersion = 3;
constexpr int32_t kCodingHuffman = 1;

struct Header {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int32_t ndims;
  int32_t coding;  // kCodingHuffman: the code section is the entropy stage's output
  int64_t dims[3];
  double abs_eb;
  double rel_eb;
  float vmin, vmax;
  int32_t anchor_stride;
  uint8_t interp[8];
  uint8_t order[8];
  int32_t reserved1;
  double alpha, beta;
  int64_t n_points, n_anchors, n_unpred;
  uint64_t checksum;
  uint64_t code_bytes;  // bytes of the code section
  uint64_t reserved2;
};
static_assert(sizeof(Header) == 160, "header layout");

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

constexpr int kSumBlocks = 152 * 2;
constexpr int kSumThreads = 256;

__global__ void __launch_bounds__(kSumThreads) checksum_kernel(const unsigned char* p,
                                                               long long nbytes,
                                                               long long word0,
                                                               unsigned long long* part) {
  unsigned long long acc = 0;
  const long long nw = (nbytes + 7) / 8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw;
       i += (long long)gridDim.x * blockDim.x) {
    uint64_t w = 0;
    const long long b0 = i * 8;
    if (b0 + 8 <= nbytes && ((reinterpret_cast<uintptr_t>(p) & 7) == 0)) {
      w = *reinterpret_cast<const uint64_t*>(p + b0);
    } else {
      for (int k = 0; k < 8 && b0 + k < nbytes; ++k) w |= (uint64_t)p[b0 + k] << (8 * k);
    }
    acc += mix64(w ^ mix64((uint64_t)(word0 + i)));
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ unsigned long long sh[kSumThreads / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int k = 0; k < kSumThreads / 32; ++k) s += sh[k];
    atomicAdd(part, s);
  }
}

uint64_t host_checksum(const unsigned char* p, size_t nbytes, uint64_t word0) {
  uint64_t acc = 0;
  const size_t nw = (nbytes + 7) / 8;
  for (size_t i = 0; i < nw; ++i) {
    uint64_t w = 0;
    for (int k = 0; k < 8 && i * 8 + k < nbytes; ++k) w |= (uint64_t)p[i * 8 + k] << (8 * k);
    acc += mix64(w ^ mix64(word0 + i));
  }
  return acc;
}

size_t pad8(size_t v) { return (v + 7) & ~(size_t)7; }

struct Layout {
  size_t anchors, uidx, uval, codes, sym, offs, sub, words, total;
};

// Offsets of every part; the code section's sizes come from its fixed part.
Layout layout_of(long long na, long long nu, long long n_sym, long long n_chunks,
                 long long n_words, int chunk) {
  Layout L;
  L.anchors = sizeof(Header);
  L.uidx = L.anchors + pad8(sizeof(float) * na);
  L.uval = L.uidx + pad8(sizeof(long long) * nu);
  L.codes = L.uval + pad8(sizeof(float) * nu);
  L.sym = L.codes + sizeof(HuffFixed);
  L.offs = L.sym + pad8(sizeof(uint16_t) * n_sym);
  L.sub = L.offs + sizeof(unsigned long long) * (n_chunks + 1);
  L.words = L.sub + (chunk > 0 ? entropy_sub_bytes(n_chunks, chunk) : 0);
  L.total = L.words + pad8(sizeof(uint32_t) * n_words);
  return L;
}

Layout layout_of(const qoz_blob* b, const HuffEncoded& h) {
  return layout_of(b->na, b->nu, h.fixed.n_sym, h.n_chunks, h.n_words, h.chunk);
}

// The device-resident parts, each with its place in the stream.
struct Part {
  const void* p;
  size_t bytes, off;
};

int parts_of(const qoz_blob* b, const HuffEncoded& h, const Layout& L, Part* out) {
  const char* sec = static_cast<const char*>(h.d_section);
  const Part ps[7] = {
      {b->d_anchors, sizeof(float) * b->na, L.anchors},
      {b->d_uidx, sizeof(long long) * b->nu, L.uidx},
      {b->d_uval, sizeof(float) * b->nu, L.uval},
      {sec, sizeof(HuffFixed), L.codes},
      {sec + sizeof(HuffFixed), L.offs - L.sym, L.sym},  // zero-padded on the device
      {sec + sizeof(HuffFixed) + h.sym_bytes, L.words - L.offs, L.offs},  // offsets, run table
      {h.d_words, sizeof(uint32_t) * h.n_words, L.words}};
  int k = 0;
  for (const Part& p : ps)
    if (p.bytes) out[k++] = p;
  return k;
}

// Device-side checksum of the payload parts (word offsets per layout).
cudaError_t device_payload_sum(const Part* parts, int np, unsigned long long* d_acc,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long), s);
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    checksum_kernel<<<kSumBlocks, kSumThreads, 0, s>>>((const unsigned char*)parts[i].p,
                                                       (long long)parts[i].bytes,
                                                       (long long)(parts[i].off / 8), d_acc);
    note_launch(1);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace
}  // namespace qoz

using namespace qoz;

extern "C" {

qoz_status qoz_blob_copy_arrays(const qoz_blob* b, uint16_t* d_codes, int64_t* d_unpred_idx,
                                float* d_unpred_val, float* d_anchors, void* stream) {
  if (!b) return fail(QOZ_EINVAL, "NULL blob");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (d_codes && b->N)
    e = cudaMemcpyAsync(d_codes, b->d_codes, sizeof(uint16_t) * b->N, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_unpred_idx && b->nu)
    e = cudaMemcpyAsync(d_unpred_idx, b->d_uidx, sizeof(long long) * b->nu,
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d_unpred_val && b->nu)
    e = cudaMemcpyAsync(d_unpred_val, b->d_uval, sizeof(float) * b->nu, cudaMemcpyDeviceToDevice,
                        s);
  if (e == cudaSuccess && d_anchors && b->na)
    e = cudaMemcpyAsync(d_anchors, b->d_anchors, sizeof(float) * b->na, cudaMemcpyDeviceToDevice,
                        s);
  if (e != cudaSuccess) return cuda_fail(e, "copy arrays");
  return QOZ_OK;
}

namespace {

// Header of a serialized blob, checksum not yet set.
Header header_of(const qoz_blob* b, const Layout& L) {
  Header h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(Header);
  h.ndims = b->shape.ndims;
  for (int i = 0; i < 3; ++i) h.dims[i] = i < b->shape.ndims ? b->shape.dims[i] : 0;
  h.abs_eb = b->abs_eb;
  h.rel_eb = b->rel_eb;
  h.vmin = b->vmin;
  h.vmax = b->vmax;
  h.anchor_stride = b->params.anchor_stride;
  memcpy(h.interp, b->params.interp, 8);
  memcpy(h.order, b->params.order, 8);
  h.alpha = b->params.alpha;
  h.beta = b->params.beta;
  h.n_points = b->N;
  h.n_anchors = b->na;
  h.n_unpred = b->nu;
  h.coding = kCodingHuffman;
  h.code_bytes = L.total - L.codes;
  return h;
}

// Enqueues the payload checksum and the part copies; the device checksum
// lands in the header's checksum slot of out (8 bytes at a fixed offset).
cudaError_t enqueue_payload(const qoz_blob* b, const HuffEncoded& h, const Layout& L,
                            unsigned char* out, cudaStream_t s) {
  Part parts[7];
  const int np = parts_of(b, h, L, parts);
  // zero the padding after each part (under 8 bytes each) so that the
  // stream is a pure function of the blob; the copies fill the rest
  for (int i = 0; i < np; ++i) {
    const size_t end = parts[i].off + parts[i].bytes;
    const size_t next = i + 1 < np ? parts[i + 1].off : L.total;
    if (next > end) memset(out + end, 0, next - end);
  }
  unsigned long long* d_acc = nullptr;
  cudaError_t e = dev_alloc((void**)&d_acc, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  e = device_payload_sum(parts, np, d_acc, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out + offsetof(Header, checksum), d_acc, sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s);
  for (int i = 0; i < np && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(out + parts[i].off, parts[i].p, parts[i].bytes, cudaMemcpyDeviceToHost,
                        s);
  dev_free(d_acc, s);
  return e;
}

// Writes the header once the payload checksum has landed in out.
void finish_header(Header h, unsigned char* out) {
  unsigned long long acc;
  memcpy(&acc, out + offsetof(Header, checksum), sizeof(acc));
  h.checksum = 0;
  h.checksum = acc + host_checksum((const unsigned char*)&h, sizeof(Header), 0);
  memcpy(out, &h, sizeof(Header));
}

struct PendingHeader {
  Header h;
  unsigned char* out;
};

void CUDART_CB header_callback(void* p) {
  PendingHeader* ph = static_cast<PendingHeader*>(p);
  finish_header(ph->h, ph->out);
  delete ph;
}

}  // namespace

qoz_status qoz_blob_serialize(const qoz_blob* b, void* h_buf, size_t cap, size_t* used,
                              void* stream) {
  if (!b || !used) return fail(QOZ_EINVAL, "NULL argument");
  cudaStream_t s = stream ? (cudaStream_t)stream : b->stream;
  HuffEncoded h;
  qoz_status st = huff_encode(b, s, &h, h_buf == nullptr);
  if (st != QOZ_OK) return st;
  const Layout L = layout_of(b, h);
  *used = L.total;
  if (!h_buf) {
    huff_free(&h, s);
    return QOZ_OK;
  }
  if (cap < L.total) {
    huff_free(&h, s);
    return fail(QOZ_EINVAL, "buffer holds %zu bytes, %zu needed", cap, L.total);
  }
  unsigned char* out = (unsigned char*)h_buf;
  const Header hd = header_of(b, L);
  cudaError_t e = enqueue_payload(b, h, L, out, s);
  huff_free(&h, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "serialize");
  finish_header(hd, out);
  return QOZ_OK;
}

qoz_status qoz_blob_serialize_async(const qoz_blob* b, void* h_buf, size_t cap, size_t* used,
                                    void* stream) {
  if (!b || !used || !h_buf) return fail(QOZ_EINVAL, "NULL argument");
  cudaStream_t s = stream ? (cudaStream_t)stream : b->stream;
  HuffEncoded h;
  qoz_status st = huff_encode(b, s, &h, false);
  if (st != QOZ_OK) return st;
  const Layout L = layout_of(b, h);
  *used = L.total;
  if (cap < L.total) {
    huff_free(&h, s);
    return fail(QOZ_EINVAL, "buffer holds %zu bytes, %zu needed", cap, L.total);
  }
  unsigned char* out = (unsigned char*)h_buf;
  PendingHeader* ph = new PendingHeader{header_of(b, L), out};
  cudaError_t e = enqueue_payload(b, h, L, out, s);
  huff_free(&h, s);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(s, header_callback, ph);
  if (e != cudaSuccess) {
    delete ph;
    return cuda_fail(e, "serialize");
  }
  return QOZ_OK;
}

qoz_status qoz_blob_serialize_bound(const qoz_blob* b, size_t* bound) {
  if (!b || !bound) return fail(QOZ_EINVAL, "NULL argument");
  // an optimal prefix code averages under 17 bits on a 65536-symbol
  // alphabet; each chunk adds at most one partly filled word
  const long long nch = (b->N + kEntropyChunkMin - 1) / kEntropyChunkMin;  // at most
  const long long words = (b->N * 17 + 31) / 32 + nch;
  *bound = layout_of(b->na, b->nu, 65536, nch, words, kEntropyChunkMin).total;
  return QOZ_OK;
}

// Host checks of a code section's fixed part against the field: chunking,
// counts, a complete prefix code (Kraft's equality) and the symbol order.
static bool code_section_ok(const HuffFixed& f, long long N, const unsigned char* sym_bytes,
                     size_t avail) {
  if (f.chunk < 8 || f.chunk > (uint32_t)kEntropyChunk || f.chunk % 8 != 0 || f.flags != 0)
    return false;
  const long long nch = (N + f.chunk - 1) / f.chunk;
  if ((long long)f.n_chunks != nch) return false;
  if (f.n_sym > 65536 || f.max_len > (uint32_t)kMaxCodeLen || f.bl_count[0] != 0) return false;
  if ((N > 0) != (f.n_sym > 0)) return false;
  unsigned long long sum = 0, kraft = 0;
  for (int l = 1; l < 64; ++l) {
    if (l > (int)f.max_len && f.bl_count[l]) return false;
    sum += f.bl_count[l];
    if (l <= (int)f.max_len) kraft += (unsigned long long)f.bl_count[l] << (f.max_len - l);
  }
  if (sum != f.n_sym) return false;
  if (f.n_sym == 1 && !(f.max_len == 1 && f.bl_count[1] == 1)) return false;
  if (f.n_sym >= 2 && kraft != (1ull << f.max_len)) return false;
  if (avail < sizeof(uint16_t) * f.n_sym) return false;
  // symbols: increasing within each length, each used once
  std::vector<unsigned char> seen(65536, 0);
  size_t k = 0;
  for (int l = 1; l <= (int)f.max_len; ++l) {
    int prev = -1;
    for (unsigned j = 0; j < f.bl_count[l]; ++j, ++k) {
      uint16_t v;
      memcpy(&v, sym_bytes + 2 * k, 2);
      if ((int)v <= prev || seen[v]) return false;
      seen[v] = 1;
      prev = v;
    }
  }
  return true;
}

qoz_status qoz_blob_deserialize(const void* h_buf, size_t size, void* stream, qoz_blob** out) {
  if (!h_buf || !out) return fail(QOZ_EINVAL, "NULL argument");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (size < sizeof(Header)) return fail(QOZ_ECORRUPT, "stream shorter than its header");
  Header h;
  memcpy(&h, h_buf, sizeof(Header));
  if (fault_injected("header") || memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion ||
      h.header_bytes != sizeof(Header) || h.coding != kCodingHuffman)
    return fail(QOZ_ECORRUPT, "bad magic / version");
  qoz_shape shape;
  shape.ndims = h.ndims;
  for (int i = 0; i < 3; ++i) shape.dims[i] = h.dims[i];
  qoz_params p;
  memset(&p, 0, sizeof(p));
  p.anchor_stride = h.anchor_stride;
  memcpy(p.interp, h.interp, 8);
  memcpy(p.order, h.order, 8);
  p.alpha = h.alpha;
  p.beta = h.beta;
  Resolved r;
  if (resolve(shape, &p, &r) != QOZ_OK) return fail(QOZ_ECORRUPT, "header: invalid shape/params");
  long long na = 1;
  for (int i = 0; i < 3; ++i) na *= (r.n[i] + r.p.anchor_stride - 1) / r.p.anchor_stride;
  if (h.n_points != r.N || h.n_anchors != na || h.n_unpred < 0 || h.n_unpred > r.N ||
      !(h.abs_eb >= 0.0) || !std::isfinite(h.abs_eb))
    return fail(QOZ_ECORRUPT, "header: inconsistent counts or bound");
  const unsigned char* in = (const unsigned char*)h_buf;
  // the code section's fixed part gives the remaining sizes
  const Layout L0 = layout_of(na, h.n_unpred, 0, 0, 0, 0);
  if (size < L0.codes + sizeof(HuffFixed)) return fail(QOZ_ECORRUPT, "stream truncated");
  HuffFixed f;
  memcpy(&f, in + L0.codes, sizeof(f));
  if (f.n_sym > 65536 || (long long)f.n_chunks < 0 || f.n_chunks > (uint64_t)r.N + 1 ||
      f.n_words > (uint64_t)(size / 4) || f.chunk < 8 || f.chunk > (uint32_t)kEntropyChunk ||
      f.chunk % 8 != 0)
    return fail(QOZ_ECORRUPT, "code section: inconsistent sizes");
  const Layout L = layout_of(na, h.n_unpred, f.n_sym, (long long)f.n_chunks, (long long)f.n_words,
                             (int)f.chunk);
  if (size < L.total || h.code_bytes != L.total - L.codes)
    return fail(QOZ_ECORRUPT, "stream truncated (%zu < %zu)", size, L.total);
  if (!code_section_ok(f, r.N, in + L.sym, L.offs - L.sym))
    return fail(QOZ_ECORRUPT, "code section: not a complete canonical code");
  {
    // word offsets: from 0, non-decreasing, ending at the word count
    unsigned long long prev = 0;
    for (uint64_t c = 0; c <= f.n_chunks; ++c) {
      unsigned long long v;
      memcpy(&v, in + L.offs + 8 * c, 8);
      if ((c == 0 && v != 0) || v < prev || v > f.n_words) return fail(QOZ_ECORRUPT, "chunk offsets");
      if (c == f.n_chunks && v != f.n_words) return fail(QOZ_ECORRUPT, "chunk offsets");
      prev = v;
    }
  }
  // host check of the unpredictable list: strictly increasing, inside the field
  {
    const long long* ui = (const long long*)(in + L.uidx);
    for (long long k = 0; k < h.n_unpred; ++k) {
      long long v;
      memcpy(&v, ui + k, sizeof(v));
      long long prev = -1;
      if (k > 0) memcpy(&prev, ui + k - 1, sizeof(prev));
      if (v < 0 || v >= r.N || v <= prev) return fail(QOZ_ECORRUPT, "unpredictable list order");
    }
  }
  configure_pool_once();
  qoz_blob* b = new qoz_blob();
  memset(b, 0, sizeof(*b));
  b->shape = shape;
  for (int i = 0; i < 3; ++i) b->n[i] = r.n[i];
  b->N = r.N;
  b->L = r.L;
  b->params = r.p;
  b->abs_eb = h.abs_eb;
  b->rel_eb = h.rel_eb;
  b->vmin = h.vmin;
  b->vmax = h.vmax;
  b->na = na;
  b->nu = h.n_unpred;
  b->stream = s;
  cudaGetDevice(&b->device);
  HuffEncoded hc;
  memset(&hc, 0, sizeof(hc));
  hc.fixed = f;
  hc.chunk = (int)f.chunk;
  hc.n_chunks = (long long)f.n_chunks;
  hc.n_words = (long long)f.n_words;
  hc.sym_bytes = pad8_bytes(sizeof(uint16_t) * 65536);
  auto cleanup = [&](qoz_status st) {
    huff_free(&hc, s);
    qoz_blob_free(b);
    return st;
  };
  unsigned long long* d_acc = nullptr;
  cudaError_t e;
  hc.sub_bytes = entropy_sub_bytes(hc.n_chunks, hc.chunk);
  const size_t sec = sizeof(HuffFixed) + hc.sym_bytes + 8 * (hc.n_chunks + 1) + hc.sub_bytes;
  if ((e = dev_alloc((void**)&b->d_codes, sizeof(uint16_t) * b->N, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_anchors, sizeof(float) * na, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_uidx, sizeof(long long) * b->nu, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_uval, sizeof(float) * b->nu, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_hist, sizeof(unsigned) * 65536, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&b->d_err, sizeof(int), s)) != cudaSuccess ||
      (e = dev_alloc(&hc.d_section, sec, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&hc.d_words, sizeof(uint32_t) * hc.n_words + 8, s)) != cudaSuccess ||
      (e = dev_alloc((void**)&d_acc, sizeof(unsigned long long), s)) != cudaSuccess)
    return cleanup(fail(QOZ_ENOMEM, "deserialize allocation"));
  char* dsec = static_cast<char*>(hc.d_section);
  e = cudaMemsetAsync(b->d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hc.d_section, 0, sec, s);
  if (e == cudaSuccess && na)
    e = cudaMemcpyAsync(b->d_anchors, in + L.anchors, sizeof(float) * na, cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess && b->nu)
    e = cudaMemcpyAsync(b->d_uidx, in + L.uidx, sizeof(long long) * b->nu,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && b->nu)
    e = cudaMemcpyAsync(b->d_uval, in + L.uval, sizeof(float) * b->nu, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dsec, in + L.codes, L.offs - L.codes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dsec + sizeof(HuffFixed) + hc.sym_bytes, in + L.offs, L.words - L.offs,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && hc.n_words)
    e = cudaMemcpyAsync(hc.d_words, in + L.words, sizeof(uint32_t) * hc.n_words,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_check(huff_decode(hc.d_section, hc.d_words, hc.n_chunks, hc.chunk, f.n_sym, b->N,
                                 b->d_codes,
                                 b->d_err, s));
  Part parts[7];
  const int np = e == cudaSuccess ? parts_of(b, hc, L, parts) : 0;
  if (e == cudaSuccess) e = device_payload_sum(parts, np, d_acc, s);
  if (e == cudaSuccess) e = launch_histogram(b->d_codes, b->N, b->d_hist, b->na, s);
  unsigned long long acc = 0;
  int derr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, d_acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(d_acc, s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "deserialize"));
  const uint64_t want = h.checksum;
  h.checksum = 0;
  const uint64_t got = acc + host_checksum((const unsigned char*)&h, sizeof(Header), 0);
  if (got != want) return cleanup(fail(QOZ_ECORRUPT, "checksum mismatch"));
  if (derr) return cleanup(fail(QOZ_ECORRUPT, "code stream does not decode"));
  huff_free(&hc, s);
  cudaMemsetAsync(b->d_err, 0, sizeof(int), s);
  *out = b;
  return QOZ_OK;
}

}  // extern "C"
