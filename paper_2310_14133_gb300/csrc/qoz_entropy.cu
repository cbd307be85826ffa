// Entropy stage: canonical Huffman coding of the quantization codes, the
// encoder that the rate estimate of Sec. 6.1 stands for (the paper follows
// Huffman coding with a dictionary coder; that lossless pass is not part of
// this stage).
//
// Definitions (the paper names Huffman coding but fixes none of these):
//   - symbols: the 16-bit code of every point in field order, anchors
//     included (they carry code 0);
//   - construction: the used symbols sorted by (count, symbol) form the leaf
//     queue, merged nodes a second queue in creation order; each pick takes
//     the node-queue head when its weight is strictly below the leaf head's
//     (or no leaf is left), otherwise the leaf; a symbol's code length is its
//     depth, a lone symbol gets length 1;
//   - canonical codes (RFC 1951 Sec. 3.2.2): consecutive integers in
//     (length, symbol) order;
//   - stream: chunks of C symbols (entropy_chunk: the largest power of two
//     from 256 to 4096 that gives at least 8192 chunks, recorded in the
//     section's fixed part), each starting on a 32-bit
//     word, codes most significant bit first, words filled from their most
//     significant bit, the tail of a chunk's last word zero;
//   - run table: a chunk of 1024 symbols or more is cut into runs of
//     kEntropyRun (512) symbols, and the coded length in bits of each run
//     but the last is stored (uint16), so a decoder can start at every run.
//
// Kernels: one CTA builds the table (shared memory up to kHuffSmemSym used
// symbols, a global workspace beyond); the encoder counts each chunk's words
// and its runs' bits, scans the word counts into offsets and writes the
// chunks (one warp per chunk, each lane a run of consecutive symbols); the
// decoder gives each run its own thread, which starts at the bit the run
// table gives and decodes with a 12-bit lookup table and, for longer codes,
// the canonical codes' interval ends, checking every index against the
// stream it was given and that the run ends where the next one starts.
// Smaller fields get smaller chunks so that their decode still spreads over
// thousands of threads.
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "../../include/qoz.h"
#include "qoz_host.h"
#include "qoz_internal.h"

namespace qoz {
namespace {

constexpr int kSymbols = 65536;
constexpr int kTabThreads = 1024;
constexpr int kHuffSmemSym = 4096;  // used symbols handled in shared memory
constexpr int kLut = 12;            // bits of the decoder's lookup table
constexpr int kDecSmemSym = 12288;  // symbols the decoder keeps in shared memory
constexpr int kDecThreads = 256;    // decoder: one run of a chunk per thread
constexpr int kRingWords = 32;      // decoder: stream words staged per thread
constexpr int kRingGroup = 8;       // decoder: words per asynchronous refill

// Workspace of the table kernel (device memory).
struct HuffWork {
  unsigned long long keys[kSymbols];   // (count << 16 | symbol), then (length << 16 | symbol)
  unsigned long long nodew[kSymbols];  // merged-node weights
  int child[2 * kSymbols];             // children of each merged node (leaf i, node n + j)
  unsigned char depth[kSymbols];       // merged-node depths
  unsigned char leaf_len[kSymbols];    // code length of leaf i (sorted order)
  unsigned char len[kSymbols];         // code length per symbol (encoder)
  unsigned long long code[kSymbols];   // canonical code per symbol << 6 | its length (encoder)
  int err;  // 1: a code longer than kMaxCodeLen; 2: a code without a table entry
};

__device__ __forceinline__ void bitonic_sort(unsigned long long* k, int P) {
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned long long a = k[i], b = k[j];
          if ((a > b) == up) {
            k[i] = b;
            k[j] = a;
          }
        }
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(kTabThreads)
    huff_table_kernel(const unsigned* __restrict__ hist, long long extra0, int chunk,
                      HuffWork* w, HuffFixed* fx, uint16_t* sym_out) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int nsh, maxlen_sh, err_sh;
  __shared__ unsigned bl[64];
  __shared__ unsigned long long first_code[64];
  __shared__ int first_index[64];
  const int t = threadIdx.x;
  if (t == 0) {
    nsh = 0;
    maxlen_sh = 0;
    err_sh = 0;
  }
  if (t < 64) bl[t] = 0;
  for (int s = t; s < kSymbols; s += kTabThreads) {
    w->len[s] = 0;
    w->code[s] = 0ull;
  }
  __syncthreads();
  // used symbols in any order (sorted next); anchors add to symbol 0.  The
  // histogram is read as 16-byte vectors, four loads in flight per thread.
  unsigned long long* gk = w->keys;
  const uint4* h4 = reinterpret_cast<const uint4*>(hist);
  constexpr int kVec = kSymbols / 4 / kTabThreads;  // 16
  for (int j0 = 0; j0 < kVec; j0 += 4) {
    uint4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = h4[(j0 + j) * kTabThreads + t];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s0 = 4 * ((j0 + j) * kTabThreads + t);
      const unsigned cv[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned long long c =
            (unsigned long long)cv[k] + (s0 + k == 0 ? (unsigned long long)extra0 : 0ull);
        if (c) gk[atomicAdd(&nsh, 1)] = (c << 16) | (unsigned long long)(s0 + k);
      }
    }
  }
  __syncthreads();
  const int n = nsh;
  const bool small = n <= kHuffSmemSym;
  unsigned long long* keys = small ? reinterpret_cast<unsigned long long*>(sm) : w->keys;
  unsigned long long* nodew = small ? keys + kHuffSmemSym : w->nodew;
  int* child = small ? reinterpret_cast<int*>(nodew + kHuffSmemSym) : w->child;
  unsigned char* depth = small ? reinterpret_cast<unsigned char*>(child + 2 * kHuffSmemSym)
                               : w->depth;
  unsigned char* leaf_len = small ? depth + kHuffSmemSym : w->leaf_len;
  int P = 1;
  while (P < n) P <<= 1;
  if (small)
    for (int i = t; i < n; i += kTabThreads) keys[i] = gk[i];
  for (int i = n + t; i < P; i += kTabThreads) keys[i] = ~0ull;
  __syncthreads();
  bitonic_sort(keys, P);

  if (t == 0 && n == 1) {
    leaf_len[0] = 1;
    maxlen_sh = 1;
  } else if (t == 0 && n > 1) {
    // two-queue merge, heads in registers
    int li = 0, ni = 0, nn = 0;
    unsigned long long hl = keys[0] >> 16, hn = 0ull;
    for (int m = 0; m < n - 1; ++m) {
      int id[2];
      unsigned long long wt[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (ni < nn && (li >= n || hn < hl)) {
          id[k] = n + ni;
          wt[k] = hn;
          ++ni;
          hn = ni < nn ? nodew[ni] : 0ull;
        } else {
          id[k] = li;
          wt[k] = hl;
          ++li;
          hl = li < n ? (keys[li] >> 16) : ~0ull;
        }
      }
      const unsigned long long sum = wt[0] + wt[1];
      nodew[nn] = sum;
      child[2 * nn] = id[0];
      child[2 * nn + 1] = id[1];
      if (ni == nn) hn = sum;
      ++nn;
    }
    // depths from the root (the last merged node) down
    int mx = 0, bad = 0;
    depth[n - 2] = 0;
    for (int j = n - 2; j >= 0; --j) {
      const int d = depth[j] + 1;
      if (d > kMaxCodeLen) {
        bad = 1;
        break;
      }
      for (int k = 0; k < 2; ++k) {
        const int ch = child[2 * j + k];
        if (ch >= n)
          depth[ch - n] = (unsigned char)d;
        else {
          leaf_len[ch] = (unsigned char)d;
          mx = d > mx ? d : mx;
        }
      }
    }
    maxlen_sh = mx;
    err_sh = bad;
  }
  __syncthreads();
  if (err_sh) {
    if (t == 0) w->err = 1;
    return;
  }
  // lengths per symbol; keys become (length << 16 | symbol)
  for (int i = t; i < n; i += kTabThreads) {
    const int s = (int)(keys[i] & 0xffffull);
    const int L = leaf_len[i];
    w->len[s] = (unsigned char)L;
    atomicAdd(&bl[L], 1u);
    keys[i] = ((unsigned long long)L << 16) | (unsigned long long)s;
  }
  __syncthreads();
  bitonic_sort(keys, P);
  const int maxlen = maxlen_sh;
  if (t == 0) {
    unsigned long long c = 0ull;
    int idx = 0;
    first_code[0] = 0ull;
    first_index[0] = 0;
    for (int b = 1; b <= maxlen; ++b) {
      c = (c + (b == 1 ? 0ull : bl[b - 1])) << 1;
      first_code[b] = c;
      first_index[b] = idx;
      idx += (int)bl[b];
    }
    fx->n_sym = (uint32_t)n;
    fx->max_len = (uint32_t)maxlen;
    fx->chunk = (uint32_t)chunk;
    fx->flags = 0u;
    for (int b = 0; b < 64; ++b) fx->bl_count[b] = b <= maxlen ? bl[b] : 0u;
    w->err = 0;
  }
  __syncthreads();
  for (int i = t; i < n; i += kTabThreads) {
    const int L = (int)(keys[i] >> 16);
    const int s = (int)(keys[i] & 0xffffull);
    w->code[s] = ((first_code[L] + (unsigned long long)(i - first_index[L])) << 6) |
                 (unsigned long long)L;
    sym_out[i] = (uint16_t)s;
  }
}

// Words of each chunk (one warp per chunk; the lanes read the chunk's codes
// as consecutive 16-byte vectors and sum their code lengths).

__device__ __forceinline__ void load8(const uint16_t* __restrict__ sym, long long i, long long n,
                                      uint32_t v[4]) {
  if (i + 8 <= n) {
    const uint4 q = *reinterpret_cast<const uint4*>(sym + i);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    for (int k = 0; k < 4; ++k) {
      const uint32_t lo = i + 2 * k < n ? sym[i + 2 * k] : 0u;
      const uint32_t hi = i + 2 * k + 1 < n ? sym[i + 2 * k + 1] : 0u;
      v[k] = lo | (hi << 16);
    }
  }
}

__global__ void __launch_bounds__(256)
    huff_count_kernel(const uint16_t* __restrict__ sym, long long n,
                      const unsigned char* __restrict__ len, long long nchunks, int chunk,
                      unsigned long long* __restrict__ offs, uint16_t* __restrict__ sub,
                      int* err) {
  const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nchunks) return;
  const long long base = c * chunk;
  const int runs = entropy_runs(chunk);
  unsigned bits = 0, rbits = 0;
  bool missing = false;  // a code the table has no entry for
  // step j covers codes 256 j .. 256 j + 255 of the chunk: two steps per run
  for (int j = 0; j < chunk / 256; ++j) {
    const long long i = base + 8ll * (j * 32 + lane);
    if (i < n) {
      uint32_t v[4];
      load8(sym, i, n, v);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (i + k >= n) break;
        const unsigned L = len[(v[k >> 1] >> (16 * (k & 1))) & 0xffffu];
        missing |= L == 0u;
        rbits += L;
      }
    }
    if (runs > 1 && (j & 1)) {  // a run ends: its length into the table (all but the last)
      unsigned r = rbits;
      for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
      if (lane == 0 && (j >> 1) + 1 < runs) sub[c * (runs - 1) + (j >> 1)] = (uint16_t)r;
      bits += rbits;
      rbits = 0;
    }
  }
  bits += rbits;
  if (missing) atomicOr(err, 2);
  for (int off = 16; off > 0; off >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, off);
  if (lane == 0) offs[c] = (bits + 31) / 32;
}

// Exclusive scan of the per-chunk word counts in place (one CTA); offs[n]
// receives the total, which also lands in the section's fixed part.  Each
// warp owns a contiguous segment and reads it lane-strided (coalesced),
// eight rounds of loads in flight.
__global__ void __launch_bounds__(1024)
    chunk_scan_kernel(unsigned long long* offs, long long nchunks, HuffFixed* fx) {
  __shared__ unsigned long long wsum[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long seg = (nchunks + 31) / 32;
  const long long b = warp * seg, e = b + seg < nchunks ? b + seg : nchunks;
  unsigned long long s = 0;
  for (long long i0 = b; i0 < e; i0 += 32 * 8) {
    unsigned long long v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const long long i = i0 + 32 * k + lane;
      v[k] = i < e ? offs[i] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) wsum[warp] = s;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long x = wsum[lane];
    unsigned long long inc = x;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    wsum[lane] = inc - x;
    if (lane == 31) {
      offs[nchunks] = inc;
      fx->n_chunks = (uint64_t)nchunks;
      fx->n_words = (uint64_t)inc;
    }
  }
  __syncthreads();
  unsigned long long carry = wsum[warp];
  for (long long i0 = b; i0 < e; i0 += 32 * 8) {
    unsigned long long v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const long long i = i0 + 32 * k + lane;
      v[k] = i < e ? offs[i] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      unsigned long long inc = v[k];
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
      }
      const long long i = i0 + 32 * k + lane;
      if (i < e) offs[i] = carry + inc - v[k];
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
}

// The chunks' bits (one warp per chunk).  The chunk's codes are read as
// consecutive 16-byte vectors and transposed through shared memory into one
// run of kRun consecutive codes per lane (rows padded by one word: the
// lanes' reads fall in distinct banks).  A lane places its run from its bit
// offset in the chunk; words the run covers whole are stored, the first and
// last (shared with the neighbouring runs) are OR-ed into the zeroed stream.
constexpr int kEncWarps = 4;  // 33 KB of static shared memory per CTA at 4096

// Appends L <= 32 bits to the lane's accumulator (nacc < 32 pending bits
// before, so at most one word completes).
__device__ __forceinline__ void put_bits(unsigned long long& acc, int& nacc, unsigned long long v,
                                         int L, uint32_t* out, long long& wi, bool& first,
                                         bool shared_first, long long nwc) {
  acc = (acc << L) | v;
  nacc += L;
  if (nacc >= 32) {
    nacc -= 32;
    const uint32_t w = (uint32_t)(acc >> nacc);
    acc &= (1ull << nacc) - 1ull;
    if (QOZ_IN(wi, nwc)) {
      if (first && shared_first)
        atomicOr(out + wi, w);
      else
        out[wi] = w;
    }
    ++wi;
    first = false;
  }
}

template <bool LONG, int CHUNK>
__global__ void __launch_bounds__(32 * kEncWarps)
    huff_encode_kernel(const uint16_t* __restrict__ sym, long long n,
                       const unsigned long long* __restrict__ entry, long long nchunks,
                       const unsigned long long* __restrict__ offs, uint32_t* words) {
  constexpr int kRun = CHUNK / 32;  // symbols of one lane's run
  constexpr int kVecPerChunk = CHUNK / 8;
  constexpr int kRowWords = kRun / 2 + 1;
  __shared__ uint32_t stage[kEncWarps][32 * kRowWords];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long c = (long long)blockIdx.x * kEncWarps + warp;
  if (c >= nchunks) return;
  const long long base = c * CHUNK;
  uint32_t* st = stage[warp];
  for (int j = 0; j < kVecPerChunk / 32; ++j) {
    const int q = j * 32 + lane;  // vector q holds codes 8q .. 8q + 7 of the chunk
    uint32_t v[4];
    load8(sym, base + 8ll * q, n, v);
    const int row = q / (kRun / 8), col = 4 * (q % (kRun / 8));
#pragma unroll
    for (int k = 0; k < 4; ++k) st[row * kRowWords + col + k] = v[k];
  }
  __syncwarp();
  const long long b = base + (long long)lane * kRun;
  const int cnt = b >= n ? 0 : (int)(b + kRun < n ? kRun : n - b);
  const uint32_t* mine = st + lane * kRowWords;
  auto sym_at = [&](int k) -> int { return (int)((mine[k >> 1] >> (16 * (k & 1))) & 0xffffu); };
  unsigned long long bits = 0;
  for (int k = 0; k < cnt; ++k) bits += entry[sym_at(k)] & 63ull;
  unsigned long long start = bits;  // inclusive scan over the lanes
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, start, off);
    if (lane >= off) start += v;
  }
  start -= bits;
  if (bits == 0) return;
  uint32_t* out = words + offs[c];
  const long long nwc = (long long)(offs[c + 1] - offs[c]);  // the chunk's words
  (void)nwc;
  long long wi = (long long)(start >> 5);
  int nacc = (int)(start & 31);  // pending bits (leading zeros of the first word)
  unsigned long long acc = 0ull;
  bool first = true;
  const bool shared_first = (start & 31) != 0;
  for (int k = 0; k < cnt; ++k) {
    const unsigned long long en = entry[sym_at(k)];
    const int L = (int)(en & 63ull);
    const unsigned long long cv = en >> 6;
    if (LONG && L > 32) {  // the high part first
      put_bits(acc, nacc, cv >> 32, L - 32, out, wi, first, shared_first, nwc);
      put_bits(acc, nacc, cv & 0xffffffffull, 32, out, wi, first, shared_first, nwc);
    } else {
      put_bits(acc, nacc, cv, L, out, wi, first, shared_first, nwc);
    }
  }
  if (nacc > 0 && QOZ_IN(wi, nwc)) atomicOr(out + wi, (uint32_t)(acc << (32 - nacc)));
}

// Decoder tables in shared memory: 12-bit lookup (symbol << 8 | length, 0
// for prefixes of longer codes) and the canonical first code / index per
// length.
struct DecTables {
  uint32_t lut[1 << kLut];
  unsigned long long first_code[64];
  // end of length L's codes, left-justified in 64 bits: canonical codes of
  // increasing length occupy consecutive intervals, so a code's length is
  // the first L whose end exceeds the next 64 stream bits
  unsigned long long end[64];
  unsigned first_index[64];
  unsigned count[64];
};

// A code longer than kLut bits at bit pos of its chunk, x the 32 stream bits
// from pos on: the length from the canonical intervals while the code fits
// in x, then bit by bit from the stream.  Returns (length, symbol), the
// symbol negative when no code matches.
__device__ __noinline__ int2 decode_long(const DecTables& T, uint32_t x, unsigned long long pos,
                                         const uint32_t* __restrict__ W, unsigned long long nw,
                                         int maxlen, unsigned nsym,
                                         const uint16_t* __restrict__ syms) {
  const unsigned long long top = (unsigned long long)x << 32;
  const int lim = maxlen < 32 ? maxlen : 32;
  int L = kLut + 1;
  while (L <= lim && top >= T.end[L]) ++L;
  if (L <= lim) {
    const unsigned long long d = (unsigned long long)(x >> (32 - L)) - T.first_code[L];
    if (d < T.count[L] && T.first_index[L] + d < nsym)
      return make_int2(L, (int)syms[T.first_index[L] + d]);
    return make_int2(L, -1);
  }
  L = lim;
  unsigned long long v = L > 0 ? (unsigned long long)(x >> (32 - L)) : 0ull;
  while (L < maxlen) {
    ++L;
    const unsigned long long q = pos + (unsigned long long)(L - 1);
    const uint32_t w = (q >> 5) < nw ? W[q >> 5] : 0u;
    v = (v << 1) | ((w >> (31 - (q & 31))) & 1u);
    if (v >= T.first_code[L] && v - T.first_code[L] < T.count[L]) {
      const unsigned long long k = T.first_index[L] + (v - T.first_code[L]);
      return make_int2(L, k < nsym ? (int)syms[k] : -1);
    }
  }
  return make_int2(L, -1);
}

__global__ void __launch_bounds__(kDecThreads)
    huff_decode_kernel(const uint32_t* __restrict__ words,
                       const unsigned long long* __restrict__ offs,
                       const uint16_t* __restrict__ sub, long long nchunks, int chunk,
                       int runs, long long n, const HuffFixed* __restrict__ fx,
                       const uint16_t* __restrict__ syms, unsigned nss,
                       uint16_t* __restrict__ out, int* err) {
  __shared__ DecTables T;
  // dynamic: the threads' word rings, then nss <= n_sym symbols
  extern __shared__ __align__(16) uint32_t ring_all[];
  uint16_t* ssym = reinterpret_cast<uint16_t*>(ring_all + kDecThreads * (kRingWords + 1));
  const int t = threadIdx.x;
  const int maxlen = (int)fx->max_len;
  const unsigned nsym = fx->n_sym;
  for (int i = t; i < (1 << kLut); i += blockDim.x) T.lut[i] = 0u;
  if (t == 0) {
    unsigned long long c = 0ull;
    unsigned idx = 0;
    for (int b = 0; b < 64; ++b) {
      if (b >= 1) c = (c + (b == 1 ? 0ull : fx->bl_count[b - 1])) << 1;
      T.first_code[b] = c;
      T.first_index[b] = idx;
      T.count[b] = b >= 1 && b <= maxlen ? fx->bl_count[b] : 0u;
      idx += T.count[b];
      const unsigned long long lim = c + T.count[b];
      T.end[b] = b == 0 ? 0ull : (lim >= (1ull << b) ? ~0ull : lim << (64 - b));
    }
  }
  __syncthreads();
  // lookup entries, one per kLut-bit prefix: the code whose interval holds
  // the prefix (symbol << 8 | length) if its length is at most kLut; for a
  // prefix of longer codes 0x80 | the shortest length among them; 0 for a
  // prefix of no code
  for (int k = t; k < (1 << kLut); k += blockDim.x) {
    const unsigned long long top = (unsigned long long)k << (64 - kLut);
    int L = 1;
    while (L <= maxlen && top >= T.end[L]) ++L;
    if (L > maxlen) continue;
    if (L > kLut) {
      T.lut[k] = 0x80u | (uint32_t)L;
      continue;
    }
    const unsigned long long d = (top >> (64 - L)) - T.first_code[L];
    if (d < T.count[L] && T.first_index[L] + d < nsym)
      T.lut[k] = ((uint32_t)syms[T.first_index[L] + d] << 8) | (uint32_t)L;
  }
  // the first nss symbols (the long codes' among them) in shared memory
  for (unsigned k = t; k < nss; k += blockDim.x) ssym[k] = syms[k];
  __syncthreads();
  // one thread per run of a chunk: its first bit is the sum of the lengths
  // the table records for the runs before it
  const long long item = blockIdx.x * (long long)blockDim.x + t;
  if (item >= nchunks * runs) return;
  const long long c = item / runs;
  const int run = (int)(item - c * runs);
  const unsigned long long w0 = offs[c], w1 = offs[c + 1];
  if (w1 < w0 || w1 - w0 > 0xffffffffull) {
    atomicOr(err, 4);
    return;
  }
  unsigned long long first = 0;  // the run's first bit in the chunk
  for (int k = 0; k < run; ++k) first += sub[c * (runs - 1) + k];
  const unsigned long long cbits = 32ull * (w1 - w0);
  if (first > cbits) {
    atomicOr(err, 4);
    return;
  }
  const unsigned nw = (unsigned)(w1 - w0 - (first >> 5));  // words from the run's first on
  const uint32_t* W = words + w0 + (first >> 5);
  // The chunk's words pass through this thread's ring of kRingWords words
  // in shared memory (four groups of kRingGroup), filled by asynchronous
  // copies a group at a time: when the window's second word enters group m,
  // group m + 2 is issued into the slots of group m - 2 and group m is
  // waited for (two groups may stay in flight).  Words past the chunk's end
  // read as zero.
  uint32_t* ring = ring_all + t * (kRingWords + 1);
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  auto issue_group = [&](unsigned g) {
#pragma unroll
    for (int k = 0; k < kRingGroup; ++k) {
      const unsigned wi = kRingGroup * g + k;
      const bool in = wi < nw;
      const uint32_t* src = in ? W + wi : words;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(
                       ring_s + 4 * (wi & (kRingWords - 1))),
                   "l"(src), "r"(in ? 4 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  issue_group(0);
  issue_group(1);
  issue_group(2);
  asm volatile("cp.async.wait_group 2;\n" ::: "memory");
  // the window: words wcur and wcur + 1 (w0r, w1r), sh bits of w0r consumed
  unsigned wcur = 0;
  uint32_t w0r = ring[0], w1r = ring[1];
  int sh = (int)(first & 31);
  // the window moves on by one word when adv (without a branch but for the
  // rare refill)
  auto advance = [&](bool adv) {
    w0r = adv ? w1r : w0r;
    wcur += adv ? 1u : 0u;
    const unsigned nx = wcur + 1;
    if (adv && (nx & (kRingGroup - 1)) == 0) {
      issue_group(nx / kRingGroup + 2);
      asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    }
    const uint32_t nxt = ring[nx & (kRingWords - 1)];
    w1r = adv ? nxt : w1r;
  };
  // one code: the 32 stream bits from the window's position and the lookup
  // table; a longer code's length from the canonical interval ends, starting
  // at the shortest length under its prefix, its symbol from shared memory;
  // codes beyond 32 bits and prefixes of no code out of line
  const int lim = maxlen < 32 ? maxlen : 32;
  auto decode = [&](int& sym) -> bool {
    const uint32_t x = __funnelshift_l(w1r, w0r, (unsigned)sh);
    const uint32_t ent = T.lut[x >> (32 - kLut)];
    int L = (int)(ent & 0xffu);
    sym = (int)(ent >> 8);
    if (L & 0x80) {
      L &= 0x7f;
      if (L <= lim) {
        const unsigned long long top = (unsigned long long)x << 32;
        while (L < lim && top >= T.end[L]) ++L;
        const unsigned long long d = (unsigned long long)(x >> (32 - L)) - T.first_code[L];
        const unsigned long long k = T.first_index[L] + d;
        if (top < T.end[L] && d < T.count[L] && k < nsym)
          sym = k < nss ? (int)ssym[k] : (int)syms[k];
        else
          L = 0;
      } else {
        L = 0;
      }
    }
    if (L == 0) {
      const int2 r = decode_long(T, x, 32ull * wcur + (unsigned long long)sh, W, nw, maxlen,
                                 nsym, syms);
      L = r.x;
      sym = r.y;
      if (sym < 0) return false;
      if (L > 32) {  // a code longer than a word: the window moves twice
        L -= 32;
        advance(true);
      }
    }
    sh += L;
    const bool adv = sh >= 32;
    sh -= adv ? 32 : 0;
    advance(adv);
    return true;
  };
  const long long b = c * chunk + (long long)run * kEntropyRun;
  const long long cend = c * chunk + chunk < n ? c * chunk + chunk : n;
  const long long rend = runs > 1 && b + kEntropyRun < cend ? b + kEntropyRun : cend;
  const int cnt = b < rend ? (int)(rend - b) : 0;
  uint16_t* o = out + b;
  int i = 0;
  for (; i + 8 <= cnt; i += 8) {  // chunks start on multiples of eight codes
    uint32_t g[4];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int sym;
      if (!decode(sym)) {
        atomicOr(err, 4);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        return;
      }
      g[k >> 1] = (k & 1) ? (g[k >> 1] | ((uint32_t)sym << 16)) : (uint32_t)sym;
    }
    *reinterpret_cast<uint4*>(o + i) = make_uint4(g[0], g[1], g[2], g[3]);
  }
  for (; i < cnt; ++i) {
    int sym;
    if (!decode(sym)) {
      atomicOr(err, 4);
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      return;
    }
    o[i] = (uint16_t)sym;
  }
  // the codes must end inside the chunk's words, and a run but the last
  // exactly where the table puts the next one
  const unsigned long long end = 32ull * ((first >> 5) + wcur) + (unsigned long long)sh;
  if (end > cbits || (run + 1 < runs && end != first + sub[c * (runs - 1) + run]))
    atomicOr(err, 4);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

}  // namespace

size_t huff_fixed_bytes() { return sizeof(HuffFixed); }

void huff_free(HuffEncoded* h, cudaStream_t s) {
  dev_free(h->d_work, s);
  dev_free(h->d_section, s);
  dev_free(h->d_words, s);
  memset(h, 0, sizeof(*h));
}

qoz_status huff_encode(const qoz_blob* b, cudaStream_t s, HuffEncoded* h, bool sizes_only) {
  memset(h, 0, sizeof(*h));
  h->chunk = entropy_chunk(b->N);
  h->n_chunks = (b->N + h->chunk - 1) / h->chunk;
  // the section's fixed part and symbol list, then the chunk offsets and
  // the run table
  h->sym_bytes = pad8_bytes(sizeof(uint16_t) * kSymbols);
  h->sub_bytes = entropy_sub_bytes(h->n_chunks, h->chunk);
  const size_t sec = sizeof(HuffFixed) + h->sym_bytes +
                     sizeof(unsigned long long) * (h->n_chunks + 1) + h->sub_bytes;
  cudaError_t e = dev_alloc(&h->d_work, sizeof(HuffWork), s);
  if (e == cudaSuccess) e = dev_alloc(&h->d_section, sec, s);
  if (e != cudaSuccess) {
    huff_free(h, s);
    return fail(QOZ_ENOMEM, "entropy workspace");
  }
  HuffWork* w = static_cast<HuffWork*>(h->d_work);
  HuffFixed* fx = static_cast<HuffFixed*>(h->d_section);
  uint16_t* syms = reinterpret_cast<uint16_t*>(static_cast<char*>(h->d_section) + sizeof(HuffFixed));
  unsigned long long* offs = reinterpret_cast<unsigned long long*>(
      static_cast<char*>(h->d_section) + sizeof(HuffFixed) + h->sym_bytes);
  uint16_t* sub_tab = reinterpret_cast<uint16_t*>(offs + (h->n_chunks + 1));
  e = cudaMemsetAsync(h->d_section, 0, sec, s);
  constexpr size_t kTabSmem = (size_t)kHuffSmemSym * (8 + 8 + 8 + 1 + 1);
  static unsigned long long attr_done = 0;
  if (e == cudaSuccess)
    e = ensure_smem_attr((const void*)huff_table_kernel, &attr_done, kTabSmem);
  if (e == cudaSuccess) {
    huff_table_kernel<<<1, kTabThreads, kTabSmem, s>>>(b->d_hist, b->na, h->chunk, w, fx, syms);
    note_launch(1);
    e = launch_check(cudaGetLastError());
  }
  const long long nch = h->n_chunks;
  const unsigned grid = (unsigned)((nch * 32 + 255) / 256);
  if (e == cudaSuccess && nch > 0) {
    huff_count_kernel<<<grid, 256, 0, s>>>(b->d_codes, b->N, w->len, nch, h->chunk, offs,
                                           sub_tab, &w->err);
    note_launch(1);
    e = launch_check(cudaGetLastError());
  }
  if (e == cudaSuccess) {
    chunk_scan_kernel<<<1, 1024, 0, s>>>(offs, nch, fx);
    note_launch(1);
    e = launch_check(cudaGetLastError());
  }
  // sizes to the host (one synchronisation): the stream's length is known
  // only once the table and the counts exist
  HuffFixed hf;
  int werr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, fx, sizeof(hf), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&werr, &w->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    huff_free(h, s);
    return cuda_fail(e, "entropy table");
  }
  if (werr & 1) {
    huff_free(h, s);
    return fail(QOZ_EUNSUPPORTED, "a Huffman code longer than %d bits", kMaxCodeLen);
  }
  if (werr) {
    huff_free(h, s);
    return fail(QOZ_ECORRUPT, "the blob's histogram does not cover its codes");
  }
  h->fixed = hf;
  h->n_words = (long long)hf.n_words;
  if (h->n_words > 0 && !sizes_only) {
    e = dev_alloc((void**)&h->d_words, sizeof(uint32_t) * (size_t)h->n_words + 8, s);
    if (e != cudaSuccess) {
      huff_free(h, s);
      return fail(QOZ_ENOMEM, "entropy stream");
    }
    e = cudaMemsetAsync(h->d_words, 0, sizeof(uint32_t) * (size_t)h->n_words + 8, s);
    if (e == cudaSuccess) {
      const unsigned eg = (unsigned)((nch + kEncWarps - 1) / kEncWarps);
      auto enc = [&](auto lng, auto ck) {
        huff_encode_kernel<decltype(lng)::value, decltype(ck)::value>
            <<<eg, 32 * kEncWarps, 0, s>>>(b->d_codes, b->N, w->code, nch, offs, h->d_words);
      };
      auto by_chunk = [&](auto lng) {
        switch (h->chunk) {
          case 256: enc(lng, std::integral_constant<int, 256>()); break;
          case 512: enc(lng, std::integral_constant<int, 512>()); break;
          case 1024: enc(lng, std::integral_constant<int, 1024>()); break;
          case 2048: enc(lng, std::integral_constant<int, 2048>()); break;
          default: enc(lng, std::integral_constant<int, 4096>()); break;
        }
      };
      if (hf.max_len > 32)
        by_chunk(std::true_type());
      else
        by_chunk(std::false_type());
      note_launch(1);
      e = launch_check(cudaGetLastError());
    }
    if (e != cudaSuccess) {
      huff_free(h, s);
      return cuda_fail(e, "entropy encode");
    }
  }
  dev_free(h->d_work, s);
  h->d_work = nullptr;
  return QOZ_OK;
}

cudaError_t huff_decode(const void* d_section, const uint32_t* d_words, long long nchunks,
                        int chunk, unsigned n_sym, long long N, uint16_t* d_codes, int* d_err,
                        cudaStream_t s) {
  const int runs = entropy_runs(chunk);
  if (nchunks <= 0) return cudaSuccess;
  const HuffFixed* fx = static_cast<const HuffFixed*>(d_section);
  const uint16_t* syms =
      reinterpret_cast<const uint16_t*>(static_cast<const char*>(d_section) + sizeof(HuffFixed));
  const unsigned long long* offs = reinterpret_cast<const unsigned long long*>(
      static_cast<const char*>(d_section) + sizeof(HuffFixed) + pad8_bytes(sizeof(uint16_t) * kSymbols));
  // symbols held in shared memory: all of them up to kDecSmemSym, the first
  // kDecSmemSym otherwise; beside them the threads' word rings
  const unsigned nss = n_sym < (unsigned)kDecSmemSym ? n_sym : (unsigned)kDecSmemSym;
  constexpr size_t kRingBytes = sizeof(uint32_t) * kDecThreads * (kRingWords + 1);
  static unsigned long long attr_done = 0;
  cudaError_t e = ensure_smem_attr((const void*)huff_decode_kernel, &attr_done,
                                   kRingBytes + sizeof(uint16_t) * kDecSmemSym);
  if (e != cudaSuccess) return e;
  const uint16_t* sub = reinterpret_cast<const uint16_t*>(offs + (nchunks + 1));
  const unsigned grid = (unsigned)((nchunks * runs + kDecThreads - 1) / kDecThreads);
  huff_decode_kernel<<<grid, kDecThreads, kRingBytes + sizeof(uint16_t) * nss, s>>>(
      d_words, offs, sub, nchunks, chunk, runs, N, fx, syms, nss, d_codes, d_err);
  note_launch(1);
  return cudaGetLastError();
}

}  // namespace qoz

#ifdef QOZ_DEBUG_BOUNDS
namespace qoz {
// This translation unit's record of failed index checks (bounds-checking build).
unsigned long long bounds_take_entropy(bool reset) { return bounds_take(reset); }
}  // namespace qoz
#endif
