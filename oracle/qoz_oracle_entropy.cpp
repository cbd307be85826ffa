/*
 * QoZ oracle, entropy stage: canonical Huffman coding of the quantization
 * codes.
 *
 * TEST INFRASTRUCTURE ONLY (see qoz_oracle.h).  The paper's pipeline ends in
 * Huffman coding of the quantization bins followed by a dictionary coder
 * (Sec. 6.1 estimates the rate of exactly this stage).  It does not fix the
 * tie rule of the Huffman construction, the code order or the stream layout;
 * the readings taken here (this project's definitions) are:
 *
 *   - symbols: the 16-bit code of every point in field order, anchors
 *     included (they carry code 0);
 *   - Huffman construction: the symbols with a non-zero count, sorted by
 *     (count, symbol), form the leaf queue; merged nodes form a second queue
 *     in creation order; each pick takes the node-queue head when that queue
 *     is non-empty and its weight is strictly below the leaf-queue head's
 *     (or the leaf queue is empty), otherwise the leaf; a symbol's code
 *     length is its depth in the final tree, and a lone symbol gets length 1;
 *   - canonical codes: the assignment of RFC 1951 Sec. 3.2.2 (codes of one
 *     length are consecutive integers in symbol order, shorter lengths
 *     first);
 *   - stream: chunks of `chunk` symbols; each chunk starts on a fresh 32-bit
 *     word, its codes are written most significant bit first, and words fill
 *     from their most significant bit; the unused tail of a chunk's last word
 *     is zero; offs[c] is the word offset of chunk c (offs[n_chunks] = total);
 *   - sub-runs: a chunk of at least 1024 codes is cut into runs of 512, and
 *     the stream records the coded length of each run but the last, so that
 *     a decoder can start a thread at every run;
 *
 * Plain sequential code; the tree is built explicitly and walked for depths.
 */
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "qoz_oracle.h"

extern "C" {

int orc_huffman_lengths(const uint64_t* hist, int K, uint8_t* len) {
  std::memset(len, 0, (size_t)K);
  std::vector<std::pair<uint64_t, int>> leaves;
  for (int s = 0; s < K; ++s)
    if (hist[s] > 0) leaves.push_back({hist[s], s});
  if (leaves.empty()) return 0;
  if (leaves.size() == 1) {
    len[leaves[0].second] = 1;
    return 1;
  }
  std::sort(leaves.begin(), leaves.end());
  const int n = (int)leaves.size();
  // tree nodes: 0..n-1 leaves (sorted order), n.. merged nodes
  std::vector<uint64_t> w(2 * n - 1);
  std::vector<int> left(2 * n - 1, -1), right(2 * n - 1, -1);
  for (int i = 0; i < n; ++i) w[i] = leaves[i].first;
  int li = 0, ni = n, nn = n;  // leaf head, node head, next node id
  auto pick = [&]() {
    const bool node_ok = ni < nn;
    const bool leaf_ok = li < n;
    if (node_ok && (!leaf_ok || w[ni] < w[li])) return ni++;
    return li++;
  };
  while (nn < 2 * n - 1) {
    const int a = pick();
    const int b = pick();
    w[nn] = w[a] + w[b];
    left[nn] = a;
    right[nn] = b;
    ++nn;
  }
  // depths from the root (the last node) down
  std::vector<int> depth(2 * n - 1, 0);
  int maxlen = 0;
  for (int v = 2 * n - 2; v >= n; --v) {
    depth[left[v]] = depth[v] + 1;
    depth[right[v]] = depth[v] + 1;
  }
  for (int i = 0; i < n; ++i) {
    len[leaves[i].second] = (uint8_t)depth[i];
    maxlen = std::max(maxlen, depth[i]);
  }
  return maxlen;
}

void orc_canonical_codes(const uint8_t* len, int K, uint64_t* code) {
  int maxlen = 0;
  for (int s = 0; s < K; ++s) maxlen = std::max(maxlen, (int)len[s]);
  std::vector<uint64_t> bl_count(maxlen + 2, 0), next_code(maxlen + 2, 0);
  for (int s = 0; s < K; ++s)
    if (len[s]) bl_count[len[s]]++;
  uint64_t c = 0;
  for (int bits = 1; bits <= maxlen; ++bits) {
    c = (c + bl_count[bits - 1]) << 1;
    next_code[bits] = c;
  }
  for (int s = 0; s < K; ++s) {
    code[s] = 0;
    if (len[s]) code[s] = next_code[len[s]]++;
  }
}

int64_t orc_huffman_encode(const uint16_t* sym, int64_t n, int chunk, const uint8_t* len,
                           const uint64_t* code, uint64_t* offs, uint32_t* words,
                           int64_t cap_words) {
  const int64_t nchunks = (n + chunk - 1) / chunk;
  int64_t w = 0;
  for (int64_t c = 0; c < nchunks; ++c) {
    offs[c] = (uint64_t)w;
    int fill = 0;  // bits used in the current word
    bool open = false;
    const int64_t e = std::min(n, (c + 1) * chunk);
    for (int64_t i = c * chunk; i < e; ++i) {
      const int L = len[sym[i]];
      if (L == 0) return -1;  // symbol without a code
      for (int b = L - 1; b >= 0; --b) {  // most significant bit first
        if (!open) {
          if (w >= cap_words) return -2;
          words[w] = 0;
          open = true;
          fill = 0;
        }
        const uint32_t bit = (uint32_t)((code[sym[i]] >> b) & 1u);
        words[w] |= bit << (31 - fill);
        if (++fill == 32) {
          ++w;
          open = false;
        }
      }
    }
    if (open) ++w;
  }
  offs[nchunks] = (uint64_t)w;
  return w;
}

int orc_huffman_subruns(const uint16_t* sym, int64_t n, int chunk, const uint8_t* len,
                        uint16_t* sub) {
  const int S = chunk >= 1024 ? chunk / 512 : 1;
  if (S == 1) return 1;
  const int64_t nchunks = (n + chunk - 1) / chunk;
  for (int64_t c = 0; c < nchunks; ++c)
    for (int j = 0; j + 1 < S; ++j) {
      uint32_t bits = 0;
      for (int64_t i = c * chunk + (int64_t)j * 512; i < c * chunk + (int64_t)(j + 1) * 512 && i < n;
           ++i) {
        if (len[sym[i]] == 0) return -1;
        bits += len[sym[i]];
      }
      sub[c * (S - 1) + j] = (uint16_t)bits;  // at most 512 * 58 bits
    }
  return S;
}

int orc_huffman_decode(const uint32_t* words, const uint64_t* offs, int64_t n, int chunk,
                       const uint8_t* len, const uint64_t* code, int K, uint16_t* out) {
  std::map<std::pair<int, uint64_t>, int> table;  // (length, code) -> symbol
  int maxlen = 0;
  for (int s = 0; s < K; ++s)
    if (len[s]) {
      table[{(int)len[s], code[s]}] = s;
      maxlen = std::max(maxlen, (int)len[s]);
    }
  const int64_t nchunks = (n + chunk - 1) / chunk;
  for (int64_t c = 0; c < nchunks; ++c) {
    uint64_t bitpos = 0;
    const uint64_t nbits = (offs[c + 1] - offs[c]) * 32;
    const int64_t e = std::min(n, (c + 1) * chunk);
    for (int64_t i = c * chunk; i < e; ++i) {
      uint64_t v = 0;
      int L = 0;
      for (;;) {
        if (bitpos >= nbits || L >= maxlen) return 1;  // truncated or no such code
        const uint32_t wd = words[offs[c] + bitpos / 32];
        v = (v << 1) | ((wd >> (31 - bitpos % 32)) & 1u);
        ++bitpos;
        ++L;
        auto it = table.find({L, v});
        if (it != table.end()) {
          out[i] = (uint16_t)it->second;
          break;
        }
      }
    }
  }
  return 0;
}

}  // extern "C"
