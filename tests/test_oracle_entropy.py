"""Pins of the oracle's entropy stage (canonical Huffman coding of the
quantization codes) against values fixed outside it: a textbook Huffman
example, the canonical-code example of RFC 1951, Kraft's equality, the
optimal cost (itself pinned by brute force in test_oracle_metrics.py),
prefix-freeness, a hand-worked bit layout and round trips."""

import itertools

import numpy as np
import pytest

import oracle as orc


@pytest.fixture(scope="module", autouse=True)
def _built():
    orc.build()


def _hist(counts, K=16):
    h = np.zeros(K, dtype=np.uint64)
    for s, c in counts.items():
        h[s] = c
    return h


def test_clrs_example_lengths():
    # Cormen et al., Introduction to Algorithms, Sec. 16.3: frequencies
    # a..f = 45, 13, 12, 16, 9, 5 (thousands) give code lengths 1, 3, 3, 3,
    # 4, 4 and 224 (thousand) bits
    h = _hist({0: 45, 1: 13, 2: 12, 3: 16, 4: 9, 5: 5})
    ln, mx = orc.huffman_lengths(h)
    assert list(ln[:6]) == [1, 3, 3, 3, 4, 4] and mx == 4
    assert int(np.sum(ln.astype(np.int64) * h.astype(np.int64))) == 224


def test_rfc1951_canonical_codes():
    # RFC 1951 Sec. 3.2.2: lengths (3, 3, 3, 3, 3, 2, 4, 4) for A..H give the
    # codes 010, 011, 100, 101, 110, 00, 1110, 1111
    ln = np.array([3, 3, 3, 3, 3, 2, 4, 4], dtype=np.uint8)
    code = orc.canonical_codes(ln)
    assert [int(c) for c in code] == [0b010, 0b011, 0b100, 0b101, 0b110, 0b00, 0b1110, 0b1111]


def test_tie_rule():
    # three equal counts: leaves 0 and 1 merge first (the leaf wins ties
    # against the merged node), so symbol 2 ends up one level higher
    ln, _ = orc.huffman_lengths(_hist({0: 1, 1: 1, 2: 1}, K=3))
    assert list(ln) == [2, 2, 1]
    ln, _ = orc.huffman_lengths(_hist({3: 7, 9: 7, 1: 7, 4: 7}, K=10))
    assert [int(ln[s]) for s in (1, 3, 4, 9)] == [2, 2, 2, 2]


def test_single_and_empty():
    ln, mx = orc.huffman_lengths(_hist({5: 10}))
    assert mx == 1 and int(ln[5]) == 1 and int(ln.sum()) == 1
    ln, mx = orc.huffman_lengths(np.zeros(8, dtype=np.uint64))
    assert mx == 0 and int(ln.sum()) == 0


def _prefix_free(ln, code):
    used = [(int(ln[s]), int(code[s])) for s in range(ln.size) if ln[s]]
    for (la, ca), (lb, cb) in itertools.permutations(used, 2):
        if la <= lb and (cb >> (lb - la)) == ca:
            return False
    return True


@pytest.mark.parametrize("seed", range(12))
def test_kraft_optimality_prefix_free(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(2, 300))
    h = np.zeros(K, dtype=np.uint64)
    used = rng.choice(K, size=int(rng.integers(2, K + 1)), replace=False)
    # skewed counts, many ties among the small ones
    h[used] = np.maximum(1, rng.geometric(0.05, size=used.size) ** int(rng.integers(1, 3)))
    ln, mx = orc.huffman_lengths(h)
    assert np.all((ln > 0) == (h > 0))
    kraft = sum(2.0 ** -int(ln[s]) for s in range(K) if ln[s])
    assert kraft == pytest.approx(1.0, abs=1e-12)
    assert int(np.sum(ln.astype(np.int64) * h.astype(np.int64))) == orc.huffman_bits(h)
    code = orc.canonical_codes(ln)
    if K <= 120:
        assert _prefix_free(ln, code)
    # canonical order: codes of one length increase with the symbol, and
    # every code of a shorter length sorts before (as a left-aligned value)
    keys = sorted((int(ln[s]), s) for s in range(K) if ln[s])
    vals = [int(code[s]) << (mx - L) for L, s in keys]
    assert vals == sorted(vals) and len(set(vals)) == len(vals)


def test_bit_layout_hand_worked():
    # RFC 1951's table; symbols F, A, G, B in one chunk: 00 010 1110 011 ->
    # 0001 0111 0011 then zeros, MSB-first in the chunk's first word
    ln = np.array([3, 3, 3, 3, 3, 2, 4, 4], dtype=np.uint8)
    code = orc.canonical_codes(ln)
    words, offs = orc.huffman_encode(np.array([5, 0, 6, 1]), ln, code, chunk=4)
    assert list(offs) == [0, 1]
    assert [int(w) for w in words] == [0b0001_0111_0011 << 20]
    # two chunks of two symbols: each starts on its own word
    words, offs = orc.huffman_encode(np.array([5, 0, 6, 1]), ln, code, chunk=2)
    assert list(offs) == [0, 1, 2]
    assert [int(w) for w in words] == [0b00010 << 27, 0b1110011 << 25]


def test_word_boundary_crossing():
    # 33 one-bit codes in one chunk spill one bit into a second word
    h = np.zeros(2, dtype=np.uint64)
    h[:] = [5, 7]
    ln, _ = orc.huffman_lengths(h)
    code = orc.canonical_codes(ln)
    sym = np.array([1] * 33, dtype=np.uint16)  # symbol 1: the longer count, code 1
    words, offs = orc.huffman_encode(sym, ln, code, chunk=64)
    assert int(ln[1]) == 1 and int(code[1]) == 1
    assert list(offs) == [0, 2] and [int(w) for w in words] == [0xFFFFFFFF, 1 << 31]


@pytest.mark.parametrize("n,chunk,seed", [(0, 16, 0), (1, 16, 1), (100, 16, 2), (4097, 4096, 3),
                                          (20000, 333, 4), (5000, 4096, 5)])
def test_round_trip(n, chunk, seed):
    rng = np.random.default_rng(seed)
    sym = (32768 + np.round(rng.laplace(0, 3.0, size=n))).astype(np.uint16)
    if n > 10:
        sym[rng.integers(0, n, size=5)] = 0  # the unpredictable marker
    h = np.bincount(sym, minlength=65536).astype(np.uint64)
    ln, mx = orc.huffman_lengths(h)
    code = orc.canonical_codes(ln)
    words, offs = orc.huffman_encode(sym, ln, code, chunk=chunk)
    assert offs.size == (n + chunk - 1) // chunk + 1
    total = int(np.sum(ln[sym].astype(np.int64)))
    assert int(offs[-1]) >= (total + 31) // 32
    assert int(offs[-1]) <= (total + 31) // 32 + (offs.size - 1)
    out = orc.huffman_decode(words, offs, n, ln, code, chunk=chunk)
    assert np.array_equal(out, sym)


def test_chunk_size_rule(orc):
    """The writer's chunk size (this project's layout; the paper fixes
    none): the largest of 4096 .. 256 codes that still gives 8192 chunks,
    else 256; worked by hand at the sizes of the workloads (48^3, 256^3,
    512^3, 1024^3) and at the switch points."""
    assert orc.entropy_chunk(0) == 256
    assert orc.entropy_chunk(48 ** 3) == 256          # 432 chunks
    assert orc.entropy_chunk(256 * 8192) == 256       # exactly 8192 chunks of 256
    assert orc.entropy_chunk(512 * 8191) == 256       # 8191 chunks of 512: too few
    assert orc.entropy_chunk(512 * 8191 + 1) == 512   # 8192 chunks, the last one short
    assert orc.entropy_chunk(256 ** 3) == 2048        # 8192 chunks of 2048
    assert orc.entropy_chunk(512 ** 3) == 4096
    assert orc.entropy_chunk(1024 ** 3) == 4096
    # the default stream of a small symbol list is one chunk of the rule's size
    ln = np.array([1, 1], dtype=np.uint8)
    words, offs = orc.huffman_encode(np.array([0, 1, 1, 0] * 100, np.uint16), ln,
                                     orc.canonical_codes(ln))
    assert offs.size == 400 // 256 + 2 and offs[-1] == words.size


def test_subrun_table_hand_worked(orc):
    """Chunks of 1024 codes hold two runs of 512; the table records the first
    run's coded length.  Chunk 0: 512 codes of a 1-bit symbol, then 512 of a
    2-bit one; chunk 1 (476 codes, all 2-bit): its first run is the 476 codes
    there are, 952 bits."""
    ln = np.array([1, 2, 2], dtype=np.uint8)
    sym = np.array([0] * 512 + [1] * 512 + [2] * 476, dtype=np.uint16)
    assert orc.huffman_subruns(sym, ln, chunk=1024).tolist() == [512, 952]
    # chunks below 1024 codes carry no table
    assert orc.huffman_subruns(sym, ln, chunk=512).size == 0
    # four runs per chunk of 2048: three entries, the last two of the short
    # second chunk past its end (0 bits)
    sym2 = np.array([0] * 2048 + [1] * 600, dtype=np.uint16)
    assert orc.huffman_subruns(sym2, ln, chunk=2048).tolist() == [512, 512, 512, 1024, 176, 0]


def _decode_from(words, bitpos, count, ln, codes):
    """Plain prefix decoding of `count` codes from bit `bitpos` of the words
    (test side, independent of the oracle's decoder)."""
    table = {(int(ln[s]), int(codes[s])): s for s in range(ln.size) if ln[s]}
    out = []
    for _ in range(count):
        v, L = 0, 0
        while True:
            w = int(words[bitpos // 32])
            v = (v << 1) | ((w >> (31 - bitpos % 32)) & 1)
            bitpos += 1
            L += 1
            if (L, v) in table:
                out.append(table[(L, v)])
                break
            assert L < 64
    return out, bitpos


def test_subrun_table_starts_decode_their_runs(orc):
    """Every run starts at the bit the table says: decoding from the chunk
    start plus the preceding runs' lengths yields exactly that run's codes
    and ends where the next run starts (a skewed alphabet with long codes)."""
    rng = np.random.default_rng(17)
    n = 5000
    sym = np.minimum(rng.geometric(0.35, n) - 1, 40).astype(np.uint16)
    hist = np.bincount(sym, minlength=64).astype(np.uint64)
    ln, _ = orc.huffman_lengths(hist)
    cd = orc.canonical_codes(ln)
    chunk = 2048
    words, offs = orc.huffman_encode(sym, ln, cd, chunk=chunk)
    sub = orc.huffman_subruns(sym, ln, chunk=chunk)
    S = chunk // 512
    for c in range(offs.size - 1):
        start = 32 * int(offs[c])
        for j in range(S):
            b = c * chunk + j * 512
            cnt = max(0, min(512, n - b))
            got, end = _decode_from(words, start, cnt, ln, cd)
            assert got == sym[b:b + cnt].tolist()
            if j + 1 < S:
                assert end - start == int(sub[c * (S - 1) + j])
                start = end
