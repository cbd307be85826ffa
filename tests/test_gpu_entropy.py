"""GPU parity of the entropy stage: the code section of a serialized blob
(table and chunked stream) against the oracle's Huffman lengths, canonical
codes and encoding of the same codes, bit for bit; the GPU decoder on streams
the oracle wrote; round trips and corruption handling."""

import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HEADER = 160
FIXED = 288
CHUNK = 4096


# header fields (byte offsets): counts, checksum, code-section size
OFF_ANCHORS, OFF_CHECKSUM, OFF_CODE_BYTES = 120, 136, 144


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2310_14133_gb300 import build
    build.build()
    import paper_2310_14133_gb300 as q
    return q


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def pad8(v):
    return (v + 7) & ~7


def parse(buf):
    """Sections of a serialized stream (format 3) as numpy views."""
    b = bytes(buf.numpy()) if hasattr(buf, "numpy") else bytes(buf)
    n_anchors, n_unpred = struct.unpack_from("<qq", b, OFF_ANCHORS)
    off = HEADER + pad8(4 * n_anchors) + pad8(8 * n_unpred) + pad8(4 * n_unpred)
    n_sym, max_len, chunk, flags, n_chunks, n_words = struct.unpack_from("<IIIIQQ", b, off)
    bl = np.frombuffer(b, dtype=np.uint32, count=64, offset=off + 32)
    so = off + FIXED
    syms = np.frombuffer(b, dtype=np.uint16, count=n_sym, offset=so)
    oo = so + pad8(2 * n_sym)
    offs = np.frombuffer(b, dtype=np.uint64, count=n_chunks + 1, offset=oo)
    runs = chunk // 512 if chunk >= 1024 else 1
    ro = oo + 8 * (n_chunks + 1)
    sub = np.frombuffer(b, dtype=np.uint16, count=n_chunks * (runs - 1), offset=ro)
    wo = ro + pad8(2 * n_chunks * (runs - 1))
    words = np.frombuffer(b, dtype=np.uint32, count=n_words, offset=wo)
    return dict(code_off=off, n_sym=n_sym, max_len=max_len, chunk=chunk, flags=flags,
                n_chunks=n_chunks, n_words=n_words, bl=bl, syms=syms, offs=offs, sub=sub,
                sub_off=ro, words_off=wo, words=words, total=wo + pad8(4 * n_words))


def expected(orc, codes, chunk=None):
    """The oracle's table and stream for the codes of all points."""
    chunk = orc.entropy_chunk(codes.size) if chunk is None else chunk
    h = np.bincount(codes.ravel(), minlength=65536).astype(np.uint64)
    ln, mx = orc.huffman_lengths(h)
    cd = orc.canonical_codes(ln)
    words, offs = orc.huffman_encode(codes.ravel(), ln, cd, chunk=chunk)
    sub = orc.huffman_subruns(codes.ravel(), ln, chunk=chunk)
    used = np.nonzero(ln)[0]
    order = sorted(used, key=lambda s: (int(ln[s]), int(s)))
    bl = np.bincount(ln[used], minlength=64).astype(np.uint32)
    return dict(ln=ln, cd=cd, mx=mx, words=words, offs=offs, sub=sub,
                syms=np.array(order, np.uint16), bl=bl)


def check_section(orc, q, blob, buf):
    codes = blob.arrays()[0].cpu().numpy().view(np.uint16)
    sec = parse(buf)
    ref = expected(orc, codes)
    assert sec["chunk"] == orc.entropy_chunk(codes.size) and sec["flags"] == 0
    assert sec["n_sym"] == ref["syms"].size and sec["max_len"] == ref["mx"]
    assert np.array_equal(sec["bl"], ref["bl"]), "codes per length"
    assert np.array_equal(sec["syms"], ref["syms"]), "symbol order"
    assert np.array_equal(sec["offs"], ref["offs"]), "chunk word offsets"
    assert np.array_equal(sec["sub"], ref["sub"]), "run table"
    assert np.array_equal(sec["words"], ref["words"]), "stream words"
    assert sec["total"] == buf.numel()
    # the stream's length is exactly the sum of the code lengths, per chunk
    nbits = int(np.sum(ref["ln"][codes.ravel()].astype(np.int64)))
    assert sec["n_words"] >= (nbits + 31) // 32
    return sec, ref


CASES = [
    ((40, 50, 60), 1e-3, 8),
    ((33, 33, 33), 1e-4, 9),
    ((1, 300, 517), 1e-3, 10),   # 2D-like, ragged chunk tail
    ((7, 1, 9), 1e-2, 11),
    ((1, 1, 1), 1e-3, 12),       # one point: an anchor, one symbol
    ((64, 64, 64), 1e-2, 13),
    ((128, 256, 256), 1e-3, 14),  # chunks of 1024: two runs each
    ((201, 255, 333), 1e-4, 15),  # chunks of 2048: four runs, ragged tail
]


@pytest.mark.parametrize("shape,rel,seed", CASES)
def test_code_section_matches_oracle(q, orc, shape, rel, seed):
    import synth
    x = synth.grf(shape, 5.0 / 3.0, seed=seed, n_modes=48).cuda()
    blob = q.compress(x, rel)
    buf = blob.serialize()
    check_section(orc, q, blob, buf)
    b2 = q.deserialize(buf.clone())
    c1 = blob.arrays()[0].cpu().numpy()
    c2 = b2.arrays()[0].cpu().numpy()
    assert np.array_equal(c1, c2)
    out1, out2 = q.decompress(blob), q.decompress(b2)
    torch.cuda.synchronize()
    assert torch.equal(out1.view(torch.int32), out2.view(torch.int32))
    blob.free()
    b2.free()


def test_many_symbols_global_workspace(q, orc):
    # a tiny bound on noise: thousands of distinct codes (the table kernel's
    # global-memory path beyond 4096 used symbols)
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.standard_normal((48, 64, 80)).astype(np.float32)).cuda()
    blob = q.compress_abs(x, 1e-4, q.make_params(3))
    buf = blob.serialize()
    sec, _ = check_section(orc, q, blob, buf)
    assert sec["n_sym"] > 4096
    b2 = q.deserialize(buf.clone())
    assert torch.equal(b2.arrays()[0], blob.arrays()[0])
    blob.free()
    b2.free()


def _checksum(b):
    """The stream's checksum (sum of mixed 8-byte words, the field zero)."""
    def mix(z):
        z = (z + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))
    a = bytearray(b)
    a[OFF_CHECKSUM:OFF_CHECKSUM + 8] = bytes(8)
    a += bytes((-len(a)) % 8)
    w = np.frombuffer(bytes(a), dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(np.sum(mix(w ^ mix(np.arange(w.size, dtype=np.uint64))), dtype=np.uint64))


@pytest.mark.parametrize("chunk", [CHUNK, 2048, 512, 200])
def test_gpu_decodes_oracle_stream(q, orc, chunk):
    # replace the GPU's code section by one the oracle wrote (layout as
    # specified; a reader takes any chunk size that is a multiple of 8 up to
    # 4096), fix the checksum, and decode on the GPU
    import synth
    x = synth.grf((36, 40, 70), 5.0 / 3.0, seed=21, n_modes=48).cuda()
    blob = q.compress(x, 1e-3)
    buf = bytes(blob.serialize().numpy())
    codes = blob.arrays()[0].cpu().numpy().view(np.uint16)
    ref = expected(orc, codes, chunk)
    sec = parse(buf)
    fixed = struct.pack("<IIIIQQ", ref["syms"].size, ref["mx"], chunk, 0, ref["offs"].size - 1,
                        ref["words"].size) + ref["bl"].tobytes()
    body = fixed + ref["syms"].tobytes()
    body += bytes(pad8(len(body)) - len(body))
    body += ref["offs"].astype(np.uint64).tobytes()
    body += ref["sub"].astype(np.uint16).tobytes()
    body += bytes(pad8(len(body)) - len(body))
    body += ref["words"].tobytes()
    body += bytes(pad8(len(body)) - len(body))
    out = bytearray(buf[:sec["code_off"]]) + body
    struct.pack_into("<Q", out, OFF_CODE_BYTES, len(body))
    struct.pack_into("<Q", out, OFF_CHECKSUM, _checksum(bytes(out)))
    t = torch.frombuffer(bytearray(out), dtype=torch.uint8)
    b2 = q.deserialize(t)
    assert np.array_equal(b2.arrays()[0].cpu().numpy().view(np.uint16), codes)
    blob.free()
    b2.free()


def test_corrupt_code_sections(q):
    import synth
    x = synth.grf((30, 40, 50), 5.0 / 3.0, seed=3, n_modes=32).cuda()
    blob = q.compress(x, 1e-3)
    buf = blob.serialize()
    sec = parse(buf)
    raw = bytes(buf.numpy())

    def expect_corrupt(data):
        with pytest.raises(q.QozError) as ei:
            q.deserialize(torch.frombuffer(bytearray(data), dtype=torch.uint8))
        assert ei.value.status == 4

    # a flipped stream bit: caught by the checksum or the decoder
    b = bytearray(raw)
    b[sec["words_off"] + 5] ^= 0x40
    expect_corrupt(b)
    # an incomplete code (one length count changed)
    b = bytearray(raw)
    L = int(sec["max_len"])
    struct.pack_into("<I", b, sec["code_off"] + 32 + 4 * L, int(sec["bl"][L]) + 1)
    expect_corrupt(b)
    # offsets that run backwards
    b = bytearray(raw)
    oo = sec["code_off"] + FIXED + pad8(2 * sec["n_sym"])
    if sec["n_chunks"] >= 2:
        struct.pack_into("<Q", b, oo + 8, int(sec["offs"][2]) + 1)
        expect_corrupt(b)
    # truncated inside the stream words
    expect_corrupt(raw[: len(raw) - 12])
    # chunk sizes a reader does not take (checksum made valid, so the code
    # section's own check rejects them)
    for bad in (12, 8192, 0):
        b = bytearray(raw)
        struct.pack_into("<I", b, sec["code_off"] + 8, bad)
        struct.pack_into("<Q", b, OFF_CHECKSUM, _checksum(bytes(b)))
        expect_corrupt(b)
    blob.free()


def test_async_matches_sync_and_bound(q):
    import synth
    x = synth.grf((50, 60, 70), 5.0 / 3.0, seed=31, n_modes=32).cuda()
    blob = q.compress(x, 1e-3)
    ref = blob.serialize()
    bound = blob.serialize_bound()
    assert ref.numel() <= bound
    s = torch.cuda.Stream()
    out = torch.full((bound,), 0xAB, dtype=torch.uint8, pin_memory=True)
    used = blob.serialize_async(out, stream=s)
    s.synchronize()
    assert used == ref.numel() and torch.equal(out[:used], ref)
    # smaller than the raw 16-bit codes
    assert used < 2 * x.numel()
    blob.free()


def test_corrupt_run_table(q):
    """A run-table entry off by one (checksum made valid): the runs no longer
    meet where the table says, and the decoder reports the stream corrupt."""
    import synth
    x = synth.grf((128, 256, 256), 5.0 / 3.0, seed=5, n_modes=32).cuda()
    blob = q.compress(x, 1e-3)
    buf = blob.serialize()
    sec = parse(buf)
    assert sec["chunk"] == 1024 and sec["sub"].size == sec["n_chunks"]
    raw = bytearray(bytes(buf.numpy()))
    k = sec["sub_off"] + 2 * (sec["n_chunks"] // 2)
    struct.pack_into("<H", raw, k, struct.unpack_from("<H", raw, k)[0] + 1)
    struct.pack_into("<Q", raw, OFF_CHECKSUM, _checksum(bytes(raw)))
    with pytest.raises(q.QozError) as ei:
        q.deserialize(torch.frombuffer(raw, dtype=torch.uint8))
    assert ei.value.status == 4
    blob.free()

