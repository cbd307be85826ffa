"""Pins for the oracle's metrics (Sec. 3: PSNR Eq. (psnr), SSIM Eq. (ssim),
Eq. (ssim2), the error autocorrelation Eq. (ac)) and rate estimate (Sec. 6.1:
Huffman coding of the pooled quantization bins), against closed forms, a
library SSIM and brute force."""

import itertools
import math

import numpy as np
import pytest
from scipy import ndimage


def test_identity(orc):
    rng = np.random.default_rng(1)
    a = rng.standard_normal((12, 13, 14)).astype(np.float32)
    assert orc.max_abs_err(a, a) == 0.0
    assert orc.psnr(a, a, 5.0) == math.inf
    m, nw, s = orc.ssim(a, a, 5.0)
    assert nw == 3 * 4 * 4
    assert m == pytest.approx(1.0, abs=1e-14)


def test_constant_error_psnr(orc):
    rng = np.random.default_rng(2)
    a = rng.uniform(-10, 10, (40, 50)).astype(np.float32)
    delta = np.float32(0.125)
    b = a + delta  # exact for these magnitudes? not always; use exact differences
    d = b.astype(np.float64) - a.astype(np.float64)
    vr = 20.0
    mse = float(np.mean(d * d))
    assert orc.mse(a, b) == pytest.approx(mse, rel=1e-12)
    # dyadic values keep a + delta exact, so the closed form holds exactly
    a2 = (np.round(a * 8) / 8).astype(np.float32)
    b2 = (a2 + delta).astype(np.float32)
    assert orc.max_abs_err(a2, b2) == 0.125
    assert orc.psnr(a2, b2, vr) == pytest.approx(20 * math.log10(vr / 0.125), rel=1e-13)


def _ssim_library(a, b, vr, win, step):
    """Textbook SSIM from scipy's box filter: local statistics at every window
    centre, then the windows that start at multiples of `step` and lie fully
    inside are averaged."""
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    c1 = (0.01 * vr) ** 2
    c2 = (0.03 * vr) ** 2
    f = lambda v: ndimage.uniform_filter(v, size=win, mode="constant")
    mx, my = f(a), f(b)
    vx = f(a * a) - mx * mx
    vy = f(b * b) - my * my
    cxy = f(a * b) - mx * my
    s = ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    half = win // 2
    sl = tuple(slice(half, n - half, step) for n in a.shape)
    return float(np.mean(s[sl])), int(s[sl].size)


@pytest.mark.parametrize("shape,win,step", [((30, 31, 29), 7, 2), ((64, 70), 7, 2),
                                            ((20, 21, 22), 5, 3), ((17, 40), 7, 1)])
def test_ssim_matches_library(orc, shape, win, step):
    rng = np.random.default_rng(3)
    a = np.cumsum(rng.standard_normal(shape), axis=0).astype(np.float32)
    b = (a + rng.normal(0, 0.3, shape)).astype(np.float32)
    vr = float(a.max()) - float(a.min())
    want, nw = _ssim_library(a, b, vr, win, step)
    got, nw2, _ = orc.ssim(a, b, vr, win, step)
    assert nw2 == nw
    assert got == pytest.approx(want, rel=1e-9)


def test_ssim_constant_shift_closed_form(orc):
    # X' = X + c: equal variances and covariance = variance, so each window's
    # SSIM is (2 mu (mu + c) + c1) / (mu^2 + (mu + c)^2 + c1)
    rng = np.random.default_rng(4)
    a = (np.round(rng.uniform(-4, 4, (21, 22, 23)) * 16) / 16).astype(np.float32)
    c = 0.5
    b = (a + np.float32(c)).astype(np.float32)
    vr = 8.0
    c1 = (0.01 * vr) ** 2
    vals = []
    for i in range(0, 21 - 6, 2):
        for j in range(0, 22 - 6, 2):
            for k in range(0, 23 - 6, 2):
                mu = float(np.mean(a[i:i + 7, j:j + 7, k:k + 7].astype(np.float64)))
                vals.append((2 * mu * (mu + c) + c1) / (mu * mu + (mu + c) ** 2 + c1))
    got, nw, _ = orc.ssim(a, b, vr)
    assert nw == len(vals)
    assert got == pytest.approx(float(np.mean(vals)), rel=1e-10)


# --------------------------------------------------------------- Huffman

def _brute_force_prefix_cost(counts):
    """Minimum of sum(count * length) over all length vectors that satisfy
    Kraft's inequality (a prefix code exists iff sum 2^-len <= 1)."""
    k = len(counts)
    if k == 1:
        return counts[0]
    best = None
    for lens in itertools.product(range(1, k), repeat=k):
        if sum(2.0 ** -l for l in lens) <= 1.0 + 1e-12:
            c = sum(a * l for a, l in zip(counts, lens))
            best = c if best is None else min(best, c)
    return best


def test_huffman_small_known(orc):
    h = np.zeros(65536, np.uint64)
    h[[5, 9, 100, 40000]] = [1, 1, 2, 4]          # lengths 3,3,2,1
    assert orc.huffman_bits(h) == 14
    h = np.zeros(65536, np.uint64)
    h[32768] = 1000                                # one symbol: 1 bit each
    assert orc.huffman_bits(h) == 1000
    assert orc.huffman_bits(np.zeros(65536, np.uint64)) == 0


@pytest.mark.parametrize("seed", range(12))
def test_huffman_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 8))
    counts = [int(v) for v in rng.integers(1, 1000, size=k)]
    if seed % 3 == 0:
        counts = [int(2 ** i) for i in range(k)]     # skewed (deep) case
    h = np.zeros(65536, np.uint64)
    pos = rng.choice(65536, size=k, replace=False)
    h[pos] = counts
    assert orc.huffman_bits(h) == _brute_force_prefix_cost(counts)


def test_estimate_bits_and_histogram(orc):
    rng = np.random.default_rng(6)
    x = np.cumsum(rng.standard_normal((40, 41, 42)), axis=2).astype(np.float32)
    p = orc.make_params(3, interp=1, order=0, alpha=1.5, beta=4)
    r = orc.compress(x, 0.05, p)
    h = orc.histogram(r["codes"], 32)
    na = len(r["anchors"])
    assert int(h.sum()) == x.size - na
    # anchors are excluded; every non-anchor point lands in its code's bin
    lv_anchor = np.zeros(x.shape, bool)
    lv_anchor[::32, ::32, ::32] = True
    want = np.bincount(r["codes"][~lv_anchor].ravel(), minlength=65536)
    assert np.array_equal(h, want.astype(np.uint64))
    nu = len(r["unpred_idx"])
    assert orc.estimate_bits(h, nu, na) == orc.huffman_bits(h) + 32 * nu + 32 * na


# ---- Eq. (ac): autocorrelation of the compression errors

def _ac_pair(e):
    """Original zeros and reconstruction e: the errors are e exactly."""
    e = np.asarray(e, dtype=np.float32)
    return np.zeros_like(e), e


def test_ac_alternating_errors(orc):
    # e_i = (-1)^i: mean 0, variance 1, every lag-1 product -1 and every
    # lag-2 product +1, so AC(1) = -1 and AC(2) = 1 exactly
    a, b = _ac_pair([(-1.0) ** i for i in range(1000)])
    assert orc.autocorr(a, b, 1) == -1.0
    assert orc.autocorr(a, b, 2) == 1.0


@pytest.mark.parametrize("period,k", [(8, 1), (8, 2), (10, 3), (16, 4)])
def test_ac_cosine_closed_form(orc, period, k):
    # e_i = cos(w i) over whole periods: AC(k) = cos(w k) + O(1 / ((N - k) sin w))
    n = 100000 - 100000 % period
    w = 2.0 * np.pi / period
    a, b = _ac_pair(np.cos(w * np.arange(n)))
    assert orc.autocorr(a, b, k) == pytest.approx(np.cos(w * k), abs=2e-4)


def test_ac_ar1_process(orc):
    # e_i = phi e_{i-1} + white noise: AC(k) -> phi^k
    rng = np.random.default_rng(3)
    phi, n = 0.6, 400000
    eta = rng.standard_normal(n)
    e = np.empty(n)
    e[0] = eta[0]
    for i in range(1, n):
        e[i] = phi * e[i - 1] + eta[i]
    a, b = _ac_pair(e)
    assert orc.autocorr(a, b, 1) == pytest.approx(phi, abs=0.01)
    assert orc.autocorr(a, b, 2) == pytest.approx(phi ** 2, abs=0.01)


def test_ac_affine_invariance_and_degenerate(orc):
    rng = np.random.default_rng(4)
    e = rng.standard_normal(5000).astype(np.float32)
    a, b = _ac_pair(e)
    a2, b2 = _ac_pair(2.0 * e.astype(np.float64) + 3.0)
    assert orc.autocorr(a2, b2, 1) == pytest.approx(orc.autocorr(a, b, 1), abs=1e-6)
    # the sign convention of the error does not matter
    assert orc.autocorr(b, a, 1) == pytest.approx(orc.autocorr(a, b, 1), abs=1e-12)
    # constant error (zero variance) and lags past the end give 0
    a, b = _ac_pair(np.full(100, 0.25))
    assert orc.autocorr(a, b, 1) == 0.0
    a, b = _ac_pair([1.0, -1.0, 2.0])
    assert orc.autocorr(a, b, 3) == 0.0


def test_ac_blocks_pairs_stay_inside(orc):
    # one block is the plain definition
    rng = np.random.default_rng(5)
    e = rng.standard_normal(777)
    a, b = _ac_pair(e)
    assert orc.autocorr_blocks(e.astype(np.float32).astype(np.float64), [777], 1) == \
        pytest.approx(orc.autocorr(a, b, 1), abs=1e-12)
    # blocks [1, 1, 1, 1] and [-1, -1, -1, -1]: mean 0, variance 1; every pair
    # inside a block gives +1, the one pair across the boundary (-1) is not
    # counted, so AC = 1 exactly
    assert orc.autocorr_blocks([1, 1, 1, 1, -1, -1, -1, -1], [4, 4], 1) == 1.0
    # the same errors as one block: 6 pairs of +1 and one of -1 -> 5/7
    assert orc.autocorr_blocks([1, 1, 1, 1, -1, -1, -1, -1], [8], 1) == pytest.approx(5.0 / 7.0)
