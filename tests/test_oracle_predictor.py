"""Pins for the oracle's predictor and quantizer (Sec. 5), independent of the
oracle's own code: interpolation-error closed forms, the level structure of
Sec. 5.2.2, the error-bound contract of Sec. 3 and exact round trips."""

import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Eq. (ebl)

def test_level_bounds_golden(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "level_bounds.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for e, a, b, l, el in rows:
        got = orc.level_bounds(float(e), float(a), float(b), int(l))[int(l) - 1]
        assert got == pytest.approx(float(el), rel=1e-15)


def test_level_bounds_policy(orc):
    # Sec. 5.2.2 policy: e_l <= e, e_1 = e, e_l non-increasing in l
    for a in (1.0, 1.25, 1.5, 1.75, 2.0, 3.0):
        for b in (1.0, 1.5, 2.0, 3.0, 4.0):
            el = orc.level_bounds(0.37, a, b, 8)
            assert el[0] == 0.37
            assert np.all(el <= 0.37)
            assert np.all(np.diff(el) <= 0)
            # beta caps the reduction: e_l >= e / beta
            assert np.all(el >= 0.37 / b * (1 - 1e-15))


# ---------------------------------------------------------- level structure

def _coord_level(c, s):
    """Level at which a coordinate first appears: anchors (c % s == 0) are
    above every level; otherwise 1 + number of trailing zero bits."""
    if c % s == 0:
        return 10 ** 6
    lv = 1
    while c % 2 == 0:
        c //= 2
        lv += 1
    return lv


def _point_levels(shape, s):
    lv = np.full(shape, 10 ** 6, dtype=np.int64)
    for a, n in enumerate(shape):
        cl = np.array([_coord_level(c, s) for c in range(n)])
        sh = [1] * len(shape)
        sh[a] = n
        lv = np.minimum(lv, cl.reshape(sh))
    return lv


@pytest.mark.parametrize("shape,s", [((5, 5, 5), 4), ((9, 9, 9), 8), ((17, 17), 16),
                                     ((33, 17, 9), 32), ((64, 64, 64), 32), ((64, 64), 64),
                                     ((3, 70, 41), 32), ((1, 1, 7), 4)])
def test_every_point_once(orc, shape, s):
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape).astype(np.float32)
    p = orc.make_params(len(shape), interp=1, order=0, anchor_stride=s)
    r = orc.compress(x, 1e-2, p)
    lv = _point_levels(shape, s)
    L = int(np.log2(s))
    n_anchor = int(np.sum(lv > L))
    assert n_anchor == len(r["anchors"]) == orc.anchor_count(shape, s)
    for l in range(1, L + 1):
        assert r["cnt"][l - 1] == int(np.sum(lv == l)), l
    assert int(np.sum(r["cnt"])) + n_anchor == x.size


def test_level1_share():
    # Sec. 5.2.2: level 1 holds 87.5 % (3D) / 75 % (2D) of the points
    lv3 = _point_levels((64, 64, 64), 32)
    lv2 = _point_levels((64, 64), 64)
    assert int(np.sum(lv3 == 1)) == 229376 == 64 ** 3 * 7 // 8
    assert int(np.sum(lv2 == 1)) == 3072 == 64 ** 2 * 3 // 4


def test_level1_share_oracle(orc):
    x = np.zeros((64, 64, 64), np.float32)
    r = orc.compress(x, 0.1, orc.make_params(3))
    assert r["cnt"][0] == 229376
    x = np.zeros((64, 64), np.float32)
    r = orc.compress(x, 0.1, orc.make_params(2))
    assert r["cnt"][0] == 3072


def _pass_axis_targets(shape, s, order_axes_of_level, ax):
    """For each level l: boolean mask of the points of level l predicted along
    axis `ax` (the last axis of the level's order whose coordinate is at level
    l, all later axes being coarser)."""
    L = int(np.log2(s))
    nd = len(shape)
    coords = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    clv = [np.vectorize(lambda c: _coord_level(int(c), s))(coords[a]) for a in range(nd)]
    plv = np.minimum.reduce(clv)
    out = {}
    for l in range(1, L + 1):
        axes = order_axes_of_level(l)
        k = axes.index(ax)
        m = (plv == l) & (clv[ax] == l)
        for j in axes[k + 1:]:
            m &= clv[j] > l
        out[l] = m
    return out, coords


def _complete_homogeneous(m, pts):
    """h_m(pts): sum of all degree-m monomials in the points (h_0 = 1)."""
    if m < 0:
        return 0.0
    if m == 0:
        return 1.0
    import itertools
    return float(sum(np.prod(c) for c in itertools.combinations_with_replacement(pts, m)))


def _stencil_nodes(kind, c, n, h):
    """Node offsets of the stencil the reading of Sec. 5.2.2 uses at coordinate
    c (axis length n, half-stride h): cubic on -3h,-h,h,3h when all exist,
    quadratic on the three that exist around a missing outer node, linear on
    -h,h, linear extrapolation from -3h,-h without a right neighbour, else the
    left neighbour alone."""
    has_b1 = c + h < n
    has_a3 = c - 3 * h >= 0
    has_b3 = c + 3 * h < n
    if not has_b1:
        return [-3 * h, -h] if has_a3 else [-h]
    if kind == 1 and has_a3 and has_b3:
        return [-3 * h, -h, h, 3 * h]
    if kind == 1 and has_a3:
        return [-3 * h, -h, h]
    if kind == 1 and has_b3:
        return [-h, h, 3 * h]
    return [-h, h]


def _closed_form_residual(kind, c, n, h, deg):
    """g(c) - pred for g(t) = t**deg, from the error of polynomial
    interpolation on nodes T: g[T, c] * prod(c - t), where the divided
    difference of t**deg over the k+2 points T + {c} is the complete
    homogeneous polynomial h_(deg-k-1) of those points."""
    nodes = [c + o for o in _stencil_nodes(kind, c, n, h)]
    k = len(nodes) - 1
    dd = _complete_homogeneous(deg - k - 1, nodes + [c])
    return dd * float(np.prod([c - t for t in nodes]))


@pytest.mark.parametrize("nd,shape,s,ax,kind,deg,order", [
    (3, (5, 9, 33), 32, 2, 0, 2, 0),
    (3, (5, 9, 33), 32, 2, 1, 3, 0),
    (3, (17, 6, 7), 16, 0, 1, 4, 3),
    (3, (17, 6, 7), 16, 0, 1, 3, 5),
    (3, (7, 29, 5), 8, 1, 0, 2, 2),
    (3, (7, 29, 5), 8, 1, 1, 3, 4),
    (2, (30, 11), 16, 0, 1, 3, 1),
    (2, (9, 40), 32, 1, 0, 2, 0),
    (2, (9, 17), 16, 1, 1, 4, 1),
])
def test_stencils_against_interpolation_error(orc, nd, shape, s, ax, kind, deg, order):
    """e = 0 keeps every reconstruction equal to the input (exact predictions
    quantize to bin 0, the rest are stored verbatim), so each residual is the
    interpolation error of g(t) = t^deg along the pass axis.  Points whose
    pass axis is another axis see a constant and must be exact."""
    n = shape[ax]
    g = np.arange(n, dtype=np.float64) ** deg
    sh = [1] * nd
    sh[ax] = n
    x = np.broadcast_to(g.reshape(sh), shape).astype(np.float32).copy()
    p = orc.make_params(nd, interp=kind, order=order, anchor_stride=s)
    r = orc.compress(x, 0.0, p)
    assert np.array_equal(r["recon"], x)
    axes_of = lambda l: list(orc.order_axes(nd, order))
    masks, coords = _pass_axis_targets(shape, s, axes_of, ax)
    expect_nonzero = np.zeros(shape, dtype=bool)
    for l, m in masks.items():
        h = 2 ** (l - 1)
        res = np.array([_closed_form_residual(kind, int(c), n, h, deg) for c in coords[ax][m]])
        assert r["l1"][l - 1] == pytest.approx(float(np.sum(np.abs(res))), rel=1e-12, abs=1e-9)
        expect_nonzero[m] = res != 0
    unpred = np.zeros(x.size, dtype=bool)
    unpred[r["unpred_idx"]] = True
    assert np.array_equal(unpred.reshape(shape), expect_nonzero)
    lv = _point_levels(shape, s)
    predicted = (lv <= int(np.log2(s))) & ~expect_nonzero
    assert np.all(r["codes"][predicted] == 32768)


@pytest.mark.parametrize("order", range(6))
@pytest.mark.parametrize("kind", [0, 1])
def test_integer_linear_field_exact(orc, order, kind):
    # every stencil except the lone-left-neighbour one reproduces degree-1
    # polynomials; that one only occurs along axes no longer than the anchor
    # stride, so with all axes longer than 32 every code is the zero bin
    z, y, x = np.meshgrid(np.arange(37), np.arange(33), np.arange(45), indexing="ij")
    f = (7 + 3 * z - 2 * y + 5 * x).astype(np.float32)
    p = orc.make_params(3, interp=kind, order=order, alpha=1.5, beta=4.0)
    r = orc.compress(f, 0.01, p)
    lv = _point_levels(f.shape, 32)
    assert np.all(r["codes"][lv <= 5] == 32768)
    assert np.all(r["codes"][lv > 5] == 0)
    assert len(r["unpred_idx"]) == 0
    assert np.array_equal(r["recon"], f)


def test_cubic_field_interior_exact(orc):
    # a sum of per-axis cubics: the 4-point stencil is exact (Sec. 5.2.2
    # cubic spline interpolation; error term vanishes for degree <= 3)
    z, y, x = np.meshgrid(np.arange(40), np.arange(40), np.arange(40), indexing="ij")
    f = (z ** 3 - 4 * y ** 3 + 2 * x ** 3 + x * x).astype(np.float64)
    f32 = (f / 64.0).astype(np.float32)
    p = orc.make_params(3, interp=1, order=0, anchor_stride=32)
    r = orc.compress(f32, 0.0, p)
    assert np.array_equal(r["recon"], f32)
    # points whose pass stencil has all four nodes are exact (code = zero bin)
    lv = _point_levels(f32.shape, 32)
    axes = list(orc.order_axes(3, 0))
    n = 40
    full = np.zeros(f32.shape, bool)
    for ax in range(3):
        masks, coords = _pass_axis_targets(f32.shape, 32, lambda l: axes, ax)
        for l, m in masks.items():
            h = 2 ** (l - 1)
            c = coords[ax]
            full |= m & (c - 3 * h >= 0) & (c + 3 * h < n)
    assert full.sum() > 0.7 * (lv <= 5).sum()
    assert np.all(r["codes"][full] == 32768)


# ------------------------------------------------------------------ quantizer

def test_quantizer_bins_and_ties(orc):
    """One level (anchor stride 2), 2D field (1, n): odd points are predicted
    from exact even neighbours equal to 0, so the residual is the value
    itself.  e = 0.5 makes the bin width 1: the bin index is the residual
    rounded half away from zero; |q| must stay below 32768."""
    vals = [0.25, 0.5, -0.5, 1.49, 2.5, -2.5, 7.0, 32767.4, 32767.5, -32767.5, 1.0e5,
            float("nan"), float("inf")]
    expect_q = [0, 1, -1, 1, 3, -3, 7, 32767, None, None, None, None, None]
    n = 2 * len(vals) + 1
    x = np.zeros((1, n), np.float32)
    x[0, 1::2] = vals
    p = orc.make_params(2, interp=0, order=1, anchor_stride=2)
    r = orc.compress(x, 0.5, p)
    for i, q in enumerate(expect_q):
        c = int(r["codes"][0, 2 * i + 1])
        if q is None:
            assert c == 0
            assert (2 * i + 1) in set(r["unpred_idx"].tolist())
        else:
            assert c == q + 32768
            assert abs(float(x[0, 2 * i + 1]) - float(r["recon"][0, 2 * i + 1])) <= 0.5
    assert len(r["unpred_idx"]) == sum(q is None for q in expect_q)
    # unpredictable values come back verbatim, sorted by index
    assert np.all(np.diff(r["unpred_idx"]) > 0)
    got = r["unpred_val"]
    want = x.reshape(-1)[r["unpred_idx"]]
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_zero_bound_constant_field(orc):
    # vrange = 0 -> e = 0: exact predictions stay predictable
    x = np.full((9, 10, 11), 3.25, np.float32)
    r = orc.compress(x, 0.0, orc.make_params(3))
    assert len(r["unpred_idx"]) == 0
    assert np.array_equal(r["recon"], x)


# ------------------------------------------------- error bound (Sec. 3) + round trip

@pytest.mark.parametrize("seed", range(4))
def test_error_bound_and_round_trip(orc, seed):
    rng = np.random.default_rng(seed)
    nd = 3 if seed % 2 == 0 else 2
    shape = tuple(int(v) for v in rng.integers(20, 70, size=nd))
    x = np.cumsum(rng.standard_normal(shape), axis=-1).astype(np.float32)
    x *= np.float32(10.0 ** rng.uniform(-2, 4))
    mn, mx, _ = orc.value_range(x)
    e = float(10.0 ** rng.uniform(-5, -1)) * (float(mx) - float(mn))
    ords = rng.integers(0, 6 if nd == 3 else 2, size=8).tolist()
    kinds = rng.integers(0, 2, size=8).tolist()
    p = orc.make_params(nd, interp=kinds, order=ords, alpha=float(rng.choice([1, 1.25, 2])),
                        beta=float(rng.choice([1.5, 3, 4])))
    r = orc.compress(x, e, p)
    err = np.abs(x.astype(np.float64) - r["recon"].astype(np.float64))
    assert err.max() <= e
    L = int(np.log2(p.anchor_stride))
    el = orc.level_bounds(e, p.alpha, p.beta, L)
    lv = _point_levels(shape, p.anchor_stride)
    for l in range(1, L + 1):
        if np.any(lv == l):
            assert err[lv == l].max() <= np.float32(el[l - 1])
    y = orc.decompress(r["codes"], e, p, r["anchors"], r["unpred_idx"], r["unpred_val"])
    assert np.array_equal(y.view(np.uint32), r["recon"].view(np.uint32))


def test_nonfinite_points_unpredictable(orc):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((20, 21, 22)).astype(np.float32)
    x[3, 4, 5] = np.nan
    x[10, 11, 13] = np.inf
    x[0, 0, 1] = -np.inf
    mn, mx, cnt = orc.value_range(x)
    assert cnt == x.size - 3 and np.isfinite(mn) and np.isfinite(mx)
    p = orc.make_params(3)
    e = 1e-3 * (float(mx) - float(mn))
    r = orc.compress(x, e, p)
    idx = set(r["unpred_idx"].tolist())
    for pt in [(3, 4, 5), (10, 11, 13), (0, 0, 1)]:
        assert np.ravel_multi_index(pt, x.shape) in idx
    y = orc.decompress(r["codes"], e, p, r["anchors"], r["unpred_idx"], r["unpred_val"])
    assert np.array_equal(y.view(np.uint32), r["recon"].view(np.uint32))
    fin = np.isfinite(x)
    assert np.all(np.abs(x[fin].astype(np.float64) - y[fin]) <= e)


def test_value_range_finite_values_only(orc):
    # Sec. 7.1.4's value range is over the finite values: min and max equal
    # numpy's over the finite subset wherever the non-finite values sit
    # (first, last, between), and a field with none gives 0, 0 and count 0
    rng = np.random.default_rng(9)
    x = rng.standard_normal(1000).astype(np.float32)
    for pos in (0, 999, 500):
        y = x.copy()
        y[pos] = np.nan
        y[(pos + 7) % 1000] = -np.inf
        y[(pos + 13) % 1000] = np.inf
        fin = np.isfinite(y)
        mn, mx, cnt = orc.value_range(y)
        assert cnt == 997 and mn == y[fin].min() and mx == y[fin].max()
    mn, mx, cnt = orc.value_range(np.full(16, np.nan, np.float32))
    assert (mn, mx, cnt) == (0.0, 0.0, 0)
    mn, mx, cnt = orc.value_range(np.array([np.inf, 2.5, -np.inf], np.float32))
    assert (mn, mx, cnt) == (2.5, 2.5, 1)
