"""Pins of the oracle's learned-tuner parts (features, network, Adam)
against closed forms and finite differences, on the CPU.

The features are this project's definition (the paper prints none), so the
pins are the mathematics of each feature on fields where it has a closed
form: linear fields (zero second differences, exact interpolation, exact
Lorenzo prediction, constant gradient), quadratics (known second
differences and interpolation residuals), and trilinear products (Lorenzo
residual equal to the mixed third difference)."""

import math

import numpy as np
import pytest

import oracle as orc

B_EDGE = 17   # one block of 17 points per axis: the whole field


def _one_block(shape):
    nd = len(shape)
    org = np.zeros((1, 3), dtype=np.int64)
    return org, tuple(shape[:nd])


def _feats(x, rel=1e-3, vrange=None):
    vr = float(x.max()) - float(x.min()) if vrange is None else vrange
    org, bd = _one_block(x.shape)
    return orc.features_blocks(x, rel, vr, org, bd), rel * vr


def test_linear_field_3d():
    n = (B_EDGE, 13, 11)
    i, j, k = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    a, b, c, d = 5.0, 2.0, -3.0, 1.0
    x = (a + b * i + c * j + d * k).astype(np.float32)
    f, e = _feats(x)
    assert f[0] == pytest.approx(-3.0)
    assert f[2] == 1.0
    assert f[3] == pytest.approx(math.log2(x.size) / 30)
    # population deviation of a linear field on a full grid
    var = sum(cf * cf * (m * m - 1) / 12.0 for cf, m in zip((b, c, d), n))
    vr = float(x.max()) - float(x.min())
    assert f[1] == pytest.approx(math.log10(vr / math.sqrt(var)), rel=1e-12)
    for s, cf in enumerate((b, c, d)):
        assert f[4 + s] == pytest.approx(math.log2(1 + abs(cf) / e), rel=1e-12)
        assert f[7 + s] == 0.0
    g = math.sqrt(b * b + c * c + d * d) / e
    gh = f[10:34]
    assert gh[min(23, max(0, math.floor(math.log2(g)) + 12))] == 1.0 and gh.sum() == 1.0
    lh = f[34:58]
    assert lh[0] == 1.0 and lh.sum() == 1.0          # Lorenzo exact on linear fields
    assert np.all(f[58:64] == 0.0)                    # both stencils exact to degree 1


def test_quadratic_along_x():
    n = (5, 6, 33)
    k = np.arange(n[2], dtype=np.float64)
    x = np.broadcast_to(k * k, n).astype(np.float32).copy()
    f, e = _feats(x)
    # first differences 2k+1, k = 0..n-2: mean n-1; second differences 2
    assert f[6] == pytest.approx(math.log2(1 + (n[2] - 1) / e), rel=1e-12)
    assert f[9] == pytest.approx(math.log2(1 + 2.0 / e), rel=1e-12)
    assert f[4] == 0.0 and f[5] == 0.0 and f[7] == 0.0 and f[8] == 0.0
    # linear interpolation misses a parabola by h^2 at every target; cubic is
    # exact; targets exist only along x (the other axes are too short for
    # h = 1 stencils, i - 3 >= 0 and i + 3 <= n - 1 need n >= 7)
    for jh, h in enumerate((1, 2, 4)):
        assert f[58 + jh] == pytest.approx(math.log2(1 + h * h / e), rel=1e-12)
        assert f[61 + jh] == 0.0


@pytest.mark.parametrize("nd", [2, 3])
def test_lorenzo_mixed_difference(nd):
    n = (9, 10, 11)[:nd] if nd == 3 else (12, 15)
    grids = np.meshgrid(*[np.arange(v, dtype=np.float64) for v in n], indexing="ij")
    x = np.prod(grids, axis=0).astype(np.float32)
    # the Lorenzo residual is the mixed backward difference: 1 everywhere
    f, e = _feats(x, rel=1e-2)
    lh = f[34:58]
    b = min(23, max(0, math.floor(math.log2(1.0 / e)) + 12))
    assert lh[b] == 1.0 and lh.sum() == 1.0
    if nd == 2:
        assert f[2] == pytest.approx(2 / 3) and f[6] == 0.0 and f[9] == 0.0


def test_constant_field_and_blocks():
    x = np.full((20, 20, 20), 3.5, dtype=np.float32)
    f, _ = _feats(x, vrange=0.0)
    assert f[1] == 0.0 and np.all(f[4:10] == 0.0)
    assert f[10] == 1.0 and f[34] == 1.0     # g = 0 and zero residual: bin 0
    # sampled features cover only the sampled blocks: a field that differs
    # outside them has the same features
    rng = np.random.default_rng(1)
    y = rng.normal(size=(200, 200, 200)).astype(np.float32)
    org, bd, _ = orc.sample_blocks(y.shape, 32, 0.005)
    mask = np.zeros(y.shape, bool)
    for o in org:
        mask[o[0]:o[0] + bd[0], o[1]:o[1] + bd[1], o[2]:o[2] + bd[2]] = True
    y2 = y.copy()
    y2[~mask] = 0.0
    f1 = orc.features(y, 1e-3, 10.0, 32, 0.005)
    f2 = orc.features(y2, 1e-3, 10.0, 32, 0.005)
    assert np.array_equal(f1[[0, 1, 2]], f2[[0, 1, 2]]) and np.array_equal(f1[4:], f2[4:])


def _net(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    P = rng.normal(0, scale, orc.NPARAM)
    mean = rng.normal(0, 1, orc.NFEAT)
    sd = rng.uniform(0.5, 2.0, orc.NFEAT)
    sd[5] = 0.0                       # a constant feature: std taken as 1
    return P, mean, sd


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 2, (B, orc.NFEAT))
    lab = np.stack([rng.integers(0, n, B) for _, n in orc.HEADS], axis=1).astype(np.int32)
    return X, lab


def test_zero_network_loss_closed_form():
    P = np.zeros(orc.NPARAM)
    X, lab = _batch(2, 7)
    loss, g = orc.mlp_loss_grad(P, np.zeros(64), np.ones(64), X, lab)
    assert loss == pytest.approx(math.log(2 * 6 * 5 * 3), rel=1e-14)
    # with zero hidden activations only the output bias has a gradient:
    # softmax (uniform) minus the label frequency
    b3 = g[-orc.NOUT:]
    for off, n in orc.HEADS:
        freq = np.bincount(lab[:, [o for o, _ in orc.HEADS].index(off)], minlength=n) / len(lab)
        assert np.allclose(b3[off:off + n], 1.0 / n - freq, atol=1e-15)
    assert np.all(g[:-orc.NOUT] == 0.0)


def test_gradient_finite_differences():
    P, mean, sd = _net(3)
    X, lab = _batch(4, 5)
    loss, g = orc.mlp_loss_grad(P, mean, sd, X, lab)
    rng = np.random.default_rng(5)
    # every parameter block: W1, b1, W2, b2, W3, b3
    bounds = np.cumsum([0, 128 * 64, 128, 128 * 128, 128, 16 * 128, 16])
    idx = np.concatenate([rng.integers(bounds[i], bounds[i + 1], 12) for i in range(6)])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (orc.mlp_loss_grad(Pp, mean, sd, X, lab, False)[0] -
              orc.mlp_loss_grad(Pm, mean, sd, X, lab, False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i
    # the softmax gradient of each head sums to zero over its logits
    b3 = g[-orc.NOUT:]
    for off, n in orc.HEADS:
        assert abs(b3[off:off + n].sum()) < 1e-14


def test_forward_matches_loss():
    P, mean, sd = _net(6)
    X, lab = _batch(7, 9)
    o = orc.mlp_forward(P, mean, sd, X)
    loss = 0.0
    for s in range(len(X)):
        for hd, (off, n) in enumerate(orc.HEADS):
            z = o[s, off:off + n]
            loss += np.log(np.exp(z - z.max()).sum()) + z.max() - z[lab[s, hd]]
    assert orc.mlp_loss_grad(P, mean, sd, X, lab, False)[0] == pytest.approx(loss / len(X),
                                                                             rel=1e-13)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(8)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    m, v = np.zeros(50), np.zeros(50)
    p0 = p.copy()
    orc.adam_step(p, g, m, v, 1, lr=0.01, eps=1e-8)
    # t = 1: bias-corrected moments are g and g^2
    assert np.allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def _one_path_net():
    """Weights with one nonzero per layer: feature 3 -> hidden-1 unit 5 ->
    hidden-2 unit 7 -> logit 10 (W1[5, 3] = 2, W2[7, 5] = 3, W3[10, 7] = 1,
    biases 0 except b3[4] = 0.5), normalisation mean 1, deviation 2 on
    feature 3.  Packing: W1 (128 x 64) row-major, b1, W2 (128 x 128), b2,
    W3 (16 x 128), b3."""
    P = np.zeros(orc.NPARAM)
    o_w1, o_b1 = 0, 128 * 64
    o_w2 = o_b1 + 128
    o_b2 = o_w2 + 128 * 128
    o_w3 = o_b2 + 128
    o_b3 = o_w3 + 16 * 128
    assert o_b3 + 16 == orc.NPARAM
    P[o_w1 + 5 * 64 + 3] = 2.0
    P[o_w2 + 7 * 128 + 5] = 3.0
    P[o_w3 + 10 * 128 + 7] = 1.0
    P[o_b3 + 4] = 0.5
    mean, sd = np.zeros(64), np.ones(64)
    mean[3], sd[3] = 1.0, 2.0
    return P, mean, sd


def test_forward_hand_worked_path():
    # f3 = 5: z3 = (5 - 1) / 2 = 2, h1[5] = relu(2 * 2) = 4, h2[7] = relu(3 * 4)
    # = 12, logit 10 = 12; logit 4 is its bias 0.5; the others 0.  f3 = -3:
    # z3 = -2, h1[5] = relu(-4) = 0, so only the bias remains.  Any other
    # feature has no path to the output.
    P, mean, sd = _one_path_net()
    X = np.zeros((3, 64))
    X[0, 3] = 5.0
    X[1, 3] = -3.0
    X[2, :] = 100.0
    X[2, 3] = 1.0          # z3 = 0: the other features alone
    out = orc.mlp_forward(P, mean, sd, X)
    want = np.zeros((3, 16))
    want[:, 4] = 0.5
    want[0, 10] = 12.0
    assert np.array_equal(out, want)


def test_adam_second_step_closed_form():
    # g1 = 1, g2 = -1 (Kingma and Ba, Algorithm 1, beta1 0.9, beta2 0.999):
    # m2 = 0.9 * 0.1 - 0.1 = -0.01, bias-corrected -0.01 / (1 - 0.81) = -1/19;
    # v2 = 0.999 * 0.001 + 0.001 = 0.001999, bias-corrected 0.001999 /
    # (1 - 0.998001) = 1.  So the second step moves the parameter by
    # +lr / 19 / (1 + eps).
    p = np.array([0.25])
    m, v = np.zeros(1), np.zeros(1)
    orc.adam_step(p, np.array([1.0]), m, v, 1, lr=0.01, eps=1e-8)
    p1 = p.copy()
    orc.adam_step(p, np.array([-1.0]), m, v, 2, lr=0.01, eps=1e-8)
    assert m[0] == pytest.approx(-0.01, rel=1e-12)
    assert v[0] == pytest.approx(0.001999, rel=1e-12)
    assert p[0] - p1[0] == pytest.approx(0.01 / 19 / (1 + 1e-8), rel=1e-10)
