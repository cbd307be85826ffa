"""The synthetic inputs follow their stated recipe: a Gaussian random field
whose shell-integrated spectrum falls as k^-p (fitted from a windowed FFT),
scaled to deviation 3, reproducible from its seed."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402


def _shell_slope(x, lo, hi):
    """Least-squares slope of log E(k) against log k over shells lo..hi, E the
    power of a Hann-windowed FFT summed over |k| in [q - 1/2, q + 1/2)."""
    n, d = x.shape[0], x.ndim
    w1 = np.hanning(n)
    w = w1
    for _ in range(d - 1):
        w = np.multiply.outer(w, w1)
    P = np.abs(np.fft.fftn((x - x.mean()) * w)) ** 2
    k = np.fft.fftfreq(n) * n
    K = np.sqrt(sum(np.meshgrid(*([k ** 2] * d), indexing="ij")))
    q = np.arange(lo, hi + 1)
    E = np.array([P[(K >= v - 0.5) & (K < v + 0.5)].sum() for v in q])
    return np.polyfit(np.log(q), np.log(E), 1)[0]


@pytest.mark.parametrize("shape,p,lo,hi", [((256, 256), 1.0, 4, 56), ((256, 256), 5 / 3, 4, 56),
                                           ((256, 256), 3.0, 4, 56),
                                           ((64, 64, 64), 5 / 3, 3, 14),
                                           ((64, 64, 64), 3.0, 3, 14)])
def test_spectrum_slope(shape, p, lo, hi):
    x = synth.grf(shape, p, seed=3, n_modes=4096).numpy().astype(np.float64)
    assert _shell_slope(x, lo, hi) == pytest.approx(-p, abs=0.2)


def test_deviation_and_seed():
    x = synth.grf((256, 256), 1.0, seed=3, n_modes=4096)
    assert float(x.double().std()) == pytest.approx(3.0, rel=0.05)
    assert x.dtype == torch.float32 and tuple(x.shape) == (256, 256)
    assert torch.equal(x, synth.grf((256, 256), 1.0, seed=3, n_modes=4096))
    assert not torch.equal(x, synth.grf((256, 256), 1.0, seed=4, n_modes=4096))


def test_trend_field_range():
    # the 64^3 k^-5/3 field plus its linear trend: values in about [-10, 10]
    x = synth.grf_trend_field(64)
    assert tuple(x.shape) == (64, 64, 64)
    assert -16.0 < float(x.min()) < -4.0 and 4.0 < float(x.max()) < 16.0
