"""Field generators (see the package docstring)."""

from __future__ import annotations

import math

import numpy as np
import torch


def _unit_vectors(rng: np.random.Generator, m: int, d: int) -> np.ndarray:
    v = rng.standard_normal((m, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def _coords(n: int, device) -> torch.Tensor:
    return torch.arange(n, device=device, dtype=torch.float64)


def grf(dims, slope: float, seed: int, n_modes: int | None = None, sigma: float = 3.0,
        device="cpu", chunk_points: int = 1 << 24) -> torch.Tensor:
    """Gaussian random field (sum of random Fourier modes), float32, dims
    slowest-first (2D or 3D)."""
    dims = tuple(int(d) for d in dims)
    d = len(dims)
    assert d in (2, 3)
    m = n_modes or (512 if d == 3 else 256)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_ref = min(dims)
    kmax = max(n_ref / 4.0, 1.0)
    direc = _unit_vectors(rng, m, d)
    kmag = np.exp(rng.uniform(0.0, math.log(kmax), size=m)) if kmax > 1 else np.ones(m)
    kvec = direc * kmag[:, None]                      # cycles per n_ref cells
    phase = rng.uniform(0.0, 2.0 * math.pi, size=m)
    amp = kmag ** ((1.0 - slope) / 2.0)
    norm = math.sqrt(float(np.sum(amp * amp)) / 2.0)

    dev = torch.device(device)
    kv = torch.tensor(kvec, dtype=torch.float64, device=dev)
    ph = torch.tensor(phase, dtype=torch.float64, device=dev)
    am = torch.tensor(amp / norm * sigma, dtype=torch.float64, device=dev)
    # per-axis complex exponentials exp(i 2 pi k_a r_a / n_ref), computed in
    # float64 and reduced modulo 2 pi before the cast
    def axis_exp(a):
        r = _coords(dims[a], dev)
        t = torch.remainder(kv[:, a:a + 1] * r[None, :] / n_ref, 1.0) * (2.0 * math.pi)
        return torch.polar(torch.ones_like(t), t)    # complex128 [m, n_a]

    out = torch.empty(dims, dtype=torch.float32, device=dev)
    e_last = axis_exp(d - 1)                          # [m, nx]
    lhs_r = torch.cat([e_last.real, e_last.imag], 0).to(torch.float32)  # [2m, nx]
    w0 = am * torch.polar(torch.ones_like(ph), ph)    # complex128 [m]
    if d == 2:
        e0 = axis_exp(0)                              # [m, ny]
        w = w0[:, None] * e0                          # [m, ny]
        wr = torch.cat([w.real, -w.imag], 0).to(torch.float32)  # [2m, ny]
        out.copy_(wr.t() @ lhs_r)
        return out
    e0 = axis_exp(0)
    e1 = axis_exp(1)
    zc = max(1, chunk_points // max(1, dims[1] * dims[2]))
    for z0 in range(0, dims[0], zc):
        z1 = min(dims[0], z0 + zc)
        w = (w0[:, None, None] * e0[:, z0:z1, None] * e1[:, None, :])  # [m, zc, ny]
        w = w.reshape(m, -1)
        wr = torch.cat([w.real, -w.imag], 0).to(torch.float32)      # [2m, zc*ny]
        out[z0:z1].copy_((wr.t() @ lhs_r).reshape(z1 - z0, dims[1], dims[2]))
    return out


def linear_trend(dims, device="cpu") -> torch.Tensor:
    """2 * sum_a (r_a / n_a) - 3, the trend added to the 64^3 field."""
    dims = tuple(int(d) for d in dims)
    dev = torch.device(device)
    out = torch.zeros(dims, dtype=torch.float64, device=dev)
    for a, n in enumerate(dims):
        shape = [1] * len(dims)
        shape[a] = n
        out = out + (_coords(n, dev) / n).reshape(shape)
    return (2.0 * out - 3.0).to(torch.float32)


def fronts(dims, seed_base: int = 2000, count: int = 8, amp: float = 3.0,
           width: float = 2.0, device="cpu", chunk_points: int = 1 << 24) -> torch.Tensor:
    """Sum of `count` sharp fronts a_j tanh((n_j . r - c_j) / width) at random
    planes; front j draws from seed seed_base + j."""
    dims = tuple(int(d) for d in dims)
    d = len(dims)
    dev = torch.device(device)
    out = torch.zeros(dims, dtype=torch.float32, device=dev)
    params = []
    for j in range(count):
        rng = np.random.Generator(np.random.PCG64(seed_base + j))
        nrm = _unit_vectors(rng, 1, d)[0]
        p = rng.uniform(0.0, 1.0, size=d) * np.array(dims)
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        params.append((nrm, float(nrm @ p), sign * amp))
    plane = dims[1] * dims[2] if d == 3 else dims[1]
    zc = max(1, chunk_points // plane)
    for z0 in range(0, dims[0], zc):
        z1 = min(dims[0], z0 + zc)
        acc = torch.zeros((z1 - z0,) + dims[1:], dtype=torch.float64, device=dev)
        for nrm, c, a in params:
            s = torch.zeros_like(acc)
            for ax in range(d):
                n_ax = (z1 - z0) if ax == 0 else dims[ax]
                r = _coords(n_ax, dev) + (z0 if ax == 0 else 0)
                shape = [1] * d
                shape[ax] = n_ax
                s = s + nrm[ax] * r.reshape(shape)
            acc = acc + a * torch.tanh((s - c) / width)
        out[z0:z1] = acc.to(torch.float32)
    return out


def zonal_bands(ny: int, nx: int, seed: int, device="cpu") -> torch.Tensor:
    """Smooth zonal (row-dependent) bands sum_j a_j cos(2 pi j row / ny + psi_j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    psi = rng.uniform(0.0, 2.0 * math.pi, size=8)
    dev = torch.device(device)
    row = _coords(ny, dev)
    col = torch.zeros(ny, dtype=torch.float64, device=dev)
    for j in range(1, 9):
        col = col + (4.0 / j) * torch.cos(2.0 * math.pi * j * row / ny + float(psi[j - 1]))
    return col[:, None].expand(ny, nx).to(torch.float32).contiguous()


def vortex_tubes(dims, seed: int, count: int = 64, device="cpu",
                 chunk_points: int = 1 << 24) -> torch.Tensor:
    """Gaussian-profile tubes A exp(-d^2 / (2 rho^2)) around random lines,
    rho ~ U[4, 12] cells, |A| ~ U[2, 4] with a random sign."""
    dims = tuple(int(d) for d in dims)
    assert len(dims) == 3
    rng = np.random.Generator(np.random.PCG64(seed))
    dev = torch.device(device)
    tubes = []
    for _ in range(count):
        p = rng.uniform(0.0, 1.0, size=3) * np.array(dims)
        u = _unit_vectors(rng, 1, 3)[0]
        rho = rng.uniform(4.0, 12.0)
        a = rng.uniform(2.0, 4.0) * (1.0 if rng.uniform() < 0.5 else -1.0)
        tubes.append((p, u, rho, a))
    out = torch.zeros(dims, dtype=torch.float32, device=dev)
    zc = max(1, chunk_points // (dims[1] * dims[2]))
    y = _coords(dims[1], dev)[None, :, None]
    x = _coords(dims[2], dev)[None, None, :]
    for z0 in range(0, dims[0], zc):
        z1 = min(dims[0], z0 + zc)
        z = (_coords(z1 - z0, dev) + z0)[:, None, None]
        acc = torch.zeros((z1 - z0, dims[1], dims[2]), dtype=torch.float32, device=dev)
        for p, u, rho, a in tubes:
            dz, dy, dx = z - p[0], y - p[1], x - p[2]
            along = dz * u[0] + dy * u[1] + dx * u[2]
            d2 = dz * dz + dy * dy + dx * dx - along * along
            acc += (a * torch.exp(-d2 / (2.0 * rho * rho))).to(torch.float32)
        out[z0:z1] = acc
    return out


# ---------------------------------------------------------------- workloads

def grf_trend_field(n: int = 64, device="cpu") -> torch.Tensor:
    """n^3 k^-5/3 field (seed 1) plus a linear trend, values in about [-10, 10]."""
    return grf((n, n, n), 5.0 / 3.0, seed=1, device=device) + linear_trend((n, n, n), device)


def grf_fronts_field(n: int = 512, device="cpu") -> torch.Tensor:
    """n^3 k^-5/3 field (seed 2) plus 8 tanh fronts of width 2 cells (NYX-sized)."""
    dims = (n, n, n)
    return grf(dims, 5.0 / 3.0, seed=2, device=device) + fronts(dims, 2000, device=device)


UNEVEN_CHOICES = (100, 128, 256, 384, 500)


def mixed_batch_fields(count2d: int = 48, count3d: int = 48, device="cpu", shape2d=(1800, 3600)):
    """Batch of CESM-ATM-shaped 2D fields (zonal bands + k^-3 noise, seeds
    3000+i) and uneven 3D k^-5/3 fields (dims from UNEVEN_CHOICES, seeds
    3100+i).  Yields (name, tensor) lazily."""
    for i in range(count2d):
        f = zonal_bands(shape2d[0], shape2d[1], 3000 + i, device) + grf(
            shape2d, 3.0, seed=3000 + i, sigma=1.0, device=device)
        yield f"band2d_{i}", f
    for i in range(count3d):
        rng = np.random.Generator(np.random.PCG64(3100 + i))
        dims = tuple(int(v) for v in rng.choice(UNEVEN_CHOICES, size=3))
        yield f"grf3d_{i}", grf(dims, 5.0 / 3.0, seed=3100 + i, device=device)


def training_field_spec(index: int):
    """Training-field recipe i: slope ~ U[1, 4], edge from {64,96,128,192,256},
    relative bound log-uniform in [1e-5, 1e-2], seed 40000 + i."""
    rng = np.random.Generator(np.random.PCG64(40000 + index))
    slope = float(rng.uniform(1.0, 4.0))
    edge = int(rng.choice((64, 96, 128, 192, 256)))
    rel = float(10.0 ** rng.uniform(-5.0, -2.0))
    return {"seed": 40000 + index, "slope": slope, "dims": (edge, edge, edge), "rel_eb": rel}


def vortex_field(n: int = 1024, device="cpu") -> torch.Tensor:
    """n^3 k^-5/3 field (seed 5) with 64 Gaussian vortex tubes."""
    dims = (n, n, n)
    return grf(dims, 5.0 / 3.0, seed=5, device=device) + vortex_tubes(dims, 5, device=device)
