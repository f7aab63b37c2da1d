"""Seeded synthetic float32 fields shaped like the paper's workloads.

The paper evaluates on NYX (3D cosmology), ATM (2D climate, 1800x3600) and
Hurricane (3D, 100x500x500) fields (Table 1, Section "Experimental Setting").
Those datasets are not available, so these generators stand in for them with
Gaussian random fields (GRFs) of power-law spectra, tanh fronts, log-normal
densities and fill regions.  This module holds none of the rate-distortion
method's arithmetic; it only makes inputs, and both the CUDA path and the
oracle consume the same bytes in every parity test.

Recipe (all fields C-order, last axis fastest):
  1. white noise N(0, 1) from a seeded generator;
  2. real FFT; multiply by sqrt(P(k)), P(k) = k^alpha, k = |f| in cycles per
     cell (per-axis FFT frequencies), P(0) = 0;
  3. inverse real FFT; standardise to mean 0, variance 1.
Seeds: config c, field i -> 20180600 + 1000*c + i.

Two backends: numpy (PCG64, host) and torch (device or host, torch.Generator).
They follow the same recipe but draw different noise, so a field is only ever
compared with itself.
"""
from __future__ import annotations

import math

import numpy as np


def seed_for(config: int, field: int = 0) -> int:
    return 20180600 + 1000 * config + field


# --------------------------------------------------------------------------
# numpy backend
# --------------------------------------------------------------------------

def _kmag_np(shape):
    axes = []
    for i, n in enumerate(shape):
        f = np.fft.rfftfreq(n) if i == len(shape) - 1 else np.fft.fftfreq(n)
        axes.append(f)
    grids = np.meshgrid(*axes, indexing="ij", sparse=True)
    k2 = sum(g * g for g in grids)
    return np.sqrt(k2)


def grf_np(shape, alpha: float, seed: int) -> np.ndarray:
    """Unit-variance GRF with spectrum k^alpha (numpy, float32 result)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal(shape)
    spec = np.fft.rfftn(noise)
    k = _kmag_np(shape)
    with np.errstate(divide="ignore"):
        amp = np.where(k > 0, k ** (alpha / 2.0), 0.0)
    g = np.fft.irfftn(spec * amp, s=shape, axes=tuple(range(len(shape))))
    g -= g.mean()
    s = g.std()
    if s > 0:
        g /= s
    return g.astype(np.float32)


def rescale(x: np.ndarray, lo: float, hi: float) -> np.ndarray:
    xmin, xmax = float(x.min()), float(x.max())
    if xmax == xmin:
        return np.full_like(x, lo, dtype=np.float32)
    y = (x.astype(np.float64) - xmin) / (xmax - xmin) * (hi - lo) + lo
    return y.astype(np.float32)


def tanh_fronts_np(shape, n_fronts: int, width: float, seed: int) -> np.ndarray:
    """Sum of a_j tanh(n_j . (r - c_j) / width): seeded unit normals n_j,
    centres c_j uniform in the box, amplitudes a_j ~ U[0.5, 1.5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape],
                        indexing="ij", sparse=True)
    out = np.zeros(shape, np.float64)
    for _ in range(n_fronts):
        nrm = rng.standard_normal(len(shape))
        nrm /= np.linalg.norm(nrm)
        c = rng.uniform(0, 1, len(shape)) * np.array(shape)
        a = rng.uniform(0.5, 1.5)
        s = sum(nrm[i] * (grids[i] - c[i]) for i in range(len(shape)))
        out += a * np.tanh(s / width)
    return out


def config1_field(seed: int | None = None, shape=(256, 256)) -> np.ndarray:
    """2D GRF, spectrum k^-3, rescaled to [-1, 1]."""
    seed = seed_for(1) if seed is None else seed
    return rescale(grf_np(shape, -3.0, seed), -1.0, 1.0)


def config2_field(seed: int | None = None, shape=(100, 500, 500)) -> np.ndarray:
    """3D GRF k^-11/3 plus 8 tanh fronts of width 2 cells, scaled to [0, 300]
    (a Hurricane-shaped field)."""
    seed = seed_for(2) if seed is None else seed
    g = grf_np(shape, -11.0 / 3.0, seed).astype(np.float64)
    g += tanh_fronts_np(shape, 8, 2.0, seed + 500)
    return rescale(g, 0.0, 300.0)


def config3_field(i: int, seed: int | None = None, shape=(512, 512, 512)) -> np.ndarray:
    """Field i of the NYX-shaped snapshot: 0 is the log-normal density
    exp(2 G), G a unit GRF with k^-2; 1..3 are velocity components, unit
    GRFs with k^-11/3."""
    seed = seed_for(3) if seed is None else seed
    if i == 0:
        return np.exp(2.0 * grf_np(shape, -2.0, seed).astype(np.float64)).astype(np.float32)
    return grf_np(shape, -11.0 / 3.0, seed + i)


def config3_fields(seed: int | None = None, shape=(512, 512, 512)) -> list:
    """The density and the three velocity components (a NYX-shaped snapshot)."""
    return [config3_field(i, seed, shape) for i in range(4)]


def fill_region_np(x: np.ndarray, seed: int, fill: float = 1e-20) -> np.ndarray:
    """Cells where an independent k^-3 GRF is below its 25th percentile are
    set to `fill` (ATM-style missing-value fill)."""
    g = grf_np(x.shape, -3.0, seed)
    mask = g < np.percentile(g, 25.0)
    y = x.copy()
    y[mask] = np.float32(fill)
    return y


# --------------------------------------------------------------------------
# torch backend (device generation of the large fields)
# --------------------------------------------------------------------------

def grf_torch(shape, alpha: float, seed: int, device="cuda", chunk_dtype=None):
    """Unit-variance GRF with spectrum k^alpha generated with torch.fft on
    `device`; float32 result on that device."""
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    noise = torch.randn(shape, generator=gen, device=device, dtype=torch.float32)
    spec = torch.fft.rfftn(noise)
    del noise
    k2 = None
    for i, n in enumerate(shape):
        f = (torch.fft.rfftfreq(n, device=device) if i == len(shape) - 1
             else torch.fft.fftfreq(n, device=device))
        view = [1] * len(shape)
        view[i] = f.numel()
        f = f.view(view) ** 2
        k2 = f if k2 is None else k2 + f
    k = torch.sqrt(k2)
    amp = torch.where(k > 0, k.clamp_min(1e-30) ** (alpha / 2.0), torch.zeros_like(k))
    spec.mul_(amp)
    del amp, k, k2
    g = torch.fft.irfftn(spec, s=shape)
    del spec
    g.sub_(g.mean())
    s = g.std()
    if float(s) > 0:
        g.div_(s)
    return g.to(torch.float32).contiguous()


def rescale_torch(x, lo: float, hi: float):
    xmin, xmax = x.min(), x.max()
    return ((x - xmin) / (xmax - xmin) * (hi - lo) + lo).to(x.dtype).contiguous()


def tanh_fronts_torch(shape, n_fronts: int, width: float, seed: int, device="cuda"):
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    out = torch.zeros(shape, device=device, dtype=torch.float32)
    coords = [torch.arange(n, device=device, dtype=torch.float32) for n in shape]
    for _ in range(n_fronts):
        nrm = rng.standard_normal(len(shape))
        nrm /= np.linalg.norm(nrm)
        c = rng.uniform(0, 1, len(shape)) * np.array(shape)
        a = rng.uniform(0.5, 1.5)
        s = None
        for i in range(len(shape)):
            view = [1] * len(shape)
            view[i] = shape[i]
            t = ((coords[i] - float(c[i])) * float(nrm[i])).view(view)
            s = t if s is None else s + t
        out.add_(torch.tanh(s / width) * float(a))
    return out


def config2_field_torch(seed=None, shape=(100, 500, 500), device="cuda"):
    seed = seed_for(2) if seed is None else seed
    g = grf_torch(shape, -11.0 / 3.0, seed, device)
    g.add_(tanh_fronts_torch(shape, 8, 2.0, seed + 500, device))
    return rescale_torch(g, 0.0, 300.0)


def config3_fields_torch(seed=None, shape=(512, 512, 512), device="cuda"):
    import torch

    seed = seed_for(3) if seed is None else seed
    dens = torch.exp(2.0 * grf_torch(shape, -2.0, seed, device)).contiguous()
    out = [dens]
    for i in range(3):
        out.append(grf_torch(shape, -11.0 / 3.0, seed + 1 + i, device))
    return out


def snapshot_specs(seed: int | None = None) -> list:
    """The batched snapshot: 79 2D 1800x3600 fields (spectral exponent drawn
    from U[-4, -2]; the 8 with index = 0 mod 10 get a 1e-20 fill region),
    13 Hurricane-shaped 100x500x500 fields and 6 512^3 fields (density, three
    velocities and two more log-normal fields with sigma 1.0 and 1.5).  Each
    spec: dict(kind, shape, alpha, seed, eb_rel)."""
    seed = seed_for(4) if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    ebs = (1e-3, 1e-4, 1e-5)
    specs = []
    for i in range(79):
        specs.append(dict(kind="atm", shape=(1800, 3600), alpha=float(rng.uniform(-4, -2)),
                          seed=seed + i, fill=(i % 10 == 0), eb_rel=float(rng.choice(ebs))))
    for i in range(13):
        specs.append(dict(kind="hurricane", shape=(100, 500, 500), alpha=-11.0 / 3.0,
                          seed=seed + 100 + i, fill=False, eb_rel=float(rng.choice(ebs))))
    nyx = [("density", 2.0), ("vx", None), ("vy", None), ("vz", None),
           ("lognormal", 1.0), ("lognormal", 1.5)]
    for i, (kind, sigma) in enumerate(nyx):
        specs.append(dict(kind="nyx_" + kind, shape=(512, 512, 512),
                          alpha=-2.0 if sigma else -11.0 / 3.0, sigma=sigma,
                          seed=seed + 200 + i, fill=False, eb_rel=float(rng.choice(ebs))))
    return specs


def make_field_torch(spec: dict, device="cuda"):
    """Materialise one snapshot spec on `device` (torch backend)."""
    import torch

    shape = tuple(spec["shape"])
    if spec["kind"] == "hurricane":
        return config2_field_torch(spec["seed"], shape, device)
    g = grf_torch(shape, spec["alpha"], spec["seed"], device)
    if spec.get("sigma"):
        g = torch.exp(float(spec["sigma"]) * g).contiguous()
    if spec.get("fill"):
        m = grf_torch(shape, -3.0, spec["seed"] + 7, device)
        thr = torch.quantile(m.flatten()[:: max(1, m.numel() // 1_000_000)].float(), 0.25)
        g = torch.where(m < thr, torch.full_like(g, 1e-20), g).contiguous()
    return g


def serving_requests(rate: float, n: int, seed: int, population: int = 256) -> list:
    """Poisson arrivals at `rate` req/s; each request names one field of a
    pre-generated population (2D ny~logU[512,1800], nx~logU[512,3600] or 3D
    cube side ~logU[64,512], each w.p. 1/2; alpha ~ U[-4,-2]) and an error
    bound from {1e-2..1e-6}.  Returns dicts (t_arrival, field_index, eb_rel)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate)
        out.append(dict(t=t, field=int(rng.integers(population)),
                        eb_rel=float(10.0 ** -rng.integers(2, 7))))
    return out


def serving_population(seed: int, population: int = 256) -> list:
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(population):
        if rng.random() < 0.5:
            ny = int(round(math.exp(rng.uniform(math.log(512), math.log(1800)))))
            nx = int(round(math.exp(rng.uniform(math.log(512), math.log(3600)))))
            shape = (ny, nx)
        else:
            s = int(round(math.exp(rng.uniform(math.log(64), math.log(512)))))
            shape = (s, s, s)
        specs.append(dict(kind="grf", shape=shape, alpha=float(rng.uniform(-4, -2)),
                          seed=seed + 1 + i, fill=False))
    return specs
