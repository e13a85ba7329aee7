"""Seeded synthetic scalar fields shaped like the volumes of the paper's experiments.

This module only draws random numbers and synthesises float32 grids. It holds none
of the Morse-Smale arithmetic, so both the CPU oracle and the CUDA path may read
its output: every array it returns is float32, C-contiguous, shape [nz, ny, nx]
(vertex (x, y, z) at index x + nx*(y + ny*z)).

The paper measures on public Open SciVis volumes of 64^3 to 512x512x112 vertices
(Table 1); those are not available here, so these generators stand in for them:

* ``cosine_lattice``  32^3 cos(2 pi x/16)+cos(2 pi y/16)+cos(2 pi z/16) + U[0,1e-3]
* ``grf``             Gaussian random field with power spectrum P(k) ~ k^-alpha
* ``gaussian_blobs``  sum of isotropic Gaussian blobs + N(0, 1e-3) noise
* ``batch_volumes``   64 GRFs of uneven anisotropic sizes (axes in 48..192)
* ``serving_stream``  8 advected GRF streams and a Poisson request trace

All synthesis runs in float64 and is cast to float32 once at the end.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def cosine_lattice(n: int = 32, period: float = 16.0, noise: float = 1e-3, seed: int = 0) -> np.ndarray:
    """cos(2 pi x/period) + cos(2 pi y/period) + cos(2 pi z/period) + U[0, noise], x,y,z in 0..n-1."""
    rng = _rng(seed)
    t = np.cos(2.0 * np.pi * np.arange(n, dtype=np.float64) / period)
    f = t[None, None, :] + t[None, :, None] + t[:, None, None]
    f = f + rng.uniform(0.0, noise, size=(n, n, n))
    return np.ascontiguousarray(f.astype(np.float32))


def _spectral_amplitude(shape_zyx, alpha: float) -> np.ndarray:
    """sqrt(P(k)) with P(k) = k^-alpha, k = |frequency| in cycles/voxel, P(0) = 0 (rfftn layout)."""
    nz, ny, nx = shape_zyx
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    nz_mask = k > 0
    amp[nz_mask] = k[nz_mask] ** (-alpha / 2.0)
    return amp


def _grf_spectrum(rng: np.random.Generator, shape_zyx, alpha: float) -> np.ndarray:
    white = rng.standard_normal(size=shape_zyx)
    return np.fft.rfftn(white) * _spectral_amplitude(shape_zyx, alpha)


def _normalise(f: np.ndarray) -> np.ndarray:
    f = f - f.mean()
    s = f.std()
    if s > 0:
        f = f / s
    return np.ascontiguousarray(f.astype(np.float32))


def grf(shape_zyx, alpha: float = 3.0, seed: int = 1) -> np.ndarray:
    """Periodic Gaussian random field: white N(0,1) -> rfftn -> * sqrt(P(k)) -> irfftn -> zero mean, unit std."""
    shape_zyx = tuple(int(s) for s in shape_zyx)
    rng = _rng(seed)
    spec = _grf_spectrum(rng, shape_zyx, alpha)
    return _normalise(np.fft.irfftn(spec, s=shape_zyx, axes=(0, 1, 2)))


def gaussian_blobs(n: int = 512, n_blobs: int = 2000, sigma_range=(2.0, 20.0), noise_std: float = 1e-3,
                   seed: int = 2, truncate: float = 5.0) -> np.ndarray:
    """Sum of isotropic Gaussian blobs plus N(0, noise_std) noise on an n^3 grid.

    Draw order: centres U[0,n)^3 (columns x,y,z), sigmas U[sigma_range], amplitudes U[-1,1],
    then the noise. Each blob is evaluated separably as the outer product of 1D exp factors,
    truncated to the box within ``truncate`` sigma of its centre (clipped to the grid).
    """
    rng = _rng(seed)
    centres = rng.uniform(0.0, float(n), size=(n_blobs, 3))
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=n_blobs)
    amps = rng.uniform(-1.0, 1.0, size=n_blobs)
    f = rng.normal(0.0, noise_std, size=(n, n, n))
    for (cx, cy, cz), s, a in zip(centres, sigmas, amps):
        lo = [max(0, int(np.ceil(c - truncate * s))) for c in (cx, cy, cz)]
        hi = [min(n - 1, int(np.floor(c + truncate * s))) for c in (cx, cy, cz)]
        if any(h < l for l, h in zip(lo, hi)):
            continue
        gx = a * np.exp(-0.5 * ((np.arange(lo[0], hi[0] + 1) - cx) / s) ** 2)
        gy = np.exp(-0.5 * ((np.arange(lo[1], hi[1] + 1) - cy) / s) ** 2)
        gz = np.exp(-0.5 * ((np.arange(lo[2], hi[2] + 1) - cz) / s) ** 2)
        f[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += (
            gz[:, None, None] * gy[None, :, None] * gx[None, None, :])
    return np.ascontiguousarray(f.astype(np.float32))


def batch_volume(seed: int, alpha: float = 2.5, lo: int = 48, hi: int = 192) -> np.ndarray:
    """One batch volume: draws its axis sizes (nx, ny, nz) uniformly in [lo, hi], then a GRF."""
    rng = _rng(seed)
    nx, ny, nz = (int(v) for v in rng.integers(lo, hi + 1, size=3))
    spec = _grf_spectrum(rng, (nz, ny, nx), alpha)
    return _normalise(np.fft.irfftn(spec, s=(nz, ny, nx), axes=(0, 1, 2)))


def batch_volumes(n: int = 64, first_seed: int = 100, alpha: float = 2.5):
    return [batch_volume(first_seed + i, alpha) for i in range(n)]


@dataclass
class ServingStream:
    """One advected field: a base GRF shifted by velocity * t in Fourier space at step t."""
    size: int
    seed: int
    spectrum: np.ndarray
    velocity: np.ndarray
    mean: float
    std: float

    def step_device(self, t: int, device="cuda"):
        """The same step synthesised with torch.fft on `device` (for feeding a server at
        request rate); float32 [n, n, n] tensor.  Matches step() to float32 rounding."""
        import torch

        n = self.size
        spec = getattr(self, "_spec_dev", None)
        if spec is None or spec.device != torch.device(device):
            spec = self._spec_dev = torch.from_numpy(self.spectrum).to(device)
        kz = torch.fft.fftfreq(n, device=device, dtype=torch.float64)[:, None, None]
        ky = torch.fft.fftfreq(n, device=device, dtype=torch.float64)[None, :, None]
        kx = torch.fft.rfftfreq(n, device=device, dtype=torch.float64)[None, None, :]
        vx, vy, vz = (float(v) * float(t) for v in self.velocity)
        phase = torch.exp(-2j * np.pi * (kx * vx + ky * vy + kz * vz))
        f = torch.fft.irfftn(spec * phase, s=(n, n, n), dim=(0, 1, 2))
        return ((f - self.mean) / self.std).to(torch.float32).contiguous()

    def step(self, t: int) -> np.ndarray:
        n = self.size
        kz = np.fft.fftfreq(n)[:, None, None]
        ky = np.fft.fftfreq(n)[None, :, None]
        kx = np.fft.rfftfreq(n)[None, None, :]
        vx, vy, vz = self.velocity * float(t)
        phase = np.exp(-2j * np.pi * (kx * vx + ky * vy + kz * vz))
        f = np.fft.irfftn(self.spectrum * phase, s=(n, n, n), axes=(0, 1, 2))
        return np.ascontiguousarray(((f - self.mean) / self.std).astype(np.float32))


def serving_streams(n_streams: int = 8, lo: int = 64, hi: int = 384, alpha: float = 3.0,
                    first_seed: int = 200):
    """Per-stream cube sizes linspace(lo, hi, n_streams) rounded; stream s uses seed first_seed+s.

    Draw order per stream: the white noise of the base field, then the velocity U[-1,1]^3
    (voxels per step).
    """
    sizes = [int(round(v)) for v in np.linspace(lo, hi, n_streams)]
    out = []
    for s, n in enumerate(sizes):
        rng = _rng(first_seed + s)
        spec = _grf_spectrum(rng, (n, n, n), alpha)
        vel = rng.uniform(-1.0, 1.0, size=3)
        base = np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))
        out.append(ServingStream(n, first_seed + s, spec, vel, float(base.mean()), float(base.std())))
    return out


def request_trace(n_requests: int = 500, rate_hz: float = 200.0, n_streams: int = 8, seed: int = 300):
    """Poisson arrivals: request i targets stream i mod n_streams at step i // n_streams."""
    rng = _rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    return [(float(arrivals[i]), i % n_streams, i // n_streams) for i in range(n_requests)]


def config_field(name: str) -> np.ndarray:
    """Single-volume workloads by name: 'cos32', 'grf256', 'blobs512' (and small variants for tests)."""
    if name == "cos32":
        return cosine_lattice()
    if name == "grf256":
        return grf((256, 256, 256), alpha=3.0, seed=1)
    if name == "blobs512":
        return gaussian_blobs()
    raise KeyError(name)
