"""Seeded synthetic workloads of the buoyancy-driven-cavity step.

Shared by the tests, the bench and the oracle-side scripts as the one source
of INPUTS (sizes, parameters, seeds, wall-temperature fields).  It holds none
of the method's arithmetic: the initial noise is drawn inside each
implementation from the seed (splitmix64 keyed by global node index), and
everything here is either a constant of a configuration or a seeded numpy
draw that is passed in as data.

The paper measures uniform meshes 32^3 .. 1024^3 of a differentially heated
cube at Ra = 1e5 (Section 2) and times a 256^3 problem on one and two P100s
(Section 4.6, Tables 3-4); it uses no dataset.
"""
from __future__ import annotations

import numpy as np

# configuration 1: the scheme as written, FP64
CFG1 = dict(name="cavity32_ra1e4_fp64", n=(32, 32, 32), Ra=1e4, Pr=0.71, noise=1e-3, seed=0, steps=200)
# configuration 2: 128^3, Ra 1e5, FP64 and FP32-mixed, 8 blocks three ways
CFG2 = dict(name="cavity128_ra1e5", n=(128, 128, 128), Ra=1e5, Pr=0.71, noise=1e-3, seed=0, steps=2000,
            decomps=((8, 1, 1), (4, 2, 1), (2, 2, 2)))
# configuration 3: 256^3, Ra 1e6, FP32-mixed
CFG3 = dict(name="cavity256_ra1e6_fp32", n=(256, 256, 256), Ra=1e6, Pr=0.71, noise=1e-4, seed=0, steps=5000)


# configuration 5: the discrete adjoint (gradient of the mean hot-wall Nusselt
# number w.r.t. the hot-wall temperature field and Ra), FP32-mixed forward
CFG5 = dict(name="adjoint128_fp32", n=(128, 128, 128), Ra=1e5, Pr=0.71, noise=1e-3, seed=0, steps=500, ckpt=50,
            theta_seed=11, theta_sigma=0.01)


# configuration 4: a batch of independent cavities advanced together
CFG4 = dict(name="batch64_fp32", ncav=64, nmin=24, nmax=96, ra_log10=(3.0, 6.0), Pr=0.71, noise=1e-3, steps=1000)

_MASK64 = (1 << 64) - 1


def _splitmix64(x: int) -> int:
    """splitmix64 output for state x (Steele, Lea & Flood 2014), as an input draw."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def batch_cavities(ncav: int = CFG4["ncav"], nmin: int = CFG4["nmin"], nmax: int = CFG4["nmax"],
                   ra_log10=CFG4["ra_log10"]):
    """Cavity b of the batch: n_d = nmin + draw mod (nmax - nmin + 1) for d = x, y, z, and
    log10 Ra uniform on ra_log10 from the next draw; the seed of its initial noise is b."""
    out = []
    span = nmax - nmin + 1
    for b in range(ncav):
        key = (b << 40) + (1 << 39)
        n = tuple(nmin + _splitmix64(key + d) % span for d in range(3))
        u = (_splitmix64(key + 3) >> 11) * (1.0 / 9007199254740992.0)
        ra = 10.0 ** (ra_log10[0] + (ra_log10[1] - ra_log10[0]) * u)
        out.append(dict(n=n, Ra=ra, seed=b))
    return out


def wall_temperature(ny: int, nz: int, seed: int, base: float = 1.0, sigma: float = 0.01) -> np.ndarray:
    """Hot-wall temperature base + N(0, sigma^2) per wall node, (j-1) + ny (k-1) order."""
    rng = np.random.default_rng(seed)
    return base + sigma * rng.standard_normal(ny * nz)


def smooth_state(n: tuple[int, int, int], seed: int, amp=(50.0, 2.0, 2.0, 2.0, 0.2)) -> np.ndarray:
    """A smooth random interior state [5, nz, ny, nx] (p, u, v, w, T): a few
    seeded low Fourier modes per field, T around the conduction profile."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    x = np.arange(1, nx + 1) / (nx + 1)
    y = np.arange(1, ny + 1) / (ny + 1)
    z = np.arange(1, nz + 1) / (nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    out = np.zeros((5, nz, ny, nx))
    for f in range(5):
        for _ in range(3):
            kx, ky, kz = rng.integers(1, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            out[f] += amp[f] * rng.uniform(-1, 1) * np.sin(np.pi * kx * X + ph[0]) * \
                np.sin(np.pi * ky * Y + ph[1]) * np.sin(np.pi * kz * Z + ph[2])
    out[4] += 1.0 - X
    return out
