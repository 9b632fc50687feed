"""Seeded synthetic inputs and the named workloads (parameters only, no method arithmetic).

Shared by the tests, the smoke check and bench.py.  The numbers restate the problem sizes
of the plates / duct experiments (Sec. 2.4, Tables 1-2) and the serving mix.
"""
import numpy as np


def random_h(cells, nv, vmax, seed, odd_v3=True):
    """Smooth, Maxwellian-weighted random VDF perturbations, shape (cells, nv, nv, nv).

    h = exp(-|v|^2) * (low-order random polynomial in v with per-cell coefficients); odd in
    v3 when odd_v3 (the parity of Poiseuille and thermal-transpiration solutions)."""
    rng = np.random.default_rng(seed)
    v = -vmax + (np.arange(nv) + 0.5) * (2.0 * vmax / nv)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    g = np.exp(-(V1 * V1 + V2 * V2 + V3 * V3))
    mons = [np.ones_like(V1), V1, V2, V1 * V1, V2 * V2, V1 * V2, V1 ** 3,
            V1 * V1 + V2 * V2 + V3 * V3]
    c = rng.standard_normal((cells, len(mons)))
    poly = np.tensordot(c, np.stack(mons), axes=1)
    noise = 0.05 * rng.standard_normal((cells, nv, nv, nv))
    if odd_v3:
        h = g * V3 * (poly + noise + noise[..., ::-1])
    else:
        h = g * (poly + noise)
    return h



def fourier_start(nv, vmax, seed):
    """Start vector of the Fourier-mode power iteration: v3 exp(-|v|^2) (1 + 0.3 n) with n a
    standard-normal field even in v3, so the vector is odd in v3 (real, shape (nv, nv, nv))."""
    rng = np.random.default_rng(seed)
    v = -vmax + (np.arange(nv) + 0.5) * (2.0 * vmax / nv)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    n = rng.standard_normal((nv, nv, nv))
    n = 0.5 * (n + n[..., ::-1])
    return V3 * np.exp(-(V1 * V1 + V2 * V2 + V3 * V3)) * (1.0 + 0.3 * n)

# Plates, 16^3, 20 uniform sections, delta = 1, M = 16 (small case the oracle finishes in
# seconds).
PLATES_16 = dict(dim=1, ns=20, grid_kind=0, delta=1.0, nv=16, vmax=6.0, M=16)

# Plates, 32^3, 100 clustered sections (Sec. 2.4 map), M = 32: the eight cases
# delta in {0.1, 1, 10, 100} x {Poiseuille, thermal transpiration}, batched.
PLATES_32_DELTAS = (0.1, 1.0, 10.0, 100.0)
PLATES_32 = dict(dim=1, ns=100, grid_kind=1, nv=32, vmax=6.0, M=32)

# Duct, aspect ratio 2, 64 x 32 cells, delta = 10, 32^3, M = 32.
DUCT_64x32 = dict(dim=2, nx=64, ny=32, width=2.0, delta=10.0, nv=32, vmax=6.0, M=32)


def serving_requests(n=256, seed=20261203, rate=None):
    """Mixed stream: plates (50..200 sections) and ducts (20x20..80x40), delta log-uniform
    on [0.01, 100], nv in {24, 32}, Poiseuille / thermal transpiration 50/50, M = 32,
    Poisson arrival times at `rate` requests/s (None: all at t = 0)."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    for _ in range(n):
        if rate:
            t += rng.exponential(1.0 / rate)
        plate = rng.random() < 0.5
        nv = 24 if rng.random() < 0.5 else 32
        delta = float(10 ** rng.uniform(-2, 2))
        forcing = int(rng.random() < 0.5)
        if plate:
            geo = dict(dim=1, ns=int(rng.integers(50, 201)), grid_kind=1)
        else:
            sq = rng.random() < 0.5
            ny = int(rng.integers(20, 41))
            nx = ny if sq else min(2 * ny, 80)
            geo = dict(dim=2, nx=nx, ny=ny, width=nx / ny)
        out.append(dict(t=t, nv=nv, vmax=6.0, M=32, delta=delta, forcing=forcing, **geo))
    return out
