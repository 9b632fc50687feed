"""Pins of the oracle's upwind sweeps: exactness on solutions the stencils must reproduce,
second-order convergence, the clustered grid's smallest section (Sec. 2.4), and the
free-molecular duct against independent ray lengths."""
import numpy as np
import pytest

from oracle import transport, velocity


def test_P10_clustered_grid_smallest_section():
    x = transport.nodes_clustered(100)
    assert x[0] == -0.5 and abs(x[-1]) < 1e-15
    d = np.diff(x)
    assert np.all(d > 0)
    # Sec. 2.4 prints "1.24e-6"; the map gives 10 s^3 to leading order at s = 1/200
    assert abs(d.min() - 1.2406e-6) < 5e-10
    assert abs(d.min() - 10 * (1 / 200) ** 3 * (1 - 1.5 / 200 + 0.6 / 200 ** 2)) < 1e-12


def test_backward_coeffs_exact_for_quadratics():
    for (a, b, c) in [(-0.3, -0.1, 0.25), (0.0, 0.5, 0.6)]:
        ka, kb, kc = transport.backward_coeffs(a, b, c)
        for f, df in [(lambda x: 1 + 0 * x, 0.0), (lambda x: x, 1.0),
                      (lambda x: x * x, 2 * c)]:
            assert abs(ka * f(c) + kb * f(b) + kc * f(a) - df) < 1e-12


@pytest.mark.parametrize("grid", ["uniform", "clustered"])
def test_sweep_1d_exact_for_mirror_linear_profile(grid):
    nv = 8
    V1, V2, V3, _ = velocity.grid(nv, 6.0)
    x = transport.nodes_uniform(10) if grid == "uniform" else transport.nodes_clustered(12)
    rng = np.random.default_rng(0)
    g = rng.standard_normal((nv, nv, nv))
    nu = 0.5 + rng.random((nv, nv, nv))
    gm = g[::-1]                        # g at the mirror velocity (-v1, v2, v3)
    X = x[:, None, None, None]
    pos = V1[None] > 0
    # v1 > 0: g (x + 1/2), zero at the wall; v1 < 0: mirror image g(v*) (1/2 - x)
    hex_ = np.where(pos, g * (X + 0.5), gm * (0.5 - X))
    dh = np.where(pos, g + 0 * X, -gm + 0 * X)
    rhs = nu * hex_ + V1 * dh
    h = transport.sweep_1d(rhs, nu, V1, x)
    assert np.max(np.abs(h - hex_)) < 1e-12 * np.max(np.abs(hex_))


def test_sweep_1d_second_order():
    nv = 4
    V1, V2, V3, _ = velocity.grid(nv, 3.0)
    nu = 1.0 + 0 * V1
    errs = []
    for ns in (40, 80, 160):
        x = transport.nodes_uniform(ns)
        X = x[:, None, None, None]
        # exact: v1>0 h = sin(pi (x+1/2))^2-ish profile vanishing at the wall,
        # mirrored for v1 < 0 so the symmetry plane condition holds
        f = lambda s: np.sin(2.0 * (s + 0.5)) * (s + 0.5)
        df = lambda s: 2.0 * np.cos(2.0 * (s + 0.5)) * (s + 0.5) + np.sin(2.0 * (s + 0.5))
        pos = V1[None] > 0
        hex_ = np.where(pos, f(X) + 0 * V1, f(-X) + 0 * V1)
        dh = np.where(pos, df(X) + 0 * V1, -df(-X) + 0 * V1)
        rhs = nu * hex_ + V1 * dh
        h = transport.sweep_1d(rhs, nu, V1, x)
        errs.append(np.max(np.abs(h - hex_)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_sweep_2d_exact_for_bilinear_distance_profile():
    nv = 8
    V1, V2, V3, _ = velocity.grid(nv, 6.0)
    nx, ny, width = 7, 5, 1.4
    rng = np.random.default_rng(2)
    g = rng.standard_normal((nv, nv, nv))
    nu = 0.5 + rng.random((nv, nv, nv))
    xc = (np.arange(nx) + 0.5) * width / nx
    yc = (np.arange(ny) + 0.5) / ny
    Xc = xc[:, None, None, None, None]
    Yc = yc[None, :, None, None, None]
    # distance from the inflow faces along the march directions
    dx_ = np.where(V1 > 0, Xc, width - Xc)
    dy_ = np.where(V2 > 0, Yc, 1.0 - Yc)
    hex_ = g * dx_ * dy_
    rhs = nu * hex_ + np.abs(V1) * g * dy_ + np.abs(V2) * g * dx_
    h = transport.sweep_2d(rhs, nu, V1, V2, nx, ny, width)
    assert np.max(np.abs(h - hex_)) < 1e-12 * np.max(np.abs(hex_))


def test_P15_free_molecular_duct_vs_ray_lengths():
    """delta = 0: v.grad h = S with h = 0 on inflow faces has h = S * t_back, t_back the
    flight time to the wall along -v in the cross-section.  The upwind sweep (nu = 0)
    must approach it as the grid is refined."""
    nv = 8
    V1, V2, V3, _ = velocity.grid(nv, 4.0)
    S = velocity.source(V1, V2, V3, 0)
    width = 1.0
    errs = []
    for n in (16, 32):
        xc = (np.arange(n) + 0.5) / n
        Xc = xc[:, None, None, None, None]
        Yc = xc[None, :, None, None, None]
        tx = np.where(V1 > 0, Xc, width - Xc) / np.abs(V1)
        ty = np.where(V2 > 0, Yc, 1.0 - Yc) / np.abs(V2)
        hex_ = S * np.minimum(tx, ty)
        rhs = np.broadcast_to(S, (n, n) + S.shape).copy()
        h = transport.sweep_2d(rhs, 0 * S, V1, V2, n, n, width)
        # the flow rate converges; pointwise the corner kink of min(tx, ty) limits order
        Mex = np.mean(np.sum(V3 * hex_, axis=(-3, -2, -1)))
        Mfd = np.mean(np.sum(V3 * h, axis=(-3, -2, -1)))
        errs.append(abs(Mfd - Mex) / abs(Mex))
    assert errs[1] < errs[0] and errs[1] < 0.03, errs
