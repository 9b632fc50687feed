"""Pins of the oracle's CIS / SIS drivers: exactness of the diffusion solves, agreement of
CIS and SIS (Sec. 2.4: within 0.5%), independence of the converged flow rate from N
(Sec. 2.5: within 0.1%), the Onsager-Casimir relation M_T = Q_P (Sec. 2.4), SIS speed-up,
and 2D runs."""
import numpy as np
import pytest

from oracle import solver, transport


def test_diffusion_1d_exact_for_linear_Y():
    rng = np.random.default_rng(0)
    for x in (transport.nodes_uniform(9), transport.nodes_clustered(13)):
        W1 = rng.standard_normal(len(x))
        Uh = rng.standard_normal(len(x))
        nd, c = 2.7, -0.8
        # dY/dx = -nd * sigma * x + G1 = c  =>  G1 = c + nd * x  (sigma = 1)
        G1 = c + nd * x
        U = solver.diffusion_1d(Uh, W1, G1, x, nd, 1.0)
        Y = Uh[0] + W1[0] + c * (x - x[0])
        assert np.max(np.abs(U - (Y - W1))) < 1e-12
        assert abs(U[0] - Uh[0]) < 1e-15          # wall value kept from the VDF


def test_poisson_2d_exact_for_quadratic():
    nx, ny, width = 9, 7, 1.8
    dx, dy = width / nx, 1.0 / ny
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(xc, yc, indexing="ij")
    q = 0.3 + X * (width - X) * 1.1 + Y * (1 - Y) * 0.7 + 0.2 * X * Y
    lap = -2.2 - 1.4                                     # exact 5-point Laplacian of q
    Uh = q + np.where((X > dx) & (X < width - dx) & (Y > dy) & (Y < 1 - dy), 5.0, 0.0)
    Z = np.zeros_like(q)
    U = solver.poisson_2d(Uh, Z, Z, Z, Z, Z, width, -lap, 1.0)
    assert np.max(np.abs(U - q)) < 1e-11


def test_poisson_2d_moment_terms_signs():
    # with U = 0 on the ring, RHS terms d1 G1 alone must act like a source -d11 W1
    nx, ny, width = 8, 8, 1.0
    dx = width / nx
    xc = (np.arange(nx) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc, indexing="ij")
    Z = np.zeros_like(X)
    g = np.sin(np.pi * X)
    U_g = solver.poisson_2d(Z, Z, Z, Z, g, Z, width, 0.0, 1.0)
    # W1 = -∫ G1 dx  gives -d11 W1 = d1 G1 in the continuum; compare the discrete solves
    W = np.cos(np.pi * X) / np.pi
    U_w = solver.poisson_2d(Z, W, Z, Z, Z, Z, width, 0.0, 1.0)
    assert np.max(np.abs(U_g - U_w)) < 0.05 * np.max(np.abs(U_g))


@pytest.fixture(scope="module")
def c1_runs():
    out = {}
    for scheme in ("sis", "cis"):
        pb = solver.Problem(dim=1, ns=20, grid="uniform", delta=1.0, nv=16, M=16, R=4.5,
                            scheme=scheme, eps=1e-9)
        r, ok = solver.solve(pb)
        assert ok
        out[scheme] = r
    return out


def test_cis_and_sis_reach_same_solution(c1_runs):
    s, c = c1_runs["sis"], c1_runs["cis"]
    assert abs(s.M - c.M) < 5e-3 * abs(c.M)
    assert abs(s.Q - c.Q) < 5e-3 * abs(c.Q)
    assert s.iters < c.iters


def test_converged_flow_rate_independent_of_N(c1_runs):
    ref = c1_runs["sis"]
    for N in (1.0, 1.5):
        pb = solver.Problem(dim=1, ns=20, grid="uniform", delta=1.0, nv=16, M=16, R=4.5,
                            N=N, scheme="sis", eps=1e-9)
        r, ok = solver.solve(pb)
        assert ok
        assert abs(r.M - ref.M) < 1e-3 * abs(ref.M)


def test_P14_onsager_mass_flow_T_equals_heat_flow_P(c1_runs):
    pb = solver.Problem(dim=1, ns=20, grid="uniform", delta=1.0, nv=16, M=16, R=4.5,
                        forcing=1, scheme="sis", eps=1e-9)
    r, ok = solver.solve(pb)
    assert ok
    QP = c1_runs["sis"].Q
    # exact for the continuous LBE; the 16^3 velocity grid leaves a few percent
    assert abs(r.M - QP) < 0.05 * abs(QP)
    assert r.M < 0 and QP < 0


def test_sis_faster_than_cis_near_continuum():
    its = {}
    for scheme in ("sis", "cis"):
        pb = solver.Problem(dim=1, ns=10, grid="uniform", delta=5.0, nv=8, vmax=4.0, M=8,
                            scheme=scheme, eps=1e-7, max_iter=2000)
        r, ok = solver.solve(pb)
        assert ok
        its[scheme] = r.iters
    assert its["cis"] > 3 * its["sis"], its


def test_2d_sis_and_cis_converge():
    res = {}
    for scheme in ("sis", "cis"):
        pb = solver.Problem(dim=2, nx=8, ny=6, width=1.5, delta=2.0, nv=8, vmax=4.0, M=8,
                            scheme=scheme, eps=1e-8)
        r, ok = solver.solve(pb)
        assert ok
        res[scheme] = r
    assert res["sis"].iters < res["cis"].iters
    # 8x6 cells: the two fixed points differ by the discretisation, a few percent
    assert abs(res["sis"].M - res["cis"].M) < 0.05 * res["cis"].M
