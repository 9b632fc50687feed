"""Pins of the binary-mixture oracle (oracle/mixture.py; Sec. 4, Eq. Boltzmann_lin and the
mixture SIS).  Exact pins: the equal-mass limit (M1), the explicit cyclic sum (M2), mass
conservation per species (M5).  Pins at the resolution the dense oracle affords (nv = 12,
vmax = 4.5): brute-force collision integral (M3), invariants (M4), momentum and energy (M5);
a swap of the two reduced masses in the collision map fails each of them by a factor of
five or more.  Viscosity (M7): the closed form against a Monte Carlo Galerkin on the weak
form of the collision integral.  SIS: M8, M9."""
import numpy as np
import pytest

from oracle import fsm, mixture as mx, solver

NE_AR = (39.95 / 20.18, 1.0 / 0.711)


@pytest.fixture(scope="module")
def F12():
    return mx.MixFSM(mx.Mixture(NE_AR[0], NE_AR[1], 0.4), 12, 4.5, 8)


def _poly(F, a, c):
    mons = [1 + 0 * F.V1, F.V1, F.V2, F.V3, F.V1 * F.V2, F.V1 * F.V3, F.V2 * F.V3,
            F.V1 ** 2, F.V3 ** 3, F.V1 * F.V2 * F.V3]
    return F.f[a] * sum(ci * m for ci, m in zip(c, mons))


def test_M1_equal_species_is_the_single_species_operator():
    """m_B = m_A, d_B = d_A: L_a = chi_a G1(h_A + h_B) + G2(h_a), where G1 and G2 are the
    f_eq-first and h-first halves of oracle.fsm's operator at the same strength."""
    F1 = fsm.FSM(8, 6.0, 8)
    b = fsm.kernel_K(1.0) / (4.0 * np.pi)
    mix = mx.Mixture(1.0, 1.0, 0.3)
    Fm = mx.MixFSM(mix, 8, 6.0, 8, b0=b)
    rng = np.random.default_rng(1)
    hA, hB = rng.standard_normal((2, 3, 8, 8, 8))

    def g1(h):
        H = fsm.fft3(h)
        out = sum(F1.wp[p] * F1.A[p] * fsm.ifft3(F1.psi[p] * H).real for p in range(F1.M))
        return out - F1.feq * F1.loss_conv(h)

    def g2(h):
        H = fsm.fft3(h)
        return sum(F1.wp[p] * F1.B[p] * fsm.ifft3(F1.phi[p] * H).real for p in range(F1.M))

    lpA, LA, lpB, LB = Fm.apply(hA, hB, 1.3)
    for chi, h, lp, L in ((0.3, hA, lpA, LA), (0.7, hB, lpB, LB)):
        ref = 1.3 * (chi * g1(hA + hB) + g2(h))
        assert np.max(np.abs(lp - ref)) < 1e-13 * np.max(np.abs(ref))
        refL = ref - 1.3 * F1.nu * h
        assert np.max(np.abs(L - refL)) < 1e-13 * np.max(np.abs(refL))


def test_M2_matrix_gains_equal_the_explicit_cyclic_sum():
    F = mx.MixFSM(mx.Mixture(2.0, 1.4, 0.5), 4, 4.0, 4)
    rng = np.random.default_rng(2)
    g = rng.standard_normal((4, 4, 4))
    gh = np.fft.fftn(g).reshape(-1) / 64
    for a in range(2):
        for b in range(2):
            for K, ref in ((F.gain_second(a, b), F.direct_gain(a, b, F.f[a], g)),
                           (F.gain_first(a, b), F.direct_gain(a, b, g, F.f[b]))):
                Q = (np.fft.ifftn((K @ gh).reshape(4, 4, 4)) * 64).real
                assert np.max(np.abs(Q - ref)) < 1e-12 * np.max(np.abs(ref))


def test_M3_matches_bruteforce_collision_integral(F12):
    mix = F12.mix

    def hfun(a, p):
        v1, v2, v3 = p[..., 0], p[..., 1], p[..., 2]
        return ((v3 * (1 + 0.5 * v1 * v1 - 0.3 * v2) + 0.2 * v1 * v2)
                * mix.feq(a, v1, v2, v3) * (1.0 if a == 0 else -0.7))

    P = np.stack([F12.V1, F12.V2, F12.V3], -1)
    _, LA, _, LB = F12.apply(hfun(0, P), hfun(1, P), 1.0)
    vv = F12.V1[:, 0, 0]
    for a, L in ((0, LA), (1, LB)):
        scale = np.max(np.abs(L))
        for idx in ((6, 5, 7), (7, 4, 6), (5, 6, 8)):
            v = np.array([vv[i] for i in idx])
            bf = mx.bruteforce_L(mix, F12.b0, a, hfun, v, 1.0, n_vs=32, vs_max=6.0, n_sphere=12)
            assert abs(L[idx] - bf) < 0.08 * scale, (a, idx, L[idx], bf)


def test_M4_collision_invariants(F12):
    F, r = F12, F12.mix.r
    Z = np.zeros_like(F.f[0])
    c2 = F.V1 ** 2 + F.V2 ** 2 + F.V3 ** 2
    for x, y in ((F.f[0], Z), (Z, F.f[1]), (F.V1 * F.f[0], r[1] * F.V1 * F.f[1]),
                 (F.V3 * F.f[0], r[1] * F.V3 * F.f[1]), (c2 * F.f[0], r[1] * c2 * F.f[1])):
        _, LA, _, LB = F.apply(x, y, 1.0)
        ref = max(np.max(np.abs(F.nu[0] * x)), np.max(np.abs(F.nu[1] * y)))
        assert max(np.max(np.abs(LA)), np.max(np.abs(LB))) < 0.1 * ref


def test_M5_conservation(F12):
    F, r = F12, F12.mix.r
    rng = np.random.default_rng(3)
    # mass, per species, is exact for any h (the k = 0 mode of gain and loss coincide)
    hA = _poly(F, 0, rng.standard_normal(10)) + rng.standard_normal(F.f[0].shape) * F.f[0]
    hB = _poly(F, 1, rng.standard_normal(10)) + rng.standard_normal(F.f[0].shape) * F.f[1]
    _, LA, _, LB = F.apply(hA, hB, 2.0)
    ref = np.sum(np.abs(2.0 * F.nu[0] * hA)) + np.sum(np.abs(2.0 * F.nu[1] * hB))
    assert abs(np.sum(LA)) < 1e-13 * ref and abs(np.sum(LB)) < 1e-13 * ref
    # momentum and energy of the mixture, to the resolution of the grid (smooth h)
    hA, hB = _poly(F, 0, rng.standard_normal(10)), _poly(F, 1, rng.standard_normal(10))
    _, LA, _, LB = F.apply(hA, hB, 2.0)
    ref = np.sum(np.abs(2.0 * F.nu[0] * hA)) + np.sum(np.abs(2.0 * F.nu[1] * hB))
    c2 = F.V1 ** 2 + F.V2 ** 2 + F.V3 ** 2
    for psi in (F.V1, F.V2, F.V3, c2):
        assert abs(np.sum(psi * LA) + r[1] * np.sum(psi * LB)) < 0.03 * ref
    # and the shear moment of a shear perturbation is not conserved (guards against L == 0)
    _, LA, _, _ = F.apply(F.V1 * F.V3 * F.f[0], 0.0 * F.f[1], 1.0)
    assert np.sum(F.V1 * F.V3 * LA) < -0.1 * np.sum(np.abs(F.V1 * F.V3 * LA))


def test_M6_dissipative(F12):
    rng = np.random.default_rng(4)
    for _ in range(3):
        h = [_poly(F12, a, rng.standard_normal(10)) for a in range(2)]
        _, LA, _, LB = F12.apply(h[0], h[1])
        assert np.sum(h[0] * LA / F12.f[0]) + np.sum(h[1] * LB / F12.f[1]) < 0.0


def test_M7_viscosity_closed_form():
    assert abs(mx.eta1(1.0, 1.0, 0.3) - 5.0 / (16.0 * np.sqrt(np.pi))) < 1e-15
    assert abs(mx.eta1(2.0, 1.5, 1.0) - 5.0 / (16.0 * np.sqrt(np.pi))) < 1e-15          # pure A
    assert abs(mx.eta1(2.0, 1.5, 0.0) - 5.0 / 16.0 * np.sqrt(2.0 / np.pi) / 2.25) < 1e-15  # pure B
    # single species: b_AA reproduces oracle.fsm's strength (nu_bar = 1.25 delta)
    assert abs(4 * np.pi * mx.Mixture(1.0, 1.0, 0.6).b_AA(2.0) - fsm.kernel_K(2.0)) < 1e-15
    for args in ((NE_AR[0], NE_AR[1], 0.5), (3.0, 0.8, 0.3)):
        assert abs(mx.mc_galerkin_viscosity(mx.Mixture(*args)) - 1.0) < 0.01, args


def _cis_pair(nv=8, ns=6, delta=0.7, iters=3):
    mix_pb = mx.MixProblem(1.0, 1.0, 0.3, delta=delta, ns=ns, nv=nv, vmax=6.0, M=8, scheme="cis")
    mr = mx.MixRun(mix_pb)
    sp = solver.Run(solver.Problem(dim=1, ns=ns, delta=delta, nv=nv, vmax=6.0, M=8, scheme="cis"))
    for _ in range(iters):
        mr.step()
        sp.step()
    return mr, sp


def test_M8_identical_species_cis_is_the_single_species_cis():
    mr, sp = _cis_pair()
    for a, chi in ((0, 0.3), (1, 0.7)):
        assert np.max(np.abs(mr.h[a] - chi * sp.h)) < 1e-13 * np.max(np.abs(sp.h))


def test_M9_sis_and_cis_reach_the_same_solution(F12):
    """At a fixed point the SIS correction vanishes only up to the discretisation (the
    diffusion equations use the discrete momentum balance); the paper reports 0.5 %."""
    kw = dict(delta=1.0, ns=8, nv=12, vmax=4.5, M=8, eps=1e-10, max_iter=400)
    sis = mx.MixRun(mx.MixProblem(*NE_AR, 0.4, scheme="sis", **kw), F=F12)
    cis = mx.MixRun(mx.MixProblem(*NE_AR, 0.4, scheme="cis", **kw), F=F12)
    assert sis.solve() and cis.solve()
    assert np.max(np.abs(sis.rates - cis.rates) / np.abs(cis.rates)) < 1.5e-2
    assert sis.iters < cis.iters
    assert sis.rates[0] > sis.rates[1] > 0.0        # the lighter species flows faster


def test_M8_2d_identical_species_cis_is_the_single_species_duct_cis():
    kw = dict(delta=0.7, nv=8, vmax=6.0, M=8, scheme="cis")
    mr = mx.MixRun(mx.MixProblem(1.0, 1.0, 0.3, dim=2, nx=5, ny=4, width=1.5, **kw))
    sp = solver.Run(solver.Problem(dim=2, nx=5, ny=4, width=1.5, **kw))
    for _ in range(3):
        mr.step()
        sp.step()
    for a, chi in ((0, 0.3), (1, 0.7)):
        assert np.max(np.abs(mr.h[a] - chi * sp.h)) < 1e-13 * np.max(np.abs(sp.h))


def test_porous_sweep_exact_without_solids_and_geometry():
    """The periodic sweep converges to the exact uniform solution h = rhs / nu when nothing is
    solid; the staircase's solid area and the interior cells of the correction are as stated."""
    F = fsm.FSM(8, 5.0, 8)
    rng = np.random.default_rng(5)
    nu = 0.5 + rng.random(F.V1.shape)
    rhs = np.broadcast_to(rng.standard_normal(F.V1.shape), (6, 6) + F.V1.shape).copy()
    solid = np.zeros((6, 6), dtype=bool)
    h = np.zeros_like(rhs)
    for _ in range(400):
        h = mx.sweep_porous(rhs, nu, F.V1, F.V2, solid, h)
    assert np.max(np.abs(h - rhs / nu)) < 1e-10 * np.max(np.abs(rhs / nu))
    s = mx.porous_solid(100, 0.4)
    assert abs(s.mean() - 0.4) < 0.01
    inner = mx.porous_interior(s)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            assert not np.any(inner & np.roll(s, (-di, -dj), axis=(0, 1)))


def test_porous_solution_is_symmetric():
    """The converged flow in the unit cell has the cell's mirror and diagonal symmetries
    (exactly: the periodic scheme does, whatever the sweep order), and the lighter species
    flows faster."""
    F = mx.MixFSM(mx.Mixture(*NE_AR, 0.5), 8, 5.0, 8, R=3.75)
    kw = dict(delta=5.0, nv=8, vmax=5.0, M=8, R=3.75, eps=1e-11, max_iter=600, dim=2, nx=10, ny=10, solid=0.4)
    run = mx.MixRun(mx.MixProblem(*NE_AR, 0.5, **kw), F=F)
    assert run.solve()
    for U in run.U:
        s = np.max(np.abs(U))
        for V in (U[::-1, :], U[:, ::-1], U.T):
            assert np.max(np.abs(U - V)) < 1e-9 * s
    assert run.rates[0] > run.rates[1] > 0.0


def test_porous_poisson_reproduces_a_periodic_discrete_eigenfunction():
    """The interior Poisson solve of the porous correction against a manufactured solution:
    U = cos(2 pi x) + 0.5 sin(4 pi y) is an eigenfunction of the periodic five-point Laplacian
    (eigenvalues (2 cos(2 pi k d) - 2) / d^2 per axis), so with U held on the non-interior cells
    the solve must return it on the interior to rounding (the diagonal, the neighbour
    couplings, the wrap across the cell's sides and the ring terms all enter)."""
    n = 24
    d = 1.0 / n
    c = (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(c, c, indexing="ij")
    U = np.cos(2 * np.pi * X) + 0.5 * np.sin(4 * np.pi * Y)
    lam1 = (2 * np.cos(2 * np.pi * d) - 2) / d ** 2
    lam2 = (2 * np.cos(4 * np.pi * d) - 2) / d ** 2
    lap = lam1 * np.cos(2 * np.pi * X) + lam2 * 0.5 * np.sin(4 * np.pi * Y)
    inner = mx.porous_interior(mx.porous_solid(n, 0.3))
    assert inner.sum() > 100 and (~inner).sum() > 50
    Uh = np.where(inner, 0.0, U)
    got = mx.porous_poisson(inner, Uh, lap)
    assert np.max(np.abs(got - U)) < 1e-12


def test_duct_poisson_reproduces_a_quadratic():
    """The duct correction's Poisson solve (chi lap U = rhs on the interior, U held on the ring)
    against U = x^2 + 3 y^2 - x y, whose five-point differences are exact: lap U = 8 with
    unequal spacings width / nx and 1 / ny."""
    from types import SimpleNamespace
    nx, ny, width, chi = 9, 7, 1.5, 0.37
    x = (np.arange(nx) + 0.5) * width / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y, indexing="ij")
    U = X ** 2 + 3 * Y ** 2 - X * Y
    Uh = U.copy()
    Uh[1:-1, 1:-1] = 0.0
    rhs = np.full((nx - 2, ny - 2), 8.0 * chi)
    got = mx.MixRun.poisson(SimpleNamespace(pb=SimpleNamespace(width=width)), Uh, rhs, chi)
    assert np.max(np.abs(got - U)) < 1e-12


def test_march_integrates_a_linear_profile_exactly():
    """The once-integrated diffusion equation is marched from the wall with the sweep's upwind
    differences (two points at the first node, three after), which are exact for a linear
    profile: dY/dx = 3 with Y(x0) = 2 gives Y = 2 + 3 (x - x0) on the clustered nodes."""
    from types import SimpleNamespace
    from oracle import transport
    x = transport.nodes_clustered(40)
    Y = mx.MixRun.march(SimpleNamespace(x=x), 2.0, np.full(len(x), 3.0))
    assert np.max(np.abs(Y - (2.0 + 3.0 * (x - x[0])))) < 1e-12
