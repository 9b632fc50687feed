"""Pins of the oracle's fast-spectral collision operator against facts that do not come
from the oracle itself: the explicit spectral convolution, a brute-force quadrature of the
collision integral, the closed-form hard-sphere collision frequency, the Maxwellian and
collision-invariant identities, symmetry/negativity of L, and nu_bar/delta = 1.25.
"""
import numpy as np
import pytest
from scipy.special import erf

from oracle import fsm


@pytest.fixture(scope="module")
def F32():
    return fsm.FSM(32, 6.0, 32, R=4.5)


@pytest.fixture(scope="module")
def F16():
    return fsm.FSM(16, 6.0, 16)


def test_directions_rule():
    # the hemisphere rule integrates polynomials in mu exactly and sums to 2 pi
    for M in (4, 8, 16, 32, 64):
        e, w = fsm.directions(M)
        assert e.shape == (M, 3)
        assert np.allclose(np.sum(e * e, 1), 1.0)
        assert np.all(e[:, 2] > 0)
        assert abs(np.sum(w) - 2 * np.pi) < 1e-13
        # ∫_hemisphere mu^2 = 2 pi / 3 ; ∫ e1^2 = 2 pi / 3 (needs >= 4 azimuths)
        assert abs(np.sum(w * e[:, 2] ** 2) - 2 * np.pi / 3) < 1e-12
        if M >= 8:
            assert abs(np.sum(w * e[:, 0] ** 2) - 2 * np.pi / 3) < 1e-12


def test_phi_psi_closed_forms():
    # phi(s) = 2∫_0^R ρ cos(ρ s) dρ and psi(a) = ∫_0^{2π} phi(a cos t) dt, by quadrature
    R = 4.5
    x, w = np.polynomial.legendre.leggauss(200)
    rho = 0.5 * R * (x + 1)
    wr = 0.5 * R * w
    for s in (0.0, 1e-4, 0.3, 2.0, 7.5):
        ref = 2 * np.sum(wr * rho * np.cos(rho * s))
        assert abs(fsm.phi(np.array([s]), R)[0] - ref) < 1e-10 * R * R
    t = (np.arange(400) + 0.5) * 2 * np.pi / 400
    for a in (0.0, 1e-4, 0.7, 3.0, 6.0):
        ref = np.sum(fsm.phi(a * np.cos(t), R)) * 2 * np.pi / 400
        assert abs(fsm.psi(np.array([a]), R)[0] - ref) < 1e-9 * R * R


def test_P1_fft_gain_equals_explicit_spectral_sum():
    F = fsm.FSM(8, 4.0, 8)
    rng = np.random.default_rng(7)
    h = F.feq * rng.standard_normal(F.feq.shape)
    fast = F.gain(h)
    slow = F.direct_spectral_gain(F.feq, h) + F.direct_spectral_gain(h, F.feq)
    assert np.max(np.abs(fast - slow)) <= 1e-12 * np.max(np.abs(slow))


def _poly_h(p):
    v1, v2, v3 = p[..., 0], p[..., 1], p[..., 2]
    return (np.exp(-np.sum(p * p, -1)) / np.pi ** 1.5
            * (v3 + 0.5 * v1 * v3 + 0.3 * v3 * (v1 * v1 + v2 * v2 + v3 * v3) + 0.2 * v1))


def test_P2_fsm_matches_bruteforce_collision_integral(F32):
    h = _poly_h(np.stack([F32.V1, F32.V2, F32.V3], -1))
    _, L = F32.apply(h[None], delta=2.0)
    L = L[0]
    scale = np.max(np.abs(L))
    for idx in [(16, 16, 16), (18, 16, 20)]:
        v = np.array([F32.V1[idx], F32.V2[idx], F32.V3[idx]])
        bf = fsm.brute_force_L(_poly_h, v, delta=2.0, n_vs=36, n_sphere=10)
        assert abs(L[idx] - bf) < 2e-4 * scale, (idx, L[idx], bf)


def test_P3_nu_matches_hard_sphere_closed_form(F32):
    K = fsm.kernel_K(1.0)
    vn = np.sqrt(F32.V1 ** 2 + F32.V2 ** 2 + F32.V3 ** 2)
    cf = K * (np.exp(-vn ** 2) / np.sqrt(np.pi) + (vn + 1 / (2 * vn)) * erf(vn))
    m = vn <= 2.0
    # angular quadrature (M = 32) and truncation at R limit the agreement
    assert np.max(np.abs(F32.nu[m] - cf[m]) / cf[m]) < 2e-3
    # with many directions and the wider cutoff R = 2S the remaining gap is truncation
    Fh = fsm.FSM(24, 6.0, 128)
    vn = np.sqrt(Fh.V1 ** 2 + Fh.V2 ** 2 + Fh.V3 ** 2)
    cf = K * (np.exp(-vn ** 2) / np.sqrt(np.pi) + (vn + 1 / (2 * vn)) * erf(vn))
    m = vn <= 2.0
    assert np.max(np.abs(Fh.nu[m] - cf[m]) / cf[m]) < 5e-5


def test_P4_maxwellian_gain_equals_loss(F32):
    g = 0.5 * F32.gain(F32.feq)        # gain(h) is symmetrised: h = f_eq gives 2 Q+(f,f)
    ref = F32.nu * F32.feq
    assert np.max(np.abs(g - ref)) < 1e-8 * np.max(ref)


@pytest.mark.parametrize("which", ["1", "v1", "v2", "v3", "v2sq"])
def test_P5_collision_invariants_in_null_space(F32, which):
    V = {"1": 1.0 + 0 * F32.V1, "v1": F32.V1, "v2": F32.V2, "v3": F32.V3,
         "v2sq": F32.V1 ** 2 + F32.V2 ** 2 + F32.V3 ** 2}[which]
    h = F32.feq * V
    _, L = F32.apply(h)
    tol = 5e-7 if which == "v2sq" else 5e-8
    assert np.max(np.abs(L)) < tol * np.max(np.abs(F32.nu * h))


def test_P6_conservation_moments_of_Lh(F32):
    h = _poly_h(np.stack([F32.V1, F32.V2, F32.V3], -1)) + F32.feq * np.cos(F32.V1) * F32.V3
    _, L = F32.apply(h, delta=3.0)
    ref = np.sum(np.abs(3.0 * F32.nu * h))
    for psi_ in (1.0 + 0 * F32.V1, F32.V1, F32.V2, F32.V3,
                 F32.V1 ** 2 + F32.V2 ** 2 + F32.V3 ** 2):
        assert abs(np.sum(psi_ * L)) < 1e-6 * ref
    # and the shear moment is not conserved (guards against L == 0)
    assert abs(np.sum(F32.V1 * F32.V3 * L)) > 1e-2 * np.sum(np.abs(F32.V1 * F32.V3 * L))


def test_P7_symmetric_and_dissipative(F32):
    rng = np.random.default_rng(1)
    F = F32
    mons = [1 + 0 * F.V1, F.V1, F.V2, F.V3, F.V1 * F.V2, F.V1 * F.V3, F.V2 * F.V3,
            F.V1 ** 2, F.V3 ** 3, F.V1 * F.V2 * F.V3]

    def rand_h():
        c = rng.standard_normal(len(mons))
        return F.feq * sum(ci * m for ci, m in zip(c, mons))

    for _ in range(2):
        g, h = rand_h(), rand_h()
        _, Lg = F.apply(g)
        _, Lh = F.apply(h)
        a = np.sum(g * Lh / F.feq)
        b = np.sum(Lg * h / F.feq)
        assert abs(a - b) < 1e-5 * max(abs(a), abs(b))
        assert np.sum(h * Lh / F.feq) < 0.0


def test_P9_nu_bar(F16, F32):
    assert abs(fsm.kernel_K(1.0) * 2 * np.sqrt(2 / np.pi) - 1.25) < 1e-15
    assert abs(F32.nu_bar(1.0) - 1.25) < 2e-4      # truncation at R = 4.5
    assert abs(F16.nu_bar(2.0) - 2.5) < 2e-4


def test_operator_linear_in_delta(F16):
    rng = np.random.default_rng(3)
    h = F16.feq * rng.standard_normal(F16.feq.shape)
    lp1, L1 = F16.apply(h, 1.0)
    lp3, L3 = F16.apply(h, 3.0)
    assert np.allclose(lp3, 3 * lp1, rtol=1e-13, atol=1e-16)
    assert np.allclose(L3, 3 * L1, rtol=1e-13, atol=1e-16)
