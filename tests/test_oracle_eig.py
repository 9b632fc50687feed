"""Pins of the Fourier-mode convergence analysis (Sec. 2.3): the BGK closed forms of the CIS
and SIS maps, and the paper's qualitative findings for the LBE (CIS omega -> 1 as delta grows;
SIS omega saturates near 0.6, Sec. 4.2; both equal in the free-molecular limit)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import eig, fsm


@pytest.fixture(scope="module")
def F16():
    return fsm.FSM(16, 6.0, 16)


def test_P11_bgk_cis_eigenvalue_closed_form(F16):
    for d in (10.0, 30.0):
        ex = quad(lambda v: d * d * np.exp(-v * v) / np.sqrt(np.pi) / (d * d + 4 * np.pi ** 2 * v * v),
                  -np.inf, np.inf)[0]
        om = eig.omega(lambda e: eig.bgk_cis_map(F16, e, d), F16, iters=15)
        assert abs(om - ex) < 2e-3 * ex, (d, om, ex)


def test_P12_lbe_cis_vs_sis_eigenvalues(F16):
    om = {}
    for d in (0.1, 10.0, 100.0):
        om[d] = (eig.omega(lambda e: eig.cis_map(F16, e, d), F16, iters=30),
                 eig.omega(lambda e: eig.sis_map(F16, e, d), F16, iters=30))
    # free-molecular: both fast
    assert om[0.1][0] < 0.05 and om[0.1][1] < 0.05
    # near continuum: CIS stalls, SIS stays near the paper's omega ~ 0.6
    assert om[100.0][0] > 0.99
    assert om[10.0][1] < 0.5 * om[10.0][0]
    assert 0.45 < om[100.0][1] < 0.7


def test_power_ratios_from_given_start_reach_bgk_closed_form(F16):
    """The start-vector form of the power iteration (used to compare with the GPU driver)
    converges to the same BGK closed-form eigenvalue as P11."""
    from paper_1612_04488_gb300 import workloads
    d = 10.0
    ex = quad(lambda v: d * d * np.exp(-v * v) / np.sqrt(np.pi) / (d * d + 4 * np.pi ** 2 * v * v),
              -np.inf, np.inf)[0]
    r = eig.power_ratios(lambda e: eig.bgk_cis_map(F16, e, d), workloads.fourier_start(16, 6.0, seed=2), 15)
    assert abs(r[-1] - ex) < 2e-3 * ex, (r[-1], ex)


def _bgk_sis_closed_form(d, N):
    """Dominant |eigenvalue| of the SIS map with the BGK operator, from the map's action on
    the functionals U(e) = ∫ v3 e and S(e) = ∫ v1 v3 e.  The half step is U(e) g with
    g = 2 d v3 f_eq / (d + 2 pi i v1); A1 = 2 d (N - 1) S(e) (the gain's v1-odd part
    vanishes); the correction leaves e' = U(e) phi + c S(e) v3 f_eq with
    c = -2 i d (N - 1) / pi and U(phi) = -A2(g).  With g1(v) = pi^-1/2 exp(-v^2) /
    (d^2 + 4 pi^2 v^2), K = ∫ (2v^2 - 1) g1 and J = ∫ v^2 g1: U(phi) = -d^2 K,
    S(g) = -2 pi i d J, U(v3 f_eq) = 1/2, S(v3 f_eq) = 0, so lambda^2 + d^2 K lambda
    + 2 d^2 (N - 1) J = 0."""
    g1 = lambda v: np.exp(-v * v) / np.sqrt(np.pi) / (d * d + 4 * np.pi ** 2 * v * v)
    K = quad(lambda v: (2 * v * v - 1) * g1(v), -np.inf, np.inf)[0]
    J = quad(lambda v: v * v * g1(v), -np.inf, np.inf)[0]
    return max(abs(x) for x in np.roots([1.0, d * d * K, 2 * d * d * (N - 1) * J]))


def test_P16_bgk_sis_eigenvalue_closed_form(F16):
    """The oracle's SIS map, driven by the BGK operator, against the closed form: the
    geometric mean of the power-iteration ratios (the two eigenvalues can be a complex pair of
    equal modulus, so single ratios oscillate).  N != 1 exercises the A1 term (sign and
    2 pi factor), delta sets the balance of the A2 term and the correction."""
    for d, N in ((10.0, 1.0), (10.0, 1.25), (10.0, 2.0), (30.0, 1.25), (30.0, 2.0)):
        op = eig.bgk_operator(F16, d)
        r = eig.power_ratios(lambda e: eig.sis_map(F16, e, d, N=N, op=op), (F16.feq * F16.V3).astype(complex),
                             200)
        om = float(np.exp(np.mean(np.log(r[100:]))))
        ex = _bgk_sis_closed_form(d, N)
        assert abs(om - ex) < 0.02 * ex, (d, N, om, ex)


def test_cis_map_with_bgk_operator_is_the_bgk_map(F16):
    rng = np.random.default_rng(4)
    e = (rng.standard_normal(F16.feq.shape) * F16.feq).astype(complex)
    a = eig.cis_map(F16, e, 10.0, op=eig.bgk_operator(F16, 10.0))
    b = eig.bgk_cis_map(F16, e, 10.0)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-15 * np.abs(b).max())
