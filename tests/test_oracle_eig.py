"""Pins of the Fourier-mode convergence analysis (Sec. 2.3): the BGK closed form, and
the paper's qualitative findings for the LBE (CIS omega -> 1 as delta grows; SIS omega
saturates near 0.6, Sec. 4.2; both equal in the free-molecular limit)."""
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
