"""Pins of the oracle's moment functions against closed forms of Gaussian moments (per axis
<v^2> = 1/2, <v^4> = 3/4, <v^6> = 15/8 under exp(-v^2)/sqrt(pi); the midpoint grid on [-6, 6]^3
integrates them to ~1e-14 at 32 points per axis): the macroscopic quantities of Sec. 2 (U3, q3, F201/4, F021/4,
F111/4), the L-moments of the N-penalised diffusion equation, and the flow rates."""
import numpy as np
import pytest

from oracle import fsm, solver


@pytest.fixture(scope="module")
def F():
    return fsm.FSM(32, 6.0, 8, 4.5)  # dv = 0.375: Gaussian moments to ~1e-14


def mom(F, h):
    return np.array([float(x) for x in solver.cell_moments(F, h)])


def test_moments_of_the_flow_velocity_mode(F):
    # h = v3 f_eq: U3 = <v3^2> = 1/2; q3 = <c^2 v3^2> - 5/2 <v3^2> = 5/4 - 5/4 = 0;
    # F201/4 = 2<v1^2 v3^2> - <v3^2> = 0; likewise F021/4; F111/4 = 0 by parity
    assert np.allclose(mom(F, F.V3 * F.feq), [0.5, 0.0, 0.0, 0.0, 0.0], atol=1e-12)


def test_moments_of_shear_and_heat_modes(F):
    # h = v1^2 v3 f_eq: U3 = 1/4; F201/4 = 2<v1^4><v3^2> - <v1^2><v3^2> = 3/4 - 1/4 = 1/2;
    # F021/4 = 2<v2^2><v1^2><v3^2> - <v1^2><v3^2> = 0;
    # q3 = <c^2 v1^2 v3^2> - 5/2 <v1^2 v3^2> = (3/8 + 1/8 + 3/8) - 5/8 = 1/4
    U, q, W1, W2, X = mom(F, F.V1 ** 2 * F.V3 * F.feq)
    assert abs(U - 0.25) < 1e-12 and abs(W1 - 0.5) < 1e-12 and abs(W2) < 1e-12 and abs(X) < 1e-12
    assert abs(q - 0.25) < 1e-12
    # h = v1 v2 v3 f_eq: F111/4 = 2<v1^2 v2^2 v3^2> = 1/4, everything else 0 by parity
    assert np.allclose(mom(F, F.V1 * F.V2 * F.V3 * F.feq), [0, 0, 0, 0, 0.25], atol=1e-12)
    # h = c^2 v3 f_eq: q3 = <c^4 v3^2> - 5/2 <c^2 v3^2> = 35/8 - 25/8 = 5/4, U3 = 5/4
    U, q, *_ = mom(F, (F.V1 ** 2 + F.V2 ** 2 + F.V3 ** 2) * F.V3 * F.feq)
    assert abs(U - 1.25) < 1e-12 and abs(q - 1.25) < 1e-12


def test_l_moments_closed_forms(F):
    # with L h = 0: G1 = 2 N delta <v1^2 v3^2> = N delta / 2 for h = v1 v3 f_eq, G2 = 0
    h = F.V1 * F.V3 * F.feq
    G1, G2 = solver.l_moments(F, np.zeros_like(h), h, 3.0)
    assert abs(G1 - 1.5) < 1e-12 and abs(G2) < 1e-12
    # the flow-velocity mode is a collision invariant: L (v3 f_eq) = 0, and G = 0 by parity
    lp, L = F.apply(F.V3 * F.feq, 1.0)
    G1, G2 = solver.l_moments(F, L, F.V3 * F.feq, 1.25)
    assert abs(G1) < 1e-10 and abs(G2) < 1e-10


def test_flow_rates_trapezoid_exact_for_linear_profiles():
    x = np.sort(np.concatenate([[-0.5, 0.0], np.random.default_rng(1).uniform(-0.5, 0.0, 9)]))
    M, Q = solver.flow_rates_1d(np.ones_like(x), x, x)
    assert abs(M - 1.0) < 1e-14 and abs(Q - (-0.25)) < 1e-14  # 2 int 1 dx, 2 int x dx
