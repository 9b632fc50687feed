"""Fourier-mode convergence analysis of CIS and SIS (oracle; test infrastructure only).

Sec. 2.3: a system periodic in x1 with one mode exp(2 pi i x1).  For the CIS
(Eq. conv_iteration) the error e obeys e^(k+1) = L+(e^(k)) / (nu_eq + 2 pi i v1).  For the
SIS (Eq. acceleratred_iteration and the U3 formula after it) the half step is the same,
then U3^(k+1) = (-2 pi i A1 - 4 pi^2 A2) / (4 pi^2) with A1 = 2 ∫ v1 v3 (L + N delta) e^(k)
and A2 = ∫ (2 v1^2 - 1) v3 e^(k+1/2) (the N-penalised form; the source is dropped because
the error iteration is homogeneous), and the correction of Eq. guided.  The convergence
factor omega is the modulus of the dominant eigenvalue of that linear map; the paper fits
U3(k) = U_inf + C exp(-lambda k), omega = exp(-lambda), which power iteration reproduces.

Pins: with L replaced by the linearized BGK operator delta (2 U3 v3 f_eq - h) (collision
frequency 1), the CIS map is rank one and omega = delta^2 ∫ pi^-1/2 exp(-v^2) /
(delta^2 + 4 pi^2 v^2) dv; the SIS map has rank two (its range is spanned by the half step's
shape and v3 f_eq) and its eigenvalues solve a quadratic whose coefficients are 1D integrals
of the same kind (tests/test_oracle_eig.py).  Both maps take the operator as an argument so
that the pins exercise the same code as the hard-sphere analysis.
"""
import numpy as np


def _lplus(F, e, delta):
    """L+ applied to complex e (L+ is real-linear)."""
    lr, Lr = F.apply(e.real, delta)
    li, Li = F.apply(e.imag, delta)
    return lr + 1j * li, Lr + 1j * Li


def fsm_operator(F, delta):
    """e -> (L+ e, L e, nu) for the hard-sphere operator of the fast spectral method."""
    def op(e):
        lp, Le = _lplus(F, e, delta)
        return lp, Le, F.nu
    return op


def bgk_operator(F, delta):
    """e -> (L+ e, L e, nu) for the linearized BGK operator L e = delta (2 U3(e) v3 f_eq - e),
    U3(e) = ∫ v3 e (collision frequency 1)."""
    w = F.dv ** 3

    def op(e):
        lp = delta * 2.0 * np.sum(F.V3 * e) * w * F.V3 * F.feq
        return lp, lp - delta * e, 1.0
    return op


def cis_map(F, e, delta, op=None):
    lp, _, nu = (op or fsm_operator(F, delta))(e)
    return lp / (delta * nu + 2j * np.pi * F.V1)


def sis_map(F, e, delta, N=1.25, op=None):
    w = F.dv ** 3
    lp, Le, nu = (op or fsm_operator(F, delta))(e)
    eh = lp / (delta * nu + 2j * np.pi * F.V1)
    A1 = 2.0 * np.sum(F.V1 * F.V3 * (Le + N * delta * e)) * w
    A2 = np.sum((2.0 * F.V1 ** 2 - 1.0) * F.V3 * eh) * w
    Uh = np.sum(F.V3 * eh) * w
    Un = (-2j * np.pi * A1 - 4.0 * np.pi ** 2 * A2) / (4.0 * np.pi ** 2)
    return eh + 2.0 * (Un - Uh) * F.V3 * F.feq


def bgk_cis_map(F, e, delta):
    w = F.dv ** 3
    U = np.sum(F.V3 * e) * w
    return delta * 2.0 * U * F.V3 * F.feq / (delta + 2j * np.pi * F.V1)


def omega(step, F, iters=60, seed=0):
    """Dominant |eigenvalue| by power iteration restricted to errors odd in v3 (the
    parity of Poiseuille and thermal-transpiration solutions; the even-in-v3 collision
    invariants never enter those flows)."""
    rng = np.random.default_rng(seed)
    n = rng.standard_normal(F.feq.shape)
    n = 0.5 * (n + n[..., ::-1])                  # even in v3, so e is odd in v3
    e = F.feq * F.V3 * (1.0 + 0.3 * n)
    e = e.astype(complex)
    r = 0.0
    for _ in range(iters):
        n0 = np.sqrt(np.sum(np.abs(e) ** 2))
        e = step(e) / n0
        r = np.sqrt(np.sum(np.abs(e) ** 2))
    return float(r)


def power_ratios(step, e0, iters, odd_v3=True):
    """Power iteration from a given start vector: e_{k+1} = P step(e_k) / |e_k|, returning the
    ratios |e_{k+1}| (they converge to the modulus of the dominant eigenvalue).  With odd_v3,
    P projects onto functions odd in v3 (the parity of the plate and duct errors), so that
    rounding cannot seed the even, density-type modes that the SIS does not accelerate."""
    e = np.asarray(e0).astype(complex)
    out = []
    for _ in range(iters):
        n0 = np.sqrt(np.sum(np.abs(e) ** 2))
        e = step(e) / n0
        if odd_v3:
            e = 0.5 * (e - e[..., ::-1])
        out.append(float(np.sqrt(np.sum(np.abs(e) ** 2))))
    return np.array(out)
