"""Discrete velocity space (oracle; test infrastructure only).

Velocities are normalised by the most probable speed (Sec. 2).  The paper leaves the
velocity discretisation to its FSM reference, so the grid is this reading: N points per
axis at cell midpoints of [-vmax, vmax], v_j = -vmax + (j + 1/2) dv, dv = 2 vmax / N.  The
grid is symmetric, has no v = 0 node and is periodic with period 2 vmax, which is what
the spectral collision operator assumes.

Index order of a velocity array is (i1, i2, i3) with i3 fastest.
"""
import numpy as np


def axis(nv, vmax):
    """1D midpoint nodes and spacing."""
    dv = 2.0 * vmax / nv
    return -vmax + (np.arange(nv) + 0.5) * dv, dv


def grid(nv, vmax):
    """Return (V1, V2, V3, dv): 3D arrays of the velocity components, shape (nv,)*3."""
    v, dv = axis(nv, vmax)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    return V1, V2, V3, dv


def feq(V1, V2, V3):
    """Equilibrium VDF f_eq = pi^(-3/2) exp(-|v|^2) (Sec. 2, first displayed equation)."""
    return np.exp(-(V1 * V1 + V2 * V2 + V3 * V3)) / np.pi ** 1.5


def source(V1, V2, V3, forcing):
    """Source term S with X_P = X_T = -1 (Sec. 2, equation for S).

    forcing 0 = Poiseuille:            S = v3 f_eq
    forcing 1 = thermal transpiration: S = v3 (|v|^2 - 5/2) f_eq
    """
    f = feq(V1, V2, V3)
    if forcing == 0:
        return V3 * f
    if forcing == 1:
        return V3 * (V1 * V1 + V2 * V2 + V3 * V3 - 2.5) * f
    raise ValueError("forcing must be 0 (Poiseuille) or 1 (thermal transpiration)")
