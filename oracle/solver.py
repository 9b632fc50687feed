"""CIS and SIS for the single-species LBE (oracle; test infrastructure only).

CIS, Sec. 2 Eq. LBE_iteration: nu_eq h^(k+1) + v.grad h^(k+1) = L+(h^(k)) + S.

SIS, Sec. 2.2 with the N-penalised split L = (L + N delta h) - N delta h of the abstract /
Sec. 2.5 footnote to Eq. LBE_penlty.  One iteration from h^(k):
  1. L-evaluation: rhs = L+ h^(k) + S, and G_j = 2 ∫ v_j v3 (L h^(k) + N delta h^(k)) dv.
  2. Kinetic half step (Eq. syn_LBE): h^(k+1/2) by the upwind sweep.
  3. Moments of h^(k+1/2): U3, q3, W1 = F201/4 = ∫(2v1^2-1) v3 h, W2 = F021/4,
     X12 = F111/4 = 2 ∫ v1 v2 v3 h.
  4. Diffusion correction of U3.
     1D (Eq. first_order with the N-penalty): with Y = U3 + W1,
        dY/dx1 = -N delta sigma x1 + G1,  Y(x0) = U3^(k+1/2)(x0) + W1(x0),
     where P13 = x1 for Poiseuille (sigma = 1) and 0 for thermal transpiration
     (sigma = 0), marched with the same upwind stencil as the sweep (first order at the
     wall).  U3^(k+1) = Y - W1.
     2D (Eq. diffusion_LBE with the N-penalty): five-point Laplacian,
        lap U3 = -N delta sigma - (d11 W1 + 2 d12 X12 + d22 W2) + d1 G1 + d2 G2
     on interior cells, U3 = U3^(k+1/2) on the wall-adjacent ring ("near the boundary",
     Sec. 2.2 third bullet); central differences for the moment terms; solved exactly
     (dense LU).
  5. Correction (Eq. guided): h^(k+1) = h^(k+1/2) + 2 (U3^(k+1) - U3^(k+1/2)) v3 f_eq.
  6. Flow rates of h^(k+1): 1D M = 2 ∫_{-1/2}^0 U3 dx1, Q = 2 ∫ q3 dx1 (trapezoid on the
     nodes, Sec. 2.4); 2D: cell averages (the M, Q equation of Sec. 2).
Stop when the relative changes of M and Q between iterations are both < eps (Sec. 2.4).
N <= 0 selects N = nu_bar / delta = 1.25 for hard spheres (Sec. 2.5).

Pins: tests/test_oracle_solver.py (CIS and SIS reach the same solution; Table 1 hard-sphere
values; Onsager symmetry; the BGK closed-form iteration eigenvalue; kappa -> 1/12).
"""
import numpy as np

from . import fsm as fsm_mod
from . import transport, velocity


HS_NU_BAR_OVER_DELTA = 1.25


class Problem:
    """Plain parameter record (see include/lbe.h for the meaning of each field)."""

    def __init__(self, dim=1, ns=20, grid="uniform", nx=64, ny=32, width=2.0, delta=1.0,
                 N=0.0, nv=16, vmax=6.0, M=16, R=0.0, forcing=0, scheme="sis", eps=1e-8,
                 max_iter=500):
        self.dim, self.ns, self.grid = dim, ns, grid
        self.nx, self.ny, self.width = nx, ny, width
        self.delta, self.N = float(delta), float(N)
        self.nv, self.vmax, self.M, self.R = nv, float(vmax), M, float(R)
        self.forcing, self.scheme = forcing, scheme
        self.eps, self.max_iter = eps, max_iter

    def n_delta(self):
        n = self.N if self.N > 0 else HS_NU_BAR_OVER_DELTA
        return n * self.delta


def make_fsm(pb):
    return fsm_mod.FSM(pb.nv, pb.vmax, pb.M, pb.R if pb.R > 0 else None)


def nodes_1d(pb):
    if pb.grid == "uniform":
        return transport.nodes_uniform(pb.ns)
    if pb.grid == "clustered":
        return transport.nodes_clustered(pb.ns)
    raise ValueError(pb.grid)


def cell_moments(F, h):
    """Moments over the trailing velocity axes: U3, q3, W1, W2, X12."""
    w = F.dv ** 3
    c2 = F.V1 ** 2 + F.V2 ** 2 + F.V3 ** 2
    ax = (-3, -2, -1)
    U = np.sum(F.V3 * h, axis=ax) * w
    q = np.sum((c2 - 2.5) * F.V3 * h, axis=ax) * w
    W1 = np.sum((2.0 * F.V1 ** 2 - 1.0) * F.V3 * h, axis=ax) * w
    W2 = np.sum((2.0 * F.V2 ** 2 - 1.0) * F.V3 * h, axis=ax) * w
    X12 = 2.0 * np.sum(F.V1 * F.V2 * F.V3 * h, axis=ax) * w
    return U, q, W1, W2, X12


def l_moments(F, Lh, h, n_delta):
    """G_j = 2 ∫ v_j v3 (L h + N delta h) dv, j = 1, 2."""
    w = F.dv ** 3
    t = Lh + n_delta * h
    ax = (-3, -2, -1)
    return (2.0 * np.sum(F.V1 * F.V3 * t, axis=ax) * w,
            2.0 * np.sum(F.V2 * F.V3 * t, axis=ax) * w)


def flow_rates_1d(U, q, x):
    return 2.0 * np.trapezoid(U, x), 2.0 * np.trapezoid(q, x)


def diffusion_1d(Uh, W1, G1, x, n_delta, sigma):
    """March dY/dx = -N delta sigma x + G1 from the wall, Y = U + W1; return U^(k+1)."""
    a, b, c = transport.march_coeffs(x)
    Y = np.zeros(len(x))
    Y[0] = Uh[0] + W1[0]
    for i in range(1, len(x)):
        r = -n_delta * sigma * x[i] + G1[i] - b[i] * Y[i - 1]
        if i >= 2:
            r -= c[i] * Y[i - 2]
        Y[i] = r / a[i]
    return Y - W1


def poisson_2d(Uh, W1, W2, X12, G1, G2, width, n_delta, sigma):
    """Five-point solve of Eq. diffusion_LBE (N-penalised) with the ring U = Uh."""
    nx, ny = Uh.shape
    dx, dy = width / nx, 1.0 / ny
    U = Uh.copy()
    ii = np.arange(1, nx - 1)
    jj = np.arange(1, ny - 1)
    I, J = np.meshgrid(ii, jj, indexing="ij")
    rhs = (-n_delta * sigma
           - (W1[I + 1, J] - 2.0 * W1[I, J] + W1[I - 1, J]) / dx ** 2
           - 2.0 * (X12[I + 1, J + 1] - X12[I + 1, J - 1] - X12[I - 1, J + 1]
                    + X12[I - 1, J - 1]) / (4.0 * dx * dy)
           - (W2[I, J + 1] - 2.0 * W2[I, J] + W2[I, J - 1]) / dy ** 2
           + (G1[I + 1, J] - G1[I - 1, J]) / (2.0 * dx)
           + (G2[I, J + 1] - G2[I, J - 1]) / (2.0 * dy))
    mx, my = nx - 2, ny - 2
    n = mx * my
    A = np.zeros((n, n))
    b = rhs.reshape(-1).copy()
    for p in range(mx):
        for q in range(my):
            k = p * my + q
            A[k, k] = -2.0 / dx ** 2 - 2.0 / dy ** 2
            for dp, dq, wgt in ((1, 0, 1.0 / dx ** 2), (-1, 0, 1.0 / dx ** 2),
                                (0, 1, 1.0 / dy ** 2), (0, -1, 1.0 / dy ** 2)):
                pp, qq = p + dp, q + dq
                if 0 <= pp < mx and 0 <= qq < my:
                    A[k, pp * my + qq] = wgt
                else:
                    b[k] -= wgt * Uh[pp + 1, qq + 1]
    U[1:-1, 1:-1] = np.linalg.solve(A, b).reshape(mx, my)
    return U


class Run:
    """Iteration state and history of one solve."""

    def __init__(self, pb, F=None):
        self.pb = pb
        self.F = make_fsm(pb) if F is None else F
        F = self.F
        self.S = velocity.source(F.V1, F.V2, F.V3, pb.forcing)
        self.nu = pb.delta * F.nu
        if pb.dim == 1:
            self.x = nodes_1d(pb)
            shape = (len(self.x),) + F.V1.shape
        else:
            shape = (pb.nx, pb.ny) + F.V1.shape
        self.h = np.zeros(shape)
        self.M = 0.0
        self.Q = 0.0
        self.iters = 0
        self.history = []
        self.U = None

    def sweep(self, rhs):
        F, pb = self.F, self.pb
        if pb.dim == 1:
            return transport.sweep_1d(rhs, self.nu, F.V1, self.x)
        return transport.sweep_2d(rhs, self.nu, F.V1, F.V2, pb.nx, pb.ny, pb.width)

    def rates(self, U, q):
        if self.pb.dim == 1:
            return flow_rates_1d(U, q, self.x)
        return float(np.mean(U)), float(np.mean(q))

    def step(self):
        """One CIS or SIS iteration; returns (M, Q) of the new iterate."""
        F, pb = self.F, self.pb
        nd = pb.n_delta()
        sigma = 1.0 if pb.forcing == 0 else 0.0
        lplus, Lh = F.apply(self.h, pb.delta)
        rhs = lplus + self.S
        hh = self.sweep(rhs)
        if pb.scheme == "cis":
            self.h = hh
            U, q, *_ = cell_moments(F, hh)
        else:
            G1, G2 = l_moments(F, Lh, self.h, nd)
            Uh, qh, W1, W2, X12 = cell_moments(F, hh)
            if pb.dim == 1:
                Un = diffusion_1d(Uh, W1, G1, self.x, nd, sigma)
            else:
                Un = poisson_2d(Uh, W1, W2, X12, G1, G2, pb.width, nd, sigma)
            dU = Un - Uh
            self.h = hh + 2.0 * dU[(...,) + (None,) * 3] * F.V3 * F.feq
            U, q, *_ = cell_moments(F, self.h)
        self.U = U
        Mn, Qn = self.rates(U, q)
        self.iters += 1
        self.history.append((Mn, Qn))
        return Mn, Qn

    def solve(self, eps=None, max_iter=None):
        """Iterate until both relative changes are < eps (Sec. 2.4).  Returns converged?"""
        eps = self.pb.eps if eps is None else eps
        max_iter = self.pb.max_iter if max_iter is None else max_iter
        while self.iters < max_iter:
            Mo, Qo = self.M, self.Q
            self.M, self.Q = self.step()
            if (abs(self.M - Mo) < eps * abs(self.M)) and (abs(self.Q - Qo) < eps * abs(self.Q)):
                return True
        return False


def solve(pb, F=None):
    r = Run(pb, F)
    ok = r.solve()
    return r, ok
