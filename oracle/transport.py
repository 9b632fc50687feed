"""Upwind finite-difference transport sweeps (oracle; test infrastructure only).

Each sweep solves, for every discrete velocity, the steady transport equation of
Eq. LBE_iteration / Eq. syn_LBE,
    nu h + v1 dh/dx1 (+ v2 dh/dx2) = rhs,
with the "second-order upwind finite difference" of Sec. 2 (below Eq. LBE_iteration):
the three-point backward (upwind) derivative on possibly non-uniform nodes, first order at
the first node after an inflow boundary.

1D plates (Sec. 2.4): nodes x_0 = -1/2 (diffuse wall) ... x_Ns = 0 (specular symmetry
plane).  Diffuse wall: incoming h = 0 for v1 > 0 (the paper's "h(v2>0)=0" is read as
v1 > 0; h is odd in v3 so the wall density perturbation vanishes).  Symmetry plane:
h(x_Ns, v1<0) = h(x_Ns, -v1); the v1 < 0 march uses the mirror ghost node
x_{Ns+1} = -x_{Ns-1} with h(x_{Ns+1}, v1) = h(x_{Ns-1}, -v1), so every interior node is
second order.

2D ducts: cell centres of a uniform nx x ny grid on [0, a] x [0, 1], diffuse walls on all
four faces (incoming h = 0 on the face).  The march in each direction starts at the inflow
face, which is an extra node at distance dx/2 carrying h = 0; the first cell is first
order, the rest use the three-point backward formula (which reaches the face node at the
second cell).

Node grids: uniform, or the wall-clustered map of Sec. 2.4,
x = (10 - 15 s + 6 s^2) s^3 - 1/2, s = (0 .. Ns) / (2 Ns).

Pins: tests/test_oracle_transport.py (exactness for linear-in-x solutions, second-order
convergence, the 1.24e-6 smallest section, free-molecular duct vs ray lengths).
"""
import numpy as np


def nodes_uniform(ns):
    return -0.5 + 0.5 * np.arange(ns + 1) / ns


def nodes_clustered(ns):
    """Sec. 2.4: x1 = (10 - 15 s + 6 s^2) s^3 - 0.5, s = (0, 1, ..., Ns) / (2 Ns)."""
    s = np.arange(ns + 1) / (2.0 * ns)
    return (10.0 - 15.0 * s + 6.0 * s * s) * s ** 3 - 0.5


def backward_coeffs(xm2, xm1, x0):
    """d/dx at x0 from values at (x0, xm1, xm2): a f0 + b f1 + c f2 (Lagrange)."""
    h1 = x0 - xm1
    h2 = xm1 - xm2
    a = (2.0 * h1 + h2) / (h1 * (h1 + h2))
    b = -(h1 + h2) / (h1 * h2)
    c = h1 / (h2 * (h1 + h2))
    return a, b, c


def march_coeffs(pos):
    """Upwind coefficients along a march whose node 0 is the inflow boundary.

    pos: coordinates along the march direction (increasing).  Returns arrays (a, b, c)
    for nodes 1..n-1: node 1 is first order, others three-point backward."""
    n = len(pos)
    a = np.zeros(n)
    b = np.zeros(n)
    c = np.zeros(n)
    a[1] = 1.0 / (pos[1] - pos[0])
    b[1] = -a[1]
    for i in range(2, n):
        a[i], b[i], c[i] = backward_coeffs(pos[i - 2], pos[i - 1], pos[i])
    return a, b, c


def sweep_1d(rhs, nu, V1, x):
    """Solve nu h + v1 dh/dx = rhs on the half channel (see module docstring).

    rhs: (Ns+1, nv, nv, nv); nu, V1: (nv, nv, nv); x: (Ns+1,) nodes, x[0] = -1/2 wall,
    x[-1] = 0 symmetry.  Velocity axis 0 is v1; the grid must be symmetric in v1."""
    n = len(x)
    nv = V1.shape[0]
    h = np.zeros(rhs.shape)
    pos = V1[nv // 2:]            # v1 > 0 half (midpoint grid is symmetric)
    neg_sl = slice(0, nv // 2)    # v1 < 0 half, index j mirrors nv-1-j
    pos_sl = slice(nv // 2, nv)
    a, b, c = march_coeffs(x)
    # v1 > 0: march from the wall, h(x0) = 0
    for i in range(1, n):
        acc = rhs[i, pos_sl] - pos * (b[i] * h[i - 1, pos_sl]
                                      + (c[i] * h[i - 2, pos_sl] if i >= 2 else 0.0))
        h[i, pos_sl] = acc / (nu[pos_sl] + pos * a[i])
    # v1 < 0: specular reflection at the symmetry plane, then march toward the wall
    h[n - 1, neg_sl] = h[n - 1, pos_sl][::-1]
    # march coordinate y = -x; upwind neighbours of node i are i+1, i+2.  The ghost node
    # i+2 = Ns+1 sits at x = -x_{Ns-1}, i.e. y = x_{Ns-1}, and carries the mirror value.
    speed = -V1[neg_sl]
    for i in range(n - 2, -1, -1):
        y0 = -x[i]
        y1 = -x[i + 1]
        y2 = -x[i + 2] if i + 2 <= n - 1 else x[n - 2]
        h2 = h[i + 2, neg_sl] if i + 2 <= n - 1 else h[n - 2, pos_sl][::-1]
        aa, bb, cc = backward_coeffs(y2, y1, y0)
        acc = rhs[i, neg_sl] - speed * (bb * h[i + 1, neg_sl] + cc * h2)
        h[i, neg_sl] = acc / (nu[neg_sl] + speed * aa)
    return h


def sweep_2d(rhs, nu, V1, V2, nx, ny, width):
    """Solve nu h + v1 dh/dx1 + v2 dh/dx2 = rhs on [0,width] x [0,1] (cell centres).

    rhs: (nx, ny, nv, nv, nv) with cell (i, j) at ((i+1/2) dx, (j+1/2) dy)."""
    dx = width / nx
    dy = 1.0 / ny
    px = np.concatenate([[0.0], (np.arange(nx) + 0.5) * dx])
    py = np.concatenate([[0.0], (np.arange(ny) + 0.5) * dy])
    ax, bx, cx = march_coeffs(px)
    ay, by, cy = march_coeffs(py)
    h = np.zeros(rhs.shape)
    nv = V1.shape[0]
    halves = (slice(0, nv // 2), slice(nv // 2, nv))
    for s1 in (0, 1):
        for s2 in (0, 1):
            sl = (halves[s1], halves[s2], slice(None))
            u1 = np.abs(V1[sl])
            u2 = np.abs(V2[sl])
            nus = nu[sl]
            order_i = range(nx) if s1 == 1 else range(nx - 1, -1, -1)
            order_j = list(range(ny)) if s2 == 1 else list(range(ny - 1, -1, -1))
            hq = np.zeros((nx, ny) + u1.shape)   # march-ordered copy, index = march step
            rq = rhs[(slice(None), slice(None)) + sl]
            for mi, i in enumerate(order_i):
                for mj, j in enumerate(order_j):
                    acc = rq[i, j].copy()
                    # x-direction neighbours (march step mi), node index mi+1 in px
                    k = mi + 1
                    if mi >= 1:
                        acc -= u1 * bx[k] * hq[mi - 1, mj]
                    if mi >= 2:
                        acc -= u1 * cx[k] * hq[mi - 2, mj]
                    k2 = mj + 1
                    if mj >= 1:
                        acc -= u2 * by[k2] * hq[mi, mj - 1]
                    if mj >= 2:
                        acc -= u2 * cy[k2] * hq[mi, mj - 2]
                    hq[mi, mj] = acc / (nus + u1 * ax[k] + u2 * ay[k2])
            for mi, i in enumerate(order_i):
                for mj, j in enumerate(order_j):
                    h[(i, j) + sl] = hq[mi, mj]
    return h
