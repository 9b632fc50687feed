"""Hard-sphere linearized collision operator by the fast spectral method (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What the paper fixes (Sec. 2, Eq. LBE_collision and the nu_eq equation):
    L h   = L+ h - nu_eq h,
    L+ h  = ∬ B [f_eq(v') h(v*') + f_eq(v*') h(v') - f_eq(v) h(v*)] dΩ dv*,
    nu_eq = ∬ B f_eq(v*) dΩ dv*.
For hard spheres B = b |v - v*| per unit solid angle.  The paper cites its fast spectral
method (Sec. 2.4) without writing it out, so the discrete operator is this reading,
written from the collision integral in the Carleman representation:

* Collision strength.  nu_bar = ∫ nu_eq f_eq dv = 1.25 delta (Sec. 2.5), and for
  B = b|u|, nu_bar = 4 pi b E|v - v*| = 4 pi b * 2 sqrt(2/pi), so
  K := 4 pi b = 5 sqrt(2 pi) delta / 16.
* Gain.  With v' = v + x, v*' = v + y, x ⊥ y, hard spheres give the constant Carleman
  kernel 4 b, and after folding the radial integrals to the whole line,
      Q+(f, g)(v) = b ∫_{S2} ∫_{S2} δ(e·e') ∫∫_{|ρ|,|ρ'|<=R} |ρ||ρ'| f(v+ρe) g(v+ρ'e'),
  truncated at |x|, |y| <= R.  In Fourier space the ρ-integral along e gives
  phi(ξ·e), the ρ'-integral over the great circle ⊥ e gives psi(|ξ - (ξ·e)e|):
      phi(s) = 2 ∫_0^R ρ cos(ρ s) dρ,     psi(a) = 4 pi R J1(R a) / a.
  The sphere integral over e is even in e; it is taken as 2 x a hemisphere rule with M
  directions (Gauss-Legendre in cos(theta) on [0, 1] times a midpoint rule in azimuth).
* Loss.  The same Carleman truncation applied to f(v) g(v + x + y) gives, per direction,
  the multiplier phi_p psi_p; summed with the same rule this is G_hat.  Each direction
  then satisfies f_eq(v+x) f_eq(v+y) = f_eq(v) f_eq(v+x+y), so the discrete gain and
  loss cancel on f_eq and on the collision invariants direction by direction.
* nu_eq is the same discrete convolution, nu_eq = F^-1(G_hat F(f_eq)).
* Nyquist planes (index -N/2 on any axis) are zeroed in every multiplier.
* Spectral transforms are the plain DFT on the velocity grid; F^-1(m F(h)) is a cyclic
  convolution, so the grid offset cancels.

Linearization: L+ h = Q+(f_eq, h) + Q+(h, f_eq) - f_eq F^-1(G_hat F(h)) and
L h = L+ h - nu_eq h.  Everything is linear in delta; tables are built for delta = 1.

Pins (tests/test_oracle_fsm.py): explicit spectral convolution (P1), brute-force
velocity quadrature of the collision integral (P2), closed-form hard-sphere nu_eq (P3),
Maxwellian gain = loss (P4), collision invariants in the null space (P5), vanishing
mass/momentum/energy moments of L h (P6), symmetry and sign of L (P7), nu_bar/delta =
1.25 (P9).
"""
import numpy as np
from scipy.special import j1

from . import velocity


def kernel_K(delta=1.0):
    """K = 4 pi b chosen so that nu_bar = 1.25 delta (Sec. 2.5, the nu_bar equation)."""
    return 5.0 * np.sqrt(2.0 * np.pi) * delta / 16.0


def default_R(vmax):
    """Truncation radius R = 2 S with S = 2 vmax / (3 + sqrt 2) (anti-aliasing choice)."""
    return 4.0 * vmax / (3.0 + np.sqrt(2.0))


def directions(M):
    """Hemisphere rule: n_t Gauss-Legendre nodes in mu = cos(theta) on [0,1] times n_a
    midpoint azimuths, n_t = 2**floor(log2(M)/2), n_a = M / n_t.  Weights sum to 2 pi."""
    if M < 2 or (M & (M - 1)) != 0:
        raise ValueError("M must be a power of two >= 2")
    n_t = 2 ** (int(np.log2(M)) // 2)
    n_a = M // n_t
    x, wx = np.polynomial.legendre.leggauss(n_t)
    mu = 0.5 * (x + 1.0)
    wmu = 0.5 * wx
    az = (np.arange(n_a) + 0.5) * 2.0 * np.pi / n_a
    e, w = [], []
    for i in range(n_t):
        st = np.sqrt(1.0 - mu[i] * mu[i])
        for k in range(n_a):
            e.append((st * np.cos(az[k]), st * np.sin(az[k]), mu[i]))
            w.append(wmu[i] * 2.0 * np.pi / n_a)
    return np.array(e), np.array(w)


def phi(s, R):
    """phi(s) = 2 ∫_0^R ρ cos(ρ s) dρ = 2 R^2 [sin x / x - 2 sin^2(x/2) / x^2], x = R s."""
    x = R * np.asarray(s, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = R * R * (1.0 - xs * xs / 4.0 + xs ** 4 / 72.0)
    xl = x[~small]
    out[~small] = 2.0 * R * R * (np.sin(xl) / xl - 2.0 * np.sin(0.5 * xl) ** 2 / (xl * xl))
    return out


def psi(a, R):
    """psi(a) = 2 ∫_0^{2pi} ∫_0^R ρ cos(ρ a cos t) dρ dt = 4 pi R^2 J1(x)/x, x = R a."""
    x = R * np.asarray(a, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = 4.0 * np.pi * R * R * (0.5 - xs * xs / 16.0 + xs ** 4 / 384.0)
    xl = x[~small]
    out[~small] = 4.0 * np.pi * R * R * j1(xl) / xl
    return out


def frequencies(nv, vmax):
    """Signed integer frequencies in DFT order, xi = l pi / vmax, and the Nyquist mask."""
    l = np.fft.fftfreq(nv, 1.0 / nv).round().astype(np.int64)
    xi = l * np.pi / vmax
    X1, X2, X3 = np.meshgrid(xi, xi, xi, indexing="ij")
    L1, L2, L3 = np.meshgrid(l, l, l, indexing="ij")
    nyq = (L1 == -nv // 2) | (L2 == -nv // 2) | (L3 == -nv // 2)
    return X1, X2, X3, nyq


def fft3(a):
    return np.fft.fftn(a, axes=(-3, -2, -1))


def ifft3(a):
    return np.fft.ifftn(a, axes=(-3, -2, -1))


class FSM:
    """Tables of the discrete operator for one (nv, vmax, M, R) at delta = 1."""

    def __init__(self, nv, vmax=6.0, M=16, R=None):
        self.nv, self.vmax, self.M = nv, float(vmax), M
        self.R = default_R(vmax) if R is None else float(R)
        self.V1, self.V2, self.V3, self.dv = velocity.grid(nv, vmax)
        self.feq = velocity.feq(self.V1, self.V2, self.V3)
        X1, X2, X3, nyq = frequencies(nv, vmax)
        e, w = directions(M)
        self.e, self.w = e, w
        b = kernel_K(1.0) / (4.0 * np.pi)
        self.wp = 2.0 * b * w          # hemisphere rule doubled, times b
        xi2 = X1 * X1 + X2 * X2 + X3 * X3
        self.phi = np.empty((M,) + X1.shape)
        self.psi = np.empty((M,) + X1.shape)
        for p in range(M):
            s = X1 * e[p, 0] + X2 * e[p, 1] + X3 * e[p, 2]
            perp = np.sqrt(np.maximum(xi2 - s * s, 0.0))
            ph = phi(s, self.R)
            ps = psi(perp, self.R)
            ph[nyq] = 0.0
            ps[nyq] = 0.0
            self.phi[p] = ph
            self.psi[p] = ps
        self.Ghat = np.einsum("p,pijk->ijk", self.wp, self.phi * self.psi)
        Feq = fft3(self.feq)
        self.A = ifft3(self.phi * Feq).real     # A_p = F^-1(phi_p F(f_eq))
        self.B = ifft3(self.psi * Feq).real     # B_p = F^-1(psi_p F(f_eq))
        self.nu = ifft3(self.Ghat * Feq).real   # nu_eq at delta = 1

    # ---- operator pieces (delta = 1) -------------------------------------------------
    def gain(self, h):
        """Q+(f_eq, h) + Q+(h, f_eq) for h of shape (..., nv, nv, nv)."""
        H = fft3(h)
        out = np.zeros(h.shape)
        for p in range(self.M):
            a = ifft3(self.psi[p] * H).real     # F^-1(psi_p F h), pairs with A_p
            bb = ifft3(self.phi[p] * H).real    # F^-1(phi_p F h), pairs with B_p
            out += self.wp[p] * (self.A[p] * a + self.B[p] * bb)
        return out

    def loss_conv(self, h):
        """F^-1(G_hat F(h)) = ∬ B h(v*) dΩ dv* in the truncated discrete form."""
        return ifft3(self.Ghat * fft3(h)).real

    def apply(self, h, delta=1.0):
        """Return (L+ h, L h) at rarefaction delta (Eq. LBE_collision)."""
        lplus = delta * (self.gain(h) - self.feq * self.loss_conv(h))
        return lplus, lplus - delta * self.nu * h

    def nu_bar(self, delta=1.0):
        """nu_bar = ∫ nu_eq f_eq dv (Sec. 2.5)."""
        return delta * float(np.sum(self.nu * self.feq)) * self.dv ** 3

    # ---- independent evaluations used as pins ---------------------------------------
    def direct_spectral_gain(self, f, g):
        """Q+(f, g) by the explicit cyclic spectral sum (pin P1), small nv only:
        F(Q+)_n = nv^-3 sum_{k + k' = n mod nv} beta(k, k') F(f)_k F(g)_k',
        beta(k, k') = sum_p wp_p phi_p(k) psi_p(k')."""
        n = self.nv
        Ff = fft3(f).reshape(-1)
        Fg = fft3(g).reshape(-1)
        ph = self.phi.reshape(self.M, -1)
        ps = self.psi.reshape(self.M, -1)
        beta = (ph * self.wp[:, None]).T @ ps          # [k, k']
        idx = np.arange(n)
        K1, K2, K3 = np.meshgrid(idx, idx, idx, indexing="ij")
        K1, K2, K3 = K1.reshape(-1), K2.reshape(-1), K3.reshape(-1)
        Qhat = np.zeros(n ** 3, dtype=complex)
        for j in range(n ** 3):
            j1_, j2_, j3_ = K1[j], K2[j], K3[j]
            kp = ((j1_ - K1) % n) * n * n + ((j2_ - K2) % n) * n + (j3_ - K3) % n
            Qhat[j] = np.sum(beta[np.arange(n ** 3), kp] * Ff * Fg[kp])
        Qhat /= n ** 3
        return ifft3(Qhat.reshape(n, n, n)).real


def brute_force_L(hfun, v, delta=1.0, n_vs=48, vs_max=6.0, n_sphere=24):
    """L h at one velocity v by direct quadrature of the collision integral (pin P2).

    L h(v) = ∬ b|u| [f_eq(v') h(v*') + f_eq(v*') h(v') - f_eq(v) h(v*) - h(v) f_eq(v*)]
    dσ dv* with v' = (v+v*)/2 + |u|σ/2, v*' = (v+v*)/2 - |u|σ/2, u = v - v*.  hfun must
    accept arrays of shape (..., 3).  Midpoint rule in v* on [-vs_max, vs_max]^3, product
    Gauss-Legendre x midpoint rule on the sphere.  No truncation in |u|.
    """
    b = kernel_K(delta) / (4.0 * np.pi)
    xs = -vs_max + (np.arange(n_vs) + 0.5) * (2.0 * vs_max / n_vs)
    dvs = (2.0 * vs_max / n_vs) ** 3
    VS = np.stack(np.meshgrid(xs, xs, xs, indexing="ij"), -1).reshape(-1, 3)
    x, wx = np.polynomial.legendre.leggauss(n_sphere)
    az = (np.arange(2 * n_sphere) + 0.5) * np.pi / n_sphere
    st = np.sqrt(1.0 - x * x)
    sig = np.stack([np.outer(st, np.cos(az)), np.outer(st, np.sin(az)),
                    np.outer(x, np.ones_like(az))], -1).reshape(-1, 3)
    wsig = np.outer(wx, np.full(az.shape, np.pi / n_sphere)).reshape(-1)

    def fe(p):
        return np.exp(-np.sum(p * p, -1)) / np.pi ** 1.5

    v = np.asarray(v, dtype=np.float64)
    u = v[None, :] - VS
    un = np.sqrt(np.sum(u * u, -1))
    cm = 0.5 * (v[None, :] + VS)
    total = 0.0
    for s, ws in zip(sig, wsig):
        vp = cm + 0.5 * un[:, None] * s[None, :]
        vsp = cm - 0.5 * un[:, None] * s[None, :]
        gainv = fe(vp) * hfun(vsp) + fe(vsp) * hfun(vp)
        total += ws * np.sum(b * un * gainv) * dvs
    loss = 4.0 * np.pi * b * np.sum(un * (fe(v[None, :]) * hfun(VS)
                                         + hfun(v[None, :]) * fe(VS))) * dvs
    return total - loss
