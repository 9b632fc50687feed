"""Binary hard-sphere mixture: linearized collision operators and the SIS (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4 fixes the equations (the Maxwellian f_alpha,eq, the LBE for h_alpha with
L_alpha = sum_beta Q_ab(f_a,eq, h_b) + Q_ab(h_a, f_b,eq), the source, the definitions of
U_alpha, P_alpha13, q_alpha, the flow rates, Eqs. LBE_penlty, LBE2_true1, LBE2_true2 and the
N_alpha equation) but cites its spectral method for Q_ab without writing it out.  The
discrete operator is therefore this reading, derived from the collision integral:

* Species A and B: masses m_A, m_B (r_a = m_a / m_A), hard-sphere diameters d_A, d_B
  (collision diameter d_ab = (d_a + d_b) / 2), molar fractions chi_a.  Velocities are in
  units of v_mA, so f_a,eq = chi_a (r_a / pi)^(3/2) exp(-r_a |v|^2).
* A collision of an alpha molecule (velocity v) with a beta molecule (v*), u = v - v*,
  mu_b = m_b / (m_a + m_b), unit vector n along the line of centres:
  v' = v - 2 mu_b (u.n) n,  v*' = v* + 2 mu_a (u.n) n  (momentum and energy conserved).
  With x = -(u.n) n and y = -(u - (u.n) n), so x ⊥ y:
      v* = v + x + y,   v' = v + 2 mu_b x,   v*' = v + c x + y,   c = mu_b - mu_a.
  Hard spheres collide at the rate d_ab^2 (u.n) per unit solid angle of n (u.n > 0), and
  the change of variables (u, n) -> (x, y) leaves the constant kernel 4 b_ab = d_ab^2,
  b_ab being the strength per unit solid angle in the sigma representation (B = b_ab |u|):
      Q+_ab(f, g)(v) = 4 b_ab ∬ δ(x·y) f(v + 2 mu_b x) g(v + c x + y) dx dy,
      Q-_ab(f, g)(v) = f(v) 4 b_ab ∬ δ(x·y) g(v + x + y) dx dy,
  both truncated at |x|, |y| <= R.  For equal masses (mu = 1/2, c = 0) this is the
  single-species form of ``oracle.fsm``.
* Fourier form.  With f_j = sum_l f^_l w^(l j) on the periodic grid (f^ = DFT / N^3), the
  x-integral along a line through the origin in direction e gives phi((2 mu_b xi_l + c xi_m)·e)
  and the y-integral over the plane ⊥ e gives psi(|xi_m ⊥ e|) (``oracle.fsm``'s phi, psi);
  the sphere integral over e is the hemisphere rule of ``oracle.fsm`` doubled:
      beta_ab(l, m) = sum_p wp_p phi((2 mu_b xi_l + c xi_m)·e_p) psi_p(m),  wp = 2 b w,
      F(Q+_ab(f, g))_k = sum_{l + m = k mod N} beta_ab(l, m) f^_l g^_m.
  phi's argument mixes both spectra unless the masses are equal, so this gain is not a sum
  of products of separate transforms: the oracle writes out the cyclic sum as a dense
  matrix on the spectrum of the unknown (the Maxwellian being the other argument).  The
  loss keeps the product form of ``oracle.fsm``: G^_ab = sum_p wp_p phi_p psi_p (mass
  independent), nu_ab = F^-1(G^_ab F(f_b,eq)).  Nyquist modes are zeroed in the factor
  that carries them (phi: the f-slot mode; psi and G^: the g-slot mode), as in
  ``oracle.fsm``.
* Linearization:
      L+_a h = sum_b [Q+_ab(f_a,eq, h_b) + Q+_ab(h_a, f_b,eq) - f_a,eq F^-1(G^_ab F h_b)],
      L_a h  = L+_a h - nu_a h_a,   nu_a = sum_b nu_ab.
* Collision strength (rarefaction).  delta = p0 l / (mu v_m) with v_m = sqrt(2 kT / m),
  m = chi_A m_A + chi_B m_B (Sec. 4, the flow-rate normalisation), and mu read as the first
  Chapman-Enskog approximation of the mixture viscosity -- the approximation under which
  the single-species nu_bar = 1.25 delta of Sec. 2.5 holds.  In units m_A = kT = d_A = 1,
  n0 l d_A^2 = delta mu1 sqrt(2 / m), so b_ab = delta mu1 sqrt(2 / m) d_ab^2 / 4.  For
  hard spheres mu1 is the closed form of the Chapman-Enskog theory (``eta1``); the pin
  ``galerkin_viscosity`` recomputes it from the discrete operator itself.

Pins (tests/test_oracle_mixture.py): the equal-mass limit equals ``oracle.fsm`` (M1), the
explicit cyclic sum equals the matrix form (M2), brute-force sigma-representation quadrature
of the collision integral for unequal masses (M3), collision invariants (M4), conservation
(M5), the sign of the dissipation (M6), the viscosity closed form against a Monte Carlo
Galerkin on the weak form of the collision integral (M7); for the SIS:
identical species reproduce the single-species CIS iteration exactly, between plates and in a
duct (M8), SIS and CIS reach the same solution to the discretisation, as the paper reports for
one species (M9).
"""
import numpy as np

from . import fsm as fsm_mod
from . import transport, velocity


def eta1(r_B, dr, chi_A):
    """First Chapman-Enskog approximation of the viscosity of a binary hard-sphere mixture
    in units m_A = kT = d_A = 1 (rigid spheres: collision integrals Omega* = A* = 1).
    r_B = m_B / m_A, dr = d_B / d_A, chi_A = molar fraction of A."""
    m1, m2 = 1.0, float(r_B)
    x1, x2 = float(chi_A), 1.0 - float(chi_A)
    s12 = 0.5 * (1.0 + dr)
    e1 = 5.0 / 16.0 * np.sqrt(m1 / np.pi)
    e2 = 5.0 / 16.0 * np.sqrt(m2 / np.pi) / dr ** 2
    e12 = 5.0 / 16.0 * np.sqrt(2.0 * m1 * m2 / (np.pi * (m1 + m2))) / s12 ** 2
    q = (m1 + m2) ** 2 / (4.0 * m1 * m2)
    X = x1 * x1 / e1 + 2.0 * x1 * x2 / e12 + x2 * x2 / e2
    Y = 0.6 * (x1 * x1 / e1 * (m1 / m2) + 2.0 * x1 * x2 / e12 * q * e12 * e12 / (e1 * e2)
               + x2 * x2 / e2 * (m2 / m1))
    Z = 0.6 * (x1 * x1 * m1 / m2 + 2.0 * x1 * x2 * (q * (e12 / e1 + e12 / e2) - 1.0)
               + x2 * x2 * m2 / m1)
    return (1.0 + Z) / (X + Y)


class Mixture:
    """Species data: r = (1, m_B/m_A), d = (1, d_B/d_A), chi = (chi_A, 1 - chi_A)."""

    def __init__(self, mass_ratio, diam_ratio, chi_A):
        self.r = np.array([1.0, float(mass_ratio)])
        self.d = np.array([1.0, float(diam_ratio)])
        self.chi = np.array([float(chi_A), 1.0 - float(chi_A)])
        self.mbar = float(np.sum(self.chi * self.r))

    def dab(self, a, b):
        return 0.5 * (self.d[a] + self.d[b])

    def b_AA(self, delta):
        """b_AA = delta mu1 sqrt(2 / m) / 4 (module docstring)."""
        return delta * eta1(self.r[1], self.d[1], self.chi[0]) * np.sqrt(2.0 / self.mbar) / 4.0

    def feq(self, a, V1, V2, V3):
        r = self.r[a]
        return self.chi[a] * (r / np.pi) ** 1.5 * np.exp(-r * (V1 * V1 + V2 * V2 + V3 * V3))


class MixFSM:
    """Dense discrete operator of one mixture on one (nv, vmax, M, R) grid.

    ``b0`` fixes b_AA (the other strengths scale with d_ab^2); by default b0 is the value at
    delta = 1, and ``apply`` scales linearly in delta (the operator is linear in b_AA)."""

    def __init__(self, mix, nv, vmax=6.0, M=16, R=None, b0=None):
        self.mix, self.nv, self.vmax, self.M = mix, nv, float(vmax), M
        self.R = fsm_mod.default_R(vmax) if R is None else float(R)
        self.b0 = mix.b_AA(1.0) if b0 is None else float(b0)
        self.V1, self.V2, self.V3, self.dv = velocity.grid(nv, vmax)
        self.f = [mix.feq(a, self.V1, self.V2, self.V3) for a in range(2)]
        X1, X2, X3, nyq = fsm_mod.frequencies(nv, vmax)
        self.X = np.stack([X1.reshape(-1), X2.reshape(-1), X3.reshape(-1)], 1)   # xi per mode
        self.nyq = nyq.reshape(-1)
        self.e, self.w = fsm_mod.directions(M)
        n = nv ** 3
        self.n = n
        # k - m (mod N per axis) as a flat mode index, for every (k, m)
        idx = np.arange(nv)
        I1, I2, I3 = [a.reshape(-1) for a in np.meshgrid(idx, idx, idx, indexing="ij")]
        self.D = (((I1[:, None] - I1[None, :]) % nv) * nv * nv
                  + ((I2[:, None] - I2[None, :]) % nv) * nv + (I3[:, None] - I3[None, :]) % nv)
        self.fhat = [np.fft.fftn(fa).reshape(-1) / n for fa in self.f]
        xi2 = np.sum(self.X * self.X, 1)
        self.s = np.empty((M, n))
        self.phi_own = np.empty((M, n))
        self.psi = np.empty((M, n))
        for p in range(M):
            s = self.X @ self.e[p]
            perp = np.sqrt(np.maximum(xi2 - s * s, 0.0))
            ph = fsm_mod.phi(s, self.R)
            ps = fsm_mod.psi(perp, self.R)
            ph[self.nyq] = 0.0
            ps[self.nyq] = 0.0
            self.s[p], self.phi_own[p], self.psi[p] = s, ph, ps
        self._beta = {}
        self.Lmat = [[self._block(a, b) for b in range(2)] for a in range(2)]
        self._beta = {}
        self.nu = [sum(self._nu_ab(a, b) for b in range(2)) for a in range(2)]

    # ---- tables ------------------------------------------------------------------------
    def strength(self, a, b):
        return self.b0 * (self.mix.dab(a, b) / self.mix.d[0]) ** 2

    def wp(self, a, b):
        return 2.0 * self.strength(a, b) * self.w

    def mu_c(self, a, b):
        ra, rb = self.mix.r[a], self.mix.r[b]
        return rb / (ra + rb), (rb - ra) / (ra + rb)

    def Ghat(self, a, b):
        return np.einsum("p,pk->k", self.wp(a, b), self.phi_own * self.psi)

    def _nu_ab(self, a, b):
        Fb = np.fft.fftn(self.f[b])
        return np.fft.ifftn(self.Ghat(a, b).reshape(Fb.shape) * Fb).real

    def beta(self, a, b):
        """Kernel modes beta_ab(l, m) = sum_p wp_p phi((2 mu_b xi_l + c xi_m)·e_p) psi_p(m)
        for every pair of flat mode indices (l: the v + 2 mu_b x slot, m: the v + c x + y
        slot), Nyquist l zeroed in phi and Nyquist m in psi."""
        mu, c = self.mu_c(a, b)
        wp = self.wp(a, b)
        keep = (~self.nyq).astype(float)
        B = np.zeros((self.n, self.n))
        for p in range(self.M):
            s = self.s[p]
            x = self.R * (2.0 * mu * s[:, None] + c * s[None, :])
            # phi(s) = 2 R^2 [sin x / x - 2 sin^2(x/2) / x^2] written with sinc
            ph = 2.0 * self.R ** 2 * (np.sinc(x / np.pi) - 0.5 * np.sinc(x / (2.0 * np.pi)) ** 2)
            B += (wp[p] * keep)[:, None] * ph * self.psi[p][None, :]
        self._beta[(a, b)] = B
        return B

    def gain_second(self, a, b):
        """Spectral matrix of h_b -> Q+_ab(f_a,eq, h_b):  sum_m beta_ab(k - m, m) f^_a,eq(k - m) h^_m."""
        cols = np.arange(self.n)[None, :]
        return self.fhat[a][self.D] * self.beta(a, b)[self.D, cols]

    def gain_first(self, a, b):
        """Spectral matrix of h_a -> Q+_ab(h_a, f_b,eq):  sum_l beta_ab(l, k - l) h^_l f^_b,eq(k - l)."""
        cols = np.arange(self.n)[None, :]
        return self.beta(a, b)[cols, self.D] * self.fhat[b][self.D]

    def fourier_block(self, a, b):
        """Spectral matrix K[k, m] of h_b -> L+_a restricted to h_b (module docstring): the
        gain Q+_ab(f_a,eq, h_b) less the loss f_a,eq F^-1(G^_ab F h_b), whose spectrum is
        sum_m f^_a,eq(k - m) G^_ab(m) h^_m, plus sum_c Q+_ac(h_a, f_c,eq) when b == a."""
        K = self.gain_second(a, b) - self.fhat[a][self.D] * self.Ghat(a, b)[None, :]
        if a == b:
            for cc in range(2):
                K = K + self.gain_first(a, cc)
        return K

    def _block(self, a, b):
        """Velocity-space matrix of the same map: L[j, i] = sum_k w^(k j) sum_m K[k, m] w^(-m i) / N^3."""
        N, n = self.nv, self.n
        K = self.fourier_block(a, b).reshape((N, N, N, N, N, N))
        T = np.fft.fftn(K, axes=(3, 4, 5))
        Lv = np.fft.ifftn(T, axes=(0, 1, 2)).reshape(n, n)
        self.max_imag = max(getattr(self, "max_imag", 0.0), float(np.max(np.abs(Lv.imag))))
        return Lv.real

    # ---- operator ----------------------------------------------------------------------
    def apply(self, hA, hB, delta=1.0):
        """Return (L+_A, L_A, L+_B, L_B) at rarefaction delta; h of shape (..., nv, nv, nv)."""
        shp = hA.shape
        h = [hA.reshape(-1, self.n).T, hB.reshape(-1, self.n).T]
        out = []
        for a in range(2):
            lp = (self.Lmat[a][0] @ h[0] + self.Lmat[a][1] @ h[1]).T.reshape(shp) * delta
            out += [lp, lp - delta * self.nu[a] * (hA if a == 0 else hB)]
        return tuple(out)

    def nu_bar(self, a, delta=1.0):
        return delta * float(np.sum(self.nu[a] * self.f[a])) * self.dv ** 3

    def N_alpha(self, a):
        """N_a = ∫ nu_a,eq f_a,eq dv / (delta chi_a) (Sec. 4), independent of delta."""
        return self.nu_bar(a, 1.0) / self.mix.chi[a]

    # ---- independent evaluations used as pins ------------------------------------------
    def direct_gain(self, a, b, f, g):
        """Q+_ab(f, g) by the explicit cyclic sum over (l, m) (pin M2; small nv only)."""
        N, n = self.nv, self.n
        Ff = np.fft.fftn(f).reshape(-1) / n
        Fg = np.fft.fftn(g).reshape(-1) / n
        mu, c = self.mu_c(a, b)
        wp = self.wp(a, b)
        Q = np.zeros(n, dtype=complex)
        for l in range(n):
            if self.nyq[l]:
                continue
            for m in range(n):
                beta = 0.0
                for p in range(self.M):
                    arg = 2.0 * mu * self.s[p][l] + c * self.s[p][m]
                    beta += wp[p] * fsm_mod.phi(np.array([arg]), self.R)[0] * self.psi[p][m]
                Q[self._add(l, m)] += beta * Ff[l] * Fg[m]
        return (np.fft.ifftn(Q.reshape(N, N, N)) * n).real

    def _add(self, l, m):
        N = self.nv
        a = np.unravel_index(l, (N, N, N))
        b = np.unravel_index(m, (N, N, N))
        return int(((a[0] + b[0]) % N) * N * N + ((a[1] + b[1]) % N) * N + (a[2] + b[2]) % N)


def bruteforce_L(mix, b0, a, hfun, v, delta=1.0, n_vs=40, vs_max=6.0, n_sphere=20):
    """L_a h at one velocity v by direct quadrature of the collision integrals in the sigma
    representation (pin M3):  sum_b ∬ b_ab |u| [f_a(v') h_b(v*') + h_a(v') f_b(v*')
    - f_a(v) h_b(v*) - h_a(v) f_b(v*)] dsigma dv*, V = mu_a v + mu_b v*, v' = V + mu_b |u| s,
    v*' = V - mu_a |u| s.  hfun(species, points[..., 3]) gives h.  Midpoint rule in v*,
    Gauss-Legendre x midpoint on the sphere, no truncation in |u|."""
    xs = -vs_max + (np.arange(n_vs) + 0.5) * (2.0 * vs_max / n_vs)
    dvs = (2.0 * vs_max / n_vs) ** 3
    VS = np.stack(np.meshgrid(xs, xs, xs, indexing="ij"), -1).reshape(-1, 3)
    x, wx = np.polynomial.legendre.leggauss(n_sphere)
    az = (np.arange(2 * n_sphere) + 0.5) * np.pi / n_sphere
    st = np.sqrt(1.0 - x * x)
    sig = np.stack([np.outer(st, np.cos(az)), np.outer(st, np.sin(az)),
                    np.outer(x, np.ones_like(az))], -1).reshape(-1, 3)
    wsig = np.outer(wx, np.full(az.shape, np.pi / n_sphere)).reshape(-1)

    def fe(s, p):
        return mix.feq(s, p[..., 0], p[..., 1], p[..., 2])

    v = np.asarray(v, dtype=np.float64)
    u = v[None, :] - VS
    un = np.sqrt(np.sum(u * u, -1))
    total = 0.0
    for b in range(2):
        bab = delta * b0 * (mix.dab(a, b) / mix.d[0]) ** 2
        ra, rb = mix.r[a], mix.r[b]
        mua, mub = ra / (ra + rb), rb / (ra + rb)
        V = mua * v[None, :] + mub * VS
        for s, ws in zip(sig, wsig):
            vp = V + mub * un[:, None] * s[None, :]
            vsp = V - mua * un[:, None] * s[None, :]
            g = fe(a, vp) * hfun(b, vsp) + hfun(a, vp) * fe(b, vsp)
            total += ws * np.sum(bab * un * g) * dvs
        loss = 4.0 * np.pi * bab * np.sum(un * (fe(a, v[None, :]) * hfun(b, VS)
                                                + hfun(a, v[None, :]) * fe(b, VS))) * dvs
        total -= loss
    return total


def galerkin_viscosity(F, delta=1.0):
    """First Chapman-Enskog approximation from the discrete operator (pin M7): the shear flow
    U3 = gamma x1 perturbs h_a = f_a,eq (2 r_a gamma x1 v3 + Phi_a), and L_a(Phi f) = 2 r_a
    gamma v1 v3 f_a,eq; Galerkin on the trial functions v1 v3 f_a,eq gives P13 =
    sum_a 2 r_a ∫ v1 v3 Phi_a f_a,eq, and mu = -P13 delta / (gamma sqrt(m)) in units of the
    viscosity that defines delta (1 when the discrete operator matches the closed form)."""
    w = F.dv ** 3
    t = [F.V1 * F.V3 * F.f[a] for a in range(2)]
    I = np.zeros((2, 2))
    for b in range(2):
        hA = t[0] if b == 0 else np.zeros_like(t[0])
        hB = t[1] if b == 1 else np.zeros_like(t[1])
        _, LA, _, LB = F.apply(hA, hB, delta)
        I[0, b] = np.sum(F.V1 * F.V3 * LA) * w
        I[1, b] = np.sum(F.V1 * F.V3 * LB) * w
    rhs = np.array([2.0 * F.mix.r[a] * np.sum(F.V1 * F.V3 * t[a]) * w for a in range(2)])
    coef = np.linalg.solve(I, rhs)
    P13 = sum(2.0 * F.mix.r[a] * coef[a] * np.sum(F.V1 * F.V3 * t[a]) * w for a in range(2))
    return -P13 * delta / np.sqrt(F.mix.mbar)


def mc_galerkin_viscosity(mix, n=1_000_000, chunks=2, seed=7):
    """The same first Chapman-Enskog approximation without the discrete operator (pin M7):
    the Galerkin brackets I[g, b] = ∫ v1 v3 L_g(h^(b)) dv, h^(b)_a = [a = b] v1 v3 f_b,eq, by
    Monte Carlo on the weak form of the collision integral,
        ∫ psi(v) Q_gd(F, G)(v) dv = ∭ b_gd |u| F(v) G(v*) [psi(v') - psi(v)] dsigma dv dv*,
    sampling v ~ f_g,eq / chi_g, v* ~ f_d,eq / chi_d and sigma uniformly on the sphere
    (delta = 1).  Returns mu / mu1 as ``galerkin_viscosity`` does."""
    rng = np.random.default_rng(seed)
    b0 = mix.b_AA(1.0)
    I = np.zeros((2, 2))
    for g in range(2):
        for d in range(2):
            bgd = b0 * (mix.dab(g, d) / mix.d[0]) ** 2
            rg, rd = mix.r[g], mix.r[d]
            mug, mud = rg / (rg + rd), rd / (rg + rd)
            acc = np.zeros(2)
            for _ in range(chunks):
                v = rng.standard_normal((n, 3)) / np.sqrt(2.0 * rg)
                vs = rng.standard_normal((n, 3)) / np.sqrt(2.0 * rd)
                sg = rng.standard_normal((n, 3))
                sg /= np.linalg.norm(sg, axis=1)[:, None]
                un = np.linalg.norm(v - vs, axis=1)
                vp = mug * v + mud * vs + mud * un[:, None] * sg
                base = (4.0 * np.pi * bgd * mix.chi[g] * mix.chi[d] * un
                        * (vp[:, 0] * vp[:, 2] - v[:, 0] * v[:, 2]))
                acc += [np.mean(base * v[:, 0] * v[:, 2]), np.mean(base * vs[:, 0] * vs[:, 2])]
            acc /= chunks
            I[g, g] += acc[0]      # h_g at v (the Q_gd(h_g, f_d,eq) term)
            I[g, d] += acc[1]      # h_d at v* (the Q_gd(f_g,eq, h_d) term)
    tt = np.array([mix.chi[a] / (4.0 * mix.r[a] ** 2) for a in range(2)])   # ∫ v1^2 v3^2 f_a,eq
    coef = np.linalg.solve(I, 2.0 * mix.r * tt)
    P13 = float(np.sum(2.0 * mix.r * coef * tt))
    return -P13 / np.sqrt(mix.mbar)


# ---- porous cell: a square array of cylinders (the unit cell, periodic) ----------------------
def porous_solid(n, solid_fraction):
    """Staircase of the centred circular cylinder of area `solid_fraction` in the periodic unit
    cell of n x n cells: cell (i, j), centre ((i + 1/2) / n, (j + 1/2) / n), is solid when its
    centre lies inside the circle."""
    c = (np.arange(n) + 0.5) / n - 0.5
    X, Y = np.meshgrid(c, c, indexing="ij")
    return X * X + Y * Y < solid_fraction / np.pi


def upwind_porous(solid1, solid2, d):
    """(a, b, c) of d/ds at a fluid cell from itself, its upwind neighbour and the next one
    (spacing d).  A solid neighbour ends the line at its face, half a cell away, where the
    diffuse wall emits h = 0: first order from the face next to a solid neighbour, three
    points through the face one cell further up."""
    if solid1:
        return 2.0 / d, 0.0, 0.0
    if solid2:
        a, b, _ = transport.backward_coeffs(-1.5 * d, -d, 0.0)
        return a, b, 0.0
    return transport.backward_coeffs(-2.0 * d, -d, 0.0)


def sweep_porous(rhs, nu, V1, V2, solid, hprev):
    """nu h + v1 dh/dx1 + v2 dh/dx2 = rhs in the periodic unit cell with solid cells (h = 0).
    For each quadrant of (v1, v2) the cells are swept in upwind order, rows in x2 and cells in
    x1; a periodic neighbour that is not yet swept takes its value from `hprev`, the previous
    sweep's result (the sweep is done in place over it), so a converged iteration satisfies the
    periodic scheme itself."""
    n = solid.shape[0]
    d = 1.0 / n
    out = hprev.copy()
    for s1 in (1, -1):
        for s2 in (1, -1):
            sel = (np.sign(V1) == s1) & (np.sign(V2) == s2)
            u1, u2, nuq = np.abs(V1[sel]), np.abs(V2[sel]), nu[sel]
            for jj in range(n):
                j = jj if s2 > 0 else n - 1 - jj
                for ii in range(n):
                    i = ii if s1 > 0 else n - 1 - ii
                    if solid[i, j]:
                        out[i, j][sel] = 0.0
                        continue
                    i1, i2 = (i - s1) % n, (i - 2 * s1) % n
                    j1, j2 = (j - s2) % n, (j - 2 * s2) % n
                    ax, bx, cx = upwind_porous(solid[i1, j], solid[i2, j], d)
                    ay, by, cy = upwind_porous(solid[i, j1], solid[i, j2], d)
                    num = (rhs[i, j][sel] - u1 * (bx * out[i1, j][sel] + cx * out[i2, j][sel])
                           - u2 * (by * out[i, j1][sel] + cy * out[i, j2][sel]))
                    out[i, j][sel] = num / (nuq + u1 * ax + u2 * ay)
    return out


def porous_interior(solid):
    """Fluid cells whose eight neighbours (periodic) are fluid; the other fluid cells form the
    wall-adjacent ring of the diffusion correction."""
    fluid = ~solid
    inner = fluid.copy()
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            inner &= np.roll(fluid, (-di, -dj), axis=(0, 1))
    return inner


# ---- synthetic iterative scheme for plates (Sec. 4) ------------------------------------------
def porous_poisson(inner, Uh, rhs):
    """lap U = rhs on the cells of ``inner`` (five-point periodic differences on the n x n unit
    cell, spacing 1/n), U = Uh on every other cell; dense LU.  Returns U on all cells."""
    n = Uh.shape[0]
    d = 1.0 / n
    idx = -np.ones((n, n), dtype=int)
    idx[inner] = np.arange(int(inner.sum()))
    m = int(inner.sum())
    A = np.zeros((m, m))
    b = rhs[inner].copy()
    for (i, j), k in zip(np.argwhere(inner), range(m)):
        A[k, k] = -4.0 / d ** 2
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            ii, jj = (i + di) % n, (j + dj) % n
            if inner[ii, jj]:
                A[k, idx[ii, jj]] = 1.0 / d ** 2
            else:
                b[k] -= Uh[ii, jj] / d ** 2
    U = Uh.copy()
    U[inner] = np.linalg.solve(A, b)
    return U


class MixProblem:
    """Poiseuille flow of a binary mixture between plates (dim 1, Table 4's setting) or through
    a rectangular duct [0, width] x [0, 1] of nx x ny cells (dim 2, Table 5's setting)."""

    def __init__(self, mass_ratio=39.95 / 20.18, diam_ratio=1.0 / 0.711, chi_A=0.5, delta=1.0,
                 ns=20, grid="uniform", nv=12, vmax=6.0, M=16, R=0.0, N_A=0.0, N_B=0.0,
                 scheme="sis", eps=1e-8, max_iter=500, dim=1, nx=8, ny=8, width=1.0, solid=0.0):
        self.mix = Mixture(mass_ratio, diam_ratio, chi_A)
        self.dim, self.nx, self.ny, self.width = dim, nx, ny, float(width)
        self.solid = float(solid)  # > 0: the periodic unit cell (nx = ny) with a cylinder of this area
        self.delta, self.ns, self.grid = float(delta), ns, grid
        self.nv, self.vmax, self.M, self.R = nv, float(vmax), M, float(R)
        self.N = (float(N_A), float(N_B))
        self.scheme, self.eps, self.max_iter = scheme, eps, max_iter


class MixRun:
    """Iteration state of one mixture solve.  One SIS iteration from h^(k) (reading of
    Eqs. LBE_penlty, LBE2_true1, LBE2_true2 in 1D):
      1. L-evaluation: rhs_a = L+_a h^(k) + S_a (S_a = v3 f_a,eq, X_P = -1) and
         G_a = 2 ∫ v1 v3 (L_a h^(k) + N_a delta h_a^(k)) dv.
      2. Kinetic half step: nu_a delta h + v1 dh/dx1 = rhs_a (upwind sweep, wall h = 0 inflow).
      3. Moments of h^(k+1/2): U_a = ∫ v3 h_a / chi_a, W_a = ∫ (2 v1^2 - 1) v3 h_a
         (= F^a_201 / 4), P_a13 = 2 r_a ∫ v1 v3 h_a.
      4. Diffusion correction, the once-integrated Eqs. LBE2_true2 / LBE2_true1 (every term
         is odd about the symmetry plane x1 = 0, so the constant vanishes):
            d(chi_a U_a + W_a)/dx1 = G_a - (N_a delta / r_a) P~_a13,
         P~_B13 = P_B13 of h^(k+1/2), P~_A13 = x1 - P_B13 (the mixture relation
         dP13/dx1 = 1 with P13(0) = 0); marched from the wall node with the sweep's stencil,
         Y(x0) = chi_a U_a(x0) + W_a(x0).
      5. Correction (Eq. guided for each species): h_a += 2 r_a (U_a^(k+1) - U_a^(k+1/2)) v3 f_a,eq.
      6. Flow rates: M_a = sqrt(m / m_A) 2 ∫_{-1/2}^0 U_a dx1, Q_a likewise with
         q_a = ∫ (r_a |v|^2 - 5/2) v3 h_a.
    In a duct (dim 2) step 4 is Eqs. LBE2_true1 / LBE2_true2 themselves, per species,
         chi_a lap U_a = -(N_a delta / r_a) D_a - (d11 W_a1 + 2 d12 X_a12 + d22 W_a2)
                         + d1 G_a1 + d2 G_a2,
    with X_a12 = F^a_111 / 4, D_B = d1 P_B13 + d2 P_B23 of h^(k+1/2) and D_A = 1 - D_B (the
    mixture relation dP13/dx1 + dP23/dx2 = 1), the five-point Laplacian and central
    differences on interior cells, and U_a = U_a^(k+1/2) on the wall-adjacent ring, as for one
    species; flow rates are sqrt(m / m_A) times cell averages.
    CIS: h^(k+1) = h^(k+1/2).  Stop when the relative changes of M_A, M_B, Q_A, Q_B are all < eps.
    N_a <= 0 selects the N_alpha equation of Sec. 4."""

    def __init__(self, pb, F=None):
        self.pb = pb
        self.F = MixFSM(pb.mix, pb.nv, pb.vmax, pb.M, pb.R if pb.R > 0 else None) if F is None else F
        F = self.F
        if pb.dim == 1:
            self.x = transport.nodes_uniform(pb.ns) if pb.grid == "uniform" else transport.nodes_clustered(pb.ns)
            shape = (len(self.x),) + F.V1.shape
        else:
            shape = (pb.nx, pb.ny) + F.V1.shape
            if pb.solid > 0:
                self.solid = porous_solid(pb.nx, pb.solid)
                self.inner = porous_interior(self.solid)
                self.hprev = [np.zeros(shape), np.zeros(shape)]
        self.h = [np.zeros(shape), np.zeros(shape)]
        self.S = [F.V3 * F.f[a] for a in range(2)]
        self.Nd = [(pb.N[a] if pb.N[a] > 0 else F.N_alpha(a)) * pb.delta for a in range(2)]
        self.rates = np.zeros(4)
        self.iters = 0
        self.U = None

    def moments(self, a, h):
        F, w = self.F, self.F.dv ** 3
        r, chi = self.pb.mix.r[a], self.pb.mix.chi[a]
        ax = (-3, -2, -1)
        c2 = F.V1 ** 2 + F.V2 ** 2 + F.V3 ** 2
        U = np.sum(F.V3 * h, axis=ax) * w / chi
        q = np.sum((r * c2 - 2.5) * F.V3 * h, axis=ax) * w
        W = np.sum((2.0 * F.V1 ** 2 - 1.0) * F.V3 * h, axis=ax) * w
        P = 2.0 * r * np.sum(F.V1 * F.V3 * h, axis=ax) * w
        return U, q, W, P

    def moments2(self, a, h):
        """W_a2 = F^a_021 / 4, X_a12 = F^a_111 / 4 and P_a23 (duct terms)."""
        F, w = self.F, self.F.dv ** 3
        ax = (-3, -2, -1)
        W2 = np.sum((2.0 * F.V2 ** 2 - 1.0) * F.V3 * h, axis=ax) * w
        X12 = 2.0 * np.sum(F.V1 * F.V2 * F.V3 * h, axis=ax) * w
        P23 = 2.0 * self.pb.mix.r[a] * np.sum(F.V2 * F.V3 * h, axis=ax) * w
        return W2, X12, P23

    def poisson(self, Uh, rhs, chi):
        """chi lap U = rhs on interior cells (five-point, dense LU), U = Uh on the ring."""
        pb = self.pb
        nx, ny = Uh.shape
        dx, dy = pb.width / nx, 1.0 / ny
        mx, my = nx - 2, ny - 2
        A = np.zeros((mx * my, mx * my))
        b = rhs.reshape(-1) / chi
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
        U = Uh.copy()
        U[1:-1, 1:-1] = np.linalg.solve(A, b).reshape(mx, my)
        return U

    def step_porous(self, L, hh):
        """Steps 3-5 in the periodic unit cell: Eqs. LBE2_true1 / LBE2_true2 on the cells of
        ``porous_interior`` with periodic central differences, U = U^(k+1/2) on the ring."""
        F, pb, mix = self.F, self.pb, self.pb.mix
        n = pb.nx
        d = 1.0 / n
        w = F.dv ** 3
        ax = (-3, -2, -1)

        def sh(f, di, dj):
            return np.roll(f, (-di, -dj), axis=(0, 1))   # f[(i + di) % n, (j + dj) % n]

        def d1(f):
            return (sh(f, 1, 0) - sh(f, -1, 0)) / (2.0 * d)

        def d2(f):
            return (sh(f, 0, 1) - sh(f, 0, -1)) / (2.0 * d)

        mo = [self.moments(a, hh[a]) + self.moments2(a, hh[a]) for a in range(2)]
        DB = d1(mo[1][3]) + d2(mo[1][6])
        D = [1.0 - DB, DB]
        inner = self.inner
        new = []
        for a in range(2):
            Uh, _, W1, _, W2, X12, _ = mo[a]
            G1 = 2.0 * np.sum(F.V1 * F.V3 * (L[a] + self.Nd[a] * self.h[a]), axis=ax) * w
            G2 = 2.0 * np.sum(F.V2 * F.V3 * (L[a] + self.Nd[a] * self.h[a]), axis=ax) * w
            rhs = (-self.Nd[a] / mix.r[a] * D[a]
                   - (sh(W1, 1, 0) - 2.0 * W1 + sh(W1, -1, 0)) / d ** 2
                   - 2.0 * (sh(X12, 1, 1) - sh(X12, 1, -1) - sh(X12, -1, 1) + sh(X12, -1, -1)) / (4.0 * d * d)
                   - (sh(W2, 0, 1) - 2.0 * W2 + sh(W2, 0, -1)) / d ** 2
                   + d1(G1) + d2(G2)) / mix.chi[a]
            Un = porous_poisson(inner, Uh, rhs)
            new.append(hh[a] + 2.0 * mix.r[a] * (Un - Uh)[(...,) + (None,) * 3] * F.V3 * F.f[a])
        return new

    def step2(self, L, hh):
        """Steps 3-5 in a duct: returns the corrected h of both species."""
        F, pb, mix = self.F, self.pb, self.pb.mix
        nx, ny = pb.nx, pb.ny
        dx, dy = pb.width / nx, 1.0 / ny
        I, J = np.meshgrid(np.arange(1, nx - 1), np.arange(1, ny - 1), indexing="ij")
        w = F.dv ** 3
        ax = (-3, -2, -1)

        def d1(f):
            return (f[I + 1, J] - f[I - 1, J]) / (2.0 * dx)

        def d2(f):
            return (f[I, J + 1] - f[I, J - 1]) / (2.0 * dy)

        mo = [self.moments(a, hh[a]) + self.moments2(a, hh[a]) for a in range(2)]
        DB = d1(mo[1][3]) + d2(mo[1][6])
        D = [1.0 - DB, DB]
        new = []
        for a in range(2):
            Uh, _, W1, _, W2, X12, _ = mo[a]
            G1 = 2.0 * np.sum(F.V1 * F.V3 * (L[a] + self.Nd[a] * self.h[a]), axis=ax) * w
            G2 = 2.0 * np.sum(F.V2 * F.V3 * (L[a] + self.Nd[a] * self.h[a]), axis=ax) * w
            rhs = (-self.Nd[a] / mix.r[a] * D[a]
                   - (W1[I + 1, J] - 2.0 * W1[I, J] + W1[I - 1, J]) / dx ** 2
                   - 2.0 * (X12[I + 1, J + 1] - X12[I + 1, J - 1] - X12[I - 1, J + 1] + X12[I - 1, J - 1])
                   / (4.0 * dx * dy)
                   - (W2[I, J + 1] - 2.0 * W2[I, J] + W2[I, J - 1]) / dy ** 2
                   + d1(G1) + d2(G2))
            Un = self.poisson(Uh, rhs, mix.chi[a])
            new.append(hh[a] + 2.0 * mix.r[a] * (Un - Uh)[(...,) + (None,) * 3] * F.V3 * F.f[a])
        return new

    def march(self, Y0, src):
        a, b, c = transport.march_coeffs(self.x)
        Y = np.zeros(len(self.x))
        Y[0] = Y0
        for i in range(1, len(self.x)):
            r = src[i] - b[i] * Y[i - 1]
            if i >= 2:
                r -= c[i] * Y[i - 2]
            Y[i] = r / a[i]
        return Y

    def step(self):
        F, pb = self.F, self.pb
        mix, d = pb.mix, pb.delta
        lpA, LA, lpB, LB = F.apply(self.h[0], self.h[1], d)
        lp, L = [lpA, lpB], [LA, LB]
        if pb.dim == 1:
            hh = [transport.sweep_1d(lp[a] + self.S[a], d * F.nu[a], F.V1, self.x) for a in range(2)]
        elif pb.solid > 0:
            hh = [sweep_porous(lp[a] + self.S[a], d * F.nu[a], F.V1, F.V2, self.solid, self.hprev[a])
                  for a in range(2)]
            self.hprev = hh
        else:
            hh = [transport.sweep_2d(lp[a] + self.S[a], d * F.nu[a], F.V1, F.V2, pb.nx, pb.ny, pb.width)
                  for a in range(2)]
        if pb.scheme == "cis":
            self.h = hh
        elif pb.dim == 2 and pb.solid > 0:
            self.h = self.step_porous(L, hh)
        elif pb.dim == 2:
            self.h = self.step2(L, hh)
        else:
            w = F.dv ** 3
            G = [2.0 * np.sum(F.V1 * F.V3 * (L[a] + self.Nd[a] * self.h[a]), axis=(-3, -2, -1)) * w
                 for a in range(2)]
            mo = [self.moments(a, hh[a]) for a in range(2)]
            Ptil = [self.x - mo[1][3], mo[1][3]]
            new = []
            for a in range(2):
                Uh, _, W, _ = mo[a]
                chi, r = mix.chi[a], mix.r[a]
                Y = self.march(chi * Uh[0] + W[0], G[a] - self.Nd[a] / r * Ptil[a])
                Un = (Y - W) / chi
                dU = Un - Uh
                new.append(hh[a] + 2.0 * r * dU[(...,) + (None,) * 3] * F.V3 * F.f[a])
            self.h = new
        mo = [self.moments(a, self.h[a]) for a in range(2)]
        s = np.sqrt(mix.mbar)
        self.U = [mo[0][0], mo[1][0]]
        self.iters += 1
        if pb.dim == 2:
            return np.array([s * np.mean(mo[0][0]), s * np.mean(mo[1][0]), s * np.mean(mo[0][1]),
                             s * np.mean(mo[1][1])])
        return np.array([s * 2.0 * np.trapezoid(mo[0][0], self.x), s * 2.0 * np.trapezoid(mo[1][0], self.x),
                         s * 2.0 * np.trapezoid(mo[0][1], self.x), s * 2.0 * np.trapezoid(mo[1][1], self.x)])

    def solve(self, eps=None, max_iter=None):
        eps = self.pb.eps if eps is None else eps
        max_iter = self.pb.max_iter if max_iter is None else max_iter
        while self.iters < max_iter:
            old = self.rates
            self.rates = self.step()
            if np.all(np.abs(self.rates - old) < eps * np.abs(self.rates)):
                return True
        return False
