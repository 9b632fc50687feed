// Host construction of the discrete hard-sphere collision operator's tables (double).
//
// Operator (Sec. 2, Eq. LBE_collision, hard spheres, fast spectral form):
//   gain(h) = sum_p w'_p [ A_p F^-1(psi_p F h) + B_p F^-1(phi_p F h) ],
//   A_p = F^-1(phi_p F f_eq), B_p = F^-1(psi_p F f_eq), w'_p = 2 b w_p, K = 4 pi b,
//   loss(h) = f_eq F^-1(G F h) + nu_eq h,   G = sum_p w'_p phi_p psi_p,  nu_eq = F^-1(G F f_eq),
//   phi(s) = 2 int_0^R r cos(r s) dr,  psi(a) = 4 pi R J1(R a) / a,
//   phi_p(xi) = phi(xi . e_p), psi_p(xi) = psi(|xi - (xi . e_p) e_p|),
//   K = 5 sqrt(2 pi) / 16 at delta = 1 so that nu_bar = 1.25 delta (Sec. 2.5).
// Directions: n_t Gauss-Legendre nodes in cos(theta) on [0,1] times n_a midpoint azimuths,
// n_t = 2^floor(log2(M)/2); the sphere integral is even in e, hence the hemisphere x 2.
// F is the plain DFT on the midpoint grid (the multipliers act as cyclic convolutions, so
// the grid offset cancels); Nyquist planes are zeroed in every multiplier.
#include <algorithm>
#include <cmath>
#include <complex>
#include <stdexcept>
#include <vector>

#include "lbe_internal.h"

namespace lbe {

namespace {

using cd = std::complex<double>;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            double dp = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double pn = (n == 1) ? z : p1, pnm1 = (n == 1) ? 1.0 : p0;
        double dp = n * (z * pn - pnm1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

double phi_fn(double s, double R) {
    double x = R * s;
    if (std::fabs(x) < 1e-3) return R * R * (1.0 - x * x / 4.0 + x * x * x * x / 72.0);
    double sh = std::sin(0.5 * x);
    return 2.0 * R * R * (std::sin(x) / x - 2.0 * sh * sh / (x * x));
}

double psi_fn(double a, double R) {
    double x = R * a;
    if (std::fabs(x) < 1e-3) return 4.0 * M_PI * R * R * (0.5 - x * x / 16.0 + x * x * x * x / 384.0);
    return 4.0 * M_PI * R * R * std::cyl_bessel_j(1.0, x) / x;
}

// In-place separable 3D DFT (direct, O(n^4)), sign -1 forward, +1 inverse (no scaling).
void dft3(std::vector<cd>& a, int n, int sign) {
    std::vector<cd> tw(n);
    for (int m = 0; m < n; ++m) tw[m] = std::polar(1.0, sign * 2.0 * M_PI * m / n);
    std::vector<cd> line(n), out(n);
    const int strides[3] = {n * n, n, 1};
    for (int ax = 0; ax < 3; ++ax) {
        int s = strides[ax];
        for (int base = 0; base < n * n * n; ++base) {
            // base enumerates line starts: index along axis must be 0
            if ((base / s) % n != 0) continue;
            for (int j = 0; j < n; ++j) line[j] = a[base + j * s];
            for (int k = 0; k < n; ++k) {
                cd acc = 0;
                for (int j = 0; j < n; ++j) acc += line[j] * tw[(j * k) % n];
                out[k] = acc;
            }
            for (int k = 0; k < n; ++k) a[base + k * s] = out[k];
        }
    }
}

}  // namespace

double default_R(double vmax) { return 0.75 * vmax; }

double carleman_phi(double s, double R) { return phi_fn(s, R); }
double carleman_psi(double a, double R) { return psi_fn(a, R); }
void host_dft3(std::vector<std::complex<double>>& a, int n, int sign) { dft3(a, n, sign); }

void hemisphere_rule(int M, std::vector<double>& e, std::vector<double>& w) {
    int nt = 1;
    while (nt * nt * 4 <= M) nt *= 2;  // nt = 2^floor(log2(M)/2)
    const int na = M / nt;
    std::vector<double> gx, gw;
    gauss_legendre(nt, gx, gw);
    e.resize(3 * (size_t)M);
    w.resize(M);
    for (int i = 0; i < nt; ++i) {
        const double mu = 0.5 * (gx[i] + 1.0), wmu = 0.5 * gw[i], st = std::sqrt(1.0 - mu * mu);
        for (int k = 0; k < na; ++k) {
            const double az = (k + 0.5) * 2.0 * M_PI / na;
            const int p = i * na + k;
            e[3 * p + 0] = st * std::cos(az);
            e[3 * p + 1] = st * std::sin(az);
            e[3 * p + 2] = mu;
            w[p] = wmu * 2.0 * M_PI / na;
        }
    }
}

void build_host_tables(HostTables& t, int nv, double vmax, int M, double R) {
    const int n = nv, n3 = nv * nv * nv;
    t.nv = nv;
    t.M = M;
    t.vmax = vmax;
    t.R = R;
    t.dv = 2.0 * vmax / nv;
    t.v.resize(n);
    for (int j = 0; j < n; ++j) t.v[j] = -vmax + (j + 0.5) * t.dv;
    t.feq.resize(n3);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double c2 = t.v[i] * t.v[i] + t.v[j] * t.v[j] + t.v[k] * t.v[k];
                t.feq[(i * n + j) * n + k] = std::exp(-c2) / std::pow(M_PI, 1.5);
            }
    // directions
    int nt = 1;
    while (nt * nt * 4 <= M) nt *= 2;  // nt = 2^floor(log2(M)/2)
    const int na = M / nt;
    std::vector<double> gx, gw;
    gauss_legendre(nt, gx, gw);
    std::vector<double> e(3 * M), wp(M);
    const double K = 5.0 * std::sqrt(2.0 * M_PI) / 16.0;
    const double b = K / (4.0 * M_PI);
    // Storage order: directions grouped by their orbit under the reflections v2 -> -v2,
    // v3 -> -v3 (azimuth k -> n_a-1-k, k -> k+n_a/2): first every ring's k < n_a/4, then
    // n_a/4 <= k < n_a/2, then the rest.  The first M/4 (M/2) directions are one
    // representative per orbit of the group {1, R2, R3, R2R3} ({1, R3}).
    auto klass = [&](int k) { return (na % 4 == 0 && k < na / 4) ? 0 : (k < na / 2 ? 1 : 2); };
    std::vector<std::pair<int, int>> order;  // (class, i*na+k) sorted
    for (int i = 0; i < nt; ++i)
        for (int k = 0; k < na; ++k) order.push_back({klass(k), i * na + k});
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int, int>& a, const std::pair<int, int>& b) { return a.first < b.first; });
    std::vector<int> slot_of(M);
    for (int q = 0; q < M; ++q) slot_of[order[q].second] = q;
    t.sym_reps1 = (na % 2 == 0) ? M / 2 : 0;
    t.sym_reps2 = (na % 4 == 0) ? M / 4 : 0;
    for (int i = 0; i < nt; ++i) {
        double mu = 0.5 * (gx[i] + 1.0), wmu = 0.5 * gw[i];
        double st = std::sqrt(1.0 - mu * mu);
        for (int k = 0; k < na; ++k) {
            double az = (k + 0.5) * 2.0 * M_PI / na;
            int p = slot_of[i * na + k];
            e[3 * p + 0] = st * std::cos(az);
            e[3 * p + 1] = st * std::sin(az);
            e[3 * p + 2] = mu;
            wp[p] = 2.0 * b * wmu * 2.0 * M_PI / na;
        }
    }
    // frequencies in DFT order
    std::vector<double> xi(n);
    for (int k = 0; k < n; ++k) xi[k] = ((k < n / 2) ? k : k - n) * M_PI / vmax;
    const double inv_n3 = 1.0 / n3;
    t.mult.assign(2 * (size_t)(M + 1) * n3, 0.0);
    std::vector<double> G(n3, 0.0);
    for (int p = 0; p < M; ++p) {
        for (int a = 0; a < n; ++a)
            for (int bb = 0; bb < n; ++bb)
                for (int c = 0; c < n; ++c) {
                    int idx = (a * n + bb) * n + c;
                    if (a == n / 2 || bb == n / 2 || c == n / 2) continue;  // Nyquist planes
                    double s = xi[a] * e[3 * p] + xi[bb] * e[3 * p + 1] + xi[c] * e[3 * p + 2];
                    double x2 = xi[a] * xi[a] + xi[bb] * xi[bb] + xi[c] * xi[c];
                    double perp = std::sqrt(std::max(x2 - s * s, 0.0));
                    double ph = phi_fn(s, R), ps = psi_fn(perp, R);
                    t.mult[2 * ((size_t)p * n3 + idx) + 0] = ps * inv_n3;
                    t.mult[2 * ((size_t)p * n3 + idx) + 1] = ph * inv_n3;
                    G[idx] += wp[p] * ph * ps;
                }
    }
    for (int idx = 0; idx < n3; ++idx) t.mult[2 * ((size_t)M * n3 + idx)] = G[idx] * inv_n3;
    // A_p, B_p, nu_eq from F f_eq
    std::vector<cd> Feq(n3);
    for (int i = 0; i < n3; ++i) Feq[i] = t.feq[i];
    dft3(Feq, n, -1);
    t.ab.assign(2 * (size_t)M * n3, 0.0);
    std::vector<cd> work(n3);
    for (int p = 0; p < M; ++p) {
        for (int i = 0; i < n3; ++i) {
            cd m(t.mult[2 * ((size_t)p * n3 + i)], t.mult[2 * ((size_t)p * n3 + i) + 1]);
            work[i] = m * Feq[i];                 // (psi + i phi) F f_eq / n^3
        }
        dft3(work, n, +1);
        for (int i = 0; i < n3; ++i) {
            t.ab[2 * ((size_t)p * n3 + i) + 0] = wp[p] * work[i].imag();  // w' A_p
            t.ab[2 * ((size_t)p * n3 + i) + 1] = wp[p] * work[i].real();  // w' B_p
        }
    }
    for (int i = 0; i < n3; ++i) work[i] = t.mult[2 * ((size_t)M * n3 + i)] * Feq[i];
    dft3(work, n, +1);
    t.nu1.resize(n3);
    for (int i = 0; i < n3; ++i) t.nu1[i] = work[i].real();
    double dv3 = t.dv * t.dv * t.dv;
    t.cU = 0;
    t.cq = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                int idx = (i * n + j) * n + k;
                double v3 = t.v[k], c2 = t.v[i] * t.v[i] + t.v[j] * t.v[j] + v3 * v3;
                t.cU += v3 * v3 * t.feq[idx] * dv3;
                t.cq += (c2 - 2.5) * v3 * v3 * t.feq[idx] * dv3;
            }
}

}  // namespace lbe
