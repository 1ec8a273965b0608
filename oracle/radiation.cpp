// Oracle radiation half: grid sampling (Sec. 2.4), plasma state and thermal synchrotron
// coefficients (Sec. 2.5), polarized transfer (Sec. 2.3.2) and the per-pixel driver.
// Test infrastructure only (see oracle.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "oracle.h"
#include "oracle_internal.hpp"

namespace ora {

// CGS constants (CODATA 2018 / IAU 2015 nominal solar mass).
static const double C_LIGHT = 2.99792458e10;
static const double E_CHARGE = 4.80320471e-10;
static const double M_ELECTRON = 9.1093837015e-28;
static const double M_PROTON = 1.67262192369e-24;
static const double H_PLANCK = 6.62607015e-27;
static const double G_NEWTON = 6.67430e-8;
static const double M_SUN = 1.98841e33;

// ---------------------------------------------------------------------------------------
// Modified Bessel function of the second kind from its integral representation
//   K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt,
// returned scaled as exp(x) K_nu(x). The integrand is even and decays double-exponentially,
// so the trapezoid rule with step 0.02 converges far below double rounding.
// ---------------------------------------------------------------------------------------
double bessel_kx(double nu, double x) {
    const double h = 0.02;
    double sum = 0.5;   // t = 0 term: exp(0) cosh(0) / 2
    for (int i = 1; i < 100000; ++i) {
        double t = i * h;
        double term = std::exp(-x * (std::cosh(t) - 1.0)) * std::cosh(nu * t);
        sum += term;
        if (term < 1e-19 * sum) break;
    }
    return h * sum;
}

// ---------------------------------------------------------------------------------------
// Thermal synchrotron coefficients in the fluid frame (Sec. 2.5). The paper cites the fits
// without printing them; the forms below are the published thermal fits:
//   emission: j_S = n e^2 nu / (sqrt(3) c K_2(1/Theta)) * I_S(x),  S = I, Q
//             j_V = 4 n e^2 nu cot(theta) / (3 sqrt(3) c Theta K_2(1/Theta)) * I_V(x)
//             x = nu / nu_c', nu_c' = (3/2) nu_B sin(theta) Theta^2, nu_B = e B / (2 pi m c)
//             (Mahadevan, Narayan & Yi 1996 / Dexter 2016 shapes, Maxwell-Juettner
//              normalisation kept exact through K_2, Leung et al. 2011)
//   absorption: Kirchhoff, alpha_S = j_S / B_nu(T_e)
//   rotation:   rho_Q = n e^2 nu_B^2 sin^2 / (m c nu^3) f_m(X) [K_1/K_2 + 6 Theta]
//               rho_V = 2 n e^2 nu_B cos / (m c nu^2) K_0/K_2 g_m(X)
//               X = Theta sqrt(sqrt(2) sin(theta) 1e3 nu_B / nu)   (Shcherbakov 2008)
// Sign convention: Stokes Q > 0 is polarization perpendicular to the projected field.
// ---------------------------------------------------------------------------------------
void coefficients(double ne, double th_e, double bg, double nu, double cth, double out[8]) {
    for (int q = 0; q < 8; ++q) out[q] = 0.0;
    if (ne <= 0.0 || th_e <= 0.0 || bg <= 0.0) return;
    double sth2 = 1.0 - cth * cth;
    double sth = std::sqrt(sth2 > 0.0 ? sth2 : 0.0);
    double nub = E_CHARGE * bg / (2.0 * M_PI * M_ELECTRON * C_LIGHT);
    double z = 1.0 / th_e;
    double k2x = bessel_kx(2.0, z);   // exp(z) K_2(z)
    double k1x = bessel_kx(1.0, z);
    double k0x = bessel_kx(0.0, z);
    if (sth > 0.0) {
        double nucp = 1.5 * nub * sth * th_e * th_e;
        double x = nu / nucp;
        double x13 = std::cbrt(x);
        double x23 = x13 * x13;
        // 1 / K_2(z) = exp(z) / (exp(z) K_2(z)); exp(z) joins the shape functions' factor
        // exp(-1.8899 x^1/3) in one exponential, which stays finite (and underflows to 0)
        // for cold plasma where exp(z) = exp(1 / Theta_e) alone overflows
        double ex = std::exp(z - 1.8899 * x13);
        double ii = 2.5651 * (1.0 + 1.92 / x13 + 0.9977 / x23) * ex;
        double iq = 2.5651 * (1.0 + 0.932 / x13 + 0.4998 / x23) * ex;
        double iv = (1.8138 / x + 3.423 / x23 + 0.02955 / std::sqrt(x) + 2.0377 / x13) * ex;
        double pre = ne * E_CHARGE * E_CHARGE * nu / (std::sqrt(3.0) * C_LIGHT) / k2x;
        out[0] = pre * ii;
        out[1] = pre * iq;
        out[2] = pre * 4.0 / (3.0 * th_e) * (cth / sth) * iv;
        double hnu_kt = H_PLANCK * nu / (th_e * M_ELECTRON * C_LIGHT * C_LIGHT);
        double bnu = 2.0 * H_PLANCK * nu * nu * nu / (C_LIGHT * C_LIGHT) / std::expm1(hnu_kt);
        out[3] = out[0] / bnu;
        out[4] = out[1] / bnu;
        out[5] = out[2] / bnu;
    }
    double xx = th_e * std::sqrt(std::sqrt(2.0) * sth * 1.0e3 * nub / nu);
    double fm = 2.011 * std::exp(-std::pow(xx, 1.035) / 4.7) -
                std::cos(0.5 * xx) * std::exp(-std::pow(xx, 1.2) / 2.73) -
                0.011 * std::exp(-xx / 47.2);
    double gm = 1.0 - 0.11 * std::log(1.0 + 0.035 * xx);
    double base = ne * E_CHARGE * E_CHARGE / (M_ELECTRON * C_LIGHT);
    out[6] = base * nub * nub * sth2 / (nu * nu * nu) * fm * (k1x / k2x + 6.0 * th_e);
    out[7] = 2.0 * base * nub * cth / (nu * nu) * (k0x / k2x) * gm;
}

// ---------------------------------------------------------------------------------------
// Grid sampling (Sec. 2.4): trilinear in (ln r, theta, phi) between cell centres, phi
// periodic, theta and r clamped to the edge cells; outside [r_min, r_max] there is no data.
// ---------------------------------------------------------------------------------------
// One snapshot (spatial sampling only); slow light combines snapshots below.
static int32_t sample_snapshot(const ora_grid* gr, const float* data, double a, const double x[4],
                               double prim[8]);

int32_t sample_grid(const ora_grid* gr, double a, const double x[4], double prim[8]) {
    if (gr->n_snapshots <= 1) return sample_snapshot(gr, gr->prim, a, x, prim);
    // Slow light: the sample's time t_camera + x^t on the snapshot axis, clamped to its ends
    const size_t snap = (size_t)8 * gr->n_phi * gr->n_theta * gr->n_r;
    const int ns = gr->n_snapshots;
    double s = (gr->t_camera + x[0] - gr->t_first) / gr->dt;
    if (s < 0.0) s = 0.0;
    if (s > ns - 1) s = ns - 1;
    if (gr->time_interp == 0) {
        const int k = (int)std::floor(s + 0.5);
        return sample_snapshot(gr, gr->prim + k * snap, a, x, prim);
    }
    int k0 = (int)std::floor(s);
    if (k0 > ns - 2) k0 = ns - 2;
    const double w = s - k0;
    double p0[8], p1[8];
    if (!sample_snapshot(gr, gr->prim + k0 * snap, a, x, p0)) return 0;
    sample_snapshot(gr, gr->prim + (k0 + 1) * snap, a, x, p1);
    for (int v = 0; v < 8; ++v) prim[v] = (1.0 - w) * p0[v] + w * p1[v];
    return 1;
}

static int32_t sample_snapshot(const ora_grid* gr, const float* data, double a, const double x[4],
                               double prim[8]) {
    double r, th, ph;
    cks_to_sks_point(x, a, &r, &th, &ph);
    if (!(r >= gr->r_min && r <= gr->r_max)) return 0;
    const int nr = gr->n_r, nt = gr->n_theta, np = gr->n_phi;
    double dlr = std::log(gr->r_max / gr->r_min) / nr;
    double dth = M_PI / nt;
    double dph = 2.0 * M_PI / np;
    auto at = [&](int v, int k, int j, int i) -> double {
        return (double)data[(((size_t)v * np + k) * nt + j) * nr + i];
    };
    if (gr->interp == 0) {
        int i = (int)std::floor(std::log(r / gr->r_min) / dlr);
        int j = (int)std::floor(th / dth);
        int k = (int)std::floor(ph / dph);
        i = std::min(std::max(i, 0), nr - 1);
        j = std::min(std::max(j, 0), nt - 1);
        k = ((k % np) + np) % np;
        for (int v = 0; v < 8; ++v) prim[v] = at(v, k, j, i);
        return 1;
    }
    auto axis = [](double fi, int n, int& i0, int& i1, double& w) {
        if (n == 1) { i0 = i1 = 0; w = 0.0; return; }
        if (fi < 0.0) fi = 0.0;
        if (fi > n - 1) fi = n - 1;
        i0 = (int)std::floor(fi);
        if (i0 > n - 2) i0 = n - 2;
        i1 = i0 + 1;
        w = fi - i0;
    };
    int i0, i1, j0, j1;
    double wr, wt;
    axis(std::log(r / gr->r_min) / dlr - 0.5, nr, i0, i1, wr);
    axis(th / dth - 0.5, nt, j0, j1, wt);
    double fk = ph / dph - 0.5;
    double fkf = std::floor(fk);
    int k0 = (((int)fkf) % np + np) % np;
    int k1 = (k0 + 1) % np;
    double wp = fk - fkf;
    for (int v = 0; v < 8; ++v) {
        double s = 0.0;
        s += (1 - wp) * (1 - wt) * (1 - wr) * at(v, k0, j0, i0);
        s += (1 - wp) * (1 - wt) * wr * at(v, k0, j0, i1);
        s += (1 - wp) * wt * (1 - wr) * at(v, k0, j1, i0);
        s += (1 - wp) * wt * wr * at(v, k0, j1, i1);
        s += wp * (1 - wt) * (1 - wr) * at(v, k1, j0, i0);
        s += wp * (1 - wt) * wr * at(v, k1, j0, i1);
        s += wp * wt * (1 - wr) * at(v, k1, j1, i0);
        s += wp * wt * wr * at(v, k1, j1, i1);
        prim[v] = s;
    }
    return 1;
}

// ---------------------------------------------------------------------------------------
// Plasma state at a sample point (Secs. 2 and 2.5). Returns 1 if the point carries plasma
// (inside the grid, finite interpolated data, sigma <= sigma_cut, positive density, pressure
// and field: the sigma cut is the only data cut of the paper's default set-up).
// u, b are contravariant CKS components.
// ---------------------------------------------------------------------------------------
int32_t plasma(const ora_grid* gr, const ora_metric* met, const double x[4], double u[4],
               double b[4], double* ne, double* th_e, double* bg, double* qv) {
    const double m = met->mass, a = met->spin;
    double prim[8];
    if (!sample_grid(gr, a, x, prim)) return 0;
    // non-finite data carry no plasma (the paper does not treat them; read like a sample
    // outside the grid)
    for (int q = 0; q < 8; ++q)
        if (!std::isfinite(prim[q])) return 0;
    double r, th, ph;
    cks_to_sks_point(x, a, &r, &th, &ph);
    double rho = prim[0], ugas = prim[1];
    // Velocity and field vectors mapped to CKS (Sec. 2: data in spherical KS are transformed
    // to the singularity-free Cartesian system before use).
    normal_to_cks(x, r, th, ph, m, a, met->flat, prim + 2, u);
    double jac[9];
    sks_jacobian(r, th, ph, a, jac);
    double bcap[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c)
        for (int i = 0; i < 3; ++i) bcap[c + 1] += jac[3 * c + i] * prim[5 + i];
    double glo[16];
    metric_cks(x, m, a, met->flat, glo, nullptr);
    double ulo[4];
    for (int al = 0; al < 4; ++al) {
        double s = 0.0;
        for (int be = 0; be < 4; ++be) s += glo[4 * al + be] * u[be];
        ulo[al] = s;
    }
    // b^t = B^i u_i, b^i = (B^i + b^t u^i) / u^t
    b[0] = bcap[1] * ulo[1] + bcap[2] * ulo[2] + bcap[3] * ulo[3];
    for (int c = 1; c < 4; ++c) b[c] = (bcap[c] + b[0] * u[c]) / u[0];
    double bsq = 0.0;
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be) bsq += glo[4 * al + be] * b[al] * b[be];
    double p = (gr->gamma_ad - 1.0) * ugas;
    if (!(rho > 0.0) || !(p > 0.0) || !(bsq > 0.0)) return 0;
    double sigma = bsq / rho;
    if (sigma > gr->sigma_cut) return 0;
    double beta_inv = bsq / (2.0 * p);
    double b2 = beta_inv * beta_inv;                          // beta^{-2}
    double ti_te = (gr->r_high + b2 * gr->r_low) / (1.0 + b2);
    double rr = gr->ne_over_ni;
    double te = gr->mu * M_PROTON / M_ELECTRON * (p / rho) * (rr + 1.0) / (rr + ti_te);
    *th_e = te;
    *ne = rho * gr->rho_unit_cgs / (gr->mu * M_PROTON) / (1.0 + 1.0 / rr);
    *bg = std::sqrt(bsq) * C_LIGHT * std::sqrt(4.0 * M_PI * gr->rho_unit_cgs);
    if (qv) {   // the tracked quantities of the auxiliary images (Sec. 4)
        qv[0] = rho; qv[1] = *ne; qv[2] = p; qv[3] = te; qv[4] = *bg; qv[5] = sigma;
        qv[6] = beta_inv;
    }
    return 1;
}

// ---------------------------------------------------------------------------------------
// Unpolarized segment (Eq. unpolarized): exact solution of dI/dl = j - alpha I over dl with
// constant coefficients; alpha dl >= 100 gives j / alpha, alpha = 0 gives I + j dl.
// ---------------------------------------------------------------------------------------
double unpolarized_step(double j, double alpha, double dl, double i0) {
    if (alpha > 0.0) {
        const double dtau = alpha * dl;
        if (dtau >= 100.0) return j / alpha;
        return std::exp(-dtau) * (i0 + std::expm1(dtau) * j / alpha);
    }
    return i0 + j * dl;
}

// ---------------------------------------------------------------------------------------
// Constant-coefficient polarized step: dS/dl = J - M S over dl, with M the Mueller-type
// matrix of absorption and rotation (U-terms zero in the field-aligned basis). The exact
// solution is the exponential of the augmented 5x5 matrix [[-M dl, J dl], [0, 0]], computed
// by scaling and squaring with a Taylor series in long double. For alpha_I dl >= 100 the
// solution is the steady state M^{-1} J (the polarized form of the Delta tau_max rule,
// Eq. unpolarized).
// ---------------------------------------------------------------------------------------
typedef long double LD;

static void build_m(const double c[8], LD M[4][4]) {
    const LD aI = c[3], aQ = c[4], aV = c[5], rQ = c[6], rV = c[7];
    const LD aU = 0, rU = 0;
    LD m[4][4] = {{aI, aQ, aU, aV}, {aQ, aI, rV, -rU}, {aU, -rV, aI, rQ}, {aV, rU, -rQ, aI}};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) M[i][j] = m[i][j];
}

void stokes_step(const double c[8], const double s0[4], double dl, double s1[4]) {
    LD M[4][4];
    build_m(c, M);
    LD J[4] = {c[0], c[1], 0.0L, c[2]};
    if (c[3] * dl >= 100.0) {
        // Solve M S = J by Gaussian elimination with partial pivoting.
        LD a[4][5];
        for (int i = 0; i < 4; ++i) {
            for (int j = 0; j < 4; ++j) a[i][j] = M[i][j];
            a[i][4] = J[i];
        }
        for (int col = 0; col < 4; ++col) {
            int p = col;
            for (int i = col + 1; i < 4; ++i)
                if (fabsl(a[i][col]) > fabsl(a[p][col])) p = i;
            for (int j = 0; j < 5; ++j) std::swap(a[p][j], a[col][j]);
            for (int i = col + 1; i < 4; ++i) {
                LD f = a[i][col] / a[col][col];
                for (int j = col; j < 5; ++j) a[i][j] -= f * a[col][j];
            }
        }
        LD x[4];
        for (int i = 3; i >= 0; --i) {
            LD s = a[i][4];
            for (int j = i + 1; j < 4; ++j) s -= a[i][j] * x[j];
            x[i] = s / a[i][i];
        }
        for (int i = 0; i < 4; ++i) s1[i] = (double)x[i];
        return;
    }
    LD B[5][5] = {};
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) B[i][j] = -M[i][j] * dl;
        B[i][4] = J[i] * dl;
    }
    LD norm = 0;
    for (int i = 0; i < 5; ++i) {
        LD s = 0;
        for (int j = 0; j < 5; ++j) s += fabsl(B[i][j]);
        norm = std::max(norm, s);
    }
    int sq = 0;
    while (norm > 0.5L) { norm *= 0.5L; ++sq; }
    LD scale = ldexpl(1.0L, -sq);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) B[i][j] *= scale;
    LD E[5][5] = {}, T[5][5] = {};
    for (int i = 0; i < 5; ++i) E[i][i] = T[i][i] = 1.0L;
    for (int n = 1; n < 40; ++n) {
        LD nt[5][5] = {};
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                LD s = 0;
                for (int q = 0; q < 5; ++q) s += T[i][q] * B[q][j];
                nt[i][j] = s / n;
            }
        LD mx = 0;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) { T[i][j] = nt[i][j]; E[i][j] += nt[i][j]; mx = std::max(mx, fabsl(nt[i][j])); }
        if (mx < 1e-30L) break;
    }
    for (int s = 0; s < sq; ++s) {
        LD e2[5][5] = {};
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                LD acc = 0;
                for (int q = 0; q < 5; ++q) acc += E[i][q] * E[q][j];
                e2[i][j] = acc;
            }
        std::memcpy(E, e2, sizeof(E));
    }
    for (int i = 0; i < 4; ++i) {
        LD acc = E[i][4];
        for (int j = 0; j < 4; ++j) acc += E[i][j] * (LD)s0[j];
        s1[i] = (double)acc;
    }
}

// ---------------------------------------------------------------------------------------
// Coordinate (parallel-transport) terms of Eq. polarized_n, read as
//   dN^{ab}/dl = -k^c (Gamma^a_{cd} N^{db} + Gamma^b_{cd} N^{ad})  (= A N + N A^T),
// with A^a_d = -k^c Gamma^a_{cd}, advanced by the predictor-corrector of Table tab:pc
// (stage 1 at the start point, stage 2 evaluated at the supplied second point).
// ---------------------------------------------------------------------------------------
static void transport_matrix(const ora_metric* met, const double x[4], const double klo[4],
                             double A[16]) {
    double gam[64], ghi[16];
    christoffel(x, met->mass, met->spin, met->flat, gam);
    metric_cks(x, met->mass, met->spin, met->flat, nullptr, ghi);
    double kup[4];
    for (int a = 0; a < 4; ++a) {
        double s = 0.0;
        for (int b = 0; b < 4; ++b) s += ghi[4 * a + b] * klo[b];
        kup[a] = s;
    }
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 4; ++d) {
            double s = 0.0;
            for (int c = 0; c < 4; ++c) s += kup[c] * gam[16 * a + 4 * c + d];
            A[4 * a + d] = -s;
        }
}

static void transport_rhs(const double A[16], const double N[16], double out[16]) {
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            double s = 0.0;
            for (int d = 0; d < 4; ++d) s += A[4 * a + d] * N[4 * d + b] + A[4 * b + d] * N[4 * a + d];
            out[4 * a + b] = s;
        }
}

void transport_step(const ora_metric* met, const double x0[4], const double k0[4],
                    const double x1[4], const double k1[4], double h, double nre[16],
                    double nim[16]) {
    double A0[16], A1[16];
    transport_matrix(met, x0, k0, A0);
    transport_matrix(met, x1, k1, A1);
    for (double* N : {nre, nim}) {
        double f0[16], nh[16], f1[16];
        transport_rhs(A0, N, f0);
        for (int q = 0; q < 16; ++q) nh[q] = N[q] + 0.5 * h * f0[q];
        transport_rhs(A1, nh, f1);
        for (int q = 0; q < 16; ++q) N[q] += h * f1[q];
    }
}

// ---------------------------------------------------------------------------------------
// Fluid-frame polarization basis (Moscibrodzka & Gammie 2018 convention as read here):
// e3 = spatial direction of k, e2 = field direction perpendicular to e3, e1 = e2 x e3.
// Stokes <-> coherency: N11 = (I+Q)/2, N22 = (I-Q)/2, N12 = (U + iV)/2.
// ---------------------------------------------------------------------------------------
static double dot4(const double g[16], const double a[4], const double b[4]) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) s += g[4 * i + j] * a[i] * b[j];
    return s;
}

static void lower(const double g[16], const double a[4], double out[4]) {
    for (int i = 0; i < 4; ++i) {
        double s = 0.0;
        for (int j = 0; j < 4; ++j) s += g[4 * i + j] * a[j];
        out[i] = s;
    }
}

static int perm_sign(int a, int b, int c, int d) {
    int p[4] = {a, b, c, d};
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
            if (p[i] == p[j]) return 0;
    int s = 1;
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
            if (p[i] > p[j]) s = -s;
    return s;
}

static double det4(const double m[16]) {
    double s = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c)
                for (int d = 0; d < 4; ++d) {
                    int e = perm_sign(a, b, c, d);
                    if (e) s += e * m[a] * m[4 + b] * m[8 + c] * m[12 + d];
                }
    return s;
}

void tetrad(const double glo[16], const double u[4], const double kup[4], const double b[4],
            double e1[4], double e2[4]) {
    double ku = dot4(glo, kup, u);
    double e3[4];
    for (int i = 0; i < 4; ++i) e3[i] = (kup[i] + ku * u[i]) / (-ku);
    double bu = dot4(glo, b, u);
    double bp[4];
    for (int i = 0; i < 4; ++i) bp[i] = b[i] + bu * u[i];
    double b3 = dot4(glo, bp, e3);
    for (int i = 0; i < 4; ++i) bp[i] -= b3 * e3[i];
    double bb = dot4(glo, bp, bp);
    double bsq = dot4(glo, b, b);
    if (!(bb > 1e-20 * bsq)) {
        // Field along the ray: any transverse direction serves (only I and V couple).
        const double trial[2][4] = {{0, 0, 0, 1}, {0, 1, 0, 0}};
        for (int t = 0; t < 2; ++t) {
            for (int i = 0; i < 4; ++i) bp[i] = trial[t][i];
            double pu = dot4(glo, bp, u);
            for (int i = 0; i < 4; ++i) bp[i] += pu * u[i];
            double p3 = dot4(glo, bp, e3);
            for (int i = 0; i < 4; ++i) bp[i] -= p3 * e3[i];
            bb = dot4(glo, bp, bp);
            if (bb > 1e-6) break;
        }
    }
    double inv = 1.0 / std::sqrt(bb);
    for (int i = 0; i < 4; ++i) e2[i] = bp[i] * inv;
    // e1^a = [abcd] u_b e2_c e3_d / sqrt(-g)
    double ul[4], e2l[4], e3l[4];
    lower(glo, u, ul);
    lower(glo, e2, e2l);
    lower(glo, e3, e3l);
    double sg = std::sqrt(-det4(glo));
    for (int a = 0; a < 4; ++a) {
        double s = 0.0;
        for (int bi = 0; bi < 4; ++bi)
            for (int c = 0; c < 4; ++c)
                for (int d = 0; d < 4; ++d) {
                    int e = perm_sign(a, bi, c, d);
                    if (e) s += e * ul[bi] * e2l[c] * e3l[d];
                }
        e1[a] = s / sg;
    }
}

void n_to_s(const double glo[16], const double e1[4], const double e2[4], const double nre[16],
            const double nim[16], double s[4]) {
    double l1[4], l2[4];
    lower(glo, e1, l1);
    lower(glo, e2, l2);
    double n11 = 0.0, n22 = 0.0, n12r = 0.0, n12i = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            n11 += l1[a] * l1[b] * nre[4 * a + b];
            n22 += l2[a] * l2[b] * nre[4 * a + b];
            n12r += l1[a] * l2[b] * nre[4 * a + b];
            n12i += l1[a] * l2[b] * nim[4 * a + b];
        }
    s[0] = n11 + n22;
    s[1] = n11 - n22;
    s[2] = 2.0 * n12r;
    s[3] = 2.0 * n12i;
}

void s_to_n(const double e1[4], const double e2[4], const double s[4], double nre[16],
            double nim[16]) {
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            nre[4 * a + b] = 0.5 * (s[0] + s[1]) * e1[a] * e1[b] + 0.5 * (s[0] - s[1]) * e2[a] * e2[b] +
                             0.5 * s[2] * (e1[a] * e2[b] + e2[a] * e1[b]);
            nim[4 * a + b] = 0.5 * s[3] * (e1[a] * e2[b] - e2[a] * e1[b]);
        }
}

// ---------------------------------------------------------------------------------------
// Samples along one geodesic (Sec. 2.2): each accepted step contributes its midpoint, or,
// when its proper length (evaluated at the midpoint) exceeds ds_max and the step reaches
// into the grid (start, midpoint or end inside r_max), n = ceil(ds / ds_max) equal
// sub-segments sampled at their centres from the quartic through y0, y1, h f0, h f1, y_mid.
// Each sample carries its affine length and the node on its camera side.
// ---------------------------------------------------------------------------------------
struct Sample {
    double x[4], k[4];     // sample point (state)
    double xn[4], kn[4];   // camera-side node
    double dl;             // affine length of the segment (> 0)
};

static void quartic(const Step& s, double th, double out[8]) {
    for (int q = 0; q < 8; ++q) {
        double y0 = s.y0[q], y1 = s.y1[q], ym = s.ym[q];
        double d0 = s.h * s.f0[q], d1 = s.h * s.f1[q];
        double D1 = y1 - y0 - d0, D2 = d1 - d0, D3 = ym - y0 - 0.5 * d0;
        double c2 = -5.0 * D1 + D2 + 16.0 * D3;
        double c3 = 14.0 * D1 - 3.0 * D2 - 32.0 * D3;
        double c4 = -8.0 * D1 + 2.0 * D2 + 16.0 * D3;
        out[q] = y0 + th * (d0 + th * (c2 + th * (c3 + th * c4)));
    }
}

static double proper_length_rate(const ora_metric* met, const double y[8]) {
    // ds/dl = (g_pq k^p k^q)^{1/2} with k^p = k^a + beta^a k^t the normal-frame components.
    double glo[16], ghi[16];
    metric_cks(y, met->mass, met->spin, met->flat, glo, ghi);
    double kup[4];
    for (int a = 0; a < 4; ++a) {
        double s = 0.0;
        for (int b = 0; b < 4; ++b) s += ghi[4 * a + b] * y[4 + b];
        kup[a] = s;
    }
    double kp[3];
    for (int c = 0; c < 3; ++c) kp[c] = kup[c + 1] + (-ghi[c + 1] / ghi[0]) * kup[0];
    double s = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) s += glo[4 * (c + 1) + d + 1] * kp[c] * kp[d];
    return std::sqrt(s);
}

static void make_samples(const ora_metric* met, const ora_grid* gr, const std::vector<Step>& steps,
                         std::vector<Sample>& out) {
    for (const Step& s : steps) {
        int nsub = 1;
        // Subdivide steps that reach into the grid: start, midpoint or end inside r_max.
        double rm = std::fmin(r_of_x(s.ym, met->spin),
                              std::fmin(r_of_x(s.y0, met->spin), r_of_x(s.y1, met->spin)));
        if (rm < gr->r_max) {
            double ds = std::fabs(s.h) * proper_length_rate(met, s.ym);
            if (ds > met->ds_max) nsub = (int)std::ceil(ds / met->ds_max);
        }
        for (int j = 0; j < nsub; ++j) {
            Sample sp;
            double ysamp[8], ynode[8];
            if (nsub == 1) {
                std::memcpy(ysamp, s.ym, sizeof(ysamp));
                std::memcpy(ynode, s.y0, sizeof(ynode));
            } else {
                quartic(s, (j + 0.5) / nsub, ysamp);
                if (j == 0) std::memcpy(ynode, s.y0, sizeof(ynode));
                else quartic(s, (double)j / nsub, ynode);
            }
            for (int q = 0; q < 4; ++q) {
                sp.x[q] = ysamp[q]; sp.k[q] = ysamp[4 + q];
                sp.xn[q] = ynode[q]; sp.kn[q] = ynode[4 + q];
            }
            sp.dl = std::fabs(s.h) / nsub;
            out.push_back(sp);
        }
    }
}

// ---------------------------------------------------------------------------------------
// One pixel, the whole path: camera -> geodesic -> samples -> transfer (source to camera)
// -> Stokes in the camera basis.
// ---------------------------------------------------------------------------------------
struct PixelResult {
    double stokes[4];
    double end[8];
    int32_t status;
    int64_t attempts, accepted, samples;
    double aux[ORA_AUX_COUNT];
};

// Auxiliary images (Sec. 4, "Auxiliary Images"), per pixel:
//   [0] Kerr-Schild time from the geodesic's termination to the camera, -x^t at the end;
//   [1] proper length of the whole geodesic, sum over steps of |h| (g_pq k^p k^q)^1/2 at the
//       step's midpoint; [2] affine parameter, sum of |h|;
//   [3] I_j = integral of j_I dl, [4] tau = integral of alpha_I dl, over the samples, with the
//       unpolarized invariants per unit affine parameter of the transfer;
//   [5 + k]  <q_k>_lambda = integral q dl / [2];
//   [12 + k] <q_k>_Ij = integral q j_I dl / I_j (0 if I_j = 0);
//   [19 + k] <q_k>_tau, the solution of d<q>/dtau = q - <q> from the source end (0 there),
//            exact for constant q over each sample: <q> -> e^-dtau <q> + (1 - e^-dtau) q;
//   q = rho (code units), n_e, p (code units), Theta_e, B (gauss), sigma, beta^-1. Samples
//   without plasma (outside the grid or cut) contribute q = 0 and no emission or absorption.
static void trace_pixel(const ora_camera* cam, const ora_metric* met, const ora_grid* gr,
                        double freq, int pix, int unpolarized, PixelResult& res) {
    const int i = pix % cam->n, j = pix / cam->n;
    double x[4], k[4], hv[4], vv[4], nnorm, r_cam, ucam[4];
    camera_pixel(cam, met, i, j, x, k, hv, vv, &nnorm, &r_cam, ucam);
    double y0[8];
    for (int q = 0; q < 4; ++q) { y0[q] = x[q]; y0[4 + q] = k[q]; }
    std::vector<Step> steps;
    res.status = integrate(met, r_cam, y0, &steps, res.end, &res.attempts, &res.accepted, nullptr);
    std::vector<Sample> samples;
    make_samples(met, gr, steps, samples);
    res.samples = (int64_t)samples.size();
    for (int a = 0; a < ORA_AUX_COUNT; ++a) res.aux[a] = 0.0;
    res.aux[0] = -res.end[0];
    for (const Step& st : steps) {
        res.aux[1] += std::fabs(st.h) * proper_length_rate(met, st.ym);
        res.aux[2] += std::fabs(st.h);
    }
    double qlam[7] = {0}, qij[7] = {0}, qtau[7] = {0}, i_unpol = 0.0;

    const double length_unit = G_NEWTON * gr->mass_msun * M_SUN / (C_LIGHT * C_LIGHT);
    double nre[16] = {0}, nim[16] = {0};
    bool started = false;
    const int ns = (int)samples.size();
    // Forward order: from the source end (last sample) to the camera.
    for (int m = ns - 1; m >= 0; --m) {
        const Sample& sp = samples[m];
        if (!unpolarized && m < ns - 1 && started) {
            const Sample& prev = samples[m + 1];
            double h = 0.5 * (prev.dl + sp.dl);
            transport_step(met, prev.x, prev.k, prev.xn, prev.kn, h, nre, nim);
        }
        double u[4], b[4], ne, te, bg, qv[7];
        if (!plasma(gr, met, sp.x, u, b, &ne, &te, &bg, qv)) continue;
        double glo[16], ghi[16];
        metric_cks(sp.x, met->mass, met->spin, met->flat, glo, ghi);
        double kup[4];
        for (int a = 0; a < 4; ++a) {
            double s = 0.0;
            for (int c = 0; c < 4; ++c) s += ghi[4 * a + c] * sp.k[c];
            kup[a] = s;
        }
        double ku = 0.0, kb = 0.0;
        for (int a = 0; a < 4; ++a) { ku += sp.k[a] * u[a]; kb += sp.k[a] * b[a]; }
        double nu_fl = nnorm * freq * (-ku);
        double bmag = std::sqrt(dot4(glo, b, b));
        double cth = kb / ((-ku) * bmag);
        if (cth > 1.0) cth = 1.0;
        if (cth < -1.0) cth = -1.0;
        double co[8];
        coefficients(ne, te, bg, nu_fl, cth, co);
        double gfac = freq / nu_fl;
        double path = length_unit * (-ku);
        double coef[8] = {co[0] * gfac * gfac * gfac * path, co[1] * gfac * gfac * gfac * path,
                          co[2] * gfac * gfac * gfac * path, co[3] * path, co[4] * path,
                          co[5] * path, co[6] * path, co[7] * path};
        // auxiliary accumulations (unpolarized invariants j_I = coef[0], alpha_I = coef[3])
        const double dtau = coef[3] * sp.dl;
        res.aux[3] += coef[0] * sp.dl;
        res.aux[4] += dtau;
        for (int q = 0; q < 7; ++q) {
            qlam[q] += qv[q] * sp.dl;
            qij[q] += qv[q] * coef[0] * sp.dl;
            qtau[q] = std::exp(-dtau) * qtau[q] - std::expm1(-dtau) * qv[q];
        }
        if (unpolarized) {
            i_unpol = unpolarized_step(coef[0], coef[3], sp.dl, i_unpol);
            started = true;
            continue;
        }
        double e1[4], e2[4];
        tetrad(glo, u, kup, b, e1, e2);
        double s[4], s1[4];
        n_to_s(glo, e1, e2, nre, nim, s);
        stokes_step(coef, s, sp.dl, s1);
        s_to_n(e1, e2, s1, nre, nim);
        started = true;
    }
    for (int q = 0; q < 7; ++q) {
        res.aux[5 + q] = res.aux[2] > 0.0 ? qlam[q] / res.aux[2] : 0.0;
        res.aux[12 + q] = res.aux[3] > 0.0 ? qij[q] / res.aux[3] : 0.0;
        res.aux[19 + q] = qtau[q];
    }
    if (unpolarized) {
        res.stokes[0] = i_unpol;
        res.stokes[1] = res.stokes[2] = res.stokes[3] = 0.0;
        return;
    }
    if (started && ns > 0) {
        const Sample& last = samples[0];
        transport_step(met, last.x, last.k, last.xn, last.kn, 0.5 * last.dl, nre, nim);
    }
    // Camera readout with e1 = H, e2 = V at the pixel.
    double glo[16];
    metric_cks(x, met->mass, met->spin, met->flat, glo, nullptr);
    n_to_s(glo, hv, vv, nre, nim, res.stokes);
}

}  // namespace ora

// ------------------------------- C entry points ----------------------------------------
extern "C" {

int32_t ora_sample_grid(const ora_grid* grid, double spin, const double x[4], double prim[8]) {
    return ora::sample_grid(grid, spin, x, prim);
}
int32_t ora_plasma(const ora_grid* grid, const ora_metric* met, const double x[4], double u[4],
                   double b[4], double* ne, double* theta_e, double* b_gauss) {
    return ora::plasma(grid, met, x, u, b, ne, theta_e, b_gauss, nullptr);
}
double ora_unpolarized_step(double j, double alpha, double dl, double i0) {
    return ora::unpolarized_step(j, alpha, dl, i0);
}
double ora_bessel_kx(double nu, double x) { return ora::bessel_kx(nu, x); }
void ora_coefficients(double ne, double theta_e, double b_gauss, double nu, double cos_theta,
                      double out[8]) {
    ora::coefficients(ne, theta_e, b_gauss, nu, cos_theta, out);
}
void ora_stokes_step(const double coef[8], const double s0[4], double dlam, double s1[4]) {
    ora::stokes_step(coef, s0, dlam, s1);
}
void ora_transport_step(const ora_metric* met, const double x0[4], const double k0[4],
                        const double x1[4], const double k1[4], double h, double n_re[16],
                        double n_im[16]) {
    ora::transport_step(met, x0, k0, x1, k1, h, n_re, n_im);
}

int64_t ora_ray_samples(const ora_metric* met, const ora_grid* grid, double r_cam,
                        const double y0[8], int64_t max_out, double* out) {
    std::vector<ora::Step> steps;
    double yf[8];
    int64_t att, acc;
    ora::integrate(met, r_cam, y0, &steps, yf, &att, &acc, nullptr);
    std::vector<ora::Sample> smp;
    ora::make_samples(met, grid, steps, smp);
    int64_t n = (int64_t)smp.size();
    for (int64_t q = 0; q < n && q < max_out; ++q) {
        double* o = out + 17 * q;
        for (int c = 0; c < 4; ++c) {
            o[c] = smp[q].x[c]; o[4 + c] = smp[q].k[c];
            o[8 + c] = smp[q].xn[c]; o[12 + c] = smp[q].kn[c];
        }
        o[16] = smp[q].dl;
    }
    return n;
}

void ora_fluid_frame(const double glo[16], const double u[4], const double kup[4],
                     const double b[4], double e1[4], double e2[4]) {
    ora::tetrad(glo, u, kup, b, e1, e2);
}

void ora_n_to_s(const double glo[16], const double e1[4], const double e2[4],
                const double n_re[16], const double n_im[16], double s[4]) {
    ora::n_to_s(glo, e1, e2, n_re, n_im, s);
}

void ora_s_to_n(const double e1[4], const double e2[4], const double s[4], double n_re[16],
                double n_im[16]) {
    ora::s_to_n(e1, e2, s, n_re, n_im);
}

void ora_trace(const ora_camera* cam, const ora_metric* met, const ora_grid* grid, double freq,
               int64_t npix, const int32_t* pix, int32_t nthreads, double* out_stokes,
               int32_t* out_status, int64_t* out_attempts, int64_t* out_accepted,
               int64_t* out_samples, double* out_end, int32_t unpolarized, double* out_aux) {
    int nt = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
    if (nt < 1) nt = 1;
    std::atomic<int64_t> next(0);
    auto work = [&]() {
        while (true) {
            int64_t q = next.fetch_add(1);
            if (q >= npix) break;
            ora::PixelResult r;
            ora::trace_pixel(cam, met, grid, freq, pix[q], unpolarized, r);
            for (int s = 0; s < 4; ++s) out_stokes[4 * q + s] = r.stokes[s];
            if (out_aux)
                for (int a = 0; a < ORA_AUX_COUNT; ++a) out_aux[ORA_AUX_COUNT * q + a] = r.aux[a];
            if (out_end)
                for (int s = 0; s < 8; ++s) out_end[8 * q + s] = r.end[s];
            if (out_status) out_status[q] = r.status;
            if (out_attempts) out_attempts[q] = r.attempts;
            if (out_accepted) out_accepted[q] = r.accepted;
            if (out_samples) out_samples[q] = r.samples;
        }
    };
    if (nt == 1) {
        work();
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) th.emplace_back(work);
        for (auto& t : th) t.join();
    }
}

}  // extern "C"
