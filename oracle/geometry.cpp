// Oracle geometry: Kerr metric in Cartesian Kerr-Schild coordinates, derivatives by dual
// numbers, the camera of Sec. 2.1 and the adaptive Dormand-Prince integrator of Sec. 2.2.
// Test infrastructure only (see oracle.h).
#include "oracle.h"
#include "oracle_internal.hpp"

#include <cmath>
#include <cstring>
#include <vector>

namespace ora {

// ---------------------------------------------------------------------------------------
// Auxiliary functions of Eq. (cks_aux): r(x, y, z), f, l_alpha. Templated so that the same
// text evaluates plain values (double) and value + gradient (Dual).
// ---------------------------------------------------------------------------------------
template <class T>
static void cks_aux(const T& x, const T& y, const T& z, double a, double m, int flat,
                    T& r, T& f, T l_lo[4]) {
    T rr2 = x * x + y * y + z * z;                                   // R^2
    T q = rr2 - a * a;
    T r2 = 0.5 * (q + sqrt(q * q + 4.0 * a * a * z * z));           // r^2
    r = sqrt(r2);
    if (flat) {
        f = T(0.0);
    } else {
        f = 2.0 * m * r * r2 / (r2 * r2 + a * a * z * z);
    }
    T den = r2 + a * a;
    l_lo[0] = T(1.0);                                               // l_t = +1 (ingoing KS)
    l_lo[1] = (r * x + a * y) / den;
    l_lo[2] = (r * y - a * x) / den;
    l_lo[3] = z / r;
}

template <class T>
static void metric_lo(const T x[4], double a, double m, int flat, T g[16]) {
    T r, f, l[4];
    cks_aux(x[1], x[2], x[3], a, m, flat, r, f, l);
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be) {
            double eta = (al == be) ? (al == 0 ? -1.0 : 1.0) : 0.0;
            g[4 * al + be] = eta + f * l[al] * l[be];
        }
}

template <class T>
static void metric_hi(const T x[4], double a, double m, int flat, T g[16]) {
    T r, f, l[4];
    cks_aux(x[1], x[2], x[3], a, m, flat, r, f, l);
    T lu[4] = {-l[0], l[1], l[2], l[3]};                            // l^alpha = eta^{ab} l_b
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be) {
            double eta = (al == be) ? (al == 0 ? -1.0 : 1.0) : 0.0;
            g[4 * al + be] = eta - f * lu[al] * lu[be];
        }
}

double r_of_x(const double x[4], double a) {
    double r, f, l[4];
    cks_aux(x[1], x[2], x[3], a, 0.0, 1, r, f, l);
    return r;
}

void metric_cks(const double x[4], double m, double a, int flat, double glo[16], double ghi[16]) {
    if (glo) metric_lo(x, a, m, flat, glo);
    if (ghi) metric_hi(x, a, m, flat, ghi);
}

// d_mu g_{ab} (mu = 0..3, d_t = 0) by dual numbers: dg[mu][a][b].
void metric_lo_deriv(const double x[4], double m, double a, int flat, double dg[64]) {
    Dual X[4];
    X[0] = Dual(x[0]);
    for (int i = 1; i < 4; ++i) X[i] = Dual::var(x[i], i - 1);
    Dual g[16];
    metric_lo(X, a, m, flat, g);
    for (int ab = 0; ab < 16; ++ab) {
        dg[ab] = 0.0;
        for (int i = 0; i < 3; ++i) dg[16 * (i + 1) + ab] = g[ab].d[i];
    }
}

// Christoffel symbols of the second kind from their definition:
// Gamma^a_{bc} = 1/2 g^{ad} (d_b g_{dc} + d_c g_{db} - d_d g_{bc}).
void christoffel(const double x[4], double m, double a, int flat, double gam[64]) {
    double ghi[16], dg[64];
    metric_cks(x, m, a, flat, nullptr, ghi);
    metric_lo_deriv(x, m, a, flat, dg);
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be)
            for (int ga = 0; ga < 4; ++ga) {
                double s = 0.0;
                for (int de = 0; de < 4; ++de)
                    s += ghi[4 * al + de] *
                         (dg[16 * be + 4 * de + ga] + dg[16 * ga + 4 * de + be] -
                          dg[16 * de + 4 * be + ga]);
                gam[16 * al + 4 * be + ga] = 0.5 * s;
            }
}

// Test knob, off (0) unless a test sets it: right-hand-side component i is scaled by
// (1 + (-1)^i k 2^-52), a perturbation of about k ulps (alternating in sign: a common factor
// would only rescale the affine parameter, which leaves the path unchanged), which shows how
// far the adaptive step control carries rounding-level differences to the end of a geodesic.
static int g_rhs_perturb_ulps = 0;

void set_rhs_perturbation(int ulps) { g_rhs_perturb_ulps = ulps; }

// Eq. (geodesic) in Hamiltonian form with H = 1/2 g^{ab} k_a k_b:
// dx^a/dl = dH/dk_a = g^{ab} k_b,  dk_t/dl = 0,  dk_a/dl = -dH/dx^a.
void geodesic_rhs(const double y[8], double m, double a, int flat, double dy[8]) {
    Dual X[4];
    X[0] = Dual(y[0]);
    for (int i = 1; i < 4; ++i) X[i] = Dual::var(y[i], i - 1);
    Dual g[16];
    metric_hi(X, a, m, flat, g);
    const double* k = y + 4;
    Dual h(0.0);
    for (int al = 0; al < 4; ++al)
        for (int be = 0; be < 4; ++be) h = h + 0.5 * g[4 * al + be] * (k[al] * k[be]);
    for (int al = 0; al < 4; ++al) {
        double s = 0.0;
        for (int be = 0; be < 4; ++be) s += g[4 * al + be].v * k[be];
        dy[al] = s;
    }
    dy[4] = 0.0;
    for (int i = 0; i < 3; ++i) dy[5 + i] = -h.d[i];
    if (g_rhs_perturb_ulps != 0) {
        for (int i = 0; i < 8; ++i)
            dy[i] *= 1.0 + ((i & 1) ? -1.0 : 1.0) * g_rhs_perturb_ulps * 0x1p-52;
    }
}

// ---------------------------------------------------------------------------------------
// Spherical Kerr-Schild (Sec. 2): printed metric, coordinate maps and their Jacobian.
// ---------------------------------------------------------------------------------------
void metric_sks(double r, double th, double m, double a, double g[16]) {
    double s = std::sin(th), c = std::cos(th);
    double f = 2.0 * m * r * r * r / (r * r * r * r + a * a * r * r * c * c);  // z = r cos(th)
    std::memset(g, 0, 16 * sizeof(double));
    g[0] = -(1.0 - f);
    g[1] = g[4] = f;
    g[3] = g[12] = -a * f * s * s;
    g[5] = 1.0 + f;
    g[7] = g[13] = -a * (1.0 + f) * s * s;
    g[10] = 2.0 * m * r / f;
    g[15] = (r * r + a * a + a * a * f * s * s) * s * s;
}

void sks_to_cks_point(double r, double th, double ph, double a, double x[4]) {
    x[0] = 0.0;
    x[1] = std::sin(th) * (r * std::cos(ph) - a * std::sin(ph));
    x[2] = std::sin(th) * (r * std::sin(ph) + a * std::cos(ph));
    x[3] = r * std::cos(th);
}

// J[a][i] = d x^a / d x^i for a = x,y,z and i = r,theta,phi.
void sks_jacobian(double r, double th, double ph, double a, double jac[9]) {
    double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
    jac[0] = st * cp;  jac[1] = ct * (r * cp - a * sp);  jac[2] = st * (-r * sp - a * cp);
    jac[3] = st * sp;  jac[4] = ct * (r * sp + a * cp);  jac[5] = st * (r * cp - a * sp);
    jac[6] = ct;       jac[7] = -r * st;                 jac[8] = 0.0;
}

void cks_to_sks_point(const double x[4], double a, double* r, double* th, double* ph) {
    double rr = r_of_x(x, a);
    *r = rr;
    double c = x[3] / rr;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    *th = std::acos(c);
    double p = std::atan2(x[2], x[1]) - std::atan(a / rr);
    const double twopi = 2.0 * M_PI;
    p = std::fmod(p, twopi);
    if (p < 0.0) p += twopi;
    if (p >= twopi) p -= twopi;
    *ph = p;
}

// Gauss-Jordan inverse with partial pivoting (n <= 5).
bool invert(int n, const double* a, double* inv) {
    double m[5][10];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) m[i][j] = (j < n) ? a[n * i + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int i = c + 1; i < n; ++i)
            if (std::fabs(m[i][c]) > std::fabs(m[p][c])) p = i;
        if (m[p][c] == 0.0) return false;
        if (p != c)
            for (int j = 0; j < 2 * n; ++j) std::swap(m[p][j], m[c][j]);
        double d = m[c][c];
        for (int j = 0; j < 2 * n; ++j) m[c][j] /= d;
        for (int i = 0; i < n; ++i)
            if (i != c) {
                double f = m[i][c];
                for (int j = 0; j < 2 * n; ++j) m[i][j] -= f * m[c][j];
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[n * i + j] = m[i][j + n];
    return true;
}

double det3(const double* g) {
    return g[0] * (g[4] * g[8] - g[5] * g[7]) - g[1] * (g[3] * g[8] - g[5] * g[6]) +
           g[2] * (g[3] * g[7] - g[4] * g[6]);
}

// Normal-frame spatial vector u^p (Sec. 2) given in spherical KS components at the CKS point
// x (spherical r, th, ph) -> contravariant CKS u^alpha. The spatial normal-frame vector maps
// with the Jacobian (same time slicing), u^n = (1 + g_pq u^p u^q)^{1/2}, A^n = alpha A^t and
// A^p = A^a + beta^a A^t with lapse and shift read from the CKS inverse metric. This route
// stays regular on the polar axis, where the spherical metric is singular.
void normal_to_cks(const double x[4], double r, double th, double ph, double m, double a,
                   int flat, const double up[3], double u[4]) {
    double jac[9];
    sks_jacobian(r, th, ph, a, jac);
    double v[3];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s += jac[3 * c + i] * up[i];
        v[c] = s;
    }
    double glo[16], ghi[16];
    metric_cks(x, m, a, flat, glo, ghi);
    double q = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) q += glo[4 * (c + 1) + d + 1] * v[c] * v[d];
    double un = std::sqrt(1.0 + q);
    double lapse = 1.0 / std::sqrt(-ghi[0]);
    u[0] = un / lapse;
    for (int c = 0; c < 3; ++c) u[c + 1] = v[c] - (-ghi[c + 1] / ghi[0]) * u[0];
}

// Covariant spherical KS spatial components k_i -> CKS k_a = (d x^i / d x^a) k_i, with the
// derivatives of r, theta, phi (as functions of x, y, z) from dual numbers. Components with
// k_i = 0 are skipped so that the polar axis (where d theta, d phi diverge) is handled.
void sks_covector_to_cks(const double x[4], double a, const double ki[3], double ka[3]) {
    Dual X = Dual::var(x[1], 0), Y = Dual::var(x[2], 1), Z = Dual::var(x[3], 2);
    Dual r, f, l[4];
    cks_aux(X, Y, Z, a, 0.0, 1, r, f, l);
    for (int c = 0; c < 3; ++c) ka[c] = ki[0] * r.d[c];
    if (ki[1] != 0.0) {
        // theta = acos(z / r): d theta = -d(z/r) / sqrt(1 - (z/r)^2)
        Dual zr = Z / r;
        double s = std::sqrt(1.0 - zr.v * zr.v);
        for (int c = 0; c < 3; ++c) ka[c] += ki[1] * (-zr.d[c] / s);
    }
    if (ki[2] != 0.0) {
        // phi = atan2(y, x) - atan(a / r)
        double rho2 = x[1] * x[1] + x[2] * x[2];
        double dxy[3] = {-x[2] / rho2, x[1] / rho2, 0.0};
        for (int c = 0; c < 3; ++c) {
            double datan = -a / (r.v * r.v + a * a) * r.d[c];
            ka[c] += ki[2] * (dxy[c] - datan);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Camera (Sec. 2.1), plane-parallel.
// ---------------------------------------------------------------------------------------
struct CameraFrame {
    double x[4];          // centre, CKS
    double u[4], ulo[4];  // camera 4-velocity
    double hh[4], vv[4];  // H, V in the coordinate frame (contravariant)
    double kk[4];         // K in the coordinate frame (contravariant)
    double r_cam;
};

static void camera_frame(const ora_camera* cam, const ora_metric* met, CameraFrame& cf) {
    const double m = met->mass, a = met->spin;
    sks_to_cks_point(cam->r, cam->theta, cam->phi, a, cf.x);
    cf.r_cam = cam->r;
    double glo[16], ghi[16];
    metric_cks(cf.x, m, a, met->flat, glo, ghi);

    // 4-velocity from the normal-frame u^p; covariant k from the spherical k_i.
    normal_to_cks(cf.x, cam->r, cam->theta, cam->phi, m, a, met->flat, cam->u_p, cf.u);
    for (int al = 0; al < 4; ++al) {
        double s = 0.0;
        for (int be = 0; be < 4; ++be) s += glo[4 * al + be] * cf.u[be];
        cf.ulo[al] = s;
    }
    double klo[4];
    sks_covector_to_cks(cf.x, a, cam->k_p, klo + 1);
    // k_t from the null condition, future-directed root (k^t > 0).
    {
        double A = ghi[0], B = 0.0, C = 0.0;
        for (int c = 1; c < 4; ++c) B += ghi[c] * klo[c];
        for (int c = 1; c < 4; ++c)
            for (int d = 1; d < 4; ++d) C += ghi[4 * c + d] * klo[c] * klo[d];
        double disc = std::sqrt(B * B - A * C);
        double r1 = (-B + disc) / A, r2 = (-B - disc) / A;
        double kt1 = A * r1 + B, kt2 = A * r2 + B;   // k^t = g^{tt} k_t + g^{ta} k_a
        klo[0] = (kt1 > 0.0) ? r1 : r2;
        (void)kt2;
    }

    // Camera-frame metric (primed), Sec. 2.1.
    const double* ul = cf.ulo;
    double gp_lo[9], gp_hi[9];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
            int A = c + 1, B = d + 1;
            gp_lo[3 * c + d] = glo[4 * A + B] - ul[A] / ul[0] * glo[B] - ul[B] / ul[0] * glo[A] +
                               ul[A] * ul[B] / (ul[0] * ul[0]) * glo[0];
            gp_hi[3 * c + d] = ghi[4 * A + B] + cf.u[A] * cf.u[B];
        }
    // Line of sight K.
    double kp_lo[3], kp_hi[3];
    for (int c = 0; c < 3; ++c) kp_lo[c] = klo[c + 1] - ul[c + 1] / ul[0] * klo[0];
    double kt_p = 0.0;
    for (int al = 0; al < 4; ++al) kt_p -= cf.u[al] * klo[al];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) s += gp_hi[3 * c + d] * kp_lo[d];
        kp_hi[c] = s;
    }
    double nrm = 0.0;
    for (int c = 0; c < 3; ++c) nrm += kp_lo[c] * kp_hi[c];
    nrm = 1.0 / std::sqrt(nrm);
    for (int c = 0; c < 3; ++c) { kp_lo[c] *= nrm; kp_hi[c] *= nrm; }
    kt_p *= nrm;
    cf.kk[0] = cf.u[0] * kt_p;
    for (int c = 0; c < 3; ++c) cf.kk[0] -= ul[c + 1] / ul[0] * kp_hi[c];
    for (int c = 0; c < 3; ++c) cf.kk[c + 1] = kp_hi[c] + cf.u[c + 1] * kt_p;

    // Vertical v by Gram-Schmidt of U = z (or y on the polar axis).
    double U[3] = {0.0, 0.0, 1.0};
    if (cf.x[1] == 0.0 && cf.x[2] == 0.0) { U[1] = 1.0; U[2] = 0.0; }
    double uk = 0.0;
    for (int c = 0; c < 3; ++c) uk += U[c] * kp_lo[c];
    double v_hi[3], v_lo[3];
    for (int c = 0; c < 3; ++c) v_hi[c] = U[c] - uk * kp_hi[c];
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) s += gp_lo[3 * c + d] * v_hi[d];
        v_lo[c] = s;
    }
    double vn = 0.0;
    for (int c = 0; c < 3; ++c) vn += v_lo[c] * v_hi[c];
    vn = 1.0 / std::sqrt(vn);
    for (int c = 0; c < 3; ++c) { v_hi[c] *= vn; v_lo[c] *= vn; }
    // Horizontal h^a = [abc] v_b K_c / sqrt(D).
    double sd = std::sqrt(det3(gp_lo));
    double h_hi[3];
    h_hi[0] = (v_lo[1] * kp_lo[2] - v_lo[2] * kp_lo[1]) / sd;
    h_hi[1] = (v_lo[2] * kp_lo[0] - v_lo[0] * kp_lo[2]) / sd;
    h_hi[2] = (v_lo[0] * kp_lo[1] - v_lo[1] * kp_lo[0]) / sd;
    double cps = std::cos(cam->psi), sps = std::sin(cam->psi);
    double Hp[3], Vp[3];
    for (int c = 0; c < 3; ++c) {
        Hp[c] = h_hi[c] * cps - v_hi[c] * sps;
        Vp[c] = v_hi[c] * cps + h_hi[c] * sps;
    }
    // Back to the coordinate frame with zero primed time component.
    cf.hh[0] = 0.0;
    cf.vv[0] = 0.0;
    for (int c = 0; c < 3; ++c) {
        cf.hh[0] -= ul[c + 1] / ul[0] * Hp[c];
        cf.vv[0] -= ul[c + 1] / ul[0] * Vp[c];
        cf.hh[c + 1] = Hp[c];
        cf.vv[c + 1] = Vp[c];
    }
}

// Null root for k^t at fixed spatial k^a (Sec. 2.1).
static double null_kt(const double glo[16], const double ka[3]) {
    double A = glo[0], B = 0.0, C = 0.0;
    for (int c = 0; c < 3; ++c) B += glo[c + 1] * ka[c];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) C += glo[4 * (c + 1) + d + 1] * ka[c] * ka[d];
    if (A == 0.0) return -C / (2.0 * B);
    double disc = std::sqrt(B * B - A * C);
    double r1 = (-B + disc) / A, r2 = (-B - disc) / A;
    if (A < 0.0) return (r1 > 0.0) ? r1 : r2;            // unique positive root
    double lo = std::fmin(r1, r2), hi = std::fmax(r1, r2);  // ergoregion: lesser positive root
    return (lo > 0.0) ? lo : hi;
}

void camera_pixel(const ora_camera* cam, const ora_metric* met, int i, int j, double x[4],
                  double k[4], double hvec[4], double vvec[4], double* nnorm, double* r_cam,
                  double ucam[4]) {
    CameraFrame cf;
    camera_frame(cam, met, cf);
    double n = cam->n;
    double aa = (i - n / 2.0 + 0.5) * cam->width / n;
    double bb = (j - n / 2.0 + 0.5) * cam->width / n;
    for (int al = 0; al < 4; ++al) x[al] = cf.x[al] + aa * cf.hh[al] + bb * cf.vv[al];
    double glo[16];
    metric_cks(x, met->mass, met->spin, met->flat, glo, nullptr);
    double kup[4];
    kup[1] = cf.kk[1]; kup[2] = cf.kk[2]; kup[3] = cf.kk[3];
    kup[0] = null_kt(glo, kup + 1);
    for (int al = 0; al < 4; ++al) {
        double s = 0.0;
        for (int be = 0; be < 4; ++be) s += glo[4 * al + be] * kup[be];
        k[al] = s;
    }
    for (int al = 0; al < 4; ++al) { hvec[al] = cf.hh[al]; vvec[al] = cf.vv[al]; }
    if (cam->nu_at_infinity) {
        *nnorm = 1.0 / (-k[0]);                      // -n k_t = nu (per unit nu)
    } else {
        double s = 0.0;
        for (int al = 0; al < 4; ++al) s += k[al] * cf.u[al];
        *nnorm = 1.0 / (-s);                         // -n k.u = nu (per unit nu)
    }
    if (r_cam) *r_cam = cf.r_cam;
    if (ucam)
        for (int al = 0; al < 4; ++al) ucam[al] = cf.u[al];
}

// ---------------------------------------------------------------------------------------
// Dormand-Prince RK5(4)7M, Table tab:dp.
// ---------------------------------------------------------------------------------------
void dp_tableau(double A[49], double b5[7], double b4[7], double bm[7], double c[7]) {
    for (int q = 0; q < 49; ++q) A[q] = 0.0;
    auto s = [&](int i, int j, double v) { A[7 * i + j] = v; };
    s(1, 0, 1.0 / 5.0);
    s(2, 0, 3.0 / 40.0);        s(2, 1, 9.0 / 40.0);
    s(3, 0, 44.0 / 45.0);       s(3, 1, -56.0 / 15.0);      s(3, 2, 32.0 / 9.0);
    s(4, 0, 19372.0 / 6561.0);  s(4, 1, -25360.0 / 2187.0); s(4, 2, 64448.0 / 6561.0);
    s(4, 3, -212.0 / 729.0);
    s(5, 0, 9017.0 / 3168.0);   s(5, 1, -355.0 / 33.0);     s(5, 2, 46732.0 / 5247.0);
    s(5, 3, 49.0 / 176.0);      s(5, 4, -5103.0 / 18656.0);
    s(6, 0, 35.0 / 384.0);      s(6, 1, 0.0);               s(6, 2, 500.0 / 1113.0);
    s(6, 3, 125.0 / 192.0);     s(6, 4, -2187.0 / 6784.0);  s(6, 5, 11.0 / 84.0);
    const double B5[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0,
                          11.0 / 84.0, 0.0};
    const double B4[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                          -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};
    const double BM[7] = {6025192743.0 / 30085553152.0, 0.0, 51252292925.0 / 65400821598.0,
                          -2691868925.0 / 45128329728.0, 187940372067.0 / 1594534317056.0,
                          -1776094331.0 / 19743644256.0, 11237099.0 / 235043384.0};
    const double C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
    for (int i = 0; i < 7; ++i) { b5[i] = B5[i]; b4[i] = B4[i]; bm[i] = BM[i]; c[i] = C[i]; }
}

double horizon_radius(const ora_metric* met) {
    double m = met->mass, a = met->spin;
    double d = m * m - a * a;
    return m + std::sqrt(d > 0.0 ? d : 0.0);
}

// ---------------------------------------------------------------------------------------
// Fixed-rule Runge-Kutta integrators (Sec. 2.2): classical RK4 (Table tab:rk4) or Heun's RK2
// (Table tab:rk2), with the step -f_step (r - r_hor) taken at the start of each step
// (Eq. rk_step; negative: backward from the camera). The paper gives the sample point only for
// DP; here a step's sample is its cubic Hermite midpoint (y0 + y1)/2 + h (f0 - f1)/8, and the
// quartic used for subdivision is then that cubic (it meets all five conditions).
// Termination as for DP.
// ---------------------------------------------------------------------------------------
static int32_t integrate_rk(const ora_metric* met, double r_cam, const double ystart[8],
                            std::vector<Step>* steps, double yf[8], int64_t* attempts_out,
                            int64_t* accepted_out, std::vector<double>* path) {
    const double m = met->mass, a = met->spin;
    const int flat = met->flat;
    const double r_hor = horizon_radius(met);
    const double r_in = met->r_in_over_rhor * r_hor;
    double y[8], f[8];
    for (int q = 0; q < 8; ++q) y[q] = ystart[q];
    geodesic_rhs(y, m, a, flat, f);
    bool been_inside = r_of_x(y, a) < r_cam;
    int64_t n = 0;
    int32_t status = ORA_OK;
    while (true) {
        if (n >= met->max_steps) { status = ORA_MAX_STEPS; break; }
        ++n;
        const double r0 = r_of_x(y, a);
        const double h = -met->f_step * (r0 - r_hor);
        double y1[8], ys[8], k2[8], k3[8], k4[8];
        if (met->integrator == 1) {
            for (int q = 0; q < 8; ++q) ys[q] = y[q] + 0.5 * h * f[q];
            geodesic_rhs(ys, m, a, flat, k2);
            for (int q = 0; q < 8; ++q) ys[q] = y[q] + 0.5 * h * k2[q];
            geodesic_rhs(ys, m, a, flat, k3);
            for (int q = 0; q < 8; ++q) ys[q] = y[q] + h * k3[q];
            geodesic_rhs(ys, m, a, flat, k4);
            for (int q = 0; q < 8; ++q)
                y1[q] = y[q] + h * (f[q] / 6.0 + k2[q] / 3.0 + k3[q] / 3.0 + k4[q] / 6.0);
        } else {
            for (int q = 0; q < 8; ++q) ys[q] = y[q] + h * f[q];
            geodesic_rhs(ys, m, a, flat, k2);
            for (int q = 0; q < 8; ++q) y1[q] = y[q] + h * (0.5 * f[q] + 0.5 * k2[q]);
        }
        bool bad = false;
        for (int q = 0; q < 8; ++q) bad = bad || !(y1[q] == y1[q]);
        if (bad) { status = ORA_NAN; break; }
        double f1[8];
        geodesic_rhs(y1, m, a, flat, f1);
        if (steps) {
            Step sp;
            for (int q = 0; q < 8; ++q) {
                sp.y0[q] = y[q];
                sp.y1[q] = y1[q];
                sp.f0[q] = f[q];
                sp.f1[q] = f1[q];
                sp.ym[q] = 0.5 * (y[q] + y1[q]) + 0.125 * h * (f[q] - f1[q]);
            }
            sp.h = h;
            steps->push_back(sp);
        }
        for (int q = 0; q < 8; ++q) { y[q] = y1[q]; f[q] = f1[q]; }
        if (path) path->insert(path->end(), y, y + 8);
        const double r = r_of_x(y, a);
        if (r < r_in) { status = ORA_HORIZON; break; }
        if (been_inside && r > r_cam) { status = ORA_ESCAPED; break; }
        if (r < r_cam) been_inside = true;
        if (std::fabs(met->f_step * (r - r_hor)) < 1e-12 * r) { status = ORA_UNDERFLOW; break; }
    }
    for (int q = 0; q < 8; ++q) yf[q] = y[q];
    if (attempts_out) *attempts_out = n;
    if (accepted_out) *accepted_out = n;
    return status;
}

int32_t integrate(const ora_metric* met, double r_cam, const double ystart[8],
                  std::vector<Step>* steps, double yf[8], int64_t* attempts_out,
                  int64_t* accepted_out, std::vector<double>* path) {
    if (met->integrator != 0)
        return integrate_rk(met, r_cam, ystart, steps, yf, attempts_out, accepted_out, path);
    double A[49], b5[7], b4[7], bm[7], c[7];
    dp_tableau(A, b5, b4, bm, c);
    const double m = met->mass, a = met->spin;
    const int flat = met->flat;
    const double r_hor = horizon_radius(met);
    const double r_in = met->r_in_over_rhor * r_hor;

    double y[8], f[8];
    for (int q = 0; q < 8; ++q) y[q] = ystart[q];
    geodesic_rhs(y, m, a, flat, f);
    double h = -met->h0_frac * (r_cam - r_hor);     // backward in affine parameter
    bool been_inside = r_of_x(y, a) < r_cam;
    bool prev_rejected = false;
    int64_t attempts = 0, accepted = 0;
    int32_t status = ORA_OK;

    while (true) {
        if (attempts >= met->max_steps) { status = ORA_MAX_STEPS; break; }
        ++attempts;
        double k[7][8];
        for (int q = 0; q < 8; ++q) k[0][q] = f[q];
        double ys[8];
        for (int st = 1; st < 7; ++st) {
            for (int q = 0; q < 8; ++q) {
                double s = 0.0;
                for (int p = 0; p < st; ++p) s += A[7 * st + p] * k[p][q];
                ys[q] = y[q] + h * s;
            }
            geodesic_rhs(ys, m, a, flat, k[st]);
        }
        // ys is now the 7th-stage argument, which is the 5th-order solution (FSAL).
        // y5 - y4 = h sum_p (b5_p - b4_p) k_p: the same difference of the two solutions,
        // evaluated without subtracting two nearly equal sums (which would lose about as
        // many digits as the tolerance has).
        double y5[8], d54[8];
        for (int q = 0; q < 8; ++q) {
            double s5 = 0.0, sd = 0.0;
            for (int p = 0; p < 7; ++p) { s5 += b5[p] * k[p][q]; sd += (b5[p] - b4[p]) * k[p][q]; }
            y5[q] = y[q] + h * s5;
            d54[q] = h * sd;
        }
        double eps = 0.0;
        bool bad = false;
        for (int q = 0; q < 8; ++q) {
            double sc = met->tol_abs + met->tol_rel * std::fmax(std::fabs(y[q]), std::fabs(y5[q]));
            double e = std::fabs(d54[q]) / sc;
            if (!(e == e)) bad = true;
            eps = std::fmax(eps, e);
        }
        if (bad) { status = ORA_NAN; break; }
        if (eps <= 1.0) {
            if (steps) {
                Step sp;
                for (int q = 0; q < 8; ++q) {
                    double s = 0.0;
                    for (int p = 0; p < 7; ++p) s += bm[p] * k[p][q];
                    sp.ym[q] = y[q] + 0.5 * h * s;          // midpoint weights scaled by h/2
                    sp.y0[q] = y[q];
                    sp.y1[q] = y5[q];
                    sp.f0[q] = k[0][q];
                    sp.f1[q] = k[6][q];
                }
                sp.h = h;
                steps->push_back(sp);
            }
            for (int q = 0; q < 8; ++q) { y[q] = y5[q]; f[q] = k[6][q]; }
            ++accepted;
            if (path) path->insert(path->end(), y, y + 8);
            double fac = (eps == 0.0) ? 10.0 : 0.9 * std::pow(eps, -0.2);
            fac = std::fmin(10.0, std::fmax(0.2, fac));
            if (prev_rejected) fac = std::fmin(fac, 1.0);
            h *= fac;
            prev_rejected = false;
            double r = r_of_x(y, a);
            if (r < r_in) { status = ORA_HORIZON; break; }
            if (been_inside && r > r_cam) { status = ORA_ESCAPED; break; }
            if (r < r_cam) been_inside = true;
        } else {
            double fac = std::fmax(0.2, 0.9 * std::pow(eps, -0.2));
            h *= fac;
            prev_rejected = true;
        }
        if (std::fabs(h) < 1e-12 * r_of_x(y, a)) { status = ORA_UNDERFLOW; break; }
    }
    for (int q = 0; q < 8; ++q) yf[q] = y[q];
    if (attempts_out) *attempts_out = attempts;
    if (accepted_out) *accepted_out = accepted;
    return status;
}

}  // namespace ora

// ------------------------------- C entry points ----------------------------------------
extern "C" {

void ora_metric_cks(const double x[4], double mass, double spin, int flat, double g_lo[16],
                    double g_hi[16]) {
    ora::metric_cks(x, mass, spin, flat, g_lo, g_hi);
}
void ora_metric_sks(double r, double theta, double mass, double spin, double g_lo[16]) {
    ora::metric_sks(r, theta, mass, spin, g_lo);
}
void ora_christoffel(const double x[4], double mass, double spin, int flat, double gam[64]) {
    ora::christoffel(x, mass, spin, flat, gam);
}
void ora_set_rhs_perturbation(int32_t ulps) { ora::set_rhs_perturbation(ulps); }
void ora_geodesic_rhs(const double y[8], double mass, double spin, int flat, double dy[8]) {
    ora::geodesic_rhs(y, mass, spin, flat, dy);
}
void ora_dp_tableau(double a[49], double b5[7], double b4[7], double bmid[7], double c[7]) {
    ora::dp_tableau(a, b5, b4, bmid, c);
}
double ora_r_of_x(const double x[4], double spin) { return ora::r_of_x(x, spin); }

void ora_camera_pixel(const ora_camera* cam, const ora_metric* met, int32_t i, int32_t j,
                      double x[4], double k[4], double hvec[4], double vvec[4], double* nnorm) {
    ora::camera_pixel(cam, met, i, j, x, k, hvec, vvec, nnorm, nullptr, nullptr);
}

int32_t ora_geodesic(const ora_metric* met, double r_cam, const double y0[8], double yf[8],
                     int64_t* attempts, int64_t* accepted, double* path, int64_t max_path,
                     int64_t* n_path) {
    std::vector<double> p;
    int32_t st = ora::integrate(met, r_cam, y0, nullptr, yf, attempts, accepted,
                                path ? &p : nullptr);
    if (path) {
        int64_t n = (int64_t)(p.size() / 8);
        if (n > max_path) n = max_path;
        for (int64_t q = 0; q < 8 * n; ++q) path[q] = p[q];
        if (n_path) *n_path = n;
    }
    return st;
}

}  // extern "C"
