// Internal declarations shared by the oracle's own translation units (test infrastructure).
#pragma once
#include <cmath>
#include <vector>

#include "oracle.h"

namespace ora {

// Forward-mode dual number carrying d/dx, d/dy, d/dz.
struct Dual {
    double v;
    double d[3];
    Dual() : v(0.0), d{0.0, 0.0, 0.0} {}
    explicit Dual(double x) : v(x), d{0.0, 0.0, 0.0} {}
    static Dual var(double x, int i) {
        Dual r(x);
        r.d[i] = 1.0;
        return r;
    }
};
inline Dual operator+(const Dual& a, const Dual& b) {
    Dual r(a.v + b.v);
    for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
    Dual r(a.v - b.v);
    for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
inline Dual operator-(const Dual& a) {
    Dual r(-a.v);
    for (int i = 0; i < 3; ++i) r.d[i] = -a.d[i];
    return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
    Dual r(a.v * b.v);
    for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
    Dual r(a.v / b.v);
    for (int i = 0; i < 3; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
    return r;
}
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator*(double a, const Dual& b) { return Dual(a) * b; }
inline Dual operator*(const Dual& a, double b) { return a * Dual(b); }
inline Dual operator/(const Dual& a, double b) { return a / Dual(b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual sqrt(const Dual& a) {
    double s = std::sqrt(a.v);
    Dual r(s);
    for (int i = 0; i < 3; ++i) r.d[i] = a.d[i] / (2.0 * s);
    return r;
}
using std::sqrt;

// geometry.cpp
double r_of_x(const double x[4], double a);
void metric_cks(const double x[4], double m, double a, int flat, double glo[16], double ghi[16]);
void metric_lo_deriv(const double x[4], double m, double a, int flat, double dg[64]);
void christoffel(const double x[4], double m, double a, int flat, double gam[64]);
void geodesic_rhs(const double y[8], double m, double a, int flat, double dy[8]);
void set_rhs_perturbation(int ulps);
void metric_sks(double r, double th, double m, double a, double g[16]);
void sks_to_cks_point(double r, double th, double ph, double a, double x[4]);
void sks_jacobian(double r, double th, double ph, double a, double jac[9]);
void cks_to_sks_point(const double x[4], double a, double* r, double* th, double* ph);
bool invert(int n, const double* a, double* inv);
void normal_to_cks(const double x[4], double r, double th, double ph, double m, double a,
                   int flat, const double up[3], double u[4]);
void sks_covector_to_cks(const double x[4], double a, const double ki[3], double ka[3]);
void camera_pixel(const ora_camera* cam, const ora_metric* met, int i, int j, double x[4],
                  double k[4], double hvec[4], double vvec[4], double* nnorm, double* r_cam,
                  double ucam[4]);
void dp_tableau(double A[49], double b5[7], double b4[7], double bm[7], double c[7]);
double horizon_radius(const ora_metric* met);

// One accepted DP step as needed by sampling: start/end states, stage derivatives at both
// ends, the fourth-order midpoint (Shampine 1986) and the signed step h.
struct Step {
    double y0[8], y1[8], f0[8], f1[8], ym[8];
    double h;
};
int32_t integrate(const ora_metric* met, double r_cam, const double ystart[8],
                  std::vector<Step>* steps, double yf[8], int64_t* attempts_out,
                  int64_t* accepted_out, std::vector<double>* path);

}  // namespace ora
