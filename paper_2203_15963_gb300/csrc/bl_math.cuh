// Device math for the Blacklight hot path (White 2022), templated on the arithmetic type.
// Geodesics always use double; sampling, plasma, coefficients and transfer use T = double
// (FP64 form) or T = float (mixed form).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace bl {

// Modified Bessel I_0, I_1 for 0 <= x <= 3.75 (used for x <= 2). FP32: the polynomials of
// Abramowitz & Stegun 9.8.1 and 9.8.3 in t = x / 3.75 (|error| < 1.6e-7 for I_0, 8e-9 for
// I_1 / x, below FP32 rounding).
__device__ __forceinline__ float cyl_bessel_i0(float x) {
    const float t = x * (1.0f / 3.75f), t2 = t * t;
    return 1.0f + t2 * (3.5156229f + t2 * (3.0899424f + t2 * (1.2067492f + t2 * (0.2659732f +
           t2 * (0.0360768f + t2 * 0.0045813f)))));
}
__device__ __forceinline__ float cyl_bessel_i1(float x) {
    const float t = x * (1.0f / 3.75f), t2 = t * t;
    return x * (0.5f + t2 * (0.87890594f + t2 * (0.51498869f + t2 * (0.15084934f + t2 * (0.02658733f +
           t2 * (0.00301532f + t2 * 0.00032411f))))));
}
// FP64 (used for 0 <= x <= 2 only): the defining power series, I_0(x) = sum_k t^k / (k!)^2
// and I_1(x) = (x/2) sum_k t^k / (k! (k+1)!) with t = x^2 / 4 <= 1, summed by Horner's rule
// through k = 12 (the next terms are below 2e-18 of the sums); all terms are positive, so
// the sums are accurate to a few units in the last place.
__constant__ double c_i0_series[13] = {
    1.0, 1.0, 1.0 / 4.0, 1.0 / 36.0, 1.0 / 576.0, 1.0 / 14400.0, 1.0 / 518400.0,
    1.0 / 25401600.0, 1.0 / 1625702400.0, 1.0 / 131681894400.0, 1.0 / 13168189440000.0,
    1.0 / 1593350922240000.0, 1.0 / 229442532802560000.0};
__constant__ double c_i1_series[13] = {
    1.0, 1.0 / 2.0, 1.0 / 12.0, 1.0 / 144.0, 1.0 / 2880.0, 1.0 / 86400.0, 1.0 / 3628800.0,
    1.0 / 203212800.0, 1.0 / 14631321600.0, 1.0 / 1316818944000.0, 1.0 / 144850083840000.0,
    1.0 / 19120211066880000.0, 1.0 / 2982752926433280000.0};
__device__ __forceinline__ double cyl_bessel_i0(double x) {
    const double t = 0.25 * x * x;
    double s = c_i0_series[12];
#pragma unroll
    for (int k = 11; k >= 0; --k) s = fma(s, t, c_i0_series[k]);
    return s;
}
__device__ __forceinline__ double cyl_bessel_i1(double x) {
    const double t = 0.25 * x * x;
    double s = c_i1_series[12];
#pragma unroll
    for (int k = 11; k >= 0; --k) s = fma(s, t, c_i1_series[k]);
    return 0.5 * x * s;
}

// Quotient a / b on the coefficient and transport path: in FP32 the hardware reciprocal times
// a (__fdividef: within 2 ulp for |b| < 2^126, far inside the FP32 form's error budget), in
// FP64 the IEEE quotient.
template <class T>
__device__ __forceinline__ T fq(T a, T b) {
    if constexpr (sizeof(T) == 4) return __fdividef(a, b);
    else return a / b;
}

// exp, log, cube root and cos on the FP32 coefficient path through the hardware
// approximations: __expf within 2 + 1.2 |x| ulp, __logf within 2^-21.4 absolute on [0.5, 2]
// and 3 ulp elsewhere, the cube root as exp(log(x) / 3) from those two, __cosf within about
// 2^-21 absolute for |x| <= pi (its argument here multiplies a term that vanishes where it is
// not). FP64: the libm functions.
template <class T>
__device__ __forceinline__ T fexp(T x) {
    if constexpr (sizeof(T) == 4) return __expf(x);
    else return exp(x);
}
template <class T>
__device__ __forceinline__ T flog(T x) {
    if constexpr (sizeof(T) == 4) return __logf(x);
    else return log(x);
}
template <class T>
__device__ __forceinline__ T fcbrt(T x) {   // x >= 0
    if constexpr (sizeof(T) == 4) return __expf(__logf(x) * (1.0f / 3.0f));
    else return cbrt(x);
}
template <class T>
__device__ __forceinline__ T fcos(T x) {
    if constexpr (sizeof(T) == 4) return __cosf(x);
    else return cos(x);
}
// Square root on the FP32 coefficient path: the PTX approximate square root (sqrt.approx.f32,
// within about one ulp, sqrt(0) = 0, without the IEEE form's correction steps); FP64: the IEEE
// square root.
template <class T>
__device__ __forceinline__ T fsqrt(T x) {
    if constexpr (sizeof(T) == 4) {
        float y;
        asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    } else {
        return sqrt(x);
    }
}
// CGS constants (CODATA 2018; IAU 2015 nominal solar mass).
constexpr double kC = 2.99792458e10;
constexpr double kE = 4.80320471e-10;
constexpr double kMe = 9.1093837015e-28;
constexpr double kMp = 1.67262192369e-24;
constexpr double kH = 6.62607015e-27;
constexpr double kG = 6.67430e-8;
constexpr double kMsun = 1.98841e33;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------
// Kerr metric in Cartesian Kerr-Schild form (Sec. 2, Eq. cks_aux):
//   g_ab = eta_ab + f l_a l_b,  g^ab = eta^ab - f l^a l^b,  l_a = (1, lx, ly, lz),
//   f = 2 M r^3 / (r^4 + a^2 z^2),  2 r^2 = R^2 - a^2 + ((R^2 - a^2)^2 + 4 a^2 z^2)^{1/2}.
// Derivatives are hand-expanded: with D = ((R^2 - a^2)^2 + 4 a^2 z^2)^{1/2},
//   dr/dx = r x / D, dr/dy = r y / D, dr/dz = z (r^2 + a^2) / (r D).
// ---------------------------------------------------------------------------------------
template <class T>
struct KSGeom {
    T r, f;
    T l[4];         // covariant l_a, l[0] = 1
    T df[3];        // d_c f
    T dl[3][3];     // d_c l_b (b spatial)
};

template <class T>
__device__ __forceinline__ void ks_geom(T x, T y, T z, T a, T m, bool flat, bool derivs,
                                        KSGeom<T>& G) {
    // Special functions kept to two reciprocal square roots and one reciprocal:
    // D = D2 rsqrt(D2), r = r2 rsqrt(r2), and 1/P, 1/s4 from 1/(P s4).
    constexpr T c1 = T(1), c2 = T(2), c3 = T(3), c4 = T(4), cHalf = T(0.5), c0 = T(0);
    const T rr2 = x * x + y * y + z * z;
    const T q = rr2 - a * a;
    const T D2 = q * q + c4 * a * a * z * z;
    const T iD = rsqrt(D2);
    const T D = D2 * iD;
    const T r2 = cHalf * (q + D);
    const T ir = rsqrt(r2);
    const T r = r2 * ir;
    const T s4 = r2 * r2 + a * a * z * z;
    const T P = r2 + a * a;
    const T iPs = c1 / (P * s4);
    const T is4 = P * iPs;
    const T iP = s4 * iPs;
    const T f = flat ? c0 : c2 * m * r * r2 * is4;
    G.r = r;
    G.f = f;
    G.l[0] = c1;
    G.l[1] = (r * x + a * y) * iP;
    G.l[2] = (r * y - a * x) * iP;
    G.l[3] = z * ir;
    if (!derivs) return;
    const T dr[3] = {r * x * iD, r * y * iD, z * P * ir * iD};
    for (int c = 0; c < 3; ++c) {
        const T extra = (c == 2) ? c2 * a * a * z : c0;
        G.df[c] = flat ? c0 : f * (c3 * dr[c] * ir - (c4 * r2 * r * dr[c] + extra) * is4);
        const T two_r_dr_iP = c2 * r * dr[c] * iP;
        G.dl[c][0] = (dr[c] * x + (c == 0 ? r : c0) + (c == 1 ? a : c0)) * iP - G.l[1] * two_r_dr_iP;
        G.dl[c][1] = (dr[c] * y + (c == 1 ? r : c0) - (c == 0 ? a : c0)) * iP - G.l[2] * two_r_dr_iP;
        G.dl[c][2] = ((c == 2 ? c1 : c0) - G.l[3] * dr[c]) * ir;
    }
}

// r of a CKS point (Eq. cks_aux:r).
template <class T>
__device__ __forceinline__ T ks_r(T x, T y, T z, T a) {
    const T q = x * x + y * y + z * z - a * a;
    return sqrt(T(0.5) * (q + sqrt(q * q + T(4) * a * a * z * z)));
}

// Lower / raise with g = eta + f l l (contravariant l^a = (-1, lx, ly, lz)).
template <class T>
__device__ __forceinline__ void lower4(const KSGeom<T>& G, const T v[4], T out[4]) {
    const T lv = G.l[0] * v[0] + G.l[1] * v[1] + G.l[2] * v[2] + G.l[3] * v[3];
    out[0] = -v[0] + G.f * lv;
    out[1] = v[1] + G.f * G.l[1] * lv;
    out[2] = v[2] + G.f * G.l[2] * lv;
    out[3] = v[3] + G.f * G.l[3] * lv;
}
template <class T>
__device__ __forceinline__ void raise4(const KSGeom<T>& G, const T w[4], T out[4]) {
    const T lw = -w[0] + G.l[1] * w[1] + G.l[2] * w[2] + G.l[3] * w[3];   // l^a w_a
    out[0] = -w[0] + G.f * lw;                                           // -f l^t lw, l^t = -1
    out[1] = w[1] - G.f * G.l[1] * lw;
    out[2] = w[2] - G.f * G.l[2] * lw;
    out[3] = w[3] - G.f * G.l[3] * lw;
}
template <class T>
__device__ __forceinline__ T dot4(const KSGeom<T>& G, const T u[4], const T v[4]) {
    const T lu = G.l[0] * u[0] + G.l[1] * u[1] + G.l[2] * u[2] + G.l[3] * u[3];
    const T lv = G.l[0] * v[0] + G.l[1] * v[1] + G.l[2] * v[2] + G.l[3] * v[3];
    return -u[0] * v[0] + u[1] * v[1] + u[2] * v[2] + u[3] * v[3] + G.f * lu * lv;
}

// Eq. (geodesic): dx^a/dl = g^ab k_b; dk_t/dl = 0; dk_c/dl = -1/2 d_c g^ab k_a k_b
//   = L (1/2 d_c f L + f sum_b d_c l_b k_b),  L = l^a k_a.
// Returns r at the evaluation point (used for the termination tests).
__device__ __forceinline__ double geodesic_rhs(const double y[8], double a, double m, bool flat,
                                               double dy[8]) {
    KSGeom<double> G;
    ks_geom<double>(y[1], y[2], y[3], a, m, flat, true, G);
    const double* k = y + 4;
    const double L = -k[0] + G.l[1] * k[1] + G.l[2] * k[2] + G.l[3] * k[3];
    dy[0] = -k[0] + G.f * L;
    dy[1] = k[1] - G.f * G.l[1] * L;
    dy[2] = k[2] - G.f * G.l[2] * L;
    dy[3] = k[3] - G.f * G.l[3] * L;
    dy[4] = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double S = G.dl[c][0] * k[1] + G.dl[c][1] * k[2] + G.dl[c][2] * k[3];
        dy[5 + c] = L * (0.5 * G.df[c] * L + G.f * S);
    }
    return G.r;
}

// ---------------------------------------------------------------------------------------
// Coordinate terms of Eq. (polarized_n), read as parallel transport of the coherency
// tensor: dN/dl = A N + N A^T with A^a_d = -k^c Gamma^a_cd. For g = eta + f l l the
// contraction is C_ed = k^c Gamma_ecd = 1/2 (D_ed + P_de - P_ed) with
//   D_ed = k^c d_c g_ed,  P_me = d_m g_ec k^c,  and A = -g^{-1} C.
// ---------------------------------------------------------------------------------------
// The needed contractions are formed directly from r, f and l (no 3x3 table d_c l_b):
//   k.grad r, d_c f = F1 d_c r - [c = z] 2 a^2 z f / s4 with F1 = f (3 / r - 4 r^3 / s4),
//   kdl_e = k^c d_c l_e, M_m = d_m (l_c) k^c (fixed k), the curl Q_de = d_d l_e - d_e l_d,
// D is symmetric and W_ed = P_de - P_ed antisymmetric, so C_ed = (D_ed + W_ed) / 2 and
// C_de = (D_ed - W_ed) / 2 from the 10 + 6 independent entries.
template <class T>
__device__ __forceinline__ void transport_matrix(const T xv[3], const T klo[4], T a, T m,
                                                 bool flat, T A[4][4]) {
    constexpr T c0 = T(0), c1 = T(1), c2 = T(2), c3 = T(3), c4 = T(4), cHalf = T(0.5);
    const T x = xv[0], y = xv[1], z = xv[2];
    const T aa = a * a;
    const T q = x * x + y * y + z * z - aa;
    const T aaz2 = aa * z * z;
    const T D2 = q * q + c4 * aaz2;
    const T iD = rsqrt(D2);
    const T r2 = cHalf * (q + D2 * iD);
    const T ir = rsqrt(r2);
    const T r = r2 * ir;
    const T s4 = r2 * r2 + aaz2;
    const T P = r2 + aa;
    const T iPs = fq(c1, P * s4);
    const T is4 = P * iPs;
    const T iP = s4 * iPs;
    const T f = flat ? c0 : c2 * m * r * r2 * is4;
    const T lx = (r * x + a * y) * iP, ly = (r * y - a * x) * iP, lz = z * ir;
    // k^a = g^ab k_b
    const T lw = -klo[0] + lx * klo[1] + ly * klo[2] + lz * klo[3];
    const T kt = -klo[0] + f * lw, kx = klo[1] - f * lx * lw, ky = klo[2] - f * ly * lw,
            kz = klo[3] - f * lz * lw;
    // d_c r, k.grad r, d_c f
    const T riD = r * iD;
    const T drx = riD * x, dry = riD * y, drz = z * P * ir * iD;
    const T kdr = kx * drx + ky * dry + kz * drz;
    const T F1 = f * (c3 * ir - c4 * r2 * r * is4);
    const T fz = c2 * aa * z * f * is4;
    const T df[4] = {c0, F1 * drx, F1 * dry, F1 * drz - fz};
    const T kdf = F1 * kdr - kz * fz;
    const T t2 = c2 * r * iP;
    // kdl_e = k^c d_c l_e (l_t constant)
    const T kdl[4] = {c0, (kdr * x + r * kx + a * ky) * iP - t2 * kdr * lx,
                      (kdr * y + r * ky - a * kx) * iP - t2 * kdr * ly, (kz - lz * kdr) * ir};
    const T l[4] = {c1, lx, ly, lz};
    const T Lp = kt + lx * kx + ly * ky + lz * kz;       // l_c k^c
    // M_m = d_m (l_c) k^c at fixed k: with A' = x k^x + y k^y, B' = y k^x - x k^y
    const T Ap = x * kx + y * ky, Bp = y * kx - x * ky;
    const T Lxy = (r * Ap + a * Bp) * iP;
    const T V = (Ap - c2 * r * Lxy) * iP - kz * ir * lz;
    const T M[4] = {c0, drx * V + (r * kx - a * ky) * iP, dry * V + (r * ky + a * kx) * iP,
                    drz * V + kz * ir};
    // curl of l: Q_xy = d_x l_y - d_y l_x, Q_xz, Q_yz
    const T Qxy = -c2 * a * iP - t2 * (drx * ly - dry * lx);
    const T Qxz = -lz * drx * ir - drz * x * iP + t2 * drz * lx;
    const T Qyz = -lz * dry * ir - drz * y * iP + t2 * drz * ly;
    const T fLp = f * Lp;
    // C = (D + W) / 2 on and above the diagonal, (D - W) / 2 below, with
    // D_ed = kdf l_e l_d + f (kdl_e l_d + l_e kdl_d) and
    // W_ed = Lp (df_d l_e - df_e l_d) + f Lp Q_de + f (l_e M_d - l_d M_e),
    // Q_de = d_d l_e - d_e l_d. The time index is written out (l_0 = 1, kdl_0 = df_0 = M_0 = 0,
    // Q_0d = 0, W_ee = 0): IEEE arithmetic may not drop a product with a zero by itself.
    T C[4][4];
    C[0][0] = cHalf * kdf;
#pragma unroll
    for (int d = 1; d < 4; ++d) {
        const T D0 = kdf * l[d] + f * kdl[d];
        const T W0 = Lp * df[d] + f * M[d];
        C[0][d] = cHalf * (D0 + W0);
        C[d][0] = cHalf * (D0 - W0);
    }
#pragma unroll
    for (int e = 1; e < 4; ++e) {
        C[e][e] = cHalf * (kdf * l[e] * l[e] + f * (c2 * (kdl[e] * l[e])));
#pragma unroll
        for (int d = e + 1; d < 4; ++d) {
            const T Ded = kdf * l[e] * l[d] + f * (kdl[e] * l[d] + l[e] * kdl[d]);
            const T Qde = (d == 2) ? -Qxy : (e == 1 ? -Qxz : -Qyz);
            const T Wed = Lp * (df[d] * l[e] - df[e] * l[d]) + fLp * Qde +
                          f * (l[e] * M[d] - l[d] * M[e]);
            C[e][d] = cHalf * (Ded + Wed);
            C[d][e] = cHalf * (Ded - Wed);
        }
    }
    // A = -g^{-1} C with g^{ae} = eta^{ae} - f l^a l^e, l^a = (-1, l1, l2, l3)
    const T lu[4] = {-c1, lx, ly, lz};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const T lc = lu[0] * C[0][d] + lu[1] * C[1][d] + lu[2] * C[2][d] + lu[3] * C[3][d];
        A[0][d] = C[0][d] + f * lu[0] * lc;
#pragma unroll
        for (int e = 1; e < 4; ++e) A[e][d] = -C[e][d] + f * lu[e] * lc;
    }
}

// Coherency tensor stored as its real symmetric part (10) and imaginary antisymmetric part
// (6): re = [00 01 02 03 11 12 13 22 23 33], im = [01 02 03 12 13 23].
template <class T>
struct Coh {
    T re[10];
    T im[6];
};

template <class T>
__device__ __forceinline__ void coh_unpack(const Coh<T>& n, T R[4][4], T I[4][4]) {
    R[0][0] = n.re[0]; R[0][1] = R[1][0] = n.re[1]; R[0][2] = R[2][0] = n.re[2];
    R[0][3] = R[3][0] = n.re[3]; R[1][1] = n.re[4]; R[1][2] = R[2][1] = n.re[5];
    R[1][3] = R[3][1] = n.re[6]; R[2][2] = n.re[7]; R[2][3] = R[3][2] = n.re[8];
    R[3][3] = n.re[9];
    I[0][0] = I[1][1] = I[2][2] = I[3][3] = T(0);
    I[0][1] = n.im[0]; I[1][0] = -n.im[0]; I[0][2] = n.im[1]; I[2][0] = -n.im[1];
    I[0][3] = n.im[2]; I[3][0] = -n.im[2]; I[1][2] = n.im[3]; I[2][1] = -n.im[3];
    I[1][3] = n.im[4]; I[3][1] = -n.im[4]; I[2][3] = n.im[5]; I[3][2] = -n.im[5];
}

// out = base + h (A N + N A^T) for both parts (structure preserving).
template <class T>
__device__ __forceinline__ void coh_axpy(const Coh<T>& base, const Coh<T>& n, const T A[4][4],
                                         T h, Coh<T>& out) {
    T R[4][4], I[4][4];
    coh_unpack(n, R, I);
    T AR[4][4], AI[4][4];   // A N (the diagonal of A I is not needed, and I_jj = 0)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            T sr = T(0), si = T(0);
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                sr += A[i][d] * R[d][j];
                if (d != j) si += A[i][d] * I[d][j];
            }
            AR[i][j] = sr;
            AI[i][j] = si;
        }
    // (A N + N A^T)_ij = AN_ij + AN_ji for the symmetric part, AN_ij - AN_ji for the
    // antisymmetric part (N^T = +-N).
    int q = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) { out.re[q] = base.re[q] + h * (AR[i][j] + AR[j][i]); ++q; }
    q = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) { out.im[q] = base.im[q] + h * (AI[i][j] - AI[j][i]); ++q; }
}

// Predictor-corrector of Table tab:pc: N_h = N + h/2 F(A0, N), N' = N + h F(A1, N_h).
template <class T>
__device__ __forceinline__ void coh_pc_step(Coh<T>& n, const T A0[4][4], const T A1[4][4], T h) {
    Coh<T> nh;
    coh_axpy(n, n, A0, T(0.5) * h, nh);
    Coh<T> out;
    coh_axpy(n, nh, A1, h, out);
    n = out;
}

// ---------------------------------------------------------------------------------------
// Modified Bessel functions K_0, K_1 from the polynomial approximations of Abramowitz &
// Stegun 9.8.5-9.8.8 (|error| < 2.2e-7 relative to the scaled value); K_2 from the
// recurrence K_2 = K_0 + (2/x) K_1. bessel_k012 takes x and 1/x and returns K_n(x) itself
// for x <= 2 (false) and exp(x) K_n(x) for x > 2 (true), where K_n alone underflows for
// large x: callers that only need ratios, or fold exp(x) into an exponential of their own,
// skip the exp(x) of the small-argument branch.
// ---------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ bool bessel_k012(T x, T ix, T& k0, T& k1, T& k2) {
    bool scaled;
    if (x <= T(2)) {
        const T t = T(0.5) * x;
        const T t2 = t * t;
        const T lg = flog(t);
        const T i0 = cyl_bessel_i0(x);
        const T i1 = cyl_bessel_i1(x);
        const T p0 = T(-0.57721566) + t2 * (T(0.42278420) + t2 * (T(0.23069756) + t2 * (T(0.03488590) +
                     t2 * (T(0.00262698) + t2 * (T(0.00010750) + t2 * T(0.00000740))))));
        const T p1 = T(1) + t2 * (T(0.15443144) + t2 * (T(-0.67278579) + t2 * (T(-0.18156897) +
                     t2 * (T(-0.01919402) + t2 * (T(-0.00110404) + t2 * T(-0.00004686))))));
        k0 = -lg * i0 + p0;
        k1 = (x * lg * i1 + p1) * ix;
        scaled = false;
    } else {
        const T u = T(2) * ix;
        const T sx = rsqrt(x);
        k0 = sx * (T(1.25331414) + u * (T(-0.07832358) + u * (T(0.02189568) + u * (T(-0.01062446) +
                   u * (T(0.00587872) + u * (T(-0.00251540) + u * T(0.00053208)))))));
        k1 = sx * (T(1.25331414) + u * (T(0.23498619) + u * (T(-0.03655620) + u * (T(0.01504268) +
                   u * (T(-0.00780353) + u * (T(0.00325614) + u * T(-0.00068245)))))));
        scaled = true;
    }
    k2 = k0 + T(2) * ix * k1;
    return scaled;
}

// exp(x) K_n(x), n = 0, 1, 2, at every x (the stage entry point and the model's targets).
template <class T>
__device__ __forceinline__ void bessel_k012_scaled(T x, T& k0, T& k1, T& k2) {
    if (!bessel_k012(x, fq(T(1), x), k0, k1, k2)) {
        const T ex = fexp(x);
        k0 = k0 * ex;
        k1 = k1 * ex;
        k2 = k2 * ex;
    }
}

// ---------------------------------------------------------------------------------------
// Thermal synchrotron coefficients in the fluid frame (Sec. 2.5), CGS:
//   j_S = n e^2 nu / (sqrt 3 c K_2(1/Theta)) I_S(x) (S = I, Q),
//   j_V = 4 n e^2 nu cot(theta) / (3 sqrt 3 c Theta K_2(1/Theta)) I_V(x),
//   x = nu / (3/2 nu_B sin(theta) Theta^2), nu_B = e B / (2 pi m_e c);
//   alpha_S = j_S / B_nu(T_e) (Kirchhoff);
//   rho_Q = n e^2 nu_B^2 sin^2 / (m_e c nu^3) f_m(X) (K_1/K_2 + 6 Theta),
//   rho_V = 2 n e^2 nu_B cos / (m_e c nu^2) (K_0/K_2) g_m(X),
//   X = Theta (sqrt 2 sin(theta) 1e3 nu_B / nu)^{1/2}.
// Q > 0 is polarization perpendicular to the projected field.
// ---------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void synchrotron_coefficients(T ne, T th, T bg, T nu, T cth, T out[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q] = T(0);
    if (!(ne > T(0)) || !(th > T(0)) || !(bg > T(0))) return;
    const T sth2 = T(1) - cth * cth;
    const T sth = fsqrt(sth2 > T(0) ? sth2 : T(0));
    const T nub = T(kE / (2.0 * kPi * kMe * kC)) * bg;
    const T z = fq(T(1), th);
    const T inu = fq(T(1), nu);
    // K_n(z), scaled by exp(z) only for z > 2 (1 / z = Theta_e)
    T k0, k1, k2;
    const bool kscaled = bessel_k012(z, th, k0, k1, k2);
    const T ik2 = fq(T(1), k2);
    // 1 / x = 3/2 nu_B sin(theta) Theta^2 / nu; X^2 = (sqrt 2 1e3 / 1.5) / x, so X and the
    // emissivity's x^-1/2 share one square root
    const T ix = T(1.5) * nub * sth * th * th * inu;
    const T six = fsqrt(ix);
    if (sth > T(0)) {
        const T ix13 = fcbrt(ix);
        const T x13 = fq(T(1), ix13);
        const T ix23 = ix13 * ix13;
        // 1 / K_2(z) = exp(z) / k2 where k2 is scaled, and exp(z) is then taken together with
        // the shape functions' exp(-1.8899 x^1/3): their product stays finite (and underflows
        // to 0 for cold plasma) where exp(z) = exp(1 / Theta_e) alone would overflow
        const T ex = fexp((kscaled ? z : T(0)) - T(1.8899) * x13);
        const T ii = T(2.5651) * (T(1) + T(1.92) * ix13 + T(0.9977) * ix23) * ex;
        const T iq = T(2.5651) * (T(1) + T(0.932) * ix13 + T(0.4998) * ix23) * ex;
        // 1 / x = (x^-1/3)^3
        const T iv = (T(1.8138) * ix23 * ix13 + T(3.423) * ix23 + T(0.02955) * six +
                      T(2.0377) * ix13) * ex;
        const T pre = ne * T(kE * kE / (1.7320508075688772 * kC)) * nu * ik2;
        out[0] = pre * ii;
        out[1] = pre * iq;
        out[2] = pre * (T(4.0 / 3.0) * z) * fq(cth, sth) * iv;
        const T hkt = T(kH / (kMe * kC * kC)) * nu * z;
        // 1 / B_nu = c^2 expm1(h nu / k T) / (2 h nu^3), ordered to stay inside float range
        const T cnu = T(kC) * inu;
        const T ibnu = expm1(hkt) * (cnu * cnu) * (T(0.5 / kH) * inu);
        out[3] = out[0] * ibnu;
        out[4] = out[1] * ibnu;
        out[5] = out[2] * ibnu;
    }
    const T X = T(30.705195677312716) * six;
    // X^1.035 and X^1.2 as exponentials of one shared logarithm (X = 0 gives log X = -inf and
    // both powers 0, as pow does)
    const T lX = flog(X);
    const T p1 = fexp(T(1.035) * lX);
    const T p2 = fexp(T(1.2) * lX);
    const T fm = T(2.011) * fexp(-p1 * T(1.0 / 4.7)) - fcos(T(0.5) * X) * fexp(-p2 * T(1.0 / 2.73)) -
                 T(0.011) * fexp(-X * T(1.0 / 47.2));
    const T gm = T(1) - T(0.11) * log1p(T(0.035) * X);
    const T base = ne * T(kE * kE / (kMe * kC));
    const T inu2 = inu * inu;
    out[6] = base * nub * nub * sth2 * (inu2 * inu) * fm * (k1 * ik2 + T(6) * th);
    out[7] = T(2) * base * nub * cth * inu2 * (k0 * ik2) * gm;
}

// ---------------------------------------------------------------------------------------
// Unpolarized segment (Eq. unpolarized): exact solution of dI/dl = j - alpha I over dl with
// constant coefficients; optical depth >= 100 gives j / alpha, alpha = 0 gives I + j dl.
// ---------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T unpolarized_step(T j, T alpha, T dl, T i0) {
    if (alpha > T(0)) {
        const T dtau = alpha * dl;
        if (dtau >= T(100)) return j / alpha;
        return exp(-dtau) * (i0 + expm1(dtau) * j / alpha);
    }
    return i0 + j * dl;
}

// 1/k for the Taylor terms k = 1..14 of the Stokes step, correctly rounded in each type (a
// table read instead of a division inside a loop of run-time length).
__constant__ double c_inv_int64[15] = {0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6,
                                       1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12,
                                       1.0 / 13, 1.0 / 14};
__constant__ float c_inv_int32[15] = {0.0f, 1.0f, 1.0f / 2, 1.0f / 3, 1.0f / 4, 1.0f / 5,
                                      1.0f / 6, 1.0f / 7, 1.0f / 8, 1.0f / 9, 1.0f / 10,
                                      1.0f / 11, 1.0f / 12, 1.0f / 13, 1.0f / 14};
template <class T>
__device__ __forceinline__ T inv_int(int k) {
    if constexpr (sizeof(T) == 8) return c_inv_int64[k];
    else return c_inv_int32[k];
}

// ---------------------------------------------------------------------------------------
// Exact constant-coefficient polarized step over dl: S' = E S + T with
// [E T; 0 1] = exp([[-M dl, J dl], [0, 0]]), M the absorption/rotation matrix (U-terms zero).
// Scaling and squaring: the augmented matrix is scaled by 2^-s to norm <= 1/2, its
// exponential taken by a Horner-form Taylor polynomial, then squared s times. For
// alpha_I dl >= 100 the steady state M^{-1} J is returned (Eq. unpolarized's tau_max rule).
// ---------------------------------------------------------------------------------------
// Steady state M^{-1} J of the polarized step (optical depth alpha_I dl >= 100, the polarized
// form of Eq. unpolarized's tau_max rule): Gaussian elimination with partial pivoting on
// [M | J]. Out of line: rarely taken, and kept off the transfer loop's instruction footprint.
template <class T>
struct StokesV {
    T v[4];
};
template <class T>
struct StokesC {
    T c[8];
};

template <class T>
__device__ __noinline__ StokesV<T> stokes_steady(const StokesC<T> cc) {
    const T* c = cc.c;
    StokesV<T> out;
    T* s1 = out.v;
    const T aI = c[3], aQ = c[4], aV = c[5], rQ = c[6], rV = c[7];
    const T M[4][4] = {{aI, aQ, T(0), aV}, {aQ, aI, rV, T(0)}, {T(0), -rV, aI, rQ}, {aV, T(0), -rQ, aI}};
    const T J[4] = {c[0], c[1], T(0), c[2]};
    // Gaussian elimination with partial pivoting on [M | J].
    T a[4][5];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) a[i][j] = M[i][j];
        a[i][4] = J[i];
    }
    for (int col = 0; col < 4; ++col) {
        int p = col;
        for (int i = col + 1; i < 4; ++i)
            if (fabs(a[i][col]) > fabs(a[p][col])) p = i;
        if (p != col)
            for (int j = 0; j < 5; ++j) { T t = a[p][j]; a[p][j] = a[col][j]; a[col][j] = t; }
        const T inv = T(1) / a[col][col];
        for (int i = col + 1; i < 4; ++i) {
            const T fct = a[i][col] * inv;
            for (int j = col; j < 5; ++j) a[i][j] -= fct * a[col][j];
        }
    }
    for (int i = 3; i >= 0; --i) {
        T s = a[i][4];
        for (int j = i + 1; j < 4; ++j) s -= a[i][j] * s1[j];
        s1[i] = s / a[i][i];
    }
    return out;
}

// exp([Z z; 0 0]) applied to [s0; 1] for a scaled ||Z|| <= 1/2 that needed s >= 2 halvings:
// the Taylor polynomial of degree m of the matrix and of phi_1(Z) z, then s squarings of the
// augmented matrix. Out of line: rare (||M dl|| > 1), and large.
template <class T>
__device__ __noinline__ StokesV<T> stokes_expm(const StokesC<T> cc, T dl, int s,
                                               const StokesV<T> sv0) {
    const T* s0 = sv0.v;
    StokesV<T> out;
    T* s1 = out.v;
    // Z = -M dl 2^-s, z = J dl 2^-s (as in stokes_step, rebuilt here off the common path)
    const T aI = cc.c[3], aQ = cc.c[4], aV = cc.c[5], rQ = cc.c[6], rV = cc.c[7];
    const T sc = ldexp(T(1), -s);
    const T dls = dl * sc;
    const T Z[4][4] = {{-aI * dls, -aQ * dls, T(0), -aV * dls},
                       {-aQ * dls, -aI * dls, -rV * dls, T(0)},
                       {T(0), rV * dls, -aI * dls, -rQ * dls},
                       {-aV * dls, T(0), rQ * dls, -aI * dls}};
    const T z[4] = {cc.c[0] * dls, cc.c[1] * dls, T(0), cc.c[2] * dls};
    // Taylor degree: ||Z|| <= 1/2, truncation 2^-(m+1)/(m+1)! below the type's rounding.
    constexpr int m = sizeof(T) == 8 ? 13 : 8;
    // E = I + Z (I + Z/2 (I + Z/3 (...))),  t = (I + Z/2 (I + Z/3 (...))) z  (phi_1(Z) z)
    T E[4][4], tv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) E[i][j] = (i == j) ? T(1) : T(0);
        tv[i] = z[i] / T(m + 1);
    }
    for (int k = m; k >= 1; --k) {
        const T ik = T(1) / T(k);
        T En[4][4], tn[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                T acc = T(0);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc += Z[i][q] * E[q][j];
                En[i][j] = (i == j ? T(1) : T(0)) + acc * ik;
            }
        }
        if (k >= 2) {
            // tv <- z / k + Z tv / k  builds sum_n Z^n z / (n+1)!
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                T acc = T(0);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc += Z[i][q] * tv[q];
                tn[i] = (z[i] + acc) * ik;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) tv[i] = tn[i];
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                T acc = T(0);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc += Z[i][q] * tv[q];
                tn[i] = z[i] + acc;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) tv[i] = tn[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) E[i][j] = En[i][j];
    }
    // Squaring: [E t; 0 1]^2 = [E^2, E t + t; 0 1].
    for (int q = 0; q < s; ++q) {
        T E2[4][4], t2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                T acc = T(0);
#pragma unroll
                for (int r = 0; r < 4; ++r) acc += E[i][r] * E[r][j];
                E2[i][j] = acc;
            }
            T acc = tv[i];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc += E[i][r] * tv[r];
            t2[i] = acc;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            tv[i] = t2[i];
#pragma unroll
            for (int j = 0; j < 4; ++j) E[i][j] = E2[i][j];
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T acc = tv[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc += E[i][j] * s0[j];
        s1[i] = acc;
    }
    return out;
}

template <class T>
__device__ __forceinline__ void stokes_step(const T c[8], const T s0[4], T dl, T s1[4]) {
    const T aI = c[3], aQ = c[4], aV = c[5], rQ = c[6], rV = c[7];
    const T M[4][4] = {{aI, aQ, T(0), aV}, {aQ, aI, rV, T(0)}, {T(0), -rV, aI, rQ}, {aV, T(0), -rQ, aI}};
    const T J[4] = {c[0], c[1], T(0), c[2]};
    if (aI * dl >= T(100)) {
        StokesC<T> cc;
#pragma unroll
        for (int i = 0; i < 8; ++i) cc.c[i] = c[i];
        const StokesV<T> r = stokes_steady<T>(cc);
#pragma unroll
        for (int i = 0; i < 4; ++i) s1[i] = r.v[i];
        return;
    }
    // Z = -M dl, z = J dl. M_02 = M_13 = M_20 = M_31 = 0 and J_2 = 0 (no U terms) are left
    // out of the sums below: IEEE arithmetic may not drop a product with a zero by itself.
    // The series of exp([Z z; 0 0]) converges at the rate of Z alone (its z column only
    // multiplies), so scaling and Taylor degree follow the infinity norm of Z.
    auto mz = [](int i, int j) {
        return (i == 0 && j == 2) || (i == 1 && j == 3) || (i == 2 && j == 0) || (i == 3 && j == 1);
    };
    T Z[4][4], z[4];
    T nrm = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T rs = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Z[i][j] = mz(i, j) ? T(0) : -M[i][j] * dl;
            if (!mz(i, j)) rs += fabs(Z[i][j]);
        }
        z[i] = i == 2 ? T(0) : J[i] * dl;
        nrm = rs > nrm ? rs : nrm;
    }
    int s = 0;
    if (nrm > T(0.5)) {
        int e;
        frexp(nrm / T(0.5), &e);
        s = e;   // nrm / 2^s <= 0.5
    }
    const T sc = ldexp(T(1), -s);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (!mz(i, j)) Z[i][j] *= sc;
        if (i != 2) z[i] *= sc;
    }
    if (s <= 1) {
        // Only the action on [s0; 1] is needed: with A = [Z z; 0 0] (scaled), exp(A) x is
        // x + A (x + A/2 (x + ... (x + A x / d))), the last component staying 1, so each term
        // is one 4x4 matrix-vector product (16 FMAs) instead of a matrix product (64). The
        // scaled map is applied 2^s times (at most twice) in place of the squarings. The
        // degree d is the smallest whose truncation, ||Z||^d (||Z|| ||s0|| + ||z||) / (d+1)!,
        // is below the unit roundoff u relative to ||Z|| ||s0|| + ||z||: the first d with
        // ||Z|| <= theta_d = (u (d+1)!)^(1/d) (u = 2^-53 in FP64, 2^-24 in FP32), at most 14
        // (FP64) or 8 (FP32) for ||Z|| <= 1/2.
        constexpr int dmax = sizeof(T) == 8 ? 14 : 8;
        constexpr float th64[14] = {2.2e-16f, 2.58e-8f, 1.38e-5f, 3.39e-4f, 2.40e-3f, 9.07e-3f,
                                    2.39e-2f, 5.01e-2f, 9.03e-2f, 0.146f, 0.218f, 0.306f,
                                    0.411f, 0.531f};
        constexpr float th32[8] = {1.19e-7f, 5.98e-4f, 1.126e-2f, 5.17e-2f, 0.1338f, 0.2587f,
                                   0.4225f, 0.6192f};
        const float nz = (float)(nrm * sc);
        int d = 1;
#pragma unroll
        for (int q = 0; q < dmax - 1; ++q)
            if (nz > (sizeof(T) == 8 ? th64[q] : th32[q])) d = q + 2;
        T v[4] = {s0[0], s0[1], s0[2], s0[3]};
#pragma unroll 1
        for (int rep = 0; rep < (1 << s); ++rep) {
            T t[4] = {v[0], v[1], v[2], v[3]};
#pragma unroll 1
            for (int k = d; k >= 1; --k) {
                const T ik = inv_int<T>(k);
                T tn[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    T acc = z[i];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (!mz(i, q)) acc += Z[i][q] * t[q];
                    tn[i] = v[i] + acc * ik;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) t[i] = tn[i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = t[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) s1[i] = v[i];
        return;
    }
    StokesC<T> cc;
#pragma unroll
    for (int i = 0; i < 8; ++i) cc.c[i] = c[i];
    StokesV<T> v0;
#pragma unroll
    for (int i = 0; i < 4; ++i) v0.v[i] = s0[i];
    const StokesV<T> r = stokes_expm<T>(cc, dl, s, v0);
#pragma unroll
    for (int i = 0; i < 4; ++i) s1[i] = r.v[i];
}

}  // namespace bl
