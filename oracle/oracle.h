/*
 * CPU FP64 oracle for the Blacklight hot path (White 2022, "Blacklight: A General-Relativistic
 * Ray-Tracing and Analysis Tool").
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to judge the CUDA path: only the test-suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * It is written to be read against the paper, not to be fast:
 *   - metric derivatives come from forward-mode dual numbers, not hand-expanded formulas;
 *   - Christoffel symbols come from their definition in terms of d g_{ab};
 *   - the constant-coefficient polarized step is the exponential of the augmented 5x5
 *     matrix (scaling and squaring + Taylor series, long double);
 *   - modified Bessel functions come from trapezoid quadrature of their integral form.
 *
 * Each reading of a point the paper leaves open is stated next to the code that takes it.
 *
 * Parity unpinned: the polarized synchrotron fitting functions (the paper cites them without
 * printing them) are pinned only at their limits, by Kirchhoff's law, by symmetry, and (total,
 * linear and circular emissivity) against quadrature of the exact emissivity integrals.
 */
#ifndef BL_ORACLE_H
#define BL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double r, theta, phi;      /* camera centre, spherical Kerr-Schild */
    double u_p[3];             /* normal-frame velocity of the centre */
    double k_p[3];             /* received momentum, covariant spherical KS spatial components */
    double width;              /* full image width w (units of M) */
    int32_t n;                 /* pixels per side */
    double psi;                /* roll angle */
    int32_t kind;              /* 0 = plane-parallel */
    int32_t nu_at_infinity;    /* 1: -n k_t = nu ; 0: -n k.u = nu */
} ora_camera;

typedef struct {
    double mass, spin;
    double r_in_over_rhor;     /* inner termination radius / outer horizon radius */
    double tol_abs, tol_rel;   /* DP tolerances f_abs, f_rel */
    double ds_max;             /* proper-length subdivision limit */
    double h0_frac;            /* initial step = -h0_frac (r_cam - r_hor) */
    int64_t max_steps;         /* attempted-step limit */
    int32_t flat;              /* 1: Minkowski metric, same coordinates */
    /* integrator: 0 Dormand-Prince RK5(4) (Table tab:dp); 1 classical RK4 (Table tab:rk4);
     * 2 Heun RK2 (Table tab:rk2), both with steps -f_step (r - r_hor) (Eq. rk_step) */
    int32_t integrator;
    double f_step;
} ora_metric;

typedef struct {
    const float* prim;         /* host, [8][n_phi][n_theta][n_r], r fastest */
    int32_t n_r, n_theta, n_phi;
    double r_min, r_max;
    double gamma_ad, r_high, r_low, mu, ne_over_ni, sigma_cut, rho_unit_cgs, mass_msun;
    int32_t interp;            /* 1 trilinear, 0 nearest */
    /* Slow light (Sec. 4, "Slow Light"): prim holds n_snapshots consecutive grids at times
     * t_first + s dt; a sample at coordinate time x^t is taken at t_camera + x^t, linearly
     * between the two adjacent snapshots (time_interp 1) or from the nearest one (0), with the
     * time clamped to the first and last snapshot. n_snapshots <= 1: one grid, no time. */
    int32_t n_snapshots;
    int32_t time_interp;
    double t_first, dt, t_camera;
} ora_grid;

enum { ORA_OK = 0, ORA_HORIZON = 1, ORA_ESCAPED = 2, ORA_MAX_STEPS = 3, ORA_UNDERFLOW = 4,
       ORA_NAN = 5 };

/* ---- geometry (Sec. 2) ---- */
void ora_metric_cks(const double x[4], double mass, double spin, int flat,
                    double g_lo[16], double g_hi[16]);
void ora_metric_sks(double r, double theta, double mass, double spin, double g_lo[16]);
void ora_christoffel(const double x[4], double mass, double spin, int flat, double gam[64]);
void ora_geodesic_rhs(const double y[8], double mass, double spin, int flat, double dy[8]);
/* Test knob: scale geodesic right-hand-side component i by (1 + (-1)^i ulps 2^-52) in all
 * later oracle calls of this process (0, the default, switches it off). */
void ora_set_rhs_perturbation(int32_t ulps);
void ora_dp_tableau(double a[49], double b5[7], double b4[7], double bmid[7], double c[7]);
double ora_r_of_x(const double x[4], double spin);

/* ---- camera (Sec. 2.1) ---- */
/* pixel (i = horizontal, j = vertical): x^a, covariant k_a, H^a, V^a (contravariant), and the
 * frequency normalisation n. */
void ora_camera_pixel(const ora_camera* cam, const ora_metric* met, int32_t i, int32_t j,
                      double x[4], double k[4], double hvec[4], double vvec[4], double* nnorm);

/* ---- geodesic (Sec. 2.2): integrate backward from y0; returns status.
 * path (optional): receives up to max_path accepted-step end states [8]. */
int32_t ora_geodesic(const ora_metric* met, double r_cam, const double y0[8], double yf[8],
                     int64_t* attempts, int64_t* accepted, double* path, int64_t max_path,
                     int64_t* n_path);

/* ---- sampling, plasma, coefficients, transfer (Secs. 2.3-2.5) ---- */
/* auxiliary values per pixel of ora_trace (out_aux [npix][ORA_AUX_COUNT]); the list is in
 * radiation.cpp above trace_pixel */
#define ORA_AUX_COUNT 26
/* Eq. unpolarized: one constant-coefficient segment */
double ora_unpolarized_step(double j, double alpha, double dl, double i0);
int32_t ora_sample_grid(const ora_grid* grid, double spin, const double x[4], double prim[8]);
int32_t ora_plasma(const ora_grid* grid, const ora_metric* met, const double x[4],
                   double u[4], double b[4], double* ne, double* theta_e, double* b_gauss);
double ora_bessel_kx(double nu, double x);   /* exp(x) K_nu(x) */
/* out: j_I, j_Q, j_V, alpha_I, alpha_Q, alpha_V, rho_Q, rho_V (CGS, fluid frame) */
void ora_coefficients(double ne, double theta_e, double b_gauss, double nu, double cos_theta,
                      double out[8]);
/* coef: e_I, e_Q, e_V, a_I, a_Q, a_V, r_Q, r_V per unit affine parameter */
void ora_stokes_step(const double coef[8], const double s0[4], double dlam, double s1[4]);
/* one predictor-corrector coordinate step of the coherency tensor (re, im parts, [4][4]) */
void ora_transport_step(const ora_metric* met, const double x0[4], const double k0[4],
                        const double x1[4], const double k1[4], double h,
                        double n_re[16], double n_im[16]);

/* samples of one ray (camera-side first): [n][17] = x[4], k[4], node x[4], node k[4], dl;
 * returns the sample count (only the first max_out are written) */
int64_t ora_ray_samples(const ora_metric* met, const ora_grid* grid, double r_cam,
                        const double y0[8], int64_t max_out, double* out);
/* fluid-frame polarization basis and the Stokes <-> coherency maps (Sec. 2.3.2) */
void ora_fluid_frame(const double glo[16], const double u[4], const double kup[4],
                     const double b[4], double e1[4], double e2[4]);
void ora_n_to_s(const double glo[16], const double e1[4], const double e2[4],
                const double n_re[16], const double n_im[16], double s[4]);
void ora_s_to_n(const double e1[4], const double e2[4], const double s[4], double n_re[16],
                double n_im[16]);

/* ---- whole path ----
 * pix: flat pixel indices (j * n + i); out_stokes [npix][4] (I, Q, U, V in erg/s/cm^2/sr/Hz);
 * out_end [npix][8] end state; counters per pixel. nthreads <= 0 means all hardware threads. */
void ora_trace(const ora_camera* cam, const ora_metric* met, const ora_grid* grid, double freq,
               int64_t npix, const int32_t* pix, int32_t nthreads, double* out_stokes,
               int32_t* out_status, int64_t* out_attempts, int64_t* out_accepted,
               int64_t* out_samples, double* out_end, int32_t unpolarized, double* out_aux);

#ifdef __cplusplus
}
#endif
#endif
