/*
 * blacklight.h -- C ABI of the GB300 (sm_103a) ray-tracing library for the hot path of
 * White 2022, "Blacklight: A General-Relativistic Ray-Tracing and Analysis Tool".
 *
 * The library computes, for every pixel of one or more plane-parallel cameras, a null
 * geodesic traced backward through Kerr spacetime in Cartesian Kerr-Schild coordinates
 * (Sec. 2, Eq. cks_aux; Sec. 2.2, Eq. geodesic) with the adaptive Dormand-Prince RK5(4)
 * integrator (Table tab:dp), samples a spherical Kerr-Schild fluid grid along it (Sec. 2.4),
 * derives the thermal-electron plasma state (Sec. 2.5), and integrates polarized radiative
 * transfer (Sec. 2.3.2, Eqs. polarized_s / polarized_n with Strang splitting and the
 * predictor-corrector of Table tab:pc) to Stokes I, Q, U, V at the camera.
 *
 * Conventions shared by every entry point:
 *   - All structs are plain data; their first field `size` must equal sizeof(struct) (ABI
 *     version check). All pointers are borrowed: the caller owns them and keeps them valid
 *     until the work on `stream` has finished.
 *   - Device pointers must belong to the current CUDA device. `stream` is a cudaStream_t
 *     (NULL = legacy default stream). Work is stream-ordered; without BL_ASYNC the call
 *     synchronises `stream` and reports per-ray anomalies in its return value.
 *   - Return value: 0 = success; > 0 = completed with per-ray anomalies (BL_WRAYS; see the
 *     per-ray status array); < 0 = error, nothing was launched or the launch failed
 *     (BL_EINVAL bad argument, BL_ENOMEM allocation failed, BL_ECUDA CUDA runtime error,
 *     BL_EUNSUPPORTED valid but not implemented). blacklight_last_error_detail() names the
 *     offending field (thread-local string, valid until the next call on that thread).
 *   - Device code never traps: rays that fail set their status word instead. Every device
 *     wait is bounded; a wait that runs out makes its kernel stop and the call return
 *     BL_ETIMEOUT, with the context still usable.
 *   - Lengths are in units of M = G M_bh / c^2; plasma and radiation in CGS.
 */
#ifndef BLACKLIGHT_H
#define BLACKLIGHT_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Camera (Sec. 2.1). The centre is given in spherical Kerr-Schild coordinates; u_p is the
 * centre's normal-frame velocity (Sec. 2, A^p = A^i + beta^i A^t), k_p the received
 * momentum direction as covariant spherical KS spatial components k_i. Pixel (i, j) sits at
 * a, b = (i or j - n/2 + 1/2) w / n along the horizontal H and vertical V directions. */
typedef struct bl_camera {
    uint32_t size;
    double r, theta, phi;
    double u_p[3];
    double k_p[3];
    double width;           /* full width w of the image plane */
    int32_t n;              /* pixels per side, 1..65536 */
    double psi;             /* roll about the line of sight */
    int32_t kind;           /* 0 = plane-parallel (only kind supported) */
    int32_t nu_at_infinity; /* 1: -n k_t = nu (Sec. 2.1); 0: -n k_a u^a = nu at the camera */
} bl_camera_t;

/* Spacetime and integrator controls (Sec. 2.2). */
typedef struct bl_metric {
    uint32_t size;
    double mass;            /* M (1 for lengths in M) */
    double spin;            /* a, |a| < M */
    double r_in_over_rhor;  /* inner termination radius in units of the outer horizon, > 1 */
    double tol_abs, tol_rel;/* DP tolerances f_abs, f_rel > 0 */
    double ds_max;          /* proper-length limit for step subdivision, > 0 */
    double h0_frac;         /* first step = -h0_frac (r_cam - r_hor) */
    int64_t max_steps;      /* attempted DP steps per ray before MAX_STEPS */
    int32_t flat;           /* 1: Minkowski metric in the same coordinates (Sec. 4, flat) */
    int32_t precision;      /* BL_PREC_FP64, BL_PREC_MIXED or BL_PREC_FAST */
    int32_t integrator;     /* BL_INT_DP (default), BL_INT_RK4 or BL_INT_RK2; all images of a
                               call share it */
    double f_step;          /* RK4/RK2: step -f_step (r - r_hor) (Eq. rk_step), 0 < f_step < 1 */
} bl_metric_t;

/* Geodesic integrators (Sec. 2.2). BL_INT_DP: adaptive Dormand-Prince RK5(4) (Table tab:dp)
 * with tol_abs, tol_rel, h0_frac. BL_INT_RK4 / BL_INT_RK2: classical RK4 (Table tab:rk4) and
 * Heun's method (Table tab:rk2) with the fixed rule of Eq. rk_step, always in FP64 (the
 * precision field then only selects the transfer arithmetic); a step's sample is its cubic
 * Hermite midpoint (y0 + y1)/2 + dl (f0 - f1)/8 (the paper defines the midpoint sample only for
 * DP), and max_steps counts steps. */
enum { BL_INT_DP = 0, BL_INT_RK4 = 1, BL_INT_RK2 = 2 };

/* Fluid grid and plasma model (Secs. 2.4-2.5). prim is a DEVICE pointer to float32
 * [8][n_phi][n_theta][n_r] (r fastest): rho, u_gas, u^p_(r,theta,phi) (normal frame),
 * B^(r,theta,phi) (coordinate components), on cells log-spaced in r over [r_min, r_max],
 * uniform in theta over [0, pi] and in phi over [0, 2 pi). */
typedef struct bl_grid {
    uint32_t size;
    const float* prim;
    int32_t n_r, n_theta, n_phi;
    double r_min, r_max;
    double gamma_ad;        /* adiabatic index: p = (gamma_ad - 1) u_gas */
    double r_high, r_low;   /* T_i / T_e prescription */
    double mu, ne_over_ni;  /* molecular weight, electron-to-ion number ratio */
    double sigma_cut;       /* sigma = b^2 / rho above this is vacuum */
    double rho_unit_cgs;    /* code density unit in g / cm^3 */
    double mass_msun;       /* black-hole mass in solar masses (sets the length unit) */
    int32_t interp;         /* 1 = trilinear, 0 = nearest */
    const float* coef_mlp;  /* NULL: coefficients from the exact fits (Sec. 2.5). Otherwise a
                               DEVICE parameter vector of the learned coefficient model
                               (BL_MLP_PARAMS floats, see blacklight_mlp_train), used for
                               samples inside its domain; all images of one call must pass the
                               same pointer, and the precision must be BL_PREC_MIXED or
                               BL_PREC_FAST (FP32 transfer). */
    /* Slow light (Sec. 4, "Slow Light"). n_snapshots <= 1: prim is one grid (fast light).
     * n_snapshots > 1: prim holds that many consecutive grids [n_snapshots][8][...] at
     * coordinate times t_first + s * dt_snapshots (dt_snapshots > 0); the camera centre is at
     * coordinate time t_camera, and a sample whose coordinate time along the ray is x^t (the
     * ray starts at the camera with x^t = 0 and runs backward) takes the fluid data at
     * t_camera + x^t, linearly between the two adjacent snapshots (time_interp 1) or from the
     * nearest snapshot (time_interp 0), clamped to the first and last snapshot. */
    int32_t n_snapshots;
    int32_t time_interp;
    double t_first;
    double dt_snapshots;
    double t_camera;
    /* Memory order of prim: BL_GRID_PLANES as described above, or BL_GRID_CELLS
     * [n_phi][n_theta][n_r][8] (per snapshot), the 8 values of a cell contiguous in 32 bytes,
     * prim 16-byte aligned; blacklight_grid_pack writes it. The values and the results are the
     * same in both; with cells each of the 8 corners a trilinear sample reads is two 16-byte
     * loads instead of eight scalar loads from eight planes. */
    int32_t layout;
} bl_grid_t;

enum { BL_GRID_PLANES = 0, BL_GRID_CELLS = 1 };

/* Outputs. stokes is a DEVICE pointer to [4][n][n] (I, Q, U, V; row j = vertical index
 * major) in erg s^-1 cm^-2 sr^-1 Hz^-1, float64 (dtype 0) or float32 (dtype 1). status,
 * steps (attempted DP steps) and samples (transfer samples) are optional DEVICE int32 [n][n]
 * (may be NULL). end_state is an optional DEVICE float64 [n][n][8] receiving the geodesic end
 * point (x^a, k_a). */
typedef struct bl_out {
    uint32_t size;
    void* stokes;
    int32_t dtype;
    int32_t* status;
    int32_t* steps;
    double* end_state;
    int32_t* samples;
    void* aux;              /* optional DEVICE [BL_AUX_COUNT][n][n] auxiliary images (Sec. 4,
                               "Auxiliary Images"), same dtype as stokes, or NULL */
} bl_out_t;

/* Auxiliary images, planes of bl_out_t.aux:
 *   0 Kerr-Schild time from the geodesic's termination to the camera (-x^t at the end)
 *   1 proper length of the geodesic, sum over steps of |dl| (g_pq k^p k^q)^1/2 at the step's
 *     midpoint;  2 elapsed affine parameter, sum of |dl|
 *   3 I_j = integral of j_I dl;  4 tau = integral of alpha_I dl  (unpolarized invariants per
 *     unit affine parameter, observed frequency)
 *   5-11  <q>_lambda = integral q dl / [2]
 *   12-18 <q>_Ij = integral q j_I dl / I_j  (0 where I_j = 0)
 *   19-25 <q>_tau, the solution of d<q>/dtau = q - <q> from the source end
 *   q in the order rho (code units), n_e (cm^-3), p (code units), Theta_e, B (gauss), sigma,
 *   beta^-1; samples without plasma contribute q = 0. */
#define BL_AUX_COUNT 26

enum {
    BL_OK = 0,
    BL_WRAYS = 1,
    BL_EINVAL = -1,
    BL_ENOMEM = -2,
    BL_ECUDA = -3,
    BL_EUNSUPPORTED = -4,
    BL_ETIMEOUT = -5        /* a bounded device wait ran out; the kernel stopped cleanly */
};

/* Per-ray status words. */
enum {
    BL_RAY_OK = 0,          /* not terminated (only before tracing) */
    BL_RAY_HORIZON = 1,     /* crossed the inner radius (Sec. 2.2) */
    BL_RAY_ESCAPED = 2,     /* crossed the camera radius outward (Sec. 2.2) */
    BL_RAY_MAX_STEPS = 3,   /* max_steps attempts without terminating */
    BL_RAY_UNDERFLOW = 4,   /* |step| fell below 1e-12 r */
    BL_RAY_NAN = 5,         /* non-finite state */
    BL_RAY_OVERFLOW = 6     /* sample store full: Stokes not computed (NaN) */
};

/* Arithmetic of the path:
 *   BL_PREC_FP64  geodesics, sampling, plasma, coefficients and transfer in FP64;
 *   BL_PREC_MIXED geodesics and step control in FP64, the rest in FP32;
 *   BL_PREC_FAST  geodesics in double-float (pairs of FP32, ~48-bit significand, step
 *                 control in FP32), the rest in FP32.
 * The FP32 part takes quotients, exp, log, cos, sin-cos and square roots from the hardware
 * approximations (errors of order 1e-6 relative, below the FP32 forms' image error against
 * the FP64 form: ~2e-6 relative L2 on a 16x16 image, ~1e-4 at 1024x1024); the FP64 form
 * uses IEEE arithmetic and the libm functions. */
enum { BL_PREC_FP64 = 0, BL_PREC_MIXED = 1, BL_PREC_FAST = 2 };
/* flags: BL_ASYNC returns without synchronising; BL_TIMING records CUDA events on `stream`
 * around the geodesic and transfer kernels of every wave (read with
 * blacklight_last_kernel_ms); BL_UNPOLARIZED integrates unpolarized transfer (Sec. 2.3.1,
 * Eq. unpolarized) instead of the polarized equations: Stokes I only, Q = U = V = 0 (not with
 * the learned coefficient model). */
enum { BL_ASYNC = 1u, BL_TIMING = 2u, BL_UNPOLARIZED = 8u };

/* Trace n_images cameras with persistent launch pairs (geodesics, then transfer). Image q
 * uses cams[q], mets[q], grids[q], freqs_hz[q] (observed frequency, > 0) and outs[q]. All
 * images must share metric.precision. The rays of all images are traced in waves of at most
 * 2^20 rays, one launch pair per wave, reusing one workspace. workspace may be NULL (the
 * library then allocates stream-ordered scratch and frees it before returning) or a DEVICE
 * buffer, 256-byte aligned, the call uses instead: blacklight_workspace_size() bytes give the
 * default waves; a
 * smaller buffer is accepted and runs smaller waves (BL_EINVAL if it cannot hold one ray).
 * Results do not depend on the wave size.
 * Ray order (scheduling only; results do not depend on it): a DP batch of at least 65536 rays
 * whose images all have n a multiple of 8 and cell-layout grids is queued as 8x8 pixel blocks,
 * longest predicted work first. The prediction is the DP attempt count of each block's centre ray, integrated
 * beforehand with the double-float geodesic kernel (1/64 of the rays, no transfer, at most 512
 * attempts a ray; in BL_PREC_FAST with both tolerances 1000 times larger, capped at 1e-3;
 * five extra launches). Other batches queue each image's rays in Morton order (n a power of
 * two) or rows. */
int blacklight_trace_batch(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                           const bl_grid_t* grids, const double* freqs_hz, const bl_out_t* outs,
                           void* workspace, size_t workspace_bytes, void* stream,
                           uint32_t flags);

/* Repack a grid of n_snapshots >= 1 consecutive snapshots from BL_GRID_PLANES to
 * BL_GRID_CELLS on `stream` (asynchronous, one kernel):
 *   cells[((s n_phi + k) n_theta + j) n_r + i][v] = planes[(((s 8 + v) n_phi + k) n_theta + j) n_r + i].
 * planes and cells are DEVICE pointers to 8 n_r n_theta n_phi n_snapshots floats each, not
 * overlapping; cells must be 16-byte aligned and stays owned by the caller. BL_EINVAL on
 * sizes < 1, NULL, host or misaligned pointers. */
int blacklight_grid_pack(const float* planes, float* cells, int32_t n_r, int32_t n_theta,
                         int32_t n_phi, int32_t n_snapshots, void* stream);

/* One image: blacklight_trace_batch with n_images = 1 and library-managed scratch. */
int blacklight_trace(const bl_camera_t* cam, const bl_metric_t* met, const bl_grid_t* grid,
                     double freq_hz, const bl_out_t* out, void* stream, uint32_t flags);

/* blacklight_trace for callers that cannot allocate device memory (no cudaMalloc,
 * cudaMallocAsync or cudaFree on any path). The paper has no counterpart: this exists for
 * callers that trace inside an allocator they do not control -- a fixed memory budget set at
 * start-up, a foreign memory pool, or a context where allocation is forbidden. Instead of
 * allocating, it uses a fixed 64 MiB scratch array compiled into the library (held by every
 * device that loads the library until the process exits), which limits it to images of at
 * most 1024 rays (e.g. 32x32); larger cameras return BL_EINVAL with an explanation. Within
 * that limit every integrator and precision is accepted: rays whose sample records need more
 * than the array holds at once (long fixed-step RK4/RK2 rays) run in several smaller waves.
 * Inputs and outputs are caller-owned device memory as for blacklight_trace.
 * The array is reserved on a device when the library's device code is loaded there, which
 * under CUDA's default lazy loading is the first call into the library on that device (this
 * entry point's or any other): make one call, e.g. a small trace, while allocation is still
 * allowed. The first call on each device also looks up the array's device address (make that
 * call before any stream capture). All calls share the one array: calls whose work overlaps
 * on the GPU (other streams, other host threads) race and corrupt each other; order them on
 * one stream. The call always synchronises `stream` before returning, so that BL_WRAYS and
 * BL_ETIMEOUT are reported from the shared counters; BL_ASYNC and BL_TIMING are ignored. */
int blacklight_trace_noalloc(const bl_camera_t* cam, const bl_metric_t* met,
                             const bl_grid_t* grid, double freq_hz, const bl_out_t* out,
                             void* stream, uint32_t flags);

/* Same as blacklight_trace, but grid->prim (and grid->coef_mlp if set) and
 * out->stokes/status/steps/end_state are HOST pointers: the call copies the grid in, traces,
 * and copies the results out (all stream-ordered, device scratch allocated and freed
 * inside). Always synchronous. */
int blacklight_trace_host(const bl_camera_t* cam, const bl_metric_t* met, const bl_grid_t* grid,
                          double freq_hz, const bl_out_t* out, void* stream);

/* blacklight_trace_batch with HOST buffers: grids[q].prim (and coef_mlp) and every pointer in
 * outs[q] are host pointers (pinned memory copies fastest). A grid whose prim pointer appears
 * in several images is copied to the device once (and repacked to the cell layout there);
 * all images are then traced in one batched launch and the outputs copied back. The grid
 * copies run on a non-blocking stream the library keeps for each device, concurrently with
 * the camera and geodesic kernels on `stream` (which do not read the grids); the transfer
 * kernel waits for them. Synchronous: returns after `stream` has finished the call's work;
 * device scratch is allocated and freed inside. flags: BL_UNPOLARIZED (BL_ASYNC and BL_TIMING
 * are ignored). */
int blacklight_trace_host_batch(int32_t n_images, const bl_camera_t* cams,
                                const bl_metric_t* mets, const bl_grid_t* grids,
                                const double* freqs_hz, const bl_out_t* outs, void* stream,
                                uint32_t flags);

/* Geodesics only (Sec. 2.2): writes out->end_state, out->status and out->steps (attempted
 * DP steps); out->stokes is ignored. */
int blacklight_geodesics(const bl_camera_t* cam, const bl_metric_t* met, const bl_out_t* out,
                         void* stream, uint32_t flags);

/* ---------------------------------------------------------------------------------------
 * Plans: a batched trace prepared once and replayed as a CUDA graph (the paper's code has no
 * counterpart; it re-traces from scratch on CPU threads). blacklight_plan_create validates
 * the arguments exactly like blacklight_trace_batch, allocates the workspace, uploads the
 * image descriptors, optionally autotunes the launch configuration, and captures the launch
 * sequence (counter reset, camera frames, one geodesic + transfer pair per wave of 2^20 rays)
 * in a CUDA graph; blacklight_plan_run replays it with one graph launch. The plan binds the
 * pointers in grids and outs and the camera/metric/frequency values: between runs the caller
 * may rewrite the contents of grids[q].prim (a new snapshot) and read the outputs, but must
 * create a new plan for other pointers or parameters. Runs on different streams must not
 * overlap (they share the plan's workspace).
 * --------------------------------------------------------------------------------------- */
typedef struct bl_plan bl_plan_t;
typedef struct bl_launch_config {
    uint32_t size;
    int32_t ray_order;        /* 0 Morton order within each image (n a power of two), 1 rows,
                                 2 the work-ordered queue of 8x8 blocks described at
                                 blacklight_trace_batch (the default where the batch allows it;
                                 BL_EINVAL elsewhere) */
    int32_t geo_ctas_per_sm;  /* persistent geodesic CTAs per SM, 0 = occupancy limit */
    int32_t tr_ctas_per_sm;   /* persistent transfer CTAs per SM, 0 = occupancy limit */
    float run_ms;             /* autotuned plans: device time of one run with this configuration */
    int32_t ilv_block;        /* batches of equal images on cell-layout grids queue their rays
                                 interleaved in blocks of this many rays of one image: a power
                                 of two in [64, 4096] dividing the rays of an image, 0 = the
                                 default (256); reported as 0 where the batch does not
                                 interleave */
} bl_launch_config_t;
/* flags for blacklight_plan_create: search ray order, interleave block and CTAs per SM
 * (coordinate descent over timed runs of the plan's own workload; the images' outputs are
 * written while tuning). The choice is cached per device and workload shape for the life of
 * the process. */
enum { BL_PLAN_AUTOTUNE = 4u };
/* config: NULL = defaults (the work-ordered queue where the batch allows it, else Morton;
 * occupancy limits), ignored with BL_PLAN_AUTOTUNE. `stream`
 * is used for the tuning runs and the capture (the legacy default stream is replaced by a
 * private stream for the capture). */
int blacklight_plan_create(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                           const bl_grid_t* grids, const double* freqs_hz, const bl_out_t* outs,
                           const bl_launch_config_t* config, uint32_t flags, void* stream,
                           bl_plan_t** plan);
/* Replay the plan on `stream` (asynchronous). */
int blacklight_plan_run(bl_plan_t* plan, void* stream);
/* Synchronise `stream` and report the last run: 0, or BL_WRAYS if some ray ended abnormally. */
int blacklight_plan_check(bl_plan_t* plan, void* stream);
/* The plan's launch configuration. */
int blacklight_plan_config(const bl_plan_t* plan, bl_launch_config_t* out);
/* Free the plan (synchronises the device). NULL is ignored. */
int blacklight_plan_destroy(bl_plan_t* plan);


/* Adaptive ray tracing (Sec. 4, "Adaptive Ray Tracing"). The root n x n image is split into
 * square blocks of `block` pixels; each traced block is judged on its own pixels' Stokes I:
 * when at least min_count pixels have a criterion value above `threshold`, every pixel of the
 * block is split into four and the four child blocks are traced at the next level (pixel
 * size halved), up to max_level. Criteria, with one-sided differences at block edges:
 *   BL_CRIT_ABS_GRAD  (D_i^2 + D_j^2)^1/2, D_i = (I[i+1] - I[i-1]) / 2
 *   BL_CRIT_REL_GRAD  same with D_i = 2 (I[i+1] - I[i-1]) / (I[i-1] + 2 I[i] + I[i+1])
 *   BL_CRIT_ABS_LAPL  |D_i + D_j|, D_i = I[i-1] - 2 I[i] + I[i+1]
 *   BL_CRIT_REL_LAPL  |D_i + D_j|, D_i = 4 (I[i-1] - 2 I[i] + I[i+1]) / (I[i-1] + 2 I[i] + I[i+1])
 * A criterion that evaluates to NaN (e.g. 0/0 in dark regions) does not count. */
typedef struct bl_adapt {
    uint32_t size;
    int32_t block;          /* block side in pixels; must divide the root n */
    int32_t max_level;      /* 0 = no refinement */
    int32_t criterion;      /* BL_CRIT_* */
    double threshold;
    int32_t min_count;      /* pixels of a block that must exceed the threshold, >= 1 */
    double min_intensity;   /* pixels with Stokes I below this never count (0 = all count);
                               keeps relative criteria from acting on numerically dark pixels */
} bl_adapt_t;

enum { BL_CRIT_ABS_GRAD = 0, BL_CRIT_REL_GRAD = 1, BL_CRIT_ABS_LAPL = 2, BL_CRIT_REL_LAPL = 3 };

/* Trace n_images cameras adaptively (one launch pair per level and wave for all images; the
 * levels follow each other on the device, without host round trips). outs[q].stokes
 * receives the composite image at the finest resolution, DEVICE [4][nf][nf] with
 * nf = n * 2^max_level, each pixel taking the value of the finest traced pixel covering it
 * (dtype 0 float64 / 1 float32); outs[q].status/steps/samples/end_state/aux are ignored.
 * level_rays (optional HOST int32 [n_images][max_level + 1]) receives the rays traced per level.
 * Synchronises `stream` at the end. A level holds at most 2^26 rays (BL_EUNSUPPORTED beyond). */
int blacklight_trace_adaptive(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                              const bl_grid_t* grids, const double* freqs_hz,
                              const bl_adapt_t* adapt, const bl_out_t* outs, int32_t* level_rays,
                              void* stream);
/* An adaptive trace (see blacklight_trace_adaptive) prepared as a plan: every level's launches,
 * the composites, the refinement decisions and the next level's block lists run on the device
 * without host round trips, captured in one CUDA graph. flags: 0 or BL_UNPOLARIZED. Run with
 * blacklight_plan_run; blacklight_plan_check or blacklight_plan_level_rays report the last run
 * (BL_EUNSUPPORTED if a level needed more than 2^26 rays). */
int blacklight_plan_create_adaptive(int32_t n_images, const bl_camera_t* cams,
                                    const bl_metric_t* mets, const bl_grid_t* grids,
                                    const double* freqs_hz, const bl_adapt_t* adapt,
                                    const bl_out_t* outs, uint32_t flags, void* stream,
                                    bl_plan_t** plan);
/* Rays traced per level in the last run of an adaptive plan (HOST int32 [n_images][max_level
 * + 1]); synchronises `stream`; returns like blacklight_plan_check. */
int blacklight_plan_level_rays(bl_plan_t* plan, int32_t* level_rays, void* stream);

/* Workspace bytes blacklight_trace_batch uses for these images with its default waves
 * (at most 2^20 rays each). */
size_t blacklight_workspace_size(int32_t n_images, const bl_camera_t* cams,
                                 const bl_metric_t* mets);

/* ---------------------------------------------------------------------------------------
 * Learned coefficient model. The paper evaluates the thermal synchrotron fits of Sec. 2.5
 * directly; this library can instead evaluate their transcendental parts with a small
 * perceptron (3 -> 64 -> 64 -> 7, SiLU, BF16 weights and activations on the tensor cores,
 * FP32 accumulation), trained on the GPU on samples of the exact fits, with the exact fits
 * kept for samples outside its domain.
 *   inputs  (log10 x, log10 Theta_e, |cos theta_B|), x = nu / nu_c, nu_c = 1.5 nu_B
 *           sin(theta_B) Theta_e^2, on the domain [-3, 6] x [-1, 2] x [0, 1];
 *   outputs o1..o7: ln of the I, Q, V emissivity shape prefactors (I_S(x) = exp(o_S -
 *           1.8899 x^1/3)), the Faraday conversion and rotation shapes f_m, g_m, ln(e^z K_2(z))
 *           and ln(K_0(z) / K_2(z)) with z = 1 / Theta_e. The remaining factors (n_e, nu, B,
 *           the angle factors, the Planck function) are exact.
 * Parameters: float [BL_MLP_PARAMS] = W1 [64][4] (column 3 = first-layer bias), W2 [64][64],
 * b2 [64], W3 [7][64], b3 [7], output offset [7], output scale [7], output trend A [7][3].
 * The model is o = offset + scale * y + A f, y the network output and f the three inputs
 * mapped linearly to [-1, 1]; offset, A and scale are fixed before training. All arrays are DEVICE pointers unless stated; calls are stream-ordered
 * and synchronise `stream` before returning; BL_ECUDA if a tensor-core wait ran out (never
 * expected; the kernels stop instead of waiting forever).
 * --------------------------------------------------------------------------------------- */
#define BL_MLP_PARAMS 4906

/* Glorot-uniform weights, zero biases, offset 0, scale 1, A 0, from the SplitMix64 stream
 * `seed`. */
int blacklight_mlp_init(float* params, uint64_t seed, void* stream);
/* n samples uniform on the input domain (SplitMix64 stream `seed`) into inputs [n][3] and
 * the exact learned quantities (FP64 fits, stored as float) into targets [n][7]. */
int blacklight_mlp_dataset(int64_t n, uint64_t seed, float* inputs, float* targets,
                           void* stream);
/* Exact learned quantities targets [n][7] of inputs [n][3]. */
int blacklight_mlp_targets(int64_t n, const float* inputs, float* targets, void* stream);
/* Set offset and A of params to the least-squares affine fit of targets [n][7] on the mapped
 * inputs [n][3], and scale to the root mean square of its residual. */
int blacklight_mlp_normalise(int64_t n, const float* inputs, const float* targets, float* params,
                             void* stream);

typedef struct bl_mlp_train {
    uint32_t size;
    int64_t n;               /* training samples (>= batch) */
    const float* inputs;     /* DEVICE [n][3] */
    const float* targets;    /* DEVICE [n][7] */
    int32_t batch;           /* samples per step: a multiple of 128 */
    int64_t steps;           /* Adam steps; step t uses samples t*batch .. (mod n) */
    double lr_start, lr_end; /* learning rate, geometric from lr_start to lr_end */
    double beta1, beta2, eps;/* Adam (Kingma & Ba 2015) */
} bl_mlp_train_t;
/* Train params in place (mean squared error of the normalised outputs). loss_history:
 * optional DEVICE float [steps] receiving each step's mean squared error. */
int blacklight_mlp_train(const bl_mlp_train_t* cfg, float* params, float* loss_history,
                         void* stream);
/* Gradient of the mean squared error over the n samples into grad [BL_MLP_PARAMS] (zero for
 * offset, scale and A) and the error itself into *loss (HOST float). */
int blacklight_mlp_grad(const float* params, int64_t n, const float* inputs, const float* targets,
                        float* grad, float* loss, void* stream);
/* Model outputs o [n][7] (denormalised) for inputs [n][3]. */
int blacklight_mlp_forward(const float* params, int64_t n, const float* inputs, float* outputs,
                           void* stream);
/* Like blacklight_coefficients (precision FP32) with the learned model inside its domain and
 * the exact fits outside it. in [n][5], out [n][8], float64. */
int blacklight_mlp_coefficients(const float* params, int64_t n, const double* in, double* out,
                                void* stream);

/* Component entry points (same device functions as the traced path), for checking each
 * stage on its own. All arrays are DEVICE pointers; n elements; precision selects the FP64
 * or FP32 device code.
 *   coefficients (Sec. 2.5): in [n][5] = n_e, Theta_e, B (gauss), nu (fluid frame), cos
 *     theta_B; out [n][8] = j_I, j_Q, j_V, alpha_I, alpha_Q, alpha_V, rho_Q, rho_V.
 *   stokes_step (Sec. 2.3.2): coef [n][8] = e_I, e_Q, e_V, a_I, a_Q, a_V, r_Q, r_V per unit
 *     affine parameter; s0 [n][4]; dl [n]; out s1 [n][4]: exact constant-coefficient step.
 *   bessel_k (scaled): in x [n]; out [n][3] = exp(x) K_0, K_1, K_2. */
int blacklight_coefficients(int64_t n, const double* in, double* out, int32_t precision,
                            void* stream);
int blacklight_stokes_step(int64_t n, const double* coef, const double* s0, const double* dl,
                           double* s1, int32_t precision, void* stream);
int blacklight_bessel_k(int64_t n, const double* x, double* out, int32_t precision,
                        void* stream);

/* Refinement decisions alone (Sec. 4): I is DEVICE float64 [n_blocks][block][block] (row-major
 * Stokes I of each block), flags DEVICE int8 [n_blocks] receives 1 where the block refines
 * under the criterion of bl_adapt_t (adapt->max_level is ignored). */
int blacklight_adapt_flags(int64_t n_blocks, const double* I, const bl_adapt_t* adapt,
                           int8_t* flags, void* stream);

/* Device memory the library allocates stream-ordered (scratch of calls without a caller
 * workspace, host-buffer staging) comes from the current device's default memory pool, which
 * by default returns freed memory to the system at every synchronisation, so a later call maps
 * it again (tens of ms for the ~20 GB of a 9 x 256^2 batch). This sets the pool's release
 * threshold: up to `bytes` of freed memory stay reserved for reuse (UINT64_MAX: all; 0: the
 * CUDA default). The setting belongs to the process's default pool for this device and
 * applies to every user of it. */
int blacklight_set_memory_retention(uint64_t bytes);

/* Self-test of the bounded device wait used by the tensor-core kernels: one CTA initialises
 * an mbarrier and waits on it for at most max_cycles SM cycles (1 <= max_cycles <= 2^32); with
 * arrive = 1 it arrives first (returns 0), with arrive = 0 nothing arrives and the wait runs out
 * (returns BL_ETIMEOUT). No fault, no unbounded wait. */
int blacklight_selftest_wait(int64_t max_cycles, int32_t arrive, void* stream);

/* Arithmetic peaks of the current device, measured (the paper has no counterpart: these are
 * the denominators of the rooflines a benchmark reports). Each probe is a kernel of
 * independent multiply-add chains x <- x a + b (2 flops a step) on every SM at full
 * occupancy, timed with CUDA events on `stream` after one warm-up launch; the best of `reps`
 * launches of ~15 ms each is kept (a burst figure: the SM clock during the probes is the
 * caller's to record).
 *   fp64_tflops: native FP64 FMA;  fp32_tflops: native FP32 FMA;
 *   df64_tflops: the double-float multiply-add of this library's double-float integrator
 *     (a compensated product plus sum of two-float values, counted as 2 flops).
 * sm_count is cudaDevAttrMultiProcessorCount and sm_clock_khz cudaDevAttrClockRate (the
 * maximum SM clock) of the device. 1 <= reps <= 100, else BL_EINVAL. Synchronous. */
typedef struct {
    uint32_t size;          /* sizeof(bl_peaks_t) */
    int32_t sm_count;
    int32_t sm_clock_khz;
    double fp64_tflops;
    double fp32_tflops;
    double df64_tflops;
    double probe_ms;        /* device time of one timed launch of each probe, summed */
} bl_peaks_t;
int blacklight_measure_peaks(bl_peaks_t* out, int32_t reps, void* stream);

const char* blacklight_strerror(int code);
const char* blacklight_last_error_detail(void);
/* Kernels launched by this thread since the last reset (launch accounting for benchmarks). */
uint64_t blacklight_launch_count(int reset);
/* Device time of the geodesic phase (ms[0]: the rays' initial states and the geodesic kernel)
 * and of the transfer kernel (ms[1]) of this thread's last call made with BL_TIMING, summed
 * over its waves; waits for that call's work. Returns 0, or BL_EINVAL if no timed call was
 * made. */
int blacklight_last_kernel_ms(float ms[2]);

#ifdef __cplusplus
}
#endif
#endif
