// Internal data layout shared by the kernels and the host entry points.
#pragma once
#include <stdint.h>

namespace bl {

// Per-sample record written by the geodesic kernel and replayed by the transfer kernel:
// sample position x,y,z and covariant k_x,k_y,k_z; the node on the sample's camera side
// (same 6 values); the segment's affine length. k_t is constant per ray (Sec. 2.2) and is
// kept in the ray header.
constexpr int kRecVals = 13;   // values of a record the transfer uses; value 13 is the time
template <class R> struct RecStride;
template <> struct RecStride<double> { static constexpr int v = 14; };   // 112 B, 16-B aligned
template <> struct RecStride<float> { static constexpr int v = 16; };    // 64 B

constexpr int kChunk = 32;          // records per pool chunk
constexpr int kMaxChunks = 128;     // chunks per ray -> at most 4096 samples per ray

// Rays of the images of a batch are queued in blocks of 2^kIlvShift consecutive rays of one
// image when the batch interleaves its images (the default; plans may tune the block size).
constexpr int kIlvShift = 8;
constexpr int64_t kIlvBlock = int64_t(1) << kIlvShift;

struct ImageDesc {
    // camera (Sec. 2.1)
    double cam_r, cam_th, cam_ph, u_p[3], k_p[3], width, psi;
    int32_t n, nu_inf;
    // metric and integrator (Sec. 2.2)
    double mass, spin, r_in_over_rhor, tol_abs, tol_rel, ds_max, h0_frac;
    int64_t max_steps;
    int32_t flat, precision;
    int32_t integrator;
    int32_t ilv;            // > 1: the batch's rays are queued interleaved over ilv images
                            // in blocks of 2^ilv_shift rays (same values in every descriptor)
    int32_t ilv_shift;
    double f_step;
    // grid and plasma (Secs. 2.4-2.5)
    const float* prim;
    int32_t nr, nt, nph, interp;
    double r_min, r_max, gamma_ad, r_high, r_low, mu, ne_ni, sigma_cut, rho_unit, length_unit;
    // slow light: n_snap snapshots, spacing dt_snap; t_rel0 = t_first - t_camera, so that a
    // sample at ray time x^t sits at (x^t - t_rel0) / dt_snap on the snapshot axis
    int32_t n_snap, time_interp;
    double t_rel0, dt_snap;
    double freq;
    // outputs
    void* stokes;
    int32_t dtype, pad_;
    int32_t* status;
    int32_t* steps;
    double* end_state;
    int32_t* samples;
    void* aux;              // auxiliary images [26][n_rays] (dtype as stokes) or nullptr
    int64_t ray_offset;     // first global ray index of this image
    int64_t n_rays;         // rays traced for this image (n * n, or blocks x block^2)
    int32_t order;          // ray order: 0 Morton (n a power of 2), 1 rows
    int32_t layout;         // grid memory order: 0 planes [8][phi][theta][r], 1 cells [...][8]
    // filled by the camera-frame kernel
    double x_cam[4], u_cam[4], kk[4], hh[4], vv[4];
    double r_cam, r_hor;
    // per-image constants of the transfer, in double (d_*) and float (f_*), derived once on
    // the host (and H, V by the camera-frame kernel) so that samples do no conversions
    double d_c[20];
    float f_c[20];
    float f_hh[4], f_vv[4];
};

// indices into d_c / f_c
enum {
    kcGam1 = 0,      // gamma_ad - 1
    kcTePre,         // mu m_p / m_e
    kcNePre,         // rho_unit / (mu m_p)
    kcBgPre,         // c (4 pi rho_unit)^1/2
    kcDlr,           // ln(r_max / r_min) / n_r
    kcLogRmin,       // ln r_min
    kcRmin, kcRmax, kcSigma, kcRhigh, kcRlow, kcNeNi, kcFreq, kcLen, kcSpin, kcMass,
    kcIDlr,          // 1 / kcDlr
    kcNeFac,         // n_e per unit code density: kcNePre / (1 + n_i / n_e)
    kcCount
};

struct RayHdr {
    double kt;       // conserved covariant k_t
    double nnorm;    // frequency normalisation n per unit nu (Sec. 2.1)
    int32_t nrec;    // samples recorded
    int32_t status;  // BL_RAY_*
    int32_t last_in; // last record of a step that came within 1.001 r_max of the hole (-1:
                     // none); the records beyond it lie outside the grid and carry no plasma
};

// Initial state of a ray (Sec. 2.1, camera pixel): y = (x^a, k_a) and the frequency
// normalisation, written by ray_init_kernel before the geodesic kernel of a wave.
struct RayInit {
    double y[8];
    double nnorm;
};

// Rays taken from a device block list (adaptive levels) instead of consecutive image ranges:
// ray r traces pixel (bx B + r % B, by B + (r / B) % B) of image q, where (q, bx, by) =
// entries[r / B^2]; the number of blocks is read from the device, so a kernel earlier in the
// same stream may produce the list. Outputs are then indexed by r.
struct BlockSource {
    const int32_t* entries;               // [blocks][3] or nullptr (image ranges)
    const unsigned long long* count;      // blocks in the list
    int32_t block;                        // B
    int32_t pix_out;                      // 1: outputs at the pixel (cost-ordered queue of a
                                          // whole-image trace); 0: at the ray's list index
};

// Side inputs of the transfer variants that split their per-sample work over passes: the
// learned model's outputs (8 floats a pool record) and its parameters, or, in the FP64 form,
// each record's precomputed scaled coefficients and fluid-frame basis (24 doubles a pool
// record) with a flag byte (1: the sample carries plasma).
struct SideIn {
    const float* mlp_y;
    const float* mlp_params;
    const double* pre;
    const unsigned char* pre_flag;
    const int32_t* first;    // FP64 transport pass: each ray's farthest plasma sample, or -1
    const int32_t* perm;     // the transfer's ray order (wave ray indices), or nullptr
};
constexpr int kPreVals = 24;

struct Counters {
    unsigned long long next_ray_geo;
    unsigned long long next_ray_tr;
    unsigned long long pool_next;
    unsigned long long next_ray_mi;    // learned-coefficient model inputs: rays handed out
    unsigned long long bad_rays;
    unsigned long long mlp_timeouts;   // CTAs whose tensor-core wait ran out (never expected)
};

}  // namespace bl
