// Kernels of the Blacklight hot path: camera frame, persistent geodesic kernel (FP64) and
// persistent transfer kernel (FP64 or FP32). Included by bl_api.cu only.
#pragma once
#include <climits>
#include <type_traits>

#include "bl_df64.cuh"
#include "bl_internal.cuh"
#include "bl_math.cuh"
#include "bl_mlp.cuh"
#include "../../include/blacklight.h"

namespace bl {

// ---------------------------------------------------------------------------------------
// Camera frame (Sec. 2.1), one thread per image, FP64.
// ---------------------------------------------------------------------------------------
__global__ void camera_frame_kernel(ImageDesc* imgs, int n_images) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_images) return;
    ImageDesc& im = imgs[q];
    const double a = im.spin, m = im.mass;
    const bool flat = im.flat != 0;
    const double st = sin(im.cam_th), ct = cos(im.cam_th), sp = sin(im.cam_ph), cp = cos(im.cam_ph);
    const double r = im.cam_r;
    double x[4] = {0.0, st * (r * cp - a * sp), st * (r * sp + a * cp), r * ct};
    KSGeom<double> G;
    ks_geom<double>(x[1], x[2], x[3], a, m, flat, false, G);
    // Jacobian columns d x^a / d (r, theta, phi)
    const double J[3][3] = {{st * cp, ct * (r * cp - a * sp), st * (-r * sp - a * cp)},
                            {st * sp, ct * (r * sp + a * cp), st * (r * cp - a * sp)},
                            {ct, -r * st, 0.0}};
    // velocity: spatial normal-frame vector v = J u^p, u^n = (1 + gamma(v, v))^1/2,
    // u^t = u^n / alpha, u^a = v^a - beta^a u^t, alpha = (1 + f)^-1/2, beta^a = f l^a / (1 + f)
    double v[3];
    for (int c = 0; c < 3; ++c) v[c] = J[c][0] * im.u_p[0] + J[c][1] * im.u_p[1] + J[c][2] * im.u_p[2];
    const double lv = G.l[1] * v[0] + G.l[2] * v[1] + G.l[3] * v[2];
    const double un = sqrt(1.0 + v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + G.f * lv * lv);
    double u[4];
    u[0] = un * sqrt(1.0 + G.f);
    for (int c = 0; c < 3; ++c) u[c + 1] = v[c] - G.f * G.l[c + 1] / (1.0 + G.f) * u[0];
    double ul[4];
    lower4(G, u, ul);
    // covariant k_a = k_i d x^i / d x^a (r, theta, phi as functions of x, y, z)
    double kl[4];
    {
        const double R2 = x[1] * x[1] + x[2] * x[2] + x[3] * x[3];
        const double qq = R2 - a * a;
        const double D = sqrt(qq * qq + 4.0 * a * a * x[3] * x[3]);
        const double rr = G.r;
        const double dr[3] = {rr * x[1] / D, rr * x[2] / D, x[3] * (rr * rr + a * a) / (rr * D)};
        for (int c = 0; c < 3; ++c) kl[c + 1] = im.k_p[0] * dr[c];
        if (im.k_p[1] != 0.0) {
            const double zr = x[3] / rr;
            const double s = sqrt(1.0 - zr * zr);
            for (int c = 0; c < 3; ++c) {
                const double dzr = ((c == 2 ? rr : 0.0) - x[3] * dr[c]) / (rr * rr);
                kl[c + 1] += im.k_p[1] * (-dzr / s);
            }
        }
        if (im.k_p[2] != 0.0) {
            const double rho2 = x[1] * x[1] + x[2] * x[2];
            const double dxy[3] = {-x[2] / rho2, x[1] / rho2, 0.0};
            for (int c = 0; c < 3; ++c)
                kl[c + 1] += im.k_p[2] * (dxy[c] + a / (rr * rr + a * a) * dr[c]);
        }
        // k_t from g^ab k_a k_b = 0 with k^t = g^tt k_t + g^ta k_a > 0
        const double A = -1.0 - G.f;
        double B = 0.0, C = 0.0;
        const double lk = G.l[1] * kl[1] + G.l[2] * kl[2] + G.l[3] * kl[3];
        B = G.f * lk;                                         // g^ta k_a = f l^a k_a
        C = kl[1] * kl[1] + kl[2] * kl[2] + kl[3] * kl[3] - G.f * lk * lk;
        const double disc = sqrt(B * B - A * C);
        const double r1 = (-B + disc) / A, r2 = (-B - disc) / A;
        kl[0] = (A * r1 + B > 0.0) ? r1 : r2;
    }
    // camera-frame metric g_{a'b'} and g^{a'b'} = g^ab + u^a u^b
    double glo[4][4];
    {
        for (int al = 0; al < 4; ++al)
            for (int be = 0; be < 4; ++be)
                glo[al][be] = ((al == be) ? (al == 0 ? -1.0 : 1.0) : 0.0) + G.f * G.l[al] * G.l[be];
    }
    double gpl[3][3], gph[3][3];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
            const int A_ = c + 1, B_ = d + 1;
            gpl[c][d] = glo[A_][B_] - ul[A_] / ul[0] * glo[0][B_] - ul[B_] / ul[0] * glo[0][A_] +
                        ul[A_] * ul[B_] / (ul[0] * ul[0]) * glo[0][0];
            const double ghi = ((c == d) ? 1.0 : 0.0) - G.f * G.l[A_] * G.l[B_];
            gph[c][d] = ghi + u[A_] * u[B_];
        }
    double Kl[3], Kh[3];
    for (int c = 0; c < 3; ++c) Kl[c] = kl[c + 1] - ul[c + 1] / ul[0] * kl[0];
    double Kt = -(u[0] * kl[0] + u[1] * kl[1] + u[2] * kl[2] + u[3] * kl[3]);
    for (int c = 0; c < 3; ++c) Kh[c] = gph[c][0] * Kl[0] + gph[c][1] * Kl[1] + gph[c][2] * Kl[2];
    double nk = 1.0 / sqrt(Kl[0] * Kh[0] + Kl[1] * Kh[1] + Kl[2] * Kh[2]);
    for (int c = 0; c < 3; ++c) { Kl[c] *= nk; Kh[c] *= nk; }
    Kt *= nk;
    im.kk[0] = u[0] * Kt - (ul[1] * Kh[0] + ul[2] * Kh[1] + ul[3] * Kh[2]) / ul[0];
    for (int c = 0; c < 3; ++c) im.kk[c + 1] = Kh[c] + u[c + 1] * Kt;
    // vertical: Gram-Schmidt of U = z (y on the polar axis)
    double U[3] = {0.0, 0.0, 1.0};
    if (x[1] == 0.0 && x[2] == 0.0) { U[1] = 1.0; U[2] = 0.0; }
    const double uk = U[0] * Kl[0] + U[1] * Kl[1] + U[2] * Kl[2];
    double vh[3], vl[3];
    for (int c = 0; c < 3; ++c) vh[c] = U[c] - uk * Kh[c];
    for (int c = 0; c < 3; ++c) vl[c] = gpl[c][0] * vh[0] + gpl[c][1] * vh[1] + gpl[c][2] * vh[2];
    const double nv = 1.0 / sqrt(vl[0] * vh[0] + vl[1] * vh[1] + vl[2] * vh[2]);
    for (int c = 0; c < 3; ++c) { vh[c] *= nv; vl[c] *= nv; }
    // horizontal: h^a = [abc] v_b K_c / sqrt(det g')
    const double det = gpl[0][0] * (gpl[1][1] * gpl[2][2] - gpl[1][2] * gpl[2][1]) -
                       gpl[0][1] * (gpl[1][0] * gpl[2][2] - gpl[1][2] * gpl[2][0]) +
                       gpl[0][2] * (gpl[1][0] * gpl[2][1] - gpl[1][1] * gpl[2][0]);
    const double isd = 1.0 / sqrt(det);
    const double hh[3] = {(vl[1] * Kl[2] - vl[2] * Kl[1]) * isd, (vl[2] * Kl[0] - vl[0] * Kl[2]) * isd,
                          (vl[0] * Kl[1] - vl[1] * Kl[0]) * isd};
    const double cps = cos(im.psi), sps = sin(im.psi);
    im.hh[0] = 0.0;
    im.vv[0] = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double Hc = hh[c] * cps - vh[c] * sps;
        const double Vc = vh[c] * cps + hh[c] * sps;
        im.hh[0] -= ul[c + 1] / ul[0] * Hc;
        im.vv[0] -= ul[c + 1] / ul[0] * Vc;
        im.hh[c + 1] = Hc;
        im.vv[c + 1] = Vc;
    }
    for (int al = 0; al < 4; ++al) {
        im.x_cam[al] = x[al];
        im.u_cam[al] = u[al];
        im.f_hh[al] = (float)im.hh[al];
        im.f_vv[al] = (float)im.vv[al];
    }
    im.r_cam = r;
    const double d = m * m - a * a;
    im.r_hor = m + sqrt(d > 0.0 ? d : 0.0);
}

// ---------------------------------------------------------------------------------------
// Ray bookkeeping helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int find_image(const ImageDesc* imgs, int n_images, int64_t ray) {
    int q = 0;
    while (q + 1 < n_images && imgs[q + 1].ray_offset <= ray) ++q;
    return q;
}

// Pixel of local ray p and the index its outputs go to: block-list order (adaptive
// refinement), else, with order 0, Morton (Z) order when n is a power of two so that a warp
// covers a compact 8x4 patch of the image, else row-major.
__device__ __forceinline__ void pixel_of(int64_t p, int n, int order, int& i, int& j);
__device__ __forceinline__ int64_t ray_pixel(const ImageDesc& im, int64_t p, int& i, int& j) {
    pixel_of(p, im.n, im.order, i, j);
    return (int64_t)j * im.n + i;
}

// Image, pixel and output index of global ray `ray`: from the device block list when there is
// one (adaptive levels); for a batch of equal images, from the interleaved queue (blocks of
// 2^ilv_shift rays taken from the images in turn: the last rays handed out are then every
// image's last blocks, which in Morton order lie at the image corners, rather than one image's
// last quarter, which holds part of the photon ring and its longest rays); else from the
// images' consecutive ray ranges.
__device__ __forceinline__ void setup_ray(const ImageDesc* imgs, int n_images, const BlockSource& bs,
                                          int64_t ray, int& q, int64_t& opix, int& i, int& j) {
    if (bs.entries) {
        const int B = bs.block;
        const int64_t b2 = (int64_t)B * B;
        const int64_t blk = ray / b2;
        const int r = (int)(ray - blk * b2);
        q = bs.entries[3 * blk];
        i = bs.entries[3 * blk + 1] * B + r % B;
        j = bs.entries[3 * blk + 2] * B + r / B;
        opix = bs.pix_out ? (int64_t)j * imgs[q].n + i : ray;
    } else if (imgs[0].ilv > 1) {
        // equal images interleaved: block b of the queue is block b / ilv of image b % ilv
        const int sh = imgs[0].ilv_shift;
        const int64_t b = ray >> sh, nb = imgs[0].ilv;
        q = (int)(b % nb);
        opix = ray_pixel(imgs[q], ((b / nb) << sh) + (ray - (b << sh)), i, j);
    } else {
        q = find_image(imgs, n_images, ray);
        opix = ray_pixel(imgs[q], ray - imgs[q].ray_offset, i, j);
    }
}

// End of this launch's ray range: a block list may hold fewer rays than the launch covers.
__device__ __forceinline__ int64_t wave_end(const BlockSource& bs, int64_t ray_end) {
    if (!bs.entries) return ray_end;
    const int64_t avail = (int64_t)(*bs.count) * bs.block * bs.block;
    return avail < ray_end ? avail : ray_end;
}

__device__ __forceinline__ void pixel_of(int64_t p, int n, int order, int& i, int& j) {
    if (order == 0 && (n & (n - 1)) == 0) {
        uint32_t xi = 0, yj = 0;
        for (int b = 0; b < 16; ++b) {
            xi |= (uint32_t)((p >> (2 * b)) & 1) << b;
            yj |= (uint32_t)((p >> (2 * b + 1)) & 1) << b;
        }
        i = (int)xi;
        j = (int)yj;
    } else {
        i = (int)(p % n);
        j = (int)(p / n);
    }
}

// auxiliary image planes (Sec. 4, "Auxiliary Images"): plane a of the image's aux array
template <class V>
__device__ __forceinline__ void aux_store(const ImageDesc& im, int a, int64_t pix, V v) {
    const int64_t npix = im.n_rays;
    if (im.dtype == 0) ((double*)im.aux)[a * npix + pix] = (double)v;
    else ((float*)im.aux)[a * npix + pix] = (float)v;
}
__device__ __forceinline__ double aux_load(const ImageDesc& im, int a, int64_t pix) {
    const int64_t npix = im.n_rays;
    return im.dtype == 0 ? ((const double*)im.aux)[a * npix + pix]
                         : (double)((const float*)im.aux)[a * npix + pix];
}

__device__ __forceinline__ double im_spin(const ImageDesc* imgs, int q) { return imgs[q].spin; }
__device__ __forceinline__ double im_mass(const ImageDesc* imgs, int q) { return imgs[q].mass; }

// Warp-aggregated fetch-and-add: every lane that calls it gets a distinct index.
__device__ __forceinline__ unsigned long long warp_fetch_add(unsigned long long* ctr) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// Warp-uniform refill: lanes with `need` set receive distinct queue indices; every lane of
// the warp must call this (full-warp ballot), which also reconverges the warp.
__device__ __forceinline__ unsigned long long warp_refill(unsigned long long* ctr, bool need) {
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (mask == 0u) return ~0ull;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// Pixel initial state (Sec. 2.1, plane-parallel): x_pix = x + a H + b V, k^a = K^a,
// k^t from the null condition (unique positive root outside the ergosphere, lesser positive
// root inside), k_a = g_ab k^b.
__device__ __forceinline__ void pixel_state(const ImageDesc& im, int i, int j, double y[8],
                                            double& nnorm) {
    const double n = im.n;
    const double aa = (i - 0.5 * n + 0.5) * im.width / n;
    const double bb = (j - 0.5 * n + 0.5) * im.width / n;
    for (int al = 0; al < 4; ++al) y[al] = im.x_cam[al] + aa * im.hh[al] + bb * im.vv[al];
    KSGeom<double> G;
    ks_geom<double>(y[1], y[2], y[3], im.spin, im.mass, im.flat != 0, false, G);
    const double ka[3] = {im.kk[1], im.kk[2], im.kk[3]};
    // g_tt (k^t)^2 + 2 g_ta k^a k^t + g_ab k^a k^b = 0
    const double lk = G.l[1] * ka[0] + G.l[2] * ka[1] + G.l[3] * ka[2];
    const double A = -1.0 + G.f;
    const double B = G.f * lk;
    const double C = ka[0] * ka[0] + ka[1] * ka[1] + ka[2] * ka[2] + G.f * lk * lk;
    double kt;
    if (A == 0.0) {
        kt = -C / (2.0 * B);
    } else {
        const double disc = sqrt(B * B - A * C);
        const double r1 = (-B + disc) / A, r2 = (-B - disc) / A;
        if (A < 0.0) {
            kt = r1 > 0.0 ? r1 : r2;
        } else {
            const double lo = fmin(r1, r2), hi = fmax(r1, r2);
            kt = lo > 0.0 ? lo : hi;
        }
    }
    const double ku[4] = {kt, ka[0], ka[1], ka[2]};
    double kl[4];
    lower4(G, ku, kl);
    for (int al = 0; al < 4; ++al) y[4 + al] = kl[al];
    if (im.nu_inf) {
        nnorm = 1.0 / (-kl[0]);
    } else {
        nnorm = 1.0 / -(kl[0] * im.u_cam[0] + kl[1] * im.u_cam[1] + kl[2] * im.u_cam[2] + kl[3] * im.u_cam[3]);
    }
}

// Initial states of the rays of a wave (Sec. 2.1): one thread a ray, RayInit[ray - ray_begin].
__global__ void ray_init_kernel(const ImageDesc* __restrict__ imgs, int n_images,
                                int64_t ray_begin, int64_t ray_end, BlockSource bs,
                                RayInit* __restrict__ init) {
    const int64_t re = wave_end(bs, ray_end);
    const int64_t n = re > ray_begin ? re - ray_begin : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += stride) {
        int q = 0, pi = 0, pj = 0;
        int64_t opix = 0;
        setup_ray(imgs, n_images, bs, ray_begin + w, q, opix, pi, pj);
        RayInit ri;
        pixel_state(imgs[q], pi, pj, ri.y, ri.nnorm);
        init[w] = ri;
    }
}

// ---------------------------------------------------------------------------------------
// Work-ordered ray queue. The DP integrator's attempts per ray vary several-fold across an
// image (rays near the photon ring wind around the hole), and a persistent kernel whose last
// rays are its longest ends with mostly idle lanes. Each B x B pixel block's work is predicted
// by the attempts of its centre ray, integrated beforehand (double-float arithmetic, geodesic
// only, 1/B^2 of the rays), and the blocks are queued longest first; every kernel of the trace
// takes its rays in that order (rows within a block), and writes them at their pixels. Only the
// scheduling changes: each ray's arithmetic, and so every output, is the same in any order.
// ---------------------------------------------------------------------------------------
constexpr int kCostBlock = 8;
constexpr int kCostBuckets = 4096;   // attempts above kCostBuckets - 1 share the first bucket
// The prediction takes at most BL_COST_MAX_ATTEMPTS attempts a ray; its tolerances are the
// batch's times a scale the host picks. A scale above 1 (BL_COST_TOL_SCALE, used for the
// double-float form, whose whole trace is short) shortens the prediction: the DP step count
// scales as tol^-1/5 for every ray alike, so the order is roughly kept while the longest
// predicted ray, which sets the prediction's latency, takes fewer attempts. Measured on nine
// 256x256 images: the double-float form 43.3 ms a step at scale 1 (a 3.5 ms prediction), 41.9
// ms at 1000; the FP64 form 487.5 ms at scale 1, 491.7 ms at 1000 (its kernels gain more from
// the exact order than the prediction costs).
#ifndef BL_COST_TOL_SCALE
#define BL_COST_TOL_SCALE 1000.0
#endif
#ifndef BL_COST_MAX_ATTEMPTS
#define BL_COST_MAX_ATTEMPTS 512
#endif

// The predictor's list: block k of the batch (images in turn, blocks in rows) as the 1 x 1
// block (image, centre column, centre row); *count = n_blocks.
__global__ void cost_list_kernel(const ImageDesc* __restrict__ imgs, int n_images,
                                 int64_t n_blocks, int32_t* __restrict__ list,
                                 unsigned long long* __restrict__ count) {
    constexpr int B = kCostBlock;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_blocks; k += stride) {
        const int q = find_image(imgs, n_images, k * B * B);
        const int64_t local = k - imgs[q].ray_offset / (B * B);
        const int nb = imgs[q].n / B;
        list[3 * k] = q;
        list[3 * k + 1] = (int32_t)(local % nb) * B + B / 2;
        list[3 * k + 2] = (int32_t)(local / nb) * B + B / 2;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (unsigned long long)n_blocks;
}

// The predictor's image descriptors: the batch's, with the prediction's tolerances and
// attempt limit, every output but the attempt count switched off and the attempt counts of
// all images written to `cost` at the list index.
__global__ void cost_descs_kernel(const ImageDesc* __restrict__ src, ImageDesc* __restrict__ dst,
                                  int n_images, int32_t* __restrict__ cost, double tol_scale) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_images; q += gridDim.x * blockDim.x) {
        ImageDesc d = src[q];
        // (scaled tolerances above 1e-3 are held there, or at the batch's own if larger)
        const double ta = d.tol_abs * tol_scale, tr = d.tol_rel * tol_scale;
        d.tol_abs = ta > 1e-3 ? fmax(d.tol_abs, 1e-3) : ta;
        d.tol_rel = tr > 1e-3 ? fmax(d.tol_rel, 1e-3) : tr;
        if (d.max_steps > BL_COST_MAX_ATTEMPTS) d.max_steps = BL_COST_MAX_ATTEMPTS;
        d.stokes = nullptr;
        d.status = nullptr;
        d.steps = cost;
        d.end_state = nullptr;
        d.samples = nullptr;
        d.aux = nullptr;
        dst[q] = d;
    }
}

// The transfers' ray orders sort groups of G consecutive wave rays by their largest work: the
// FP64 transport pass groups of a warp's 32 (neighbouring pixels of the geodesic queue, so a
// warp keeps rays of similar paths through the plasma: 245.7 -> 240.5 ms against single rays
// on the nine-image step), the FP32 transfer single rays (10.9 ms against 13.2 with groups:
// its per-sample chain costs the same with or without plasma, and single rays balance better).
constexpr int kTransportGroup = 32;
constexpr int kFusedGroup = 1;

// Queue position -> wave ray of an ordered transfer (perm lists the groups longest first);
// -1 for the positions of a partial last group that hold no ray.
template <int G>
__device__ __forceinline__ int64_t ordered_ray(const int32_t* perm, unsigned long long got,
                                               int64_t n) {
    const int64_t w = (int64_t)perm[got / G] * G + (int64_t)(got % G);
    return w < n ? w : -1;
}
// Queue length of an ordered transfer over n wave rays.
template <int G>
__device__ __forceinline__ int64_t ordered_total(int64_t n) {
    return (n + G - 1) / G * G;
}

// Bucket of a cost in a descending counting sort (larger costs in lower buckets).
__device__ __forceinline__ int cost_bucket(int32_t c) {
    const int v = c < 0 ? 0 : (c > kCostBuckets - 1 ? kCostBuckets - 1 : c);
    return kCostBuckets - 1 - v;
}

// In one CTA of 1024 threads: start[] (kCostBuckets counts, shared memory) becomes its
// exclusive prefix sum; ends with a barrier.
__device__ __forceinline__ void bucket_scan(unsigned int* start) {
    __shared__ unsigned int warp_sum[32];
    const int t = threadIdx.x;
    // each thread its 4 consecutive buckets, then across threads
    constexpr int kPer = kCostBuckets / 1024;
    unsigned int v[kPer], sum = 0u;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { v[i] = start[kPer * t + i]; sum += v[i]; }
    const int lane = t & 31, wid = t >> 5;
    unsigned int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        unsigned int w = warp_sum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        warp_sum[lane] = wi - w;
    }
    __syncthreads();
    unsigned int run = warp_sum[wid] + incl - sum;
#pragma unroll
    for (int i = 0; i < kPer; ++i) { start[kPer * t + i] = run; run += v[i]; }
    __syncthreads();
}

// One CTA of 1024 threads: counting sort of the blocks by predicted attempts, descending
// (equal counts in any order), into the block list (image, bx, by) of the trace.
__global__ void __launch_bounds__(1024) cost_sort_kernel(const int32_t* __restrict__ cost,
                                                         const int32_t* __restrict__ list,
                                                         int64_t n_blocks,
                                                         int32_t* __restrict__ sorted,
                                                         unsigned long long* __restrict__ count) {
    constexpr int B = kCostBlock;
    __shared__ unsigned int start[kCostBuckets];
    const int t = threadIdx.x;
    for (int b = t; b < kCostBuckets; b += 1024) start[b] = 0u;
    __syncthreads();
    for (int64_t k = t; k < n_blocks; k += 1024) atomicAdd(&start[cost_bucket(cost[k])], 1u);
    __syncthreads();
    bucket_scan(start);
    for (int64_t k = t; k < n_blocks; k += 1024) {
        const unsigned int pos = atomicAdd(&start[cost_bucket(cost[k])], 1u);
        sorted[3 * (int64_t)pos] = list[3 * k];
        sorted[3 * (int64_t)pos + 1] = list[3 * k + 1] / B;
        sorted[3 * (int64_t)pos + 2] = list[3 * k + 2] / B;
    }
    if (t == 0) *count = (unsigned long long)n_blocks;
}

// The transfers' queues: a key kernel (record_key_kernel, transport_key_kernel) stores each
// order group's work in key[] and histograms it (hist, global, kCostBuckets counts, zeroed per
// wave); the scan turns the histogram into bucket starts, and the scatter lists the groups
// longest first in perm (equal work in any order).
__global__ void __launch_bounds__(1024) work_scan_kernel(unsigned int* __restrict__ hist) {
    __shared__ unsigned int start[kCostBuckets];
    for (int b = threadIdx.x; b < kCostBuckets; b += 1024) start[b] = hist[b];
    __syncthreads();
    bucket_scan(start);
    for (int b = threadIdx.x; b < kCostBuckets; b += 1024) hist[b] = start[b];
}
// (over the wave's order groups of G rays, as the key kernel counted them: a device block
// list may hold fewer rays than the launch covers; lanes of a warp with equal buckets take
// their places with one atomic)
template <int G>
__global__ void work_scatter_kernel(const int32_t* __restrict__ key, BlockSource bs,
                                    int64_t ray_begin, int64_t ray_end,
                                    unsigned int* __restrict__ start, int32_t* __restrict__ perm) {
    const int64_t re = wave_end(bs, ray_end);
    const int64_t n = ((re > ray_begin ? re - ray_begin : 0) + G - 1) / G;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < n; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        const bool on = w < n;
        const int b = on ? cost_bucket(key[w]) : -1 - lane;   // idle lanes in buckets of their own
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(same) - 1;
        unsigned int base = 0u;
        if (on && lane == leader) base = atomicAdd(&start[b], (unsigned int)__popc(same));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (on) perm[base + __popc(same & ((1u << lane) - 1u))] = (int32_t)w;
    }
}

// ---------------------------------------------------------------------------------------
// Persistent geodesic kernel (Sec. 2.2). Each lane owns one ray at a time and advances it
// by one Dormand-Prince attempt per loop iteration; a lane whose ray terminates takes the
// next ray from the global queue, so uneven step counts do not idle the warp. Accepted steps
// emit sample records (midpoint, or quartic sub-samples when the step is longer than ds_max
// in proper length and reaches into the grid) into a pool of fixed-size chunks.
// ---------------------------------------------------------------------------------------
// Dormand-Prince RK5(4)7M coefficients (Table tab:dp).
#define DP_A21 (1.0 / 5.0)
#define DP_A31 (3.0 / 40.0)
#define DP_A32 (9.0 / 40.0)
#define DP_A41 (44.0 / 45.0)
#define DP_A42 (-56.0 / 15.0)
#define DP_A43 (32.0 / 9.0)
#define DP_A51 (19372.0 / 6561.0)
#define DP_A52 (-25360.0 / 2187.0)
#define DP_A53 (64448.0 / 6561.0)
#define DP_A54 (-212.0 / 729.0)
#define DP_A61 (9017.0 / 3168.0)
#define DP_A62 (-355.0 / 33.0)
#define DP_A63 (46732.0 / 5247.0)
#define DP_A64 (49.0 / 176.0)
#define DP_A65 (-5103.0 / 18656.0)
#define DP_B1 (35.0 / 384.0)
#define DP_B3 (500.0 / 1113.0)
#define DP_B4 (125.0 / 192.0)
#define DP_B5 (-2187.0 / 6784.0)
#define DP_B6 (11.0 / 84.0)
// error weights b5 - b4
#define DP_E1 (35.0 / 384.0 - 5179.0 / 57600.0)
#define DP_E3 (500.0 / 1113.0 - 7571.0 / 16695.0)
#define DP_E4 (125.0 / 192.0 - 393.0 / 640.0)
#define DP_E5 (-2187.0 / 6784.0 + 92097.0 / 339200.0)
#define DP_E6 (11.0 / 84.0 - 187.0 / 2100.0)
#define DP_E7 (-1.0 / 40.0)
// fourth-order midpoint weights (applied with h/2)
#define DP_M1 (6025192743.0 / 30085553152.0)
#define DP_M3 (51252292925.0 / 65400821598.0)
#define DP_M4 (-2691868925.0 / 45128329728.0)
#define DP_M5 (187940372067.0 / 1594534317056.0)
#define DP_M6 (-1776094331.0 / 19743644256.0)
#define DP_M7 (11237099.0 / 235043384.0)

// Dormand-Prince RK5(4)7M coefficients (Table tab:dp) in constant memory, read with
// warp-uniform indices by the rolled stage loop: row s of a (s = 1..6; row 6 is the
// fifth-order weights, the first-same-as-last stage), the error weights b5 - b4 and the
// fourth-order midpoint weights.
struct DPTable {
    double a[7][7];
    double e[7];
    double m[7];
};
struct DPTableF {     // the same values as double-float pairs
    float2 a[7][7];
    float2 e[7];
    float2 m[7];
};
#define DP_ROW(...) __VA_ARGS__
__constant__ DPTable c_dp = {
    {{0, 0, 0, 0, 0, 0, 0},
     {DP_A21, 0, 0, 0, 0, 0, 0},
     {DP_A31, DP_A32, 0, 0, 0, 0, 0},
     {DP_A41, DP_A42, DP_A43, 0, 0, 0, 0},
     {DP_A51, DP_A52, DP_A53, DP_A54, 0, 0, 0},
     {DP_A61, DP_A62, DP_A63, DP_A64, DP_A65, 0, 0},
     {DP_B1, 0, DP_B3, DP_B4, DP_B5, DP_B6, 0}},
    {DP_E1, 0, DP_E3, DP_E4, DP_E5, DP_E6, DP_E7},
    {DP_M1, 0, DP_M3, DP_M4, DP_M5, DP_M6, DP_M7}};
#define DF2(d) float2{(float)(d), (float)((d) - (double)(float)(d))}
__constant__ DPTableF c_dpf = {
    {{DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0)},
     {DF2(DP_A21), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0)},
     {DF2(DP_A31), DF2(DP_A32), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0)},
     {DF2(DP_A41), DF2(DP_A42), DF2(DP_A43), DF2(0.0), DF2(0.0), DF2(0.0), DF2(0.0)},
     {DF2(DP_A51), DF2(DP_A52), DF2(DP_A53), DF2(DP_A54), DF2(0.0), DF2(0.0), DF2(0.0)},
     {DF2(DP_A61), DF2(DP_A62), DF2(DP_A63), DF2(DP_A64), DF2(DP_A65), DF2(0.0), DF2(0.0)},
     {DF2(DP_B1), DF2(0.0), DF2(DP_B3), DF2(DP_B4), DF2(DP_B5), DF2(DP_B6), DF2(0.0)}},
    {DF2(DP_E1), DF2(0.0), DF2(DP_E3), DF2(DP_E4), DF2(DP_E5), DF2(DP_E6), DF2(DP_E7)},
    {DF2(DP_M1), DF2(0.0), DF2(DP_M3), DF2(DP_M4), DF2(DP_M5), DF2(DP_M6), DF2(DP_M7)}};

template <class G> struct DPCoef;
template <> struct DPCoef<double> {
    static __device__ __forceinline__ double a(int s, int j) { return c_dp.a[s][j]; }
    static __device__ __forceinline__ double e(int j) { return c_dp.e[j]; }
    static __device__ __forceinline__ double m(int j) { return c_dp.m[j]; }
};

template <class R>
struct RecordSink {
    R* pool;
    int32_t* chunks;         // [rays][kMaxChunks]
    unsigned long long pool_chunks;
    Counters* ctr;
};

// Arithmetic used by the geodesic integrator: native double, or df64 (double-float).
template <class G> struct GeoArith;
template <> struct GeoArith<double> {
    static __device__ __forceinline__ double from(double d) { return d; }
    static __device__ __forceinline__ double to(double g) { return g; }
    static __device__ __forceinline__ float tof(double g) { return (float)g; }
};
template <> struct GeoArith<float> {
    static __device__ __forceinline__ float from(double d) { return (float)d; }
    static __device__ __forceinline__ double to(float g) { return (double)g; }
    static __device__ __forceinline__ float tof(float g) { return g; }
};
template <> struct GeoArith<df64> {
    static __device__ __forceinline__ df64 from(double d) { return df64(d); }
    static __device__ __forceinline__ double to(const df64& g) { return df_to_double(g); }
    static __device__ __forceinline__ float tof(const df64& g) { return g.hi + g.lo; }
};

// Short sums of products in the integrator arithmetic: plain expressions in double, the
// compensated accumulator (one renormalisation per sum) in double-float.
__device__ __forceinline__ double g_fma(double a, double b, double c) { return a * b + c; }
__device__ __forceinline__ double g_dot2(double a, double b, double c, double d) { return a * b + c * d; }
__device__ __forceinline__ double g_dot3(double a, double b, double c, double d, double e,
                                         double f) { return a * b + c * d + e * f; }
__device__ __forceinline__ df64 g_fma(const df64& a, const df64& b, const df64& c) {
    DFDot s;
    s.first(a, b);
    s.add_term(c);
    return s.get();
}
__device__ __forceinline__ df64 g_dot2(const df64& a, const df64& b, const df64& c, const df64& d) {
    DFDot s;
    s.first(a, b);
    s.add(c, d);
    return s.get();
}
__device__ __forceinline__ df64 g_dot3(const df64& a, const df64& b, const df64& c, const df64& d,
                                       const df64& e, const df64& f) {
    DFDot s;
    s.first(a, b);
    s.add(c, d);
    s.add(e, f);
    return s.get();
}

// 1/x in the integrator arithmetic (no multiplication by an exact 1 in double-float).
__device__ __forceinline__ double g_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ df64 g_rcp(const df64& x) { return rcp(x); }

// A product inside a chain of products: unnormalised in double-float, plain in double.
__device__ __forceinline__ double g_mul_nn(double a, double b) { return a * b; }
__device__ __forceinline__ df64 g_mul_nn(const df64& a, const df64& b) { return df_mul_nn(a, b); }

// Exact scaling by a power of two in the integrator arithmetic.
__device__ __forceinline__ double scale2(double x, float f) { return x * (double)f; }
__device__ __forceinline__ df64 scale2(const df64& x, float f) { return df_scale(x, f); }

// Eq. (geodesic) right-hand side in arithmetic G; returns r at the evaluation point.
// With g^ab = eta^ab - f l^a l^b and L = l^a k_a, dx^a/dl = g^ab k_b and
// dk_c/dl = L (1/2 d_c f L + f d_c L), where d_c L is the derivative at fixed k. Instead of the
// nine derivatives d_c l_b (bl_math.cuh's form, kept for the transport matrices), d_c L is
// formed directly: with A = x k_x + y k_y and B = y k_x - x k_y, l_x k_x + l_y k_y =
// (r A + a B) / (r^2 + a^2) =: L_xy and l_z k_z = z k_z / r, so
//   d_c L = d_c r V + (r k_x - a k_y, r k_y + a k_x, k_z)_c / (r^2 + a^2 or r),
//   V = (A - 2 r L_xy) / (r^2 + a^2) - k_z z / r^2,
// and d_c f = F1 d_c r - [c = z] 2 a^2 z f / (r^4 + a^2 z^2), F1 = f (3 / r - 4 r^3 / (r^4 + a^2 z^2)).
// The same quantities as the nine-derivative form, in about 40 fewer operations.
template <class G>
__device__ __forceinline__ G geodesic_rhs_g(const G y[8], const G& a, const G& m, bool flat, G dy[8]) {
    constexpr G c0 = G(0), c3 = G(3);
    const G x = y[1], yy = y[2], z = y[3];
    const G kt = y[4], kx = y[5], ky = y[6], kz = y[7];
    // r (Eq. cks_aux:r), f and l as in ks_geom: two reciprocal square roots, one reciprocal
    const G aa = a * a;
    const G q = g_dot3(x, x, yy, yy, z, z) - aa;
    const G aaz2 = g_mul_nn(aa, z) * z;
    const G D2 = g_fma(q, q, scale2(aaz2, 4.0f));
    const G iD = rsqrt(D2);
    const G r2 = scale2(g_fma(D2, iD, q), 0.5f);
    const G ir = rsqrt(r2);
    const G r = r2 * ir;
    const G s4 = g_fma(r2, r2, aaz2);
    const G P = r2 + aa;
    const G iPs = g_rcp(P * s4);
    const G is4 = P * iPs;
    const G iP = s4 * iPs;
    const G f = flat ? c0 : g_mul_nn(g_mul_nn(scale2(m, 2.0f), r), r2) * is4;
    const G lx = g_dot2(r, x, a, yy) * iP, ly = g_dot2(r, yy, -a, x) * iP, lz = z * ir;
    // L = l^a k_a (l^t = -1)
    const G A_ = g_dot2(x, kx, yy, ky);
    const G B_ = g_dot2(yy, kx, -x, ky);
    const G Lxy = g_dot2(r, A_, a, B_) * iP;
    const G L = g_fma(lz, kz, Lxy - kt);
    const G fL = f * L;
    dy[0] = fL - kt;
    dy[1] = g_fma(-lx, fL, kx);
    dy[2] = g_fma(-ly, fL, ky);
    dy[3] = g_fma(-lz, fL, kz);
    dy[4] = c0;
    // d_c r
    const G riD = r * iD;
    const G drx = riD * x, dry = riD * yy, drz = g_mul_nn(g_mul_nn(z, P), ir) * iD;
    // d_c L at fixed k, and d_c f
    const G w = kz * ir;
    const G V = g_dot2(g_fma(-scale2(r, 2.0f), Lxy, A_), iP, -w, lz);
    const G Sx = g_dot2(drx, V, g_dot2(r, kx, -a, ky), iP);
    const G Sy = g_dot2(dry, V, g_dot2(r, ky, a, kx), iP);
    const G Sz = g_fma(drz, V, w);
    const G F1 = f * g_dot2(c3, ir, -(scale2(r2, 4.0f) * r), is4);
    const G dfx = F1 * drx, dfy = F1 * dry;
    const G dfz = g_fma(F1, drz, -(g_mul_nn(g_mul_nn(scale2(aa, 2.0f), z), f) * is4));
    const G halfL = scale2(L, 0.5f);
    dy[5] = L * g_dot2(dfx, halfL, f, Sx);
    dy[6] = L * g_dot2(dfy, halfL, f, Sy);
    dy[7] = L * g_dot2(dfz, halfL, f, Sz);
    return r;
}

template <> struct DPCoef<df64> {
    static __device__ __forceinline__ df64 a(int s, int j) { const float2 v = c_dpf.a[s][j]; return df64(v.x, v.y); }
    static __device__ __forceinline__ df64 e(int j) { const float2 v = c_dpf.e[j]; return df64(v.x, v.y); }
    static __device__ __forceinline__ df64 m(int j) { const float2 v = c_dpf.m[j]; return df64(v.x, v.y); }
};

// Accumulator of a sum of coefficient x stage-derivative products in the integrator
// arithmetic: the compensated double-float dot product, or plain (fused) double.
template <class G> struct StageDot;
template <> struct StageDot<double> {
    double s;
    __device__ __forceinline__ void first(double a, double x) { s = a * x; }
    __device__ __forceinline__ void add(double a, double x) { s = s + a * x; }
    __device__ __forceinline__ double get() const { return s; }
    __device__ __forceinline__ double axpy(double h, double y) const { return y + h * s; }
};
template <> struct StageDot<df64> {
    DFDot d;
    __device__ __forceinline__ void first(const df64& a, const df64& x) { d.first(a, x); }
    __device__ __forceinline__ void add(const df64& a, const df64& x) { d.add(a, x); }
    __device__ __forceinline__ df64 get() const { return d.get(); }
    __device__ __forceinline__ df64 axpy(const df64& h, const df64& y) const { return d.axpy(h, y); }
    __device__ __forceinline__ float value_f() const { return d.s + d.c; }
};


template <class R, class G>
__device__ __forceinline__ R to_rec(const G& v) {
    if constexpr (sizeof(R) == sizeof(float)) return (R)GeoArith<G>::tof(v);
    else return (R)GeoArith<G>::to(v);
}

// Append one record for `ray`; returns false when the store is full.
template <class R, class G>
__device__ __forceinline__ bool append_record(const RecordSink<R>& S, int64_t ray, int32_t& nrec,
                                              const G ys[8], const G yn[8], double dl) {
    const int32_t slot = nrec % kChunk;
    const int32_t ch = nrec / kChunk;
    if (ch >= kMaxChunks) return false;
    int32_t* tab = S.chunks + ray * kMaxChunks;
    if (slot == 0) {
        const unsigned long long c = warp_fetch_add(&S.ctr->pool_next);
        if (c >= S.pool_chunks) return false;
        tab[ch] = (int32_t)c;
    }
    const int64_t idx = (int64_t)tab[ch] * kChunk + slot;
    R* rec = S.pool + idx * RecStride<R>::v;
    // the record is assembled in registers and stored as 16-byte vectors (records are 64 B
    // (float) or 112 B (double) apart from a 256-byte aligned pool)
    const R v[14] = {to_rec<R>(ys[1]), to_rec<R>(ys[2]), to_rec<R>(ys[3]), to_rec<R>(ys[5]),
                     to_rec<R>(ys[6]), to_rec<R>(ys[7]), to_rec<R>(yn[1]), to_rec<R>(yn[2]),
                     to_rec<R>(yn[3]), to_rec<R>(yn[5]), to_rec<R>(yn[6]), to_rec<R>(yn[7]),
                     (R)dl, to_rec<R>(ys[0])};   // value 13: coordinate time (slow light)
    if constexpr (std::is_same<R, float>::value) {
        float4* q = reinterpret_cast<float4*>(rec);
        q[0] = make_float4(v[0], v[1], v[2], v[3]);
        q[1] = make_float4(v[4], v[5], v[6], v[7]);
        q[2] = make_float4(v[8], v[9], v[10], v[11]);
        q[3] = make_float4(v[12], v[13], 0.0f, 0.0f);
    } else {
        double2* q = reinterpret_cast<double2*>(rec);
#pragma unroll
        for (int i = 0; i < 7; ++i) q[i] = make_double2(v[2 * i], v[2 * i + 1]);
    }
    ++nrec;
    return true;
}

// Resident CTAs per SM the geodesic kernel is compiled for (the register budget follows:
// 65536 / (128 x this)).
#ifndef BL_GEO_MIN_CTAS
#define BL_GEO_MIN_CTAS 3
#endif
// Stage derivatives of a geodesic kernel: in dynamic shared memory, thread-fastest (the
// double-float and mixed forms), or a per-thread local array (the FP64 form, whose high
// occupancy leaves no shared memory for them).
template <class G, bool kSmem> struct KStore;
template <class G> struct KStore<G, true> {
    G* p;
    __device__ __forceinline__ G& at(int j, int s) { return p[(j * 7 + s) * 128]; }
};
template <class G> struct KStore<G, false> {
    G k[7][7];
    __device__ __forceinline__ G& at(int j, int s) { return k[j][s]; }
};
// Records of a subdivided step from the FP32 quartic about the step's start (coefficients
// y0, d0 = h f0, c2, c3, c4 per component): nsub samples at the centres of equal parts.
template <class R>
__device__ __forceinline__ bool emit_quartic_f(const RecordSink<R>& sink, int64_t wray, int32_t& nrec,
                                       const float y0f[8], const float d0f[8], const float c2f[8],
                                       const float c3f[8], const float c4f[8], int nsub,
                                       double hd) {
    bool ok = true;
    const float invf = 1.0f / (float)nsub;
    for (int s = 0; s < nsub && ok; ++s) {
        float ysm[8], ynd[8];
        const float ts = (s + 0.5f) * invf, tn = s * invf;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            ysm[c] = y0f[c] + ts * (d0f[c] + ts * (c2f[c] + ts * (c3f[c] + ts * c4f[c])));
            ynd[c] = (s == 0) ? y0f[c]
                              : y0f[c] + tn * (d0f[c] + tn * (c2f[c] + tn * (c3f[c] + tn * c4f[c])));
        }
        ok = append_record(sink, wray, nrec, ysm, ynd, hd / nsub);
    }
    return ok;
}

// eps^(-1/5) for the FP64 step control (factor 0.9 eps^-1/5, clamped to [0.2, 10] by the
// caller): a single-precision seed refined by two Newton steps for y^-5 = eps,
// y <- y (6 - eps y^5) / 5, each squaring the relative error (1e-6 -> 3e-12 -> rounding), in
// 12 FP64 operations instead of a double-precision pow. Arguments whose factor lies beyond
// the clamp return a value beyond it.
__device__ __forceinline__ double inv_fifth_root(double e) {
    if (e < 1e-6) return 1e3;
    if (e > 1e30) return 1e-3;
    double y = (double)__powf((float)e, -0.2f);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double y2 = y * y;
        const double y5 = y2 * y2 * y;
        y = (y * 0.2) * fma(-e, y5, 6.0);
    }
    return y;
}

template <class R, class G, bool kKsmem>
__device__ __forceinline__ void geodesic_body(const ImageDesc* __restrict__ imgs,
                                              int n_images, int64_t ray_begin, int64_t ray_end,
                                              RayHdr* __restrict__ hdr, RecordSink<R> sink,
                                              int record, BlockSource bs,
                                              const RayInit* __restrict__ init) {
    // rays [ray_begin, ray_end) of the batch form this wave; hdr, init and the chunk tables
    // are indexed by ray - ray_begin
    const int64_t re = wave_end(bs, ray_end);
    const int64_t total_rays = re > ray_begin ? re - ray_begin : 0;
    using A = GeoArith<G>;
    // compile-time constants in the integrator arithmetic (a run-time double -> df64 split
    // would cost FP64 conversions)
    constexpr G kDP_A21 = G(DP_A21);
    constexpr G kDP_A31 = G(DP_A31);
    constexpr G kDP_A32 = G(DP_A32);
    constexpr G kDP_A41 = G(DP_A41);
    constexpr G kDP_A42 = G(DP_A42);
    constexpr G kDP_A43 = G(DP_A43);
    constexpr G kDP_A51 = G(DP_A51);
    constexpr G kDP_A52 = G(DP_A52);
    constexpr G kDP_A53 = G(DP_A53);
    constexpr G kDP_A54 = G(DP_A54);
    constexpr G kDP_A61 = G(DP_A61);
    constexpr G kDP_A62 = G(DP_A62);
    constexpr G kDP_A63 = G(DP_A63);
    constexpr G kDP_A64 = G(DP_A64);
    constexpr G kDP_A65 = G(DP_A65);
    constexpr G kDP_B1 = G(DP_B1);
    constexpr G kDP_B3 = G(DP_B3);
    constexpr G kDP_B4 = G(DP_B4);
    constexpr G kDP_B5 = G(DP_B5);
    constexpr G kDP_B6 = G(DP_B6);
    constexpr G kDP_E1 = G(DP_E1);
    constexpr G kDP_E3 = G(DP_E3);
    constexpr G kDP_E4 = G(DP_E4);
    constexpr G kDP_E5 = G(DP_E5);
    constexpr G kDP_E6 = G(DP_E6);
    constexpr G kDP_E7 = G(DP_E7);
    constexpr G kDP_M1 = G(DP_M1);
    constexpr G kDP_M3 = G(DP_M3);
    constexpr G kDP_M4 = G(DP_M4);
    constexpr G kDP_M5 = G(DP_M5);
    constexpr G kDP_M6 = G(DP_M6);
    constexpr G kDP_M7 = G(DP_M7);
    constexpr G kHalf = G(0.5);
    constexpr G kM5 = G(-5.0);
    constexpr G k16 = G(16.0);
    constexpr G k14 = G(14.0);
    constexpr G kThree = G(3.0);
    constexpr G k32 = G(32.0);
    constexpr G kM8 = G(-8.0);
    constexpr G k2c = G(2.0);
    constexpr bool kNative = std::is_same<G, double>::value;
    Counters* ctr = sink.ctr;
    bool active = false;
    int64_t ray = 0;
    int q = 0, pi = 0, pj = 0;
    int64_t opix = 0;   // output index of the current ray
    int64_t wray = 0;   // index of the current ray within this wave
    G y[8];
    // K(0, c) = f(y); K(1..6, c) stage derivatives of the current attempt. In shared memory
    // (thread-fastest, conflict-free): 448 B a thread, which as a local array would take 172 KB
    // of L1 per SM and miss to L2.
    // The k_t component is constant along the ray (dk_t/dl = 0), so its derivatives are not
    // stored: 7 slots a stage, and KR(j, 4) reads as an exact zero.
#define KSLOT(c) ((c) < 4 ? (c) : (c) - 1)
    KStore<G, kKsmem> Ks;
    if constexpr (kKsmem) {
        extern __shared__ __align__(16) unsigned char geo_smem[];
        Ks.p = reinterpret_cast<G*>(geo_smem) + threadIdx.x;
    }
#define KX(j, c) Ks.at(j, KSLOT(c))
#define KR(j, c) ((c) == 4 ? G(0) : KX(j, c))
    G h = G(0);
    double nnorm = 0.0;
    bool been_inside = false, prev_rej = false;
    int64_t attempts = 0;
    int32_t nrec = 0, status = 0;
    double r_cam = 0.0, r_in = 0.0, ds_max = 0.0, r_grid = 0.0;
    G a = G(0), m = G(0);
    double tol_abs = 0.0, tol_rel = 0.0;
    int64_t max_steps = 0;
    bool flat = false;
    double r_cur = 0.0;     // r at y
    bool want_aux = false;  // auxiliary images: proper length and affine parameter
    double aux_len = 0.0, aux_lam = 0.0;
    int32_t last_in = -1;   // last record of a step reaching within 1.001 r_max

    bool exhausted = false;
    // All 32 lanes stay in the loop until the whole warp is out of work, so the warp
    // reconverges every iteration and the attempt is issued once for all lanes that hold a
    // ray (lanes without one are masked).
    while (true) {
        const bool need = !active && !exhausted;
        const unsigned long long got = warp_refill(&ctr->next_ray_geo, need);
        if (need) {
            if ((int64_t)got >= total_rays) {
                exhausted = true;
            } else {
                wray = (int64_t)got;
                ray = ray_begin + wray;
                active = true;
            }
        }
        if (!__any_sync(0xffffffffu, active)) break;
        if (!active) continue;
        if (need) {   // a ray taken from the queue in this iteration: set it up
            setup_ray(imgs, n_images, bs, ray, q, opix, pi, pj);
            const ImageDesc& im = imgs[q];
            // the pixel's initial state: in the double-float form from ray_init_kernel (its
            // FP64 set-up stays out of this loop), in the FP64-arithmetic forms computed here
            // (measured faster for them: mixed form 190 against 235 ms with the precomputed
            // states)
            if constexpr (kNative) {
                double yd[8];
                pixel_state(im, pi, pj, yd, nnorm);
#pragma unroll
                for (int c = 0; c < 8; ++c) y[c] = yd[c];
            } else {
                const RayInit& ri = init[wray];
#pragma unroll
                for (int c = 0; c < 8; ++c) y[c] = A::from(ri.y[c]);
                nnorm = ri.nnorm;
            }
            a = A::from(im.spin); m = A::from(im.mass); flat = im.flat != 0;
            r_cam = im.r_cam;
            r_in = im.r_in_over_rhor * im.r_hor;
            ds_max = im.ds_max;
            r_grid = im.r_max;
            tol_abs = im.tol_abs; tol_rel = im.tol_rel;
            max_steps = im.max_steps;
            want_aux = record && im.aux != nullptr;
            aux_len = aux_lam = 0.0;
            h = A::from(-im.h0_frac * (r_cam - im.r_hor));
            prev_rej = false;
        }
        // ---- one Dormand-Prince attempt (Table tab:dp) ----
        // Rolled stage loop: one right-hand-side body run six times keeps the kernel small
        // enough for the instruction cache. K(0) holds f(y) (first same as last), K(s) the
        // stage derivatives; stage 6 is evaluated at the fifth-order solution y5. A ray's first
        // attempt starts at stage 0, which evaluates f(y) at the stage point y, so that the
        // set-up path needs no copy of the right-hand side.
        G ys[8], y5[8];
        double r5 = 0.0;
#pragma unroll 1
        for (int st = need ? 0 : 1; st < 7; ++st) {
            if (st == 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) ys[c] = y[c];
            } else {
                // earlier stages outer (rolled), components inner: each coefficient is read
                // once per stage term; every component keeps its order of operations
                StageDot<G> acc[8];
                {
                    const G a0 = DPCoef<G>::a(st, 0);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c != 4) acc[c].first(a0, KX(0, c));
                }
                // the last row's second coefficient (b_2 of the fifth-order weights) is zero
#pragma unroll 1
                for (int j = st == 6 ? 2 : 1; j < st; ++j) {
                    const G aj = DPCoef<G>::a(st, j);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c != 4) acc[c].add(aj, KX(j, c));
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) ys[c] = (c == 4) ? y[4] : acc[c].axpy(h, y[c]);
            }
            G fs[8];
            const G rr = geodesic_rhs_g<G>(ys, a, m, flat, fs);
#pragma unroll
            for (int c = 0; c < 8; ++c) if (c != 4) KX(st, c) = fs[c];
            if (st == 0) {
                r_cur = A::to(rr);
                been_inside = r_cur < r_cam;
            }
            if (st == 6) {
                r5 = kNative ? A::to(rr) : (double)A::tof(rr);
#pragma unroll
                for (int c = 0; c < 8; ++c) y5[c] = ys[c];
            }
        }
        // Error norm eps = max_c |y5_c - y4_c| / (f_abs + f_rel max(|y_c|, |y5_c|)) with
        // y5 - y4 = h sum (b5 - b4) k. Native double keeps the FP64 form's arithmetic; the
        // df64 form takes the ratio in float (it only steers the step size).
        double eps;
        bool finite = true;
        {
            G errv[8];
            float errf[8];
            {
                StageDot<G> acc[8];
                {
                    const G e0 = DPCoef<G>::e(0);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c != 4) acc[c].first(e0, KX(0, c));
                }
#pragma unroll 1
                for (int j = 2; j < 7; ++j) {
                    const G ej = DPCoef<G>::e(j);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c != 4) acc[c].add(ej, KX(j, c));
                }
                if constexpr (kNative) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) errv[c] = (c == 4) ? G(0) : h * acc[c].get();
                } else {
                    // the double-float form uses the estimate in FP32 only: h_hi (s + c) there
                    const float hf = A::tof(h);
#pragma unroll
                    for (int c = 0; c < 8; ++c) errf[c] = (c == 4) ? 0.0f : hf * acc[c].value_f();
                }
            }
            if constexpr (kNative) {
                double num = 0.0, den = 1.0;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const double err = fabs(A::to(errv[c]));
                    const double sc = tol_abs + tol_rel * fmax(fabs(A::to(y[c])), fabs(A::to(y5[c])));
                    finite = finite && isfinite(err) && isfinite(A::to(y5[c]));
                    if (err * den > num * sc) { num = err; den = sc; }
                }
                eps = num / den;
            } else {
                float num = 0.0f, den = 1.0f;
                const float ta = (float)tol_abs, tr = (float)tol_rel;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const float err = fabsf(errf[c]);
                    const float sc = ta + tr * fmaxf(fabsf(A::tof(y[c])), fabsf(A::tof(y5[c])));
                    finite = finite && isfinite(err) && isfinite(A::tof(y5[c]));
                    if (err * den > num * sc) { num = err; den = sc; }
                }
                eps = (double)(num / den);
            }
        }
        ++attempts;
        bool done = false;
        if (!finite) {
            status = BL_RAY_NAN;
            done = true;
        } else if (eps <= 1.0) {
            // accepted: samples of this step (camera side first)
            if (record) {
                // FP32 records (fast and mixed forms): the midpoint's increment
                // (h/2) sum_j b_mid,j k_j and the quartic coefficients are formed in FP32 from the
                // state; they move a record by about one FP32 ulp and leave the integration and
                // its step decisions untouched. FP64 records (FP64 form): all in double.
                constexpr bool kFRec = sizeof(R) == sizeof(float);
                G ym[8];
                float ymf[8], incm[8];
                if constexpr (kFRec) {
                    const float hh = 0.5f * A::tof(h);
                    float acc[8];
                    {
                        const float m0 = c_dpf.m[0].x;
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[c] = m0 * A::tof(KR(0, c));
                    }
#pragma unroll 1
                    for (int j = 2; j < 7; ++j) {
                        const float mj = c_dpf.m[j].x;
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (c != 4) acc[c] = fmaf(mj, A::tof(KX(j, c)), acc[c]);
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        incm[c] = hh * acc[c];
                        if constexpr (!kNative) ymf[c] = y[c].hi + (y[c].lo + incm[c]);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        G acc = DPCoef<G>::m(0) * KR(0, c);
#pragma unroll 1
                        for (int j = 2; j < 7; ++j) acc = acc + DPCoef<G>::m(j) * KR(j, c);
                        ym[c] = y[c] + (kHalf * h) * acc;
                    }
                }
                const double r0 = r_cur, r1 = r5;
                const double hd = kNative ? A::to(h) : (double)A::tof(h);
                double rmid, kt_up, fmid;
                if constexpr (kNative) {
                    double ymd[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        if constexpr (kFRec) {
                            ymd[c] = A::to(y[c]) + (double)incm[c];
                            ymf[c] = (float)ymd[c];
                        } else {
                            ymd[c] = A::to(ym[c]);
                        }
                    }
                    KSGeom<double> Gm;
                    ks_geom<double>(ymd[1], ymd[2], ymd[3], im_spin(imgs, q), im_mass(imgs, q), flat, false, Gm);
                    const double L = -ymd[4] + Gm.l[1] * ymd[5] + Gm.l[2] * ymd[6] + Gm.l[3] * ymd[7];
                    kt_up = -ymd[4] + Gm.f * L;
                    rmid = Gm.r;
                    fmid = Gm.f;
                } else {
                    KSGeom<float> Gm;
                    ks_geom<float>(ymf[1], ymf[2], ymf[3], (float)im_spin(imgs, q), (float)im_mass(imgs, q),
                                   flat, false, Gm);
                    const float L = -ymf[4] + Gm.l[1] * ymf[5] + Gm.l[2] * ymf[6] + Gm.l[3] * ymf[7];
                    kt_up = -ymf[4] + Gm.f * L;
                    rmid = Gm.r;
                    fmid = Gm.f;
                }
                if (want_aux) {
                    aux_lam += fabs(hd);
                    aux_len += fabs(hd) * fabs(kt_up) / sqrt(1.0 + fmid);
                }
                const double rmin = fmin(rmid, fmin(r0, r1));
                int nsub = 1;
                if (rmin < r_grid) {
                    // ds/dl = (g_pq k^p k^q)^1/2 = alpha |k^t| for a null ray
                    if constexpr (kNative) {
                        const double ds = fabs(hd) * fabs(kt_up) / sqrt(1.0 + fmid);
                        if (ds > ds_max) {
                            const double nd = ceil(ds / ds_max);
                            nsub = nd > 4096.0 ? 4097 : (int)nd;
                        }
                    } else {
                        const float ds = fabsf((float)hd) * fabsf((float)kt_up) * rsqrtf(1.0f + (float)fmid);
                        if (ds > (float)ds_max) {
                            const float nd = ceilf(ds / (float)ds_max);
                            nsub = nd > 4096.0f ? 4097 : (int)nd;
                        }
                    }
                }
                bool ok = true;
                if (nsub == 1) {
                    if constexpr (kFRec) {
                        float yf[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c) yf[c] = A::tof(y[c]);
                        ok = append_record(sink, wray, nrec, ymf, yf, fabs(hd));
                    } else {
                        ok = append_record(sink, wray, nrec, ym, y, fabs(hd));
                    }
                } else if constexpr (kFRec) {
                    // float records: the quartic through y0, y1, h f0, h f1 and y_mid
                    // (Shampine 1986), in FP32 about y0 (y_mid - y0 is the midpoint increment)
                    const float hf = A::tof(h);
                    float y0f[8], d0f[8], c2f[8], c3f[8], c4f[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float d0 = hf * A::tof(KR(0, c));
                        const float D1 = A::tof(y5[c] - y[c]) - d0;
                        const float D2 = hf * A::tof(KR(6, c)) - d0;
                        const float D3 = incm[c] - 0.5f * d0;
                        y0f[c] = A::tof(y[c]);
                        d0f[c] = d0;
                        c2f[c] = -5.0f * D1 + D2 + 16.0f * D3;
                        c3f[c] = 14.0f * D1 - 3.0f * D2 - 32.0f * D3;
                        c4f[c] = -8.0f * D1 + 2.0f * D2 + 16.0f * D3;
                    }
                    ok = emit_quartic_f(sink, wray, nrec, y0f, d0f, c2f, c3f, c4f, nsub, fabs(hd));
                } else {
                    double y0d[8], d0[8], c2[8], c3[8], c4[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        y0d[c] = A::to(y[c]);
                        d0[c] = hd * A::to(KR(0, c));
                        const double D1 = A::to(y5[c]) - y0d[c] - d0[c];
                        const double D2 = hd * A::to(KR(6, c)) - d0[c];
                        const double D3 = A::to(ym[c]) - y0d[c] - 0.5 * d0[c];
                        c2[c] = -5.0 * D1 + D2 + 16.0 * D3;
                        c3[c] = 14.0 * D1 - 3.0 * D2 - 32.0 * D3;
                        c4[c] = -8.0 * D1 + 2.0 * D2 + 16.0 * D3;
                    }
                    const double inv = 1.0 / nsub;
                    for (int s = 0; s < nsub && ok; ++s) {
                        double ysm[8], ynd[8];
                        const double ts = (s + 0.5) * inv, tn = s * inv;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            ysm[c] = y0d[c] + ts * (d0[c] + ts * (c2[c] + ts * (c3[c] + ts * c4[c])));
                            ynd[c] = (s == 0) ? y0d[c]
                                              : y0d[c] + tn * (d0[c] + tn * (c2[c] + tn * (c3[c] + tn * c4[c])));
                        }
                        ok = append_record(sink, wray, nrec, ysm, ynd, fabs(hd) * inv);
                    }
                }
                if (!ok) { status = BL_RAY_OVERFLOW; done = true; }
                else if (kNative && rmin <= r_grid * 1.001) last_in = nrec - 1;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) { y[c] = y5[c]; if (c != 4) KX(0, c) = KX(6, c); }
            if constexpr (kNative) {
                double fac = (eps == 0.0) ? 10.0 : 0.9 * inv_fifth_root(eps);
                fac = fmin(10.0, fmax(0.2, fac));
                if (prev_rej) fac = fmin(fac, 1.0);
                h = h * A::from(fac);
            } else {
                const float ef = (float)eps;
                float fac = (ef == 0.0f) ? 10.0f : 0.9f * powf(ef, -0.2f);
                fac = fminf(10.0f, fmaxf(0.2f, fac));
                if (prev_rej) fac = fminf(fac, 1.0f);
                h = h * G(fac);
            }
            prev_rej = false;
            r_cur = r5;
            if (!done) {
                if (r_cur < r_in) { status = BL_RAY_HORIZON; done = true; }
                else if (been_inside && r_cur > r_cam) { status = BL_RAY_ESCAPED; done = true; }
                else if (r_cur < r_cam) been_inside = true;
            }
        } else {
            double fac;
            if constexpr (kNative) {
                fac = fmax(0.2, 0.9 * inv_fifth_root(eps));
                h = h * A::from(fac);
            } else {
                h = h * G(fmaxf(0.2f, 0.9f * powf((float)eps, -0.2f)));
            }
            prev_rej = true;
        }
        if (!done) {
            if ((kNative ? fabs(A::to(h)) : (double)fabsf(A::tof(h))) < 1e-12 * r_cur) {
                status = BL_RAY_UNDERFLOW;
                done = true;
            }
            else if (attempts >= max_steps) { status = BL_RAY_MAX_STEPS; done = true; }
        }
        if (done) {
            const ImageDesc& im = imgs[q];
            const int64_t pix = opix;
            if (im.status) im.status[pix] = status;
            if (im.steps) im.steps[pix] = (int32_t)(attempts < 2147483647 ? attempts : 2147483647);
            if (im.end_state)
                for (int c = 0; c < 8; ++c) im.end_state[pix * 8 + c] = A::to(y[c]);
            if (im.samples) im.samples[pix] = nrec;
            if (want_aux) {
                aux_store(im, 0, pix, -A::to(y[0]));
                aux_store(im, 1, pix, aux_len);
                aux_store(im, 2, pix, aux_lam);
            }
            RayHdr hd;
            hd.kt = A::to(y[4]);
            hd.nnorm = nnorm;
            hd.nrec = nrec;
            hd.status = status;
            // (the double-float kernel, issue bound at its register limit, does not track it:
            // 27.3 -> 29.9 ms when it did; its rays start from the far end)
            hd.last_in = kNative ? last_in : nrec - 1;
            hdr[wray] = hd;
            if (status != BL_RAY_HORIZON && status != BL_RAY_ESCAPED)
                atomicAdd(&ctr->bad_rays, 1ull);
            active = false;
            attempts = 0;
            nrec = 0;
            status = 0;
            last_in = -1;
        }
    }
}
#undef KX
#undef KR
#undef KSLOT

template <class R, class G>
__global__ void __launch_bounds__(128, BL_GEO_MIN_CTAS) geodesic_kernel(const ImageDesc* __restrict__ imgs,
                                                          int n_images, int64_t ray_begin,
                                                          int64_t ray_end,
                                                          RayHdr* __restrict__ hdr,
                                                          RecordSink<R> sink, int record,
                                                          BlockSource bs,
                                                          const RayInit* __restrict__ init) {
    geodesic_body<R, G, true>(imgs, n_images, ray_begin, ray_end, hdr, sink, record, bs, init);
}

// Resident CTAs per SM the FP64-form geodesic kernel is compiled for: 16 (32 registers, the
// SM's 64 warps; stage derivatives in local memory) measured 189.7 ms on the 9 x 256^2 step,
// against 199.6 ms at 3 CTAs with them in shared memory (4: 203.9; in local memory 4: 201.7,
// 6: 202.7, 8: 207.6). The mixed form (FP32 records, whose midpoints are formed in FP32)
// stays in the shared-memory kernel at 3 CTAs: 148.8 ms there against 160.5 ms in this one.
#ifndef BL_GEO64_MIN_CTAS
#define BL_GEO64_MIN_CTAS 16
#endif
// The FP64 form (FP64 state, FP64 records) with its own register budget.
__global__ void __launch_bounds__(128, BL_GEO64_MIN_CTAS) geodesic_kernel_fp64(
        const ImageDesc* __restrict__ imgs, int n_images, int64_t ray_begin, int64_t ray_end,
        RayHdr* __restrict__ hdr, RecordSink<double> sink, int record, BlockSource bs,
        const RayInit* __restrict__ init) {
    geodesic_body<double, double, false>(imgs, n_images, ray_begin, ray_end, hdr, sink, record, bs,
                                         init);
}

// Per-image constant in the transfer arithmetic.
template <class T>
__device__ __forceinline__ T ic(const ImageDesc& im, int k) {
    if constexpr (std::is_same<T, float>::value) return im.f_c[k];
    else return im.d_c[k];
}

// ---------------------------------------------------------------------------------------
// Plasma state at a sample (Secs. 2, 2.4, 2.5) in arithmetic T.
// ---------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------
// Fixed-rule geodesic integrators (Sec. 2.2): classical RK4 (Table tab:rk4) and Heun's RK2
// (Table tab:rk2) in FP64, step -f_step (r - r_hor) at the start of each step (Eq. rk_step).
// Each step's sample is its cubic Hermite midpoint (y0 + y1)/2 + h (f0 - f1)/8; a step longer
// than ds_max in proper length is subdivided by the same cubic. Persistent like
// geodesic_kernel, with the same records, outputs and termination rules.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void hermite(const double y0[8], const double y1[8], const double f0[8],
                                        const double f1[8], double h, double t, double out[8]) {
    const double t2 = t * t, t3 = t2 * t;
    const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2,
                 h11 = t3 - t2;
#pragma unroll
    for (int c = 0; c < 8; ++c) out[c] = h00 * y0[c] + h10 * h * f0[c] + h01 * y1[c] + h11 * h * f1[c];
}

template <class R>
__global__ void __launch_bounds__(128, 3) geodesic_rk_kernel(const ImageDesc* __restrict__ imgs,
                                                             int n_images, int64_t ray_begin,
                                                             int64_t ray_end,
                                                             RayHdr* __restrict__ hdr,
                                                             RecordSink<R> sink, int record,
                                                             BlockSource bs) {
    const int64_t re = wave_end(bs, ray_end);
    const int64_t total_rays = re > ray_begin ? re - ray_begin : 0;
    Counters* ctr = sink.ctr;
    bool active = false, exhausted = false;
    int64_t ray = 0, wray = 0, opix = 0;
    int q = 0, pi = 0, pj = 0;
    double y[8], f[8];
    double nnorm = 0.0, r_cur = 0.0, r_cam = 0.0, r_in = 0.0, r_hor = 0.0, ds_max = 0.0;
    double r_grid = 0.0, a = 0.0, m = 0.0, f_step = 0.0;
    int integ = 1;
    bool flat = false, been_inside = false, want_aux = false;
    int64_t nsteps = 0, max_steps = 0;
    int32_t nrec = 0, status = 0;
    double aux_len = 0.0, aux_lam = 0.0;
    while (true) {
        const bool need = !active && !exhausted;
        const unsigned long long got = warp_refill(&ctr->next_ray_geo, need);
        if (need) {
            if ((int64_t)got >= total_rays) exhausted = true;
            else { wray = (int64_t)got; ray = ray_begin + wray; active = true; }
        }
        if (!__any_sync(0xffffffffu, active)) break;
        if (!active) continue;
        if (need) {
            setup_ray(imgs, n_images, bs, ray, q, opix, pi, pj);
            const ImageDesc& im = imgs[q];
            pixel_state(im, pi, pj, y, nnorm);
            a = im.spin; m = im.mass; flat = im.flat != 0;
            r_cam = im.r_cam; r_hor = im.r_hor;
            r_in = im.r_in_over_rhor * im.r_hor;
            ds_max = im.ds_max; r_grid = im.r_max;
            f_step = im.f_step; integ = im.integrator;
            max_steps = im.max_steps;
            want_aux = record && im.aux != nullptr;
            aux_len = aux_lam = 0.0;
            r_cur = geodesic_rhs(y, a, m, flat, f);
            been_inside = r_cur < r_cam;
            nsteps = 0; nrec = 0; status = BL_RAY_OK;
        }
        // one step
        const double h = -f_step * (r_cur - r_hor);
        double y1[8], ys[8], k2[8];
        if (integ == 1) {
            double k3[8], k4[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) ys[c] = y[c] + 0.5 * h * f[c];
            geodesic_rhs(ys, a, m, flat, k2);
#pragma unroll
            for (int c = 0; c < 8; ++c) ys[c] = y[c] + 0.5 * h * k2[c];
            geodesic_rhs(ys, a, m, flat, k3);
#pragma unroll
            for (int c = 0; c < 8; ++c) ys[c] = y[c] + h * k3[c];
            geodesic_rhs(ys, a, m, flat, k4);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                y1[c] = y[c] + h * (f[c] / 6.0 + k2[c] / 3.0 + k3[c] / 3.0 + k4[c] / 6.0);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) ys[c] = y[c] + h * f[c];
            geodesic_rhs(ys, a, m, flat, k2);
#pragma unroll
            for (int c = 0; c < 8; ++c) y1[c] = y[c] + h * (0.5 * f[c] + 0.5 * k2[c]);
        }
        ++nsteps;
        bool finite = true;
#pragma unroll
        for (int c = 0; c < 8; ++c) finite = finite && isfinite(y1[c]);
        bool done = false;
        if (!finite) {
            status = BL_RAY_NAN;
            done = true;
        } else {
            double f1[8];
            const double r1 = geodesic_rhs(y1, a, m, flat, f1);
            if (record) {
                double ym[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) ym[c] = 0.5 * (y[c] + y1[c]) + 0.125 * h * (f[c] - f1[c]);
                KSGeom<double> Gm;
                ks_geom<double>(ym[1], ym[2], ym[3], a, m, flat, false, Gm);
                const double L = -ym[4] + Gm.l[1] * ym[5] + Gm.l[2] * ym[6] + Gm.l[3] * ym[7];
                const double kt_up = -ym[4] + Gm.f * L;
                const double ds = fabs(h) * fabs(kt_up) / sqrt(1.0 + Gm.f);
                if (want_aux) { aux_lam += fabs(h); aux_len += ds; }
                int nsub = 1;
                if (fmin(Gm.r, fmin(r_cur, r1)) < r_grid && ds > ds_max) {
                    const double nd = ceil(ds / ds_max);
                    nsub = nd > 4096.0 ? 4097 : (int)nd;
                }
                bool ok = true;
                if (nsub == 1) {
                    ok = append_record(sink, wray, nrec, ym, y, fabs(h));
                } else {
                    const double inv = 1.0 / nsub;
                    for (int sb = 0; sb < nsub && ok; ++sb) {
                        double ysm[8], ynd[8];
                        hermite(y, y1, f, f1, h, (sb + 0.5) * inv, ysm);
                        if (sb == 0) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) ynd[c] = y[c];
                        } else {
                            hermite(y, y1, f, f1, h, sb * inv, ynd);
                        }
                        ok = append_record(sink, wray, nrec, ysm, ynd, fabs(h) * inv);
                    }
                }
                if (!ok) { status = BL_RAY_OVERFLOW; done = true; }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) { y[c] = y1[c]; f[c] = f1[c]; }
            r_cur = r1;
            if (!done) {
                if (r_cur < r_in) { status = BL_RAY_HORIZON; done = true; }
                else if (been_inside && r_cur > r_cam) { status = BL_RAY_ESCAPED; done = true; }
                else {
                    if (r_cur < r_cam) been_inside = true;
                    if (fabs(f_step * (r_cur - r_hor)) < 1e-12 * r_cur) { status = BL_RAY_UNDERFLOW; done = true; }
                    else if (nsteps >= max_steps) { status = BL_RAY_MAX_STEPS; done = true; }
                }
            }
        }
        if (done) {
            const ImageDesc& im = imgs[q];
            const int64_t pix = opix;
            if (im.status) im.status[pix] = status;
            if (im.steps) im.steps[pix] = (int32_t)(nsteps < 2147483647 ? nsteps : 2147483647);
            if (im.end_state)
                for (int c = 0; c < 8; ++c) im.end_state[pix * 8 + c] = y[c];
            if (im.samples) im.samples[pix] = nrec;
            if (want_aux) {
                aux_store(im, 0, pix, -y[0]);
                aux_store(im, 1, pix, aux_len);
                aux_store(im, 2, pix, aux_lam);
            }
            RayHdr hd;
            hd.kt = y[4];
            hd.nnorm = nnorm;
            hd.nrec = nrec;
            hd.status = status;
            hd.last_in = nrec - 1;   // (fixed-step integrators: no skip)
            hdr[wray] = hd;
            if (status != BL_RAY_HORIZON && status != BL_RAY_ESCAPED)
                atomicAdd(&ctr->bad_rays, 1ull);
            active = false;
        }
    }
}

template <class T>
struct Plasma {
    T u[4], b[4];         // contravariant CKS
    T ul[4];              // covariant u
    T ne, th, bg, bsq;
    T rho, p, binv;       // code-unit density and pressure, b^2 / (2 p)
};

// The 8 primitives of cell `cell` of a grid in the cell layout ([...][8], 32 bytes a cell,
// 16-byte aligned): two read-only 16-byte loads.
__device__ __forceinline__ void load_cell(const float* __restrict__ base, size_t cell, float c[8]) {
    const float4* p = reinterpret_cast<const float4*>(base) + 2 * cell;
    const float4 a = __ldg(p), b = __ldg(p + 1);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}

// Plane layout [s][8][cells] -> cell layout [s][cells][8]; one thread per cell, reads
// coalesced per plane, writes two 16-byte vectors.
__global__ void grid_pack_kernel(const float* __restrict__ planes, float* __restrict__ cells,
                                 int64_t cells_per_snap, int64_t n_cells) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += stride) {
        const int64_t s = c / cells_per_snap, x = c - s * cells_per_snap;
        const float* src = planes + s * 8 * cells_per_snap + x;
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldg(src + k * cells_per_snap);
        float4* dst = reinterpret_cast<float4*>(cells) + 2 * c;
        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

// A grid value (float) in the sampling arithmetic T. float -> double is exact; it is done
// with integer operations on the bit pattern instead of a conversion instruction, which on
// this hardware shares the scarce FP64 pipe with the arithmetic (a trilinear sample converts
// 64 values): the exponent is rebiased (127 -> 1023, all ones kept for inf and NaN) and the
// significand widened; zeros keep their sign; subnormal floats (exponent field 0, nonzero)
// take the conversion instruction.
template <class T>
__device__ __forceinline__ T grid_val(float f) {
    if constexpr (sizeof(T) == 4) {
        return f;
    } else {
        const uint32_t b = __float_as_uint(f);
        const uint32_t e = b & 0x7f800000u, sgn = b & 0x80000000u;
        if (e == 0u && (b & 0x7fffffffu) != 0u) return (double)f;
        uint32_t hi = sgn | (((b & 0x7fffffffu) >> 3) + 0x38000000u);
        if (e == 0x7f800000u) hi += 0x38000000u;
        const uint32_t lo = b << 29;
        return e == 0u ? __hiloint2double((int)sgn, 0) : __hiloint2double((int)hi, (int)lo);
    }
}

// x is neither NaN nor infinite (exponent field not all ones)
__device__ __forceinline__ bool finite_bits(float x) {
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// Fused multiply-add in T, written out: the grid sums below fix their rounding in the source
// (a sum of two products may otherwise be fused either way), so that both grid layouts and
// every kernel variant produce the same bits.
__device__ __forceinline__ float t_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double t_fma(double a, double b, double c) { return fma(a, b, c); }

// The bit patterns of a cell's three magnetic-field components OR-ed together (values 5..7:
// B^r, B^theta, B^phi); with the sign bit cleared it is zero exactly when the field is +-0.
__device__ __forceinline__ unsigned int cell_field_bits(const float* __restrict__ prim, int layout,
                                                        size_t plane, size_t cell) {
    if (layout == 1) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(prim) + 2 * cell + 1);
        return __float_as_uint(v.y) | __float_as_uint(v.z) | __float_as_uint(v.w);
    }
    return __float_as_uint(__ldg(prim + 5 * plane + cell)) |
           __float_as_uint(__ldg(prim + 6 * plane + cell)) |
           __float_as_uint(__ldg(prim + 7 * plane + cell));
}

// field_test: first read the stencil's magnetic field alone and return false (no plasma) when
// every corner's field is zero -- exact (b = 0 fails the b^2 > 0 test below), and it skips the
// interpolation and the plasma state at such samples.
template <class T, bool kSlow = false>
__device__ __forceinline__ bool plasma_at(const ImageDesc& im, const T x[3], T t,
                                          const KSGeom<T>& G, Plasma<T>& P, bool field_test) {
    const T a = ic<T>(im, kcSpin);
    const T r = G.r;
    if (!(r >= ic<T>(im, kcRmin) && r <= ic<T>(im, kcRmax))) return false;
    T cth = fq(x[2], r);
    cth = cth > T(1) ? T(1) : (cth < T(-1) ? T(-1) : cth);
    const T th = acos(cth);
    const T sth = fsqrt(T(1) - cth * cth);
    const T twopi = T(2.0 * kPi);
    // phi = arg(x + i y) - arg(r + i a) = arg((x + i y)(r - i a)), in (-pi, pi]; one wrap
    // puts it in [0, 2 pi) (fmod by 2 pi would return such a value unchanged). Its sine and
    // cosine are that complex number normalised (on the axis, where it vanishes, phi = 0).
    const T zre = x[0] * r + x[1] * a, zim = x[1] * r - x[0] * a;
    T ph = atan2(zim, zre);
    if (ph < T(0)) ph += twopi;
    if (ph >= twopi) ph -= twopi;
    const int nr = im.nr, nt = im.nt, np = im.nph;
    const size_t plane = (size_t)np * nt * nr;
    // slow light: the two snapshots around the sample's time and the weight of the second
    const float* __restrict__ prim = im.prim;
    const float* __restrict__ prim1 = nullptr;
    T wt1 = T(0);
    if (kSlow && im.n_snap > 1) {
        const int ns = im.n_snap;
        T fs = (t - (T)im.t_rel0) / (T)im.dt_snap;
        fs = fs < T(0) ? T(0) : (fs > T(ns - 1) ? T(ns - 1) : fs);
        int s0;
        if (im.time_interp == 0) {
            s0 = (int)floor(fs + T(0.5));
        } else {
            s0 = (int)floor(fs);
            if (s0 > ns - 2) s0 = ns - 2;
            wt1 = fs - T(s0);
            prim1 = prim + (size_t)(s0 + 1) * 8 * plane;
        }
        prim += (size_t)s0 * 8 * plane;
    }
    T pv[8];
    // fractional cell coordinates: (ln r - ln r_min) / dlr, theta / (pi / n_theta),
    // phi / (2 pi / n_phi), each as a product with the precomputed reciprocal cell size
    const T idlr = ic<T>(im, kcIDlr);
    const T lrmin = ic<T>(im, kcLogRmin);
    const T idth = T(nt) * T(1.0 / kPi);
    const T idph = T(np) * T(0.5 / kPi);
    if (im.interp == 0) {
        int i = (int)floor((flog(r) - lrmin) * idlr);
        int j = (int)floor(th * idth);
        int k = (int)floor(ph * idph);
        i = min(max(i, 0), nr - 1);
        j = min(max(j, 0), nt - 1);
        k = ((k % np) + np) % np;
        const size_t base = ((size_t)k * nt + j) * nr + i;
        // a cell without magnetic field holds no plasma (b = 0, below): its field
        // components alone decide that
        if (field_test) {
            unsigned int fb = cell_field_bits(prim, im.layout, plane, base);
            if (kSlow && prim1) fb |= cell_field_bits(prim1, im.layout, plane, base);
            if ((fb & 0x7fffffffu) == 0u) return false;
        }
        if (im.layout == 1) {
            float c[8];
            load_cell(prim, base, c);
#pragma unroll
            for (int v = 0; v < 8; ++v) pv[v] = grid_val<T>(c[v]);
            if (kSlow && prim1) {
                load_cell(prim1, base, c);
#pragma unroll
                for (int v = 0; v < 8; ++v) pv[v] = t_fma(wt1, grid_val<T>(c[v]), (T(1) - wt1) * pv[v]);
            }
        } else {
#pragma unroll
            for (int v = 0; v < 8; ++v) pv[v] = grid_val<T>(__ldg(prim + v * plane + base));
            if (kSlow && prim1) {
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    pv[v] = t_fma(wt1, grid_val<T>(__ldg(prim1 + v * plane + base)), (T(1) - wt1) * pv[v]);
            }
        }
    } else {
        int i0, j0;
        T wr, wt;
        {
            T fi = (flog(r) - lrmin) * idlr - T(0.5);
            if (nr == 1) { i0 = 0; wr = T(0); }
            else {
                fi = fi < T(0) ? T(0) : (fi > T(nr - 1) ? T(nr - 1) : fi);
                i0 = (int)floor(fi);
                if (i0 > nr - 2) i0 = nr - 2;
                wr = fi - T(i0);
            }
        }
        {
            T fj = th * idth - T(0.5);
            if (nt == 1) { j0 = 0; wt = T(0); }
            else {
                fj = fj < T(0) ? T(0) : (fj > T(nt - 1) ? T(nt - 1) : fj);
                j0 = (int)floor(fj);
                if (j0 > nt - 2) j0 = nt - 2;
                wt = fj - T(j0);
            }
        }
        const int i1 = nr == 1 ? 0 : i0 + 1, j1 = nt == 1 ? 0 : j0 + 1;
        const T fk = ph * idph - T(0.5);
        const T fkf = floor(fk);
        const int k0 = (((int)fkf) % np + np) % np;
        const int k1 = (k0 + 1) % np;
        const T wp = fk - fkf;
        const size_t o00 = ((size_t)k0 * nt + j0) * nr, o01 = ((size_t)k0 * nt + j1) * nr;
        const size_t o10 = ((size_t)k1 * nt + j0) * nr, o11 = ((size_t)k1 * nt + j1) * nr;
        // a stencil whose eight cells carry no magnetic field holds no plasma (b = 0, below):
        // the field components alone decide that, before the interpolation
        if (field_test) {
            const size_t cell[8] = {o00 + i0, o00 + i1, o01 + i0, o01 + i1,
                                    o10 + i0, o10 + i1, o11 + i0, o11 + i1};
            unsigned int fb = 0u;
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                fb |= cell_field_bits(prim, im.layout, plane, cell[n]);
                if (kSlow && prim1) fb |= cell_field_bits(prim1, im.layout, plane, cell[n]);
            }
            if ((fb & 0x7fffffffu) == 0u) return false;
        }
        const T w000 = (T(1) - wp) * (T(1) - wt) * (T(1) - wr), w001 = (T(1) - wp) * (T(1) - wt) * wr;
        const T w010 = (T(1) - wp) * wt * (T(1) - wr), w011 = (T(1) - wp) * wt * wr;
        const T w100 = wp * (T(1) - wt) * (T(1) - wr), w101 = wp * (T(1) - wt) * wr;
        const T w110 = wp * wt * (T(1) - wr), w111 = wp * wt * wr;
        if (im.layout == 1) {
            // cell layout: the 8 corners as 16 vector loads, summed in the plane form's order
            auto tri8 = [&](const float* __restrict__ pp, T out[8]) {
                const size_t cell[8] = {o00 + i0, o00 + i1, o01 + i0, o01 + i1,
                                        o10 + i0, o10 + i1, o11 + i0, o11 + i1};
                const T w[8] = {w000, w001, w010, w011, w100, w101, w110, w111};
                float c[8];
                load_cell(pp, cell[0], c);
#pragma unroll
                for (int v = 0; v < 8; ++v) out[v] = w[0] * grid_val<T>(c[v]);
#pragma unroll
                for (int n = 1; n < 8; ++n) {
                    load_cell(pp, cell[n], c);
#pragma unroll
                    for (int v = 0; v < 8; ++v) out[v] = t_fma(w[n], grid_val<T>(c[v]), out[v]);
                }
            };
            tri8(prim, pv);
            if (kSlow && prim1) {
                T pv1[8];
                tri8(prim1, pv1);
#pragma unroll
                for (int v = 0; v < 8; ++v) pv[v] = t_fma(wt1, pv1[v], (T(1) - wt1) * pv[v]);
            }
        } else {
            // accumulated one corner at a time with explicit fused multiply-adds, as the cell
            // layout does: both layouts round alike
            auto tri = [&](const float* __restrict__ pp) -> T {
                T acc = w000 * grid_val<T>(__ldg(pp + o00 + i0));
                acc = t_fma(w001, grid_val<T>(__ldg(pp + o00 + i1)), acc);
                acc = t_fma(w010, grid_val<T>(__ldg(pp + o01 + i0)), acc);
                acc = t_fma(w011, grid_val<T>(__ldg(pp + o01 + i1)), acc);
                acc = t_fma(w100, grid_val<T>(__ldg(pp + o10 + i0)), acc);
                acc = t_fma(w101, grid_val<T>(__ldg(pp + o10 + i1)), acc);
                acc = t_fma(w110, grid_val<T>(__ldg(pp + o11 + i0)), acc);
                return t_fma(w111, grid_val<T>(__ldg(pp + o11 + i1)), acc);
            };
#pragma unroll
            for (int v = 0; v < 8; ++v) pv[v] = tri(prim + v * plane);
            if (kSlow && prim1) {
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    pv[v] = t_fma(wt1, tri(prim1 + v * plane), (T(1) - wt1) * pv[v]);
            }
        }
    }
    // non-finite data (a NaN or infinite primitive at any corner of the stencil) carry no
    // plasma; the test reads the exponent bits (integer operations)
    {
        bool fin = true;
#pragma unroll
        for (int v = 0; v < 8; ++v) fin = fin && finite_bits(pv[v]);
        if (!fin) return false;
    }
    // spherical -> Cartesian KS vectors (Jacobian columns d x^a / d(r, theta, phi))
    T sph = T(0), cph = T(1);
    {
        const T zz = zre * zre + zim * zim;
        if (zz > T(0)) {
            const T iz = rsqrt(zz);
            cph = zre * iz;
            sph = zim * iz;
        }
    }
    const T J[3][3] = {{sth * cph, cth * (r * cph - a * sph), sth * (-r * sph - a * cph)},
                       {sth * sph, cth * (r * sph + a * cph), sth * (r * cph - a * sph)},
                       {cth, -r * sth, T(0)}};
    T v[3], B[3];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        v[c] = J[c][0] * pv[2] + J[c][1] * pv[3] + J[c][2] * pv[4];
        B[c] = J[c][0] * pv[5] + J[c][1] * pv[6] + J[c][2] * pv[7];
    }
    v[2] = J[2][0] * pv[2] + J[2][1] * pv[3];   // J[2][2] = d z / d phi = 0
    B[2] = J[2][0] * pv[5] + J[2][1] * pv[6];
    const T f = G.f;
    const T lv = G.l[1] * v[0] + G.l[2] * v[1] + G.l[3] * v[2];
    const T un = fsqrt(T(1) + v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + f * lv * lv);
    P.u[0] = un * fsqrt(T(1) + f);
    const T sh = fq(f, T(1) + f) * P.u[0];
#pragma unroll
    for (int c = 0; c < 3; ++c) P.u[c + 1] = v[c] - G.l[c + 1] * sh;
    lower4(G, P.u, P.ul);
    P.b[0] = B[0] * P.ul[1] + B[1] * P.ul[2] + B[2] * P.ul[3];
    const T iut = fq(T(1), P.u[0]);
#pragma unroll
    for (int c = 0; c < 3; ++c) P.b[c + 1] = (B[c] + P.b[0] * P.u[c + 1]) * iut;
    P.bsq = dot4(G, P.b, P.b);
    const T rho = pv[0];
    const T p = ic<T>(im, kcGam1) * pv[1];
    if (!(rho > T(0)) || !(p > T(0)) || !(P.bsq > T(0))) return false;
    if (fq(P.bsq, rho) > ic<T>(im, kcSigma)) return false;
    const T binv = fq(P.bsq, T(2) * p);
    const T b2 = binv * binv;
    const T ratio = fq(ic<T>(im, kcRhigh) + b2 * ic<T>(im, kcRlow), T(1) + b2);
    const T rr = ic<T>(im, kcNeNi);
    const T th_e = fq(ic<T>(im, kcTePre) * fq(p, rho) * (rr + T(1)), rr + ratio);
    P.th = th_e;
    P.ne = rho * ic<T>(im, kcNeFac);
    P.bg = fsqrt(P.bsq) * ic<T>(im, kcBgPre);
    P.rho = rho;
    P.p = p;
    P.binv = binv;
    return true;
}

// Fluid-frame basis: e3 along the photon's spatial direction, e2 along the field projected
// perpendicular to e3, e1^a = [abcd] u_b e2_c e3_d (sqrt(-g) = 1 in Cartesian KS).
template <class T>
__device__ __forceinline__ void fluid_basis(const KSGeom<T>& G, const Plasma<T>& P, const T kl[4],
                                            const T ku[4], T e1[4], T e2[4], T e1l[4], T e2l[4]) {
    const T kdu = kl[0] * P.u[0] + kl[1] * P.u[1] + kl[2] * P.u[2] + kl[3] * P.u[3];
    const T iw = fq(T(-1), kdu);
    T e3[4], e3l[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { e3[c] = (ku[c] + kdu * P.u[c]) * iw; e3l[c] = (kl[c] + kdu * P.ul[c]) * iw; }
    const T bu = P.b[0] * P.ul[0] + P.b[1] * P.ul[1] + P.b[2] * P.ul[2] + P.b[3] * P.ul[3];
    T bp[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) bp[c] = P.b[c] + bu * P.u[c];
    T b3 = bp[0] * e3l[0] + bp[1] * e3l[1] + bp[2] * e3l[2] + bp[3] * e3l[3];
#pragma unroll
    for (int c = 0; c < 4; ++c) bp[c] -= b3 * e3[c];
    T bpl[4];
    lower4(G, bp, bpl);
    T bb = bp[0] * bpl[0] + bp[1] * bpl[1] + bp[2] * bpl[2] + bp[3] * bpl[3];
    const T tiny = sizeof(T) == 8 ? T(1e-20) : T(1e-10);
    if (!(bb > tiny * P.bsq)) {
        // field along the ray: any transverse direction (only I and V couple there)
        for (int t = 0; t < 2; ++t) {
            T tv[4] = {T(0), T(0), T(0), T(0)};
            tv[t == 0 ? 3 : 1] = T(1);
            T tl[4];
            lower4(G, tv, tl);
            const T pu = tl[0] * P.u[0] + tl[1] * P.u[1] + tl[2] * P.u[2] + tl[3] * P.u[3];
#pragma unroll
            for (int c = 0; c < 4; ++c) bp[c] = tv[c] + pu * P.u[c];
            b3 = bp[0] * e3l[0] + bp[1] * e3l[1] + bp[2] * e3l[2] + bp[3] * e3l[3];
#pragma unroll
            for (int c = 0; c < 4; ++c) bp[c] -= b3 * e3[c];
            lower4(G, bp, bpl);
            bb = bp[0] * bpl[0] + bp[1] * bpl[1] + bp[2] * bpl[2] + bp[3] * bpl[3];
            if (bb > T(1e-6)) break;
        }
    }
    const T ib = rsqrt(bb);
#pragma unroll
    for (int c = 0; c < 4; ++c) { e2[c] = bp[c] * ib; e2l[c] = bpl[c] * ib; }
    // e1^a = (-1)^a det(minor_a) of the rows (u_l, e2_l, e3_l)
    const T* A0 = P.ul;
    const T* A1 = e2l;
    const T* A2 = e3l;
    auto det3c = [&](int c0, int c1, int c2) -> T {
        return A0[c0] * (A1[c1] * A2[c2] - A1[c2] * A2[c1]) - A0[c1] * (A1[c0] * A2[c2] - A1[c2] * A2[c0]) +
               A0[c2] * (A1[c0] * A2[c1] - A1[c1] * A2[c0]);
    };
    e1[0] = det3c(1, 2, 3);
    e1[1] = -det3c(0, 2, 3);
    e1[2] = det3c(0, 1, 3);
    e1[3] = -det3c(0, 1, 2);
    lower4(G, e1, e1l);
}

// Stokes from the coherency tensor in the basis (e1, e2): N11 = (I+Q)/2, N22 = (I-Q)/2,
// N12 = (U + iV)/2.
template <class T>
__device__ __forceinline__ void coh_to_stokes(const Coh<T>& n, const T e1l[4], const T e2l[4], T s[4]) {
    // n11 = e1 R e1, n22 = e2 R e2, n12 = e1 (R + i I) e2, through R e1, R e2 and I e2
    T R[4][4], I[4][4];
    coh_unpack(n, R, I);
    T v1[4], v2[4], w2[4];
#pragma unroll
    for (int a_ = 0; a_ < 4; ++a_) {
        T x1 = T(0), x2 = T(0), xi = T(0);
#pragma unroll
        for (int b_ = 0; b_ < 4; ++b_) {
            x1 += R[a_][b_] * e1l[b_];
            x2 += R[a_][b_] * e2l[b_];
            if (b_ != a_) xi += I[a_][b_] * e2l[b_];
        }
        v1[a_] = x1; v2[a_] = x2; w2[a_] = xi;
    }
    T n11 = T(0), n22 = T(0), n12r = T(0), n12i = T(0);
#pragma unroll
    for (int a_ = 0; a_ < 4; ++a_) {
        n11 += e1l[a_] * v1[a_];
        n22 += e2l[a_] * v2[a_];
        n12r += e1l[a_] * v2[a_];
        n12i += e1l[a_] * w2[a_];
    }
    s[0] = n11 + n22;
    s[1] = n11 - n22;
    s[2] = T(2) * n12r;
    s[3] = T(2) * n12i;
}

template <class T>
__device__ __forceinline__ void stokes_to_coh(const T e1[4], const T e2[4], const T s[4], Coh<T>& n) {
    // N = p e1 e1 + q e2 e2 + u (e1 e2 + e2 e1) + i v (e1 e2 - e2 e1), with the vectors
    // scaled once
    const T p = T(0.5) * (s[0] + s[1]), qv = T(0.5) * (s[0] - s[1]), uu = T(0.5) * s[2], vv = T(0.5) * s[3];
    T pe1[4], qe2[4], ue1[4], ue2[4], ve1[4];
#pragma unroll
    for (int a_ = 0; a_ < 4; ++a_) {
        pe1[a_] = p * e1[a_]; qe2[a_] = qv * e2[a_]; ue1[a_] = uu * e1[a_]; ue2[a_] = uu * e2[a_];
        ve1[a_] = vv * e1[a_];
    }
    int k = 0;
#pragma unroll
    for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
        for (int b_ = a_; b_ < 4; ++b_)
            n.re[k++] = pe1[a_] * e1[b_] + qe2[a_] * e2[b_] + ue1[a_] * e2[b_] + ue2[a_] * e1[b_];
    k = 0;
#pragma unroll
    for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
        for (int b_ = a_ + 1; b_ < 4; ++b_) n.im[k++] = ve1[a_] * e2[b_] - ve1[b_] * e2[a_];
}

// One sample record as 16-byte vector loads (records are 16-byte aligned).
template <class R>
__device__ __forceinline__ void load_record(const R* __restrict__ rec, R out[RecStride<R>::v]) {
    if constexpr (std::is_same<R, float>::value) {
        const float4* p = reinterpret_cast<const float4*>(rec);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 v = __ldg(p + i);
            out[4 * i] = v.x; out[4 * i + 1] = v.y; out[4 * i + 2] = v.z; out[4 * i + 3] = v.w;
        }
    } else {
        const double2* p = reinterpret_cast<const double2*>(rec);
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const double2 v = __ldg(p + i);
            out[2 * i] = v.x; out[2 * i + 1] = v.y;
        }
    }
}

template <class R>
__device__ __forceinline__ const R* record_ptr(const R* __restrict__ pool, const int32_t* __restrict__ chunks,
                                               int64_t ray, int32_t idx) {
    const int32_t ch = chunks[ray * kMaxChunks + idx / kChunk];
    return pool + ((int64_t)ch * kChunk + (idx % kChunk)) * RecStride<R>::v;
}
// Position of record idx of a ray in the pool (records counted from the pool's start).
__device__ __forceinline__ int64_t record_index(const int32_t* __restrict__ chunks, int64_t ray,
                                                int32_t idx) {
    return (int64_t)chunks[ray * kMaxChunks + idx / kChunk] * kChunk + (idx % kChunk);
}

// ---------------------------------------------------------------------------------------
// Persistent transfer kernel (Sec. 2.3.2). Each lane replays one ray's samples from the
// source end to the camera, one sample per loop iteration: merged N half-steps by the
// predictor-corrector (stage 1 at the previous sample, stage 2 at the node it shares with
// the current one), then, where the sample carries plasma, N -> S in the fluid frame, the
// exact constant-coefficient Stokes step, and S -> N. A lane whose ray is done reads out the
// Stokes parameters in the camera basis (H, V) and takes the next ray.
// ---------------------------------------------------------------------------------------
// Features of a transfer-kernel variant (compile-time, so that each variant carries only the
// registers it needs).
enum { kFSlow = 1, kFUnpol = 2, kFAux = 4, kFMlp = 8 };

// Auxiliary accumulators of one ray (Sec. 4, "Auxiliary Images"): I_j, tau and the lambda-,
// emission- and tau-weighted sums of rho, n_e, p, Theta_e, B, sigma, beta^-1.
template <class T>
struct AuxAcc {
    T ij, tau, ql[7], qi[7], qt[7];
    __device__ __forceinline__ void reset() {
        ij = tau = T(0);
#pragma unroll
        for (int k = 0; k < 7; ++k) ql[k] = qi[k] = qt[k] = T(0);
    }
    // one sample: emissivity e and absorptivity a per unit affine parameter over dl
    __device__ __forceinline__ void add(const Plasma<T>& P, T e, T a, T dl) {
        const T q[7] = {P.rho, P.ne, P.p, P.th, P.bg, P.bsq / P.rho, P.binv};
        const T dtau = a * dl;
        const T ex = exp(-dtau), om = -expm1(-dtau);
        ij += e * dl;
        tau += dtau;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            ql[k] += q[k] * dl;
            qi[k] += q[k] * e * dl;
            qt[k] = ex * qt[k] + om * q[k];
        }
    }
};

template <class T>
__device__ __forceinline__ void aux_finish(const ImageDesc& im, int64_t pix, const AuxAcc<T>& A) {
    const double lam = aux_load(im, 2, pix);     // written by the geodesic kernel
    aux_store(im, 3, pix, A.ij);
    aux_store(im, 4, pix, A.tau);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        aux_store(im, 5 + k, pix, lam > 0.0 ? (double)A.ql[k] / lam : 0.0);
        aux_store(im, 12 + k, pix, A.ij > T(0) ? A.qi[k] / A.ij : T(0));
        aux_store(im, 19 + k, pix, A.qt[k]);
    }
}

// The record a ray's transfer starts from: the far-side records beyond its last step that
// came within 1.001 r_max of the hole lie outside the grid's shell (their sample radius
// exceeds r_max by far more than its FP32 rounding), carry no plasma and leave the coherency
// zero, so the transfer starts at that step's last record (record 0 where no step did, for
// the read-out at its node).
__device__ __forceinline__ int32_t transfer_start(const RayHdr& hd) {
    const int32_t last = hd.nrec - 1;
    return hd.last_in < last ? (hd.last_in > 0 ? hd.last_in : 0) : last;
}

// A warp's 32 consecutive wave rays (w = lane of the warp's first ray + lane) with keys k
// (lanes with on = false hold none): the key of each order group -- the group's largest --
// into key[group] and the histogram of the counting sort (lanes of a warp with equal buckets
// add with one atomic).
template <int G>
__device__ __forceinline__ void group_key(int32_t k, bool on, int64_t w, int32_t* __restrict__ key,
                                          unsigned int* __restrict__ hist) {
    static_assert(G == 1 || G == 32, "order groups: single rays or warps");
    const int lane = threadIdx.x & 31;
    if constexpr (G == 32) {
        const int32_t gk = __reduce_max_sync(0xffffffffu, k);
        if (lane == 0 && gk >= 0) {
            key[w / 32] = gk;
            atomicAdd(&hist[cost_bucket(gk)], 1u);
        }
    } else {
        if (on) key[w] = k;
        const int b = on ? cost_bucket(k) : -1 - lane;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        if (on && lane == __ffs(same) - 1) atomicAdd(&hist[b], (unsigned int)__popc(same));
    }
}

// The fused transfer's ray order: each wave ray's records to process (0 for rays without a
// transfer) into key[] and the histogram of the counting sort (lanes of a warp with equal
// buckets add with one atomic); work_scan_kernel and work_scatter_kernel finish the order.
__global__ void record_key_kernel(const RayHdr* __restrict__ hdr, BlockSource bs,
                                  int64_t ray_begin, int64_t ray_end, int32_t* __restrict__ key,
                                  unsigned int* __restrict__ hist) {
    const int64_t re = wave_end(bs, ray_end);
    const int64_t n = re > ray_begin ? re - ray_begin : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < n; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        const bool on = w < n;
        int32_t k = -1;
        if (on) {
            const RayHdr hd = hdr[w];
            k = (hd.status == BL_RAY_OVERFLOW || hd.nrec == 0) ? 0 : transfer_start(hd) + 1;
        }
        group_key<kFusedGroup>(k, on, w, key, hist);
    }
}

template <class T, class R, int kF>
__device__ __forceinline__ void transfer_body(const ImageDesc* __restrict__ imgs,
                                              int n_images, int64_t ray_begin, int64_t ray_end,
                                              const RayHdr* __restrict__ hdr,
                                              const R* __restrict__ pool,
                                              const int32_t* __restrict__ chunks,
                                              Counters* ctr, BlockSource bs, SideIn side) {
    const float* __restrict__ mlp_y = side.mlp_y;
    const float* __restrict__ mlp_params = side.mlp_params;
    constexpr bool kSlow = (kF & kFSlow) != 0;
    constexpr bool kUnpol = (kF & kFUnpol) != 0;
    constexpr bool kAux = (kF & kFAux) != 0;
    // learned coefficients: the model's outputs come from the pool pass (mlp_y, 8 floats a
    // record), the record's last value flags the samples the model evaluated
    constexpr bool kMlp = (kF & kFMlp) != 0;
    static_assert(!kMlp || std::is_same<R, float>::value, "the learned model needs FP32 records");
    constexpr bool kIdx = kMlp;   // the transfer needs each record's pool index
    // the stencil field test of plasma_at: always in the FP64 form; in FP32 where the rays are
    // not queued by record count -- that order predicts a ray's cost from its records, which
    // stops holding once field-free records are cheap (nine 256^2 images, fast form: cell-layout
    // grids in the record-count order 11.6 ms with the test switched off there, 13.3 with it on;
    // plane-layout grids in the consecutive queue 18.9 ms with the test, 25.8 before it). A
    // run-time switch in one kernel, so that both queue orders run the same arithmetic; FP32
    // compiles it into the plain polarized and unpolarized variants only, which keeps the
    // register budgets of the slow-light, auxiliary-image and learned variants.
    constexpr bool kFieldTestable = sizeof(T) == sizeof(double) || (!kSlow && !kAux && !kMlp);
    const bool field_test = kFieldTestable && (sizeof(T) == sizeof(double) || side.perm == nullptr);
    int64_t nxt_k = 0;
    const int64_t re = wave_end(bs, ray_end);
    const int64_t n_rays = re > ray_begin ? re - ray_begin : 0;
    const int64_t total_rays = side.perm ? ordered_total<kFusedGroup>(n_rays) : n_rays;
    int64_t wray = 0;
    bool active = false;
    int64_t ray = 0, opix = 0;
    int q = 0, pi = 0, pj = 0;
    int32_t idx = 0;
    Coh<T> N;
    T Iu = T(0);            // unpolarized intensity (Eq. unpolarized)
    AuxAcc<T> AX;
    bool started = false;
    T prev[kRecVals];
    R nxt[RecStride<R>::v];
    T kt = T(0), a = T(0), m = T(0), nu_norm = T(0);
    bool flat = false;

    bool exhausted = false;
    while (true) {
        const bool need = !active && !exhausted;
        const unsigned long long got = warp_refill(&ctr->next_ray_tr, need);
        if (need) {
            if ((int64_t)got >= total_rays) exhausted = true;
            else {
                // the wave's rays in the order of their record counts where there is one
                wray = side.perm ? ordered_ray<kFusedGroup>(side.perm, got, n_rays) : (int64_t)got;
                ray = ray_begin + wray;
            }
        }
        if (!__any_sync(0xffffffffu, active || (need && !exhausted))) break;
        if (!active && !(need && !exhausted)) continue;
        if (!active && wray < 0) continue;   // a partial order group's empty position
        if (!active) {
            setup_ray(imgs, n_images, bs, ray, q, opix, pi, pj);
            const ImageDesc& im = imgs[q];
            const RayHdr hd = hdr[wray];
            if (hd.status == BL_RAY_OVERFLOW || hd.nrec == 0) {
                const int64_t npix = im.n_rays;
                const int64_t pix = opix;
                const double val = hd.status == BL_RAY_OVERFLOW ? nan("") : 0.0;
                for (int s = 0; s < 4; ++s) {
                    if (im.dtype == 0) ((double*)im.stokes)[s * npix + pix] = val;
                    else ((float*)im.stokes)[s * npix + pix] = (float)val;
                }
                if constexpr (kAux) {
                    if (im.aux) {
                        AuxAcc<T> z;
                        z.reset();
                        aux_finish(im, pix, z);
                    }
                }
                continue;
            }
            idx = transfer_start(hd);
            load_record<R>(record_ptr(pool, chunks, wray, idx), nxt);
            if constexpr (kIdx) nxt_k = record_index(chunks, wray, idx);
            kt = (T)hd.kt;
            nu_norm = (T)(hd.nnorm * im.freq);
            a = ic<T>(im, kcSpin);
            m = ic<T>(im, kcMass);
            flat = im.flat != 0;
#pragma unroll
            for (int c = 0; c < 10; ++c) N.re[c] = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) N.im[c] = T(0);
            Iu = T(0);
            if constexpr (kAux) AX.reset();
            started = false;
            active = true;
        }
        const ImageDesc& im = imgs[q];
        // idx < 0: every sample is in, and this iteration only takes the last half-step to the
        // camera node and reads the pixel out (sharing the transport code of the sample steps)
        const bool finishing = idx < 0;
        T cur[kRecVals];
        T nxt_t = T(0);   // the sample's coordinate time
        int64_t cur_k = 0;
        bool cur_flag = false;
        if (!finishing) {
            // record idx was prefetched into nxt; start fetching idx - 1 before using it
#pragma unroll
            for (int c = 0; c < kRecVals; ++c) cur[c] = (T)nxt[c];
            nxt_t = (T)nxt[13];
            if constexpr (kIdx) cur_k = nxt_k;
            if constexpr (kMlp) cur_flag = __float_as_uint((float)nxt[15]) != 0u;
            if (idx > 0) {
                load_record<R>(record_ptr(pool, chunks, wray, idx - 1), nxt);
                if constexpr (kIdx) nxt_k = record_index(chunks, wray, idx - 1);
            }
        }
        if (!kUnpol && started) {
            // merged N half-steps from the previous sample to this one (to the camera node on
            // the finishing iteration, where the far half is empty)
            T A0[4][4], A1[4][4];
            const T kp[4] = {kt, prev[3], prev[4], prev[5]};
            const T kn[4] = {kt, prev[9], prev[10], prev[11]};
            transport_matrix<T>(prev, kp, a, m, flat, A0);
            transport_matrix<T>(prev + 6, kn, a, m, flat, A1);
            coh_pc_step(N, A0, A1, T(0.5) * (prev[12] + (finishing ? T(0) : cur[12])));
        }
        if (finishing) {
            const int64_t npix = im.n_rays;
            T sv[4] = {Iu, T(0), T(0), T(0)};
            if constexpr (!kUnpol) {
                // read out in the camera basis at the camera-side node
                KSGeom<T> G;
                ks_geom<T>(prev[6], prev[7], prev[8], a, m, flat, false, G);
                T hv[4], vv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if constexpr (std::is_same<T, float>::value) { hv[c] = im.f_hh[c]; vv[c] = im.f_vv[c]; }
                    else { hv[c] = im.hh[c]; vv[c] = im.vv[c]; }
                }
                T hl[4], vl[4];
                lower4(G, hv, hl);
                lower4(G, vv, vl);
                coh_to_stokes(N, hl, vl, sv);
            }
            for (int c = 0; c < 4; ++c) {
                if (im.dtype == 0) ((double*)im.stokes)[c * npix + opix] = (double)sv[c];
                else ((float*)im.stokes)[c * npix + opix] = (float)sv[c];
            }
            if constexpr (kAux) if (im.aux) aux_finish(im, opix, AX);
            active = false;
            continue;
        }
        {
            const T xs[3] = {cur[0], cur[1], cur[2]};
            KSGeom<T> G;
            ks_geom<T>(xs[0], xs[1], xs[2], a, m, flat, false, G);
            Plasma<T> P;
            if (plasma_at<T, kSlow>(im, xs, nxt_t, G, P, field_test)) {
                const T kl[4] = {kt, cur[3], cur[4], cur[5]};
                T ku[4];
                raise4(G, kl, ku);
                const T kdu = kl[0] * P.u[0] + kl[1] * P.u[1] + kl[2] * P.u[2] + kl[3] * P.u[3];
                const T kdb = kl[0] * P.b[0] + kl[1] * P.b[1] + kl[2] * P.b[2] + kl[3] * P.b[3];
                const T nu_fl = nu_norm * (-kdu);
                T cth = fq(kdb, (-kdu) * fsqrt(P.bsq));
                cth = cth > T(1) ? T(1) : (cth < T(-1) ? T(-1) : cth);
                T co[8];
                bool learned = false;
                if constexpr (kMlp) {
                    const mlp::ModelIn mi = mlp::model_inputs(P.th, P.bg, nu_fl, cth);
                    if (cur_flag && mi.ok && P.ne > T(0)) {
                        // (loaded here: loading them one sample ahead with the record measured
                        // slower, 61.2 against 58.9 ms at 1024^2)
                        const float4* yq = reinterpret_cast<const float4*>(mlp_y + 8 * cur_k);
                        const float4 y0 = __ldg(yq), y1 = __ldg(yq + 1);
                        const float y[7] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z};
                        float o[7];
                        mlp::model_outputs_from_y(mlp_params, y, mi.f, o);
                        mlp::coefficients_from(o, P.ne, P.th, P.bg, nu_fl, cth, co);
                        learned = true;
                    }
                }
                if (!learned) synchrotron_coefficients<T>(P.ne, P.th, P.bg, nu_fl, cth, co);
                const T g = fq(ic<T>(im, kcFreq), nu_fl);
                const T path = ic<T>(im, kcLen) * (-kdu);
                const T eg = g * g * g * path;
                const T coef[8] = {co[0] * eg, co[1] * eg, co[2] * eg, co[3] * path,
                                   co[4] * path, co[5] * path, co[6] * path, co[7] * path};
                if constexpr (kAux) AX.add(P, coef[0], coef[3], cur[12]);
                if constexpr (kUnpol) {
                    Iu = unpolarized_step<T>(coef[0], coef[3], cur[12], Iu);
                } else {
                    T e1[4], e2[4], e1l[4], e2l[4];
                    fluid_basis<T>(G, P, kl, ku, e1, e2, e1l, e2l);
                    T s0[4], s1[4];
                    coh_to_stokes(N, e1l, e2l, s0);
                    stokes_step<T>(coef, s0, cur[12], s1);
                    stokes_to_coh(e1, e2, s1, N);
                }
                started = true;
            }
        }
#pragma unroll
        for (int c = 0; c < kRecVals; ++c) prev[c] = cur[c];
        --idx;
    }
}
// The transfer kernel: FP32 (mixed and fast forms) in CTAs of 128 threads, the polarized and
// unpolarized variants held to 4 CTAs an SM (128 registers; with the field test uncapped they
// take 142 and 3 CTAs), the slow-light and auxiliary-image variants uncapped; FP64 capped
// (BL_TR64_MAXNREG) in CTAs of 64 threads, which keeps more warps an SM resident.
#ifndef BL_TR32_MIN_CTAS
#define BL_TR32_MIN_CTAS 4
#endif
template <class T, class R, int kF>
__global__ void __launch_bounds__(128, (kF & (kFSlow | kFAux)) ? 0 : BL_TR32_MIN_CTAS) transfer_kernel(const ImageDesc* __restrict__ imgs,
                                                       int n_images, int64_t ray_begin,
                                                       int64_t ray_end,
                                                       const RayHdr* __restrict__ hdr,
                                                       const R* __restrict__ pool,
                                                       const int32_t* __restrict__ chunks,
                                                       Counters* ctr, BlockSource bs,
                                                       SideIn side) {
    transfer_body<T, R, kF>(imgs, n_images, ray_begin, ray_end, hdr, pool, chunks, ctr, bs, side);
}
// Register cap and CTA size of the FP64 transfer kernel. Its FP64 arithmetic runs at 1/64 of
// the FP32 rate with long dependent latencies, so resident warps matter more than spills to
// L1: measured on the 9 x 256^2 step, 96 registers (20 warps an SM) 459 ms, 80: 441 ms, 72:
// 429 ms, 64 (32 warps an SM): 405 ms, 56: 395 ms, 48 (42 warps an SM): 385 ms, 40: 373 ms,
// 32 (64 warps, the SM's limit): 349 ms.
#ifndef BL_TR64_MAXNREG
#define BL_TR64_MAXNREG 32
#endif
#ifndef BL_TR64_THREADS
#define BL_TR64_THREADS 64
#endif
// The transfer of the learned-coefficient form (its model outputs from the pool pass),
// compiled for 4 resident CTAs an SM (128 registers; uncapped it takes 142 registers and 3
// CTAs, measured 62.5 against 58.9 ms at 1024^2).
template <bool kSlow>
__global__ void __launch_bounds__(128, 4) transfer_learned_kernel(
        const ImageDesc* __restrict__ imgs, int n_images, int64_t ray_begin, int64_t ray_end,
        const RayHdr* __restrict__ hdr, const float* __restrict__ pool,
        const int32_t* __restrict__ chunks, Counters* ctr, BlockSource bs, SideIn side) {
    transfer_body<float, float, kFMlp | (kSlow ? kFSlow : 0)>(
        imgs, n_images, ray_begin, ray_end, hdr, pool, chunks, ctr, bs, side);
}

constexpr int kTransferFp64Threads = BL_TR64_THREADS;
template <int kF>
__global__ void __maxnreg__(BL_TR64_MAXNREG) transfer_kernel_fp64(const ImageDesc* __restrict__ imgs,
                                                     int n_images, int64_t ray_begin,
                                                     int64_t ray_end,
                                                     const RayHdr* __restrict__ hdr,
                                                     const double* __restrict__ pool,
                                                     const int32_t* __restrict__ chunks,
                                                     Counters* ctr, BlockSource bs,
                                                     SideIn side) {
    transfer_body<double, double, kF>(imgs, n_images, ray_begin, ray_end, hdr, pool, chunks,
                                      ctr, bs, side);
}


// ---------------------------------------------------------------------------------------
// FP64 form, first pass of the transfer: everything a sample needs that does not depend on
// the ray's running coherency -- geometry, plasma state, the scaled synchrotron coefficients
// and the fluid-frame basis -- for every record, written per record (kPreVals doubles and a
// flag byte). The arithmetic is that of the transfer kernel's sample step, operation for
// operation; the second pass (transport_fp64_kernel) runs the transport and the Stokes steps.
// Work is compacted per warp: a warp takes rays in turn and tests its records 32 at a time
// with a conservative FP32 test of the grid's radial shell (records outside get flag 0 at
// once); the records that pass go to the warp's queue in shared memory, and whenever it holds
// 32 the warp evaluates them with every lane busy, whatever rays they belong to (a warp per
// ray left lanes idle on each ray's last 32 records and on records outside the grid: 26.2
// of 32 lanes active). Each ray's farthest plasma sample and plasma-sample count are combined
// with atomics (one per ray in a batch) for the transport pass's start and order.
// ---------------------------------------------------------------------------------------
// Resident CTAs an SM of the FP64 sample pass (16: 32 registers, the SM's 64 warps; measured
// on the 9 x 256^2 step with the transport pass at 32 registers: 4 CTAs 326.3 ms for both
// passes, 8: 324.4, 16: 322.7; the single fused kernel 346.7 ms).
#ifndef BL_PRE64_MIN_CTAS
#define BL_PRE64_MIN_CTAS 16
#endif
// Cell index along one axis of the grid lookup (plasma_at) from a fractional coordinate u
// (trilinear: u = cell coordinate - 1/2, the stencil's lower cell, clamped so that both cells
// exist; nearest: u = cell coordinate, the cell, clamped).
__device__ __forceinline__ int lookup_cell(float u, int n, bool tri) {
    if (tri) {
        if (n == 1) return 0;
        u = fminf(fmaxf(u, 0.0f), (float)(n - 1));
        const int i = (int)floorf(u);
        return i > n - 2 ? n - 2 : i;
    }
    const int i = (int)floorf(u);
    return min(max(i, 0), n - 1);
}
// The cell a coordinate known to within +-m maps to, or -1 when the interval straddles a
// cell boundary (the map u -> cell is monotone, so equal ends fix every point between).
__device__ __forceinline__ int certain_cell(float u, float m, int n, bool tri) {
    const int lo = lookup_cell(u - m, n, tri), hi = lookup_cell(u + m, n, tri);
    return lo == hi ? lo : -1;
}
__device__ __forceinline__ int certain_cell_periodic(float u, float m) {
    const float lo = floorf(u - m), hi = floorf(u + m);
    return lo == hi ? (int)lo : INT_MIN;
}

// Whether the grid lookup of a sample at this position (plasma_at, one snapshot) certainly
// reads a stencil whose corners all carry zero magnetic field -- the sample then has b = 0
// and no synchrotron plasma (plasma_at requires b^2 > 0), whatever else the cells hold. The
// stencil is located in FP32 from the record's FP32 position: r^2 as the radial shell test
// forms it, theta = atan2(sin, cos) with sin^2 = (x^2 + y^2) / (r^2 + a^2) and cos = z / r
// (x^2 + y^2 = (r^2 + a^2) sin^2 theta in Cartesian Kerr-Schild), the azimuth as plasma_at
// forms it. Each fractional coordinate carries a margin of 1e-3 cells plus four times a bound
// on its FP32 error (the rounding of r^2 grows with (R^2 + a^2) / r^2, R^2 = x^2 + y^2 + z^2)
// and the rounding of the FP32 scale factors;
// a coordinate whose margin interval straddles a cell boundary, or a point within 1e-15 of
// the axis, is reported as not certain (false: the FP64 lookup decides). A true answer is
// exact: the FP64 lookup then reads the same stencil and returns no plasma.
__device__ __forceinline__ bool stencil_field_free(const ImageDesc& im, float x, float y, float z,
                                                   float r2, float aa) {
    const float rho2 = x * x + y * y;
    if (!(rho2 > 1e-30f)) return false;
    const float R2 = rho2 + z * z;
    const float eps = 3e-7f * (R2 + aa) / r2 + 2e-7f;
    const float r = sqrtf(r2);
    const float a = im.f_c[kcSpin];
    const float th = atan2f(sqrtf(rho2 / (r2 + aa)), z / r);
    float ph = atan2f(y * r - x * a, x * r + y * a);
    const float twopi = 6.28318530717958648f;
    if (ph < 0.0f) ph += twopi;
    if (ph >= twopi) ph -= twopi;
    const int nr = im.nr, nt = im.nt, np = im.nph;
    const bool tri = im.interp != 0;
    const float off = tri ? 0.5f : 0.0f;
    const float idlr = im.f_c[kcIDlr];
    const float idth = (float)nt * 0.318309886183790672f;
    const float idph = (float)np * 0.159154943091895336f;
    // margins: the coordinate's own FP32 error, and 4e-7 |u| for the FP32 scale factors
    const float ur = (logf(r) - im.f_c[kcLogRmin]) * idlr - off;
    const float ut = th * idth - off;
    const float up = ph * idph - off;
    const int i0 = certain_cell(ur, 1e-3f + idlr * (4.0f * eps + 1e-6f) + 4e-7f * fabsf(ur), nr, tri);
    const int j0 = certain_cell(ut, 1e-3f + idth * (4.0f * eps + 1e-6f) + 4e-7f * fabsf(ut), nt, tri);
    const int kf = certain_cell_periodic(up, 1e-3f + idph * (2.0f * eps + 1e-6f) + 4e-7f * fabsf(up));
    if (i0 < 0 || j0 < 0 || kf == INT_MIN) return false;
    const int k0 = ((kf % np) + np) % np;
    const int i1 = (tri && nr > 1) ? i0 + 1 : i0, j1 = (tri && nt > 1) ? j0 + 1 : j0;
    const int k1 = tri ? (k0 + 1) % np : k0;
    const size_t plane = (size_t)np * nt * nr;
    unsigned int bits = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const size_t cell = ((size_t)((c & 4) ? k1 : k0) * nt + ((c & 2) ? j1 : j0)) * nr +
                            ((c & 1) ? i1 : i0);
        bits |= cell_field_bits(im.prim, im.layout, plane, cell);
    }
    return (bits & 0x7fffffffu) == 0u;   // +-0 in every field component of every corner
}

struct SampleItem {
    int64_t k;       // pool record
    int32_t wray;    // ray within the wave
    int32_t idx;     // record within the ray
    int32_t q;       // image
    int32_t pad_;
};
constexpr int kSampleQueue = 64;   // per warp: fewer than 32 waiting + one batch of 32 tests

template <bool kSlow>
__global__ void __launch_bounds__(128, BL_PRE64_MIN_CTAS) fp64_samples_kernel(const ImageDesc* __restrict__ imgs,
                                                           int n_images, int64_t ray_begin,
                                                           int64_t ray_end,
                                                           const RayHdr* __restrict__ hdr,
                                                           const double* __restrict__ pool,
                                                           const int32_t* __restrict__ chunks,
                                                           Counters* ctr, BlockSource bs,
                                                           double* __restrict__ pre,
                                                           unsigned char* __restrict__ pre_flag,
                                                           int32_t* __restrict__ tfirst,
                                                           int32_t* __restrict__ tnpl) {
    using T = double;
    __shared__ SampleItem qbuf[4][kSampleQueue];   // 128 threads: 4 warps
    const int lane = threadIdx.x & 31;
    SampleItem* Q = qbuf[threadIdx.x >> 5];
    int qn = 0;   // items waiting (warp-uniform)

    // the queue's first n items, lane i taking item i
    auto evaluate = [&](int n) {
        bool plasma = false;
        int32_t wray = -1, idx = -1;
        if (lane < n) {
            const SampleItem it = Q[lane];
            wray = it.wray;
            idx = it.idx;
            const RayHdr hd = hdr[it.wray];
            const ImageDesc& im = imgs[it.q];
            const T kt = hd.kt, nu_norm = hd.nnorm * im.freq;
            const T a = ic<T>(im, kcSpin), m = ic<T>(im, kcMass);
            const bool flat = im.flat != 0;
            T cur[RecStride<double>::v];
            load_record<double>(pool + it.k * RecStride<double>::v, cur);
            const T xs[3] = {cur[0], cur[1], cur[2]};
            KSGeom<T> G;
            ks_geom<T>(xs[0], xs[1], xs[2], a, m, flat, false, G);
            Plasma<T> P;
            if (plasma_at<T, kSlow>(im, xs, cur[13], G, P, true)) {
                const T kl[4] = {kt, cur[3], cur[4], cur[5]};
                T ku[4];
                raise4(G, kl, ku);
                const T kdu = kl[0] * P.u[0] + kl[1] * P.u[1] + kl[2] * P.u[2] + kl[3] * P.u[3];
                const T kdb = kl[0] * P.b[0] + kl[1] * P.b[1] + kl[2] * P.b[2] + kl[3] * P.b[3];
                const T nu_fl = nu_norm * (-kdu);
                T cth = fq(kdb, (-kdu) * fsqrt(P.bsq));
                cth = cth > T(1) ? T(1) : (cth < T(-1) ? T(-1) : cth);
                T co[8];
                synchrotron_coefficients<T>(P.ne, P.th, P.bg, nu_fl, cth, co);
                const T g = fq(ic<T>(im, kcFreq), nu_fl);
                const T path = ic<T>(im, kcLen) * (-kdu);
                const T eg = g * g * g * path;
                T v[kPreVals] = {co[0] * eg, co[1] * eg, co[2] * eg, co[3] * path,
                                 co[4] * path, co[5] * path, co[6] * path, co[7] * path};
                fluid_basis<T>(G, P, kl, ku, v + 8, v + 12, v + 16, v + 20);
                double2* out = reinterpret_cast<double2*>(pre + kPreVals * it.k);
#pragma unroll
                for (int i = 0; i < kPreVals / 2; ++i) out[i] = make_double2(v[2 * i], v[2 * i + 1]);
                plasma = true;
            }
            pre_flag[it.k] = plasma ? 1 : 0;
        }
        // per ray of the batch: its plasma samples lie at increasing lanes (records enter the
        // queue in order), so the highest lane of a ray's group holds its farthest one
        const unsigned grp = __match_any_sync(0xffffffffu, plasma ? wray : -1 - lane);
        if (plasma && lane == 31 - __clz(grp)) {
            atomicMax(&tfirst[wray], idx);
            atomicAdd(&tnpl[wray], __popc(grp));
        }
    };

    // one loop with one evaluation site (the kernel's code stays small for the instruction
    // cache): each turn takes a ray if the current one is done, tests its next 32 records, and
    // evaluates a batch when 32 items wait or, with the rays exhausted, whatever remains
    const int64_t re = wave_end(bs, ray_end);
    const int64_t total_rays = re > ray_begin ? re - ray_begin : 0;
    int64_t wray = 0;
    int32_t base = 0, nrec = 0;
    int q = 0;
    float aa = 0.0f, r2lo = 0.0f, r2hi = 0.0f;
    bool exhausted = false;
    while (true) {
        if (base >= nrec && !exhausted) {
            unsigned long long got = 0;
            if (lane == 0) got = atomicAdd(&ctr->next_ray_mi, 1ull);
            got = __shfl_sync(0xffffffffu, got, 0);
            if ((int64_t)got >= total_rays) {
                exhausted = true;
            } else {
                wray = (int64_t)got;
                int pi, pj;
                int64_t opix;
                setup_ray(imgs, n_images, bs, ray_begin + wray, q, opix, pi, pj);
                const RayHdr hd = hdr[wray];
                base = 0;
                nrec = 0;
                if (hd.status != BL_RAY_OVERFLOW && hd.nrec > 0) {
                    const ImageDesc& im = imgs[q];
                    // shell test in FP32 on r^2 with 1e-4 margins (the exact test follows in
                    // evaluate): 2 r^2 = R^2 - a^2 + ((R^2 - a^2)^2 + 4 a^2 z^2)^1/2
                    aa = (float)(im.spin * im.spin);
                    r2lo = (float)(im.r_min * im.r_min * (1.0 - 1e-4));
                    r2hi = (float)(im.r_max * im.r_max * (1.0 + 1e-4));
                    // records beyond the last one near the grid carry no plasma
                    // (transfer_start)
                    nrec = hd.last_in + 1 < hd.nrec ? hd.last_in + 1 : hd.nrec;
                }
            }
        }
        if (base < nrec) {
            const int32_t idx = base + lane;
            bool cand = false;
            int64_t k = 0;
            if (idx < nrec) {
                k = record_index(chunks, wray, idx);
                const double* rp = pool + k * RecStride<double>::v;
                const float x = (float)__ldg(rp), y = (float)__ldg(rp + 1), z = (float)__ldg(rp + 2);
                const float qq = x * x + y * y + z * z - aa;
                const float r2 = 0.5f * (qq + sqrtf(qq * qq + 4.0f * aa * z * z));
                cand = r2 >= r2lo && r2 <= r2hi;
                // a stencil without magnetic field holds no plasma (stencil_field_free);
                // one snapshot only
                if (!kSlow && cand) cand = !stencil_field_free(imgs[q], x, y, z, r2, aa);
                if (!cand) pre_flag[k] = 0;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, cand);
            if (cand) {
                SampleItem& it = Q[qn + __popc(mask & ((1u << lane) - 1u))];
                it.k = k;
                it.wray = (int32_t)wray;
                it.idx = idx;
                it.q = q;
            }
            qn += __popc(mask);
            base += 32;
            __syncwarp();
        }
        if (qn >= 32 || (exhausted && qn > 0)) {
            const int n = qn < 32 ? qn : 32;
            evaluate(n);
            __syncwarp();
            SampleItem keep;
            const bool moves = lane < qn - n;
            if (moves) keep = Q[n + lane];
            __syncwarp();
            if (moves) Q[lane] = keep;
            qn -= n;
            __syncwarp();
        }
        if (exhausted && qn == 0) break;
    }
}

// The transport pass's key for each group of wave rays from the sample pass's results: the
// farthest plasma sample (tfirst, -1: none) and the plasma-sample count (npl): the steps from
// there to the camera plus half a step per Stokes step; with the histogram of the counting
// sort.
__global__ void transport_key_kernel(const int32_t* __restrict__ tfirst,
                                     const int32_t* __restrict__ npl, int32_t* __restrict__ key,
                                     BlockSource bs, int64_t ray_begin, int64_t ray_end,
                                     unsigned int* __restrict__ hist) {
    const int64_t re = wave_end(bs, ray_end);
    const int64_t n = re > ray_begin ? re - ray_begin : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < n; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        const bool on = w < n;
        const int32_t k = on ? tfirst[w] + 1 + (npl[w] >> 1) : -1;
        group_key<kTransportGroup>(k, on, w, key, hist);
    }
}

// ---------------------------------------------------------------------------------------
// FP64 form, second pass of the transfer: along each ray from the source end, the merged N
// half-steps of the predictor-corrector (Table tab:pc) and, at every sample the first pass
// found plasma at, the Stokes step with that pass's coefficients and basis; at the camera
// node the read-out in the camera basis. The same operations in the same order as the single
// kernel (transfer_body), with a smaller live state: only N and the two records of the
// current half-steps, re-read from the pool instead of carried (FP64 registers are the
// scarce resource; their spills were the kernel's main stall).
// ---------------------------------------------------------------------------------------
#ifndef BL_TRANSPORT64_MAXNREG
#define BL_TRANSPORT64_MAXNREG 32
#endif
__global__ void __maxnreg__(BL_TRANSPORT64_MAXNREG) transport_fp64_kernel(
        const ImageDesc* __restrict__ imgs, int n_images, int64_t ray_begin, int64_t ray_end,
        const RayHdr* __restrict__ hdr, const double* __restrict__ pool,
        const int32_t* __restrict__ chunks, Counters* ctr, BlockSource bs, SideIn side,
        const int32_t* __restrict__ perm) {
    using T = double;
    const int64_t re = wave_end(bs, ray_end);
    const int64_t n_rays = re > ray_begin ? re - ray_begin : 0;
    const int64_t total_rays = perm ? ordered_total<kTransportGroup>(n_rays) : n_rays;
    int64_t wray = 0, ray = 0, opix = 0;
    bool active = false, started = false;
    int q = 0, pi = 0, pj = 0;
    int32_t idx = 0;
    Coh<T> N;
    T kt = T(0), a = T(0), m = T(0);
    bool flat = false;
    bool exhausted = false;
    while (true) {
        const bool need = !active && !exhausted;
        const unsigned long long got = warp_refill(&ctr->next_ray_tr, need);
        if (need) {
            if ((int64_t)got >= total_rays) exhausted = true;
            else {
                // the sample pass's work order (longest first) where there is one
                wray = perm ? ordered_ray<kTransportGroup>(perm, got, n_rays) : (int64_t)got;
                ray = ray_begin + wray;
            }
        }
        if (!__any_sync(0xffffffffu, active || (need && !exhausted))) break;
        if (!active && !(need && !exhausted)) continue;
        if (!active && wray < 0) continue;   // a partial order group's empty position
        if (!active) {
            setup_ray(imgs, n_images, bs, ray, q, opix, pi, pj);
            const ImageDesc& im = imgs[q];
            const RayHdr hd = hdr[wray];
            if (hd.status == BL_RAY_OVERFLOW || hd.nrec == 0) {
                const int64_t npix = im.n_rays;
                const double val = hd.status == BL_RAY_OVERFLOW ? nan("") : 0.0;
                for (int s = 0; s < 4; ++s) ((double*)im.stokes)[s * npix + opix] = val;
                continue;
            }
            // from the farthest plasma sample where the sample pass found it (the records
            // beyond it leave N = 0 untouched); with none, straight to the read-out
            idx = side.first ? side.first[wray] : hd.nrec - 1;
            kt = hd.kt;
            a = ic<T>(im, kcSpin);
            m = ic<T>(im, kcMass);
            flat = im.flat != 0;
#pragma unroll
            for (int c = 0; c < 10; ++c) N.re[c] = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) N.im[c] = T(0);
            started = false;
            active = true;
        }
        const ImageDesc& im = imgs[q];
        const bool finishing = idx < 0;
        // this sample's segment length (none on the finishing half-step to the camera node)
        T dl_cur = T(0);
        int64_t cur_k = 0;
        if (!finishing) {
            cur_k = record_index(chunks, wray, idx);
            dl_cur = __ldg(pool + cur_k * RecStride<double>::v + 12);
        }
        if (started || finishing) {
            // the previous sample's record: its point and node carry the two half-steps
            const double* pr = pool + record_index(chunks, wray, idx + 1) * RecStride<double>::v;
            if (started) {
                const T h = T(0.5) * (__ldg(pr + 12) + dl_cur);
                T A[4][4];
                Coh<T> nh;
                {
                    const T x0[3] = {__ldg(pr), __ldg(pr + 1), __ldg(pr + 2)};
                    const T k0[4] = {kt, __ldg(pr + 3), __ldg(pr + 4), __ldg(pr + 5)};
                    transport_matrix<T>(x0, k0, a, m, flat, A);
                }
                coh_axpy(N, N, A, T(0.5) * h, nh);
                {
                    const T x1[3] = {__ldg(pr + 6), __ldg(pr + 7), __ldg(pr + 8)};
                    const T k1[4] = {kt, __ldg(pr + 9), __ldg(pr + 10), __ldg(pr + 11)};
                    transport_matrix<T>(x1, k1, a, m, flat, A);
                }
                Coh<T> out;
                coh_axpy(N, nh, A, h, out);
                N = out;
            }
            if (finishing) {
                // read out in the camera basis at the camera-side node of the last record
                KSGeom<T> G;
                ks_geom<T>(__ldg(pr + 6), __ldg(pr + 7), __ldg(pr + 8), a, m, flat, false, G);
                T hl[4], vl[4];
                lower4(G, im.hh, hl);
                lower4(G, im.vv, vl);
                T sv[4];
                coh_to_stokes(N, hl, vl, sv);
                const int64_t npix = im.n_rays;
                for (int c = 0; c < 4; ++c) ((double*)im.stokes)[c * npix + opix] = sv[c];
                active = false;
                continue;
            }
        }
        if (side.pre_flag[cur_k]) {
            const double2* pq = reinterpret_cast<const double2*>(side.pre + kPreVals * cur_k);
            T v[kPreVals];
#pragma unroll
            for (int i = 0; i < kPreVals / 2; ++i) {
                const double2 d = __ldg(pq + i);
                v[2 * i] = d.x;
                v[2 * i + 1] = d.y;
            }
            T s0[4], s1[4];
            coh_to_stokes(N, v + 16, v + 20, s0);
            stokes_step<T>(v, s0, dl_cur, s1);
            stokes_to_coh(v + 8, v + 12, s1, N);
            started = true;
        }
        --idx;
    }
}

// ---------------------------------------------------------------------------------------
// Learned coefficients, first pass: the model inputs of every sample record. One warp takes a
// ray, its lanes 32 consecutive records at a time (the records of a chunk lie together in the
// pool): geometry, plasma state and the fluid-frame frequency and pitch angle at the sample,
// as the transfer computes them, then the model's input row (mlp::input_row) into the record's
// last 8 bytes -- zeros where the sample has no plasma or lies outside the model's domain.
// ---------------------------------------------------------------------------------------
template <bool kSlow>
__global__ void __launch_bounds__(128) mlp_inputs_kernel(const ImageDesc* __restrict__ imgs,
                                                         int n_images, int64_t ray_begin,
                                                         int64_t ray_end,
                                                         const RayHdr* __restrict__ hdr,
                                                         float* __restrict__ pool,
                                                         const int32_t* __restrict__ chunks,
                                                         Counters* ctr, BlockSource bs) {
    using T = float;
    const int lane = threadIdx.x & 31;
    const int64_t re = wave_end(bs, ray_end);
    const int64_t total_rays = re > ray_begin ? re - ray_begin : 0;
    while (true) {
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(&ctr->next_ray_mi, 1ull);
        got = __shfl_sync(0xffffffffu, got, 0);
        if ((int64_t)got >= total_rays) break;
        const int64_t wray = (int64_t)got, ray = ray_begin + wray;
        int q, pi, pj;
        int64_t opix;
        setup_ray(imgs, n_images, bs, ray, q, opix, pi, pj);
        const RayHdr hd = hdr[wray];
        if (hd.status == BL_RAY_OVERFLOW || hd.nrec == 0) continue;
        const ImageDesc& im = imgs[q];
        const T kt = (T)hd.kt, nu_norm = (T)(hd.nnorm * im.freq);
        const T a = ic<T>(im, kcSpin), m = ic<T>(im, kcMass);
        const bool flat = im.flat != 0;
        for (int32_t base = 0; base < hd.nrec; base += 32) {
            const int32_t idx = base + lane;
            if (idx >= hd.nrec) break;
            float* rec = pool + record_index(chunks, wray, idx) * RecStride<float>::v;
            float v[RecStride<float>::v];
            load_record<float>(rec, v);
            const T xs[3] = {v[0], v[1], v[2]};
            KSGeom<T> G;
            ks_geom<T>(xs[0], xs[1], xs[2], a, m, flat, false, G);
            Plasma<T> P;
            uint2 row = make_uint2(0u, 0u);
            if (plasma_at<T, kSlow>(im, xs, v[13], G, P, false)) {
                const T kl[4] = {kt, v[3], v[4], v[5]};
                const T kdu = kl[0] * P.u[0] + kl[1] * P.u[1] + kl[2] * P.u[2] + kl[3] * P.u[3];
                const T kdb = kl[0] * P.b[0] + kl[1] * P.b[1] + kl[2] * P.b[2] + kl[3] * P.b[3];
                const T nu_fl = nu_norm * (-kdu);
                T cth = fq(kdb, (-kdu) * fsqrt(P.bsq));
                cth = cth > T(1) ? T(1) : (cth < T(-1) ? T(-1) : cth);
                const mlp::ModelIn mi = mlp::model_inputs(P.th, P.bg, nu_fl, cth);
                if (mi.ok && P.ne > T(0)) row = mlp::input_row(mi.f);
            }
            *reinterpret_cast<uint2*>(rec + 14) = row;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Adaptive refinement (Sec. 4): per-block criterion and composite assembly.
// ---------------------------------------------------------------------------------------
// Criterion value of pixel (u, v) of a B x B block whose Stokes I is I[v * B + u].
template <class V>
__device__ __forceinline__ double adapt_value(const V* I, int B, int u, int v, int crit) {
    auto at = [&](int uu, int vv) -> double { return (double)I[vv * B + uu]; };
    // differences along one axis at position w of B with the two neighbours of w, one-sided
    // (shifted stencil) at the block edges
    auto d1 = [&](bool along_u, int w) -> double {
        if (B < 2) return 0.0;
        auto val = [&](int k) -> double { return along_u ? at(k, v) : at(u, k); };
        int lo = w - 1, hi = w + 1;
        double num, den;
        if (w == 0) { lo = 0; hi = 1; }
        else if (w == B - 1) { lo = B - 2; hi = B - 1; }
        const bool central = (hi - lo) == 2;
        if (crit == BL_CRIT_ABS_GRAD) {
            num = val(hi) - val(lo);
            return central ? 0.5 * num : num;
        }
        // relative gradient
        num = val(hi) - val(lo);
        den = central ? (val(lo) + 2.0 * val(w) + val(hi)) : 0.5 * (val(lo) + val(hi)) * 2.0;
        return central ? 2.0 * num / den : 2.0 * num / den;
    };
    auto d2 = [&](bool along_u, int w) -> double {
        if (B < 3) return 0.0;
        auto val = [&](int k) -> double { return along_u ? at(k, v) : at(u, k); };
        int c = w;
        if (c == 0) c = 1;
        else if (c == B - 1) c = B - 2;
        const double lap = val(c - 1) - 2.0 * val(c) + val(c + 1);
        if (crit == BL_CRIT_ABS_LAPL) return lap;
        return 4.0 * lap / (val(c - 1) + 2.0 * val(c) + val(c + 1));
    };
    if (crit == BL_CRIT_ABS_GRAD || crit == BL_CRIT_REL_GRAD) {
        const double di = d1(true, u), dj = d1(false, v);
        return sqrt(di * di + dj * dj);
    }
    return fabs(d2(true, u) + d2(false, v));
}

// One thread per block: flags[b] = 1 when at least min_count pixels exceed the threshold.
template <class V>
__global__ void adapt_criterion_kernel(const V* __restrict__ I, int64_t n_blocks, int B, int crit,
                                       double threshold, int min_count, double min_intensity,
                                       int8_t* __restrict__ flags,
                                       const unsigned long long* __restrict__ n_dev = nullptr) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= (n_dev ? (int64_t)*n_dev : n_blocks)) return;
    const V* blk = I + b * (int64_t)B * B;
    int count = 0;
    for (int v = 0; v < B; ++v)
        for (int u = 0; u < B; ++u)
            if ((double)blk[v * B + u] >= min_intensity &&
                adapt_value(blk, B, u, v, crit) > threshold) ++count;   // NaN never counts
    flags[b] = count >= min_count ? 1 : 0;
}

// Output image of one adaptive trace: the finest-level composite, nf x nf per Stokes plane.
struct OutDesc {
    void* stokes;
    int32_t nf, dtype;
};

// Paint the rays of one level (block list bs, Stokes in planes of length cap) into the
// finest-level composites: the ray of level pixel (i, j) covers the s x s finest pixels
// starting at (i s, j s).
template <class V>
__global__ void adapt_composite_kernel(const V* __restrict__ st, int64_t cap, BlockSource bs,
                                       int s, const OutDesc* __restrict__ outs) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t b2 = (int64_t)bs.block * bs.block;
    if (p >= (int64_t)(*bs.count) * b2) return;
    const int64_t blk = p / b2;
    const int r = (int)(p - blk * b2);
    const int q = bs.entries[3 * blk];
    const int i = bs.entries[3 * blk + 1] * bs.block + r % bs.block;
    const int j = bs.entries[3 * blk + 2] * bs.block + r / bs.block;
    const OutDesc o = outs[q];
    const int64_t plane = (int64_t)o.nf * o.nf;
    for (int c = 0; c < 4; ++c) {
        const V v = st[c * cap + p];
        for (int dj = 0; dj < s; ++dj)
            for (int di = 0; di < s; ++di) {
                const int64_t k = c * plane + (int64_t)(j * s + dj) * o.nf + (i * s + di);
                if (o.dtype == 0) ((double*)o.stokes)[k] = (double)v;
                else ((float*)o.stokes)[k] = (float)v;
            }
    }
}

// Children of the refined blocks of one level, in parent order (each parent (q, bx, by) gives
// (q, 2 bx + dx, 2 by + dy), dy then dx), written as the next level's block list; one CTA of
// 1024 threads scans the flags. Blocks beyond the next list's capacity are counted in
// *overflow and not written. per_image[q] accumulates the next level's blocks of image q.
__global__ void __launch_bounds__(1024) adapt_refine_kernel(
        const int8_t* __restrict__ flags, const int32_t* __restrict__ entries,
        const unsigned long long* __restrict__ count, int32_t* __restrict__ next_entries,
        unsigned long long* __restrict__ next_count, unsigned long long cap_next,
        unsigned long long* __restrict__ per_image, unsigned long long* __restrict__ overflow) {
    __shared__ unsigned int warp_tot[32];
    __shared__ unsigned long long base;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t n = (int64_t)*count;
    if (t == 0) base = 0;
    __syncthreads();
    for (int64_t start = 0; start < n; start += 1024) {
        const int64_t b = start + t;
        const bool f = b < n && flags[b] != 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[w] = __popc(m);
        __syncthreads();
        unsigned before = 0, total = 0;
        for (int k = 0; k < 32; ++k) {
            if (k < w) before += warp_tot[k];
            total += warp_tot[k];
        }
        if (f) {
            const unsigned long long out = base + before + __popc(m & ((1u << lane) - 1u));
            if (4 * out + 4 <= cap_next) {
                const int32_t q = entries[3 * b], bx = entries[3 * b + 1], by = entries[3 * b + 2];
                int32_t* dst = next_entries + 12 * out;
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        dst[0] = q; dst[1] = 2 * bx + dx; dst[2] = 2 * by + dy;
                        dst += 3;
                    }
                atomicAdd(&per_image[q], 4ull);
            } else {
                atomicAdd(overflow, 1ull);
            }
        }
        __syncthreads();
        if (t == 0) base += total;
        __syncthreads();
    }
    if (t == 0) *next_count = 4 * base < cap_next ? 4 * base : cap_next / 4 * 4;
}

// ---------------------------------------------------------------------------------------
// Component kernels (checks of single stages against the oracle).
// ---------------------------------------------------------------------------------------
template <class T>
__global__ void coefficients_kernel(int64_t n, const double* __restrict__ in, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T c[8];
    synchrotron_coefficients<T>((T)in[5 * i], (T)in[5 * i + 1], (T)in[5 * i + 2], (T)in[5 * i + 3],
                                (T)in[5 * i + 4], c);
    for (int q = 0; q < 8; ++q) out[8 * i + q] = (double)c[q];
}

template <class T>
__global__ void stokes_step_kernel(int64_t n, const double* __restrict__ coef, const double* __restrict__ s0,
                                   const double* __restrict__ dl, double* __restrict__ s1) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T c[8], a[4], b[4];
    for (int q = 0; q < 8; ++q) c[q] = (T)coef[8 * i + q];
    for (int q = 0; q < 4; ++q) a[q] = (T)s0[4 * i + q];
    stokes_step<T>(c, a, (T)dl[i], b);
    for (int q = 0; q < 4; ++q) s1[4 * i + q] = (double)b[q];
}

template <class T>
__global__ void bessel_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T k0, k1, k2;
    bessel_k012_scaled<T>((T)x[i], k0, k1, k2);
    out[3 * i] = k0;
    out[3 * i + 1] = k1;
    out[3 * i + 2] = k2;
}

}  // namespace bl
