// C ABI of the Blacklight GB300 library: argument checks, workspace layout, launches.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <cstddef>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/blacklight.h"
#include "bl_kernels.cuh"
#include "bl_peak.cuh"

namespace {

thread_local char g_detail[512] = "";
thread_local uint64_t g_launches = 0;
// events around the geodesic and transfer kernels of the last BL_TIMING call on this thread
// BL_TIMING events of the last timed call on this thread: for wave w, [2w] precedes its
// geodesic launch, [2w+1] separates geodesics from transfer, [2w+2] follows the transfer.
thread_local std::vector<cudaEvent_t> g_ev;
thread_local int g_timed_waves = 0;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(BL_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define BL_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Average pool chunks reserved per ray (32 samples each); rays whose samples do not fit are
// reported with status BL_RAY_OVERFLOW.
constexpr int64_t kChunksPerRay = 16;
// Rays are traced in waves of at most this many: the geodesic and transfer kernels run once
// per wave, and the per-ray headers, chunk tables and sample pool are sized for one wave
// (about 33 GiB with float records, 58 GiB with double records), so the workspace stays
// bounded whatever the number of images or pixels.
constexpr int64_t kWaveRays = 1 << 20;

struct Layout {
    size_t counters, descs, hdr, init, chunks, pool, mlp_y, pre, pre_flag, tkey, tnpl, tperm,
        tfirst, thist, pred, total;
    int64_t rays;          // rays of the whole call
    int64_t wave;          // rays per wave (the workspace holds one wave)
    int64_t pool_chunks;
    int64_t pred_blocks;   // blocks of the work-ordered queue (0: the queue is not reordered)
};

// The work-ordered queue's scratch (after the layout's other regions): the predictor's
// counters, image descriptors, 1 x 1 block list, attempt counts, ray headers and initial
// states, the sorted block list and the two list lengths.
struct PredOff {
    size_t ctr, descs, list, cost, hdr, init, sorted, count, end;
};
PredOff pred_offsets(size_t base, int32_t n_images, int64_t nb) {
    PredOff o{};
    size_t off = base;
    o.ctr = off;    off = align_up(off + sizeof(bl::Counters));
    o.descs = off;  off = align_up(off + sizeof(bl::ImageDesc) * (size_t)n_images);
    o.list = off;   off = align_up(off + 3 * sizeof(int32_t) * (size_t)nb);
    o.cost = off;   off = align_up(off + sizeof(int32_t) * (size_t)nb);
    o.hdr = off;    off = align_up(off + sizeof(bl::RayHdr) * (size_t)nb);
    o.init = off;   off = align_up(off + sizeof(bl::RayInit) * (size_t)nb);
    o.sorted = off; off = align_up(off + 3 * sizeof(int32_t) * (size_t)nb);
    o.count = off;  off = align_up(off + 2 * sizeof(unsigned long long));
    o.end = off;
    return o;
}

// The FP64 transfer runs as two passes (fp64_samples_kernel, then the transport and Stokes
// steps) when set; 0 keeps the single fused kernel.
#ifndef BL_TR64_SPLIT
#define BL_TR64_SPLIT 1
#endif
constexpr bool kFp64Split = BL_TR64_SPLIT != 0;


// mlp: room for the learned model's outputs, 8 floats for every record of the pool
Layout make_layout_wave(int32_t n_images, int64_t rays, int64_t wave, int precision,
                        bool transfer, int64_t cpr = kChunksPerRay, bool mlp = false,
                        int64_t pred_blocks = 0) {
    Layout L{};
    L.rays = rays;
    L.pred_blocks = pred_blocks;
    L.wave = wave;
    L.pool_chunks = transfer ? L.wave * cpr : 0;
    const size_t rec = precision != BL_PREC_FP64 ? sizeof(float) * bl::RecStride<float>::v
                                                 : sizeof(double) * bl::RecStride<double>::v;
    size_t off = 0;
    L.counters = off; off = align_up(off + sizeof(bl::Counters));
    L.descs = off;    off = align_up(off + sizeof(bl::ImageDesc) * (size_t)n_images);
    L.hdr = off;      off = align_up(off + sizeof(bl::RayHdr) * (size_t)L.wave);
    L.init = off;     off = align_up(off + sizeof(bl::RayInit) * (size_t)L.wave);
    L.chunks = off;   off = align_up(off + sizeof(int32_t) * bl::kMaxChunks * (size_t)L.wave);
    L.pool = off;     off = align_up(off + rec * bl::kChunk * (size_t)L.pool_chunks);
    L.mlp_y = off;
    if (mlp && transfer) off = align_up(off + 8 * sizeof(float) * bl::kChunk * (size_t)L.pool_chunks);
    // FP64 form: the sample pass's coefficients and basis, and a flag byte, a pool record
    L.pre = off;
    L.pre_flag = off;
    if (precision == BL_PREC_FP64 && transfer && kFp64Split) {
        off = align_up(off + bl::kPreVals * sizeof(double) * bl::kChunk * (size_t)L.pool_chunks);
        L.pre_flag = off;
        off = align_up(off + bl::kChunk * (size_t)L.pool_chunks);
    }
    // the transfer's ray order: each ray's work, the wave's rays longest first, each ray's
    // first transported sample (FP64 transport pass), the histogram of the counting sort
    L.tkey = L.tnpl = L.tperm = L.tfirst = L.thist = off;
    if (transfer) {
        L.tkey = off;   off = align_up(off + sizeof(int32_t) * (size_t)L.wave);
        L.tnpl = off;   off = align_up(off + sizeof(int32_t) * (size_t)L.wave);
        L.tperm = off;  off = align_up(off + sizeof(int32_t) * (size_t)L.wave);
        L.tfirst = off; off = align_up(off + sizeof(int32_t) * (size_t)L.wave);
        L.thist = off;  off = align_up(off + sizeof(unsigned int) * bl::kCostBuckets);
    }
    L.pred = off;
    if (pred_blocks > 0) off = pred_offsets(off, n_images, pred_blocks).end;
    L.total = off;
    return L;
}

Layout make_layout_rays(int32_t n_images, int64_t rays, int precision, bool transfer = true,
                        int64_t cpr = kChunksPerRay, bool mlp = false, int64_t pred_blocks = 0) {
    return make_layout_wave(n_images, rays, rays < kWaveRays ? rays : kWaveRays, precision,
                            transfer, cpr, mlp, pred_blocks);
}

// The largest wave (>= 1 ray) whose layout fits in `bytes`; wave = 0 if none does.
Layout fit_layout(int32_t n_images, int64_t rays, int precision, bool transfer, size_t bytes,
                  int64_t cpr, bool mlp = false, int64_t pred_blocks = 0) {
    Layout L = make_layout_rays(n_images, rays, precision, transfer, cpr, mlp, pred_blocks);
    if (L.total <= bytes) return L;
    int64_t lo = 0, hi = L.wave;        // total(lo) fits (or lo = 0), total(hi) does not
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (make_layout_wave(n_images, rays, mid, precision, transfer, cpr, mlp, pred_blocks).total <= bytes) lo = mid;
        else hi = mid;
    }
    return make_layout_wave(n_images, rays, lo, precision, transfer, cpr, mlp, pred_blocks);
}

int64_t count_rays(int32_t n_images, const bl_camera_t* cams) {
    int64_t rays = 0;
    for (int q = 0; q < n_images; ++q) rays += (int64_t)cams[q].n * cams[q].n;
    return rays;
}

// Average record chunks to reserve per ray. The adaptive DP integrator records a few hundred
// samples per ray; the fixed-rule RK integrators take about 2 ln(r_cam / r_hor) / f_step steps
// on a ray that passes the hole and leaves again, one sample each.
int64_t chunks_per_ray(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets) {
    int64_t c = kChunksPerRay;
    for (int q = 0; q < n_images; ++q) {
        if (mets[q].integrator == BL_INT_DP || !(mets[q].f_step > 0.0)) continue;
        const double a = mets[q].spin / mets[q].mass;
        const double r_hor = mets[q].mass * (1.0 + std::sqrt(std::fmax(1.0 - a * a, 0.0)));
        const double recs = 2.5 * std::log(std::fmax(cams[q].r / r_hor, 2.0)) / mets[q].f_step + 128.0;
        const int64_t need = (int64_t)std::ceil(recs / bl::kChunk) + 1;
        if (need > c) c = need;
    }
    return c < bl::kMaxChunks ? c : bl::kMaxChunks;
}

// Blocks of the work-ordered queue for a batch, or 0 where it is not used: DP integration
// (the fixed-step integrators' work hardly varies), every image's n a multiple of the block
// size, at least kCostMinRays rays (below that the prediction's own latency, about that of
// the longest predicted ray, is not repaid), and grids in the cell layout where the batch has
// grids (grids = nullptr: sized as if it does). The queue mixes the images' blocks; with
// several plane-layout grids in use at once their 64 scalar gathers a sample miss L2 more
// (fast form, nine images: transfer 25.7 -> 38.8 ms), so such batches keep the consecutive
// queue.
constexpr int64_t kCostMinRays = 1 << 16;
int64_t cost_blocks(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                    const bl_grid_t* grids = nullptr) {
    if (mets[0].integrator != BL_INT_DP) return 0;
    if (grids)
        for (int q = 0; q < n_images; ++q)
            if (grids[q].layout != BL_GRID_CELLS) return 0;
    for (int q = 0; q < n_images; ++q)
        if (cams[q].n % bl::kCostBlock) return 0;
    const int64_t rays = count_rays(n_images, cams);
    return rays >= kCostMinRays ? rays / ((int64_t)bl::kCostBlock * bl::kCostBlock) : 0;
}

Layout make_layout(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                   bool mlp = false) {
    return make_layout_rays(n_images, count_rays(n_images, cams), mets[0].precision, true,
                            chunks_per_ray(n_images, cams, mets), mlp,
                            cost_blocks(n_images, cams, mets));
}

int check_camera(const bl_camera_t* c, int q) {
    if (!c) return fail(BL_EINVAL, "cams[%d] is NULL", q);
    if (c->size != sizeof(bl_camera_t)) return fail(BL_EINVAL, "cams[%d].size mismatch", q);
    if (!(c->n >= 1 && c->n <= 65536)) return fail(BL_EINVAL, "cams[%d].n out of range", q);
    if (!(c->width > 0.0) || !std::isfinite(c->width)) return fail(BL_EINVAL, "cams[%d].width", q);
    if (!(c->r > 0.0) || !std::isfinite(c->r)) return fail(BL_EINVAL, "cams[%d].r", q);
    if (!std::isfinite(c->theta) || !std::isfinite(c->phi) || !std::isfinite(c->psi))
        return fail(BL_EINVAL, "cams[%d] angles", q);
    if (c->kind != 0) return fail(BL_EUNSUPPORTED, "cams[%d].kind: only plane-parallel", q);
    if (c->k_p[0] == 0.0 && c->k_p[1] == 0.0 && c->k_p[2] == 0.0)
        return fail(BL_EINVAL, "cams[%d].k_p is zero", q);
    return 0;
}

int check_metric(const bl_metric_t* m, int q) {
    if (!m) return fail(BL_EINVAL, "mets[%d] is NULL", q);
    if (m->size != sizeof(bl_metric_t)) return fail(BL_EINVAL, "mets[%d].size mismatch", q);
    if (!(m->mass > 0.0)) return fail(BL_EINVAL, "mets[%d].mass must be > 0", q);
    if (!(std::fabs(m->spin) < m->mass)) return fail(BL_EINVAL, "mets[%d].spin: need |a| < M", q);
    if (!(m->r_in_over_rhor > 1.0)) return fail(BL_EINVAL, "mets[%d].r_in_over_rhor must be > 1", q);
    if (!(m->tol_abs > 0.0) || !(m->tol_rel > 0.0)) return fail(BL_EINVAL, "mets[%d] tolerances", q);
    if (!(m->ds_max > 0.0)) return fail(BL_EINVAL, "mets[%d].ds_max must be > 0", q);
    if (!(m->h0_frac > 0.0)) return fail(BL_EINVAL, "mets[%d].h0_frac must be > 0", q);
    if (!(m->max_steps > 0)) return fail(BL_EINVAL, "mets[%d].max_steps must be > 0", q);
    if (m->precision != BL_PREC_FP64 && m->precision != BL_PREC_MIXED &&
        m->precision != BL_PREC_FAST)
        return fail(BL_EINVAL, "mets[%d].precision", q);
    if (m->integrator != BL_INT_DP && m->integrator != BL_INT_RK4 && m->integrator != BL_INT_RK2)
        return fail(BL_EINVAL, "mets[%d].integrator", q);
    if (m->integrator != BL_INT_DP && !(m->f_step > 0.0 && m->f_step < 1.0))
        return fail(BL_EINVAL, "mets[%d].f_step must be in (0, 1)", q);
    return 0;
}

int check_grid(const bl_grid_t* g, int q) {
    if (!g) return fail(BL_EINVAL, "grids[%d] is NULL", q);
    if (g->size != sizeof(bl_grid_t)) return fail(BL_EINVAL, "grids[%d].size mismatch", q);
    if (!g->prim) return fail(BL_EINVAL, "grids[%d].prim is NULL", q);
    if (g->n_r < 1 || g->n_theta < 1 || g->n_phi < 1) return fail(BL_EINVAL, "grids[%d] dims", q);
    if (!(g->r_min > 0.0) || !(g->r_max > g->r_min)) return fail(BL_EINVAL, "grids[%d] r range", q);
    if (!(g->gamma_ad > 1.0)) return fail(BL_EINVAL, "grids[%d].gamma_ad", q);
    if (!(g->mu > 0.0) || !(g->ne_over_ni > 0.0)) return fail(BL_EINVAL, "grids[%d] composition", q);
    if (!(g->rho_unit_cgs > 0.0) || !(g->mass_msun > 0.0)) return fail(BL_EINVAL, "grids[%d] units", q);
    if (g->interp != 0 && g->interp != 1) return fail(BL_EINVAL, "grids[%d].interp", q);
    if (g->layout != BL_GRID_PLANES && g->layout != BL_GRID_CELLS)
        return fail(BL_EINVAL, "grids[%d].layout", q);
    if (g->layout == BL_GRID_CELLS && ((uintptr_t)g->prim & 15u) != 0)
        return fail(BL_EINVAL, "grids[%d].prim must be 16-byte aligned for BL_GRID_CELLS", q);
    if (g->n_snapshots > 1) {
        if (!(g->dt_snapshots > 0.0) || !std::isfinite(g->dt_snapshots) ||
            !std::isfinite(g->t_first) || !std::isfinite(g->t_camera))
            return fail(BL_EINVAL, "grids[%d]: slow light needs dt_snapshots > 0 and finite times", q);
        if (g->time_interp != 0 && g->time_interp != 1)
            return fail(BL_EINVAL, "grids[%d].time_interp", q);
    } else if (g->n_snapshots < 0) {
        return fail(BL_EINVAL, "grids[%d].n_snapshots < 0", q);
    }
    return 0;
}

int check_out(const bl_out_t* o, int q, bool need_stokes) {
    if (!o) return fail(BL_EINVAL, "outs[%d] is NULL", q);
    if (o->size != sizeof(bl_out_t)) return fail(BL_EINVAL, "outs[%d].size mismatch", q);
    if (need_stokes && !o->stokes) return fail(BL_EINVAL, "outs[%d].stokes is NULL", q);
    if (o->dtype != 0 && o->dtype != 1) return fail(BL_EINVAL, "outs[%d].dtype", q);
    return 0;
}

int device_pointer(const void* p, const char* what) {
    if (!p) return 0;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BL_EINVAL, "%s is not a CUDA pointer", what);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(BL_EINVAL, "%s must be device memory", what);
    int dev = 0;
    cudaGetDevice(&dev);
    if (at.device != dev) return fail(BL_EINVAL, "%s is on device %d, current is %d", what, at.device, dev);
    return 0;
}

void fill_desc(bl::ImageDesc& d, const bl_camera_t& c, const bl_metric_t& m, const bl_grid_t& g,
               double freq, const bl_out_t& o, int64_t offset) {
    memset(&d, 0, sizeof(d));
    d.cam_r = c.r; d.cam_th = c.theta; d.cam_ph = c.phi;
    for (int i = 0; i < 3; ++i) { d.u_p[i] = c.u_p[i]; d.k_p[i] = c.k_p[i]; }
    d.width = c.width; d.psi = c.psi; d.n = c.n; d.nu_inf = c.nu_at_infinity;
    d.mass = m.mass; d.spin = m.spin; d.r_in_over_rhor = m.r_in_over_rhor;
    d.tol_abs = m.tol_abs; d.tol_rel = m.tol_rel; d.ds_max = m.ds_max; d.h0_frac = m.h0_frac;
    d.max_steps = m.max_steps; d.flat = m.flat; d.precision = m.precision;
    d.integrator = m.integrator; d.f_step = m.f_step;
    d.prim = g.prim; d.nr = g.n_r; d.nt = g.n_theta; d.nph = g.n_phi; d.interp = g.interp;
    d.layout = g.layout;
    d.r_min = g.r_min; d.r_max = g.r_max; d.gamma_ad = g.gamma_ad; d.r_high = g.r_high;
    d.r_low = g.r_low; d.mu = g.mu; d.ne_ni = g.ne_over_ni; d.sigma_cut = g.sigma_cut;
    d.rho_unit = g.rho_unit_cgs;
    d.n_snap = g.n_snapshots > 1 ? g.n_snapshots : 1;
    d.time_interp = g.time_interp;
    d.t_rel0 = g.t_first - g.t_camera;
    d.dt_snap = g.n_snapshots > 1 ? g.dt_snapshots : 1.0;
    d.length_unit = bl::kG * g.mass_msun * bl::kMsun / (bl::kC * bl::kC);
    d.freq = freq;
    {
        double* c = d.d_c;
        c[bl::kcGam1] = g.gamma_ad - 1.0;
        c[bl::kcTePre] = g.mu * bl::kMp / bl::kMe;
        c[bl::kcNePre] = g.rho_unit_cgs / (g.mu * bl::kMp);
        c[bl::kcBgPre] = bl::kC * std::sqrt(4.0 * bl::kPi * g.rho_unit_cgs);
        c[bl::kcDlr] = std::log(g.r_max / g.r_min) / g.n_r;
        c[bl::kcLogRmin] = std::log(g.r_min);
        c[bl::kcRmin] = g.r_min;
        c[bl::kcRmax] = g.r_max;
        c[bl::kcSigma] = g.sigma_cut;
        c[bl::kcRhigh] = g.r_high;
        c[bl::kcRlow] = g.r_low;
        c[bl::kcNeNi] = g.ne_over_ni;
        c[bl::kcFreq] = freq;
        c[bl::kcLen] = d.length_unit;
        c[bl::kcSpin] = m.spin;
        c[bl::kcMass] = m.mass;
        c[bl::kcIDlr] = 1.0 / c[bl::kcDlr];
        c[bl::kcNeFac] = c[bl::kcNePre] / (1.0 + 1.0 / g.ne_over_ni);
        static_assert(bl::kcCount <= 20, "per-image constants");
        for (int i = 0; i < bl::kcCount; ++i) d.f_c[i] = (float)c[i];
    }
    d.stokes = o.stokes; d.dtype = o.dtype; d.status = o.status; d.steps = o.steps;
    d.end_state = o.end_state;
    d.samples = o.samples;
    d.aux = o.aux;
    d.ray_offset = offset;
    d.n_rays = (int64_t)c.n * c.n;
    d.ilv = 0;
    d.ilv_shift = bl::kIlvShift;
}

// Queue the rays of a batch of equal images interleaved (see setup_ray) when every image has
// the same number of rays, a whole number of kIlvBlock-ray blocks, at consecutive offsets, and
// its grid (if any) in the cell layout. Grids in the plane layout keep the consecutive queue:
// their 64 scalar gathers a sample, spread over three grids at once, missed L2 enough to
// outweigh the shorter tail (transfer 27.6 -> 40.9 ms on the 9-image step). Scheduling only:
// each ray's result is the same in either queue order.
bool set_interleave(std::vector<bl::ImageDesc>& d, int shift = bl::kIlvShift) {
    const size_t n = d.size();
    const int64_t blk = int64_t(1) << shift;
    bool eq = n > 1 && d[0].n_rays > 0 && d[0].n_rays % blk == 0;
    for (size_t q = 0; q < n && eq; ++q)
        eq = d[q].n_rays == d[0].n_rays && d[q].ray_offset == (int64_t)q * d[0].n_rays &&
             (d[q].prim == nullptr || d[q].layout == BL_GRID_CELLS);
    for (auto& x : d) {
        x.ilv = eq ? (int32_t)n : 0;
        x.ilv_shift = shift;
    }
    return eq;
}

// Dynamic shared memory of a mixed- or double-float-form geodesic CTA: the stage derivatives,
// 7 stages x 7 components (k_t's are zero) of 8 bytes for each of its 128 threads. The FP64
// form keeps them in local memory and takes no dynamic shared memory.
constexpr size_t kGeoSmem = (size_t)7 * 7 * 128 * 8;

struct DevInfo {
    int sms = 0;
    int geo_blocks[3] = {0, 0, 0};  // per SM, indexed by precision: [fp64, mixed, fast]
    int tr_occ[2][8] = {};          // transfer variants: [double, float][feature bits]
    int tr_mlp_occ[2] = {0, 0};     // learned-coefficient transfer: [fast light, slow light]
    int mi_occ[2] = {0, 0};         // learned-coefficient model inputs: [fast, slow light]
    int pre_occ[2] = {0, 0};        // FP64 sample pass: [fast, slow light]
    int tr_pre_occ[2] = {0, 0};     // FP64 transfer after the sample pass: [fast, slow light]
    int fwd_pool_occ = 0;           // the model over the sample pool
    int rk_occ[2] = {0, 0};         // RK2/RK4 geodesic kernel: [double records, float records]
    // CTAs per SM of the transfer variant a launch uses
    int transfer(int precision, const float* mlp, int feat) const {
        if (mlp) return tr_mlp_occ[(feat & bl::kFSlow) ? 1 : 0];
        if (precision == BL_PREC_FP64 && kFp64Split && !(feat & (bl::kFUnpol | bl::kFAux)))
            return tr_pre_occ[(feat & bl::kFSlow) ? 1 : 0];
        return tr_occ[precision == BL_PREC_FP64 ? 0 : 1][feat & 7];
    }
};

template <class T, class R, int F>
int occ_transfer(int* out) {
    if constexpr (std::is_same<T, double>::value) {
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bl::transfer_kernel_fp64<F>,
                                                              bl::kTransferFp64Threads, 0));
    } else {
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bl::transfer_kernel<T, R, F>, 128, 0));
    }
    if (*out < 1) *out = 1;
    return 0;
}

template <class T, class R>
int occ_transfer_all(int out[8]) {
    int rc = 0;
    if (!rc) rc = occ_transfer<T, R, 0>(&out[0]);
    if (!rc) rc = occ_transfer<T, R, 1>(&out[1]);
    if (!rc) rc = occ_transfer<T, R, 2>(&out[2]);
    if (!rc) rc = occ_transfer<T, R, 3>(&out[3]);
    if (!rc) rc = occ_transfer<T, R, 4>(&out[4]);
    if (!rc) rc = occ_transfer<T, R, 5>(&out[5]);
    if (!rc) rc = occ_transfer<T, R, 6>(&out[6]);
    if (!rc) rc = occ_transfer<T, R, 7>(&out[7]);
    return rc;
}

int dev_info(DevInfo& out) {
    static std::mutex mu;
    static std::vector<DevInfo> cache;
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1);
    DevInfo& di = cache[dev];
    if (di.sms == 0) {
        BL_CUDA(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
        // the stage derivatives exceed the default 48 KB of shared memory
        BL_CUDA(cudaFuncSetAttribute(bl::geodesic_kernel<float, double>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGeoSmem));
        BL_CUDA(cudaFuncSetAttribute(bl::geodesic_kernel<float, bl::df64>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGeoSmem));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.geo_blocks[0], bl::geodesic_kernel_fp64, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.geo_blocks[1], bl::geodesic_kernel<float, double>, 128, kGeoSmem));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.geo_blocks[2], bl::geodesic_kernel<float, bl::df64>, 128, kGeoSmem));
        for (int i = 0; i < 3; ++i)
            if (di.geo_blocks[i] < 1) di.geo_blocks[i] = 1;
        int rc = occ_transfer_all<double, double>(di.tr_occ[0]);
        if (!rc) rc = occ_transfer_all<float, float>(di.tr_occ[1]);
        if (rc) { di.sms = 0; return rc; }
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.tr_mlp_occ[0], bl::transfer_learned_kernel<false>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.tr_mlp_occ[1], bl::transfer_learned_kernel<true>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.mi_occ[0], bl::mlp_inputs_kernel<false>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.mi_occ[1], bl::mlp_inputs_kernel<true>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.fwd_pool_occ, bl::mlp::forward_pool_kernel, 128, 0));
        for (int i = 0; i < 2; ++i)
            if (di.mi_occ[i] < 1) di.mi_occ[i] = 1;
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.pre_occ[0], bl::fp64_samples_kernel<false>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.pre_occ[1], bl::fp64_samples_kernel<true>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.tr_pre_occ[0], bl::transport_fp64_kernel, bl::kTransferFp64Threads, 0));
        di.tr_pre_occ[1] = di.tr_pre_occ[0];
        for (int i = 0; i < 2; ++i) {
            if (di.pre_occ[i] < 1) di.pre_occ[i] = 1;
            if (di.tr_pre_occ[i] < 1) di.tr_pre_occ[i] = 1;
        }
        if (di.fwd_pool_occ < 1) di.fwd_pool_occ = 1;
        for (int i = 0; i < 2; ++i)
            if (di.tr_mlp_occ[i] < 1) di.tr_mlp_occ[i] = 1;
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.rk_occ[0], bl::geodesic_rk_kernel<double>, 128, 0));
        BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.rk_occ[1], bl::geodesic_rk_kernel<float>, 128, 0));
        for (int i = 0; i < 2; ++i)
            if (di.rk_occ[i] < 1) di.rk_occ[i] = 1;
    }
    out = di;
    return 0;
}

// One launch of the transfer variant with feature bits F (grid: CTAs; the FP64 kernel runs
// CTAs of kTransferFp64Threads threads).
template <class T, class R>
void launch_transfer(int feat, unsigned grid, cudaStream_t st, const bl::ImageDesc* d, int n,
                     int64_t b, int64_t e, const bl::RayHdr* hdr, const R* pool,
                     const int32_t* chunks, bl::Counters* ctr, bl::BlockSource bs,
                     bl::SideIn side = bl::SideIn{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}) {
    if constexpr (std::is_same<T, double>::value) {
        constexpr int th = bl::kTransferFp64Threads;
        switch (feat & 7) {
            case 0: bl::transfer_kernel_fp64<0><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 1: bl::transfer_kernel_fp64<1><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 2: bl::transfer_kernel_fp64<2><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 3: bl::transfer_kernel_fp64<3><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 4: bl::transfer_kernel_fp64<4><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 5: bl::transfer_kernel_fp64<5><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 6: bl::transfer_kernel_fp64<6><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            default: bl::transfer_kernel_fp64<7><<<grid, th, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
        }
    } else {
        if (feat & bl::kFMlp) {
            if constexpr (std::is_same<R, float>::value) {
                if (feat & bl::kFSlow)
                    bl::transfer_learned_kernel<true><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side);
                else
                    bl::transfer_learned_kernel<false><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side);
            }
            return;
        }
        switch (feat & 7) {
            case 0: bl::transfer_kernel<T, R, 0><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 1: bl::transfer_kernel<T, R, 1><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 2: bl::transfer_kernel<T, R, 2><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 3: bl::transfer_kernel<T, R, 3><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 4: bl::transfer_kernel<T, R, 4><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 5: bl::transfer_kernel<T, R, 5><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            case 6: bl::transfer_kernel<T, R, 6><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
            default: bl::transfer_kernel<T, R, 7><<<grid, 128, 0, st>>>(d, n, b, e, hdr, pool, chunks, ctr, bs, side); break;
        }
    }
}

// Launch shape of the persistent kernels: CTAs per SM (0 = the occupancy limit).
struct LaunchCfg {
    int geo_ctas = 0, tr_ctas = 0;
    int feat = 0;           // transfer variant: bl::kFSlow | kFUnpol | kFAux
    int integrator = BL_INT_DP;
    bool keep_bad = false;  // leave the bad-ray count of earlier launches in place
    bl::BlockSource bs{nullptr, nullptr, 0, 0};   // rays from a device block list (adaptive)
    cudaEvent_t gate = nullptr;   // the first transfer launch waits for it (grids still arriving)
    bool cost_order = true;       // work-ordered queue where the layout has room for it
    // the fused transfer's record-count order; off where a grid is in the plane layout (the
    // order mixes images, whose 64 scalar gathers a sample then miss L2 more: fast form on nine
    // plane-layout images, transfer 25.8 -> 32.5 ms)
    bool order_transfer = true;
};

// Every image's grid in the cell layout.
bool all_cells(const bl::ImageDesc* d, size_t n) {
    for (size_t q = 0; q < n; ++q)
        if (d[q].layout != BL_GRID_CELLS) return false;
    return true;
}

// The kernel sequence of one trace on prepared workspace whose image descriptors are already
// on the device: counter reset, camera frames, then one geodesic + transfer pair per wave of
// rays, in stream order (the part a plan captures in a CUDA graph).
int launch_kernels(int32_t n_images, char* ws, const Layout& L, int precision, bool transfer,
                   cudaStream_t st, bool timing, const float* mlp, const LaunchCfg& cfg_in) {
    DevInfo di;
    int rc = dev_info(di);
    if (rc) return rc;
    const int64_t n_waves = L.wave > 0 ? (L.rays + L.wave - 1) / L.wave : 0;
    if (timing) {
        while ((int64_t)g_ev.size() < 2 * n_waves + 1) {
            cudaEvent_t e = nullptr;
            BL_CUDA(cudaEventCreate(&e));
            g_ev.push_back(e);
        }
    }
    g_timed_waves = 0;
    bl::Counters* ctr = (bl::Counters*)(ws + L.counters);
    bl::ImageDesc* d_desc = (bl::ImageDesc*)(ws + L.descs);
    bl::RayHdr* hdr = (bl::RayHdr*)(ws + L.hdr);
    int32_t* chunks = (int32_t*)(ws + L.chunks);
    BL_CUDA(cudaMemsetAsync(ctr, 0, cfg_in.keep_bad ? offsetof(bl::Counters, bad_rays)
                                                    : sizeof(bl::Counters), st));
    bl::camera_frame_kernel<<<(n_images + 63) / 64, 64, 0, st>>>(d_desc, n_images);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    LaunchCfg cfg = cfg_in;
    if (L.pred_blocks > 0 && cfg.cost_order && !cfg.bs.entries) {
        // work-ordered queue: list the blocks' centre rays, integrate them (double-float
        // geodesics, attempt counts only), sort the blocks by their counts, longest first
        const int64_t nb = L.pred_blocks;
        const PredOff po = pred_offsets(L.pred, n_images, nb);
        bl::Counters* pctr = (bl::Counters*)(ws + po.ctr);
        bl::ImageDesc* pdesc = (bl::ImageDesc*)(ws + po.descs);
        int32_t* plist = (int32_t*)(ws + po.list);
        int32_t* pcost = (int32_t*)(ws + po.cost);
        int32_t* psorted = (int32_t*)(ws + po.sorted);
        unsigned long long* pcount = (unsigned long long*)(ws + po.count);
        BL_CUDA(cudaMemsetAsync(pctr, 0, sizeof(bl::Counters), st));
        const int64_t lb = (nb + 255) / 256, lcap = (int64_t)di.sms * 8;
        bl::cost_list_kernel<<<(unsigned)(lb < lcap ? lb : lcap), 256, 0, st>>>(d_desc, n_images, nb,
                                                                                plist, pcount);
        bl::cost_descs_kernel<<<(n_images + 63) / 64, 64, 0, st>>>(
            d_desc, pdesc, n_images, pcost, precision == BL_PREC_FAST ? BL_COST_TOL_SCALE : 1.0);
        const bl::BlockSource pbs{plist, pcount, 1, 0};
        bl::ray_init_kernel<<<(unsigned)(lb < lcap ? lb : lcap), 256, 0, st>>>(
            pdesc, n_images, 0, nb, pbs, (bl::RayInit*)(ws + po.init));
        // few rays: at most one CTA an SM, so each runs at its latency
        const int64_t pg = (nb + 127) / 128, pcap = (int64_t)di.sms * di.geo_blocks[2];
        bl::RecordSink<float> psink{nullptr, nullptr, 0ull, pctr};
        bl::geodesic_kernel<float, bl::df64><<<(unsigned)(pg < pcap ? pg : pcap), 128, kGeoSmem, st>>>(
            pdesc, n_images, 0, nb, (bl::RayHdr*)(ws + po.hdr), psink, 0, pbs,
            (const bl::RayInit*)(ws + po.init));
        bl::cost_sort_kernel<<<1, 1024, 0, st>>>(pcost, plist, nb, psorted, pcount + 1);
        g_launches += 5;
        BL_CUDA(cudaGetLastError());
        cfg.bs = bl::BlockSource{psorted, pcount + 1, bl::kCostBlock, 1};
    }
    const int pidx = precision;
    auto pick = [](int want, int occ) { return want > 0 && want < occ ? want : occ; };
    const unsigned geo_grid = (unsigned)(di.sms * pick(cfg.geo_ctas, di.geo_blocks[pidx]));
    const unsigned tr_grid = (unsigned)(di.sms * pick(cfg.tr_ctas, di.transfer(precision, mlp, cfg.feat)));
    const int record = transfer ? 1 : 0;
    const bool slow = (cfg.feat & bl::kFSlow) != 0;
    for (int64_t w = 0; w < n_waves; ++w) {
        const int64_t b = w * L.wave;
        const int64_t e = b + L.wave < L.rays ? b + L.wave : L.rays;
        // the work and pool counters restart with each wave; bad_rays accumulates
        if (w > 0) BL_CUDA(cudaMemsetAsync(ctr, 0, offsetof(bl::Counters, bad_rays), st));
        if (timing) BL_CUDA(cudaEventRecord(g_ev[2 * w], st));
        if (cfg.integrator != BL_INT_DP) {
            const int ri = precision == BL_PREC_FP64 ? 0 : 1;
            const unsigned rk_grid = (unsigned)(di.sms * pick(cfg.geo_ctas, di.rk_occ[ri]));
            if (precision == BL_PREC_FP64) {
                bl::RecordSink<double> sink{(double*)(ws + L.pool), chunks, (unsigned long long)L.pool_chunks, ctr};
                bl::geodesic_rk_kernel<double><<<rk_grid, 128, 0, st>>>(d_desc, n_images, b, e, hdr, sink, record, cfg.bs);
            } else {
                bl::RecordSink<float> sink{(float*)(ws + L.pool), chunks, (unsigned long long)L.pool_chunks, ctr};
                bl::geodesic_rk_kernel<float><<<rk_grid, 128, 0, st>>>(d_desc, n_images, b, e, hdr, sink, record, cfg.bs);
            }
        } else {
            // double-float form: the wave's pixel initial states first, then the integrator
            bl::RayInit* init = (bl::RayInit*)(ws + L.init);
            if (precision == BL_PREC_FAST) {
                const int64_t wn = e - b;
                const int64_t ib = (wn + 255) / 256, icap = (int64_t)di.sms * 8;
                bl::ray_init_kernel<<<(unsigned)(ib < icap ? (ib > 0 ? ib : 1) : icap), 256, 0, st>>>(
                    d_desc, n_images, b, e, cfg.bs, init);
                ++g_launches;
                BL_CUDA(cudaGetLastError());
            }
            if (precision == BL_PREC_FP64) {
                bl::RecordSink<double> sink{(double*)(ws + L.pool), chunks, (unsigned long long)L.pool_chunks, ctr};
                bl::geodesic_kernel_fp64<<<geo_grid, 128, 0, st>>>(
                    d_desc, n_images, b, e, hdr, sink, record, cfg.bs, init);
            } else {
                bl::RecordSink<float> sink{(float*)(ws + L.pool), chunks, (unsigned long long)L.pool_chunks, ctr};
                if (precision == BL_PREC_MIXED)
                    bl::geodesic_kernel<float, double><<<geo_grid, 128, kGeoSmem, st>>>(
                        d_desc, n_images, b, e, hdr, sink, record, cfg.bs, init);
                else
                    bl::geodesic_kernel<float, bl::df64><<<geo_grid, 128, kGeoSmem, st>>>(
                        d_desc, n_images, b, e, hdr, sink, record, cfg.bs, init);
            }
        }
        ++g_launches;
        BL_CUDA(cudaGetLastError());
        if (timing) BL_CUDA(cudaEventRecord(g_ev[2 * w + 1], st));
        if (transfer) {
            // the geodesic kernel does not read the grids: only the transfer waits for them
            if (w == 0 && cfg.gate) BL_CUDA(cudaStreamWaitEvent(st, cfg.gate, 0));
            const float* fpool = (const float*)(ws + L.pool);
            const double* dpool = (const double*)(ws + L.pool);
            int32_t* tkey = (int32_t*)(ws + L.tkey);
            int32_t* tperm = (int32_t*)(ws + L.tperm);
            unsigned int* thist = (unsigned int*)(ws + L.thist);
            const int64_t sb = (e - b + 255) / 256, scap = (int64_t)di.sms * 8;
            const unsigned sgrid = (unsigned)(sb < scap ? (sb > 0 ? sb : 1) : scap);
            // the fused transfer's ray order: by the records each ray's transfer processes,
            // longest first (a counting sort)
            auto order_by_records = [&]() -> int {
                BL_CUDA(cudaMemsetAsync(thist, 0, sizeof(unsigned int) * bl::kCostBuckets, st));
                bl::record_key_kernel<<<sgrid, 256, 0, st>>>(hdr, cfg.bs, b, e, tkey, thist);
                bl::work_scan_kernel<<<1, 1024, 0, st>>>(thist);
                bl::work_scatter_kernel<bl::kFusedGroup><<<sgrid, 256, 0, st>>>(tkey, cfg.bs, b, e, thist, tperm);
                g_launches += 3;
                BL_CUDA(cudaGetLastError());
                return 0;
            };
            if (mlp) {
                // learned coefficients in three passes: the model inputs of every record, the
                // model over the record pool in full tensor-core tiles, then the transfer
                // reading the model's outputs
                float* mpool = (float*)(ws + L.pool);
                float* my = (float*)(ws + L.mlp_y);
                const unsigned mi_grid = (unsigned)(di.sms * di.mi_occ[slow ? 1 : 0]);
                if (slow)
                    bl::mlp_inputs_kernel<true><<<mi_grid, 128, 0, st>>>(
                        d_desc, n_images, b, e, hdr, mpool, chunks, ctr, cfg.bs);
                else
                    bl::mlp_inputs_kernel<false><<<mi_grid, 128, 0, st>>>(
                        d_desc, n_images, b, e, hdr, mpool, chunks, ctr, cfg.bs);
                ++g_launches;
                BL_CUDA(cudaGetLastError());
                bl::mlp::forward_pool_kernel<<<(unsigned)(di.sms * di.fwd_pool_occ), 128, 0, st>>>(
                    mlp, fpool, &ctr->pool_next, (unsigned long long)L.pool_chunks, my,
                    &ctr->mlp_timeouts);
                ++g_launches;
                BL_CUDA(cudaGetLastError());
                if (cfg.order_transfer && (rc = order_by_records())) return rc;
                launch_transfer<float, float>(cfg.feat | bl::kFMlp, tr_grid, st, d_desc, n_images, b,
                                              e, hdr, fpool, chunks, ctr, cfg.bs,
                                              bl::SideIn{my, mlp, nullptr, nullptr, nullptr,
                                                         cfg.order_transfer ? tperm : nullptr});
            } else if (precision != BL_PREC_FP64) {
                if (cfg.order_transfer && (rc = order_by_records())) return rc;
                launch_transfer<float, float>(cfg.feat, tr_grid, st, d_desc, n_images, b, e, hdr,
                                              fpool, chunks, ctr, cfg.bs,
                                              bl::SideIn{nullptr, nullptr, nullptr, nullptr, nullptr,
                                                         cfg.order_transfer ? tperm : nullptr});
            } else if (kFp64Split && !(cfg.feat & (bl::kFUnpol | bl::kFAux))) {
                // FP64 in two passes: the sample pass, then transport and Stokes steps
                // then the transport pass takes the wave's rays longest first (a counting sort
                // of the sample pass's work estimates)
                double* pre = (double*)(ws + L.pre);
                unsigned char* pflag = (unsigned char*)(ws + L.pre_flag);
                int32_t* tfirst = (int32_t*)(ws + L.tfirst);
                int32_t* tnpl = (int32_t*)(ws + L.tnpl);
                // per wave ray: farthest plasma sample -1 and no plasma samples until found
                BL_CUDA(cudaMemsetAsync(tfirst, 0xff, sizeof(int32_t) * (size_t)(e - b), st));
                BL_CUDA(cudaMemsetAsync(tnpl, 0, sizeof(int32_t) * (size_t)(e - b), st));
                BL_CUDA(cudaMemsetAsync(thist, 0, sizeof(unsigned int) * bl::kCostBuckets, st));
                const unsigned pre_grid = (unsigned)(di.sms * di.pre_occ[slow ? 1 : 0]);
                if (slow)
                    bl::fp64_samples_kernel<true><<<pre_grid, 128, 0, st>>>(
                        d_desc, n_images, b, e, hdr, dpool, chunks, ctr, cfg.bs, pre, pflag,
                        tfirst, tnpl);
                else
                    bl::fp64_samples_kernel<false><<<pre_grid, 128, 0, st>>>(
                        d_desc, n_images, b, e, hdr, dpool, chunks, ctr, cfg.bs, pre, pflag,
                        tfirst, tnpl);
                bl::transport_key_kernel<<<sgrid, 256, 0, st>>>(tfirst, tnpl, tkey, cfg.bs, b, e, thist);
                bl::work_scan_kernel<<<1, 1024, 0, st>>>(thist);
                bl::work_scatter_kernel<bl::kTransportGroup><<<sgrid, 256, 0, st>>>(tkey, cfg.bs, b, e, thist, tperm);
                g_launches += 4;
                BL_CUDA(cudaGetLastError());
                bl::transport_fp64_kernel<<<tr_grid, bl::kTransferFp64Threads, 0, st>>>(
                    d_desc, n_images, b, e, hdr, dpool, chunks, ctr, cfg.bs,
                    bl::SideIn{nullptr, nullptr, pre, pflag, tfirst}, tperm);
            } else {
                if (cfg.order_transfer && (rc = order_by_records())) return rc;
                launch_transfer<double, double>(cfg.feat, tr_grid, st, d_desc, n_images, b, e,
                                                hdr, dpool, chunks, ctr, cfg.bs,
                                                bl::SideIn{nullptr, nullptr, nullptr, nullptr, nullptr,
                                                           cfg.order_transfer ? tperm : nullptr});
            }
            ++g_launches;
            BL_CUDA(cudaGetLastError());
        }
        if (timing) BL_CUDA(cudaEventRecord(g_ev[2 * w + 2], st));
    }
    if (timing) g_timed_waves = (int)n_waves;
    return 0;
}

// Upload the image descriptors, then launch_kernels.
int launch_all(int32_t n_images, const std::vector<bl::ImageDesc>& descs, char* ws,
               const Layout& L, int precision, bool transfer, cudaStream_t st, bool timing,
               const float* mlp = nullptr, const LaunchCfg& cfg = LaunchCfg()) {
    BL_CUDA(cudaMemcpyAsync(ws + L.descs, descs.data(), sizeof(bl::ImageDesc) * n_images,
                            cudaMemcpyHostToDevice, st));
    LaunchCfg c = cfg;
    for (const auto& d : descs) {
        if (d.n_snap > 1) c.feat |= bl::kFSlow;
        if (d.aux) c.feat |= bl::kFAux;
    }
    c.integrator = descs.empty() ? BL_INT_DP : descs[0].integrator;
    c.order_transfer = all_cells(descs.data(), descs.size());
    return launch_kernels(n_images, ws, L, precision, transfer, st, timing, mlp, c);
}

int finish(char* ws, const Layout& L, cudaStream_t st, bool sync) {
    if (!sync) return 0;
    bl::Counters c{};
    BL_CUDA(cudaMemcpyAsync(&c, ws + L.counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    BL_CUDA(cudaStreamSynchronize(st));
    if (c.mlp_timeouts)
        return fail(BL_ETIMEOUT, "%llu CTAs stopped: tensor-core wait ran out", c.mlp_timeouts);
    return c.bad_rays ? BL_WRAYS : BL_OK;
}

// The learned-model pointer shared by all images (nullptr: exact fits), checked.
int common_mlp(int32_t n_images, const bl_grid_t* grids, int precision, const float** out,
               uint32_t flags = 0, const bl_out_t* outs = nullptr) {
    *out = nullptr;
    if (!grids) return 0;
    const float* p = grids[0].coef_mlp;
    if (p && (flags & BL_UNPOLARIZED))
        return fail(BL_EUNSUPPORTED, "coef_mlp with BL_UNPOLARIZED");
    if (p && outs)
        for (int q = 0; q < n_images; ++q)
            if (outs[q].aux) return fail(BL_EUNSUPPORTED, "coef_mlp with auxiliary images");
    for (int q = 1; q < n_images; ++q)
        if (grids[q].coef_mlp != p) return fail(BL_EINVAL, "grids[%d].coef_mlp differs from grids[0]", q);
    if (p && precision == BL_PREC_FP64)
        return fail(BL_EUNSUPPORTED, "coef_mlp needs FP32 transfer (BL_PREC_MIXED or BL_PREC_FAST)");
    if (p) {
        int rc = device_pointer(p, "grids[].coef_mlp");
        if (rc) return rc;
    }
    *out = p;
    return 0;
}

int check_batch(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                const bl_grid_t* grids, const double* freqs, const bl_out_t* outs, bool transfer,
                int* precision_out) {
    int precision = -1;
    if (n_images < 1) return fail(BL_EINVAL, "n_images must be >= 1");
    if (!cams || !mets || !outs || (transfer && (!grids || !freqs)))
        return fail(BL_EINVAL, "NULL array argument");
    for (int q = 0; q < n_images; ++q) {
        int rc = check_camera(&cams[q], q);
        if (!rc) rc = check_metric(&mets[q], q);
        if (!rc && transfer) rc = check_grid(&grids[q], q);
        if (!rc) rc = check_out(&outs[q], q, transfer);
        if (rc) return rc;
        if (transfer && !(freqs[q] > 0.0 && std::isfinite(freqs[q])))
            return fail(BL_EINVAL, "freqs[%d] must be > 0", q);
        if (precision < 0) precision = mets[q].precision;
        else if (precision != mets[q].precision)
            return fail(BL_EINVAL, "all images must share metric.precision");
        if (mets[q].integrator != mets[0].integrator)
            return fail(BL_EINVAL, "all images must share metric.integrator");
        char what[64];
        snprintf(what, sizeof(what), "outs[%d].stokes", q);
        if (transfer && (rc = device_pointer(outs[q].stokes, what))) return rc;
        snprintf(what, sizeof(what), "outs[%d].status", q);
        if ((rc = device_pointer(outs[q].status, what))) return rc;
        snprintf(what, sizeof(what), "outs[%d].steps", q);
        if ((rc = device_pointer(outs[q].steps, what))) return rc;
        snprintf(what, sizeof(what), "outs[%d].end_state", q);
        if ((rc = device_pointer(outs[q].end_state, what))) return rc;
        snprintf(what, sizeof(what), "outs[%d].samples", q);
        if ((rc = device_pointer(outs[q].samples, what))) return rc;
        snprintf(what, sizeof(what), "outs[%d].aux", q);
        if ((rc = device_pointer(outs[q].aux, what))) return rc;
        if (!transfer && outs[q].aux)
            return fail(BL_EINVAL, "outs[%d].aux: auxiliary images need the transfer", q);
        snprintf(what, sizeof(what), "grids[%d].prim", q);
        if (transfer && (rc = device_pointer(grids[q].prim, what))) return rc;
    }
    *precision_out = precision;
    return 0;
}

int trace_impl(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
               const bl_grid_t* grids, const double* freqs, const bl_out_t* outs, void* workspace,
               size_t workspace_bytes, void* stream, uint32_t flags, bool transfer,
               cudaEvent_t gate = nullptr) {
    g_detail[0] = 0;
    int precision = -1;
    {
        int rc = check_batch(n_images, cams, mets, grids, freqs, outs, transfer, &precision);
        if (rc) return rc;
    }
    // geodesics only: no records, so no pool
    const int64_t rays = count_rays(n_images, cams);
    const int64_t cpr = chunks_per_ray(n_images, cams, mets);
    // learned coefficients (validated below) need room for the model's outputs
    const bool use_mlp = transfer && grids && grids[0].coef_mlp != nullptr;
    const int64_t pb = cost_blocks(n_images, cams, mets, transfer ? grids : nullptr);
    Layout L = make_layout_rays(n_images, rays, precision, transfer, cpr, use_mlp, pb);
    std::vector<bl::ImageDesc> descs(n_images);
    int64_t off = 0;
    static const bl_grid_t kNoGrid = {sizeof(bl_grid_t), nullptr, 1, 1, 1, 1.0, 2.0, 4.0 / 3.0,
                                      1.0, 1.0, 0.5, 1.0, 1.0, 1.0, 1.0, 1};
    for (int q = 0; q < n_images; ++q) {
        fill_desc(descs[q], cams[q], mets[q], transfer ? grids[q] : kNoGrid,
                  transfer ? freqs[q] : 1.0, outs[q], off);
        off += (int64_t)cams[q].n * cams[q].n;
    }
    set_interleave(descs);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    bool own = false;
    if (ws) {
        if ((uintptr_t)ws % kAlign)
            return fail(BL_EINVAL, "workspace must be %zu-byte aligned", kAlign);
        // a workspace smaller than the default layout runs the rays in more, smaller waves
        L = fit_layout(n_images, rays, precision, transfer, workspace_bytes, cpr, use_mlp, pb);
        if (L.wave < 1)
            return fail(BL_EINVAL, "workspace too small: %zu < %zu bytes (one ray)",
                        workspace_bytes,
                        make_layout_wave(n_images, rays, 1, precision, transfer, cpr, use_mlp, pb).total);
        int rc = device_pointer(ws, "workspace");
        if (rc) return rc;
    } else {
        cudaError_t e = cudaMallocAsync((void**)&ws, L.total, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(BL_ENOMEM, "cudaMallocAsync(%zu bytes): %s", L.total, cudaGetErrorString(e));
        }
        own = true;
    }
    const float* mlp = nullptr;
    int rc = transfer ? common_mlp(n_images, grids, precision, &mlp, flags, outs) : 0;
    if (rc) {
        if (own) cudaFreeAsync(ws, st);
        return rc;
    }
    LaunchCfg cfg;
    if (flags & BL_UNPOLARIZED) cfg.feat |= bl::kFUnpol;
    cfg.gate = gate;
    rc = launch_all(n_images, descs, ws, L, precision, transfer, st, (flags & BL_TIMING) != 0, mlp,
                    cfg);
    if (rc == 0) rc = finish(ws, L, st, !(flags & BL_ASYNC));
    if (own) {
        cudaError_t e = cudaFreeAsync(ws, st);
        if (rc == 0 && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
    }
    return rc;
}

// ---------------------------------------------------------------------------------------
// Plans: prepared batched traces replayed as CUDA graphs, with an optional autotuner.
// ---------------------------------------------------------------------------------------
struct TuneKey {
    int dev, precision, mlp, n_images;
    int64_t rays;
    bool operator<(const TuneKey& o) const {
        if (dev != o.dev) return dev < o.dev;
        if (precision != o.precision) return precision < o.precision;
        if (mlp != o.mlp) return mlp < o.mlp;
        if (n_images != o.n_images) return n_images < o.n_images;
        return rays < o.rays;
    }
};
struct TuneVal {
    int order, ilv_shift;
    LaunchCfg cfg;
    float ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

}  // namespace

namespace { struct AdaptRun; }

struct bl_plan {
    int dev = 0;
    int32_t n_images = 0;
    int precision = 0;
    const float* mlp = nullptr;
    int feat = 0;            // transfer variant feature bits
    std::vector<bl::ImageDesc> descs;
    Layout L{};
    char* ws = nullptr;
    int order = 0;
    int ilv_shift = bl::kIlvShift;
    LaunchCfg cfg;
    float run_ms = 0.0f;
    int64_t kernels_per_run = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    AdaptRun* adapt = nullptr;   // adaptive plans: the device-driven multi-level sequence
};

namespace {

// order 0: Morton within each image, 1: rows, 2: the work-ordered queue of 8 x 8 blocks
int plan_set_order(bl_plan& P, int order, cudaStream_t st, int ilv_shift = -1) {
    for (auto& d : P.descs) d.order = order == 2 ? 0 : order;
    P.order = order;
    if (ilv_shift >= 0) {
        set_interleave(P.descs, ilv_shift);
        P.ilv_shift = ilv_shift;
    }
    BL_CUDA(cudaMemcpyAsync(P.ws + P.L.descs, P.descs.data(),
                            sizeof(bl::ImageDesc) * P.descs.size(), cudaMemcpyHostToDevice, st));
    return 0;
}

// Device time of one run with the given configuration (best of two, after one warm-up).
int plan_time(bl_plan& P, const LaunchCfg& cfg, cudaStream_t st, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BL_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(ce, "cudaEventCreate"); }
    int rc = 0;
    float best = 1e30f;
    for (int it = 0; it < 3 && rc == 0; ++it) {
        if (it > 0 && (ce = cudaEventRecord(e0, st)) != cudaSuccess) rc = cuda_fail(ce, "record");
        LaunchCfg c = cfg;
        c.feat = P.feat;
        c.integrator = P.descs[0].integrator;
        c.cost_order = P.order == 2;
        c.order_transfer = all_cells(P.descs.data(), P.descs.size());
        if (!rc) rc = launch_kernels(P.n_images, P.ws, P.L, P.precision, true, st, false, P.mlp, c);
        if (!rc && it > 0) {
            if ((ce = cudaEventRecord(e1, st)) != cudaSuccess) rc = cuda_fail(ce, "record");
            else if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(ce, "sync");
            else {
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (t < best) best = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return rc;
}

// Coordinate descent: ray order at the occupancy limits, then geodesic CTAs per SM, then
// transfer CTAs per SM. A candidate replaces the current choice only if it is faster by more
// than kTuneMargin (run-to-run variation of these persistent kernels is about 1-2 %).
constexpr float kTuneMargin = 0.03f;
int plan_autotune(bl_plan& P, cudaStream_t st) {
    DevInfo di;
    int rc = dev_info(di);
    if (rc) return rc;
    const TuneKey key{P.dev, P.precision, P.mlp ? 1 : 0, P.n_images, P.L.rays};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            P.cfg = it->second.cfg;
            P.run_ms = it->second.ms;
            return plan_set_order(P, it->second.order, st, it->second.ilv_shift);
        }
    }
    float best = 0.0f, t = 0.0f;
    LaunchCfg cfg;
    // ray order: the work-ordered queue where the batch allows it, else Morton; then the others
    int order = P.L.pred_blocks > 0 ? 2 : 0;
    int ilv_shift = bl::kIlvShift;
    if ((rc = plan_set_order(P, order, st, ilv_shift)) || (rc = plan_time(P, cfg, st, &best))) return rc;
    for (int o = 0; o < 2; ++o) {
        if (o == order) continue;
        if ((rc = plan_set_order(P, o, st)) || (rc = plan_time(P, cfg, st, &t))) return rc;
        if (t < best * (1.0f - kTuneMargin)) { best = t; order = o; }
    }
    if ((rc = plan_set_order(P, order, st))) return rc;
    // interleave block of a batch of equal images: 64 to 4096 rays (not used by the
    // work-ordered queue)
    if (P.descs[0].ilv > 1 && order != 2) {
        for (int sh = 6; sh <= 12; sh += 2) {
            if (sh == bl::kIlvShift) continue;
            std::vector<bl::ImageDesc> probe = P.descs;
            if (!set_interleave(probe, sh)) continue;
            if ((rc = plan_set_order(P, order, st, sh)) || (rc = plan_time(P, cfg, st, &t))) return rc;
            if (t < best * (1.0f - kTuneMargin)) { best = t; ilv_shift = sh; }
        }
        if ((rc = plan_set_order(P, order, st, ilv_shift))) return rc;
    }
    const int geo_max = di.geo_blocks[P.precision];
    const int tr_max = di.transfer(P.precision, P.mlp, P.feat);
    int geo_best = geo_max;
    for (int c = 1; c < geo_max; ++c) {
        LaunchCfg trial = cfg;
        trial.geo_ctas = c;
        if ((rc = plan_time(P, trial, st, &t))) return rc;
        if (t < best * (1.0f - kTuneMargin)) { best = t; geo_best = c; }
    }
    cfg.geo_ctas = geo_best;
    int tr_best = tr_max;
    for (int c = 1; c < tr_max; ++c) {
        LaunchCfg trial = cfg;
        trial.tr_ctas = c;
        if ((rc = plan_time(P, trial, st, &t))) return rc;
        if (t < best * (1.0f - kTuneMargin)) { best = t; tr_best = c; }
    }
    cfg.tr_ctas = tr_best;
    P.cfg = cfg;
    P.run_ms = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TuneVal{order, P.ilv_shift, cfg, best};
    return 0;
}

int adapt_enqueue(AdaptRun& R, cudaStream_t st);

int plan_capture(bl_plan& P, cudaStream_t user) {
    DevInfo di;                      // occupancy queries happen before, not during, capture
    if (int rc0 = dev_info(di)) return rc0;
    cudaStream_t st = user;
    bool own = false;
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) {
        BL_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    // descriptors must be on the device before the captured kernels first run
    cudaError_t e = cudaStreamSynchronize(user);
    int rc = e == cudaSuccess ? 0 : cuda_fail(e, "cudaStreamSynchronize");
    const uint64_t before = g_launches;
    if (!rc) {
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamBeginCapture");
    }
    if (!rc) {
        if (P.adapt) {
            rc = adapt_enqueue(*P.adapt, st);
        } else {
            LaunchCfg c = P.cfg;
            c.feat = P.feat;
            c.integrator = P.descs[0].integrator;
            c.cost_order = P.order == 2;
            c.order_transfer = all_cells(P.descs.data(), P.descs.size());
            rc = launch_kernels(P.n_images, P.ws, P.L, P.precision, true, st, false, P.mlp, c);
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
        if (!rc) {
            P.graph = g;
            e = cudaGraphInstantiate(&P.exec, P.graph, 0);
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    P.kernels_per_run = (int64_t)(g_launches - before);
    g_launches = before;          // capture launches nothing; runs are counted when replayed
    if (own) cudaStreamDestroy(st);
    return rc;
}

// ---------------------------------------------------------------------------------------
// Fixed scratch for blacklight_trace_noalloc. Some callers cannot allocate device memory
// while they trace -- for example code running inside a memory pool they do not own, or a
// host process whose allocator must not grow after start-up -- so this entry point works in
// a statically sized buffer that lives in the library's device image instead. Every device
// that loads the library holds these 64 MiB until the process exits.
// ---------------------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = 64ull << 20;
constexpr int64_t kNoAllocMaxRays = 1024;     // e.g. one 32x32 image
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The array's name is a host-side stand-in in host code; the device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
int noalloc_scratch(char** out) {
    static std::mutex mu;
    static std::vector<char*> addr;
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        addr[dev] = (char*)p;
    }
    *out = addr[dev];
    return 0;
}

int check_adapt(const bl_adapt_t* ad, const bl_camera_t* cams, int32_t n_images) {
    if (!ad) return fail(BL_EINVAL, "adapt is NULL");
    if (ad->size != sizeof(bl_adapt_t)) return fail(BL_EINVAL, "adapt.size mismatch");
    if (ad->block < 1 || ad->max_level < 0 || ad->max_level > 8 || ad->min_count < 1 ||
        ad->min_count > ad->block * ad->block)
        return fail(BL_EINVAL, "adapt: block >= 1, 0 <= max_level <= 8, 1 <= min_count <= block^2");
    if (ad->criterion < BL_CRIT_ABS_GRAD || ad->criterion > BL_CRIT_REL_LAPL)
        return fail(BL_EINVAL, "adapt.criterion");
    if (!std::isfinite(ad->threshold)) return fail(BL_EINVAL, "adapt.threshold");
    if (!(ad->min_intensity >= 0.0)) return fail(BL_EINVAL, "adapt.min_intensity must be >= 0");
    for (int q = 0; q < n_images; ++q) {
        if (cams[q].n % ad->block) return fail(BL_EINVAL, "cams[%d].n must be a multiple of block", q);
        if ((int64_t)cams[q].n << ad->max_level > 65536)
            return fail(BL_EINVAL, "cams[%d]: n * 2^max_level exceeds 65536", q);
    }
    return 0;
}

// ---------------------------------------------------------------------------------------
// Adaptive tracing (Sec. 4) driven entirely on the device: each level's blocks of all images
// form one device block list (image, bx, by); the persistent kernels take their rays from it,
// the level is painted into the composites, its blocks are judged, and a one-CTA scan writes
// the next level's list. No host round trip between levels, so the whole sequence can be
// captured in a CUDA graph.
// ---------------------------------------------------------------------------------------
constexpr int64_t kMaxAdaptLevelRays = 1ll << 26;   // capacity of one level (67M rays)

struct AdaptRun {
    int32_t n_images = 0, max_level = 0, B = 0, precision = 0, feat = 0;
    const float* mlp = nullptr;
    bl_adapt_t ad{};
    size_t vsize = 4;
    std::vector<int64_t> cap_blocks;        // per level
    int64_t max_cap_rays = 0;
    Layout L{};                             // trace workspace (waves)
    char* mem = nullptr;                    // one allocation for everything below
    size_t mem_bytes = 0;
    char* ws = nullptr;
    bl::ImageDesc* descs = nullptr;         // [levels][n_images]
    std::vector<int32_t*> entries;          // per level
    unsigned long long* counts = nullptr;   // [levels] blocks, then [levels][n_images], overflow
    int8_t* flags = nullptr;
    char* lvl = nullptr;                    // [4][max_cap_rays] compact Stokes
    bl::OutDesc* outd = nullptr;
    // host copies uploaded once
    std::vector<bl::ImageDesc> h_descs;
    std::vector<int32_t> h_root;
    std::vector<unsigned long long> h_counts0;
    std::vector<bl::OutDesc> h_outd;
};

int adapt_prepare(AdaptRun& R, int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                  const bl_grid_t* grids, const double* freqs, const bl_adapt_t* ad,
                  const bl_out_t* outs, const float* mlp, uint32_t flags, cudaStream_t st,
                  bool persistent) {
    R.n_images = n_images;
    R.max_level = ad->max_level;
    R.B = ad->block;
    R.ad = *ad;
    R.precision = mets[0].precision;
    R.mlp = mlp;
    R.vsize = R.precision == BL_PREC_FP64 ? sizeof(double) : sizeof(float);
    if (flags & BL_UNPOLARIZED) R.feat |= bl::kFUnpol;
    for (int q = 0; q < n_images; ++q)
        if (grids[q].n_snapshots > 1) R.feat |= bl::kFSlow;
    const int64_t b2 = (int64_t)R.B * R.B;
    int64_t root = 0;
    for (int q = 0; q < n_images; ++q) root += (int64_t)(cams[q].n / R.B) * (cams[q].n / R.B);
    R.cap_blocks.resize(R.max_level + 1);
    for (int l = 0; l <= R.max_level; ++l) {
        double c = (double)root * std::pow(4.0, l);
        const double lim = (double)(kMaxAdaptLevelRays / b2);
        R.cap_blocks[l] = (int64_t)(c < lim ? c : lim);
        if (R.cap_blocks[l] < root && l == 0) R.cap_blocks[l] = root;
        R.max_cap_rays = std::max(R.max_cap_rays, R.cap_blocks[l] * b2);
    }
    R.L = make_layout_rays(n_images, R.max_cap_rays, R.precision, true,
                           chunks_per_ray(n_images, cams, mets), R.mlp != nullptr);
    // one allocation: trace workspace, descriptors, block lists, counts, flags, Stokes, outputs
    const int levels = R.max_level + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_ws = take(R.L.total);
    const size_t o_desc = take(sizeof(bl::ImageDesc) * levels * n_images);
    std::vector<size_t> o_ent(levels);
    for (int l = 0; l < levels; ++l) o_ent[l] = take(sizeof(int32_t) * 3 * R.cap_blocks[l]);
    const size_t n_counts = levels + (size_t)levels * n_images + 1;
    const size_t o_cnt = take(sizeof(unsigned long long) * n_counts);
    int64_t max_flags = 1;
    for (int l = 0; l < R.max_level; ++l) max_flags = std::max(max_flags, R.cap_blocks[l]);
    const size_t o_flags = take((size_t)max_flags);
    const size_t o_lvl = take(4 * R.vsize * (size_t)R.max_cap_rays);
    const size_t o_out = take(sizeof(bl::OutDesc) * n_images);
    R.mem_bytes = off;
    cudaError_t e = persistent ? cudaMalloc((void**)&R.mem, off)
                               : cudaMallocAsync((void**)&R.mem, off, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        R.mem = nullptr;
        return fail(BL_ENOMEM, "adaptive buffers (%zu bytes): %s", off, cudaGetErrorString(e));
    }
    R.ws = R.mem + o_ws;
    R.descs = (bl::ImageDesc*)(R.mem + o_desc);
    R.entries.resize(levels);
    for (int l = 0; l < levels; ++l) R.entries[l] = (int32_t*)(R.mem + o_ent[l]);
    R.counts = (unsigned long long*)(R.mem + o_cnt);
    R.flags = (int8_t*)(R.mem + o_flags);
    R.lvl = R.mem + o_lvl;
    R.outd = (bl::OutDesc*)(R.mem + o_out);
    // level descriptors: camera at n 2^L, compact Stokes in planes of the level's capacity
    R.h_descs.resize((size_t)levels * n_images);
    for (int l = 0; l < levels; ++l)
        for (int q = 0; q < n_images; ++q) {
            bl_camera_t c = cams[q];
            c.n = cams[q].n << l;
            bl_out_t o{sizeof(bl_out_t), nullptr, R.precision == BL_PREC_FP64 ? 0 : 1, nullptr,
                       nullptr, nullptr, nullptr, nullptr};
            bl::ImageDesc& d = R.h_descs[(size_t)l * n_images + q];
            fill_desc(d, c, mets[q], grids[q], freqs[q], o, 0);
            d.stokes = R.lvl;
            d.n_rays = R.cap_blocks[l] * b2;
        }
    // root block list (image-major, blocks row by row) and level-0 counts
    R.h_root.clear();
    R.h_counts0.assign(n_counts, 0ull);
    R.h_counts0[0] = (unsigned long long)root;
    for (int q = 0; q < n_images; ++q) {
        const int nb = cams[q].n / R.B;
        for (int by = 0; by < nb; ++by)
            for (int bx = 0; bx < nb; ++bx) {
                R.h_root.push_back(q); R.h_root.push_back(bx); R.h_root.push_back(by);
            }
        R.h_counts0[levels + q] = (unsigned long long)nb * nb;
    }
    R.h_outd.resize(n_images);
    for (int q = 0; q < n_images; ++q)
        R.h_outd[q] = bl::OutDesc{outs[q].stokes, cams[q].n << R.max_level, outs[q].dtype};
    BL_CUDA(cudaMemcpyAsync(R.descs, R.h_descs.data(), sizeof(bl::ImageDesc) * R.h_descs.size(),
                            cudaMemcpyHostToDevice, st));
    BL_CUDA(cudaMemcpyAsync(R.entries[0], R.h_root.data(), sizeof(int32_t) * R.h_root.size(),
                            cudaMemcpyHostToDevice, st));
    BL_CUDA(cudaMemcpyAsync(R.outd, R.h_outd.data(), sizeof(bl::OutDesc) * n_images,
                            cudaMemcpyHostToDevice, st));
    // the host vectors must outlive the copies from pageable memory: synchronise
    BL_CUDA(cudaStreamSynchronize(st));
    return 0;
}

// Enqueue one adaptive trace (all levels) on st.
int adapt_enqueue(AdaptRun& R, cudaStream_t st) {
    const int levels = R.max_level + 1;
    const int64_t b2 = (int64_t)R.B * R.B;
    const size_t n_counts = levels + (size_t)levels * R.n_images + 1;
    // counts: level 0 from the host values; the rest zero
    BL_CUDA(cudaMemcpyAsync(R.counts, R.h_counts0.data(), sizeof(unsigned long long) * n_counts,
                            cudaMemcpyHostToDevice, st));
    BL_CUDA(cudaMemsetAsync(R.ws + R.L.counters, 0, sizeof(bl::Counters), st));
    unsigned long long* per_image = R.counts + levels;
    unsigned long long* overflow = R.counts + levels + (size_t)levels * R.n_images;
    for (int l = 0; l < levels; ++l) {
        BL_CUDA(cudaMemcpyAsync(R.ws + R.L.descs, R.descs + (size_t)l * R.n_images,
                                sizeof(bl::ImageDesc) * R.n_images, cudaMemcpyDeviceToDevice, st));
        Layout Ll = R.L;
        Ll.rays = R.cap_blocks[l] * b2;
        LaunchCfg cfg;
        cfg.feat = R.feat;
        cfg.integrator = R.h_descs[0].integrator;
        cfg.keep_bad = true;
        cfg.bs = bl::BlockSource{R.entries[l], R.counts + l, R.B};
        cfg.order_transfer = all_cells(R.h_descs.data(), (size_t)R.n_images);
        int rc = launch_kernels(R.n_images, R.ws, Ll, R.precision, true, st, false, R.mlp, cfg);
        if (rc) return rc;
        const int s = 1 << (R.max_level - l);
        const unsigned grid_r = (unsigned)((Ll.rays + 255) / 256);
        if (R.precision == BL_PREC_FP64)
            bl::adapt_composite_kernel<double><<<grid_r, 256, 0, st>>>((const double*)R.lvl, Ll.rays, cfg.bs, s, R.outd);
        else
            bl::adapt_composite_kernel<float><<<grid_r, 256, 0, st>>>((const float*)R.lvl, Ll.rays, cfg.bs, s, R.outd);
        ++g_launches;
        BL_CUDA(cudaGetLastError());
        if (l == R.max_level) break;
        const unsigned grid_b = (unsigned)((R.cap_blocks[l] + 127) / 128);
        const bl_adapt_t& ad = R.ad;
        if (R.precision == BL_PREC_FP64)
            bl::adapt_criterion_kernel<double><<<grid_b, 128, 0, st>>>((const double*)R.lvl, R.cap_blocks[l], R.B, ad.criterion, ad.threshold, ad.min_count, ad.min_intensity, R.flags, R.counts + l);
        else
            bl::adapt_criterion_kernel<float><<<grid_b, 128, 0, st>>>((const float*)R.lvl, R.cap_blocks[l], R.B, ad.criterion, ad.threshold, ad.min_count, ad.min_intensity, R.flags, R.counts + l);
        bl::adapt_refine_kernel<<<1, 1024, 0, st>>>(R.flags, R.entries[l], R.counts + l,
                                                    R.entries[l + 1], R.counts + l + 1,
                                                    (unsigned long long)R.cap_blocks[l + 1],
                                                    per_image + (size_t)(l + 1) * R.n_images,
                                                    overflow);
        g_launches += 2;
        BL_CUDA(cudaGetLastError());
    }
    return 0;
}

// Read back the level counts and anomalies of the last run (synchronises st).
int adapt_finish(AdaptRun& R, int32_t* level_rays, cudaStream_t st) {
    const int levels = R.max_level + 1;
    const size_t n_counts = levels + (size_t)levels * R.n_images + 1;
    std::vector<unsigned long long> h(n_counts);
    bl::Counters c{};
    BL_CUDA(cudaMemcpyAsync(h.data(), R.counts, sizeof(unsigned long long) * n_counts,
                            cudaMemcpyDeviceToHost, st));
    BL_CUDA(cudaMemcpyAsync(&c, R.ws + R.L.counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    BL_CUDA(cudaStreamSynchronize(st));
    const int64_t b2 = (int64_t)R.B * R.B;
    if (level_rays)
        for (int q = 0; q < R.n_images; ++q)
            for (int l = 0; l < levels; ++l)
                level_rays[q * levels + l] = (int32_t)(h[levels + (size_t)l * R.n_images + q] * b2);
    if (c.mlp_timeouts) return fail(BL_ETIMEOUT, "tensor-core wait ran out in %llu CTAs", c.mlp_timeouts);
    if (h[n_counts - 1])
        return fail(BL_EUNSUPPORTED, "adaptive refinement exceeded a level's capacity of %lld rays",
                    (long long)kMaxAdaptLevelRays);
    return c.bad_rays ? BL_WRAYS : BL_OK;
}

int check_adaptive_args(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                        const bl_grid_t* grids, const double* freqs_hz, const bl_adapt_t* adapt,
                        const bl_out_t* outs, uint32_t flags, int* precision_out,
                        const float** mlp_out) {
    if (n_images < 1) return fail(BL_EINVAL, "n_images must be >= 1");
    if (!cams || !mets || !grids || !freqs_hz || !outs) return fail(BL_EINVAL, "NULL array argument");
    int precision = -1;
    for (int q = 0; q < n_images; ++q) {
        int rc = check_camera(&cams[q], q);
        if (!rc) rc = check_metric(&mets[q], q);
        if (!rc) rc = check_grid(&grids[q], q);
        if (!rc) rc = check_out(&outs[q], q, true);
        if (rc) return rc;
        if (!(freqs_hz[q] > 0.0 && std::isfinite(freqs_hz[q]))) return fail(BL_EINVAL, "freqs[%d] must be > 0", q);
        if (precision < 0) precision = mets[q].precision;
        else if (precision != mets[q].precision) return fail(BL_EINVAL, "all images must share metric.precision");
        char what[64];
        snprintf(what, sizeof(what), "outs[%d].stokes", q);
        if ((rc = device_pointer(outs[q].stokes, what))) return rc;
        snprintf(what, sizeof(what), "grids[%d].prim", q);
        if ((rc = device_pointer(grids[q].prim, what))) return rc;
    }
    int rc = check_adapt(adapt, cams, n_images);
    if (rc) return rc;
    if (flags & ~(uint32_t)BL_UNPOLARIZED) return fail(BL_EINVAL, "adaptive flags: BL_UNPOLARIZED only");
    const float* mlp = nullptr;
    if ((rc = common_mlp(n_images, grids, precision, &mlp, flags))) return rc;
    for (int q = 0; q < n_images; ++q)
        if (mets[q].integrator != mets[0].integrator)
            return fail(BL_EINVAL, "all images must share metric.integrator");
    *precision_out = precision;
    *mlp_out = mlp;
    return 0;
}

int trace_adaptive_impl(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                        const bl_grid_t* grids, const double* freqs, const bl_adapt_t* ad,
                        const bl_out_t* outs, int32_t* level_rays, cudaStream_t st,
                        const float* mlp, uint32_t flags) {
    AdaptRun R;
    int rc = adapt_prepare(R, n_images, cams, mets, grids, freqs, ad, outs, mlp, flags, st, false);
    if (rc) return rc;
    rc = adapt_enqueue(R, st);
    if (!rc) rc = adapt_finish(R, level_rays, st);
    cudaFreeAsync(R.mem, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == 0 && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

}  // namespace

extern "C" {

int blacklight_trace_adaptive(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                              const bl_grid_t* grids, const double* freqs_hz,
                              const bl_adapt_t* adapt, const bl_out_t* outs, int32_t* level_rays,
                              void* stream) {
    g_detail[0] = 0;
    int precision = -1;
    const float* mlp = nullptr;
    int rc = check_adaptive_args(n_images, cams, mets, grids, freqs_hz, adapt, outs, 0,
                                 &precision, &mlp);
    if (rc) return rc;
    return trace_adaptive_impl(n_images, cams, mets, grids, freqs_hz, adapt, outs, level_rays,
                               (cudaStream_t)stream, mlp, 0);
}

int blacklight_adapt_flags(int64_t n_blocks, const double* I, const bl_adapt_t* adapt,
                           int8_t* flags, void* stream) {
    g_detail[0] = 0;
    if (n_blocks < 0 || (n_blocks > 0 && (!I || !flags))) return fail(BL_EINVAL, "bad arguments");
    if (!adapt || adapt->size != sizeof(bl_adapt_t) || adapt->block < 1 || adapt->min_count < 1 ||
        adapt->criterion < BL_CRIT_ABS_GRAD || adapt->criterion > BL_CRIT_REL_LAPL)
        return fail(BL_EINVAL, "adapt");
    if (n_blocks == 0) return 0;
    int rc = device_pointer(I, "I");
    if (!rc) rc = device_pointer(flags, "flags");
    if (rc) return rc;
    bl::adapt_criterion_kernel<double><<<(unsigned)((n_blocks + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        I, n_blocks, adapt->block, adapt->criterion, adapt->threshold, adapt->min_count,
        adapt->min_intensity, flags);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_trace_noalloc(const bl_camera_t* cam, const bl_metric_t* met,
                             const bl_grid_t* grid, double freq_hz, const bl_out_t* out,
                             void* stream, uint32_t flags) {
    g_detail[0] = 0;
    if (!cam || !met) return fail(BL_EINVAL, "NULL argument");
    int rc = check_camera(cam, 0);
    if (!rc) rc = check_metric(met, 0);
    if (rc) return rc;
    const int64_t rays = (int64_t)cam->n * cam->n;
    if (rays > kNoAllocMaxRays)
        return fail(BL_EINVAL, "blacklight_trace_noalloc: %lld rays exceed its fixed scratch "
                    "(at most %lld rays, %zu bytes); use blacklight_trace",
                    (long long)rays, (long long)kNoAllocMaxRays, kNoAllocBytes);
    char* ws = nullptr;
    rc = noalloc_scratch(&ws);
    if (rc) return rc;
    // The counters at the head of the scratch are zeroed on the stream before each launch;
    // the rest is written before it is read, so stale contents from the last call are inert.
    // When one wave of all rays does not fit (long fixed-step RK4/RK2 rays need up to 128
    // record chunks each), trace_impl runs the rays in smaller waves inside the same array.
    // The call always waits for its work: the anomaly counters live in the shared array, and
    // the next call would zero them before an asynchronous caller could read them.
    return trace_impl(1, cam, met, grid, &freq_hz, out, ws, kNoAllocBytes, stream,
                      flags & ~(uint32_t)(BL_TIMING | BL_ASYNC), true);
}

int blacklight_plan_create(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                           const bl_grid_t* grids, const double* freqs_hz, const bl_out_t* outs,
                           const bl_launch_config_t* config, uint32_t flags, void* stream,
                           bl_plan_t** plan) {
    g_detail[0] = 0;
    if (!plan) return fail(BL_EINVAL, "plan is NULL");
    *plan = nullptr;
    int precision = -1;
    int rc = check_batch(n_images, cams, mets, grids, freqs_hz, outs, true, &precision);
    if (rc) return rc;
    if (config && !(flags & BL_PLAN_AUTOTUNE)) {
        if (config->size != sizeof(bl_launch_config_t)) return fail(BL_EINVAL, "config.size mismatch");
        if (config->ray_order < 0 || config->ray_order > 2 || config->geo_ctas_per_sm < 0 ||
            config->tr_ctas_per_sm < 0)
            return fail(BL_EINVAL, "config: ray_order 0, 1 or 2, CTAs per SM >= 0");
        if (config->ray_order == 2 && cost_blocks(n_images, cams, mets, grids) == 0)
            return fail(BL_EINVAL, "config.ray_order 2 needs DP integration, cell-layout grids, "
                                   "every n a multiple of %d and at least %lld rays",
                        bl::kCostBlock, (long long)kCostMinRays);
        const int b = config->ilv_block;
        if (b != 0 && (b < 64 || b > 4096 || (b & (b - 1)) != 0))
            return fail(BL_EINVAL, "config.ilv_block: 0 or a power of two in [64, 4096]");
    }
    const float* mlp = nullptr;
    if ((rc = common_mlp(n_images, grids, precision, &mlp, flags, outs))) return rc;
    bl_plan* P = new bl_plan();
    if (flags & BL_UNPOLARIZED) P->feat |= bl::kFUnpol;
    BL_CUDA(cudaGetDevice(&P->dev));
    P->n_images = n_images;
    P->precision = precision;
    P->mlp = mlp;
    P->L = make_layout_rays(n_images, count_rays(n_images, cams), precision, true,
                            chunks_per_ray(n_images, cams, mets), mlp != nullptr,
                            cost_blocks(n_images, cams, mets, grids));
    P->descs.resize(n_images);
    int64_t off = 0;
    for (int q = 0; q < n_images; ++q) {
        fill_desc(P->descs[q], cams[q], mets[q], grids[q], freqs_hz[q], outs[q], off);
        if (P->descs[q].n_snap > 1) P->feat |= bl::kFSlow;
        if (P->descs[q].aux) P->feat |= bl::kFAux;
        off += (int64_t)cams[q].n * cams[q].n;
    }
    set_interleave(P->descs);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc((void**)&P->ws, P->L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return fail(BL_ENOMEM, "cudaMalloc(%zu bytes): %s", P->L.total, cudaGetErrorString(e));
    }
    if (flags & BL_PLAN_AUTOTUNE) {
        rc = plan_autotune(*P, st);
    } else {
        int sh = bl::kIlvShift;
        if (config) {
            P->cfg.geo_ctas = config->geo_ctas_per_sm;
            P->cfg.tr_ctas = config->tr_ctas_per_sm;
            if (config->ilv_block > 0) {
                sh = 0;
                while ((1 << sh) < config->ilv_block) ++sh;
            }
        }
        rc = plan_set_order(*P, config ? config->ray_order : (P->L.pred_blocks > 0 ? 2 : 0), st, sh);
    }
    if (!rc) rc = plan_capture(*P, st);
    if (rc) {
        blacklight_plan_destroy(P);
        return rc;
    }
    *plan = P;
    return 0;
}

int blacklight_plan_run(bl_plan_t* plan, void* stream) {
    g_detail[0] = 0;
    if (!plan || !plan->exec) return fail(BL_EINVAL, "plan is NULL or not built");
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    if (dev != plan->dev) return fail(BL_EINVAL, "plan belongs to device %d, current is %d", plan->dev, dev);
    BL_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
    g_launches += (uint64_t)plan->kernels_per_run;
    return 0;
}

int blacklight_plan_check(bl_plan_t* plan, void* stream) {
    g_detail[0] = 0;
    if (!plan) return fail(BL_EINVAL, "plan is NULL");
    if (plan->adapt) return adapt_finish(*plan->adapt, nullptr, (cudaStream_t)stream);
    if (!plan->ws) return fail(BL_EINVAL, "plan is not built");
    return finish(plan->ws, plan->L, (cudaStream_t)stream, true);
}

int blacklight_plan_config(const bl_plan_t* plan, bl_launch_config_t* out) {
    g_detail[0] = 0;
    if (!plan || !out || out->size != sizeof(bl_launch_config_t))
        return fail(BL_EINVAL, "plan is NULL or out.size mismatch");
    DevInfo di;
    int rc = dev_info(di);
    if (rc) return rc;
    const int geo_max = di.geo_blocks[plan->precision];
    const int tr_max = di.transfer(plan->precision, plan->mlp, plan->feat);
    out->ray_order = plan->order;
    out->geo_ctas_per_sm = plan->cfg.geo_ctas > 0 && plan->cfg.geo_ctas < geo_max ? plan->cfg.geo_ctas : geo_max;
    out->tr_ctas_per_sm = plan->cfg.tr_ctas > 0 && plan->cfg.tr_ctas < tr_max ? plan->cfg.tr_ctas : tr_max;
    out->run_ms = plan->run_ms;
    out->ilv_block = plan->descs[0].ilv > 1 && plan->order != 2 ? (1 << plan->descs[0].ilv_shift) : 0;
    return 0;
}

int blacklight_plan_destroy(bl_plan_t* plan) {
    if (!plan) return 0;
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->ws) cudaFree(plan->ws);
    if (plan->adapt) {
        if (plan->adapt->mem) cudaFree(plan->adapt->mem);
        delete plan->adapt;
    }
    delete plan;
    return 0;
}

int blacklight_plan_create_adaptive(int32_t n_images, const bl_camera_t* cams,
                                    const bl_metric_t* mets, const bl_grid_t* grids,
                                    const double* freqs_hz, const bl_adapt_t* adapt,
                                    const bl_out_t* outs, uint32_t flags, void* stream,
                                    bl_plan_t** plan) {
    g_detail[0] = 0;
    if (!plan) return fail(BL_EINVAL, "plan is NULL");
    *plan = nullptr;
    int precision = -1;
    const float* mlp = nullptr;
    int rc = check_adaptive_args(n_images, cams, mets, grids, freqs_hz, adapt, outs, flags,
                                 &precision, &mlp);
    if (rc) return rc;
    bl_plan* P = new bl_plan();
    BL_CUDA(cudaGetDevice(&P->dev));
    P->n_images = n_images;
    P->precision = precision;
    P->mlp = mlp;
    P->adapt = new AdaptRun();
    cudaStream_t st = (cudaStream_t)stream;
    rc = adapt_prepare(*P->adapt, n_images, cams, mets, grids, freqs_hz, adapt, outs, mlp, flags,
                       st, true);
    if (!rc) rc = plan_capture(*P, st);
    if (rc) {
        blacklight_plan_destroy(P);
        return rc;
    }
    *plan = P;
    return 0;
}

int blacklight_plan_level_rays(bl_plan_t* plan, int32_t* level_rays, void* stream) {
    g_detail[0] = 0;
    if (!plan || !plan->adapt) return fail(BL_EINVAL, "not an adaptive plan");
    return adapt_finish(*plan->adapt, level_rays, (cudaStream_t)stream);
}

int blacklight_trace_batch(int32_t n_images, const bl_camera_t* cams, const bl_metric_t* mets,
                           const bl_grid_t* grids, const double* freqs_hz, const bl_out_t* outs,
                           void* workspace, size_t workspace_bytes, void* stream, uint32_t flags) {
    return trace_impl(n_images, cams, mets, grids, freqs_hz, outs, workspace, workspace_bytes,
                      stream, flags, true);
}

int blacklight_trace(const bl_camera_t* cam, const bl_metric_t* met, const bl_grid_t* grid,
                     double freq_hz, const bl_out_t* out, void* stream, uint32_t flags) {
    return trace_impl(1, cam, met, grid, &freq_hz, out, nullptr, 0, stream, flags, true);
}

int blacklight_geodesics(const bl_camera_t* cam, const bl_metric_t* met, const bl_out_t* out,
                         void* stream, uint32_t flags) {
    return trace_impl(1, cam, met, nullptr, nullptr, out, nullptr, 0, stream, flags, false);
}

size_t blacklight_workspace_size(int32_t n_images, const bl_camera_t* cams,
                                 const bl_metric_t* mets) {
    if (n_images < 1 || !cams || !mets) return 0;
    return make_layout(n_images, cams, mets).total;
}

int blacklight_trace_host(const bl_camera_t* cam, const bl_metric_t* met, const bl_grid_t* grid,
                          double freq_hz, const bl_out_t* out, void* stream) {
    g_detail[0] = 0;
    if (!cam || !met || !grid || !out) return fail(BL_EINVAL, "NULL argument");
    int rc = check_camera(cam, 0);
    if (!rc) rc = check_metric(met, 0);
    if (!rc) rc = check_grid(grid, 0);
    if (!rc) rc = check_out(out, 0, true);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t npix = (size_t)cam->n * cam->n;
    const size_t gbytes = sizeof(float) * 8 * (size_t)grid->n_r * grid->n_theta * grid->n_phi *
                          (size_t)(grid->n_snapshots > 1 ? grid->n_snapshots : 1);
    const size_t sbytes = 4 * npix * (out->dtype == 0 ? sizeof(double) : sizeof(float));
    char* dev = nullptr;
    const size_t off_s = align_up(gbytes), off_st = off_s + align_up(sbytes),
                 off_sp = off_st + align_up(npix * 4), off_e = off_sp + align_up(npix * 4),
                 off_m = off_e + align_up(npix * 8 * sizeof(double)),
                 off_a = off_m + (grid->coef_mlp ? align_up(sizeof(float) * BL_MLP_PARAMS) : 0),
                 abytes = out->aux ? (size_t)BL_AUX_COUNT * npix *
                                     (out->dtype == 0 ? sizeof(double) : sizeof(float)) : 0,
                 total = off_a + align_up(abytes);
    cudaError_t e = cudaMallocAsync((void**)&dev, total, st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(BL_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e)); }
    bl_grid_t g = *grid;
    g.prim = (const float*)dev;
    bl_out_t o = *out;
    o.stokes = dev + off_s;
    o.status = out->status ? (int32_t*)(dev + off_st) : nullptr;
    o.steps = out->steps ? (int32_t*)(dev + off_sp) : nullptr;
    o.end_state = out->end_state ? (double*)(dev + off_e) : nullptr;
    o.samples = nullptr;
    o.aux = out->aux ? (void*)(dev + off_a) : nullptr;
    rc = 0;
    e = cudaMemcpyAsync(dev, grid->prim, gbytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy grid to device");
    if (!rc && grid->coef_mlp) {
        g.coef_mlp = (const float*)(dev + off_m);
        e = cudaMemcpyAsync(dev + off_m, grid->coef_mlp, sizeof(float) * BL_MLP_PARAMS,
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy coefficient model to device");
    }
    if (!rc) rc = trace_impl(1, cam, met, &g, &freq_hz, &o, nullptr, 0, stream, BL_ASYNC, true);
    if (rc >= 0) {
        e = cudaMemcpyAsync(out->stokes, o.stokes, sbytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->status)
            e = cudaMemcpyAsync(out->status, o.status, npix * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->steps)
            e = cudaMemcpyAsync(out->steps, o.steps, npix * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->end_state)
            e = cudaMemcpyAsync(out->end_state, o.end_state, npix * 64, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->aux)
            e = cudaMemcpyAsync(out->aux, o.aux, abytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy results to host");
    }
    cudaFreeAsync(dev, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (rc == 0 && se != cudaSuccess) rc = cuda_fail(se, "cudaStreamSynchronize");
    return rc;
}

// ---------------------------------------------------------------------------------------
// Learned coefficient model
// ---------------------------------------------------------------------------------------
static_assert(BL_MLP_PARAMS == bl::mlp::kParams, "parameter count");
}  // extern "C"

namespace {

// Run `launch(err)` with a zeroed device error flag; BL_ECUDA if a kernel reported a timeout.
template <class F>
int with_tc_flag(cudaStream_t st, F launch) {
    int* err = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&err, sizeof(int), st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(BL_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e)); }
    int rc = 0;
    e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync");
    if (!rc) rc = launch(err);
    int h = 0;
    if (!rc) {
        e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "read error flag");
    }
    cudaFreeAsync(err, st);
    e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    if (!rc && h) rc = fail(BL_ETIMEOUT, "tensor-core wait ran out");
    return rc;
}

int mlp_grid_size() {
    DevInfo di;
    if (dev_info(di)) return 0;
    return di.sms * 4;
}

int mlp_train_attr() {
    static std::mutex mu;
    static std::vector<bool> done;
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, false);
    if (!done[dev]) {
        BL_CUDA(cudaFuncSetAttribute(bl::mlp::train_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bl::mlp::kTrainSmem));
        done[dev] = true;
    }
    return 0;
}

}  // namespace

extern "C" {

int blacklight_mlp_init(float* params, uint64_t seed, void* stream) {
    g_detail[0] = 0;
    int rc = device_pointer(params, "params");
    if (rc) return rc;
    bl::mlp::init_kernel<<<(BL_MLP_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, seed);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_mlp_dataset(int64_t n, uint64_t seed, float* inputs, float* targets, void* stream) {
    g_detail[0] = 0;
    if (n < 0) return fail(BL_EINVAL, "n < 0");
    if (n == 0) return 0;
    int rc = device_pointer(inputs, "inputs");
    if (!rc) rc = device_pointer(targets, "targets");
    if (rc) return rc;
    bl::mlp::dataset_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, seed, inputs, targets);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_mlp_targets(int64_t n, const float* inputs, float* targets, void* stream) {
    g_detail[0] = 0;
    if (n < 0) return fail(BL_EINVAL, "n < 0");
    if (n == 0) return 0;
    int rc = device_pointer(inputs, "inputs");
    if (!rc) rc = device_pointer(targets, "targets");
    if (rc) return rc;
    bl::mlp::targets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, inputs, targets);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_mlp_normalise(int64_t n, const float* inputs, const float* targets, float* params,
                             void* stream) {
    g_detail[0] = 0;
    if (n < 4) return fail(BL_EINVAL, "n < 4");
    int rc = device_pointer(inputs, "inputs");
    if (!rc) rc = device_pointer(targets, "targets");
    if (!rc) rc = device_pointer(params, "params");
    if (rc) return rc;
    bl::mlp::normalise_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(n, inputs, targets, params);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_mlp_grad(const float* params, int64_t n, const float* inputs, const float* targets,
                        float* grad, float* loss, void* stream) {
    g_detail[0] = 0;
    if (n < 1 || !loss) return fail(BL_EINVAL, "n < 1 or loss is NULL");
    int rc = device_pointer(params, "params");
    if (!rc) rc = device_pointer(inputs, "inputs");
    if (!rc) rc = device_pointer(targets, "targets");
    if (!rc) rc = device_pointer(grad, "grad");
    if (!rc) rc = mlp_train_attr();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    float* dloss = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dloss, sizeof(float), st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(BL_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e)); }
    rc = with_tc_flag(st, [&](int* err) -> int {
        BL_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * BL_MLP_PARAMS, st));
        BL_CUDA(cudaMemsetAsync(dloss, 0, sizeof(float), st));
        bl::mlp::train_kernel<<<(unsigned)((n + 127) / 128), 128, bl::mlp::kTrainSmem, st>>>(
            params, n, inputs, targets, 0, n, (double)n, grad, dloss, nullptr, nullptr, err);
        ++g_launches;
        BL_CUDA(cudaGetLastError());
        float h = 0.0f;
        BL_CUDA(cudaMemcpyAsync(&h, dloss, sizeof(float), cudaMemcpyDeviceToHost, st));
        BL_CUDA(cudaStreamSynchronize(st));
        *loss = (float)(h / (7.0 * (double)n));
        return 0;
    });
    cudaFreeAsync(dloss, st);
    return rc;
}

int blacklight_mlp_train(const bl_mlp_train_t* cfg, float* params, float* loss_history,
                         void* stream) {
    g_detail[0] = 0;
    if (!cfg || cfg->size != sizeof(bl_mlp_train_t)) return fail(BL_EINVAL, "cfg.size mismatch");
    if (cfg->batch < 128 || cfg->batch % 128 || cfg->n < cfg->batch || cfg->steps < 0)
        return fail(BL_EINVAL, "need batch a positive multiple of 128, n >= batch, steps >= 0");
    if (!(cfg->lr_start > 0.0) || !(cfg->lr_end > 0.0) || !(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) ||
        !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0) || !(cfg->eps > 0.0))
        return fail(BL_EINVAL, "learning rates and eps must be > 0, 0 <= beta < 1");
    int rc = device_pointer(params, "params");
    if (!rc) rc = device_pointer(cfg->inputs, "cfg.inputs");
    if (!rc) rc = device_pointer(cfg->targets, "cfg.targets");
    if (!rc && loss_history) rc = device_pointer(loss_history, "loss_history");
    if (!rc) rc = mlp_train_attr();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // m, v [BL_MLP_PARAMS] each, then per-tile gradient sums [tiles][trained parameters] and
    // per-tile losses [tiles]: the tiles' sums are reduced in a fixed order, so a training run
    // is reproducible bit for bit
    const int64_t tiles = cfg->batch / 128;
    const size_t n_part = (size_t)tiles * bl::mlp::kOffMean;
    float* buf = nullptr;
    const size_t bytes = sizeof(float) * (2 * (size_t)BL_MLP_PARAMS + n_part + (size_t)tiles);
    cudaError_t e = cudaMallocAsync((void**)&buf, bytes, st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(BL_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e)); }
    float *m = buf, *v = buf + BL_MLP_PARAMS, *part = buf + 2 * BL_MLP_PARAMS,
          *part_loss = part + n_part;
    rc = with_tc_flag(st, [&](int* err) -> int {
        BL_CUDA(cudaMemsetAsync(buf, 0, bytes, st));
        const unsigned blocks = (unsigned)tiles;
        const double b1 = cfg->beta1, b2 = cfg->beta2;
        double p1 = 1.0, p2 = 1.0;
        for (int64_t t = 0; t < cfg->steps; ++t) {
            const int64_t first = (int64_t)((t * (int64_t)cfg->batch) % cfg->n);
            bl::mlp::train_kernel<<<blocks, 128, bl::mlp::kTrainSmem, st>>>(
                params, cfg->n, cfg->inputs, cfg->targets, first, cfg->batch, (double)cfg->batch,
                nullptr, nullptr, part, part_loss, err);
            const double frac = cfg->steps > 1 ? (double)t / (double)(cfg->steps - 1) : 0.0;
            const double lr = cfg->lr_start * pow(cfg->lr_end / cfg->lr_start, frac);
            p1 *= b1;
            p2 *= b2;
            bl::mlp::adam_kernel<<<(bl::mlp::kOffMean + 255) / 256, 256, 0, st>>>(
                params, part, (int)tiles, m, v, (float)lr, (float)b1, (float)b2, (float)cfg->eps,
                (float)(1.0 - p1), (float)(1.0 - p2), part_loss,
                loss_history ? loss_history + t : nullptr, (float)(1.0 / (7.0 * cfg->batch)));
            g_launches += 2;
            BL_CUDA(cudaGetLastError());
        }
        return 0;
    });
    cudaFreeAsync(buf, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (!rc && se != cudaSuccess) rc = cuda_fail(se, "cudaStreamSynchronize");
    return rc;
}

int blacklight_mlp_forward(const float* params, int64_t n, const float* inputs, float* outputs,
                           void* stream) {
    g_detail[0] = 0;
    if (n < 0) return fail(BL_EINVAL, "n < 0");
    if (n == 0) return 0;
    int rc = device_pointer(params, "params");
    if (!rc) rc = device_pointer(inputs, "inputs");
    if (!rc) rc = device_pointer(outputs, "outputs");
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t tiles = (n + 127) / 128;
    const int g = mlp_grid_size();
    const unsigned grid = (unsigned)(tiles < g ? tiles : g);
    return with_tc_flag(st, [&](int* err) -> int {
        bl::mlp::forward_kernel<<<grid, 128, 0, st>>>(params, n, inputs, outputs, err);
        ++g_launches;
        BL_CUDA(cudaGetLastError());
        return 0;
    });
}

int blacklight_mlp_coefficients(const float* params, int64_t n, const double* in, double* out,
                                void* stream) {
    g_detail[0] = 0;
    if (n < 0) return fail(BL_EINVAL, "n < 0");
    if (n == 0) return 0;
    int rc = device_pointer(params, "params");
    if (!rc) rc = device_pointer(in, "in");
    if (!rc) rc = device_pointer(out, "out");
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t tiles = (n + 127) / 128;
    const int g = mlp_grid_size();
    const unsigned grid = (unsigned)(tiles < g ? tiles : g);
    return with_tc_flag(st, [&](int* err) -> int {
        bl::mlp::coefficients_kernel<<<grid, 128, 0, st>>>(params, n, in, out, err);
        ++g_launches;
        BL_CUDA(cudaGetLastError());
        return 0;
    });
}

}  // extern "C"

namespace {

// A non-blocking stream per device for input copies that overlap kernels on the caller's
// stream (created once, kept for the process).
int copy_stream(cudaStream_t* out) {
    static std::mutex mu;
    static std::vector<cudaStream_t> streams;
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)streams.size() <= dev) streams.resize(dev + 1, nullptr);
    if (!streams[dev]) BL_CUDA(cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking));
    *out = streams[dev];
    return 0;
}

// Plane -> cell repacking of n_snap snapshots of `per_snap` cells (stream-ordered).
int launch_grid_pack(const float* planes, float* cells, int64_t per_snap, int64_t n_snap,
                     cudaStream_t st) {
    DevInfo di;
    int rc = dev_info(di);
    if (rc) return rc;
    const int64_t n = per_snap * n_snap;
    const int64_t want = (n + 255) / 256, cap = (int64_t)di.sms * 8;
    bl::grid_pack_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, st>>>(planes, cells, per_snap, n);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    return 0;
}

}  // namespace

extern "C" {

int blacklight_grid_pack(const float* planes, float* cells, int32_t n_r, int32_t n_theta,
                         int32_t n_phi, int32_t n_snapshots, void* stream) {
    g_detail[0] = 0;
    if (!planes || !cells) return fail(BL_EINVAL, "NULL grid pointer");
    if (n_r < 1 || n_theta < 1 || n_phi < 1 || n_snapshots < 1)
        return fail(BL_EINVAL, "grid sizes must be >= 1");
    if (((uintptr_t)cells & 15u) != 0) return fail(BL_EINVAL, "cells must be 16-byte aligned");
    int rc = device_pointer(planes, "planes");
    if (!rc) rc = device_pointer(cells, "cells");
    if (rc) return rc;
    const int64_t per_snap = (int64_t)n_r * n_theta * n_phi;
    const uintptr_t bytes = (uintptr_t)(sizeof(float) * 8 * per_snap * n_snapshots);
    const uintptr_t a = (uintptr_t)planes, b = (uintptr_t)cells;
    if (a < b + bytes && b < a + bytes) return fail(BL_EINVAL, "planes and cells overlap");
    return launch_grid_pack(planes, cells, per_snap, n_snapshots, (cudaStream_t)stream);
}

int blacklight_trace_host_batch(int32_t n_images, const bl_camera_t* cams,
                                const bl_metric_t* mets, const bl_grid_t* grids,
                                const double* freqs_hz, const bl_out_t* outs, void* stream,
                                uint32_t flags) {
    g_detail[0] = 0;
    if (n_images < 1 || !cams || !mets || !grids || !freqs_hz || !outs)
        return fail(BL_EINVAL, "NULL array argument or n_images < 1");
    for (int q = 0; q < n_images; ++q) {
        int rc = check_camera(&cams[q], q);
        if (!rc) rc = check_metric(&mets[q], q);
        if (!rc) rc = check_grid(&grids[q], q);
        if (!rc) rc = check_out(&outs[q], q, true);
        if (rc) return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // distinct grids (by host pointer), their sizes and offsets in one device allocation.
    // Grids given in the plane layout are copied into staging regions of their own and
    // repacked into the cell layout on the device (each trilinear corner then costs two vector
    // loads). The copies run on a side stream while the geodesic kernel, which does not read
    // the grids, runs on `stream`; only the transfer kernel waits for them.
    std::vector<const float*> uniq;
    std::vector<size_t> gsz, goff;
    std::vector<int> gidx(n_images), gfirst;
    size_t off = 0;
    for (int q = 0; q < n_images; ++q) {
        const bl_grid_t& g = grids[q];
        const size_t bytes = sizeof(float) * 8 * (size_t)g.n_r * g.n_theta * g.n_phi *
                             (size_t)(g.n_snapshots > 1 ? g.n_snapshots : 1);
        int k = -1;
        for (size_t u = 0; u < uniq.size(); ++u)
            if (uniq[u] == g.prim) { k = (int)u; break; }
        if (k < 0) {
            k = (int)uniq.size();
            uniq.push_back(g.prim);
            gsz.push_back(bytes);
            goff.push_back(off);
            gfirst.push_back(q);
            off = align_up(off + bytes);
        } else if (gsz[k] < bytes) {
            return fail(BL_EINVAL, "grids[%d] shares its prim pointer with a smaller grid", q);
        } else if (grids[gfirst[k]].layout != g.layout) {
            return fail(BL_EINVAL, "grids[%d] shares its prim pointer with another layout", q);
        }
        gidx[q] = k;
    }
    std::vector<size_t> ostage(uniq.size(), 0);
    for (size_t u = 0; u < uniq.size(); ++u)
        if (grids[gfirst[u]].layout == BL_GRID_PLANES) { ostage[u] = off; off = align_up(off + gsz[u]); }
    const size_t o_mlp = off;
    if (grids[0].coef_mlp) off = align_up(off + sizeof(float) * BL_MLP_PARAMS);
    std::vector<size_t> o_out(n_images);
    for (int q = 0; q < n_images; ++q) {
        const size_t npix = (size_t)cams[q].n * cams[q].n;
        const size_t es = outs[q].dtype == 0 ? sizeof(double) : sizeof(float);
        o_out[q] = off;
        off = align_up(off + 4 * npix * es);                                   // stokes
        if (outs[q].status) off = align_up(off + npix * 4);
        if (outs[q].steps) off = align_up(off + npix * 4);
        if (outs[q].samples) off = align_up(off + npix * 4);
        if (outs[q].end_state) off = align_up(off + npix * 64);
        if (outs[q].aux) off = align_up(off + (size_t)BL_AUX_COUNT * npix * es);
    }
    const Layout L = make_layout(n_images, cams, mets, grids[0].coef_mlp != nullptr);
    const size_t o_ws = off;
    off = align_up(off + L.total);
    char* dev = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dev, off, st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(BL_ENOMEM, "cudaMallocAsync(%zu): %s", off, cudaGetErrorString(e)); }
    int rc = 0;
    // side stream for the input copies: it starts after the allocation on `stream`, and
    // `gate` marks the end of its work (the transfer kernel and every exit path wait for it)
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_alloc = nullptr, gate = nullptr;
    rc = copy_stream(&cs);
    if (!rc && (e = cudaEventCreateWithFlags(&ev_alloc, cudaEventDisableTiming)) != cudaSuccess)
        rc = cuda_fail(e, "cudaEventCreate");
    if (!rc && (e = cudaEventCreateWithFlags(&gate, cudaEventDisableTiming)) != cudaSuccess)
        rc = cuda_fail(e, "cudaEventCreate");
    if (!rc && (e = cudaEventRecord(ev_alloc, st)) != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
    if (!rc && (e = cudaStreamWaitEvent(cs, ev_alloc, 0)) != cudaSuccess) rc = cuda_fail(e, "cudaStreamWaitEvent");
    for (size_t u = 0; u < uniq.size() && !rc; ++u) {
        const bl_grid_t& g = grids[gfirst[u]];
        const bool pack = g.layout == BL_GRID_PLANES;
        e = cudaMemcpyAsync(dev + (pack ? ostage[u] : goff[u]), uniq[u], gsz[u],
                            cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy grid to device");
        if (!rc && pack)
            rc = launch_grid_pack((const float*)(dev + ostage[u]), (float*)(dev + goff[u]),
                                  (int64_t)g.n_r * g.n_theta * g.n_phi,
                                  g.n_snapshots > 1 ? g.n_snapshots : 1, cs);
    }
    if (!rc && grids[0].coef_mlp) {
        e = cudaMemcpyAsync(dev + o_mlp, grids[0].coef_mlp, sizeof(float) * BL_MLP_PARAMS,
                            cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy coefficient model to device");
    }
    if (cs && gate) {
        e = cudaEventRecord(gate, cs);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
    }
    std::vector<bl_grid_t> dg(grids, grids + n_images);
    std::vector<bl_out_t> dout(outs, outs + n_images);
    for (int q = 0; q < n_images; ++q) {
        dg[q].prim = (const float*)(dev + goff[gidx[q]]);
        dg[q].layout = BL_GRID_CELLS;
        if (grids[q].coef_mlp) dg[q].coef_mlp = (const float*)(dev + o_mlp);
        const size_t npix = (size_t)cams[q].n * cams[q].n;
        const size_t es = outs[q].dtype == 0 ? sizeof(double) : sizeof(float);
        size_t p = o_out[q];
        dout[q].stokes = dev + p; p = align_up(p + 4 * npix * es);
        if (outs[q].status) { dout[q].status = (int32_t*)(dev + p); p = align_up(p + npix * 4); }
        if (outs[q].steps) { dout[q].steps = (int32_t*)(dev + p); p = align_up(p + npix * 4); }
        if (outs[q].samples) { dout[q].samples = (int32_t*)(dev + p); p = align_up(p + npix * 4); }
        if (outs[q].end_state) { dout[q].end_state = (double*)(dev + p); p = align_up(p + npix * 64); }
        if (outs[q].aux) { dout[q].aux = dev + p; }
    }
    if (!rc)
        rc = trace_impl(n_images, cams, mets, dg.data(), freqs_hz, dout.data(), dev + o_ws, L.total,
                        stream, BL_ASYNC | (flags & BL_UNPOLARIZED), true, gate);
    // whatever happened above, nothing on `stream` (results, the free) may overtake the copies
    if (gate) cudaStreamWaitEvent(st, gate, 0);
    for (int q = 0; q < n_images && rc >= 0; ++q) {
        const size_t npix = (size_t)cams[q].n * cams[q].n;
        const size_t es = outs[q].dtype == 0 ? sizeof(double) : sizeof(float);
        e = cudaMemcpyAsync(outs[q].stokes, dout[q].stokes, 4 * npix * es, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && outs[q].status)
            e = cudaMemcpyAsync(outs[q].status, dout[q].status, npix * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && outs[q].steps)
            e = cudaMemcpyAsync(outs[q].steps, dout[q].steps, npix * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && outs[q].samples)
            e = cudaMemcpyAsync(outs[q].samples, dout[q].samples, npix * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && outs[q].end_state)
            e = cudaMemcpyAsync(outs[q].end_state, dout[q].end_state, npix * 64, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && outs[q].aux)
            e = cudaMemcpyAsync(outs[q].aux, dout[q].aux, (size_t)BL_AUX_COUNT * npix * es,
                                cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy results to host");
    }
    if (rc >= 0) {
        const int r2 = finish(dev + o_ws, L, st, true);   // per-ray anomalies of the launch
        if (r2 != 0) rc = r2;
    }
    cudaFreeAsync(dev, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (rc == 0 && se != cudaSuccess) rc = cuda_fail(se, "cudaStreamSynchronize");
    if (ev_alloc) cudaEventDestroy(ev_alloc);
    if (gate) cudaEventDestroy(gate);
    return rc;
}

int blacklight_coefficients(int64_t n, const double* in, double* out, int32_t precision,
                            void* stream) {
    g_detail[0] = 0;
    if (n < 0 || (n > 0 && (!in || !out))) return fail(BL_EINVAL, "bad arguments");
    if (n == 0) return 0;
    int rc = device_pointer(in, "in");
    if (!rc) rc = device_pointer(out, "out");
    if (rc) return rc;
    const int64_t blocks = (n + 127) / 128;
    if (precision == BL_PREC_MIXED)
        bl::coefficients_kernel<float><<<blocks, 128, 0, (cudaStream_t)stream>>>(n, in, out);
    else
        bl::coefficients_kernel<double><<<blocks, 128, 0, (cudaStream_t)stream>>>(n, in, out);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_stokes_step(int64_t n, const double* coef, const double* s0, const double* dl,
                           double* s1, int32_t precision, void* stream) {
    g_detail[0] = 0;
    if (n < 0 || (n > 0 && (!coef || !s0 || !dl || !s1))) return fail(BL_EINVAL, "bad arguments");
    if (n == 0) return 0;
    int rc = device_pointer(coef, "coef");
    if (!rc) rc = device_pointer(s0, "s0");
    if (!rc) rc = device_pointer(dl, "dl");
    if (!rc) rc = device_pointer(s1, "s1");
    if (rc) return rc;
    const int64_t blocks = (n + 127) / 128;
    if (precision == BL_PREC_MIXED)
        bl::stokes_step_kernel<float><<<blocks, 128, 0, (cudaStream_t)stream>>>(n, coef, s0, dl, s1);
    else
        bl::stokes_step_kernel<double><<<blocks, 128, 0, (cudaStream_t)stream>>>(n, coef, s0, dl, s1);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

int blacklight_bessel_k(int64_t n, const double* x, double* out, int32_t precision, void* stream) {
    g_detail[0] = 0;
    if (n < 0 || (n > 0 && (!x || !out))) return fail(BL_EINVAL, "bad arguments");
    if (n == 0) return 0;
    int rc = device_pointer(x, "x");
    if (!rc) rc = device_pointer(out, "out");
    if (rc) return rc;
    const int64_t blocks = (n + 127) / 128;
    if (precision == BL_PREC_MIXED)
        bl::bessel_kernel<float><<<blocks, 128, 0, (cudaStream_t)stream>>>(n, x, out);
    else
        bl::bessel_kernel<double><<<blocks, 128, 0, (cudaStream_t)stream>>>(n, x, out);
    ++g_launches;
    BL_CUDA(cudaGetLastError());
    BL_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return 0;
}

}  // extern "C"

namespace {

// Best-of-reps rate (flops per second) of one probe launch; ms_out += one launch's time.
template <class K, class L>
int time_probe(K kernel, L launch, int reps, cudaStream_t st, double flops, double* rate,
               double* ms_out) {
    int per_sm = 0;
    BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, bl::kPeakThreads, 0));
    int dev = 0, sms = 0;
    BL_CUDA(cudaGetDevice(&dev));
    BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    const double total = flops * (double)grid * bl::kPeakThreads;
    cudaEvent_t e0, e1;
    BL_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(ce, "cudaEventCreate"); }
    double best = 0.0, last_ms = 0.0;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) { launch(grid, st); ++g_launches; e = cudaGetLastError(); }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms > 0.0f) {   // launch 0 is the warm-up
            const double v = total / (ms * 1e-3);
            if (v > best) best = v;
            last_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "peak probe");
    *rate = best;
    *ms_out += last_ms;
    return 0;
}

}  // namespace

extern "C" {

int blacklight_measure_peaks(bl_peaks_t* out, int32_t reps, void* stream) {
    g_detail[0] = 0;
    if (!out || out->size != sizeof(bl_peaks_t)) return fail(BL_EINVAL, "out: NULL or size mismatch");
    if (reps < 1 || reps > 100) return fail(BL_EINVAL, "reps must be in [1, 100]");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    BL_CUDA(cudaDeviceGetAttribute(&out->sm_count, cudaDevAttrMultiProcessorCount, dev));
    BL_CUDA(cudaDeviceGetAttribute(&out->sm_clock_khz, cudaDevAttrClockRate, dev));
    // the probes' results are stored only under a condition that never holds; the sink is a
    // small stream-ordered buffer they never write
    float* sink = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&sink, 65536 * sizeof(double), st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(BL_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e)); }
    // chain lengths for ~15 ms a launch on a GB300-class device
    constexpr int kIt64 = 4096, kIt32 = 1 << 18, kItDf = 1 << 15;
    constexpr int kCh = 8, kChDf = 4;
    out->probe_ms = 0.0;
    double r64 = 0.0, r32 = 0.0, rdf = 0.0;
    int rc = time_probe(bl::fma_chain_kernel<double, kCh>,
                        [&](unsigned g, cudaStream_t s) {
                            bl::fma_chain_kernel<double, kCh><<<g, bl::kPeakThreads, 0, s>>>(
                                (double*)sink, kIt64, 0.999999, 1e-6);
                        }, reps, st, 2.0 * kCh * kIt64, &r64, &out->probe_ms);
    if (!rc)
        rc = time_probe(bl::fma_chain_kernel<float, kCh>,
                        [&](unsigned g, cudaStream_t s) {
                            bl::fma_chain_kernel<float, kCh><<<g, bl::kPeakThreads, 0, s>>>(
                                sink, kIt32, 0.999999f, 1e-6f);
                        }, reps, st, 2.0 * kCh * kIt32, &r32, &out->probe_ms);
    if (!rc)
        rc = time_probe(bl::df64_chain_kernel<kChDf>,
                        [&](unsigned g, cudaStream_t s) {
                            const bl::df64 a(0.999999), b(1e-6);
                            bl::df64_chain_kernel<kChDf><<<g, bl::kPeakThreads, 0, s>>>(
                                sink, kItDf, a.hi, a.lo, b.hi, b.lo);
                        }, reps, st, 2.0 * kChDf * kItDf, &rdf, &out->probe_ms);
    cudaFreeAsync(sink, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (rc) return rc;
    if (es != cudaSuccess) return cuda_fail(es, "cudaStreamSynchronize");
    out->fp64_tflops = r64 * 1e-12;
    out->fp32_tflops = r32 * 1e-12;
    out->df64_tflops = rdf * 1e-12;
    return 0;
}

int blacklight_set_memory_retention(uint64_t bytes) {
    g_detail[0] = 0;
    int dev = 0;
    BL_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    BL_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t v = bytes;
    BL_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &v));
    return 0;
}

int blacklight_selftest_wait(int64_t max_cycles, int32_t arrive, void* stream) {
    g_detail[0] = 0;
    if (max_cycles < 1 || max_cycles > (1ll << 32) || (arrive != 0 && arrive != 1))
        return fail(BL_EINVAL, "max_cycles in [1, 2^32], arrive 0 or 1");
    return with_tc_flag((cudaStream_t)stream, [&](int* err) -> int {
        bl::mlp::wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(max_cycles, arrive, err);
        ++g_launches;
        BL_CUDA(cudaGetLastError());
        return 0;
    });
}

const char* blacklight_strerror(int code) {
    switch (code) {
        case BL_OK: return "success";
        case BL_WRAYS: return "completed; some rays did not terminate normally (see status)";
        case BL_EINVAL: return "invalid argument";
        case BL_ENOMEM: return "device memory allocation failed";
        case BL_ECUDA: return "CUDA runtime error";
        case BL_EUNSUPPORTED: return "unsupported option";
        case BL_ETIMEOUT: return "a bounded device wait ran out";
        default: return "unknown error code";
    }
}

const char* blacklight_last_error_detail(void) { return g_detail; }

int blacklight_last_kernel_ms(float ms[2]) {
    g_detail[0] = 0;
    if (!ms) return fail(BL_EINVAL, "ms is NULL");
    if (g_timed_waves < 1) return fail(BL_EINVAL, "no call with BL_TIMING on this thread");
    const int w_n = g_timed_waves;
    BL_CUDA(cudaEventSynchronize(g_ev[2 * w_n]));
    ms[0] = ms[1] = 0.0f;
    for (int w = 0; w < w_n; ++w) {
        float a = 0.0f, b = 0.0f;
        BL_CUDA(cudaEventElapsedTime(&a, g_ev[2 * w], g_ev[2 * w + 1]));
        BL_CUDA(cudaEventElapsedTime(&b, g_ev[2 * w + 1], g_ev[2 * w + 2]));
        ms[0] += a;
        ms[1] += b;
    }
    return 0;
}

uint64_t blacklight_launch_count(int reset) {
    uint64_t v = g_launches;
    if (reset) g_launches = 0;
    return v;
}

}  // extern "C"
