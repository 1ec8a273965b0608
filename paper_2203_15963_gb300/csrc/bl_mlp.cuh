// Learned thermal-synchrotron coefficient model: a 3 -> 64 -> 64 -> 7 SiLU perceptron whose
// seven outputs replace the transcendental parts of the fits of Sec. 2.5 (Bessel factors of
// the Maxwell-Juettner normalisation, the emissivity shape polynomials, the Faraday shapes);
// the closed-form prefactors stay exact. Weights are BF16 in shared memory, products run on
// the tensor cores (tcgen05, FP32 accumulation in tensor memory), one 128-sample tile per
// CTA with one sample per thread.
//
// Model (all float):
//   inputs  log10 x in [-3, 6] (x = nu / nu_c, nu_c = 1.5 nu_B sin(theta) Theta^2),
//           log10 Theta_e in [-1, 2], |cos theta_B| in [0, 1], each mapped to [-1, 1], and a
//           constant 1 that carries the first layer's bias;
//   outputs o = offset + scale * y + A f, y = W3 silu(W2 silu(W1 [f, 1]) + b2) + b3, with
//           o1..o3 = ln of the I, Q, V shape prefactors (the exp(-1.8899 x^1/3) factor kept
//           exact), o4, o5 = f_m, g_m (Faraday conversion and rotation shapes),
//           o6 = ln(e^z K_2(z)), o7 = ln(K_0(z) / K_2(z)), z = 1 / Theta_e.
// Parameter vector (float, kParams values): W1 [64][4], W2 [64][64], b2 [64], W3 [7][64],
// b3 [7], offset [7], scale [7], A [7][3]. Offset, A and scale are fixed before training (the
// least-squares affine fit of the targets and its residual's standard deviation), so the
// network learns only the non-linear remainder.
#pragma once
#include "bl_internal.cuh"
#include "bl_math.cuh"
#include "bl_tc.cuh"

namespace bl {
namespace mlp {

constexpr int kHidden = 64, kOut = 7;
constexpr int kOffW1 = 0, kOffW2 = 256, kOffB2 = 4352, kOffW3 = 4416, kOffB3 = 4864,
              kOffMean = 4871, kOffScale = 4878, kOffA = 4885, kParams = 4906;
constexpr float kLxLo = -3.0f, kLxHi = 6.0f, kLtLo = -1.0f, kLtHi = 2.0f;
constexpr long long kWaitCycles = 1ll << 31;   // ~1 s at 2 GHz

__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
// z sigma(z) = z/2 (1 + tanh(z/2)) with the hardware tanh (relative error about 2^-11, below
// the bf16 rounding of the stored activation, 2^-9): one special-function operation instead
// of two. Inference in the trace only; training keeps silu above.
__device__ __forceinline__ float silu_tanh(float z) {
    const float hz = 0.5f * z;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(hz));
    return fmaf(hz, t, hz);
}
__device__ __forceinline__ float silu_grad(float z) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// ---------------------------------------------------------------------------------------
// Model inputs of one plasma sample and the reconstruction of the eight coefficients
// ---------------------------------------------------------------------------------------
struct ModelIn {
    float f[3];     // network inputs in [-1, 1]
    bool ok;        // inside the trained domain
};

__device__ __forceinline__ ModelIn model_inputs(float th, float bg, float nu, float cth) {
    ModelIn m;
    const float sth = sqrtf(fmaxf(1.0f - cth * cth, 0.0f));
    const float nub = (float)(kE / (2.0 * kPi * kMe * kC)) * bg;
    const float nuc = 1.5f * nub * sth * th * th;
    const float lx = log10f(nu / nuc);
    const float lt = log10f(th);
    m.ok = th > 0.0f && bg > 0.0f && nuc > 0.0f && lx >= kLxLo && lx <= kLxHi && lt >= kLtLo &&
           lt <= kLtHi;
    m.f[0] = m.ok ? 2.0f * (lx - kLxLo) / (kLxHi - kLxLo) - 1.0f : 0.0f;
    m.f[1] = m.ok ? 2.0f * (lt - kLtLo) / (kLtHi - kLtLo) - 1.0f : 0.0f;
    m.f[2] = 2.0f * fabsf(cth) - 1.0f;
    return m;
}

// j_{I,Q,V}, alpha_{I,Q,V}, rho_{Q,V} from the learned quantities o[7] and the exact
// prefactors (same formulae as synchrotron_coefficients with its transcendental parts
// replaced). Requires ne, th, bg > 0 and sin(theta_B) > 0 (guaranteed by model_inputs).
__device__ __forceinline__ void coefficients_from(const float o[7], float ne, float th, float bg,
                                                  float nu, float cth, float out[8]) {
    const float sth2 = fmaxf(1.0f - cth * cth, 0.0f);
    const float sth = sqrtf(sth2);
    const float nub = (float)(kE / (2.0 * kPi * kMe * kC)) * bg;
    const float z = 1.0f / th;
    const float x = nu / (1.5f * nub * sth * th * th);
    const float lex = -1.8899f * cbrtf(x) + z - o[5];
    const float pre = ne * (float)(kE * kE / (1.7320508075688772 * kC)) * nu;
    out[0] = pre * expf(o[0] + lex);
    out[1] = pre * expf(o[1] + lex);
    out[2] = pre * (4.0f / (3.0f * th)) * (cth / sth) * expf(o[2] + lex);
    const float hkt = (float)(kH / (kMe * kC * kC)) * nu / th;
    const float cnu = (float)kC / nu;
    const float ibnu = expm1f(hkt) * (cnu * cnu) * ((float)(0.5 / kH) / nu);
    out[3] = out[0] * ibnu;
    out[4] = out[1] * ibnu;
    out[5] = out[2] * ibnu;
    const float k0k2 = expf(o[6]);
    const float k1k2 = (1.0f - k0k2) * z * 0.5f;
    const float base = ne * (float)(kE * kE / (kMe * kC));
    out[6] = base * nub * nub * sth2 / (nu * nu * nu) * o[3] * (k1k2 + 6.0f * th);
    out[7] = 2.0f * base * nub * cth / (nu * nu) * k0k2 * o[4];
}

// The seven learned quantities from the exact fits, in FP64 (training targets).
__device__ __forceinline__ void exact_targets(double lx, double lt, double o[7]) {
    const double x = pow(10.0, lx);
    const double u = 1.0 / cbrt(x);
    const double X = sqrt(1.4142135623730951e3 / (1.5 * x));
    o[0] = log(2.5651 * (1.0 + 1.92 * u + 0.9977 * u * u));
    o[1] = log(2.5651 * (1.0 + 0.932 * u + 0.4998 * u * u));
    o[2] = log(1.8138 / x + 3.423 * u * u + 0.02955 / sqrt(x) + 2.0377 * u);
    o[3] = 2.011 * exp(-pow(X, 1.035) / 4.7) - cos(0.5 * X) * exp(-pow(X, 1.2) / 2.73) -
           0.011 * exp(-X / 47.2);
    o[4] = 1.0 - 0.11 * log1p(0.035 * X);
    double k0, k1, k2;
    bessel_k012_scaled<double>(pow(10.0, -lt), k0, k1, k2);
    o[5] = log(k2);
    o[6] = log(k0 / k2);
}

// SplitMix64 (Steele, Lea & Flood 2014): the i-th output of the generator seeded with seed.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double uniform01(uint64_t seed, uint64_t i) {
    return (double)(splitmix64(seed, i) >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------------------
// Inference: one 128-sample tile per call, all 128 threads of the CTA take part
// ---------------------------------------------------------------------------------------
struct __align__(128) FwdSmem {
    unsigned char w1[64 * 16 * 2];   // [64][16]: W1 columns 0-2, bias in column 3
    unsigned char w2[64 * 64 * 2];   // [64][64]
    unsigned char w3[16 * 64 * 2];   // [16][64], rows 7-15 zero
    unsigned char x[128 * 16 * 2];   // [128][16]: inputs, 1, zeros
    unsigned char h[128 * 64 * 2];   // [128][64]: hidden activations
    float b2[64], b3[8], mean[8], scale[8], A[24];
    uint64_t bar;
    uint32_t tmem;
};
constexpr uint32_t kFwdCols = 64;

// Stage the weights and set up tensor memory and the barrier (every thread calls this).
__device__ __forceinline__ void fwd_init(FwdSmem& S, const float* __restrict__ P) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < 64 * 16; i += nt) {
        const int j = i >> 4, k = i & 15;
        tc::st_bf16(S.w1, j, k, 16, k < 4 ? P[kOffW1 + 4 * j + k] : 0.0f);
    }
    for (int i = t; i < 64 * 64; i += nt) tc::st_bf16(S.w2, i >> 6, i & 63, 64, P[kOffW2 + i]);
    for (int i = t; i < 16 * 64; i += nt) {
        const int o = i >> 6, j = i & 63;
        tc::st_bf16(S.w3, o, j, 64, o < kOut ? P[kOffW3 + 64 * o + j] : 0.0f);
    }
    for (int i = t; i < 128 * 16; i += nt) {
        const int r = i >> 4, k = i & 15;
        tc::st_bf16(S.x, r, k, 16, k == 3 ? 1.0f : 0.0f);
    }
    for (int i = t; i < 64; i += nt) S.b2[i] = P[kOffB2 + i];
    for (int i = t; i < 8; i += nt) {
        S.b3[i] = i < kOut ? P[kOffB3 + i] : 0.0f;
        S.mean[i] = i < kOut ? P[kOffMean + i] : 0.0f;
        S.scale[i] = i < kOut ? P[kOffScale + i] : 0.0f;
    }
    for (int i = t; i < 24; i += nt) S.A[i] = i < 3 * kOut ? P[kOffA + i] : 0.0f;
    if (t < 32) tc::tmem_alloc(&S.tmem, kFwdCols);
    if (t == 0) tc::mbar_init(&S.bar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Wait for the MMA group committed in phase `phase`, the same outcome on every thread.
__device__ __forceinline__ bool cta_wait(FwdSmem& S, uint32_t& phase) {
    const bool ok = tc::mbar_wait(&S.bar, phase, kWaitCycles);
    phase ^= 1u;
    const bool all = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
    return all;
}

// hidden layer epilogue: 64 accumulator columns of this thread's row (+ bias), SiLU, BF16
// row of the next A operand
template <bool kTanh>
__device__ __forceinline__ void hidden_epilogue(FwdSmem& S, const float* bias) {
    auto act = [](float z) { return kTanh ? silu_tanh(z) : silu(z); };
    const int t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v[16];
        tc::tmem_ld16(tc::tmem_lane_addr(S.tmem, 16 * c), v);
        // 8 consecutive columns of a row are one 16-byte row of a core matrix: one vector store
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            uint32_t w[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int j = 8 * g + 2 * p;
                w[p] = tc::pack_bf16x2(act(v[j] + (bias ? bias[16 * c + j] : 0.0f)),
                                       act(v[j + 1] + (bias ? bias[16 * c + j + 1] : 0.0f)));
            }
            *reinterpret_cast<uint4*>(S.h + tc::kmajor(t, 16 * c + 8 * g, 64)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

__device__ __forceinline__ void issue_barrier_then(FwdSmem& S) {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
}

// Forward pass of this thread's sample (f[3]; rows whose thread passes valid = false are
// computed on zero inputs and ignored; a tile without a valid row issues no MMA and leaves o
// at zero). kTanh selects the hardware-tanh activation. Returns false if a tensor-core wait
// timed out.
// Columns 0-3 of a sample's A-operand row as two packed bf16 pairs: the three inputs and the
// constant 1 of the first-layer bias.
__device__ __forceinline__ uint2 input_row(const float f[3]) {
    return make_uint2(tc::pack_bf16x2(f[0], f[1]), tc::pack_bf16x2(f[2], 1.0f));
}

// The network of a tile whose rows arrive packed (input_row); o is y = W3 h2 + b3 before the
// affine output map. Same waits and masking as fwd_tile.
template <bool kTanh>
__device__ __forceinline__ bool fwd_tile_y(FwdSmem& S, uint32_t& phase, uint2 row, bool valid,
                                           float y[7]) {
    const int t = threadIdx.x;
    *reinterpret_cast<uint2*>(S.x + tc::kmajor(t, 0, 16)) = valid ? row : make_uint2(0u, 0u);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    if (!__syncthreads_or(valid)) {
        tc::fence_after_sync();
#pragma unroll
        for (int k = 0; k < kOut; ++k) y[k] = 0.0f;
        return true;
    }
    if (t == 0) {
        tc::fence_after_sync();
        tc::gemm_bf16(S.tmem, S.x, S.w1, 64, 16);
        tc::mma_commit(&S.bar);
    }
    if (!cta_wait(S, phase)) return false;
    hidden_epilogue<kTanh>(S, nullptr);          // first-layer bias is in W1
    issue_barrier_then(S);
    if (t == 0) {
        tc::fence_after_sync();
        tc::gemm_bf16(S.tmem, S.h, S.w2, 64, 64);
        tc::mma_commit(&S.bar);
    }
    if (!cta_wait(S, phase)) return false;
    hidden_epilogue<kTanh>(S, S.b2);
    issue_barrier_then(S);
    if (t == 0) {
        tc::fence_after_sync();
        tc::gemm_bf16(S.tmem, S.h, S.w3, 16, 64);
        tc::mma_commit(&S.bar);
    }
    if (!cta_wait(S, phase)) return false;
    float v[16];
    tc::tmem_ld16(tc::tmem_lane_addr(S.tmem, 0), v);
#pragma unroll
    for (int k = 0; k < kOut; ++k) y[k] = v[k] + S.b3[k];
    tc::fence_before_sync();
    return true;
}

template <bool kTanh = false>
__device__ __forceinline__ bool fwd_tile(FwdSmem& S, uint32_t& phase, const float f[3], bool valid,
                                         float o[7]) {
    const int t = threadIdx.x;
    // columns 0-3 of the row: the three inputs and the constant 1 of the first-layer bias
    *reinterpret_cast<uint2*>(S.x + tc::kmajor(t, 0, 16)) =
        make_uint2(tc::pack_bf16x2(valid ? f[0] : 0.0f, valid ? f[1] : 0.0f),
                   tc::pack_bf16x2(valid ? f[2] : 0.0f, 1.0f));
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    if (!__syncthreads_or(valid)) {
        tc::fence_after_sync();
#pragma unroll
        for (int k = 0; k < kOut; ++k) o[k] = 0.0f;
        return true;
    }
    if (t == 0) {
        tc::fence_after_sync();
        tc::gemm_bf16(S.tmem, S.x, S.w1, 64, 16);
        tc::mma_commit(&S.bar);
    }
    if (!cta_wait(S, phase)) return false;
    hidden_epilogue<kTanh>(S, nullptr);          // first-layer bias is in W1
    issue_barrier_then(S);
    if (t == 0) {
        tc::fence_after_sync();
        tc::gemm_bf16(S.tmem, S.h, S.w2, 64, 64);
        tc::mma_commit(&S.bar);
    }
    if (!cta_wait(S, phase)) return false;
    hidden_epilogue<kTanh>(S, S.b2);
    issue_barrier_then(S);
    if (t == 0) {
        tc::fence_after_sync();
        tc::gemm_bf16(S.tmem, S.h, S.w3, 16, 64);
        tc::mma_commit(&S.bar);
    }
    if (!cta_wait(S, phase)) return false;
    float v[16];
    tc::tmem_ld16(tc::tmem_lane_addr(S.tmem, 0), v);
#pragma unroll
    for (int k = 0; k < kOut; ++k)
        o[k] = S.mean[k] + S.scale[k] * (v[k] + S.b3[k]) + S.A[3 * k] * f[0] +
               S.A[3 * k + 1] * f[1] + S.A[3 * k + 2] * f[2];
    tc::fence_before_sync();
    return true;
}

// Release tensor memory. After a timed-out wait the outstanding MMA group is waited for
// once more (bounded) before the columns are freed.
__device__ __forceinline__ void fwd_finish(FwdSmem& S, uint32_t phase, bool ok) {
    if (!ok) tc::mbar_wait(&S.bar, phase ^ 1u, kWaitCycles);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(S.tmem, kFwdCols);
}

// outputs o [n][7] for raw inputs [n][3] (log10 x, log10 Theta_e, |cos|); persistent tiles
__global__ void __launch_bounds__(128) forward_kernel(const float* __restrict__ P, int64_t n,
                                                      const float* __restrict__ in,
                                                      float* __restrict__ out, int* err) {
    __shared__ FwdSmem S;
    fwd_init(S, P);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t tiles = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int64_t i = tile * 128 + threadIdx.x;
        const bool valid = i < n;
        float f[3] = {0.0f, 0.0f, 0.0f};
        if (valid) {
            f[0] = 2.0f * (in[3 * i] - kLxLo) / (kLxHi - kLxLo) - 1.0f;
            f[1] = 2.0f * (in[3 * i + 1] - kLtLo) / (kLtHi - kLtLo) - 1.0f;
            f[2] = 2.0f * fabsf(in[3 * i + 2]) - 1.0f;
        }
        float o[7];
        ok = fwd_tile(S, phase, f, valid, o);
        if (ok && valid)
            for (int k = 0; k < kOut; ++k) out[7 * i + k] = o[k];
    }
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    fwd_finish(S, phase, ok);
}

// The learned model over a trace's sample records (the middle pass of the learned-coefficient
// transfer): record k of the pool carries its sample's input row in its last 8 bytes (values
// 14-15, written by the model-input kernel; zero where the sample has no plasma or lies
// outside the model's domain); the model's outputs o[7] (padded to 8) go to out[8 k ..].
// Each CTA scans its share of the pool's used records 128 at a time and queues the records
// that carry an input row in shared memory; whenever 128 wait it runs the network on a full
// tile of them (each row of a tile is computed independently of the others, so the outputs do
// not depend on which records share a tile). The used record count is read on the device (the
// pool cursor after the geodesic kernel), so the launch needs no host round trip.
constexpr int kPoolQueue = 256;   // fewer than 128 waiting + one scanned batch of 128
__global__ void __launch_bounds__(128) forward_pool_kernel(const float* __restrict__ P,
                                                           const float* __restrict__ pool,
                                                           const unsigned long long* __restrict__ pool_next,
                                                           unsigned long long pool_chunks,
                                                           float* __restrict__ out,
                                                           unsigned long long* timeouts) {
    __shared__ FwdSmem S;
    __shared__ int64_t qrec[kPoolQueue];   // (the rows are read again at evaluation: 2 KB
                                           // more of queue would cost a CTA an SM)
    __shared__ int wsum[4];
    fwd_init(S, P);
    uint32_t phase = 0;
    bool ok = true;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned long long used_chunks = *pool_next < pool_chunks ? *pool_next : pool_chunks;
    const int64_t n = (int64_t)used_chunks * kChunk;
    const int64_t tiles = (n + 127) / 128;
    int qn = 0;   // records waiting (the same on every thread)
    for (int64_t tile = blockIdx.x; ok; tile += gridDim.x) {
        const bool more = tile < tiles;
        if (more) {
            // scan 128 records; the ones with an input row join the queue in record order
            const int64_t k = tile * 128 + t;
            uint2 row = make_uint2(0u, 0u);
            if (k < n) row = __ldg(reinterpret_cast<const uint2*>(pool + 16 * k + 14));
            const bool valid = row.y != 0u;          // the constant-1 column is set
            const unsigned mask = __ballot_sync(0xffffffffu, valid);
            if (lane == 0) wsum[wid] = __popc(mask);
            __syncthreads();
            int off = __popc(mask & ((1u << lane) - 1u)), total = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (w < wid) off += wsum[w];
                total += wsum[w];
            }
            if (valid) qrec[qn + off] = k;
            qn += total;
            __syncthreads();
        }
        if (qn >= 128 || (!more && qn > 0)) {
            const int m = qn < 128 ? qn : 128;
            const bool valid = t < m;
            const int64_t k = valid ? qrec[t] : 0;
            const uint2 row = valid ? __ldg(reinterpret_cast<const uint2*>(pool + 16 * k + 14))
                                    : make_uint2(0u, 0u);
            float y[7];
            ok = fwd_tile_y<true>(S, phase, row, valid, y);
            if (ok && valid) {
                float4* q = reinterpret_cast<float4*>(out + 8 * k);
                q[0] = make_float4(y[0], y[1], y[2], y[3]);
                q[1] = make_float4(y[4], y[5], y[6], 0.0f);
            }
            // the waiting remainder moves to the queue's front
            const bool moves = t < qn - m;
            int64_t keep_rec = 0;
            __syncthreads();
            if (moves) keep_rec = qrec[m + t];
            __syncthreads();
            if (moves) qrec[t] = keep_rec;
            qn -= m;
            __syncthreads();
        }
        if (!more && qn == 0) break;
    }
    if (!ok && t == 0) atomicAdd(timeouts, 1ull);
    fwd_finish(S, phase, ok);
}

// The affine output map o = offset + scale y + A f of the model, for a sample whose inputs f
// were those of its packed row (the transfer reads y from the pool pass and applies it).
__device__ __forceinline__ void model_outputs_from_y(const float* __restrict__ P, const float y[7],
                                                     const float f[3], float o[7]) {
#pragma unroll
    for (int k = 0; k < kOut; ++k)
        o[k] = __ldg(P + kOffMean + k) + __ldg(P + kOffScale + k) * y[k] +
               __ldg(P + kOffA + 3 * k) * f[0] + __ldg(P + kOffA + 3 * k + 1) * f[1] +
               __ldg(P + kOffA + 3 * k + 2) * f[2];
}

// coefficients [n][8] of plasma samples in [n][5] (n_e, Theta_e, B, nu, cos theta_B): the
// model inside its domain, the exact fits (FP32) outside it
__global__ void __launch_bounds__(128) coefficients_kernel(const float* __restrict__ P, int64_t n,
                                                           const double* __restrict__ in,
                                                           double* __restrict__ out, int* err) {
    __shared__ FwdSmem S;
    fwd_init(S, P);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t tiles = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int64_t i = tile * 128 + threadIdx.x;
        const bool valid = i < n;
        float s[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (valid)
            for (int q = 0; q < 5; ++q) s[q] = (float)in[5 * i + q];
        const ModelIn m = model_inputs(s[1], s[2], s[3], s[4]);
        const bool use = valid && m.ok && s[0] > 0.0f;
        float o[7];
        ok = fwd_tile(S, phase, m.f, use, o);
        if (ok && valid) {
            float c[8];
            if (use) coefficients_from(o, s[0], s[1], s[2], s[3], s[4], c);
            else synchrotron_coefficients<float>(s[0], s[1], s[2], s[3], s[4], c);
            for (int q = 0; q < 8; ++q) out[8 * i + q] = (double)c[q];
        }
    }
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    fwd_finish(S, phase, ok);
}

// ---------------------------------------------------------------------------------------
// Training: forward and backward of one 128-sample tile per CTA, all nine products on the
// tensor cores. Weight gradients contract over the samples (K = 128): their A operand is the
// transposed error (rows = units; the rows beyond the layer's units read neighbouring
// shared memory and produce accumulator rows that are never read), their B operand the
// transposed activations with a row of ones appended, whose column yields the bias gradient.
// ---------------------------------------------------------------------------------------
constexpr uint32_t kTdZ2T = 0;        // [64][128] dZ2^T  (A, 128-row window to 32768)
constexpr uint32_t kTdZ1T = 16384;    // [64][128] dZ1^T  (A window to 49152)
constexpr uint32_t kTdZ3T = 32768;    // [8][128]  dY^T   (A window to 65536)
constexpr uint32_t kTH1T = 34816;     // [80][128] H1^T, ones row 64 (B)
constexpr uint32_t kTH2T = 55296;     // [80][128] H2^T, ones row 64 (B)
constexpr uint32_t kTXT = 75776;      // [16][128] X^T (B): inputs, ones row 3
constexpr uint32_t kTX = 79872;       // [128][16] X (A)
constexpr uint32_t kTH1 = 83968;      // [128][64] H1 (A)
constexpr uint32_t kTH2 = 100352;     // [128][64] H2 (A)
constexpr uint32_t kTdZ3 = 116736;    // [128][16] dY (A)
constexpr uint32_t kTdZ2 = 120832;    // [128][64] dZ2 (A)
constexpr uint32_t kTW1 = 137216;     // [64][16] W1 (B)
constexpr uint32_t kTW2 = 139264;     // [64][64] W2 (B)
constexpr uint32_t kTW3 = 147456;     // [16][64] W3 (B)
constexpr uint32_t kTW3T = 149504;    // [64][16] W3^T (B)
constexpr uint32_t kTW2T = 151552;    // [64][64] W2^T (B)
constexpr uint32_t kTF32 = 159744;    // b2[64] b3[8] mean[8] scale[8] red[32] A[24]
constexpr uint32_t kTBar = 161024;    // mbarrier, tensor-memory base
constexpr uint32_t kTrainSmem = 161280;
// tensor-memory columns (512 allocated)
constexpr int kCZ1 = 0, kCZ2 = 64, kCZ3 = 128, kCdH2 = 160, kCdW3 = 224, kCdH1 = 304,
              kCdW2 = 368, kCdW1 = 448;
constexpr uint32_t kTrainCols = 512;

// Gradients of the mean squared error over n_total samples x 7 outputs and the summed squared
// error; block b takes the 128-sample tile b of the `count` samples starting at sample `first`
// of the n-sample set (wrapping around). With part == nullptr the tiles add into grad[kParams]
// and *loss atomically (summation order, and so the last bits, vary between runs). Otherwise
// tile b stores its own sums, part[b][kOffMean] (every trained parameter) and part_loss[b], for
// a reduction in a fixed order (adam_kernel), which makes training reproducible bit for bit.
__global__ void __launch_bounds__(128, 1) train_kernel(const float* __restrict__ P, int64_t n,
                                                       const float* __restrict__ in,
                                                       const float* __restrict__ tg,
                                                       int64_t first, int64_t count,
                                                       double n_total, float* __restrict__ grad,
                                                       float* __restrict__ loss,
                                                       float* __restrict__ part,
                                                       float* __restrict__ part_loss, int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float* b2 = (float*)(sm + kTF32);
    float* b3 = b2 + 64;
    float* mean = b3 + 8;
    float* scale = mean + 8;
    float* red = scale + 8;
    float* Atr = red + 32;
    uint64_t* bar = (uint64_t*)(sm + kTBar);
    uint32_t* tbase = (uint32_t*)(sm + kTBar + 8);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // ---- stage weights, constant rows and padding
    for (int i = t; i < 64 * 16; i += 128) {
        const int j = i >> 4, k = i & 15;
        const float w = k < 4 ? P[kOffW1 + 4 * j + k] : 0.0f;
        tc::st_bf16(sm + kTW1, j, k, 16, w);
    }
    for (int i = t; i < 64 * 64; i += 128) {
        const int j = i >> 6, k = i & 63;
        const float w = P[kOffW2 + i];
        tc::st_bf16(sm + kTW2, j, k, 64, w);      // W2[j][k]: out j, in k
        tc::st_bf16(sm + kTW2T, k, j, 64, w);     // W2^T[k][j]
    }
    for (int i = t; i < 16 * 64; i += 128) {
        const int o = i >> 6, j = i & 63;
        const float w = o < kOut ? P[kOffW3 + 64 * o + j] : 0.0f;
        tc::st_bf16(sm + kTW3, o, j, 64, w);
        tc::st_bf16(sm + kTW3T, j, o, 16, w);
    }
    for (int i = t; i < 16 * 128; i += 128) {     // X^T rows 3-15 and X columns 3-15
        const int k = i >> 7, s = i & 127;
        if (k >= 3) {
            tc::st_bf16(sm + kTXT, k, s, 128, k == 3 ? 1.0f : 0.0f);
            tc::st_bf16(sm + kTX, s, k, 16, k == 3 ? 1.0f : 0.0f);
        }
    }
    for (int i = t; i < 16 * 128; i += 128) {     // ones row 64 and zero rows 65-79
        const int r = 64 + (i >> 7), s = i & 127;
        tc::st_bf16(sm + kTH1T, r, s, 128, r == 64 ? 1.0f : 0.0f);
        tc::st_bf16(sm + kTH2T, r, s, 128, r == 64 ? 1.0f : 0.0f);
    }
    for (int i = t; i < 128 * 16; i += 128) {     // dY columns 7-15, dY^T row 7
        const int s = i >> 4, k = i & 15;
        if (k >= kOut) tc::st_bf16(sm + kTdZ3, s, k, 16, 0.0f);
    }
    tc::st_bf16(sm + kTdZ3T, 7, t, 128, 0.0f);
    if (t < 64) b2[t] = P[kOffB2 + t];
    if (t < 8) {
        b3[t] = t < kOut ? P[kOffB3 + t] : 0.0f;
        mean[t] = t < kOut ? P[kOffMean + t] : 0.0f;
        scale[t] = t < kOut ? P[kOffScale + t] : 1.0f;
    }
    if (t < 24) Atr[t] = t < 3 * kOut ? P[kOffA + t] : 0.0f;
    if (warp == 0) tc::tmem_alloc(tbase, kTrainCols);
    if (t == 0) tc::mbar_init(bar, 1);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tbase;
    uint32_t phase = 0;
    bool ok = true;
    auto wait = [&]() -> bool {
        const bool w = tc::mbar_wait(bar, phase, kWaitCycles);
        phase ^= 1u;
        const bool all = __syncthreads_and(w) != 0;
        tc::fence_after_sync();
        return all;
    };
    auto barrier = [&]() {
        tc::fence_smem_to_async();
        tc::fence_before_sync();
        __syncthreads();
    };

    // ---- this thread's sample: block b takes samples first + 128 b + t (mod n), t < count
    const int64_t base = (int64_t)blockIdx.x * 128;
    const bool valid = base + t < count;
    const int64_t i = (first + base + t) % n;
    float f[3] = {0.0f, 0.0f, 0.0f}, tn[7];
    if (valid) {
        f[0] = 2.0f * (in[3 * i] - kLxLo) / (kLxHi - kLxLo) - 1.0f;
        f[1] = 2.0f * (in[3 * i + 1] - kLtLo) / (kLtHi - kLtLo) - 1.0f;
        f[2] = 2.0f * fabsf(in[3 * i + 2]) - 1.0f;
    }
    __syncthreads();   // offset, scale and A staged
    for (int k = 0; k < kOut; ++k)
        tn[k] = valid ? (tg[7 * i + k] - mean[k] - Atr[3 * k] * f[0] - Atr[3 * k + 1] * f[1] -
                         Atr[3 * k + 2] * f[2]) / scale[k]
                      : 0.0f;
    for (int k = 0; k < 3; ++k) {
        tc::st_bf16(sm + kTX, t, k, 16, f[k]);
        tc::st_bf16(sm + kTXT, k, t, 128, f[k]);
    }

    do {
        // ---- forward
        barrier();
        if (t == 0) {
            tc::fence_after_sync();
            tc::gemm_bf16(tm + kCZ1, sm + kTX, sm + kTW1, 64, 16);
            tc::mma_commit(bar);
        }
        if (!(ok = wait())) break;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCZ1 + 16 * c), v);
            for (int j = 0; j < 16; ++j) {
                const float h = silu(v[j]);
                tc::st_bf16(sm + kTH1, t, 16 * c + j, 64, h);
                tc::st_bf16(sm + kTH1T, 16 * c + j, t, 128, h);
            }
        }
        barrier();
        if (t == 0) {
            tc::fence_after_sync();
            tc::gemm_bf16(tm + kCZ2, sm + kTH1, sm + kTW2, 64, 64);
            tc::mma_commit(bar);
        }
        if (!(ok = wait())) break;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCZ2 + 16 * c), v);
            for (int j = 0; j < 16; ++j) {
                const float h = silu(v[j] + b2[16 * c + j]);
                tc::st_bf16(sm + kTH2, t, 16 * c + j, 64, h);
                tc::st_bf16(sm + kTH2T, 16 * c + j, t, 128, h);
            }
        }
        barrier();
        if (t == 0) {
            tc::fence_after_sync();
            tc::gemm_bf16(tm + kCZ3, sm + kTH2, sm + kTW3, 16, 64);
            tc::mma_commit(bar);
        }
        if (!(ok = wait())) break;
        // ---- loss and output error dY = 2 (y - t) / (n_total 7)
        float se = 0.0f;
        {
            float v[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCZ3), v);
            const float sc = (float)(2.0 / (n_total * kOut));
            for (int k = 0; k < kOut; ++k) {
                const float e = valid ? v[k] + b3[k] - tn[k] : 0.0f;
                se += e * e;
                const float dy = sc * e;
                tc::st_bf16(sm + kTdZ3, t, k, 16, dy);
                tc::st_bf16(sm + kTdZ3T, k, t, 128, dy);
            }
        }
        for (int off = 16; off > 0; off >>= 1) se += __shfl_xor_sync(0xffffffffu, se, off);
        if (lane == 0) red[warp] = se;
        // ---- dH2 = dY W3, dW3 (+ db3) = dY^T [H2, 1]
        barrier();
        if (t == 0) {
            tc::fence_after_sync();
            const float tile_loss = red[0] + red[1] + red[2] + red[3];
            if (part_loss) part_loss[blockIdx.x] = tile_loss;
            else atomicAdd(loss, tile_loss);
            tc::gemm_bf16(tm + kCdH2, sm + kTdZ3, sm + kTW3T, 64, 16);
            tc::gemm_bf16(tm + kCdW3, sm + kTdZ3T, sm + kTH2T, 80, 128);
            tc::mma_commit(bar);
        }
        if (!(ok = wait())) break;
        // ---- dZ2 = dH2 * silu'(Z2)
        for (int c = 0; c < 4; ++c) {
            float dh[16], z[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCdH2 + 16 * c), dh);
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCZ2 + 16 * c), z);
            for (int j = 0; j < 16; ++j) {
                const float d = dh[j] * silu_grad(z[j] + b2[16 * c + j]);
                tc::st_bf16(sm + kTdZ2, t, 16 * c + j, 64, d);
                tc::st_bf16(sm + kTdZ2T, 16 * c + j, t, 128, d);
            }
        }
        // ---- dH1 = dZ2 W2, dW2 (+ db2) = dZ2^T [H1, 1]
        barrier();
        if (t == 0) {
            tc::fence_after_sync();
            tc::gemm_bf16(tm + kCdH1, sm + kTdZ2, sm + kTW2T, 64, 64);
            tc::gemm_bf16(tm + kCdW2, sm + kTdZ2T, sm + kTH1T, 80, 128);
            tc::mma_commit(bar);
        }
        if (!(ok = wait())) break;
        // ---- dZ1 = dH1 * silu'(Z1)
        for (int c = 0; c < 4; ++c) {
            float dh[16], z[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCdH1 + 16 * c), dh);
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCZ1 + 16 * c), z);
            for (int j = 0; j < 16; ++j)
                tc::st_bf16(sm + kTdZ1T, 16 * c + j, t, 128, dh[j] * silu_grad(z[j]));
        }
        // ---- dW1 (+ db1 in column 3) = dZ1^T X
        barrier();
        if (t == 0) {
            tc::fence_after_sync();
            tc::gemm_bf16(tm + kCdW1, sm + kTdZ1T, sm + kTXT, 16, 128);
            tc::mma_commit(bar);
        }
        if (!(ok = wait())) break;
        // ---- accumulate this tile's weight gradients (rows = units: lanes 0-63)
        float* const own = part ? part + (size_t)blockIdx.x * kOffMean : nullptr;
        auto put = [&](int idx, float val) {
            if (own) own[idx] = val;
            else atomicAdd(&grad[idx], val);
        };
        if (warp < 2) {
            const int j = t;                    // unit of layers 1 and 2
            for (int c = 0; c < 5; ++c) {       // dW2 columns 0-63, db2 in column 64
                float v[16];
                tc::tmem_ld16(tc::tmem_lane_addr(tm, kCdW2 + 16 * c), v);
                for (int q = 0; q < 16; ++q) {
                    const int col = 16 * c + q;
                    if (col < 64) put(kOffW2 + 64 * j + col, v[q]);
                    else if (col == 64) put(kOffB2 + j, v[q]);
                }
            }
            float v[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tm, kCdW1), v);
            for (int q = 0; q < 4; ++q) put(kOffW1 + 4 * j + q, v[q]);
        }
        if (warp == 0) {
            for (int c = 0; c < 5; ++c) {       // dW3 rows 0-6, db3 in column 64
                float v[16];
                tc::tmem_ld16(tc::tmem_lane_addr(tm, kCdW3 + 16 * c), v);
                if (lane < kOut)
                    for (int q = 0; q < 16; ++q) {
                        const int col = 16 * c + q;
                        if (col < 64) put(kOffW3 + 64 * lane + col, v[q]);
                        else if (col == 64) put(kOffB3 + lane, v[q]);
                    }
            }
        }
    } while (false);
    if (!ok) {
        if (t == 0) atomicExch(err, 1);
        tc::mbar_wait(bar, phase ^ 1u, kWaitCycles);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, kTrainCols);
}

// One Adam step (Kingma & Ba 2015) on every trained parameter; clears the gradient. c1, c2
// are the bias corrections 1 - beta1^t, 1 - beta2^t. Also moves the step's summed squared
// error into loss_hist (mean over n_total x 7) and clears it.
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ part, int n_tiles,
                            float* __restrict__ m, float* __restrict__ v, float lr, float beta1,
                            float beta2, float eps, float c1, float c2,
                            const float* __restrict__ part_loss, float* loss_hist,
                            float inv_count) {
    // one Adam step from the tiles' gradient sums, added in tile order
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss_hist) {
        float l = 0.0f;
        for (int b = 0; b < n_tiles; ++b) l += part_loss[b];
        *loss_hist = l * inv_count;
    }
    if (i >= kOffMean) return;
    float g = 0.0f;
    for (int b = 0; b < n_tiles; ++b) g += part[(size_t)b * kOffMean + i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// n uniform samples of the input box (SplitMix64 stream `seed`: draws 3i, 3i+1, 3i+2) and
// their targets from the exact fits.
__global__ void dataset_kernel(int64_t n, uint64_t seed, float* __restrict__ in,
                               float* __restrict__ tg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lx = kLxLo + (kLxHi - kLxLo) * uniform01(seed, 3 * i);
    const double lt = kLtLo + (kLtHi - kLtLo) * uniform01(seed, 3 * i + 1);
    const double c = uniform01(seed, 3 * i + 2);
    in[3 * i] = (float)lx;
    in[3 * i + 1] = (float)lt;
    in[3 * i + 2] = (float)c;
    double o[7];
    exact_targets((double)(float)lx, (double)(float)lt, o);
    for (int k = 0; k < kOut; ++k) tg[7 * i + k] = (float)o[k];
}

__global__ void targets_kernel(int64_t n, const float* __restrict__ in, float* __restrict__ tg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double o[7];
    exact_targets((double)in[3 * i], (double)in[3 * i + 1], o);
    for (int k = 0; k < kOut; ++k) tg[7 * i + k] = (float)o[k];
}

// Glorot-uniform weights from SplitMix64 stream `seed` (draw i for parameter i), zero biases,
// output mean 0 and scale 1.
__global__ void init_kernel(float* __restrict__ P, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float u = (float)(2.0 * uniform01(seed, (uint64_t)i) - 1.0);
    float v = 0.0f;
    if (i < kOffW2) v = (i & 3) == 3 ? 0.0f : u * sqrtf(6.0f / (3 + 64));
    else if (i < kOffB2) v = u * sqrtf(6.0f / (64 + 64));
    else if (i >= kOffW3 && i < kOffB3) v = u * sqrtf(6.0f / (64 + 7));
    else if (i >= kOffScale && i < kOffA) v = 1.0f;
    P[i] = v;
}

// Offset, trend A and scale of the model from n training samples (one block of 256 threads):
// least squares of the targets on (f, 1), f the mapped inputs, by the normal equations in
// double precision, and the root mean square of the residual.
__device__ __forceinline__ void features_of(const float* in, int64_t i, double f[4]) {
    f[0] = 2.0f * (in[3 * i] - kLxLo) / (kLxHi - kLxLo) - 1.0f;
    f[1] = 2.0f * (in[3 * i + 1] - kLtLo) / (kLtHi - kLtLo) - 1.0f;
    f[2] = 2.0f * fabsf(in[3 * i + 2]) - 1.0f;
    f[3] = 1.0;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    return s;
}

__global__ void normalise_kernel(int64_t n, const float* __restrict__ in,
                                 const float* __restrict__ tg, float* __restrict__ P) {
    __shared__ double sh[32];
    __shared__ double G[4][4], R[4][7], beta[4][7];
    // normal equations: G = sum f f^T, R = sum f o^T
    double g[10], r[28];
    for (int q = 0; q < 10; ++q) g[q] = 0.0;
    for (int q = 0; q < 28; ++q) r[q] = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double f[4];
        features_of(in, i, f);
        int q = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = a; b < 4; ++b) g[q++] += f[a] * f[b];
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < kOut; ++k) r[7 * a + k] += f[a] * (double)tg[7 * i + k];
    }
    {
        int q = 0;
        for (int a = 0; a < 4; ++a)
            for (int b = a; b < 4; ++b) {
                const double v = block_sum(g[q++], sh);
                if (threadIdx.x == 0) { G[a][b] = v; G[b][a] = v; }
            }
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < kOut; ++k) {
                const double v = block_sum(r[7 * a + k], sh);
                if (threadIdx.x == 0) R[a][k] = v;
            }
    }
    if (threadIdx.x == 0) {
        // Gaussian elimination with partial pivoting on [G | R]
        double M[4][11];
        for (int a = 0; a < 4; ++a) {
            for (int b = 0; b < 4; ++b) M[a][b] = G[a][b];
            for (int k = 0; k < kOut; ++k) M[a][4 + k] = R[a][k];
        }
        for (int c = 0; c < 4; ++c) {
            int p = c;
            for (int a = c + 1; a < 4; ++a) if (fabs(M[a][c]) > fabs(M[p][c])) p = a;
            for (int b = 0; b < 11; ++b) { const double tmp = M[c][b]; M[c][b] = M[p][b]; M[p][b] = tmp; }
            for (int a = c + 1; a < 4; ++a) {
                const double fct = M[a][c] / M[c][c];
                for (int b = c; b < 11; ++b) M[a][b] -= fct * M[c][b];
            }
        }
        for (int k = 0; k < kOut; ++k)
            for (int a = 3; a >= 0; --a) {
                double v = M[a][4 + k];
                for (int b = a + 1; b < 4; ++b) v -= M[a][b] * beta[b][k];
                beta[a][k] = v / M[a][a];
            }
    }
    __syncthreads();
    // residual root mean square
    double e[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double f[4];
        features_of(in, i, f);
        for (int k = 0; k < kOut; ++k) {
            const double d = (double)tg[7 * i + k] - (beta[0][k] * f[0] + beta[1][k] * f[1] +
                                                      beta[2][k] * f[2] + beta[3][k]);
            e[k] += d * d;
        }
    }
    for (int k = 0; k < kOut; ++k) {
        const double v = block_sum(e[k], sh);
        if (threadIdx.x == 0) {
            const double rms = sqrt(v / (double)n);
            P[kOffMean + k] = (float)beta[3][k];
            P[kOffScale + k] = (float)(rms > 1e-30 ? rms : 1.0);
            for (int a = 0; a < 3; ++a) P[kOffA + 3 * k + a] = (float)beta[a][k];
        }
    }
}

// Self-test of the bounded mbarrier wait: with arrive = 0 nothing arrives and the wait must
// run out after max_cycles (sets *err); with arrive = 1 the barrier's phase completes first.
__global__ void wait_selftest_kernel(long long max_cycles, int arrive, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(&bar)) : "memory");
    __syncthreads();
    const bool ok = tc::mbar_wait(&bar, 0u, max_cycles);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace mlp
}  // namespace bl
