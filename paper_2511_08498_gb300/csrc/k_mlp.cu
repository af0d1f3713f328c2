// Learned Voigt-profile surrogate: a 3 -> 64 -> 64 -> 1 multilayer perceptron
// with tanh-form GELU activations that predicts ln H(a, x - u) from the
// wavelength offset x (Doppler widths, rest frame), the damping a and the
// projected velocity u (Doppler widths).  It stands in for the on-the-fly
// profile evaluation of the Core-and-Voigt treatment (Section 3.2); the exact
// HUM1WEI24 evaluation remains the fallback and the accuracy reference.
//
// Precision: weights are used as BF16 (rounded from an FP32 master copy), the
// hidden activations that feed the tensor cores are BF16, every sum is FP32.
//
// Tensor cores (tcgen05, kind::f16, accumulators in tensor memory) do every
// contraction over the hidden width or over the samples of a tile; CUDA cores
// do the 3-input first layer, the activations and the output dot product.
// One CTA of 128 threads owns tiles of 128 samples, thread t = sample t = TMEM
// lane t.  Per tile:
//   forward   D2 = H1 W2^T                      (M 128, N 64, K 64)
//   backward  D3 = Delta2 W2                    (M 128, N 64, K 64)   -> dL/dh1
//             D4 += [Delta2^T; (dy h2)^T] [H1^T; 1]^T
//                                               (M 128, N 80, K 128)  -> dW2, db2, dw3
//             D5 += Delta1^T [F^T; 1]^T         (M 128, N 16, K 128)  -> dW1, db1
// (tensor-memory columns: D2 0-63, D3 64-127, D4 128-207, D5 224-239 of 256)
// D4 and D5 accumulate over all tiles of the CTA and are added to the global
// gradient once at the end.  Every mbarrier wait is bounded; on expiry the CTA
// records DEX_ERR_TIMEOUT, waits (bounded) once more, frees its tensor memory
// and returns.
#include <cmath>
#include <cstddef>

#include "dex_internal.h"
#include "mlp.cuh"
#include "umma.cuh"
#include "voigt.cuh"

namespace dex {

namespace {

using namespace umma;
using mlp::Act;
using mlp::gelu;
using mlp::kB1;
using mlp::kB2;
using mlp::kB3;
using mlp::kH;
using mlp::kW1;
using mlp::kW2;
using mlp::kW3;

constexpr int kTile = 128;  // samples per tile (MMA M)
constexpr int kWaitPolls = 1 << 20;

// tile geometry (rows R of each K-major operand)
constexpr int kRowsH1T = 80;  // 64 hidden units, the ones row 64, zero rows 65..79
constexpr int kRowsFT = 16;   // 3 features, the ones row 3, zero rows 4..15

// TMEM columns
constexpr uint32_t kColD2 = 0, kColD3 = 64, kColD4 = 128, kColD5 = 224;
constexpr uint32_t kColsTrain = 256, kColsInfer = 64;

struct SmemInfer {
    unsigned char W2[kH * kH * 2];        // B of D2: rows out j, K in i
    unsigned char H1[kTile * kH * 2];     // A of D2: rows sample, K in i
    float w1[kH * 3], b1[kH], b2[kH], w3[kH], b3;
    alignas(16) float w1t[3][kH];         // w1 by input feature: neighbouring units side by side
    unsigned long long mbar;
    unsigned int tmem;
};

struct SmemTrain {
    unsigned char W2[kH * kH * 2];              // B of D2
    unsigned char W2T[kH * kH * 2];             // B of D3: rows in i, K out j
    unsigned char H1[kTile * kH * 2];           // A of D2
    unsigned char D2[kTile * kH * 2];           // A of D3: rows sample, K out j
    unsigned char D2T[kTile * kTile * 2];       // A of D4 (rows j: delta2, rows 64 + j: dy h2), then A of D5
    unsigned char H1T[kRowsH1T * kTile * 2];    // B of D4: rows i (+ ones row), K sample
    unsigned char FT[kRowsFT * kTile * 2];      // B of D5: rows feature (+ ones row), K sample
    float w1[kH * 3], b1[kH], b2[kH], w3[kH], b3;
    float red_loss[4], red_gb3[4];
    unsigned long long mbar;
    unsigned int tmem;
};

// dynamic shared memory requested per CTA: at most 4 inference / 2 training
// CTAs fit on an SM, so their tensor-memory allocations always fit (512 columns)
constexpr size_t kSmemInfer = 48 * 1024;
constexpr size_t kSmemTrain = 110 * 1024;
static_assert(sizeof(SmemInfer) <= kSmemInfer, "inference shared memory");
// the packed inference loads read float2 pairs of these arrays at even indices
static_assert(offsetof(SmemInfer, b1) % 8 == 0 && offsetof(SmemInfer, b2) % 8 == 0 &&
                  offsetof(SmemInfer, w3) % 8 == 0 && offsetof(SmemInfer, w1t) % 8 == 0,
              "inference weight alignment");
static_assert(sizeof(SmemTrain) <= kSmemTrain, "training shared memory");

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void put_bf16(unsigned char* tile, int off, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(tile + off) = __float2bfloat16_rn(v);
}

// input features: x / 16, log10(a) + 2, u / 16; false (and zeros) for a
// non-finite input or a <= 0
__device__ __forceinline__ bool features(const float* xau, long long s, float* f)
{
    const float x = xau[3 * s], a = xau[3 * s + 1], u = xau[3 * s + 2];
    if (!(a > 0.0f) || !isfinite(a) || !isfinite(x) || !isfinite(u)) {
        f[0] = f[1] = f[2] = 0.0f;
        return false;
    }
    mlp::features(x, a, u, f);
    return true;
}

template <class S>
__device__ void stage_weights(S& sm, const float* __restrict__ p, bool transposed_copy, unsigned char* W2T)
{
    const int t = threadIdx.x;
    for (int q = t; q < kH * kH; q += blockDim.x) {
        const int j = q / kH, i = q - j * kH;
        const float w = p[kW2 + q];
        put_bf16(sm.W2, tile_offset(j, i, kH), w);
        if (transposed_copy) put_bf16(W2T, tile_offset(i, j, kH), w);
    }
    for (int q = t; q < kH * 3; q += blockDim.x) sm.w1[q] = bf16_round(p[kW1 + q]);
    if (t < kH) {
        sm.b1[t] = p[kB1 + t];
        sm.b2[t] = p[kB2 + t];
        sm.w3[t] = bf16_round(p[kW3 + t]);
    }
    if (t == 0) sm.b3 = p[kB3];
}

// layer 1 + GELU for sample row t: writes h1 (BF16) to H1 (row t), and when
// H1T is given to H1T (column t); returns nothing else (z1 is recomputed).
template <class S>
__device__ __forceinline__ void layer1(S& sm, const float* f, int t, unsigned char* H1T)
{
#pragma unroll 1
    for (int i0 = 0; i0 < kH; i0 += 8) {
        __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q;
            const float z = fmaf(sm.w1[3 * i + 2], f[2], fmaf(sm.w1[3 * i + 1], f[1], fmaf(sm.w1[3 * i], f[0], sm.b1[i])));
            hb[q] = __float2bfloat16_rn(gelu(z).g);
            if (H1T) *reinterpret_cast<__nv_bfloat16*>(H1T + tile_offset(i, t, kRowsH1T)) = hb[q];
        }
        *reinterpret_cast<uint4*>(sm.H1 + tile_offset(t, i0, kTile)) = *reinterpret_cast<const uint4*>(hb);
    }
}

// GELU of two hidden units at once on the packed FP32 pipe (FMUL2/FFMA2/FADD2):
// every lane rounded exactly as mlp::gelu(z).g
__device__ __forceinline__ float2 gelu2(float2 z)
{
    const float c = 0.79788456080286536f, k = 0.044715f;
    const float m2log2e = -2.8853900817779268f;
    const float2 z2 = __fmul2_rn(z, z);
    const float2 u = __fmul2_rn(__fmul2_rn(make_float2(c, c), z), __ffma2_rn(make_float2(k, k), z2, make_float2(1.0f, 1.0f)));
    const float2 a = __fmul2_rn(u, make_float2(m2log2e, m2log2e));
    const float2 d = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(mlp::mlp_ex2(a.x), mlp::mlp_ex2(a.y)));
    return __fmul2_rn(z, make_float2(mlp::mlp_rcp(d.x), mlp::mlp_rcp(d.y)));
}

// layer 1 + GELU for sample row t (inference): units in pairs on the packed pipe,
// every value rounded as in layer1()
__device__ __forceinline__ void layer1_infer(SmemInfer& sm, const float* f, int t)
{
    const float2 f0 = make_float2(f[0], f[0]), f1 = make_float2(f[1], f[1]), f2 = make_float2(f[2], f[2]);
#pragma unroll 1
    for (int i0 = 0; i0 < kH; i0 += 8) {
        __align__(16) __nv_bfloat162 hb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + 2 * q;
            const float2 b = *reinterpret_cast<const float2*>(&sm.b1[i]);
            const float2 w0 = *reinterpret_cast<const float2*>(&sm.w1t[0][i]);
            const float2 w1 = *reinterpret_cast<const float2*>(&sm.w1t[1][i]);
            const float2 w2 = *reinterpret_cast<const float2*>(&sm.w1t[2][i]);
            const float2 z = __ffma2_rn(w2, f2, __ffma2_rn(w1, f1, __ffma2_rn(w0, f0, b)));
            hb[q] = __float22bfloat162_rn(gelu2(z));
        }
        *reinterpret_cast<uint4*>(sm.H1 + tile_offset(t, i0, kTile)) = *reinterpret_cast<const uint4*>(hb);
    }
}

// one MMA chain: D (+)= A B^T over K/16 K-steps, issued by the calling thread
__device__ __forceinline__ void mma_chain(uint32_t d, const unsigned char* A, int rowsA, const unsigned char* B,
                                          int rowsB, int K, uint32_t idesc, bool accumulate)
{
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    for (int k = 0; k < K / 16; ++k)
        mma_bf16(d, smem_desc(a0 + k * kstep_bytes(rowsA)), smem_desc(b0 + k * kstep_bytes(rowsB)), idesc,
                 accumulate || k > 0);
}

// make every thread's shared-memory writes and TMEM reads ordered before the
// MMAs thread 0 issues next
__device__ __forceinline__ void sync_for_mma()
{
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// bounded wait by every thread; returns true on success for the whole CTA
__device__ __forceinline__ bool wait_all(unsigned long long* mbar, uint32_t& phase)
{
    const bool ok = mbar_wait(mbar, phase, kWaitPolls);
    phase ^= 1u;
    const bool all = !__syncthreads_or(ok ? 0 : 1);
    fence_after_sync();
    return all;
}

// ------------------------------------------------------------ inference --
__global__ void __launch_bounds__(128, 1) k_mlp_forward(const MlpParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SmemInfer& sm = *reinterpret_cast<SmemInfer*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    stage_weights(sm, P.params, false, nullptr);
    for (int q = t; q < kH * 3; q += blockDim.x) sm.w1t[q % 3][q / 3] = bf16_round(P.params[kW1 + q]);
    if (t == 0) mbar_init(&sm.mbar, 1);
    if (warp == 0) tmem_alloc(&sm.tmem, kColsInfer);
    sync_for_mma();
    const uint32_t tm = sm.tmem;
    uint32_t phase = 0;
    const long long n_tiles = (P.n + kTile - 1) / kTile;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long long s = tile * kTile + t;
        bool valid = s < P.n;
        float f[3] = {0.0f, 0.0f, 0.0f};
        if (valid && !features(P.xau, s, f)) {
            raise_status(P.status, DEX_ERR_NUMERIC);
            valid = false;
        }
        layer1_infer(sm, f, t);
        sync_for_mma();
        if (t == 0) {
            mma_chain(tm + kColD2, sm.H1, kTile, sm.W2, kH, kH, idesc_bf16_f32(kTile, kH), false);
            mma_commit(&sm.mbar);
        }
        if (!(ok = wait_all(&sm.mbar, phase))) break;
        // output unit: two partial sums (even and odd hidden units) on the packed pipe
        float2 y2 = make_float2(sm.b3, 0.0f);
#pragma unroll 1
        for (int c = 0; c < kH; c += 16) {
            float z[16];
            tmem_ld16(tmem_at(tm, warp * 32, kColD2 + c), z);
#pragma unroll
            for (int q = 0; q < 16; q += 2) {
                const float2 b = *reinterpret_cast<const float2*>(&sm.b2[c + q]);
                const float2 w = *reinterpret_cast<const float2*>(&sm.w3[c + q]);
                y2 = __ffma2_rn(w, gelu2(__fadd2_rn(make_float2(z[q], z[q + 1]), b)), y2);
            }
        }
        const float y = y2.x + y2.y;
        if (valid) P.out[s] = y;
    }
    if (!ok) {
        raise_status(P.status, DEX_ERR_TIMEOUT);
        mbar_wait(&sm.mbar, phase ^ 1u, kWaitPolls);  // the MMA still in flight, if any
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, kColsInfer);
}

// ------------------------------------------------------------- training --
__global__ void __launch_bounds__(128, 1) k_mlp_grad(const MlpParams P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SmemTrain& sm = *reinterpret_cast<SmemTrain*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    stage_weights(sm, P.params, true, sm.W2T);
    // constant rows: H1T row 64 = 1, rows 65..79 = 0; FT row 3 = 1, rows 4..15 = 0
    for (int q = t; q < (kRowsH1T - kH) * kTile; q += blockDim.x) {
        const int r = kH + q / kTile, k = q % kTile;
        put_bf16(sm.H1T, tile_offset(r, k, kRowsH1T), r == kH ? 1.0f : 0.0f);
    }
    for (int q = t; q < (kRowsFT - 3) * kTile; q += blockDim.x) {
        const int r = 3 + q / kTile, k = q % kTile;
        put_bf16(sm.FT, tile_offset(r, k, kRowsFT), r == 3 ? 1.0f : 0.0f);
    }
    if (t == 0) mbar_init(&sm.mbar, 1);
    if (warp == 0) tmem_alloc(&sm.tmem, kColsTrain);
    sync_for_mma();
    const uint32_t tm = sm.tmem;
    uint32_t phase = 0;
    const long long n_tiles = (P.n + kTile - 1) / kTile;
    bool ok = true, any = false;
    float loss = 0.0f, gb3 = 0.0f;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long long s = tile * kTile + t;
        bool valid = s < P.n;
        float f[3] = {0.0f, 0.0f, 0.0f}, target = 0.0f;
        if (valid) {
            target = P.target[s];
            if (!features(P.xau, s, f) || !isfinite(target)) {
                raise_status(P.status, DEX_ERR_NUMERIC);
                valid = false;
                f[0] = f[1] = f[2] = 0.0f;
            }
        }
        layer1(sm, f, t, sm.H1T);
#pragma unroll
        for (int k = 0; k < 3; ++k) put_bf16(sm.FT, tile_offset(k, t, kRowsFT), f[k]);
        sync_for_mma();
        if (t == 0) {
            mma_chain(tm + kColD2, sm.H1, kTile, sm.W2, kH, kH, idesc_bf16_f32(kTile, kH), false);
            mma_commit(&sm.mbar);
        }
        if (!(ok = wait_all(&sm.mbar, phase))) break;

        // forward output (first pass over z2 in tensor memory), then dy
        float y = sm.b3;
#pragma unroll 1
        for (int c = 0; c < kH; c += 16) {
            float z[16];
            tmem_ld16(tmem_at(tm, warp * 32, kColD2 + c), z);
#pragma unroll
            for (int q = 0; q < 16; ++q) y = fmaf(sm.w3[c + q], gelu(z[q] + sm.b2[c + q]).g, y);
        }
        const float r = valid ? y - target : 0.0f;
        const float dy = 2.0f * r;
        loss = fmaf(r, r, loss);
        gb3 += dy;
        // second pass: delta2 = dy w3 g'(z2) into the rows of D2 (K-major by j) and
        // the columns of D2T, dy h2 into the columns of D2T's rows 64 + j
#pragma unroll 1
        for (int c = 0; c < kH; c += 16) {
            float z[16];
            tmem_ld16(tmem_at(tm, warp * 32, kColD2 + c), z);
            __align__(16) __nv_bfloat16 db[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = c + q;
                const Act a = gelu(z[q] + sm.b2[j]);
                db[q] = __float2bfloat16_rn(dy * sm.w3[j] * a.dg);
                *reinterpret_cast<__nv_bfloat16*>(sm.D2T + tile_offset(j, t, kTile)) = db[q];
                put_bf16(sm.D2T, tile_offset(kH + j, t, kTile), dy * a.g);
            }
            *reinterpret_cast<uint4*>(sm.D2 + tile_offset(t, c, kTile)) = *reinterpret_cast<const uint4*>(db);
            *reinterpret_cast<uint4*>(sm.D2 + tile_offset(t, c + 8, kTile)) = *reinterpret_cast<const uint4*>(db + 8);
        }
        sync_for_mma();
        if (t == 0) {
            mma_chain(tm + kColD3, sm.D2, kTile, sm.W2T, kH, kH, idesc_bf16_f32(kTile, kH), false);
            mma_chain(tm + kColD4, sm.D2T, kTile, sm.H1T, kRowsH1T, kTile, idesc_bf16_f32(kTile, kRowsH1T), any);
            mma_commit(&sm.mbar);
        }
        if (!(ok = wait_all(&sm.mbar, phase))) break;

        // delta1 = (dL/dh1) g'(z1) into the columns of the D2T buffer (rows 0..63)
#pragma unroll 1
        for (int c = 0; c < kH; c += 16) {
            float dh[16];
            tmem_ld16(tmem_at(tm, warp * 32, kColD3 + c), dh);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = c + q;
                const float z1 =
                    fmaf(sm.w1[3 * i + 2], f[2], fmaf(sm.w1[3 * i + 1], f[1], fmaf(sm.w1[3 * i], f[0], sm.b1[i])));
                put_bf16(sm.D2T, tile_offset(i, t, kTile), dh[q] * gelu(z1).dg);
            }
        }
        sync_for_mma();
        if (t == 0) {
            mma_chain(tm + kColD5, sm.D2T, kTile, sm.FT, kRowsFT, kTile, idesc_bf16_f32(kTile, kRowsFT), any);
            mma_commit(&sm.mbar);
        }
        if (!(ok = wait_all(&sm.mbar, phase))) break;
        any = true;
    }
    if (!ok) {
        raise_status(P.status, DEX_ERR_TIMEOUT);
        mbar_wait(&sm.mbar, phase ^ 1u, kWaitPolls);
    } else {
        const float inv_n = 1.0f / (float)P.n;
        // loss and db3: warp sums, then one atomic per CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loss += __shfl_xor_sync(0xffffffffu, loss, o);
            gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
        }
        if (lane == 0) {
            sm.red_loss[warp] = loss;
            sm.red_gb3[warp] = gb3;
        }
        __syncthreads();
        if (t == 0 && any) {
            atomicAdd(P.loss, (sm.red_loss[0] + sm.red_loss[1] + sm.red_loss[2] + sm.red_loss[3]) * inv_n);
            atomicAdd(P.grad + kB3, (sm.red_gb3[0] + sm.red_gb3[1] + sm.red_gb3[2] + sm.red_gb3[3]) * inv_n);
        }
        if (any) {
            // D4 row r < 64: dW2[r][0..63], db2[r] (column 64); row 64 + j: dw3[j] (column 64)
            float v[16];
#pragma unroll 1
            for (int c = 0; c < kH; c += 16) {
                tmem_ld16(tmem_at(tm, warp * 32, kColD4 + c), v);
                if (t < kH)
#pragma unroll
                    for (int q = 0; q < 16; ++q) atomicAdd(P.grad + kW2 + t * kH + c + q, v[q] * inv_n);
            }
            tmem_ld16(tmem_at(tm, warp * 32, kColD4 + kH), v);
            if (t < kH) atomicAdd(P.grad + kB2 + t, v[0] * inv_n);
            else atomicAdd(P.grad + kW3 + (t - kH), v[0] * inv_n);
            // D5 row r < 64: dW1[r][0..2], db1[r] (column 3)
            tmem_ld16(tmem_at(tm, warp * 32, kColD5), v);
            if (t < kH) {
#pragma unroll
                for (int k = 0; k < 3; ++k) atomicAdd(P.grad + kW1 + 3 * t + k, v[k] * inv_n);
                atomicAdd(P.grad + kB1 + t, v[3] * inv_n);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, kColsTrain);
}

// ----------------------------------------------------------------- Adam --
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = fmaf(b1, m[q], (1.0f - b1) * gq);
    const float vq = fmaf(b2, v[q], (1.0f - b2) * gq * gq);
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq * c1) / (sqrtf(vq * c2) + eps);
}

// ------------------------------------------------------ training targets --
__global__ void k_mlp_targets(long long n, const float* __restrict__ xau, float* __restrict__ out, VoigtCoef C)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    out[s] = logf(voigt_h(C, xau[3 * s + 1], xau[3 * s] - xau[3 * s + 2]));
}

}  // namespace

int mlp_param_count() { return mlp::kParams; }

static int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

cudaError_t launch_mlp_forward(cudaStream_t s, const MlpParams& P)
{
    if (P.n == 0) return cudaSuccess;
    const int sms = sm_count();
    if (sms == 0) return cudaErrorInvalidDevice;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemInfer);
    if (e != cudaSuccess) return e;
    const long long tiles = (P.n + kTile - 1) / kTile;
    const long long grid = tiles < 4LL * sms ? tiles : 4LL * sms;
    k_mlp_forward<<<(unsigned)grid, 128, kSmemInfer, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(cudaStream_t s, const MlpParams& P)
{
    cudaError_t e = cudaMemsetAsync(P.grad, 0, sizeof(float) * mlp_param_count(), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.loss, 0, sizeof(float), s);
    if (e != cudaSuccess || P.n == 0) return e;
    const int sms = sm_count();
    if (sms == 0) return cudaErrorInvalidDevice;
    e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTrain);
    if (e != cudaSuccess) return e;
    const long long tiles = (P.n + kTile - 1) / kTile;
    const long long grid = tiles < 2LL * sms ? tiles : 2LL * sms;
    k_mlp_grad<<<(unsigned)grid, 128, kSmemTrain, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(cudaStream_t s, float* p, const float* g, float* m, float* v, int step, float lr,
                            float b1, float b2, float eps)
{
    const int n = mlp_param_count();
    const float c1 = (float)(1.0 / (1.0 - pow((double)b1, step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)b2, step)));
    k_mlp_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_targets(cudaStream_t s, long long n, const float* xau, float* out)
{
    if (n == 0) return cudaSuccess;
    k_mlp_targets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, xau, out, voigt_coefficients());
    return cudaGetLastError();
}

}  // namespace dex
