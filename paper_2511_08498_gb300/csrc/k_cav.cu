// "Core and Voigt" (CaV) treatment of a moving medium (Section 3.2): the line
// profile is evaluated on the fly per segment and wavelength from MIP chains of
// the direction-independent line parameters.
//
// Voxel record (8 floats, the same for every wavelength): eta*, chi*, damping a,
// 1/v_th, v_x, v_z, eta_c, chi_c (velocities and v_th in km/s, wavelengths as
// velocity offsets dv from the rest wavelength).  For propagation direction w
// (= -d of the traced ray) and wavelength dv:
//   u = dv + v.w,  s = lambda0/lambda = 1/(1 + dv/c),  phi = H(a/s^2, u/v_th) / (sqrt(pi) v_th),
//   eta = eta* s phi + eta_c,  chi = chi* s phi + chi_c          (Section 3.2 scalings)
// with H by HUM1WEI24.  The traversal is the shared hierarchical DDA (hdda.cuh).
//
// Level selection (k_cav_mips_build): box-filter chains of the 8 parameters;
// a 2x2 group of level m passes when the IoD of ln(eta Ds), ln(chi Ds) of its
// children -- each evaluated at the Doppler shift closest to line centre that
// its speed allows, |u| = max(0, |dv| - |v|) -- is below the thresholds, or the
// largest such chi Ds is below chi_ds_min; the block level is the largest m with
// every group of every level <= m passing for every wavelength of the batch.
// With n_test_dirs = K > 0 a group must also pass the same test on its children
// evaluated as a ray along each w_k samples them, u = dv + v_child . w_k: the
// closest-to-core values of children moving in different directions can agree
// while the profiles a ray sees are shifted apart.
#include "hdda.cuh"
#include "mlp.cuh"
#include "vlm.cuh"
#include "voigt.cuh"

namespace dex {

namespace {

constexpr int kCavStride = 8;

// eta, chi of one voxel at propagation-projected shift u for wavelength l
__device__ __forceinline__ void cav_eta_chi(const CavParams& M, const float* v, int l, float u, float& eta, float& chi)
{
    const float inv = v[3];
    const float H = voigt_h(M.coef, v[2] * M.is2[l], u * inv);
    const float phi = H * inv * kInvSqrtPi;
    const float sl = M.s[l];
    eta = fmaf(v[0] * sl, phi, v[6]);
    chi = fmaf(v[1] * sl, phi, v[7]);
}

// The same treatment with the learned surrogate as the profile: inside the
// surrogate's training domain H = exp(network(x, a', u)) with x = dv / v_th,
// a' = a / s^2 and u = -(v.w) / v_th (so that x - u is the Voigt argument);
// outside it, and as its accuracy reference, the HUM1WEI24 evaluation above.  The network
// runs in float32 on the CUDA cores, one evaluation per segment and wavelength,
// with its weights in the kernel's parameter space.
__device__ __forceinline__ float surrogate_or_exact(const CavMlpParams& M, float a, float x, float u)
{
    if (a >= mlp::kAMin && a <= mlp::kAMax && fabsf(x) <= mlp::kXMax && fabsf(u) <= mlp::kUMax)
        return __expf(mlp::ln_h_fp32(M.w, x, a, u));
    return voigt_h(M.cav.coef, a, x - u);
}

template <int W>
struct CavMlpModel {
    static constexpr int kStride = kCavStride;
    static constexpr bool kPerBatch = false;
    static constexpr int kMinBlocks = 1;  // the network's 64 hidden values stay in registers
    static constexpr bool kEarlyLoad = false;
    static constexpr bool kZeroNoop = false;  // profile parameters of zero are not a no-op
    using Params = CavMlpParams;
    struct Voxel {
        float p[kCavStride];
    };
    __device__ __forceinline__ static Voxel load(const float* q)
    {
        Voxel v;
        const float4 a = __ldg(reinterpret_cast<const float4*>(q)), b = __ldg(reinterpret_cast<const float4*>(q) + 1);
        v.p[0] = a.x; v.p[1] = a.y; v.p[2] = a.z; v.p[3] = a.w;
        v.p[4] = b.x; v.p[5] = b.y; v.p[6] = b.z; v.p[7] = b.w;
        return v;
    }
    __device__ __forceinline__ static void integrate(const Params& M, const Voxel& v, int b, float wx, float wz,
                                                     float nl2, float* I, float* T)
    {
        const float proj = fmaf(v.p[4], wx, v.p[5] * wz);
        const float inv = v.p[3];
        const float u = -proj * inv;
#pragma unroll 1
        for (int w = 0; w < W; ++w) {
            const int l = b * W + w;
            const float H = surrogate_or_exact(M, v.p[2] * M.cav.is2[l], M.cav.dv[l] * inv, u);
            const float phi = H * inv * kInvSqrtPi;
            const float sl = M.cav.s[l];
            const float eta = fmaf(v.p[0] * sl, phi, v.p[6]);
            const float chi = fmaf(v.p[1] * sl, phi, v.p[7]);
            const float S = chi > 0.0f ? __fdividef(eta, chi) : 0.0f;
            segment(S, chi, nl2, I[w], T[w]);
        }
    }
};

template <int W>
struct CavModel {
    static constexpr int kStride = kCavStride;
    static constexpr bool kPerBatch = false;
    static constexpr int kMinBlocks = 4;
    static constexpr bool kEarlyLoad = false;
    static constexpr bool kZeroNoop = false;  // profile parameters of zero are not a no-op
    using Params = CavParams;
    struct Voxel {
        float p[kCavStride];
    };
    __device__ __forceinline__ static Voxel load(const float* q)
    {
        Voxel v;
        const float4 a = __ldg(reinterpret_cast<const float4*>(q)), b = __ldg(reinterpret_cast<const float4*>(q) + 1);
        v.p[0] = a.x; v.p[1] = a.y; v.p[2] = a.z; v.p[3] = a.w;
        v.p[4] = b.x; v.p[5] = b.y; v.p[6] = b.z; v.p[7] = b.w;
        return v;
    }
    __device__ __forceinline__ static void integrate(const Params& M, const Voxel& v, int b, float wx, float wz,
                                                     float nl2, float* I, float* T)
    {
        const float proj = fmaf(v.p[4], wx, v.p[5] * wz);
        // not unrolled: eight inlined copies of the four-branch Voigt evaluation made
        // the solve instruction-fetch bound (1024 x 512, 64 wavelengths: 9.4 s against
        // 2.3 s with one copy; bit-identical)
#pragma unroll 1
        for (int w = 0; w < W; ++w) {
            const int l = b * W + w;
            float eta, chi;
            cav_eta_chi(M, v.p, l, M.dv[l] + proj, eta, chi);
            const float S = chi > 0.0f ? __fdividef(eta, chi) : 0.0f;
            segment(S, chi, nl2, I[w], T[w]);
        }
    }
};

// flag[blk] = 1 if any parameter that makes emission or opacity is non-zero in the block
__global__ void __launch_bounds__(256) k_cav_block_flags(int nx, int nbx, CavFields F, int* __restrict__ flag)
{
    const int blk = blockIdx.x;
    const int bx = blk % nbx, bz = blk / nbx;
    const long long c = (long long)(bz * DEX_BLOCK + (threadIdx.x >> 4)) * nx + bx * DEX_BLOCK + (threadIdx.x & 15);
    const int any = (F.eta_star[c] != 0.0f) | (F.chi_star[c] != 0.0f) | (F.eta_c[c] != 0.0f) | (F.chi_c[c] != 0.0f);
    const int r = __syncthreads_or(any);
    if (threadIdx.x == 0) flag[blk] = r ? 1 : 0;
}

template <int W>
__global__ void __launch_bounds__(256) k_cav_mips_build(const CavMipParams P, const CavParams M)
{
    __shared__ float sp[level_offset(5)][kCavStride];
    const int a = blockIdx.x;
    if (a >= *P.n_active) return;
    const int b = blockIdx.y;
    const int blk = P.active[a];
    const int bx = blk % P.nbx, bz = blk / P.nbx;
    const int t = threadIdx.x;
    const long long c = (long long)(bz * DEX_BLOCK + (t >> 4)) * P.nx + bx * DEX_BLOCK + (t & 15);
    float* brick = P.bricks + (size_t)a * P.chain * kCavStride;
    const bool writer = (b == 0);  // parameters are the same for every batch

    {
        float v[kCavStride];
        const float vth = P.F.vth[c];
        v[0] = P.F.eta_star[c];
        v[1] = P.F.chi_star[c];
        v[2] = P.F.damping[c];
        v[3] = vth > 0.0f ? 1.0f / vth : 0.0f;
        v[4] = P.F.vx[c];
        v[5] = P.F.vz[c];
        v[6] = P.F.eta_c[c];
        v[7] = P.F.chi_c[c];
        bool bad = false;
#pragma unroll
        for (int q = 0; q < kCavStride; ++q) {
            if (!isfinite(v[q]) || ((q != 4 && q != 5) && v[q] < 0.0f)) bad = true;
            sp[t][q] = v[q];
        }
        if (bad) raise_status(P.status, DEX_ERR_NUMERIC);
        if (writer) {
            float4* o = reinterpret_cast<float4*>(brick + (size_t)t * kCavStride);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
    }
    __syncthreads();

    int level = 0;
    bool ok = true;
    for (int m = 1; m <= P.max_mip; ++m) {
        const int side = DEX_BLOCK >> m, side_p = side << 1;
        const int off = level_offset(m), off_p = level_offset(m - 1);
        const float ds = (float)(1 << m);
        const float ln_ds = (float)m * 0.69314718f;
        bool pass = true;
        if (t < side * side) {
            const int vx_ = t % side, vz_ = t / side;
            const int c0 = off_p + (2 * vz_) * side_p + 2 * vx_;
            const int ch[4] = {c0, c0 + 1, c0 + side_p, c0 + side_p + 1};
            float v[kCavStride];
#pragma unroll
            for (int q = 0; q < kCavStride; ++q)
                v[q] = 0.25f * ((sp[ch[0]][q] + sp[ch[1]][q]) + (sp[ch[2]][q] + sp[ch[3]][q]));
#pragma unroll
            for (int q = 0; q < kCavStride; ++q) sp[off + t][q] = v[q];
            if (writer) {
                float4* o = reinterpret_cast<float4*>(brick + (size_t)(off + t) * kCavStride);
                o[0] = make_float4(v[0], v[1], v[2], v[3]);
                o[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
            for (int w = 0; w < W; ++w) {
                const int l = b * W + w;
                if (l >= P.n_lambda) break;
                float e[4], x[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float* cp = sp[ch[k]];
                    const float speed = sqrtf(cp[4] * cp[4] + cp[5] * cp[5]);
                    cav_eta_chi(M, cp, l, fmaxf(fabsf(M.dv[l]) - speed, 0.0f), e[k], x[k]);
                }
                const GroupStat se = reduce_group(e[0], e[1], e[2], e[3], ln_ds, false);
                const GroupStat sc = reduce_group(x[0], x[1], x[2], x[3], ln_ds, false);
                const float kmax = fmaxf(fmaxf(x[0], x[1]), fmaxf(x[2], x[3]));
                pass = pass && ((se.iod < P.thr_eta && sc.iod < P.thr_chi) || (kmax * ds < P.chi_ds_min));
                // directional tests: the children as a ray propagating along w_k samples them,
                // each at its own (mean) velocity projected on w_k
                for (int d = 0; d < P.n_test_dirs && pass; ++d) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float* cp = sp[ch[k]];
                        cav_eta_chi(M, cp, l, M.dv[l] + fmaf(cp[4], P.test_wx[d], cp[5] * P.test_wz[d]), e[k], x[k]);
                    }
                    const GroupStat de = reduce_group(e[0], e[1], e[2], e[3], ln_ds, false);
                    const GroupStat dc = reduce_group(x[0], x[1], x[2], x[3], ln_ds, false);
                    const float dmax = fmaxf(fmaxf(x[0], x[1]), fmaxf(x[2], x[3]));
                    pass = (de.iod < P.thr_eta && dc.iod < P.thr_chi) || (dmax * ds < P.chi_ds_min);
                }
            }
        }
        const int all = __syncthreads_and(pass ? 1 : 0);
        if (ok && all) level = m;
        else ok = false;
    }
    if (t == 0) {
        if (P.level_cap != nullptr) level = min(level, max((int)P.level_cap[blk], 0));
        const unsigned long long state = (unsigned long long)(level + 1);
        atomicOr(P.words + (size_t)b * P.n_words + blk / DEX_STATES_PER_WORD,
                 state << (DEX_STATE_BITS * (blk % DEX_STATES_PER_WORD)));
    }
}

// kernel parameters are limited to 32764 bytes
static_assert(sizeof(HddaParams) + sizeof(CavMlpParams) <= 32764, "CaV-surrogate kernel parameters too large");

template <typename K, typename MP>
cudaError_t launch_cav_solve_t(K kernel, dim3 grid, size_t smem, cudaStream_t s, const HddaParams& P, const MP& M)
{
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 256, smem, s>>>(P, M);
    return cudaSuccess;
}

}  // namespace

void fill_cav_params(CavParams& M, int n_lambda, int W, const float* dv, float c_kms)
{
    M.coef = voigt_coefficients();
    M.n_lambda = n_lambda;
    const int n_pad = ((n_lambda + W - 1) / W) * W;
    for (int l = 0; l < n_pad; ++l) {
        const float d = l < n_lambda ? dv[l] : 0.0f;
        const double s = 1.0 / (1.0 + (double)d / (double)c_kms);
        M.dv[l] = d;
        M.s[l] = (float)s;
        M.is2[l] = (float)(1.0 / (s * s));
    }
}

cudaError_t launch_cav_grid_build(cudaStream_t s, int nx, int nz, const CavFields& F, int* block_offset, int* active,
                                  int* n_active)
{
    const int nbx = nx / DEX_BLOCK, nbz = nz / DEX_BLOCK;
    k_cav_block_flags<<<(unsigned)(nbx * nbz), 256, 0, s>>>(nx, nbx, F, block_offset);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_block_layout(s, nbx, nbz, block_offset, active, n_active);
}

cudaError_t launch_cav_mips_build(cudaStream_t s, const CavMipParams& P, const CavParams& M)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(P.words, 0, sizeof(unsigned long long) * (size_t)P.n_words * P.n_batch, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    switch (P.W) {
        case 1: k_cav_mips_build<1><<<grid, 256, 0, s>>>(P, M); break;
        case 2: k_cav_mips_build<2><<<grid, 256, 0, s>>>(P, M); break;
        case 4: k_cav_mips_build<4><<<grid, 256, 0, s>>>(P, M); break;
        case 8: k_cav_mips_build<8><<<grid, 256, 0, s>>>(P, M); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_solve_cav_mlp(cudaStream_t s, const HddaParams& P, const CavMlpParams& M)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    const size_t smem = sizeof(unsigned long long) * (size_t)P.n_words;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    cudaError_t e = cudaSuccess;
    switch (P.W) {
#define DEX_LAUNCH(WW)                                                                                           \
    case WW:                                                                                                     \
        if (P.seg_count) e = launch_cav_solve_t(k_solve_hdda_t<WW, true, CavMlpModel<WW>>, grid, smem, s, P, M);   \
        else e = launch_cav_solve_t(k_solve_hdda_t<WW, false, CavMlpModel<WW>>, grid, smem, s, P, M);              \
        break;
        DEX_LAUNCH(1)
        DEX_LAUNCH(2)
        DEX_LAUNCH(4)
        DEX_LAUNCH(8)
#undef DEX_LAUNCH
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_solve_cav(cudaStream_t s, const HddaParams& P, const CavParams& M)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    const size_t smem = sizeof(unsigned long long) * (size_t)P.n_words;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    cudaError_t e = cudaSuccess;
    switch (P.W) {
#define DEX_LAUNCH(WW)                                                                                     \
    case WW:                                                                                               \
        if (P.seg_count) e = launch_cav_solve_t(k_solve_hdda_t<WW, true, CavModel<WW>>, grid, smem, s, P, M); \
        else e = launch_cav_solve_t(k_solve_hdda_t<WW, false, CavModel<WW>>, grid, smem, s, P, M);           \
        break;
        DEX_LAUNCH(1)
        DEX_LAUNCH(2)
        DEX_LAUNCH(4)
        DEX_LAUNCH(8)
#undef DEX_LAUNCH
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace dex
