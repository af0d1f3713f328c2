// Velocity interpolation treatment of a moving medium (Section 3.1).
//
// Every MIP voxel (level m, MIP 0 included) stores, per wavelength batch, a
// header (mean v_x, mean v_z, V = largest speed of its MIP-0 cells, 0) and the
// emissivity and opacity at NV projected velocities v_s = -V + 2 V s / (NV - 1):
//   eta_s = mean over the voxel's MIP-0 cells of the cell's eta at u = dv + v_s,
// likewise chi_s (the line model of k_cav.cu, Voigt by voigt_h).  Along a ray
// (propagation w = -d) the voxel's eta, chi are the linear interpolation of its
// grid at the projected velocity v_mean . w, clamped to [-V, V].  The level of a
// block per batch comes from Eq. IoD on the rest-frame values (projected
// velocity 0), Section 3.1, with the always-average rule; with n_test_dirs = K
// > 0 also from the same test on the children's grids interpolated as a ray
// along each of K in-plane directions samples them.
#include "hdda.cuh"
#include "vlm.cuh"
#include "voigt.cuh"

namespace dex {

namespace {

constexpr int kNV = DEX_VEL_SAMPLES;

template <int W>
struct VelModel {
    static constexpr int kRec = 2 * W;                 // eta[W], chi[W] of one grid velocity
    static constexpr int kStride = 4 + kNV * kRec;
    static constexpr bool kPerBatch = true;
    static constexpr int kMinBlocks = 4;
    static constexpr bool kEarlyLoad = false;
    static constexpr bool kZeroNoop = false;  // profile parameters of zero are not a no-op
    struct Params {
        int unused;
    };
    struct Voxel {
        float vx, vz, V;
        const float* p;
    };
    __device__ __forceinline__ static Voxel load(const float* q)
    {
        const float4 h = __ldg(reinterpret_cast<const float4*>(q));
        return Voxel{h.x, h.y, h.z, q + 4};
    }
    __device__ __forceinline__ static void integrate(const Params&, const Voxel& v, int, float wx, float wz,
                                                     float nl2, float* I, float* T)
    {
        const float proj = fminf(fmaxf(fmaf(v.vx, wx, v.vz * wz), -v.V), v.V);
        const float f = v.V > 0.0f ? __fdividef(proj + v.V, 2.0f * v.V) * (float)(kNV - 1) : 0.0f;
        const int i0 = min((int)f, kNV - 2);
        const float t = f - (float)i0;
        const Record<W> r0 = load_record<W>(v.p + i0 * kRec);
        const Record<W> r1 = load_record<W>(v.p + (i0 + 1) * kRec);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            // records hold (eta, chi) here: Record's S slot carries eta
            const float eta = fmaf(t, r1.S[w] - r0.S[w], r0.S[w]);
            const float chi = fmaf(t, r1.chi[w] - r0.chi[w], r0.chi[w]);
            const float S = chi > 0.0f ? __fdividef(eta, chi) : 0.0f;
            segment(S, chi, nl2, I[w], T[w]);
        }
    }
};

// eta, chi of MIP-0 cell parameters p (8 floats as in k_cav.cu) at shift u for wavelength l
__device__ __forceinline__ void cell_eta_chi(const CavParams& M, const float* p, int l, float u, float& eta,
                                             float& chi)
{
    const float inv = p[3];
    const float H = voigt_h(M.coef, p[2] * M.is2[l], u * inv);
    const float phi = H * inv * kInvSqrtPi;
    const float sl = M.s[l];
    eta = fmaf(p[0] * sl, phi, p[6]);
    chi = fmaf(p[1] * sl, phi, p[7]);
}

template <int W>
__global__ void __launch_bounds__(256) k_vel_mips_build(const CavMipParams P, const CavParams M)
{
    constexpr int REC = VelModel<W>::kStride;
    __shared__ float sp[256][8];                          // MIP-0 cell parameters
    __shared__ float s_e[level_offset(5)][W];             // rest-frame eta chain
    __shared__ float s_c[level_offset(5)][W];             // rest-frame chi chain
    __shared__ float s_v[level_offset(5)][3];             // mean vx, mean vz, max speed
    const int a = blockIdx.x;
    if (a >= *P.n_active) return;
    const int b = blockIdx.y;
    const int blk = P.active[a];
    const int bx = blk % P.nbx, bz = blk / P.nbx;
    const int t = threadIdx.x;
    const long long c = (long long)(bz * DEX_BLOCK + (t >> 4)) * P.nx + bx * DEX_BLOCK + (t & 15);
    float* brick = P.bricks + ((size_t)b * P.cap_active + a) * P.chain * REC;

    {
        const float vth = P.F.vth[c];
        float v[8] = {P.F.eta_star[c], P.F.chi_star[c], P.F.damping[c], vth > 0.0f ? 1.0f / vth : 0.0f,
                      P.F.vx[c],       P.F.vz[c],       P.F.eta_c[c],   P.F.chi_c[c]};
        bool bad = false;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (!isfinite(v[q]) || ((q != 4 && q != 5) && v[q] < 0.0f)) bad = true;
            sp[t][q] = v[q];
        }
        if (bad) raise_status(P.status, DEX_ERR_NUMERIC);
        s_v[t][0] = v[4];
        s_v[t][1] = v[5];
        s_v[t][2] = sqrtf(v[4] * v[4] + v[5] * v[5]);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int l = min(b * W + w, P.n_lambda - 1);
            float e, x;
            cell_eta_chi(M, v, l, M.dv[l], e, x);  // rest frame: projected velocity 0
            s_e[t][w] = e;
            s_c[t][w] = x;
        }
    }
    __syncthreads();

    // rest-frame chain + velocity statistics + level decision (as the static build, box filter)
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
            s_v[off + t][0] = 0.25f * ((s_v[ch[0]][0] + s_v[ch[1]][0]) + (s_v[ch[2]][0] + s_v[ch[3]][0]));
            s_v[off + t][1] = 0.25f * ((s_v[ch[0]][1] + s_v[ch[1]][1]) + (s_v[ch[2]][1] + s_v[ch[3]][1]));
            s_v[off + t][2] = fmaxf(fmaxf(s_v[ch[0]][2], s_v[ch[1]][2]), fmaxf(s_v[ch[2]][2], s_v[ch[3]][2]));
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const GroupStat se = reduce_group(s_e[ch[0]][w], s_e[ch[1]][w], s_e[ch[2]][w], s_e[ch[3]][w], ln_ds,
                                                  false);
                const float k0 = s_c[ch[0]][w], k1 = s_c[ch[1]][w], k2 = s_c[ch[2]][w], k3 = s_c[ch[3]][w];
                const GroupStat sc = reduce_group(k0, k1, k2, k3, ln_ds, false);
                const float kmax = fmaxf(fmaxf(k0, k1), fmaxf(k2, k3));
                if (b * W + w < P.n_lambda)
                    pass = pass && ((se.iod < P.thr_eta && sc.iod < P.thr_chi) || (kmax * ds < P.chi_ds_min));
                s_e[off + t][w] = se.val;
                s_c[off + t][w] = sc.val;
            }
        }
        const int all = __syncthreads_and(pass ? 1 : 0);
        if (ok && all) level = m;
        else ok = false;
    }

    // velocity grids of every level: work items (voxel, grid velocity, wavelength)
    for (int m = 0; m <= P.max_mip; ++m) {
        const int side = DEX_BLOCK >> m, f = 1 << m, nvox = side * side;
        const int off = level_offset(m);
        for (int q = t; q < nvox * kNV * W; q += blockDim.x) {
            const int w = q % W, s = (q / W) % kNV, vox = q / (W * kNV);
            const int l = min(b * W + w, P.n_lambda - 1);
            const float V = s_v[off + vox][2];
            const float vs = fmaf(2.0f * V, (float)s / (float)(kNV - 1), -V);
            const int vx0 = (vox % side) * f, vz0 = (vox / side) * f;
            float se = 0.0f, sc = 0.0f;
            for (int cz = 0; cz < f; ++cz)
                for (int cx = 0; cx < f; ++cx) {
                    float e, x;
                    cell_eta_chi(M, sp[(vz0 + cz) * DEX_BLOCK + vx0 + cx], l, M.dv[l] + vs, e, x);
                    se += e;
                    sc += x;
                }
            const float inv_n = 1.0f / (float)(f * f);
            float* rec = brick + (size_t)(off + vox) * REC;
            rec[4 + s * 2 * W + w] = se * inv_n;
            rec[4 + s * 2 * W + W + w] = sc * inv_n;
            if (s == 0 && w == 0)
                *reinterpret_cast<float4*>(rec) = make_float4(s_v[off + vox][0], s_v[off + vox][1], V, 0.0f);
        }
    }

    // directional tests (n_test_dirs = K > 0): a level that passed the rest-frame test
    // must also pass it on its children as a ray along each w_k samples them -- each
    // child's velocity grid interpolated at its mean velocity projected on w_k, as
    // the traversal does -- since rest-frame values of children moving in different
    // directions can agree while the profiles a ray sees are shifted apart
    if (P.n_test_dirs > 0 && level > 0) {
        __syncthreads();  // the grids above are written by the whole CTA
        int dlevel = 0;
        for (int m = 1; m <= level; ++m) {
            const int side = DEX_BLOCK >> m, side_p = side << 1;
            const int off_p = level_offset(m - 1);
            const float ds = (float)(1 << m);
            const float ln_ds = (float)m * 0.69314718f;
            bool pass = true;
            if (t < side * side) {
                const int vx_ = t % side, vz_ = t / side;
                const int c0 = off_p + (2 * vz_) * side_p + 2 * vx_;
                const int ch[4] = {c0, c0 + 1, c0 + side_p, c0 + side_p + 1};
                for (int d = 0; d < P.n_test_dirs && pass; ++d) {
                    float e[4][W], x[4][W];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float* rec = brick + (size_t)ch[k] * REC;
                        const float4 h = *reinterpret_cast<const float4*>(rec);
                        const float proj = fminf(fmaxf(fmaf(h.x, P.test_wx[d], h.y * P.test_wz[d]), -h.z), h.z);
                        const float f = h.z > 0.0f ? (proj + h.z) / (2.0f * h.z) * (float)(kNV - 1) : 0.0f;
                        const int i0 = min((int)f, kNV - 2);
                        const float u = f - (float)i0;
                        const float* r0 = rec + 4 + i0 * 2 * W;
                        const float* r1 = r0 + 2 * W;
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            e[k][w] = fmaf(u, r1[w] - r0[w], r0[w]);
                            x[k][w] = fmaf(u, r1[W + w] - r0[W + w], r0[W + w]);
                        }
                    }
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        if (b * W + w >= P.n_lambda) continue;
                        const GroupStat se = reduce_group(e[0][w], e[1][w], e[2][w], e[3][w], ln_ds, false);
                        const GroupStat sc = reduce_group(x[0][w], x[1][w], x[2][w], x[3][w], ln_ds, false);
                        const float kmax = fmaxf(fmaxf(x[0][w], x[1][w]), fmaxf(x[2][w], x[3][w]));
                        pass = pass && ((se.iod < P.thr_eta && sc.iod < P.thr_chi) || (kmax * ds < P.chi_ds_min));
                    }
                }
            }
            if (!__syncthreads_and(pass ? 1 : 0)) break;
            dlevel = m;
        }
        level = dlevel;
    }
    if (t == 0) {
        if (P.level_cap != nullptr) level = min(level, max((int)P.level_cap[blk], 0));
        const unsigned long long state = (unsigned long long)(level + 1);
        atomicOr(P.words + (size_t)b * P.n_words + blk / DEX_STATES_PER_WORD,
                 state << (DEX_STATE_BITS * (blk % DEX_STATES_PER_WORD)));
    }
}

template <typename K, typename MP>
cudaError_t launch_kernel(K kernel, dim3 grid, size_t smem, cudaStream_t s, const HddaParams& P, const MP& M)
{
    if (smem > 32 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 256, smem, s>>>(P, M);
    return cudaSuccess;
}

}  // namespace

int vel_record_floats(int W) { return 4 + kNV * 2 * W; }

cudaError_t launch_vel_mips_build(cudaStream_t s, const CavMipParams& P, const CavParams& M)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(P.words, 0, sizeof(unsigned long long) * (size_t)P.n_words * P.n_batch, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    switch (P.W) {
        case 1: k_vel_mips_build<1><<<grid, 256, 0, s>>>(P, M); break;
        case 2: k_vel_mips_build<2><<<grid, 256, 0, s>>>(P, M); break;
        case 4: k_vel_mips_build<4><<<grid, 256, 0, s>>>(P, M); break;
        case 8: k_vel_mips_build<8><<<grid, 256, 0, s>>>(P, M); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_solve_velinterp(cudaStream_t s, const HddaParams& P)
{
    if (P.cap_active == 0 || P.n_batch == 0) return cudaSuccess;
    const size_t smem = sizeof(unsigned long long) * (size_t)P.n_words;
    dim3 grid((unsigned)P.cap_active, (unsigned)P.n_batch);
    cudaError_t e = cudaSuccess;
    switch (P.W) {
#define DEX_LAUNCH(WW)                                                                                  \
    case WW:                                                                                            \
        if (P.seg_count)                                                                                \
            e = launch_kernel(k_solve_hdda_t<WW, true, VelModel<WW>>, grid, smem, s, P,                 \
                              typename VelModel<WW>::Params{});                                         \
        else                                                                                            \
            e = launch_kernel(k_solve_hdda_t<WW, false, VelModel<WW>>, grid, smem, s, P,                \
                              typename VelModel<WW>::Params{});                                         \
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
