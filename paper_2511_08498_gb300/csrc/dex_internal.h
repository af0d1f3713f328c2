// Internal launch interfaces between the C-ABI layer (dex_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dex_common.cuh"
#include "voigt.cuh"

namespace dex {

struct DenseParams {
    int nx, nz, n_lambda, W, n_batch;
    int exclude_own;        // leave out each probe's own-cell emission (the first segment)
    long long n_cells;
    const float* planes;
    int n_probe;
    const int* probes;      // nullptr: every cell, tiled launch
    float i_bc;
    float* J;
    float* I;
    unsigned long long* seg_count;
    unsigned int* status;
    Quadrature quad;
};

struct MipParams {
    int nx, nz, nbx, nbz, n_lambda, W, n_batch, max_mip, chain, n_words, cap_active, storage;
    bool log_mean;
    float thr_eta, thr_chi, chi_ds_min;
    const float* eta;
    const float* chi;
    const int* active;
    const int* n_active;
    const signed char* level_cap;
    float* bricks;
    unsigned long long* words;
    unsigned int* status;
};

// Grids of at most this many blocks stage the one-word-per-block table (32 KB).
constexpr int kInfoMaxBlocks = 8192;
// The paired walk always stages it, for grids of up to 2048 x 2048 (64 KB of
// dynamic shared memory: with its 16 KB J tile, two 256-thread CTAs per SM
// hold 160 KB).
constexpr int kPairInfoMaxBlocks = 16384;

// Distance thresholds of levels 1..4 padded to four, as the traversal compares
// them (the number of thresholds band[m-1] <= t is the highest level allowed):
// +inf for the levels beyond the n_band given (never reached), 0 for all four
// when there is no limit (n_band < 0: every level allowed from t = 0).
inline void pad_bands(int n_band, float* band)
{
    for (int q = 0; q < 4; ++q)
        band[q] = n_band < 0 ? 0.0f : (q < n_band ? band[q] : __builtin_huge_valf());
}

// Pairs of wavelength batches walked together (DEX_TRAVERSAL_PAIRED): the
// batches are paired mirror-wise within consecutive groups of `group` batches
// (group <= 0 or >= n_batch: one group of all), b with g0 + size - 1 - (b - g0);
// a group of odd size leaves its middle batch alone.
__host__ __device__ inline int pair_group_size(int n_batch, int group)
{
    return group <= 0 || group > n_batch ? n_batch : group;
}
__host__ __device__ inline int pair_count(int n_batch, int group)
{
    const int g = pair_group_size(n_batch, group);
    int n = 0;
    for (int g0 = 0; g0 < n_batch; g0 += g) n += (n_batch - g0 < g ? n_batch - g0 : g) / 2;
    return n;
}
__host__ __device__ inline void pair_batches(int p, int n_batch, int group, int& b1, int& b2)
{
    const int g = pair_group_size(n_batch, group);
    for (int g0 = 0; g0 < n_batch; g0 += g) {
        const int size = n_batch - g0 < g ? n_batch - g0 : g, np = size / 2;
        if (p < np) {
            b1 = g0 + p;
            b2 = g0 + size - 1 - p;
            return;
        }
        p -= np;
    }
    b1 = b2 = -1;
}

// Lone batches of the pairing: the middle batch of every group of odd size.
__host__ __device__ inline int pair_lone_count(int n_batch, int group)
{
    const int g = pair_group_size(n_batch, group);
    int n = 0;
    for (int g0 = 0; g0 < n_batch; g0 += g) n += (n_batch - g0 < g ? n_batch - g0 : g) & 1;
    return n;
}
__host__ __device__ inline int pair_lone_batch(int q, int n_batch, int group)
{
    const int g = pair_group_size(n_batch, group);
    for (int g0 = 0; g0 < n_batch; g0 += g) {
        const int size = n_batch - g0 < g ? n_batch - g0 : g;
        if (size & 1) {
            if (q == 0) return g0 + size / 2;
            --q;
        }
    }
    return -1;
}

struct HddaParams {
    int nx, nz, nbx, nbz, n_lambda, W, n_batch, chain, n_words, cap_active, storage;
    int pair_group;  // DEX_TRAVERSAL_PAIRED: batches paired within groups of this many (0: one group)
    int n_band;      // < 0: no distance limit; else level m needs block entry t >= band[m-1]
                     // (band padded to four by pad_bands)
    int traversal;   // DEX_TRAVERSAL_PER_BATCH, _SHARED or _PAIRED (static model, W = 8)
    int exclude_own; // leave out each probe's own-voxel emission (static model, W = 8, float32)
    float band[4];
    long long n_cells;
    const float* bricks;
    const unsigned long long* words;
    const int* block_offset;
    const int* active;
    const int* n_active;
    float i_bc;
    float* J;
    float* I;
    unsigned long long* seg_count;
    unsigned int* status;
    Quadrature quad;
};

struct AtomParams {
    dex_atom atom;
    int n_lambda;
    double nu[DEX_MAX_ATOM_LAMBDA];    // sample frequencies (Hz)
    double wq[DEX_MAX_ATOM_LAMBDA];    // trapezoid weight in frequency within the sample's line
    signed char tag[DEX_MAX_ATOM_LAMBDA];
    double nu0[DEX_MAX_LINES];
    double b_ul[DEX_MAX_LINES];
    double b_lu[DEX_MAX_LINES];
};

cudaError_t launch_lte_pops(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T,
                            const float* nh, double* pops);
cudaError_t launch_atom_eta_chi(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T,
                                const float* ne, const double* pops, float* eta, float* chi);
cudaError_t launch_rates(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T, const float* J,
                         double* jbar);
cudaError_t launch_se_solve(cudaStream_t s, const AtomParams& P, long long n_cells, const float* T, const float* ne,
                            const float* nh, const double* jbar, const double* rho, double* pops);

// Directions grouped by the path from a cell centre to its boundary,
// l = 1 / (2 max(|d_x|, |d_z|)) cells, with the summed quadrature weight of each group
struct OwnCellOperator {
    int n;
    float ell[DEX_MAX_DIRS];
    float w[DEX_MAX_DIRS];
};
cudaError_t launch_mali_rates(cudaStream_t s, const AtomParams& P, const OwnCellOperator& O, long long n_cells,
                              const float* T, const float* ne, const double* pops, const float* J, double* rho,
                              double* jeff);
cudaError_t launch_max_rel_change(cudaStream_t s, int n_level, long long n_cells, const float* T, const double* old_p,
                                  const double* new_p, double* out);

// Core-and-Voigt: per-cell parameter fields (device pointers) and per-wavelength constants
struct CavFields {
    const float* eta_star;
    const float* chi_star;
    const float* damping;
    const float* vth;
    const float* vx;
    const float* vz;
    const float* eta_c;
    const float* chi_c;
};

struct CavParams {
    VoigtCoef coef;
    int n_lambda;
    float dv[DEX_MAX_CAV_LAMBDA];   // wavelength offsets (km/s), padded to whole batches
    float s[DEX_MAX_CAV_LAMBDA];    // lambda0 / lambda
    float is2[DEX_MAX_CAV_LAMBDA];  // (lambda / lambda0)^2
};

// Core-and-Voigt with the learned profile: the CaV tables plus the network's
// parameters (W1, W2, w3 rounded to bfloat16 values), passed by value
struct CavMlpParams {
    CavParams cav;
    float w[4481];
};

constexpr int kMaxTestDirs = 16;

struct CavMipParams {
    int nx, nz, nbx, nbz, n_lambda, W, n_batch, max_mip, chain, n_words, cap_active;
    float thr_eta, thr_chi, chi_ds_min;
    int n_test_dirs;                   // directional level tests (0: the paper's test alone)
    float test_wx[kMaxTestDirs];       // their propagation directions
    float test_wz[kMaxTestDirs];
    CavFields F;
    const int* active;
    const int* n_active;
    const signed char* level_cap;
    float* bricks;
    unsigned long long* words;
    unsigned int* status;
};

void fill_cav_params(CavParams& M, int n_lambda, int W, const float* dv, float c_kms);
cudaError_t launch_block_layout(cudaStream_t s, int nbx, int nbz, int* block_offset, int* active, int* n_active);
cudaError_t launch_cav_grid_build(cudaStream_t s, int nx, int nz, const CavFields& F, int* block_offset, int* active,
                                  int* n_active);
cudaError_t launch_cav_mips_build(cudaStream_t s, const CavMipParams& P, const CavParams& M);
cudaError_t launch_solve_cav(cudaStream_t s, const HddaParams& P, const CavParams& M);
cudaError_t launch_solve_cav_mlp(cudaStream_t s, const HddaParams& P, const CavMlpParams& M);

int vel_record_floats(int W);
cudaError_t launch_vel_mips_build(cudaStream_t s, const CavMipParams& P, const CavParams& M);
cudaError_t launch_solve_velinterp(cudaStream_t s, const HddaParams& P);

struct AtmDesc {
    int nx, nz, nbx, nbz, n_lambda, chain, n_words, cap_active, n_dir, n_band;
    float band[4];
    float i_bc;
    long long item_base;
    const float* bricks;
    const unsigned long long* words;
    const int* block_offset;
    const int* active;
    const int* n_active;
    const float* dirs;
    const float* weights;
    float* J;
};

struct BatchParams {
    int n_atm;
    long long n_items;
    int paired;             // W = 8: work units are pairs of batches (pair_batches) and lone batches
    int pair_group;         //   paired within groups of this many batches (0: one group)
    int parts;              // work items per active block and batch: 256 / probes per item
    int chunk;              // work items claimed per queue increment
    unsigned int* queue;
    unsigned long long* done_ns;
    unsigned long long* start_ns;
    unsigned int* status;
    AtmDesc atm[DEX_MAX_BATCH_ATM];
};

// packet: probes per work item (256, 128 or 64); info: stage one word per block
// (offset * 8 + state) instead of the packed state words; occupancy (W = 8): a
// 64-register budget (four 256-thread CTAs per SM) instead of the compiler's;
// smem_bytes: the largest table of the batch
cudaError_t launch_batch_solve(cudaStream_t s, const BatchParams& P, int ctas, int W, int packet, bool info,
                               bool occupancy, size_t smem_bytes);
// work units of one atmosphere: its batches, or with P.paired its pairs and lone batches
inline int batch_units(const BatchParams& P, int n_batch)
{
    return P.paired ? pair_count(n_batch, P.pair_group) + pair_lone_count(n_batch, P.pair_group) : n_batch;
}
cudaError_t noalloc_scratch(unsigned int** out);

int chain_length(int max_mip);
int record_floats(int W, int storage);
// special-function-unit 2^x throughput (k_probe.cu); synchronises the stream
cudaError_t measure_ex2_rate(cudaStream_t s, double* ops_per_s);
cudaError_t measure_fp32_rate(cudaStream_t s, double* ops_per_s);
// a bounded mbarrier wait that runs out (self-test of the timeout path)
cudaError_t launch_wait_timeout(cudaStream_t s, int polls, unsigned int* status);

// learned profile surrogate (k_mlp.cu)
struct MlpParams {
    long long n;                 // samples
    const float* xau;            // [n][3]: x, a, u
    const float* target;         // [n] ln H (training)
    const float* params;         // mlp_param_count() FP32 master parameters
    float* out;                  // [n] predicted ln H (inference)
    float* grad;                 // mlp_param_count() gradient of the mean loss (training)
    float* loss;                 // mean squared error (training)
    unsigned int* status;
};
int mlp_param_count();
cudaError_t launch_mlp_forward(cudaStream_t s, const MlpParams& P);
cudaError_t launch_mlp_grad(cudaStream_t s, const MlpParams& P);
cudaError_t launch_mlp_adam(cudaStream_t s, float* p, const float* g, float* m, float* v, int step, float lr,
                            float b1, float b2, float eps);
cudaError_t launch_mlp_targets(cudaStream_t s, long long n, const float* xau, float* out);

cudaError_t launch_voigt(cudaStream_t s, long long n, const float* a, const float* x, float* h);
cudaError_t launch_synth_static_line(cudaStream_t s, long long n_cells, int n_lambda, const float* chi_c,
                                     const float* s_c, const float* s_l, const float* ratio, const float* dld,
                                     const float* dlam, float* eta, float* chi);
cudaError_t launch_grid_build(cudaStream_t s, int nx, int nz, int n_lambda, const float* eta, const float* chi,
                              int* block_offset, int* active, int* n_active);
cudaError_t launch_mips_build(cudaStream_t s, const MipParams& p);
cudaError_t launch_solve_hdda(cudaStream_t s, const HddaParams& p);
// one traversal per ray for up to four wavelength batches (k_hdda_mb.cu)
bool solve_hdda_shared_applies(const HddaParams& p);
cudaError_t launch_solve_hdda_shared(cudaStream_t s, const HddaParams& p);
bool solve_hdda_paired_applies(const HddaParams& p);
cudaError_t launch_solve_hdda_paired(cudaStream_t s, const HddaParams& p);

// --------------------------------------------------- radiance cascades --
struct RcParams {
    int nx, nz, nbx, nbz, n_lambda, W, n_batch, chain, n_words, cap_active, storage;
    int spacing, pnx, pnz, n_dir, level_cap;  // this cascade: probe lattice, directions, MIP cap
    int dir_fastest;                           // thread order: directions (1) or probes (0) fastest
    int paired, pair_group;                    // W = 8: one walk per pair of batches (pair_batches)
    float t_s, t_e, i_bc;                      // radiance interval, boundary intensity
    const float* bricks;
    const unsigned long long* words;
    const int* block_offset;
    const float* dirs;                         // [n_dir][2] of this cascade
    const float* upper;                        // merged radiance of the cascade above, or nullptr
    float* out;                                // [n_batch][n_dir][pnz * pnx][W] merged radiance
    unsigned long long* seg_count;
    unsigned int* status;
};
cudaError_t launch_rc_cascade(cudaStream_t s, const RcParams& P);
cudaError_t launch_rc_mean(cudaStream_t s, const RcParams& P, const float* L0, float* J);

// ------------------------------------------------------------------- 3D --
// Grids [nz][ny][nx] (x fastest) cut into DEX_BLOCK3^3 blocks; block index
// (bz * nby + by) * nbx + bx; level m of a block's chain holds (8 >> m)^3
// voxels, row-major [z][y][x].
struct Quadrature3 {
    int n_dir;
    float dx[DEX_MAX_DIRS];
    float dy[DEX_MAX_DIRS];
    float dz[DEX_MAX_DIRS];
    float w[DEX_MAX_DIRS];
};

struct Dense3Params {
    int nx, ny, nz, n_lambda, W, n_batch;
    long long n_cells;
    const float* planes;
    int n_probe;
    const int* probes;      // nullptr: every cell
    float i_bc;
    float* J;
    float* I;
    unsigned long long* seg_count;
    unsigned int* status;
    Quadrature3 quad;
};

struct Mip3Params {
    int nx, ny, nz, nbx, nby, nbz, n_lambda, W, n_batch, max_mip, chain, n_words, cap_active, storage;
    bool log_mean;
    float thr_eta, thr_chi, chi_ds_min;
    const float* eta;
    const float* chi;
    const int* active;
    const int* n_active;
    const signed char* level_cap;
    float* bricks;
    unsigned long long* words;
    unsigned int* status;
};

struct Hdda3Params {
    int nx, ny, nz, nbx, nby, nbz, n_lambda, W, n_batch, max_mip, chain, n_words, cap_active, storage;
    int traversal;  // DEX_TRAVERSAL_PAIRED: one walk per pair of batches; otherwise one per batch
    int pair_group; // batches paired within groups of this many (0: one group), as HddaParams
    int n_band;
    float band[4];
    long long n_cells;
    const float* bricks;
    const unsigned long long* words;
    const int* block_offset;
    const int* active;
    const int* n_active;
    float i_bc;
    float* J;
    float* I;
    unsigned long long* seg_count;
    unsigned int* status;
    Quadrature3 quad;
};

int chain_length3(int max_mip);
cudaError_t launch_solve_dense3(cudaStream_t s, const Dense3Params& P);
cudaError_t launch_grid3_build(cudaStream_t s, int nx, int ny, int nz, int n_lambda, const float* eta, const float* chi,
                               int* block_offset, int* active, int* n_active);
cudaError_t launch_mips3_build(cudaStream_t s, const Mip3Params& P);
cudaError_t launch_solve_hdda3(cudaStream_t s, const Hdda3Params& P);
bool solve_hdda3_paired_applies(const Hdda3Params& P);

cudaError_t launch_pack_planes(cudaStream_t s, long long n_cells, int n_lambda, int W,
                               const float* eta, const float* chi, float* planes, unsigned int* status);
cudaError_t launch_solve_dense(cudaStream_t s, const DenseParams& p);

}  // namespace dex
