/*
 * dexgb -- GB300 (sm_103a) formal solution of the radiative transfer equation
 * on sparse, variance-limited mipmapped 2D grids (arxiv 2511.08498).
 *
 * C ABI.  Every entry point takes plain pointers and sizes; no C++ or PyTorch
 * types cross this boundary.
 *
 * Conventions
 *  - Geometry: a 2D grid of nx * nz unit square voxels ("cells"), x horizontal,
 *    z vertical; cell (i, j) has index c = j * nx + i and centre (i + 0.5, j + 0.5).
 *    Per-cell arrays are row-major [nz][nx]; wavelength-dependent ones are
 *    wavelength-major [n_lambda][nz][nx] unless stated otherwise.
 *  - Emissivity eta and opacity chi are per unit length (cell side = 1).
 *  - Ownership: the caller allocates and owns every buffer passed in; pointers
 *    marked "device" must be device memory of the context's GPU, "host" must be
 *    host memory.  The library keeps no pointer after a call returns, except the
 *    context's own status word.
 *  - Asynchrony: compute calls enqueue kernels on the context's stream and
 *    return before they finish.  Argument errors are returned immediately as a
 *    status code (nothing is enqueued).  Errors found on the device (a ray
 *    exceeding its step cap, a negative or NaN opacity) are recorded in the
 *    context's device status word and reported by dex_ctx_check().
 *  - No call falls back to the CPU: without a usable GPU, dex_ctx_create fails.
 */
#ifndef DEXGB_H
#define DEXGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
enum {
    DEX_OK = 0,
    DEX_ERR_ARG = 1,            /* invalid argument (nothing was enqueued)           */
    DEX_ERR_CUDA = 2,           /* a CUDA runtime call failed                         */
    DEX_ERR_TRAVERSAL_CAP = 4,  /* device: a ray exceeded its traversal step cap      */
    DEX_ERR_NUMERIC = 8,        /* device: negative or non-finite opacity/emissivity  */
    DEX_ERR_UNSUPPORTED = 16,   /* configuration outside the compiled variants        */
    DEX_ERR_TIMEOUT = 32        /* device: a bounded wait on the tensor cores expired  */
};

#define DEX_VERSION 100
#define DEX_MAX_DIRS 256        /* quadrature directions per solve                    */
#define DEX_BLOCK 16            /* block side of the sparse grid (Section 2.3)        */
#define DEX_BLOCK3 8            /* block side of the sparse 3D grid (Section 2.3)     */
#define DEX_STATE_BITS 3        /* bits per packed block state (Section 2.3.1)        */
#define DEX_STATES_PER_WORD 21  /* floor(64 / 3) block states per 64-bit word         */

typedef struct dex_ctx dex_ctx;

/* Library version (DEX_VERSION). */
int dex_version(void);

/* Human-readable name of a status code (static string). */
const char* dex_status_string(int status);

/*
 * Create a context bound to CUDA device `device` and stream `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  Allocates one 4-byte device
 * status word.  Returns DEX_ERR_CUDA when no usable device exists.
 */
int dex_ctx_create(int device, void* stream, dex_ctx** out);

/* Destroy a context (waits for its stream, frees the status word). NULL is a no-op. */
int dex_ctx_destroy(dex_ctx* ctx);

/* Rebind the context to another stream of the same device. */
int dex_ctx_set_stream(dex_ctx* ctx, void* stream);

/*
 * Traversal of the static accelerated solve (dex_formal_solve_hdda) for W = 8:
 *   DEX_TRAVERSAL_PER_BATCH (default): one walk per ray and wavelength batch.
 *   DEX_TRAVERSAL_SHARED: one walk per ray for two wavelength batches, b and
 *     n_batch - 1 - b.  In every block the walk steps through the voxels of the
 *     finer of the two batches' levels there, and each batch integrates its own
 *     voxel (at its own level, Section 4.1) when the walk leaves it, over the
 *     length between the same two planes its own walk would use: J, I and the
 *     executed segment count equal those of the per-batch walk.  Needs at least
 *     two batches and grids of at most 24576 blocks (the CTA stages one 32-bit
 *     word per block); otherwise the per-batch walk runs.  On a GB300 it is the
 *     slower of the two on the static-line workload (its larger per-thread
 *     state halves the resident warps).
 *   DEX_TRAVERSAL_PAIRED: one walk per ray for each pair of batches: b and
 *     n_batch - 1 - b by default, else as dex_ctx_set_pair_group sets (a line's
 *     batches lie symmetrically about its centre, so a pair sees the same part
 *     of the profile and tends to take the same levels); one thread carries
 *     the pair's 16 wavelengths.  The walk uses, in
 *     every block, the smaller of the two batches' levels (Section 2.2), capped
 *     by the distance limits as usual (Section 4.1): no batch is integrated more
 *     coarsely than at its own levels, and where the two agree the result is
 *     that of the per-batch walk.  J and I equal, bit for bit, those of the
 *     per-batch walk given state words that hold the pair's minimum for both
 *     batches.  The middle batch of a group of odd size is solved by the
 *     per-batch walk.  Needs W = 8 and grids of at most 16384 blocks (the
 *     own-cell emission may be left out, dex_ctx_set_own_cell, as for the
 *     per-batch walk); otherwise dex_formal_solve_hdda returns
 *     DEX_ERR_UNSUPPORTED.  The executed segment
 *     count counts each segment of the walk once per batch of the pair.  The
 *     3D solve (dex_formal_solve_hdda3) honours this mode too.
 * Any other mode -> DEX_ERR_ARG.  The setting belongs to the context.
 */
/*
 * Own-cell emission in the formal solutions (context setting, default 1 =
 * included).  With include = 0, dex_formal_solve_dense and dex_formal_solve_hdda
 * leave out the emission of each probe's own cell (the first segment of every
 * ray; for the accelerated solve the probe's own voxel, which is its MIP-0 cell
 * wherever the distance limits keep the probe's block at level 0): I and J then
 * hold the radiation arriving from beyond the cell, attenuated by it (Jext, the
 * input of dex_mali_rates).  The accelerated solve supports it for W = 8 and
 * float32 bricks; every other solver returns DEX_ERR_UNSUPPORTED while it is
 * off.  include not 0 or 1 -> DEX_ERR_ARG.
 */
int dex_ctx_set_own_cell(dex_ctx* ctx, int include);

#define DEX_TRAVERSAL_PER_BATCH 0
#define DEX_TRAVERSAL_SHARED 1
#define DEX_TRAVERSAL_PAIRED 2
int dex_ctx_set_traversal(dex_ctx* ctx, int mode);

/*
 * Which batches the paired walk (DEX_TRAVERSAL_PAIRED) pairs (context setting,
 * default 0).  The batches are taken in consecutive groups of `group` batches
 * (group = 0, or group >= n_batch: one group of all batches) and paired
 * mirror-wise inside each group: batch g0 + q with g0 + size - 1 - q, where g0
 * is the group's first batch and size its number of batches (the last group
 * may be short); the middle batch of a group of odd size is solved alone.  A
 * wavelength grid that holds several lines one after the other, each line's
 * samples filling whole batches, pairs each line's batches with each other
 * when group is the batches per line.  group < 0 -> DEX_ERR_ARG.
 */
int dex_ctx_set_pair_group(dex_ctx* ctx, int group);

/*
 * Synchronise the context's stream, read and clear the device status word.
 * Returns DEX_OK or the OR of the device error bits (DEX_ERR_TRAVERSAL_CAP,
 * DEX_ERR_NUMERIC), or DEX_ERR_CUDA if the stream reported a CUDA error.
 */
int dex_ctx_check(dex_ctx* ctx);

/* Message of the last error returned by a call on this context (static until the next call). */
const char* dex_last_error(const dex_ctx* ctx);

/* ------------------------------------------------- wavelength-batch planes --
 *
 * The solvers read per-voxel data as interleaved wavelength-batch records: for
 * a batch width W (1, 2, 4 or 8) and n_batch = ceil(n_lambda / W) batches,
 *     planes[b][c][0 .. W-1]   = S (source function) of wavelengths b*W + w
 *     planes[b][c][W .. 2W-1]  = chi of the same wavelengths
 * with S = eta / chi where chi > 0.  A transparent emitter (chi = 0, eta > 0)
 * is stored as chi = eta * 2^-60, S = 2^60, which adds eta * length to the
 * intensity to float32 precision for eta <= 2^36 (larger values are rejected
 * with DEX_ERR_NUMERIC).  eta = chi = 0 is stored as S = chi = 0.  Wavelengths
 * beyond n_lambda are zero.  One record is 8*W bytes (W = 8: one 64-byte unit).
 *
 * Alignment: for W = 8 the float32 records (planes and bricks) and the bfloat16
 * bricks are read with 256-bit loads, so those arrays must be 32-byte aligned;
 * otherwise 16-byte (W = 1: 8-byte) alignment suffices.  A misaligned array is
 * rejected with DEX_ERR_ARG before anything is enqueued.
 */

/*
 * Pack eta, chi ([n_lambda][n_cells] float32, device) into planes
 * ([n_batch][n_cells][2W] float32, device).  A negative or non-finite chi or
 * eta, or a transparent emitter above 2^36, sets DEX_ERR_NUMERIC in the device
 * status word (the voxel is stored as empty).
 */
int dex_pack_planes(dex_ctx* ctx, int n_cells, int n_lambda, int W,
                    const float* eta, const float* chi, float* planes);

/* Number of floats of the planes array: n_batch * n_cells * 2W. */
size_t dex_planes_floats(int n_cells, int n_lambda, int W);

/* ------------------------------------------------------ plain formal solve --
 *
 * Section 1, Eq. RteIntegral with eta, chi constant per voxel (Section 4.1);
 * long characteristics (Section 1): from the centre of every probe cell, along
 * each quadrature direction d_k, the ray p(t) = p_c + t d_k is traced to the
 * grid boundary through the full-resolution grid with exact per-voxel path
 * lengths (Amanatides & Woo DDA, Section 2.3).  I_k is the intensity arriving
 * at the probe along that ray from the boundary, where it equals i_bc:
 *     I_k = i_bc e^{-sum tau} + sum_i S_i (1 - e^{-tau_i}) e^{-sum_{j<i} tau_j},
 * voxels i ordered from the probe outward, tau_i = chi_i l_i.
 * J = sum_k w_k I_k (mean intensity).
 *
 *   nx, nz     grid size (1 .. 65536 each)
 *   planes     device, wavelength-batch records of every cell (layout above)
 *   dirs       host [n_dir][2] (d_x, d_z), unit vectors; weights host [n_dir];
 *              1 <= n_dir <= DEX_MAX_DIRS
 *   n_probe    number of probes; n_probe < 0 means every cell (probes must be
 *              NULL, probe p = cell p); n_probe == 0 is a no-op
 *   probes     device [n_probe] cell indices (ignored when n_probe <= 0)
 *   J          device [n_lambda][n_probe] float32 output (overwritten)
 *   I          device [n_lambda][n_dir][n_probe] float32 output, or NULL
 *   seg_count  device uint64 accumulator, or NULL: adds the number of
 *              non-zero-length voxel segments traversed (one per ray and voxel,
 *              counted once per wavelength batch)
 */
int dex_formal_solve_dense(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, const float* planes,
                           int n_dir, const float* dirs, const float* weights,
                           int n_probe, const int* probes, float i_bc,
                           float* J, float* I, unsigned long long* seg_count);

/* ------------------------------------------ static continuum + line model --
 *
 * Section 2, Eqs. EtaTot and ChiTot (eta = sum of line terms + background,
 * chi likewise) for one line over a continuum, with a line profile normalised
 * to its peak:  chi_l = ratio chi_c exp(-(dlam / dld)^2),  chi = chi_c + chi_l,
 * eta = chi_c S_c + chi_l S_l.
 *   chi_c, s_c, s_l, ratio, dld : device [n_cells] (continuum opacity, continuum
 *                                 and line source functions, peak line/continuum
 *                                 opacity ratio, Doppler width in the units of dlam)
 *   dlam                        : device [n_lambda] offsets from line centre
 *   eta, chi                    : device [n_lambda][n_cells] outputs
 */
int dex_synth_static_line(dex_ctx* ctx, int n_cells, int n_lambda, const float* chi_c, const float* s_c,
                          const float* s_l, const float* ratio, const float* dld, const float* dlam,
                          float* eta, float* chi);

/* ------------------------------------------------------ sparse block grid --
 *
 * Section 2.3: the grid is cut into DEX_BLOCK x DEX_BLOCK blocks (nx and nz must
 * be multiples of DEX_BLOCK); a block is empty when eta = chi = 0 in all its
 * cells at every wavelength (one sparsity map shared by all wavelengths,
 * Section 4.1).  Section 2.3.1: non-empty ("active") blocks are ranked along
 * the Morton Z-order curve of their block coordinates (bx in the even bits),
 * and a dense lookup table gives each block's rank.
 *
 *   eta, chi      device [n_lambda][nz][nx]
 *   block_offset  device [nbz * nbx] output: rank of block bz*nbx+bx, or -1 if empty
 *   active        device [nbz * nbx] output: active[r] = block index of rank r
 *                 (entries >= *n_active are left untouched)
 *   n_active      device int output: number of active blocks
 */
int dex_grid_build(dex_ctx* ctx, int nx, int nz, int n_lambda, const float* eta, const float* chi,
                   int* block_offset, int* active, int* n_active);

/* Packed 3-bit block-state words per wavelength batch: ceil(nbx * nbz / 21). */
size_t dex_state_words(int nx, int nz);

/* Voxel records of one active block's MIP chain, levels 0..max_mip: sum (16 >> m)^2. */
int dex_chain_voxels(int max_mip);

/* Record storage formats of the static bricks (accumulation along rays is float32 in all):
 *   DEX_STORE_F32  : S[W], chi[W] float32 (2W floats per voxel), stored per brick row:
 *                    the S[W] of the row's voxels in x order, then their chi[W]
 *   DEX_STORE_BF16 : S[W], chi[W] bfloat16, round to nearest    (W floats; W = 4 or 8)
 *   DEX_STORE_F16  : float32 max S, max chi, 2 pad words, then S / max S and chi / max chi
 *                    as float16, round to nearest (4 + W floats; W = 4 or 8).  Values
 *                    below 2^-14 of their record's maximum lose precision (subnormals)
 *                    and below 2^-24 of it become 0. */
enum { DEX_STORE_F32 = 0, DEX_STORE_BF16 = 1, DEX_STORE_F16 = 2 };

/* Floats of the brick array: n_batch * capacity * dex_chain_voxels(max_mip) * record floats. */
size_t dex_brick_floats(int capacity, int n_lambda, int W, int max_mip, int storage);

/* Variance-limited mipmapping parameters (Section 2.2, Section 4.1). */
typedef struct {
    float iod_eta;     /* IoD threshold for ln(eta Ds) (paper: 1)                          */
    float iod_chi;     /* IoD threshold for ln(chi Ds) (paper: 1)                          */
    float chi_ds_min;  /* always average where the largest child chi * Ds is below this (0.25) */
    int max_mip;       /* highest level, 0..4 (0: sparse skipping only)                   */
    int log_mean;      /* 1: log-space (geometric) mean of the children; 0: box filter     */
    int storage;       /* DEX_STORE_F32 / _BF16 / _F16 record format of the bricks         */
    int n_test_dirs;   /* moving-medium builds: 0 = the level test of Sections 3.1 / 3.2
                          alone; K in 1..16 = a group must also pass the IoD test on its
                          children's emissivity and opacity as a ray along each of K
                          in-plane propagation directions w_k = (cos 2 pi k / K,
                          sin 2 pi k / K) samples them (see dex_cav_mips_build);
                          ignored by the static builds                                     */
} dex_vlm_params;

/*
 * Build the MIP chains of every active block for each wavelength batch and
 * select each block's level (Sections 2.1, 2.2, 2.3.1).
 *   active, n_active  from dex_grid_build (device); capacity = host upper bound
 *                     on n_active (grid size of the launch; bricks are sized by it)
 *   params            host pointer
 *   level_cap         device [nbz * nbx] per-block upper bound on the level, or NULL
 *   bricks            device [n_batch][capacity][chain][record] output records (format
 *                     params->storage; alignment as for the planes above):
 *                     level m of a block starts at voxel sum_{k<m} (16 >> k)^2 and
 *                     is row-major over its (16 >> m)^2 voxels; in float32 each row of
 *                     side = 16 >> m voxels is S of voxels 0..side-1 (W floats each),
 *                     then chi of them (a warp's rays at neighbouring voxels of a row
 *                     then read contiguous runs); the other formats store one record
 *                     per voxel
 *   state_words       device [n_batch][dex_state_words] output (zeroed by the call):
 *                     block k's state (0 = empty, level + 1) in word k / 21, bits 3 (k % 21)
 * The level of a block is the largest m <= max_mip such that every 2x2 group of
 * every level 1..m inside it passes for every wavelength of the batch: both IoD
 * values below their thresholds, or largest child chi * Ds < chi_ds_min.
 */
int dex_mips_build(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, const float* eta, const float* chi,
                   const int* active, const int* n_active, int capacity, const dex_vlm_params* params,
                   const signed char* level_cap, float* bricks, unsigned long long* state_words);

/*
 * Accelerated formal solution (Section 2.3, Algorithm 1): the same long
 * characteristics as dex_formal_solve_dense, from the centre of every cell of
 * every active block, traversed with a hierarchical DDA that crosses empty
 * blocks in one step and steps at each block's selected MIP level.
 *   bricks, state_words, block_offset, active, n_active, capacity: from the calls above
 *   storage   the record format the bricks were built with (DEX_STORE_*)
 *   n_band, band  host [n_band] (n_band <= 4) non-decreasing distances, or band = NULL
 *       for no limit: a block first entered at ray parameter t is sampled at level
 *       min(selected level, #{m : band[m-1] <= t}), the long-characteristics form of
 *       the per-cascade maximum MIP level of Section 4.1 (full resolution near the
 *       probe, coarser levels only further out; n_band = 0 forces level 0)
 *   J   device [n_lambda][nz][nx] output; zeroed by the call, written at probe cells
 *   I   device [n_lambda][n_dir][nz][nx] output or NULL (zeroed by the call)
 *   seg_count  device uint64 accumulator or NULL: adds the voxel segments integrated
 */
int dex_formal_solve_hdda(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, int storage,
                          const float* bricks,
                          const unsigned long long* state_words, const int* block_offset, const int* active,
                          const int* n_active, int capacity, int n_dir, const float* dirs, const float* weights,
                          int n_band, const float* band, float i_bc, float* J, float* I,
                          unsigned long long* seg_count);

/* ------------------------------------------------ level populations (SE) --
 *
 * A multi-level atom with radiative lines and collisional coupling (cgs units).
 * Populations are float64 [n_level][n_cells]; temperature, electron and
 * hydrogen densities float32 [n_cells] (T <= 0 marks an empty cell: zero
 * populations, zero emissivity/opacity).  Wavelength samples are host arrays:
 * lambda_nm[n_lambda] and line_tag[n_lambda] (index of the line a sample
 * belongs to, or -1 for a background-only sample); n_lambda <= DEX_MAX_ATOM_LAMBDA.
 */
#define DEX_MAX_LEVELS 4
#define DEX_MAX_LINES 4
#define DEX_MAX_ATOM_LAMBDA 256

typedef struct {
    int n_level;                                  /* <= DEX_MAX_LEVELS                      */
    double energy_erg[DEX_MAX_LEVELS];            /* level energies above the ground level  */
    double g[DEX_MAX_LEVELS];                     /* statistical weights                    */
    int n_line;                                   /* <= DEX_MAX_LINES                       */
    int line_lower[DEX_MAX_LINES];
    int line_upper[DEX_MAX_LINES];
    double line_A[DEX_MAX_LINES];                 /* Einstein A_ul (1/s)                    */
    double line_lambda0_nm[DEX_MAX_LINES];        /* rest wavelengths                       */
    double upsilon[DEX_MAX_LEVELS][DEX_MAX_LEVELS]; /* collision strengths, [i][j] with i < j */
    double mass_amu;                              /* atomic mass (Doppler widths)           */
    double background_sigma;                      /* grey background opacity per electron (cm^2) */
    double cell_cm;                               /* voxel side: eta, chi are per voxel     */
} dex_atom;

/* Boltzmann (LTE) populations summing to n_H: the iteration's starting point. */
int dex_lte_populations(dex_ctx* ctx, const dex_atom* atom, int n_cells, const float* temperature,
                        const float* nh, double* pops);

/*
 * Section 2, Eqs. Eta and Chi (complete redistribution) for every line, plus a
 * grey background chi_c = background_sigma n_e with Planck source function:
 *   eta = (h nu / 4 pi) n_u A_ul phi(nu),  chi = (h nu / 4 pi)(n_l B_lu - n_u B_ul) phi(nu),
 * B_ul = A_ul c^2 / (2 h nu0^3), B_lu = (g_u / g_l) B_ul, phi a Doppler profile
 * (width nu0/c sqrt(2kT/m)) renormalised to unit trapezoid quadrature over the
 * line's samples.  Outputs float32 [n_lambda][n_cells], per voxel (x cell_cm).
 */
int dex_atom_eta_chi(dex_ctx* ctx, const dex_atom* atom, int n_cells, int n_lambda, const double* lambda_nm,
                     const int* line_tag, const float* temperature, const float* ne, const double* pops,
                     float* eta, float* chi);

/*
 * Radiative-rate reduction: Jbar[l][c] = sum_k w_k phi_k(c) J[k][c] over line l's
 * samples (trapezoid weights in frequency, the same renormalised profile), in
 * float64.  J: float32 [n_lambda][n_cells]; jbar: float64 [n_line][n_cells].
 */
int dex_rates_accumulate(dex_ctx* ctx, const dex_atom* atom, int n_cells, int n_lambda, const double* lambda_nm,
                         const int* line_tag, const float* temperature, const float* J, double* jbar);

/*
 * Per-cell statistical equilibrium in float64: rates R_lu = B_lu Jbar,
 * R_ul = A_ul + B_ul Jbar, collisional C_ij = n_e 8.629e-6 / (g_i sqrt T) Upsilon_ij
 * e^{-dE/kT} (i < j) with detailed balance for C_ji; sum_j n_j P_ji = n_i sum_j P_ij,
 * the ground-level equation replaced by sum_i n_i = n_H.  pops: float64 output.
 */
int dex_se_solve(dex_ctx* ctx, const dex_atom* atom, int n_cells, const float* temperature, const float* ne,
                 const float* nh, const double* jbar, double* pops);

/*
 * MALI (Section 4.1: multilevel accelerated lambda iteration with same-transition
 * preconditioning and a diagonal approximate operator, after Rybicki & Hummer
 * 1992).  One iteration from populations n' (pops) and the J of their emissivity
 * and opacity (the formal solution of dex_atom_eta_chi's output):
 *
 *   dex_mali_rates       per line and cell, in float64,
 *                          rho      = 1 - Psibar,
 *                          Psibar   = sum_k w_k phi_k Lambda*_k chi_line,k / chi_k,
 *                          Jbar_eff = sum_k w_k phi_k (J_k - Lambda*_k eta_line,k / chi_k),
 *                        over the line's samples (trapezoid weights in frequency,
 *                        the renormalised profile of dex_rates_accumulate), with
 *                        eta, chi of n' (float64, per cell) and the diagonal
 *                        operator of the long-characteristics solve
 *                          Lambda*_k = sum_d w_d (1 - e^{-chi_k l_d}),
 *                          l_d = 1 / (2 max(|d_x|, |d_z|)) cells
 *                        (the path from the probe's centre to its cell boundary;
 *                        the own cell adds S (1 - e^{-chi l_d}) to I_d).  The
 *                        input Jext is the formal solution with each probe's
 *                        own-cell emission left out (dex_ctx_set_own_cell(ctx, 0)),
 *                        J = Jext + Lambda* (eta_line + eta_c) / chi, and the call
 *                        evaluates Jbar_eff = sum_k w_k phi_k (Jext_k + Lambda*_k
 *                        eta_c,k / chi_k) and rho = sum_k w_k phi_k ((1 - Lambda*_k)
 *                        chi_line,k + chi_c) / chi_k (the profile has unit
 *                        quadrature): the same numbers, without the cancellations
 *                        of J minus the own-cell term and of 1 minus Psibar, which
 *                        in cells thick at every sampled frequency exceed float32.
 *                        dirs, weights: host [n_dir][2], [n_dir] as in the
 *                        solvers.  rho, jeff: float64 device [n_line][n_cells].
 *   dex_se_solve_preconditioned
 *                        the statistical equilibrium of dex_se_solve with the
 *                        preconditioned radiative rates R_ul = A_ul rho + B_ul
 *                        Jbar_eff, R_lu = B_lu Jbar_eff: the MALI populations.
 *   dex_max_rel_change   out (device, one double) = max over cells with T > 0 and
 *                        over levels of |new - old| / new (the convergence
 *                        measure of Section 4.1); a non-finite value propagates.
 *
 * Arguments as dex_rates_accumulate / dex_se_solve; null buffers or bad sizes ->
 * DEX_ERR_ARG.  The caller owns every buffer.
 */
int dex_mali_rates(dex_ctx* ctx, const dex_atom* atom, int n_cells, int n_lambda, const double* lambda_nm,
                   const int* line_tag, const float* temperature, const float* ne, const double* pops,
                   const float* Jext, int n_dir, const float* dirs, const float* weights, double* rho, double* jeff);
int dex_se_solve_preconditioned(dex_ctx* ctx, const dex_atom* atom, int n_cells, const float* temperature,
                                const float* ne, const float* nh, const double* rho, const double* jeff, double* pops);
int dex_max_rel_change(dex_ctx* ctx, int n_level, int n_cells, const float* temperature, const double* old_pops,
                       const double* new_pops, double* out);

/* ------------------------------------------------------------------ Voigt --
 *
 * Section 3.2: the Voigt function H(a, x) = Re w(x + i a) by HUM1WEI24
 * (Humlicek 1982 region I for |x| + a >= 15, Weideman 1994 with 24 terms
 * otherwise), float32; the form the Core-and-Voigt solver evaluates per segment.
 * a, x, h: device [n] (a >= 0).
 */
int dex_voigt(dex_ctx* ctx, int n, const float* a, const float* x, float* h);

/* ------------------------------------------------------ Core and Voigt --
 *
 * Section 3.2: a moving medium with one spectral line over an isotropic
 * background.  Per cell (device [nz][nx] float32 fields): line strengths eta*,
 * chi* (per km/s), Voigt damping a, thermal width v_th (km/s), velocity v_x, v_z
 * (km/s), background eta_c, chi_c.  Wavelengths are velocity offsets dv (km/s)
 * from the rest wavelength; c_kms is the speed of light in km/s.  For a ray
 * traced toward +d the radiation propagates along w = -d and
 *   u = dv + v.w,  s = 1/(1 + dv/c),  phi = H(a/s^2, u/v_th)/(sqrt(pi) v_th),
 *   eta = eta* s phi + eta_c,  chi = chi* s phi + chi_c,
 * with H by HUM1WEI24 (dex_voigt).  n_lambda <= DEX_MAX_CAV_LAMBDA.
 */
#define DEX_MAX_CAV_LAMBDA 256

typedef struct {
    const float* eta_star;
    const float* chi_star;
    const float* damping;
    const float* vth;
    const float* vx;
    const float* vz;
    const float* eta_c;
    const float* chi_c;
} dex_cav_fields;

/* Sparsity map + Morton layout from the CaV fields (block empty when eta*, chi*,
 * eta_c, chi_c all vanish in it); outputs as dex_grid_build. */
int dex_cav_grid_build(dex_ctx* ctx, int nx, int nz, const dex_cav_fields* fields, int* block_offset, int* active,
                       int* n_active);

/* Floats of the CaV parameter bricks: capacity * dex_chain_voxels(max_mip) * 8. */
size_t dex_cav_brick_floats(int capacity, int max_mip);

/*
 * Box-filter MIP chains of the 8 voxel parameters (one set for all wavelengths:
 * bricks [capacity][chain][8] = eta*, chi*, a, 1/v_th, v_x, v_z, eta_c, chi_c) and
 * the block level per wavelength batch: Eq. IoD of ln(eta Ds), ln(chi Ds) with each
 * child's eta, chi evaluated at the Doppler shift closest to line centre its speed
 * allows (|u| = max(0, |dv| - |v|), Section 3.2), plus the always-average rule.
 * dv: host [n_lambda].  Other arguments as dex_mips_build (log_mean is ignored).
 */
int dex_cav_mips_build(dex_ctx* ctx, int nx, int nz, const dex_cav_fields* fields, int n_lambda, int W,
                       const float* dv, float c_kms, const int* active, const int* n_active, int capacity,
                       const dex_vlm_params* params, const signed char* level_cap, float* bricks,
                       unsigned long long* state_words);

/*
 * CaV formal solution: the hierarchical DDA of dex_formal_solve_hdda over the
 * parameter bricks, evaluating eta, chi per segment and wavelength for the ray's
 * direction (HUM1WEI24 Voigt profile).  Arguments as dex_formal_solve_hdda plus
 * dv (host [n_lambda]) and c_kms.
 */
int dex_formal_solve_cav(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* dv,
                         float c_kms, const float* bricks, const unsigned long long* state_words,
                         const int* block_offset, const int* active, const int* n_active, int capacity, int n_dir,
                         const float* dirs, const float* weights, int n_band, const float* band, float i_bc,
                         float* J, float* I, unsigned long long* seg_count);

/* The Core-and-Voigt solve with the learned surrogate network (see
 * dex_mlp_forward below) as the line profile: inside the network's training
 * domain (1e-3 <= a' <= 1e-1, |x| <= 16, |u| <= 10 with x = dv / v_th,
 * a' = a / s^2, u = -(v . w) / v_th) H = exp(network(x, a', u)), evaluated in
 * float32 on the CUDA cores with W1, W2, w3 rounded to bfloat16; outside it the
 * HUM1WEI24 evaluation of dex_formal_solve_cav.  mlp_params: HOST array of
 * dex_mlp_param_count() floats (copied into the launch; non-finite -> DEX_ERR_ARG).
 * Other arguments as dex_formal_solve_cav.  The paper has no counterpart. */
int dex_formal_solve_cav_mlp(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* dv,
                             float c_kms, const float* bricks, const unsigned long long* state_words,
                             const int* block_offset, const int* active, const int* n_active, int capacity,
                             int n_dir, const float* dirs, const float* weights, int n_band, const float* band,
                             float i_bc, const float* mlp_params, float* J, float* I, unsigned long long* seg_count);

/* --------------------------------------------------- velocity interpolation --
 *
 * Section 3.1 with the line model above: every MIP voxel (MIP 0 included)
 * stores, per wavelength batch, its mean velocity, V = the largest speed of its
 * MIP-0 cells, and eta, chi at DEX_VEL_SAMPLES projected velocities
 * v_s = -V + 2 V s / (DEX_VEL_SAMPLES - 1) (each the mean over the voxel's MIP-0
 * cells of the cell's eta, chi at u = dv + v_s).  Along a ray the voxel's eta,
 * chi are interpolated linearly at the projected mean velocity, clamped to
 * [-V, V].  Block levels come from Eq. IoD on the rest-frame (projected
 * velocity 0) values.  Record: 4 + DEX_VEL_SAMPLES * 2W floats
 * (v_x, v_z, V, 0, then for each grid velocity eta[W], chi[W]).
 */
#define DEX_VEL_SAMPLES 8

/* Floats of the velocity-grid bricks: n_batch * capacity * chain * (4 + 16 W). */
size_t dex_vel_brick_floats(int capacity, int n_lambda, int W, int max_mip);

/* Build the velocity-grid MIP chains and the per-batch block levels; arguments as
 * dex_cav_mips_build (bricks sized by dex_vel_brick_floats). */
int dex_vel_mips_build(dex_ctx* ctx, int nx, int nz, const dex_cav_fields* fields, int n_lambda, int W,
                       const float* dv, float c_kms, const int* active, const int* n_active, int capacity,
                       const dex_vlm_params* params, const signed char* level_cap, float* bricks,
                       unsigned long long* state_words);

/* Formal solution with velocity interpolation; arguments as dex_formal_solve_hdda. */
int dex_formal_solve_velinterp(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* bricks,
                               const unsigned long long* state_words, const int* block_offset, const int* active,
                               const int* n_active, int capacity, int n_dir, const float* dirs, const float* weights,
                               int n_band, const float* band, float i_bc, float* J, float* I,
                               unsigned long long* seg_count);

/* ---------------------------------------------------- batched atmospheres --
 *
 * Many independent atmospheres solved by one persistent launch: a fixed grid of
 * CTAs pulls work items (atmosphere, wavelength batch, active block) from a
 * device counter until none are left; each item is the 256-probe block solve of
 * dex_formal_solve_hdda (static records).  The atmospheres share the batch
 * width W and differ in size, wavelengths, quadrature and sparsity.
 */
#define DEX_MAX_BATCH_ATM 32

typedef struct {
    int nx, nz, n_lambda, max_mip, capacity;      /* as for dex_formal_solve_hdda          */
    const float* bricks;                          /* device, from dex_mips_build           */
    const unsigned long long* state_words;        /* device                                */
    const int* block_offset;                      /* device, from dex_grid_build           */
    const int* active;                            /* device                                */
    const int* n_active;                          /* device                                */
    int n_dir;                                    /* 1 .. DEX_MAX_DIRS                     */
    const float* dirs;                            /* DEVICE [n_dir][2] unit vectors         */
    const float* weights;                         /* DEVICE [n_dir]                        */
    int n_band;                                   /* distance limits as dex_formal_solve_hdda; */
    float band[4];                                /*   n_band < 0: none                    */
    float i_bc;
    float* J;                                     /* device [n_lambda][nz][nx], zeroed here */
} dex_batch_item;

/*
 * Solve n_atm (<= DEX_MAX_BATCH_ATM) atmospheres in one persistent launch.
 *   atms     host [n_atm] descriptors (device pointers inside)
 *   ctas     persistent grid size (0: 3 per SM)
 *   queue    device scratch: one unsigned int, the work counter (reset by the call)
 *   done_ns  device [n_atm] or NULL: completion time of each atmosphere's last item
 *            (GPU global timer, ns), start_ns device [1] or NULL: the earliest CTA start
 * Every J is zeroed by the call, then written at the probe cells.
 */
int dex_batch_solve(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, int ctas, unsigned int* queue,
                    unsigned long long* done_ns, unsigned long long* start_ns);

/*
 * Launch configuration of the batched solve (the knobs an autotuner sweeps; no
 * paper counterpart -- the paper batches wavelengths within one model, Section 4.1):
 *   ctas     persistent grid size (0: 3 per SM)
 *   packet   probes per work item: 256 (a whole block), 128 or 64 (a 16 x 8 or
 *            16 x 4 part of it; the CTA then has that many threads)
 *   chunk    work items a CTA claims per increment of the queue counter (1..64)
 *   staging  how the CTA stages its atmosphere-batch's block table in shared
 *            memory: 0 the packed 3-bit state words (plus the global offset
 *            table), 1 one word per block, offset * 8 + state (every grid of
 *            the batch at most 8192 blocks)
 *   occupancy  0: the compiler's register budget; 1 (W = 8 only): 64 registers
 *            a thread, so that 1024 threads a SM are resident (some spilling)
 * Every probe accumulates J over the directions in one thread in the order of
 * dex_formal_solve_hdda, so J is bit-identical for every configuration.
 * dex_batch_solve is dex_batch_solve_config with {ctas, 256, 1, 0, 0}.  Invalid
 * values -> DEX_ERR_ARG.
 * With the context's traversal set to DEX_TRAVERSAL_PAIRED (W = 8; every grid
 * of at most 8192 blocks, else DEX_ERR_UNSUPPORTED) the work units are each
 * atmosphere's pairs of batches (dex_ctx_set_pair_group) and lone batches, and
 * J equals that of dex_formal_solve_hdda's paired walk bit for bit; staging
 * and occupancy then do not apply (one word per block is staged, at most 128
 * registers a thread).  dex_batch_solve and dex_batch_solve_noalloc follow the
 * setting too.
 */
typedef struct {
    int ctas;
    int packet;
    int chunk;
    int staging;
    int occupancy;
} dex_batch_config;

int dex_batch_solve_config(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, const dex_batch_config* cfg,
                           unsigned int* queue, unsigned long long* done_ns, unsigned long long* start_ns);

/*
 * Allocation-free variant of dex_batch_solve (the paper has no counterpart:
 * this is a deployment convenience of this library).
 *
 * For callers that cannot allocate device memory when they solve: a host
 * application that owns every byte of the device through its own pool, or a
 * time-critical loop where a cudaMalloc -- which may synchronise the device --
 * is not acceptable.  Such a caller has no place to put the one scratch word
 * (the work counter) that dex_batch_solve takes as `queue`.  This entry point
 * keeps that scratch in a statically sized device array inside the library
 * instead: DEX_NOALLOC_SCRATCH_WORDS words (256 bytes), held on every GPU that
 * loads the library until the process exits.  The caller still provides all
 * inputs and outputs (descriptors, J, optional done_ns / start_ns).
 *
 * - It calls no cudaMalloc/cudaFree and no other allocating routine, on the
 *   device or the host; the counter is reset by the call before the launch.
 *   The CUDA driver itself reserves device memory when it first loads the
 *   library's kernels into a context (code and static data, this array
 *   included), and it may do that lazily on the first call of any dex_* entry
 *   point on the device: a caller that must not see that happen during its solve
 *   makes one call at initialisation, before any stream capture.
 * - Every call looks up the array's device address on the current device (a
 *   runtime table look-up, not an allocation), so a cudaDeviceReset between
 *   calls is safe: the next call uses the new context's array.
 * - Every call shares the same array: calls that overlap on the GPU (different
 *   streams, or different contexts on one device) race on the counter.
 *   Serialise them.
 * - Limits as dex_batch_solve: n_atm <= DEX_MAX_BATCH_ATM and at most 2^32 - 1
 *   work items in total; larger requests are rejected with DEX_ERR_ARG.
 * Arguments and results otherwise as dex_batch_solve (no `queue`).
 */
#define DEX_NOALLOC_SCRATCH_WORDS 64

int dex_batch_solve_noalloc(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, int ctas,
                            unsigned long long* done_ns, unsigned long long* start_ns);

/* Measured throughput (operations per second) of the special-function unit's
 * 2^x (ex2.approx.ftz.f32) on the context's device: every segment-wavelength
 * update of the solvers needs one, so this is the ceiling their update rate is
 * reported against.  Runs a short probe kernel (8 x SMs CTAs, ~1 ms) on the
 * context's stream and synchronises it; allocates and frees 1.2 MB of device
 * memory.  No paper counterpart (a measurement utility). */
int dex_measure_ex2_rate(dex_ctx* ctx, double* ops_per_s);

/* Measured throughput (lane operations per second) of the FP32 pipe on packed
 * fused multiply-adds (FFMA2: two lane operations per instruction) on the
 * context's device: the unit every multiply and add of the segment update
 * (Eq. RteIntegral with the 1 - e^{-tau} series) occupies, and with ten of them
 * per segment-wavelength the tighter of the solvers' two arithmetic ceilings.
 * Runs a short probe kernel (8 x SMs CTAs, ~1 ms) on the context's stream and
 * synchronises it; allocates and frees 1.2 MB of device memory.  No paper
 * counterpart (a measurement utility). */
int dex_measure_fp32_rate(dex_ctx* ctx, double* ops_per_s);

/* Self-test of the device-side failure path: one thread waits on an mbarrier
 * that nothing arrives on, with the same bounded wait the tensor-core kernels
 * use, giving up after `polls` (1 .. 1e6) polls; the next dex_ctx_check then
 * returns DEX_ERR_TIMEOUT and the context stays usable.  No fault, no hang. */
int dex_selftest_wait_timeout(dex_ctx* ctx, int polls);

/* ------------------------------------------------------------------------
 * Learned Voigt-profile surrogate.  The paper evaluates the Voigt profile of
 * the Core-and-Voigt treatment on the fly (Section 3.2); this library adds a
 * small network trained on the profiles that evaluation produces, as an
 * alternative to it.  The paper has no counterpart of these calls.
 *
 * Network: features f = (x / 16, log10(a) + 2, u / 16) of the wavelength offset
 * x from line centre in Doppler widths (rest frame), the damping a and the
 * projected velocity u in Doppler widths; h1 = GELU(W1 f + b1) (64),
 * h2 = GELU(W2 h1 + b2) (64), y = w3 . h2 + b3 predicts ln H(a, x - u).
 * GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
 * Parameters: one float32 array of dex_mlp_param_count() = 4481 values:
 *   W1 [64][3] at 0, b1 [64] at 192, W2 [64][64] (row = output) at 256,
 *   b2 [64] at 4352, w3 [64] at 4416, b3 at 4480.
 * The kernels use W1, W2, w3 rounded to bfloat16 (round to nearest even) and
 * the bfloat16-rounded h1 as tensor-core operands; all sums are float32.
 * Samples xau are [n][3] float32 (x, a, u), device memory, 0 <= n <= 2^38
 * (DEX_ERR_ARG otherwise).  A sample with a non-finite value or a <= 0 is
 * skipped and sets DEX_ERR_NUMERIC.
 * ---------------------------------------------------------------------- */
int dex_mlp_param_count(void);

/* ln H predictions out[n] (device) for n >= 0 samples. */
int dex_mlp_forward(dex_ctx* ctx, long long n, const float* xau, const float* params, float* out);

/* Mean squared error L = (1/n) sum (y - target)^2 over n >= 0 samples and its
 * gradient with respect to every parameter: grad (device, dex_mlp_param_count()
 * floats) and loss (device, one float) are overwritten.  Gradients through the
 * tensor cores use bfloat16 operands: the per-sample output errors of layer 2
 * (delta2 = dy w3 GELU'(z2)), dy h2, the layer-1 errors and the features. */
int dex_mlp_grad(dex_ctx* ctx, long long n, const float* xau, const float* target, const float* params,
                 float* grad, float* loss);

/* One Adam step (Kingma & Ba 2015) on the float32 parameters, step >= 1:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * All arrays device memory of dex_mlp_param_count() floats. */
int dex_mlp_adam(dex_ctx* ctx, float* params, const float* grad, float* m, float* v, int step, float lr,
                 float beta1, float beta2, float eps);

/* Training targets ln H(a, x - u) from the library's own Voigt evaluation
 * (dex_voigt's scheme), out[n] device. */
int dex_mlp_targets(dex_ctx* ctx, long long n, const float* xau, float* out);

/* ============================================================== 3D grids ==
 *
 * Section 2.3: the adapted grid "generalises directly to 3D": cubic blocks of
 * DEX_BLOCK3^3 = 8^3 voxels, each empty or at one MIP level in 0..3 (Section
 * 2.3.1: a block reduces to a single entry at level 3), MIP groups of 2x2x2
 * voxels (Section 2.1).  Grids are [nz][ny][nx] with x fastest: cell
 * c = (k * ny + j) * nx + i.  Directions are host [n_dir][3] (d_x, d_y, d_z)
 * finite unit vectors, 1 <= n_dir <= DEX_MAX_DIRS, weights host [n_dir].
 * Every 3D call needs nx * ny * nz <= 2^31 - 1 cells and each extent <= 2048
 * (the Morton layout walks a cube of at most 256^3 block codes).
 */

/*
 * Plain full-resolution 3D formal solution: dex_formal_solve_dense on three
 * axes.  From the centre of every probe cell along each d_k the ray is traced
 * to the grid boundary (where the intensity is i_bc) through every voxel with
 * exact path lengths; I_k and J = sum_k w_k I_k as in 2D.
 *   planes     device wavelength-batch records of every cell (dex_pack_planes
 *              with n_cells = nx * ny * nz)
 *   n_probe    < 0: every cell (probes NULL, probe p = cell p); 0: no-op
 *   probes     device [n_probe] cell indices
 *   J          device [n_lambda][n_probe] output (overwritten)
 *   I          device [n_lambda][n_dir][n_probe] output or NULL
 *   seg_count  device uint64 accumulator or NULL (non-zero-length segments)
 */
int dex_formal_solve_dense3(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, int W, const float* planes,
                            int n_dir, const float* dirs, const float* weights, int n_probe, const int* probes,
                            float i_bc, float* J, float* I, unsigned long long* seg_count);

/*
 * Sparsity map and Morton layout of a 3D grid (nx, ny, nz positive multiples of
 * 8).  A block is empty when eta = chi = 0 in all its cells at every
 * wavelength; active blocks are ranked along the Z-order curve of (bx, by, bz)
 * (bit b of bx, by, bz at bits 3b, 3b + 1, 3b + 2).
 *   eta, chi      device [n_lambda][nz][ny][nx]
 *   block_offset  device [nbz * nby * nbx] output: rank of block (bz * nby + by) * nbx + bx, or -1
 *   active        device [nbz * nby * nbx] output: block index of each rank
 *   n_active      device int output
 */
int dex_grid3_build(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, const float* eta, const float* chi,
                    int* block_offset, int* active, int* n_active);

/* Packed 3-bit block-state words per wavelength batch: ceil(nbx * nby * nbz / 21). */
size_t dex_state_words3(int nx, int ny, int nz);

/* Voxel records of one 3D chain, levels 0..max_mip (max_mip <= 3): sum (8 >> m)^3. */
int dex_chain_voxels3(int max_mip);

/* Floats of the 3D brick array: n_batch * capacity * dex_chain_voxels3(max_mip) * record floats. */
size_t dex_brick3_floats(int capacity, int n_lambda, int W, int max_mip, int storage);

/*
 * 3D MIP chains and level selection (dex_mips_build on 2x2x2 groups; the IoD
 * test, always-average rule, means and per-batch level rule are the same).
 * params->max_mip must be in 0..3.  Level m of a block starts at record
 * sum_{k<m} (8 >> k)^3 and is row-major [z][y][x] over (8 >> m)^3 voxels.
 *   level_cap  device [nbz * nby * nbx] per-block upper bound, or NULL
 *   bricks, state_words  outputs as in dex_mips_build (state words zeroed by the call)
 */
int dex_mips3_build(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, int W, const float* eta,
                    const float* chi, const int* active, const int* n_active, int capacity,
                    const dex_vlm_params* params, const signed char* level_cap, float* bricks,
                    unsigned long long* state_words);

/*
 * Accelerated 3D formal solution (Section 2.3, Algorithm 1 on three axes): from
 * the centre of every cell of every active block, hierarchical DDA over the
 * 8^3 blocks, empty blocks crossed in one step, each non-empty block sampled at
 * its level capped by the distance limits (n_band <= 4 non-decreasing
 * thresholds, band = NULL for none; as dex_formal_solve_hdda).
 *   J   device [n_lambda][nz][ny][nx] output; zeroed by the call, written at probe cells
 *   I   device [n_lambda][n_dir][nz][ny][nx] output or NULL (zeroed by the call)
 *   seg_count  device uint64 accumulator or NULL: adds the voxel segments integrated
 * With the context's traversal set to DEX_TRAVERSAL_PAIRED (W = 8 and at most
 * 8192 state words, else DEX_ERR_UNSUPPORTED) one walk serves each pair of
 * batches b, n_batch - 1 - b on the smaller of their levels, as in the 2D
 * solve; every other traversal setting gives one walk per batch.
 */
int dex_formal_solve_hdda3(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, int W, int max_mip, int storage,
                           const float* bricks, const unsigned long long* state_words, const int* block_offset,
                           const int* active, const int* n_active, int capacity, int n_dir, const float* dirs,
                           const float* weights, int n_band, const float* band, float i_bc, float* J, float* I,
                           unsigned long long* seg_count);

/* ===================================================== radiance cascades ==
 *
 * The radiance-cascade formal solution the paper's code wraps around its
 * traversal (Section 4.1 "Model Configuration"), in 2D: with branching factor 2
 * cascade i has probes on a lattice of spacing 2^i (probe (px, pz) at
 * (2^i (px + 1/2), 2^i (pz + 1/2))), n0 4^i directions and the radiance
 * interval [t0 4^(i-1), t0 4^i] (cascade 0: [0, t0]; the paper: n0 = 4,
 * t0 = 1.5, 6 cascades, level caps [0, 0, 1, 2, 3, 4]).  Each interval is
 * traced through the sparse mipmapped grid of dex_mips_build at
 * min(block level, level_cap[i]) (empty blocks skipped), giving emission I and
 * transmission T.  Merged radiance L = I + T R, from the top cascade down: R is
 * i_bc if the ray leaves the grid inside its interval or on the top cascade,
 * else the bilinear interpolation at the probe of the mean over the 4 child
 * directions 4k .. 4k+3 of the cascade above (4 nearest probes, indices clamped
 * at the lattice edge).  J = the mean of L over the n0 cascade-0 directions.
 */

/* Floats of the workspace: 2 * n_batch * n0 * nx * nz * W (two cascades' merged radiance). */
size_t dex_rc_workspace_floats(int nx, int nz, int n_lambda, int W, int n0);

/*
 *   nx, nz        multiples of 16 and of 2^(n_cascades - 1); n0 * nx * nz <= 2^31 - 1
 *   bricks ... capacity, max_mip, storage: from dex_grid_build / dex_mips_build
 *                 (storage: F32 with W = 1, 2, 4, 8; BF16 or F16 with W = 8)
 *   n_cascades    1 .. 8;  n0: 1 .. 64 cascade-0 directions;  t0 > 0 (cascade-0 interval end)
 *   level_cap     host [n_cascades], each in 0 .. max_mip
 *   dirs          device [sum_i n0 4^i][2]: the directions of cascade 0, then 1, ...
 *                 (unit vectors; direction k of cascade i+1's block 4k .. 4k+3 should
 *                 split direction k of cascade i)
 *   workspace     device, dex_rc_workspace_floats floats (16-byte aligned)
 *   J             device [n_lambda][nz][nx] output: zeroed by the call, written at every
 *                 cell of every non-empty block
 *   seg_count     device uint64 accumulator or NULL: adds the voxel segments integrated
 * With the context's traversal set to DEX_TRAVERSAL_PAIRED and W = 8, every
 * interval walks once for each pair of batches (dex_ctx_set_pair_group) on the
 * smaller of their levels, capped by the cascade's cap, lone batches alone;
 * each segment then counts once per batch of the pair.
 */
int dex_rc_solve(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, int storage, const float* bricks,
                 const unsigned long long* state_words, const int* block_offset, int capacity, int n_cascades,
                 int n0, float t0, const int* level_cap, const float* dirs, float i_bc, float* workspace, float* J,
                 unsigned long long* seg_count);

#ifdef __cplusplus
}
#endif

#endif /* DEXGB_H */
