// C-ABI entry points of libdexgb: argument checks, context, launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "dex_internal.h"
#include "dexgb.h"

struct dex_ctx {
    int device;
    cudaStream_t stream;
    unsigned int* status;  // device word, OR of DEX_ERR_* bits raised by kernels
    int traversal = DEX_TRAVERSAL_PER_BATCH;  // static accelerated solve: one walk per wavelength batch
    int pair_group = 0;                        // paired walk: batches paired within groups of this many
    int own_cell = 1;                          // solvers include each probe's own-cell emission
    char msg[512];
};

namespace {

int fail(dex_ctx* ctx, int code, const char* fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->msg, sizeof(ctx->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

int ok(dex_ctx* ctx)
{
    if (ctx) ctx->msg[0] = '\0';
    return DEX_OK;
}

int cuda_fail(dex_ctx* ctx, cudaError_t e, const char* where)
{
    return fail(ctx, DEX_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Make the context's device current for the calling thread.
int bind(dex_ctx* ctx)
{
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return DEX_OK;
}

bool valid_W(int W) { return W == 1 || W == 2 || W == 4 || W == 8; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
// Alignment the record loads need: W = 8 float32 (64-byte) and bfloat16 (32-byte)
// records are read with 256-bit loads; other records with 128-bit (W = 1: 64-bit) loads.
size_t rec_align(int W, int storage)
{
    if (W == 8 && (storage == DEX_STORE_F32 || storage == DEX_STORE_BF16)) return 32;
    return W == 1 ? 8 : 16;
}

int fill_quadrature(dex_ctx* ctx, int n_dir, const float* dirs, const float* weights, dex::Quadrature& q)
{
    if (n_dir < 1 || n_dir > DEX_MAX_DIRS)
        return fail(ctx, DEX_ERR_ARG, "n_dir must be in [1, %d], got %d", DEX_MAX_DIRS, n_dir);
    if (!dirs || !weights) return fail(ctx, DEX_ERR_ARG, "dirs and weights (host arrays) are required");
    q.n_dir = n_dir;
    for (int k = 0; k < n_dir; ++k) {
        const float dx = dirs[2 * k], dz = dirs[2 * k + 1];
        const float n2 = dx * dx + dz * dz;
        if (!std::isfinite(dx) || !std::isfinite(dz) || std::fabs(n2 - 1.0f) > 1e-4f)
            return fail(ctx, DEX_ERR_ARG, "direction %d is not a finite unit vector", k);
        if (!std::isfinite(weights[k])) return fail(ctx, DEX_ERR_ARG, "weight %d is not finite", k);
        q.dx[k] = dx;
        q.dz[k] = dz;
        q.w[k] = weights[k];
    }
    return DEX_OK;
}

constexpr double kH_ = 6.62607015e-27;
constexpr double kC_ = 2.99792458e10;

// Validate the atom and the wavelength samples; fill the launch parameters
// (frequencies, per-line trapezoid weights in frequency, Einstein B).
int fill_atom(dex_ctx* ctx, const dex_atom* atom, int n_lambda, const double* lambda_nm, const int* line_tag,
              dex::AtomParams& P)
{
    if (!atom) return fail(ctx, DEX_ERR_ARG, "atom required");
    if (atom->n_level < 2 || atom->n_level > DEX_MAX_LEVELS)
        return fail(ctx, DEX_ERR_ARG, "n_level must be in [2, %d]", DEX_MAX_LEVELS);
    if (atom->n_line < 0 || atom->n_line > DEX_MAX_LINES)
        return fail(ctx, DEX_ERR_ARG, "n_line must be in [0, %d]", DEX_MAX_LINES);
    for (int l = 0; l < atom->n_line; ++l) {
        const int lo = atom->line_lower[l], up = atom->line_upper[l];
        if (lo < 0 || up >= atom->n_level || lo >= up) return fail(ctx, DEX_ERR_ARG, "line %d has bad levels", l);
        if (!(atom->line_A[l] > 0.0) || !(atom->line_lambda0_nm[l] > 0.0))
            return fail(ctx, DEX_ERR_ARG, "line %d needs A > 0 and lambda0 > 0", l);
    }
    for (int i = 0; i < atom->n_level; ++i)
        if (!(atom->g[i] > 0.0)) return fail(ctx, DEX_ERR_ARG, "statistical weight %d must be > 0", i);
    if (!(atom->mass_amu > 0.0) || !(atom->cell_cm > 0.0) || !(atom->background_sigma >= 0.0))
        return fail(ctx, DEX_ERR_ARG, "mass, cell size must be > 0 and background_sigma >= 0");
    if (n_lambda < 0 || n_lambda > DEX_MAX_ATOM_LAMBDA)
        return fail(ctx, DEX_ERR_ARG, "n_lambda must be in [0, %d]", DEX_MAX_ATOM_LAMBDA);
    if (n_lambda > 0 && (!lambda_nm || !line_tag)) return fail(ctx, DEX_ERR_ARG, "lambda_nm and line_tag required");
    P.atom = *atom;
    P.n_lambda = n_lambda;
    for (int k = 0; k < n_lambda; ++k) {
        if (!(lambda_nm[k] > 0.0)) return fail(ctx, DEX_ERR_ARG, "wavelength %d must be > 0", k);
        if (line_tag[k] < -1 || line_tag[k] >= atom->n_line) return fail(ctx, DEX_ERR_ARG, "bad line tag %d", k);
        P.nu[k] = kC_ / (lambda_nm[k] * 1e-7);
        P.tag[k] = (signed char)line_tag[k];
        P.wq[k] = 0.0;
    }
    for (int l = 0; l < atom->n_line; ++l) {
        P.nu0[l] = kC_ / (atom->line_lambda0_nm[l] * 1e-7);
        P.b_ul[l] = atom->line_A[l] * kC_ * kC_ / (2.0 * kH_ * P.nu0[l] * P.nu0[l] * P.nu0[l]);
        P.b_lu[l] = atom->g[atom->line_upper[l]] / atom->g[atom->line_lower[l]] * P.b_ul[l];
        // trapezoid weights over the line's samples in increasing frequency
        int idx[DEX_MAX_ATOM_LAMBDA], n = 0;
        for (int k = 0; k < n_lambda; ++k)
            if (line_tag[k] == l) idx[n++] = k;
        for (int a = 1; a < n; ++a)  // insertion sort by frequency
            for (int b = a; b > 0 && P.nu[idx[b]] < P.nu[idx[b - 1]]; --b) {
                const int t = idx[b];
                idx[b] = idx[b - 1];
                idx[b - 1] = t;
            }
        for (int a = 0; a + 1 < n; ++a) {
            const double h = P.nu[idx[a + 1]] - P.nu[idx[a]];
            P.wq[idx[a]] += 0.5 * h;
            P.wq[idx[a + 1]] += 0.5 * h;
        }
    }
    return DEX_OK;
}

// float -> nearest bfloat16 (ties to even), as a float; finite inputs
float bf16_round_host(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

}  // namespace

extern "C" {

int dex_version(void) { return DEX_VERSION; }

const char* dex_status_string(int s)
{
    switch (s) {
        case DEX_OK: return "ok";
        case DEX_ERR_ARG: return "invalid argument";
        case DEX_ERR_CUDA: return "CUDA error";
        case DEX_ERR_TRAVERSAL_CAP: return "ray traversal exceeded its step cap";
        case DEX_ERR_NUMERIC: return "negative or non-finite emissivity/opacity";
        case DEX_ERR_UNSUPPORTED: return "unsupported configuration";
        case DEX_ERR_TIMEOUT: return "a bounded device-side wait expired";
        default: return "combined device error bits";
    }
}

int dex_ctx_create(int device, void* stream, dex_ctx** out)
{
    if (!out) return DEX_ERR_ARG;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return DEX_ERR_CUDA;
    if (device < 0 || device >= n) return DEX_ERR_ARG;
    dex_ctx* ctx = new (std::nothrow) dex_ctx();
    if (!ctx) return DEX_ERR_ARG;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->msg[0] = '\0';
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        delete ctx;
        return DEX_ERR_CUDA;
    }
    *out = ctx;
    return DEX_OK;
}

int dex_ctx_destroy(dex_ctx* ctx)
{
    if (!ctx) return DEX_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->status);
    delete ctx;
    return DEX_OK;
}

int dex_ctx_set_traversal(dex_ctx* ctx, int mode)
{
    if (!ctx) return DEX_ERR_ARG;
    if (mode != DEX_TRAVERSAL_PER_BATCH && mode != DEX_TRAVERSAL_SHARED && mode != DEX_TRAVERSAL_PAIRED)
        return fail(ctx, DEX_ERR_ARG,
                    "traversal mode must be DEX_TRAVERSAL_PER_BATCH, DEX_TRAVERSAL_SHARED or DEX_TRAVERSAL_PAIRED");
    ctx->traversal = mode;
    return ok(ctx);
}

int dex_ctx_set_pair_group(dex_ctx* ctx, int group)
{
    if (!ctx) return DEX_ERR_ARG;
    if (group < 0) return fail(ctx, DEX_ERR_ARG, "pair group must be >= 0, got %d", group);
    ctx->pair_group = group;
    return ok(ctx);
}

int dex_ctx_set_own_cell(dex_ctx* ctx, int include)
{
    if (!ctx) return DEX_ERR_ARG;
    if (include != 0 && include != 1) return fail(ctx, DEX_ERR_ARG, "include must be 0 or 1");
    ctx->own_cell = include;
    return ok(ctx);
}

// solvers without the own-cell option refuse to run while it is off
static int own_cell_required(dex_ctx* ctx, const char* who)
{
    if (ctx->own_cell) return DEX_OK;
    return fail(ctx, DEX_ERR_UNSUPPORTED, "%s always includes the own-cell emission (dex_ctx_set_own_cell)", who);
}

int dex_ctx_set_stream(dex_ctx* ctx, void* stream)
{
    if (!ctx) return DEX_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return ok(ctx);
}

int dex_ctx_check(dex_ctx* ctx)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = bind(ctx)) return r;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    unsigned int h = 0;
    e = cudaMemcpy(&h, ctx->status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(h));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status readback");
    if (h) return fail(ctx, (int)h, "device reported: %s%s%s", (h & DEX_ERR_TRAVERSAL_CAP) ? "traversal cap " : "",
                       (h & DEX_ERR_NUMERIC) ? "numeric " : "", (h & DEX_ERR_TIMEOUT) ? "wait timeout" : "");
    return ok(ctx);
}

const char* dex_last_error(const dex_ctx* ctx) { return ctx ? ctx->msg : "no context"; }

size_t dex_planes_floats(int n_cells, int n_lambda, int W)
{
    if (n_cells < 0 || n_lambda < 0 || !valid_W(W)) return 0;
    const size_t n_batch = (size_t)((n_lambda + W - 1) / W);
    return n_batch * (size_t)n_cells * (size_t)(2 * W);
}

int dex_pack_planes(dex_ctx* ctx, int n_cells, int n_lambda, int W, const float* eta, const float* chi,
                    float* planes)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n_cells < 0 || n_lambda < 0) return fail(ctx, DEX_ERR_ARG, "negative size");
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_cells == 0 || n_lambda == 0) return ok(ctx);
    if (!eta || !chi || !planes) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(planes, rec_align(W, DEX_STORE_F32)))
        return fail(ctx, DEX_ERR_ARG, "planes must be %zu-byte aligned", rec_align(W, DEX_STORE_F32));
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_pack_planes(ctx->stream, n_cells, n_lambda, W, eta, chi, planes, ctx->status);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pack_planes launch");
    return ok(ctx);
}

int dex_formal_solve_dense(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, const float* planes, int n_dir,
                           const float* dirs, const float* weights, int n_probe, const int* probes, float i_bc,
                           float* J, float* I, unsigned long long* seg_count)
{
    if (!ctx) return DEX_ERR_ARG;
    if (nx < 1 || nz < 1 || nx > 65536 || nz > 65536)
        return fail(ctx, DEX_ERR_ARG, "grid size must be in [1, 65536], got %d x %d", nx, nz);
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 0) return fail(ctx, DEX_ERR_ARG, "negative n_lambda");
    const long long n_cells = (long long)nx * nz;
    if (n_probe < 0) {  // every cell is a probe
        if (probes) return fail(ctx, DEX_ERR_ARG, "n_probe < 0 (every cell) takes no probe list");
        if (n_cells > 0x7fffffffLL) return fail(ctx, DEX_ERR_ARG, "grid too large for an all-cell solve");
        n_probe = (int)n_cells;
    } else if (n_probe > 0 && !probes) {
        return fail(ctx, DEX_ERR_ARG, "probe list required for n_probe > 0");
    }
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    dex::DenseParams P{};
    P.exclude_own = ctx->own_cell ? 0 : 1;
    if (int r = fill_quadrature(ctx, n_dir, dirs, weights, P.quad)) return r;
    if (n_lambda == 0 || n_probe == 0) return ok(ctx);
    if (!planes || !J) return fail(ctx, DEX_ERR_ARG, "planes and J are required");
    if (!aligned(planes, rec_align(W, DEX_STORE_F32)))
        return fail(ctx, DEX_ERR_ARG, "planes must be %zu-byte aligned", rec_align(W, DEX_STORE_F32));
    P.nx = nx;
    P.nz = nz;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.n_cells = n_cells;
    P.planes = planes;
    P.n_probe = n_probe;
    P.probes = probes;
    P.i_bc = i_bc;
    P.J = J;
    P.I = I;
    P.seg_count = seg_count;
    P.status = ctx->status;
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_solve_dense(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve_dense launch");
    return ok(ctx);
}

int dex_synth_static_line(dex_ctx* ctx, int n_cells, int n_lambda, const float* chi_c, const float* s_c,
                          const float* s_l, const float* ratio, const float* dld, const float* dlam, float* eta,
                          float* chi)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n_cells < 0 || n_lambda < 0) return fail(ctx, DEX_ERR_ARG, "negative size");
    if (n_cells == 0 || n_lambda == 0) return ok(ctx);
    if (!chi_c || !s_c || !s_l || !ratio || !dld || !dlam || !eta || !chi)
        return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_synth_static_line(ctx->stream, n_cells, n_lambda, chi_c, s_c, s_l, ratio, dld,
                                                  dlam, eta, chi);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "synth_static_line launch");
    return ok(ctx);
}

static int check_sparse_grid(dex_ctx* ctx, int nx, int nz)
{
    if (nx < DEX_BLOCK || nz < DEX_BLOCK || nx % DEX_BLOCK || nz % DEX_BLOCK)
        return fail(ctx, DEX_ERR_ARG, "sparse grids need nx, nz positive multiples of %d, got %d x %d", DEX_BLOCK,
                    nx, nz);
    const long long nb = (long long)(nx / DEX_BLOCK) * (nz / DEX_BLOCK);
    if (nb > (long long)DEX_STATES_PER_WORD * 24576 || nx > 65536 || nz > 65536)
        return fail(ctx, DEX_ERR_ARG, "sparse grid too large (%lld blocks)", nb);
    return DEX_OK;
}

size_t dex_state_words(int nx, int nz)
{
    if (nx < DEX_BLOCK || nz < DEX_BLOCK) return 0;
    const size_t nb = (size_t)(nx / DEX_BLOCK) * (size_t)(nz / DEX_BLOCK);
    return (nb + DEX_STATES_PER_WORD - 1) / DEX_STATES_PER_WORD;
}

int dex_chain_voxels(int max_mip)
{
    if (max_mip < 0 || max_mip > 4) return 0;
    return dex::chain_length(max_mip);
}

static bool valid_storage(int W, int storage)
{
    return storage == DEX_STORE_F32 || ((storage == DEX_STORE_BF16 || storage == DEX_STORE_F16) && (W == 4 || W == 8));
}

size_t dex_brick_floats(int capacity, int n_lambda, int W, int max_mip, int storage)
{
    if (capacity < 0 || n_lambda < 0 || !valid_W(W) || max_mip < 0 || max_mip > 4 || !valid_storage(W, storage))
        return 0;
    const size_t n_batch = (size_t)((n_lambda + W - 1) / W);
    return n_batch * (size_t)capacity * (size_t)dex::chain_length(max_mip) * (size_t)dex::record_floats(W, storage);
}

int dex_grid_build(dex_ctx* ctx, int nx, int nz, int n_lambda, const float* eta, const float* chi,
                   int* block_offset, int* active, int* n_active)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (!eta || !chi || !block_offset || !active || !n_active) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_grid_build(ctx->stream, nx, nz, n_lambda, eta, chi, block_offset, active, n_active);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "grid_build launch");
    return ok(ctx);
}

int dex_mips_build(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, const float* eta, const float* chi,
                   const int* active, const int* n_active, int capacity, const dex_vlm_params* params,
                   const signed char* level_cap, float* bricks, unsigned long long* state_words)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (!params) return fail(ctx, DEX_ERR_ARG, "params required");
    if (params->max_mip < 0 || params->max_mip > 4)
        return fail(ctx, DEX_ERR_ARG, "max_mip must be in [0, 4], got %d", params->max_mip);
    if (std::isnan(params->iod_eta) || std::isnan(params->iod_chi) || std::isnan(params->chi_ds_min))
        return fail(ctx, DEX_ERR_ARG, "NaN threshold");
    if (!valid_storage(W, params->storage))
        return fail(ctx, DEX_ERR_ARG, "storage %d not available for W = %d (bfloat16/float16 need W = 4 or 8)",
                    params->storage, W);
    const int nb = (nx / DEX_BLOCK) * (nz / DEX_BLOCK);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %d]", nb);
    if (!eta || !chi || !active || !n_active || !bricks || !state_words) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(bricks, rec_align(W, params->storage)))
        return fail(ctx, DEX_ERR_ARG, "bricks must be %zu-byte aligned", rec_align(W, params->storage));
    dex::MipParams P{};
    P.nx = nx;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK;
    P.nbz = nz / DEX_BLOCK;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.max_mip = params->max_mip;
    P.chain = dex::chain_length(params->max_mip);
    P.n_words = (int)dex_state_words(nx, nz);
    P.cap_active = capacity;
    P.storage = params->storage;
    P.log_mean = params->log_mean != 0;
    P.thr_eta = params->iod_eta;
    P.thr_chi = params->iod_chi;
    P.chi_ds_min = params->chi_ds_min;
    P.eta = eta;
    P.chi = chi;
    P.active = active;
    P.n_active = n_active;
    P.level_cap = level_cap;
    P.bricks = bricks;
    P.words = state_words;
    P.status = ctx->status;
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_mips_build(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mips_build launch");
    return ok(ctx);
}

static int solve_sparse(dex_ctx* ctx, int kind, int nx, int nz, int n_lambda, int W, int max_mip, int storage,
                        const float* bricks, const unsigned long long* state_words, const int* block_offset,
                        const int* active, const int* n_active, int capacity, int n_dir, const float* dirs,
                        const float* weights, int n_band, const float* band, float i_bc, float* J, float* I,
                        unsigned long long* seg_count)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (max_mip < 0 || max_mip > 4) return fail(ctx, DEX_ERR_ARG, "max_mip must be in [0, 4]");
    if (kind == 0 ? !valid_storage(W, storage) : storage != DEX_STORE_F32)
        return fail(ctx, DEX_ERR_ARG, "storage %d not available here", storage);
    const int nb = (nx / DEX_BLOCK) * (nz / DEX_BLOCK);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %d]", nb);
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    dex::HddaParams P{};
    P.storage = storage;
    P.n_band = -1;
    P.traversal = kind == 0 ? ctx->traversal : DEX_TRAVERSAL_PER_BATCH;
    P.pair_group = ctx->pair_group;
    P.exclude_own = ctx->own_cell ? 0 : 1;
    if (P.exclude_own && (kind != 0 || W != 8 || storage != DEX_STORE_F32))
        return fail(ctx, DEX_ERR_UNSUPPORTED,
                    "leaving out the own-cell emission needs the static solve with W = 8 and float32 bricks");
    if (band != nullptr && n_band >= 0) {
        if (n_band > 4) return fail(ctx, DEX_ERR_ARG, "at most 4 distance thresholds, got %d", n_band);
        for (int q = 0; q < n_band; ++q) {
            if (std::isnan(band[q]) || (q > 0 && band[q] < band[q - 1]))
                return fail(ctx, DEX_ERR_ARG, "distance thresholds must be non-decreasing numbers");
            P.band[q] = band[q];
        }
        P.n_band = n_band;
    }
    dex::pad_bands(P.n_band, P.band);
    if (int r = fill_quadrature(ctx, n_dir, dirs, weights, P.quad)) return r;
    if (!bricks || !state_words || !block_offset || !active || !n_active || !J)
        return fail(ctx, DEX_ERR_ARG, "null buffer");
    const size_t ral = kind == 0 ? rec_align(W, storage) : (W == 1 ? 8 : 16);
    if (!aligned(bricks, ral)) return fail(ctx, DEX_ERR_ARG, "bricks must be %zu-byte aligned", ral);
    P.nx = nx;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK;
    P.nbz = nz / DEX_BLOCK;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.chain = dex::chain_length(max_mip);
    P.n_words = (int)dex_state_words(nx, nz);
    P.cap_active = capacity;
    P.n_cells = (long long)nx * nz;
    P.bricks = bricks;
    P.words = state_words;
    P.block_offset = block_offset;
    P.active = active;
    P.n_active = n_active;
    P.i_bc = i_bc;
    P.J = J;
    P.I = I;
    P.seg_count = seg_count;
    P.status = ctx->status;
    if (kind == 0 && P.traversal == DEX_TRAVERSAL_PAIRED && !dex::solve_hdda_paired_applies(P))
        return fail(ctx, DEX_ERR_UNSUPPORTED, "the paired walk needs W = 8 and at most %d blocks",
                    dex::kPairInfoMaxBlocks);
    if (int r = bind(ctx)) return r;
    cudaError_t e = cudaMemsetAsync(J, 0, sizeof(float) * (size_t)n_lambda * (size_t)P.n_cells, ctx->stream);
    if (e == cudaSuccess && I)
        e = cudaMemsetAsync(I, 0, sizeof(float) * (size_t)n_lambda * (size_t)n_dir * (size_t)P.n_cells, ctx->stream);
    if (e == cudaSuccess)
        e = kind == 2 ? dex::launch_solve_velinterp(ctx->stream, P) : dex::launch_solve_hdda(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve_hdda launch");
    return ok(ctx);
}
int dex_formal_solve_hdda(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, int storage,
                          const float* bricks, const unsigned long long* state_words, const int* block_offset,
                          const int* active, const int* n_active, int capacity, int n_dir, const float* dirs,
                          const float* weights, int n_band, const float* band, float i_bc, float* J, float* I,
                          unsigned long long* seg_count)
{
    return solve_sparse(ctx, 0, nx, nz, n_lambda, W, max_mip, storage, bricks, state_words, block_offset, active, n_active,
                        capacity, n_dir, dirs, weights, n_band, band, i_bc, J, I, seg_count);
}

int dex_lte_populations(dex_ctx* ctx, const dex_atom* atom, int n_cells, const float* temperature, const float* nh,
                        double* pops)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::AtomParams* P = new (std::nothrow) dex::AtomParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    int r = fill_atom(ctx, atom, 0, nullptr, nullptr, *P);
    if (!r && n_cells < 0) r = fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!r && n_cells > 0 && (!temperature || !nh || !pops)) r = fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!r) r = bind(ctx);
    if (!r) {
        cudaError_t e = dex::launch_lte_pops(ctx->stream, *P, n_cells, temperature, nh, pops);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "lte_pops launch") : ok(ctx);
    }
    delete P;
    return r;
}

int dex_atom_eta_chi(dex_ctx* ctx, const dex_atom* atom, int n_cells, int n_lambda, const double* lambda_nm,
                     const int* line_tag, const float* temperature, const float* ne, const double* pops, float* eta,
                     float* chi)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::AtomParams* P = new (std::nothrow) dex::AtomParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    int r = fill_atom(ctx, atom, n_lambda, lambda_nm, line_tag, *P);
    if (!r && n_cells < 0) r = fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!r && n_cells > 0 && n_lambda > 0 && (!temperature || !ne || !pops || !eta || !chi))
        r = fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!r) r = bind(ctx);
    if (!r) {
        cudaError_t e = dex::launch_atom_eta_chi(ctx->stream, *P, n_cells, temperature, ne, pops, eta, chi);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "atom_eta_chi launch") : ok(ctx);
    }
    delete P;
    return r;
}

int dex_rates_accumulate(dex_ctx* ctx, const dex_atom* atom, int n_cells, int n_lambda, const double* lambda_nm,
                         const int* line_tag, const float* temperature, const float* J, double* jbar)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::AtomParams* P = new (std::nothrow) dex::AtomParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    int r = fill_atom(ctx, atom, n_lambda, lambda_nm, line_tag, *P);
    if (!r && n_cells < 0) r = fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!r && n_cells > 0 && (!temperature || !J || !jbar)) r = fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!r) r = bind(ctx);
    if (!r) {
        cudaError_t e = dex::launch_rates(ctx->stream, *P, n_cells, temperature, J, jbar);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "rates launch") : ok(ctx);
    }
    delete P;
    return r;
}

int dex_se_solve(dex_ctx* ctx, const dex_atom* atom, int n_cells, const float* temperature, const float* ne,
                 const float* nh, const double* jbar, double* pops)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::AtomParams* P = new (std::nothrow) dex::AtomParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    int r = fill_atom(ctx, atom, 0, nullptr, nullptr, *P);
    if (!r && n_cells < 0) r = fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!r && n_cells > 0 && (!temperature || !ne || !nh || !pops || (atom->n_line > 0 && !jbar)))
        r = fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!r) r = bind(ctx);
    if (!r) {
        cudaError_t e = dex::launch_se_solve(ctx->stream, *P, n_cells, temperature, ne, nh, jbar, nullptr, pops);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "se_solve launch") : ok(ctx);
    }
    delete P;
    return r;
}

int dex_mali_rates(dex_ctx* ctx, const dex_atom* atom, int n_cells, int n_lambda, const double* lambda_nm,
                   const int* line_tag, const float* temperature, const float* ne, const double* pops, const float* J,
                   int n_dir, const float* dirs, const float* weights, double* rho, double* jeff)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::AtomParams* P = new (std::nothrow) dex::AtomParams();
    dex::OwnCellOperator* O = new (std::nothrow) dex::OwnCellOperator();
    int r = (!P || !O) ? fail(ctx, DEX_ERR_ARG, "host allocation failed") : DEX_OK;
    if (!r) r = fill_atom(ctx, atom, n_lambda, lambda_nm, line_tag, *P);
    if (!r && n_cells < 0) r = fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!r && n_cells > 0 && atom->n_line > 0 && (!temperature || !ne || !pops || !J || !rho || !jeff))
        r = fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!r) {
        dex::Quadrature* q = new (std::nothrow) dex::Quadrature();
        if (!q) r = fail(ctx, DEX_ERR_ARG, "host allocation failed");
        else r = fill_quadrature(ctx, n_dir, dirs, weights, *q);
        if (!r) {
            // group the directions by their own-cell path l = 1 / (2 max(|dx|, |dz|))
            O->n = 0;
            for (int k = 0; k < n_dir; ++k) {
                const float ell = 0.5f / std::max(std::fabs(q->dx[k]), std::fabs(q->dz[k]));
                int g = 0;
                while (g < O->n && O->ell[g] != ell) ++g;
                if (g == O->n) {
                    O->ell[g] = ell;
                    O->w[g] = 0.0f;
                    ++O->n;
                }
                O->w[g] += q->w[k];
            }
        }
        delete q;
    }
    if (!r) r = bind(ctx);
    if (!r) {
        cudaError_t e = dex::launch_mali_rates(ctx->stream, *P, *O, n_cells, temperature, ne, pops, J, rho, jeff);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "mali_rates launch") : ok(ctx);
    }
    delete P;
    delete O;
    return r;
}

int dex_se_solve_preconditioned(dex_ctx* ctx, const dex_atom* atom, int n_cells, const float* temperature,
                                const float* ne, const float* nh, const double* rho, const double* jeff, double* pops)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::AtomParams* P = new (std::nothrow) dex::AtomParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    int r = fill_atom(ctx, atom, 0, nullptr, nullptr, *P);
    if (!r && n_cells < 0) r = fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!r && n_cells > 0 && (!temperature || !ne || !nh || !pops || (atom->n_line > 0 && (!rho || !jeff))))
        r = fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!r) r = bind(ctx);
    if (!r) {
        cudaError_t e = dex::launch_se_solve(ctx->stream, *P, n_cells, temperature, ne, nh, jeff, rho, pops);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "se_solve launch") : ok(ctx);
    }
    delete P;
    return r;
}

int dex_max_rel_change(dex_ctx* ctx, int n_level, int n_cells, const float* temperature, const double* old_pops,
                       const double* new_pops, double* out)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n_level < 1 || n_level > DEX_MAX_LEVELS) return fail(ctx, DEX_ERR_ARG, "n_level must be in [1, %d]", DEX_MAX_LEVELS);
    if (n_cells < 0) return fail(ctx, DEX_ERR_ARG, "negative n_cells");
    if (!out || (n_cells > 0 && (!temperature || !old_pops || !new_pops))) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(out, 8)) return fail(ctx, DEX_ERR_ARG, "out must be 8-byte aligned");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_max_rel_change(ctx->stream, n_level, n_cells, temperature, old_pops, new_pops, out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "max_rel_change launch");
    return ok(ctx);
}

int dex_voigt(dex_ctx* ctx, int n, const float* a, const float* x, float* h)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n < 0) return fail(ctx, DEX_ERR_ARG, "negative n");
    if (n == 0) return ok(ctx);
    if (!a || !x || !h) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_voigt(ctx->stream, n, a, x, h);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "voigt launch");
    return ok(ctx);
}

static int cav_fields(dex_ctx* ctx, const dex_cav_fields* f, dex::CavFields& F)
{
    if (!f) return fail(ctx, DEX_ERR_ARG, "fields required");
    if (!f->eta_star || !f->chi_star || !f->damping || !f->vth || !f->vx || !f->vz || !f->eta_c || !f->chi_c)
        return fail(ctx, DEX_ERR_ARG, "every CaV field pointer is required");
    F = dex::CavFields{f->eta_star, f->chi_star, f->damping, f->vth, f->vx, f->vz, f->eta_c, f->chi_c};
    return DEX_OK;
}

static int cav_lambda(dex_ctx* ctx, int n_lambda, const float* dv, float c_kms)
{
    if (n_lambda < 1 || n_lambda > DEX_MAX_CAV_LAMBDA)
        return fail(ctx, DEX_ERR_ARG, "n_lambda must be in [1, %d]", DEX_MAX_CAV_LAMBDA);
    if (!dv) return fail(ctx, DEX_ERR_ARG, "dv (host) required");
    if (!(c_kms > 0.0f) || !std::isfinite(c_kms)) return fail(ctx, DEX_ERR_ARG, "c_kms must be > 0");
    for (int l = 0; l < n_lambda; ++l)
        if (!std::isfinite(dv[l]) || !(1.0f + dv[l] / c_kms > 0.0f)) return fail(ctx, DEX_ERR_ARG, "bad dv[%d]", l);
    return DEX_OK;
}

int dex_cav_grid_build(dex_ctx* ctx, int nx, int nz, const dex_cav_fields* fields, int* block_offset, int* active,
                       int* n_active)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    dex::CavFields F;
    if (int r = cav_fields(ctx, fields, F)) return r;
    if (!block_offset || !active || !n_active) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_cav_grid_build(ctx->stream, nx, nz, F, block_offset, active, n_active);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cav_grid_build launch");
    return ok(ctx);
}

size_t dex_cav_brick_floats(int capacity, int max_mip)
{
    if (capacity < 0 || max_mip < 0 || max_mip > 4) return 0;
    return (size_t)capacity * (size_t)dex::chain_length(max_mip) * 8;
}

static int moving_mips_build(dex_ctx* ctx, bool velgrid, int nx, int nz, const dex_cav_fields* fields,
                             int n_lambda, int W, const float* dv, float c_kms, const int* active,
                             const int* n_active, int capacity, const dex_vlm_params* params,
                             const signed char* level_cap, float* bricks, unsigned long long* state_words)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (int r = cav_lambda(ctx, n_lambda, dv, c_kms)) return r;
    dex::CavMipParams P{};
    if (int r = cav_fields(ctx, fields, P.F)) return r;
    if (!params) return fail(ctx, DEX_ERR_ARG, "params required");
    if (params->max_mip < 0 || params->max_mip > 4) return fail(ctx, DEX_ERR_ARG, "max_mip must be in [0, 4]");
    if (std::isnan(params->iod_eta) || std::isnan(params->iod_chi) || std::isnan(params->chi_ds_min))
        return fail(ctx, DEX_ERR_ARG, "NaN threshold");
    const int nb = (nx / DEX_BLOCK) * (nz / DEX_BLOCK);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %d]", nb);
    if (!active || !n_active || !bricks || !state_words) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(bricks, 16)) return fail(ctx, DEX_ERR_ARG, "bricks must be 16-byte aligned");
    P.nx = nx;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK;
    P.nbz = nz / DEX_BLOCK;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.max_mip = params->max_mip;
    P.chain = dex::chain_length(params->max_mip);
    P.n_words = (int)dex_state_words(nx, nz);
    P.cap_active = capacity;
    P.thr_eta = params->iod_eta;
    P.thr_chi = params->iod_chi;
    P.chi_ds_min = params->chi_ds_min;
    if (params->n_test_dirs < 0 || params->n_test_dirs > dex::kMaxTestDirs)
        return fail(ctx, DEX_ERR_ARG, "n_test_dirs must be in [0, %d]", dex::kMaxTestDirs);
    P.n_test_dirs = params->n_test_dirs;
    for (int k = 0; k < P.n_test_dirs; ++k) {
        const double th = 2.0 * 3.14159265358979323846 * (double)k / (double)P.n_test_dirs;
        P.test_wx[k] = (float)std::cos(th);
        P.test_wz[k] = (float)std::sin(th);
    }
    P.active = active;
    P.n_active = n_active;
    P.level_cap = level_cap;
    P.bricks = bricks;
    P.words = state_words;
    P.status = ctx->status;
    dex::CavParams* M = new (std::nothrow) dex::CavParams();
    if (!M) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    dex::fill_cav_params(*M, n_lambda, W, dv, c_kms);
    int r = bind(ctx);
    if (!r) {
        cudaError_t e = velgrid ? dex::launch_vel_mips_build(ctx->stream, P, *M)
                                : dex::launch_cav_mips_build(ctx->stream, P, *M);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "mips build launch") : ok(ctx);
    }
    delete M;
    return r;
}

int dex_cav_mips_build(dex_ctx* ctx, int nx, int nz, const dex_cav_fields* fields, int n_lambda, int W,
                       const float* dv, float c_kms, const int* active, const int* n_active, int capacity,
                       const dex_vlm_params* params, const signed char* level_cap, float* bricks,
                       unsigned long long* state_words)
{
    return moving_mips_build(ctx, false, nx, nz, fields, n_lambda, W, dv, c_kms, active, n_active, capacity, params,
                             level_cap, bricks, state_words);
}

size_t dex_vel_brick_floats(int capacity, int n_lambda, int W, int max_mip)
{
    if (capacity < 0 || n_lambda < 0 || !valid_W(W) || max_mip < 0 || max_mip > 4) return 0;
    const size_t n_batch = (size_t)((n_lambda + W - 1) / W);
    return n_batch * (size_t)capacity * (size_t)dex::chain_length(max_mip) * (size_t)dex::vel_record_floats(W);
}

int dex_vel_mips_build(dex_ctx* ctx, int nx, int nz, const dex_cav_fields* fields, int n_lambda, int W,
                       const float* dv, float c_kms, const int* active, const int* n_active, int capacity,
                       const dex_vlm_params* params, const signed char* level_cap, float* bricks,
                       unsigned long long* state_words)
{
    return moving_mips_build(ctx, true, nx, nz, fields, n_lambda, W, dv, c_kms, active, n_active, capacity, params,
                             level_cap, bricks, state_words);
}

static int solve_cav(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* dv, float c_kms,
                     const float* bricks, const unsigned long long* state_words, const int* block_offset,
                     const int* active, const int* n_active, int capacity, int n_dir, const float* dirs,
                     const float* weights, int n_band, const float* band, float i_bc, float* J, float* I,
                     unsigned long long* seg_count, const float* mlp_params)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (int r = cav_lambda(ctx, n_lambda, dv, c_kms)) return r;
    if (max_mip < 0 || max_mip > 4) return fail(ctx, DEX_ERR_ARG, "max_mip must be in [0, 4]");
    const int nb = (nx / DEX_BLOCK) * (nz / DEX_BLOCK);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %d]", nb);
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    dex::HddaParams P{};
    if (int r = fill_quadrature(ctx, n_dir, dirs, weights, P.quad)) return r;
    P.n_band = -1;
    if (band != nullptr && n_band >= 0) {
        if (n_band > 4) return fail(ctx, DEX_ERR_ARG, "at most 4 distance thresholds, got %d", n_band);
        for (int q = 0; q < n_band; ++q) {
            if (std::isnan(band[q]) || (q > 0 && band[q] < band[q - 1]))
                return fail(ctx, DEX_ERR_ARG, "distance thresholds must be non-decreasing numbers");
            P.band[q] = band[q];
        }
        P.n_band = n_band;
    }
    dex::pad_bands(P.n_band, P.band);
    if (!bricks || !state_words || !block_offset || !active || !n_active || !J)
        return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(bricks, 16)) return fail(ctx, DEX_ERR_ARG, "bricks must be 16-byte aligned");
    P.nx = nx;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK;
    P.nbz = nz / DEX_BLOCK;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.chain = dex::chain_length(max_mip);
    P.n_words = (int)dex_state_words(nx, nz);
    P.cap_active = capacity;
    P.n_cells = (long long)nx * nz;
    P.bricks = bricks;
    P.words = state_words;
    P.block_offset = block_offset;
    P.active = active;
    P.n_active = n_active;
    P.i_bc = i_bc;
    P.J = J;
    P.I = I;
    P.seg_count = seg_count;
    P.status = ctx->status;
    dex::CavMlpParams* M = new (std::nothrow) dex::CavMlpParams();
    if (!M) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    dex::fill_cav_params(M->cav, n_lambda, W, dv, c_kms);
    if (mlp_params) {
        const int n = dex::mlp_param_count();
        for (int q = 0; q < n; ++q) {
            if (!std::isfinite(mlp_params[q])) {
                delete M;
                return fail(ctx, DEX_ERR_ARG, "network parameter %d not finite", q);
            }
            const bool weight = q < 192 || (q >= 256 && q < 4352) || (q >= 4416 && q < 4480);
            M->w[q] = weight ? bf16_round_host(mlp_params[q]) : mlp_params[q];
        }
    }
    int r = bind(ctx);
    if (!r) {
        cudaError_t e = cudaMemsetAsync(J, 0, sizeof(float) * (size_t)n_lambda * (size_t)P.n_cells, ctx->stream);
        if (e == cudaSuccess && I)
            e = cudaMemsetAsync(I, 0, sizeof(float) * (size_t)n_lambda * (size_t)n_dir * (size_t)P.n_cells,
                                ctx->stream);
        if (e == cudaSuccess)
            e = mlp_params ? dex::launch_solve_cav_mlp(ctx->stream, P, *M) : dex::launch_solve_cav(ctx->stream, P, M->cav);
        r = e != cudaSuccess ? cuda_fail(ctx, e, "solve_cav launch") : ok(ctx);
    }
    delete M;
    return r;
}

int dex_formal_solve_cav(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* dv,
                         float c_kms, const float* bricks, const unsigned long long* state_words,
                         const int* block_offset, const int* active, const int* n_active, int capacity, int n_dir,
                         const float* dirs, const float* weights, int n_band, const float* band, float i_bc,
                         float* J, float* I, unsigned long long* seg_count)
{
    return solve_cav(ctx, nx, nz, n_lambda, W, max_mip, dv, c_kms, bricks, state_words, block_offset, active,
                     n_active, capacity, n_dir, dirs, weights, n_band, band, i_bc, J, I, seg_count, nullptr);
}

int dex_formal_solve_cav_mlp(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* dv,
                             float c_kms, const float* bricks, const unsigned long long* state_words,
                             const int* block_offset, const int* active, const int* n_active, int capacity,
                             int n_dir, const float* dirs, const float* weights, int n_band, const float* band,
                             float i_bc, const float* mlp_params, float* J, float* I, unsigned long long* seg_count)
{
    if (!ctx) return DEX_ERR_ARG;
    if (!mlp_params) return fail(ctx, DEX_ERR_ARG, "null network parameters");
    return solve_cav(ctx, nx, nz, n_lambda, W, max_mip, dv, c_kms, bricks, state_words, block_offset, active,
                     n_active, capacity, n_dir, dirs, weights, n_band, band, i_bc, J, I, seg_count, mlp_params);
}

int dex_formal_solve_velinterp(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, const float* bricks,
                               const unsigned long long* state_words, const int* block_offset, const int* active,
                               const int* n_active, int capacity, int n_dir, const float* dirs, const float* weights,
                               int n_band, const float* band, float i_bc, float* J, float* I,
                               unsigned long long* seg_count)
{
    return solve_sparse(ctx, 2, nx, nz, n_lambda, W, max_mip, DEX_STORE_F32, bricks, state_words, block_offset, active, n_active,
                        capacity, n_dir, dirs, weights, n_band, band, i_bc, J, I, seg_count);
}

// Validate the batch descriptors and fill the launch parameters (no launch).
static int fill_batch(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, dex::BatchParams& P,
                      size_t& max_words, int parts = 1, size_t* max_blocks = nullptr)
{
    if (n_atm < 1 || n_atm > DEX_MAX_BATCH_ATM)
        return fail(ctx, DEX_ERR_ARG, "n_atm must be in [1, %d], got %d", DEX_MAX_BATCH_ATM, n_atm);
    if (!atms) return fail(ctx, DEX_ERR_ARG, "atms (host) required");
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    long long base = 0;
    max_words = 0;
    size_t blocks_max = 0;
    P.n_atm = n_atm;
    // the context's paired walk: work units are pairs of batches and lone batches
    P.paired = ctx->traversal == DEX_TRAVERSAL_PAIRED ? 1 : 0;
    P.pair_group = ctx->pair_group;
    if (P.paired && W != 8) return fail(ctx, DEX_ERR_UNSUPPORTED, "the paired walk needs W = 8");
    for (int a = 0; a < n_atm; ++a) {
        const dex_batch_item& it = atms[a];
        if (int r = check_sparse_grid(ctx, it.nx, it.nz)) return r;
        if (it.n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: n_lambda must be >= 1", a);
        if (it.max_mip < 0 || it.max_mip > 4) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: bad max_mip", a);
        const int nb = (it.nx / DEX_BLOCK) * (it.nz / DEX_BLOCK);
        if (it.capacity < 0 || it.capacity > nb) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: bad capacity", a);
        if (it.n_dir < 1 || it.n_dir > DEX_MAX_DIRS) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: bad n_dir", a);
        if (!it.bricks || !it.state_words || !it.block_offset || !it.active || !it.n_active || !it.dirs ||
            !it.weights || !it.J)
            return fail(ctx, DEX_ERR_ARG, "atmosphere %d: null buffer", a);
        if (!aligned(it.bricks, rec_align(W, DEX_STORE_F32)))
            return fail(ctx, DEX_ERR_ARG, "atmosphere %d: bricks must be %zu-byte aligned", a, rec_align(W, DEX_STORE_F32));
        if (it.n_band > 4) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: at most 4 distance thresholds", a);
        if (!std::isfinite(it.i_bc)) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: i_bc not finite", a);
        dex::AtmDesc& A = P.atm[a];
        A.nx = it.nx;
        A.nz = it.nz;
        A.nbx = it.nx / DEX_BLOCK;
        A.nbz = it.nz / DEX_BLOCK;
        A.n_lambda = it.n_lambda;
        A.chain = dex::chain_length(it.max_mip);
        A.n_words = (int)dex_state_words(it.nx, it.nz);
        A.cap_active = it.capacity;
        A.n_dir = it.n_dir;
        A.n_band = it.n_band < 0 ? -1 : it.n_band;
        for (int q = 0; q < 4; ++q) A.band[q] = it.band[q];
        for (int q = 1; q < (A.n_band > 0 ? A.n_band : 0); ++q)
            if (!(A.band[q] >= A.band[q - 1])) return fail(ctx, DEX_ERR_ARG, "atmosphere %d: bad thresholds", a);
        dex::pad_bands(A.n_band, A.band);
        A.i_bc = it.i_bc;
        A.item_base = base;
        A.bricks = it.bricks;
        A.words = it.state_words;
        A.block_offset = it.block_offset;
        A.active = it.active;
        A.n_active = it.n_active;
        A.dirs = it.dirs;
        A.weights = it.weights;
        A.J = it.J;
        base += (long long)dex::batch_units(P, (it.n_lambda + W - 1) / W) * it.capacity * parts;
        if ((size_t)A.n_words > max_words) max_words = (size_t)A.n_words;
        if ((size_t)nb > blocks_max) blocks_max = (size_t)nb;
    }
    if (max_blocks) *max_blocks = blocks_max;
    if (P.paired && blocks_max > (size_t)dex::kInfoMaxBlocks)
        return fail(ctx, DEX_ERR_UNSUPPORTED, "the paired walk needs grids of at most %d blocks", dex::kInfoMaxBlocks);
    if (base > 0xffffffffLL) return fail(ctx, DEX_ERR_ARG, "too many work items");
    P.n_items = base;
    P.parts = parts;
    P.chunk = 1;
    return DEX_OK;
}

// Zero every J, then launch the persistent solve with the given work counter.
static int batch_launch(dex_ctx* ctx, dex::BatchParams& P, const dex_batch_item* atms, int W, int ctas,
                        size_t max_words, unsigned int* queue, unsigned long long* done_ns,
                        unsigned long long* start_ns, int packet = 256, bool info = false, size_t max_blocks = 0,
                        bool occupancy = false)
{
    if (int r = own_cell_required(ctx, "the batched solve")) return r;
    P.queue = queue;
    P.done_ns = done_ns;
    P.start_ns = start_ns;
    P.status = ctx->status;
    if (ctas <= 0) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        ctas = 3 * (sms > 0 ? sms : 152);
    }
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < P.n_atm && e == cudaSuccess; ++a)
        e = cudaMemsetAsync(atms[a].J, 0, sizeof(float) * (size_t)atms[a].n_lambda * atms[a].nx * atms[a].nz,
                            ctx->stream);
    if (e == cudaSuccess && done_ns) e = cudaMemsetAsync(done_ns, 0, sizeof(unsigned long long) * P.n_atm, ctx->stream);
    if (e == cudaSuccess && start_ns) e = cudaMemsetAsync(start_ns, 0xff, sizeof(unsigned long long), ctx->stream);
    // the paired walk stages one word per block (max_blocks: the largest grid)
    const size_t smem = info || P.paired ? sizeof(int) * max_blocks : sizeof(unsigned long long) * max_words;
    if (e == cudaSuccess) e = dex::launch_batch_solve(ctx->stream, P, ctas, W, packet, info, occupancy, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch_solve launch");
    return ok(ctx);
}

int dex_batch_solve(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, int ctas, unsigned int* queue,
                    unsigned long long* done_ns, unsigned long long* start_ns)
{
    if (!ctx) return DEX_ERR_ARG;
    if (!queue) return fail(ctx, DEX_ERR_ARG, "queue (device scratch word) required");
    dex::BatchParams* P = new (std::nothrow) dex::BatchParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    size_t max_words = 0, max_blocks = 0;
    int r = fill_batch(ctx, n_atm, atms, W, *P, max_words, 1, &max_blocks);
    if (!r) r = bind(ctx);
    if (!r) r = batch_launch(ctx, *P, atms, W, ctas, max_words, queue, done_ns, start_ns, 256, false, max_blocks);
    delete P;
    return r;
}

int dex_batch_solve_config(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, const dex_batch_config* cfg,
                           unsigned int* queue, unsigned long long* done_ns, unsigned long long* start_ns)
{
    if (!ctx) return DEX_ERR_ARG;
    if (!cfg) return fail(ctx, DEX_ERR_ARG, "config required");
    if (!queue) return fail(ctx, DEX_ERR_ARG, "queue (device scratch word) required");
    if (cfg->packet != 256 && cfg->packet != 128 && cfg->packet != 64)
        return fail(ctx, DEX_ERR_ARG, "packet must be 256, 128 or 64 probes, got %d", cfg->packet);
    if (cfg->chunk < 1 || cfg->chunk > 64) return fail(ctx, DEX_ERR_ARG, "chunk must be in [1, 64], got %d", cfg->chunk);
    if (cfg->staging != 0 && cfg->staging != 1) return fail(ctx, DEX_ERR_ARG, "staging must be 0 or 1");
    if (cfg->occupancy != 0 && cfg->occupancy != 1) return fail(ctx, DEX_ERR_ARG, "occupancy must be 0 or 1");
    if (cfg->occupancy == 1 && W != 8) return fail(ctx, DEX_ERR_ARG, "the 64-register budget is built for W = 8");
    if (cfg->ctas < 0) return fail(ctx, DEX_ERR_ARG, "ctas must be >= 0");
    dex::BatchParams* P = new (std::nothrow) dex::BatchParams();
    if (!P) return fail(ctx, DEX_ERR_ARG, "host allocation failed");
    size_t max_words = 0, max_blocks = 0;
    int r = fill_batch(ctx, n_atm, atms, W, *P, max_words, 256 / cfg->packet, &max_blocks);
    if (!r && cfg->staging == 1 && max_blocks > (size_t)dex::kInfoMaxBlocks)
        r = fail(ctx, DEX_ERR_ARG, "one-word-per-block staging needs grids of at most %d blocks", dex::kInfoMaxBlocks);
    if (!r) {
        P->chunk = cfg->chunk;
        r = bind(ctx);
    }
    if (!r)
        r = batch_launch(ctx, *P, atms, W, cfg->ctas, max_words, queue, done_ns, start_ns, cfg->packet,
                         cfg->staging == 1, max_blocks, cfg->occupancy == 1);
    delete P;
    return r;
}

int dex_batch_solve_noalloc(dex_ctx* ctx, int n_atm, const dex_batch_item* atms, int W, int ctas,
                            unsigned long long* done_ns, unsigned long long* start_ns)
{
    if (!ctx) return DEX_ERR_ARG;
    dex::BatchParams P{};  // on the stack: this call makes no allocation at all
    size_t max_words = 0, max_blocks = 0;
    if (int r = fill_batch(ctx, n_atm, atms, W, P, max_words, 1, &max_blocks)) return r;
    if (int r = bind(ctx)) return r;
    unsigned int* scratch = nullptr;
    cudaError_t e = dex::noalloc_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "static scratch address");
    return batch_launch(ctx, P, atms, W, ctas, max_words, scratch, done_ns, start_ns, 256, false, max_blocks);
}

}  // extern "C"

// ------------------------------------------------------------------ MLP --
int dex_mlp_param_count(void) { return dex::mlp_param_count(); }

int dex_mlp_forward(dex_ctx* ctx, long long n, const float* xau, const float* params, float* out)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n < 0 || n > (1LL << 38)) return fail(ctx, DEX_ERR_ARG, "n must be in [0, 2^38]");
    if (n == 0) return ok(ctx);
    if (!xau || !params || !out) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    dex::MlpParams P{};
    P.n = n;
    P.xau = xau;
    P.params = params;
    P.out = out;
    P.status = ctx->status;
    cudaError_t e = dex::launch_mlp_forward(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp forward launch");
    return ok(ctx);
}

int dex_mlp_grad(dex_ctx* ctx, long long n, const float* xau, const float* target, const float* params,
                 float* grad, float* loss)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n < 0 || n > (1LL << 38)) return fail(ctx, DEX_ERR_ARG, "n must be in [0, 2^38]");
    if (!params || !grad || !loss || (n > 0 && (!xau || !target))) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    dex::MlpParams P{};
    P.n = n;
    P.xau = xau;
    P.target = target;
    P.params = params;
    P.grad = grad;
    P.loss = loss;
    P.status = ctx->status;
    cudaError_t e = dex::launch_mlp_grad(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp gradient launch");
    return ok(ctx);
}

int dex_mlp_adam(dex_ctx* ctx, float* params, const float* grad, float* m, float* v, int step, float lr,
                 float beta1, float beta2, float eps)
{
    if (!ctx) return DEX_ERR_ARG;
    if (!params || !grad || !m || !v) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return fail(ctx, DEX_ERR_ARG, "invalid Adam hyper-parameters");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_mlp_adam(ctx->stream, params, grad, m, v, step, lr, beta1, beta2, eps);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp adam launch");
    return ok(ctx);
}

int dex_mlp_targets(dex_ctx* ctx, long long n, const float* xau, float* out)
{
    if (!ctx) return DEX_ERR_ARG;
    if (n < 0 || n > (1LL << 38)) return fail(ctx, DEX_ERR_ARG, "n must be in [0, 2^38]");
    if (n == 0) return ok(ctx);
    if (!xau || !out) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_mlp_targets(ctx->stream, n, xau, out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mlp targets launch");
    return ok(ctx);
}

// ---------------------------------------------------------- measurement --
int dex_measure_ex2_rate(dex_ctx* ctx, double* ops_per_s)
{
    if (!ctx) return DEX_ERR_ARG;
    if (!ops_per_s) return fail(ctx, DEX_ERR_ARG, "null output");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::measure_ex2_rate(ctx->stream, ops_per_s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ex2 rate probe");
    return ok(ctx);
}

int dex_measure_fp32_rate(dex_ctx* ctx, double* ops_per_s)
{
    if (!ctx) return DEX_ERR_ARG;
    if (!ops_per_s) return fail(ctx, DEX_ERR_ARG, "null output");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::measure_fp32_rate(ctx->stream, ops_per_s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fp32 rate probe");
    return ok(ctx);
}

int dex_selftest_wait_timeout(dex_ctx* ctx, int polls)
{
    if (!ctx) return DEX_ERR_ARG;
    if (polls < 1 || polls > 1000000) return fail(ctx, DEX_ERR_ARG, "polls must be in [1, 1e6]");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_wait_timeout(ctx->stream, polls, ctx->status);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test launch");
    return ok(ctx);
}

// ------------------------------------------------------------------- 3D --
static int check_extent3(dex_ctx* ctx, int nx, int ny, int nz, bool blocks)
{
    if (nx < 1 || ny < 1 || nz < 1 || nx > 2048 || ny > 2048 || nz > 2048)
        return fail(ctx, DEX_ERR_ARG, "3D grid extents must be in [1, 2048], got %d x %d x %d", nx, ny, nz);
    if ((long long)nx * ny * nz > 0x7fffffffLL) return fail(ctx, DEX_ERR_ARG, "3D grid above 2^31 - 1 cells");
    if (blocks && (nx % DEX_BLOCK3 || ny % DEX_BLOCK3 || nz % DEX_BLOCK3))
        return fail(ctx, DEX_ERR_ARG, "sparse 3D grids need extents that are multiples of %d", DEX_BLOCK3);
    return DEX_OK;
}

static int fill_quadrature3(dex_ctx* ctx, int n_dir, const float* dirs, const float* weights, dex::Quadrature3& q)
{
    if (n_dir < 1 || n_dir > DEX_MAX_DIRS)
        return fail(ctx, DEX_ERR_ARG, "n_dir must be in [1, %d], got %d", DEX_MAX_DIRS, n_dir);
    if (!dirs || !weights) return fail(ctx, DEX_ERR_ARG, "dirs and weights (host arrays) are required");
    q.n_dir = n_dir;
    for (int k = 0; k < n_dir; ++k) {
        const float dx = dirs[3 * k], dy = dirs[3 * k + 1], dz = dirs[3 * k + 2];
        const float n2 = dx * dx + dy * dy + dz * dz;
        if (!std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz) || std::fabs(n2 - 1.0f) > 1e-4f)
            return fail(ctx, DEX_ERR_ARG, "direction %d is not a finite unit vector", k);
        if (!std::isfinite(weights[k])) return fail(ctx, DEX_ERR_ARG, "weight %d is not finite", k);
        q.dx[k] = dx;
        q.dy[k] = dy;
        q.dz[k] = dz;
        q.w[k] = weights[k];
    }
    return DEX_OK;
}

int dex_formal_solve_dense3(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, int W, const float* planes,
                            int n_dir, const float* dirs, const float* weights, int n_probe, const int* probes,
                            float i_bc, float* J, float* I, unsigned long long* seg_count)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = own_cell_required(ctx, "the 3D plain solve")) return r;
    if (int r = check_extent3(ctx, nx, ny, nz, false)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 0) return fail(ctx, DEX_ERR_ARG, "negative n_lambda");
    const long long n_cells = (long long)nx * ny * nz;
    if (n_probe < 0) {
        if (probes) return fail(ctx, DEX_ERR_ARG, "n_probe < 0 (every cell) takes no probe list");
        n_probe = (int)n_cells;
    } else if (n_probe > 0 && !probes) {
        return fail(ctx, DEX_ERR_ARG, "probe list required for n_probe > 0");
    }
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    dex::Dense3Params P{};
    if (int r = fill_quadrature3(ctx, n_dir, dirs, weights, P.quad)) return r;
    if (n_lambda == 0 || n_probe == 0) return ok(ctx);
    if (!planes || !J) return fail(ctx, DEX_ERR_ARG, "planes and J are required");
    if (!aligned(planes, rec_align(W, DEX_STORE_F32)))
        return fail(ctx, DEX_ERR_ARG, "planes must be %zu-byte aligned", rec_align(W, DEX_STORE_F32));
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.n_cells = n_cells;
    P.planes = planes;
    P.n_probe = n_probe;
    P.probes = probes;
    P.i_bc = i_bc;
    P.J = J;
    P.I = I;
    P.seg_count = seg_count;
    P.status = ctx->status;
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_solve_dense3(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve_dense3 launch");
    return ok(ctx);
}

size_t dex_state_words3(int nx, int ny, int nz)
{
    if (nx < DEX_BLOCK3 || ny < DEX_BLOCK3 || nz < DEX_BLOCK3) return 0;
    const size_t nb = (size_t)(nx / DEX_BLOCK3) * (size_t)(ny / DEX_BLOCK3) * (size_t)(nz / DEX_BLOCK3);
    return (nb + DEX_STATES_PER_WORD - 1) / DEX_STATES_PER_WORD;
}

int dex_chain_voxels3(int max_mip)
{
    if (max_mip < 0 || max_mip > 3) return 0;
    return dex::chain_length3(max_mip);
}

size_t dex_brick3_floats(int capacity, int n_lambda, int W, int max_mip, int storage)
{
    if (capacity < 0 || n_lambda < 0 || !valid_W(W) || max_mip < 0 || max_mip > 3 || !valid_storage(W, storage))
        return 0;
    const size_t n_batch = (size_t)((n_lambda + W - 1) / W);
    return n_batch * (size_t)capacity * (size_t)dex::chain_length3(max_mip) * (size_t)dex::record_floats(W, storage);
}

int dex_grid3_build(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, const float* eta, const float* chi,
                    int* block_offset, int* active, int* n_active)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_extent3(ctx, nx, ny, nz, true)) return r;
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (!eta || !chi || !block_offset || !active || !n_active) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_grid3_build(ctx->stream, nx, ny, nz, n_lambda, eta, chi, block_offset, active,
                                            n_active);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "grid3_build launch");
    return ok(ctx);
}

int dex_mips3_build(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, int W, const float* eta, const float* chi,
                    const int* active, const int* n_active, int capacity, const dex_vlm_params* params,
                    const signed char* level_cap, float* bricks, unsigned long long* state_words)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = check_extent3(ctx, nx, ny, nz, true)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (!params) return fail(ctx, DEX_ERR_ARG, "params required");
    if (params->max_mip < 0 || params->max_mip > 3)
        return fail(ctx, DEX_ERR_ARG, "3D max_mip must be in [0, 3], got %d", params->max_mip);
    if (std::isnan(params->iod_eta) || std::isnan(params->iod_chi) || std::isnan(params->chi_ds_min))
        return fail(ctx, DEX_ERR_ARG, "NaN threshold");
    if (!valid_storage(W, params->storage))
        return fail(ctx, DEX_ERR_ARG, "storage %d not available for W = %d", params->storage, W);
    const long long nb = (long long)(nx / DEX_BLOCK3) * (ny / DEX_BLOCK3) * (nz / DEX_BLOCK3);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %lld]", nb);
    if (!eta || !chi || !active || !n_active || !bricks || !state_words) return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(bricks, rec_align(W, params->storage)))
        return fail(ctx, DEX_ERR_ARG, "bricks must be %zu-byte aligned", rec_align(W, params->storage));
    dex::Mip3Params P{};
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK3;
    P.nby = ny / DEX_BLOCK3;
    P.nbz = nz / DEX_BLOCK3;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.max_mip = params->max_mip;
    P.chain = dex::chain_length3(params->max_mip);
    P.n_words = (int)dex_state_words3(nx, ny, nz);
    P.cap_active = capacity;
    P.storage = params->storage;
    P.log_mean = params->log_mean != 0;
    P.thr_eta = params->iod_eta;
    P.thr_chi = params->iod_chi;
    P.chi_ds_min = params->chi_ds_min;
    P.eta = eta;
    P.chi = chi;
    P.active = active;
    P.n_active = n_active;
    P.level_cap = level_cap;
    P.bricks = bricks;
    P.words = state_words;
    P.status = ctx->status;
    if (int r = bind(ctx)) return r;
    cudaError_t e = dex::launch_mips3_build(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mips3_build launch");
    return ok(ctx);
}

int dex_formal_solve_hdda3(dex_ctx* ctx, int nx, int ny, int nz, int n_lambda, int W, int max_mip, int storage,
                           const float* bricks, const unsigned long long* state_words, const int* block_offset,
                           const int* active, const int* n_active, int capacity, int n_dir, const float* dirs,
                           const float* weights, int n_band, const float* band, float i_bc, float* J, float* I,
                           unsigned long long* seg_count)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = own_cell_required(ctx, "the 3D accelerated solve")) return r;
    if (int r = check_extent3(ctx, nx, ny, nz, true)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (max_mip < 0 || max_mip > 3) return fail(ctx, DEX_ERR_ARG, "3D max_mip must be in [0, 3]");
    if (!valid_storage(W, storage)) return fail(ctx, DEX_ERR_ARG, "storage %d not available for W = %d", storage, W);
    const long long nb = (long long)(nx / DEX_BLOCK3) * (ny / DEX_BLOCK3) * (nz / DEX_BLOCK3);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %lld]", nb);
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    dex::Hdda3Params P{};
    P.storage = storage;
    P.traversal = ctx->traversal == DEX_TRAVERSAL_PAIRED ? DEX_TRAVERSAL_PAIRED : DEX_TRAVERSAL_PER_BATCH;
    P.pair_group = ctx->pair_group;
    P.n_band = -1;
    if (band != nullptr && n_band >= 0) {
        if (n_band > 4) return fail(ctx, DEX_ERR_ARG, "at most 4 distance thresholds, got %d", n_band);
        for (int q = 0; q < n_band; ++q) {
            if (std::isnan(band[q]) || (q > 0 && band[q] < band[q - 1]))
                return fail(ctx, DEX_ERR_ARG, "distance thresholds must be non-decreasing numbers");
            P.band[q] = band[q];
        }
        P.n_band = n_band;
    }
    if (int r = fill_quadrature3(ctx, n_dir, dirs, weights, P.quad)) return r;
    if (!bricks || !state_words || !block_offset || !active || !n_active || !J)
        return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(bricks, rec_align(W, storage)))
        return fail(ctx, DEX_ERR_ARG, "bricks must be %zu-byte aligned", rec_align(W, storage));
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK3;
    P.nby = ny / DEX_BLOCK3;
    P.nbz = nz / DEX_BLOCK3;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.max_mip = max_mip;
    P.chain = dex::chain_length3(max_mip);
    P.n_words = (int)dex_state_words3(nx, ny, nz);
    P.cap_active = capacity;
    P.n_cells = (long long)nx * ny * nz;
    P.bricks = bricks;
    P.words = state_words;
    P.block_offset = block_offset;
    P.active = active;
    P.n_active = n_active;
    P.i_bc = i_bc;
    P.J = J;
    P.I = I;
    P.seg_count = seg_count;
    P.status = ctx->status;
    if (P.traversal == DEX_TRAVERSAL_PAIRED && !dex::solve_hdda3_paired_applies(P))
        return fail(ctx, DEX_ERR_UNSUPPORTED, "the paired 3D walk needs W = 8 and at most 8192 state words");
    if (int r = bind(ctx)) return r;
    cudaError_t e = cudaMemsetAsync(J, 0, sizeof(float) * (size_t)n_lambda * (size_t)P.n_cells, ctx->stream);
    if (e == cudaSuccess && I)
        e = cudaMemsetAsync(I, 0, sizeof(float) * (size_t)n_lambda * (size_t)n_dir * (size_t)P.n_cells, ctx->stream);
    if (e == cudaSuccess) e = dex::launch_solve_hdda3(ctx->stream, P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve_hdda3 launch");
    return ok(ctx);
}

// ----------------------------------------------------- radiance cascades --
// cascades with at least this many directions order their threads directions
// first (measured on the 1024^2 workload: cascades 4 and 5 of the paper's six)
static constexpr int kRcDirFastestMin = 1024;
size_t dex_rc_workspace_floats(int nx, int nz, int n_lambda, int W, int n0)
{
    if (nx < 1 || nz < 1 || n_lambda < 0 || !valid_W(W) || n0 < 1) return 0;
    const size_t n_batch = (size_t)((n_lambda + W - 1) / W);
    return 2 * n_batch * (size_t)n0 * (size_t)nx * (size_t)nz * (size_t)W;
}

int dex_rc_solve(dex_ctx* ctx, int nx, int nz, int n_lambda, int W, int max_mip, int storage, const float* bricks,
                 const unsigned long long* state_words, const int* block_offset, int capacity, int n_cascades,
                 int n0, float t0, const int* level_cap, const float* dirs, float i_bc, float* workspace, float* J,
                 unsigned long long* seg_count)
{
    if (!ctx) return DEX_ERR_ARG;
    if (int r = own_cell_required(ctx, "the cascade solve")) return r;
    if (int r = check_sparse_grid(ctx, nx, nz)) return r;
    if (!valid_W(W)) return fail(ctx, DEX_ERR_ARG, "batch width W must be 1, 2, 4 or 8, got %d", W);
    if (n_lambda < 1) return fail(ctx, DEX_ERR_ARG, "n_lambda must be >= 1");
    if (max_mip < 0 || max_mip > 4) return fail(ctx, DEX_ERR_ARG, "max_mip must be in [0, 4]");
    if (!(storage == DEX_STORE_F32 || (W == 8 && (storage == DEX_STORE_BF16 || storage == DEX_STORE_F16))))
        return fail(ctx, DEX_ERR_ARG, "storage %d not available for W = %d", storage, W);
    if (n_cascades < 1 || n_cascades > 8) return fail(ctx, DEX_ERR_ARG, "n_cascades must be in [1, 8]");
    if (n0 < 1 || n0 > 64) return fail(ctx, DEX_ERR_ARG, "n0 must be in [1, 64]");
    const int top = 1 << (n_cascades - 1);
    if (nx % top || nz % top)
        return fail(ctx, DEX_ERR_ARG, "nx, nz must be multiples of 2^(n_cascades - 1) = %d", top);
    if ((long long)n0 * nx * nz > 0x7fffffffLL) return fail(ctx, DEX_ERR_ARG, "n0 * nx * nz above 2^31 - 1");
    if (!(t0 > 0.0f) || !std::isfinite(t0)) return fail(ctx, DEX_ERR_ARG, "t0 must be a positive number");
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    if (!level_cap) return fail(ctx, DEX_ERR_ARG, "level_cap (host) required");
    for (int i = 0; i < n_cascades; ++i)
        if (level_cap[i] < 0 || level_cap[i] > max_mip)
            return fail(ctx, DEX_ERR_ARG, "level_cap[%d] must be in [0, max_mip]", i);
    const int nb = (nx / DEX_BLOCK) * (nz / DEX_BLOCK);
    if (capacity < 0 || capacity > nb) return fail(ctx, DEX_ERR_ARG, "capacity must be in [0, %d]", nb);
    if (!bricks || !state_words || !block_offset || !dirs || !workspace || !J)
        return fail(ctx, DEX_ERR_ARG, "null buffer");
    if (!aligned(bricks, rec_align(W, storage)) || !aligned(workspace, 16))
        return fail(ctx, DEX_ERR_ARG, "misaligned buffer (bricks %zu-byte, workspace 16-byte)", rec_align(W, storage));
    dex::RcParams P{};
    P.nx = nx;
    P.nz = nz;
    P.nbx = nx / DEX_BLOCK;
    P.nbz = nz / DEX_BLOCK;
    P.n_lambda = n_lambda;
    P.W = W;
    P.n_batch = (n_lambda + W - 1) / W;
    P.chain = dex::chain_length(max_mip);
    P.n_words = (int)dex_state_words(nx, nz);
    P.cap_active = capacity;
    P.storage = storage;
    P.paired = ctx->traversal == DEX_TRAVERSAL_PAIRED && W == 8 ? 1 : 0;
    P.pair_group = ctx->pair_group;
    P.i_bc = i_bc;
    P.bricks = bricks;
    P.words = state_words;
    P.block_offset = block_offset;
    P.seg_count = seg_count;
    P.status = ctx->status;
    if (int r = bind(ctx)) return r;
    const size_t n_cells = (size_t)nx * nz;
    const size_t half = (size_t)P.n_batch * (size_t)n0 * n_cells * (size_t)W;
    cudaError_t e = cudaMemsetAsync(J, 0, sizeof(float) * (size_t)n_lambda * n_cells, ctx->stream);
    // direction offsets: cascade i starts at n0 (4^i - 1) / 3
    const float* upper = nullptr;
    float* out = nullptr;
    for (int i = n_cascades - 1; i >= 0 && e == cudaSuccess; --i) {
        const long long pow4 = 1LL << (2 * i);
        P.spacing = 1 << i;
        P.pnx = nx >> i;
        P.pnz = nz >> i;
        P.n_dir = (int)(n0 * pow4);
        P.level_cap = level_cap[i];
        // long intervals from few probes: a warp of neighbouring directions from one
        // probe reads neighbouring bricks; short ones keep lanes on neighbouring probes
        P.dir_fastest = P.n_dir >= kRcDirFastestMin ? 1 : 0;
        P.t_s = i == 0 ? 0.0f : t0 * (float)(pow4 / 4);
        P.t_e = t0 * (float)pow4;
        P.dirs = dirs + 2 * (size_t)(n0 * ((pow4 - 1) / 3));
        out = workspace + ((n_cascades - 1 - i) % 2 == 0 ? 0 : half);
        P.upper = upper;
        P.out = out;
        e = dex::launch_rc_cascade(ctx->stream, P);
        upper = out;
    }
    if (e == cudaSuccess) {
        P.n_dir = n0;
        e = dex::launch_rc_mean(ctx->stream, P, out, J);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rc_solve launch");
    return ok(ctx);
}
