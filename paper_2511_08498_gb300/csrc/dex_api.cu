// C-ABI entry points of libdexgb: argument checks, context, launches.
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
    if (h) return fail(ctx, (int)h, "device reported: %s%s", (h & DEX_ERR_TRAVERSAL_CAP) ? "traversal cap " : "",
                       (h & DEX_ERR_NUMERIC) ? "numeric" : "");
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
    if (!aligned(planes, 8 * (W < 2 ? 1 : 2))) return fail(ctx, DEX_ERR_ARG, "planes must be 16-byte aligned");
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
    if (!probes) n_probe = (int)std::min<long long>(n_cells, 0x7fffffff);
    if (n_probe < 0) return fail(ctx, DEX_ERR_ARG, "negative n_probe");
    if (!std::isfinite(i_bc)) return fail(ctx, DEX_ERR_ARG, "i_bc not finite");
    dex::DenseParams P{};
    if (int r = fill_quadrature(ctx, n_dir, dirs, weights, P.quad)) return r;
    if (n_lambda == 0 || n_probe == 0) return ok(ctx);
    if (!planes || !J) return fail(ctx, DEX_ERR_ARG, "planes and J are required");
    if (!aligned(planes, W == 1 ? 8 : 16)) return fail(ctx, DEX_ERR_ARG, "planes misaligned");
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

}  // extern "C"
