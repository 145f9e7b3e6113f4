// Allocation-free Sigma solve: igr_solve_sigma_noalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// Sigma solve: code running inside another framework's memory budget,
// allocation-free real-time loops, or library hooks that may not call
// cudaMalloc or a caching allocator. For them this file keeps the solve's
// scratch (the IGR source b and the second Jacobi buffer) in one statically
// sized device array that the CUDA module provides when the library is
// loaded; the call itself allocates nothing.
//
// The array is a file-scope __device__ object. Host code cannot use its name
// as a device address (in host code the symbol is only a host-side stand-in),
// so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and caches it. The
// cached address belongs to the device's primary context: a cudaDeviceReset
// between calls (which tears that context down) is not supported.
#include <stdio.h>

#include <mutex>

#include "../../include/igr.h"
#include "igr_internal.h"

using namespace igr;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[IGR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_lock;
void *g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch per device
// message of the calling thread's last failed call
thread_local char g_noalloc_err[512] = "";

igr_status fail(igr_status s, const char *msg, cudaError_t e = cudaSuccess)
{
    if (e != cudaSuccess)
        snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s", msg);
    return s;
}

// device address of the scratch array on the current device (set up once)
igr_status scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(IGR_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(IGR_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(IGR_ERR_CUDA, "cudaGetSymbolAddress of the static scratch array", e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return IGR_OK;
}

}  // namespace

extern "C" {

size_t igr_noalloc_max_cells(igr_precision prec)
{
    const Ops *o = ops_for(prec);
    return o ? IGR_NOALLOC_SCRATCH_BYTES / (2 * (size_t)o->storage_bytes) : 0;
}

const char *igr_noalloc_last_error(void) { return g_noalloc_err; }

igr_status igr_solve_sigma_noalloc(const igr_config *cfg, const void *q, void *sigma_inout,
                                   int sweeps, void *cuda_stream)
{
    if (const char *why = validate_config(cfg)) return fail(IGR_ERR_INVALID_ARG, why);
    if (!q || !sigma_inout) return fail(IGR_ERR_INVALID_ARG, "q and sigma_inout are required");
    if (sweeps < 0) return fail(IGR_ERR_INVALID_ARG, "sweeps < 0");
    const int sb = ops_for(cfg->prec)->storage_bytes;
    if (!is_aligned(q, sb) || !is_aligned(sigma_inout, sb))
        return fail(IGR_ERR_INVALID_ARG, "q and sigma_inout must be aligned to their element size");
    for (int f = 0; f < 6; f++)
        if (cfg->bc[f] == IGR_BC_INFLOW)
            return fail(IGR_ERR_UNSUPPORTED, "the allocation-free solve takes periodic and outflow faces only");
    if (cfg->prec == IGR_F32_F16INC || cfg->prec == IGR_F32_BF16INC)
        return fail(IGR_ERR_UNSUPPORTED, "the allocation-free solve takes the modes that store q in one type");
    const Ops *o = ops_for(cfg->prec);
    Geom g;
    g.nx = cfg->nx;
    g.ny = cfg->ny;
    g.nz = cfg->nz;
    for (int f = 0; f < 6; f++) g.bc[f] = cfg->bc[f];
    g.plane = (long long)cfg->nx * cfg->ny;
    g.n = g.plane * cfg->nz;
    size_t need = 2 * (size_t)g.n * o->storage_bytes;
    if (need > IGR_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "grid of %lld cells needs %zu scratch bytes; the static array holds %zu "
                 "(at most %zu cells in this precision)",
                 g.n, need, (size_t)IGR_NOALLOC_SCRATCH_BYTES, igr_noalloc_max_cells(cfg->prec));
        return fail(IGR_ERR_INVALID_ARG, msg);
    }
    void *base = nullptr;
    igr_status s = scratch_address(&base);
    if (s != IGR_OK) return s;
    Phys p;
    p.dx = cfg->dx;
    p.gamma = cfg->gamma;
    p.alpha = cfg->alpha;
    p.cfl = cfg->cfl;
    p.order = cfg->order == 3 ? 3 : 5;
    p.mu = cfg->mu;
    p.zeta = cfg->zeta;
    Tiles t = default_tiles(g);
    if (!is_aligned(q, vec4_align(sb)) || !is_aligned(sigma_inout, vec4_align(sb)))
        t.vec_source = t.vec_jacobi = 0;  // the 1-cell forms: same bits, element alignment only
    Inflow none;
    none.W = nullptr;
    none.J = nullptr;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // scratch layout: b (n values), then the second Jacobi buffer (n values).
    // Both are fully written before they are read, so nothing needs clearing.
    void *b = base;
    void *other = (unsigned char *)base + (size_t)g.n * o->storage_bytes;
    cudaError_t e = o->source(g, p, t, none, q, nullptr, b, nullptr, st);
    if (e != cudaSuccess) return fail(IGR_ERR_CUDA, "source kernel launch", e);
    void *src = sigma_inout, *dst = other;
    if (cfg->sigma_solver == SOLVER_RBGS) {  // in place: red then black cells
        for (int it = 0; it < sweeps; it++)
            for (int colour = 0; colour < 2; colour++) {
                e = o->jacobi(g, p, t, q, b, sigma_inout, sigma_inout, colour, st);
                if (e != cudaSuccess) return fail(IGR_ERR_CUDA, "Gauss-Seidel kernel launch", e);
            }
    } else {
        for (int it = 0; it < sweeps; it++) {
            e = o->jacobi(g, p, t, q, b, src, dst, -1, st);
            if (e != cudaSuccess) return fail(IGR_ERR_CUDA, "Jacobi kernel launch", e);
            void *tmp = src;
            src = dst;
            dst = tmp;
        }
    }
    if (src != sigma_inout) {
        e = cudaMemcpyAsync(sigma_inout, src, (size_t)g.n * o->storage_bytes,
                            cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail(IGR_ERR_CUDA, "copy of the result", e);
    }
    return IGR_OK;
}

}  // extern "C"
