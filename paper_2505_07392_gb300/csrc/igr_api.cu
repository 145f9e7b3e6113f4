// Host runtime of the IGR solver: the C ABI of include/igr.h.
//
// A context owns, in the storage type of its precision mode:
//   qA, qB, qC   three state buffers (5 n each). The RK stage reads its
//                input with a stencil, so it cannot write in place; stage 1
//                writes qB, stage 2 qC, stage 3 writes back into qA (the RK
//                base, read only at the same cell by the same thread).
//   sig[2]       Sigma ping-pong pair; Sigma persists across stages and steps
//                as the warm start of the Jacobi sweeps.
//   b            IGR source.
// In the increment modes qA is the FP32 state q^n, qB and qC hold the 16-bit
// increments d_1, d_2 of stages 1 and 2, stage 3 writes q^n+1 into a second
// FP32 buffer (qalt; the two alternate), and rho16 holds the stage density
// in the storage type for the sweeps.
// plus the -z inflow tables (arithmetic type), the per-block wave-speed
// maxima and a small block of device scalars (dt, t, speed, error flag).
// A time step never returns to the host: dt is reduced and applied on the
// device.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/igr.h"
#include "igr_internal.h"

using namespace igr;

// z-slabs of the last stage whose read-back overlaps the rest of the stage
constexpr int kOutSlabs = 8;

struct igr_ctx {
    igr_config cfg;
    std::vector<igr_jet> jets;
    Geom g;
    Phys p;
    Tiles tiles;
    const Ops *ops;
    igr_allocator alloc;
    bool own_alloc;
    cudaStream_t st;
    int device;
    void *q[3];         // q^n, q^1, q^2 (q[2] unused with host_rk_base); increment
                        // modes: q^n (FP32), d_1, d_2 (storage type)
    void *qalt;         // increment modes: the FP32 buffer stage 3 writes q^n+1 into
    void *rho16;        // increment modes: the stage density in the storage type
    bool inc;           // an increment mode
    void *hbase;        // host_rk_base: pinned host buffer of the RK base (5 n values)
    void *hbase_dev;    // its device-mapped address
    void *sig[2];
    void *b;
    void *W, *J;
    double *blockmax;
    long long blockmax_len;
    double *diag_part;  // per-block diagnostics partials (allocated by the first igr_diagnose)
    Scalars *sc;
    double *jets_dev;
    int cur;            // index of the current Sigma buffer
    int speed_nblocks;  // valid entries of blockmax for the current state (0: stale)
    int warn_flags;     // IGR_WARN_* seen at synchronising calls since the last igr_get_flags
    bool profiling;
    std::vector<cudaEvent_t> ev;  // start/stop pairs of the pending launches
    // igr_step_host: a stream for the read-back and an event per z-slab of
    // the last stage (created by its first call)
    cudaStream_t copy_st;
    cudaEvent_t slab_ev[kOutSlabs + 1];
    cudaEvent_t in_ev[2];  // igr_step_host: rho and m copied in (c->st), the energy field too (copy_st)
    std::vector<int> ev_class;
    long long prof_launches[KC_COUNT];
    double prof_ms[KC_COUNT];
    char err[512];
    // adjoint workspace (allocated by the first igr_adjoint_step)
    struct Adj {
        bool ready;
        void *qs[2];                       // stage-2/3 inputs (storage, 5 n)
        void *its;                         // Sigma iterates, 3 x (sweeps + 1) x n (storage)
        void *b;                           // source (storage, n)
        void *lq0, *lqs, *lout, *Lb;       // adjoints (arithmetic type, 5 n)
        void *lsig, *lb, *mu, *nl, *rb;    // adjoints (arithmetic type, n)
        void *lamJ;                        // adjoint of the inflow tables (5 x plane)
        double *gw;                        // jet gradient (njets)
        Scalars *sc;                       // dt of the recomputed stages
        std::vector<void *> all;
    } adj;
};

static char g_create_err[512] = "";

// smallest z-chunk (planes per block) a launch may use
static constexpr int kMinZChunk = 4;

static igr_status fail(igr_ctx *c, igr_status s, const char *fmt, ...)
{
    char *buf = c ? c->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return s;
}

#define CU(ctx, call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, IGR_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

// ------------------------------------------------------------ small kernels

// W[j][i] = sum_n s_n, J[v][j][i] = sum_n s_n q_jet_n[v],
// s_n = (1 - tanh((r_n - R_n) / (edge_n dx))) / 2 at the cell centre (x, y).
template <typename T>
__global__ void k_inflow_tables(int nx, int ny, double dx, double gamma, const double *jets,
                                int njets, T *W, T *J)
{
    long long plane = (long long)nx * ny;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < plane;
         f += (long long)gridDim.x * blockDim.x) {
        int i = (int)(f % nx), j = (int)(f / nx);
        double x = (i + 0.5) * dx, y = (j + 0.5) * dx;
        double w = 0.0, acc[5] = {0, 0, 0, 0, 0};
        for (int n = 0; n < njets; n++) {
            const double *jt = jets + 7 * n;
            double r = sqrt((x - jt[0]) * (x - jt[0]) + (y - jt[1]) * (y - jt[1]));
            double s = 0.5 * (1.0 - tanh((r - jt[2]) / (jt[6] * dx)));
            double rho = jt[3], vw = jt[4], p = jt[5];
            double qj[5] = {rho, 0.0, 0.0, rho * vw, p / (gamma - 1.0) + 0.5 * rho * vw * vw};
            w += s;
            for (int v = 0; v < 5; v++) acc[v] += s * qj[v];
        }
        W[f] = (T)w;
        for (int v = 0; v < 5; v++) J[v * plane + f] = (T)acc[v];
    }
}

__device__ __forceinline__ double load_any(const void *p, int dt, long long i)
{
    switch (dt) {
    case IGR_DT_F64: return ((const double *)p)[i];
    case IGR_DT_F32: return ((const float *)p)[i];
    case IGR_DT_F16: return __half2float(((const __half *)p)[i]);
    default: return __bfloat162float(((const __nv_bfloat16 *)p)[i]);
    }
}
__device__ __forceinline__ void store_any(void *p, int dt, long long i, double v)
{
    switch (dt) {
    case IGR_DT_F64: ((double *)p)[i] = v; break;
    case IGR_DT_F32: ((float *)p)[i] = (float)v; break;
    case IGR_DT_F16: ((__half *)p)[i] = __double2half(v); break;
    default: ((__nv_bfloat16 *)p)[i] = __double2bfloat16(v); break;
    }
}

// dst[i] = src[i] converted (round to nearest even), or 0 when src is NULL
__global__ void k_convert(const void *src, int sdt, void *dst, int ddt, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        store_any(dst, ddt, i, src ? load_any(src, sdt, i) : 0.0);
}

__device__ __forceinline__ double nanmax_d(double a, double b) { return (a > b || a != a) ? a : b; }

// dt from the per-block wave-speed maxima (or the fixed dt), t += dt
__device__ __forceinline__ void finalize_dt_body(const double *blockmax, int nblocks, Scalars *sc, double cfl_dx,
                                                 double fixed_dt);
__global__ void k_finalize_dt(const double *blockmax, int nblocks, Scalars *sc, double cfl_dx,
                              double fixed_dt)
{
    finalize_dt_body(blockmax, nblocks, sc, cfl_dx, fixed_dt);
}

// the same for several instances at once, one block each
struct DtInst {
    const double *blockmax;
    int nblocks;
    Scalars *sc;
    double cfl_dx;
};
struct DtGroup {
    int count;
    DtInst d[kGroupMax];
};
__global__ void k_finalize_dt_group(const __grid_constant__ DtGroup a)
{
    const DtInst &d = a.d[blockIdx.x];
    finalize_dt_body(d.blockmax, d.nblocks, d.sc, d.cfl_dx, 0.0);
}

__device__ __forceinline__ void finalize_dt_body(const double *blockmax, int nblocks, Scalars *sc, double cfl_dx,
                                                 double fixed_dt)
{
    __shared__ double red[32];
    double m = 0.0;
    if (fixed_dt <= 0.0)
        for (int t = threadIdx.x; t < nblocks; t += blockDim.x) m = nanmax_d(m, blockmax[t]);
    for (int o = 16; o > 0; o >>= 1) m = nanmax_d(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = nanmax_d(m, red[w]);
        double dt = fixed_dt > 0.0 ? fixed_dt : cfl_dx / m;
        if (fixed_dt <= 0.0) sc->speed = m;
        if (!(dt > 0.0) || isinf(dt)) sc->err |= ERRF_NONFINITE;
        sc->dt = dt;
        sc->t += dt;
    }
}

// ------------------------------------------------------------ helpers

// element type of Sigma, b and the increments
static int storage_dtype(igr_precision p)
{
    switch (p) {
    case IGR_F64: return IGR_DT_F64;
    case IGR_F32: return IGR_DT_F32;
    case IGR_F32_F16STORE: case IGR_F32_F16INC: return IGR_DT_F16;
    default: return IGR_DT_BF16;
    }
}
static bool is_inc(igr_precision p) { return p == IGR_F32_F16INC || p == IGR_F32_BF16INC; }
// element type of the state q
static int state_dtype(igr_precision p) { return is_inc(p) ? IGR_DT_F32 : storage_dtype(p); }
static size_t dtype_bytes(int dt) { return dt == IGR_DT_F64 ? 8 : dt == IGR_DT_F32 ? 4 : 2; }

const Ops *igr::ops_for(int p)
{
    switch (p) {
    case IGR_F64: return &ops_f64;
    case IGR_F32: return &ops_f32;
    case IGR_F32_F16STORE: return &ops_f16;
    case IGR_F32_BF16STORE: return &ops_bf16;
    case IGR_F32_F16INC: return &ops_f16inc;
    case IGR_F32_BF16INC: return &ops_bf16inc;
    }
    return nullptr;
}

// Longest z-chunk (at most 128 planes, at least 16) that still gives the
// kernel six waves of blocks on 152 SMs holding `resident` blocks each: every
// block starts by loading the planes below its chunk, so longer chunks
// amortise that prologue, while too few blocks leave SMs idle in the last
// wave. (tx, ty): columns per block.
static int default_zc(const Geom &g, int tx, int ty, int resident)
{
    long long cols = (long long)((g.nx + tx - 1) / tx) * ((g.ny + ty - 1) / ty);
    int zc = 128;
    while (zc > 16 && cols * ((g.nz + zc - 1) / zc) < 6LL * 152 * resident) zc /= 2;
    return zc > g.nz ? g.nz : zc;
}

Tiles igr::default_tiles(const Geom &g)
{
    Tiles t;
    t.vec_source = vec4_default_source(g.nx);
    t.vec_jacobi = vec4_default_jacobi(g.nx);
    t.zc_source = default_zc(g, t.vec_source ? 128 : 32, 8, 3);
    t.zc_jacobi = default_zc(g, t.vec_jacobi ? 128 : 32, 8, 3);
    t.zc_flux = default_zc(g, 32, 15, 1);
    t.z_begin = t.z_end = 0;
    return t;
}

const char *igr::validate_config(const igr_config *c)
{
    if (!c) return "cfg is NULL";
    if (c->nx < 4 || c->ny < 4 || c->nz < 4) return "nx, ny, nz must each be >= 4";
    if ((long long)c->nx * c->ny > (1ll << 31) - 1) return "nx*ny must fit in a 32-bit int";
    if ((long long)c->nx * c->ny * c->nz >= (1ll << 32)) return "the grid must have fewer than 2^32 cells";
    if (!(c->dx > 0) || !(c->gamma > 1) || !(c->alpha >= 0) || !(c->cfl > 0) || isinf(c->dx))
        return "need dx > 0, gamma > 1, alpha >= 0, cfl > 0";
    if (c->sweeps < 1) return "sweeps must be >= 1";
    if (c->prec < IGR_F64 || c->prec > IGR_F32_BF16INC) return "unknown precision mode";
    if (is_inc(c->prec) && c->host_rk_base) return "host_rk_base is not available in the increment modes";
    for (int f = 0; f < 6; f++)
        if (c->bc[f] < IGR_BC_PERIODIC || c->bc[f] > IGR_BC_INFLOW) return "unknown boundary condition";
    for (int a = 0; a < 3; a++)
        if ((c->bc[2 * a] == IGR_BC_PERIODIC) != (c->bc[2 * a + 1] == IGR_BC_PERIODIC))
            return "a periodic axis must be periodic on both faces";
    for (int f = 0; f < 6; f++)
        if (c->bc[f] == IGR_BC_INFLOW && f != 4) return "IGR_BC_INFLOW is supported on the -z face only";
    if (c->njets < 0 || (c->njets > 0 && !c->jets)) return "jets is NULL with njets > 0";
    if (c->host_rk_base != 0 && c->host_rk_base != 1) return "host_rk_base must be 0 or 1";
    if (c->order != 0 && c->order != 3 && c->order != 5) return "order must be 3 or 5 (0 means 5)";
    if (c->sigma_solver != SOLVER_JACOBI && c->sigma_solver != SOLVER_RBGS) return "unknown sigma_solver";
    if (!(c->mu >= 0.0) || !(c->zeta >= 0.0) || isinf(c->mu) || isinf(c->zeta))
        return "mu and zeta must be finite and >= 0";
    if (c->sigma_solver == SOLVER_RBGS) {
        const int len[3] = {c->nx, c->ny, c->nz};
        for (int a = 0; a < 3; a++)
            if (c->bc[2 * a] == IGR_BC_PERIODIC && len[a] % 2)
                return "red-black sweeps need an even number of cells along every periodic axis";
    }
    if (c->njets > 0 && c->bc[4] != IGR_BC_INFLOW) return "jets need an IGR_BC_INFLOW -z face";
    for (int n = 0; n < c->njets; n++) {
        const igr_jet &j = c->jets[n];
        if (!(j.rho > 0) || !(j.p > 0) || !(j.edge_width > 0) || !(j.radius >= 0))
            return "jet needs rho > 0, p > 0, edge_width > 0, radius >= 0";
    }
    return nullptr;
}

struct Layout {
    size_t state, incr, sig, b, W, J, blockmax, scalars, jets;
};

static Layout layout_of(const igr_config *c)
{
    Geom g;
    g.nx = c->nx; g.ny = c->ny; g.nz = c->nz;
    g.plane = (long long)c->nx * c->ny;
    g.n = g.plane * c->nz;
    const Ops *o = ops_for(c->prec);
    Tiles t = default_tiles(g);
    Layout L;
    L.state = (size_t)5 * g.n * o->state_bytes;
    L.incr = (size_t)5 * g.n * o->storage_bytes;  // a stage increment (increment modes)
    L.sig = (size_t)g.n * o->storage_bytes;
    L.b = L.sig;
    L.W = (size_t)g.plane * o->compute_bytes;
    L.J = 5 * L.W;
    t.zc_flux = kMinZChunk;  // the tuner may pick chunks down to kMinZChunk planes
    long long fb = o->flux_blocks(g, t);
    L.blockmax = (size_t)(fb > 4096 ? fb : 4096) * sizeof(double);
    L.scalars = 2 * sizeof(Scalars);  // [0] stepping, [1] igr_get_dt
    L.jets = (size_t)(c->njets > 0 ? c->njets : 1) * 7 * sizeof(double);
    return L;
}

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

static void *default_alloc(size_t bytes, void *)
{
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}
static void default_free(void *p, void *) { cudaFree(p); }

static igr_status ctx_alloc(igr_ctx *c, void **out, size_t bytes)
{
    *out = c->alloc.alloc(round256(bytes), c->alloc.user);
    if (!*out) return fail(c, IGR_ERR_OOM, "device allocation of %zu bytes failed", bytes);
    return IGR_OK;
}

// ------------------------------------------------------------ profiling

// Every launch is also an NVTX range named for its kernel class (for a
// timeline tool; without one attached a range costs a pointer test).
static const char *const kClassRange[KC_COUNT] = {"igr.source", "igr.jacobi", "igr.flux", "igr.other"};

static void prof_begin(igr_ctx *c, int cls)
{
    nvtxRangePushA(kClassRange[cls]);
    if (!c->profiling) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->st);
    c->ev.push_back(a);
    c->ev.push_back(b);
    c->ev_class.push_back(cls);
}
static void prof_end(igr_ctx *c)
{
    nvtxRangePop();
    if (!c->profiling) return;
    cudaEventRecord(c->ev.back(), c->st);
}
static void prof_collect(igr_ctx *c)
{
    for (size_t n = 0; n < c->ev_class.size(); n++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[2 * n], c->ev[2 * n + 1]);
        c->prof_ms[c->ev_class[n]] += ms;
        c->prof_launches[c->ev_class[n]] += 1;
        cudaEventDestroy(c->ev[2 * n]);
        cudaEventDestroy(c->ev[2 * n + 1]);
    }
    c->ev.clear();
    c->ev_class.clear();
}

// ------------------------------------------------------------ stage logic

static Inflow inflow_of(igr_ctx *c)
{
    Inflow in;
    in.W = c->W;
    in.J = c->J;
    return in;
}

// `sweeps` sweeps warm-started from s_first: Jacobi ping-pongs between
// s_first and s_other; red-black Gauss-Seidel updates s_first in place (two
// half-sweeps each). *result is the buffer holding the solution.
static igr_status launch_sweeps(igr_ctx *c, const Tiles &t, const void *q, const void *b,
                                void *s_first, void *s_other, int sweeps, void **result)
{
    if (c->cfg.sigma_solver == SOLVER_RBGS) {
        for (int it = 0; it < sweeps; it++)
            for (int colour = 0; colour < 2; colour++) {
                prof_begin(c, KC_JACOBI);
                CU(c, c->ops->jacobi(c->g, c->p, t, q, b, s_first, s_first, colour, c->st));
                prof_end(c);
            }
        *result = s_first;
        return IGR_OK;
    }
    void *src = s_first, *dst = s_other;
    for (int it = 0; it < sweeps; it++) {
        prof_begin(c, KC_JACOBI);
        CU(c, c->ops->jacobi(c->g, c->p, t, q, b, src, dst, -1, c->st));
        prof_end(c);
        void *t = src;
        src = dst;
        dst = t;
    }
    *result = src;
    return IGR_OK;
}

static igr_status refresh_speed(igr_ctx *c);
static igr_status finalize_dt(igr_ctx *c, double fixed_dt);

// One stage: source, sweeps, flux. With host_out (the last stage of
// igr_step_host) the flux runs in z-slabs of whole chunks, and each slab's
// planes of `out` are copied to host_out on copy_st as soon as the slab is
// done, while the next slabs compute; c->st then waits for the copies.
// qd: the stage's increments (increment modes, stages 2 and 3), else NULL.
// With q_ready (stage 1 of igr_step_host) the energy field of qs may still
// be arriving: the source and the sweeps read only rho and m, so they run
// first; then c->st waits for q_ready and the step's dt is formed from the
// whole state just before the flux, its first reader.
static igr_status run_stage(igr_ctx *c, int mode, const void *qs, const void *qd, const void *qn, void *out,
                            void *base_out = nullptr, void *host_out = nullptr, cudaEvent_t q_ready = nullptr)
{
    prof_begin(c, KC_SOURCE);
    CU(c, c->ops->source(c->g, c->p, c->tiles, inflow_of(c), qs, qd, c->b, c->rho16, c->st));
    prof_end(c);
    void *res;
    // the sweeps read the density as field 0 of their q: the state itself, or
    // the stage density the source kernel stored (increment modes)
    const void *qj = c->inc ? c->rho16 : qs;
    igr_status s = launch_sweeps(c, c->tiles, qj, c->b, c->sig[c->cur], c->sig[1 - c->cur], c->cfg.sweeps, &res);
    if (s != IGR_OK) return s;
    c->cur = res == c->sig[0] ? 0 : 1;
    if (q_ready) {
        CU(c, cudaStreamWaitEvent(c->st, q_ready, 0));
        s = refresh_speed(c);
        if (s == IGR_OK) s = finalize_dt(c, 0.0);
        if (s != IGR_OK) return s;
    }
    if (!host_out) {
        prof_begin(c, KC_FLUX);
        CU(c, c->ops->flux(c->g, c->p, c->tiles, inflow_of(c), mode, qs, qd, c->sig[c->cur], qn, out,
                           nullptr, base_out, c->sc, c->blockmax, &c->sc->err, c->st));
        prof_end(c);
        return IGR_OK;
    }
    const int zc = c->tiles.zc_flux, nchunk = (c->g.nz + zc - 1) / zc;
    const int per = (nchunk + kOutSlabs - 1) / kOutSlabs;  // chunks per slab
    const size_t sb = c->ops->state_bytes, plane = (size_t)c->g.plane;
    for (int c0 = 0, k = 0; c0 < nchunk; c0 += per, k++) {
        Tiles t = c->tiles;
        t.z_begin = c0 * zc;
        t.z_end = std::min(c->g.nz, (c0 + per) * zc);
        prof_begin(c, KC_FLUX);
        CU(c, c->ops->flux(c->g, c->p, t, inflow_of(c), mode, qs, qd, c->sig[c->cur], qn, out, nullptr,
                           base_out, c->sc, c->blockmax, &c->sc->err, c->st));
        prof_end(c);
        CU(c, cudaEventRecord(c->slab_ev[k], c->st));
        CU(c, cudaStreamWaitEvent(c->copy_st, c->slab_ev[k], 0));
        const size_t off = (size_t)t.z_begin * plane, len = (size_t)(t.z_end - t.z_begin) * plane;
        for (int u = 0; u < 5; u++) {
            const size_t at = ((size_t)u * c->g.n + off) * sb;
            CU(c, cudaMemcpyAsync((char *)host_out + at, (const char *)out + at, len * sb,
                                  cudaMemcpyDeviceToHost, c->copy_st));
        }
    }
    CU(c, cudaEventRecord(c->slab_ev[kOutSlabs], c->copy_st));
    CU(c, cudaStreamWaitEvent(c->st, c->slab_ev[kOutSlabs], 0));
    return IGR_OK;
}

static igr_status refresh_speed(igr_ctx *c)
{
    if (c->speed_nblocks > 0) return IGR_OK;
    int nb = 0;
    prof_begin(c, KC_OTHER);
    CU(c, c->ops->speed(c->g, c->p, c->q[0], c->blockmax, &nb, c->st));
    prof_end(c);
    c->speed_nblocks = nb;
    return IGR_OK;
}

static igr_status read_flags(igr_ctx *c)
{
    CU(c, cudaStreamSynchronize(c->st));
    if (c->profiling) prof_collect(c);
    int err = 0;
    CU(c, cudaMemcpy(&err, &c->sc->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        int zero = 0;
        CU(c, cudaMemcpy(&c->sc->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        c->warn_flags |= err & ERRF_FACE;
        if (err & ERRF_NONFINITE)
            return fail(c, IGR_ERR_NONFINITE, "a stage produced a non-finite value or time step");
    }
    return IGR_OK;
}

// ------------------------------------------------------------ the C ABI

extern "C" {

const char *igr_version(void) { return "igr-gb300 0.1 (sm_103a)"; }

const char *igr_last_error(const igr_ctx *ctx) { return ctx ? ctx->err : g_create_err; }

size_t igr_memory_bytes(const igr_config *cfg)
{
    if (validate_config(cfg)) return 0;
    Layout L = layout_of(cfg);
    if (is_inc(cfg->prec))  // two FP32 states, two increments, the stage density
        return 2 * round256(L.state) + 2 * round256(L.incr) + round256(L.b) +
               (cfg->sigma_solver == SOLVER_RBGS ? 1 : 2) * round256(L.sig) + round256(L.b) +
               round256(L.W) + round256(L.J) + round256(L.blockmax) + round256(L.scalars) + round256(L.jets);
    return (cfg->host_rk_base ? 2 : 3) * round256(L.state) +
           (cfg->sigma_solver == SOLVER_RBGS ? 1 : 2) * round256(L.sig) + round256(L.b) +
           round256(L.W) + round256(L.J) + round256(L.blockmax) + round256(L.scalars) + round256(L.jets);
}

igr_status igr_create(const igr_config *cfg, const igr_allocator *allocator, void *cuda_stream,
                      igr_ctx **out)
{
    if (!out) return fail(nullptr, IGR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (const char *why = validate_config(cfg)) return fail(nullptr, IGR_ERR_INVALID_ARG, "%s", why);
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(nullptr, IGR_ERR_INVALID_ARG, "allocator needs alloc and free");
    igr_ctx *c = new (std::nothrow) igr_ctx();
    if (!c) return fail(nullptr, IGR_ERR_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->jets.assign(cfg->jets, cfg->jets + cfg->njets);
    c->cfg.jets = c->jets.data();
    c->g.nx = cfg->nx;
    c->g.ny = cfg->ny;
    c->g.nz = cfg->nz;
    for (int f = 0; f < 6; f++) c->g.bc[f] = cfg->bc[f];
    c->g.plane = (long long)cfg->nx * cfg->ny;
    c->g.n = c->g.plane * cfg->nz;
    c->p.dx = cfg->dx;
    c->p.gamma = cfg->gamma;
    c->p.alpha = cfg->alpha;
    c->p.cfl = cfg->cfl;
    c->p.order = cfg->order == 3 ? 3 : 5;
    c->p.mu = cfg->mu;
    c->p.zeta = cfg->zeta;
    c->tiles = default_tiles(c->g);
    c->ops = ops_for(cfg->prec);
    if (allocator) {
        c->alloc = *allocator;
    } else {
        c->alloc.alloc = default_alloc;
        c->alloc.free = default_free;
        c->alloc.user = nullptr;
    }
    c->st = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);

    Layout L = layout_of(cfg);
    igr_status s = IGR_OK;
    c->inc = is_inc(cfg->prec);
    const int nstate = cfg->host_rk_base ? 2 : 3;
    for (int n = 0; n < nstate && s == IGR_OK; n++) s = ctx_alloc(c, &c->q[n], c->inc && n > 0 ? L.incr : L.state);
    if (s == IGR_OK && c->inc) s = ctx_alloc(c, &c->qalt, L.state);
    if (s == IGR_OK && c->inc) s = ctx_alloc(c, &c->rho16, L.b);
    if (s == IGR_OK && cfg->host_rk_base) {
        if (cudaHostAlloc(&c->hbase, L.state, cudaHostAllocMapped) != cudaSuccess) {
            c->hbase = nullptr;
            s = fail(c, IGR_ERR_OOM, "pinned host allocation of %zu bytes failed", L.state);
        } else if (cudaHostGetDevicePointer(&c->hbase_dev, c->hbase, 0) != cudaSuccess) {
            s = fail(c, IGR_ERR_UNSUPPORTED, "the device cannot map host memory");
        } else {
            memset(c->hbase, 0, L.state);
        }
    }
    const int nsig = cfg->sigma_solver == SOLVER_RBGS ? 1 : 2;  // red-black sweeps work in place
    for (int n = 0; n < nsig && s == IGR_OK; n++) s = ctx_alloc(c, &c->sig[n], L.sig);
    if (s == IGR_OK) s = ctx_alloc(c, &c->b, L.b);
    if (s == IGR_OK) s = ctx_alloc(c, &c->W, L.W);
    if (s == IGR_OK) s = ctx_alloc(c, &c->J, L.J);
    if (s == IGR_OK) s = ctx_alloc(c, (void **)&c->blockmax, L.blockmax);
    if (s == IGR_OK) s = ctx_alloc(c, (void **)&c->sc, L.scalars);
    if (s == IGR_OK) s = ctx_alloc(c, (void **)&c->jets_dev, L.jets);
    c->blockmax_len = (long long)(L.blockmax / sizeof(double));
    if (s != IGR_OK) {
        snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
        igr_destroy(c);
        return s;
    }
    // zero state, Sigma, scalars; build the inflow tables
    cudaError_t e = cudaSuccess;
    for (int n = 0; n < nstate && e == cudaSuccess; n++)
        e = cudaMemsetAsync(c->q[n], 0, c->inc && n > 0 ? L.incr : L.state, c->st);
    if (e == cudaSuccess && c->inc) e = cudaMemsetAsync(c->qalt, 0, L.state, c->st);
    if (e == cudaSuccess && c->inc) e = cudaMemsetAsync(c->rho16, 0, L.b, c->st);
    for (int n = 0; n < nsig && e == cudaSuccess; n++) e = cudaMemsetAsync(c->sig[n], 0, L.sig, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->b, 0, L.b, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sc, 0, L.scalars, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->W, 0, L.W, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->J, 0, L.J, c->st);
    if (e == cudaSuccess && cfg->njets > 0) {
        std::vector<double> jt(7 * cfg->njets);
        for (int n = 0; n < cfg->njets; n++) {
            const igr_jet &j = cfg->jets[n];
            double v[7] = {j.cx, j.cy, j.radius, j.rho, j.w, j.p, j.edge_width};
            memcpy(&jt[7 * n], v, sizeof v);
        }
        e = cudaMemcpy(c->jets_dev, jt.data(), jt.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            int blocks = (int)((c->g.plane + 255) / 256);
            if (blocks > 4096) blocks = 4096;
            if (c->ops->compute_bytes == 8)
                k_inflow_tables<double><<<blocks, 256, 0, c->st>>>(
                    cfg->nx, cfg->ny, cfg->dx, cfg->gamma, c->jets_dev, cfg->njets, (double *)c->W,
                    (double *)c->J);
            else
                k_inflow_tables<float><<<blocks, 256, 0, c->st>>>(
                    cfg->nx, cfg->ny, cfg->dx, cfg->gamma, c->jets_dev, cfg->njets, (float *)c->W,
                    (float *)c->J);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof g_create_err, "igr_create: %s", cudaGetErrorString(e));
        igr_destroy(c);
        return IGR_ERR_CUDA;
    }
    c->cur = 0;
    c->speed_nblocks = 0;
    *out = c;
    return IGR_OK;
}

igr_status igr_destroy(igr_ctx *c)
{
    if (!c) return IGR_OK;
    cudaStreamSynchronize(c->st);
    if (c->profiling) prof_collect(c);
    void *bufs[] = {c->q[0], c->q[1], c->q[2], c->qalt, c->rho16, c->sig[0], c->sig[1], c->b, c->W, c->J,
                    c->blockmax, c->sc, c->jets_dev, c->diag_part};
    for (void *p : bufs)
        if (p) c->alloc.free(p, c->alloc.user);
    for (void *p : c->adj.all)
        if (p) c->alloc.free(p, c->alloc.user);
    if (c->hbase) cudaFreeHost(c->hbase);
    if (c->copy_st) {
        cudaStreamSynchronize(c->copy_st);
        for (cudaEvent_t e : c->slab_ev) cudaEventDestroy(e);
        for (cudaEvent_t e : c->in_ev) cudaEventDestroy(e);
        cudaStreamDestroy(c->copy_st);
    }
    delete c;
    return IGR_OK;
}

// Copy count values from a caller buffer of type dt into a context buffer of
// type ddt (converted on the device when they differ). Host buffers must have
// the state's type; in the increment modes a host Sigma (FP32) is staged in
// the first increment buffer, which holds nothing between steps, and
// converted there.
static igr_status copy_in(igr_ctx *c, const void *src, void *dst, long long count, igr_dtype dt,
                          int on_device, int ddt)
{
    const size_t db = dtype_bytes(dt);
    if (on_device && !is_aligned(src, db))
        return fail(c, IGR_ERR_INVALID_ARG, "device buffer not aligned to its element size");
    if (!on_device && (int)dt != state_dtype(c->cfg.prec))
        return fail(c, IGR_ERR_UNSUPPORTED, "host buffers must use the state dtype (%d)",
                    state_dtype(c->cfg.prec));
    if ((int)dt == ddt) {
        CU(c, cudaMemcpyAsync(dst, src, count * db, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->st));
        return IGR_OK;
    }
    const void *from = src;
    if (!on_device) {  // increment modes only (dt = FP32, ddt = the storage type)
        CU(c, cudaMemcpyAsync(c->q[1], src, count * db, cudaMemcpyHostToDevice, c->st));
        from = c->q[1];
    }
    k_convert<<<2048, 256, 0, c->st>>>(from, dt, dst, ddt, count);
    CU(c, cudaGetLastError());
    return IGR_OK;
}

// Copy count values of type sdt from a context buffer into a caller buffer
// of type dt (the same rules as copy_in).
static igr_status copy_out(igr_ctx *c, const void *src, void *dst, long long count, igr_dtype dt,
                           int on_device, int sdt)
{
    const size_t db = dtype_bytes(dt);
    if (on_device && !is_aligned(dst, db))
        return fail(c, IGR_ERR_INVALID_ARG, "device buffer not aligned to its element size");
    if (!on_device && (int)dt != state_dtype(c->cfg.prec))
        return fail(c, IGR_ERR_UNSUPPORTED, "host buffers must use the state dtype (%d)",
                    state_dtype(c->cfg.prec));
    if ((int)dt == sdt) {
        CU(c, cudaMemcpyAsync(dst, src, count * db, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->st));
        return IGR_OK;
    }
    void *to = on_device ? dst : c->q[1];
    k_convert<<<2048, 256, 0, c->st>>>(src, sdt, to, dt, count);
    CU(c, cudaGetLastError());
    if (!on_device) CU(c, cudaMemcpyAsync(dst, to, count * db, cudaMemcpyDeviceToHost, c->st));
    return IGR_OK;
}

igr_status igr_set_state(igr_ctx *c, const void *q, const void *sigma, igr_dtype dtype, int on_device)
{
    if (!c || !q) return fail(c, IGR_ERR_INVALID_ARG, "ctx and q are required");
    if (dtype < IGR_DT_F64 || dtype > IGR_DT_BF16) return fail(c, IGR_ERR_INVALID_ARG, "bad dtype");
    igr_status s = copy_in(c, q, c->q[0], 5 * c->g.n, dtype, on_device, state_dtype(c->cfg.prec));
    if (s != IGR_OK) return s;
    c->cur = 0;
    if (sigma) {
        s = copy_in(c, sigma, c->sig[0], c->g.n, dtype, on_device, storage_dtype(c->cfg.prec));
        if (s != IGR_OK) return s;
    } else {
        CU(c, cudaMemsetAsync(c->sig[0], 0, c->g.n * dtype_bytes(storage_dtype(c->cfg.prec)), c->st));
    }
    c->speed_nblocks = 0;
    // a new trajectory: flags pending from the replaced state are dropped
    c->warn_flags = 0;
    CU(c, cudaMemsetAsync(&c->sc->err, 0, sizeof(int), c->st));
    if (!on_device) CU(c, cudaStreamSynchronize(c->st));
    return IGR_OK;
}

igr_status igr_set_conserved(igr_ctx *c, const void *q, igr_dtype dtype, int on_device)
{
    if (!c || !q) return fail(c, IGR_ERR_INVALID_ARG, "ctx and q are required");
    if (dtype < IGR_DT_F64 || dtype > IGR_DT_BF16) return fail(c, IGR_ERR_INVALID_ARG, "bad dtype");
    igr_status s = copy_in(c, q, c->q[0], 5 * c->g.n, dtype, on_device, state_dtype(c->cfg.prec));
    if (s != IGR_OK) return s;
    c->speed_nblocks = 0;  // dt from the new q
    c->warn_flags = 0;
    CU(c, cudaMemsetAsync(&c->sc->err, 0, sizeof(int), c->st));
    if (!on_device) CU(c, cudaStreamSynchronize(c->st));
    return IGR_OK;
}

igr_status igr_get_state(igr_ctx *c, void *q, void *sigma, igr_dtype dtype, int on_device)
{
    if (!c || !q) return fail(c, IGR_ERR_INVALID_ARG, "ctx and q are required");
    if (dtype < IGR_DT_F64 || dtype > IGR_DT_BF16) return fail(c, IGR_ERR_INVALID_ARG, "bad dtype");
    igr_status s = copy_out(c, c->q[0], q, 5 * c->g.n, dtype, on_device, state_dtype(c->cfg.prec));
    if (s == IGR_OK && sigma)
        s = copy_out(c, c->sig[c->cur], sigma, c->g.n, dtype, on_device, storage_dtype(c->cfg.prec));
    if (s != IGR_OK) return s;
    return read_flags(c);
}

}  // extern "C"

// One SSP-RK3 step; with host_out the final state is also copied there,
// overlapped with the last stage (see run_stage).
// dt of the step (the CFL rule on the wave-speed maxima of the current
// state, or fixed_dt > 0) into the device scalars
static igr_status finalize_dt(igr_ctx *c, double fixed_dt)
{
    prof_begin(c, KC_OTHER);
    k_finalize_dt<<<1, 1024, 0, c->st>>>(c->blockmax, c->speed_nblocks, c->sc, c->cfg.cfl * c->cfg.dx,
                                        fixed_dt);
    CU(c, cudaGetLastError());
    prof_end(c);
    return IGR_OK;
}

// One SSP-RK3 step. q_ready (igr_step_host): the energy field of q^n is
// still being copied in until that event; stage 1 forms dt after its sweeps.
static igr_status one_step(igr_ctx *c, double fixed_dt, void *host_out, cudaEvent_t q_ready = nullptr)
{
    igr_status s;
    if (!q_ready) {
        if (fixed_dt <= 0.0) {
            s = refresh_speed(c);
            if (s != IGR_OK) return s;
        }
        s = finalize_dt(c, fixed_dt);
        if (s != IGR_OK) return s;
    }
    if (c->hbase) {
        // RK base in host memory: stage 1 copies q^n there while it reads it,
        // stages 2 and 3 read it back; the two device buffers alternate
        s = run_stage(c, FLUX_STAGE1, c->q[0], nullptr, c->q[0], c->q[1], c->hbase_dev, nullptr, q_ready);
        if (s == IGR_OK) s = run_stage(c, FLUX_STAGE2, c->q[1], nullptr, c->hbase_dev, c->q[0]);
        if (s == IGR_OK) s = run_stage(c, FLUX_STAGE3, c->q[0], nullptr, c->hbase_dev, c->q[1], nullptr, host_out);
        std::swap(c->q[0], c->q[1]);
    } else if (c->inc) {
        // FP32 state q^n, 16-bit increments: stage s reads q^n + d_s
        s = run_stage(c, FLUX_STAGE1, c->q[0], nullptr, c->q[0], c->q[1], nullptr, nullptr, q_ready);
        if (s == IGR_OK) s = run_stage(c, FLUX_STAGE2, c->q[0], c->q[1], c->q[0], c->q[2]);
        if (s == IGR_OK) s = run_stage(c, FLUX_STAGE3, c->q[0], c->q[2], c->q[0], c->qalt, nullptr, host_out);
        std::swap(c->q[0], c->qalt);
    } else {
        s = run_stage(c, FLUX_STAGE1, c->q[0], nullptr, c->q[0], c->q[1], nullptr, nullptr, q_ready);
        if (s == IGR_OK) s = run_stage(c, FLUX_STAGE2, c->q[1], nullptr, c->q[0], c->q[2]);
        if (s == IGR_OK) s = run_stage(c, FLUX_STAGE3, c->q[2], nullptr, c->q[0], c->q[0], nullptr, host_out);
    }
    if (s != IGR_OK) return s;
    c->speed_nblocks = (int)c->ops->flux_blocks(c->g, c->tiles);
    return IGR_OK;
}

extern "C" {

igr_status igr_step(igr_ctx *c, int nsteps, double fixed_dt, double *t_inout)
{
    if (!c) return fail(c, IGR_ERR_INVALID_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(c, IGR_ERR_INVALID_ARG, "nsteps < 0");
    if (fixed_dt != fixed_dt) return fail(c, IGR_ERR_INVALID_ARG, "fixed_dt is NaN");
    double t0 = 0.0;
    if (t_inout) {
        CU(c, cudaMemcpyAsync(&t0, &c->sc->t, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CU(c, cudaStreamSynchronize(c->st));
    }
    for (int n = 0; n < nsteps; n++) {
        nvtxRangePushA("igr.step");
        igr_status s = one_step(c, fixed_dt, nullptr);
        nvtxRangePop();
        if (s != IGR_OK) return s;
    }
    if (t_inout) {
        double t1 = 0.0;
        CU(c, cudaMemcpyAsync(&t1, &c->sc->t, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        igr_status s = read_flags(c);
        *t_inout += t1 - t0;
        if (s != IGR_OK) return s;
    }
    return IGR_OK;
}

igr_status igr_step_host(igr_ctx *c, const void *q_in, void *q_out, int nsteps, igr_dtype dtype)
{
    if (!c || !q_in || !q_out) return fail(c, IGR_ERR_INVALID_ARG, "ctx, q_in and q_out are required");
    if (nsteps < 1) return fail(c, IGR_ERR_INVALID_ARG, "nsteps < 1");
    if ((int)dtype != state_dtype(c->cfg.prec))
        return fail(c, IGR_ERR_UNSUPPORTED, "host buffers must use the state dtype (%d)",
                    state_dtype(c->cfg.prec));
    if (!c->copy_st) {
        CU(c, cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->slab_ev) CU(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (cudaEvent_t &e : c->in_ev) CU(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    // q in (the host buffer has the state type); Sigma stays on the device
    // (as with igr_set_conserved). rho and m come first on c->st, then the
    // energy field on copy_st while stage 1's source and sweeps, which read
    // rho and m only, run; stage 1 waits for it before its dt and flux.
    const size_t sb = c->ops->state_bytes, nb = (size_t)c->g.n * sb;
    CU(c, cudaMemcpyAsync(c->q[0], q_in, 4 * nb, cudaMemcpyHostToDevice, c->st));
    CU(c, cudaEventRecord(c->in_ev[0], c->st));
    CU(c, cudaStreamWaitEvent(c->copy_st, c->in_ev[0], 0));
    CU(c, cudaMemcpyAsync((char *)c->q[0] + 4 * nb, (const char *)q_in + 4 * nb, nb, cudaMemcpyHostToDevice,
                          c->copy_st));
    CU(c, cudaEventRecord(c->in_ev[1], c->copy_st));
    c->speed_nblocks = 0;
    c->warn_flags = 0;
    CU(c, cudaMemsetAsync(&c->sc->err, 0, sizeof(int), c->st));
    igr_status s;
    for (int n = 0; n < nsteps; n++) {
        s = one_step(c, 0.0, n == nsteps - 1 ? q_out : nullptr, n == 0 ? c->in_ev[1] : nullptr);
        if (s != IGR_OK) return s;
    }
    return read_flags(c);  // synchronises the stream, which waits for the copies
}

igr_status igr_solve_sigma(igr_ctx *c, const void *q, void *sigma_inout, int sweeps, igr_dtype dtype)
{
    if (!c || !q || !sigma_inout) return fail(c, IGR_ERR_INVALID_ARG, "ctx, q, sigma are required");
    if (sweeps < 0) return fail(c, IGR_ERR_INVALID_ARG, "sweeps < 0");
    if ((int)dtype != storage_dtype(c->cfg.prec))
        return fail(c, IGR_ERR_UNSUPPORTED, "dtype must be the storage dtype");
    const size_t sb = c->ops->storage_bytes, qb = c->ops->state_bytes;
    if (!is_aligned(q, qb) || !is_aligned(sigma_inout, sb))
        return fail(c, IGR_ERR_INVALID_ARG, "q and sigma_inout must be aligned to their element size");
    Tiles t = c->tiles;
    if (!is_aligned(q, vec4_align((int)qb)) || !is_aligned(sigma_inout, vec4_align((int)sb)))
        t.vec_source = t.vec_jacobi = 0;  // the 1-cell forms: same bits, element alignment only
    prof_begin(c, KC_SOURCE);
    CU(c, c->ops->source(c->g, c->p, t, inflow_of(c), q, nullptr, c->b, c->rho16, c->st));
    prof_end(c);
    // the context's second Sigma buffer is scratch: sweeps alternate between
    // the caller's buffer and it, and an odd count copies the result back
    void *scratch = c->sig[1 - c->cur];
    void *res;
    igr_status s = launch_sweeps(c, t, c->inc ? c->rho16 : q, c->b, sigma_inout, scratch, sweeps, &res);
    if (s != IGR_OK) return s;
    if (res != sigma_inout)
        CU(c, cudaMemcpyAsync(sigma_inout, res, c->g.n * (size_t)c->ops->storage_bytes,
                              cudaMemcpyDeviceToDevice, c->st));
    return IGR_OK;
}

igr_status igr_rhs(igr_ctx *c, const void *q, const void *sigma, void *rhs, igr_dtype dtype)
{
    if (!c || !q || !sigma || !rhs) return fail(c, IGR_ERR_INVALID_ARG, "ctx, q, sigma, rhs are required");
    if ((int)dtype != storage_dtype(c->cfg.prec))
        return fail(c, IGR_ERR_UNSUPPORTED, "dtype must be the storage dtype");
    if (!is_aligned(q, c->ops->state_bytes) || !is_aligned(sigma, c->ops->storage_bytes) ||
        !is_aligned(rhs, c->ops->compute_bytes))
        return fail(c, IGR_ERR_INVALID_ARG, "q, sigma and rhs must be aligned to their element size");
    prof_begin(c, KC_FLUX);
    CU(c, c->ops->flux(c->g, c->p, c->tiles, inflow_of(c), FLUX_RHS, q, nullptr, sigma, nullptr, nullptr,
                       rhs, nullptr, c->sc, c->blockmax, &c->sc->err, c->st));
    prof_end(c);
    return IGR_OK;
}

igr_status igr_rk_combine(igr_ctx *c, const void *qn, const void *qs, const void *L, void *out,
                          long long count, int stage, double dt)
{
    if (!c || !qn || !qs || !L || !out) return fail(c, IGR_ERR_INVALID_ARG, "null buffer");
    if (count < 0 || stage < 1 || stage > 3) return fail(c, IGR_ERR_INVALID_ARG, "bad count or stage");
    if (!is_aligned(qn, c->ops->state_bytes) || !is_aligned(qs, c->ops->state_bytes) ||
        !is_aligned(out, c->ops->state_bytes) || !is_aligned(L, c->ops->compute_bytes))
        return fail(c, IGR_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    double w = stage == 1 ? 1.0 : stage == 2 ? 0.25 : 2.0 / 3.0;
    if (count == 0) return IGR_OK;
    prof_begin(c, KC_OTHER);
    CU(c, c->ops->rk_combine(qn, qs, L, out, count, dt, w, c->st));
    prof_end(c);
    return IGR_OK;
}

igr_status igr_get_dt(igr_ctx *c, double *dt)
{
    if (!c || !dt) return fail(c, IGR_ERR_INVALID_ARG, "ctx and dt are required");
    igr_status s = refresh_speed(c);
    if (s != IGR_OK) return s;
    // reduce into the second scalar slot so the step's scalars are untouched
    Scalars *tmp = c->sc + 1;
    CU(c, cudaMemsetAsync(tmp, 0, sizeof(Scalars), c->st));
    k_finalize_dt<<<1, 1024, 0, c->st>>>(c->blockmax, c->speed_nblocks, tmp, c->cfg.cfl * c->cfg.dx, 0.0);
    CU(c, cudaGetLastError());
    Scalars h;
    CU(c, cudaMemcpyAsync(&h, tmp, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
    CU(c, cudaStreamSynchronize(c->st));
    *dt = h.dt;
    return IGR_OK;
}

igr_status igr_sync(igr_ctx *c)
{
    if (!c) return fail(c, IGR_ERR_INVALID_ARG, "ctx is NULL");
    return read_flags(c);
}

igr_status igr_profile_enable(igr_ctx *c, int on)
{
    if (!c) return fail(c, IGR_ERR_INVALID_ARG, "ctx is NULL");
    CU(c, cudaStreamSynchronize(c->st));
    prof_collect(c);
    c->profiling = on != 0;
    for (int k = 0; k < KC_COUNT; k++) {
        c->prof_launches[k] = 0;
        c->prof_ms[k] = 0.0;
    }
    return IGR_OK;
}

igr_status igr_profile_read(igr_ctx *c, int kc, long long *launches, double *total_ms)
{
    if (!c || kc < 0 || kc >= KC_COUNT || !launches || !total_ms)
        return fail(c, IGR_ERR_INVALID_ARG, "bad profile query");
    CU(c, cudaStreamSynchronize(c->st));
    prof_collect(c);
    *launches = c->prof_launches[kc];
    *total_ms = c->prof_ms[kc];
    return IGR_OK;
}


// ------------------------------------------------------------ launch shapes

static int clamp_zc(int zc, int nz) { return zc < kMinZChunk ? kMinZChunk : (zc > nz ? nz : zc); }

igr_status igr_set_tiles(igr_ctx *c, int zc_source, int zc_jacobi, int zc_flux)
{
    if (!c || zc_source < 1 || zc_jacobi < 1 || zc_flux < 1)
        return fail(c, IGR_ERR_INVALID_ARG, "z-chunks must be >= 1");
    c->tiles.zc_source = clamp_zc(zc_source, c->g.nz);
    c->tiles.zc_jacobi = clamp_zc(zc_jacobi, c->g.nz);
    c->tiles.zc_flux = clamp_zc(zc_flux, c->g.nz);
    return IGR_OK;
}

igr_status igr_get_tiles(igr_ctx *c, int *zc_source, int *zc_jacobi, int *zc_flux)
{
    if (!c || !zc_source || !zc_jacobi || !zc_flux) return fail(c, IGR_ERR_INVALID_ARG, "null argument");
    *zc_source = c->tiles.zc_source;
    *zc_jacobi = c->tiles.zc_jacobi;
    *zc_flux = c->tiles.zc_flux;
    return IGR_OK;
}

igr_status igr_set_kernel_forms(igr_ctx *c, int source_vec4, int jacobi_vec4)
{
    if (!c) return fail(c, IGR_ERR_INVALID_ARG, "ctx is NULL");
    if (source_vec4 < -1 || source_vec4 > 1 || jacobi_vec4 < -1 || jacobi_vec4 > 1)
        return fail(c, IGR_ERR_INVALID_ARG, "forms are -1 (default), 0 (1 cell) or 1 (4 cells)");
    if ((source_vec4 == 1 || jacobi_vec4 == 1) && c->g.nx % 4)
        return fail(c, IGR_ERR_INVALID_ARG, "the 4-cell form needs nx %% 4 == 0 (nx = %d)", c->g.nx);
    c->tiles.vec_source = source_vec4 < 0 ? vec4_default_source(c->g.nx) : source_vec4;
    c->tiles.vec_jacobi = jacobi_vec4 < 0 ? vec4_default_jacobi(c->g.nx) : jacobi_vec4;
    return IGR_OK;
}

igr_status igr_get_kernel_forms(igr_ctx *c, int *source_vec4, int *jacobi_vec4)
{
    if (!c || !source_vec4 || !jacobi_vec4) return fail(c, IGR_ERR_INVALID_ARG, "null argument");
    *source_vec4 = c->tiles.vec_source;
    *jacobi_vec4 = c->tiles.vec_jacobi;
    return IGR_OK;
}

}  // extern "C"

// mean milliseconds of `reps` launches of fn() on the context stream
template <typename F> static igr_status time_launches(igr_ctx *c, int reps, F fn, float *ms)
{
    cudaEvent_t a, b;
    CU(c, cudaEventCreate(&a));
    CU(c, cudaEventCreate(&b));
    CU(c, fn());  // warm-up
    CU(c, cudaEventRecord(a, c->st));
    for (int r = 0; r < reps; r++) CU(c, fn());
    CU(c, cudaEventRecord(b, c->st));
    CU(c, cudaEventSynchronize(b));
    CU(c, cudaEventElapsedTime(ms, a, b));
    *ms /= reps;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return IGR_OK;
}

extern "C" {

igr_status igr_autotune(igr_ctx *c, int reps)
{
    if (!c || reps < 1) return fail(c, IGR_ERR_INVALID_ARG, "ctx and reps >= 1 are required");
    if (c->profiling) return fail(c, IGR_ERR_INVALID_ARG, "disable profiling before tuning");
    const int cand[] = {4, 8, 16, 32, 64, 128};
    Tiles best = c->tiles;
    float tbest[3] = {1e30f, 1e30f, 1e30f};
    void *sig = c->sig[c->cur], *scratch = c->sig[1 - c->cur];
    if (c->cfg.sigma_solver == SOLVER_RBGS)
        CU(c, cudaMemcpyAsync(c->q[1], sig, c->g.n * (size_t)c->ops->storage_bytes, cudaMemcpyDeviceToDevice,
                              c->st));
    const int nforms = c->g.nx % 4 == 0 ? 2 : 1;  // the 4-cell forms need rows of a multiple of 4
    for (int zc : cand) {
        if (zc > c->g.nz && zc != cand[0]) continue;
        Tiles t = c->tiles;
        t.zc_source = t.zc_jacobi = t.zc_flux = clamp_zc(zc, c->g.nz);
        float ms;
        igr_status s;
        // each kernel class writes only scratch: b, the other Sigma buffer, the stage-1 output
        for (int v = 0; v < nforms; v++) {
            t.vec_source = t.vec_jacobi = v;
            s = time_launches(c, reps, [&] {
                return c->ops->source(c->g, c->p, t, inflow_of(c), c->q[0], nullptr, c->b, c->rho16, c->st);
            }, &ms);
            if (s != IGR_OK) return s;
            if (ms < tbest[0]) { tbest[0] = ms; best.zc_source = t.zc_source; best.vec_source = v; }
            s = time_launches(c, reps, [&] {
                // red-black: a half-sweep in place on a copy of Sigma in the stage-1 output buffer
                const void *qj = c->inc ? c->rho16 : c->q[0];
                return c->cfg.sigma_solver == SOLVER_RBGS
                           ? c->ops->jacobi(c->g, c->p, t, qj, c->b, c->q[1], c->q[1], 0, c->st)
                           : c->ops->jacobi(c->g, c->p, t, qj, c->b, sig, scratch, -1, c->st);
            }, &ms);
            if (s != IGR_OK) return s;
            if (ms < tbest[1]) { tbest[1] = ms; best.zc_jacobi = t.zc_jacobi; best.vec_jacobi = v; }
        }
        s = time_launches(c, reps, [&] {
            return c->ops->flux(c->g, c->p, t, inflow_of(c), FLUX_STAGE1, c->q[0], nullptr, sig, c->q[0], c->q[1],
                                nullptr, nullptr, c->sc, c->blockmax, &c->sc->err, c->st);
        }, &ms);
        if (s != IGR_OK) return s;
        if (ms < tbest[2]) { tbest[2] = ms; best.zc_flux = t.zc_flux; }
    }
    c->tiles = best;
    return IGR_OK;
}

// ------------------------------------------------------------ batches

struct igr_batch {
    std::vector<igr_ctx *> inst;
    // instances largest first (cells; ties in the caller's order): the order
    // of their blocks in a grouped launch. The long-running blocks of the
    // large instances start first and the short ones of the small instances
    // fill the last waves (measured on 64 Taylor-Green instances of 48^3 to
    // 128^3: 4.55e9 -> 5.03e9 cell-updates/s in FP32, 4.33e9 -> 5.20e9 with
    // FP16 increments, against the caller's order)
    std::vector<int> order;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaStream_t user;  // the caller's stream (may be the legacy stream, which cannot be captured)
    cudaStream_t main;  // the batch's own stream, ordered after `user` at entry and before it at exit
    cudaEvent_t fork, enter, leave;
    struct Host {  // host-side stepping state of one instance
        int cur, speed_nblocks;
        Tiles tiles;
        void *q0;  // the current state buffer (the increment modes alternate two)
        bool operator==(const Host &o) const
        {
            return cur == o.cur && speed_nblocks == o.speed_nblocks && q0 == o.q0 &&
                   tiles.zc_source == o.tiles.zc_source &&
                   tiles.zc_jacobi == o.tiles.zc_jacobi && tiles.zc_flux == o.tiles.zc_flux &&
                   tiles.vec_source == o.tiles.vec_source && tiles.vec_jacobi == o.tiles.vec_jacobi;
        }
    };
    struct Graph {
        std::vector<Host> before, after;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    char err[512];
};

static igr_status bfail(igr_batch *b, igr_status s, const char *msg)
{
    snprintf(b->err, sizeof b->err, "%s", msg);
    return s;
}

static std::vector<igr_batch::Host> host_state(const igr_batch *b)
{
    std::vector<igr_batch::Host> h(b->inst.size());
    for (size_t i = 0; i < h.size(); i++)
        h[i] = {b->inst[i]->cur, b->inst[i]->speed_nblocks, b->inst[i]->tiles, b->inst[i]->q[0]};
    return h;
}

static void set_host_state(igr_batch *b, const std::vector<igr_batch::Host> &h)
{
    for (size_t i = 0; i < h.size(); i++) {
        igr_ctx *c = b->inst[i];
        c->cur = h[i].cur;
        c->speed_nblocks = h[i].speed_nblocks;
        if (c->inc && c->q[0] != h[i].q0) std::swap(c->q[0], c->qalt);
    }
}

// one step of every instance, each on its own stream, forked from and joined
// back into the batch's stream
static igr_status step_forkjoin(igr_batch *b)
{
    if (cudaEventRecord(b->fork, b->main) != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "fork record");
    for (size_t i = 0; i < b->inst.size(); i++) {
        if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "fork wait");
        igr_status s = igr_step(b->inst[i], 1, 0.0, nullptr);
        if (s != IGR_OK) return bfail(b, s, igr_last_error(b->inst[i]));
        if (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "join record");
        if (cudaStreamWaitEvent(b->main, b->join[i], 0) != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "join wait");
    }
    return IGR_OK;
}

// Inputs and output of stage `stage` of a context's step (see one_step).
struct StageIO {
    const void *qs, *qd, *qn;
    void *out;
};
static StageIO stage_io(const igr_ctx *c, int stage)
{
    if (c->inc) {
        if (stage == 1) return {c->q[0], nullptr, c->q[0], c->q[1]};
        if (stage == 2) return {c->q[0], c->q[1], c->q[0], c->q[2]};
        return {c->q[0], c->q[2], c->q[0], c->qalt};
    }
    if (stage == 1) return {c->q[0], nullptr, c->q[0], c->q[1]};
    if (stage == 2) return {c->q[1], nullptr, c->q[0], c->q[2]};
    return {c->q[2], nullptr, c->q[0], c->q[0]};
}

// One step of every instance with grouped launches: each kernel class runs
// as one launch over all instances' blocks (per precision and kernel form),
// instead of one launch per instance. Every instance keeps its own buffers,
// launch shape and CFL dt, and runs the same kernel bodies on the same data
// as a step of its own context, so the results are bitwise the same. Needs a
// valid wave-speed reduction in every instance (not the first step after a
// set_state).
static igr_status step_grouped(igr_batch *b)
{
    cudaStream_t st = b->main;
    const int n = (int)b->inst.size();
    // instances of one precision run together; batches are usually uniform
    std::vector<const Ops *> kinds;
    for (igr_ctx *c : b->inst)
        if (std::find(kinds.begin(), kinds.end(), c->ops) == kinds.end()) kinds.push_back(c->ops);
    // dt of every instance from the wave-speed maxima of its last stage
    for (int i0 = 0; i0 < n; i0 += kGroupMax) {
        DtGroup a;
        a.count = std::min(n - i0, (int)kGroupMax);
        for (int i = 0; i < a.count; i++) {
            igr_ctx *c = b->inst[i0 + i];
            a.d[i] = {c->blockmax, c->speed_nblocks, c->sc, c->cfg.cfl * c->cfg.dx};
        }
        k_finalize_dt_group<<<a.count, 1024, 0, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "grouped dt launch");
    }
    int maxs = 0;
    for (igr_ctx *c : b->inst) maxs = std::max(maxs, c->cfg.sweeps);
    std::vector<igr_ctx *> inst(n);
    for (int i = 0; i < n; i++) inst[i] = b->inst[b->order[i]];
    std::vector<SourceCall> sc;
    std::vector<JacobiCall> jc;
    std::vector<FluxCall> fc;
    for (int stage = 1; stage <= 3; stage++) {
        for (const Ops *o : kinds) {
            sc.clear();
            for (igr_ctx *c : inst)
                if (c->ops == o) {
                    const StageIO io = stage_io(c, stage);
                    sc.push_back({c->g, c->p, c->tiles, inflow_of(c), io.qs, io.qd, c->b, c->rho16});
                }
            if (o->source_group(sc.data(), (int)sc.size(), st) != cudaSuccess)
                return bfail(b, IGR_ERR_CUDA, "grouped source launch");
            // sweep k of every instance that makes at least k + 1 sweeps
            for (int k = 0; k < maxs; k++)
                for (int colour = -1; colour < 2; colour++) {
                    jc.clear();
                    for (igr_ctx *c : inst) {
                        const bool rb = c->cfg.sigma_solver == SOLVER_RBGS;
                        if (c->ops != o || k >= c->cfg.sweeps || (rb ? colour < 0 : colour >= 0)) continue;
                        const void *qj = c->inc ? c->rho16 : stage_io(c, stage).qs;
                        void *src = c->sig[c->cur], *dst = rb ? src : c->sig[1 - c->cur];
                        jc.push_back({c->g, c->p, c->tiles, qj, c->b, src, dst});
                    }
                    if (jc.empty()) continue;
                    if (o->jacobi_group(jc.data(), (int)jc.size(), colour, st) != cudaSuccess)
                        return bfail(b, IGR_ERR_CUDA, "grouped sweep launch");
                    for (igr_ctx *c : inst)  // Jacobi sweeps alternate the two Sigma buffers
                        if (c->ops == o && k < c->cfg.sweeps && c->cfg.sigma_solver != SOLVER_RBGS && colour < 0)
                            c->cur = 1 - c->cur;
                }
            fc.clear();
            for (igr_ctx *c : inst)
                if (c->ops == o) {
                    const StageIO io = stage_io(c, stage);
                    fc.push_back({c->g, c->p, c->tiles, inflow_of(c), io.qs, io.qd, c->sig[c->cur], io.qn, io.out,
                                  c->sc, c->blockmax, &c->sc->err});
                }
            if (o->flux_group(fc.data(), (int)fc.size(), stage, st) != cudaSuccess)
                return bfail(b, IGR_ERR_CUDA, "grouped flux launch");
        }
    }
    for (igr_ctx *c : inst) {
        if (c->inc) std::swap(c->q[0], c->qalt);
        c->speed_nblocks = (int)c->ops->flux_blocks(c->g, c->tiles);
    }
    return IGR_OK;
}

static igr_status step_batch_steps(igr_batch *b, int nsteps);

igr_status igr_create_batch(const igr_config *cfgs, int n, const igr_allocator *allocator,
                            void *cuda_stream, igr_batch **out)
{
    if (!out || !cfgs || n < 1) return fail(nullptr, IGR_ERR_INVALID_ARG, "cfgs, n >= 1 and out are required");
    *out = nullptr;
    for (int i = 0; i < n; i++)
        if (cfgs[i].host_rk_base)  // captured graphs hold fixed state pointers
            return fail(nullptr, IGR_ERR_UNSUPPORTED, "host_rk_base is not available in batches");
    igr_batch *b = new (std::nothrow) igr_batch();
    if (!b) return fail(nullptr, IGR_ERR_OOM, "host allocation failed");
    b->user = (cudaStream_t)cuda_stream;
    igr_status s = IGR_OK;
    if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->enter, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->leave, cudaEventDisableTiming) != cudaSuccess)
        s = fail(nullptr, IGR_ERR_CUDA, "stream/event creation failed");
    for (int i = 0; i < n && s == IGR_OK; i++) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            s = fail(nullptr, IGR_ERR_CUDA, "stream/event creation failed");
            break;
        }
        b->streams.push_back(st);
        b->join.push_back(ev);
        igr_ctx *c = nullptr;
        s = igr_create(&cfgs[i], allocator, st, &c);
        if (s == IGR_OK) b->inst.push_back(c);
    }
    if (s != IGR_OK) {
        char msg[512];
        snprintf(msg, sizeof msg, "%s", g_create_err);
        igr_destroy_batch(b);
        snprintf(g_create_err, sizeof g_create_err, "%s", msg);
        return s;
    }
    b->order.resize(n);
    for (int i = 0; i < n; i++) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->inst[x]->g.n > b->inst[y]->g.n; });
    *out = b;
    return IGR_OK;
}

// Time reps grouped launches of one kernel class over every instance (the
// tiles of instance i in t[i]; each launch writes only scratch: b and the
// stage density, the other Sigma buffer or a copy of Sigma for red-black
// sweeps, the stage-1 output), after one warm-up, on the batch's stream.
static igr_status time_class(igr_batch *b, int cls, const std::vector<Tiles> &t, int reps, float *ms)
{
    cudaStream_t st = b->main;
    std::vector<const Ops *> kinds;
    for (igr_ctx *c : b->inst)
        if (std::find(kinds.begin(), kinds.end(), c->ops) == kinds.end()) kinds.push_back(c->ops);
    std::vector<SourceCall> sc;
    std::vector<JacobiCall> jc;
    std::vector<FluxCall> fc;
    auto launch = [&]() -> cudaError_t {
        for (const Ops *o : kinds) {
            cudaError_t e = cudaSuccess;
            if (cls == KC_SOURCE) {
                sc.clear();
                for (int i : b->order) {
                    igr_ctx *c = b->inst[i];
                    if (c->ops == o)
                        sc.push_back({c->g, c->p, t[i], inflow_of(c), c->q[0], nullptr, c->b, c->rho16});
                }
                e = o->source_group(sc.data(), (int)sc.size(), st);
            } else if (cls == KC_JACOBI) {
                for (int colour = -1; colour < 1 && e == cudaSuccess; colour++) {
                    jc.clear();
                    for (int i : b->order) {
                        igr_ctx *c = b->inst[i];
                        const bool rb = c->cfg.sigma_solver == SOLVER_RBGS;
                        if (c->ops != o || rb != (colour == 0)) continue;
                        const void *qj = c->inc ? c->rho16 : c->q[0];
                        if (rb)  // a half-sweep in place on the copy of Sigma in the stage-1 output buffer
                            jc.push_back({c->g, c->p, t[i], qj, c->b, c->q[1], c->q[1]});
                        else
                            jc.push_back({c->g, c->p, t[i], qj, c->b, c->sig[c->cur], c->sig[1 - c->cur]});
                    }
                    if (!jc.empty()) e = o->jacobi_group(jc.data(), (int)jc.size(), colour, st);
                }
            } else {
                fc.clear();
                for (int i : b->order) {
                    igr_ctx *c = b->inst[i];
                    if (c->ops == o)
                        fc.push_back({c->g, c->p, t[i], inflow_of(c), c->q[0], nullptr, c->sig[c->cur], c->q[0],
                                      c->q[1], c->sc, c->blockmax, &c->sc->err});
                }
                e = o->flux_group(fc.data(), (int)fc.size(), 1, st);
            }
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "event creation failed");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return bfail(b, IGR_ERR_CUDA, "event creation failed");
    }
    cudaError_t e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; r++) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return bfail(b, IGR_ERR_CUDA, cudaGetErrorString(e));
    *ms /= reps;
    return IGR_OK;
}

igr_status igr_autotune_batch(igr_batch *b, int reps)
{
    if (!b || reps < 1) return IGR_ERR_INVALID_ARG;
    const int n = (int)b->inst.size();
    for (igr_ctx *c : b->inst)
        if (c->profiling) return bfail(b, IGR_ERR_INVALID_ARG, "disable profiling before tuning");
    // 1. every distinct problem tuned alone (its first instance), the shape
    //    given to the instances of the same problem
    for (int i = 0; i < n; i++) {
        igr_ctx *c = b->inst[i];
        int same = -1;
        for (int k = 0; k < i && same < 0; k++) {
            const igr_ctx *d = b->inst[k];
            if (d->g.nx == c->g.nx && d->g.ny == c->g.ny && d->g.nz == c->g.nz &&
                std::equal(d->g.bc, d->g.bc + 6, c->g.bc) && d->cfg.prec == c->cfg.prec &&
                d->p.order == c->p.order && d->cfg.sigma_solver == c->cfg.sigma_solver &&
                d->p.mu == c->p.mu && d->p.zeta == c->p.zeta && d->cfg.njets == c->cfg.njets)
                same = k;
        }
        if (same >= 0) {
            c->tiles = b->inst[same]->tiles;
            continue;
        }
        igr_status s = igr_autotune(c, reps);
        if (s != IGR_OK) return bfail(b, s, igr_last_error(c));
    }
    // 2. the batch together: per kernel class, every instance's z-chunk
    //    scaled by a common factor (clamped to its grid), the fastest kept;
    //    the other instances' blocks are what fills the GPU now, so longer
    //    chunks than a lone instance wants pay
    for (int i = 0; i < n; i++) {
        igr_ctx *c = b->inst[i];
        if (c->cfg.sigma_solver == SOLVER_RBGS)
            if (cudaMemcpyAsync(c->q[1], c->sig[c->cur], c->g.n * (size_t)c->ops->storage_bytes,
                                cudaMemcpyDeviceToDevice, c->st) != cudaSuccess ||
                cudaStreamSynchronize(c->st) != cudaSuccess)
                return bfail(b, IGR_ERR_CUDA, "copy of Sigma for tuning");
    }
    const int factors[] = {1, 2, 4, 8, 16, 32};
    for (int cls : {KC_FLUX, KC_JACOBI, KC_SOURCE}) {
        std::vector<Tiles> base(n), t(n), best;
        for (int i = 0; i < n; i++) base[i] = b->inst[i]->tiles;
        float tbest = 1e30f;
        for (int f : factors) {
            bool changed = f == 1;
            for (int i = 0; i < n; i++) {
                t[i] = base[i];
                const int nz = b->inst[i]->g.nz;
                int &z = cls == KC_FLUX ? t[i].zc_flux : cls == KC_JACOBI ? t[i].zc_jacobi : t[i].zc_source;
                const int z0 = z;
                z = clamp_zc(z0 * f, nz);
                changed = changed || z != z0;
            }
            if (!changed) break;  // every chunk already spans its grid
            float ms;
            igr_status s = time_class(b, cls, t, reps, &ms);
            if (s != IGR_OK) return s;
            if (ms < tbest) {
                tbest = ms;
                best = t;
            }
        }
        for (int i = 0; i < n; i++) b->inst[i]->tiles = best[i];
    }
    return IGR_OK;
}

igr_ctx *igr_batch_instance(igr_batch *b, int i)
{
    return (b && i >= 0 && i < (int)b->inst.size()) ? b->inst[i] : nullptr;
}

igr_status igr_step_batch(igr_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return IGR_ERR_INVALID_ARG;
    if (cudaEventRecord(b->enter, b->user) != cudaSuccess || cudaStreamWaitEvent(b->main, b->enter, 0) != cudaSuccess)
        return bfail(b, IGR_ERR_CUDA, "ordering after the caller's stream");
    igr_status st = step_batch_steps(b, nsteps);
    if (cudaEventRecord(b->leave, b->main) != cudaSuccess || cudaStreamWaitEvent(b->user, b->leave, 0) != cudaSuccess)
        return bfail(b, IGR_ERR_CUDA, "ordering the caller's stream after the batch");
    return st;
}

static igr_status step_batch_steps(igr_batch *b, int nsteps)
{
    for (int n = 0; n < nsteps; n++) {
        bool steady = true;
        for (igr_ctx *c : b->inst)
            steady = steady && !c->profiling && c->speed_nblocks == (int)c->ops->flux_blocks(c->g, c->tiles);
        if (!steady) {  // first step after set_state (the dt needs a stand-alone reduction)
            igr_status s = step_forkjoin(b);
            if (s != IGR_OK) return s;
            continue;
        }
        std::vector<igr_batch::Host> now = host_state(b);
        igr_batch::Graph *gr = nullptr;
        for (auto &g : b->graphs)
            if (g.before == now) gr = &g;
        if (!gr) {
            igr_batch::Graph g;
            g.before = now;
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, IGR_ERR_CUDA, "begin capture");
            igr_status s = step_grouped(b);
            cudaError_t e = cudaStreamEndCapture(b->main, &graph);
            if (s != IGR_OK) return s;
            if (e != cudaSuccess) return bfail(b, IGR_ERR_CUDA, cudaGetErrorString(e));
            g.after = host_state(b);
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return bfail(b, IGR_ERR_CUDA, cudaGetErrorString(e));
            set_host_state(b, g.before);
            b->graphs.push_back(g);
            gr = &b->graphs.back();
        }
        if (cudaGraphLaunch(gr->exec, b->main) != cudaSuccess) return bfail(b, IGR_ERR_CUDA, "graph launch");
        set_host_state(b, gr->after);
    }
    return IGR_OK;
}

igr_status igr_sync_batch(igr_batch *b)
{
    if (!b) return IGR_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->main) != cudaSuccess || cudaStreamSynchronize(b->user) != cudaSuccess)
        return bfail(b, IGR_ERR_CUDA, "synchronize");
    for (igr_ctx *c : b->inst) {
        igr_status s = igr_sync(c);
        if (s != IGR_OK) return bfail(b, s, igr_last_error(c));
    }
    return IGR_OK;
}

const char *igr_batch_last_error(const igr_batch *b) { return b ? b->err : g_create_err; }

igr_status igr_destroy_batch(igr_batch *b)
{
    if (!b) return IGR_OK;
    if (b->main) cudaStreamSynchronize(b->main);
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    for (igr_ctx *c : b->inst) igr_destroy(c);
    for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->enter) cudaEventDestroy(b->enter);
    if (b->leave) cudaEventDestroy(b->leave);
    if (b->main) cudaStreamDestroy(b->main);
    delete b;
    return IGR_OK;
}


// ------------------------------------------------------------ adjoint

static igr_status adj_alloc(igr_ctx *c, void **p, size_t bytes)
{
    igr_status s = ctx_alloc(c, p, bytes);
    if (s == IGR_OK) c->adj.all.push_back(*p);
    return s;
}

static igr_status ensure_adjoint(igr_ctx *c)
{
    if (c->adj.ready) return IGR_OK;
    size_t n = (size_t)c->g.n, sb = c->ops->storage_bytes, cb = c->ops->compute_bytes;
    int S = c->cfg.sweeps;
    igr_status s = IGR_OK;
    for (int i = 0; i < 2 && s == IGR_OK; i++) s = adj_alloc(c, &c->adj.qs[i], 5 * n * sb);
    if (s == IGR_OK) s = adj_alloc(c, &c->adj.its, 3 * (size_t)(S + 1) * n * sb);
    if (s == IGR_OK) s = adj_alloc(c, &c->adj.b, n * sb);
    void **five[] = {&c->adj.lq0, &c->adj.lqs, &c->adj.lout, &c->adj.Lb};
    for (void **p : five)
        if (s == IGR_OK) s = adj_alloc(c, p, 5 * n * cb);
    void **one[] = {&c->adj.lsig, &c->adj.lb, &c->adj.mu, &c->adj.nl, &c->adj.rb};
    for (void **p : one)
        if (s == IGR_OK) s = adj_alloc(c, p, n * cb);
    if (s == IGR_OK) s = adj_alloc(c, &c->adj.lamJ, 5 * (size_t)c->g.plane * cb);
    if (s == IGR_OK) s = adj_alloc(c, (void **)&c->adj.gw, (size_t)(c->cfg.njets > 0 ? c->cfg.njets : 1) * sizeof(double));
    if (s == IGR_OK) s = adj_alloc(c, (void **)&c->adj.sc, sizeof(Scalars));
    if (s != IGR_OK) return s;
    CU(c, cudaMemsetAsync(c->adj.sc, 0, sizeof(Scalars), c->st));
    c->adj.ready = true;
    return IGR_OK;
}

igr_status igr_adjoint_step(igr_ctx *c, const void *q_n, const void *sigma_n, const void *lam_q_np1,
                            const void *lam_sigma_np1, void *lam_q_n, void *lam_sigma_n, double *grad_jet_w,
                            double dt, igr_dtype dtype)
{
    if (!c || !q_n || !sigma_n || !lam_q_np1 || !lam_sigma_np1 || !lam_q_n || !lam_sigma_n)
        return fail(c, IGR_ERR_INVALID_ARG, "null buffer");
    if (!(dt > 0.0)) return fail(c, IGR_ERR_INVALID_ARG, "the adjoint needs a fixed dt > 0");
    if ((int)dtype != storage_dtype(c->cfg.prec))
        return fail(c, IGR_ERR_UNSUPPORTED, "q_n and sigma_n must use the storage dtype");
    {
        const size_t sb = c->ops->storage_bytes, cb = c->ops->compute_bytes;
        if (!is_aligned(q_n, sb) || !is_aligned(sigma_n, sb) || !is_aligned(lam_q_np1, cb) ||
            !is_aligned(lam_sigma_np1, cb) || !is_aligned(lam_q_n, cb) || !is_aligned(lam_sigma_n, cb))
            return fail(c, IGR_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    }
    if (c->inc)
        return fail(c, IGR_ERR_UNSUPPORTED, "the adjoint covers the modes that store the state in one type");
    if (c->p.order != 5 || c->cfg.sigma_solver != SOLVER_JACOBI || c->p.mu != 0.0 || c->p.zeta != 0.0)
        return fail(c, IGR_ERR_UNSUPPORTED,
                    "the adjoint covers the inviscid scheme with 5th-order faces and Jacobi sweeps");
    if (c->profiling) return fail(c, IGR_ERR_INVALID_ARG, "disable profiling before the adjoint");
    igr_status s = ensure_adjoint(c);
    if (s != IGR_OK) return s;
    auto &A = c->adj;
    const Ops *o = c->ops;
    size_t n = (size_t)c->g.n, sb = o->storage_bytes, cb = o->compute_bytes;
    int S = c->cfg.sweeps;
    auto it = [&](int st, int k) { return (void *)((unsigned char *)A.its + ((size_t)st * (S + 1) + k) * n * sb); };
    const double wst[3] = {1.0, 0.25, 2.0 / 3.0};
    Scalars hsc = {};
    hsc.dt = dt;
    CU(c, cudaMemcpyAsync(A.sc, &hsc, sizeof(Scalars), cudaMemcpyHostToDevice, c->st));
    CU(c, cudaStreamSynchronize(c->st));  // hsc lives on this stack frame
    // forward recompute: stage inputs and every Sigma iterate
    const void *qs[3] = {q_n, A.qs[0], A.qs[1]};
    CU(c, cudaMemcpyAsync(it(0, 0), sigma_n, n * sb, cudaMemcpyDeviceToDevice, c->st));
    for (int st = 0; st < 3; st++) {
        CU(c, o->source(c->g, c->p, c->tiles, inflow_of(c), qs[st], nullptr, A.b, nullptr, c->st));
        for (int k = 0; k < S; k++)
            CU(c, o->jacobi(c->g, c->p, c->tiles, qs[st], A.b, it(st, k), it(st, k + 1), -1, c->st));
        if (st < 2) {
            CU(c, o->flux(c->g, c->p, c->tiles, inflow_of(c), st == 0 ? FLUX_STAGE1 : FLUX_STAGE2, qs[st],
                          nullptr, it(st, S), q_n, (void *)qs[st + 1], nullptr, nullptr, A.sc, c->blockmax,
                          &A.sc->err, c->st));
            CU(c, cudaMemcpyAsync(it(st + 1, 0), it(st, S), n * sb, cudaMemcpyDeviceToDevice, c->st));
        }
    }
    // reverse
    void *lout = A.lout, *lqs = A.lqs, *lsig = A.lsig, *nl = A.nl;
    CU(c, cudaMemcpyAsync(lout, lam_q_np1, 5 * n * cb, cudaMemcpyDeviceToDevice, c->st));
    CU(c, cudaMemcpyAsync(lsig, lam_sigma_np1, n * cb, cudaMemcpyDeviceToDevice, c->st));
    CU(c, cudaMemsetAsync(A.lq0, 0, 5 * n * cb, c->st));
    CU(c, cudaMemsetAsync(A.lamJ, 0, 5 * (size_t)c->g.plane * cb, c->st));
    CU(c, cudaMemsetAsync(A.rb, 0, n * cb, c->st));
    for (int st = 2; st >= 0; st--) {
        CU(c, o->adj_rk(lout, A.lq0, lqs, A.Lb, 5 * (long long)n, wst[st], dt, c->st));
        CU(c, o->adj_rhs(c->g, c->p, inflow_of(c), qs[st], it(st, S), A.Lb, lqs, lsig, A.lamJ, c->st));
        CU(c, cudaMemsetAsync(A.lb, 0, n * cb, c->st));
        for (int k = S - 1; k >= 0; k--) {
            CU(c, o->adj_jacobi(c->g, c->p, qs[st], it(st, k), it(st, k + 1), lsig, nl, A.lb, A.rb, A.mu, c->st));
            std::swap(lsig, nl);
        }
        CU(c, o->adj_rho(c->g, qs[st], A.rb, lqs, c->st));
        CU(c, o->adj_source(c->g, c->p, inflow_of(c), qs[st], A.lb, lqs, A.lamJ, c->st));
        if (st == 0)  // the first stage reads q_n itself: lq0 += lqs
            CU(c, o->adj_rk(lqs, A.lq0, lqs, A.Lb, 5 * (long long)n, 0.0, 0.0, c->st));
        else
            std::swap(lout, lqs);
    }
    CU(c, cudaMemcpyAsync(lam_q_n, A.lq0, 5 * n * cb, cudaMemcpyDeviceToDevice, c->st));
    CU(c, cudaMemcpyAsync(lam_sigma_n, lsig, n * cb, cudaMemcpyDeviceToDevice, c->st));
    if (grad_jet_w && c->cfg.njets > 0) {
        CU(c, cudaMemsetAsync(A.gw, 0, c->cfg.njets * sizeof(double), c->st));
        CU(c, o->adj_jets(c->g, c->p, c->jets_dev, c->cfg.njets, A.lamJ, A.gw, c->st));
        std::vector<double> h(c->cfg.njets);
        CU(c, cudaMemcpyAsync(h.data(), A.gw, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CU(c, cudaStreamSynchronize(c->st));
        for (int j = 0; j < c->cfg.njets; j++) grad_jet_w[j] += h[j];
    }
    return IGR_OK;
}


igr_status igr_diagnose(igr_ctx *c, igr_diagnostics *out)
{
    if (!c || !out) return fail(c, IGR_ERR_INVALID_ARG, "ctx and out are required");
    if (!c->diag_part) {
        igr_status s = ctx_alloc(c, (void **)&c->diag_part, sizeof(double) * DIAG_PARTS * DIAG_BLOCKS_MAX);
        if (s != IGR_OK) return s;
    }
    int nb = 0;
    Inflow in{c->W, c->J};
    prof_begin(c, KC_OTHER);
    CU(c, c->ops->diag(c->g, c->p, in, c->q[0], c->sig[c->cur], c->diag_part, &nb, c->st));
    prof_end(c);
    std::vector<double> part((size_t)nb * DIAG_PARTS);
    CU(c, cudaMemcpyAsync(part.data(), c->diag_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          c->st));
    igr_status s = read_flags(c);  // synchronises
    if (s != IGR_OK) return s;
    double acc[DIAG_PARTS] = {0, 0, 0, 0, 0, 0, 0, INFINITY, INFINITY, 0};
    for (int b = 0; b < nb; b++) {  // fixed order: deterministic
        const double *x = part.data() + (size_t)b * DIAG_PARTS;
        for (int t = 0; t < 7; t++) acc[t] += x[t];
        acc[7] = fmin(acc[7], x[7]);
        acc[8] = fmin(acc[8], x[8]);
        acc[9] = fmax(acc[9], x[9]);
    }
    double vol = c->p.dx * c->p.dx * c->p.dx;
    out->mass = acc[0] * vol;
    for (int a = 0; a < 3; a++) out->momentum[a] = acc[1 + a] * vol;
    out->energy = acc[4] * vol;
    out->rho_min = acc[7];
    out->p_min = acc[8];
    out->sigma_absmax = acc[9];
    out->b_norm = sqrt(acc[6]);
    out->sigma_residual = acc[6] > 0 ? sqrt(acc[5] / acc[6]) : sqrt(acc[5]);
    return IGR_OK;
}

igr_status igr_debug_bounds_hits(unsigned long long *hits, int clear)
{
    if (!hits) return fail(nullptr, IGR_ERR_INVALID_ARG, "hits is NULL");
    unsigned long long sum = 0;
    for (const Ops *o : {&ops_f64, &ops_f32, &ops_f16, &ops_bf16, &ops_f16inc, &ops_bf16inc}) {
        unsigned long long h = o->bounds_hits(clear);
        if (h == ~0ull) return fail(nullptr, IGR_ERR_UNSUPPORTED, "not a bounds-checking debug build");
        sum += h;
    }
    *hits = sum;
    return IGR_OK;
}

igr_status igr_debug_bounds_selftest(void)
{
    unsigned long long h;
    igr_status s = igr_debug_bounds_hits(&h, 0);
    if (s != IGR_OK) return s;
    int *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(int)) != cudaSuccess) return fail(nullptr, IGR_ERR_OOM, "selftest buffer");
    cudaError_t e = ops_f32.bounds_selftest(sink, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(sink);
    if (e != cudaSuccess) return fail(nullptr, IGR_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
    return IGR_OK;
}

igr_status igr_get_flags(igr_ctx *c, int *flags)
{
    if (!c || !flags) return fail(c, IGR_ERR_INVALID_ARG, "ctx and flags are required");
    igr_status s = read_flags(c);
    *flags = c->warn_flags;
    c->warn_flags = 0;
    return s;
}

}  // extern "C"
