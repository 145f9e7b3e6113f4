// Internal interface between the host runtime (igr_api.cu) and the kernel
// translation units (igr_kernels.cu, compiled once per storage type).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/igr.h"

namespace igr {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2 };

// Kernel classes for per-launch timing.
enum { KC_SOURCE = 0, KC_JACOBI = 1, KC_FLUX = 2, KC_OTHER = 3, KC_COUNT = 4 };

struct Geom {
    int nx, ny, nz;
    int bc[6];          // faces -x,+x,-y,+y,-z,+z
    long long plane;    // nx * ny
    long long n;        // nx * ny * nz
};

struct Phys {
    double dx, gamma, alpha, cfl;
    int order;   // face reconstruction: 5 or 3
    double mu, zeta;  // shear and bulk viscosity (0: Euler)
};

// Sigma sweep kinds (igr_config.sigma_solver)
enum { SOLVER_JACOBI = 0, SOLVER_RBGS = 1 };

// bits of Scalars::err
enum { ERRF_NONFINITE = 1, ERRF_FACE = 2 };

// Device-resident scalars of a context.
struct Scalars {
    double dt;          // time step of the current step
    double t;           // accumulated simulated time
    double speed;       // max_d(|u_d| + c) of the state at the start of the step
    int err;            // ERRF_NONFINITE: a non-finite value or dt; ERRF_FACE: a face with rho or p <= 0
    int pad;
};

// Inflow tables on the -z face, in the arithmetic type:
// W[j][i] = sum_n s_n, J[v][j][i] = sum_n s_n q_jet_n[v].
struct Inflow {
    const void *W;
    const void *J;
};

// Launch shapes chosen by the runtime.
struct Tiles {
    int zc_source;  // z-planes per block of the source kernel
    int zc_jacobi;  // z-planes per block of the Jacobi kernel
    int zc_flux;    // z-planes per block of the flux kernel
    int vec_source; // 1: 4 cells per thread (128-cell rows; nx % 4 == 0), 0: one cell per thread
    int vec_jacobi; // the same for the Jacobi kernel
    int z_begin;    // a flux launch covers planes [z_begin, z_end) only (z_begin a multiple
    int z_end;      // of zc_flux, z_end a multiple or nz); z_end = 0: all planes
};

// Default form of the source and Jacobi kernels for rows of nx cells. The
// 4-cell form runs fewer instructions per cell (source 80 against 140,
// Jacobi 69 against 79, FP16 storage) but covers rows in blocks of 128
// cells, the 1-cell form in blocks of 32; the lanes beyond nx idle. The
// 4-cell form is taken where its share of busy lanes is at least the
// instruction ratio (num / den) times the 1-cell form's.
inline int vec4_default(int nx, int num, int den)
{
    if (nx % 4) return 0;
    const long long t4 = (nx + 127LL) / 128 * 128, t1 = (nx + 31LL) / 32 * 32;
    return t1 * den >= t4 * num ? 1 : 0;  // nx / t4 >= (num / den) (nx / t1)
}
inline int vec4_default_source(int nx) { return vec4_default(nx, 80, 140); }
inline int vec4_default_jacobi(int nx) { return vec4_default(nx, 69, 79); }

// Alignment of caller device pointers. Every kernel reads and writes whole
// elements, so a pointer must be aligned to its element size. The 4-cell
// forms of the source and Jacobi kernels also load and store 4 consecutive
// values at once (8 bytes at 16-bit storage, 16 bytes for FP32 and, as two
// 16-byte accesses, for FP64), so they need the field bases aligned to that;
// a call whose pointers are not takes the 1-cell forms, which give the same
// bits.
inline bool is_aligned(const void *p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }
inline size_t vec4_align(int storage_bytes) { return storage_bytes * 4 > 16 ? 16 : (size_t)storage_bytes * 4; }

// Stage modes of the flux kernel.
enum { FLUX_RHS = 0, FLUX_STAGE1 = 1, FLUX_STAGE2 = 2, FLUX_STAGE3 = 3 };

// Kernel set of one storage type. Every entry enqueues on `st` and returns
// the launch error (cudaGetLastError) without synchronising.
struct Ops {
    int storage_bytes;  // bytes per stored value (Sigma, b; the increments of the increment modes)
    int compute_bytes;  // bytes per arithmetic value (8 for FP64, else 4)
    int state_bytes;    // bytes per value of the state q^n (the storage type; 4 in the increment modes)
    // b = alpha [tr(G^2) + tr(G)^2] from the stage state q (+ increments qd in the
    // increment modes, NULL in stage 1 and in every other mode); in the increment
    // modes rho_out gets the stage density in the storage type, which the sweeps
    // read as their q (NULL otherwise)
    cudaError_t (*source)(const Geom &, const Phys &, const Tiles &, const Inflow &,
                          const void *q, const void *qd, void *b, void *rho_out, cudaStream_t st);
    // one Jacobi sweep s_out <- (b + beta sum c s_in) / (1/rho + beta sum c) with
    // colour < 0; with colour 0 or 1 one red-black Gauss-Seidel half-sweep in
    // place (s_in == s_out), updating the cells with (i + j + k) % 2 == colour
    cudaError_t (*jacobi)(const Geom &, const Phys &, const Tiles &, const void *q,
                          const void *b, const void *s_in, void *s_out, int colour, cudaStream_t st);
    // flux divergence and RK stage (mode FLUX_STAGE*), or L(q; Sigma) into rhs (FLUX_RHS).
    // Stage 3 also writes the per-block maximum wave speed of its output to blockmax.
    // Stage 1 with base_out != NULL also copies its input qs there (the RK base of
    // stages 2 and 3 when it lives in host memory). In the increment modes the
    // stage input is qs (= q^n) plus the increments qd (stages 2 and 3; NULL in
    // stage 1 and in every other mode), stages 1 and 2 write increments to out
    // and stage 3 writes the FP32 state q^n+1 to out.
    cudaError_t (*flux)(const Geom &, const Phys &, const Tiles &, const Inflow &, int mode,
                        const void *qs, const void *qd, const void *sig, const void *qn, void *out,
                        void *rhs, void *base_out, const Scalars *sc, double *blockmax, int *err,
                        cudaStream_t st);
    // number of blocks of the flux launch (entries of blockmax it writes)
    long long (*flux_blocks)(const Geom &, const Tiles &);
    // per-block maximum wave speed of q; returns the block count in *nblocks
    cudaError_t (*speed)(const Geom &, const Phys &, const void *q, double *blockmax,
                         int *nblocks, cudaStream_t st);
    // out = qn + w ((qs - qn) + dt L) over n values, exactly as the flux
    // kernel's epilogue stores it (L in the arithmetic type; in the increment
    // modes the FP32 state update of stage 3 on FP32 arrays)
    cudaError_t (*rk_combine)(const void *qn, const void *qs, const void *L, void *out,
                              long long n, double dt, double w, cudaStream_t st);

    // ---- adjoint (all adjoint buffers in the arithmetic type) ----
    // lq0 += (1 - w) lout; lqs = w lout; Lb = w dt lout   (5 n values)
    cudaError_t (*adj_rk)(const void *lout, void *lq0, void *lqs, void *Lb, long long n5, double w,
                          double dt, cudaStream_t st);
    // reverse of L(qs; sig): Lb -> lqs (5 fields), lsig, lamJ (5 x plane), by atomics
    cudaError_t (*adj_rhs)(const Geom &, const Phys &, const Inflow &, const void *qs,
                           const void *sig, const void *Lb, void *lqs, void *lsig, void *lamJ,
                           cudaStream_t st);
    // one reversed Jacobi sweep s_k -> F: lsig (in: adjoint of F) -> nl (adjoint
    // of s_k); lb += mu; rb += d/d(1/rho); mu is scratch
    cudaError_t (*adj_jacobi)(const Geom &, const Phys &, const void *q, const void *sk,
                              const void *F, const void *lsig, void *nl, void *lb, void *rb,
                              void *mu, cudaStream_t st);
    // lqs[rho] -= rb / rho^2; rb = 0
    cudaError_t (*adj_rho)(const Geom &, const void *q, void *rb, void *lqs, cudaStream_t st);
    // reverse of the IGR source: lb -> lqs (rho, m), lamJ, by atomics
    cudaError_t (*adj_source)(const Geom &, const Phys &, const Inflow &, const void *q,
                              const void *lb, void *lqs, void *lamJ, cudaStream_t st);
    // gw[n] += sum over the inflow face of s_n (rho_n lamJ_mz + rho_n w_n lamJ_E)
    cudaError_t (*adj_jets)(const Geom &, const Phys &, const double *jets, int njets,
                            const void *lamJ, double *gw, cudaStream_t st);

    // ---- diagnostics (FP64) ----
    // per-block partials (DIAG_PARTS doubles each) of the state's totals,
    // extrema and the elliptic residual; *nblocks <= DIAG_MAXBLOCKS blocks
    cudaError_t (*diag)(const Geom &, const Phys &, const Inflow &, const void *q, const void *sig,
                        double *part, int *nblocks, cudaStream_t st);

    // ---- debug build (IGR_DEBUG_BOUNDS) ----
    // out-of-range indices counted by the forward kernels since the last clear
    // (~0 when the library is not a debug build); a self-test forming one
    // out-of-range index (checked, never dereferenced; sink is never written)
    unsigned long long (*bounds_hits)(int clear);
    cudaError_t (*bounds_selftest)(int *sink, cudaStream_t st);

    // ---- grouped launches over independent instances (batches) ----
    // One launch per kernel class covers every instance's blocks; each
    // instance keeps its own grid, launch shape and buffers, so its results
    // are bitwise those of its own launches. The launchers split the calls
    // into groups a single launch can take (the same kernel form, at most
    // kGroupMax instances).
    cudaError_t (*source_group)(const struct SourceCall *calls, int n, cudaStream_t st);
    cudaError_t (*jacobi_group)(const struct JacobiCall *calls, int n, int colour, cudaStream_t st);
    cudaError_t (*flux_group)(const struct FluxCall *calls, int n, int mode, cudaStream_t st);
};

// One instance's arguments of a grouped launch (the same as the single
// launch's, see Ops::source, Ops::jacobi, Ops::flux).
struct SourceCall {
    Geom g;
    Phys p;
    Tiles t;
    Inflow in;
    const void *q, *qd;
    void *b, *rho_out;
};
struct JacobiCall {
    Geom g;
    Phys p;
    Tiles t;
    const void *q, *b, *s_in;
    void *s_out;
};
struct FluxCall {
    Geom g;
    Phys p;
    Tiles t;
    Inflow in;
    const void *qs, *qd, *sig, *qn;
    void *out;
    const Scalars *sc;
    double *blockmax;
    int *err;
};

// instances per grouped launch: their descriptors travel as one kernel
// parameter (at most 32 KB)
enum { kGroupMax = 64 };

// layout of one block's diagnostics partials: sums of rho, mx, my, mz, E,
// (A Sigma - b)^2, b^2; minima of rho and p; maximum |Sigma|
enum { DIAG_PARTS = 10, DIAG_BLOCKS_MAX = 152 * 8 };

extern const Ops ops_f64, ops_f32, ops_f16, ops_bf16, ops_f16inc, ops_bf16inc;

// shared by the host entry points (igr_api.cu, igr_noalloc.cu)
const Ops *ops_for(int precision);             // kernel set of an igr_precision
Tiles default_tiles(const Geom &g);            // launch shapes for a grid
const char *validate_config(const igr_config *c);  // NULL when valid

}  // namespace igr
