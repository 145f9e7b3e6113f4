/*
 * igr.h - C ABI of the GB300 IGR Euler stage solver.
 *
 * One call of igr_step advances the 3D compressible Euler equations with
 * information geometric regularization (IGR) by SSP-RK3 time steps on a
 * uniform Cartesian grid. Each of the three stages runs, on one GPU:
 *   1. velocity gradients and the IGR source
 *        b = alpha [tr((grad u)^2) + tr^2(grad u)]       (Eq. igrelliptic, left side)
 *   2. warm-started Jacobi sweeps for the entropic pressure Sigma of
 *        Sigma/rho - alpha div(grad Sigma / rho) = b      (Eq. igrelliptic)
 *      with the 7-point stencil and face coefficient (1/rho_i + 1/rho_nb)/2
 *   3. 5th-order finite-volume face reconstruction of (rho, m, E, Sigma),
 *      local Lax-Friedrichs flux of the IGR-modified Euler system with
 *      pressure p + Sigma                         (Eqs. igrmabalance-igrenbalance)
 *   4. flux divergence and the SSP-RK3 stage update (Gottlieb-Shu)
 * following Sec. "Discretization" and Algorithm 1 of the paper.
 *
 * Conventions for every function:
 *  - Return value: an igr_status. No exception or longjmp crosses the ABI.
 *    On failure igr_last_error(ctx) gives a one-line message.
 *  - State layout: q is [5][nz][ny][nx] contiguous (x fastest), variables
 *    (rho, rho u, rho v, rho w, E), interior cells only. Sigma is
 *    [nz][ny][nx]. No ghost cells: boundary conditions act by index mapping.
 *  - Element types: the "storage dtype" of a precision mode is that of
 *    Sigma and b (FP64, FP32, binary16 or bfloat16); the "state dtype" is
 *    that of q: the storage dtype, except FP32 in the increment modes
 *    (IGR_F32_F16INC, IGR_F32_BF16INC).
 *  - Device pointers are borrowed. Calls that take them are asynchronous on
 *    the context's stream; the caller keeps the memory alive until that
 *    stream has passed the call. Host pointers are read or written before
 *    the call returns.
 *  - Alignment: a device pointer must be aligned to its element size (2, 4
 *    or 8 bytes), else the call returns IGR_ERR_INVALID_ARG before any
 *    launch. Where a call could take the 4-cell kernel forms (igr_solve_sigma,
 *    igr_solve_sigma_noalloc), pointers that are element-aligned but not
 *    aligned to 4 elements (8 bytes at 16-bit storage, 16 bytes for FP32 and
 *    FP64; a sliced tensor can start anywhere) make that call take the
 *    1-cell forms, which give the same bits. Buffers from cudaMalloc or a
 *    caching allocator are 256-byte aligned.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Asynchronous faults (CUDA errors, non-finite results) surface at the
 *    next call that synchronises: igr_get_state, igr_sync, igr_step_host,
 *    or igr_step with a non-NULL t_inout.
 */
#ifndef IGR_H
#define IGR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IGR_OK = 0,
    IGR_ERR_INVALID_ARG = 1, /* rejected before any launch */
    IGR_ERR_OOM = 2,         /* an allocation failed */
    IGR_ERR_CUDA = 3,        /* a CUDA call failed */
    IGR_ERR_NONFINITE = 4,   /* a stage produced a NaN/Inf value or time step */
    IGR_ERR_TIMEOUT = 5,     /* reserved for bounded device-side waits */
    IGR_ERR_UNSUPPORTED = 6  /* a valid request that the library does not implement */
} igr_status;

/* Arithmetic and storage of a context. */
typedef enum {
    IGR_F64 = 0,           /* FP64 storage and arithmetic */
    IGR_F32 = 1,           /* FP32 storage and arithmetic */
    IGR_F32_F16STORE = 2,  /* FP32 arithmetic, q/Sigma/b stored as IEEE binary16,
                              RK combination in FP64, round-to-nearest-even on store */
    IGR_F32_BF16STORE = 3, /* as above with bfloat16 storage */
    IGR_F32_F16INC = 4,    /* FP32 arithmetic; the state q^n in FP32 (the RK accumulation
                              never rounds to 16 bits); RK stages 1 and 2 store the
                              increments d_s = q_s - q^n as IEEE binary16 (a stage reads
                              q_s = RN32(q^n + d_s)); Sigma, b and the sweeps' density in
                              binary16. Increments must stay within binary16's range
                              (|d| < 65504), else the step reports IGR_ERR_NONFINITE. */
    IGR_F32_BF16INC = 5    /* as IGR_F32_F16INC with bfloat16 increments, Sigma and b */
} igr_precision;

/* Element type of a buffer passed across the ABI. */
typedef enum { IGR_DT_F64 = 0, IGR_DT_F32 = 1, IGR_DT_F16 = 2, IGR_DT_BF16 = 3 } igr_dtype;

/* Boundary condition of one domain face. */
typedef enum {
    IGR_BC_PERIODIC = 0, /* wrap (must be set on both faces of an axis) */
    IGR_BC_OUTFLOW = 1,  /* zero gradient: out-of-domain cells copy the nearest cell */
    IGR_BC_INFLOW = 2    /* jets (only on the -z face): the out-of-domain state is
                            (1 - sum_n s_n) q_nearest + sum_n s_n q_jet_n with
                            s_n = (1 - tanh((r_n - R_n)/(edge_width_n dx)))/2;
                            Sigma sees zero gradient */
} igr_bc;

/* A circular jet on the -z face: centre (cx, cy) and radius in length units,
 * primitive state (rho, w along +z, p), edge width in cells. */
typedef struct {
    double cx, cy, radius, rho, w, p, edge_width;
} igr_jet;

/* Optional caller-supplied device allocator (e.g. a framework's caching
 * allocator). alloc returns device memory aligned to 256 bytes or NULL. */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} igr_allocator;

typedef struct {
    int nx, ny, nz;     /* cells per axis, each >= 4 */
    double dx;          /* cell size (cubic cells) */
    double gamma;       /* ideal-gas ratio of specific heats, Eq. (state_eqn) */
    double alpha;       /* IGR alpha, proportional to dx^2 */
    double cfl;         /* dt = cfl dx / max_cells max_d(|u_d| + c) */
    int sweeps;         /* Jacobi sweeps per stage, >= 1 */
    igr_precision prec;
    igr_bc bc[6];       /* faces -x, +x, -y, +y, -z, +z */
    const igr_jet *jets;/* njets jets on an IGR_BC_INFLOW -z face (copied) */
    int njets;
    int host_rk_base;   /* 0: in-core. 1: keep the RK base q^n (5 n values) in pinned,
                           device-mapped host memory (cudaHostAlloc) instead of a third
                           device state buffer: stage 1 writes it while it reads its
                           input, stages 2 and 3 read it over the CPU-GPU link (NVLink-C2C
                           on Grace systems). Device memory drops from 18 to 13 values
                           per cell; results are bitwise those of the in-core mode. Not
                           available in batches. Ignored by igr_solve_sigma_noalloc. */
    int order;          /* face reconstruction (Sec. "Discretization": third- or
                           fifth-order finite volumes): 5 (0 means 5) or 3, the
                           quadratic through three cell averages of each biased
                           stencil */
    int sigma_solver;   /* Sigma sweeps (Sec. "Discretization": Jacobi or Gauss-Seidel):
                           IGR_SOLVER_JACOBI (two Sigma buffers) or IGR_SOLVER_RBGS,
                           red-black Gauss-Seidel in place (red cells, i + j + k even,
                           then black; one Sigma buffer; every periodic axis must
                           have even length). igr_adjoint_step covers order 5 with
                           Jacobi only. */
    double mu, zeta;    /* shear and bulk viscosity, Eq. (constitutive_law); 0, 0 is the
                           Euler system. Nonzero adds tau = mu (grad u + grad u^T)
                           + (zeta - 2 mu/3)(div u) I to the momentum flux and u . tau
                           to the energy flux, with second-order face derivatives (the
                           two cells across the face; tangential derivatives averaged
                           over both). dt keeps the convective CFL rule: the caller
                           keeps dt within the viscous limit ~ rho dx^2 / mu. Not in
                           igr_adjoint_step. */
} igr_config;

#define IGR_SOLVER_JACOBI 0
#define IGR_SOLVER_RBGS 1

typedef struct igr_ctx igr_ctx; /* opaque */

/* Validate cfg and allocate the context on the current CUDA device:
 * three state buffers (5 fields each; two with host_rk_base, plus the host
 * buffer of the RK base), two Sigma buffers, the source b,
 * the inflow tables and a few scalars, all in the storage type of
 * cfg->prec; in the increment modes two FP32 state buffers, two buffers of
 * 16-bit increments and the stage density instead of the three state
 * buffers (68 bytes per cell with Jacobi sweeps, against 72 for IGR_F32 and
 * 36 for IGR_F32_F16STORE). allocator may be NULL (cudaMalloc). cuda_stream is a
 * cudaStream_t (NULL = legacy default stream). The state and Sigma start
 * at zero; call igr_set_state before stepping. */
igr_status igr_create(const igr_config *cfg, const igr_allocator *allocator, void *cuda_stream,
                      igr_ctx **out);

/* Device bytes igr_create allocates for cfg (0 if cfg is invalid); with
 * host_rk_base the pinned host buffer (5 n stored values) is not counted. */
size_t igr_memory_bytes(const igr_config *cfg);

/* Synchronise the stream, free every buffer, destroy the context. NULL is a no-op. */
igr_status igr_destroy(igr_ctx *ctx);

/* Copy a state into the context. q holds 5 n values, sigma n values
 * (NULL sets Sigma = 0, the cold start). dtype is the element type of q
 * and sigma; on_device = 1 means device pointers (any dtype, converted on
 * the device), 0 means host pointers (dtype must be the state dtype). */
igr_status igr_set_state(igr_ctx *ctx, const void *q, const void *sigma, igr_dtype dtype,
                         int on_device);

/* Replace q alone (5 n values; dtype and on_device as for igr_set_state)
 * and keep Sigma, the warm start of the next elliptic solve. This is the
 * call for a host-driven loop that reads q out after each step
 * (igr_get_state with sigma = NULL) and hands it back, possibly changed:
 * Sigma never leaves the device. The next step recomputes dt from the new q. */
igr_status igr_set_conserved(igr_ctx *ctx, const void *q, igr_dtype dtype, int on_device);

/* Copy the state out (q: 5 n values, sigma: n values or NULL), same
 * dtype/on_device rules as igr_set_state. Synchronises the stream and
 * reports pending asynchronous errors. */
igr_status igr_get_state(igr_ctx *ctx, void *q, void *sigma, igr_dtype dtype, int on_device);

/* Advance nsteps SSP-RK3 steps. fixed_dt > 0 uses that dt; otherwise each
 * step takes dt = cfl dx / max_d(|u_d| + c) of the state at its start,
 * computed on the device (no host round trip). If t_inout is non-NULL the
 * call synchronises, adds the elapsed simulated time to *t_inout and
 * reports asynchronous errors; with NULL it only enqueues. */
igr_status igr_step(igr_ctx *ctx, int nsteps, double fixed_dt, double *t_inout);

/* nsteps SSP-RK3 steps from host memory to host memory: q_in (5 n values,
 * the state dtype, best pinned) is copied in, Sigma stays on the device
 * (as with igr_set_conserved), the steps run, and the final q is written to
 * q_out. rho and m are copied first; the energy field follows on a second
 * stream while the first stage's source and sweeps (which read rho and m
 * only) run, and the first step's dt is formed just before its first flux.
 * The last stage's flux kernel runs in z-slabs and each slab is copied out
 * while the next ones compute, so part of the read-back overlaps the last
 * stage. q_in and q_out may be the same buffer and must not be written
 * during the call. dt follows the CFL rule. Synchronises and reports
 * asynchronous errors. */
igr_status igr_step_host(igr_ctx *ctx, const void *q_in, void *q_out, int nsteps, igr_dtype dtype);

/* Sigma solve alone, on caller device buffers: q in the state dtype,
 * sigma_inout in the storage dtype (dtype names the storage dtype): b from
 * q, then `sweeps` Jacobi sweeps warm-started from sigma_inout; the result
 * overwrites sigma_inout. Uses the context's b, second Sigma buffer and (in
 * the increment modes) stage-density buffer as scratch (the context state
 * is untouched). */
igr_status igr_solve_sigma(igr_ctx *ctx, const void *q, void *sigma_inout, int sweeps,
                           igr_dtype dtype);

/* Spatial operator L(q; Sigma) = -div F_hat (no elliptic solve, no RK):
 * q is a device buffer in the state dtype, sigma in the storage dtype
 * (dtype), rhs is a device buffer of 5 n values in the arithmetic type
 * (FP64 for IGR_F64, FP32 otherwise). */
igr_status igr_rhs(igr_ctx *ctx, const void *q, const void *sigma, void *rhs, igr_dtype dtype);

/* Discrete adjoint of one SSP-RK3 step with a fixed dt: the transpose of the
 * Jacobian of (q, Sigma) -> (q', Sigma') that igr_step(ctx, 1, dt) computes
 * (Sigma enters through the warm start of the Jacobi sweeps, so it is part
 * of the state), applied to (lam_q_np1, lam_sigma_np1):
 *   lam_q_n     = (dq'/dq)^T lam_q_np1 + (dSigma'/dq)^T lam_sigma_np1
 *   lam_sigma_n = (dq'/dSigma)^T lam_q_np1 + (dSigma'/dSigma)^T lam_sigma_np1
 *   grad_jet_w[j] += the same product's derivative in jet j's velocity w_j.
 * It is the hand-written reverse of every piece of the stage (RK combination,
 * flux divergence, local LF flux with p + Sigma, 5th-order reconstruction,
 * Jacobi sweeps in the variable mu = lambda / diagonal, IGR source, boundary
 * and jet-blend index mapping); the forward step is recomputed from (q_n,
 * sigma_n) and every Sigma iterate kept. Non-smooth points follow the
 * forward's branch (max(aL, aR): the side taken, aR on a tie; |u|: sign(u)).
 * q_n, sigma_n: device buffers in the storage dtype (dtype); lam_*: device
 * buffers in the arithmetic type (FP64 for IGR_F64, else FP32; 5 n and n
 * values; outputs may not alias inputs); grad_jet_w: host array of njets
 * doubles or NULL (synchronises when given). The first call allocates a
 * workspace of about (29 + 3 sweeps) n stored values plus 30 n arithmetic
 * values through the context's allocator. The scatter steps use atomics, so
 * FP32 results vary in the last bits from run to run. The increment modes
 * return IGR_ERR_UNSUPPORTED. */
igr_status igr_adjoint_step(igr_ctx *ctx, const void *q_n, const void *sigma_n,
                            const void *lam_q_np1, const void *lam_sigma_np1, void *lam_q_n,
                            void *lam_sigma_n, double *grad_jet_w, double dt, igr_dtype dtype);

/* The SSP-RK3 stage combination alone, exactly as the stage kernel stores it:
 *   out = qn + w [(qs - qn) + dt L],  w = 1, 1/4, 2/3 for stage = 1, 2, 3
 * (Gottlieb-Shu SSP-RK3 in increment form). qn, qs, out: device buffers of
 * count values in the state dtype; L: device buffer in the arithmetic type
 * (FP64 for IGR_F64, FP32 otherwise). In IGR_F32_F16STORE and
 * IGR_F32_BF16STORE the stored value is the FP64 evaluation of the
 * expression rounded to nearest-even; in the increment modes it is the FP32
 * state update of stage 3 (stages 1 and 2 there store the increment
 * w [(qs - qn) + dt L] rounded to 16 bits). out may alias qn. For
 * verification and tooling. */
igr_status igr_rk_combine(igr_ctx *ctx, const void *qn, const void *qs, const void *L, void *out,
                          long long count, int stage, double dt);

/* ---- Allocation-free Sigma solve --------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory where they need a Sigma solve (code working
 * inside another framework's fixed memory budget, allocation-free real-time
 * loops, hooks that may not call cudaMalloc or a caching allocator).
 *
 * igr_solve_sigma_noalloc does what igr_solve_sigma does (b from q, then
 * `sweeps` Jacobi sweeps warm-started from sigma_inout, result in
 * sigma_inout) without a context and without allocating anything: its
 * scratch (b and the second Jacobi buffer, 2 n values of the storage type)
 * lives in one static device array of IGR_NOALLOC_SCRATCH_BYTES that every
 * GPU loading this library holds until the process exits.
 *  - q, sigma_inout: device buffers in the storage type of cfg->prec.
 *  - Grids needing more than the array holds (see igr_noalloc_max_cells) are
 *    rejected with IGR_ERR_INVALID_ARG; IGR_BC_INFLOW faces and the
 *    increment modes with IGR_ERR_UNSUPPORTED. The call issues no cudaMalloc/cudaFree and no
 *    allocating library routine.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture. The address is kept for later calls, so a
 *    cudaDeviceReset between calls is not supported.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents (every value is written before it is read, so nothing needs
 *    clearing). Calls whose work overlaps on the GPU (concurrent streams or
 *    threads) race on it: serialise them.
 *  - Errors: the status; the message is in igr_noalloc_last_error(). */
#define IGR_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
igr_status igr_solve_sigma_noalloc(const igr_config *cfg, const void *q, void *sigma_inout,
                                   int sweeps, void *cuda_stream);
/* Largest grid (cells) igr_solve_sigma_noalloc takes in precision prec. */
size_t igr_noalloc_max_cells(igr_precision prec);
/* Message of the calling thread's last failed igr_solve_sigma_noalloc call
 * (one buffer per thread). Never NULL. */
const char *igr_noalloc_last_error(void);

/* Time step dt = cfl dx / max_d(|u_d| + c) of the current state.
 * Synchronises. */
igr_status igr_get_dt(igr_ctx *ctx, double *dt);

/* Synchronise the stream and report pending asynchronous errors. */
igr_status igr_sync(igr_ctx *ctx);

/* Warnings seen since the last call or the last igr_set_state (synchronises):
 * IGR_WARN_FACE_POSITIVITY when a reconstructed face state had rho <= 0 or
 * p <= 0 (its LF speed is then not a number and the other side's speed is
 * used, as in the scheme's definition; the step goes on). Errors are returned
 * as by igr_sync. igr_set_state drops the warnings and errors still pending
 * from the state it replaces. */
#define IGR_WARN_FACE_POSITIVITY 2
igr_status igr_get_flags(igr_ctx *ctx, int *flags);

/* Diagnostics of the current state, evaluated in FP64 on the device from the
 * stored values (every stored value converts to double exactly):
 *  - totals over cells of rho, m and E times dx^3 (conserved exactly up to
 *    round-off under periodic boundaries);
 *  - minima of rho and p = (gamma - 1)(E - |m|^2 / (2 rho)), maximum |Sigma|;
 *  - the residual of the elliptic equation for Sigma (Eq. igrelliptic):
 *    ||A Sigma - b||_2 / ||b||_2 over cells (||A Sigma||_2 when b = 0), with
 *    A the operator the Jacobi sweeps relax (face coefficients
 *    (1/rho_i + 1/rho_nb)/2, faces on non-periodic boundaries dropped) and b
 *    the IGR source of the current state. After igr_step, Sigma is the last
 *    stage's solve and the state has advanced since, so this measures how
 *    well Sigma solves the equation for the state it is paired with.
 * Per-block partial sums are reduced in a fixed order (deterministic). The
 * first call allocates (10 x 1216 doubles) through the context allocator.
 * Synchronises; errors as igr_sync. */
typedef struct {
    double mass, momentum[3], energy;
    double rho_min, p_min, sigma_absmax;
    double b_norm;          /* ||b||_2 over cells */
    double sigma_residual;  /* ||A Sigma - b||_2 / ||b||_2 */
} igr_diagnostics;
igr_status igr_diagnose(igr_ctx *ctx, igr_diagnostics *out);

/* ---- Bounds-checking debug build ------------------------------------
 * A second library, libigr_debug.so, is compiled with IGR_DEBUG_BOUNDS: every
 * global index the forward kernels (source, Jacobi, flux, stage epilogue)
 * form is compared with its array's length, and an index out of range is
 * counted and replaced by 0, so nothing is accessed out of bounds. This
 * stands in for a memory checker (compute-sanitizer is not used).
 * igr_debug_bounds_hits returns the count summed over all precisions since
 * the last clear (clear != 0 resets it); igr_debug_bounds_selftest launches a
 * kernel that forms one out-of-range index (checked, never dereferenced),
 * which adds exactly 1. Both synchronise and return IGR_ERR_UNSUPPORTED in
 * the normal library. */
igr_status igr_debug_bounds_hits(unsigned long long *hits, int clear);
igr_status igr_debug_bounds_selftest(void);

/* Per-kernel timing with CUDA events on the context stream. While enabled,
 * every launch is bracketed by an event pair; igr_profile_read synchronises
 * and returns, for kernel class k (0 source, 1 jacobi, 2 flux, 3 other),
 * the launch count and total milliseconds since enabling. */
igr_status igr_profile_enable(igr_ctx *ctx, int on);
igr_status igr_profile_read(igr_ctx *ctx, int kernel_class, long long *launches, double *total_ms);

/* ---- Launch shapes and the autotuner ----------------------------------
 * Each kernel class marches blocks up chunks of z-planes; the chunk length
 * is the tunable launch shape (>= 4 planes, at most nz). The source and
 * Jacobi kernels also come in two forms: one cell per thread (rows in
 * blocks of 32 cells) and four cells per thread (rows in blocks of 128
 * cells; only for nx % 4 == 0), which runs fewer instructions per cell but
 * idles more lanes on short rows. By default the four-cell form is taken
 * where its share of busy lanes is at least its instruction ratio (source
 * 80/140, Jacobi 69/79) times the one-cell form's.
 * Results do not depend on the launch shape: every face flux comes out of
 * the same instructions whatever the chunking, both forms evaluate the same
 * sequence of rounded operations, and there are no atomics, so outputs are
 * bitwise identical for every choice.
 * igr_set_kernel_forms: source_vec4 and jacobi_vec4 each -1 (the default
 * rule), 0 (one cell per thread) or 1 (four cells; IGR_ERR_INVALID_ARG when
 * nx % 4 != 0).
 * igr_autotune times each class on the current state for the candidate
 * lengths 4..128 and, where nx % 4 == 0, both forms (reps launches each, on
 * the context stream; only scratch buffers are written) and keeps the
 * fastest; call it after igr_set_state. It synchronises. */
igr_status igr_set_tiles(igr_ctx *ctx, int zc_source, int zc_jacobi, int zc_flux);
igr_status igr_get_tiles(igr_ctx *ctx, int *zc_source, int *zc_jacobi, int *zc_flux);
igr_status igr_set_kernel_forms(igr_ctx *ctx, int source_vec4, int jacobi_vec4);
igr_status igr_get_kernel_forms(igr_ctx *ctx, int *source_vec4, int *jacobi_vec4);
igr_status igr_autotune(igr_ctx *ctx, int reps);

/* ---- Batches of independent instances -----------------------------------
 * n independent contexts (any sizes and configurations) advanced together.
 * igr_create_batch creates one context per config, each on its own stream
 * forked from and joined into cuda_stream. igr_batch_instance(b, i) gives
 * instance i's context for igr_set_state / igr_get_state / igr_autotune /
 * igr_get_dt (not for igr_step or igr_step_host: step the batch). igr_step_batch advances
 * every instance by nsteps SSP-RK3 steps, each with its own CFL dt. A step
 * runs each kernel class as one grouped launch over all instances' blocks
 * (one launch per precision, kernel form and scheme among the instances, at
 * most 64 instances each), so the GPU fills even when every instance is
 * small; every instance keeps its own buffers, launch shape and dt, and its
 * results are bitwise those of a context stepping alone. The step is
 * captured once as a CUDA graph and replayed, except the first step after a
 * set_state, which launches per instance directly. Asynchronous on
 * cuda_stream; igr_sync_batch synchronises and reports any instance's error. */
typedef struct igr_batch igr_batch;
igr_status igr_create_batch(const igr_config *cfgs, int n, const igr_allocator *allocator,
                            void *cuda_stream, igr_batch **out);
igr_ctx *igr_batch_instance(igr_batch *b, int i);
igr_status igr_step_batch(igr_batch *b, int nsteps);
/* igr_autotune_batch chooses every instance's launch shape for running in
 * the batch: first each distinct problem (grid, boundaries, precision,
 * scheme) alone as igr_autotune does, its shape given to the instances of
 * the same problem; then, per kernel class, all instances' z-chunks scaled
 * by a common factor 1..32 (clamped to each grid) with the grouped launches
 * timed over the whole batch (reps each, on the batch's stream), the fastest
 * kept. In a batch the other instances' blocks fill the GPU, so the chunks
 * come out longer than a lone instance's. Only scratch buffers are written:
 * states, Sigma and dt are unchanged. Call it after every instance's
 * igr_set_state; it synchronises. Results of later steps are bitwise the
 * same for any launch shape. Grouped launches order the instances largest
 * first (cells), whatever the order of cfgs. */
igr_status igr_autotune_batch(igr_batch *b, int reps);
igr_status igr_sync_batch(igr_batch *b);
const char *igr_batch_last_error(const igr_batch *b);
igr_status igr_destroy_batch(igr_batch *b);

/* Message of the last failure on ctx (or of the last failed igr_create when
 * ctx is NULL). Never NULL. */
const char *igr_last_error(const igr_ctx *ctx);

/* Library version string. */
const char *igr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IGR_H */
