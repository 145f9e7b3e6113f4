// Stage kernels of the IGR Euler solver, compiled once per storage type
// (IGR_STORAGE = double | float | __half | __nv_bfloat16, exported as the
// kernel set IGR_OPS).
//
// Layout: structure of arrays, q[v][k][j][i] with x fastest, interior cells
// only; boundary conditions act by index mapping (periodic wrap, zero-
// gradient clamp, jet blend on the -z face), never through ghost storage.
//
// All three kernels are 2.5D: a block owns a TX x TY tile of (x, y) columns
// and marches up a chunk of z-planes, keeping the column's z-neighbours in
// registers and taking x/y neighbours from the plane just loaded.
//
//   k_source  grad u (2nd-order central) and the IGR source
//             b = alpha [tr(G^2) + tr(G)^2]            (Eq. igrelliptic)
//   k_jacobi  one Jacobi sweep of the 7-point operator
//             A s = s/rho - alpha div(grad s / rho)    (Eq. igrelliptic)
//   k_flux    5th-order face values of (rho, m, E, Sigma), local
//             Lax-Friedrichs flux with pressure p + Sigma
//             (Eqs. igrmabalance-igrenbalance, Sec. "Discretization"),
//             divergence, and the SSP-RK3 stage combination
//             out = qn + w [(qs - qn) + dt L]   (w = 1, 1/4, 2/3);
//             stage 3 also reduces max_d(|u_d| + c) of its output for the
//             next dt. No atomics on the data path: every face flux is
//             computed once per tile and the divergence sums in a fixed
//             order, so results are deterministic.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <stdio.h>

#include <type_traits>

#include "igr_internal.h"

#ifndef IGR_STORAGE
#error "IGR_STORAGE must name the storage type"
#endif

namespace igr {
namespace {

using S = IGR_STORAGE;

// arithmetic type C and RK-combination type A of each storage type
template <typename T> struct Num;
template <> struct Num<double> { using C = double; using A = double; };
template <> struct Num<float> { using C = float; using A = float; };
template <> struct Num<__half> { using C = float; using A = double; };
template <> struct Num<__nv_bfloat16> { using C = float; using A = double; };
using C = Num<S>::C;
using A = Num<S>::A;

// Type of the conserved state q^n. It is the storage type, except in the
// increment modes (IGR_BASE=float, with 16-bit S): there q^n is kept in FP32
// and RK stages 1 and 2 store the 16-bit increments d_s = q_s - q^n, so a
// stage reads its input as q_s = RN32(q^n + d_s) and the RK accumulation of
// q^n never rounds to 16 bits. Sigma, b and the increments use S.
#ifdef IGR_BASE
using QB = IGR_BASE;
constexpr bool kInc = true;
#else
using QB = S;
constexpr bool kInc = false;
#endif

// Offsets inside one field are 32-bit (grids hold fewer than 2^32 cells);
// each field has its own base pointer, so an address is one 32x32->64 step.
using idx = unsigned;
// Index checks of the debug build (IGR_DEBUG_BOUNDS, a separate library):
// every global index the forward kernels form, and every shared-memory index
// that depends on more than the thread's position in its block (halo slots,
// the flux kernel's tile and face-buffer offsets), is compared with its
// array's length; an index out of range is counted and replaced by 0, so
// nothing is accessed out of bounds and the count is read on the host. In
// the normal build the checks compile to nothing.
#ifdef IGR_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds_hits;
// element offset c of an array of n values (offsets are unsigned: a
// negative one wraps to a value >= n on the grids the checks run on)
__device__ __forceinline__ idx ck(idx c, long long n)
{
    if ((long long)c >= n) {
        atomicAdd(&g_bounds_hits, 1ull);
        return 0;
    }
    return c;
}
// pointer p to w consecutive values of the array of n values at base
template <class T>
__device__ __forceinline__ T *ckp(T *p, T *base, long long n, int w)
{
    const long long d = p - base;
    if (d < 0 || d + w > n) {
        atomicAdd(&g_bounds_hits, 1ull);
        return base;
    }
    return p;
}
// 64-bit element offset c of an array of n values
__device__ __forceinline__ size_t ckl(size_t c, long long n)
{
    if ((long long)c >= n) {
        atomicAdd(&g_bounds_hits, 1ull);
        return 0;
    }
    return c;
}
#define CKP(p, base, n) ckp((p), (base), (long long)(n), 1)
#define CKP4(p, base, n) ckp((p), (base), (long long)(n), 4)
// shared-memory element index c of a tile of n elements
__device__ __forceinline__ int cks(int c, int n)
{
    if (c < 0 || c >= n) {
        atomicAdd(&g_bounds_hits, 1ull);
        return 0;
    }
    return c;
}
// the first of 4 consecutive shared values of a vector access: in range and
// a multiple of 4 (16-byte aligned for 4-byte values)
__device__ __forceinline__ int cks4(int c, int n)
{
    if (c < 0 || c + 3 >= n || (c & 3)) {
        atomicAdd(&g_bounds_hits, 1ull);
        return 0;
    }
    return c;
}
#else
__device__ __forceinline__ idx ck(idx c, long long) { return c; }
__device__ __forceinline__ size_t ckl(size_t c, long long) { return c; }
#define CKP(p, base, n) (p)
#define CKP4(p, base, n) (p)
__device__ __forceinline__ int cks(int c, int) { return c; }
__device__ __forceinline__ int cks4(int c, int) { return c; }
#endif

template <int N> struct Fin { const S *p[N]; };   // fields read
template <int N> struct Fout { S *p[N]; };        // fields written
struct Frhs { C *p[5]; };
struct QBIn { const QB *p[5]; };                  // the state q^n (RK base)
struct QBOut { QB *p[5]; };                       // a new state q^n+1

// ------------------------------------------------------------ load/store
__device__ __forceinline__ double ldc(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldc(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldc(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ldc(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

// Raw loads for prefetching: the value stays in its storage type until it is
// used, so no instruction waits on the load before then (a conversion right
// after the load would stall there and hide nothing).
__device__ __forceinline__ S ldr(const S *p) { return __ldg(p); }
__device__ __forceinline__ double cv(double v) { return v; }
__device__ __forceinline__ float cv(float v) { return v; }
__device__ __forceinline__ float cv(__half v) { return __half2float(v); }
__device__ __forceinline__ float cv(__nv_bfloat16 v) { return __bfloat162float(v); }

// Reading the state of a stage: the base fields b (type QB) plus, in the
// increment modes from stage 2 on, the increments d (type S). HASD says
// whether increments are read; without them the state is the base itself.
struct QIn {
    const QB *b[5];
    const S *d[5];
    size_t fs;  // values between consecutive fields of b and of d (the increment
                // modes address the fields from b[0] and d[0] with it)
};
struct QRawInc {  // one raw state value of the increment modes
    QB b;
    S d;
};
template <bool INC> struct StateIO;
template <> struct StateIO<false> {  // (used where the state has the storage type)
    using Raw = S;
    template <bool HASD> static __device__ __forceinline__ S ld(const QIn &q, int u, idx c)
    {
        return ldr(reinterpret_cast<const S *>(q.b[u]) + c);
    }
    template <bool HASD> static __device__ __forceinline__ C val(S r) { return cv(r); }
};
template <> struct StateIO<true> {
    using Raw = QRawInc;
    template <bool HASD> static __device__ __forceinline__ QRawInc ld(const QIn &q, int u, idx c)
    {
        QRawInc r;
        r.b = __ldg(q.b[0] + u * q.fs + c);
        r.d = HASD ? ldr(q.d[0] + u * q.fs + c) : S(0.0f);
        return r;
    }
    // the stage value q_s = RN32(q^n + d_s) (q^n itself without increments)
    template <bool HASD> static __device__ __forceinline__ C val(const QRawInc &r)
    {
        return HASD ? C(__fadd_rn(float(cv(r.b)), float(cv(r.d)))) : C(cv(r.b));
    }
};
using QRaw = StateIO<kInc>::Raw;
template <bool HASD> __device__ __forceinline__ QRaw ldqr(const QIn &q, int u, idx c)
{
    return StateIO<kInc>::ld<HASD>(q, u, c);
}
template <bool HASD> __device__ __forceinline__ C cvq(const QRaw &r) { return StateIO<kInc>::val<HASD>(r); }
template <bool HASD> __device__ __forceinline__ C ldq(const QIn &q, int u, idx c)
{
    return cvq<HASD>(ldqr<HASD>(q, u, c));
}

// store v rounded to nearest even; returns the stored value in type C
__device__ __forceinline__ double stc(double *p, double v) { *p = v; return v; }
__device__ __forceinline__ float stc(float *p, float v) { *p = v; return v; }
__device__ __forceinline__ float stc(__half *p, double v)
{
    __half h = __double2half(v);
    *p = h;
    return __half2float(h);
}
__device__ __forceinline__ float stc(__half *p, float v)
{
    __half h = __float2half_rn(v);
    *p = h;
    return __half2float(h);
}
__device__ __forceinline__ float stc(__nv_bfloat16 *p, double v)
{
    __nv_bfloat16 h = __double2bfloat16(v);
    *p = h;
    return __bfloat162float(h);
}
__device__ __forceinline__ float stc(__nv_bfloat16 *p, float v)
{
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    *p = h;
    return __bfloat162float(h);
}

// ------------------------------------------------------------ arithmetic
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double sqrt_c(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_c(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// products that are never fused into a following add: velocities u = m/rho
// must round before they are differenced, so equal neighbours give an exact 0
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
// rounded operations that the compiler neither fuses nor reorders, for
// sequences that two kernel forms must evaluate identically
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a / b as the sweeps evaluate it: a times the approximate reciprocal in
// FP32, the correctly rounded quotient in FP64
__device__ __forceinline__ double quot(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float quot(float a, float b) { return __fmul_rn(a, rcp(b)); }

// NaN-propagating maximum (a NaN wave speed must reach dt)
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

// Pairs of arithmetic values for packed FP32x2 operations (add.rn.f32x2,
// mul.rn.f32x2, fma.rn.f32x2 on sm_100 and later: each lane rounds exactly
// like the scalar operation); FP64 pairs take two scalar operations.
template <typename T> struct PairOf;
template <> struct PairOf<float> { using T = float2; };
template <> struct PairOf<double> { using T = double2; };
using C2 = typename PairOf<C>::T;

__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b)
{
    return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c)
{
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ C2 pset(C x, C y)
{
    C2 r;
    r.x = x;
    r.y = y;
    return r;
}
__device__ __forceinline__ C2 bcast(C v) { return pset(v, v); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 padd(double2 a, double2 b)
{
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}

// ------------------------------------------------------------ indexing
__device__ __forceinline__ int wrap(int c, int n)
{
    c %= n;
    return c < 0 ? c + n : c;
}
// in-range index for coordinate c along an axis of n cells
__device__ __forceinline__ int map_axis(int c, int n, int bclo, int bchi)
{
    if (c < 0) return bclo == BC_PERIODIC ? wrap(c, n) : 0;
    if (c >= n) return bchi == BC_PERIODIC ? wrap(c, n) : n - 1;
    return c;
}

// 5th-order finite-volume face values at face i+1/2 from cell averages
// v[i-2..i+3]: the quartic through the five cell averages of the left-
// (resp. right-) biased stencil, evaluated at the face.
__device__ __forceinline__ C rec_left(C a, C b, C c, C d, C e)
{
    return C(2.0 / 60.0) * a - C(13.0 / 60.0) * b + C(47.0 / 60.0) * c + C(27.0 / 60.0) * d -
           C(3.0 / 60.0) * e;
}
__device__ __forceinline__ C rec_right(C b, C c, C d, C e, C f)
{
    return C(-3.0 / 60.0) * b + C(27.0 / 60.0) * c + C(47.0 / 60.0) * d - C(13.0 / 60.0) * e +
           C(2.0 / 60.0) * f;
}

// Doubled local Lax-Friedrichs flux along axis D from face states (rho, mx,
// my, mz, E, Sigma) on the left and right:
//   G = 2 F_hat = (F_L + F_R) - lam (q_R - q_L),
//   F = (m_D, m u_D + (p + Sigma) e_D, (E + p + Sigma) u_D),
//   p = (gamma - 1)(E - |m|^2 / (2 rho)), lam = max(|u_D| + c) over both sides,
//   c = sqrt(gamma p / rho).
// (The factor 1/2 is applied once, in the divergence.) Flags a non-positive
// face density or pressure.
// The warning flag of non-positive face states. In the 16-bit storage forms
// it is a running minimum of the face densities and pressures, tested once
// per block (fewer instructions per face: their flux kernel ran 2.4% faster
// at full size); FP32 and FP64 storage keep a boolean per face (the minimum
// measured 0.9% slower there). A face whose four values are all NaN sets
// the boolean and not the minimum; its outputs raise the non-finite error.
constexpr bool kFaceMin = sizeof(S) == 2;
using FaceFlag = std::conditional<kFaceMin, C, bool>::type;
__device__ __forceinline__ void flag_face(bool &f, C a, C b, C c, C d) { f |= !(fmin(fmin(a, b), fmin(c, d)) > C(0)); }
template <class T> __device__ __forceinline__ void flag_face(T &f, C a, C b, C c, C d)
{
    f = fmin(f, fmin(fmin(a, b), fmin(c, d)));
}
__device__ __forceinline__ bool flag_bad(bool f) { return f; }
template <class T> __device__ __forceinline__ bool flag_bad(T f) { return !(f > T(0)); }
template <int D>
__device__ __forceinline__ void lf_flux2(const C *L, const C *R, C gamma, C gm1, C *G, FaceFlag &bad)
{
    C rL = rcp(L[0]), rR = rcp(R[0]);
    C uL = L[1 + D] * rL, uR = R[1 + D] * rR;
    C pL = gm1 * (L[4] - C(0.5) * ((L[1] * L[1] + L[2] * L[2] + L[3] * L[3]) * rL));
    C pR = gm1 * (R[4] - C(0.5) * ((R[1] * R[1] + R[2] * R[2] + R[3] * R[3]) * rR));
    flag_face(bad, L[0], R[0], pL, pR);
    C aL = fabs(uL) + sqrt_c(gamma * pL * rL);
    C aR = fabs(uR) + sqrt_c(gamma * pR * rR);
    C lam = fmax(aL, aR);  // a NaN speed comes with a flagged face
    C PL = pL + L[5], PR = pR + R[5];
    G[0] = (L[1 + D] + R[1 + D]) - lam * (R[0] - L[0]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C f = L[1 + a] * uL + R[1 + a] * uR;
        if (a == D) f += PL + PR;
        G[1 + a] = f - lam * (R[1 + a] - L[1 + a]);
    }
    G[4] = ((L[4] + PL) * uL + (R[4] + PR) * uR) - lam * (R[4] - L[4]);
}

// wave speed max_d |u_d| + c at a cell
__device__ __forceinline__ C cell_speed(C rho, C mx, C my, C mz, C E, C gamma, C gm1)
{
    C r = rcp(rho);
    C p = gm1 * (E - C(0.5) * (mx * mx + my * my + mz * mz) * r);
    C um = fmax(fabs(mx), fmax(fabs(my), fabs(mz))) * r;
    return um + sqrt_c(gamma * p * r);
}

// block-wide NaN-propagating max of v; thread 0 of the block gets the result
template <int NT>
__device__ __forceinline__ double block_max(double v)
{
    __shared__ double red[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < NT / 32; w++) v = nanmax(v, red[w]);
    }
    return v;
}

// ------------------------------------------------ 16-bit RK combination
// The stage combination v = qn + w ((qs - qn) + dt L) is specified in FP64
// and then rounded to the 16-bit storage format. FP64 runs at a small
// fraction of the FP32 rate on this GPU, so it is evaluated in FP32 with a
// rigorous bound e on |v32 - v64|:
//   d = RN(qs - qn), p = RN(dt32 L + d), v = RN(w32 p + qn) with dt32, w32
//   the FP32 roundings of dt, w (w <= 1) gives, to first order,
//   |v32 - v64| <= 2^-24 (|v| + 3 |p| + 2 |d|) <= 2^-22 (|v| + |p| + |d|),
//   the slack covering the FP64 evaluation's own rounding and the FP32
//   evaluation of e; where a rounding result is an FP32 subnormal its error
//   is absolute (at most 2^-150), so e adds 2^-148 for the three roundings.
// So v64 lies in [RD(v32 - e), RU(v32 + e)] (directed FP32 roundings).
// Rounding to nearest-even is monotone: when both ends of that interval round
// to the same storage value (with -0 equal to +0), so does v64. Both ends are
// converted by one packed conversion and compared as a pair. Otherwise (for
// smooth data, about e / spacing of the values, well under one in a
// thousand) the combination is redone in FP64. The stored value therefore
// always equals the FP64 evaluation rounded to nearest-even, with zeros
// stored as +0.
template <typename T> struct Narrow;
template <> struct Narrow<__half> {
    using T2 = __half2;
    static __device__ __forceinline__ __half rn(double v) { return __double2half(v); }
    // (RN(a), RN(b)) in the low and high halves, one conversion
    static __device__ __forceinline__ __half2 rn2(float a, float b) { return __floats2half2_rn(a, b); }
    static __device__ __forceinline__ bool eq2(__half2 a, __half2 b) { return __hbeq2(a, b); }
    static __device__ __forceinline__ __half2 swap(__half2 a) { return __lowhigh2highlow(a); }
    static __device__ __forceinline__ __half lo(__half2 a) { return __low2half(a); }
    static __device__ __forceinline__ __half hi(__half2 a) { return __high2half(a); }
    // zeros are stored as +0 (-0 + +0 = +0 under round-to-nearest)
    static __device__ __forceinline__ __half canon(__half h) { return __hadd(h, __ushort_as_half(0)); }
    static __device__ __forceinline__ __half2 canon2(__half2 h)
    {
        return __hadd2(h, __halves2half2(__ushort_as_half(0), __ushort_as_half(0)));
    }
};
template <> struct Narrow<__nv_bfloat16> {
    using T2 = __nv_bfloat162;
    static __device__ __forceinline__ __nv_bfloat16 rn(double v) { return __double2bfloat16(v); }
    static __device__ __forceinline__ __nv_bfloat162 rn2(float a, float b) { return __floats2bfloat162_rn(a, b); }
    static __device__ __forceinline__ bool eq2(__nv_bfloat162 a, __nv_bfloat162 b) { return __hbeq2(a, b); }
    static __device__ __forceinline__ __nv_bfloat162 swap(__nv_bfloat162 a) { return __lowhigh2highlow(a); }
    static __device__ __forceinline__ __nv_bfloat16 lo(__nv_bfloat162 a) { return __low2bfloat16(a); }
    static __device__ __forceinline__ __nv_bfloat16 hi(__nv_bfloat162 a) { return __high2bfloat16(a); }
    static __device__ __forceinline__ __nv_bfloat16 canon(__nv_bfloat16 h)
    {
        return __hadd(h, __ushort_as_bfloat16(0));
    }
    static __device__ __forceinline__ __nv_bfloat162 canon2(__nv_bfloat162 h)
    {
        return __hadd2(h, __halves2bfloat162(__ushort_as_bfloat16(0), __ushort_as_bfloat16(0)));
    }
};

// FP64 evaluation, out of line so that only the rare lanes that need it run
// FP64 instructions
template <typename T>
__device__ __noinline__ T rk_fp64(float qn, float qs, float L, double dt, double w)
{
    double vd = __dadd_rn(double(qn),
                          __dmul_rn(w, __dadd_rn(__dsub_rn(double(qs), double(qn)),
                                                 __dmul_rn(dt, double(L)))));
    return Narrow<T>::canon(Narrow<T>::rn(vd));
}

// FP32 evaluation v of one combination and the bound e on |v - v64|
__device__ __forceinline__ float rk_eval32(float qn, float qs, float L, float dt32, float w32, float &e)
{
    float d = __fsub_rn(qs, qn);
    float pp = __fmaf_rn(dt32, L, d);
    float v = __fmaf_rn(w32, pp, qn);
    // relative rounding errors, plus 2^-148 for the three roundings whose
    // results may be FP32 subnormals (absolute error up to 2^-150 each)
    e = __fmaf_rn(fabsf(v) + fabsf(pp) + fabsf(d), 0x1p-22f, 0x1p-148f);
    return v;
}

// Two combinations rounded to the storage format (low, high); ok = false
// when either rounding could differ from the FP64 evaluation's
template <typename T>
__device__ __forceinline__ typename Narrow<T>::T2 rk_narrow_pair(float qn0, float qs0, float L0, float qn1,
                                                                 float qs1, float L1, float dt32, float w32,
                                                                 bool &ok)
{
    using NR = Narrow<T>;
    float e0, e1;
    const float v0 = rk_eval32(qn0, qs0, L0, dt32, w32, e0);
    const float v1 = rk_eval32(qn1, qs1, L1, dt32, w32, e1);
    const typename NR::T2 a = NR::rn2(__fsub_rd(v0, e0), __fsub_rd(v1, e1));
    const typename NR::T2 b = NR::rn2(__fadd_ru(v0, e0), __fadd_ru(v1, e1));
    ok = NR::eq2(a, b);
    return NR::canon2(b);
}

// One combination rounded to the storage format; ok as for the pair
template <typename T>
__device__ __forceinline__ T rk_narrow_one(float qn, float qs, float L, float dt32, float w32, bool &ok)
{
    using NR = Narrow<T>;
    float e;
    const float v = rk_eval32(qn, qs, L, dt32, w32, e);
    const typename NR::T2 x = NR::rn2(__fsub_rd(v, e), __fadd_ru(v, e));
    ok = NR::eq2(x, NR::swap(x));
    return NR::canon(NR::hi(x));
}

constexpr bool kNarrow = sizeof(S) == 2;

// The 16-bit stage combination of one cell's five values: two pairs and a
// single value, one branch per cell for the rare FP64 re-evaluations (a pair
// that failed is redone in FP64 for both of its values)
template <typename T>
__device__ __forceinline__ void rk_narrow5(const C qn[5], const C qs[5], const C L[5], C dt32, double dt,
                                           C w32, double w, T h[5])
{
    using NR = Narrow<T>;
    bool ok01, ok23, ok4;
    const typename NR::T2 h01 = rk_narrow_pair<T>(qn[0], qs[0], L[0], qn[1], qs[1], L[1], dt32, w32, ok01);
    const typename NR::T2 h23 = rk_narrow_pair<T>(qn[2], qs[2], L[2], qn[3], qs[3], L[3], dt32, w32, ok23);
    h[0] = NR::lo(h01);
    h[1] = NR::hi(h01);
    h[2] = NR::lo(h23);
    h[3] = NR::hi(h23);
    h[4] = rk_narrow_one<T>(qn[4], qs[4], L[4], dt32, w32, ok4);
    if (!(ok01 && ok23 && ok4)) {
#pragma unroll
        for (int u = 0; u < 5; u++)
            if (!(u < 2 ? ok01 : u < 4 ? ok23 : ok4)) h[u] = rk_fp64<T>(qn[u], qs[u], L[u], dt, w);
    }
}

// Stage combination of the five conserved values of one cell, stored at
// offset c of each output field; returns the stored values in type C.
__device__ __forceinline__ void rk_store5(const Fout<5> &out, idx c, const C qn[5], const C qs[5],
                                          const C L[5], C dt32, double dt, C w32, double w, C o[5])
{
    if constexpr (kNarrow) {
        S h[5];
        rk_narrow5<S>(qn, qs, L, dt32, dt, w32, w, h);
#pragma unroll
        for (int u = 0; u < 5; u++) {
            out.p[u][c] = h[u];
            o[u] = cv(h[u]);
        }
    } else {
#pragma unroll
        for (int u = 0; u < 5; u++) o[u] = stc(out.p[u] + c, qn[u] + w32 * ((qs[u] - qn[u]) + dt32 * L[u]));
    }
}

// Block coordinates of a stage kernel's body: those of the launch itself, or,
// in a grouped launch over several instances, the block's place in its own
// instance's grid.
struct BlockPos {
    int x, y, z, gx, gy;
    static __device__ __forceinline__ BlockPos of_launch()
    {
        return {(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x, (int)gridDim.y};
    }
    // the l-th block of a grid of gx x gy x * blocks
    static __device__ __forceinline__ BlockPos of_index(int l, int gx, int gy)
    {
        return {l % gx, (l / gx) % gy, l / (gx * gy), gx, gy};
    }
};

// --------------------------------------------- tiles of the 7-point kernels
constexpr int BX = 32, BY = 8, BT = BX * BY;
constexpr int HX = BX + 2, HY = BY + 2;   // plane tile with a halo of 1
constexpr int NHALO1 = 2 * BX + 2 * BY;   // halo cells (corners are never read)

// position of halo cell e (0 <= e < NHALO1) in the HX x HY tile
__device__ __forceinline__ void halo1_cell(int e, int &lx, int &ly)
{
    if (e < BX) { lx = 1 + e; ly = 0; }
    else if (e < 2 * BX) { lx = 1 + e - BX; ly = HY - 1; }
    else if (e < 2 * BX + BY) { lx = 0; ly = 1 + e - 2 * BX; }
    else { lx = HX - 1; ly = 1 + e - 2 * BX - BY; }
}

// --------------------------------------------------------------- source
// z-index of plane kk in [-1, nz]: periodic wrap or zero-gradient clamp
__device__ __forceinline__ int zmap(int kk, const Geom &g)
{
    return kk < 0 ? (g.bc[4] == BC_PERIODIC ? kk + g.nz : 0)
                  : (kk >= g.nz ? (g.bc[5] == BC_PERIODIC ? kk - g.nz : g.nz - 1) : kk);
}

// u = m / rho of the cell at in-plane offset f of plane kk (kk may leave the
// domain through -z/+z: periodic wrap, zero-gradient clamp or the jet blend);
// *rho_s gets the cell's (unblended) density
template <bool HASD>
__device__ __forceinline__ void col_u(const QIn &q, const Geom &g, const C *W, const C *J, idx f,
                                      int kk, C u[3], C *rho_s = nullptr)
{
    idx c = ck((idx)map_axis(kk, g.nz, g.bc[4], g.bc[5]) * (idx)g.plane + f, g.n);
    C rho = ldq<HASD>(q, 0, c), m0 = ldq<HASD>(q, 1, c), m1 = ldq<HASD>(q, 2, c), m2 = ldq<HASD>(q, 3, c);
    if (rho_s) *rho_s = rho;
    if (kk < 0 && g.bc[4] == BC_INFLOW) {
        idx pl = (idx)g.plane;
        f = ck(f, g.plane);
        C w = C(1) - W[f];
        rho = fma_rn(w, rho, J[f]);
        m0 = fma_rn(w, m0, J[pl + f]);
        m1 = fma_rn(w, m1, J[2 * pl + f]);
        m2 = fma_rn(w, m2, J[3 * pl + f]);
    }
    // products rounded before they are differenced: equal neighbours give an exact 0
    C r = rcp(rho);
    u[0] = mul_rn(m0, r);
    u[1] = mul_rn(m1, r);
    u[2] = mul_rn(m2, r);
}

// b = alpha [tr(G^2) + tr(G)^2] (Eq. igrelliptic) from the undivided central
// differences D = 2 dx G of u, with alpha_s = alpha / (2 dx)^2:
//   b = alpha_s [sum_ab D_ab D_ba + (sum_a D_aa)^2],
// in one fixed order of rounded operations, so that the two forms of the
// source kernel give the same bits
__device__ __forceinline__ C source_b(const C (&D)[3][3], C alpha_s)
{
    const C tr = add_rn(add_rn(D[0][0], D[1][1]), D[2][2]);
    C sq = mul_rn(D[0][0], D[0][0]);
    sq = fma_rn(D[1][1], D[1][1], sq);
    sq = fma_rn(D[2][2], D[2][2], sq);
    C x = mul_rn(D[0][1], D[1][0]);
    x = fma_rn(D[0][2], D[2][0], x);
    x = fma_rn(D[1][2], D[2][1], x);
    const C tr2 = fma_rn(C(2), x, sq);  // sum_ab D_ab D_ba
    return mul_rn(alpha_s, fma_rn(tr, tr, tr2));
}

// grad u by central differences from a shared plane tile U (x, y) and the
// column's registers (z); b from source_b. In the increment modes the kernel
// also stores the stage's density rounded to the storage type (rho_out),
// which the Jacobi sweeps of the stage read.
template <bool HASD>
__device__ __forceinline__ void source_body(const QIn q, S *__restrict__ b, S *__restrict__ rho_out,
                                            const Geom g, C alpha_s, const C *W, const C *J, int zc,
                                            const BlockPos bp)
{
    __shared__ C U[3][HY][HX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int x0 = bp.x * BX, y0 = bp.y * BY;
    const int i = x0 + tx, j = y0 + ty;
    const bool active = i < g.nx && j < g.ny;
    const int k0 = bp.z * zc, k1 = min(g.nz, k0 + zc);
    const idx pl = (idx)g.plane;
    // the own slot of the tile holds the mapped cell (it is a neighbour of
    // active cells even when this thread is outside the domain)
    const idx f = (idx)(map_axis(j, g.ny, g.bc[2], g.bc[3]) * g.nx + map_axis(i, g.nx, g.bc[0], g.bc[1]));
    const bool hv = tid < NHALO1;
    int hs = 0;
    idx hf = 0;
    if (hv) {
        int lx, ly;
        halo1_cell(tid, lx, ly);
        hs = ly * HX + lx;
        hf = (idx)(map_axis(y0 + ly - 1, g.ny, g.bc[2], g.bc[3]) * g.nx +
                   map_axis(x0 + lx - 1, g.nx, g.bc[0], g.bc[1]));
    }
    C um[3], u0[3], up[3];
    C rho0 = C(1), rhop = C(1);  // density of the column at k and k + 1 (increment modes)
    col_u<HASD>(q, g, W, J, f, k0 - 1, um);
    col_u<HASD>(q, g, W, J, f, k0, u0, &rho0);
    // raw values one iteration ahead (loads overlap the previous plane's work):
    // the column at k + 1 and the halo at k (planes >= 0 need no jet blend)
    QRaw nc[4], nh[4];
    auto raw4 = [&](idx off, int kk, QRaw v[4]) {
        idx c = ck((idx)zmap(kk, g) * pl + off, g.n);
#pragma unroll
        for (int a = 0; a < 4; a++) v[a] = ldqr<HASD>(q, a, c);
    };
    raw4(f, k0 + 1, nc);
    if (hv) raw4(hf, k0, nh);
    for (int k = k0; k < k1; k++) {
        rhop = cvq<HASD>(nc[0]);
        C r = rcp(rhop);
#pragma unroll
        for (int a = 0; a < 3; a++) up[a] = mul_rn(cvq<HASD>(nc[1 + a]), r);
        C hu[3];
        if (hv) {
            C rh = rcp(cvq<HASD>(nh[0]));
#pragma unroll
            for (int a = 0; a < 3; a++) hu[a] = mul_rn(cvq<HASD>(nh[1 + a]), rh);
        }
        if (k + 1 < k1) {
            raw4(f, k + 2, nc);
            if (hv) raw4(hf, k + 1, nh);
        }
        __syncthreads();  // readers of the previous plane are done
#pragma unroll
        for (int a = 0; a < 3; a++) {
            U[a][ty + 1][tx + 1] = u0[a];
            if (hv) (&U[a][0][0])[cks(hs, HY * HX)] = hu[a];
        }
        __syncthreads();
        if (active) {
            C D[3][3];  // D[a][c]: undivided central difference of u_a along c
#pragma unroll
            for (int a = 0; a < 3; a++) {
                D[a][0] = U[a][ty + 1][tx + 2] - U[a][ty + 1][tx];
                D[a][1] = U[a][ty + 2][tx + 1] - U[a][ty][tx + 1];
                D[a][2] = up[a] - um[a];
            }
            stc(CKP(b + (idx)k * pl + (idx)(j * g.nx + i), b, g.n), source_b(D, alpha_s));
            if constexpr (kInc) stc(CKP(rho_out + (idx)k * pl + (idx)(j * g.nx + i), rho_out, g.n), rho0);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            um[a] = u0[a];
            u0[a] = up[a];
        }
        rho0 = rhop;
    }
}
template <bool HASD>
__global__ void __launch_bounds__(BT) k_source(QIn q, S *__restrict__ b, S *__restrict__ rho_out, Geom g,
                                                C alpha_s, const C *W, const C *J, int zc)
{
    source_body<HASD>(q, b, rho_out, g, alpha_s, W, J, zc, BlockPos::of_launch());
}


// --------------------------------------------------------------- Jacobi
// One sweep s_out = (b + beta sum_f c_f s_nb) / (1/rho + beta sum_f c_f),
// c_f = (1/rho_i + 1/rho_nb)/2; a face on a non-periodic boundary carries no
// term. 1/rho and sigma of plane k sit in a shared tile with a halo of 1;
// the z-neighbours stay in registers.
//
// colour >= 0 makes it one half of a red-black Gauss-Seidel sweep, in place
// (s_in == s_out): only the cells with (i + j + k) % 2 == colour change.
// Their neighbours all have the other colour (periodic axes have even
// length), which no thread writes during the launch, so every updated value
// is the same whatever the order of execution; values read from cells of
// the updated colour feed only results that are discarded.

// One update of one cell: e[f] the face factor (beta / 2, 0 for a face on a
// non-periodic boundary), rn[f] the reciprocal density and sn[f] Sigma of
// the neighbour across face f, faces in the order -x, +x, -y, +y, -z, +z. A
// fixed order of rounded operations, lane for lane that of the packed form
// of k_jacobi_v4, so that every form of the sweep gives the same bits.
__device__ __forceinline__ C jacobi_cell(C r0, const C (&e)[6], const C (&rn)[6], const C (&sn)[6], C bv)
{
    C c[6];
#pragma unroll
    for (int f = 0; f < 6; f++) c[f] = mul_rn(e[f], add_rn(r0, rn[f]));
    C diag = r0;
#pragma unroll
    for (int f = 0; f < 6; f++) diag = add_rn(diag, c[f]);
    C off = mul_rn(c[0], sn[0]);
#pragma unroll
    for (int f = 1; f < 6; f++) off = fma_rn(c[f], sn[f], off);
    return quot(add_rn(bv, off), diag);
}

__device__ __forceinline__ void jacobi_body(const S *__restrict__ q, const S *__restrict__ b, const S *sin,
                                            S *sout, const Geom g, C beta, int zc, int colour,
                                            const BlockPos bp)
{
    __shared__ C R[HY][HX], SG[HY][HX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int x0 = bp.x * BX, y0 = bp.y * BY;
    const int i = x0 + tx, j = y0 + ty;
    const bool active = i < g.nx && j < g.ny;
    const int k0 = bp.z * zc, k1 = min(g.nz, k0 + zc);
    const idx pl = (idx)g.plane;
    const idx f = (idx)(map_axis(j, g.ny, g.bc[2], g.bc[3]) * g.nx + map_axis(i, g.nx, g.bc[0], g.bc[1]));
    const bool hv = tid < NHALO1;
    int hs = 0;
    idx hf = 0;
    if (hv) {
        int lx, ly;
        halo1_cell(tid, lx, ly);
        hs = ly * HX + lx;
        hf = (idx)(map_axis(y0 + ly - 1, g.ny, g.bc[2], g.bc[3]) * g.nx +
                   map_axis(x0 + lx - 1, g.nx, g.bc[0], g.bc[1]));
    }
    const C hb = C(0.5) * beta;
    // a face term exists unless the face is a non-periodic domain boundary
    const C exm = (i > 0 || g.bc[0] == BC_PERIODIC) ? hb : C(0);
    const C exp_ = (i < g.nx - 1 || g.bc[1] == BC_PERIODIC) ? hb : C(0);
    const C eym = (j > 0 || g.bc[2] == BC_PERIODIC) ? hb : C(0);
    const C eyp = (j < g.ny - 1 || g.bc[3] == BC_PERIODIC) ? hb : C(0);
    C rm, sm, r0, s0, rp, sp;
    {
        idx c = ck((idx)zmap(k0 - 1, g) * pl + f, g.n);
        rm = rcp(ldc(q + c));
        sm = ldc(sin + c);
        c = ck((idx)k0 * pl + f, g.n);
        r0 = rcp(ldc(q + c));
        s0 = ldc(sin + c);
    }
    // raw values one iteration ahead: column at k + 1, halo and b at k
    S ncr, ncs, nhr = S(1.0f), nhs = S(0.0f), nb;
    auto pre = [&](int kk) {
        idx c = ck((idx)zmap(kk + 1, g) * pl + f, g.n);
        ncr = ldr(q + c);
        ncs = ldr(sin + c);
        if (hv) {
            idx h = ck((idx)kk * pl + hf, g.n);
            nhr = ldr(q + h);
            nhs = ldr(sin + h);
        }
        nb = ldr(CKP(b + (idx)kk * pl + f, b, g.n));
    };
    pre(k0);
    for (int k = k0; k < k1; k++) {
        rp = rcp(cv(ncr));
        sp = cv(ncs);
        C hr = rcp(cv(nhr)), hsg = cv(nhs), bv = cv(nb);
        if (k + 1 < k1) pre(k + 1);
        __syncthreads();
        R[ty + 1][tx + 1] = r0;
        SG[ty + 1][tx + 1] = s0;
        if (hv) {
            (&R[0][0])[cks(hs, HY * HX)] = hr;
            (&SG[0][0])[cks(hs, HY * HX)] = hsg;
        }
        __syncthreads();
        if (active) {
            const C ezm = (k > 0 || g.bc[4] == BC_PERIODIC) ? hb : C(0);
            const C ezp = (k < g.nz - 1 || g.bc[5] == BC_PERIODIC) ? hb : C(0);
            // faces in the order -x, +x, -y, +y, -z, +z
            const C e[6] = {exm, exp_, eym, eyp, ezm, ezp};
            const C rn[6] = {R[ty + 1][tx], R[ty + 1][tx + 2], R[ty][tx + 1], R[ty + 2][tx + 1], rm, rp};
            const C sn[6] = {SG[ty + 1][tx], SG[ty + 1][tx + 2], SG[ty][tx + 1], SG[ty + 2][tx + 1], sm, sp};
            if (colour < 0 || ((i + j + k) & 1) == colour)
                stc(CKP(sout + (idx)k * pl + (idx)(j * g.nx + i), sout, g.n), jacobi_cell(r0, e, rn, sn, bv));
        }
        rm = r0; sm = s0;
        r0 = rp; s0 = sp;
    }
}
__global__ void __launch_bounds__(BT) k_jacobi(const S *__restrict__ q, const S *__restrict__ b,
                                                const S *sin, S *sout, Geom g, C beta, int zc,
                                                int colour)
{
    jacobi_body(q, b, sin, sout, g, beta, zc, colour, BlockPos::of_launch());
}


// Vector form of the sweep for rows whose length is a multiple of 4: each
// thread owns 4 consecutive cells of a row (one 4-wide load/store per field),
// takes x-neighbours from its own registers, y-neighbours as aligned 4-wide
// shared loads. Same arithmetic per cell, in the same order, as k_jacobi.
__device__ __forceinline__ void ld4(const double *p, double v[4])
{
    double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const float *p, float v[4])
{
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const __half *p, float v[4])
{
    uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&a.x));
    float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&a.y));
    v[0] = lo.x; v[1] = lo.y; v[2] = hi.x; v[3] = hi.y;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16 *p, float v[4])
{
    uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
    float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&a.x));
    float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&a.y));
    v[0] = lo.x; v[1] = lo.y; v[2] = hi.x; v[3] = hi.y;
}
__device__ __forceinline__ void st4(double *p, const double v[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float *p, const float v[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(__half *p, const float v[4])
{
    __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}
__device__ __forceinline__ void st4(__nv_bfloat16 *p, const float v[4])
{
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}

// four consecutive stored values kept raw after one vector load
template <typename T> struct Vec4;
template <> struct Vec4<double> { double2 a, b; };
template <> struct Vec4<float> { float4 a; };
template <> struct Vec4<__half> { uint2 a; };
template <> struct Vec4<__nv_bfloat16> { uint2 a; };
using V4 = Vec4<S>;

__device__ __forceinline__ Vec4<double> ld4r(const double *p)
{
    return {__ldg(reinterpret_cast<const double2 *>(p)), __ldg(reinterpret_cast<const double2 *>(p) + 1)};
}
__device__ __forceinline__ Vec4<float> ld4r(const float *p) { return {__ldg(reinterpret_cast<const float4 *>(p))}; }
__device__ __forceinline__ Vec4<__half> ld4r(const __half *p) { return {__ldg(reinterpret_cast<const uint2 *>(p))}; }
__device__ __forceinline__ Vec4<__nv_bfloat16> ld4r(const __nv_bfloat16 *p)
{
    return {__ldg(reinterpret_cast<const uint2 *>(p))};
}
__device__ __forceinline__ void cv4(const Vec4<double> &v, double o[4])
{
    o[0] = v.a.x; o[1] = v.a.y; o[2] = v.b.x; o[3] = v.b.y;
}
__device__ __forceinline__ void cv4(const Vec4<float> &v, float o[4])
{
    o[0] = v.a.x; o[1] = v.a.y; o[2] = v.a.z; o[3] = v.a.w;
}
union H2U { unsigned u; __half2 h; };
union B2U { unsigned u; __nv_bfloat162 h; };
__device__ __forceinline__ void cv4(const Vec4<__half> &v, float o[4])
{
    H2U lo, hi;
    lo.u = v.a.x;
    hi.u = v.a.y;
    float2 a = __half22float2(lo.h), b = __half22float2(hi.h);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void cv4(const Vec4<__nv_bfloat16> &v, float o[4])
{
    B2U lo, hi;
    lo.u = v.a.x;
    hi.u = v.a.y;
    float2 a = __bfloat1622float2(lo.h), b = __bfloat1622float2(hi.h);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ Vec4<double> pack4(double a, double b, double c, double d)
{
    return {make_double2(a, b), make_double2(c, d)};
}
__device__ __forceinline__ Vec4<float> pack4(float a, float b, float c, float d) { return {make_float4(a, b, c, d)}; }
__device__ __forceinline__ Vec4<__half> pack4(__half a, __half b, __half c, __half d)
{
    return {make_uint2(__half_as_ushort(a) | ((unsigned)__half_as_ushort(b) << 16),
                       __half_as_ushort(c) | ((unsigned)__half_as_ushort(d) << 16))};
}
__device__ __forceinline__ Vec4<__nv_bfloat16> pack4(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c,
                                                      __nv_bfloat16 d)
{
    return {make_uint2(__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16),
                       __bfloat16_as_ushort(c) | ((unsigned)__bfloat16_as_ushort(d) << 16))};
}

constexpr int VX = 4, TXV = BX * VX;        // 128 cells per tile row

// 4 consecutive values of a 16-byte aligned shared row (one 128-bit access
// for FP32, two for FP64; scalar accesses at stride 4 would conflict 4-way)
__device__ __forceinline__ void sh_st4(float *p, const float v[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sh_st4(double *p, const double v[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void sh_ld4(const float *p, float v[4])
{
    float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void sh_ld4(const double *p, double v[4])
{
    double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
constexpr int HXV = TXV + 2 * VX;           // interior at column VX (16-byte aligned)
constexpr int NYH = 2 * BX, NXH = 2 * BY;   // 4-wide y-halo tasks, scalar x-halo tasks

// The update of four cells (x-consecutive, of one row) as two packed FP32x2
// pairs, cells (0, 1) and (2, 3); lane for lane the sequence of jacobi_cell
// (faces -x, +x, -y, +y, -z, +z). r0, s0: the cells; rl, sl / rr, sr: the
// x-neighbours left of cell 0 and right of cell 3; ry0 / ry1 (sy0 / sy1):
// the rows below / above; rm, sm / rp, sp: the planes below / above; bv:
// the source; hb = beta / 2 and the face factors of the four cells' outer
// faces (the inner x-faces are always hb).
__device__ __forceinline__ void jacobi4_packed(const float (&r0)[4], const float (&s0)[4], float rl, float sl,
                                               float rr, float sr, const float (&ry0)[4], const float (&ry1)[4],
                                               const float (&sy0)[4], const float (&sy1)[4], const float (&rm)[4],
                                               const float (&sm)[4], const float (&rp)[4], const float (&sp)[4],
                                               const float (&bv)[4], float hb, float exm, float exp_, float eym,
                                               float eyp, float ezm, float ezp, float (&o)[4])
{
    const float2 r01 = make_float2(r0[0], r0[1]), r23 = make_float2(r0[2], r0[3]), r12 = make_float2(r0[1], r0[2]);
    const float2 s12 = make_float2(s0[1], s0[2]);
    const float2 rxm[2] = {make_float2(rl, r0[0]), r12}, rxp[2] = {r12, make_float2(r0[3], rr)};
    const float2 sxm[2] = {make_float2(sl, s0[0]), s12}, sxp[2] = {s12, make_float2(s0[3], sr)};
    const float2 exmp[2] = {make_float2(exm, hb), make_float2(hb, hb)};
    const float2 expp[2] = {make_float2(hb, hb), make_float2(hb, exp_)};
    const float2 rc[2] = {r01, r23};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int c = 2 * h;
        float2 c0 = pmul(exmp[h], padd(rc[h], rxm[h]));
        float2 c1 = pmul(expp[h], padd(rc[h], rxp[h]));
        float2 c2 = pmul(make_float2(eym, eym), padd(rc[h], make_float2(ry0[c], ry0[c + 1])));
        float2 c3 = pmul(make_float2(eyp, eyp), padd(rc[h], make_float2(ry1[c], ry1[c + 1])));
        float2 c4 = pmul(make_float2(ezm, ezm), padd(rc[h], make_float2(rm[c], rm[c + 1])));
        float2 c5 = pmul(make_float2(ezp, ezp), padd(rc[h], make_float2(rp[c], rp[c + 1])));
        float2 diag = padd(padd(padd(padd(padd(padd(rc[h], c0), c1), c2), c3), c4), c5);
        float2 off = pmul(c0, sxm[h]);
        off = pfma(c1, sxp[h], off);
        off = pfma(c2, make_float2(sy0[c], sy0[c + 1]), off);
        off = pfma(c3, make_float2(sy1[c], sy1[c + 1]), off);
        off = pfma(c4, make_float2(sm[c], sm[c + 1]), off);
        off = pfma(c5, make_float2(sp[c], sp[c + 1]), off);
        float2 num = padd(make_float2(bv[c], bv[c + 1]), off);
        float2 res = pmul(num, make_float2(rcp(diag.x), rcp(diag.y)));
        o[c] = res.x;
        o[c + 1] = res.y;
    }
}
__device__ __forceinline__ void jacobi4_packed(const double (&)[4], const double (&)[4], double, double, double,
                                               double, const double (&)[4], const double (&)[4],
                                               const double (&)[4], const double (&)[4], const double (&)[4],
                                               const double (&)[4], const double (&)[4], const double (&)[4],
                                               const double (&)[4], double, double, double, double, double,
                                               double, double, double (&)[4])
{
}  // FP64 takes the scalar cells; this overload only lets the FP32 call compile in the FP64 build

// 4 raw values of field a at cells (x .. x+3) of row-plane offset rowoff:
// one 4-wide load when the cells lie inside the row, mapped single loads otherwise
template <class T>
__device__ __forceinline__ Vec4<T> ld4_mapped(const T *__restrict__ a, const Geom &g, idx rowoff, int x)
{
    if (x + VX <= g.nx) return ld4r(CKP4(a + rowoff + x, a, g.n));
    T v[VX];
#pragma unroll
    for (int c = 0; c < VX; c++)
        v[c] = __ldg(CKP(a + rowoff + (idx)map_axis(x + c, g.nx, g.bc[0], g.bc[1]), a, g.n));
    return pack4(v[0], v[1], v[2], v[3]);
}

// 4 raw state values (cells x .. x+3) and their stage values, as StateIO
struct QRaw4Inc {
    Vec4<QB> b;
    V4 d;
};
template <bool INC> struct StateIO4;
template <> struct StateIO4<false> {  // (used where the state has the storage type)
    using Raw = V4;
    template <bool HASD>
    static __device__ __forceinline__ V4 ld(const QIn &q, int u, const Geom &g, idx rowoff, int x)
    {
        return ld4_mapped(reinterpret_cast<const S *>(q.b[u]), g, rowoff, x);
    }
    template <bool HASD> static __device__ __forceinline__ void val(const V4 &r, C o[4]) { cv4(r, o); }
    // cells off .. off+3 inside one row: one 4-wide load
    template <bool HASD>
    static __device__ __forceinline__ V4 ldd(const QIn &q, int u, const Geom &g, idx off)
    {
        const S *f = reinterpret_cast<const S *>(q.b[u]);
        return ld4r(CKP4(f + off, f, g.n));
    }
};
template <> struct StateIO4<true> {
    using Raw = QRaw4Inc;
    template <bool HASD>
    static __device__ __forceinline__ QRaw4Inc ld(const QIn &q, int u, const Geom &g, idx rowoff, int x)
    {
        QRaw4Inc r;
        r.b = ld4_mapped(q.b[0] + u * q.fs, g, rowoff, x);
        if constexpr (HASD) r.d = ld4_mapped(q.d[0] + u * q.fs, g, rowoff, x);
        return r;
    }
    template <bool HASD>
    static __device__ __forceinline__ QRaw4Inc ldd(const QIn &q, int u, const Geom &g, idx off)
    {
        QRaw4Inc r;
        r.b = ld4r(CKP4(q.b[0] + u * q.fs + off, q.b[0], 5 * g.n));
        if constexpr (HASD) r.d = ld4r(CKP4(q.d[0] + u * q.fs + off, q.d[0], 5 * g.n));
        return r;
    }
    template <bool HASD> static __device__ __forceinline__ void val(const QRaw4Inc &r, C o[4])
    {
        cv4(r.b, o);
        if constexpr (HASD) {
            C d[4];
            cv4(r.d, d);
#pragma unroll
            for (int c = 0; c < 4; c++) o[c] = C(__fadd_rn(float(o[c]), float(d[c])));
        }
    }
};
using QRaw4 = StateIO4<kInc>::Raw;
template <bool HASD>
__device__ __forceinline__ QRaw4 ldq4(const QIn &q, int u, const Geom &g, idx rowoff, int x)
{
    return StateIO4<kInc>::ld<HASD>(q, u, g, rowoff, x);
}
template <bool HASD> __device__ __forceinline__ void cvq4(const QRaw4 &r, C o[4])
{
    StateIO4<kInc>::val<HASD>(r, o);
}

// The four-cell sweep of any block (tiles that cross the grid's edge in x
// or y: lanes past the row's end, rows past the last, mapped loads).
__device__ __forceinline__ void jacobi_v4_edge(const S *__restrict__ q, const S *__restrict__ b, const S *sin,
                                               S *sout, const Geom &g, C beta, int zc, int colour,
                                               const BlockPos &bp, C (*R)[HXV], C (*SG)[HXV])
{
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int x0 = bp.x * TXV, y0 = bp.y * BY;
    const int i0 = x0 + VX * tx, j = y0 + ty;
    const bool active = i0 < g.nx && j < g.ny;
    const int k0 = bp.z * zc, k1 = min(g.nz, k0 + zc);
    const idx pl = (idx)g.plane;
    const idx rowj = (idx)(map_axis(j, g.ny, g.bc[2], g.bc[3]) * g.nx);
    // halo tasks: 4-wide cells of the rows above/below the tile, then single
    // cells left/right of each row
    int htask = tid < NYH ? 0 : (tid < NYH + NXH ? 1 : 2);
    int hsy = 0, hsx = 0, hx = 0;
    idx hrow = 0;
    if (htask == 0) {
        int side = tid / BX, t = tid % BX;
        hsy = side ? HY - 1 : 0;
        hsx = VX + VX * t;
        hx = x0 + VX * t;
        hrow = (idx)(map_axis(y0 + (side ? BY : -1), g.ny, g.bc[2], g.bc[3]) * g.nx);
    } else if (htask == 1) {
        int e = tid - NYH, side = e / BY, r = e % BY;
        hsy = 1 + r;
        hsx = side ? VX + TXV : VX - 1;
        hx = map_axis(side ? x0 + TXV : x0 - 1, g.nx, g.bc[0], g.bc[1]);
        hrow = (idx)(map_axis(y0 + r, g.ny, g.bc[2], g.bc[3]) * g.nx);
    }
    const C hb = C(0.5) * beta;
    const C exm = (i0 > 0 || g.bc[0] == BC_PERIODIC) ? hb : C(0);
    const C exp_ = (i0 + VX - 1 < g.nx - 1 || g.bc[1] == BC_PERIODIC) ? hb : C(0);
    const C eym = (j > 0 || g.bc[2] == BC_PERIODIC) ? hb : C(0);
    const C eyp = (j < g.ny - 1 || g.bc[3] == BC_PERIODIC) ? hb : C(0);

    C rm[VX], sm[VX], r0[VX], s0[VX], rp[VX], sp[VX];
    {
        C t[VX];
        cv4(ld4_mapped(q, g, (idx)zmap(k0 - 1, g) * pl + rowj, i0), t);
        cv4(ld4_mapped(sin, g, (idx)zmap(k0 - 1, g) * pl + rowj, i0), sm);
#pragma unroll
        for (int c = 0; c < VX; c++) rm[c] = rcp(t[c]);
        cv4(ld4_mapped(q, g, (idx)k0 * pl + rowj, i0), t);
        cv4(ld4_mapped(sin, g, (idx)k0 * pl + rowj, i0), s0);
#pragma unroll
        for (int c = 0; c < VX; c++) r0[c] = rcp(t[c]);
    }
    // raw values one iteration ahead: own cells at k + 1, halo and b at k
    V4 ncr, ncs, nb, nhr, nhs;
    S nxr = S(1.0f), nxs = S(0.0f);
    auto pre = [&](int kk) {
        idx pz = (idx)zmap(kk + 1, g) * pl + rowj;
        ncr = ld4_mapped(q, g, pz, i0);
        ncs = ld4_mapped(sin, g, pz, i0);
        if (active) nb = ld4r(CKP4(b + (idx)kk * pl + rowj + (idx)i0, b, g.n));
        if (htask == 0) {
            nhr = ld4_mapped(q, g, (idx)kk * pl + hrow, hx);
            nhs = ld4_mapped(sin, g, (idx)kk * pl + hrow, hx);
        } else if (htask == 1) {
            nxr = ldr(CKP(q + (idx)kk * pl + hrow + hx, q, g.n));
            nxs = ldr(CKP(sin + (idx)kk * pl + hrow + hx, sin, g.n));
        }
    };
    pre(k0);
    for (int k = k0; k < k1; k++) {
        C bv[VX], hr[VX], hsg[VX], t[VX];
        cv4(ncr, t);
        cv4(ncs, sp);
#pragma unroll
        for (int c = 0; c < VX; c++) rp[c] = rcp(t[c]);
        if (active) cv4(nb, bv);
        if (htask == 0) {
            cv4(nhr, t);
            cv4(nhs, hsg);
#pragma unroll
            for (int c = 0; c < VX; c++) hr[c] = rcp(t[c]);
        } else if (htask == 1) {
            hr[0] = rcp(cv(nxr));
            hsg[0] = cv(nxs);
        }
        if (k + 1 < k1) pre(k + 1);
        __syncthreads();
        sh_st4(&R[ty + 1][VX + VX * tx], r0);
        sh_st4(&SG[ty + 1][VX + VX * tx], s0);
        if (htask == 0) {
            sh_st4(&R[cks(hsy, HY)][cks4(hsx, HXV)], hr);
            sh_st4(&SG[cks(hsy, HY)][cks4(hsx, HXV)], hsg);
        } else if (htask == 1) {
            R[cks(hsy, HY)][cks(hsx, HXV)] = hr[0];
            SG[cks(hsy, HY)][cks(hsx, HXV)] = hsg[0];
        }
        __syncthreads();
        if (active) {
            const C ezm = (k > 0 || g.bc[4] == BC_PERIODIC) ? hb : C(0);
            const C ezp = (k < g.nz - 1 || g.bc[5] == BC_PERIODIC) ? hb : C(0);
            const int col = VX + VX * tx;
            C ry0[VX], ry1[VX], sy0[VX], sy1[VX], o[VX];
            sh_ld4(&R[ty][col], ry0);
            sh_ld4(&R[ty + 2][col], ry1);
            sh_ld4(&SG[ty][col], sy0);
            sh_ld4(&SG[ty + 2][col], sy1);
            if constexpr (sizeof(C) == 4) {
                jacobi4_packed(r0, s0, R[ty + 1][col - 1], SG[ty + 1][col - 1], R[ty + 1][col + VX],
                               SG[ty + 1][col + VX], ry0, ry1, sy0, sy1, rm, sm, rp, sp, bv, hb, exm, exp_, eym,
                               eyp, ezm, ezp, o);
#pragma unroll
                for (int c = 0; c < VX; c++)
                    if (colour >= 0 && ((i0 + c + j + k) & 1) != colour) o[c] = s0[c];
            } else {
#pragma unroll
                for (int c = 0; c < VX; c++) {
                    C rxm = c > 0 ? r0[c - 1] : R[ty + 1][col - 1];
                    C sxm = c > 0 ? s0[c - 1] : SG[ty + 1][col - 1];
                    C rxp = c < VX - 1 ? r0[c + 1] : R[ty + 1][col + VX];
                    C sxp = c < VX - 1 ? s0[c + 1] : SG[ty + 1][col + VX];
                    // faces in the order -x, +x, -y, +y, -z, +z
                    const C e[6] = {c > 0 ? hb : exm, c < VX - 1 ? hb : exp_, eym, eyp, ezm, ezp};
                    const C rn[6] = {rxm, rxp, ry0[c], ry1[c], rm[c], rp[c]};
                    const C sn[6] = {sxm, sxp, sy0[c], sy1[c], sm[c], sp[c]};
                    o[c] = jacobi_cell(r0[c], e, rn, sn, bv[c]);
                    // red-black half-sweep: cells of the other colour keep (and
                    // write back) the value read at the start of the launch
                    if (colour >= 0 && ((i0 + c + j + k) & 1) != colour) o[c] = s0[c];
                }
            }
            st4(CKP4(sout + (idx)k * pl + (idx)(j * g.nx + i0), sout, g.n), o);
        }
#pragma unroll
        for (int c = 0; c < VX; c++) {
            rm[c] = r0[c]; sm[c] = s0[c];
            r0[c] = rp[c]; s0[c] = sp[c];
        }
    }
}
// The four-cell sweep of a block whose tile lies inside the grid in x and y
// (FP32 arithmetic): every lane owns four cells of a row, its loads are
// whole 4-wide rows, and the halo offsets are mapped once. Warps 0 and 1
// load the rows below and above the tile, lanes 0..15 of warp 2 the cells
// left and right of its rows. The plane tile is double buffered, so a plane
// needs one barrier. The update is jacobi4_packed, as in jacobi_v4_edge, so
// both give the same bits. RB: a red-black half-sweep of the given colour
// (cells of the other colour keep and write back Sigma).
template <bool RB>
__device__ __forceinline__ void jacobi_v4_full(const S *__restrict__ q, const S *__restrict__ b, const S *sin,
                                               S *sout, const Geom &g, C beta, int zc, int colour,
                                               const BlockPos &bp, C (*R2)[HY][HXV], C (*SG2)[HY][HXV])
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = bp.x * TXV, y0 = bp.y * BY;
    const int i0 = x0 + VX * tx, j = y0 + ty;
    const int k0 = bp.z * zc, k1 = min(g.nz, k0 + zc);
    const idx pl = (idx)g.plane;
    const idx own = (idx)j * (idx)g.nx + (idx)i0;
    // halo: warp 0 the row below the tile, warp 1 the row above (4-wide),
    // warp 2 lanes 0..7 the cells left of rows 0..7, lanes 8..15 right
    const bool yh = ty < 2, xh = ty == 2 && tx < 2 * BY;
    int hsy = 0, hsx = 0;
    idx hoff = 0;
    if (yh) {
        hsy = ty ? HY - 1 : 0;
        hsx = VX + VX * tx;
        hoff = (idx)map_axis(y0 + (ty ? BY : -1), g.ny, g.bc[2], g.bc[3]) * (idx)g.nx + (idx)i0;
    } else if (xh) {
        const int side = tx / BY, r = tx % BY;
        hsy = 1 + r;
        hsx = side ? VX + TXV : VX - 1;
        hoff = (idx)(y0 + r) * (idx)g.nx + (idx)map_axis(side ? x0 + TXV : x0 - 1, g.nx, g.bc[0], g.bc[1]);
    }
    const C hb = C(0.5) * beta;
    const C exm = (i0 > 0 || g.bc[0] == BC_PERIODIC) ? hb : C(0);
    const C exp_ = (i0 + VX - 1 < g.nx - 1 || g.bc[1] == BC_PERIODIC) ? hb : C(0);
    const C eym = (j > 0 || g.bc[2] == BC_PERIODIC) ? hb : C(0);
    const C eyp = (j < g.ny - 1 || g.bc[3] == BC_PERIODIC) ? hb : C(0);

    C rm[VX], sm[VX], r0[VX], s0[VX], rp[VX], sp[VX];
    {
        C t[VX];
        const idx zm = (idx)zmap(k0 - 1, g) * pl + own, z0 = (idx)k0 * pl + own;
        cv4(ld4r(CKP4(q + zm, q, g.n)), t);
        cv4(ld4r(CKP4(sin + zm, sin, g.n)), sm);
#pragma unroll
        for (int c = 0; c < VX; c++) rm[c] = rcp(t[c]);
        cv4(ld4r(CKP4(q + z0, q, g.n)), t);
        cv4(ld4r(CKP4(sin + z0, sin, g.n)), s0);
#pragma unroll
        for (int c = 0; c < VX; c++) r0[c] = rcp(t[c]);
    }
    // raw values one iteration ahead: own cells at k + 1, halo and b at k
    V4 ncr, ncs, nb, nhr, nhs;
    S nxr = S(1.0f), nxs = S(0.0f);
    auto pre = [&](int kk) {
        const idx pz = (idx)zmap(kk + 1, g) * pl + own, pk = (idx)kk * pl;
        ncr = ld4r(CKP4(q + pz, q, g.n));
        ncs = ld4r(CKP4(sin + pz, sin, g.n));
        nb = ld4r(CKP4(b + pk + own, b, g.n));
        if (yh) {
            nhr = ld4r(CKP4(q + pk + hoff, q, g.n));
            nhs = ld4r(CKP4(sin + pk + hoff, sin, g.n));
        } else if (xh) {
            nxr = ldr(CKP(q + pk + hoff, q, g.n));
            nxs = ldr(CKP(sin + pk + hoff, sin, g.n));
        }
    };
    pre(k0);
    const int col = VX + VX * tx;
    for (int k = k0; k < k1; k++) {
        C bv[VX], t[VX];
        // two tile buffers, planes alternating: the buffer written here was
        // last read two planes ago, before the barrier of the previous plane
        C (*R)[HXV] = R2[(k - k0) & 1], (*SG)[HXV] = SG2[(k - k0) & 1];
        sh_st4(&R[ty + 1][col], r0);
        sh_st4(&SG[ty + 1][col], s0);
        if (yh) {
            C hr[VX], hsg[VX];
            cv4(nhr, t);
            cv4(nhs, hsg);
#pragma unroll
            for (int c = 0; c < VX; c++) hr[c] = rcp(t[c]);
            sh_st4(&R[cks(hsy, HY)][cks4(hsx, HXV)], hr);
            sh_st4(&SG[cks(hsy, HY)][cks4(hsx, HXV)], hsg);
        } else if (xh) {
            R[cks(hsy, HY)][cks(hsx, HXV)] = rcp(cv(nxr));
            SG[cks(hsy, HY)][cks(hsx, HXV)] = cv(nxs);
        }
        cv4(ncr, t);
        cv4(ncs, sp);
#pragma unroll
        for (int c = 0; c < VX; c++) rp[c] = rcp(t[c]);
        cv4(nb, bv);
        if (k + 1 < k1) pre(k + 1);
        __syncthreads();
        const C ezm = (k > 0 || g.bc[4] == BC_PERIODIC) ? hb : C(0);
        const C ezp = (k < g.nz - 1 || g.bc[5] == BC_PERIODIC) ? hb : C(0);
        C ry0[VX], ry1[VX], sy0[VX], sy1[VX], o[VX];
        sh_ld4(&R[ty][col], ry0);
        sh_ld4(&R[ty + 2][col], ry1);
        sh_ld4(&SG[ty][col], sy0);
        sh_ld4(&SG[ty + 2][col], sy1);
        jacobi4_packed(r0, s0, R[ty + 1][col - 1], SG[ty + 1][col - 1], R[ty + 1][col + VX], SG[ty + 1][col + VX],
                       ry0, ry1, sy0, sy1, rm, sm, rp, sp, bv, hb, exm, exp_, eym, eyp, ezm, ezp, o);
        if constexpr (RB) {
#pragma unroll
            for (int c = 0; c < VX; c++)
                if (((i0 + c + j + k) & 1) != colour) o[c] = s0[c];
        }
        st4(CKP4(sout + (idx)k * pl + own, sout, g.n), o);
#pragma unroll
        for (int c = 0; c < VX; c++) {
            rm[c] = r0[c]; sm[c] = s0[c];
            r0[c] = rp[c]; s0[c] = sp[c];
        }
    }
}

__device__ __forceinline__ void jacobi_v4_body(const S *__restrict__ q, const S *__restrict__ b, const S *sin,
                                               S *sout, const Geom g, C beta, int zc, int colour,
                                               const BlockPos bp)
{
    __shared__ __align__(16) C R[2][HY][HXV];
    __shared__ __align__(16) C SG[2][HY][HXV];
    if constexpr (sizeof(C) == 4) {
        if (bp.x * TXV + TXV <= g.nx && bp.y * BY + BY <= g.ny) {  // block-uniform
            if (colour < 0)
                jacobi_v4_full<false>(q, b, sin, sout, g, beta, zc, colour, bp, R, SG);
            else
                jacobi_v4_full<true>(q, b, sin, sout, g, beta, zc, colour, bp, R, SG);
            return;
        }
    }
    jacobi_v4_edge(q, b, sin, sout, g, beta, zc, colour, bp, R[0], SG[0]);
}
constexpr int JACOBI_V4_BLOCKS = sizeof(S) == 2 ? 3 : sizeof(S) == 4 ? 2 : 1;  // resident per SM
__global__ void __launch_bounds__(BT, JACOBI_V4_BLOCKS) k_jacobi_v4(const S *__restrict__ q, const S *__restrict__ b,
                                                                  const S *sin, S *sout, Geom g, C beta, int zc,
                                                                  int colour)
{
    jacobi_v4_body(q, b, sin, sout, g, beta, zc, colour, BlockPos::of_launch());
}
// Grids whose every 4-cell tile lies inside (rows a multiple of 128 cells,
// a multiple of 8 rows; FP32 arithmetic) launch the full-tile body alone:
// without the edge body in the same kernel it keeps its values in registers
// (the combined kernel spills).
template <bool RB>
__global__ void __launch_bounds__(BT, JACOBI_V4_BLOCKS) k_jacobi_v4_full(const S *__restrict__ q,
                                                                       const S *__restrict__ b, const S *sin,
                                                                       S *sout, Geom g, C beta, int zc, int colour)
{
    if constexpr (sizeof(C) == 4) {
        __shared__ __align__(16) C R[2][HY][HXV];
        __shared__ __align__(16) C SG[2][HY][HXV];
        jacobi_v4_full<RB>(q, b, sin, sout, g, beta, zc, colour, BlockPos::of_launch(), R, SG);
    }
}


// Vector form of the source for rows whose length is a multiple of 4, laid
// out like k_jacobi_v4: each thread owns 4 consecutive cells of a row (one
// 4-wide load per field), u of plane k sits in a shared tile with a halo of 1
// (4-wide aligned rows), x-neighbours come from the thread's own registers
// and z-neighbours from its register queue. The central differences are
// taken undivided and 1/(2 dx)^2 is folded into alpha:
//   b = (alpha / (4 dx^2)) [sum_ab D_ab D_ba + (sum_a D_aa)^2],
//   D_ab = u_a(i + e_b) - u_a(i - e_b),
// which is Eq. igrelliptic's left side with G = D / (2 dx). k_source takes the
// same differences and source_b, so both forms give the same bits.
template <bool HASD>
__device__ __forceinline__ void source_v4_body(const QIn q, S *__restrict__ b, S *__restrict__ rho_out,
                                               const Geom g, C alpha_s, const C *W, const C *J, int zc,
                                               const BlockPos bp)
{
    __shared__ __align__(16) C U[3][HY][HXV];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int x0 = bp.x * TXV, y0 = bp.y * BY;
    const int i0 = x0 + VX * tx, j = y0 + ty;
    const bool active = i0 < g.nx && j < g.ny;
    const int k0 = bp.z * zc, k1 = min(g.nz, k0 + zc);
    const idx pl = (idx)g.plane;
    const idx rowj = (idx)(map_axis(j, g.ny, g.bc[2], g.bc[3]) * g.nx);
    // halo tasks: 4-wide cells of the rows above/below the tile, then single
    // cells left/right of each row
    int htask = tid < NYH ? 0 : (tid < NYH + NXH ? 1 : 2);
    int hsy = 0, hsx = 0, hx = 0;
    idx hrow = 0;
    if (htask == 0) {
        int side = tid / BX, t = tid % BX;
        hsy = side ? HY - 1 : 0;
        hsx = VX + VX * t;
        hx = x0 + VX * t;
        hrow = (idx)(map_axis(y0 + (side ? BY : -1), g.ny, g.bc[2], g.bc[3]) * g.nx);
    } else if (htask == 1) {
        int e = tid - NYH, side = e / BY, r = e % BY;
        hsy = 1 + r;
        hsx = side ? VX + TXV : VX - 1;
        hx = map_axis(side ? x0 + TXV : x0 - 1, g.nx, g.bc[0], g.bc[1]);
        hrow = (idx)(map_axis(y0 + r, g.ny, g.bc[2], g.bc[3]) * g.nx);
    }

    // u = m / rho of 4 cells from raw values (products rounded before they
    // are differenced: equal neighbours give an exact 0)
    auto u4 = [&](const QRaw4 (&r)[4], C u[3][VX], C rho[VX]) {
        C m[VX], rr[VX];
        cvq4<HASD>(r[0], rho);
#pragma unroll
        for (int c = 0; c < VX; c++) rr[c] = rcp(rho[c]);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cvq4<HASD>(r[1 + a], m);
#pragma unroll
            for (int c = 0; c < VX; c++) u[a][c] = mul_rn(m[c], rr[c]);
        }
    };
    // u of the own 4 cells of plane kk (the jet blend below an inflow face);
    // rho gets their (unblended) densities
    auto own_u = [&](int kk, C u[3][VX], C rho[VX]) {
        idx zb = (idx)zmap(kk, g) * pl + rowj;
        C v[4][VX];
#pragma unroll
        for (int f = 0; f < 4; f++) cvq4<HASD>(ldq4<HASD>(q, f, g, zb, i0), v[f]);
#pragma unroll
        for (int c = 0; c < VX; c++) rho[c] = v[0][c];
        if (kk < 0 && g.bc[4] == BC_INFLOW) {
#pragma unroll
            for (int c = 0; c < VX; c++) {
                idx fc = ck(rowj + (idx)map_axis(i0 + c, g.nx, g.bc[0], g.bc[1]), g.plane);
                C w = C(1) - W[fc];
#pragma unroll
                for (int f = 0; f < 4; f++) v[f][c] = fma_rn(w, v[f][c], J[(idx)f * pl + fc]);
            }
        }
#pragma unroll
        for (int c = 0; c < VX; c++) {
            C r = rcp(v[0][c]);
#pragma unroll
            for (int a = 0; a < 3; a++) u[a][c] = mul_rn(v[1 + a][c], r);
        }
    };
    C um[3][VX], u0[3][VX], up[3][VX];
    C rho0[VX], rhop[VX];  // densities of the own cells at k and k + 1
    own_u(k0 - 1, um, rhop);
    own_u(k0, u0, rho0);
    // raw values one iteration ahead: own cells at k + 1, halo at k (planes >= 0).
    // The increment modes' stages 2 and 3 (base and increments, 6 registers
    // per field and 4 cells) load the halo when it is used instead, which
    // keeps the registers under two blocks per SM with fewer spills.
    constexpr bool kHaloAhead = !(kInc && HASD);
    QRaw4 nc[4], nh[4];
    QRaw nxh[4];
    auto halo = [&](int kk) {
        if (htask == 0) {
#pragma unroll
            for (int f = 0; f < 4; f++) nh[f] = ldq4<HASD>(q, f, g, (idx)kk * pl + hrow, hx);
        } else if (htask == 1) {
#pragma unroll
            for (int f = 0; f < 4; f++) nxh[f] = ldqr<HASD>(q, f, ck((idx)kk * pl + hrow + hx, g.n));
        }
    };
    auto pre = [&](int kk) {
        idx pz = (idx)zmap(kk + 1, g) * pl + rowj;
#pragma unroll
        for (int f = 0; f < 4; f++) nc[f] = ldq4<HASD>(q, f, g, pz, i0);
        if (kHaloAhead) halo(kk);
    };
    pre(k0);
    for (int k = k0; k < k1; k++) {
        if (!kHaloAhead) halo(k);
        u4(nc, up, rhop);
        C hu[3][VX];
        if (htask == 0) {
            C hrho[VX];
            u4(nh, hu, hrho);
        } else if (htask == 1) {
            C r = rcp(cvq<HASD>(nxh[0]));
#pragma unroll
            for (int a = 0; a < 3; a++) hu[a][0] = mul_rn(cvq<HASD>(nxh[1 + a]), r);
        }
        if (k + 1 < k1) pre(k + 1);
        __syncthreads();  // readers of the previous plane are done
#pragma unroll
        for (int a = 0; a < 3; a++) {
            sh_st4(&U[a][ty + 1][VX + VX * tx], u0[a]);
            if (htask == 0) sh_st4(&U[a][cks(hsy, HY)][cks4(hsx, HXV)], hu[a]);
            else if (htask == 1) U[a][cks(hsy, HY)][cks(hsx, HXV)] = hu[a][0];
        }
        __syncthreads();
        if (active) {
            const int col = VX + VX * tx;
            C ym[3][VX], yp[3][VX], o[VX];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                sh_ld4(&U[a][ty][col], ym[a]);
                sh_ld4(&U[a][ty + 2][col], yp[a]);
            }
            C xl[3], xr[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                xl[a] = U[a][ty + 1][col - 1];
                xr[a] = U[a][ty + 1][col + VX];
            }
#pragma unroll
            for (int c = 0; c < VX; c++) {
                C D[3][3];  // D[a][d]: undivided central difference of u_a along d
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    C xm = c > 0 ? u0[a][c - 1] : xl[a];
                    C xp = c < VX - 1 ? u0[a][c + 1] : xr[a];
                    D[a][0] = xp - xm;
                    D[a][1] = yp[a][c] - ym[a][c];
                    D[a][2] = up[a][c] - um[a][c];
                }
                o[c] = source_b(D, alpha_s);
            }
            st4(CKP4(b + (idx)k * pl + (idx)(j * g.nx + i0), b, g.n), o);
            if constexpr (kInc) st4(CKP4(rho_out + (idx)k * pl + (idx)(j * g.nx + i0), rho_out, g.n), rho0);
        }
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c < VX; c++) {
                um[a][c] = u0[a][c];
                u0[a][c] = up[a][c];
            }
#pragma unroll
        for (int c = 0; c < VX; c++) rho0[c] = rhop[c];
    }
}
// 4 raw state values (cells off .. off+3 of field u, inside one row)
template <bool HASD>
__device__ __forceinline__ QRaw4 ldq4d(const QIn &q, int u, const Geom &g, idx off)
{
    return StateIO4<kInc>::ldd<HASD>(q, u, g, off);
}

// The 4-cell source of a grid whose every tile lies inside (rows a multiple
// of 128 cells, a multiple of 8 rows): the body of source_v4_body without
// lanes past the row's end, with whole 4-wide loads and halo offsets mapped
// once (warps 0 and 1: the rows below and above; lanes 0..15 of warp 2: the
// cells left and right of the rows), and the plane tile double buffered.
// The same operations per cell, so the same bits.
template <bool HASD>
__device__ __forceinline__ void source_v4_full(const QIn q, S *__restrict__ b, S *__restrict__ rho_out,
                                               const Geom g, C alpha_s, const C *W, const C *J, int zc,
                                               const BlockPos bp)
{
    __shared__ __align__(16) C U2[2][3][HY][HXV];  // plane tiles of u, two planes alternating
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = bp.x * TXV, y0 = bp.y * BY;
    const int i0 = x0 + VX * tx, j = y0 + ty;
    const int k0 = bp.z * zc, k1 = min(g.nz, k0 + zc);
    const idx pl = (idx)g.plane;
    const idx own = (idx)j * (idx)g.nx + (idx)i0;
    const bool yh = ty < 2, xh = ty == 2 && tx < 2 * BY;
    int hsy = 0, hsx = 0;
    idx hoff = 0;
    if (yh) {
        hsy = ty ? HY - 1 : 0;
        hsx = VX + VX * tx;
        hoff = (idx)map_axis(y0 + (ty ? BY : -1), g.ny, g.bc[2], g.bc[3]) * (idx)g.nx + (idx)i0;
    } else if (xh) {
        const int side = tx / BY, r = tx % BY;
        hsy = 1 + r;
        hsx = side ? VX + TXV : VX - 1;
        hoff = (idx)(y0 + r) * (idx)g.nx + (idx)map_axis(side ? x0 + TXV : x0 - 1, g.nx, g.bc[0], g.bc[1]);
    }
    auto u4 = [&](const QRaw4 (&r)[4], C u[3][VX], C rho[VX]) {
        C m[VX], rr[VX];
        cvq4<HASD>(r[0], rho);
#pragma unroll
        for (int c = 0; c < VX; c++) rr[c] = rcp(rho[c]);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cvq4<HASD>(r[1 + a], m);
#pragma unroll
            for (int c = 0; c < VX; c++) u[a][c] = mul_rn(m[c], rr[c]);
        }
    };
    auto own_u = [&](int kk, C u[3][VX], C rho[VX]) {
        const idx zb = (idx)zmap(kk, g) * pl + own;
        C v[4][VX];
#pragma unroll
        for (int f = 0; f < 4; f++) cvq4<HASD>(ldq4d<HASD>(q, f, g, zb), v[f]);
#pragma unroll
        for (int c = 0; c < VX; c++) rho[c] = v[0][c];
        if (kk < 0 && g.bc[4] == BC_INFLOW) {
#pragma unroll
            for (int c = 0; c < VX; c++) {
                const idx fc = ck(own + (idx)c, g.plane);
                C w = C(1) - W[fc];
#pragma unroll
                for (int f = 0; f < 4; f++) v[f][c] = fma_rn(w, v[f][c], J[(idx)f * pl + fc]);
            }
        }
#pragma unroll
        for (int c = 0; c < VX; c++) {
            C r = rcp(v[0][c]);
#pragma unroll
            for (int a = 0; a < 3; a++) u[a][c] = mul_rn(v[1 + a][c], r);
        }
    };
    C um[3][VX], u0[3][VX], up[3][VX];
    C rho0[VX], rhop[VX];
    own_u(k0 - 1, um, rhop);
    own_u(k0, u0, rho0);
    constexpr bool kHaloAhead = !(kInc && HASD);
    QRaw4 nc[4], nh[4];
    QRaw nxh[4];
    auto halo = [&](int kk) {
        if (yh) {
#pragma unroll
            for (int f = 0; f < 4; f++) nh[f] = ldq4d<HASD>(q, f, g, (idx)kk * pl + hoff);
        } else if (xh) {
#pragma unroll
            for (int f = 0; f < 4; f++) nxh[f] = ldqr<HASD>(q, f, ck((idx)kk * pl + hoff, g.n));
        }
    };
    auto pre = [&](int kk) {
        const idx pz = (idx)zmap(kk + 1, g) * pl + own;
#pragma unroll
        for (int f = 0; f < 4; f++) nc[f] = ldq4d<HASD>(q, f, g, pz);
        if (kHaloAhead) halo(kk);
    };
    pre(k0);
    const int col = VX + VX * tx;
    for (int k = k0; k < k1; k++) {
        if (!kHaloAhead) halo(k);
        // the buffer written here was last read two planes ago, before the
        // barrier of the previous plane: one barrier per plane
        C (*U)[HY][HXV] = U2[(k - k0) & 1];
#pragma unroll
        for (int a = 0; a < 3; a++) sh_st4(&U[a][ty + 1][col], u0[a]);
        if (yh) {
            C hu[3][VX], hrho[VX];
            u4(nh, hu, hrho);
#pragma unroll
            for (int a = 0; a < 3; a++) sh_st4(&U[a][cks(hsy, HY)][cks4(hsx, HXV)], hu[a]);
        } else if (xh) {
            C r = rcp(cvq<HASD>(nxh[0]));
#pragma unroll
            for (int a = 0; a < 3; a++) U[a][cks(hsy, HY)][cks(hsx, HXV)] = mul_rn(cvq<HASD>(nxh[1 + a]), r);
        }
        u4(nc, up, rhop);
        if (k + 1 < k1) pre(k + 1);
        __syncthreads();
        C ym[3][VX], yp[3][VX], o[VX];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            sh_ld4(&U[a][ty][col], ym[a]);
            sh_ld4(&U[a][ty + 2][col], yp[a]);
        }
        C xl[3], xr[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            xl[a] = U[a][ty + 1][col - 1];
            xr[a] = U[a][ty + 1][col + VX];
        }
#pragma unroll
        for (int c = 0; c < VX; c++) {
            C D[3][3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                C xm = c > 0 ? u0[a][c - 1] : xl[a];
                C xp = c < VX - 1 ? u0[a][c + 1] : xr[a];
                D[a][0] = xp - xm;
                D[a][1] = yp[a][c] - ym[a][c];
                D[a][2] = up[a][c] - um[a][c];
            }
            o[c] = source_b(D, alpha_s);
        }
        st4(CKP4(b + (idx)k * pl + own, b, g.n), o);
        if constexpr (kInc) st4(CKP4(rho_out + (idx)k * pl + own, rho_out, g.n), rho0);
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c < VX; c++) {
                um[a][c] = u0[a][c];
                u0[a][c] = up[a][c];
            }
#pragma unroll
        for (int c = 0; c < VX; c++) rho0[c] = rhop[c];
    }
}

// Two blocks per SM (at most 128 registers): the kernel waits on load
// latency, and one block per SM, which a free register choice gives (about
// 156 registers), runs it 1.6x slower. The increment modes' form, which
// holds raw FP32 values and 16-bit increments one plane ahead, spills a few
// registers under this bound and still runs faster. FP64 keeps one block.
constexpr int SOURCE_V4_BLOCKS = sizeof(C) == 8 ? 1 : 2;
template <bool HASD>
__global__ void __launch_bounds__(BT, SOURCE_V4_BLOCKS) k_source_v4(QIn q, S *__restrict__ b, S *__restrict__ rho_out, Geom g,
                                                   C alpha_s, const C *W, const C *J, int zc)
{
    source_v4_body<HASD>(q, b, rho_out, g, alpha_s, W, J, zc, BlockPos::of_launch());
}
template <bool HASD>
__global__ void __launch_bounds__(BT, SOURCE_V4_BLOCKS) k_source_v4_full(QIn q, S *__restrict__ b,
                                                                        S *__restrict__ rho_out, Geom g,
                                                                        C alpha_s, const C *W, const C *J, int zc)
{
    source_v4_full<HASD>(q, b, rho_out, g, alpha_s, W, J, zc, BlockPos::of_launch());
}


// ----------------------------------------------------------------- flux
// Block of TY + 1 warps over a TX x TY tile of columns. Warps 0..TY-1 own a
// row each: per plane a warp computes the x-face at the low side of each of
// its cells, the y-face below its row and, from its register queue, the
// z-face above; warp TY computes the y-faces above the last row and the
// x-faces at the high end of every row. Every warp thus does three face
// evaluations or fewer and the tile needs no face twice. The warp count is a
// multiple of 4 so that the four SM sub-partitions (16K registers each) hold
// equal shares: 16 warps of at most 128 registers in FP32 arithmetic, one
// block per SM, keep the stencil queue in registers.
constexpr int TX = 32, TY = sizeof(C) == 8 ? 7 : 15, NWARP = TY + 1, NT = 32 * NWARP;
constexpr int PW = TX + 6, PH = TY + 6;          // plane tile with a halo of 3
// tile cells that are read: the rows of the tile with the x-halo, the three
// rows above and below (no corner blocks), and the four cells diagonal to
// the interior's corners (the viscous faces' tangential neighbours)
constexpr int NPLANE = TY * PW + 6 * TX + 4;
constexpr int LPT = (NPLANE + NT - 1) / NT;      // tile cells loaded per thread
// every thread has a first tile cell (its test is dropped in the 16-bit
// forms, where that measured faster; FP32/FP64 keep it)
constexpr bool kR0 = sizeof(S) == 2 && NPLANE >= NT;

// The plane tiles keep the six face variables as three pairs, (rho, m_x),
// (m_y, m_z), (E, Sigma): a stencil point of a pair is one 8-byte (16-byte in
// FP64) shared load, and the reconstruction of a pair is one packed FP32x2
// multiply-add per term.

// 5th-order face values of a pair (weights as in rec_left / rec_right)
__device__ __forceinline__ C2 rec_left2(C2 a, C2 b, C2 c, C2 d, C2 e)
{
    C2 t = pmul(bcast(C(2.0 / 60.0)), a);
    t = pfma(bcast(C(-13.0 / 60.0)), b, t);
    t = pfma(bcast(C(47.0 / 60.0)), c, t);
    t = pfma(bcast(C(27.0 / 60.0)), d, t);
    return pfma(bcast(C(-3.0 / 60.0)), e, t);
}
__device__ __forceinline__ C2 rec_right2(C2 b, C2 c, C2 d, C2 e, C2 f)
{
    C2 t = pmul(bcast(C(-3.0 / 60.0)), b);
    t = pfma(bcast(C(27.0 / 60.0)), c, t);
    t = pfma(bcast(C(47.0 / 60.0)), d, t);
    t = pfma(bcast(C(-13.0 / 60.0)), e, t);
    return pfma(bcast(C(2.0 / 60.0)), f, t);
}

// 3rd-order face values of a pair: the quadratic through the three cell
// averages of the biased stencil (i-1..i+1 left, i..i+2 right) at the face
__device__ __forceinline__ C2 rec3_left2(C2 b, C2 c, C2 d)
{
    C2 t = pmul(bcast(C(-1.0 / 6.0)), b);
    t = pfma(bcast(C(5.0 / 6.0)), c, t);
    return pfma(bcast(C(2.0 / 6.0)), d, t);
}
__device__ __forceinline__ C2 rec3_right2(C2 c, C2 d, C2 e)
{
    C2 t = pmul(bcast(C(2.0 / 6.0)), c);
    t = pfma(bcast(C(5.0 / 6.0)), d, t);
    return pfma(bcast(C(-1.0 / 6.0)), e, t);
}

constexpr int TILE2 = 3 * PH * PW;  // pairs in one plane tile
// Layout of one plane tile: the pairs (rho, m_x) and (m_y, m_z) of a cell
// side by side, one 16-byte quad per cell (two in FP64) for cells 0..PH*PW-1,
// then the pairs (E, Sigma) of all cells. A stencil point is then one
// 16-byte shared load and one 8-byte load (FP32) instead of three 8-byte
// loads: the same shared-memory bandwidth in fewer instructions.
constexpr int QUADS = 2 * PH * PW;  // offset (in pairs) of the (E, Sigma) pairs
__device__ __forceinline__ int pair_at(int p, int e) { return p < 2 ? 2 * e + p : QUADS + e; }
// the pairs (rho, m_x), (m_y, m_z) of tile cell e
__device__ __forceinline__ void ld_quad(const float2 *T, int e, float2 &a, float2 &b)
{
    const float4 q = *reinterpret_cast<const float4 *>(T + 2 * e);
    a = make_float2(q.x, q.y);
    b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld_quad(const double2 *T, int e, double2 &a, double2 &b)
{
    a = T[2 * e];
    b = T[2 * e + 1];
}
__device__ __forceinline__ void st_quad(float2 *T, int e, float2 a, float2 b)
{
    *reinterpret_cast<float4 *>(T + 2 * e) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_quad(double2 *T, int e, double2 a, double2 b)
{
    T[2 * e] = a;
    T[2 * e + 1] = b;
}
// the three pairs of tile cell e
__device__ __forceinline__ void ld_cell(const C2 *T, int e, C2 &a, C2 &b, C2 &c)
{
    ld_quad(T, e, a, b);
    c = T[QUADS + e];
}
__device__ __forceinline__ void st_cell(C2 *T, int e, C2 a, C2 b, C2 c)
{
    st_quad(T, e, a, b);
    T[QUADS + e] = c;
}
constexpr int NFX = 5 * TY * (TX + 1), NFY = 5 * (TY + 1) * TX;  // one parity of the face buffers
constexpr int RING = 7;             // plane tiles resident: k-2..k+3 and k+4 in flight

// Storage equal to the arithmetic type: plane tiles are copied global ->
// shared with cp.async (4- or 8-byte elements), which holds no registers.
constexpr bool kAsyncTile = sizeof(S) == sizeof(C);
__device__ __forceinline__ void cp_async_elem(C *dst, const S *src)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// shared bytes: the ring of plane tiles (pairs), two sets of x- and y-face fluxes
__host__ __device__ constexpr size_t flux_smem_bytes()
{
    return RING * TILE2 * sizeof(C2) + 2 * (5 * TY * (TX + 1) + 5 * (TY + 1) * TX) * sizeof(C);
}

// tile cell e (0 <= e < NPLANE) -> position (lx, ly) in the PW x PH tile
__device__ __forceinline__ void plane_cell(int e, int &lx, int &ly)
{
    if (e < 3 * TX) { ly = e / TX; lx = 3 + e % TX; }
    else if (e < 3 * TX + TY * PW) { e -= 3 * TX; ly = 3 + e / PW; lx = e % PW; }
    else if (e < 6 * TX + TY * PW) { e -= 3 * TX + TY * PW; ly = TY + 3 + e / TX; lx = 3 + e % TX; }
    else { e -= 6 * TX + TY * PW; ly = (e & 2) ? TY + 3 : 2; lx = (e & 1) ? TX + 3 : 2; }
}

template <int D, int ORD>
__device__ __forceinline__ void face_from_stencil(const C2 (&s)[6][3], C gamma, C gm1, C *F,
                                                  FaceFlag &bad)
{
    C L[6], R[6];
#pragma unroll
    for (int p = 0; p < 3; p++) {
        C2 l = ORD == 3 ? rec3_left2(s[1][p], s[2][p], s[3][p])
                        : rec_left2(s[0][p], s[1][p], s[2][p], s[3][p], s[4][p]);
        C2 r = ORD == 3 ? rec3_right2(s[2][p], s[3][p], s[4][p])
                        : rec_right2(s[1][p], s[2][p], s[3][p], s[4][p], s[5][p]);
        L[2 * p] = l.x;
        L[2 * p + 1] = l.y;
        R[2 * p] = r.x;
        R[2 * p + 1] = r.y;
    }
    lf_flux2<D>(L, R, gamma, gm1, F, bad);
}

// face along D (0, 1) from six consecutive cells of one plane tile starting
// at element `at`, `step` elements apart
template <int D, int ORD>
__device__ __forceinline__ void tile_face(const C2 *T, int at, int step, C gamma, C gm1, C *F,
                                          FaceFlag &bad)
{
    C2 s[6][3];
#pragma unroll
    for (int m = 0; m < 6; m++) {
        if (ORD == 3 && (m == 0 || m == 5)) {
            s[m][0] = s[m][1] = s[m][2] = bcast(C(0));
        } else {
            ld_cell(T, cks(at + m * step, PH * PW), s[m][0], s[m][1], s[m][2]);
        }
    }
    face_from_stencil<D, ORD>(s, gamma, gm1, F, bad);
}

// tile_face with the stencil's point 3 (the cell the face lies below / left of
// the row warp's own cell) given: the row warp holds it from its z-stencil
template <int D, int ORD>
__device__ __forceinline__ void tile_face_c(const C2 *T, int at, int step, const C2 (&c3)[3], C gamma, C gm1,
                                            C *F, FaceFlag &bad)
{
    C2 s[6][3];
#pragma unroll
    for (int m = 0; m < 6; m++) {
        if (ORD == 3 && (m == 0 || m == 5)) {
            s[m][0] = s[m][1] = s[m][2] = bcast(C(0));
        } else if (m == 3) {
            s[m][0] = c3[0];
            s[m][1] = c3[1];
            s[m][2] = c3[2];
        } else {
            ld_cell(T, cks(at + m * step, PH * PW), s[m][0], s[m][1], s[m][2]);
        }
    }
    face_from_stencil<D, ORD>(s, gamma, gm1, F, bad);
}

// ------------------------------------------------------- viscous stresses
// Velocity u = m / rho of the tile cell at pair offset `at`.
__device__ __forceinline__ void tvel(const C2 *T, int at, C u[3])
{
    C2 a, b;
    ld_quad(T, cks(at, PH * PW), a, b);
    C r = rcp(a.x);
    u[0] = a.y * r;
    u[1] = b.x * r;
    u[2] = b.y * r;
}

// Doubled viscous flux (like lf_flux2's 2 F_hat) through the face between
// cells A and B along axis D, added to G (Eqs. igrmobalance-igrenbalance with
// the stress of Eq. constitutive_law):
//   tau_aD = mu (du_a/dx_D + du_D/dx_a) + lam delta_aD div u, lam = zeta - 2 mu / 3,
//   G[1 + a] -= 2 tau_aD,  G[4] -= 2 sum_a ((u_a(A) + u_a(B)) / 2) tau_aD,
// with second-order face derivatives: normal (u(B) - u(A)) / dx, tangential
// along t the mean of the central differences at A and B. T1/T2 give the
// tangential axes t1 < t2 (the two axes other than D) as the cells on each
// side of A and B: a1m, a1p, b1m, b1p along t1 and a2m.. along t2.
template <int D>
__device__ __forceinline__ void visc_face(const C2 *TA, int a, const C2 *TB, int b, const C2 *T1Am,
                                          int a1m, const C2 *T1Ap, int a1p, const C2 *T1Bm, int b1m,
                                          const C2 *T1Bp, int b1p, const C2 *T2Am, int a2m,
                                          const C2 *T2Ap, int a2p, const C2 *T2Bm, int b2m,
                                          const C2 *T2Bp, int b2p, C mu, C lam, C inv_dx, C *G)
{
    constexpr int t1 = D == 0 ? 1 : 0, t2 = D == 2 ? 1 : 2;
    C uA[3], uB[3], p[3], m[3], q[3], r[3], Gr[3][3];
    tvel(TA, a, uA);
    tvel(TB, b, uB);
#pragma unroll
    for (int c = 0; c < 3; c++) Gr[c][D] = (uB[c] - uA[c]) * inv_dx;
    const C qd = C(0.25) * inv_dx;
    tvel(T1Ap, a1p, p); tvel(T1Am, a1m, m); tvel(T1Bp, b1p, q); tvel(T1Bm, b1m, r);
#pragma unroll
    for (int c = 0; c < 3; c++) Gr[c][t1] = ((p[c] - m[c]) + (q[c] - r[c])) * qd;
    tvel(T2Ap, a2p, p); tvel(T2Am, a2m, m); tvel(T2Bp, b2p, q); tvel(T2Bm, b2m, r);
#pragma unroll
    for (int c = 0; c < 3; c++) Gr[c][t2] = ((p[c] - m[c]) + (q[c] - r[c])) * qd;
    const C div = (Gr[0][0] + Gr[1][1]) + Gr[2][2];
    C work = C(0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        C tau = mu * (Gr[c][D] + Gr[D][c]);
        if (c == D) tau += lam * div;
        G[1 + c] -= C(2) * tau;
        work += C(0.5) * (uA[c] + uB[c]) * tau;
    }
    G[4] -= C(2) * work;
}

// registers per thread such that NWARP / 4 warps fit one sub-partition's 16K
constexpr int FLUX_MAXREG = sizeof(C) == 8 ? 224 : 128;

// The block keeps a ring of RING plane tiles (halo 3 in x and y) in shared
// memory: plane kk lives in slot (kk - k0 + 3) mod RING. Iteration k (from
// k0 - 1 to k1 - 1), one barrier each:
//   - start the copy of plane k + 4 into the slot of plane k - 3 (read for
//     the last time before the previous barrier);
//   - row warps: divergence and stage combination of plane k - 1 (face
//     buffers of parity k - 1), then the z-face k + 1/2 from planes
//     k - 2..k + 3 of the ring at the warp's own cells;
//   - all warps (k >= k0): the x- and y-faces of plane k into the face
//     buffers of parity k;
//   - complete the copy of plane k + 4, barrier.
// Planes k0 - 3..k0 + 2 are filled before the loop (with the boundary index
// mapping and, below an inflow face, the jet blend). Every plane is read from
// global memory once per block; nothing relies on the L1 cache.
//
// In the increment modes the input q_s is read as RN32(q^n + d_s) (d_s from
// stage 2 on), stages 1 and 2 store the 16-bit increment
// d_{s+1} = RN16(w [(q_s - q^n) + dt L]) into `out`, and stage 3 stores the
// FP32 state q^n + w [(q_s - q^n) + dt L] into `outb`.
template <int mode, int ORD, bool VISC>
__device__ __forceinline__ void flux_body(const QIn qin, const S *__restrict__ sig, const QBIn qn,
                                          const Fout<5> out, const QBOut outb, const Frhs rhs,
                                          const Fout<5> base_out, const Geom g, C gamma, C half_inv_dx,
                                          const Scalars *sc, double *blockmax, int *err, const C *W,
                                          const C *J, int zc, int cz0, C mu, C lamv, const BlockPos bp)
{
    constexpr bool HASD = kInc && (mode == FLUX_STAGE2 || mode == FLUX_STAGE3);
    // The five fields of every state buffer lie g.n values apart. In the
    // increment modes, which read and write more buffers, their addresses
    // come from the first field's pointer and that stride, so the kernel
    // holds one pointer per buffer: fewer constant-bank reloads of pointers
    // (9 against 26 per cell) for more 64-bit adds, 4.5% faster at full size;
    // the other forms keep a pointer per field (the same or 1% faster).
    const size_t fs = (size_t)g.n;
    const QB *const qb0 = qin.b[0];
    const S *const qd0 = qin.d[0];
    const QB *const qn0 = qn.p[0];
    S *const out0 = out.p[0];
    QB *const outb0 = outb.p[0];
    // raw state value u at offset c (StateIO's layout, one pointer per buffer)
    auto ldq_raw = [&](int u, idx c) -> QRaw {
        if constexpr (kInc) {
            QRawInc r;
            r.b = __ldg(qb0 + u * fs + c);
            r.d = HASD ? ldr(qd0 + u * fs + c) : S(0.0f);
            return *reinterpret_cast<QRaw *>(&r);
        } else {
            return ldqr<HASD>(qin, u, c);
        }
    };
    // field u of the stored input (u < 5: q, 5: Sigma) where the state has the storage type
    auto fin = [&](int u) -> const S * { return u < 5 ? reinterpret_cast<const S *>(qin.b[u]) : sig; };
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *P = reinterpret_cast<C2 *>(smem_raw);        // [RING][3][PH][PW]
    C *FXb = reinterpret_cast<C *>(P + RING * TILE2); // [2][5][TY][TX+1]
    C *FYb = FXb + 2 * NFX;                           // [2][5][TY+1][TX]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int x0 = bp.x * TX, y0 = bp.y * TY;
    const int cz = cz0 + bp.z;  // z-chunk (a launch may cover chunks cz0.. only)
    const int k0 = cz * zc, k1 = min(g.nz, k0 + zc);
    const bool rowwarp = w < TY;  // warp-uniform
    const int i = x0 + lane, j = y0 + (rowwarp ? w : 0);
    const bool active = rowwarp && i < g.nx && j < g.ny;
    const idx pl = (idx)g.plane;
    const idx own = (idx)(j * g.nx + i);
    const int tcell = (w + 3) * PW + lane + 3;  // this row-warp lane's cell in a tile
    const C gm1 = gamma - C(1);
    FaceFlag bad = FaceFlag(kFaceMin ? 1 : 0);  // face states with rho <= 0 or p <= 0 (warning)
    bool nonfinite = false; // a non-finite output (error)
    // ring slot offsets (in pairs) of planes k-2..k+4 in iteration k, rotated
    // once per plane: plane kk sits in slot (kk - k0 + 3) mod RING
    int ro[RING];
#pragma unroll
    for (int m = 0; m < RING; m++) ro[m] = m * TILE2;  // k = k0 - 1: planes k0-3.. in slots 0..


    // tile cells this thread loads each plane: shared and in-plane offsets
    int soff[LPT];
    idx goff[LPT];
#pragma unroll
    for (int r = 0; r < LPT; r++) {
        int e = tid + r * NT;
        soff[r] = -1;
        goff[r] = 0;
        if (e < NPLANE) {
            int lx, ly;
            plane_cell(e, lx, ly);
            soff[r] = ly * PW + lx;
            goff[r] = (idx)(map_axis(y0 + ly - 3, g.ny, g.bc[2], g.bc[3]) * g.nx +
                            map_axis(x0 + lx - 3, g.nx, g.bc[0], g.bc[1]));
        }
    }

    // planes k0 - 3..k0 + 2, loaded and stored directly (index mapping in z,
    // jet blend below an inflow face)
#pragma unroll 1
    for (int kk = k0 - 3; kk < k0 + 3; kk++) {
        C2 *T = P + (kk - k0 + 3) * TILE2;
        const idx zb = (idx)zmap(kk, g) * pl;
        const bool blend = kk < 0 && g.bc[4] == BC_INFLOW;
#pragma unroll
        for (int r = 0; r < LPT; r++)
            if ((kR0 && r == 0) || soff[r] >= 0) {
                C v[6];
                const idx c = ck(zb + goff[r], g.n);
#pragma unroll
                for (int u = 0; u < 5; u++) v[u] = cvq<HASD>(ldq_raw(u, c));
                v[5] = ldc(sig + c);
                if (blend) {
                    C wf = C(1) - W[ck(goff[r], g.plane)];
#pragma unroll
                    for (int u = 0; u < 5; u++) v[u] = wf * v[u] + J[(idx)u * pl + ck(goff[r], g.plane)];
                }
                st_cell(T, cks(soff[r], PH * PW), pset(v[0], v[1]), pset(v[2], v[3]), pset(v[4], v[5]));
            }
    }

    // plane kk >= k0 + 3 of the pipeline: FP32/FP64 storage copies with
    // cp.async; 16-bit storage loads raw values into registers at `fetch`
    // and converts and stores them at `land`
    S Rg[LPT][6];     // (unused with cp.async and in the increment modes)
    QRaw Rq[LPT][5];  // increment modes: raw q^n and d_s
    S Rs[LPT];        // increment modes: raw Sigma
    auto fetch = [&](int kk, C2 *T) {
        const idx zb = (idx)zmap(kk, g) * pl;
#pragma unroll
        for (int r = 0; r < LPT; r++)
            if ((kR0 && r == 0) || soff[r] >= 0) {
                if constexpr (kInc) {
                    const idx c = ck(zb + goff[r], g.n);
#pragma unroll
                    for (int u = 0; u < 5; u++) Rq[r][u] = ldq_raw(u, c);
                    Rs[r] = ldr(sig + c);
                } else {
#pragma unroll
                    for (int u = 0; u < 6; u++) {
                        if constexpr (kAsyncTile)
                            cp_async_elem(&T[pair_at(u >> 1, cks(soff[r], PH * PW))].x + (u & 1),
                                          CKP(fin(u) + zb + goff[r], fin(u), g.n));
                        else
                            Rg[r][u] = ldr(CKP(fin(u) + zb + goff[r], fin(u), g.n));
                    }
                }
            }
        if constexpr (kAsyncTile) cp_async_commit();
    };
    auto land = [&](C2 *T) {
        if constexpr (kAsyncTile) {
            cp_async_wait_all();
        } else if constexpr (kInc) {
#pragma unroll
            for (int r = 0; r < LPT; r++)
                if ((kR0 && r == 0) || soff[r] >= 0) {
                    st_cell(T, cks(soff[r], PH * PW), pset(cvq<HASD>(Rq[r][0]), cvq<HASD>(Rq[r][1])),
                            pset(cvq<HASD>(Rq[r][2]), cvq<HASD>(Rq[r][3])), pset(cvq<HASD>(Rq[r][4]), cv(Rs[r])));
                }
        } else {
#pragma unroll
            for (int r = 0; r < LPT; r++)
                if ((kR0 && r == 0) || soff[r] >= 0)
                    st_cell(T, cks(soff[r], PH * PW), pset(cv(Rg[r][0]), cv(Rg[r][1])), pset(cv(Rg[r][2]), cv(Rg[r][3])),
                            pset(cv(Rg[r][4]), cv(Rg[r][5])));
        }
    };
    __syncthreads();

    C dt32 = C(0), w32 = C(1);
    double dt = 0.0, wd = 1.0;
    if (mode != FLUX_RHS) {
        dt = sc->dt;
        wd = mode == FLUX_STAGE1 ? 1.0 : mode == FLUX_STAGE2 ? 0.25 : 2.0 / 3.0;
        dt32 = C(dt);
        w32 = C(wd);
    }
    C smax = C(0);  // running wave-speed maximum (FP32 here: FP64 is slow on this GPU)

    C Fzm[5], Fzp[5];
    // planes k and k + 1 at a row-warp lane's cell before iteration k: the
    // z-stencils of consecutive planes share them, so each iteration loads
    // four of its six points (shared loads are the flux kernel's most
    // contended resource; the copies are register moves). Not in the
    // viscous kernels, whose extra registers would spill.
    // this lane's x-face (at the low side of its cell) and y-face (below its
    // row) of the last plane: the divergence of that plane takes them from
    // registers and only the faces of its neighbours from the face buffers
    constexpr bool kOwnFaces = sizeof(C) == 4;
    C Fxo[5], Fyo[5];
    C2 zq[2][3];
    if (!VISC && rowwarp) {
        ld_cell(P + ro[2], cks(tcell, PH * PW), zq[0][0], zq[0][1], zq[0][2]);  // plane k0 - 1
        ld_cell(P + ro[3], cks(tcell, PH * PW), zq[1][0], zq[1][1], zq[1][2]);  // plane k0
    }
    QB qnv[5];  // q^n of plane k - 1 (stages 2 and 3), loaded one iteration ahead

    // divergence and stage combination of plane kk (face buffers of parity kk)
    // The three pairs of a row-warp lane's own cell in plane k, taken from its
    // z-stencil (the stencil's centre plane): they are point 3 of the lane's
    // x- and y-face stencils in plane k and the stage input the divergence of
    // plane k combines in the next iteration, so none is loaded twice.
    C2 cc[3];
    auto finish = [&](int kk) {
        const C *FX = FXb + (kk & 1) * NFX;
        const C *FY = FYb + (kk & 1) * NFY;
        idx c = ck((idx)kk * pl + own, g.n);
        C Lv[5];
#pragma unroll
        for (int u = 0; u < 5; u++) {
            // the faces above and right of the cell from the buffers, the two
            // below and left of it computed by this lane (Fxo, Fyo; FP64
            // arithmetic reads them back, its extra registers would spill)
            const C fxl = kOwnFaces ? Fxo[u] : FX[cks((u * TY + w) * (TX + 1) + lane, NFX)];
            const C fyl = kOwnFaces ? Fyo[u] : FY[cks((u * (TY + 1) + w) * TX + lane, NFY)];
            C dfx = FX[cks((u * TY + w) * (TX + 1) + lane + 1, NFX)] - fxl;
            C dfy = FY[cks((u * (TY + 1) + w + 1) * TX + lane, NFY)] - fyl;
            C dfz = Fzp[u] - Fzm[u];
            Lv[u] = -((dfx + dfy) + dfz) * half_inv_dx;
        }
        if (mode == FLUX_RHS) {
#pragma unroll
            for (int u = 0; u < 5; u++) rhs.p[u][c] = Lv[u];
            nonfinite |= !isfinite((Lv[0] + Lv[1]) + (Lv[2] + Lv[3]) + Lv[4]);
        } else {
            const C2 a = cc[0], b = cc[1], e = cc[2];  // plane kk at this cell
            const C qsv[5] = {a.x, a.y, b.x, b.y, e.x};
            if (mode == FLUX_STAGE1 && base_out.p[0]) {
                // the RK base q^n for stages 2 and 3 (exact: qsv holds stored values)
#pragma unroll
                for (int u = 0; u < 5; u++) stc(base_out.p[u] + c, qsv[u]);
            }
            C o[5], qb[5];
#pragma unroll
            for (int u = 0; u < 5; u++) qb[u] = mode == FLUX_STAGE1 ? qsv[u] : cv(qnv[u]);
            if constexpr (kInc) {
#pragma unroll
                for (int u = 0; u < 5; u++) {
                    const C inc = w32 * ((qsv[u] - qb[u]) + dt32 * Lv[u]);
                    if (mode == FLUX_STAGE3)
                        o[u] = stc(outb0 + u * fs + c, qb[u] + inc);  // q^n+1 in FP32
                    else
                        o[u] = stc(out0 + u * fs + c, inc);  // the increment d_s+1, rounded to 16 bits
                }
            } else {
                rk_store5(out, c, qb, qsv, Lv, dt32, dt, w32, wd, o);
            }
            nonfinite |= !isfinite((o[0] + o[1]) + (o[2] + o[3]) + o[4]);
            if (mode == FLUX_STAGE3) {
                C sp = cell_speed(o[0], o[1], o[2], o[3], o[4], gamma, gm1);
                smax = (sp > smax || sp != sp) ? sp : smax;
            }
        }
    };

    for (int k = k0 - 1; k < k1; k++) {
        const bool more = k + 4 <= k1 + 2;  // plane k + 4 feeds the z-faces
        if (more) fetch(k + 4, P + ro[6]);
        const C2 *T = P + ro[2];  // plane k
        C *FX = FXb + (k & 1) * NFX;
        C *FY = FYb + (k & 1) * NFY;
        C F[5];
        const C2 *Tm = P + ro[1], *Tp = P + ro[3];  // planes k - 1, k + 1 (viscous terms)
        const C inv_dx = C(2) * half_inv_dx;
        // viscous x-face between tile cells a and a + 1 (same row)
        auto visc_x = [&](int a) {
            visc_face<0>(T, a, T, a + 1, T, a - PW, T, a + PW, T, a + 1 - PW, T, a + 1 + PW, Tm, a, Tp,
                         a, Tm, a + 1, Tp, a + 1, mu, lamv, inv_dx, F);
        };
        // viscous y-face between tile cells a and a + PW (same column)
        auto visc_y = [&](int a) {
            visc_face<1>(T, a, T, a + PW, T, a - 1, T, a + 1, T, a + PW - 1, T, a + PW + 1, Tm, a, Tp,
                         a, Tm, a + PW, Tp, a + PW, mu, lamv, inv_dx, F);
        };
        if (rowwarp) {
            if (active) {
                if (k > k0) finish(k - 1);
                if (k >= k0 && (mode == FLUX_STAGE2 || mode == FLUX_STAGE3)) {
                    idx c = ck((idx)k * pl + own, g.n);
#pragma unroll
                    for (int u = 0; u < 5; u++) qnv[u] = __ldg(kInc ? qn0 + u * fs + c : qn.p[u] + c);
                }
            }
#pragma unroll
            for (int u = 0; u < 5; u++) Fzm[u] = Fzp[u];
            C2 sz[6][3];  // z-stencil: planes k - 2..k + 3 at this cell
#pragma unroll
            for (int m = 0; m < 6; m++) {
                if (!VISC && (m == 2 || m == 3)) {  // planes k, k + 1: points 3, 4 of the previous z-stencil
#pragma unroll
                    for (int p = 0; p < 3; p++) sz[m][p] = zq[m - 2][p];
                } else {
                    ld_cell(P + ro[m], cks(tcell, PH * PW), sz[m][0], sz[m][1], sz[m][2]);
                }
            }
            if constexpr (!VISC) {
#pragma unroll
                for (int p = 0; p < 3; p++) {
                    zq[0][p] = sz[3][p];
                    zq[1][p] = sz[4][p];
                }
            }
            face_from_stencil<2, ORD>(sz, gamma, gm1, Fzp, bad);  // z-face k + 1/2
            cc[0] = sz[2][0];  // plane k at this cell
            cc[1] = sz[2][1];
            cc[2] = sz[2][2];
            if constexpr (VISC) {
                const C2 *Ta = P + ro[2], *Tb = P + ro[3];  // planes k, k + 1
                visc_face<2>(Ta, tcell, Tb, tcell, Ta, tcell - 1, Ta, tcell + 1, Tb, tcell - 1, Tb,
                             tcell + 1, Ta, tcell - PW, Ta, tcell + PW, Tb, tcell - PW, Tb, tcell + PW,
                             mu, lamv, C(2) * half_inv_dx, Fzp);
            }
            if (k >= k0) {
                // x-face at the low side of cell `lane` of row w (tile cells lane-3..lane+2)
                tile_face_c<0, ORD>(T, (w + 3) * PW + lane, 1, cc, gamma, gm1, F, bad);
                if constexpr (VISC) visc_x((w + 3) * PW + lane + 2);
#pragma unroll
                for (int u = 0; u < 5; u++) {
                    FX[cks((u * TY + w) * (TX + 1) + lane, NFX)] = F[u];
                    if constexpr (kOwnFaces) Fxo[u] = F[u];
                }
                // y-face below row w in column lane (tile rows w-3..w+2)
                tile_face_c<1, ORD>(T, w * PW + lane + 3, PW, cc, gamma, gm1, F, bad);
                if constexpr (VISC) visc_y((w + 2) * PW + lane + 3);
#pragma unroll
                for (int u = 0; u < 5; u++) {
                    FY[cks((u * (TY + 1) + w) * TX + lane, NFY)] = F[u];
                    if constexpr (kOwnFaces) Fyo[u] = F[u];
                }
            }
        } else if (k >= k0) {
            // y-face above the last row, column lane
            tile_face<1, ORD>(T, TY * PW + lane + 3, PW, gamma, gm1, F, bad);
            if constexpr (VISC) visc_y((TY + 2) * PW + lane + 3);
#pragma unroll
            for (int u = 0; u < 5; u++) FY[cks((u * (TY + 1) + TY) * TX + lane, NFY)] = F[u];
            if (lane < TY) {
                // x-face at the high end of row `lane`
                tile_face<0, ORD>(T, (lane + 3) * PW + TX, 1, gamma, gm1, F, bad);
                if constexpr (VISC) visc_x((lane + 3) * PW + TX + 2);
#pragma unroll
                for (int u = 0; u < 5; u++) FX[cks((u * TY + lane) * (TX + 1) + TX, NFX)] = F[u];
            }
        }
        if (more) land(P + ro[6]);
        __syncthreads();
        const int r0 = ro[0];
#pragma unroll
        for (int m = 0; m + 1 < RING; m++) ro[m] = ro[m + 1];
        ro[RING - 1] = r0;
    }
    // the last plane (its faces are behind the final barrier; its cell's
    // values are in cc from the last z-stencil)
    if (active) finish(k1 - 1);
    const bool badf = flag_bad(bad);
    if (nonfinite || badf) atomicOr(err, (nonfinite ? ERRF_NONFINITE : 0) | (badf ? ERRF_FACE : 0));
    if (mode == FLUX_STAGE3) {
        double m = block_max<NT>(double(smax));
        if (tid == 0)
            blockmax[(cz * (long long)bp.gy + bp.y) * bp.gx + bp.x] = m;
    }
}
template <int mode, int ORD, bool VISC>
__global__ void __maxnreg__(FLUX_MAXREG)
    k_flux(QIn qin, const S *__restrict__ sig, QBIn qn, Fout<5> out, QBOut outb, Frhs rhs, Fout<5> base_out,
           Geom g, C gamma, C half_inv_dx, const Scalars *sc, double *blockmax, int *err, const C *W,
           const C *J, int zc, int cz0, C mu, C lamv)
{
    flux_body<mode, ORD, VISC>(qin, sig, qn, out, outb, rhs, base_out, g, gamma, half_inv_dx, sc, blockmax, err,
                               W, J, zc, cz0, mu, lamv, BlockPos::of_launch());
}


// stand-alone stage combination (the flux kernel's epilogue) over n values;
// in the increment modes the FP32 state update of stage 3 on FP32 arrays
__global__ void k_rk_combine(const QB *__restrict__ qn, const QB *__restrict__ qs,
                             const C *__restrict__ L, QB *__restrict__ out, long long n, double dt,
                             double wd)
{
    C dt32 = C(dt), w32 = C(wd);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        C a = cv(__ldg(qn + c)), b = cv(__ldg(qs + c)), l = L[c];
        if constexpr (kNarrow && !kInc) {
            bool ok;
            S h = rk_narrow_one<S>(a, b, l, dt32, w32, ok);
            if (!ok) h = rk_fp64<S>(a, b, l, dt, wd);
            reinterpret_cast<S *>(out)[c] = h;
        } else {
            out[c] = a + w32 * ((b - a) + dt32 * l);
        }
    }
}

// ---------------------------------------------------------- wave speed
constexpr int SPEED_NT = 256, SPEED_MAXBLOCKS = 152 * 8;

__global__ void __launch_bounds__(SPEED_NT) k_speed(const QB *__restrict__ q, long long n, C gamma,
                                                     double *blockmax)
{
    double m = 0.0;
    C gm1 = gamma - C(1);
    for (long long c = blockIdx.x * (long long)SPEED_NT + threadIdx.x; c < n;
         c += (long long)gridDim.x * SPEED_NT)
        m = nanmax(m, double(cell_speed(ldc(q + c), ldc(q + n + c), ldc(q + 2 * n + c),
                                        ldc(q + 3 * n + c), ldc(q + 4 * n + c), gamma, gm1)));
    m = block_max<SPEED_NT>(m);
    if (threadIdx.x == 0) blockmax[blockIdx.x] = m;
}

// ------------------------------------------------------------ diagnostics
// FP64 evaluation of the state's totals, extrema and the residual of the
// elliptic equation (Eq. igrelliptic) for the stored Sigma:
//   (A s)_i = s_i (1/rho_i + beta sum_f c_f) - beta sum_f c_f s_nb,
//   c_f = (1/rho_i + 1/rho_nb) / 2, beta = alpha / dx^2, faces on a
//   non-periodic boundary dropped (the operator the Jacobi sweeps relax);
//   b_i = alpha [sum_ab G_ab G_ba + (sum_a G_aa)^2], G_ab the central
//   difference of u_a = m_a / rho along b (the source kernel's definition,
//   with the same boundary mapping and jet blend).
// Every stored value converts to double exactly, so the result is the FP64
// evaluation on the stored state. One thread per cell (grid-stride), per-block
// partial results in a fixed reduction order: deterministic.
constexpr int DIAG_NT = 256, DIAG_NV = DIAG_PARTS;

// conserved value u at (i, j, kk) through the boundary mapping, in FP64
__device__ __forceinline__ double dval(const QB *q, const Geom &g, const C *W, const C *J, int i,
                                       int j, int kk, int u)
{
    int mi = map_axis(i, g.nx, g.bc[0], g.bc[1]), mj = map_axis(j, g.ny, g.bc[2], g.bc[3]);
    int mk = map_axis(kk, g.nz, g.bc[4], g.bc[5]);
    idx f = (idx)(mj * g.nx + mi);
    double v = (double)cv(q[(size_t)u * (size_t)g.n + (size_t)mk * (size_t)g.plane + f]);
    if (kk < 0 && g.bc[4] == BC_INFLOW)
        v = (1.0 - (double)W[f]) * v + (double)J[(size_t)u * (size_t)g.plane + f];
    return v;
}

// velocity u_a at (i, j, kk), FP64
__device__ __forceinline__ void dvel(const QB *q, const Geom &g, const C *W, const C *J, int i, int j,
                                     int kk, double u[3])
{
    double rho = dval(q, g, W, J, i, j, kk, 0);
#pragma unroll
    for (int a = 0; a < 3; a++) u[a] = dval(q, g, W, J, i, j, kk, 1 + a) / rho;
}

__global__ void __launch_bounds__(DIAG_NT) k_diag(const QB *__restrict__ q, const S *__restrict__ sig,
                                                  Geom g, double gamma, double alpha, double dx,
                                                  const C *W, const C *J, double *part)
{
    // acc: sums of rho, mx, my, mz, E, (A s - b)^2, b^2; minima of rho, p; max |Sigma|
    double acc[DIAG_NV] = {0, 0, 0, 0, 0, 0, 0, INFINITY, INFINITY, 0};
    const double beta = alpha / (dx * dx), inv2dx = 0.5 / dx;
    for (long long c = blockIdx.x * (long long)DIAG_NT + threadIdx.x; c < g.n;
         c += (long long)gridDim.x * DIAG_NT) {
        int i = (int)(c % g.nx), j = (int)((c / g.nx) % g.ny), k = (int)(c / g.plane);
        double v[5];
#pragma unroll
        for (int u = 0; u < 5; u++) v[u] = (double)cv(q[(size_t)u * (size_t)g.n + (size_t)c]);
        double s0 = (double)cv(sig[c]);
#pragma unroll
        for (int u = 0; u < 5; u++) acc[u] += v[u];
        double p = (gamma - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / v[0]);
        acc[7] = fmin(acc[7], v[0]);
        acc[8] = fmin(acc[8], p);
        acc[9] = fmax(acc[9], fabs(s0));
        // b from central differences of u
        double G[3][3];
        const int di[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            double up[3], um[3];
            dvel(q, g, W, J, i + di[b][0], j + di[b][1], k + di[b][2], up);
            dvel(q, g, W, J, i - di[b][0], j - di[b][1], k - di[b][2], um);
#pragma unroll
            for (int a = 0; a < 3; a++) G[a][b] = (up[a] - um[a]) * inv2dx;
        }
        double tr = G[0][0] + G[1][1] + G[2][2], t2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) t2 += G[a][b] * G[b][a];
        double bv = alpha * (t2 + tr * tr);
        // A Sigma with the boundary faces of non-periodic sides dropped
        double r0 = 1.0 / v[0], diag = r0, off = 0.0;
        const int dir[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        const int ext[3] = {g.nx, g.ny, g.nz}, pos[3] = {i, j, k};
#pragma unroll
        for (int f = 0; f < 6; f++) {
            int ax = f >> 1;
            int pn = pos[ax] + ((f & 1) ? 1 : -1);
            if ((pn < 0 || pn >= ext[ax]) && g.bc[f] != BC_PERIODIC) continue;
            int ni = map_axis(i + dir[f][0], g.nx, g.bc[0], g.bc[1]);
            int nj = map_axis(j + dir[f][1], g.ny, g.bc[2], g.bc[3]);
            int nk = map_axis(k + dir[f][2], g.nz, g.bc[4], g.bc[5]);
            size_t nc = (size_t)nk * (size_t)g.plane + (size_t)nj * g.nx + ni;
            double cf = 0.5 * beta * (r0 + 1.0 / (double)cv(q[nc]));
            diag += cf;
            off += cf * (double)cv(sig[nc]);
        }
        double res = diag * s0 - off - bv;
        acc[5] += res * res;
        acc[6] += bv * bv;
    }
    // block reduction in a fixed order
    __shared__ double red[DIAG_NT / 32][DIAG_NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < DIAG_NV; t++) {
        double x = acc[t];
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            x = t < 7 ? x + y : (t < 9 ? fmin(x, y) : fmax(x, y));
        }
        if (lane == 0) red[w][t] = x;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_NV) {
        int t = threadIdx.x;
        double x = red[0][t];
        for (int ww = 1; ww < DIAG_NT / 32; ww++)
            x = t < 7 ? x + red[ww][t] : (t < 9 ? fmin(x, red[ww][t]) : fmax(x, red[ww][t]));
        part[blockIdx.x * DIAG_NV + t] = x;
    }
}

// ---------------------------------------------------------------- adjoint
// Reverse of one stage (discrete adjoint with dt frozen). Simple kernels: one
// thread per face or cell, grid-stride loops, and atomics where the forward
// gathers (each reverse stencil scatters to the cells it read). Adjoint
// values are in the arithmetic type C. Non-smooth points follow the forward's
// branch: the LF speed max(aL, aR) sends its adjoint to the side the forward
// took (aR on a tie), |u| takes sign(u) with sign(0) = 0.

__device__ __forceinline__ void aadd(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void aadd(double *p, double v) { atomicAdd(p, v); }

// forward value of field u (0..4 conserved, 5 Sigma) read at (i, j, kk):
// index mapping plus the jet blend of the -z inflow face
__device__ __forceinline__ C val_at(const S *q, const S *sig, const Geom &g, const C *W, const C *J,
                                    int i, int j, int kk, int u)
{
    int mi = map_axis(i, g.nx, g.bc[0], g.bc[1]), mj = map_axis(j, g.ny, g.bc[2], g.bc[3]);
    int mk = map_axis(kk, g.nz, g.bc[4], g.bc[5]);
    idx f = ck((idx)(mj * g.nx + mi), g.plane);
    idx c = ck((idx)mk * (idx)g.plane + f, g.n);
    if (u == 5) return ldc(sig + c);
    C v = ldc(q + ckl((size_t)u * (size_t)g.n + c, 5 * g.n));
    if (kk < 0 && g.bc[4] == BC_INFLOW)
        v = (C(1) - W[f]) * v + J[ckl((size_t)u * (size_t)g.plane + f, 5 * g.plane)];
    return v;
}

// adjoint of that read: scatter `a` back to the cell(s) the value came from
__device__ __forceinline__ void scatter_at(C *lq, C *lsig, C *lamJ, const Geom &g, const C *W, int i,
                                           int j, int kk, int u, C a)
{
    int mi = map_axis(i, g.nx, g.bc[0], g.bc[1]), mj = map_axis(j, g.ny, g.bc[2], g.bc[3]);
    int mk = map_axis(kk, g.nz, g.bc[4], g.bc[5]);
    idx f = ck((idx)(mj * g.nx + mi), g.plane);
    idx c = ck((idx)mk * (idx)g.plane + f, g.n);
    if (u == 5) {
        aadd(lsig + c, a);
        return;
    }
    const size_t qc = ckl((size_t)u * (size_t)g.n + c, 5 * g.n);
    if (kk < 0 && g.bc[4] == BC_INFLOW) {
        aadd(lq + qc, (C(1) - W[f]) * a);
        aadd(lamJ + ckl((size_t)u * (size_t)g.plane + f, 5 * g.plane), a);
        return;
    }
    aadd(lq + qc, a);
}

__global__ void k_adj_rk(const C *lout, C *lq0, C *lqs, C *Lb, long long n5, C w, C dt)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n5;
         c += (long long)gridDim.x * blockDim.x) {
        C a = lout[c];
        lq0[c] += (C(1) - w) * a;
        lqs[c] = w * a;
        Lb[c] = w * dt * a;
    }
}

// reverse of the physical flux along D at a face state v = (rho, m, E) and
// Sigma s: Fb (adjoint of F) and ab (adjoint of |u_D| + c) into vb, sb
template <int D>
__device__ __forceinline__ void flux_rev(const C v[5], C s, const C Fb[5], C ab, C gamma, C vb[5], C &sb)
{
    C rho = v[0], E = v[4], r = C(1) / rho;
    C u[3] = {v[1] * r, v[2] * r, v[3] * r};
    C ke = C(0.5) * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    C p = (gamma - C(1)) * (E - ke);
    C P = p + s;
    C c = sqrt(gamma * p * r);
    C ub[3] = {C(0), C(0), C(0)}, rhob = C(0), Eb = C(0), Pb = C(0), pb = C(0);
    rhob += Fb[0] * u[D];
    ub[D] += Fb[0] * rho;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        vb[1 + a] += Fb[1 + a] * u[D];
        ub[D] += Fb[1 + a] * v[1 + a];
    }
    Pb += Fb[1 + D] + Fb[4] * u[D];
    Eb += Fb[4] * u[D];
    ub[D] += Fb[4] * (E + P);
    ub[D] += ab * (u[D] > C(0) ? C(1) : (u[D] < C(0) ? C(-1) : C(0)));
    pb += ab * gamma / (C(2) * c * rho);
    rhob -= ab * c / (C(2) * rho);
    pb += Pb;
    sb += Pb;
    Eb += (gamma - C(1)) * pb;
    C keb = -(gamma - C(1)) * pb;
    rhob += keb * C(0.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int a = 0; a < 3; a++) ub[a] += keb * rho * u[a];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        vb[1 + a] += ub[a] * r;
        rhob -= ub[a] * u[a] * r;
    }
    vb[0] += rhob;
    vb[4] += Eb;
}

template <int D>
__device__ __forceinline__ C fwd_flux(const C v[5], C s, C gamma, C F[5])
{
    C rho = v[0], E = v[4], r = C(1) / rho;
    C u[3] = {v[1] * r, v[2] * r, v[3] * r};
    C p = (gamma - C(1)) * (E - C(0.5) * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    C P = p + s;
    F[0] = rho * u[D];
#pragma unroll
    for (int a = 0; a < 3; a++) F[1 + a] = v[1 + a] * u[D] + (a == D ? P : C(0));
    F[4] = (E + P) * u[D];
    return fabs(u[D]) + sqrt(gamma * p * r);
}

// one thread per face normal to D: face f sits between cells f-1 and f
template <int D>
__global__ void k_adj_rhs(const S *q, const S *sig, const C *Lb, C *lq, C *lsig, C *lamJ, Geom g, C gamma,
                          C inv_dx, const C *W, const C *J)
{
    const int nf[3] = {g.nx + (D == 0), g.ny + (D == 1), g.nz + (D == 2)};
    const int nd = D == 0 ? g.nx : D == 1 ? g.ny : g.nz;
    const long long total = (long long)nf[0] * nf[1] * nf[2];
    const C cl[6] = {C(2.0 / 60), C(-13.0 / 60), C(47.0 / 60), C(27.0 / 60), C(-3.0 / 60), C(0)};
    const C cr[6] = {C(0), C(-3.0 / 60), C(27.0 / 60), C(47.0 / 60), C(-13.0 / 60), C(2.0 / 60)};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int c3[3];
        c3[0] = (int)(t % nf[0]);
        c3[1] = (int)((t / nf[0]) % nf[1]);
        c3[2] = (int)(t / ((long long)nf[0] * nf[1]));
        const int f = c3[D];
        C Fb[5];
#pragma unroll
        for (int u = 0; u < 5; u++) {
            C hi = C(0), lo = C(0);
            if (f < nd) hi = Lb[ckl((size_t)u * g.n + ((size_t)c3[2] * g.ny + c3[1]) * g.nx + c3[0], 5 * g.n)];
            if (f >= 1) {
                int cc[3] = {c3[0], c3[1], c3[2]};
                cc[D] = f - 1;
                lo = Lb[ckl((size_t)u * g.n + ((size_t)cc[2] * g.ny + cc[1]) * g.nx + cc[0], 5 * g.n)];
            }
            Fb[u] = (hi - lo) * inv_dx;
        }
        C sv[6][6];
#pragma unroll
        for (int m = 0; m < 6; m++) {
            int cc[3] = {c3[0], c3[1], c3[2]};
            cc[D] += m - 3;
#pragma unroll
            for (int u = 0; u < 6; u++) sv[m][u] = val_at(q, sig, g, W, J, cc[0], cc[1], cc[2], u);
        }
        C L[6], R[6];
#pragma unroll
        for (int u = 0; u < 6; u++) {
            L[u] = rec_left(sv[0][u], sv[1][u], sv[2][u], sv[3][u], sv[4][u]);
            R[u] = rec_right(sv[1][u], sv[2][u], sv[3][u], sv[4][u], sv[5][u]);
        }
        C FL[5], FR[5];
        C aL = fwd_flux<D>(L, L[5], gamma, FL);
        C aR = fwd_flux<D>(R, R[5], gamma, FR);
        C lam = aL > aR ? aL : aR;
        C Lbv[5] = {C(0), C(0), C(0), C(0), C(0)}, Rbv[5] = {C(0), C(0), C(0), C(0), C(0)};
        C FLb[5], FRb[5], lamb = C(0);
#pragma unroll
        for (int u = 0; u < 5; u++) {
            FLb[u] = C(0.5) * Fb[u];
            FRb[u] = C(0.5) * Fb[u];
            Lbv[u] += C(0.5) * lam * Fb[u];
            Rbv[u] -= C(0.5) * lam * Fb[u];
            lamb -= C(0.5) * (R[u] - L[u]) * Fb[u];
        }
        C sLb = C(0), sRb = C(0);
        flux_rev<D>(L, L[5], FLb, aL > aR ? lamb : C(0), gamma, Lbv, sLb);
        flux_rev<D>(R, R[5], FRb, aL > aR ? C(0) : lamb, gamma, Rbv, sRb);
#pragma unroll
        for (int m = 0; m < 6; m++) {
            int cc[3] = {c3[0], c3[1], c3[2]};
            cc[D] += m - 3;
#pragma unroll
            for (int u = 0; u < 5; u++) {
                C a = cl[m] * Lbv[u] + cr[m] * Rbv[u];
                if (a != C(0)) scatter_at(lq, lsig, lamJ, g, W, cc[0], cc[1], cc[2], u, a);
            }
            C a = cl[m] * sLb + cr[m] * sRb;
            if (a != C(0)) scatter_at(lq, lsig, lamJ, g, W, cc[0], cc[1], cc[2], 5, a);
        }
    }
}

// neighbour of cell (i,j,k) across face d (0:-x .. 5:+z); false on a
// non-periodic domain boundary (no face term there)
__device__ __forceinline__ bool nbr(const Geom &g, int i, int j, int k, int d, idx &out)
{
    int c[3] = {i, j, k}, n[3] = {g.nx, g.ny, g.nz};
    int ax = d >> 1;
    c[ax] += (d & 1) ? 1 : -1;
    if (c[ax] < 0 || c[ax] >= n[ax]) {
        if (g.bc[d] != BC_PERIODIC) return false;
        c[ax] = c[ax] < 0 ? c[ax] + n[ax] : c[ax] - n[ax];
    }
    out = ck(((idx)c[2] * (idx)g.ny + (idx)c[1]) * (idx)g.nx + (idx)c[0], g.n);
    return true;
}

// mu = lambda / D_i, lb += mu
__global__ void k_adj_jac_mu(const S *q, const C *lsig, C *mu, C *lb, Geom g, C beta)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.n;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / g.plane);
        C ri = C(1) / ldc(q + t), diag = ri;
        for (int d = 0; d < 6; d++) {
            idx m;
            if (nbr(g, i, j, k, d, m)) diag += beta * C(0.5) * (ri + C(1) / ldc(q + m));
        }
        C mv = lsig[t] / diag;
        mu[t] = mv;
        lb[t] += mv;
    }
}

// gather form of the transposed sweep (the neighbour relation is symmetric):
// nl_m = sum_i beta c_im mu_i; rb_m += mu_m (beta/2 sum s_nb - F_m (1 + beta nf/2))
//                                  + sum_i mu_i beta/2 (s_m - F_i)
__global__ void k_adj_jac_gather(const S *q, const S *sk, const S *F, const C *mu, C *nl, C *rb, Geom g,
                                 C beta)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.n;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / g.plane);
        C rm = C(1) / ldc(q + t), sm = ldc(sk + t), Fm = ldc(F + t), mum = mu[t];
        C acc = C(0), ssum = C(0), rbm = C(0);
        int nfc = 0;
        for (int d = 0; d < 6; d++) {
            idx n;
            if (!nbr(g, i, j, k, d, n)) continue;
            C rn = C(1) / ldc(q + n), mun = mu[n];
            acc += beta * C(0.5) * (rm + rn) * mun;
            ssum += ldc(sk + n);
            nfc++;
            rbm += mun * C(0.5) * beta * (sm - ldc(F + n));
        }
        rbm += mum * (C(0.5) * beta * ssum - Fm * (C(1) + C(0.5) * beta * C(nfc)));
        nl[t] = acc;
        rb[t] += rbm;
    }
}

__global__ void k_adj_rho(const S *q, C *rb, C *lqs, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        C rho = ldc(q + t);
        lqs[t] -= rb[t] / (rho * rho);
        rb[t] = C(0);
    }
}

// reverse of the source at one cell: lambda_b -> u at the 6 neighbours -> (rho, m) there
__global__ void k_adj_source(const S *q, const C *lb, C *lq, C *lamJ, Geom g, C alpha, C inv2dx, const C *W,
                             const C *J)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.n;
         t += (long long)gridDim.x * blockDim.x) {
        C bb = lb[t];
        if (bb == C(0)) continue;
        int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / g.plane);
        C rho[2][3], m[2][3][3], u[2][3][3];  // [+/-][direction][component]
        for (int c = 0; c < 3; c++)
            for (int sgn = 0; sgn < 2; sgn++) {
                int cc[3] = {i, j, k};
                cc[c] += sgn == 0 ? 1 : -1;
                rho[sgn][c] = val_at(q, nullptr, g, W, J, cc[0], cc[1], cc[2], 0);
                for (int a = 0; a < 3; a++) {
                    m[sgn][c][a] = val_at(q, nullptr, g, W, J, cc[0], cc[1], cc[2], 1 + a);
                    u[sgn][c][a] = m[sgn][c][a] / rho[sgn][c];
                }
            }
        C G[3][3];
        for (int a = 0; a < 3; a++)
            for (int c = 0; c < 3; c++) G[a][c] = (u[0][c][a] - u[1][c][a]) * inv2dx;
        C tr = G[0][0] + G[1][1] + G[2][2];
        for (int c = 0; c < 3; c++)
            for (int a = 0; a < 3; a++) {
                C Gb = alpha * (C(2) * G[c][a] + (a == c ? C(2) * tr : C(0))) * bb;
                C ub = Gb * inv2dx;
                for (int sgn = 0; sgn < 2; sgn++) {
                    C us = sgn == 0 ? ub : -ub;
                    int cc[3] = {i, j, k};
                    cc[c] += sgn == 0 ? 1 : -1;
                    C r = rho[sgn][c];
                    scatter_at(lq, nullptr, lamJ, g, W, cc[0], cc[1], cc[2], 1 + a, us / r);
                    scatter_at(lq, nullptr, lamJ, g, W, cc[0], cc[1], cc[2], 0, -us * m[sgn][c][a] / (r * r));
                }
            }
    }
}

// gw[n] += sum over the inflow face of s_n (rho_n lamJ_mz + rho_n w_n lamJ_E); one block per jet
__global__ void k_adj_jets(const double *jets, const C *lamJ, double *gw, int nx, int ny, double dx)
{
    const double *jt = jets + 7 * blockIdx.x;
    long long plane = (long long)nx * ny;
    double acc = 0.0;
    for (long long f = threadIdx.x; f < plane; f += blockDim.x) {
        int i = (int)(f % nx), j = (int)(f / nx);
        double x = (i + 0.5) * dx, y = (j + 0.5) * dx;
        double r = sqrt((x - jt[0]) * (x - jt[0]) + (y - jt[1]) * (y - jt[1]));
        double sn = 0.5 * (1.0 - tanh((r - jt[2]) / (jt[6] * dx)));
        acc += sn * (jt[3] * double(lamJ[ckl(3 * plane + f, 5 * plane)]) +
                     jt[3] * jt[4] * double(lamJ[ckl(4 * plane + f, 5 * plane)]));
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gw[blockIdx.x] += red[0];
}

// ------------------------------------------------- grouped launches
// One launch covers the blocks of several independent instances: block b
// belongs to the instance whose first block blk0 is the largest <= b, and
// runs the instance's own body at its place in the instance's own grid.
struct SourceInst {
    QIn q;
    S *b, *rho_out;
    Geom g;
    C alpha_s;
    const C *W, *J;
    int zc, gx, gy, blk0;
};
struct JacobiInst {
    const S *q, *b, *sin;
    S *sout;
    Geom g;
    C beta;
    int zc, gx, gy, blk0;
};
struct FluxInst {
    QIn qin;
    const S *sig;
    QBIn qn;
    Fout<5> out;
    QBOut outb;
    Geom g;
    C gamma, half_inv_dx, mu, lamv;
    const Scalars *sc;
    double *blockmax;
    int *err;
    const C *W, *J;
    int zc, gx, gy, blk0;
};
template <class I> struct Group {
    int count;
    I d[kGroupMax];
};
static_assert(sizeof(Group<FluxInst>) <= 32000, "grouped launch descriptors exceed the kernel parameter space");

// index of the instance that owns block b (blk0 ascending, d[0].blk0 = 0)
template <class I> __device__ __forceinline__ int group_find(const Group<I> &a, int b)
{
    int lo = 0, hi = a.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.d[mid].blk0 <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <bool HASD>
__global__ void __launch_bounds__(BT) k_source_group(const __grid_constant__ Group<SourceInst> a)
{
    const SourceInst &d = a.d[group_find(a, blockIdx.x)];
    source_body<HASD>(d.q, d.b, d.rho_out, d.g, d.alpha_s, d.W, d.J, d.zc,
                      BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy));
}
template <bool HASD>
__global__ void __launch_bounds__(BT, SOURCE_V4_BLOCKS) k_source_v4_group(const __grid_constant__ Group<SourceInst> a)
{
    const SourceInst &d = a.d[group_find(a, blockIdx.x)];
    source_v4_body<HASD>(d.q, d.b, d.rho_out, d.g, d.alpha_s, d.W, d.J, d.zc,
                         BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy));
}
__global__ void __launch_bounds__(BT) k_jacobi_group(const __grid_constant__ Group<JacobiInst> a, int colour)
{
    const JacobiInst &d = a.d[group_find(a, blockIdx.x)];
    jacobi_body(d.q, d.b, d.sin, d.sout, d.g, d.beta, d.zc, colour,
                BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy));
}
__global__ void __launch_bounds__(BT, JACOBI_V4_BLOCKS) k_jacobi_v4_group(const __grid_constant__ Group<JacobiInst> a,
                                                                         int colour)
{
    const JacobiInst &d = a.d[group_find(a, blockIdx.x)];
    jacobi_v4_body(d.q, d.b, d.sin, d.sout, d.g, d.beta, d.zc, colour,
                   BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy));
}
template <bool HASD>
__global__ void __launch_bounds__(BT, SOURCE_V4_BLOCKS) k_source_v4_full_group(const __grid_constant__ Group<SourceInst> a)
{
    const SourceInst &d = a.d[group_find(a, blockIdx.x)];
    source_v4_full<HASD>(d.q, d.b, d.rho_out, d.g, d.alpha_s, d.W, d.J, d.zc,
                         BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy));
}
template <bool RB>
__global__ void __launch_bounds__(BT, JACOBI_V4_BLOCKS) k_jacobi_v4_full_group(const __grid_constant__ Group<JacobiInst> a,
                                                                              int colour)
{
    if constexpr (sizeof(C) == 4) {
        __shared__ __align__(16) C R[2][HY][HXV];
        __shared__ __align__(16) C SG[2][HY][HXV];
        const JacobiInst &d = a.d[group_find(a, blockIdx.x)];
        jacobi_v4_full<RB>(d.q, d.b, d.sin, d.sout, d.g, d.beta, d.zc, colour,
                           BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy), R, SG);
    }
}
template <int mode, int ORD, bool VISC>
__global__ void __maxnreg__(FLUX_MAXREG) k_flux_group(const __grid_constant__ Group<FluxInst> a)
{
    const FluxInst &d = a.d[group_find(a, blockIdx.x)];
    const Frhs none_rhs = {};
    const Fout<5> none_base = {};
    flux_body<mode, ORD, VISC>(d.qin, d.sig, d.qn, d.out, d.outb, none_rhs, none_base, d.g, d.gamma,
                               d.half_inv_dx, d.sc, d.blockmax, d.err, d.W, d.J, d.zc, 0, d.mu, d.lamv,
                               BlockPos::of_index(blockIdx.x - d.blk0, d.gx, d.gy));
}

// ------------------------------------------------------------ launchers
dim3 grid_of(const Geom &g, int bx, int by, int zc)
{
    return dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, (g.nz + zc - 1) / zc);
}

template <int N> Fin<N> fields_in(const void *base, long long n)
{
    Fin<N> f;
    for (int u = 0; u < N; u++) f.p[u] = base ? (const S *)base + u * n : nullptr;
    return f;
}

// state input: base fields q (type QB) and increments qd (type S, or NULL)
QIn state_in(const void *q, const void *qd, long long n)
{
    QIn f;
    for (int u = 0; u < 5; u++) {
        f.b[u] = q ? (const QB *)q + u * n : nullptr;
        f.d[u] = qd ? (const S *)qd + u * n : nullptr;
    }
    f.fs = (size_t)n;
    return f;
}

cudaError_t launch_source(const Geom &g, const Phys &p, const Tiles &t, const Inflow &in,
                          const void *q, const void *qd, void *b, void *rho_out, cudaStream_t st)
{
    if (kInc != (rho_out != nullptr)) return cudaErrorInvalidValue;  // the stage density: increment modes only
    if (!kInc && qd) return cudaErrorInvalidValue;
    const QIn qi = state_in(q, qd, g.n);
    const C as = C(p.alpha * 0.25 / (p.dx * p.dx));
    const C *W = (const C *)in.W, *J = (const C *)in.J;
    if (t.vec_source && g.nx % VX == 0) {
        auto kern = qd ? k_source_v4<kInc> : k_source_v4<false>;
        // 16-bit storage: grids whose tiles all lie inside take the full-tile
        // kernel (FP16 increments, full-size plume: 12.0 -> 10.7 ms); with
        // FP32 storage it measured slower (8.6 -> 10.5 ms) and is not used
        if (sizeof(S) == 2 && g.nx % TXV == 0 && g.ny % BY == 0)
            kern = qd ? k_source_v4_full<kInc> : k_source_v4_full<false>;
        kern<<<grid_of(g, TXV, BY, t.zc_source), dim3(BX, BY), 0, st>>>(qi, (S *)b, (S *)rho_out, g, as, W, J,
                                                                       t.zc_source);
        return cudaGetLastError();
    }
    auto kern = qd ? k_source<kInc> : k_source<false>;
    kern<<<grid_of(g, BX, BY, t.zc_source), dim3(BX, BY), 0, st>>>(qi, (S *)b, (S *)rho_out, g, as, W, J,
                                                                   t.zc_source);
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const Geom &g, const Phys &p, const Tiles &t, const void *q,
                          const void *b, const void *s_in, void *s_out, int colour, cudaStream_t st)
{
    if (t.vec_jacobi && g.nx % VX == 0) {
        if (sizeof(C) == 4 && g.nx % TXV == 0 && g.ny % BY == 0) {
            auto kern = colour < 0 ? k_jacobi_v4_full<false> : k_jacobi_v4_full<true>;
            kern<<<grid_of(g, TXV, BY, t.zc_jacobi), dim3(BX, BY), 0, st>>>(
                (const S *)q, (const S *)b, (const S *)s_in, (S *)s_out, g, C(p.alpha / (p.dx * p.dx)),
                t.zc_jacobi, colour);
            return cudaGetLastError();
        }
        k_jacobi_v4<<<grid_of(g, TXV, BY, t.zc_jacobi), dim3(BX, BY), 0, st>>>(
            (const S *)q, (const S *)b, (const S *)s_in, (S *)s_out, g, C(p.alpha / (p.dx * p.dx)),
            t.zc_jacobi, colour);
        return cudaGetLastError();
    }
    k_jacobi<<<grid_of(g, BX, BY, t.zc_jacobi), dim3(BX, BY), 0, st>>>(
        (const S *)q, (const S *)b, (const S *)s_in, (S *)s_out, g, C(p.alpha / (p.dx * p.dx)),
        t.zc_jacobi, colour);
    return cudaGetLastError();
}

long long flux_blocks(const Geom &g, const Tiles &t)
{
    dim3 gr = grid_of(g, TX, TY, t.zc_flux);
    return (long long)gr.x * gr.y * gr.z;
}

cudaError_t launch_flux(const Geom &g, const Phys &p, const Tiles &t, const Inflow &in, int mode,
                        const void *qs, const void *qd, const void *sig, const void *qn, void *out, void *rhs,
                        void *base_out, const Scalars *sc, double *blockmax, int *err, cudaStream_t st)
{
    // increments are read from stage 2 on, and only in the increment modes
    if ((qd != nullptr) != (kInc && (mode == FLUX_STAGE2 || mode == FLUX_STAGE3))) return cudaErrorInvalidValue;
    if (kInc && base_out) return cudaErrorInvalidValue;
    size_t smem = flux_smem_bytes();
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const QIn fi = state_in(qs, qd, g.n);
        QBIn fn;
        Fout<5> fo, fb;
        QBOut fob;
        Frhs fr;
        // the stage output: increments (S) for stages 1 and 2 of the increment
        // modes, the FP32 state for their stage 3, else the stored state (S)
        const bool out_is_state = !kInc || mode == FLUX_STAGE3;
        for (int u = 0; u < 5; u++) {
            fn.p[u] = qn ? (const QB *)qn + u * g.n : nullptr;
            fo.p[u] = out && !(kInc && out_is_state) ? (S *)out + u * g.n : nullptr;
            fob.p[u] = out && kInc && out_is_state ? (QB *)out + u * g.n : nullptr;
            fb.p[u] = base_out ? (S *)base_out + u * g.n : nullptr;
            fr.p[u] = rhs ? (C *)rhs + u * g.n : nullptr;
        }
        // the z-chunks of planes [z_begin, z_end) (all chunks when z_end = 0)
        dim3 gr = grid_of(g, TX, TY, t.zc_flux);
        const int cz0 = t.z_begin / t.zc_flux;
        if (t.z_end > 0) gr.z = (t.z_end - t.z_begin + t.zc_flux - 1) / t.zc_flux;
        kern<<<gr, NT, smem, st>>>(fi, (const S *)sig, fn, fo, fob, fr, fb, g, C(p.gamma), C(0.5 / p.dx), sc,
                                   blockmax, err, (const C *)in.W, (const C *)in.J, t.zc_flux, cz0, C(p.mu),
                                   C(p.zeta - 2.0 * p.mu / 3.0));
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess)
                fprintf(stderr, "igr: flux launch failed (%s): block %d, regs %d, max threads %d, "
                                "static smem %zu, dynamic smem %zu, local %zu\n",
                        cudaGetErrorString(e), NT, fa.numRegs, fa.maxThreadsPerBlock,
                        fa.sharedSizeBytes, smem, fa.localSizeBytes);
        }
        return e;
    };
    auto by_mode = [&](auto k0, auto k1, auto k2, auto k3) {
        switch (mode) {
        case FLUX_RHS: return go(k0);
        case FLUX_STAGE1: return go(k1);
        case FLUX_STAGE2: return go(k2);
        default: return go(k3);
        }
    };
    const bool visc = p.mu != 0.0 || p.zeta != 0.0;
    if (p.order == 3) {
        if (visc)
            return by_mode(k_flux<FLUX_RHS, 3, true>, k_flux<FLUX_STAGE1, 3, true>,
                           k_flux<FLUX_STAGE2, 3, true>, k_flux<FLUX_STAGE3, 3, true>);
        return by_mode(k_flux<FLUX_RHS, 3, false>, k_flux<FLUX_STAGE1, 3, false>,
                       k_flux<FLUX_STAGE2, 3, false>, k_flux<FLUX_STAGE3, 3, false>);
    }
    if (visc)
        return by_mode(k_flux<FLUX_RHS, 5, true>, k_flux<FLUX_STAGE1, 5, true>,
                       k_flux<FLUX_STAGE2, 5, true>, k_flux<FLUX_STAGE3, 5, true>);
    return by_mode(k_flux<FLUX_RHS, 5, false>, k_flux<FLUX_STAGE1, 5, false>,
                   k_flux<FLUX_STAGE2, 5, false>, k_flux<FLUX_STAGE3, 5, false>);
}

// ---- grouped launches: calls are split by kernel form and in chunks of
// kGroupMax; each chunk is one launch over all its instances' blocks

// run fn(first, count) over the runs of consecutive calls with equal key(call)
template <class T, class K, class F>
cudaError_t by_runs(const T *calls, int n, K key, F fn)
{
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && j - i < kGroupMax && key(calls[j]) == key(calls[i])) j++;
        cudaError_t e = fn(calls + i, j - i);
        if (e != cudaSuccess) return e;
        i = j;
    }
    return cudaSuccess;
}

cudaError_t launch_source_group(const SourceCall *calls, int n, cudaStream_t st)
{
    for (int i = 0; i < n; i++)
        if ((kInc != (calls[i].rho_out != nullptr)) || (!kInc && calls[i].qd)) return cudaErrorInvalidValue;
    // 0: one cell per thread, 1: four cells, 2: four cells, every tile inside
    // the grid (16-bit storage; as launch_source)
    auto vec = [](const SourceCall &c) {
        if (!c.t.vec_source || c.g.nx % VX != 0) return 0;
        return sizeof(S) == 2 && c.g.nx % TXV == 0 && c.g.ny % BY == 0 ? 2 : 1;
    };
    auto key = [&](const SourceCall &c) { return 2 * vec(c) + (c.qd ? 1 : 0); };
    return by_runs(calls, n, key, [&](const SourceCall *cs, int m) {
        Group<SourceInst> a;
        a.count = m;
        int blk = 0;
        const int v = vec(cs[0]);
        for (int i = 0; i < m; i++) {
            const SourceCall &c = cs[i];
            SourceInst &d = a.d[i];
            d.q = state_in(c.q, c.qd, c.g.n);
            d.b = (S *)c.b;
            d.rho_out = (S *)c.rho_out;
            d.g = c.g;
            d.alpha_s = C(c.p.alpha * 0.25 / (c.p.dx * c.p.dx));
            d.W = (const C *)c.in.W;
            d.J = (const C *)c.in.J;
            d.zc = c.t.zc_source;
            const dim3 gr = grid_of(c.g, v ? TXV : BX, BY, d.zc);
            d.gx = (int)gr.x;
            d.gy = (int)gr.y;
            d.blk0 = blk;
            blk += (int)(gr.x * gr.y * gr.z);
        }
        auto kern = v == 2 ? (cs[0].qd ? k_source_v4_full_group<kInc> : k_source_v4_full_group<false>)
                    : v ? (cs[0].qd ? k_source_v4_group<kInc> : k_source_v4_group<false>)
                        : (cs[0].qd ? k_source_group<kInc> : k_source_group<false>);
        kern<<<blk, dim3(BX, BY), 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_jacobi_group(const JacobiCall *calls, int n, int colour, cudaStream_t st)
{
    // 0: one cell per thread, 1: four cells, 2: four cells, every tile inside
    // the grid (FP32 arithmetic; as launch_jacobi)
    auto vec = [](const JacobiCall &c) {
        if (!c.t.vec_jacobi || c.g.nx % VX != 0) return 0;
        return sizeof(C) == 4 && c.g.nx % TXV == 0 && c.g.ny % BY == 0 ? 2 : 1;
    };
    return by_runs(calls, n, vec, [&](const JacobiCall *cs, int m) {
        Group<JacobiInst> a;
        a.count = m;
        int blk = 0;
        const int v = vec(cs[0]);
        for (int i = 0; i < m; i++) {
            const JacobiCall &c = cs[i];
            JacobiInst &d = a.d[i];
            d.q = (const S *)c.q;
            d.b = (const S *)c.b;
            d.sin = (const S *)c.s_in;
            d.sout = (S *)c.s_out;
            d.g = c.g;
            d.beta = C(c.p.alpha / (c.p.dx * c.p.dx));
            d.zc = c.t.zc_jacobi;
            const dim3 gr = grid_of(c.g, v ? TXV : BX, BY, d.zc);
            d.gx = (int)gr.x;
            d.gy = (int)gr.y;
            d.blk0 = blk;
            blk += (int)(gr.x * gr.y * gr.z);
        }
        if (v == 2) {
            auto kern = colour < 0 ? k_jacobi_v4_full_group<false> : k_jacobi_v4_full_group<true>;
            kern<<<blk, dim3(BX, BY), 0, st>>>(a, colour);
        } else if (v) {
            k_jacobi_v4_group<<<blk, dim3(BX, BY), 0, st>>>(a, colour);
        } else {
            k_jacobi_group<<<blk, dim3(BX, BY), 0, st>>>(a, colour);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_flux_group(const FluxCall *calls, int n, int mode, cudaStream_t st)
{
    if (mode == FLUX_RHS) return cudaErrorInvalidValue;
    for (int i = 0; i < n; i++)
        if ((calls[i].qd != nullptr) != (kInc && (mode == FLUX_STAGE2 || mode == FLUX_STAGE3)) ||
            calls[i].t.z_end != 0)
            return cudaErrorInvalidValue;
    auto kind = [](const FluxCall &c) {
        return 2 * (c.p.order == 3 ? 1 : 0) + (c.p.mu != 0.0 || c.p.zeta != 0.0 ? 1 : 0);
    };
    const size_t smem = flux_smem_bytes();
    return by_runs(calls, n, kind, [&](const FluxCall *cs, int m) {
        Group<FluxInst> a;
        a.count = m;
        int blk = 0;
        const bool out_is_state = !kInc || mode == FLUX_STAGE3;
        for (int i = 0; i < m; i++) {
            const FluxCall &c = cs[i];
            FluxInst &d = a.d[i];
            d.qin = state_in(c.qs, c.qd, c.g.n);
            d.sig = (const S *)c.sig;
            for (int u = 0; u < 5; u++) {
                d.qn.p[u] = c.qn ? (const QB *)c.qn + u * c.g.n : nullptr;
                d.out.p[u] = c.out && !(kInc && out_is_state) ? (S *)c.out + u * c.g.n : nullptr;
                d.outb.p[u] = c.out && kInc && out_is_state ? (QB *)c.out + u * c.g.n : nullptr;
            }
            d.g = c.g;
            d.gamma = C(c.p.gamma);
            d.half_inv_dx = C(0.5 / c.p.dx);
            d.mu = C(c.p.mu);
            d.lamv = C(c.p.zeta - 2.0 * c.p.mu / 3.0);
            d.sc = c.sc;
            d.blockmax = c.blockmax;
            d.err = c.err;
            d.W = (const C *)c.in.W;
            d.J = (const C *)c.in.J;
            d.zc = c.t.zc_flux;
            const dim3 gr = grid_of(c.g, TX, TY, d.zc);
            d.gx = (int)gr.x;
            d.gy = (int)gr.y;
            d.blk0 = blk;
            blk += (int)(gr.x * gr.y * gr.z);
        }
        auto go = [&](auto kern) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            kern<<<blk, NT, smem, st>>>(a);
            return cudaGetLastError();
        };
        auto by_mode = [&](auto k1, auto k2, auto k3) {
            return mode == FLUX_STAGE1 ? go(k1) : mode == FLUX_STAGE2 ? go(k2) : go(k3);
        };
        switch (kind(cs[0])) {
        case 0:
            return by_mode(k_flux_group<FLUX_STAGE1, 5, false>, k_flux_group<FLUX_STAGE2, 5, false>,
                           k_flux_group<FLUX_STAGE3, 5, false>);
        case 1:
            return by_mode(k_flux_group<FLUX_STAGE1, 5, true>, k_flux_group<FLUX_STAGE2, 5, true>,
                           k_flux_group<FLUX_STAGE3, 5, true>);
        case 2:
            return by_mode(k_flux_group<FLUX_STAGE1, 3, false>, k_flux_group<FLUX_STAGE2, 3, false>,
                           k_flux_group<FLUX_STAGE3, 3, false>);
        default:
            return by_mode(k_flux_group<FLUX_STAGE1, 3, true>, k_flux_group<FLUX_STAGE2, 3, true>,
                           k_flux_group<FLUX_STAGE3, 3, true>);
        }
    });
}

cudaError_t launch_speed(const Geom &g, const Phys &p, const void *q, double *blockmax,
                         int *nblocks, cudaStream_t st)
{
    long long want = (g.n + SPEED_NT - 1) / SPEED_NT;
    int nb = (int)(want < SPEED_MAXBLOCKS ? want : SPEED_MAXBLOCKS);
    k_speed<<<nb, SPEED_NT, 0, st>>>((const QB *)q, g.n, C(p.gamma), blockmax);
    *nblocks = nb;
    return cudaGetLastError();
}

cudaError_t launch_rk_combine(const void *qn, const void *qs, const void *L, void *out,
                              long long n, double dt, double w, cudaStream_t st)
{
    long long want = (n + 255) / 256;
    int nb = (int)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
    k_rk_combine<<<nb, 256, 0, st>>>((const QB *)qn, (const QB *)qs, (const C *)L, (QB *)out, n, dt, w);
    return cudaGetLastError();
}

int adj_blocks(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

cudaError_t launch_adj_rk(const void *lout, void *lq0, void *lqs, void *Lb, long long n5, double w,
                          double dt, cudaStream_t st)
{
    k_adj_rk<<<adj_blocks(n5), 256, 0, st>>>((const C *)lout, (C *)lq0, (C *)lqs, (C *)Lb, n5, C(w), C(dt));
    return cudaGetLastError();
}

cudaError_t launch_adj_rhs(const Geom &g, const Phys &p, const Inflow &in, const void *qs, const void *sig,
                           const void *Lb, void *lqs, void *lsig, void *lamJ, cudaStream_t st)
{
    long long nfx = (long long)(g.nx + 1) * g.ny * g.nz, nfy = (long long)g.nx * (g.ny + 1) * g.nz,
              nfz = (long long)g.nx * g.ny * (g.nz + 1);
    const C *W = (const C *)in.W, *J = (const C *)in.J;
    k_adj_rhs<0><<<adj_blocks(nfx), 256, 0, st>>>((const S *)qs, (const S *)sig, (const C *)Lb, (C *)lqs,
                                                   (C *)lsig, (C *)lamJ, g, C(p.gamma), C(1.0 / p.dx), W, J);
    k_adj_rhs<1><<<adj_blocks(nfy), 256, 0, st>>>((const S *)qs, (const S *)sig, (const C *)Lb, (C *)lqs,
                                                   (C *)lsig, (C *)lamJ, g, C(p.gamma), C(1.0 / p.dx), W, J);
    k_adj_rhs<2><<<adj_blocks(nfz), 256, 0, st>>>((const S *)qs, (const S *)sig, (const C *)Lb, (C *)lqs,
                                                   (C *)lsig, (C *)lamJ, g, C(p.gamma), C(1.0 / p.dx), W, J);
    return cudaGetLastError();
}

cudaError_t launch_adj_jacobi(const Geom &g, const Phys &p, const void *q, const void *sk, const void *F,
                              const void *lsig, void *nl, void *lb, void *rb, void *mu, cudaStream_t st)
{
    C beta = C(p.alpha / (p.dx * p.dx));
    k_adj_jac_mu<<<adj_blocks(g.n), 256, 0, st>>>((const S *)q, (const C *)lsig, (C *)mu, (C *)lb, g, beta);
    k_adj_jac_gather<<<adj_blocks(g.n), 256, 0, st>>>((const S *)q, (const S *)sk, (const S *)F,
                                                       (const C *)mu, (C *)nl, (C *)rb, g, beta);
    return cudaGetLastError();
}

cudaError_t launch_adj_rho(const Geom &g, const void *q, void *rb, void *lqs, cudaStream_t st)
{
    k_adj_rho<<<adj_blocks(g.n), 256, 0, st>>>((const S *)q, (C *)rb, (C *)lqs, g.n);
    return cudaGetLastError();
}

cudaError_t launch_adj_source(const Geom &g, const Phys &p, const Inflow &in, const void *q, const void *lb,
                              void *lqs, void *lamJ, cudaStream_t st)
{
    k_adj_source<<<adj_blocks(g.n), 256, 0, st>>>((const S *)q, (const C *)lb, (C *)lqs, (C *)lamJ, g,
                                                   C(p.alpha), C(0.5 / p.dx), (const C *)in.W, (const C *)in.J);
    return cudaGetLastError();
}

cudaError_t launch_adj_jets(const Geom &g, const Phys &p, const double *jets, int njets, const void *lamJ,
                            double *gw, cudaStream_t st)
{
    if (njets <= 0) return cudaSuccess;
    k_adj_jets<<<njets, 256, 0, st>>>(jets, (const C *)lamJ, gw, g.nx, g.ny, p.dx);
    return cudaGetLastError();
}

cudaError_t launch_diag(const Geom &g, const Phys &p, const Inflow &in, const void *q, const void *sig,
                        double *part, int *nblocks, cudaStream_t st)
{
    long long nb = (g.n + DIAG_NT - 1) / DIAG_NT;
    int blocks = (int)(nb < DIAG_BLOCKS_MAX ? nb : DIAG_BLOCKS_MAX);
    *nblocks = blocks;
    k_diag<<<blocks, DIAG_NT, 0, st>>>((const QB *)q, (const S *)sig, g, p.gamma, p.alpha, p.dx,
                                        (const C *)in.W, (const C *)in.J, part);
    return cudaGetLastError();
}

// debug build: read (and clear) the bounds-check counter; the self-test
// forms one index past the end of an array of n values (checked, not used)
__global__ void k_bounds_selftest(long long n, int *sink)
{
    idx c = ck((idx)(n + 5), n);
    if (c != 0) *sink = (int)c;  // never taken: the check returns 0
}

unsigned long long bounds_hits(int clear)
{
#ifdef IGR_DEBUG_BOUNDS
    unsigned long long h = 0;
    if (cudaMemcpyFromSymbol(&h, g_bounds_hits, sizeof h) != cudaSuccess) return ~0ull;
    if (clear) {
        unsigned long long z = 0;
        if (cudaMemcpyToSymbol(g_bounds_hits, &z, sizeof z) != cudaSuccess) return ~0ull;
    }
    return h;
#else
    (void)clear;
    return ~0ull;  // not a debug build
#endif
}

cudaError_t bounds_selftest(int *sink, cudaStream_t st)
{
    k_bounds_selftest<<<1, 1, 0, st>>>(1000, sink);
    return cudaGetLastError();
}

}  // namespace

extern const Ops IGR_OPS = {
    (int)sizeof(S), (int)sizeof(C), (int)sizeof(QB), launch_source, launch_jacobi, launch_flux, flux_blocks,
    launch_speed, launch_rk_combine, launch_adj_rk, launch_adj_rhs, launch_adj_jacobi, launch_adj_rho,
    launch_adj_source, launch_adj_jets, launch_diag, bounds_hits, bounds_selftest,
    launch_source_group, launch_jacobi_group, launch_flux_group,
};

}  // namespace igr
