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

// ------------------------------------------------------------ load/store
__device__ __forceinline__ double ldc(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldc(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldc(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ldc(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

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
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double sqrt_c(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_c(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double div_c(double a, double b) { return a / b; }
__device__ __forceinline__ float div_c(float a, float b) { return __fdividef(a, b); }

// products that are never fused into a following add: velocities u = m/rho
// must round before they are differenced, so equal neighbours give an exact 0
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// NaN-propagating maximum (a NaN wave speed must reach dt)
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

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

// Local Lax-Friedrichs flux along axis D from face states (rho, mx, my, mz,
// E, Sigma) on the left and right: F_hat = (F_L + F_R)/2 - lam (q_R - q_L)/2,
// F = (m_D, m u_D + (p + Sigma) e_D, (E + p + Sigma) u_D),
// p = (gamma - 1)(E - |m|^2 / (2 rho)), lam = max(|u_D| + c) over both sides,
// c = sqrt(gamma p / rho). Flags a non-positive face density or pressure.
template <int D>
__device__ __forceinline__ void lf_flux(const C *L, const C *R, C gamma, C gm1, C *F, bool &bad)
{
    C rL = rcp(L[0]), rR = rcp(R[0]);
    C uL = L[1 + D] * rL, uR = R[1 + D] * rR;
    C pL = gm1 * (L[4] - C(0.5) * (L[1] * L[1] + L[2] * L[2] + L[3] * L[3]) * rL);
    C pR = gm1 * (R[4] - C(0.5) * (R[1] * R[1] + R[2] * R[2] + R[3] * R[3]) * rR);
    bad |= !(L[0] > C(0) && R[0] > C(0) && pL > C(0) && pR > C(0));
    C aL = fabs(uL) + sqrt_c(gamma * pL * rL);
    C aR = fabs(uR) + sqrt_c(gamma * pR * rR);
    C h = C(0.5) * (aL > aR ? aL : aR);
    C PL = pL + L[5], PR = pR + R[5];
    F[0] = C(0.5) * (L[1 + D] + R[1 + D]) - h * (R[0] - L[0]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C f = C(0.5) * (L[1 + a] * uL + R[1 + a] * uR);
        if (a == D) f += C(0.5) * (PL + PR);
        F[1 + a] = f - h * (R[1 + a] - L[1 + a]);
    }
    F[4] = C(0.5) * ((L[4] + PL) * uL + (R[4] + PR) * uR) - h * (R[4] - L[4]);
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

constexpr int BX = 32, BY = 8;  // tile of the source and Jacobi kernels

// --------------------------------------------------------------- source
// u at column (i, j), plane kk (kk may leave the domain through -z/+z)
__device__ __forceinline__ void col_u(const S *__restrict__ q, const Geom &g, const C *W,
                                      const C *J, int i, int j, int kk, C u[3])
{
    int km = map_axis(kk, g.nz, g.bc[4], g.bc[5]);
    long long c = km * g.plane + (long long)j * g.nx + i;
    C rho = ldc(q + c), m0 = ldc(q + g.n + c), m1 = ldc(q + 2 * g.n + c), m2 = ldc(q + 3 * g.n + c);
    if (kk < 0 && g.bc[4] == BC_INFLOW) {
        long long f = (long long)j * g.nx + i;
        C w = C(1) - W[f];
        rho = w * rho + J[f];
        m0 = w * m0 + J[g.plane + f];
        m1 = w * m1 + J[2 * g.plane + f];
        m2 = w * m2 + J[3 * g.plane + f];
    }
    C r = rcp(rho);
    u[0] = mul_rn(m0, r);
    u[1] = mul_rn(m1, r);
    u[2] = mul_rn(m2, r);
}

__device__ __forceinline__ void plane_u(const S *__restrict__ q, const Geom &g, long long c, C u[3])
{
    C r = rcp(ldc(q + c));
    u[0] = mul_rn(ldc(q + g.n + c), r);
    u[1] = mul_rn(ldc(q + 2 * g.n + c), r);
    u[2] = mul_rn(ldc(q + 3 * g.n + c), r);
}

__global__ void __launch_bounds__(BX *BY) k_source(const S *__restrict__ q, S *__restrict__ b,
                                                    Geom g, C alpha, C inv2dx, const C *W,
                                                    const C *J, int zc)
{
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    int k0 = blockIdx.z * zc, k1 = min(g.nz, k0 + zc);
    int im = map_axis(i - 1, g.nx, g.bc[0], g.bc[1]), ip = map_axis(i + 1, g.nx, g.bc[0], g.bc[1]);
    int jm = map_axis(j - 1, g.ny, g.bc[2], g.bc[3]), jp = map_axis(j + 1, g.ny, g.bc[2], g.bc[3]);
    C um[3], u0[3], up[3];  // z-neighbours of the column
    col_u(q, g, W, J, i, j, k0 - 1, um);
    col_u(q, g, W, J, i, j, k0, u0);
    for (int k = k0; k < k1; k++) {
        col_u(q, g, W, J, i, j, k + 1, up);
        long long pk = k * g.plane;
        C uxm[3], uxp[3], uym[3], uyp[3];
        plane_u(q, g, pk + (long long)j * g.nx + im, uxm);
        plane_u(q, g, pk + (long long)j * g.nx + ip, uxp);
        plane_u(q, g, pk + (long long)jm * g.nx + i, uym);
        plane_u(q, g, pk + (long long)jp * g.nx + i, uyp);
        C G[3][3];  // G[a][c] = d u_a / d x_c
#pragma unroll
        for (int a = 0; a < 3; a++) {
            G[a][0] = (uxp[a] - uxm[a]) * inv2dx;
            G[a][1] = (uyp[a] - uym[a]) * inv2dx;
            G[a][2] = (up[a] - um[a]) * inv2dx;
        }
        C tr = G[0][0] + G[1][1] + G[2][2];
        C tr2 = G[0][0] * G[0][0] + G[1][1] * G[1][1] + G[2][2] * G[2][2] +
                C(2) * (G[0][1] * G[1][0] + G[0][2] * G[2][0] + G[1][2] * G[2][1]);
        stc(b + pk + (long long)j * g.nx + i, alpha * (tr2 + tr * tr));
#pragma unroll
        for (int a = 0; a < 3; a++) {
            um[a] = u0[a];
            u0[a] = up[a];
        }
    }
}

// --------------------------------------------------------------- Jacobi
__global__ void __launch_bounds__(BX *BY) k_jacobi(const S *__restrict__ q, const S *__restrict__ b,
                                                    const S *__restrict__ sin, S *__restrict__ sout,
                                                    Geom g, C beta, int zc)
{
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    int k0 = blockIdx.z * zc, k1 = min(g.nz, k0 + zc);
    // neighbour existence (a non-periodic boundary face carries no term)
    bool hxm = i > 0 || g.bc[0] == BC_PERIODIC, hxp = i < g.nx - 1 || g.bc[1] == BC_PERIODIC;
    bool hym = j > 0 || g.bc[2] == BC_PERIODIC, hyp = j < g.ny - 1 || g.bc[3] == BC_PERIODIC;
    int im = wrap(i - 1, g.nx), ip = wrap(i + 1, g.nx), jm = wrap(j - 1, g.ny), jp = wrap(j + 1, g.ny);
    long long col = (long long)j * g.nx + i;
    // column values at k-1, k, k+1 (reciprocal density and sigma)
    auto colv = [&](int kk, C &r, C &s) {
        int km = wrap(kk, g.nz);
        r = rcp(ldc(q + km * g.plane + col));
        s = ldc(sin + km * g.plane + col);
    };
    C rm, sm, r0, s0, rp, sp;
    colv(k0 - 1, rm, sm);
    colv(k0, r0, s0);
    C half_beta = C(0.5) * beta;
    for (int k = k0; k < k1; k++) {
        colv(k + 1, rp, sp);
        long long pk = k * g.plane;
        C diag = r0, off = C(0);
        // order of faces: -x, +x, -y, +y, -z, +z
        auto face = [&](bool has, long long c) {
            if (has) {
                C cf = half_beta * (r0 + rcp(ldc(q + c)));
                diag += cf;
                off += cf * ldc(sin + c);
            }
        };
        face(hxm, pk + (long long)j * g.nx + im);
        face(hxp, pk + (long long)j * g.nx + ip);
        face(hym, pk + (long long)jm * g.nx + i);
        face(hyp, pk + (long long)jp * g.nx + i);
        bool hzm = k > 0 || g.bc[4] == BC_PERIODIC, hzp = k < g.nz - 1 || g.bc[5] == BC_PERIODIC;
        if (hzm) {
            C cf = half_beta * (r0 + rm);
            diag += cf;
            off += cf * sm;
        }
        if (hzp) {
            C cf = half_beta * (r0 + rp);
            diag += cf;
            off += cf * sp;
        }
        stc(sout + pk + col, div_c(ldc(b + pk + col) + off, diag));
        rm = r0; sm = s0;
        r0 = rp; s0 = sp;
    }
}

// ----------------------------------------------------------------- flux
constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int PW = TX + 6, PH = TY + 6;  // plane tile with a halo of 3

__host__ __device__ constexpr size_t flux_smem_elems()
{
    return 6 * PH * PW + 5 * TY * (TX + 1) + 5 * (TY + 1) * TX;
}

// one column value set (rho, mx, my, mz, E, Sigma) at plane kk, with the
// -z inflow blend for kk < 0
__device__ __forceinline__ void col_load(const S *__restrict__ qs, const S *__restrict__ sig,
                                         const Geom &g, const C *W, const C *J, int i, int j,
                                         int kk, C v[6])
{
    int km = map_axis(kk, g.nz, g.bc[4], g.bc[5]);
    long long c = km * g.plane + (long long)j * g.nx + i;
#pragma unroll
    for (int u = 0; u < 5; u++) v[u] = ldc(qs + u * g.n + c);
    v[5] = ldc(sig + c);
    if (kk < 0 && g.bc[4] == BC_INFLOW) {
        long long f = (long long)j * g.nx + i;
        C w = C(1) - W[f];
#pragma unroll
        for (int u = 0; u < 5; u++) v[u] = w * v[u] + J[u * g.plane + f];
    }
}

template <int D>
__device__ __forceinline__ void face_from_stencil(const C (&s)[6][6], C gamma, C gm1, C *F,
                                                  bool &bad)
{
    C L[6], R[6];
#pragma unroll
    for (int u = 0; u < 6; u++) {
        L[u] = rec_left(s[0][u], s[1][u], s[2][u], s[3][u], s[4][u]);
        R[u] = rec_right(s[1][u], s[2][u], s[3][u], s[4][u], s[5][u]);
    }
    lf_flux<D>(L, R, gamma, gm1, F, bad);
}

__global__ void __launch_bounds__(NT) k_flux(const S *__restrict__ qs, const S *__restrict__ sig,
                                              const S *qn, S *out, C *rhs, Geom g, C gamma,
                                              C inv_dx, int mode, const Scalars *sc,
                                              double *blockmax, int *err, const C *W, const C *J,
                                              int zc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *P = reinterpret_cast<C *>(smem_raw);  // [6][PH][PW]
    C *FX = P + 6 * PH * PW;                 // [5][TY][TX+1]
    C *FY = FX + 5 * TY * (TX + 1);          // [5][TY+1][TX]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int k0 = blockIdx.z * zc, k1 = min(g.nz, k0 + zc);
    const int i = x0 + tx, j = y0 + ty;
    const bool active = i < g.nx && j < g.ny;
    const int ic = min(i, g.nx - 1), jc = min(j, g.ny - 1);
    const C gm1 = gamma - C(1);
    bool bad = false;

    A w = A(1), dt = A(0);
    if (mode != FLUX_RHS) {
        dt = A(sc->dt);
        w = mode == FLUX_STAGE1 ? A(1) : mode == FLUX_STAGE2 ? A(0.25) : A(2.0 / 3.0);
    }
    double smax = 0.0;

    // Register queue of the column's z-stencil. At iteration k the slots hold
    // planes k-2..k+3 and give the z-face k + 1/2. The loop starts one plane
    // early so that the face k0 - 1/2 comes out of the same instructions as
    // every other z-face (bitwise equal to the neighbouring chunk's copy).
    C Q[6][6];
#pragma unroll
    for (int s = 1; s < 6; s++) col_load(qs, sig, g, W, J, ic, jc, k0 - 4 + s, Q[s]);
    C Fzm[5];
    for (int k = k0 - 1; k < k1; k++) {
#pragma unroll
        for (int s = 0; s < 5; s++)
#pragma unroll
            for (int u = 0; u < 6; u++) Q[s][u] = Q[s + 1][u];
        col_load(qs, sig, g, W, J, ic, jc, k + 3, Q[5]);
        C Fzp[5];
        face_from_stencil<2>(Q, gamma, gm1, Fzp, bad);  // z-face k + 1/2
        if (k >= k0) {
            __syncthreads();  // readers of the previous plane are done
            // plane k with an x/y halo of 3 (corners are never read)
            for (int t = tid; t < PW * PH; t += NT) {
                int lx = t % PW, ly = t / PW;
                bool xin = lx >= 3 && lx < TX + 3, yin = ly >= 3 && ly < TY + 3;
                if (!xin && !yin) continue;
                int mx = map_axis(x0 + lx - 3, g.nx, g.bc[0], g.bc[1]);
                int my = map_axis(y0 + ly - 3, g.ny, g.bc[2], g.bc[3]);
                long long c = k * g.plane + (long long)my * g.nx + mx;
#pragma unroll
                for (int u = 0; u < 5; u++) P[(u * PH + ly) * PW + lx] = ldc(qs + u * g.n + c);
                P[(5 * PH + ly) * PW + lx] = ldc(sig + c);
            }
            __syncthreads();
            // x-faces: face f of row r sits between local cells f-1 and f
            for (int t = tid; t < (TX + 1) * TY; t += NT) {
                int f = t % (TX + 1), r = t / (TX + 1);
                C s[6][6];
#pragma unroll
                for (int m = 0; m < 6; m++)
#pragma unroll
                    for (int u = 0; u < 6; u++) s[m][u] = P[(u * PH + r + 3) * PW + f + m];
                C F[5];
                face_from_stencil<0>(s, gamma, gm1, F, bad);
#pragma unroll
                for (int u = 0; u < 5; u++) FX[(u * TY + r) * (TX + 1) + f] = F[u];
            }
            // y-faces: face fr of column c sits between local rows fr-1 and fr
            for (int t = tid; t < (TY + 1) * TX; t += NT) {
                int c = t % TX, fr = t / TX;
                C s[6][6];
#pragma unroll
                for (int m = 0; m < 6; m++)
#pragma unroll
                    for (int u = 0; u < 6; u++) s[m][u] = P[(u * PH + fr + m) * PW + c + 3];
                C F[5];
                face_from_stencil<1>(s, gamma, gm1, F, bad);
#pragma unroll
                for (int u = 0; u < 5; u++) FY[(u * (TY + 1) + fr) * TX + c] = F[u];
            }
            __syncthreads();
            if (active) {
                long long c = k * g.plane + (long long)j * g.nx + i;
                C Lv[5];
#pragma unroll
                for (int u = 0; u < 5; u++) {
                    C dfx = FX[(u * TY + ty) * (TX + 1) + tx + 1] - FX[(u * TY + ty) * (TX + 1) + tx];
                    C dfy = FY[(u * (TY + 1) + ty + 1) * TX + tx] - FY[(u * (TY + 1) + ty) * TX + tx];
                    C dfz = Fzp[u] - Fzm[u];
                    Lv[u] = -((dfx + dfy) + dfz) * inv_dx;
                }
                if (mode == FLUX_RHS) {
#pragma unroll
                    for (int u = 0; u < 5; u++) rhs[u * g.n + c] = Lv[u];
                } else {
                    C o[5];
#pragma unroll
                    for (int u = 0; u < 5; u++) {
                        A qsv = A(Q[2][u]);
                        A qnv = mode == FLUX_STAGE1 ? qsv : A(ldc(qn + u * g.n + c));
                        A v = qnv + w * ((qsv - qnv) + dt * A(Lv[u]));
                        o[u] = stc(out + u * g.n + c, v);
                        bad |= !isfinite(o[u]);
                    }
                    if (mode == FLUX_STAGE3)
                        smax = nanmax(smax, double(cell_speed(o[0], o[1], o[2], o[3], o[4], gamma, gm1)));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 5; u++) Fzm[u] = Fzp[u];
    }
    if (bad) atomicOr(err, 1);
    if (mode == FLUX_STAGE3) {
        double m = block_max<NT>(smax);
        if (tid == 0)
            blockmax[(blockIdx.z * (long long)gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = m;
    }
}

// ---------------------------------------------------------- wave speed
constexpr int SPEED_NT = 256, SPEED_MAXBLOCKS = 152 * 8;

__global__ void __launch_bounds__(SPEED_NT) k_speed(const S *__restrict__ q, long long n, C gamma,
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

// ------------------------------------------------------------ launchers
dim3 grid_of(const Geom &g, int bx, int by, int zc)
{
    return dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, (g.nz + zc - 1) / zc);
}

cudaError_t launch_source(const Geom &g, const Phys &p, const Tiles &t, const Inflow &in,
                          const void *q, void *b, cudaStream_t st)
{
    k_source<<<grid_of(g, BX, BY, t.zc_source), dim3(BX, BY), 0, st>>>(
        (const S *)q, (S *)b, g, C(p.alpha), C(0.5 / p.dx), (const C *)in.W, (const C *)in.J,
        t.zc_source);
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const Geom &g, const Phys &p, const Tiles &t, const void *q,
                          const void *b, const void *s_in, void *s_out, cudaStream_t st)
{
    k_jacobi<<<grid_of(g, BX, BY, t.zc_jacobi), dim3(BX, BY), 0, st>>>(
        (const S *)q, (const S *)b, (const S *)s_in, (S *)s_out, g, C(p.alpha / (p.dx * p.dx)),
        t.zc_jacobi);
    return cudaGetLastError();
}

long long flux_blocks(const Geom &g, const Tiles &t)
{
    dim3 gr = grid_of(g, TX, TY, t.zc_flux);
    return (long long)gr.x * gr.y * gr.z;
}

cudaError_t launch_flux(const Geom &g, const Phys &p, const Tiles &t, const Inflow &in, int mode,
                        const void *qs, const void *sig, const void *qn, void *out, void *rhs,
                        const Scalars *sc, double *blockmax, int *err, cudaStream_t st)
{
    static bool attr_set = false;
    size_t smem = flux_smem_elems() * sizeof(C);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_flux, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_flux<<<grid_of(g, TX, TY, t.zc_flux), dim3(TX, TY), smem, st>>>(
        (const S *)qs, (const S *)sig, (const S *)qn, (S *)out, (C *)rhs, g, C(p.gamma),
        C(1.0 / p.dx), mode, sc, blockmax, err, (const C *)in.W, (const C *)in.J, t.zc_flux);
    return cudaGetLastError();
}

cudaError_t launch_speed(const Geom &g, const Phys &p, const void *q, double *blockmax,
                         int *nblocks, cudaStream_t st)
{
    long long want = (g.n + SPEED_NT - 1) / SPEED_NT;
    int nb = (int)(want < SPEED_MAXBLOCKS ? want : SPEED_MAXBLOCKS);
    k_speed<<<nb, SPEED_NT, 0, st>>>((const S *)q, g.n, C(p.gamma), blockmax);
    *nblocks = nb;
    return cudaGetLastError();
}

}  // namespace

extern const Ops IGR_OPS = {
    (int)sizeof(S), (int)sizeof(C), launch_source, launch_jacobi, launch_flux, flux_blocks,
    launch_speed,
};

}  // namespace igr
