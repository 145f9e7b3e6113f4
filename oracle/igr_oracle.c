/*
 * FP64 CPU oracle for one SSP-RK3 step of the 3D Euler equations with
 * information geometric regularization (IGR).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA path.
 *
 * It is written plainly: ghost-cell arrays of width 3, one loop per
 * operation, all arithmetic in double, built with -ffp-contract=off.
 * Every function names the part of the paper it follows:
 *   - IGR-modified Euler system, Eqs. (igrmabalance)-(igrenbalance);
 *   - IGR elliptic equation for Sigma, Eq. (igrelliptic);
 *   - ideal-gas equation of state, Eq. (state_eqn);
 *   - discretisation (Sec. "Discretization"): 5th-order finite-volume face
 *     reconstruction, Lax-Friedrichs flux, 2nd-order velocity gradients,
 *     7-point elliptic stencil, warm-started Jacobi sweeps, 3rd-order SSP
 *     Runge-Kutta (Gottlieb-Shu);
 *   - Algorithm 1 (flux of p+Sigma in every direction, Sigma reconstructed
 *     like the conserved variables);
 *   - the alternatives the same section names: 3rd-order face values and
 *     (red-black) Gauss-Seidel sweeps, selected by orc_grid.order and
 *     orc_grid.sigma_solver (the adjoint covers the default scheme only);
 *   - viscous stresses, Eq. (constitutive_law), when orc_grid.mu or
 *     orc_grid.zeta is nonzero (Navier-Stokes form of the same system).
 * Readings where the paper is silent (face coefficient of the elliptic
 * operator, local LF speed, boundary treatment of Sigma, dt rule, jet
 * inflow ghosts) are listed next to the code that takes them.
 *
 * State layout: q[v][k][j][i], v in (rho, mx, my, mz, E), x fastest,
 * interior cells only. Sigma and b: [k][j][i].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define G 3 /* ghost width: the 5th-order stencil reaches 3 cells */
#define NV 5

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2 };

typedef struct {
    int nx, ny, nz;
    double dx, gamma, alpha, cfl;
    int sweeps;
    int bc[6];          /* faces -x,+x,-y,+y,-z,+z */
    int njets;
    const double *jets; /* njets x 7: cx, cy, radius, rho, w, p, edge_width */
    int order;          /* face reconstruction: 5 or 3 (Sec. "Discretization") */
    int sigma_solver;   /* Sigma sweeps: 0 Jacobi, 1 red-black Gauss-Seidel */
    double mu, zeta;    /* shear and bulk viscosity, Eq. (constitutive_law); 0 = Euler */
} orc_grid;

/* ---------------------------------------------------------------- indexing */

static long ncell(const orc_grid *g) { return (long)g->nx * g->ny * g->nz; }
static long nghost(const orc_grid *g)
{
    return (long)(g->nx + 2 * G) * (g->ny + 2 * G) * (g->nz + 2 * G);
}
/* interior index */
static long I(const orc_grid *g, int i, int j, int k)
{
    return ((long)k * g->ny + j) * g->nx + i;
}
/* ghost-array index; i in [-G, nx+G) */
static long GI(const orc_grid *g, int i, int j, int k)
{
    return ((long)(k + G) * (g->ny + 2 * G) + (j + G)) * (g->nx + 2 * G) + (i + G);
}

/* --------------------------------------------------------- ghost filling */

/* Conserved state of jet n, from its primitive state (rho, w along +z, p):
 * Eq. (state_eqn) gives E = p/(gamma-1) + rho w^2 / 2. */
static void jet_state(const orc_grid *g, int n, double qj[NV])
{
    const double *J = g->jets + 7 * n;
    double rho = J[3], w = J[4], p = J[5];
    qj[0] = rho;
    qj[1] = 0.0;
    qj[2] = 0.0;
    qj[3] = rho * w;
    qj[4] = p / (g->gamma - 1.0) + 0.5 * rho * w * w;
}

/* Fill the ghost layers of one field f (ghost array) along all three axes.
 * Periodic faces wrap; outflow faces copy the nearest interior cell
 * (zero gradient). An inflow face (only -z is allowed) blends every jet's
 * state into the nearest interior cell:
 *   s_n = (1 - tanh((r_n - R_n) / (edge_width_n dx))) / 2,
 *   ghost = (1 - sum_n s_n) q_interior + sum_n s_n q_jet_n,
 * with r_n the distance from the ghost cell's (x, y) centre to jet n. For a
 * field that is not a conserved variable (Sigma), inflow acts as outflow. */
static void fill_axis_x(const orc_grid *g, double *f)
{
    int nx = g->nx;
    for (int k = -G; k < g->nz + G; k++)
        for (int j = -G; j < g->ny + G; j++)
            for (int s = 1; s <= G; s++) {
                int lo = -s, hi = nx - 1 + s;
                int slo = g->bc[0] == BC_PERIODIC ? ((lo % nx) + nx) % nx : 0;
                int shi = g->bc[1] == BC_PERIODIC ? hi % nx : nx - 1;
                f[GI(g, lo, j, k)] = f[GI(g, slo, j, k)];
                f[GI(g, hi, j, k)] = f[GI(g, shi, j, k)];
            }
}
static void fill_axis_y(const orc_grid *g, double *f)
{
    int ny = g->ny;
    for (int k = -G; k < g->nz + G; k++)
        for (int s = 1; s <= G; s++)
            for (int i = -G; i < g->nx + G; i++) {
                int lo = -s, hi = ny - 1 + s;
                int slo = g->bc[2] == BC_PERIODIC ? ((lo % ny) + ny) % ny : 0;
                int shi = g->bc[3] == BC_PERIODIC ? hi % ny : ny - 1;
                f[GI(g, i, lo, k)] = f[GI(g, i, slo, k)];
                f[GI(g, i, hi, k)] = f[GI(g, i, shi, k)];
            }
}
static void fill_axis_z(const orc_grid *g, double *f, int var)
{
    int nz = g->nz;
    for (int s = 1; s <= G; s++)
        for (int j = -G; j < g->ny + G; j++)
            for (int i = -G; i < g->nx + G; i++) {
                int lo = -s, hi = nz - 1 + s;
                int slo = g->bc[4] == BC_PERIODIC ? ((lo % nz) + nz) % nz : 0;
                int shi = g->bc[5] == BC_PERIODIC ? hi % nz : nz - 1;
                double vlo = f[GI(g, i, j, slo)];
                if (g->bc[4] == BC_INFLOW && var >= 0) {
                    /* the blend weight of a ghost column outside the face's
                     * extent is that of the face cell it maps to (the x and
                     * y ghosts of the source plane hold those cells' values) */
                    int mi = i, mj = j;
                    if (mi < 0) mi = g->bc[0] == BC_PERIODIC ? ((mi % g->nx) + g->nx) % g->nx : 0;
                    if (mi >= g->nx) mi = g->bc[1] == BC_PERIODIC ? mi % g->nx : g->nx - 1;
                    if (mj < 0) mj = g->bc[2] == BC_PERIODIC ? ((mj % g->ny) + g->ny) % g->ny : 0;
                    if (mj >= g->ny) mj = g->bc[3] == BC_PERIODIC ? mj % g->ny : g->ny - 1;
                    double x = (mi + 0.5) * g->dx, y = (mj + 0.5) * g->dx;
                    double wsum = 0.0, jsum = 0.0;
                    for (int n = 0; n < g->njets; n++) {
                        const double *J = g->jets + 7 * n;
                        double r = sqrt((x - J[0]) * (x - J[0]) + (y - J[1]) * (y - J[1]));
                        double sn = 0.5 * (1.0 - tanh((r - J[2]) / (J[6] * g->dx)));
                        double qj[NV];
                        jet_state(g, n, qj);
                        wsum += sn;
                        jsum += sn * qj[var];
                    }
                    vlo = (1.0 - wsum) * vlo + jsum;
                }
                f[GI(g, i, j, lo)] = vlo;
                f[GI(g, i, j, hi)] = f[GI(g, i, j, shi)];
            }
}

/* q (interior, 5 fields) -> qg (ghost arrays, 5 fields). */
void orc_fill_ghosts(const orc_grid *g, const double *q, double *qg)
{
    long N = ncell(g), NG = nghost(g);
    for (int v = 0; v < NV; v++) {
        double *f = qg + v * NG;
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) f[GI(g, i, j, k)] = q[v * N + I(g, i, j, k)];
        fill_axis_x(g, f);
        fill_axis_y(g, f);
        fill_axis_z(g, f, v);
    }
}

/* Sigma (interior) -> ghost array: periodic wrap, zero gradient otherwise. */
static void fill_sigma_ghosts(const orc_grid *g, const double *sig, double *sg)
{
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) sg[GI(g, i, j, k)] = sig[I(g, i, j, k)];
    fill_axis_x(g, sg);
    fill_axis_y(g, sg);
    fill_axis_z(g, sg, -1);
}

/* ------------------------------------------- velocity gradients and source */

/* IGR source b = alpha [tr((grad u)^2) + tr^2(grad u)] at every interior cell,
 * Eq. (igrelliptic) left side. grad u by second-order central differences
 * (Sec. "Discretization"): G[a][c] = d u_a / d x_c
 *   = (u_a(i + e_c) - u_a(i - e_c)) / (2 dx), u = m / rho,
 * neighbours outside the domain taken from the ghost cells of q.
 * tr(G^2) = sum_{a,c} G[a][c] G[c][a]; tr^2(G) = (sum_a G[a][a])^2. */
static void source_from_ghosts(const orc_grid *g, const double *qg, double *b)
{
    long NG = nghost(g);
    const double *rho = qg, *m[3] = {qg + NG, qg + 2 * NG, qg + 3 * NG};
#pragma omp parallel for
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                int off[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                double Gm[3][3];
                for (int c = 0; c < 3; c++) {
                    long ip = GI(g, i + off[c][0], j + off[c][1], k + off[c][2]);
                    long im = GI(g, i - off[c][0], j - off[c][1], k - off[c][2]);
                    for (int a = 0; a < 3; a++) {
                        double up = m[a][ip] / rho[ip];
                        double um = m[a][im] / rho[im];
                        Gm[a][c] = (up - um) / (2.0 * g->dx);
                    }
                }
                double trG2 = 0.0;
                for (int a = 0; a < 3; a++)
                    for (int c = 0; c < 3; c++) trG2 += Gm[a][c] * Gm[c][a];
                double trG = Gm[0][0] + Gm[1][1] + Gm[2][2];
                b[I(g, i, j, k)] = g->alpha * (trG2 + trG * trG);
            }
}

void orc_source(const orc_grid *g, const double *q, double *b)
{
    double *qg = malloc(sizeof(double) * NV * nghost(g));
    orc_fill_ghosts(g, q, qg);
    source_from_ghosts(g, qg, b);
    free(qg);
}

/* ------------------------------------------------ elliptic operator for Sigma */

/* Neighbour of interior cell (i,j,k) across face dir (0:-x 1:+x 2:-y 3:+y
 * 4:-z 5:+z). Returns 0 when the face is a non-periodic domain boundary:
 * there the zero-gradient condition on Sigma makes the face term vanish. */
static int neighbour(const orc_grid *g, int i, int j, int k, int dir, long *nb)
{
    int n[3] = {g->nx, g->ny, g->nz};
    int c[3] = {i, j, k};
    int ax = dir / 2, sgn = (dir % 2) ? 1 : -1;
    c[ax] += sgn;
    if (c[ax] < 0 || c[ax] >= n[ax]) {
        if (g->bc[dir] != BC_PERIODIC) return 0;
        c[ax] = (c[ax] + n[ax]) % n[ax];
    }
    *nb = I(g, c[0], c[1], c[2]);
    return 1;
}

/* Discrete operator A of Eq. (igrelliptic), A Sigma = rho^-1 Sigma
 * - alpha div(rho^-1 grad Sigma), with the 7-point stencil
 *   (A s)_i = r_i s_i + beta sum_f c_f (s_i - s_nb(f)),
 * beta = alpha / dx^2, r = 1/rho, face coefficient c_f = (r_i + r_nb) / 2
 * (reading: the paper names only "a standard 7-point stencil"; the
 * arithmetic mean keeps A symmetric). Faces on a non-periodic boundary
 * carry no term (zero normal gradient of Sigma). */
void orc_apply_A(const orc_grid *g, const double *q, const double *s, double *out)
{
    const double *rho = q;
    double beta = g->alpha / (g->dx * g->dx);
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long c = I(g, i, j, k), nb;
                double ri = 1.0 / rho[c];
                double acc = ri * s[c];
                for (int d = 0; d < 6; d++) {
                    if (!neighbour(g, i, j, k, d, &nb)) continue;
                    double cf = 0.5 * (ri + 1.0 / rho[nb]);
                    acc += beta * cf * (s[c] - s[nb]);
                }
                out[c] = acc;
            }
}

/* Red-black Gauss-Seidel sweeps on A sigma = b (Sec. "Discretization":
 * Jacobi or Gauss-Seidel, warm-started): each sweep updates the red cells
 * (i + j + k even), then the black cells (odd), in place, each from the
 * current values of its neighbours, which are all of the other colour
 * (periodic axes have even length):
 *   sigma_i <- (b_i + beta sum_f c_f sigma_nb) / (r_i + beta sum_f c_f). */
static void rbgs(const orc_grid *g, const double *q, const double *b, double *sigma, int sweeps)
{
    const double *rho = q;
    double beta = g->alpha / (g->dx * g->dx);
    for (int it = 0; it < sweeps; it++)
        for (int colour = 0; colour < 2; colour++) {
#pragma omp parallel for
            for (int k = 0; k < g->nz; k++)
                for (int j = 0; j < g->ny; j++)
                    for (int i = 0; i < g->nx; i++) {
                        if (((i + j + k) & 1) != colour) continue;
                        long c = I(g, i, j, k), nb;
                        double ri = 1.0 / rho[c];
                        double diag = ri, off = 0.0;
                        for (int d = 0; d < 6; d++) {
                            if (!neighbour(g, i, j, k, d, &nb)) continue;
                            double cf = 0.5 * (ri + 1.0 / rho[nb]);
                            diag += beta * cf;
                            off += beta * cf * sigma[nb];
                        }
                        sigma[c] = (b[c] + off) / diag;
                    }
        }
}

/* `sweeps` Jacobi sweeps on A sigma = b, warm-started from the incoming
 * sigma (Sec. "Discretization": the previous Sigma is the initial guess):
 *   sigma_i <- (b_i + beta sum_f c_f sigma_nb) / (r_i + beta sum_f c_f),
 * every cell updated from the previous iterate only (two buffers); with
 * g->sigma_solver = 1 red-black Gauss-Seidel sweeps instead. */
void orc_jacobi(const orc_grid *g, const double *q, const double *b, double *sigma,
                int sweeps)
{
    if (g->sigma_solver == 1) {
        rbgs(g, q, b, sigma, sweeps);
        return;
    }
    long N = ncell(g);
    const double *rho = q;
    double beta = g->alpha / (g->dx * g->dx);
    double *old = malloc(sizeof(double) * N);
    for (int it = 0; it < sweeps; it++) {
        memcpy(old, sigma, sizeof(double) * N);
#pragma omp parallel for
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    long c = I(g, i, j, k), nb;
                    double ri = 1.0 / rho[c];
                    double diag = ri, off = 0.0;
                    for (int d = 0; d < 6; d++) {
                        if (!neighbour(g, i, j, k, d, &nb)) continue;
                        double cf = 0.5 * (ri + 1.0 / rho[nb]);
                        diag += beta * cf;
                        off += beta * cf * old[nb];
                    }
                    sigma[c] = (b[c] + off) / diag;
                }
    }
    free(old);
}

/* ------------------------------------------------------- fluxes and RHS */

/* 5th-order linear finite-volume face values at face i+1/2 from the cell
 * averages v[i-2..i+3] (Sec. "Discretization", Algorithm 1: the stencil
 * -2..3 along the sweep direction): the unique quartic matching the five
 * cell averages of the left-biased (resp. right-biased) stencil, evaluated
 * at the face. */
static double recon_left(const double v[6])
{
    return (2.0 * v[0] - 13.0 * v[1] + 47.0 * v[2] + 27.0 * v[3] - 3.0 * v[4]) / 60.0;
}
static double recon_right(const double v[6])
{
    return (-3.0 * v[1] + 27.0 * v[2] + 47.0 * v[3] - 13.0 * v[4] + 2.0 * v[5]) / 60.0;
}

/* 3rd-order alternative (Sec. "Discretization": third- or fifth-order finite
 * volumes): the quadratic through the three cell averages of the biased
 * stencil i-1..i+1 (left) or i..i+2 (right), evaluated at face i+1/2. */
static double recon3_left(const double v[6]) { return (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0; }
static double recon3_right(const double v[6]) { return (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0; }

static double face_left(const orc_grid *g, const double v[6])
{
    return g->order == 3 ? recon3_left(v) : recon_left(v);
}
static double face_right(const orc_grid *g, const double v[6])
{
    return g->order == 3 ? recon3_right(v) : recon_right(v);
}

/* Physical flux of the IGR-modified Euler system along axis d,
 * Eqs. (igrmabalance)-(igrenbalance) with tau = 0:
 *   (rho u_d, m u_d + (p + Sigma) e_d, (E + p + Sigma) u_d),
 * p from Eq. (state_eqn). Also returns |u_d| + c with c = sqrt(gamma p / rho)
 * (reading: the sound speed uses p, not p + Sigma). */
static double phys_flux(const orc_grid *g, const double qv[NV], double sig, int d,
                        double F[NV])
{
    double rho = qv[0], E = qv[4];
    double u[3] = {qv[1] / rho, qv[2] / rho, qv[3] / rho};
    double ke = 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double p = (g->gamma - 1.0) * (E - ke);
    double P = p + sig;
    F[0] = rho * u[d];
    for (int a = 0; a < 3; a++) F[1 + a] = qv[1 + a] * u[d] + (a == d ? P : 0.0);
    F[4] = (E + P) * u[d];
    return fabs(u[d]) + sqrt(g->gamma * p / rho);
}

/* velocity u = m / rho of ghost-array cell gi */
static void vel_at(const orc_grid *g, const double *qg, long gi, double u[3])
{
    long NG = nghost(g);
    for (int a = 0; a < 3; a++) u[a] = qg[(1 + a) * NG + gi] / qg[gi];
}

/* Viscous part of the flux through the face between cells A = c - e_d and
 * B = c along axis d (c = (i, j, k)), Eqs. (igrmobalance)-(igrenbalance)
 * with the stress of Eq. (constitutive_law)
 *   tau_ab = mu (du_a/dx_b + du_b/dx_a) + (zeta - 2 mu / 3) delta_ab div u
 * (reading: the garbled delta_ij du_i/dx_j term is the divergence, Stokes'
 * form). Velocity derivatives at the face, second order (Sec.
 * "Discretization": second-order derivatives of u suffice; reading: on the
 * compact face stencil rather than reconstructed cell-centre gradients):
 *   normal      du_a/dx_d = (u_a(B) - u_a(A)) / dx,
 *   tangential  du_a/dx_t = [(u_a(A+e_t) - u_a(A-e_t)) + (u_a(B+e_t) - u_a(B-e_t))] / (4 dx),
 * face velocity (u(A) + u(B)) / 2. The flux adds -tau_{a d} to momentum
 * component a and -sum_a u_a tau_{a d} to energy. */
static void viscous_flux(const orc_grid *g, const double *qg, int i, int j, int k, int d,
                         double Fv[NV])
{
    int c[3] = {i, j, k}, a0[3] = {i, j, k};
    a0[d] -= 1;
    double uA[3], uB[3], Gr[3][3];
    vel_at(g, qg, GI(g, a0[0], a0[1], a0[2]), uA);
    vel_at(g, qg, GI(g, c[0], c[1], c[2]), uB);
    for (int a = 0; a < 3; a++) Gr[a][d] = (uB[a] - uA[a]) / g->dx;
    for (int t = 0; t < 3; t++) {
        if (t == d) continue;
        int Ap[3] = {a0[0], a0[1], a0[2]}, Am[3] = {a0[0], a0[1], a0[2]};
        int Bp[3] = {c[0], c[1], c[2]}, Bm[3] = {c[0], c[1], c[2]};
        Ap[t] += 1; Am[t] -= 1; Bp[t] += 1; Bm[t] -= 1;
        double uAp[3], uAm[3], uBp[3], uBm[3];
        vel_at(g, qg, GI(g, Ap[0], Ap[1], Ap[2]), uAp);
        vel_at(g, qg, GI(g, Am[0], Am[1], Am[2]), uAm);
        vel_at(g, qg, GI(g, Bp[0], Bp[1], Bp[2]), uBp);
        vel_at(g, qg, GI(g, Bm[0], Bm[1], Bm[2]), uBm);
        for (int a = 0; a < 3; a++)
            Gr[a][t] = ((uAp[a] - uAm[a]) + (uBp[a] - uBm[a])) / (4.0 * g->dx);
    }
    double div = Gr[0][0] + Gr[1][1] + Gr[2][2];
    double work = 0.0;
    Fv[0] = 0.0;
    for (int a = 0; a < 3; a++) {
        double tau = g->mu * (Gr[a][d] + Gr[d][a]) + (a == d ? (g->zeta - 2.0 * g->mu / 3.0) * div : 0.0);
        Fv[1 + a] = -tau;
        work += 0.5 * (uA[a] + uB[a]) * tau;
    }
    Fv[4] = -work;
}

/* Spatial operator L(q; Sigma) = -div F_hat at every interior cell, with the
 * local Lax-Friedrichs flux (reading: local speed)
 *   F_hat = (F(q_L) + F(q_R)) / 2 - lambda (q_R - q_L) / 2,
 *   lambda = max(|u_d|+c at L, at R),
 * Sigma entering only through the pressure p + Sigma, reconstructed with
 * the same 5th-order face values as the conserved variables.
 *   L_i = -[(Fx_{i+1/2} - Fx_{i-1/2}) + (Fy..) + (Fz..)] / dx. */
static void rhs_from_ghosts(const orc_grid *g, const double *qg, const double *sg,
                            double *L)
{
    long N = ncell(g), NG = nghost(g);
    int nx = g->nx, ny = g->ny, nz = g->nz;
    memset(L, 0, sizeof(double) * NV * N);
    for (int d = 0; d < 3; d++) {
        /* face fluxes along d: face index f in [0, n_d], face f sits between
         * cells f-1 and f */
        int fx = nx + (d == 0), fy = ny + (d == 1), fz = nz + (d == 2);
        long NF = (long)fx * fy * fz;
        double *F = malloc(sizeof(double) * NV * NF);
#pragma omp parallel for
        for (int k = 0; k < fz; k++)
            for (int j = 0; j < fy; j++)
                for (int i = 0; i < fx; i++) {
                    /* stencil cells along d: face f = (i,j,k)[d] between
                     * cells f-1 and f -> cells f-3 .. f+2 */
                    double vq[NV + 1][6];
                    for (int s = 0; s < 6; s++) {
                        int c[3] = {i, j, k};
                        c[d] += s - 3;
                        long gi = GI(g, c[0], c[1], c[2]);
                        for (int v = 0; v < NV; v++) vq[v][s] = qg[v * NG + gi];
                        vq[NV][s] = sg[gi];
                    }
                    double qL[NV], qR[NV], FL[NV], FR[NV];
                    for (int v = 0; v < NV; v++) {
                        qL[v] = face_left(g, vq[v]);
                        qR[v] = face_right(g, vq[v]);
                    }
                    double sL = face_left(g, vq[NV]), sR = face_right(g, vq[NV]);
                    double aL = phys_flux(g, qL, sL, d, FL);
                    double aR = phys_flux(g, qR, sR, d, FR);
                    double lam = aL > aR ? aL : aR;
                    long fi = ((long)k * fy + j) * fx + i;
                    for (int v = 0; v < NV; v++)
                        F[v * NF + fi] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (qR[v] - qL[v]);
                    if (g->mu != 0.0 || g->zeta != 0.0) {
                        double Fv[NV];
                        viscous_flux(g, qg, i, j, k, d, Fv);
                        for (int v = 0; v < NV; v++) F[v * NF + fi] += Fv[v];
                    }
                }
        /* accumulate the flux difference of this direction */
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    int c[3] = {i, j, k};
                    int h[3] = {i, j, k};
                    h[d] += 1;
                    long lo = ((long)c[2] * fy + c[1]) * fx + c[0];
                    long hi = ((long)h[2] * fy + h[1]) * fx + h[0];
                    for (int v = 0; v < NV; v++)
                        L[v * N + I(g, i, j, k)] += F[v * NF + hi] - F[v * NF + lo];
                }
        free(F);
    }
    for (long n = 0; n < NV * N; n++) L[n] = -L[n] / g->dx;
}

/* L(q; Sigma) for given q and Sigma (no elliptic solve). */
void orc_rhs(const orc_grid *g, const double *q, const double *sigma, double *L)
{
    double *qg = malloc(sizeof(double) * NV * nghost(g));
    double *sg = malloc(sizeof(double) * nghost(g));
    orc_fill_ghosts(g, q, qg);
    fill_sigma_ghosts(g, sigma, sg);
    rhs_from_ghosts(g, qg, sg, L);
    free(qg);
    free(sg);
}

/* max over interior cells of max_d (|u_d| + c) (reading: the paper does not
 * state its time-step rule; dt = cfl dx / this maximum, from the state at
 * the start of the step). */
double orc_max_speed(const orc_grid *g, const double *q)
{
    long N = ncell(g);
    double smax = 0.0;
    for (long n = 0; n < N; n++) {
        double rho = q[n];
        double u[3] = {q[N + n] / rho, q[2 * N + n] / rho, q[3 * N + n] / rho};
        double p = (g->gamma - 1.0) *
                   (q[4 * N + n] - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
        double c = sqrt(g->gamma * p / rho);
        for (int d = 0; d < 3; d++) {
            double s = fabs(u[d]) + c;
            if (s > smax) smax = s;
        }
    }
    return smax;
}

/* One Runge-Kutta stage: the elliptic solve for Sigma (warm start from the
 * incoming sigma, `sweeps` Jacobi sweeps), then
 *   out = qn + w [(qs - qn) + dt L(qs; Sigma)],
 * the increment form of the Gottlieb-Shu SSP-RK3 stages (w = 1, 1/4, 2/3).
 * out may alias qn but not qs. */
void orc_stage(const orc_grid *g, const double *qs, const double *qn, double *sigma,
               double *out, double w, double dt)
{
    long N = ncell(g);
    double *qg = malloc(sizeof(double) * NV * nghost(g));
    double *sg = malloc(sizeof(double) * nghost(g));
    double *b = malloc(sizeof(double) * N);
    double *L = malloc(sizeof(double) * NV * N);
    orc_fill_ghosts(g, qs, qg);
    source_from_ghosts(g, qg, b);
    orc_jacobi(g, qs, b, sigma, g->sweeps);
    fill_sigma_ghosts(g, sigma, sg);
    rhs_from_ghosts(g, qg, sg, L);
    for (long n = 0; n < NV * N; n++) out[n] = qn[n] + w * ((qs[n] - qn[n]) + dt * L[n]);
    free(qg);
    free(sg);
    free(b);
    free(L);
}

/* One SSP-RK3 time step (Gottlieb-Shu), state and Sigma updated in place.
 * dt = fixed_dt if fixed_dt > 0, else cfl dx / orc_max_speed(q). Returns dt. */
double orc_step(const orc_grid *g, double *q, double *sigma, double fixed_dt)
{
    long N = ncell(g);
    double dt = fixed_dt > 0.0 ? fixed_dt : g->cfl * g->dx / orc_max_speed(g, q);
    double *q1 = malloc(sizeof(double) * NV * N);
    double *q2 = malloc(sizeof(double) * NV * N);
    orc_stage(g, q, q, sigma, q1, 1.0, dt);
    orc_stage(g, q1, q, sigma, q2, 0.25, dt);
    orc_stage(g, q2, q, sigma, q, 2.0 / 3.0, dt);
    free(q1);
    free(q2);
    return dt;
}

/* nsteps steps; returns the elapsed simulated time. */
double orc_run(const orc_grid *g, double *q, double *sigma, int nsteps, double fixed_dt)
{
    double t = 0.0;
    for (int n = 0; n < nsteps; n++) t += orc_step(g, q, sigma, fixed_dt);
    return t;
}

/* ======================================================================
 * Discrete adjoint of one SSP-RK3 step (fixed dt), in FP64.
 *
 * With dt frozen, one step maps (q, Sigma; jet velocities w) to
 * (q', Sigma'). Given the adjoints (lq, ls) of (q', Sigma'), the functions
 * below return the adjoints of (q, Sigma) and add d<lq,q'> + <ls,Sigma'>/dw
 * to gw. Each routine is the hand-written reverse of the forward routine
 * of the same name: the forward step is recomputed and stored (stage
 * inputs, Sigma iterates of every sweep), then the stages are reversed.
 * Non-smooth points take one-sided branches matching the forward: the LF
 * speed max(aL, aR) sends its adjoint to the side the forward selected,
 * |u| takes sign(u) with sign(0) = 0.
 * ====================================================================== */

/* reverse of fill_axis_x/y/z: the adjoint of each ghost cell goes back to the
 * cell it was copied from (times 1 - sum s for an inflow ghost, whose jet part
 * goes to lamJ[var][j][i]); the ghost's adjoint is consumed */
static void fill_axis_x_rev(const orc_grid *g, double *fb)
{
    int nx = g->nx;
    for (int k = g->nz + G - 1; k >= -G; k--)
        for (int j = g->ny + G - 1; j >= -G; j--)
            for (int s = G; s >= 1; s--) {
                int lo = -s, hi = nx - 1 + s;
                int slo = g->bc[0] == BC_PERIODIC ? ((lo % nx) + nx) % nx : 0;
                int shi = g->bc[1] == BC_PERIODIC ? hi % nx : nx - 1;
                fb[GI(g, shi, j, k)] += fb[GI(g, hi, j, k)];
                fb[GI(g, hi, j, k)] = 0.0;
                fb[GI(g, slo, j, k)] += fb[GI(g, lo, j, k)];
                fb[GI(g, lo, j, k)] = 0.0;
            }
}
static void fill_axis_y_rev(const orc_grid *g, double *fb)
{
    int ny = g->ny;
    for (int k = g->nz + G - 1; k >= -G; k--)
        for (int s = G; s >= 1; s--)
            for (int i = g->nx + G - 1; i >= -G; i--) {
                int lo = -s, hi = ny - 1 + s;
                int slo = g->bc[2] == BC_PERIODIC ? ((lo % ny) + ny) % ny : 0;
                int shi = g->bc[3] == BC_PERIODIC ? hi % ny : ny - 1;
                fb[GI(g, i, shi, k)] += fb[GI(g, i, hi, k)];
                fb[GI(g, i, hi, k)] = 0.0;
                fb[GI(g, i, slo, k)] += fb[GI(g, i, lo, k)];
                fb[GI(g, i, lo, k)] = 0.0;
            }
}
static void fill_axis_z_rev(const orc_grid *g, double *fb, int var, double *lamJ)
{
    int nz = g->nz;
    for (int s = G; s >= 1; s--)
        for (int j = g->ny + G - 1; j >= -G; j--)
            for (int i = g->nx + G - 1; i >= -G; i--) {
                int lo = -s, hi = nz - 1 + s;
                int slo = g->bc[4] == BC_PERIODIC ? ((lo % nz) + nz) % nz : 0;
                int shi = g->bc[5] == BC_PERIODIC ? hi % nz : nz - 1;
                fb[GI(g, i, j, shi)] += fb[GI(g, i, j, hi)];
                fb[GI(g, i, j, hi)] = 0.0;
                double a = fb[GI(g, i, j, lo)];
                fb[GI(g, i, j, lo)] = 0.0;
                if (g->bc[4] == BC_INFLOW && var >= 0) {
                    double x = (i + 0.5) * g->dx, y = (j + 0.5) * g->dx;
                    double wsum = 0.0;
                    for (int n = 0; n < g->njets; n++) {
                        const double *J = g->jets + 7 * n;
                        double r = sqrt((x - J[0]) * (x - J[0]) + (y - J[1]) * (y - J[1]));
                        wsum += 0.5 * (1.0 - tanh((r - J[2]) / (J[6] * g->dx)));
                    }
                    fb[GI(g, i, j, slo)] += (1.0 - wsum) * a;
                    if (i >= 0 && i < g->nx && j >= 0 && j < g->ny)
                        lamJ[((long)var * g->ny + j) * g->nx + i] += a;
                } else {
                    fb[GI(g, i, j, slo)] += a;
                }
            }
}

/* reverse of orc_fill_ghosts: qgb (ghost-array adjoints, consumed) is added
 * to qb (interior adjoints); lamJ (5 x ny x nx) collects the jet-table part */
static void fill_ghosts_rev(const orc_grid *g, double *qgb, double *qb, double *lamJ)
{
    long N = ncell(g), NG = nghost(g);
    for (int v = 0; v < NV; v++) {
        double *fb = qgb + v * NG;
        fill_axis_z_rev(g, fb, v, lamJ);
        fill_axis_y_rev(g, fb);
        fill_axis_x_rev(g, fb);
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) qb[v * N + I(g, i, j, k)] += fb[GI(g, i, j, k)];
    }
}

static void fill_sigma_ghosts_rev(const orc_grid *g, double *sgb, double *sb)
{
    fill_axis_z_rev(g, sgb, -1, NULL);
    fill_axis_y_rev(g, sgb);
    fill_axis_x_rev(g, sgb);
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) sb[I(g, i, j, k)] += sgb[GI(g, i, j, k)];
}

/* reverse of source_from_ghosts: bb (adjoint of b) added into qgb.
 * d b / d G[a][c] = alpha (2 G[c][a] + 2 tr(G) delta_ac). */
static void source_rev(const orc_grid *g, const double *qg, const double *bb, double *qgb)
{
    long NG = nghost(g);
    const double *rho = qg, *m[3] = {qg + NG, qg + 2 * NG, qg + 3 * NG};
    double *rhob = qgb, *mb[3] = {qgb + NG, qgb + 2 * NG, qgb + 3 * NG};
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                int off[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                double Gm[3][3];
                long ip[3], im[3];
                for (int c = 0; c < 3; c++) {
                    ip[c] = GI(g, i + off[c][0], j + off[c][1], k + off[c][2]);
                    im[c] = GI(g, i - off[c][0], j - off[c][1], k - off[c][2]);
                    for (int a = 0; a < 3; a++)
                        Gm[a][c] = (m[a][ip[c]] / rho[ip[c]] - m[a][im[c]] / rho[im[c]]) / (2.0 * g->dx);
                }
                double trG = Gm[0][0] + Gm[1][1] + Gm[2][2];
                double b_bar = bb[I(g, i, j, k)];
                for (int c = 0; c < 3; c++)
                    for (int a = 0; a < 3; a++) {
                        double Gb = g->alpha * (2.0 * Gm[c][a] + (a == c ? 2.0 * trG : 0.0)) * b_bar;
                        double ub = Gb / (2.0 * g->dx); /* + at ip, - at im */
                        long p = ip[c], q = im[c];
                        mb[a][p] += ub / rho[p];
                        rhob[p] -= ub * m[a][p] / (rho[p] * rho[p]);
                        mb[a][q] -= ub / rho[q];
                        rhob[q] += ub * m[a][q] / (rho[q] * rho[q]);
                    }
            }
}

/* reverse of `sweeps` Jacobi sweeps. it[0..sweeps] are the iterates of the
 * forward solve (it[0] the warm start). sb: in, the adjoint of it[sweeps];
 * out, the adjoint of it[0]. bb and rhob accumulate. With D_i the diagonal
 * and mu = lambda / D, the adjoint of a sweep is the same 7-point stencil
 * applied to mu (the operator is symmetric). */
static void jacobi_rev(const orc_grid *g, const double *q, double *const *it, int sweeps, double *sb,
                       double *bb, double *rhob)
{
    long N = ncell(g);
    const double *rho = q;
    double beta = g->alpha / (g->dx * g->dx);
    double *mu = malloc(sizeof(double) * N), *rb = calloc(N, sizeof(double)), *nl = malloc(sizeof(double) * N);
    for (int it_k = sweeps - 1; it_k >= 0; it_k--) {
        const double *s0 = it[it_k], *F = it[it_k + 1];
        for (long c = 0; c < N; c++) nl[c] = 0.0;
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    long c = I(g, i, j, k), nb;
                    double ri = 1.0 / rho[c], diag = ri;
                    for (int d = 0; d < 6; d++)
                        if (neighbour(g, i, j, k, d, &nb)) diag += beta * 0.5 * (ri + 1.0 / rho[nb]);
                    mu[c] = sb[c] / diag;
                }
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    long c = I(g, i, j, k), nb;
                    double ri = 1.0 / rho[c];
                    double ssum = 0.0;
                    int nf = 0;
                    bb[c] += mu[c];
                    for (int d = 0; d < 6; d++) {
                        if (!neighbour(g, i, j, k, d, &nb)) continue;
                        double cf = 0.5 * (ri + 1.0 / rho[nb]);
                        nl[nb] += beta * cf * mu[c];
                        ssum += s0[nb];
                        nf++;
                        rb[nb] += mu[c] * 0.5 * beta * (s0[nb] - F[c]);
                    }
                    rb[c] += mu[c] * (0.5 * beta * ssum - F[c] * (1.0 + 0.5 * beta * nf));
                }
        for (long c = 0; c < N; c++) sb[c] = nl[c];
    }
    for (long c = 0; c < N; c++) rhob[c] -= rb[c] / (rho[c] * rho[c]);
    free(mu);
    free(rb);
    free(nl);
}

/* reverse of phys_flux: Fb (5) and ab (adjoint of |u_d| + c) into qvb (5), sigb */
static void phys_flux_rev(const orc_grid *g, const double qv[NV], double sig, int d, const double Fb[NV],
                          double ab, double qvb[NV], double *sigb)
{
    double gm = g->gamma;
    double rho = qv[0], E = qv[4];
    double u[3] = {qv[1] / rho, qv[2] / rho, qv[3] / rho};
    double ke = 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double p = (gm - 1.0) * (E - ke);
    double P = p + sig;
    double c = sqrt(gm * p / rho);
    double ub[3] = {0, 0, 0}, rhob = 0, Eb = 0, Pb = 0, pb = 0;
    /* F0 = rho u_d, F[1+a] = m_a u_d + P delta_ad, F4 = (E + P) u_d */
    rhob += Fb[0] * u[d];
    ub[d] += Fb[0] * rho;
    for (int a = 0; a < 3; a++) {
        qvb[1 + a] += Fb[1 + a] * u[d];
        ub[d] += Fb[1 + a] * qv[1 + a];
    }
    Pb += Fb[1 + d];
    Eb += Fb[4] * u[d];
    Pb += Fb[4] * u[d];
    ub[d] += Fb[4] * (E + P);
    /* a = |u_d| + sqrt(gamma p / rho) */
    ub[d] += ab * (u[d] > 0 ? 1.0 : (u[d] < 0 ? -1.0 : 0.0));
    pb += ab * gm / (2.0 * c * rho);
    rhob += -ab * c / (2.0 * rho);
    /* P = p + Sigma; p = (gamma-1)(E - ke); ke = rho |u|^2 / 2 */
    pb += Pb;
    *sigb += Pb;
    Eb += (gm - 1.0) * pb;
    double keb = -(gm - 1.0) * pb;
    rhob += keb * 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; a++) ub[a] += keb * rho * u[a];
    /* u_a = m_a / rho */
    for (int a = 0; a < 3; a++) {
        qvb[1 + a] += ub[a] / rho;
        rhob -= ub[a] * u[a] / rho;
    }
    qvb[0] += rhob;
    qvb[4] += Eb;
}

/* reverse of rhs_from_ghosts: Lb (adjoint of L, interior) into qgb, sgb */
static void rhs_rev(const orc_grid *g, const double *qg, const double *sg, const double *Lb, double *qgb,
                    double *sgb)
{
    static const double cl[6] = {2.0 / 60, -13.0 / 60, 47.0 / 60, 27.0 / 60, -3.0 / 60, 0.0};
    static const double cr[6] = {0.0, -3.0 / 60, 27.0 / 60, 47.0 / 60, -13.0 / 60, 2.0 / 60};
    long N = ncell(g), NG = nghost(g);
    int n3[3] = {g->nx, g->ny, g->nz};
    for (int d = 0; d < 3; d++) {
        int fx = g->nx + (d == 0), fy = g->ny + (d == 1), fz = g->nz + (d == 2);
        for (int k = 0; k < fz; k++)
            for (int j = 0; j < fy; j++)
                for (int i = 0; i < fx; i++) {
                    int c3[3] = {i, j, k};
                    int f = c3[d];
                    /* F_hat at face f is -1/dx in L of cell f-1 and +1/dx in L of cell f */
                    double Fh_b[NV];
                    for (int v = 0; v < NV; v++) {
                        double lo = 0.0, hi = 0.0;
                        if (f >= 1) {
                            int cc[3] = {i, j, k};
                            cc[d] = f - 1;
                            lo = Lb[v * N + I(g, cc[0], cc[1], cc[2])];
                        }
                        if (f < n3[d]) hi = Lb[v * N + I(g, i, j, k)];
                        Fh_b[v] = (hi - lo) / g->dx;
                    }
                    long pos[6];
                    double vq[NV + 1][6];
                    for (int s = 0; s < 6; s++) {
                        int cc[3] = {i, j, k};
                        cc[d] += s - 3;
                        pos[s] = GI(g, cc[0], cc[1], cc[2]);
                        for (int v = 0; v < NV; v++) vq[v][s] = qg[v * NG + pos[s]];
                        vq[NV][s] = sg[pos[s]];
                    }
                    double qL[NV], qR[NV], FL[NV], FR[NV];
                    for (int v = 0; v < NV; v++) {
                        qL[v] = face_left(g, vq[v]);
                        qR[v] = face_right(g, vq[v]);
                    }
                    double sL = face_left(g, vq[NV]), sR = face_right(g, vq[NV]);
                    double aL = phys_flux(g, qL, sL, d, FL);
                    double aR = phys_flux(g, qR, sR, d, FR);
                    double lam = aL > aR ? aL : aR;
                    double FLb[NV], FRb[NV], qLb[NV] = {0}, qRb[NV] = {0}, sLb = 0, sRb = 0, lamb = 0;
                    for (int v = 0; v < NV; v++) {
                        FLb[v] = 0.5 * Fh_b[v];
                        FRb[v] = 0.5 * Fh_b[v];
                        qLb[v] += 0.5 * lam * Fh_b[v];
                        qRb[v] -= 0.5 * lam * Fh_b[v];
                        lamb -= 0.5 * (qR[v] - qL[v]) * Fh_b[v];
                    }
                    double aLb = aL > aR ? lamb : 0.0, aRb = aL > aR ? 0.0 : lamb;
                    phys_flux_rev(g, qL, sL, d, FLb, aLb, qLb, &sLb);
                    phys_flux_rev(g, qR, sR, d, FRb, aRb, qRb, &sRb);
                    for (int s = 0; s < 6; s++) {
                        for (int v = 0; v < NV; v++) qgb[v * NG + pos[s]] += cl[s] * qLb[v] + cr[s] * qRb[v];
                        sgb[pos[s]] += cl[s] * sLb + cr[s] * sRb;
                    }
                }
    }
}

/* Adjoint of one SSP-RK3 step with fixed dt > 0 from (q, sigma):
 * lq, ls: adjoints of q', Sigma' (inputs); lq_out, ls_out: adjoints of q,
 * Sigma (outputs, overwritten); gw (njets) accumulates the jet-velocity
 * gradient. */
void orc_adjoint_step(const orc_grid *g, const double *q, const double *sigma, double dt,
                      const double *lq, const double *ls, double *lq_out, double *ls_out, double *gw)
{
    long N = ncell(g), NG = nghost(g);
    int S = g->sweeps;
    const double wst[3] = {1.0, 0.25, 2.0 / 3.0};
    /* forward recompute with storage */
    double *qs[3], *its[3][64];
    double *qg = malloc(sizeof(double) * NV * NG), *sg = malloc(sizeof(double) * NG);
    double *b = malloc(sizeof(double) * N), *L = malloc(sizeof(double) * NV * N);
    for (int st = 0; st < 3; st++) {
        qs[st] = malloc(sizeof(double) * NV * N);
        for (int s = 0; s <= S; s++) its[st][s] = malloc(sizeof(double) * N);
    }
    memcpy(qs[0], q, sizeof(double) * NV * N);
    memcpy(its[0][0], sigma, sizeof(double) * N);
    for (int st = 0; st < 3; st++) {
        orc_fill_ghosts(g, qs[st], qg);
        source_from_ghosts(g, qg, b);
        for (int s = 0; s < S; s++) {
            memcpy(its[st][s + 1], its[st][s], sizeof(double) * N);
            orc_jacobi(g, qs[st], b, its[st][s + 1], 1);
        }
        if (st < 2) {
            fill_sigma_ghosts(g, its[st][S], sg);
            rhs_from_ghosts(g, qg, sg, L);
            for (long n = 0; n < NV * N; n++)
                qs[st + 1][n] = q[n] + wst[st] * ((qs[st][n] - q[n]) + dt * L[n]);
            memcpy(its[st + 1][0], its[st][S], sizeof(double) * N);
        }
    }
    /* reverse */
    double *lqs = calloc(NV * N, sizeof(double)), *lq0 = calloc(NV * N, sizeof(double));
    double *lsig = malloc(sizeof(double) * N), *lb = malloc(sizeof(double) * N);
    double *qgb = malloc(sizeof(double) * NV * NG), *sgb = malloc(sizeof(double) * NG);
    double *Lb = calloc(NV * N, sizeof(double));
    double *lamJ = calloc((long)NV * g->ny * g->nx, sizeof(double));
    double *lout = malloc(sizeof(double) * NV * N);
    memcpy(lout, lq, sizeof(double) * NV * N);
    memcpy(lsig, ls, sizeof(double) * N);
    for (int st = 2; st >= 0; st--) {
        double w = wst[st];
        /* out = q + w ((qs - q) + dt L(qs, Sigma^S)) */
        for (long n = 0; n < NV * N; n++) {
            lq0[n] += (1.0 - w) * lout[n];
            lqs[n] = w * lout[n];
            Lb[n] = w * dt * lout[n];
        }
        orc_fill_ghosts(g, qs[st], qg);
        fill_sigma_ghosts(g, its[st][S], sg);
        memset(qgb, 0, sizeof(double) * NV * NG);
        memset(sgb, 0, sizeof(double) * NG);
        rhs_rev(g, qg, sg, Lb, qgb, sgb);
        fill_sigma_ghosts_rev(g, sgb, lsig); /* lsig: adjoint of Sigma^S */
        memset(lb, 0, sizeof(double) * N);
        jacobi_rev(g, qs[st], its[st], S, lsig, lb, lqs); /* rho adjoint into lqs[0..N) */
        source_rev(g, qg, lb, qgb);
        fill_ghosts_rev(g, qgb, lqs, lamJ);
        /* the stage input is q (stage 1) or the previous stage's output */
        if (st == 0)
            for (long n = 0; n < NV * N; n++) lq0[n] += lqs[n];
        else
            memcpy(lout, lqs, sizeof(double) * NV * N);
    }
    memcpy(lq_out, lq0, sizeof(double) * NV * N);
    memcpy(ls_out, lsig, sizeof(double) * N);
    /* jet tables: J[v](x, y) = sum_n s_n q_jet_n[v]; d q_jet_n / d w_n = (0,0,0,rho_n, rho_n w_n) */
    for (int n = 0; n < g->njets; n++) {
        const double *Jt = g->jets + 7 * n;
        double acc = 0.0;
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                double x = (i + 0.5) * g->dx, y = (j + 0.5) * g->dx;
                double r = sqrt((x - Jt[0]) * (x - Jt[0]) + (y - Jt[1]) * (y - Jt[1]));
                double sn = 0.5 * (1.0 - tanh((r - Jt[2]) / (Jt[6] * g->dx)));
                long f = (long)j * g->nx + i;
                acc += sn * (Jt[3] * lamJ[3L * g->ny * g->nx + f] + Jt[3] * Jt[4] * lamJ[4L * g->ny * g->nx + f]);
            }
        gw[n] += acc;
    }
    for (int st = 0; st < 3; st++) {
        free(qs[st]);
        for (int s = 0; s <= S; s++) free(its[st][s]);
    }
    free(qg); free(sg); free(b); free(L); free(lqs); free(lq0); free(lsig); free(lb);
    free(qgb); free(sgb); free(Lb); free(lamJ); free(lout);
}

/* ---------------- vector-Jacobian products of the parts (for pinning) */

/* qb (5N) += (dL/dq)^T Lb, sb (N) += (dL/dSigma)^T Lb, lamJ ignored */
void orc_rhs_vjp(const orc_grid *g, const double *q, const double *sigma, const double *Lb, double *qb,
                 double *sb)
{
    long NG = nghost(g);
    double *qg = malloc(sizeof(double) * NV * NG), *sg = malloc(sizeof(double) * NG);
    double *qgb = calloc(NV * NG, sizeof(double)), *sgb = calloc(NG, sizeof(double));
    double *lamJ = calloc((long)NV * g->ny * g->nx, sizeof(double));
    orc_fill_ghosts(g, q, qg);
    fill_sigma_ghosts(g, sigma, sg);
    rhs_rev(g, qg, sg, Lb, qgb, sgb);
    fill_sigma_ghosts_rev(g, sgb, sb);
    fill_ghosts_rev(g, qgb, qb, lamJ);
    free(qg); free(sg); free(qgb); free(sgb); free(lamJ);
}

/* qb (5N) += (db/dq)^T bb */
void orc_source_vjp(const orc_grid *g, const double *q, const double *bb, double *qb)
{
    long NG = nghost(g);
    double *qg = malloc(sizeof(double) * NV * NG), *qgb = calloc(NV * NG, sizeof(double));
    double *lamJ = calloc((long)NV * g->ny * g->nx, sizeof(double));
    orc_fill_ghosts(g, q, qg);
    source_rev(g, qg, bb, qgb);
    fill_ghosts_rev(g, qgb, qb, lamJ);
    free(qg); free(qgb); free(lamJ);
}

/* Jacobi sweeps from sigma0: sb in = adjoint of the result, out = adjoint of
 * sigma0; bb (N) and rhob (N) accumulate */
void orc_jacobi_vjp(const orc_grid *g, const double *q, const double *b, const double *sigma0, int sweeps,
                    double *sb, double *bb, double *rhob)
{
    long N = ncell(g);
    double *it[64] = {0};
    for (int s = 0; s <= sweeps; s++) it[s] = malloc(sizeof(double) * N);
    memcpy(it[0], sigma0, sizeof(double) * N);
    for (int s = 0; s < sweeps; s++) {
        memcpy(it[s + 1], it[s], sizeof(double) * N);
        orc_jacobi(g, q, b, it[s + 1], 1);
    }
    jacobi_rev(g, q, it, sweeps, sb, bb, rhob);
    for (int s = 0; s <= sweeps; s++) free(it[s]);
}
