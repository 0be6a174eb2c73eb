/*
 * oracle.c -- plain, slow FP64 CPU restatement of the differentiable MAC-grid
 * fluid step of arXiv 2503.00868 ("3D Dynamic Fluid Assets from Single-View
 * Videos with Generative Gaussian Splatting").
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library; the product path never does. It shares
 * no code, header, table or helper with the CUDA implementation.
 *
 * What it computes (paper passages):
 *   - Eq. (eq::v), Sec. 3.2.2: dv/dt = -grad p / rho + div(2 nu S) + g, solved by
 *     operator splitting (Chorin) with a pressure Poisson equation.
 *   - Sec. 3.4.1: grid convection by semi-Lagrangian back-tracing (Stam).
 *   - Sec. 3.4.1: the Poisson pressure equation (solved here by (P)CG; the paper
 *     replaces the implicit solve by PeRCNN, which is fitted to solver output).
 *   - Sec. 3.4.2, Eq. (eq::optLoss): masked cosine + L2 loss on grid velocities.
 *   - Sec. 3.4.1, Fig. percnn_str_fit: a small 3D convolution network that maps a
 *     pressure right-hand side to a pressure (used as a PCG preconditioner).
 *   - Sec. 3.3.3: the volumetric-velocity initialisation, a laminar wall-function
 *     base profile and the constrained divergence projection of Eq. (eq::divProj).
 *   - Sec. 3.4.1: the recurrent convolutional (PeRCNN) pressure solver.
 *   - Sec. 3.2.2, Sec. 3.4.3: APIC transfers (Eq. eq::particle_map, the G2P and C
 *     update) per MAC face component, particle advection, and the deformation
 *     gradient and covariance update of the Gaussians.
 *   - Sec. 3.2.1, Sec. 3.5: front-to-back splatting of the Gaussians into an image.
 *
 * Readings where the paper is silent (each is restated where it is used):
 *   R1 split order: advect -> body force -> implicit viscosity -> projection, so
 *      every step ends divergence-free.
 *   R2 viscosity: constant nu, backward Euler (I + nu dt L_f) u_v = u_b per
 *      component on fluid faces.
 *   R3 advection: one forward-Euler back-trace in index space, trilinear sample
 *      of the own component, continuous index clamped to [0, n-1].
 *   R4 pressure: p = 0 in air cells, solid walls are Neumann, the all-liquid
 *      closed box removes the mean of the right-hand side.
 *   R5 MIC(0) (Bridson, Fluid Simulation for Computer Graphics, 2nd ed.):
 *      tau = 0.97, safety sigma = 0.25, lexicographic order with x fastest.
 *   R6 loss: halved squared L2 averaged over band faces plus (1 - cos) averaged
 *      over band cells on cell-centred velocities, eps = 1e-8.
 *
 * Dense array layout (C order, x fastest), all FP64:
 *   cells        (nz, ny, nx)        index (k*ny + j)*nx + i
 *   u  faces     (nz, ny, nx+1)      u(i,j,k) sits between cells (i-1,j,k), (i,j,k)
 *   v  faces     (nz, ny+1, nx)      v(i,j,k) sits between cells (i,j-1,k), (i,j,k)
 *   w  faces     (nz+1, ny, nx)      w(i,j,k) sits between cells (i,j,k-1), (i,j,k)
 * Cell types: 0 air, 1 liquid, 2 solid; cells outside the array are solid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { AIR = 0, LIQUID = 1, SOLID = 2 };
enum { FC_AIR = 0, FC_FLUID = 1, FC_FIXED = 2 };
enum { PC_NONE = 0, PC_JACOBI = 1, PC_MIC0 = 2 };
enum { ST_OK = 0, ST_NOCONV = 1, ST_BREAKDOWN = 2 };

typedef struct {
    int nx, ny, nz;
    const uint8_t *type;        /* cell types, (nz, ny, nx) */
    const double *bc[3];        /* prescribed values on fixed faces; NULL = 0 */
    double dx, dt, nu;
    double g[3];                /* body force (acceleration) per component */
    double tol_p, tol_v;        /* relative residual targets of the two solves */
    int maxit_p, maxit_v;
    int precond;                /* pressure preconditioner: PC_NONE/JACOBI/MIC0 */
    double mic_tau, mic_sigma;
    const double *percnn_w;     /* 27 taps [dz][dy][dx]; with percnn_k > 0 the projection */
    int percnn_k;               /* solves the pressure by that many recurrent sub-steps */
    int advect_grad;            /* reverse of advection: 0 the exact adjoint, 1 the upwind surrogate */
} or_grid;

typedef struct {
    int iters;
    int status;
    double relres;       /* recursive residual at exit, relative */
    double true_relres;  /* |b - A x| / |b| recomputed at exit */
} or_stats;

/* ------------------------------------------------------------------------ */
/* indexing                                                                  */
/* ------------------------------------------------------------------------ */

static void face_dims(const or_grid *g, int c, int d[3])
{
    d[0] = g->nx; d[1] = g->ny; d[2] = g->nz;
    d[c] += 1;
}

static long fidx(const int d[3], int i, int j, int k)
{
    return ((long)k * d[1] + j) * d[0] + i;
}

static long ncells(const or_grid *g) { return (long)g->nx * g->ny * g->nz; }

static long nfaces(const or_grid *g, int c)
{
    int d[3];
    face_dims(g, c, d);
    return (long)d[0] * d[1] * d[2];
}

static long cidx(const or_grid *g, int i, int j, int k)
{
    return ((long)k * g->ny + j) * g->nx + i;
}

static int cell_type(const or_grid *g, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz)
        return SOLID;
    return g->type[cidx(g, i, j, k)];
}

/* A face touching a solid cell has a prescribed (fixed) value. A face between two
 * non-solid cells with at least one liquid side is a fluid face (an unknown of the
 * viscosity solve, moved by the pressure gradient). A face between two air cells
 * holds zero. */
static int face_class(const or_grid *g, int c, int i, int j, int k)
{
    int o[3] = {0, 0, 0};
    o[c] = 1;
    int tl = cell_type(g, i - o[0], j - o[1], k - o[2]);
    int tr = cell_type(g, i, j, k);
    if (tl == SOLID || tr == SOLID) return FC_FIXED;
    if (tl == LIQUID || tr == LIQUID) return FC_FLUID;
    return FC_AIR;
}

static double bc_value(const or_grid *g, int c, long f)
{
    return g->bc[c] ? g->bc[c][f] : 0.0;
}

void or_face_class(const or_grid *g, int c, uint8_t *out)
{
    int d[3];
    face_dims(g, c, d);
    for (int k = 0; k < d[2]; k++)
        for (int j = 0; j < d[1]; j++)
            for (int i = 0; i < d[0]; i++)
                out[fidx(d, i, j, k)] = (uint8_t)face_class(g, c, i, j, k);
}

/* ------------------------------------------------------------------------ */
/* vector helpers over concatenated face fields                              */
/* ------------------------------------------------------------------------ */

static double dot(const double *a, const double *b, long n)
{
    double s = 0.0;
    for (long t = 0; t < n; t++) s += a[t] * b[t];
    return s;
}

/* ------------------------------------------------------------------------ */
/* a1 + a2: semi-Lagrangian advection with body force (Sec. 3.4.1; Eq. eq::v)  */
/* ------------------------------------------------------------------------ */

/* Per-dimension trilinear set-up for a continuous index s on an axis of n
 * samples: clamp to [0, n-1]; base = min(floor(s), n-2); frac = s - base.
 * `active` is 0 when the clamp bound (the derivative w.r.t. s is then zero). */
static void axis_setup(double s, int n, int *base, double *frac, int *active)
{
    *active = 1;
    if (s < 0.0) { s = 0.0; *active = 0; }
    if (s > (double)(n - 1)) { s = (double)(n - 1); *active = 0; }
    int b = (int)floor(s);
    if (b > n - 2) b = n - 2;
    *base = b;
    *frac = s - (double)b;
}

/* The velocity seen by face (i,j,k) of component c: its own value, and for each
 * other component e the mean of the four e-faces of the two cells that share the
 * face. */
static void face_velocity(const or_grid *g, int c, int i, int j, int k,
                          const double *const u[3], double vel[3])
{
    int dc[3];
    face_dims(g, c, dc);
    vel[c] = u[c][fidx(dc, i, j, k)];
    int L[3] = {i, j, k}, R[3] = {i, j, k};
    L[c] -= 1;
    for (int e = 0; e < 3; e++) {
        if (e == c) continue;
        int de[3];
        face_dims(g, e, de);
        int Lp[3] = {L[0], L[1], L[2]}, Rp[3] = {R[0], R[1], R[2]};
        Lp[e] += 1;
        Rp[e] += 1;
        vel[e] = 0.25 * (u[e][fidx(de, L[0], L[1], L[2])] + u[e][fidx(de, Lp[0], Lp[1], Lp[2])] +
                         u[e][fidx(de, R[0], R[1], R[2])] + u[e][fidx(de, Rp[0], Rp[1], Rp[2])]);
    }
}

typedef struct {
    int base[3];
    double frac[3];
    int active[3];
} trace_t;

static void back_trace(const or_grid *g, int c, int i, int j, int k,
                       const double vel[3], trace_t *t)
{
    int dc[3];
    face_dims(g, c, dc);
    int idx[3] = {i, j, k};
    double h = g->dt / g->dx;
    for (int e = 0; e < 3; e++) {
        double s = (double)idx[e] - h * vel[e];
        axis_setup(s, dc[e], &t->base[e], &t->frac[e], &t->active[e]);
    }
}

static double trilinear(const double *f, const int d[3], const trace_t *t)
{
    double acc = 0.0;
    for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < 2; cy++)
            for (int cx = 0; cx < 2; cx++) {
                double w = (cx ? t->frac[0] : 1.0 - t->frac[0]) *
                           (cy ? t->frac[1] : 1.0 - t->frac[1]) *
                           (cz ? t->frac[2] : 1.0 - t->frac[2]);
                acc += w * f[fidx(d, t->base[0] + cx, t->base[1] + cy, t->base[2] + cz)];
            }
    return acc;
}

void or_advect(const or_grid *g, const double *const u[3], double *const ua[3])
{
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    int cls = face_class(g, c, i, j, k);
                    if (cls == FC_FIXED) { ua[c][f] = bc_value(g, c, f); continue; }
                    if (cls == FC_AIR) { ua[c][f] = 0.0; continue; }
                    double vel[3];
                    trace_t t;
                    face_velocity(g, c, i, j, k, u, vel);
                    back_trace(g, c, i, j, k, vel, &t);
                    ua[c][f] = trilinear(u[c], d, &t) + g->dt * g->g[c];
                }
    }
}

/* The back-traced sample point of every face of component c, as used by
 * or_advect: s_out[3 f + e] = idx_e - (dt/dx) vel_e before clamping, for the
 * fluid faces f (NaN on fixed and air faces, which are not advected). A test
 * helper: trilinear interpolation is not differentiable where a coordinate of
 * s is an integer, so the reverse pass is not unique there. */
void or_advect_samples(const or_grid *g, int c, const double *const u[3], double *s_out)
{
    int d[3];
    face_dims(g, c, d);
    const double h = g->dt / g->dx;
    for (int k = 0; k < d[2]; k++)
        for (int j = 0; j < d[1]; j++)
            for (int i = 0; i < d[0]; i++) {
                long f = fidx(d, i, j, k);
                int idx[3] = {i, j, k};
                if (face_class(g, c, i, j, k) != FC_FLUID) {
                    for (int e = 0; e < 3; e++) s_out[3 * f + e] = NAN;
                    continue;
                }
                double vel[3];
                face_velocity(g, c, i, j, k, u, vel);
                for (int e = 0; e < 3; e++) s_out[3 * f + e] = (double)idx[e] - h * vel[e];
            }
}

/* Exact discrete adjoint of or_advect w.r.t. the input field: given the
 * cotangent ga of the advected field, ACCUMULATE d<ga, advect(u)>/du into gu.
 * Fixed and air faces of the output are constants and contribute nothing. */
void or_advect_adjoint(const or_grid *g, const double *const u[3],
                       const double *const ga[3], double *const gu[3])
{
    double h = g->dt / g->dx;
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                    double w = ga[c][f];
                    if (w == 0.0) continue;
                    double vel[3];
                    trace_t t;
                    face_velocity(g, c, i, j, k, u, vel);
                    back_trace(g, c, i, j, k, vel, &t);
                    /* value term: the trilinear weights */
                    double dsd[3] = {0.0, 0.0, 0.0}; /* d sample / d s_e */
                    for (int cz = 0; cz < 2; cz++)
                        for (int cy = 0; cy < 2; cy++)
                            for (int cx = 0; cx < 2; cx++) {
                                double wx = cx ? t.frac[0] : 1.0 - t.frac[0];
                                double wy = cy ? t.frac[1] : 1.0 - t.frac[1];
                                double wz = cz ? t.frac[2] : 1.0 - t.frac[2];
                                long fc = fidx(d, t.base[0] + cx, t.base[1] + cy, t.base[2] + cz);
                                gu[c][fc] += w * wx * wy * wz;
                                double val = u[c][fc];
                                dsd[0] += (cx ? 1.0 : -1.0) * wy * wz * val;
                                dsd[1] += wx * (cy ? 1.0 : -1.0) * wz * val;
                                dsd[2] += wx * wy * (cz ? 1.0 : -1.0) * val;
                            }
                    /* position term: s_e = idx_e - h * vel_e, unless clamped */
                    for (int e = 0; e < 3; e++) {
                        if (!t.active[e]) continue;
                        double gv = -h * dsd[e] * w; /* d/d vel_e */
                        if (e == c) {
                            gu[c][f] += gv;
                        } else {
                            int de[3];
                            face_dims(g, e, de);
                            int L[3] = {i, j, k}, R[3] = {i, j, k};
                            L[c] -= 1;
                            int Lp[3] = {L[0], L[1], L[2]}, Rp[3] = {R[0], R[1], R[2]};
                            Lp[e] += 1;
                            Rp[e] += 1;
                            gu[e][fidx(de, L[0], L[1], L[2])] += 0.25 * gv;
                            gu[e][fidx(de, Lp[0], Lp[1], Lp[2])] += 0.25 * gv;
                            gu[e][fidx(de, R[0], R[1], R[2])] += 0.25 * gv;
                            gu[e][fidx(de, Rp[0], Rp[1], Rp[2])] += 0.25 * gv;
                        }
                    }
                }
    }
}

/* The paper's surrogate for the reverse pass of convection (Sec. 3.4.1): the
 * derivative of the convected velocity v with respect to the velocity component
 * i that transports it is taken as -dt dv/di, with dv/di by a first-order
 * upwind difference, instead of differentiating the back-trace. Reading taken
 * (the passage gives only that derivative): the cotangent of each convected
 * fluid face f of component c passes unchanged to the same face of the input
 * (the value the face carries), and each velocity component e seen at f
 * (ubar_e of the back-trace: the own component, or the mean of four faces of
 * another) receives -dt ga_c(f) dv_c/de at f. dv_c/de is the index-space
 * difference of the convected field v along e divided by dx, taken on the
 * upstream side of ubar_e (the side the flow comes from: the lower neighbour
 * when ubar_e > 0, else the upper one), and zero where that neighbour is
 * outside the face array. v is the
 * convected field (or_advect of u); ACCUMULATES into gu. */
void or_advect_adjoint_upwind(const or_grid *g, const double *const u[3],
                              const double *const ga[3], double *const gu[3])
{
    double h = g->dt / g->dx;
    long nf[3];
    double *va[3];
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        nf[c] = (long)d[0] * d[1] * d[2];
        va[c] = (double *)calloc((size_t)nf[c], sizeof(double));
    }
    or_advect(g, u, va);
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                    double w = ga[c][f];
                    if (w == 0.0) continue;
                    gu[c][f] += w; /* the value term */
                    double vel[3];
                    face_velocity(g, c, i, j, k, u, vel);
                    int idx[3] = {i, j, k};
                    for (int e = 0; e < 3; e++) {
                        /* upwind difference of v_c along e, in index units */
                        int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                        if (vel[e] > 0.0) lo[e] -= 1; else hi[e] += 1;
                        if (lo[e] < 0 || hi[e] >= d[e]) continue;
                        (void)idx;
                        double dv = va[c][fidx(d, hi[0], hi[1], hi[2])] - va[c][fidx(d, lo[0], lo[1], lo[2])];
                        double gv = -h * dv * w; /* d/d ubar_e */
                        if (e == c) {
                            gu[c][f] += gv;
                        } else {
                            int de[3];
                            face_dims(g, e, de);
                            int L[3] = {i, j, k}, R[3] = {i, j, k};
                            L[c] -= 1;
                            int Lp[3] = {L[0], L[1], L[2]}, Rp[3] = {R[0], R[1], R[2]};
                            Lp[e] += 1;
                            Rp[e] += 1;
                            gu[e][fidx(de, L[0], L[1], L[2])] += 0.25 * gv;
                            gu[e][fidx(de, Lp[0], Lp[1], Lp[2])] += 0.25 * gv;
                            gu[e][fidx(de, R[0], R[1], R[2])] += 0.25 * gv;
                            gu[e][fidx(de, Rp[0], Rp[1], Rp[2])] += 0.25 * gv;
                        }
                    }
                }
    }
    for (int c = 0; c < 3; c++) free(va[c]);
}

/* ------------------------------------------------------------------------ */
/* a3: implicit viscosity (Eq. eq::v viscous stress, backward Euler)          */
/* ------------------------------------------------------------------------ */

/* Neighbour rule for the face Laplacian of a fluid face: a fluid neighbour is
 * coupled, a fixed neighbour is a Dirichlet value, an air neighbour or one
 * beyond the array (tangential at a box wall) is a mirror (zero flux). */

/* y = (I + nu dt L_f) x on fluid faces, zero elsewhere; Dirichlet values are
 * left out (they belong to the right-hand side). */
void or_visc_apply(const or_grid *g, const double *const x[3], double *const y[3])
{
    double cc = g->nu * g->dt / (g->dx * g->dx);
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    if (face_class(g, c, i, j, k) != FC_FLUID) { y[c][f] = 0.0; continue; }
                    double xf = x[c][f], acc = xf;
                    int idx[3] = {i, j, k};
                    for (int e = 0; e < 3; e++)
                        for (int sgn = -1; sgn <= 1; sgn += 2) {
                            int n[3] = {idx[0], idx[1], idx[2]};
                            n[e] += sgn;
                            if (n[e] < 0 || n[e] >= d[e]) continue;
                            int cl = face_class(g, c, n[0], n[1], n[2]);
                            if (cl == FC_FLUID) acc += cc * (xf - x[c][fidx(d, n[0], n[1], n[2])]);
                            else if (cl == FC_FIXED) acc += cc * xf;
                        }
                    y[c][f] = acc;
                }
    }
}

/* Dirichlet part of the right-hand side: cc * sum of fixed neighbour values. */
static void visc_dirichlet(const or_grid *g, double *const out[3])
{
    double cc = g->nu * g->dt / (g->dx * g->dx);
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    out[c][f] = 0.0;
                    if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                    int idx[3] = {i, j, k};
                    for (int e = 0; e < 3; e++)
                        for (int sgn = -1; sgn <= 1; sgn += 2) {
                            int n[3] = {idx[0], idx[1], idx[2]};
                            n[e] += sgn;
                            if (n[e] < 0 || n[e] >= d[e]) continue;
                            if (face_class(g, c, n[0], n[1], n[2]) == FC_FIXED)
                                out[c][f] += cc * bc_value(g, c, fidx(d, n[0], n[1], n[2]));
                        }
                }
    }
}

/* The face Laplacian with Dirichlet values taken from the field itself
 * ((L~ u)_f = sum over coupled and fixed neighbours of (u_f - u_n) / dx^2);
 * used by the viscosity gradient. Zero off fluid faces. */
static void visc_laplacian_full(const or_grid *g, const double *const u[3], double *const y[3])
{
    double inv = 1.0 / (g->dx * g->dx);
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    y[c][f] = 0.0;
                    if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                    int idx[3] = {i, j, k};
                    double acc = 0.0;
                    for (int e = 0; e < 3; e++)
                        for (int sgn = -1; sgn <= 1; sgn += 2) {
                            int n[3] = {idx[0], idx[1], idx[2]};
                            n[e] += sgn;
                            if (n[e] < 0 || n[e] >= d[e]) continue;
                            int cl = face_class(g, c, n[0], n[1], n[2]);
                            if (cl == FC_AIR) continue;
                            acc += u[c][f] - u[c][fidx(d, n[0], n[1], n[2])];
                        }
                    y[c][f] = acc * inv;
                }
    }
}

/* Conjugate gradients on the fluid faces for (I + nu dt L_f) x = rhs, starting
 * from x = 0, stopping at |r|/|rhs| <= tol_v. Vectors are zero off fluid faces. */
static void visc_cg(const or_grid *g, double *const rhs[3], double *const x[3], or_stats *st)
{
    long n[3] = {nfaces(g, 0), nfaces(g, 1), nfaces(g, 2)};
    long ntot = n[0] + n[1] + n[2];
    double *buf = (double *)calloc((size_t)ntot * 3, sizeof(double));
    double *r = buf, *p = buf + ntot, *q = buf + 2 * ntot;
    double *rr3[3] = {r, r + n[0], r + n[0] + n[1]};
    double *pp3[3] = {p, p + n[0], p + n[0] + n[1]};
    double *qq3[3] = {q, q + n[0], q + n[0] + n[1]};
    for (int c = 0; c < 3; c++) {
        memcpy(rr3[c], rhs[c], (size_t)n[c] * sizeof(double));
        memset(x[c], 0, (size_t)n[c] * sizeof(double));
    }
    memcpy(p, r, (size_t)ntot * sizeof(double));
    double bb = dot(r, r, ntot), rr = bb;
    st->iters = 0;
    st->status = ST_OK;
    st->relres = 0.0;
    if (bb > 0.0) {
        int it;
        for (it = 1; it <= g->maxit_v; it++) {
            or_visc_apply(g, (const double *const *)pp3, qq3);
            double pq = dot(p, q, ntot);
            if (!(pq > 0.0)) { st->status = ST_BREAKDOWN; break; }
            double alpha = rr / pq;
            for (int c = 0; c < 3; c++)
                for (long t = 0; t < n[c]; t++) x[c][t] += alpha * pp3[c][t];
            for (long t = 0; t < ntot; t++) r[t] -= alpha * q[t];
            double rr_new = dot(r, r, ntot);
            st->iters = it;
            if (sqrt(rr_new / bb) <= g->tol_v) { rr = rr_new; break; }
            double beta = rr_new / rr;
            rr = rr_new;
            for (long t = 0; t < ntot; t++) p[t] = r[t] + beta * p[t];
        }
        if (it > g->maxit_v) st->status = ST_NOCONV;
        st->relres = sqrt(rr / bb);
    }
    /* true residual */
    or_visc_apply(g, (const double *const *)x, qq3);
    double tr = 0.0;
    for (int c = 0; c < 3; c++)
        for (long t = 0; t < n[c]; t++) {
            double e = rhs[c][t] - qq3[c][t];
            tr += e * e;
        }
    st->true_relres = bb > 0.0 ? sqrt(tr / bb) : 0.0;
    free(buf);
}

/* Solve the viscosity step: fluid faces from the implicit solve, fixed faces take
 * their prescribed values, air faces are zero. `dirichlet` selects whether the
 * fixed neighbours' values enter the right-hand side (forward) or not (adjoint). */
static void visc_solve_impl(const or_grid *g, const double *const ub[3], double *const uv[3],
                            int dirichlet, or_stats *st)
{
    long n[3] = {nfaces(g, 0), nfaces(g, 1), nfaces(g, 2)};
    double *rhs[3], *x[3];
    for (int c = 0; c < 3; c++) {
        rhs[c] = (double *)calloc((size_t)n[c], sizeof(double));
        x[c] = (double *)calloc((size_t)n[c], sizeof(double));
    }
    if (dirichlet) visc_dirichlet(g, rhs);
    for (int c = 0; c < 3; c++) {
        uint8_t *cls = (uint8_t *)malloc((size_t)n[c]);
        or_face_class(g, c, cls);
        for (long t = 0; t < n[c]; t++)
            rhs[c][t] = (cls[t] == FC_FLUID) ? rhs[c][t] + ub[c][t] : 0.0;
        free(cls);
    }
    visc_cg(g, rhs, x, st);
    for (int c = 0; c < 3; c++) {
        uint8_t *cls = (uint8_t *)malloc((size_t)n[c]);
        or_face_class(g, c, cls);
        for (long t = 0; t < n[c]; t++) {
            if (cls[t] == FC_FLUID) uv[c][t] = x[c][t];
            else if (cls[t] == FC_FIXED) uv[c][t] = dirichlet ? bc_value(g, c, t) : 0.0;
            else uv[c][t] = 0.0;
        }
        free(cls);
        free(rhs[c]);
        free(x[c]);
    }
}

void or_visc_solve(const or_grid *g, const double *const ub[3], double *const uv[3], or_stats *st)
{
    visc_solve_impl(g, ub, uv, 1, st);
}

/* ------------------------------------------------------------------------ */
/* a4-a6: projection (Sec. 3.2.2 splitting; Poisson pressure equation)        */
/* ------------------------------------------------------------------------ */

/* b_i = -dx * (net outflow of cell i) for liquid cells, zero elsewhere. */
void or_divergence(const or_grid *g, const double *const u[3], double *b)
{
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long ci = cidx(g, i, j, k);
                if (g->type[ci] != LIQUID) { b[ci] = 0.0; continue; }
                double div = 0.0;
                for (int c = 0; c < 3; c++) {
                    int d[3];
                    face_dims(g, c, d);
                    int hi[3] = {i, j, k};
                    hi[c] += 1;
                    div += u[c][fidx(d, hi[0], hi[1], hi[2])] - u[c][fidx(d, i, j, k)];
                }
                b[ci] = -g->dx * div;
            }
}

/* Seven-point pressure operator on liquid cells: each non-solid neighbour adds
 * one to the diagonal, each liquid neighbour -1 off the diagonal; air cells hold
 * p = 0 and solid neighbours add nothing. Zero on non-liquid cells. */
void or_poisson_apply(const or_grid *g, const double *x, double *y)
{
    static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long ci = cidx(g, i, j, k);
                if (g->type[ci] != LIQUID) { y[ci] = 0.0; continue; }
                double acc = 0.0;
                for (int m = 0; m < 6; m++) {
                    int a = i + off[m][0], b = j + off[m][1], cc = k + off[m][2];
                    int t = cell_type(g, a, b, cc);
                    if (t == SOLID) continue;
                    acc += x[ci];
                    if (t == LIQUID) acc -= x[cidx(g, a, b, cc)];
                }
                y[ci] = acc;
            }
}

static int poisson_diag(const or_grid *g, int i, int j, int k)
{
    static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    int dcount = 0;
    for (int m = 0; m < 6; m++)
        if (cell_type(g, i + off[m][0], j + off[m][1], k + off[m][2]) != SOLID) dcount++;
    return dcount;
}

/* Coupling to the next cell along +x, +y, +z: -1 when both are liquid. */
static double poisson_off(const or_grid *g, int i, int j, int k, int e)
{
    int o[3] = {0, 0, 0};
    o[e] = 1;
    if (cell_type(g, i, j, k) != LIQUID) return 0.0;
    if (cell_type(g, i + o[0], j + o[1], k + o[2]) != LIQUID) return 0.0;
    return -1.0;
}

/* u_f -= (q_R - q_L) / dx on fluid faces; q is zero in non-liquid cells. */
void or_grad_subtract(const or_grid *g, const double *q, double *const u[3])
{
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                    int L[3] = {i, j, k};
                    L[c] -= 1;
                    double qr = cell_type(g, i, j, k) == LIQUID ? q[cidx(g, i, j, k)] : 0.0;
                    double ql = cell_type(g, L[0], L[1], L[2]) == LIQUID ? q[cidx(g, L[0], L[1], L[2])] : 0.0;
                    u[c][fidx(d, i, j, k)] -= (qr - ql) / g->dx;
                }
    }
}

/* The pressure operator is singular when the liquid touches no air cell (a
 * closed box full of liquid): its null space is then the constant on the liquid. */
int or_is_singular(const or_grid *g)
{
    static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    int any = 0;
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                if (cell_type(g, i, j, k) != LIQUID) continue;
                any = 1;
                for (int m = 0; m < 6; m++)
                    if (cell_type(g, i + off[m][0], j + off[m][1], k + off[m][2]) == AIR) return 0;
            }
    return any;
}

static void remove_liquid_mean(const or_grid *g, double *x)
{
    long n = ncells(g), cnt = 0;
    double s = 0.0;
    for (long t = 0; t < n; t++)
        if (g->type[t] == LIQUID) { s += x[t]; cnt++; }
    if (!cnt) return;
    s /= (double)cnt;
    for (long t = 0; t < n; t++)
        if (g->type[t] == LIQUID) x[t] -= s;
}

/* MIC(0) factor (Bridson): for each liquid cell in lexicographic order,
 *   e = A_ii - sum_{lower nbr m} (A_mi * prec_m)^2
 *         - tau * sum_{lower nbr m} A_mi * (sum of m's other forward couplings) * prec_m^2,
 *   e < sigma * A_ii  =>  e = A_ii;   prec_i = 1 / sqrt(e).
 * The factor is L with L_ii = 1/prec_i and L_im = A_im * prec_m (m lower). */
void or_mic0_factor(const or_grid *g, double tau, double sigma, double *prec)
{
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long ci = cidx(g, i, j, k);
                prec[ci] = 0.0;
                if (g->type[ci] != LIQUID) continue;
                double diag = (double)poisson_diag(g, i, j, k);
                double e = diag;
                /* lower neighbours along x, y, z */
                int lo[3][3] = {{i - 1, j, k}, {i, j - 1, k}, {i, j, k - 1}};
                for (int a = 0; a < 3; a++) {
                    int *m = lo[a];
                    if (cell_type(g, m[0], m[1], m[2]) != LIQUID) continue;
                    double pm = prec[cidx(g, m[0], m[1], m[2])];
                    double amc = poisson_off(g, m[0], m[1], m[2], a); /* coupling m -> this cell */
                    double other = 0.0;
                    for (int b = 0; b < 3; b++)
                        if (b != a) other += poisson_off(g, m[0], m[1], m[2], b);
                    e -= (amc * pm) * (amc * pm);
                    e -= tau * amc * other * pm * pm;
                }
                if (e < sigma * diag) e = diag;
                prec[ci] = diag > 0.0 ? 1.0 / sqrt(e) : 0.0; /* a liquid cell walled in on all sides */
            }
}

/* z = (L L^T)^{-1} r with the MIC(0) factor: forward then backward substitution. */
void or_mic0_apply(const or_grid *g, const double *prec, const double *r, double *z)
{
    long n = ncells(g);
    double *y = (double *)calloc((size_t)n, sizeof(double));
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long ci = cidx(g, i, j, k);
                if (g->type[ci] != LIQUID) continue;
                double t = r[ci];
                int lo[3][3] = {{i - 1, j, k}, {i, j - 1, k}, {i, j, k - 1}};
                for (int a = 0; a < 3; a++) {
                    int *m = lo[a];
                    if (cell_type(g, m[0], m[1], m[2]) != LIQUID) continue;
                    long mi = cidx(g, m[0], m[1], m[2]);
                    t -= poisson_off(g, m[0], m[1], m[2], a) * prec[mi] * y[mi];
                }
                y[ci] = t * prec[ci];
            }
    for (long t = 0; t < n; t++) z[t] = 0.0;
    for (int k = g->nz - 1; k >= 0; k--)
        for (int j = g->ny - 1; j >= 0; j--)
            for (int i = g->nx - 1; i >= 0; i--) {
                long ci = cidx(g, i, j, k);
                if (g->type[ci] != LIQUID) continue;
                double t = y[ci];
                int hi[3][3] = {{i + 1, j, k}, {i, j + 1, k}, {i, j, k + 1}};
                for (int a = 0; a < 3; a++) {
                    int *m = hi[a];
                    if (cell_type(g, m[0], m[1], m[2]) != LIQUID) continue;
                    t -= poisson_off(g, i, j, k, a) * prec[ci] * z[cidx(g, m[0], m[1], m[2])];
                }
                z[ci] = t * prec[ci];
            }
    free(y);
}

/* Preconditioned CG for the pressure operator from x = 0 (the null-space mean
 * of b is removed first when the operator is singular). Stops at
 * |r|/|b| <= tol_p or after maxit_p iterations. */
void or_pcg(const or_grid *g, const double *b_in, double *x, int precond, or_stats *st)
{
    long n = ncells(g);
    double *b = (double *)malloc((size_t)n * sizeof(double));
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double *p = (double *)calloc((size_t)n, sizeof(double));
    double *q = (double *)calloc((size_t)n, sizeof(double));
    double *prec = NULL;
    memcpy(b, b_in, (size_t)n * sizeof(double));
    for (long t = 0; t < n; t++) if (g->type[t] != LIQUID) b[t] = 0.0;
    int singular = or_is_singular(g);
    if (singular) remove_liquid_mean(g, b);
    if (precond == PC_MIC0) {
        prec = (double *)calloc((size_t)n, sizeof(double));
        or_mic0_factor(g, g->mic_tau, g->mic_sigma, prec);
    }
    for (long t = 0; t < n; t++) x[t] = 0.0;
    memcpy(r, b, (size_t)n * sizeof(double));
    double bb = dot(b, b, n), rr = bb;
    st->iters = 0;
    st->status = ST_OK;
    st->relres = 0.0;
    st->true_relres = 0.0;
    if (bb > 0.0) {
#define APPLY_PREC()                                                                    \
    do {                                                                                \
        if (precond == PC_MIC0) or_mic0_apply(g, prec, r, z);                           \
        else if (precond == PC_JACOBI) {                                                \
            for (int kk = 0; kk < g->nz; kk++)                                          \
                for (int jj = 0; jj < g->ny; jj++)                                      \
                    for (int ii = 0; ii < g->nx; ii++) {                                \
                        long cc = cidx(g, ii, jj, kk);                                  \
                        int dg = poisson_diag(g, ii, jj, kk);                   \
                        z[cc] = (g->type[cc] == LIQUID && dg > 0) ? r[cc] / dg : 0.0; \
                    }                                                                   \
        } else memcpy(z, r, (size_t)n * sizeof(double));                                \
    } while (0)
        APPLY_PREC();
        memcpy(p, z, (size_t)n * sizeof(double));
        double rz = dot(r, z, n);
        int it;
        for (it = 1; it <= g->maxit_p; it++) {
            or_poisson_apply(g, p, q);
            double pq = dot(p, q, n);
            if (!(pq > 0.0)) { st->status = ST_BREAKDOWN; break; }
            double alpha = rz / pq;
            for (long t = 0; t < n; t++) { x[t] += alpha * p[t]; r[t] -= alpha * q[t]; }
            rr = dot(r, r, n);
            st->iters = it;
            if (sqrt(rr / bb) <= g->tol_p) break;
            APPLY_PREC();
            double rz_new = dot(r, z, n);
            double beta = rz_new / rz;
            rz = rz_new;
            for (long t = 0; t < n; t++) p[t] = z[t] + beta * p[t];
        }
#undef APPLY_PREC
        if (it > g->maxit_p) st->status = ST_NOCONV;
        st->relres = sqrt(rr / bb);
        if (singular) remove_liquid_mean(g, x);
        or_poisson_apply(g, x, q);
        double tr = 0.0;
        for (long t = 0; t < n; t++) { double e = b[t] - q[t]; tr += e * e; }
        st->true_relres = sqrt(tr / bb);
    }
    free(b); free(r); free(z); free(p); free(q); free(prec);
}

/* Project u in place onto the discretely divergence-free fields: b = div RHS,
 * solve for q, subtract the pressure gradient. q_out (nullable) receives q. */
void or_percnn_solve(const or_grid *g, const double *W, int K, const double *b, double *p, or_stats *st);

void or_project(const or_grid *g, double *const u[3], double *q_out, or_stats *st)
{
    long n = ncells(g);
    double *b = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)calloc((size_t)n, sizeof(double));
    or_divergence(g, (const double *const *)u, b);
    if (g->percnn_k > 0 && g->percnn_w)
        or_percnn_solve(g, g->percnn_w, g->percnn_k, b, q, st);
    else
        or_pcg(g, b, q, g->precond, st);
    or_grad_subtract(g, q, u);
    if (q_out) memcpy(q_out, q, (size_t)n * sizeof(double));
    free(b);
    free(q);
}

/* ------------------------------------------------------------------------ */
/* the step and its adjoint                                                  */
/* ------------------------------------------------------------------------ */

static void alloc3(const or_grid *g, double *a[3])
{
    for (int c = 0; c < 3; c++) a[c] = (double *)calloc((size_t)nfaces(g, c), sizeof(double));
}

static void free3(double *a[3])
{
    for (int c = 0; c < 3; c++) free(a[c]);
}

/* One step: advect (+ body force, fixed faces), implicit viscosity, projection.
 * u_visc (nullable) receives the field after viscosity. st[0] viscosity, st[1]
 * pressure. */
void or_step(const or_grid *g, const double *const u_in[3], double *const u_out[3],
             double *const *u_visc, or_stats *st)
{
    double *ua[3];
    alloc3(g, ua);
    or_advect(g, u_in, ua);
    or_visc_solve(g, (const double *const *)ua, u_out, &st[0]);
    free3(ua);
    if (u_visc)
        for (int c = 0; c < 3; c++) memcpy(u_visc[c], u_out[c], (size_t)nfaces(g, c) * sizeof(double));
    or_project(g, u_out, NULL, &st[1]);
}

/* Reverse of one step. Given the input field u_in and the cotangent g_out of the
 * step's output, write the cotangent g_in of the input and add dL/dnu to *g_nu.
 *   projection:  P is an orthogonal projector on the fluid faces, so the
 *                cotangent is projected by the same operator (fixed and air
 *                faces of the output are constants: their cotangent is dropped);
 *   viscosity:   (I + nu dt L_f) is symmetric: one more solve; with
 *                A(nu) u_v = u_b + Dirichlet(nu), dL/dnu = -dt <gb, L~ u_v>;
 *   advection:   the exact discrete adjoint of the trilinear back-trace. */
void or_adjoint_step(const or_grid *g, const double *const u_in[3], const double *const g_out[3],
                     double *const g_in[3], double *g_nu, or_stats *st)
{
    double *ua[3], *uv[3], *gv[3], *gb[3], *lu[3];
    alloc3(g, ua); alloc3(g, uv); alloc3(g, gv); alloc3(g, gb); alloc3(g, lu);
    or_advect(g, u_in, ua);
    or_visc_solve(g, (const double *const *)ua, uv, &st[0]);
    /* projection adjoint */
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    gv[c][f] = face_class(g, c, i, j, k) == FC_FLUID ? g_out[c][f] : 0.0;
                }
    }
    or_project(g, gv, NULL, &st[1]);
    /* viscosity adjoint (no Dirichlet values: the cotangent of a fixed face is 0) */
    visc_solve_impl(g, (const double *const *)gv, gb, 0, &st[2]);
    visc_laplacian_full(g, (const double *const *)uv, lu);
    double s = 0.0;
    for (int c = 0; c < 3; c++) s += dot(gb[c], lu[c], nfaces(g, c));
    *g_nu += -g->dt * s;
    /* advection adjoint (body force is an additive constant) */
    for (int c = 0; c < 3; c++) memset(g_in[c], 0, (size_t)nfaces(g, c) * sizeof(double));
    if (g->advect_grad == 1)
        or_advect_adjoint_upwind(g, u_in, (const double *const *)gb, g_in);
    else
        or_advect_adjoint(g, u_in, (const double *const *)gb, g_in);
    free3(ua); free3(uv); free3(gv); free3(gb); free3(lu);
}

/* ------------------------------------------------------------------------ */
/* a7: loss of Eq. (eq::optLoss) and its gradient                             */
/* ------------------------------------------------------------------------ */

/* Band cells: kind 0 (surface) = liquid cells with at least one air neighbour;
 * kind 1 (occupied) = all liquid cells. */
void or_band_cells(const or_grid *g, int kind, uint8_t *band)
{
    static const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long ci = cidx(g, i, j, k);
                band[ci] = 0;
                if (g->type[ci] != LIQUID) continue;
                if (kind == 1) { band[ci] = 1; continue; }
                for (int m = 0; m < 6; m++)
                    if (cell_type(g, i + off[m][0], j + off[m][1], k + off[m][2]) == AIR) { band[ci] = 1; break; }
            }
}

/* L = beta/(2|B|) sum_{f in B} (u_f - t_f)^2 + alpha/|Bc| sum_{c in Bc} (1 - cos(ubar_c, tbar_c))
 * B = fluid faces with a band cell on either side; Bc = band cells; ubar = mean of a
 * cell's two faces per component; cos(a,b) = a.b / (sqrt(|a|^2+eps^2) sqrt(|b|^2+eps^2)).
 * Adds L to *loss and dL/du to grad. */
void or_loss_grad(const or_grid *g, const double *const u[3], const double *const tgt[3],
                  int kind, double alpha, double beta, double *loss, double *const grad[3])
{
    const double eps = 1e-8;
    long nc = ncells(g);
    uint8_t *band = (uint8_t *)malloc((size_t)nc);
    or_band_cells(g, kind, band);
    long nb_cells = 0, nb_faces = 0;
    for (long t = 0; t < nc; t++) nb_cells += band[t];
    /* count band faces */
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                    int L[3] = {i, j, k};
                    L[c] -= 1;
                    int inb = (cell_type(g, i, j, k) == LIQUID && band[cidx(g, i, j, k)]) ||
                              (cell_type(g, L[0], L[1], L[2]) == LIQUID && band[cidx(g, L[0], L[1], L[2])]);
                    nb_faces += inb;
                }
    }
    double l2 = 0.0, lcos = 0.0;
    if (nb_faces > 0 && beta != 0.0) {
        for (int c = 0; c < 3; c++) {
            int d[3];
            face_dims(g, c, d);
            for (int k = 0; k < d[2]; k++)
                for (int j = 0; j < d[1]; j++)
                    for (int i = 0; i < d[0]; i++) {
                        if (face_class(g, c, i, j, k) != FC_FLUID) continue;
                        int L[3] = {i, j, k};
                        L[c] -= 1;
                        int inb = (cell_type(g, i, j, k) == LIQUID && band[cidx(g, i, j, k)]) ||
                                  (cell_type(g, L[0], L[1], L[2]) == LIQUID && band[cidx(g, L[0], L[1], L[2])]);
                        if (!inb) continue;
                        long f = fidx(d, i, j, k);
                        double e = u[c][f] - tgt[c][f];
                        l2 += 0.5 * e * e;
                        grad[c][f] += beta * e / (double)nb_faces;
                    }
        }
        l2 *= beta / (double)nb_faces;
    }
    if (nb_cells > 0 && alpha != 0.0) {
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    long ci = cidx(g, i, j, k);
                    if (!band[ci]) continue;
                    double a[3], b[3];
                    long lo[3], hi[3];
                    for (int c = 0; c < 3; c++) {
                        int d[3];
                        face_dims(g, c, d);
                        int h[3] = {i, j, k};
                        h[c] += 1;
                        lo[c] = fidx(d, i, j, k);
                        hi[c] = fidx(d, h[0], h[1], h[2]);
                        a[c] = 0.5 * (u[c][lo[c]] + u[c][hi[c]]);
                        b[c] = 0.5 * (tgt[c][lo[c]] + tgt[c][hi[c]]);
                    }
                    double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
                    double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + eps * eps);
                    double nbv = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + eps * eps);
                    double cs = ab / (na * nbv);
                    lcos += 1.0 - cs;
                    for (int c = 0; c < 3; c++) {
                        double dcos = b[c] / (na * nbv) - ab * a[c] / (na * na * na * nbv);
                        double gcell = -alpha * dcos / (double)nb_cells;
                        grad[c][lo[c]] += 0.5 * gcell;
                        grad[c][hi[c]] += 0.5 * gcell;
                    }
                }
        lcos *= alpha / (double)nb_cells;
    }
    *loss += l2 + lcos;
    free(band);
}

/* ------------------------------------------------------------------------ */
/* a12/a13: the convolutional preconditioner network (Sec. 3.4.1)            */
/* ------------------------------------------------------------------------ */

/* Five 3x3x3 convolutions, channels 2 -> 16 -> 16 -> 16 -> 16 -> 1, zero
 * padding, ReLU after the first four. Weights W_l are [co][ci][3][3][3]
 * (values already rounded to bf16 by the caller), biases FP64. Inputs: channel 0
 * = r / s on liquid cells (s = max |r| over liquid cells), channel 1 = cell type
 * code (liquid 1, air 0, solid -1). Activations are rounded to bf16 after each
 * hidden layer, as the GPU stores them. Output z = s * y on liquid cells. */
#define NET_LAYERS 5
static const int net_ch[NET_LAYERS + 1] = {2, 16, 16, 16, 16, 1};

double or_bf16_round(double v)
{
    float f = (float)v;
    uint32_t bits;
    memcpy(&bits, &f, 4);
    if ((bits & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan */
    uint32_t lsb = (bits >> 16) & 1u;
    bits += 0x7fffu + lsb;
    bits &= 0xffff0000u;
    memcpy(&f, &bits, 4);
    return (double)f;
}

static void conv3d(const or_grid *g, const double *in, int ci_n, const double *W, const double *B,
                   int co_n, double *out)
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    long n = ncells(g);
    for (int co = 0; co < co_n; co++)
        for (int k = 0; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    double acc = B[co];
                    for (int ci = 0; ci < ci_n; ci++)
                        for (int dz = -1; dz <= 1; dz++)
                            for (int dy = -1; dy <= 1; dy++)
                                for (int dxo = -1; dxo <= 1; dxo++) {
                                    int a = i + dxo, b = j + dy, c = k + dz;
                                    if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                                    double wv = W[(((long)co * ci_n + ci) * 3 + (dz + 1)) * 9 + (dy + 1) * 3 + (dxo + 1)];
                                    acc += wv * in[(long)ci * n + cidx(g, a, b, c)];
                                }
                    out[(long)co * n + cidx(g, i, j, k)] = acc;
                }
}

/* acts (nullable) receives the stored (post-ReLU, bf16-rounded) input of each
 * layer: layer l's input at acts + offset_l, offsets sum(ch[m] * n, m < l). The
 * last slot holds the raw network output y (before scaling by s). Returns s. */
double or_net_forward(const or_grid *g, const double *const W[NET_LAYERS],
                      const double *const B[NET_LAYERS], const double *r, double *z, double *acts)
{
    long n = ncells(g);
    double s = 0.0;
    for (long t = 0; t < n; t++)
        if (g->type[t] == LIQUID && fabs(r[t]) > s) s = fabs(r[t]);
    double *cur = (double *)calloc((size_t)n * 16, sizeof(double));
    double *nxt = (double *)calloc((size_t)n * 16, sizeof(double));
    for (long t = 0; t < n; t++) {
        double x0 = (g->type[t] == LIQUID && s > 0.0) ? r[t] / s : 0.0;
        cur[t] = or_bf16_round(x0);
        cur[n + t] = g->type[t] == LIQUID ? 1.0 : (g->type[t] == SOLID ? -1.0 : 0.0);
    }
    long off = 0;
    for (int l = 0; l < NET_LAYERS; l++) {
        if (acts) memcpy(acts + off, cur, (size_t)net_ch[l] * n * sizeof(double));
        off += (long)net_ch[l] * n;
        conv3d(g, cur, net_ch[l], W[l], B[l], net_ch[l + 1], nxt);
        if (l < NET_LAYERS - 1)
            for (long t = 0; t < (long)net_ch[l + 1] * n; t++)
                nxt[t] = or_bf16_round(nxt[t] > 0.0 ? nxt[t] : 0.0);
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (acts) memcpy(acts + off, cur, (size_t)n * sizeof(double));
    for (long t = 0; t < n; t++) z[t] = (g->type[t] == LIQUID) ? s * cur[t] : 0.0;
    free(cur);
    free(nxt);
    return s;
}

/* Training loss for one (b, q) pair with A q = b (A the pressure operator):
 *   s = max |b| over liquid;  y = Net(b / s);  e = y - q/s on liquid cells;
 *   loss = e^T A e / ((q/s)^T A (q/s)),
 * the relative error of the predicted pressure in the energy norm of the
 * discrete Laplacian (Sec. 3.4.1: the fitted network should give the pressure of
 * the second-order Laplacian scheme). dloss/dy = 2 A e / ((q/s)^T A (q/s)).
 * Returns the loss and ADDS its gradient to gW, gB (same layouts as W, B). */
double or_net_loss_grad(const or_grid *g, const double *const W[NET_LAYERS],
                        const double *const B[NET_LAYERS], const double *b, const double *q,
                        double *const gW[NET_LAYERS], double *const gB[NET_LAYERS])
{
    long n = ncells(g);
    long tot = 0;
    for (int l = 0; l <= NET_LAYERS; l++) tot += (long)net_ch[l] * n;
    double *acts = (double *)calloc((size_t)tot, sizeof(double));
    double *z = (double *)calloc((size_t)n, sizeof(double));
    double s = or_net_forward(g, W, B, b, z, acts);
    if (s == 0.0) { free(acts); free(z); return 0.0; }
    long offs[NET_LAYERS + 1];
    offs[0] = 0;
    for (int l = 1; l <= NET_LAYERS; l++) offs[l] = offs[l - 1] + (long)net_ch[l - 1] * n;
    const double *y = acts + offs[NET_LAYERS];
    double *ev = (double *)calloc((size_t)n, sizeof(double));
    double *tq = (double *)calloc((size_t)n, sizeof(double));
    double *Aev = (double *)calloc((size_t)n, sizeof(double));
    double *Atq = (double *)calloc((size_t)n, sizeof(double));
    for (long t = 0; t < n; t++)
        if (g->type[t] == LIQUID) {
            tq[t] = q[t] / s;
            ev[t] = y[t] - tq[t];
        }
    or_poisson_apply(g, ev, Aev);
    or_poisson_apply(g, tq, Atq);
    double den = dot(tq, Atq, n), num = dot(ev, Aev, n);
    double *gy = (double *)calloc((size_t)n * 16, sizeof(double));
    double *gx = (double *)calloc((size_t)n * 16, sizeof(double));
    for (long t = 0; t < n; t++)
        if (g->type[t] == LIQUID) gy[t] = 2.0 * Aev[t] / den;
    free(ev); free(tq); free(Aev); free(Atq);
    int nx = g->nx, ny = g->ny, nz = g->nz;
    for (int l = NET_LAYERS - 1; l >= 0; l--) {
        int ci_n = net_ch[l], co_n = net_ch[l + 1];
        const double *in = acts + offs[l];
        /* ReLU mask on this layer's output (all but the last layer) */
        if (l < NET_LAYERS - 1) {
            const double *outv = acts + offs[l + 1];
            for (long t = 0; t < (long)co_n * n; t++) if (!(outv[t] > 0.0)) gy[t] = 0.0;
        }
        memset(gx, 0, (size_t)ci_n * n * sizeof(double));
        for (int co = 0; co < co_n; co++)
            for (int k = 0; k < nz; k++)
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        double go = gy[(long)co * n + cidx(g, i, j, k)];
                        if (go == 0.0) continue;
                        gB[l][co] += go;
                        for (int ci = 0; ci < ci_n; ci++)
                            for (int dz = -1; dz <= 1; dz++)
                                for (int dy = -1; dy <= 1; dy++)
                                    for (int dxo = -1; dxo <= 1; dxo++) {
                                        int a = i + dxo, bb = j + dy, c = k + dz;
                                        if (a < 0 || bb < 0 || c < 0 || a >= nx || bb >= ny || c >= nz) continue;
                                        long wi = (((long)co * ci_n + ci) * 3 + (dz + 1)) * 9 + (dy + 1) * 3 + (dxo + 1);
                                        long xi = (long)ci * n + cidx(g, a, bb, c);
                                        gW[l][wi] += go * in[xi];
                                        gx[xi] += go * W[l][wi];
                                    }
                    }
        double *tmp = gy; gy = gx; gx = tmp;
    }
    free(acts); free(z); free(gy); free(gx);
    return num / den;
}

/* ------------------------------------------------------------------------ */
/* volumetric-velocity initialisation (Sec. 3.3.3)                           */
/* ------------------------------------------------------------------------ */

/* Laminar boundary-layer profile of Sec. 3.3.3: |v| / V_inf = 3/2 e - 1/2 e^3 with
 * e = y / delta below the boundary-layer thickness, 1 above it. */
static double wall_factor(double y, double delta)
{
    if (!(delta > 0.0)) return 1.0;
    double e = y / delta;
    if (e >= 1.0) return 1.0;
    if (e <= 0.0) return 0.0;
    return 1.5 * e - 0.5 * e * e * e;
}

/* Surface speed of the column (i, k) of cells, clamped to the grid. */
static double column_speed(const or_grid *g, const double *vinf, int i, int k)
{
    if (i < 0) i = 0;
    if (i >= g->nx) i = g->nx - 1;
    if (k < 0) k = 0;
    if (k >= g->nz) k = g->nz - 1;
    return vinf[(long)k * g->nx + i];
}

/* Base velocity: on every fluid face dir_c * V_inf * wall_factor(y / delta), y the
 * height of the face centre above the floor (y = 0, the riverbed), V_inf the surface
 * speed of the face's cell column (vinf, (nz, nx)); x and z faces between two
 * columns take the mean of both. Fixed faces take their prescribed value, faces
 * between air cells 0. */
void or_wall_profile(const or_grid *g, const double dir[3], const double *vinf, double delta, double *const u[3])
{
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        for (int k = 0; k < d[2]; k++)
            for (int j = 0; j < d[1]; j++)
                for (int i = 0; i < d[0]; i++) {
                    long f = fidx(d, i, j, k);
                    int cls = face_class(g, c, i, j, k);
                    if (cls == FC_FIXED) { u[c][f] = bc_value(g, c, f); continue; }
                    if (cls != FC_FLUID) { u[c][f] = 0.0; continue; }
                    double y = (c == 1 ? (double)j : j + 0.5) * g->dx;
                    double vi;
                    if (c == 0) vi = 0.5 * (column_speed(g, vinf, i - 1, k) + column_speed(g, vinf, i, k));
                    else if (c == 2) vi = 0.5 * (column_speed(g, vinf, i, k - 1) + column_speed(g, vinf, i, k));
                    else vi = column_speed(g, vinf, i, k);
                    u[c][f] = dir[c] * vi * wall_factor(y, delta);
                }
    }
}

/* A face the constrained projection may move: a fluid face that is not held. With
 * hold_surface the faces between a liquid and an air cell (the free surface, which
 * carries the observed surface velocity) are held. */
static int pbd_free(const or_grid *g, int c, int i, int j, int k, int hold_surface)
{
    if (face_class(g, c, i, j, k) != FC_FLUID) return 0;
    if (!hold_surface) return 1;
    int o[3] = {0, 0, 0};
    o[c] = 1;
    int tl = cell_type(g, i - o[0], j - o[1], k - o[2]), tr = cell_type(g, i, j, k);
    return !((tl == LIQUID && tr == AIR) || (tl == AIR && tr == LIQUID));
}

/* Constrained divergence projection (Eq. eq::divProj), Jacobi form: per iteration,
 * for every liquid cell i the constraint C_i = (div u)_i = sum over its six faces of
 * (u_hi - u_lo)/dx, lambda_i = -C_i / (sum over its free faces of (1/dx)^2 + eps);
 * then every free face f moves by sum_i lambda_i dC_i/du_f = (lambda_lo - lambda_hi)/dx,
 * lo and hi the cells on its two sides (lambda = 0 off the liquid). All lambda of an
 * iteration come from the same field. Returns |C|_2 over the liquid after the last
 * iteration. */
double or_pbd_project(const or_grid *g, double *const u[3], int hold_surface, int iters, double eps)
{
    long n = ncells(g);
    double *lam = (double *)calloc((size_t)n, sizeof(double));
    double norm2 = 0.0;
    for (int it = 0; it <= iters; it++) {
        norm2 = 0.0;
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    long ci = cidx(g, i, j, k);
                    lam[ci] = 0.0;
                    if (g->type[ci] != LIQUID) continue;
                    double C = 0.0;
                    int nfree = 0;
                    for (int c = 0; c < 3; c++) {
                        int d[3];
                        face_dims(g, c, d);
                        int hi[3] = {i, j, k};
                        hi[c] += 1;
                        C += (u[c][fidx(d, hi[0], hi[1], hi[2])] - u[c][fidx(d, i, j, k)]) / g->dx;
                        nfree += pbd_free(g, c, i, j, k, hold_surface);
                        nfree += pbd_free(g, c, hi[0], hi[1], hi[2], hold_surface);
                    }
                    norm2 += C * C;
                    lam[ci] = -C / (nfree / (g->dx * g->dx) + eps);
                }
        if (it == iters) break;
        for (int c = 0; c < 3; c++) {
            int d[3];
            face_dims(g, c, d);
            int o[3] = {0, 0, 0};
            o[c] = 1;
            for (int k = 0; k < d[2]; k++)
                for (int j = 0; j < d[1]; j++)
                    for (int i = 0; i < d[0]; i++) {
                        if (!pbd_free(g, c, i, j, k, hold_surface)) continue;
                        int li = i - o[0], lj = j - o[1], lk = k - o[2];
                        double ll = (cell_type(g, li, lj, lk) == LIQUID) ? lam[cidx(g, li, lj, lk)] : 0.0;
                        double lh = (cell_type(g, i, j, k) == LIQUID) ? lam[cidx(g, i, j, k)] : 0.0;
                        u[c][fidx(d, i, j, k)] += (ll - lh) / g->dx;
                    }
        }
    }
    free(lam);
    return sqrt(norm2);
}

/* ------------------------------------------------------------------------ */
/* recurrent convolutional pressure solver (Sec. 3.4.1, PeRCNN)              */
/* ------------------------------------------------------------------------ */

/* z = m (W * r): the 27-tap correlation of r with W (taps [dz][dy][dx], r zero off
 * the liquid and outside the grid), kept on liquid cells (m) only. flip = 1 uses the
 * point-reflected kernel W[26 - t], the transpose of the masked operator. */
static void percnn_conv(const or_grid *g, const double *W, int flip, const double *r, double *z)
{
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long ci = cidx(g, i, j, k);
                if (g->type[ci] != LIQUID) { z[ci] = 0.0; continue; }
                double acc = 0.0;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dxo = -1; dxo <= 1; dxo++) {
                            if (cell_type(g, i + dxo, j + dy, k + dz) != LIQUID) continue;
                            int t = (dz + 1) * 9 + (dy + 1) * 3 + (dxo + 1);
                            acc += W[flip ? 26 - t : t] * r[cidx(g, i + dxo, j + dy, k + dz)];
                        }
                z[ci] = acc;
            }
}

/* The pressure by K recurrent sub-steps (my reading of the PeRCNN layer of Sec.
 * 3.4.1): the physics operator is the scheme's own 7-point L_p with the cell-type
 * boundary conditions, the fitted part a 3x3x3 kernel W acting on the residual:
 *   p_0 = 0,  r_k = b - L_p p_k,  p_{k+1} = p_k + m (W * r_k).
 * Its fixed points solve L_p p = b. For a singular operator the liquid mean of the
 * result is removed. st (nullable) gets K and |b - L_p p_K| / |b|. */
void or_percnn_solve(const or_grid *g, const double *W, int K, const double *b, double *p, or_stats *st)
{
    long n = ncells(g);
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    for (long c = 0; c < n; c++) p[c] = 0.0;
    for (int it = 0; it < K; it++) {
        or_poisson_apply(g, p, r);
        for (long c = 0; c < n; c++) r[c] = (g->type[c] == LIQUID) ? b[c] - r[c] : 0.0;
        percnn_conv(g, W, 0, r, z);
        for (long c = 0; c < n; c++) p[c] += z[c];
    }
    if (or_is_singular(g)) remove_liquid_mean(g, p);
    if (st) {
        or_poisson_apply(g, p, r);
        double rr = 0.0, bb = 0.0;
        for (long c = 0; c < n; c++)
            if (g->type[c] == LIQUID) { rr += (b[c] - r[c]) * (b[c] - r[c]); bb += b[c] * b[c]; }
        st->iters = K;
        st->status = ST_OK;
        st->relres = st->true_relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    free(r);
    free(z);
}

/* Energy-norm fit loss of the recurrent solver on one pair L_p q = b:
 *   e = p_K - q,  loss = e^T L_p e / q^T L_p q,
 * and its gradient w.r.t. the 27 taps (added to dW) by the backward recurrence:
 *   g_K = dloss/dp_K = 2 L_p e / (q^T L_p q);  for k = K-1 .. 0:
 *   dW[t] += sum_i g_{k+1,i} m_i r_k(i + t);   g_k = g_{k+1} - L_p (m W^T * (m g_{k+1})).
 * Stores every residual r_k. Returns the loss. */
double or_percnn_loss_grad(const or_grid *g, const double *W, int K, const double *b, const double *q, double *dW)
{
    long n = ncells(g);
    double *rs = (double *)malloc((size_t)n * (size_t)(K > 0 ? K : 1) * sizeof(double));
    double *p = (double *)calloc((size_t)n, sizeof(double));
    double *t1 = (double *)malloc((size_t)n * sizeof(double));
    double *gk = (double *)malloc((size_t)n * sizeof(double));
    for (int it = 0; it < K; it++) {
        double *r = rs + (size_t)it * n;
        or_poisson_apply(g, p, t1);
        for (long c = 0; c < n; c++) r[c] = (g->type[c] == LIQUID) ? b[c] - t1[c] : 0.0;
        percnn_conv(g, W, 0, r, t1);
        for (long c = 0; c < n; c++) p[c] += t1[c];
    }
    /* loss and its gradient w.r.t. p_K */
    double *e = (double *)malloc((size_t)n * sizeof(double));
    double *Ae = (double *)malloc((size_t)n * sizeof(double));
    for (long c = 0; c < n; c++) e[c] = (g->type[c] == LIQUID) ? p[c] - q[c] : 0.0;
    or_poisson_apply(g, e, Ae);
    or_poisson_apply(g, q, t1);
    double num = 0.0, den = 0.0;
    for (long c = 0; c < n; c++)
        if (g->type[c] == LIQUID) { num += e[c] * Ae[c]; den += q[c] * t1[c]; }
    double loss = den > 0.0 ? num / den : 0.0;
    for (long c = 0; c < n; c++) gk[c] = den > 0.0 ? 2.0 * Ae[c] / den : 0.0;
    for (int it = K - 1; it >= 0; it--) {
        const double *r = rs + (size_t)it * n;
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    long ci = cidx(g, i, j, k);
                    if (g->type[ci] != LIQUID || gk[ci] == 0.0) continue;
                    for (int dz = -1; dz <= 1; dz++)
                        for (int dy = -1; dy <= 1; dy++)
                            for (int dxo = -1; dxo <= 1; dxo++) {
                                if (cell_type(g, i + dxo, j + dy, k + dz) != LIQUID) continue;
                                int t = (dz + 1) * 9 + (dy + 1) * 3 + (dxo + 1);
                                dW[t] += gk[ci] * r[cidx(g, i + dxo, j + dy, k + dz)];
                            }
                }
        percnn_conv(g, W, 1, gk, t1);  /* m W^T * (m g) (gk is zero off the liquid) */
        or_poisson_apply(g, t1, e);
        for (long c = 0; c < n; c++) gk[c] = (g->type[c] == LIQUID) ? gk[c] - e[c] : 0.0;
    }
    free(rs); free(p); free(t1); free(gk); free(e); free(Ae);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* APIC transfers and Gaussian deformation (Sec. 3.2.2, Sec. 3.4.3)          */
/* ------------------------------------------------------------------------ */

/* Quadratic B-spline weights of the 3 nodes base, base+1, base+2 of one axis for a
 * particle at continuous node coordinate s (nodes at integers): base = floor(s - 1/2),
 * f = s - base in [1/2, 3/2). Returns base. */
static int bspline2(double s, double w[3])
{
    int base = (int)floor(s - 0.5);
    double f = s - base;
    w[0] = 0.5 * (1.5 - f) * (1.5 - f);
    w[1] = 0.75 - (f - 1.0) * (f - 1.0);
    w[2] = 0.5 * (f - 0.5) * (f - 0.5);
    return base;
}

/* Continuous node coordinate of position x along `axis` for face component c: the
 * nodes of component c sit at index * dx along axis c and (index + 1/2) * dx along
 * the others. */
static double node_coord(const or_grid *g, int c, int axis, double x)
{
    return x / g->dx - (axis == c ? 0.0 : 0.5);
}

/* P2G (Eq. eq::particle_map) per face component c on the MAC grid:
 *   (m v)_i = sum_p w_ip m_p [v_p,c + (C_p (x_i - x_p))_c],  v_i = (m v)_i / sum_p w_ip m_p,
 * w_ip the product of quadratic B-spline weights, nodes outside the face arrays
 * skipped, v_i = 0 where no particle contributes. x, v: [p][3]; C: [p][3][3]
 * (row c = gradient of component c); m: [p]. mass (nullable) gets sum_p w_ip m_p. */
void or_p2g(const or_grid *g, int np, const double *x, const double *v, const double *C, const double *m,
            double *const u[3], double *const mass[3])
{
    for (int c = 0; c < 3; c++) {
        int d[3];
        face_dims(g, c, d);
        long nf = (long)d[0] * d[1] * d[2];
        double *mv = (double *)calloc((size_t)nf, sizeof(double));
        double *ms = (double *)calloc((size_t)nf, sizeof(double));
        for (int p = 0; p < np; p++) {
            double w[3][3];
            int base[3];
            for (int a = 0; a < 3; a++) base[a] = bspline2(node_coord(g, c, a, x[3 * p + a]), w[a]);
            for (int kz = 0; kz < 3; kz++)
                for (int ky = 0; ky < 3; ky++)
                    for (int kx = 0; kx < 3; kx++) {
                        int i = base[0] + kx, j = base[1] + ky, k = base[2] + kz;
                        if (i < 0 || j < 0 || k < 0 || i >= d[0] || j >= d[1] || k >= d[2]) continue;
                        double wt = w[0][kx] * w[1][ky] * w[2][kz] * m[p];
                        double xi[3] = {(i + (c == 0 ? 0.0 : 0.5)) * g->dx, (j + (c == 1 ? 0.0 : 0.5)) * g->dx,
                                        (k + (c == 2 ? 0.0 : 0.5)) * g->dx};
                        double aff = 0.0;
                        for (int a = 0; a < 3; a++) aff += C[9 * p + 3 * c + a] * (xi[a] - x[3 * p + a]);
                        long f = fidx(d, i, j, k);
                        mv[f] += wt * (v[3 * p + c] + aff);
                        ms[f] += wt;
                    }
        }
        for (long f = 0; f < nf; f++) {
            u[c][f] = ms[f] > 0.0 ? mv[f] / ms[f] : 0.0;
            if (mass && mass[c]) mass[c][f] = ms[f];
        }
        free(mv);
        free(ms);
    }
}

/* G2P and the particle update (Sec. 3.2.2, Sec. 3.4.3), per particle:
 *   v_p,c = sum_i w_ip u_c,i ;  C_p[c][a] = 4/dx^2 sum_i w_ip u_c,i (x_i - x_p)_a
 * (nodes outside the face arrays contribute nothing), then when `advance`:
 *   x_p += dt v_p (clamped to [lo, hi] per axis),  F_p = (I + dt C_p) F_p,
 *   A_p = F_p A0_p F_p^T  (F, A0, A nullable; [p][3][3]). */
void or_g2p(const or_grid *g, int np, double *x, double *v, double *C, double *F, const double *A0, double *A,
            const double *const u[3], double dt, int advance, double lo, double hi)
{
    for (int p = 0; p < np; p++) {
        double xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
        for (int c = 0; c < 3; c++) {
            int d[3];
            face_dims(g, c, d);
            double w[3][3];
            int base[3];
            for (int a = 0; a < 3; a++) base[a] = bspline2(node_coord(g, c, a, xp[a]), w[a]);
            double vc = 0.0, cc[3] = {0.0, 0.0, 0.0};
            for (int kz = 0; kz < 3; kz++)
                for (int ky = 0; ky < 3; ky++)
                    for (int kx = 0; kx < 3; kx++) {
                        int i = base[0] + kx, j = base[1] + ky, k = base[2] + kz;
                        if (i < 0 || j < 0 || k < 0 || i >= d[0] || j >= d[1] || k >= d[2]) continue;
                        double wt = w[0][kx] * w[1][ky] * w[2][kz];
                        double uv = u[c][fidx(d, i, j, k)];
                        double xi[3] = {(i + (c == 0 ? 0.0 : 0.5)) * g->dx, (j + (c == 1 ? 0.0 : 0.5)) * g->dx,
                                        (k + (c == 2 ? 0.0 : 0.5)) * g->dx};
                        vc += wt * uv;
                        for (int a = 0; a < 3; a++) cc[a] += wt * uv * (xi[a] - xp[a]);
                    }
            v[3 * p + c] = vc;
            for (int a = 0; a < 3; a++) C[9 * p + 3 * c + a] = 4.0 / (g->dx * g->dx) * cc[a];
        }
        if (!advance) continue;
        for (int a = 0; a < 3; a++) {
            double nx = xp[a] + dt * v[3 * p + a];
            x[3 * p + a] = nx < lo ? lo : (nx > hi ? hi : nx);
        }
        if (F) {
            double Fn[9];
            for (int r = 0; r < 3; r++)
                for (int s = 0; s < 3; s++) {
                    double acc = F[9 * p + 3 * r + s];
                    for (int t = 0; t < 3; t++) acc += dt * C[9 * p + 3 * r + t] * F[9 * p + 3 * t + s];
                    Fn[3 * r + s] = acc;
                }
            memcpy(F + 9 * p, Fn, sizeof(Fn));
            if (A0 && A) {
                double T[9];
                for (int r = 0; r < 3; r++)
                    for (int s = 0; s < 3; s++) {
                        double acc = 0.0;
                        for (int t = 0; t < 3; t++) acc += Fn[3 * r + t] * A0[9 * p + 3 * t + s];
                        T[3 * r + s] = acc;
                    }
                for (int r = 0; r < 3; r++)
                    for (int s = 0; s < 3; s++) {
                        double acc = 0.0;
                        for (int t = 0; t < 3; t++) acc += T[3 * r + t] * Fn[3 * s + t];
                        A[9 * p + 3 * r + s] = acc;
                    }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Gaussian splatting forward rendering (Sec. 3.2.1, Sec. 3.5)               */
/* ------------------------------------------------------------------------ */

typedef struct {
    double R[9], t[3];          /* world -> camera: x_c = R x + t */
    double fx, fy, cx, cy;      /* pinhole intrinsics (pixels) */
    int width, height;
    double znear;
    double bg[3];
} or_camera;

/* Projection of one Gaussian: camera-space depth, pixel-space mean and the inverse
 * of the 2D covariance J R A R^T J^T (J the Jacobian of the pinhole projection at
 * the mean). Returns 0 when the Gaussian is culled (behind znear, degenerate). */
static int splat_project(const or_camera *cam, const double x[3], const double A[9], double *depth,
                         double mean[2], double conic[3])
{
    double xc[3];
    for (int r = 0; r < 3; r++) xc[r] = cam->R[3 * r] * x[0] + cam->R[3 * r + 1] * x[1] + cam->R[3 * r + 2] * x[2] + cam->t[r];
    if (!(xc[2] > cam->znear)) return 0;
    double z = xc[2];
    mean[0] = cam->fx * xc[0] / z + cam->cx;
    mean[1] = cam->fy * xc[1] / z + cam->cy;
    double J[6] = {cam->fx / z, 0.0, -cam->fx * xc[0] / (z * z), 0.0, cam->fy / z, -cam->fy * xc[1] / (z * z)};
    double M[6]; /* J R */
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            M[3 * r + c] = J[3 * r] * cam->R[c] + J[3 * r + 1] * cam->R[3 + c] + J[3 * r + 2] * cam->R[6 + c];
    double S[4] = {0, 0, 0, 0};
    for (int r = 0; r < 2; r++)
        for (int s = 0; s < 2; s++) {
            double acc = 0.0;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) acc += M[3 * r + a] * A[3 * a + b] * M[3 * s + b];
            S[2 * r + s] = acc;
        }
    double det = S[0] * S[3] - S[1] * S[2];
    if (!(det > 0.0)) return 0;
    conic[0] = S[3] / det;
    conic[1] = -S[1] / det;
    conic[2] = S[0] / det;
    *depth = z;
    return 1;
}

typedef struct {
    double depth;
    int idx;
} splat_key;

static int splat_key_cmp(const void *a, const void *b)
{
    const splat_key *p = (const splat_key *)a, *q = (const splat_key *)b;
    if (p->depth < q->depth) return -1;
    if (p->depth > q->depth) return 1;
    return p->idx - q->idx;
}

/* Front-to-back compositing of the splatting formula of Sec. 3.2.1 at every pixel
 * centre (px + 1/2, py + 1/2):  C = sum_i alpha_i c_i prod_{j<i} (1 - alpha_j) + T bg,
 * over the Gaussians in increasing depth (ties by index), with
 * alpha_i = min(0.99, sigma_i exp(-d^T Sigma_i^-1 d / 2)), d the offset of the pixel
 * centre from the projected mean, kept only inside the 3-sigma ellipse
 * (d^T Sigma^-1 d <= 9) and when alpha >= 1/255; the walk stops once the
 * transmittance T would fall below 1e-4. Colours are degree-0 spherical harmonics
 * (RGB). x [n][3], opacity [n], A [n][3][3], color [n][3]; rgb [h][w][3], T [h][w]. */
/* View-dependent colour (Sec. 3.2.1: the compositing sum weights SH(r; F_i), the
 * spherical-harmonic colour of Gaussian i seen along the viewing ray r). The
 * real spherical harmonics of degree <= 3 at the unit direction d = (x, y, z),
 * normalised over the sphere (the integral of Y_j^2 is 1), indexed j = l^2 +
 * l + m, with the signs of the standard 3DGS evaluator (so that coefficients
 * made for it render alike):
 *   l = 0: 1/(2 sqrt(pi))
 *   l = 1: -a y, a z, -a x                                        a = sqrt(3/(4 pi))
 *   l = 2: b xy, -b yz, c (2zz - xx - yy), -b xz, e (xx - yy)    b = sqrt(15/(4 pi)),
 *          c = sqrt(5/(16 pi)), e = sqrt(15/(16 pi))
 *   l = 3: -f y (3xx - yy), g xyz, -h y (4zz - xx - yy), k z (2zz - 3xx - 3yy),
 *          -h x (4zz - xx - yy), (g/2) z (xx - yy), -f x (xx - 3yy)
 *          f = sqrt(35/(32 pi)), g = sqrt(105/(4 pi)), h = sqrt(21/(32 pi)),
 *          k = sqrt(7/(16 pi)) */
void or_sh_basis(int degree, const double d[3], double *Y)
{
    const double PI = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    Y[0] = 0.5 / sqrt(PI);
    if (degree < 1) return;
    const double a = sqrt(3.0 / (4.0 * PI));
    Y[1] = -a * y;
    Y[2] = a * z;
    Y[3] = -a * x;
    if (degree < 2) return;
    const double b = sqrt(15.0 / (4.0 * PI)), c = sqrt(5.0 / (16.0 * PI)), e = sqrt(15.0 / (16.0 * PI));
    Y[4] = b * x * y;
    Y[5] = -b * y * z;
    Y[6] = c * (2.0 * z * z - x * x - y * y);
    Y[7] = -b * x * z;
    Y[8] = e * (x * x - y * y);
    if (degree < 3) return;
    const double f = sqrt(35.0 / (32.0 * PI)), g = sqrt(105.0 / (4.0 * PI)), h = sqrt(21.0 / (32.0 * PI)),
                 k = sqrt(7.0 / (16.0 * PI));
    Y[9] = -f * y * (3.0 * x * x - y * y);
    Y[10] = g * x * y * z;
    Y[11] = -h * y * (4.0 * z * z - x * x - y * y);
    Y[12] = k * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -h * x * (4.0 * z * z - x * x - y * y);
    Y[14] = 0.5 * g * z * (x * x - y * y);
    Y[15] = -f * x * (x * x - 3.0 * y * y);
}

/* The colour of one Gaussian: max(0, 1/2 + sum_j sh[j][k] Y_j(d)) per channel k,
 * with d the unit vector from the camera centre (-R^T t) to the mean (the 1/2
 * offset of the standard evaluator: zero coefficients give mid grey). */
static void sh_colour(int degree, const or_camera *cam, const double xm[3], const double *sh, double out[3])
{
    double C[3], d[3], Y[16], nrm = 0.0;
    for (int r = 0; r < 3; r++) C[r] = -(cam->R[r] * cam->t[0] + cam->R[3 + r] * cam->t[1] + cam->R[6 + r] * cam->t[2]);
    for (int r = 0; r < 3; r++) {
        d[r] = xm[r] - C[r];
        nrm += d[r] * d[r];
    }
    nrm = sqrt(nrm);
    for (int r = 0; r < 3; r++) d[r] = nrm > 0.0 ? d[r] / nrm : 0.0;
    or_sh_basis(degree, d, Y);
    const int nb = (degree + 1) * (degree + 1);
    for (int k = 0; k < 3; k++) {
        double v = 0.5;
        for (int j = 0; j < nb; j++) v += sh[3 * j + k] * Y[j];
        out[k] = v > 0.0 ? v : 0.0;
    }
}

/* Front-to-back compositing as below; with `near` non-NULL, near[pixel] = 1 when
 * the pixel's value turns on a decision that an evaluation in single precision
 * could take the other way, by enough to show: a Gaussian whose md lies within
 * rel of the 3-sigma cutoff 9, or whose alpha lies within rel of 1/255, while
 * its contribution at the threshold times the transmittance exceeds 2e-5; a
 * transmittance within rel of the 1e-4 floor; or two contributing Gaussians whose
 * depths differ (but are not equal) by less than 4e-6 of the depth, a few
 * single-precision roundings. The flags change no value. */
static void splat_render_impl(int n, const double *x, const double *opacity, const double *A, const double *color,
                              const or_camera *cam, double *rgb, double *T_out, unsigned char *near, double rel);

void or_splat_render(int n, const double *x, const double *opacity, const double *A, const double *color,
                     const or_camera *cam, double *rgb, double *T_out)
{
    splat_render_impl(n, x, opacity, A, color, cam, rgb, T_out, NULL, 0.0);
}

void or_splat_render_flags(int n, const double *x, const double *opacity, const double *A, const double *color,
                           const or_camera *cam, double *rgb, double *T_out, unsigned char *near, double rel)
{
    splat_render_impl(n, x, opacity, A, color, cam, rgb, T_out, near, rel);
}

/* The same compositing with the view-dependent colour of each Gaussian from its
 * spherical-harmonic coefficients sh [n][(degree + 1)^2][3] (degree 0 .. 3). */
void or_splat_render_sh(int n, const double *x, const double *opacity, const double *A, const double *sh,
                        int degree, const or_camera *cam, double *rgb, double *T_out, unsigned char *near, double rel)
{
    const int nb = (degree + 1) * (degree + 1);
    double *col = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    for (int i = 0; i < n; i++) sh_colour(degree, cam, x + 3 * i, sh + (size_t)i * nb * 3, col + 3 * i);
    splat_render_impl(n, x, opacity, A, col, cam, rgb, T_out, near, rel);
    free(col);
}

static void splat_render_impl(int n, const double *x, const double *opacity, const double *A, const double *color,
                              const or_camera *cam, double *rgb, double *T_out, unsigned char *near, double rel)
{
    double *depth = (double *)malloc((size_t)n * sizeof(double));
    double *mean = (double *)malloc((size_t)n * 2 * sizeof(double));
    double *conic = (double *)malloc((size_t)n * 3 * sizeof(double));
    int *ok = (int *)malloc((size_t)n * sizeof(int));
    splat_key *keys = (splat_key *)malloc((size_t)(n > 0 ? n : 1) * sizeof(splat_key));
    int m = 0;
    for (int i = 0; i < n; i++) {
        ok[i] = splat_project(cam, x + 3 * i, A + 9 * i, depth + i, mean + 2 * i, conic + 3 * i);
        if (ok[i]) { keys[m].depth = depth[i]; keys[m].idx = i; m++; }
    }
    qsort(keys, (size_t)m, sizeof(splat_key), splat_key_cmp);
    for (int py = 0; py < cam->height; py++)
        for (int px = 0; px < cam->width; px++) {
            double T = 1.0, c[3] = {0.0, 0.0, 0.0};
            double pu = px + 0.5, pv = py + 0.5;
            int flag = 0;
            double last_depth = -1.0;
            for (int q = 0; q < m; q++) {
                int i = keys[q].idx;
                double dx = pu - mean[2 * i], dy = pv - mean[2 * i + 1];
                double md = conic[3 * i] * dx * dx + 2.0 * conic[3 * i + 1] * dx * dy + conic[3 * i + 2] * dy * dy;
                if (near && fabs(md - 9.0) < rel * 9.0) {
                    double a_cut = opacity[i] * exp(-4.5);
                    if ((a_cut > 0.99 ? 0.99 : a_cut) * T > 2e-5) flag = 1;
                }
                if (md > 9.0) continue;
                double alpha = opacity[i] * exp(-0.5 * md);
                if (alpha > 0.99) alpha = 0.99;
                if (near && fabs(alpha * 255.0 - 1.0) < rel && T / 255.0 > 2e-5) flag = 1;
                if (alpha < 1.0 / 255.0) continue;
                double Tn = T * (1.0 - alpha);
                if (near && fabs(Tn * 1e4 - 1.0) < rel) flag = 1;
                if (Tn < 1e-4) break;
                if (near && last_depth >= 0.0 && depth[i] != last_depth && depth[i] - last_depth < 4e-6 * depth[i])
                    flag = 1;
                for (int k = 0; k < 3; k++) c[k] += alpha * T * color[3 * i + k];
                T = Tn;
                last_depth = depth[i];
            }
            long o = (long)py * cam->width + px;
            if (near) near[o] = (unsigned char)flag;
            for (int k = 0; k < 3; k++) rgb[3 * o + k] = c[k] + T * cam->bg[k];
            if (T_out) T_out[o] = T;
        }
    free(depth); free(mean); free(conic); free(ok); free(keys);
}
