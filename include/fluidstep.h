/*
 * fluidstep.h -- C ABI of the differentiable MAC-grid fluid step on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method (arXiv 2503.00868, Sec. 3.4) fits simulation parameters by
 * evolving a grid velocity field through the split incompressible Navier-Stokes
 * equations (Eq. eq::v, Sec. 3.2.2), with grid convection by back-tracing
 * (Sec. 3.4.1), under the masked loss of Eq. eq::optLoss (Sec. 3.4.2). The problem
 * statement there is v_sim^{i+n} = DiffSim^n(v^i; nu, v_in, g, dt, ...): these
 * calls provide one step of DiffSim, its reverse-mode adjoint and the loss.
 *
 * One step (fs_step) is:
 *   1. semi-Lagrangian advection: each fluid face samples its own component
 *      trilinearly at x_f - dt * u(x_f) (other components at the face are the mean
 *      of the 4 surrounding faces); the continuous index is clamped to the array;
 *   2. body force: + dt * g on fluid faces; fixed faces take their prescribed
 *      values, faces between two air cells are zero;
 *   3. implicit viscosity: (I + nu dt L_f) u_v = u_b on the fluid faces, per
 *      component, L_f the 7-point face Laplacian (fluid neighbours coupled, fixed
 *      neighbours Dirichlet, air neighbours and box-wall tangential neighbours
 *      zero-flux), solved by CG preconditioned with Jacobi, or with the multigrid
 *      V-cycle when precond = FS_PRECOND_MG;
 *   4. projection: b = -dx * div(u_v) on liquid cells, L_p q = b (7-point, p = 0
 *      in air, solid walls zero-flux) by PCG, then u -= grad q / dx on fluid faces.
 *      The pressure is p = rho * q / dt.
 *
 * Cell types: FS_AIR, FS_LIQUID, FS_SOLID; every cell outside the grid is solid.
 * A face is FIXED if a solid cell touches it, FLUID if it touches a liquid cell
 * and no solid cell, AIR otherwise.
 *
 * Memory layout. Every field the caller passes is a DEVICE array of floats (or
 * bytes) in the library layout returned by fs_layout(): element (i, j, k) of any
 * cell array or of any face component lives at
 *     (k * rows + j) * pitch + i,     rows = ny + 1, planes = nz + 1,
 * with pitch >= nx + 1 a multiple of 4, and every array holds `nelems` =
 * pitch * rows * planes elements. u-faces use i <= nx, v-faces j <= ny, w-faces
 * k <= nz; u(i,j,k) lies between cells (i-1,j,k) and (i,j,k) (likewise v, w).
 * Entries outside an array's valid range are padding: the library never reads
 * them and writes zeros there in its outputs.
 *
 * Ownership. The caller owns every array it passes and must keep it alive until
 * the call returns. The context owns its scratch (solver vectors, flags, the
 * reduction buffers, pinned read-back memory) and frees it in fs_destroy. The
 * library never frees caller memory and never returns memory to the caller.
 *
 * Streams and synchronisation. All work is enqueued on the context's stream.
 * Calls that run an iterative solve or return a scalar (fs_step, fs_project,
 * fs_adjoint_step, fs_loss_grad, fs_set_mask) read the result back from pinned
 * memory and return after the stream has reached the end of their work. A
 * context must not be used from two host threads at once.
 *
 * Errors. Every call returns an FS_* status. Argument errors (FS_EINVAL) are
 * reported before anything is enqueued. FS_ENOCONV means an iteration cap was
 * reached: the best iterate is still written and the stats are filled.
 * fs_last_error() returns a per-thread message for the last failing call.
 */
#ifndef FLUIDSTEP_H
#define FLUIDSTEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FS_OK = 0,
    FS_EINVAL = 1,      /* bad argument (sizes, null pointer, parameter range) */
    FS_ENOMEM = 2,      /* device or pinned allocation failed at init */
    FS_ECUDA = 3,       /* a CUDA call failed; see fs_last_error() */
    FS_ENOCONV = 4,     /* a solve hit its iteration cap (result still written) */
    FS_ENONFINITE = 5,  /* a non-finite value appeared in a solve */
    FS_ESTATE = 6,      /* call out of order (e.g. no mask set yet) */
    FS_ETIMEOUT = 7,    /* a bounded device-side wait ran out */
    FS_EBREAKDOWN = 8   /* a solve lost positive definiteness (p.Ap <= 0) */
};

enum { FS_AIR = 0, FS_LIQUID = 1, FS_SOLID = 2 };

enum {
    FS_PRECOND_JACOBI = 0,  /* diagonal scaling */
    FS_PRECOND_MIC0 = 1,    /* modified incomplete Cholesky, level 0 */
    FS_PRECOND_LEARNED = 2, /* the convolutional network, in flexible CG */
    FS_PRECOND_MG = 3,      /* geometric multigrid V-cycle (not in the paper: damped-Jacobi
                               smoothing, cell coarsening with air kept, trilinear transfers) */
    FS_PRECOND_LEARNED_MG = 4 /* the network, then one V-cycle on what it leaves:
                                 z = e + M(r - L_p e), e = s Net(r/s); in flexible CG */
};

enum {
    FS_ADVECT_GRAD_EXACT = 0,  /* the exact discrete adjoint of the back-trace */
    FS_ADVECT_GRAD_UPWIND = 1  /* the paper's surrogate (Sec. 3.4.1): -dt dv/de by first-order upwind
                                  differences of the convected field v, the cotangent passed through */
};

enum {
    FS_SOLVER_PCG = 0,      /* preconditioned CG to tol_p (precond selects the preconditioner) */
    FS_SOLVER_PERCNN = 1    /* K recurrent convolutional sub-steps (fs_percnn_load), Sec. 3.4.1 */
};

enum {
    FS_MASK_SURFACE = 0,   /* liquid cells with an air neighbour (the surface band) */
    FS_MASK_OCCUPIED = 1   /* every liquid cell */
};

typedef struct fs_ctx fs_ctx;

/* A MAC velocity field: three caller-owned DEVICE arrays in the library layout. */
typedef struct {
    float *u, *v, *w;
} fs_mac;

typedef struct {
    double dx;         /* cell size, > 0 */
    double dt;         /* time step, >= 0 */
    double nu;         /* kinematic viscosity, >= 0 */
    double rho;        /* density, > 0; only scales the reported pressure */
    double g[3];       /* body acceleration per component */
    int precond;       /* FS_PRECOND_* for the pressure solve; FS_PRECOND_MG and
                          FS_PRECOND_LEARNED_MG also precondition the viscosity solve with
                          the V-cycle (Jacobi otherwise) */
    int maxit_p;       /* pressure iteration cap, >= 1 */
    int maxit_v;       /* viscosity iteration cap, >= 1 */
    double tol_p;      /* pressure relative residual target |r|/|b|, > 0 */
    double tol_v;      /* viscosity relative residual target, > 0 */
    int check_every;   /* iterations between host convergence checks, >= 1 (at most 4 with
                          the multigrid preconditioner). Once a pass of the same kind has
                          run on the context, the first check comes one iteration before
                          that pass's count and later ones every two iterations */
    int spin_limit;    /* cap on every device-side spin-wait (iterations), >= 1 */
    double mic_tau;    /* MIC(0) modification, in [0, 1] */
    double mic_sigma;  /* MIC(0) safety threshold, in [0, 1) */
    int warm_start;    /* 0: every pressure solve starts from q = 0. 1: a forward projection
                          (fs_step, fs_project) starts from the last converged pressure of a
                          forward projection on this context, an adjoint projection
                          (fs_adjoint_step) from the last adjoint one, whenever that gives a
                          smaller initial residual than q = 0; the stopping test is unchanged,
                          so only the iteration count differs. fs_set_mask and
                          fs_set_params reset the kept pressures. */
    int pressure_solver;  /* FS_SOLVER_PCG (default) or FS_SOLVER_PERCNN: the pressure of every
                             projection (fs_step, fs_project, fs_adjoint_step) by the recurrent
                             convolutional solver; its map is symmetric, so the adjoint step
                             applies the same projection to the cotangent */
    int advect_grad;      /* reverse of advection in fs_adjoint_step: FS_ADVECT_GRAD_EXACT (default)
                             or FS_ADVECT_GRAD_UPWIND (the paper's surrogate gradient: each fluid
                             face's cotangent passes through, and each velocity component e seen
                             at the face receives -dt times the cotangent times the upwind
                             difference of the convected field along e, over dx) */
} fs_params;

typedef struct {
    int status;            /* FS_OK, FS_ENOCONV, FS_ENONFINITE or FS_EBREAKDOWN */
    int iters_p;           /* pressure iterations, summed over the call's solves */
    int iters_v;           /* viscosity iterations, summed over the call's solves */
    double relres_p;       /* last pressure solve: recursive |r|/|b| at exit */
    double relres_v;       /* last viscosity solve: recursive |r|/|b| at exit */
    double true_relres_p;  /* last pressure solve: |b - A q|/|b| recomputed at exit to FP64
                              accuracy (b - A q of the FP32 pressure summed from its exact
                              terms by cascaded error-free FP32 sums, the norms in
                              compensated pairs merged in FP64) */
    int fallbacks;         /* pressure solves redone with MIC(0) after the learned one failed */
    int restarts_p;        /* refinement steps of the pressure solves (summed over the call):
                              when the recursive residual meets tol_p but the FP64 residual
                              |b - A q| is above tol_p |b|, CG runs again on the correction
                              system A d = b - A q (right-hand side rounded once from FP64)
                              to tol_p |b| / 2, and the pressure is kept as the pair q + d;
                              at most two per solve. Where the first CG pass of the last
                              solve of the same kind (forward or adjoint) left an FP64
                              residual above tol_p |b|, the next first pass stops at half
                              that relative residual; the context keeps it until the next
                              fs_set_mask */
} fs_stats;

typedef struct {
    int nx, ny, nz;        /* cells */
    int pitch;             /* elements per row, >= nx + 1, multiple of 4 */
    int rows;              /* ny + 1 */
    int planes;            /* nz + 1 */
    long long nelems;      /* pitch * rows * planes: the size of every array */
} fs_layout_t;

/* Default parameters: dx = 1/ny is left to the caller (set to 1), dt = 1/30,
 * nu = 0.01, rho = 1000, g = 0, Jacobi, tolerances 1e-6, caps 20000/2000,
 * check_every 8, spin_limit 1<<22, MIC(0) tau = 0.97, sigma = 0.25, no warm start. */
void fs_default_params(fs_params *p);

/* Create a context for an nx * ny * nz grid (each >= 2) bound to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream) on the current device.
 * Allocates all scratch. Errors: FS_EINVAL for sizes or parameters,
 * FS_ENOMEM, FS_ECUDA. *out is NULL on failure. */
int fs_init_grid(fs_ctx **out, int nx, int ny, int nz, const fs_params *p, void *cuda_stream);

/* Free the context and its scratch (waits for its stream). NULL is a no-op. */
int fs_destroy(fs_ctx *c);

/* The array layout shared by every field of this context. */
int fs_layout(const fs_ctx *c, fs_layout_t *out);

/* Rebind the context to another stream. */
int fs_set_stream(fs_ctx *c, void *cuda_stream);

/* Replace the step parameters (e.g. a new nu during a fit). Same checks as init.
 * Drops the pressures kept for warm starts. */
int fs_set_params(fs_ctx *c, const fs_params *p);

/* Set the grid-type mask (Sec. 3.4.2, "grid types of surface, occupation, or
 * empty"; the liquid cells come from the particle-to-grid transfer of Sec. 3.4.1).
 * cell_type_dense: DEVICE uint8 array of nx*ny*nz values FS_AIR/FS_LIQUID/FS_SOLID
 * in dense C order (index (k*ny + j)*nx + i), read during the call.
 * bc: nullable DEVICE field (library layout) holding the prescribed velocity of
 * each fixed face (e.g. an inflow v_in on wall faces); NULL means all fixed faces
 * are zero. It is copied. Derives face classes, the surface band and whether the
 * pressure operator is singular (liquid touching no air cell: the mean of the
 * right-hand side is then removed). Errors: FS_EINVAL for a type value > 2. */
int fs_set_mask(fs_ctx *c, const uint8_t *cell_type_dense, const fs_mac *bc);

/* One step of the grid velocity evolution (Eq. eq::v split as in Sec. 3.2.2, with
 * back-traced convection of Sec. 3.4.1): u_out = Project(Visc(Advect(u_in) + dt g)).
 * u_in, u_out: DEVICE fields, must not alias. u_visc: nullable DEVICE field that
 * receives the field after viscosity (the input of the projection), which
 * fs_adjoint_step can reuse instead of recomputing it. st: nullable host stats.
 * Returns FS_ENOCONV/FS_ENONFINITE/FS_EBREAKDOWN from the solves. */
int fs_step(fs_ctx *c, const fs_mac *u_in, fs_mac *u_out, fs_mac *u_visc, fs_stats *st);

/* Pressure projection alone (Sec. 3.2.2, Poisson pressure equation), in place on u.
 * q_out: nullable DEVICE cell array (library layout) receiving q, where the
 * pressure is p = rho * q / dt (q is mean-free when the operator is singular).
 * After a refined solve the solver keeps q as a pair of FP32 terms
 * (fs_pressure_pair); q_out is their sum rounded to FP32. */
int fs_project(fs_ctx *c, fs_mac *u, float *q_out, fs_stats *st);

/* The last projection's q as the pair of FP32 terms the solver keeps it in,
 * q = q_hi + q_lo (the paper has no counterpart: a precision detail of this
 * solver). After an iterative refinement (fs_stats.restarts_p > 0) the pair is the
 * first solution and the sum of the corrections, which q_out rounds to one FP32
 * value; otherwise q_lo = 0. fs_stats.true_relres_p is the residual of the pair.
 * q_hi, q_lo: DEVICE cell arrays in the library layout (as q_out of fs_project),
 * must not alias. Before any solve both read zero. FS_EINVAL for a NULL or aliased
 * array, FS_ESTATE before fs_set_mask. */
int fs_pressure_pair(fs_ctx *c, float *q_hi, float *q_lo);

/* Reverse mode of fs_step (derived from the step; Sec. 3.4.2 optimises through
 * it). Given the step input u_in and the cotangent g_out = dL/du_out, writes
 * g_in = dL/du_in (overwritten, every face) and ADDS dL/dnu to *g_nu (host).
 * The adjoint of the projection is the projection itself (an orthogonal
 * projector on the fluid faces), the viscosity solve is self-adjoint, and the
 * advection adjoint is the exact discrete adjoint of the trilinear back-trace
 * (accumulated with atomics, so its summation order is not fixed).
 * u_visc: nullable; the u_visc that fs_step wrote for this u_in (saves one
 * advection and one viscosity solve). g_in must not alias u_in or g_out. */
int fs_adjoint_step(fs_ctx *c, const fs_mac *u_in, const fs_mac *u_visc,
                    const fs_mac *g_out, fs_mac *g_in, double *g_nu, fs_stats *st);

/* The masked loss of Eq. eq::optLoss (Sec. 3.4.2) at one frame:
 *   L = beta/(2|B|) sum_{f in B} (u_f - t_f)^2
 *     + alpha/|Bc| sum_{c in Bc} (1 - cos(ubar_c, tbar_c)),
 * Bc = band cells of `mask_kind` (FS_MASK_SURFACE or FS_MASK_OCCUPIED),
 * B = fluid faces touching a band cell, ubar = cell-centred velocity (mean of the
 * two faces per component), cos(a, b) = a.b / (sqrt(|a|^2+e^2) sqrt(|b|^2+e^2)),
 * e = 1e-8. ADDS L to *loss (host) and, if g is non-NULL, dL/du to g (device). */
int fs_loss_grad(fs_ctx *c, const fs_mac *u, const fs_mac *target, int mask_kind,
                 double alpha, double beta, double *loss, fs_mac *g);

/* The right-hand side of the pressure equation for a field u (Sec. 3.2.2):
 * b = -dx * div(u) on liquid cells (the liquid mean removed when the operator is
 * singular), zero elsewhere. u: DEVICE field; b_out: DEVICE cell array. */
int fs_divergence(fs_ctx *c, const fs_mac *u, float *b_out);

/* Volumetric-velocity initialisation, base profile (Sec. 3.3.3: the laminar
 * wall-function polynomial |v| / V_inf = 3/2 (y/delta) - 1/2 (y/delta)^3 below the
 * boundary-layer thickness delta, 1 above). Every fluid face of component c gets
 * dir[c] * V_inf * that factor, with y the height of the face centre above the
 * floor (dx * j for y faces, dx * (j + 1/2) otherwise) and V_inf the surface speed
 * of the face's cell column (the mean of the two columns for x and z faces between
 * columns). Fixed faces get their prescribed values (fs_set_mask), all other faces
 * and the padding 0.
 *   dir:   HOST, 3 doubles (the mainstream direction; not normalised here)
 *   vinf:  DEVICE, nz * nx floats, column (i, k) at k * nx + i
 *   delta: boundary-layer thickness in metres, >= 0 (0: the factor is 1)
 *   u_out: DEVICE field, overwritten.
 * FS_EINVAL on a NULL pointer or a non-finite / negative delta. */
int fs_wall_profile(fs_ctx *c, const double dir[3], const float *vinf, double delta, fs_mac *u_out);

/* Constrained divergence projection (Sec. 3.3.3, Eq. eq::divProj), Jacobi form,
 * in place on u. Per iteration every liquid cell i computes its constraint
 * C_i = (div u)_i = sum over its six faces of (u_hi - u_lo)/dx and
 * lambda_i = -C_i / (n_i / dx^2 + eps), n_i its number of free faces; then every
 * free face moves by (lambda_lo - lambda_hi) / dx (lambda = 0 off the liquid).
 * Free faces are fluid faces that are not held: fixed faces are always held, and
 * with hold_surface != 0 the faces between a liquid and an air cell (the observed
 * free surface) are held too.
 *   iters: iterations, in [0, 10^7]; eps: relaxation, >= 0
 *   div_norm (HOST, nullable): |C|_2 over the liquid after the last iteration.
 * FS_EINVAL on bad arguments, FS_ENONFINITE if the divergence is not finite. */
int fs_pbd_project(fs_ctx *c, fs_mac *u, int hold_surface, int iters, double eps, double *div_norm);

/* Pinhole camera of the splatting renderer: x_c = R x + t (R row-major), pixel
 * u = fx x_c / z_c + cx, v = fy y_c / z_c + cy; pixel (px, py) has its centre at
 * (px + 1/2, py + 1/2). Gaussians with z_c <= znear are culled. */
typedef struct {
    double R[9], t[3];
    double fx, fy, cx, cy;
    int width, height;     /* pixels, each in [1, 16384] */
    double znear;          /* > 0 */
    double bg[3];          /* background colour */
} fs_camera;

/* Forward splatting of n Gaussians into an RGB image (Sec. 3.2.1 compositing
 * formula, Sec. 3.5 rendering by splatting), into device buffers (headless):
 *   C = sum_i alpha_i c_i prod_{j<i} (1 - alpha_j) + T bg over the Gaussians in
 *   increasing depth (ties by index); alpha_i = min(0.99, sigma_i exp(-d^T S^-1 d / 2))
 *   with S = J R A_i R^T J^T the projected covariance (J the pinhole Jacobian at the
 *   mean) and d the pixel centre's offset from the projected mean, kept inside the
 *   3-sigma ellipse and when alpha >= 1/255; the walk stops once the transmittance
 *   would fall below 1e-4. Colours are RGB (degree-0 spherical harmonics;
 *   fs_splat_render_sh takes higher degrees).
 *   x [n][3], opacity [n] in [0, 1], A [n][3][3] covariances, color [n][3]: DEVICE;
 *   cam: HOST; rgb_out [height][width][3], T_out (nullable) [height][width]: DEVICE.
 * A must be symmetric positive definite. Does not need a mask. Synchronises the
 * stream once (the number of tile entries sizes a scratch buffer). FS_EINVAL on bad
 * arguments or more than 2^32 (Gaussian, 16 x 16 tile) pairs, FS_ENOMEM when the
 * scratch cannot grow. */
int fs_splat_render(fs_ctx *c, int n, const float *x, const float *opacity, const float *A, const float *color,
                    const fs_camera *cam, float *rgb_out, float *T_out);

/* fs_splat_render with view-dependent colours (Sec. 3.2.1: the compositing sum
 * weights SH(r; F_i), the spherical-harmonic colour of Gaussian i seen along the
 * ray): c_i = max(0, 1/2 + sum_j sh[i][j] Y_j(d_i)) per channel, with d_i the
 * unit vector from the camera centre -R^T t to the mean and Y_j, j = l^2 + l + m,
 * the real spherical harmonics of degree l <= sh_degree, normalised over the
 * sphere, in the sign convention of the standard 3DGS evaluator (degree 1:
 * -a y, a z, -a x with a = sqrt(3 / (4 pi))).
 *   sh [n][(sh_degree + 1)^2][3]: DEVICE; sh_degree in [0, 3]; the rest as in
 *   fs_splat_render. Degree 0 with sh[i][0] = (c_i - 1/2) / Y_0 gives colour c_i. */
int fs_splat_render_sh(fs_ctx *c, int n, const float *x, const float *opacity, const float *A, const float *sh,
                       int sh_degree, const fs_camera *cam, float *rgb_out, float *T_out);

/* Counters of the last fs_splat_render on this context, as host values (no GPU
 * work): entries = the number of (Gaussian, tile) pairs binned, max_tile = the
 * most Gaussians binned into one 16 x 16 tile. Both 0 before the first render.
 * FS_EINVAL on a NULL argument. */
int fs_splat_stats(const fs_ctx *c, unsigned long long *entries, unsigned long long *max_tile);

/* APIC particle -> grid transfer (Sec. 3.2.2, Eq. eq::particle_map), per MAC face
 * component c with quadratic B-spline weights w_ip over 3 x 3 x 3 nodes (the nodes
 * of component c sit at index * dx along axis c and (index + 1/2) * dx along the
 * others):  (m v)_i = sum_p w_ip m_p [v_p,c + (C_p (x_i - x_p))_c],
 *           u_c,i = (m v)_i / sum_p w_ip m_p, 0 where no particle reaches.
 * Does not depend on the mask. np >= 0 particles, all DEVICE arrays:
 *   x, v: [np][3] metres and m/s; C: [np][3][3] row-major (row c = gradient of
 *   component c); m: [np]; u_out: overwritten; mass_out (nullable): sum_p w_ip m_p.
 * FP32 atomic accumulation: the last bits depend on the scheduling.
 * FS_EINVAL on a NULL array or np < 0. */
int fs_p2g(fs_ctx *c, int np, const float *x, const float *v, const float *C, const float *m, fs_mac *u_out,
           fs_mac *mass_out);

/* APIC grid -> particle transfer and particle update (Sec. 3.2.2, Sec. 3.4.3):
 *   v_p,c = sum_i w_ip u_c,i,   C_p[c][a] = 4/dx^2 sum_i w_ip u_c,i (x_i - x_p)_a,
 * then when advance != 0: x_p += dt v_p clamped to [lo, hi] per axis,
 * F_p = (I + dt C_p) F_p (when F != NULL) and A_p = F_p A0_p F_p^T (when A0 and
 * A_out != NULL), the deformation and covariance of the Gaussians. All DEVICE:
 *   x [np][3] (updated when advancing), v_out [np][3], C_out [np][3][3],
 *   F [np][3][3] in/out, A0, A_out [np][3][3]; u the grid field.
 * FS_EINVAL on a NULL required array, np < 0 or non-finite dt, lo, hi. */
int fs_g2p(fs_ctx *c, int np, float *x, float *v_out, float *C_out, float *F, const float *A0, float *A_out,
           const fs_mac *u, double dt, int advance, double lo, double hi);

/* Recurrent convolutional pressure solver (Sec. 3.4.1: the PeRCNN layer that
 * replaces the implicit pressure solve during the optimisation). The scheme's own
 * 7-point operator L_p with the cell-type boundary conditions is encoded; a fitted
 * 3x3x3 kernel W acts on the residual, and `substeps` recurrent sub-steps emulate
 * the iteration of an implicit solver:
 *   p_0 = 0,  r_k = m (b - L_p p_k),  p_{k+1} = p_k + m (W * r_k),
 * m the liquid mask, * the correlation over the 27 taps [dz][dy][dx] (neighbours
 * off the liquid read 0). Fixed points solve L_p p = b. With
 * fs_params.pressure_solver = FS_SOLVER_PERCNN every projection uses it; the
 * statistics report K iterations and the true residual.
 *   w27: HOST, 27 floats; stored point-symmetrised, (w[t] + w[26 - t]) / 2, which
 *        makes the map b -> p_K symmetric (the adjoint step relies on it)
 *   substeps: K in [1, 100000]. FS_EINVAL on a NULL or non-finite kernel. */
int fs_percnn_load(fs_ctx *c, const float *w27, int substeps);

/* The stored (symmetrised) kernel and K. w27: HOST, 27 floats. FS_ESTATE when none. */
int fs_percnn_read(fs_ctx *c, float *w27, int *substeps);

/* Fit of the kernel (Sec. 3.4.1: the recurrent solver should give the pressure of
 * the second-order scheme on solver-generated pairs): for one pair L_p q = b
 * (DEVICE public-layout cell arrays) ADDS the energy-norm loss
 * (p_K - q)^T L_p (p_K - q) / q^T L_p q to *loss and its gradient w.r.t. the 27
 * stored taps to dw27 (HOST, 27 floats), by the backward recurrence over the K
 * stored residuals (K * cells floats of device memory). The gradient is w.r.t.
 * the stored taps; a caller that fits the symmetric kernel symmetrises it. */
int fs_percnn_grad(fs_ctx *c, const float *b, const float *q, double *loss, float *dw27);

/* Apply the pressure preconditioner selected in the parameters to one vector:
 * z = M^-1 r on the liquid cells (zero elsewhere). Jacobi: M = diag(L_p);
 * MIC(0): M = L L^T with the modified incomplete Cholesky factor of L_p (Bridson,
 * cited by the paper for its pressure projection, Sec. 3.2.2), factored on first
 * use after fs_set_mask, computed in lexicographic order (x fastest). Multigrid:
 * one V-cycle of damped-Jacobi smoothing on a cell hierarchy (a symmetric linear
 * operator; the paper has no counterpart), built on first use after fs_set_mask,
 * which synchronises the stream once. Learned: the network (needs fs_net_load).
 * r, z: DEVICE cell arrays in the library layout, must not alias.
 * Returns FS_ETIMEOUT if a bounded device wait of the MIC(0) wavefront ran out. */
int fs_precond_apply(fs_ctx *c, const float *r, float *z);

/* ---- learned preconditioner (Sec. 3.4.1, Fig. percnn_str_fit: a network of
 * 3x3x3 convolutions fitted to implicit-solver output stands in for the
 * pressure solve; here it serves as the preconditioner of flexible CG) ----------
 * Five 3x3x3 convolutions, channels 2 -> 16 -> 16 -> 16 -> 16 -> 1, zero padding,
 * ReLU after the first four; input channel 0 = r / s on liquid cells (s = max |r|
 * over the liquid), channel 1 = cell type code (liquid 1, air 0, solid -1);
 * output z = s * y on liquid cells. bf16 weights and activations, FP32 sums.
 * Parameters are one flat FP32 vector in PyTorch Conv3d order: W1 [16][2][3][3][3],
 * b1 [16], W2, b2, W3, b3, W4, b4 (each [16][16][3][3][3], [16]), W5 [1][16][3][3][3],
 * b5 [1]; fs_net_param_count() gives its length. With precond = FS_PRECOND_LEARNED
 * (the network alone) or FS_PRECOND_LEARNED_MG (the network followed by one
 * multigrid V-cycle on its residual, z = e + M(r - L_p e) with e = s Net(r/s): the
 * network acts as the fine-grid smoother and the V-cycle as the coarse correction)
 * the pressure solve runs flexible CG (beta = -z'.Ap / p.Ap); if that does not
 * reach the tolerance it is redone with MIC(0) and fs_stats.fallbacks counts it. */
int fs_net_param_count(void);

/* Load parameters (FP32, `count` values; HOST memory if params_on_host, else
 * DEVICE). Allocates the network's buffers on first use (FS_ENOMEM). */
int fs_net_load(fs_ctx *c, const float *params, int count, int params_on_host);

/* Copy the current FP32 master parameters to HOST memory (`count` values). */
int fs_net_read(fs_ctx *c, float *params_host, int count);

/* z = Net(r) on liquid cells; r, z DEVICE cell arrays (library layout). */
int fs_net_forward(fs_ctx *c, const float *r, float *z);

/* The kernels of the network's inference layers on this context (the learned
 * preconditioners and fs_net_forward; training always uses the first):
 *   0: warp-level mma.sync m16n8k16 BF16 MMAs, operands staged by ldmatrix;
 *   1: tcgen05.mma (M = 128 cells, N = 16 channels, K = 16 per 3x3x3 tap) with
 *      the accumulators in tensor memory, read back by tcgen05.ld.
 * Both compute the same sums (FP32 accumulation of BF16 products, in a different
 * order). FS_EINVAL for another value; a bounded wait for the MMAs that runs out
 * makes the next solve or fs_net_forward return FS_ETIMEOUT. */
int fs_net_kernel(fs_ctx *c, int which);

/* Training on one (b, q) pair with L_p q = b on the context's mask (DEVICE cell
 * arrays), for the role the context's precond selects. The loss is the relative
 * error that the preconditioner leaves, in the energy norm of the pressure
 * operator, loss = w.L_p w / (q/s).L_p (q/s) (the fitted network should give the
 * pressure of the Laplacian scheme, Sec. 3.4.1), with y = Net(b/s) on liquid
 * cells and
 *   FS_PRECOND_LEARNED_MG:  w = q/s - y - M(b/s - L_p y), M the V-cycle
 *                           (its gradient passes through M, which is symmetric);
 *   any other precond:      w = q/s - y.
 * The loss is ADDED to *loss (host) and its gradient ADDED to the context's
 * gradient accumulator. */
int fs_net_grad(fs_ctx *c, const float *b, const float *q, double *loss);

/* Copy the accumulated gradient to HOST memory (`count` values). */
int fs_net_grad_read(fs_ctx *c, float *grad_host, int count);

/* One Adam step (bias-corrected, `step` >= 1) on the FP32 master parameters with
 * the accumulated gradient times grad_scale; clears the accumulator and refreshes
 * the bf16 working copies. fix_offsets = 1 keeps every bias and the weights of the
 * cell-type input channel at their current values: when those are zero the
 * network is positively homogeneous, Net(a x) = a Net(x) for a >= 0, so the
 * preconditioner responds to a shrinking residual in proportion. */
int fs_net_adam(fs_ctx *c, double lr, double beta1, double beta2, double eps, int step, double grad_scale,
                int fix_offsets);

/* One Adam step (Kingma and Ba, 2015) on `n` FP32 parameters in DEVICE memory: the
 * optimiser of the parameter fit (Sec. 3.4.2 fits theta = log nu and the
 * correction of the initial velocity by gradient descent on the loss). With
 * g' = grad_scale g:  m = beta1 m + (1 - beta1) g',  v = beta2 v + (1 - beta2) g'^2,
 * p -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps).
 * p, m, v are updated in place, g is read only; the caller owns all four arrays
 * (m and v zero before step 1; any alignment, 16-byte aligned ones take four
 * elements per thread). Runs on the context's stream without synchronising; needs
 * no mask. FS_EINVAL for n < 0, a NULL array with n > 0, step < 1, lr < 0, a beta
 * outside [0, 1), eps <= 0 or a non-finite lr or grad_scale. */
int fs_adam_update(fs_ctx *c, float *p, const float *g, float *m, float *v, long long n, double lr, double beta1,
                   double beta2, double eps, int step, double grad_scale);

/* fs_net_grad over `batch` pairs stored back to back (each `nelems` floats of the
 * library layout) followed by fs_net_adam with grad_scale = 1/batch (beta1 0.9,
 * beta2 0.999, eps 1e-8, fix_offsets 1). *loss receives the mean loss of the batch. */
int fs_net_train_step(fs_ctx *c, const float *b_batch, const float *q_batch, int batch, double lr, int step,
                      double *loss);

/* Per-kernel timing. fs_profile(c, k) with k >= 1 resets the counters and from
 * then on brackets launches of the solver kernels (every k-th CG iteration of
 * each batch), the advection kernels and the preconditioners with CUDA events on
 * the context's stream; fs_profile(c, 0) stops. It also counts every kernel the
 * context launches (reported as the entry "all_kernels"). Timing is collected when a call synchronises, so it adds no host
 * round trip. fs_profile_read copies up to `max` entries (one per kernel kind
 * that ran) into `out` and sets *count. `bytes` is the ALGORITHMIC traffic summed
 * over the launches: for the CG kernels the flag byte of every element of the
 * launch range plus, per active element (liquid cell or fluid face), 16 bytes for
 * the fused direction update and operator apply (read r or z and p, write p and
 * Ap) and 24 bytes for the iterate update (read x, r, p, Ap, write x, r); zero for
 * kernels without a stated figure. */
typedef struct {
    char name[32];
    long long launches;      /* launches timed (every k-th of the sampled kinds) */
    double total_ms;         /* their summed duration */
    double bytes;            /* their summed algorithmic bytes */
    long long all_launches;  /* launches of this kind that did work, timed or not (>= launches) */
} fs_kernel_time;

int fs_profile(fs_ctx *c, int enable);
int fs_profile_read(fs_ctx *c, fs_kernel_time *out, int max, int *count);

/* Pressure projection that allocates nothing. The paper has no counterpart: this
 * serves callers that cannot allocate device memory (code running where a CUDA
 * allocation is forbidden or would break a fixed memory budget, such as a plugin
 * inside an application that owns the device allocator, or a real-time loop that
 * must not call cudaMalloc after start-up).
 *
 * It computes what fs_project computes with the Jacobi preconditioner, without a
 * context: u (DEVICE field in the layout fs_init_grid would use for this size:
 * pitch = nx + 1 rounded up to a multiple of 4, rows = ny + 1, planes = nz + 1)
 * is projected in place; q_out (nullable DEVICE cell array, same layout)
 * receives q; cell_type_dense is as in fs_set_mask; every fixed face keeps the
 * value it holds in u. tol is the relative residual target, maxit the iteration
 * cap, dx the cell size (it scales q only). All scratch lives in one static
 * device array of 16 MiB that every GPU loading the library holds until the
 * process exits; every grid up to 64 x 64 x 64 fits, a larger one is rejected
 * with FS_EINVAL (and a message giving the bytes it needs) before any work.
 * The call never calls cudaMalloc, cudaFree or any other allocating routine.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress) with
 * the caller's current device, so the array of that device is used; the first
 * call on a device may load the library's device code there, so make that first
 * call before any stream capture. Every call shares the one array, and each clears the parts
 * that must start at zero: calls that overlap on the GPU (on different streams or
 * host threads, for the same device) race and corrupt each other's results.
 * The call synchronises `cuda_stream` before it returns. */
int fs_project_noalloc(int nx, int ny, int nz, const uint8_t *cell_type_dense, fs_mac *u, float *q_out,
                       double dx, double tol, int maxit, void *cuda_stream, fs_stats *st);

/* The per-thread message of the last failing call ("" if none). */
const char *fs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FLUIDSTEP_H */
