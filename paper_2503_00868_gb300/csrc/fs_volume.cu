// fs_volume.cu -- volumetric-velocity initialisation (arXiv 2503.00868,
// Sec. 3.3.3): the laminar wall-function base profile and the constrained
// divergence projection of Eq. eq::divProj, on the public MAC layout.
//
// Base profile: a fluid face gets dir * V_inf * f(y / delta), f(e) = 3/2 e - 1/2 e^3
// below the boundary-layer thickness and 1 above, y the height of the face centre
// above the floor, V_inf the surface speed of the face's cell column (the mean of
// both columns for x and z faces between two columns). Fixed faces take their
// prescribed values, other faces 0.
//
// Constrained projection, Jacobi form: per iteration every liquid cell computes its
// constraint C = (div u) over its six faces and lambda = -C / (n_free / dx^2 + eps)
// into a cell-space buffer, then every free face moves by (lambda_lo - lambda_hi)/dx.
// Free faces are fluid faces that are not held; with hold_surface the faces between
// a liquid and an air cell (the observed free surface) are held.
// Per iteration: one pass over the cells (3 face arrays + flags -> lambda) and one
// over the faces (lambda + the face arrays, in place): HBM-bound streams.
#include <cmath>

#include "fs_internal.cuh"

namespace fs {
namespace {

constexpr int TH = 256;

__device__ __forceinline__ void decode_pub(const Layout &L, int t, int &i, int &j, int &k)
{
    i = t % L.P;
    const int row = t / L.P;
    j = row % L.R;
    k = row / L.R;
}

__device__ __forceinline__ float column_speed(const float *__restrict__ vinf, const Layout &L, int i, int k)
{
    i = min(max(i, 0), L.nx - 1);
    k = min(max(k, 0), L.nz - 1);
    return __ldg(vinf + (size_t)k * L.nx + i);
}

__global__ void __launch_bounds__(TH) k_wall_profile(F3 u, const uint8_t *__restrict__ ff,
                                                     const float *__restrict__ bc, const float *__restrict__ vinf,
                                                     float d0, float d1, float d2, float delta, float dx, Layout L)
{
    const float dir[3] = {d0, d1, d2};
    const long long total = 3LL * L.S;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / L.S), t = (int)(e - (long long)c * L.S);
        int i, j, k;
        decode_pub(L, t, i, j, k);
        const int fs_idx = L.face_origin(c) + t;
        const uint8_t f = ff[fs_idx];
        float v = 0.f;
        if (f & FF_FIXED) {
            v = bc ? bc[fs_idx] : 0.f;
        } else if (f & FF_FLUID) {
            const float y = (c == 1 ? (float)j : (float)j + 0.5f) * dx;
            float vi;
            if (c == 0) vi = 0.5f * (column_speed(vinf, L, i - 1, k) + column_speed(vinf, L, i, k));
            else if (c == 2) vi = 0.5f * (column_speed(vinf, L, i, k - 1) + column_speed(vinf, L, i, k));
            else vi = column_speed(vinf, L, i, k);
            float fac = 1.f;
            if (delta > 0.f) {
                const float r = y / delta;
                fac = r >= 1.f ? 1.f : (r <= 0.f ? 0.f : 1.5f * r - 0.5f * r * r * r);
            }
            v = dir[c] * vi * fac;
        }
        u.c[c][t] = v;
    }
}

// face of component c at public index t (the low face of cell t): may it move?
__device__ __forceinline__ bool pbd_free(const uint8_t *__restrict__ ff, const uint8_t *__restrict__ cf,
                                         const Layout &L, int c, int t, int off, int hold)
{
    if (!(ff[L.face_origin(c) + t] & FF_FLUID)) return false;
    if (!hold) return true;
    const uint8_t lo = cf[L.PL + t - off], hi = cf[L.PL + t];
    const bool surface = ((lo & CF_LIQ) && (hi & CF_AIR)) || ((lo & CF_AIR) && (hi & CF_LIQ));
    return !surface;
}

// lambda per liquid cell (cell space, 0 elsewhere) and |C|^2 -> s->aux[0]
__global__ void __launch_bounds__(TH) k_pbd_lambda(CF3 u, const uint8_t *__restrict__ cf,
                                                   const uint8_t *__restrict__ ff, Layout L, int hold, float inv_dx,
                                                   float eps, float *lam, SolveScal *s, double *partials)
{
    const int off[3] = {1, L.P, L.PL};
    KSum acc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.S; t += gridDim.x * blockDim.x) {
        float lv = 0.f;
        if (cf[L.PL + t] & CF_LIQ) {
            float C = 0.f;
            int nfree = 0;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                C += (u.c[c][t + off[c]] - u.c[c][t]) * inv_dx;
                nfree += pbd_free(ff, cf, L, c, t, off[c], hold) + pbd_free(ff, cf, L, c, t + off[c], off[c], hold);
            }
            acc.add(C * C);
            lv = -C / ((float)nfree * inv_dx * inv_dx + eps);
        }
        lam[L.PL + t] = lv;
    }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) s->aux[0] = tot[0];
}

// every free face moves by (lambda_lo - lambda_hi) / dx
__global__ void __launch_bounds__(TH) k_pbd_update(F3 u, const uint8_t *__restrict__ cf,
                                                   const uint8_t *__restrict__ ff, Layout L, int hold, float inv_dx,
                                                   const float *__restrict__ lam)
{
    const int off[3] = {1, L.P, L.PL};
    const long long total = 3LL * L.S;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / L.S), t = (int)(e - (long long)c * L.S);
        if (!pbd_free(ff, cf, L, c, t, off[c], hold)) continue;
        u.c[c][t] += (lam[L.PL + t - off[c]] - lam[L.PL + t]) * inv_dx;
    }
}

}  // namespace

int launch_wall_profile(fs_ctx *c, const double dir[3], const float *vinf, double delta, F3 u)
{
    const Layout &L = c->L;
    k_wall_profile<<<grid_blocks(c, 3LL * L.S, TH), TH, 0, c->stream>>>(
        u, c->fflag, c->has_bc ? c->bc : nullptr, vinf, (float)dir[0], (float)dir[1], (float)dir[2], (float)delta,
        (float)c->prm.dx, L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

// `iters` Jacobi iterations in place on u; |C|_2 over the liquid after the last.
int launch_pbd_project(fs_ctx *c, F3 u, int hold, int iters, double eps, double *norm)
{
    const Layout &L = c->L;
    const float inv_dx = (float)(1.0 / c->prm.dx);
    const int bc_ = grid_blocks(c, L.S, TH), bf = grid_blocks(c, 3LL * L.S, TH);
    CF3 uc{{u.c[0], u.c[1], u.c[2]}};
    float *lam = c->pr;  // cell-space scratch: no solve runs meanwhile
    SolveScal *s = c->scal + 2;
    for (int it = 0; it <= iters; it++) {
        k_pbd_lambda<<<bc_, TH, 0, c->stream>>>(uc, c->cflag, c->fflag, L, hold, inv_dx, (float)eps, lam, s,
                                                c->partials);
        c->n_launches += 1;
        if (it == iters) break;
        k_pbd_update<<<bf, TH, 0, c->stream>>>(u, c->cflag, c->fflag, L, hold, inv_dx, lam);
        c->n_launches += 1;
    }
    FS_CUDA(cudaGetLastError());
    SolveScal h;
    int rc = read_scal(c, 2, &h);
    if (rc) return rc;
    if (!std::isfinite(h.aux[0])) return set_error(FS_ENONFINITE, "fs_pbd_project: non-finite divergence");
    if (norm) *norm = std::sqrt(h.aux[0]);
    return FS_OK;
}

}  // namespace fs
