// fs_advect.cu -- semi-Lagrangian convection on the MAC grid (arXiv 2503.00868,
// Sec. 3.4.1: back-tracing after Stam's stable fluids) with the body force of
// Eq. eq::v, and its exact discrete adjoint.
//
// Each fluid face f of component c looks up the velocity at the face (its own
// value; each other component as the mean of the 4 surrounding faces), traces
// back one forward-Euler step in index space, s = idx - (dt/dx) * vel, clamps s
// to [0, n-1] per axis of the component's array and samples trilinearly. The
// adjoint scatters the cotangent to the 8 corners and routes the derivative
// w.r.t. the trace position back to the velocities that formed it (zero on a
// clamped axis).
#include "fs_internal.cuh"

namespace fs {
namespace {

struct Axis {
    int base;
    float frac;
    bool active;
};

// frac is formed from the integer offset so that its rounding error does not
// grow with the index.
__device__ __forceinline__ Axis trace_axis(int pos, float disp, int n)
{
    Axis a;
    const float s = (float)pos - disp;
    if (s < 0.f) { a.base = 0; a.frac = 0.f; a.active = false; }
    else if (s > (float)(n - 1)) { a.base = n - 2; a.frac = 1.f; a.active = false; }
    else {
        int b = (int)floorf(s);
        b = b > n - 2 ? n - 2 : b;
        b = b < 0 ? 0 : b;
        a.base = b;
        a.frac = (float)(pos - b) - disp;
        a.active = true;
    }
    return a;
}

struct Trace {
    Axis ax[3];
    int corner;  // public-layout index of the (base, base, base) corner
};

__device__ __forceinline__ void face_trace(const CF3 &u, const Layout &L, int c, int i, int j, int k, int idx,
                                           float h, Trace &tr)
{
    const int offs[3] = {1, L.P, L.PL};
    const int off_c = offs[c];
    float vel[3];
    vel[c] = u.c[c][idx];
#pragma unroll
    for (int e = 0; e < 3; e++) {
        if (e == c) continue;
        const float *ue = u.c[e];
        const int l = idx - off_c, oe = offs[e];
        vel[e] = 0.25f * ((ue[l] + ue[l + oe]) + (ue[idx] + ue[idx + oe]));
    }
    int dims[3] = {L.nx, L.ny, L.nz};
    dims[c] += 1;
    const int pos[3] = {i, j, k};
#pragma unroll
    for (int e = 0; e < 3; e++) tr.ax[e] = trace_axis(pos[e], h * vel[e], dims[e]);
    tr.corner = (tr.ax[2].base * L.R + tr.ax[1].base) * L.P + tr.ax[0].base;
}

// One launch per component; grid (ceil(P/128), rows, planes).
__global__ void __launch_bounds__(128) k_advect(CF3 u, float *__restrict__ vx, const uint8_t *__restrict__ ff,
                                                Layout L, int c, float h, float dtg)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= L.P) return;
    const int idx = (k * L.R + j) * L.P + i;
    const int t = L.face_origin(c) + idx;
    if (!(ff[t] & FF_FLUID)) { vx[t] = 0.f; return; }
    Trace tr;
    face_trace(u, L, c, i, j, k, idx, h, tr);
    const float *uc = u.c[c];
    const int o = tr.corner, P = L.P, PL = L.PL;
    const float fx = tr.ax[0].frac, fy = tr.ax[1].frac, fz = tr.ax[2].frac;
    const float c00 = uc[o] + fx * (uc[o + 1] - uc[o]);
    const float c10 = uc[o + P] + fx * (uc[o + P + 1] - uc[o + P]);
    const float c01 = uc[o + PL] + fx * (uc[o + PL + 1] - uc[o + PL]);
    const float c11 = uc[o + PL + P] + fx * (uc[o + PL + P + 1] - uc[o + PL + P]);
    const float c0 = c00 + fy * (c10 - c00);
    const float c1 = c01 + fy * (c11 - c01);
    vx[t] = (c0 + fz * (c1 - c0)) + dtg;
}

__global__ void __launch_bounds__(128) k_advect_adj(CF3 u, const float *__restrict__ gb, F3 g,
                                                    const uint8_t *__restrict__ ff, Layout L, int c, float h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= L.P) return;
    const int idx = (k * L.R + j) * L.P + i;
    const int t = L.face_origin(c) + idx;
    if (!(ff[t] & FF_FLUID)) return;
    const float w = gb[t];
    if (w == 0.f) return;
    Trace tr;
    face_trace(u, L, c, i, j, k, idx, h, tr);
    const float *uc = u.c[c];
    float *gcp = g.c[c];
    const int o = tr.corner, P = L.P, PL = L.PL;
    const float fx = tr.ax[0].frac, fy = tr.ax[1].frac, fz = tr.ax[2].frac;
    const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy}, wz[2] = {1.f - fz, fz};
    float ds[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int cz = 0; cz < 2; cz++)
#pragma unroll
        for (int cy = 0; cy < 2; cy++)
#pragma unroll
            for (int cx = 0; cx < 2; cx++) {
                const int a = o + cz * PL + cy * P + cx;
                atomicAdd(gcp + a, w * (wx[cx] * wy[cy] * wz[cz]));
                const float val = uc[a];
                ds[0] += (cx ? 1.f : -1.f) * wy[cy] * wz[cz] * val;
                ds[1] += wx[cx] * (cy ? 1.f : -1.f) * wz[cz] * val;
                ds[2] += wx[cx] * wy[cy] * (cz ? 1.f : -1.f) * val;
            }
    const int offs[3] = {1, P, PL};
#pragma unroll
    for (int e = 0; e < 3; e++) {
        if (!tr.ax[e].active) continue;
        const float gv = -h * ds[e] * w;
        if (e == c) {
            atomicAdd(gcp + idx, gv);
        } else {
            float *ge = g.c[e];
            const int l = idx - offs[c], oe = offs[e];
            const float q = 0.25f * gv;
            atomicAdd(ge + l, q);
            atomicAdd(ge + l + oe, q);
            atomicAdd(ge + idx, q);
            atomicAdd(ge + idx + oe, q);
        }
    }
}

// The paper's upwind surrogate of the reverse of convection (Sec. 3.4.1): the
// cotangent w of a fluid face f of component c passes to the same face, and
// each velocity component e seen at f (the own one, or the mean of four faces
// of another) receives -h w (v_c(hi) - v_c(lo)), the first-order upwind
// difference of the convected field v along e, taken on the side the flow
// comes from (lo = f - 1 when the velocity along e is > 0, else hi = f + 1) and
// zero when that neighbour is outside the component's array. A fixed face holds
// its prescribed value in v, an air face 0. One launch per component.
__global__ void __launch_bounds__(128) k_advect_adj_upwind(CF3 u, const float *__restrict__ va,
                                                           const float *__restrict__ bc, const float *__restrict__ gb,
                                                           F3 g, const uint8_t *__restrict__ ff, Layout L, int c,
                                                           float h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= L.P) return;
    const int idx = (k * L.R + j) * L.P + i;
    const int t = L.face_origin(c) + idx;
    if (!(ff[t] & FF_FLUID)) return;
    const float w = gb[t];
    if (w == 0.f) return;
    float *gcp = g.c[c];
    atomicAdd(gcp + idx, w);  // the value term
    const int offs[3] = {1, L.P, L.PL};
    float vel[3];
    vel[c] = u.c[c][idx];
#pragma unroll
    for (int e = 0; e < 3; e++) {
        if (e == c) continue;
        const float *ue = u.c[e];
        const int l = idx - offs[c], oe = offs[e];
        vel[e] = 0.25f * ((ue[l] + ue[l + oe]) + (ue[idx] + ue[idx + oe]));
    }
    int dims[3] = {L.nx, L.ny, L.nz};
    dims[c] += 1;
    const int pos[3] = {i, j, k};
    auto conv = [&](int tt) { return (ff[tt] & FF_FIXED) ? bc[tt] : va[tt]; };
#pragma unroll
    for (int e = 0; e < 3; e++) {
        const bool up = vel[e] > 0.f;
        const int lo = up ? pos[e] - 1 : pos[e], hi = up ? pos[e] : pos[e] + 1;
        if (lo < 0 || hi >= dims[e]) continue;
        const int tl = t + (lo - pos[e]) * offs[e], th = t + (hi - pos[e]) * offs[e];
        const float gv = -h * (conv(th) - conv(tl)) * w;
        if (e == c) {
            atomicAdd(gcp + idx, gv);
        } else {
            float *ge = g.c[e];
            const int l = idx - offs[c], oe = offs[e];
            const float q = 0.25f * gv;
            atomicAdd(ge + l, q);
            atomicAdd(ge + l + oe, q);
            atomicAdd(ge + idx, q);
            atomicAdd(ge + idx + oe, q);
        }
    }
}

__global__ void k_zero3(F3 g, int n)
{
    const int c = blockIdx.y;
    float4 *p = reinterpret_cast<float4 *>(g.c[c]);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n / 4; t += gridDim.x * blockDim.x)
        p[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

int launch_advect(fs_ctx *c, CF3 u)
{
    const Layout &L = c->L;
    const float h = (float)(c->prm.dt / c->prm.dx);
    dim3 grid((L.P + 127) / 128, L.R, L.Z);
    cudaEvent_t e0 = prof_mark(c);
    for (int comp = 0; comp < 3; comp++)
        k_advect<<<grid, 128, 0, c->stream>>>(u, c->vx, c->fflag, L, comp, h,
                                             (float)(c->prm.dt * c->prm.g[comp]));
    // algorithmic bytes of the three launches: the three input components read
    // once (the gathered neighbours come from cache), the face flags, and the
    // three advected components written
    prof_add(c, K_ADVECT, e0, prof_mark(c), 24.0 * (double)L.S + (double)L.nF);
    c->n_launches += 3;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_advect_adjoint(fs_ctx *c, CF3 u, F3 g)
{
    const Layout &L = c->L;
    const float h = (float)(c->prm.dt / c->prm.dx);
    dim3 gz(grid_blocks(c, L.S / 4, 256), 3);
    k_zero3<<<gz, 256, 0, c->stream>>>(g, L.S);
    dim3 grid((L.P + 127) / 128, L.R, L.Z);
    if (c->prm.advect_grad == FS_ADVECT_GRAD_UPWIND) {
        // the convected field, into a free face-space vector (vx holds the cotangent)
        for (int comp = 0; comp < 3; comp++)
            k_advect<<<grid, 128, 0, c->stream>>>(u, c->vq, c->fflag, L, comp, h, (float)(c->prm.dt * c->prm.g[comp]));
        for (int comp = 0; comp < 3; comp++)
            k_advect_adj_upwind<<<grid, 128, 0, c->stream>>>(u, c->vq, c->bc, c->vx, g, c->fflag, L, comp, h);
        c->n_launches += 7;
        FS_CUDA(cudaGetLastError());
        return FS_OK;
    }
    cudaEvent_t e0 = prof_mark(c);
    for (int comp = 0; comp < 3; comp++)
        k_advect_adj<<<grid, 128, 0, c->stream>>>(u, c->vx, g, c->fflag, L, comp, h);
    // the input field and the cotangent read once, the face flags, and the
    // scattered gradient written once (its atomic adds resolve in L2)
    prof_add(c, K_ADVECT_ADJ, e0, prof_mark(c), 36.0 * (double)L.S + (double)L.nF);
    c->n_launches += 4;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

}  // namespace fs
