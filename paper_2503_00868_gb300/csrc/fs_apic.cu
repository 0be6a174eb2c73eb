// fs_apic.cu -- APIC transfers between particles and the MAC grid, and the
// deformation of the Gaussians (arXiv 2503.00868, Sec. 3.2.2, Sec. 3.4.3).
//
// Per face component c (nodes at index * dx along axis c, (index + 1/2) * dx along
// the others), quadratic B-spline weights over 3 x 3 x 3 nodes:
//   P2G (Eq. eq::particle_map): (m v)_i = sum_p w_ip m_p [v_p,c + (C_p (x_i - x_p))_c],
//        v_i = (m v)_i / sum_p w_ip m_p (0 where no particle reaches);
//   G2P: v_p,c = sum_i w_ip u_c,i,  C_p[c][a] = 4/dx^2 sum_i w_ip u_c,i (x_i - x_p)_a;
//   advance: x_p += dt v_p (clamped), F_p = (I + dt C_p) F_p, A_p = F_p A0_p F_p^T.
// P2G scatters with FP32 atomics (one thread per particle, 2 x 81 atomic adds),
// so the summation order, and the last bits, vary from run to run; G2P gathers
// (one thread per particle, 81 node reads). Particles are arrays of structures:
// x, v [p][3]; C, F, A0, A [p][3][3] row-major; m [p].
#include <cmath>

#include "fs_internal.cuh"

namespace fs {
namespace {

constexpr int TH = 256;

struct Spline {
    int base[3];
    float w[3][3];
};

// weights of component c's nodes around position x (metres); the node coordinate
// is clamped to [-8, lim] first (a position that far out, or NaN, reaches no node
// and cannot overflow the integer base)
__device__ __forceinline__ Spline spline(const float x[3], int c, float inv_dx, float lim)
{
    Spline s;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float sc = fminf(fmaxf(x[a] * inv_dx - (a == c ? 0.f : 0.5f), -8.f), lim);
        const int b = (int)floorf(sc - 0.5f);
        const float f = sc - (float)b;
        s.base[a] = b;
        s.w[a][0] = 0.5f * (1.5f - f) * (1.5f - f);
        s.w[a][1] = 0.75f - (f - 1.f) * (f - 1.f);
        s.w[a][2] = 0.5f * (f - 0.5f) * (f - 0.5f);
    }
    return s;
}

__device__ __forceinline__ bool in_faces(const Layout &L, int c, int i, int j, int k)
{
    const int di = L.nx + (c == 0), dj = L.ny + (c == 1), dk = L.nz + (c == 2);
    return i >= 0 && j >= 0 && k >= 0 && i < di && j < dj && k < dk;
}

__global__ void __launch_bounds__(TH) k_p2g(int np, const float *__restrict__ x, const float *__restrict__ v,
                                            const float *__restrict__ C, const float *__restrict__ m, F3 mv,
                                            F3 ms, Layout L, float dx)
{
    const float inv_dx = 1.f / dx;
    const float lim = (float)(max(L.nx, max(L.ny, L.nz)) + 8);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
        const float mp = m[p];
#pragma unroll 1
        for (int c = 0; c < 3; c++) {
            const Spline s = spline(xp, c, inv_dx, lim);
            const float vc = v[3 * p + c];
            const float c0 = C[9 * p + 3 * c], c1 = C[9 * p + 3 * c + 1], c2 = C[9 * p + 3 * c + 2];
            for (int kz = 0; kz < 3; kz++)
                for (int ky = 0; ky < 3; ky++)
#pragma unroll
                    for (int kx = 0; kx < 3; kx++) {
                        const int i = s.base[0] + kx, j = s.base[1] + ky, k = s.base[2] + kz;
                        if (!in_faces(L, c, i, j, k)) continue;
                        const float wt = s.w[0][kx] * s.w[1][ky] * s.w[2][kz] * mp;
                        const float dxv = ((float)i + (c == 0 ? 0.f : 0.5f)) * dx - xp[0];
                        const float dyv = ((float)j + (c == 1 ? 0.f : 0.5f)) * dx - xp[1];
                        const float dzv = ((float)k + (c == 2 ? 0.f : 0.5f)) * dx - xp[2];
                        const int t = (k * L.R + j) * L.P + i;
                        atomicAdd(mv.c[c] + t, wt * (vc + c0 * dxv + c1 * dyv + c2 * dzv));
                        atomicAdd(ms.c[c] + t, wt);
                    }
        }
    }
}

// u = mv / ms where ms > 0 (in place on mv); mass copy when wanted
__global__ void __launch_bounds__(TH) k_p2g_norm(F3 mv, CF3 ms, F3 mass_out, long long S)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3 * S;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / S);
        const long long t = e - c * S;
        const float mm = ms.c[c][t];
        mv.c[c][t] = mm > 0.f ? mv.c[c][t] / mm : 0.f;
        if (mass_out.c[c]) mass_out.c[c][t] = mm;
    }
}

__global__ void __launch_bounds__(TH) k_g2p(int np, float *x, float *v, float *C, float *F,
                                            const float *__restrict__ A0, float *A, CF3 u, Layout L, float dx,
                                            float dt, int advance, float lo, float hi)
{
    const float inv_dx = 1.f / dx;
    const float cs = 4.f * inv_dx * inv_dx;
    const float lim = (float)(max(L.nx, max(L.ny, L.nz)) + 8);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
        float vp[3], Cp[9];
#pragma unroll 1
        for (int c = 0; c < 3; c++) {
            const Spline s = spline(xp, c, inv_dx, lim);
            float vc = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
            for (int kz = 0; kz < 3; kz++)
                for (int ky = 0; ky < 3; ky++)
#pragma unroll
                    for (int kx = 0; kx < 3; kx++) {
                        const int i = s.base[0] + kx, j = s.base[1] + ky, k = s.base[2] + kz;
                        if (!in_faces(L, c, i, j, k)) continue;
                        const float wu = s.w[0][kx] * s.w[1][ky] * s.w[2][kz] * __ldg(u.c[c] + (k * L.R + j) * L.P + i);
                        vc += wu;
                        g0 += wu * (((float)i + (c == 0 ? 0.f : 0.5f)) * dx - xp[0]);
                        g1 += wu * (((float)j + (c == 1 ? 0.f : 0.5f)) * dx - xp[1]);
                        g2 += wu * (((float)k + (c == 2 ? 0.f : 0.5f)) * dx - xp[2]);
                    }
            vp[c] = vc;
            Cp[3 * c] = cs * g0;
            Cp[3 * c + 1] = cs * g1;
            Cp[3 * c + 2] = cs * g2;
        }
#pragma unroll
        for (int a = 0; a < 3; a++) v[3 * p + a] = vp[a];
#pragma unroll
        for (int a = 0; a < 9; a++) C[9 * p + a] = Cp[a];
        if (!advance) continue;
#pragma unroll
        for (int a = 0; a < 3; a++) x[3 * p + a] = fminf(fmaxf(xp[a] + dt * vp[a], lo), hi);
        if (!F) continue;
        float Fo[9], Fn[9];
#pragma unroll
        for (int a = 0; a < 9; a++) Fo[a] = F[9 * p + a];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int s = 0; s < 3; s++)
                Fn[3 * r + s] = Fo[3 * r + s] +
                                dt * (Cp[3 * r] * Fo[s] + Cp[3 * r + 1] * Fo[3 + s] + Cp[3 * r + 2] * Fo[6 + s]);
#pragma unroll
        for (int a = 0; a < 9; a++) F[9 * p + a] = Fn[a];
        if (!A0 || !A) continue;
        float T[9];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int s = 0; s < 3; s++)
                T[3 * r + s] = Fn[3 * r] * A0[9 * p + s] + Fn[3 * r + 1] * A0[9 * p + 3 + s] +
                               Fn[3 * r + 2] * A0[9 * p + 6 + s];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int s = 0; s < 3; s++)
                A[9 * p + 3 * r + s] = T[3 * r] * Fn[3 * s] + T[3 * r + 1] * Fn[3 * s + 1] + T[3 * r + 2] * Fn[3 * s + 2];
    }
}

}  // namespace

int launch_p2g(fs_ctx *c, int np, const float *x, const float *v, const float *C, const float *m, F3 u, F3 mass)
{
    const Layout &L = c->L;
    const size_t sb = (size_t)L.S * sizeof(float);
    F3 ms{{c->fg[0], c->fg[1], c->fg[2]}};
    for (int k = 0; k < 3; k++) {
        FS_CUDA(cudaMemsetAsync(u.c[k], 0, sb, c->stream));
        FS_CUDA(cudaMemsetAsync(ms.c[k], 0, sb, c->stream));
    }
    if (np > 0) {
        k_p2g<<<grid_blocks(c, np, TH), TH, 0, c->stream>>>(np, x, v, C, m, u, ms, L, (float)c->prm.dx);
        c->n_launches += 1;
    }
    CF3 msc{{ms.c[0], ms.c[1], ms.c[2]}};
    k_p2g_norm<<<grid_blocks(c, 3LL * L.S, TH), TH, 0, c->stream>>>(u, msc, mass, (long long)L.S);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_g2p(fs_ctx *c, int np, float *x, float *v, float *C, float *F, const float *A0, float *A, CF3 u,
               double dt, int advance, double lo, double hi)
{
    if (np <= 0) return FS_OK;
    k_g2p<<<grid_blocks(c, np, TH), TH, 0, c->stream>>>(np, x, v, C, F, A0, A, u, c->L, (float)c->prm.dx,
                                                          (float)dt, advance, (float)lo, (float)hi);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

}  // namespace fs
