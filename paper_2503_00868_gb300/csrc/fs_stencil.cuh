// fs_stencil.cuh -- helpers of the CG kernels and the streaming update
// (included by fs_pcg.cu before fs_tma.cuh).
//
// With the Jacobi preconditioner the solver keeps the scaled residual
// z = D^-1 r instead of r (the update is z -= alpha D^-1 Ap, and r.z = sum d z^2,
// r.r = sum d^2 z^2), so the direction update needs no division.
#pragma once

namespace fs {
namespace {

__device__ __forceinline__ float4 ld4(const float *__restrict__ p, int t)
{
    return __ldg(reinterpret_cast<const float4 *>(p + t));
}

__device__ __forceinline__ float4 fma4(float4 a, float b, float4 c)  // a + b c
{
    return make_float4(a.x + b * c.x, a.y + b * c.y, a.z + b * c.z, a.w + b * c.w);
}

// Diagonal and its inverse per neighbour count, for this launch's coefficient.
template <class Op>
__device__ __forceinline__ void fill_diag_tables(float *dtab, float *itab, float cc)
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid < 8) {
        const float d = Op::diag((uint8_t)tid, cc);
        dtab[tid] = d;
        itab[tid] = d > 0.f ? 1.f / d : 0.f;
    }
}

// Update over the active tiles (128 x 8 of one plane), persistent grid striding
// over the ordered tile list. A thread touches its quad only when the tile's
// quad-activity word says the quad holds an active element, so the quads of a
// tile outside the liquid (or the fluid faces) cost no traffic; the next tile's
// list entry and activity word are loaded a tile ahead. Jacobi (JAC):
// x += alpha p, z -= alpha D^-1 Ap, with r.z = sum d z^2 and r.r = sum d^2 z^2.
// Otherwise: x += alpha p, r -= alpha Ap, r.r. The last block counts the
// iteration, decides convergence and (Jacobi) forms beta.
template <class Op, bool JAC>
__global__ void __launch_bounds__(256) k_update_q(float *x, float *r, const float *__restrict__ p,
                                                  const float *__restrict__ q, const uint8_t *__restrict__ fl,
                                                  const int *__restrict__ list, const unsigned *__restrict__ qmask,
                                                  int nact, TileMap M, float cc, SolveScal *s, double *partials)
{
    if (s->done) return;
    __shared__ float dtab[8], itab[8];
    if (JAC) {
        fill_diag_tables<Op>(dtab, itab, cc);
        __syncthreads();
    }
    const float alpha = (float)s->alpha;
    const int tx = threadIdx.x, ty = threadIdx.y;
    KSum rz, rr;
    int idx = blockIdx.x;
    int b = idx < nact ? __ldg(list + idx) : 0;
    unsigned qm = idx < nact ? __ldg(qmask + (size_t)idx * TILE_Y + ty) : 0u;
    while (idx < nact) {
        const int nidx = idx + gridDim.x;
        const int bn = nidx < nact ? __ldg(list + nidx) : 0;
        const unsigned qmn = nidx < nact ? __ldg(qmask + (size_t)nidx * TILE_Y + ty) : 0u;
        if ((qm >> tx) & 1u) {
            int v, k, tyi, txi;
            M.decode(b, v, k, tyi, txi);
            const int t = M.origin0 + v * M.vstride + k * M.PL + (tyi * TILE_Y + ty) * M.P + txi * TILE_X + 4 * tx;
            const uchar4 f = __ldg(reinterpret_cast<const uchar4 *>(fl + t));
            const float4 cx = *reinterpret_cast<const float4 *>(x + t);
            const float4 cr = *reinterpret_cast<const float4 *>(r + t);
            const float4 cp = ld4(p, t), cq = ld4(q, t);
            const float4 xv = fma4(cx, alpha, cp);
            float4 rv = cr;
            if (JAC) {
                rv.x -= alpha * itab[f.x & 7] * cq.x;
                rv.y -= alpha * itab[f.y & 7] * cq.y;
                rv.z -= alpha * itab[f.z & 7] * cq.z;
                rv.w -= alpha * itab[f.w & 7] * cq.w;
                const float ax = dtab[f.x & 7] * rv.x, ay = dtab[f.y & 7] * rv.y;
                const float az = dtab[f.z & 7] * rv.z, aw = dtab[f.w & 7] * rv.w;
                rz.add(ax * rv.x + ay * rv.y + az * rv.z + aw * rv.w);
                rr.add(ax * ax + ay * ay + az * az + aw * aw);
            } else {
                rv = fma4(rv, -alpha, cq);
                rr.add(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
            }
            *reinterpret_cast<float4 *>(x + t) = xv;
            *reinterpret_cast<float4 *>(r + t) = rv;
        }
        b = bn;
        qm = qmn;
        idx = nidx;
    }
    KSum vv[2] = {rr, rz};
    double tot[2];
    if (grid_reduce<2>(vv, partials, &s->ticket, tot) && threadIdx.x == 0 && threadIdx.y == 0) {
        s->iter += 1;
        s->rr = tot[0];
        if (!isfinite(tot[0]) || !isfinite(tot[1])) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (tot[0] <= s->tol2 * s->bb) { s->done = 1; s->status = FS_OK; }
        else if (s->iter >= s->maxit) { s->done = 1; s->status = FS_ENOCONV; }
        else if (JAC) {
            s->beta = tot[1] / s->rz;
            s->rz = tot[1];
        }
    }
}

}  // namespace
}  // namespace fs
