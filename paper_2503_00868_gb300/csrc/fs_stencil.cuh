// fs_stencil.cuh -- the two CG kernels of both solves as plane-tiled stencils
// (included by fs_pcg.cu, which defines PoisOp and HelmOp).
//
// A tile is 128 x 8 columns (each of the 32 x 8 threads a 16-byte quad of 4
// consecutive x elements) of ONE plane of one volume. `list` holds, in order
// (x fastest, then y, plane, volume), the tiles that contain an active element.
// A persistent grid (as many blocks as fit on the SMs) strides over the list;
// each thread issues all loads of a tile at once, and the next list entry is
// fetched a tile ahead.
//   * p = z + beta p_old is formed for the tile and a one-element halo (rows above
//     and below as quads, the two side columns as scalars) into shared memory;
//   * x and y neighbours come from shared memory; the two z neighbours are formed
//     from their own loads, which blocks working on the neighbouring planes (a
//     few list entries away, at the same time) have just brought into L2.
// Inactive entries of z, p and Ap hold zero, so no load waits on a flag byte;
// stores touch only quads holding an active element.
//
// With the Jacobi preconditioner the solver keeps the scaled residual
// z = D^-1 r instead of r (the update is z -= alpha D^-1 Ap, and r.z = sum d z^2,
// r.r = sum d^2 z^2), so the direction update needs no division.
#pragma once

namespace fs {
namespace {

constexpr int SM_W = TILE_X + 8;  // plane row: [3] left halo, [4, 4 + TILE_X) data, [4 + TILE_X] right halo

__device__ __forceinline__ float4 ld4(const float *__restrict__ p, int t)
{
    return __ldg(reinterpret_cast<const float4 *>(p + t));
}

__device__ __forceinline__ float4 fma4(float4 a, float b, float4 c)  // a + b c
{
    return make_float4(a.x + b * c.x, a.y + b * c.y, a.z + b * c.z, a.w + b * c.w);
}

__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

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

// Where a thread's quad and its halo element of tile b lie.
struct TilePos {
    int t;        // own quad (first element), -1 when outside the volume
    int h;        // halo element / quad, -1 when this thread has none
    int hkind;    // 1 quad row, 2 scalar column
    int hrow, hcol;
};

__device__ __forceinline__ TilePos tile_pos(const TileMap &M, int b)
{
    int v, k, tyi, txi;
    M.decode(b, v, k, tyi, txi);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = txi * TILE_X, j0 = tyi * TILE_Y;
    const int i = i0 + 4 * tx, j = j0 + ty;
    const int org = M.origin0 + v * M.vstride + k * M.PL;
    TilePos p;
    p.t = (i < M.P && j < M.R) ? org + j * M.P + i : -1;
    p.h = -1;
    p.hkind = 0;
    p.hrow = p.hcol = 0;
    // warp 0 the row below, warp 1 the row above (quads); warp 2 lanes 0-7 the
    // left column, lanes 8-15 the right column (scalars)
    if (ty == 0 && i < M.P) {
        p.h = org + (j0 - 1) * M.P + i; p.hkind = 1; p.hrow = 0; p.hcol = 4 + 4 * tx;
    } else if (ty == 1 && i < M.P && j0 + TILE_Y <= M.R) {
        p.h = org + (j0 + TILE_Y) * M.P + i; p.hkind = 1; p.hrow = TILE_Y + 1; p.hcol = 4 + 4 * tx;
    } else if (ty == 2 && tx < TILE_Y && j0 + tx <= M.R) {
        p.h = org + (j0 + tx) * M.P + i0 - 1; p.hkind = 2; p.hrow = tx + 1; p.hcol = 3;
    } else if (ty == 2 && tx >= TILE_Y && tx < 2 * TILE_Y && j0 + tx - TILE_Y <= M.R && i0 + TILE_X <= M.P) {
        p.h = org + (j0 + tx - TILE_Y) * M.P + i0 + TILE_X; p.hkind = 2; p.hrow = tx - TILE_Y + 1; p.hcol = 4 + TILE_X;
    }
    return p;
}

// Everything one thread loads for one tile of the operator apply.
struct SpLoad {
    TilePos pos;
    uchar4 f;
    float4 zc, oc, zm, om, zp, op, hz, ho;
};

__device__ __forceinline__ void sp_issue(SpLoad &a, const TileMap &M, int b, const float *__restrict__ z,
                                         const float *__restrict__ pold, const uint8_t *__restrict__ fl)
{
    a.pos = tile_pos(M, b);
    const int t = a.pos.t;
    if (t >= 0) {
        a.f = __ldg(reinterpret_cast<const uchar4 *>(fl + t));
        a.zc = ld4(z, t); a.oc = ld4(pold, t);
        a.zm = ld4(z, t - M.PL); a.om = ld4(pold, t - M.PL);
        a.zp = ld4(z, t + M.PL); a.op = ld4(pold, t + M.PL);
    } else {
        a.f = make_uchar4(0, 0, 0, 0);
        a.zc = a.oc = a.zm = a.om = a.zp = a.op = zero4();
    }
    if (a.pos.hkind == 1) {
        a.hz = ld4(z, a.pos.h); a.ho = ld4(pold, a.pos.h);
    } else if (a.pos.hkind == 2) {
        a.hz = make_float4(__ldg(z + a.pos.h), 0.f, 0.f, 0.f);
        a.ho = make_float4(__ldg(pold + a.pos.h), 0.f, 0.f, 0.f);
    }
}

// p_new = z + beta p_old; q = A p_new; partial sums of p_new . q; alpha at the end.
template <class Op>
__global__ void __launch_bounds__(256) k_spmv_p(const float *__restrict__ z, const float *__restrict__ pold,
                                                float *__restrict__ pnew, float *__restrict__ q,
                                                const uint8_t *__restrict__ fl, const int *__restrict__ list,
                                                int nact, TileMap M, float cc, SolveScal *s, double *partials)
{
    if (s->done) return;
    __shared__ __align__(16) float sm[TILE_Y + 2][SM_W];
    __shared__ float dtab[8], itab[8];
    KSum acc;
    fill_diag_tables<Op>(dtab, itab, cc);
    const float beta = (float)s->beta;
    const float oc = Op::offc(cc);
    const int tx = threadIdx.x, ty = threadIdx.y;
    int idx = blockIdx.x;
    int b = idx < nact ? __ldg(list + idx) : 0;
    while (idx < nact) {
        const int nidx = idx + gridDim.x;
        const int bn = nidx < nact ? __ldg(list + nidx) : 0;  // next tile index, fetched early
        SpLoad cur;
        sp_issue(cur, M, b, z, pold, fl);
        // this tile
        const float4 pc = fma4(cur.zc, beta, cur.oc);
        *reinterpret_cast<float4 *>(&sm[ty + 1][4 + 4 * tx]) = pc;
        if (cur.pos.hkind == 1)
            *reinterpret_cast<float4 *>(&sm[cur.pos.hrow][cur.pos.hcol]) = fma4(cur.hz, beta, cur.ho);
        else if (cur.pos.hkind == 2)
            sm[cur.pos.hrow][cur.pos.hcol] = cur.hz.x + beta * cur.ho.x;
        __syncthreads();
        const uchar4 fc = cur.f;
        if (cur.pos.t >= 0 && ((fc.x | fc.y | fc.z | fc.w) & Op::ACTIVE)) {
            const float4 pm = fma4(cur.zm, beta, cur.om), pp = fma4(cur.zp, beta, cur.op);
            const float4 dn = *reinterpret_cast<const float4 *>(&sm[ty][4 + 4 * tx]);
            const float4 up = *reinterpret_cast<const float4 *>(&sm[ty + 2][4 + 4 * tx]);
            const float lf = sm[ty + 1][3 + 4 * tx], rt = sm[ty + 1][8 + 4 * tx];
            float4 qv;
            qv.x = (fc.x & Op::ACTIVE) ? dtab[fc.x & 7] * pc.x - oc * ((lf + pc.y) + (dn.x + up.x) + (pm.x + pp.x)) : 0.f;
            qv.y = (fc.y & Op::ACTIVE) ? dtab[fc.y & 7] * pc.y - oc * ((pc.x + pc.z) + (dn.y + up.y) + (pm.y + pp.y)) : 0.f;
            qv.z = (fc.z & Op::ACTIVE) ? dtab[fc.z & 7] * pc.z - oc * ((pc.y + pc.w) + (dn.z + up.z) + (pm.z + pp.z)) : 0.f;
            qv.w = (fc.w & Op::ACTIVE) ? dtab[fc.w & 7] * pc.w - oc * ((pc.z + rt) + (dn.w + up.w) + (pm.w + pp.w)) : 0.f;
            *reinterpret_cast<float4 *>(pnew + cur.pos.t) = pc;
            *reinterpret_cast<float4 *>(q + cur.pos.t) = qv;
            acc.add(pc.x * qv.x + pc.y * qv.y + pc.z * qv.z + pc.w * qv.w);
        }
        __syncthreads();  // the next tile reuses the plane buffer
        b = bn;
        idx = nidx;
    }
    double vv[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(vv, partials, &s->ticket, tot) && threadIdx.x == 0 && threadIdx.y == 0) {
        const double pq = tot[0];
        s->pq = pq;
        if (!isfinite(pq)) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (!(pq > 0.0)) { s->done = 1; s->status = FS_EBREAKDOWN; }
        else s->alpha = s->rz / pq;
    }
}

struct UpLoad {
    int t;
    uchar4 f;
    float4 x, r, p, q;
};

__device__ __forceinline__ void up_issue(UpLoad &a, const TileMap &M, int b, const float *x, const float *r,
                                         const float *__restrict__ p, const float *__restrict__ q,
                                         const uint8_t *__restrict__ fl)
{
    int v, k, tyi, txi;
    M.decode(b, v, k, tyi, txi);
    const int i = txi * TILE_X + 4 * threadIdx.x, j = tyi * TILE_Y + threadIdx.y;
    a.t = (i < M.P && j < M.R) ? M.origin0 + v * M.vstride + k * M.PL + j * M.P + i : -1;
    if (a.t >= 0) {
        a.f = __ldg(reinterpret_cast<const uchar4 *>(fl + a.t));
        a.x = *reinterpret_cast<const float4 *>(x + a.t);
        a.r = *reinterpret_cast<const float4 *>(r + a.t);
        a.p = ld4(p, a.t);
        a.q = ld4(q, a.t);
    } else {
        a.f = make_uchar4(0, 0, 0, 0);
    }
}

// Jacobi (JAC): x += alpha p, z -= alpha D^-1 Ap, with r.z = sum d z^2 and
// r.r = sum d^2 z^2. Otherwise: x += alpha p, r -= alpha Ap, r.r. The last block
// counts the iteration, decides convergence and (Jacobi) forms beta.
template <class Op, bool JAC>
__global__ void __launch_bounds__(256) k_update_p(float *x, float *r, const float *__restrict__ p,
                                                  const float *__restrict__ q, const uint8_t *__restrict__ fl,
                                                  const int *__restrict__ list, int nact, TileMap M, float cc,
                                                  SolveScal *s, double *partials)
{
    if (s->done) return;
    __shared__ float dtab[8], itab[8];
    KSum rz, rr;
    if (JAC) {
        fill_diag_tables<Op>(dtab, itab, cc);
        __syncthreads();
    }
    const float alpha = (float)s->alpha;
    int idx = blockIdx.x;
    int b = idx < nact ? __ldg(list + idx) : 0;
    while (idx < nact) {
        const int nidx = idx + gridDim.x;
        const int bn = nidx < nact ? __ldg(list + nidx) : 0;  // next tile index, fetched early
        UpLoad cur;
        up_issue(cur, M, b, x, r, p, q, fl);
        const uchar4 f = cur.f;
        if (cur.t >= 0 && ((f.x | f.y | f.z | f.w) & Op::ACTIVE)) {
            const float4 xv = fma4(cur.x, alpha, cur.p);
            float4 rv = cur.r;
            if (JAC) {
                rv.x -= alpha * itab[f.x & 7] * cur.q.x;
                rv.y -= alpha * itab[f.y & 7] * cur.q.y;
                rv.z -= alpha * itab[f.z & 7] * cur.q.z;
                rv.w -= alpha * itab[f.w & 7] * cur.q.w;
                const float ax = dtab[f.x & 7] * rv.x, ay = dtab[f.y & 7] * rv.y;
                const float az = dtab[f.z & 7] * rv.z, aw = dtab[f.w & 7] * rv.w;
                rz.add(ax * rv.x + ay * rv.y + az * rv.z + aw * rv.w);
                rr.add(ax * ax + ay * ay + az * az + aw * aw);
            } else {
                rv = fma4(rv, -alpha, cur.q);
                rr.add(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
            }
            *reinterpret_cast<float4 *>(x + cur.t) = xv;
            *reinterpret_cast<float4 *>(r + cur.t) = rv;
        }
        b = bn;
        idx = nidx;
    }
    double vv[2] = {rr.value(), rz.value()}, tot[2];
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
