// fs_mg.cu -- geometric multigrid V-cycle as the preconditioner of the pressure
// CG (z = M r for the 7-point operator of Sec. 3.2.2's projection). The paper
// solves the projection with a fitted recurrent network (Sec. 3.4.1); this
// preconditioner is the library's own choice for speed, and the solve still
// stops at the same tolerance on the same operator, so it changes the number of
// iterations, not what the projection computes.
//
// Levels. Level 0 is the cell space of the context (flags CF_LIQ, CF_AIR and the
// neighbour count CF_D). A coarse cell covers 2 x 2 x 2 cells of the level above
// (cells beyond an odd edge count as solid): it is air (a Dirichlet cell, p = 0)
// when any child is air, else liquid when any child is liquid, else solid. Each
// coarse level stores the same flag bits, with its own neighbour counts, in a
// dense array with a one-cell solid halo. The operator on level l is the same
// 7-point stencil rediscretised on cells of size 2^l dx, i.e. scaled by 4^-l.
//
// V-cycle on level l for A_l e = r: two damped Jacobi sweeps from e = 0
// (omega = 0.8), the residual, restriction (the transpose of cell-centred
// trilinear prolongation, divided by 8), the V-cycle on level l + 1, prolongation
// of its correction (weights 3/4 and 1/4 per axis), and two more sweeps. The
// coarsest level (small enough for shared memory) takes a fixed number of sweeps
// in one block. Every step is linear in r with symmetric smoothing and restriction
// proportional to the transposed prolongation, so M is symmetric, as CG needs.
//
// Every kernel runs densely over a level's whole array and writes zero on cells
// that are not liquid, so a stencil at the edge of the liquid reads zeros.
#include <cmath>
#include <new>

#include "fs_internal.cuh"

namespace fs {

constexpr int MG_MAX_LEVELS = 16;
constexpr int MG_COARSE_CELLS = 3072;  // padded cells of a level solved in shared memory
constexpr int MG_COARSE_SWEEPS = 30;
constexpr float MG_OMEGA = 0.8f;

// A level's array is `rows` rows of `sy` elements, `rpp` rows per plane; element
// e of row w is cell (e - ioff, w % rpp - joff, w / rpp - koff). Kernels walk
// rows (a warp along a row), so no element index is divided.
struct MgGrid {
    int nx, ny, nz;    // cells of the level
    int sy, sz;        // element strides of a row and a plane
    int origin;        // element of cell (0, 0, 0)
    int n;             // elements of the whole array (halo, padding and guards included)
    int rows, rpp, ioff, joff, koff;
    __host__ __device__ int idx(int i, int j, int k) const { return origin + k * sz + j * sy + i; }
};

#define MG_FOR_ROWS(g)                                                                                   \
    for (int row = blockIdx.x * blockDim.y + threadIdx.y; row < (g).rows; row += gridDim.x * blockDim.y) \
        for (int e = threadIdx.x; e < (g).sy; e += blockDim.x)

struct MgLevel {
    MgGrid g;
    float scale = 1.f;  // 4^-l
    uint8_t *fl = nullptr;
    float *r = nullptr, *a = nullptr, *b = nullptr, *c = nullptr;  // right-hand side and three work arrays
};

struct MgState {
    int nlev = 0;
    MgLevel lev[MG_MAX_LEVELS];
    long long epoch = -1;  // mask epoch the hierarchy was built for
};

namespace {

constexpr int TH = 256;
const dim3 RT(32, 8);  // a warp along a row, 8 rows per block

__device__ __forceinline__ bool liq(uint8_t f) { return f & CF_LIQ; }

// A_l e at a liquid cell, without the scale
__device__ __forceinline__ float lap(const float *__restrict__ e, int t, uint8_t f, const MgGrid &g)
{
    return (float)(f & CF_D) * e[t] - ((e[t - 1] + e[t + 1]) + (e[t - g.sy] + e[t + g.sy]) + (e[t - g.sz] + e[t + g.sz]));
}

// omega / (scale d) for d = 0..6 (zero for d = 0)
__device__ __forceinline__ void fill_wtab(float *wt, float scale)
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid < 8) wt[tid] = tid > 0 && tid < 7 ? MG_OMEGA / (scale * (float)tid) : 0.f;
    __syncthreads();
}

// the first two sweeps from e = 0 in one pass: e1 = omega D^-1 r is formed on
// the fly at the cell and its six neighbours, then e2 = e1 + omega D^-1 (r - A e1)
__global__ void __launch_bounds__(256) k_mg_smooth2(MgGrid g, const uint8_t *__restrict__ fl,
                                                    const float *__restrict__ r, float *eo, float scale)
{
    __shared__ float wt[8];
    fill_wtab(wt, scale);
    MG_FOR_ROWS(g)
    {
        const int t = row * g.sy + e;
        const uint8_t f = fl[t];
        float v = 0.f;
        if (liq(f)) {
            const int d = f & CF_D;
            auto e1 = [&](int u) {
                const uint8_t fu = fl[u];
                return liq(fu) ? wt[fu & CF_D] * r[u] : 0.f;
            };
            const float c1 = e1(t);
            const float nb = (e1(t - 1) + e1(t + 1)) + (e1(t - g.sy) + e1(t + g.sy)) + (e1(t - g.sz) + e1(t + g.sz));
            v = c1 + wt[d] * (r[t] - scale * ((float)d * c1 - nb));
        }
        eo[t] = v;
    }
}

// e_out = e_in + omega D^-1 (r - A e_in)
__global__ void __launch_bounds__(256) k_mg_smooth(MgGrid g, const uint8_t *__restrict__ fl,
                                                   const float *__restrict__ r, const float *__restrict__ ein,
                                                   float *eout, float scale)
{
    __shared__ float wt[8];
    fill_wtab(wt, scale);
    MG_FOR_ROWS(g)
    {
        const int t = row * g.sy + e;
        const uint8_t f = fl[t];
        eout[t] = liq(f) ? ein[t] + wt[f & CF_D] * (r[t] - scale * lap(ein, t, f, g)) : 0.f;
    }
}

// res = r - A e
__global__ void __launch_bounds__(256) k_mg_residual(MgGrid g, const uint8_t *__restrict__ fl,
                                                     const float *__restrict__ r, const float *__restrict__ ev,
                                                     float *res, float scale)
{
    MG_FOR_ROWS(g)
    {
        const int t = row * g.sy + e;
        const uint8_t f = fl[t];
        res[t] = liq(f) ? r[t] - scale * lap(ev, t, f, g) : 0.f;
    }
}

// coarse r = (1/8) sum over the 4 x 4 x 4 fine window of w_a w_b w_c res_fine,
// w = (1/4, 3/4, 3/4, 1/4) at fine indices 2I - 1 .. 2I + 2
__global__ void __launch_bounds__(256) k_mg_restrict(MgGrid gf, const float *__restrict__ res, MgGrid gc,
                                                     const uint8_t *__restrict__ flc, float *rc)
{
    const float w[4] = {0.25f, 0.75f, 0.75f, 0.25f};
    MG_FOR_ROWS(gc)
    {
        const int t = row * gc.sy + e;
        float acc = 0.f;
        if (liq(flc[t])) {
            const int I = e - gc.ioff, J = row % gc.rpp - gc.joff, K = row / gc.rpp - gc.koff;
            for (int c = 0; c < 4; c++) {
                const int k = 2 * K - 1 + c;
                if (k < 0 || k >= gf.nz) continue;
                for (int b = 0; b < 4; b++) {
                    const int j = 2 * J - 1 + b;
                    if (j < 0 || j >= gf.ny) continue;
                    const int frow = gf.idx(0, j, k);
                    float sr = 0.f;
#pragma unroll
                    for (int a = 0; a < 4; a++) {
                        const int i = 2 * I - 1 + a;
                        if (i >= 0 && i < gf.nx) sr += w[a] * res[frow + i];
                    }
                    acc += w[c] * w[b] * sr;
                }
            }
            acc *= 0.125f;
        }
        rc[t] = acc;
    }
}

// e_fine += P e_coarse on liquid fine cells (in place)
__global__ void __launch_bounds__(256) k_mg_prolong(MgGrid gf, const uint8_t *__restrict__ fl, float *ef,
                                                    MgGrid gc, const float *__restrict__ ec)
{
    MG_FOR_ROWS(gf)
    {
        const int t = row * gf.sy + e;
        if (!liq(fl[t])) continue;
        const int i = e - gf.ioff, j = row % gf.rpp - gf.joff, k = row / gf.rpp - gf.koff;
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        const int I2 = (i & 1) ? I + 1 : I - 1, J2 = (j & 1) ? J + 1 : J - 1, K2 = (k & 1) ? K + 1 : K - 1;
        // coarse indices -1 and n land in the coarse halo, which holds zeros
        const float v = 0.421875f * ec[gc.idx(I, J, K)] +
                        0.140625f * (ec[gc.idx(I2, J, K)] + ec[gc.idx(I, J2, K)] + ec[gc.idx(I, J, K2)]) +
                        0.046875f * (ec[gc.idx(I2, J2, K)] + ec[gc.idx(I2, J, K2)] + ec[gc.idx(I, J2, K2)]) +
                        0.015625f * ec[gc.idx(I2, J2, K2)];
        ef[t] += v;
    }
}

// coarse flags from the level above: air if any child is air, else liquid if any
// child is liquid; the halo stays solid (zero)
__global__ void k_mg_coarsen(MgGrid gf, const uint8_t *__restrict__ flf, MgGrid gc, uint8_t *flc)
{
    MG_FOR_ROWS(gc)
    {
        const int t = row * gc.sy + e;
        const int I = e - gc.ioff, J = row % gc.rpp - gc.joff, K = row / gc.rpp - gc.koff;
        uint8_t out = 0;
        if (I >= 0 && J >= 0 && K >= 0 && I < gc.nx && J < gc.ny && K < gc.nz) {
            bool air = false, lq = false;
            for (int c = 0; c < 2; c++)
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++) {
                        const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;
                        if (i >= gf.nx || j >= gf.ny || k >= gf.nz) continue;
                        const uint8_t f = flf[gf.idx(i, j, k)];
                        air |= (f & CF_AIR) != 0;
                        lq |= (f & CF_LIQ) != 0;
                    }
            out = air ? CF_AIR : (lq ? CF_LIQ : 0);
        }
        flc[t] = out;
    }
}

// neighbour counts of the liquid cells: neighbours that are liquid or air
__global__ void k_mg_count(MgGrid g, uint8_t *fl)
{
    MG_FOR_ROWS(g)
    {
        const int t = row * g.sy + e;
        const uint8_t f = fl[t];
        if (!liq(f)) continue;
        const int off[6] = {-1, 1, -g.sy, g.sy, -g.sz, g.sz};
        int d = 0;
#pragma unroll
        for (int m = 0; m < 6; m++) d += (fl[t + off[m]] & (CF_LIQ | CF_AIR)) ? 1 : 0;
        fl[t] = (uint8_t)((f & ~CF_D) | d);
    }
}

// coarsest level: MG_COARSE_SWEEPS damped Jacobi sweeps from zero, in shared memory
__global__ void __launch_bounds__(TH) k_mg_coarse(MgGrid g, const uint8_t *__restrict__ fl,
                                                  const float *__restrict__ r, float *e, float scale)
{
    extern __shared__ float sm[];
    float *e0 = sm, *e1 = sm + g.n, *rs = sm + 2 * g.n;
    uint8_t *fs = reinterpret_cast<uint8_t *>(sm + 3 * g.n);
    for (int t = threadIdx.x; t < g.n; t += TH) {
        fs[t] = fl[t];
        rs[t] = r[t];
        const int d = fl[t] & CF_D;
        e0[t] = (liq(fl[t]) && d > 0) ? MG_OMEGA * r[t] / (scale * (float)d) : 0.f;
        e1[t] = 0.f;
    }
    __syncthreads();
    for (int s = 1; s < MG_COARSE_SWEEPS; s++) {
        const float *ein = (s & 1) ? e0 : e1;
        float *eout = (s & 1) ? e1 : e0;
        for (int t = threadIdx.x; t < g.n; t += TH) {
            const uint8_t f = fs[t];
            const int d = f & CF_D;
            float v = 0.f;
            if (liq(f) && d > 0) v = ein[t] + MG_OMEGA * (rs[t] - scale * lap(ein, t, f, g)) / (scale * (float)d);
            eout[t] = v;
        }
        __syncthreads();
    }
    const float *res = (MG_COARSE_SWEEPS & 1) ? e0 : e1;  // the last sweep's output
    for (int t = threadIdx.x; t < g.n; t += TH) e[t] = res[t];
}

size_t coarse_smem(const MgGrid &g) { return (size_t)g.n * 13 + 16; }

int launch_blocks(fs_ctx *c, long long n) { return grid_blocks(c, n, TH); }
int row_blocks(fs_ctx *c, const MgGrid &g) { return grid_blocks(c, g.rows, 8); }

MgGrid level0_grid(const Layout &L)
{
    MgGrid g;
    g.nx = L.nx;
    g.ny = L.ny;
    g.nz = L.nz;
    g.sy = L.P;
    g.sz = L.PL;
    g.origin = L.PL;
    g.n = L.nC;
    g.rows = L.nC / L.P;
    g.rpp = L.R;
    g.ioff = 0;
    g.joff = 0;
    g.koff = 1;
    return g;
}

MgGrid coarse_grid(int nx, int ny, int nz)
{
    MgGrid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.sy = nx + 2;
    g.sz = (nx + 2) * (ny + 2);
    g.origin = g.sz + g.sy + 1;
    g.n = g.sz * (nz + 2);
    g.rows = (ny + 2) * (nz + 2);
    g.rpp = ny + 2;
    g.ioff = 1;
    g.joff = 1;
    g.koff = 1;
    return g;
}

void free_levels(MgState *s)
{
    for (int l = 1; l < s->nlev; l++) {
        MgLevel &v = s->lev[l];
        cudaFree(v.fl);
        cudaFree(v.r);
        cudaFree(v.a);
        cudaFree(v.b);
        cudaFree(v.c);
        v = MgLevel();
    }
    cudaFree(s->lev[0].b);
    cudaFree(s->lev[0].c);
    s->lev[0] = MgLevel();
    s->nlev = 0;
    s->epoch = -1;
}

// The V-cycle on level l: r in lev[l].r (level 0: the given r), result in lev[l].a
// (level 0: the given z).
int vcycle(fs_ctx *c, MgState *s, int l)
{
    MgLevel &v = s->lev[l];
    const MgGrid &g = v.g;
    if (l == s->nlev - 1) {
        k_mg_coarse<<<1, TH, coarse_smem(g), c->stream>>>(g, v.fl, v.r, v.a, v.scale);
        c->n_launches += 1;
        return FS_OK;
    }
    const int nb = row_blocks(c, g);
    k_mg_smooth2<<<nb, RT, 0, c->stream>>>(g, v.fl, v.r, v.b, v.scale);
    k_mg_residual<<<nb, RT, 0, c->stream>>>(g, v.fl, v.r, v.b, v.c, v.scale);
    MgLevel &w = s->lev[l + 1];
    k_mg_restrict<<<row_blocks(c, w.g), RT, 0, c->stream>>>(g, v.c, w.g, w.fl, w.r);
    c->n_launches += 3;
    if (int rc = vcycle(c, s, l + 1)) return rc;
    k_mg_prolong<<<nb, RT, 0, c->stream>>>(g, v.fl, v.b, w.g, w.a);
    k_mg_smooth<<<nb, RT, 0, c->stream>>>(g, v.fl, v.r, v.b, v.c, v.scale);
    k_mg_smooth<<<nb, RT, 0, c->stream>>>(g, v.fl, v.r, v.c, v.a, v.scale);
    c->n_launches += 3;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

}  // namespace

void mg_free(fs_ctx *c)
{
    MgState *s = static_cast<MgState *>(c->mg);
    if (!s) return;
    free_levels(s);
    delete s;
    c->mg = nullptr;
}

// Builds the hierarchy for the current mask (once per mask).
static int mg_build(fs_ctx *c, MgState *s)
{
    free_levels(s);
    const Layout &L = c->L;
    MgLevel &l0 = s->lev[0];
    l0.g = level0_grid(L);
    l0.scale = 1.f;
    l0.fl = c->cflag;
    s->nlev = 1;
    auto fail = [&](const char *what) {
        cudaGetLastError();
        free_levels(s);
        return set_error(FS_ENOMEM, "multigrid %s", what);
    };
    if (cudaMalloc(&l0.b, (size_t)L.nC * 4) != cudaSuccess || cudaMalloc(&l0.c, (size_t)L.nC * 4) != cudaSuccess)
        return fail("level-0 work arrays");
    FS_CUDA(cudaMemsetAsync(l0.b, 0, (size_t)L.nC * 4, c->stream));
    FS_CUDA(cudaMemsetAsync(l0.c, 0, (size_t)L.nC * 4, c->stream));
    while (s->lev[s->nlev - 1].g.n > MG_COARSE_CELLS && s->nlev < MG_MAX_LEVELS) {
        const MgGrid &gf = s->lev[s->nlev - 1].g;
        MgLevel &v = s->lev[s->nlev];
        v.g = coarse_grid((gf.nx + 1) / 2, (gf.ny + 1) / 2, (gf.nz + 1) / 2);
        v.scale = s->lev[s->nlev - 1].scale * 0.25f;
        const size_t nb = (size_t)v.g.n;
        if (cudaMalloc(&v.fl, nb) != cudaSuccess || cudaMalloc(&v.r, nb * 4) != cudaSuccess ||
            cudaMalloc(&v.a, nb * 4) != cudaSuccess || cudaMalloc(&v.b, nb * 4) != cudaSuccess ||
            cudaMalloc(&v.c, nb * 4) != cudaSuccess) {
            s->nlev += 1;  // free what was allocated
            return fail("level arrays");
        }
        s->nlev += 1;
        for (float *p : {v.r, v.a, v.b, v.c}) FS_CUDA(cudaMemsetAsync(p, 0, nb * 4, c->stream));
        const int blocks = row_blocks(c, v.g);
        k_mg_coarsen<<<blocks, RT, 0, c->stream>>>(gf, s->lev[s->nlev - 2].fl, v.g, v.fl);
        k_mg_count<<<blocks, RT, 0, c->stream>>>(v.g, v.fl);
        c->n_launches += 2;
        FS_CUDA(cudaGetLastError());
        if (v.g.nx == 1 && v.g.ny == 1 && v.g.nz == 1) break;
    }
    if (s->lev[s->nlev - 1].g.n > MG_COARSE_CELLS)
        return set_error(FS_EINVAL, "multigrid: the coarsest level does not fit in shared memory");
    s->epoch = c->mask_epoch;
    return FS_OK;
}

// z = M r on the cell space (r and z of length nC, zero off the liquid).
int mg_apply(fs_ctx *c, const float *r, float *z)
{
    MgState *s = static_cast<MgState *>(c->mg);
    if (!s) {
        s = new (std::nothrow) MgState();
        if (!s) return set_error(FS_ENOMEM, "host allocation failed");
        c->mg = s;
    }
    if (s->epoch != c->mask_epoch)
        if (int rc = mg_build(c, s)) return rc;
    MgLevel &l0 = s->lev[0];
    l0.r = const_cast<float *>(r);
    l0.a = z;
    const int rc = vcycle(c, s, 0);
    l0.r = nullptr;
    l0.a = nullptr;
    return rc;
}

int mg_levels(const fs_ctx *c)
{
    const MgState *s = static_cast<const MgState *>(c->mg);
    return s ? s->nlev : 0;
}

}  // namespace fs
