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
// dense array with a solid halo (a plane and a row on each side, 4 elements
// before each row, the row pitch a multiple of 4). The operator on level l is the
// same 7-point stencil rediscretised on cells of size 2^l dx, i.e. scaled by 4^-l.
//
// V-cycle on level l for A_l e = r: two damped Jacobi sweeps from e = 0
// (omega = 0.8), the residual, restriction (the transpose of cell-centred
// trilinear prolongation, divided by 8), the V-cycle on level l + 1, prolongation
// of its correction (weights 3/4 and 1/4 per axis), and two more sweeps; one
// before and one after on a face volume's level 0, where the mass term of the
// Helmholtz operator makes the smoothing strong enough that the second costs more
// than the iterations it saves. The
// coarsest level (small enough for shared memory) takes a fixed number of sweeps
// in one block. Every step is linear in r with symmetric smoothing and restriction
// proportional to the transposed prolongation, so M is symmetric, as CG needs.
//
// The sweeps, the residual and the transfers take four elements per thread and
// walk a list of a level's quads that hold an unknown (built with the hierarchy).
// Every array a V-cycle writes is written only on those quads (with zeros on
// their other elements) and is zero on every other quad: the work arrays are
// zeroed when the hierarchy is built, and the level-0 output (the solver's z) is
// a context buffer that is zeroed with each new mask and that every writer
// leaves zero off the unknowns. So a stencil at the edge of the liquid reads
// zeros, and the solver's operator apply reads z = 0 off the unknowns.
//
// The same V-cycle preconditions the implicit viscosity solve, one velocity
// component at a time: each face volume is a box of unknown faces (FF_FLUID),
// prescribed faces (FF_FIXED, Dirichlet) and mirror faces (Neumann), whose flag
// bits coincide with the cell bits used here (FF_FLUID = CF_LIQ, FF_FIXED =
// CF_AIR, FF_N = CF_D), and the operator gains the mass term: A_l = m I +
// 4^-l cc L_l with m = 1 (m = 0 for the pressure).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fs_internal.cuh"

namespace fs {

constexpr int MG_MAX_LEVELS = 16;
constexpr int MG_COARSE_CELLS = 3072;  // padded cells of a level solved in shared memory
constexpr int MG_COARSE_SWEEPS = 30;
constexpr float MG_OMEGA = 0.8f;

// A level's array is `rows` rows of `sy` elements, `rpp` rows per plane; element
// e of row w is cell (e - ioff, w % rpp - joff, w / rpp - koff). The set-up
// kernels walk rows (a warp along a row), so they divide no element index.
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
    float scale = 1.f;  // 4^-l times the operator's coefficient
    float mass = 0.f;   // identity term (1 for the Helmholtz operator)
    uint8_t *fl = nullptr;
    float *r = nullptr, *a = nullptr, *b = nullptr, *c = nullptr;  // right-hand side and three work arrays
    int *ql = nullptr;  // active quads (every level but the coarsest)
    int nqa = 0;
    int *pl = nullptr;  // active restriction pairs of this level as the coarse one (levels >= 1)
    int npa = 0;
};

struct MgState {
    int nlev = 0;
    MgLevel lev[MG_MAX_LEVELS];
    long long epoch = -1;  // mask epoch the hierarchy was built for
    float coef = 0.f;      // operator coefficient it was built for
    bool own0 = true;      // level 0 work arrays belong to this hierarchy
    const int *done = nullptr;  // the calling solve's convergence flag (nullable)
    int cl = 0;                 // first level of the single-cluster launch (0: none)
    bool one0 = false;          // one smoothing sweep each side on level 0 (the face volumes)
    // r.z in the last level-0 sweep of the current apply (rzs null: not formed)
    SolveScal *rzs = nullptr;
    int rz_first = 0, rz_boff = 0, rz_btot = 0;
    int ctas = 0;               // CTAs of that cluster
    long long calls = 0;        // applies so far (profiling samples every prof_period-th)
    // algorithmic bytes of the level-0 kernels, in the order of K_MG0_SMOOTH2 ..
    // K_MG0_SMOOTH_Z (profiled when the first is > 0)
    double by0[6] = {0, 0, 0, 0, 0, 0};
};

// The pressure hierarchy and one per face volume (viscosity). The face volumes
// share two level-0 work arrays of face-space length, and their V-cycles are
// independent: volumes 1 and 2 run on two side streams, forked from and joined
// back to the context's stream.
struct MgAll {
    MgState cell, face[3];
    float *fb = nullptr, *fc = nullptr;
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
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

// omega / (m + scale d), zero where the diagonal vanishes
__device__ __forceinline__ float wtab_entry(float scale, float m, int d)
{
    const float dg = m + scale * (float)d;
    return dg > 0.f ? MG_OMEGA / dg : 0.f;
}

// the table for d = 0..7 in shared memory
__device__ __forceinline__ void fill_wtab(float *wt, float scale, float m)
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid < 8) wt[tid] = wtab_entry(scale, m, tid);
    __syncthreads();
}

// ---- four elements per thread -------------------------------------------------
// Every level but the coarsest has a row pitch, plane stride and origin that are
// multiples of 4 (level 0 by the context's layout, a coarse level by its 4-element
// x halo), so a quad of 4 consecutive elements never crosses a row and its
// float4 / uchar4 loads are aligned. A quad without an unknown is skipped; a quad
// with one is read whole (its row is interior, so every neighbour load is inside
// the array) and written whole, with zeros on the elements that are not unknowns.

__device__ __forceinline__ uchar4 ldf4(const uint8_t *__restrict__ p, int t)
{
    return __ldg(reinterpret_cast<const uchar4 *>(p + t));
}
__device__ __forceinline__ bool any_liq(uchar4 f) { return ((f.x | f.y | f.z | f.w) & CF_LIQ) != 0; }

// e_out on one element from e_in: c (centre), the sum of its six neighbours nb
__device__ __forceinline__ float sweep1(uint8_t f, float c, float nb, float rv, const float *wt, float scale, float m)
{
    return liq(f) ? c + wt[f & CF_D] * (rv - m * c - scale * ((float)(f & CF_D) * c - nb)) : 0.f;
}

// The kernels below walk a level's list of active quads (those holding an
// unknown, built with the hierarchy), each thread striding through it with the
// next entry fetched one step ahead: no flag load stands between a thread and its
// data loads, and the quads without an unknown cost nothing.
#define MG_FOR_LIST(list, na)                                                                            \
    for (int mg_i = blockIdx.x * blockDim.x + threadIdx.x, mg_st = gridDim.x * blockDim.x,               \
             q = mg_i < (na) ? __ldg((list) + mg_i) : 0, mg_next = 0;                                    \
         mg_i < (na) && ((mg_next = mg_i + mg_st < (na) ? __ldg((list) + mg_i + mg_st) : 0), true);     \
         mg_i += mg_st, q = mg_next)

// Vector loads of the item functions: through the non-coherent path for a launch
// that does not write what it reads (CG = false), or at L2 (CG = true) for the
// cluster launch, whose CTAs read what others wrote before a cluster barrier.
template <bool CG>
__device__ __forceinline__ float4 ldv4(const float *p, int t)
{
    if constexpr (CG)
        return __ldcg(reinterpret_cast<const float4 *>(p + t));
    else
        return __ldg(reinterpret_cast<const float4 *>(p + t));
}
template <bool CG>
__device__ __forceinline__ float ldv1(const float *p, int t)
{
    if constexpr (CG)
        return __ldcg(p + t);
    else
        return __ldg(p + t);
}

// one damped Jacobi sweep on quad q: eout from ein; returns r.eout over the quad
template <bool CG>
__device__ __forceinline__ float smooth_q(const MgGrid &g, const uint8_t *__restrict__ fl, const float *r,
                                          const float *ein, float *eout, const float *wt, float scale, float m, int q)
{
    const int t = q << 2;
    const uchar4 f = ldf4(fl, t);
    const float4 c = ldv4<CG>(ein, t), rv = ldv4<CG>(r, t);
    const float4 dn = ldv4<CG>(ein, t - g.sy), up = ldv4<CG>(ein, t + g.sy);
    const float4 bk = ldv4<CG>(ein, t - g.sz), fw = ldv4<CG>(ein, t + g.sz);
    const float lf = ldv1<CG>(ein, t - 1), rt = ldv1<CG>(ein, t + 4);
    float4 v;
    v.x = sweep1(f.x, c.x, (lf + c.y) + (dn.x + up.x) + (bk.x + fw.x), rv.x, wt, scale, m);
    v.y = sweep1(f.y, c.y, (c.x + c.z) + (dn.y + up.y) + (bk.y + fw.y), rv.y, wt, scale, m);
    v.z = sweep1(f.z, c.z, (c.y + c.w) + (dn.z + up.z) + (bk.z + fw.z), rv.z, wt, scale, m);
    v.w = sweep1(f.w, c.w, (c.z + rt) + (dn.w + up.w) + (bk.w + fw.w), rv.w, wt, scale, m);
    *reinterpret_cast<float4 *>(eout + t) = v;
    return rv.x * v.x + rv.y * v.y + rv.z * v.z + rv.w * v.w;
}

// res = r - A e on quad q
template <bool CG>
__device__ __forceinline__ void resid_q(const MgGrid &g, const uint8_t *__restrict__ fl, const float *r,
                                        const float *ev, float *res, float scale, float m, int q)
{
    const int t = q << 2;
    const uchar4 f = ldf4(fl, t);
    const float4 c = ldv4<CG>(ev, t), rv = ldv4<CG>(r, t);
    const float4 dn = ldv4<CG>(ev, t - g.sy), up = ldv4<CG>(ev, t + g.sy);
    const float4 bk = ldv4<CG>(ev, t - g.sz), fw = ldv4<CG>(ev, t + g.sz);
    const float lf = ldv1<CG>(ev, t - 1), rt = ldv1<CG>(ev, t + 4);
    auto one = [&](uint8_t fe, float ce, float nb, float re) {
        return liq(fe) ? re - m * ce - scale * ((float)(fe & CF_D) * ce - nb) : 0.f;
    };
    float4 v;
    v.x = one(f.x, c.x, (lf + c.y) + (dn.x + up.x) + (bk.x + fw.x), rv.x);
    v.y = one(f.y, c.y, (c.x + c.z) + (dn.y + up.y) + (bk.y + fw.y), rv.y);
    v.z = one(f.z, c.z, (c.y + c.w) + (dn.z + up.z) + (bk.z + fw.z), rv.z);
    v.w = one(f.w, c.w, (c.z + rt) + (dn.w + up.w) + (bk.w + fw.w), rv.w);
    *reinterpret_cast<float4 *>(res + t) = v;
}

// the first two sweeps from e = 0 on quad q: e1 = omega D^-1 r on the fly, then one sweep
template <bool CG>
__device__ __forceinline__ void smooth2_q(const MgGrid &g, const uint8_t *__restrict__ fl, const float *r, float *eo,
                                          const float *wt, float scale, float m, int q)
{
    const int t = q << 2;
    const uchar4 f = ldf4(fl, t);
    auto e1q = [&](int u) {  // e1 on the quad at u
        const uchar4 fu = ldf4(fl, u);
        const float4 ru = ldv4<CG>(r, u);
        return make_float4(liq(fu.x) ? wt[fu.x & CF_D] * ru.x : 0.f, liq(fu.y) ? wt[fu.y & CF_D] * ru.y : 0.f,
                           liq(fu.z) ? wt[fu.z & CF_D] * ru.z : 0.f, liq(fu.w) ? wt[fu.w & CF_D] * ru.w : 0.f);
    };
    auto e1s = [&](int u) {
        const uint8_t fu = fl[u];
        return liq(fu) ? wt[fu & CF_D] * ldv1<CG>(r, u) : 0.f;
    };
    const float4 c = e1q(t), rv = ldv4<CG>(r, t);
    const float4 dn = e1q(t - g.sy), up = e1q(t + g.sy), bk = e1q(t - g.sz), fw = e1q(t + g.sz);
    const float lf = e1s(t - 1), rt = e1s(t + 4);
    float4 v;
    v.x = sweep1(f.x, c.x, (lf + c.y) + (dn.x + up.x) + (bk.x + fw.x), rv.x, wt, scale, m);
    v.y = sweep1(f.y, c.y, (c.x + c.z) + (dn.y + up.y) + (bk.y + fw.y), rv.y, wt, scale, m);
    v.z = sweep1(f.z, c.z, (c.y + c.w) + (dn.z + up.z) + (bk.z + fw.z), rv.z, wt, scale, m);
    v.w = sweep1(f.w, c.w, (c.z + rt) + (dn.w + up.w) + (bk.w + fw.w), rv.w, wt, scale, m);
    *reinterpret_cast<float4 *>(eo + t) = v;
}

// e_fine += P e_coarse on the unknowns of an active quad q (in place). The quad's
// elements i .. i + 3 (i a multiple of 4) take their x samples from coarse
// I0 - 1 .. I0 + 2 (I0 = i / 2); indices past the coarse halo are clamped to it
// (a sample that only padding elements use).
template <bool CG>
__device__ __forceinline__ void prolong_q(const MgGrid &gf, const uint8_t *__restrict__ fl, float *ef,
                                          const MgGrid &gc, const float *ec, int q)
{
    const int qrow = gf.sy >> 2;
    const int t = q << 2;
    const uchar4 f = ldf4(fl, t);
    const int row = q / qrow, e = (q - row * qrow) << 2;
    const int i = e - gf.ioff, j = row % gf.rpp - gf.joff, k = row / gf.rpp - gf.koff;
    const int I0 = i >> 1, J = j >> 1, K = k >> 1;
    const int J2 = (j & 1) ? J + 1 : J - 1, K2 = (k & 1) ? K + 1 : K - 1;
    const int xs[4] = {max(I0 - 1, -1), I0, min(I0 + 1, gc.nx), min(I0 + 2, gc.nx)};
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    const int jj[2] = {J, J2}, kk[2] = {K, K2};
    const float wy[2] = {0.75f, 0.25f};
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const int base = gc.idx(0, jj[a], kk[b]);
            const float w = wy[a] * wy[b];
            const float cm = ldv1<CG>(ec, base + xs[0]), c0 = ldv1<CG>(ec, base + xs[1]);
            const float c1 = ldv1<CG>(ec, base + xs[2]), c2 = ldv1<CG>(ec, base + xs[3]);
            s0 += w * (0.75f * c0 + 0.25f * cm);
            s1 += w * (0.75f * c0 + 0.25f * c1);
            s2 += w * (0.75f * c1 + 0.25f * c0);
            s3 += w * (0.75f * c1 + 0.25f * c2);
        }
    float4 v = CG ? __ldcg(reinterpret_cast<const float4 *>(ef + t)) : *reinterpret_cast<const float4 *>(ef + t);
    if (liq(f.x)) v.x += s0;
    if (liq(f.y)) v.y += s1;
    if (liq(f.z)) v.z += s2;
    if (liq(f.w)) v.w += s3;
    *reinterpret_cast<float4 *>(ef + t) = v;
}

// Restriction of an active pair of the coarse level: t0 is the element of coarse
// cell (2m, J, K), and the pair (2m, 2m + 1) holds at least one unknown. Per fine
// row of the 4 x 4 window it reads the aligned quad 4m .. 4m + 3 and the scalars
// at 4m - 1 and 4m + 4 (excluded at or past nx, where the next row begins), and
// forms both cells' x weights from them.
template <bool CG>
__device__ __forceinline__ void restrict_pair(const MgGrid &gf, const float *res, const MgGrid &gc,
                                              const uint8_t *__restrict__ flc, float *rc, int t0)
{
    const float w[4] = {0.25f, 0.75f, 0.75f, 0.25f};
    const int rel = t0 - gc.origin;
    const int K = rel / gc.sz, J = (rel - K * gc.sz) / gc.sy, I0 = rel - K * gc.sz - J * gc.sy;
    const int m = I0 >> 1;
    const bool l0 = liq(flc[t0]), l1 = I0 + 1 < gc.nx && liq(flc[t0 + 1]);
    float a0 = 0.f, a1 = 0.f;
    // unrolled, so the 16 row loads are issued together
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int k = 2 * K - 1 + c;
        if (k < 0 || k >= gf.nz) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int j = 2 * J - 1 + b;
            if (j < 0 || j >= gf.ny) continue;
            const int row = gf.idx(0, j, k) + 4 * m;  // a multiple of 4
            const float4 qd = ldv4<CG>(res, row);
            const float lf = m > 0 ? ldv1<CG>(res, row - 1) : 0.f;
            const float rt = 4 * m + 4 < gf.nx ? ldv1<CG>(res, row + 4) : 0.f;
            const float wyz = w[c] * w[b];
            // coarse 2m: fine 4m - 1 .. 4m + 2; coarse 2m + 1: fine 4m + 1 .. 4m + 4
            a0 += wyz * (0.25f * lf + 0.75f * qd.x + 0.75f * qd.y + 0.25f * qd.z);
            a1 += wyz * (0.25f * qd.y + 0.75f * qd.z + 0.75f * qd.w + 0.25f * rt);
        }
    }
    if (l0) rc[t0] = 0.125f * a0;
    if (l1) rc[t0 + 1] = 0.125f * a1;
}

// one damped Jacobi sweep from zero and the residual it leaves, on quad q:
// eb = e1 = omega D^-1 r at the quad, res = r - A e1 (e1 at the neighbours formed
// on the fly)
__device__ __forceinline__ void pre1_q(const MgGrid &g, const uint8_t *__restrict__ fl, const float *r, float *eb,
                                       float *res, const float *wt, float scale, float m, int q)
{
    const int t = q << 2;
    const uchar4 f = ldf4(fl, t);
    auto e1q = [&](int u) {  // e1 on the quad at u
        const uchar4 fu = ldf4(fl, u);
        const float4 ru = ldv4<false>(r, u);
        return make_float4(liq(fu.x) ? wt[fu.x & CF_D] * ru.x : 0.f, liq(fu.y) ? wt[fu.y & CF_D] * ru.y : 0.f,
                           liq(fu.z) ? wt[fu.z & CF_D] * ru.z : 0.f, liq(fu.w) ? wt[fu.w & CF_D] * ru.w : 0.f);
    };
    auto e1s = [&](int u) {
        const uint8_t fu = fl[u];
        return liq(fu) ? wt[fu & CF_D] * ldv1<false>(r, u) : 0.f;
    };
    const float4 c = e1q(t), rv = ldv4<false>(r, t);
    const float4 dn = e1q(t - g.sy), up = e1q(t + g.sy), bk = e1q(t - g.sz), fw = e1q(t + g.sz);
    const float lf = e1s(t - 1), rt = e1s(t + 4);
    auto one = [&](uint8_t fe, float ce, float nb, float re) {
        return liq(fe) ? re - m * ce - scale * ((float)(fe & CF_D) * ce - nb) : 0.f;
    };
    float4 v;
    v.x = one(f.x, c.x, (lf + c.y) + (dn.x + up.x) + (bk.x + fw.x), rv.x);
    v.y = one(f.y, c.y, (c.x + c.z) + (dn.y + up.y) + (bk.y + fw.y), rv.y);
    v.z = one(f.z, c.z, (c.y + c.w) + (dn.z + up.z) + (bk.z + fw.z), rv.z);
    v.w = one(f.w, c.w, (c.z + rt) + (dn.w + up.w) + (bk.w + fw.w), rv.w);
    *reinterpret_cast<float4 *>(eb + t) = c;
    *reinterpret_cast<float4 *>(res + t) = v;
}

// ---- one launch per step ------------------------------------------------------

// One sweep over the active quads. With rzs (the last sweep of a V-cycle's level
// 0), it also forms r.eout, which is the solver's r.z: each block's compensated
// sum goes to the partials as block boff + blockIdx.x of btot (the blocks of the
// face volumes' launches together), and the last block to arrive sets beta =
// rz_new / rz (first: 0) and rz, as the solver's separate r.z pass does.
__global__ void __launch_bounds__(256) k_mg0_smooth(MgGrid g, const int *__restrict__ qlist, int na,
                                                    const uint8_t *__restrict__ fl, const float *__restrict__ r,
                                                    const float *__restrict__ ein, float *eout, float scale, float m,
                                                    const int *done, SolveScal *rzs, double *partials, int first,
                                                    int boff, int btot)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    __shared__ float wt[8];
    fill_wtab(wt, scale, m);
    KSum acc;
    MG_FOR_LIST(qlist, na) acc.add(smooth_q<false>(g, fl, r, ein, eout, wt, scale, m, q));
    if (!rzs || *(volatile const int *)&rzs->done) return;  // (a timed sweep runs after convergence too)
    KSum v[1] = {acc};
    double tot[1];
    if (multi_reduce<1>(v, partials, &rzs->ticket, tot, boff + (int)blockIdx.x, btot) && threadIdx.x == 0) {
        if (!isfinite(tot[0])) {
            rzs->done = 1;
            rzs->status = FS_ENONFINITE;
            return;
        }
        rzs->beta = first ? 0.0 : tot[0] / rzs->rz;
        rzs->rz = tot[0];
    }
}

__global__ void __launch_bounds__(256) k_mg0_pre1(MgGrid g, const int *__restrict__ qlist, int na,
                                                  const uint8_t *__restrict__ fl, const float *__restrict__ r,
                                                  float *eb, float *res, float scale, float m, const int *done)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    __shared__ float wt[8];
    fill_wtab(wt, scale, m);
    MG_FOR_LIST(qlist, na) pre1_q(g, fl, r, eb, res, wt, scale, m, q);
}

__global__ void __launch_bounds__(256, 8) k_mg0_residual(MgGrid g, const int *__restrict__ qlist, int na,
                                                      const uint8_t *__restrict__ fl, const float *__restrict__ r,
                                                      const float *__restrict__ ev, float *res, float scale, float m,
                                                      const int *done)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    MG_FOR_LIST(qlist, na) resid_q<false>(g, fl, r, ev, res, scale, m, q);
}

__global__ void __launch_bounds__(256) k_mg0_smooth2(MgGrid g, const int *__restrict__ qlist, int na,
                                                     const uint8_t *__restrict__ fl, const float *__restrict__ r,
                                                     float *eo, float scale, float m, const int *done)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    __shared__ float wt[8];
    fill_wtab(wt, scale, m);
    MG_FOR_LIST(qlist, na) smooth2_q<false>(g, fl, r, eo, wt, scale, m, q);
}

__global__ void __launch_bounds__(256) k_mg0_prolong(MgGrid gf, const int *__restrict__ qlist, int na,
                                                     const uint8_t *__restrict__ fl, float *ef, MgGrid gc,
                                                     const float *__restrict__ ec, const int *done)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    MG_FOR_LIST(qlist, na) prolong_q<false>(gf, fl, ef, gc, ec, q);
}

// restriction over the coarse level's list of active pairs
__global__ void __launch_bounds__(256) k_mg0_restrict(MgGrid gf, const float *__restrict__ res, MgGrid gc,
                                                      const int *__restrict__ plist, int np,
                                                      const uint8_t *__restrict__ flc, float *rc, const int *done)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    MG_FOR_LIST(plist, np) restrict_pair<false>(gf, res, gc, flc, rc, q);
}

// ---- lists of the active quads and restriction pairs ------------------------------
// Sorted and deterministic: block b owns items [b LB_ITEMS, (b + 1) LB_ITEMS), four
// consecutive items per thread; a first pass counts each block's kept items, the
// host scans the counts, and a second pass writes each block's items in order
// at its offset.
constexpr int LB_TH = 256, LB_PER = 4, LB_ITEMS = LB_TH * LB_PER;

struct QuadPred {  // a quad of the level holds an unknown
    MgGrid g;
    const uint8_t *fl;
    __device__ long long items() const { return g.n >> 2; }
    __device__ bool keep(long long q, int &out) const
    {
        out = (int)q;
        return any_liq(ldf4(fl, (int)q << 2));
    }
};
struct PairPred {  // a restriction pair (2m, 2m + 1) of the coarse level holds an unknown
    MgGrid g;
    const uint8_t *fl;
    __device__ long long items() const { return (long long)((g.nx + 1) >> 1) * g.ny * g.nz; }
    __device__ bool keep(long long it, int &out) const
    {
        const int npair = (g.nx + 1) >> 1;
        const int m = (int)(it % npair);
        const long long jk = it / npair;
        const int J = (int)(jk % g.ny), K = (int)(jk / g.ny);
        out = g.idx(2 * m, J, K);
        return liq(fl[out]) || (2 * m + 1 < g.nx && liq(fl[out + 1]));
    }
};

template <class P>
__global__ void __launch_bounds__(LB_TH) k_list_build(P pred, const int *__restrict__ offsets, int *count, int *list)
{
    __shared__ int warp_tot[LB_TH / 32];
    const long long n = pred.items();
    const long long base = (long long)blockIdx.x * LB_ITEMS + (long long)threadIdx.x * LB_PER;
    int ids[LB_PER];
    int kept = 0;
#pragma unroll
    for (int k = 0; k < LB_PER; k++) {
        int id = 0;
        const bool keep = base + k < n && pred.keep(base + k, id);
        ids[k] = keep ? id : -1;
        kept += keep ? 1 : 0;
    }
    // inclusive scan of the kept counts over the block (warp shuffles, then warps)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = kept;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int k = 0; k < LB_TH / 32; k++) {
        if (k < w) before += warp_tot[k];
        total += warp_tot[k];
    }
    if (!list) {  // counting pass
        if (threadIdx.x == 0) count[blockIdx.x] = total;
        return;
    }
    int pos = offsets[blockIdx.x] + before + incl - kept;
#pragma unroll
    for (int k = 0; k < LB_PER; k++)
        if (ids[k] >= 0) list[pos++] = ids[k];
}

// ---- set-up ------------------------------------------------------------------

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

// The coarsest level: MG_COARSE_SWEEPS damped Jacobi sweeps from zero in the
// shared memory `sm` of one block (13 bytes per element), the result written to
// e on every element; wt is the level's weight table. Each sweep reads only the
// previous one, so the result does not depend on the block size.
template <bool CG>
__device__ void coarse_block(const MgGrid &g, const uint8_t *__restrict__ fl, const float *r, float *e,
                             const float *wt, float scale, float m, float *sm)
{
    float *e0 = sm, *e1 = sm + g.n, *rs = sm + 2 * g.n;
    uint8_t *fs = reinterpret_cast<uint8_t *>(sm + 3 * g.n);
    for (int t = threadIdx.x; t < g.n; t += blockDim.x) {
        const uint8_t f = fl[t];
        const float rv = ldv1<CG>(r, t);
        fs[t] = f;
        rs[t] = liq(f) ? rv : 0.f;
        e0[t] = liq(f) ? wt[f & CF_D] * rv : 0.f;
        e1[t] = 0.f;
    }
    __syncthreads();
    for (int s = 1; s < MG_COARSE_SWEEPS; s++) {
        const float *ein = (s & 1) ? e0 : e1;
        float *eout = (s & 1) ? e1 : e0;
        for (int t = threadIdx.x; t < g.n; t += blockDim.x) {
            const uint8_t f = fs[t];
            eout[t] = liq(f) ? ein[t] + wt[f & CF_D] * (rs[t] - m * ein[t] - scale * lap(ein, t, f, g)) : 0.f;
        }
        __syncthreads();
    }
    const float *res = (MG_COARSE_SWEEPS & 1) ? e0 : e1;  // the last sweep's output
    for (int t = threadIdx.x; t < g.n; t += blockDim.x) e[t] = res[t];
}

constexpr int COARSE_TH = 1024;  // threads of the block that solves the coarsest level

__global__ void __launch_bounds__(COARSE_TH) k_mg_coarse(MgGrid g, const uint8_t *__restrict__ fl,
                                                         const float *__restrict__ r, float *e, float scale, float m,
                                                         const int *done)
{
    if (done && *(volatile const int *)done) return;  // the solve has converged
    extern __shared__ float sm[];
    __shared__ float wt[8];
    fill_wtab(wt, scale, m);
    coarse_block<false>(g, fl, r, e, wt, scale, m, sm);
}

// ---- the small levels in one cluster -------------------------------------------
// The levels whose active quads number at most MGC_MAX_QUADS take one launch of a
// single thread-block cluster (MGC_CTAS CTAs of MGC_TH threads): the same steps as
// the per-level kernels, level by level, with the cluster's hardware barrier in
// place of each kernel boundary. What one CTA writes another reads after the
// barrier (release, then acquire at cluster scope), through L2 (ld.global.cg:
// no SM's L1 can hold a stale copy). CTA 0 solves the coarsest level.
constexpr int MGC_TH = 1024;
constexpr int MGC_MAXLEV = 8;
constexpr int MGC_MAX_QUADS = 49152;

struct MgcLevel {
    MgGrid g;
    const uint8_t *fl;
    float *r, *a, *b, *c;
    const int *ql, *pl;
    int nqa, npa;
    float scale, mass;
};

struct MgClusterArgs {
    MgcLevel lev[MGC_MAXLEV];
    int nlev;
    const int *done;
};

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int cluster_ctas()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return (int)r;
}

// The V-cycle on a.lev[0] .. a.lev[nlev - 1]: r in lev[0].r, result in lev[0].a.
__global__ void __launch_bounds__(MGC_TH) k_mg_cluster(const MgClusterArgs a)
{
    if (a.done && *(volatile const int *)a.done) return;  // the solve has converged (every CTA alike)
    extern __shared__ float sm[];
    __shared__ float wts[MGC_MAXLEV][8];
    for (int i = threadIdx.x; i < MGC_MAXLEV * 8; i += blockDim.x)
        if (i / 8 < a.nlev) wts[i / 8][i % 8] = wtab_entry(a.lev[i / 8].scale, a.lev[i / 8].mass, i % 8);
    __syncthreads();
    const int tid = cluster_rank() * blockDim.x + threadIdx.x, st = cluster_ctas() * blockDim.x;
    for (int l = 0; l + 1 < a.nlev; l++) {
        const MgcLevel &L = a.lev[l], &W = a.lev[l + 1];
        for (int i = tid; i < L.nqa; i += st)
            smooth2_q<true>(L.g, L.fl, L.r, L.b, wts[l], L.scale, L.mass, __ldg(L.ql + i));
        cluster_barrier();
        for (int i = tid; i < L.nqa; i += st) resid_q<true>(L.g, L.fl, L.r, L.b, L.c, L.scale, L.mass, __ldg(L.ql + i));
        cluster_barrier();
        for (int i = tid; i < W.npa; i += st) restrict_pair<true>(L.g, L.c, W.g, W.fl, W.r, __ldg(W.pl + i));
        cluster_barrier();
    }
    if (cluster_rank() == 0) {
        const MgcLevel &L = a.lev[a.nlev - 1];
        coarse_block<true>(L.g, L.fl, L.r, L.a, wts[a.nlev - 1], L.scale, L.mass, sm);
    }
    cluster_barrier();
    for (int l = a.nlev - 2; l >= 0; l--) {
        const MgcLevel &L = a.lev[l], &W = a.lev[l + 1];
        for (int i = tid; i < L.nqa; i += st) prolong_q<true>(L.g, L.fl, L.b, W.g, W.a, __ldg(L.ql + i));
        cluster_barrier();
        for (int i = tid; i < L.nqa; i += st)
            smooth_q<true>(L.g, L.fl, L.r, L.b, L.c, wts[l], L.scale, L.mass, __ldg(L.ql + i));
        cluster_barrier();
        for (int i = tid; i < L.nqa; i += st)
            smooth_q<true>(L.g, L.fl, L.r, L.c, L.a, wts[l], L.scale, L.mass, __ldg(L.ql + i));
        if (l > 0) cluster_barrier();
    }
}

// r.z over the active quads of one or three level-0 lists (r is zero off the
// unknowns, so no other quad adds to it), in the lists' fixed order: beta =
// rz_new / rz (first: beta = 0), as the dense pass of the solver does.
struct RzLists {
    const int *ql[3];
    int n[3];
    long long base[3];
    int nv;
};

__global__ void __launch_bounds__(TH) k_mg_rz(RzLists L, const float *__restrict__ r, const float *__restrict__ z,
                                             int first, SolveScal *s, double *partials)
{
    if (s->done) return;
    KSum acc;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    for (int v = 0; v < L.nv; v++) {
        const float4 *r4 = reinterpret_cast<const float4 *>(r + L.base[v]);
        const float4 *z4 = reinterpret_cast<const float4 *>(z + L.base[v]);
        for (int i = tid; i < L.n[v]; i += st) {
            const int q = __ldg(L.ql[v] + i);
            const float4 a = __ldg(r4 + q), b = __ldg(z4 + q);
            acc.add(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w);
        }
    }
    KSum v[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        if (!isfinite(tot[0])) {
            s->done = 1;
            s->status = FS_ENONFINITE;
            return;
        }
        s->beta = first ? 0.0 : tot[0] / s->rz;
        s->rz = tot[0];
    }
}

// number of unknown cells of a level (once per mask, for the profiled byte count)
__global__ void k_mg_count_liq(MgGrid g, const uint8_t *__restrict__ fl, unsigned long long *out)
{
    unsigned long long k = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.n; t += gridDim.x * blockDim.x) k += liq(fl[t]) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    if ((threadIdx.x & 31) == 0 && k) atomicAdd(out, k);
}

size_t coarse_smem(const MgGrid &g) { return (size_t)g.n * 13 + 16; }

int row_blocks(fs_ctx *c, const MgGrid &g) { return grid_blocks(c, g.rows, 8); }

// a box of nx x ny x nz cells in the guarded layout of the context (pitch P, R
// rows per plane, a guard plane before and after): the cell space, or one face
// volume counted from its leading guard plane
MgGrid level0_grid(const Layout &L, int nx, int ny, int nz)
{
    MgGrid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.sy = L.P;
    g.sz = L.PL;
    g.origin = L.PL;
    g.n = L.S + 2 * L.PL;
    g.rows = g.n / L.P;
    g.rpp = L.R;
    g.ioff = 0;
    g.joff = 0;
    g.koff = 1;
    return g;
}

// a coarse level: a solid halo of one plane and one row on each side, and of 4
// elements before each row (at least 1 after it), with the row pitch a multiple
// of 4, so that its quads are aligned like level 0's
MgGrid coarse_grid(int nx, int ny, int nz)
{
    MgGrid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.sy = (nx + 5 + 3) / 4 * 4;
    g.sz = g.sy * (ny + 2);
    g.origin = g.sz + g.sy + 4;
    g.n = g.sz * (nz + 2);
    g.rows = (ny + 2) * (nz + 2);
    g.rpp = ny + 2;
    g.ioff = 4;
    g.joff = 1;
    g.koff = 1;
    return g;
}

void free_levels(MgState *s)
{
    for (int l = 0; l < s->nlev; l++) {
        cudaFree(s->lev[l].ql);
        cudaFree(s->lev[l].pl);
        s->lev[l].ql = s->lev[l].pl = nullptr;
        s->lev[l].nqa = s->lev[l].npa = 0;
    }
    for (int l = 1; l < s->nlev; l++) {
        MgLevel &v = s->lev[l];
        cudaFree(v.fl);
        cudaFree(v.r);
        cudaFree(v.a);
        cudaFree(v.b);
        cudaFree(v.c);
        v = MgLevel();
    }
    if (s->own0) {
        cudaFree(s->lev[0].b);
        cudaFree(s->lev[0].c);
    }
    s->lev[0] = MgLevel();
    s->nlev = 0;
    s->epoch = -1;
}

// The V-cycle on level l: r in lev[l].r, result in lev[l].a. With `sample`, the
// last level-0 sweep is timed.
// The V-cycle on level l: r in lev[l].r, result in lev[l].a. With `sample`
// (level 0 of a pressure V-cycle on the context's stream), every level-0 kernel
// and the coarse levels as a whole are timed; a timed kernel always runs in full
// (an early exit would record work not done).
// levels cl .. nlev - 1 of a hierarchy in one cluster launch
int launch_cluster(fs_ctx *c, MgState *s, int cl, cudaStream_t st)
{
    MgClusterArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nlev = s->nlev - cl;
    for (int l = cl; l < s->nlev; l++) {
        const MgLevel &v = s->lev[l];
        a.lev[l - cl] = MgcLevel{v.g, v.fl, v.r, v.a, v.b, v.c, v.ql, v.pl, v.nqa, v.npa, v.scale, v.mass};
    }
    a.done = s->done;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s->ctas);
    cfg.blockDim = dim3(MGC_TH);
    cfg.dynamicSmemBytes = coarse_smem(s->lev[s->nlev - 1].g);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s->ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FS_CUDA(cudaLaunchKernelEx(&cfg, k_mg_cluster, a));
    c->n_launches += 1;
    return FS_OK;
}

// CTAs of the single-cluster launch on this device: 16 where the device allows
// that non-portable size, else 8, else 0 (no cluster launch)
int cluster_ctas_here()
{
    static int cached = -1;
    if (cached >= 0) return cached;
    cached = 0;
    if (cudaFuncSetAttribute(k_mg_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int n : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n);
        cfg.blockDim = dim3(MGC_TH);
        cfg.dynamicSmemBytes = (size_t)MG_COARSE_CELLS * 13 + 16;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = n;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_mg_cluster, &cfg) == cudaSuccess && clusters > 0) {
            cached = n;
            break;
        }
        cudaGetLastError();
    }
    return cached;
}

// Resident blocks per SM of the list-walking kernels, for one-wave grids.
struct MgResidency {
    int smooth2, residual, pre1, restrict_, prolong, smooth;
};
const MgResidency &mg_residency()
{
    static const MgResidency r{resident_blocks((const void *)k_mg0_smooth2, 0),
                               resident_blocks((const void *)k_mg0_residual, 0),
                               resident_blocks((const void *)k_mg0_pre1, 0),
                               resident_blocks((const void *)k_mg0_restrict, 0),
                               resident_blocks((const void *)k_mg0_prolong, 0),
                               resident_blocks((const void *)k_mg0_smooth, 0)};
    return r;
}

// blocks of the sweeps k_mg0_smooth over a level's nqa active quads (also the
// block count of the r.z reduction the last level-0 sweep forms)
int smooth_blocks(const fs_ctx *c, int nqa) { return wave_blocks(c, nqa, mg_residency().smooth); }

int vcycle(fs_ctx *c, MgState *s, int l, bool sample, cudaStream_t st)
{
    if (s->cl > 0 && l == s->cl) return launch_cluster(c, s, l, st);
    MgLevel &v = s->lev[l];
    const MgGrid &g = v.g;
    if (l == s->nlev - 1) {
        k_mg_coarse<<<1, COARSE_TH, coarse_smem(g), st>>>(g, v.fl, v.r, v.a, v.scale, v.mass, s->done);
        c->n_launches += 1;
        return FS_OK;
    }
    const bool timed = sample && l == 0 && s->by0[0] > 0.0;
    const int *done = timed ? nullptr : s->done;
    // an event pair around each timed launch (an event belongs to one pair)
    cudaEvent_t e0 = nullptr;
    auto begin = [&]() {
        if (timed) e0 = prof_mark(c);
    };
    auto end = [&](int kind, double bytes) {
        if (timed) prof_add(c, kind, e0, prof_mark(c), bytes);
    };
    // four elements per thread: every level but the coarsest has quad-aligned rows;
    // each kernel over the active quads in one wave of its resident blocks
    const MgResidency &res = mg_residency();
    const int nb = smooth_blocks(c, v.nqa);
    MgLevel &w = s->lev[l + 1];
    // one sweep each side on level 0 of a face volume (the viscosity solve), two
    // elsewhere
    const bool one = l == 0 && s->one0;
    if (one) {  // the sweep from zero and the residual it leaves, in one pass
        k_mg0_pre1<<<wave_blocks(c, v.nqa, res.pre1), TH, 0, st>>>(g, v.ql, v.nqa, v.fl, v.r, v.b, v.c, v.scale, v.mass, done);
        c->n_launches += 1;
    } else {
        begin();
        k_mg0_smooth2<<<wave_blocks(c, v.nqa, res.smooth2), TH, 0, st>>>(g, v.ql, v.nqa, v.fl, v.r, v.b, v.scale, v.mass, done);
        end(K_MG0_SMOOTH2, s->by0[0]);
        begin();
        k_mg0_residual<<<wave_blocks(c, v.nqa, res.residual), TH, 0, st>>>(g, v.ql, v.nqa, v.fl, v.r, v.b, v.c, v.scale, v.mass, done);
        end(K_MG0_RESIDUAL, s->by0[1]);
        c->n_launches += 2;
    }
    begin();
    k_mg0_restrict<<<wave_blocks(c, w.npa, res.restrict_), TH, 0, st>>>(g, v.c, w.g, w.pl, w.npa, w.fl, w.r, done);
    end(K_MG0_RESTRICT, s->by0[2]);
    c->n_launches += 1;
    begin();
    if (int rc = vcycle(c, s, l + 1, false, st)) return rc;
    end(K_MG_COARSE, 0.0);
    begin();
    k_mg0_prolong<<<wave_blocks(c, v.nqa, res.prolong), TH, 0, st>>>(g, v.ql, v.nqa, v.fl, v.b, w.g, w.a, done);
    end(K_MG0_PROLONG, s->by0[3]);
    SolveScal *rzs = l == 0 ? s->rzs : nullptr;  // r.z of the solver in the last level-0 sweep
    const float *ez = v.c;                        // the input of the last sweep
    if (one) {
        ez = v.b;
    } else {
        begin();
        k_mg0_smooth<<<nb, TH, 0, st>>>(g, v.ql, v.nqa, v.fl, v.r, v.b, v.c, v.scale, v.mass, done, nullptr,
                                        nullptr, 0, 0, 0);
        end(K_MG0_SMOOTH, s->by0[4]);
        c->n_launches += 1;
    }
    begin();
    k_mg0_smooth<<<nb, TH, 0, st>>>(g, v.ql, v.nqa, v.fl, v.r, ez, v.a, v.scale, v.mass, done, rzs, c->partials,
                                    s->rz_first, s->rz_boff, s->rz_btot);
    end(K_MG0_SMOOTH_Z, s->by0[5]);
    c->n_launches += 2;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

// Builds a hierarchy under level 0 (grid g0, flags fl0, work arrays b0 and c0 of
// the level-0 length, or allocated here when null).
int mg_build(fs_ctx *c, MgState *s, const MgGrid &g0, uint8_t *fl0, float *b0, float *c0, float coef, float mass)
{
    free_levels(s);
    MgLevel &l0 = s->lev[0];
    l0.g = g0;
    l0.scale = coef;
    l0.mass = mass;
    l0.fl = fl0;
    s->nlev = 1;
    s->own0 = b0 == nullptr;
    auto fail = [&](const char *what) {
        cudaGetLastError();
        free_levels(s);
        return set_error(FS_ENOMEM, "multigrid %s", what);
    };
    if (s->own0) {
        if (cudaMalloc(&l0.b, (size_t)g0.n * 4) != cudaSuccess || cudaMalloc(&l0.c, (size_t)g0.n * 4) != cudaSuccess)
            return fail("level-0 work arrays");
        FS_CUDA(cudaMemsetAsync(l0.b, 0, (size_t)g0.n * 4, c->stream));
        FS_CUDA(cudaMemsetAsync(l0.c, 0, (size_t)g0.n * 4, c->stream));
    } else {
        l0.b = b0;
        l0.c = c0;
    }
    while (s->lev[s->nlev - 1].g.n > MG_COARSE_CELLS && s->nlev < MG_MAX_LEVELS) {
        const MgGrid &gf = s->lev[s->nlev - 1].g;
        MgLevel &v = s->lev[s->nlev];
        v.g = coarse_grid((gf.nx + 1) / 2, (gf.ny + 1) / 2, (gf.nz + 1) / 2);
        v.scale = s->lev[s->nlev - 1].scale * 0.25f;
        v.mass = mass;
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
    for (int l = 0; l + 1 < s->nlev; l++) {  // the quad kernels' alignment (true by construction)
        const MgGrid &g = s->lev[l].g;
        if (g.sy % 4 || g.sz % 4 || g.origin % 4 || g.n % 4)
            return set_error(FS_EINVAL, "multigrid: level %d rows are not quad-aligned", l);
    }
    // the lists of active quads (every level but the coarsest) and of active
    // restriction pairs (every level but the finest): counted, allocated, filled
    auto make_list = [&](bool pairs, int l, int **list, int *count) -> int {
        const MgGrid &g = s->lev[l].g;
        const long long items = pairs ? (long long)((g.nx + 1) >> 1) * g.ny * g.nz : g.n / 4;
        const int blocks = (int)std::max(1LL, (items + LB_ITEMS - 1) / LB_ITEMS);
        int *dcnt = nullptr;
        std::vector<int> hcnt(blocks);
        if (cudaMalloc(&dcnt, sizeof(int) * (size_t)blocks * 2) != cudaSuccess) {
            cudaGetLastError();
            return FS_ENOMEM;
        }
        auto launch = [&](const int *offs, int *out) {
            if (pairs)
                k_list_build<<<blocks, LB_TH, 0, c->stream>>>(PairPred{g, s->lev[l].fl}, offs, dcnt, out);
            else
                k_list_build<<<blocks, LB_TH, 0, c->stream>>>(QuadPred{g, s->lev[l].fl}, offs, dcnt, out);
            c->n_launches += 1;
        };
        int rc = FS_OK;
        launch(nullptr, nullptr);
        if ((rc = check_cuda(cudaGetLastError(), "k_list_build")) ||
            (rc = check_cuda(cudaMemcpyAsync(hcnt.data(), dcnt, sizeof(int) * (size_t)blocks,
                                             cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync")) ||
            (rc = check_cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize"))) {
            cudaFree(dcnt);
            return rc;
        }
        int total = 0;
        for (int b = 0; b < blocks; b++) {  // exclusive scan of the block counts
            const int n = hcnt[b];
            hcnt[b] = total;
            total += n;
        }
        *count = total;
        if (cudaMalloc(list, sizeof(int) * (size_t)std::max(total, 1)) != cudaSuccess) {
            cudaGetLastError();
            *list = nullptr;
            cudaFree(dcnt);
            return FS_ENOMEM;
        }
        if (!(rc = check_cuda(cudaMemcpyAsync(dcnt + blocks, hcnt.data(), sizeof(int) * (size_t)blocks,
                                              cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync"))) {
            launch(dcnt + blocks, *list);
            rc = check_cuda(cudaGetLastError(), "k_list_build");
        }
        // the host counts must outlive the copy above
        if (!rc) rc = check_cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        cudaFree(dcnt);
        return rc;
    };
    for (int l = 0; l < s->nlev; l++) {
        MgLevel &v = s->lev[l];
        int rc = FS_OK;
        if (l + 1 < s->nlev) rc = make_list(false, l, &v.ql, &v.nqa);
        if (!rc && l >= 1) rc = make_list(true, l, &v.pl, &v.npa);
        if (rc == FS_ENOMEM) return fail("active lists");
        if (rc) {
            free_levels(s);
            return rc;
        }
    }
    // the small levels in one cluster launch: from the first level below level 0
    // whose active quads fit the cluster's threads a few times over, when at
    // least one level above the coarsest is among them
    s->cl = 0;
    s->ctas = cluster_ctas_here();
    if (s->ctas > 0)
        for (int l = 1; l + 1 < s->nlev; l++)
            if (s->lev[l].nqa <= MGC_MAX_QUADS && s->nlev - l <= MGC_MAXLEV) {
                s->cl = l;
                break;
            }
    // The least each level-0 kernel must move (its algorithmic bytes): the list
    // entry and the flags of each active quad (or pair) it visits and 4 bytes per
    // unknown for each vector it reads or writes on the unknowns.
    // q0: the active quads of level 0; p1: level 1's active pairs;
    // u0, u1: the unknowns of levels 0 and 1.
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c->partials), nl[2] = {0, 0};
    FS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(nl), c->stream));
    k_mg_count_liq<<<grid_blocks(c, g0.n, TH), TH, 0, c->stream>>>(g0, fl0, cnt);
    if (s->nlev > 1)
        k_mg_count_liq<<<grid_blocks(c, s->lev[1].g.n, TH), TH, 0, c->stream>>>(s->lev[1].g, s->lev[1].fl, cnt + 1);
    FS_CUDA(cudaMemcpyAsync(nl, cnt, sizeof(nl), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    const double u0 = (double)nl[0], u1 = (double)nl[1];
    const double q0 = (double)s->lev[0].nqa, p1 = s->nlev > 1 ? (double)s->lev[1].npa : 0.0;
    s->by0[0] = 8.0 * q0 + 8.0 * u0;             // smooth2: read r, write e
    s->by0[1] = 8.0 * q0 + 12.0 * u0;            // residual: read r, e, write res
    s->by0[2] = 6.0 * p1 + 4.0 * u0 + 4.0 * u1;  // restrict: pair list and flags, read res, write level-1 r
    s->by0[3] = 8.0 * q0 + 8.0 * u0 + 4.0 * u1;  // prolong: read and write e, read the level-1 e
    s->by0[4] = 8.0 * q0 + 12.0 * u0;            // smooth: read r, e, write e
    s->by0[5] = 8.0 * q0 + 12.0 * u0;            // last smooth: read r, e, write z
    s->epoch = c->mask_epoch;
    s->coef = coef;
    return FS_OK;
}

int apply_on(fs_ctx *c, MgState *s, const float *r, float *z, const int *done, bool sample, cudaStream_t st,
             SolveScal *rzs = nullptr, int first = 0, int boff = 0, int btot = 0)
{
    s->done = done;
    s->rzs = rzs;
    s->rz_first = first;
    s->rz_boff = boff;
    s->rz_btot = btot;
    MgLevel &l0 = s->lev[0];
    l0.r = const_cast<float *>(r);
    l0.a = z;
    const int rc = vcycle(c, s, 0, sample, st);
    l0.r = nullptr;
    l0.a = nullptr;
    return rc;
}

MgAll *state(fs_ctx *c)
{
    MgAll *m = static_cast<MgAll *>(c->mg);
    if (!m) {
        m = new (std::nothrow) MgAll();
        c->mg = m;
    }
    return m;
}

}  // namespace

void mg_free(fs_ctx *c)
{
    MgAll *m = static_cast<MgAll *>(c->mg);
    if (!m) return;
    free_levels(&m->cell);
    for (MgState &f : m->face) free_levels(&f);
    cudaFree(m->fb);
    cudaFree(m->fc);
    for (int k = 0; k < 2; k++) {
        if (m->side[k]) cudaStreamDestroy(m->side[k]);
        if (m->join[k]) cudaEventDestroy(m->join[k]);
    }
    if (m->fork) cudaEventDestroy(m->fork);
    delete m;
    c->mg = nullptr;
}

// z = M r on the cell space (r and z of length nC, zero off the liquid).
// z = M r on the cell space; with rzs, r.z in the last level-0 sweep when the
// hierarchy has one (*fused tells)
static int apply_cell(fs_ctx *c, const float *r, float *z, const int *done, SolveScal *rzs, int first, bool *fused)
{
    if (fused) *fused = false;
    MgAll *m = state(c);
    if (!m) return set_error(FS_ENOMEM, "host allocation failed");
    const Layout &L = c->L;
    if (m->cell.epoch != c->mask_epoch)
        if (int rc = mg_build(c, &m->cell, level0_grid(L, L.nx, L.ny, L.nz), c->cflag, nullptr, nullptr, 1.f, 0.f))
            return rc;
    const bool fuse = rzs && m->cell.nlev >= 2;
    const bool sample = c->prof_on && (m->cell.calls++ % std::max(1, c->prof_period)) == 0;
    cudaEvent_t e0 = sample ? prof_mark(c) : nullptr;
    const int rc = fuse ? apply_on(c, &m->cell, r, z, done, sample, c->stream, rzs, first, 0,
                                   smooth_blocks(c, m->cell.lev[0].nqa))
                        : apply_on(c, &m->cell, r, z, done, sample, c->stream);
    if (sample) prof_add(c, K_MG_VCYCLE_P, e0, prof_mark(c), 0.0);
    if (fused) *fused = fuse && rc == FS_OK;
    return rc;
}

int mg_apply(fs_ctx *c, const float *r, float *z, const int *done)
{
    return apply_cell(c, r, z, done, nullptr, 0, nullptr);
}

bool mg_apply_rz(fs_ctx *c, const float *r, float *z, const int *done, SolveScal *s, int first, int &rc)
{
    bool fused = false;
    rc = apply_cell(c, r, z, done, s, first, &fused);
    return fused;
}

// z = M r on the face space for the Helmholtz operator I + cc L of the viscosity
// solve, one V-cycle per velocity component (r and z of length nF, zero off the
// unknown faces). With `done` set, every kernel returns at once once *done != 0.
static int apply_faces(fs_ctx *c, const float *r, float *z, float cc, const int *done, SolveScal *rzs, int first,
                       bool *fused)
{
    if (fused) *fused = false;
    MgAll *m = state(c);
    if (!m) return set_error(FS_ENOMEM, "host allocation failed");
    const Layout &L = c->L;
    if (!m->fb) {
        if (cudaMalloc(&m->fb, (size_t)L.nF * 4) != cudaSuccess || cudaMalloc(&m->fc, (size_t)L.nF * 4) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(m->fb);
            m->fb = nullptr;
            return set_error(FS_ENOMEM, "multigrid face work arrays");
        }
        FS_CUDA(cudaMemsetAsync(m->fb, 0, (size_t)L.nF * 4, c->stream));
        FS_CUDA(cudaMemsetAsync(m->fc, 0, (size_t)L.nF * 4, c->stream));
    }
    if (!m->fork) {  // the side streams and their events, once (the fork event last)
        for (int k = 0; k < 2; k++) {
            if (!m->side[k]) FS_CUDA(cudaStreamCreateWithFlags(&m->side[k], cudaStreamNonBlocking));
            if (!m->join[k]) FS_CUDA(cudaEventCreateWithFlags(&m->join[k], cudaEventDisableTiming));
        }
        FS_CUDA(cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming));
    }
    if (m->face[0].epoch != c->mask_epoch) {  // new mask: the shared work arrays start from zero again
        FS_CUDA(cudaMemsetAsync(m->fb, 0, (size_t)L.nF * 4, c->stream));
        FS_CUDA(cudaMemsetAsync(m->fc, 0, (size_t)L.nF * 4, c->stream));
    }
    const bool sample = c->prof_on && (m->face[0].calls++ % std::max(1, c->prof_period)) == 0;
    cudaEvent_t e0 = sample ? prof_mark(c) : nullptr;
    for (int k = 0; k < 3; k++) {
        MgState &s = m->face[k];
        const size_t base = (size_t)L.face_origin(k) - L.PL;  // the volume's leading guard plane
        if (s.epoch != c->mask_epoch) {
            const MgGrid g0 = level0_grid(L, L.nx + (k == 0), L.ny + (k == 1), L.nz + (k == 2));
            if (int rc = mg_build(c, &s, g0, c->fflag + base, m->fb + base, m->fc + base, cc, 1.f)) return rc;
            s.one0 = true;
        } else if (s.coef != cc) {  // a new viscosity or time step: rescale the levels only
            float sc = cc;
            for (int l = 0; l < s.nlev; l++, sc *= 0.25f) s.lev[l].scale = sc;
            s.coef = cc;
        }
    }
    // r.z in the three last level-0 sweeps together: their blocks are numbered
    // one after another for one reduction (volume k's from boff[k])
    bool fuse = rzs != nullptr;
    int boff[3] = {0, 0, 0}, btot = 0;
    for (int k = 0; k < 3 && fuse; k++) {
        fuse = m->face[k].nlev >= 2;
        boff[k] = btot;
        btot += smooth_blocks(c, m->face[k].lev[0].nqa);
    }
    // volume 0 on the context's stream, 1 and 2 beside it (their sweeps share the
    // GPU, so none is timed alone: the profiled sweep is the pressure V-cycle's)
    FS_CUDA(cudaEventRecord(m->fork, c->stream));
    for (int k = 0; k < 2; k++) FS_CUDA(cudaStreamWaitEvent(m->side[k], m->fork, 0));
    for (int k = 2; k >= 0; k--) {
        const size_t base = (size_t)L.face_origin(k) - L.PL;
        cudaStream_t st = k == 0 ? c->stream : m->side[k - 1];
        const int rc = fuse ? apply_on(c, &m->face[k], r + base, z + base, done, false, st, rzs, first, boff[k], btot)
                            : apply_on(c, &m->face[k], r + base, z + base, done, false, st);
        if (rc) return rc;
    }
    for (int k = 0; k < 2; k++) {
        FS_CUDA(cudaEventRecord(m->join[k], m->side[k]));
        FS_CUDA(cudaStreamWaitEvent(c->stream, m->join[k], 0));
    }
    if (sample) prof_add(c, K_MG_VCYCLE_V, e0, prof_mark(c), 0.0);
    if (fused) *fused = fuse;
    return FS_OK;
}

int mg_apply_faces(fs_ctx *c, const float *r, float *z, float cc, const int *done)
{
    return apply_faces(c, r, z, cc, done, nullptr, 0, nullptr);
}

bool mg_apply_faces_rz(fs_ctx *c, const float *r, float *z, float cc, const int *done, SolveScal *s, int first,
                       int &rc)
{
    bool fused = false;
    rc = apply_faces(c, r, z, cc, done, s, first, &fused);
    return fused;
}

// Launch counts of the level-0 kernels (fs_profile): `vcycles` V-cycles that did
// work on the pressure hierarchy, or on each of the three face volumes.
void mg_count(fs_ctx *c, long long vcycles, bool faces)
{
    const MgAll *m = static_cast<const MgAll *>(c->mg);
    if (!m || !c->prof_on) return;
    const int nlev = faces ? m->face[0].nlev : m->cell.nlev;
    if (nlev < 2) return;
    const long long k = faces ? 3 * vcycles : vcycles;
    const bool one = faces && m->face[0].one0;  // the face volumes' level 0 skips three of the six kinds
    for (int id : {K_MG0_SMOOTH2, K_MG0_RESIDUAL, K_MG0_SMOOTH})
        if (!one) prof_count(c, id, k);
    for (int id : {K_MG0_RESTRICT, K_MG0_PROLONG, K_MG0_SMOOTH_Z}) prof_count(c, id, k);
    prof_count(c, faces ? K_MG_VCYCLE_V : K_MG_VCYCLE_P, vcycles);
    if (!faces) prof_count(c, K_MG_COARSE, vcycles);
}

// r.z over the active quads of the pressure hierarchy's level 0 (or of the three
// face volumes'); false when the hierarchy has no lists (a level 0 that is its
// own coarsest level), and the caller takes the dense pass
bool mg_rz(fs_ctx *c, bool faces, const float *r, const float *z, int first, SolveScal *s)
{
    const MgAll *m = static_cast<const MgAll *>(c->mg);
    if (!m) return false;
    RzLists L;
    std::memset(&L, 0, sizeof(L));
    long long total = 0;
    L.nv = faces ? 3 : 1;
    for (int v = 0; v < L.nv; v++) {
        const MgState &h = faces ? m->face[v] : m->cell;
        if (h.nlev < 2 || h.epoch != c->mask_epoch || !h.lev[0].ql) return false;
        L.ql[v] = h.lev[0].ql;
        L.n[v] = h.lev[0].nqa;
        L.base[v] = faces ? (long long)c->L.face_origin(v) - c->L.PL : 0;
        total += L.n[v];
    }
    k_mg_rz<<<grid_blocks(c, total, TH), TH, 0, c->stream>>>(L, r, z, first, s, c->partials);
    c->n_launches += 1;
    return cudaPeekAtLastError() == cudaSuccess;
}

// The level-0 lists of active quads of the pressure hierarchy (one) or of the
// three face volumes, with each volume's first element; false when a hierarchy
// has no lists for the current mask.
bool mg_level0_lists(const fs_ctx *c, bool faces, const int **ql, int *n, long long *base)
{
    const MgAll *m = static_cast<const MgAll *>(c->mg);
    if (!m) return false;
    const int nv = faces ? 3 : 1;
    for (int v = 0; v < nv; v++) {
        const MgState &h = faces ? m->face[v] : m->cell;
        if (h.nlev < 2 || h.epoch != c->mask_epoch || !h.lev[0].ql) return false;
        ql[v] = h.lev[0].ql;
        n[v] = h.lev[0].nqa;
        base[v] = faces ? (long long)c->L.face_origin(v) - c->L.PL : 0;
    }
    return true;
}

int mg_levels(const fs_ctx *c)
{
    const MgAll *m = static_cast<const MgAll *>(c->mg);
    return m ? m->cell.nlev : 0;
}

}  // namespace fs
