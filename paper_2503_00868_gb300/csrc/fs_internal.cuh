// fs_internal.cuh -- shared declarations of the CUDA implementation of the
// differentiable MAC-grid fluid step (arXiv 2503.00868, Sec. 3.4.1-3.4.2).
//
// Internal vectors. Solver vectors live in flat, guarded buffers so that every
// 7-point stencil reads its neighbours at fixed offsets (+-1, +-pitch, +-plane)
// without bounds checks:
//   cell space  [guard: plane][cells: S][guard: plane]
//   face space  [guard][u: S][guard][v: S][guard][w: S][guard]
// where S = pitch * rows * planes is the size of one array of the public layout
// and plane = pitch * rows. Guards and padding hold zero and flag byte 0, so a
// neighbour outside the grid contributes nothing.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fluidstep.h"

namespace fs {

// ---- flag bytes ------------------------------------------------------------
// cell flags: bits 0-2 = number of non-solid neighbours (pressure diagonal)
constexpr uint8_t CF_D = 0x07;
constexpr uint8_t CF_LIQ = 0x08;
constexpr uint8_t CF_AIR = 0x10;
constexpr uint8_t CF_SOLID = 0x20;
constexpr uint8_t CF_BAND = 0x40;  // liquid with an air neighbour
// face flags: bits 0-2 = number of fluid or fixed neighbours (viscosity diagonal)
constexpr uint8_t FF_N = 0x07;
constexpr uint8_t FF_FLUID = 0x08;
constexpr uint8_t FF_FIXED = 0x10;
constexpr uint8_t FF_AIR = 0x20;

// ---- solver scalars (device memory; mirrored to pinned host memory) --------
struct SolveScal {
    double rz;      // r.z of the current iterate
    double pq;      // p.Ap
    double rr;      // r.r
    double bb;      // b.b (right-hand side)
    double tol2;    // tol^2
    double alpha;
    double beta;
    double aux[4];  // misc reductions (sums, counts, losses)
    int iter;
    int maxit;
    int done;
    int status;     // FS_OK / FS_ENOCONV / FS_ENONFINITE / FS_EBREAKDOWN
    unsigned ticket;
    int pad;
};

struct Layout {
    int nx, ny, nz;
    int P;      // pitch
    int R;      // rows = ny + 1
    int Z;      // planes = nz + 1
    int PL;     // plane = P * R
    int S;      // P * R * Z
    int nC;     // cell space length  = S + 2 * PL
    int nF;     // face space length  = 3 * (S + PL) + PL
    __host__ __device__ int face_origin(int c) const { return PL + c * (S + PL); }
};

// Tiling of a guarded space for the z-marching stencil kernels: `nvol` volumes
// (1 for cell space, 3 for face space) of P x R x Z elements starting at
// origin0 + v * vstride; tiles of TILE_X x TILE_Y columns, `tz` planes per chunk.
// Block b covers tile (tx, ty) of chunk ch of volume v, x fastest.
constexpr int TILE_X = 128;  // elements (32 threads x 4)
constexpr int TILE_Y = 8;

struct TileMap {
    int ntx, nty, tz, nch, nvol;
    int P, R, Z, PL;
    int origin0, vstride;
    int nblocks;
    __host__ __device__ void decode(int b, int &v, int &ch, int &ty, int &tx) const
    {
        tx = b % ntx;
        b /= ntx;
        ty = b % nty;
        b /= nty;
        ch = b % nch;
        v = b / nch;
    }
};

struct F3 {
    float *c[3];
};
struct CF3 {
    const float *c[3];
};

}  // namespace fs

struct fs_ctx {
    fs::Layout L;
    fs_params prm;
    cudaStream_t stream;
    int device;
    int num_sms;
    int mask_set;
    long long mask_epoch;  // incremented by every fs_set_mask (caches keyed to the mask)
    int singular;
    int has_bc;
    long long n_liquid, n_band_cells[2], n_band_faces[2];

    uint8_t *cflag;       // cell space
    uint8_t *fflag;       // face space
    float *bc;            // face space: prescribed values on fixed faces
    float *dsum;          // face space: sum of fixed neighbours' values (fluid faces)

    // pressure solve (cell space)
    float *pb, *pr, *pp[2], *pq, *px, *pz;
    // iterative refinement of the pressure solve: the first solution (head), the
    // sum of earlier corrections (tail) and the right-hand side of the correction
    // being solved. After a refined solve the pressure is the pair q_head + px.
    float *pxh, *pxt, *pbr;
    const float *q_head;  // null unless the last pressure solve was refined
    int refining;         // a correction is being solved: no warm start
    double tol2_scale;    // the stopping test is r.r <= tol_p^2 * tol2_scale * b.b (0 reads as 1)
    // warm start: last converged pressure of a forward (0) / adjoint (1) projection,
    // allocated on first use, invalidated by set_mask
    float *pw[2];
    int pw_valid[2];
    // relative residual^2 (FP64-accurate) that the first CG pass of the last
    // pressure solve of each kind left when it was above tol_p^2 (else 0): the
    // rounding floor of the FP32 iterate, which the next solve's first pass does
    // not try to go below
    double p_floor2[2];
    // iterations of the last CG pass of each kind: pressure [kind][refining],
    // viscosity [dirichlet]; 0 unknown. The host runs that many minus one before
    // its first read of the convergence flag.
    int it_last_p[2][2], it_last_v[2];
    int solve_kind;       // kind of the pressure solve being run
    // viscosity solve (face space)
    float *vx, *vr, *vp[2], *vq, *vz;  // vz: preconditioned residual of a multigrid viscosity solve
    // full-layout scratch fields (3 * S each, public layout)
    float *fu[3];         // u_visc when the caller does not keep it
    float *fg[3];         // adjoint cotangent being projected
    float *gc[3];         // cell space x3: per-cell cosine-loss gradient

    // MIC(0)
    float *mic_prec;      // cell space
    float *py;            // cell space: forward-substitution result
    int mic_ready;        // factor valid for the current mask and tau, sigma
    int mic_sched_ready;  // tile order valid for the current mask
    int *mic_order;       // liquid 8^3 tiles by tile level
    uint8_t *mic_tact;    // per tile: holds liquid
    int *mic_tflag;       // per tile: epoch of its last completed sweep
    int *mic_next;        // work counter of the running sweep
    int mic_n, mic_epoch, mic_ntiles;

    // learned preconditioner (fs_net.cu) and its flexible-CG direction ring
    // (fs_fcg.cu), allocated on first use
    void *net;
    void *fcg;
    void *percnn;         // recurrent convolutional pressure solver (fs_percnn.cu)
    void *splat;          // splatting scratch (fs_splat.cu)
    void *mg;             // multigrid hierarchy of the pressure preconditioner (fs_mg.cu)

    // reductions
    fs::SolveScal *scal;        // device [4]: 0 pressure, 1 viscosity, 2 misc, 3 misc
    fs::SolveScal *scal_host;   // pinned mirror
    double *partials;           // device [max_blocks * 8]
    int max_blocks;
    unsigned *err_word;         // device error word of bounded waits
    long long n_fluid;          // fluid faces
    fs::TileMap tm_cell, tm_face;    // z-marching tilings of cell and face space
    uint8_t *act_cell, *act_face;    // per tile block: 1 if it holds an active element
    int *list_cell, *list_face;      // the active tiles, in tile order
    int nact_cell, nact_face;
    // per listed tile, 8 words (one per tile row) with bit q set when quad q of
    // that row holds an active element
    unsigned *qmask_cell, *qmask_face;
    // z-marching work of the operator apply: {column, k0, k1, 0} chunks of active planes
    int4 *items_cell, *items_face;
    int nitems_cell, nitems_face;
    // tensor maps of the vectors the operator apply reads (3-D: pitch x rows x
    // planes of the guarded space, 136 x 10 x 1 boxes)
    CUtensorMap tmz_pr, tmz_pz, tmz_pp[2], tmz_vr, tmz_vp[2], tmz_vz;

    // per-kernel timing (fs_profile)
    int prof_on;
    int prof_period;            // time every prof_period-th CG iteration
    void *prof;                 // fs::Prof
    long long n_launches;       // kernels launched by this context since fs_profile(c, 1)
};

namespace fs {

int set_error(int code, const char *fmt, ...);
int check_cuda(cudaError_t e, const char *what);
#define FS_CUDA(call)                                              \
    do {                                                           \
        int _rc = ::fs::check_cuda((call), #call);                 \
        if (_rc) return _rc;                                       \
    } while (0)

inline int grid_blocks(const fs_ctx *c, long long n, int threads, int per_thread = 1)
{
    long long need = (n + (long long)threads * per_thread - 1) / ((long long)threads * per_thread);
    if (need < 1) need = 1;
    return (int)(need < c->max_blocks ? need : c->max_blocks);
}

// Resident 256-thread blocks per SM of a kernel with `dyn` bytes of dynamic
// shared memory; raises the kernel's dynamic shared memory limit to `dyn` on
// first use.
inline int resident_blocks(const void *fn, size_t dyn)
{
    if (dyn > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, dyn) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

// Blocks of a grid-stride launch of 256-thread blocks over n items for a kernel
// with `resident` blocks per SM: at most one full wave. A grid of max_blocks for
// a kernel that fits fewer blocks per SM would run its last blocks in a second,
// mostly empty wave, each with as much work as the first wave's.
inline int wave_blocks(const fs_ctx *c, long long n, int resident)
{
    long long need = (n + 255) / 256;
    if (need < 1) need = 1;
    const long long cap = (long long)c->num_sms * (resident > 0 ? resident : 1);
    return (int)(need < cap ? need : cap);
}

// ---- deterministic grid reduction ------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Compensated FP32 accumulation (Kahan): keeps per-thread partial sums of FP32
// products accurate to about one FP32 rounding before the FP64 tree.
// Error-free sum (Knuth's TwoSum): a + b = s + e exactly, s = fl(a + b).
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Sums K doubles over the grid. Each block writes its partials; the last block
// to arrive adds the partials in block order (so the result does not depend on
// scheduling) and returns true in all its threads with the totals in `tot`
// (valid in thread 0). Requires blockDim.x * blockDim.y a multiple of 32,
// <= 1024, and a one-dimensional grid.
template <int K>
__device__ __forceinline__ bool grid_reduce(double (&v)[K], double *partials, unsigned *ticket,
                                            double (&tot)[K])
{
    __shared__ double sh[32][K];
    __shared__ int last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sh[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double t = lane < nw ? sh[lane][k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) partials[(size_t)blockIdx.x * K + k] = t;
        }
        if (lane == 0) {
            __threadfence();
            unsigned t = atomicAdd(ticket, 1u);
            last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = 0.0;
        for (int b = tid; b < (int)gridDim.x; b += nthr)
            t += __ldcg(&partials[(size_t)b * K + k]);
        tot[k] = warp_sum(t);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sh[wid][k] = tot[k];
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double t = 0.0;
            for (int w = 0; w < nw; w++) t += sh[w][k];
            tot[k] = t;
        }
        *ticket = 0u;
    }
    return true;
}

// The same grid sum over compensated FP32 pairs, with no FP64 arithmetic before
// the final conversion (FP64 shuffles and adds are slow on this part: a grid of
// 1216 blocks took 12.3 us with the FP64 tree above and 8.2 us with this one).
// A pair (s, c) stands for s - c, as in KSum. Two pairs merge by Knuth's TwoSum:
// t = s1 + s2 with its rounding error e recovered exactly, so
// (s1 - c1) + (s2 - c2) = t - (c1 + c2 - e). The merge tree is fixed (lanes,
// then warps, then the partials in block order, strided over the last block's
// threads), so the totals do not depend on scheduling. Each pair goes to the
// partials buffer as a float2 (8 bytes per value, like a double). The totals
// are valid in thread 0 of the last block.
__device__ __forceinline__ void ks_merge(float &s, float &c, float s2, float c2)
{
    const float t = s + s2;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (s2 - bp);  // t + e == s + s2 exactly
    s = t;
    c = (c + c2) - e;
}

template <int K>
__device__ __forceinline__ void ks_warp(KSum (&v)[K])
{
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, v[k].s, o);
            const float c2 = __shfl_xor_sync(0xffffffffu, v[k].c, o);
            ks_merge(v[k].s, v[k].c, s2, c2);
        }
}

// block sum of pairs; true in warp 0, whose lanes all hold the block's totals
template <int K>
__device__ __forceinline__ bool ks_block(KSum (&v)[K])
{
    __shared__ float shs[32][K], shc[32][K];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nw = (blockDim.x * blockDim.y) >> 5;
    const int lane = tid & 31, wid = tid >> 5;
    ks_warp<K>(v);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) {
            shs[wid][k] = v[k].s;
            shc[wid][k] = v[k].c;
        }
    __syncthreads();
    if (wid != 0) return false;
#pragma unroll
    for (int k = 0; k < K; k++) {
        v[k].s = lane < nw ? shs[lane][k] : 0.f;
        v[k].c = lane < nw ? shc[lane][k] : 0.f;
    }
    ks_warp<K>(v);
    return true;
}

// A block's arrival at the ticket of a grid sum, by the thread that wrote the
// block's partials: an atomic add with release semantics (the partials are
// visible before the count) and acquire semantics (the last block to arrive sees
// every partial once its threads pass the barrier that follows), at device
// scope, in place of a full fence before and after a relaxed add.
__device__ __forceinline__ unsigned ticket_arrive(unsigned *ticket)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(ticket) : "memory");
    return old;
}

// The last block's share of the merge: thread tid takes the partials of blocks
// tid, tid + nthr, ... in that order. The loads of U of them are issued before
// the first merge, so the thread waits for about one L2 round trip per U
// partials instead of one per partial (U sized so that the merge needs no more
// registers than the streaming loops of the kernels it ends).
template <int K>
__device__ __forceinline__ void ks_gather(KSum (&v)[K], const float2 *pp, int nblocks, int tid, int nthr)
{
    constexpr int U = K == 1 ? 8 : 1;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = KSum();
    for (int b0 = tid; b0 < nblocks; b0 += U * nthr) {
        float2 q[U][K];
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
            for (int k = 0; k < K; k++)
                q[u][k] = b0 + u * nthr < nblocks ? __ldcg(&pp[(size_t)(b0 + u * nthr) * K + k])
                                                  : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (b0 + u * nthr < nblocks)
#pragma unroll
                for (int k = 0; k < K; k++) ks_merge(v[k].s, v[k].c, q[u][k].x, q[u][k].y);
    }
}

template <int K>
__device__ __forceinline__ bool grid_reduce(KSum (&v)[K], double *partials, unsigned *ticket, double (&tot)[K])
{
    __shared__ int last;
    float2 *pp = reinterpret_cast<float2 *>(partials);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
    if (ks_block<K>(v) && tid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) pp[(size_t)blockIdx.x * K + k] = make_float2(v[k].s, v[k].c);
        last = ticket_arrive(ticket) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    ks_gather<K>(v, pp, (int)gridDim.x, tid, nthr);
    __syncthreads();  // the shared staging of ks_block is reused
    if (ks_block<K>(v) && tid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) tot[k] = (double)v[k].s - (double)v[k].c;
        *ticket = 0u;
    }
    return true;
}

// grid_reduce over the blocks of several launches that run at once (the face
// volumes' V-cycles on their streams): this block is number `block` of `nblocks`
// in all; the partials are merged in that order by the last block to arrive, in
// whichever launch it is.
template <int K>
__device__ __forceinline__ bool multi_reduce(KSum (&v)[K], double *partials, unsigned *ticket, double (&tot)[K],
                                             int block, int nblocks)
{
    __shared__ int last;
    float2 *pp = reinterpret_cast<float2 *>(partials);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
    if (ks_block<K>(v) && tid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) pp[(size_t)block * K + k] = make_float2(v[k].s, v[k].c);
        last = ticket_arrive(ticket) == (unsigned)nblocks - 1;
    }
    __syncthreads();
    if (!last) return false;
    ks_gather<K>(v, pp, nblocks, tid, nthr);
    __syncthreads();  // the shared staging of ks_block is reused
    if (ks_block<K>(v) && tid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) tot[k] = (double)v[k].s - (double)v[k].c;
        *ticket = 0u;
    }
    return true;
}

// ---- launchers implemented in the .cu files --------------------------------
// fs_mask.cu
int build_mask(fs_ctx *c, const uint8_t *types_dense, const fs_mac *bc);
TileMap make_tilemap(const Layout &L, int nvol, int num_sms);
int make_tensor_maps(fs_ctx *c);   // fs_mask.cu, once per context
int zmarch_slots(const fs_ctx *c, bool face);  // fs_pcg.cu: resident blocks of the operator apply
// fs_pcg.cu
int solve_pressure(fs_ctx *c, fs_stats *st);             // pb -> px
int solve_viscosity(fs_ctx *c, bool dirichlet, fs_stats *st);  // vx (guess, rhs) -> vx
int precond_apply_public(fs_ctx *c, const float *r, float *z);  // public cell arrays
int launch_divergence(fs_ctx *c, CF3 u);                 // u -> pb, with bb/mean handling
int launch_grad_subtract(fs_ctx *c, CF3 in, F3 out, float *q_out);
int launch_compose(fs_ctx *c, F3 out);                   // vx + bc -> full field
int launch_mask_fluid(fs_ctx *c, CF3 in, F3 out);        // zero off fluid faces
int launch_to_face_space(fs_ctx *c, CF3 in);             // full field (fluid) -> vx
int launch_nu_grad(fs_ctx *c, CF3 uv, double *dot);      // <vx, L~ uv>
int launch_loss(fs_ctx *c, CF3 u, CF3 t, int kind, double alpha, double beta, F3 g,
                double *loss);
// fs_mg.cu
int mg_apply(fs_ctx *c, const float *r, float *z, const int *done);
int mg_apply_faces(fs_ctx *c, const float *r, float *z, float cc, const int *done);
void mg_free(fs_ctx *c);
void mg_count(fs_ctx *c, long long vcycles, bool faces);  // fs_mg.cu: launch counts for fs_profile
int mg_levels(const fs_ctx *c);
bool mg_level0_lists(const fs_ctx *c, bool faces, const int **ql, int *n, long long *base);  // fs_mg.cu
int pressure_pair(fs_ctx *c, float *q_hi, float *q_lo);  // fs_pcg.cu
bool mg_rz(fs_ctx *c, bool faces, const float *r, const float *z, int first, SolveScal *s);  // fs_mg.cu
// z = M r with r.z formed in the V-cycle's last level-0 sweep (beta = rz_new / rz,
// first: beta = 0, as k_rz); false when the hierarchy has no such sweep (a level
// 0 that is its own coarsest level): then z is formed but r.z is not
bool mg_apply_rz(fs_ctx *c, const float *r, float *z, const int *done, SolveScal *s, int first, int &rc);
bool mg_apply_faces_rz(fs_ctx *c, const float *r, float *z, float cc, const int *done, SolveScal *s, int first,
                       int &rc);
// fs_splat.cu
int splat_render(fs_ctx *c, int n, const float *x, const float *op, const float *A, const float *col,
                 const float *sh, int deg, const fs_camera *cam, float *rgb, float *T);
void splat_free(fs_ctx *c);
void splat_stats(const fs_ctx *c, unsigned long long *entries, unsigned long long *max_tile);
// fs_apic.cu
int launch_p2g(fs_ctx *c, int np, const float *x, const float *v, const float *C, const float *m, F3 u, F3 mass);
int launch_g2p(fs_ctx *c, int np, float *x, float *v, float *C, float *F, const float *A0, float *A, CF3 u,
               double dt, int advance, double lo, double hi);
// fs_volume.cu
int launch_wall_profile(fs_ctx *c, const double dir[3], const float *vinf, double delta, F3 u);
int launch_pbd_project(fs_ctx *c, F3 u, int hold, int iters, double eps, double *norm);
// fs_advect.cu
int launch_advect(fs_ctx *c, CF3 u);                     // u -> vx (fluid faces)
int launch_advect_adjoint(fs_ctx *c, CF3 u, F3 g);       // vx cotangent -> g (+=)
// fs_mic0.cu
int mic0_factor(fs_ctx *c);
int mic0_apply(fs_ctx *c, const float *r, float *z);
// fs_net.cu
int net_alloc(fs_ctx *c, bool training);
void net_free(fs_ctx *c);
int net_load(fs_ctx *c, const float *params, int count, bool host);
int net_read(fs_ctx *c, float *params_host);
int net_kernel(fs_ctx *c, int which);  // fs_net.cu: inference layers, 0 mma.sync, 1 tcgen05
int check_wait_error(fs_ctx *c, const char *what);  // fs_pcg.cu: bounded-wait errors of the last solve
int net_apply(fs_ctx *c, const float *r, float *z);   // cell space
int net_grad(fs_ctx *c, const float *b, const float *q, double *loss);  // public layout
int net_adam(fs_ctx *c, double lr, double beta1, double beta2, double eps, int step, double gscale,
             int fix_offsets);
int net_grad_read(fs_ctx *c, float *grad_host);
int adam_update(fs_ctx *c, float *p, const float *g, float *m, float *v, long long n, double lr, double beta1,
                double beta2, double eps, int step, double grad_scale);  // fs_optim.cu
int net_grad_clear(fs_ctx *c);
int net_param_count();
bool net_loaded(const fs_ctx *c);
// public cell array -> cell space, zero off liquid
int cell_in(fs_ctx *c, const float *src, float *dst);
int cell_out(fs_ctx *c, const float *src, float *dst);  // cell space -> public cell array

int read_scal(fs_ctx *c, int which, SolveScal *out);
// mean-free preconditioned residual over the liquid when the operator is singular
int remove_null_mode(fs_ctx *c, float *z);
// fs_fcg.cu: flexible CG with the network, pb -> px (warm: from the current x);
// final scalars in *h
int learned_apply(fs_ctx *c, const float *r, float *z, const int *done);  // fs_pcg.cu: network (+ V-cycle)
int solve_pressure_fcg(fs_ctx *c, SolveScal *h, bool warm);
int pressure_restart(fs_ctx *c);  // fs_pcg.cu: r = b - A x, p = 0 (scalars of slot 0)
void fcg_release(fs_ctx *c);
// fs_percnn.cu: recurrent convolutional pressure solver, pb -> px
int percnn_load(fs_ctx *c, const float *w27, int K);
int percnn_read(fs_ctx *c, float *w27, int *K);
bool percnn_loaded(const fs_ctx *c);
void percnn_free(fs_ctx *c);
int solve_pressure_percnn(fs_ctx *c, SolveScal *h);
int percnn_grad(fs_ctx *c, const float *b, const float *q, double *loss, float *dw_host);

// ---- per-kernel timing -------------------------------------------------------
enum KernelId : int {
    K_P_SPMV = 0,
    K_P_UPDATE,
    K_V_SPMV,
    K_V_UPDATE,
    K_ADVECT,
    K_ADVECT_ADJ,
    K_MIC_APPLY,
    K_NET_APPLY,
    K_FCG_VEC,
    K_MG_VCYCLE_P,  // one pressure V-cycle (time only)
    K_MG_VCYCLE_V,  // one viscosity V-cycle over the three face volumes (time only)
    // level 0 of a V-cycle, one entry per kernel (timed on the pressure V-cycle;
    // launches counted over the pressure and the face-volume V-cycles)
    K_MG0_SMOOTH2,   // the two pre-smoothing sweeps from zero
    K_MG0_RESIDUAL,  // the residual after them
    K_MG0_RESTRICT,  // its restriction to level 1
    K_MG0_PROLONG,   // the prolongation of the level-1 correction
    K_MG0_SMOOTH,    // the first post-smoothing sweep
    K_MG0_SMOOTH_Z,  // the last post-smoothing sweep, which writes z densely
    K_MG_COARSE,     // levels 1 and below of a pressure V-cycle (time only)
    K_COUNT
};
cudaEvent_t prof_mark(fs_ctx *c);   // records an event on the stream (nullptr when off)
void prof_add(fs_ctx *c, int id, cudaEvent_t a, cudaEvent_t b, double bytes);
void prof_count(fs_ctx *c, int id, long long launches);  // launches of a kind, timed or not
void prof_flush(fs_ctx *c);         // call after the stream has been synchronised

}  // namespace fs
