// fs_tma.cuh -- the operator apply of both CG solves with TMA-fed shared memory
// (included by fs_pcg.cu, which defines PoisOp and HelmOp).
//
// Operator apply (k_spmv_z): a block owns a 128 x 8 column of one volume and
// marches it along z over a chunk of planes [k0, k1). For every plane it needs,
// one elected thread issues two tensor copies (cp.async.bulk.tensor) of the
// 136 x 10 box around the column (x from i0-4, y from j0-1; the tensor copy
// fills everything outside the array with zeros) -- one of z, one of p_old --
// Z_NS planes ahead, into a ring of stage buffers completed by mbarriers. The
// block forms p_new = z + beta p_old for the whole box once per plane, into a
// ring of four p_new planes, and computes q = A p_new for the plane below the
// newest one from that ring. Each plane of z and p_old thus comes from HBM once
// per column (plus two planes per chunk), with several planes in flight per
// block independent of the register budget.
//
// Every mbarrier wait is bounded. A block whose wait runs out records bit 2 in
// the error word, waits (bounded again) for its own copies still in flight and
// leaves its loops, but still takes part in the grid reduction; the block that
// finishes the reduction then ends the solve with FS_ETIMEOUT.
#pragma once

#include <cuda.h>

namespace fs {
namespace {

constexpr int ZB_W = TILE_X + 8;           // box row: x from i0 - 4 to i0 + 131
constexpr int ZB_H = TILE_Y + 2;           // box rows: j0 - 1 .. j0 + 8
constexpr int ZB_ELEMS = ZB_W * ZB_H;      // 1360 floats
constexpr int ZB_BYTES = ZB_ELEMS * 4;     // 5440 bytes per box
constexpr int ZB_PITCH = 5504;             // stage buffer stride, a multiple of 128 bytes
constexpr int Z_NS = 2;                    // planes in flight per block
constexpr int Z_RING = 4;                  // p_new planes kept
constexpr unsigned TMA_SPIN = 1u << 26;    // try_wait rounds before a wait gives up
constexpr unsigned ERR_TMA = 2u;

constexpr size_t zmarch_smem() { return 128 + (size_t)Z_NS * 2 * ZB_PITCH + (size_t)Z_RING * ZB_BYTES + Z_NS * 8; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned char *align128(unsigned char *p)
{
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) & ~(uintptr_t)127);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// true when the phase with this parity completed within the spin budget
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (unsigned n = 0; n < TMA_SPIN; n++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 3-D tiled tensor copy global -> shared, completing on `bar`. The x coordinate
// must be a multiple of 4 floats (16 bytes); the callers pass i0 - 4 or i0 with
// i0 a multiple of TILE_X.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uchar4 ld_flags(const uint8_t *__restrict__ fl, int t)
{
    return __ldg(reinterpret_cast<const uchar4 *>(fl + t));
}

// ---------------------------------------------------------------------------
// q = A p_new, p_new = z + beta p_old, partial sums of p_new . q; alpha at the end.
// items[i] = {column, k0, k1, 0}, column = (v * nty + tyi) * ntx + txi.
template <class Op>
__global__ void __launch_bounds__(256) k_spmv_z(const __grid_constant__ CUtensorMap mz,
                                                const __grid_constant__ CUtensorMap mo, float *__restrict__ pnew,
                                                float *__restrict__ q, const uint8_t *__restrict__ fl,
                                                const int4 *__restrict__ items, int nitems, TileMap M, float cc,
                                                SolveScal *s, double *partials, unsigned *err)
{
    if (s->done) return;
    extern __shared__ unsigned char dyn_smem[];
    unsigned char *base = align128(dyn_smem);
    float *ring = reinterpret_cast<float *>(base + Z_NS * 2 * ZB_PITCH);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + Z_NS * 2 * ZB_PITCH + Z_RING * ZB_BYTES);
    __shared__ float dtab[8], itab[8];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    fill_diag_tables<Op>(dtab, itab, cc);
    if (tid == 0) {
        for (int i = 0; i < Z_NS; i++) mbar_init(bar + i, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const float beta = (float)s->beta;
    const float oc = Op::offc(cc);
    KSum acc;
    unsigned gbase = 0;  // plane loads of earlier items (the same in every thread)
    int cons = 0, issued = 0;  // of the current item
    bool bad = false;
    int it = blockIdx.x;
    for (; it < nitems; it += gridDim.x) {
        const int4 w = __ldg(items + it);
        const int txi = w.x % M.ntx, tyi = (w.x / M.ntx) % M.nty, v = w.x / (M.ntx * M.nty);
        const int k0 = w.y, k1 = w.z;
        const int L = k1 - k0 + 2;  // planes k0 - 1 .. k1
        const int i0 = txi * TILE_X, j0 = tyi * TILE_Y;
        const int orgv = M.origin0 + v * M.vstride;
        const int plane0 = orgv / M.PL;  // tensor plane of this volume's plane 0
        __syncthreads();                  // the previous item's readers are done
        issued = L < Z_NS ? L : Z_NS;
        if (tid == 0) {
            for (int m = 0; m < issued; m++) {
                const int st = (int)((gbase + m) % Z_NS);
                unsigned char *sb = base + st * 2 * ZB_PITCH;
                mbar_expect_tx(bar + st, 2 * ZB_BYTES);
                tma_load_3d(sb, &mz, i0 - 4, j0 - 1, plane0 + k0 - 1 + m, bar + st);
                tma_load_3d(sb + ZB_PITCH, &mo, i0 - 4, j0 - 1, plane0 + k0 - 1 + m, bar + st);
            }
        }
        const int i = i0 + 4 * tx, j = j0 + ty;
        const bool own = i < M.P && j < M.R;
        const int trow = orgv + j * M.P + i;  // + k * PL
        // flag bytes of the next three output planes, loaded ahead
        const uchar4 f0 = make_uchar4(0, 0, 0, 0);
        uchar4 fq0 = own ? ld_flags(fl, trow + k0 * M.PL) : f0;
        uchar4 fq1 = (own && k0 + 1 < k1) ? ld_flags(fl, trow + (k0 + 1) * M.PL) : f0;
        uchar4 fq2 = (own && k0 + 2 < k1) ? ld_flags(fl, trow + (k0 + 2) * M.PL) : f0;
        for (cons = 0; cons < L; cons++) {
            const int m = cons;
            const unsigned g = gbase + m;
            const int st = (int)(g % Z_NS);
            // warp 0 waits for the plane's copies; the block barrier passes the
            // completed phase (and the data it guards) on to the other warps
            const bool ok = ty != 0 || mbar_wait_bounded(bar + st, (g / Z_NS) & 1u);
            bad = __syncthreads_or(!ok);
            if (bad) break;
            {
                const float4 *bz = reinterpret_cast<const float4 *>(base + st * 2 * ZB_PITCH);
                const float4 *bo = reinterpret_cast<const float4 *>(base + st * 2 * ZB_PITCH + ZB_PITCH);
                float4 *dst = reinterpret_cast<float4 *>(ring + (m % Z_RING) * ZB_ELEMS);
                for (int e = tid; e < ZB_ELEMS / 4; e += 256) dst[e] = fma4(bz[e], beta, bo[e]);
            }
            __syncthreads();
            // stage st is free again: the plane Z_NS ahead goes into it
            if (m + Z_NS < L) {
                if (tid == 0) {
                    unsigned char *sb = base + st * 2 * ZB_PITCH;
                    mbar_expect_tx(bar + st, 2 * ZB_BYTES);
                    tma_load_3d(sb, &mz, i0 - 4, j0 - 1, plane0 + k0 - 1 + m + Z_NS, bar + st);
                    tma_load_3d(sb + ZB_PITCH, &mo, i0 - 4, j0 - 1, plane0 + k0 - 1 + m + Z_NS, bar + st);
                }
                issued++;
            }
            if (m < 2) continue;
            // q for plane k from the p_new planes k - 1, k, k + 1
            const int k = k0 + m - 2;
            const uchar4 fc = fq0;
            fq0 = fq1;
            fq1 = fq2;
            fq2 = (own && k + 3 < k1) ? ld_flags(fl, trow + (k + 3) * M.PL) : f0;
            if (own && ((fc.x | fc.y | fc.z | fc.w) & Op::ACTIVE)) {
                const float *rm = ring + ((m - 2) % Z_RING) * ZB_ELEMS;
                const float *rc = ring + ((m - 1) % Z_RING) * ZB_ELEMS;
                const float *rp = ring + (m % Z_RING) * ZB_ELEMS;
                const int o = (ty + 1) * ZB_W + 4 + 4 * tx;
                const float4 pc = *reinterpret_cast<const float4 *>(rc + o);
                const float4 dn = *reinterpret_cast<const float4 *>(rc + o - ZB_W);
                const float4 up = *reinterpret_cast<const float4 *>(rc + o + ZB_W);
                const float4 pm = *reinterpret_cast<const float4 *>(rm + o);
                const float4 pp = *reinterpret_cast<const float4 *>(rp + o);
                const float lf = rc[o - 1], rt = rc[o + 4];
                float4 qv;
                qv.x = (fc.x & Op::ACTIVE) ? dtab[fc.x & 7] * pc.x - oc * ((lf + pc.y) + (dn.x + up.x) + (pm.x + pp.x)) : 0.f;
                qv.y = (fc.y & Op::ACTIVE) ? dtab[fc.y & 7] * pc.y - oc * ((pc.x + pc.z) + (dn.y + up.y) + (pm.y + pp.y)) : 0.f;
                qv.z = (fc.z & Op::ACTIVE) ? dtab[fc.z & 7] * pc.z - oc * ((pc.y + pc.w) + (dn.z + up.z) + (pm.z + pp.z)) : 0.f;
                qv.w = (fc.w & Op::ACTIVE) ? dtab[fc.w & 7] * pc.w - oc * ((pc.z + rt) + (dn.w + up.w) + (pm.w + pp.w)) : 0.f;
                const int t = trow + k * M.PL;
                *reinterpret_cast<float4 *>(pnew + t) = pc;
                *reinterpret_cast<float4 *>(q + t) = qv;
                acc.add(pc.x * qv.x + pc.y * qv.y + pc.z * qv.z + pc.w * qv.w);
            }
        }
        if (bad) break;
        gbase += (unsigned)L;
    }
    if (bad) {
        // wait (bounded) for this block's copies still in flight, then report
        if (tid == 0) {
            for (int m = cons; m < issued; m++) {
                const unsigned g = gbase + m;
                mbar_wait_bounded(bar + g % Z_NS, (g / Z_NS) & 1u);
            }
            atomicOr(err, ERR_TMA);
        }
        __syncthreads();
    }
    KSum vv[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(vv, partials, &s->ticket, tot) && threadIdx.x == 0 && threadIdx.y == 0) {
        const double pq = tot[0];
        s->pq = pq;
        if (__ldcg(err) & ERR_TMA) { s->done = 1; s->status = FS_ETIMEOUT; }
        else if (!isfinite(pq)) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (!(pq > 0.0)) { s->done = 1; s->status = FS_EBREAKDOWN; }
        else s->alpha = s->rz / pq;
    }
}

}  // namespace
}  // namespace fs
