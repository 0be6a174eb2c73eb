// fs_splat.cu -- forward splatting of the Gaussians into an image (arXiv
// 2503.00868, Sec. 3.2.1 compositing formula, Sec. 3.5 rendering by splatting),
// into a headless device buffer.
//
// Per Gaussian (pinhole camera, x_c = R x + t): depth z, projected mean, 2D
// covariance S = J R A R^T J^T (J the projection Jacobian at the mean) and its
// inverse (the conic). At a pixel centre d = pixel - mean,
//   alpha = min(0.99, sigma exp(-d^T S^-1 d / 2)), kept inside the 3-sigma ellipse
//   (d^T S^-1 d <= 9) and when alpha >= 1/255,
// and the pixel composites front to back by depth (ties by index):
//   C = sum_i alpha_i c_i T_i + T bg,  T_i = prod_{j<i} (1 - alpha_j),
// stopping once the transmittance would fall below 1e-4. Colours are degree-0
// spherical harmonics (RGB).
//
// Pipeline: (1) project, record each Gaussian's tile rectangle (16 x 16 pixel
// tiles covering the 3-sigma ellipse's bounding box) and count entries per tile;
// (2) exclusive scan of the counts (one block); (3) write (depth bits << 32 | index)
// keys into each tile's segment; (4) a tile with more than SP_CAP keys is sorted in
// place by one block (stable LSD radix sort, 8-bit digits, through a ping-pong
// buffer); (5) one block per tile sorts a segment of at most SP_CAP keys in shared
// memory (bitonic) and composites, one thread per pixel, in batches of records
// staged in shared memory. Every sort orders the full 64-bit key, so equal depths
// fall back to index order whatever order the atomics filled the segment in.
#include <cmath>
#include <new>

#include "fs_internal.cuh"

namespace fs {

struct SplatRecord {
    float mx, my;          // projected mean (pixels)
    float ca, cb, cc;      // conic: S^-1 = [[ca, cb], [cb, cc]]
    float opacity;
    float r, g, b;
};

struct SplatState {
    SplatRecord *rec = nullptr;
    int4 *rect = nullptr;            // tile rectangle [x0, x1) x [y0, y1)
    float *depth = nullptr;
    int cap_n = 0;
    unsigned *tcount = nullptr, *toff = nullptr, *tfill = nullptr;
    int cap_t = 0;
    unsigned long long *keys = nullptr, *keys2 = nullptr;
    long long cap_k = 0, cap_k2 = 0;
    unsigned long long last_entries = 0, last_max = 0;  // counters of the last render
};

namespace {

constexpr int SP_TILE = 16;
constexpr int SP_CAP = 4096;   // keys per tile sorted in shared memory

struct Cam {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int w, h;
    float znear;
    float bg[3];
};

// Block-local table of tiles (open addressing, linear probing, no deletion): the
// (Gaussian, tile) pairs of a block's 256 Gaussians, which are usually neighbours
// in space and share tiles, are counted in shared memory and reach the global
// per-tile counters with one atomic per distinct tile. A tile that finds no slot
// within SP_PROBE probes goes to the global counter directly; since slots are
// never freed, a later lookup of that tile fails the same way.
constexpr int SP_HT = 1024;
constexpr int SP_PROBE = 16;
constexpr unsigned SP_EMPTY = 0xffffffffu;

__device__ __forceinline__ int ht_slot(unsigned *hk, unsigned t, bool insert)
{
    const unsigned h = (t * 2654435761u) >> 22;
    for (int p = 0; p < SP_PROBE; p++) {
        const unsigned sl = (h + p) & (SP_HT - 1);
        unsigned cur = hk[sl];
        if (cur == t) return (int)sl;
        if (cur == SP_EMPTY) {
            if (!insert) return -1;
            cur = atomicCAS(hk + sl, SP_EMPTY, t);
            if (cur == SP_EMPTY || cur == t) return (int)sl;
        }
    }
    return -1;
}

// View-dependent colour (Sec. 3.2.1, SH(r; F_i)): max(0, 1/2 + sum_j sh[j] Y_j(d))
// per channel, with the real spherical harmonics Y_j of degree <= 3 in the sign
// convention of the standard 3DGS evaluator and d the unit vector from the camera
// centre to the mean. The constants are the normalisations of the basis:
// sqrt(3/4pi), sqrt(15/4pi), sqrt(5/16pi), sqrt(15/16pi), sqrt(35/32pi),
// sqrt(105/4pi), sqrt(21/32pi), sqrt(7/16pi).
__device__ __forceinline__ void sh_colour(int deg, const float *__restrict__ sh, float dx, float dy, float dz,
                                          float out[3])
{
    constexpr float Y0 = 0.28209479177387814f, A1 = 0.4886025119029199f;
    constexpr float B2 = 1.0925484305920792f, C2 = 0.31539156525252005f, E2 = 0.5462742152960396f;
    constexpr float F3 = 0.5900435899266435f, G3 = 2.890611442640554f, H3 = 0.4570457994644658f,
                    K3 = 0.3731763325901154f;
    float Y[16];
    Y[0] = Y0;
    if (deg >= 1) {
        Y[1] = -A1 * dy;
        Y[2] = A1 * dz;
        Y[3] = -A1 * dx;
    }
    if (deg >= 2) {
        const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
        Y[4] = B2 * dx * dy;
        Y[5] = -B2 * dy * dz;
        Y[6] = C2 * (2.f * zz - xx - yy);
        Y[7] = -B2 * dx * dz;
        Y[8] = E2 * (xx - yy);
        if (deg >= 3) {
            Y[9] = -F3 * dy * (3.f * xx - yy);
            Y[10] = G3 * dx * dy * dz;
            Y[11] = -H3 * dy * (4.f * zz - xx - yy);
            Y[12] = K3 * dz * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -H3 * dx * (4.f * zz - xx - yy);
            Y[14] = 0.5f * G3 * dz * (xx - yy);
            Y[15] = -F3 * dx * (xx - 3.f * yy);
        }
    }
    const int nb = (deg + 1) * (deg + 1);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float v = 0.5f;
        for (int j = 0; j < nb; j++) v += sh[3 * j + k] * Y[j];
        out[k] = fmaxf(v, 0.f);
    }
}

// Projection, colour and tile counting of each Gaussian. The colour is col[i]
// (RGB) or, with sh non-null, the spherical-harmonic colour of degree `deg`
// seen from the camera centre.
__global__ void __launch_bounds__(256) k_sp_project(int n, const float *__restrict__ x,
                                                    const float *__restrict__ op, const float *__restrict__ A,
                                                    const float *__restrict__ col, const float *__restrict__ sh,
                                                    int deg, Cam cam, SplatRecord *rec, int4 *rect, float *depth,
                                                    unsigned *tcount, int ntx, int nty)
{
    __shared__ unsigned hk[SP_HT], hc[SP_HT];
    for (int base = blockIdx.x * 256; base < n; base += gridDim.x * 256) {  // uniform over the block
        for (int e = threadIdx.x; e < SP_HT; e += 256) {
            hk[e] = SP_EMPTY;
            hc[e] = 0;
        }
        __syncthreads();
        const int i = base + threadIdx.x;
        int4 rc = make_int4(0, 0, 0, 0);
        float xc[3];
        const int ii = min(i, n - 1);  // rows past n: read a valid row, record nothing
#pragma unroll
        for (int r = 0; r < 3; r++)
            xc[r] = cam.R[3 * r] * x[3 * ii] + cam.R[3 * r + 1] * x[3 * ii + 1] + cam.R[3 * r + 2] * x[3 * ii + 2] +
                    cam.t[r];
        const float z = xc[2];
        if (i < n && z > cam.znear) {
            const float mx = cam.fx * xc[0] / z + cam.cx, my = cam.fy * xc[1] / z + cam.cy;
            const float J[6] = {cam.fx / z, 0.f, -cam.fx * xc[0] / (z * z), 0.f, cam.fy / z, -cam.fy * xc[1] / (z * z)};
            float M[6];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    M[3 * r + c] = J[3 * r] * cam.R[c] + J[3 * r + 1] * cam.R[3 + c] + J[3 * r + 2] * cam.R[6 + c];
            float S[4];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    float acc = 0.f;
#pragma unroll
                    for (int a = 0; a < 3; a++)
#pragma unroll
                        for (int b = 0; b < 3; b++) acc += M[3 * r + a] * A[9 * i + 3 * a + b] * M[3 * s + b];
                    S[2 * r + s] = acc;
                }
            const float det = S[0] * S[3] - S[1] * S[2];
            if (det > 0.f && S[0] > 0.f && S[3] > 0.f) {
                SplatRecord q;
                q.mx = mx;
                q.my = my;
                q.ca = S[3] / det;
                q.cb = -S[1] / det;
                q.cc = S[0] / det;
                q.opacity = op[i];
                if (sh) {
                    // the camera centre -R^T t and the unit direction to the mean
                    float d[3], nrm = 0.f;
#pragma unroll
                    for (int r = 0; r < 3; r++) {
                        const float cr = -(cam.R[r] * cam.t[0] + cam.R[3 + r] * cam.t[1] + cam.R[6 + r] * cam.t[2]);
                        d[r] = x[3 * i + r] - cr;
                        nrm += d[r] * d[r];
                    }
                    const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                    float cv[3];
                    sh_colour(deg, sh + (size_t)i * (deg + 1) * (deg + 1) * 3, d[0] * inv, d[1] * inv, d[2] * inv, cv);
                    q.r = cv[0];
                    q.g = cv[1];
                    q.b = cv[2];
                } else {
                    q.r = col[3 * i];
                    q.g = col[3 * i + 1];
                    q.b = col[3 * i + 2];
                }
                rec[i] = q;
                depth[i] = z;
                // the 3-sigma ellipse lies in mean +- 3 sqrt(diag S); pixel centres at p + 1/2
                const float ex = 3.f * sqrtf(S[0]) + 1.f, ey = 3.f * sqrtf(S[3]) + 1.f;
                const float x0 = fmaxf(mx - ex, 0.f), x1 = fminf(mx + ex, (float)cam.w);
                const float y0 = fmaxf(my - ey, 0.f), y1 = fminf(my + ey, (float)cam.h);
                if (x0 < x1 && y0 < y1) {
                    rc.x = min((int)(x0 / SP_TILE), ntx - 1);
                    rc.y = min((int)(x1 / SP_TILE), ntx - 1) + 1;
                    rc.z = min((int)(y0 / SP_TILE), nty - 1);
                    rc.w = min((int)(y1 / SP_TILE), nty - 1) + 1;
                }
            }
        }
        if (i < n) rect[i] = rc;
        for (int ty = rc.z; ty < rc.w; ty++)
            for (int tx = rc.x; tx < rc.y; tx++) {
                const unsigned t = (unsigned)(ty * ntx + tx);
                const int sl = ht_slot(hk, t, true);
                if (sl >= 0)
                    atomicAdd(hc + sl, 1u);
                else
                    atomicAdd(tcount + t, 1u);
            }
        __syncthreads();
        for (int e = threadIdx.x; e < SP_HT; e += 256)
            if (hk[e] != SP_EMPTY) atomicAdd(tcount + hk[e], hc[e]);
        __syncthreads();
    }
}

// exclusive scan of the tile counts, one block of 1024 threads; total[0] = the
// number of entries, total[1] = the largest tile count
__global__ void __launch_bounds__(1024) k_sp_scan(const unsigned *__restrict__ cnt, unsigned *off, int nt,
                                                  unsigned long long *total)
{
    __shared__ unsigned long long part[1024];
    __shared__ unsigned pmax[1024];
    const int per = (nt + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(lo + per, nt);
    unsigned long long s = 0;
    unsigned mx = 0;
    for (int t = lo; t < hi; t++) {
        s += cnt[t];
        mx = max(mx, cnt[t]);
    }
    part[threadIdx.x] = s;
    pmax[threadIdx.x] = mx;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {  // inclusive scan (Hillis-Steele)
        const unsigned long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0ull;
    for (int t = lo; t < hi; t++) {
        off[t] = (unsigned)run;
        run += cnt[t];
    }
    for (int d = 512; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) pmax[threadIdx.x] = max(pmax[threadIdx.x], pmax[threadIdx.x + d]);
        __syncthreads();
    }
    if (threadIdx.x == 1023) total[0] = part[1023];
    if (threadIdx.x == 0) total[1] = pmax[0];
}

// Writes each (Gaussian, tile) key into its tile's segment. Pass 1 counts a
// block's pairs per tile in the shared table (pairs without a slot take a global
// position at once); one global atomic per table slot then reserves a contiguous
// range of the segment; pass 2 walks the pairs again and places them in the range.
__global__ void __launch_bounds__(256) k_sp_fill(int n, const int4 *__restrict__ rect,
                                                 const float *__restrict__ depth,
                                                 const unsigned *__restrict__ off, unsigned *fill,
                                                 unsigned long long *keys, int ntx)
{
    __shared__ unsigned hk[SP_HT], hc[SP_HT], hb[SP_HT];
    for (int base = blockIdx.x * 256; base < n; base += gridDim.x * 256) {  // uniform over the block
        for (int e = threadIdx.x; e < SP_HT; e += 256) {
            hk[e] = SP_EMPTY;
            hc[e] = 0;
        }
        __syncthreads();
        const int i = base + threadIdx.x;
        const int4 rc = i < n ? rect[i] : make_int4(0, 0, 0, 0);
        const unsigned long long key =
            i < n ? ((unsigned long long)__float_as_uint(depth[i]) << 32) | (unsigned)i : 0ull;
        for (int ty = rc.z; ty < rc.w; ty++)
            for (int tx = rc.x; tx < rc.y; tx++) {
                const unsigned t = (unsigned)(ty * ntx + tx);
                const int sl = ht_slot(hk, t, true);
                if (sl >= 0) {
                    atomicAdd(hc + sl, 1u);
                } else {
                    const unsigned pos = atomicAdd(fill + t, 1u);
                    keys[off[t] + pos] = key;
                }
            }
        __syncthreads();
        for (int e = threadIdx.x; e < SP_HT; e += 256)
            if (hk[e] != SP_EMPTY) {
                hb[e] = off[hk[e]] + atomicAdd(fill + hk[e], hc[e]);
                hc[e] = 0;
            }
        __syncthreads();
        for (int ty = rc.z; ty < rc.w; ty++)
            for (int tx = rc.x; tx < rc.y; tx++) {
                const int sl = ht_slot(hk, (unsigned)(ty * ntx + tx), false);
                if (sl >= 0) keys[hb[sl] + atomicAdd(hc + sl, 1u)] = key;
            }
        __syncthreads();
    }
}

// Stable LSD radix sort (8-bit digits) of each tile segment longer than SP_CAP,
// one block of 256 threads per tile. Digits 0-3 are the Gaussian index (those
// above the largest index are skipped), 4-7 the depth bits; a digit that all keys
// share is skipped too. A round takes 2048 keys, warp w the 256 consecutive keys
// [w * 256, w * 256 + 256) as BS_IT slots of 32; slot by slot, a key's rank among
// the warp's keys with the same digit is the warp's running count of that digit
// plus its rank within the slot (__match_any_sync), and the warps are ordered by a
// per-digit prefix, so equal digits keep their order. The result ends in `keys`.
constexpr int BS_IT = 8;

__global__ void __launch_bounds__(256) k_sp_bigsort(unsigned long long *keys, unsigned long long *tmp,
                                                    const unsigned *__restrict__ off,
                                                    const unsigned *__restrict__ cnt, int idx_digits)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned wcnt[8][256];
    __shared__ unsigned wpos[8][256];
    __shared__ unsigned wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned n = cnt[blockIdx.x];
    if (n <= SP_CAP) return;
    unsigned long long *src = keys + off[blockIdx.x], *dst = tmp + off[blockIdx.x];
    for (int w = 0; w < 8; w++) wcnt[w][tid] = 0;
    for (int dgt = 0; dgt < 8; dgt++) {
        if (dgt < 4 && dgt >= idx_digits) continue;
        const int shift = 8 * dgt;
        hist[tid] = 0;
        __syncthreads();
        for (unsigned e = tid; e < n; e += 256) atomicAdd(&hist[(unsigned)(src[e] >> shift) & 255u], 1u);
        __syncthreads();
        if (__syncthreads_or(hist[tid] == n)) continue;  // one digit for all keys
        // exclusive scan of the histogram: the digits' base positions
        const unsigned v = hist[tid];
        unsigned incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        unsigned wpre = 0;
        for (int w = 0; w < warp; w++) wpre += wsum[w];
        hist[tid] = wpre + incl - v;
        __syncthreads();
        for (unsigned r0 = 0; r0 < n; r0 += 256 * BS_IT) {
            unsigned long long kv[BS_IT];
            unsigned dg[BS_IT], rk[BS_IT];
#pragma unroll
            for (int q = 0; q < BS_IT; q++) {
                const unsigned e = r0 + warp * 256 + q * 32 + lane;
                kv[q] = e < n ? src[e] : 0ull;
                dg[q] = e < n ? ((unsigned)(kv[q] >> shift) & 255u) : 256u;
            }
#pragma unroll
            for (int q = 0; q < BS_IT; q++) {
                const unsigned mask = __match_any_sync(0xffffffffu, dg[q]);
                const unsigned before = dg[q] < 256u ? wcnt[warp][dg[q]] : 0u;
                rk[q] = before + __popc(mask & ((1u << lane) - 1u));
                __syncwarp();
                if (dg[q] < 256u && lane == __ffs(mask) - 1) wcnt[warp][dg[q]] = before + __popc(mask);
                __syncwarp();
            }
            __syncthreads();
            unsigned run = hist[tid];  // thread tid owns digit tid
            for (int w = 0; w < 8; w++) {
                wpos[w][tid] = run;
                run += wcnt[w][tid];
                wcnt[w][tid] = 0;
            }
            hist[tid] = run;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < BS_IT; q++)
                if (dg[q] < 256u) dst[wpos[warp][dg[q]] + rk[q]] = kv[q];
        }
        unsigned long long *t = src;
        src = dst;
        dst = t;
        __syncthreads();
    }
    if (src != keys + off[blockIdx.x])
        for (unsigned e = tid; e < n; e += 256) keys[off[blockIdx.x] + e] = src[e];
}

__global__ void __launch_bounds__(256) k_sp_render(const unsigned long long *__restrict__ keys,
                                                   const unsigned *__restrict__ off,
                                                   const unsigned *__restrict__ cnt,
                                                   const SplatRecord *__restrict__ rec, Cam cam, int ntx,
                                                   float *rgb, float *Tout)
{
    __shared__ unsigned long long sk[SP_CAP];
    __shared__ SplatRecord sr[256];
    const int tile = blockIdx.x;
    const int tid = threadIdx.x;
    const unsigned n = cnt[tile], base = off[tile];
    const bool big = n > SP_CAP;  // already sorted in global memory
    int m = 1;
    while (!big && m < (int)n) m <<= 1;
    if (!big)
        for (int e = tid; e < m; e += 256) sk[e] = e < (int)n ? keys[base + e] : ~0ull;
    __syncthreads();
    // bitonic sort of m keys (ascending: depth, then index)
    for (int k = 2; !big && k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int e = tid; e < m; e += 256) {
                const int p = e ^ j;
                if (p > e) {
                    const bool up = (e & k) == 0;
                    const unsigned long long a = sk[e], b = sk[p];
                    if ((a > b) == up) {
                        sk[e] = b;
                        sk[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    const int px = (tile % ntx) * SP_TILE + (tid % SP_TILE), py = (tile / ntx) * SP_TILE + (tid / SP_TILE);
    const bool inside = px < cam.w && py < cam.h;
    const float pu = px + 0.5f, pv = py + 0.5f;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    bool done = !inside;
    for (int b0 = 0; b0 < (int)n; b0 += 256) {
        if (__syncthreads_and(done)) break;
        if (b0 + tid < (int)n)
            sr[tid] = rec[(unsigned)((big ? keys[base + b0 + tid] : sk[b0 + tid]) & 0xffffffffu)];
        __syncthreads();
        const int nb = min(256, (int)n - b0);
        for (int q = 0; q < nb && !done; q++) {
            const SplatRecord g = sr[q];
            const float dx = pu - g.mx, dy = pv - g.my;
            const float md = g.ca * dx * dx + 2.f * g.cb * dx * dy + g.cc * dy * dy;
            if (md > 9.f) continue;
            float alpha = fminf(0.99f, g.opacity * expf(-0.5f * md));
            if (alpha < 1.f / 255.f) continue;
            const float Tn = T * (1.f - alpha);
            if (Tn < 1e-4f) {
                done = true;
                break;
            }
            c0 += alpha * T * g.r;
            c1 += alpha * T * g.g;
            c2 += alpha * T * g.b;
            T = Tn;
        }
    }
    if (inside) {
        const long long o = (long long)py * cam.w + px;
        rgb[3 * o] = c0 + T * cam.bg[0];
        rgb[3 * o + 1] = c1 + T * cam.bg[1];
        rgb[3 * o + 2] = c2 + T * cam.bg[2];
        if (Tout) Tout[o] = T;
    }
}

template <typename T>
int grow(T **p, long long &cap, long long need)
{
    if (need <= cap && *p) return FS_OK;
    cudaFree(*p);
    *p = nullptr;
    cap = 0;
    const long long n = need > 0 ? need : 1;
    if (cudaMalloc((void **)p, (size_t)n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FS_ENOMEM, "splatting scratch of %lld elements", n);
    }
    cap = n;
    return FS_OK;
}

}  // namespace

void splat_free(fs_ctx *c)
{
    SplatState *s = static_cast<SplatState *>(c->splat);
    if (!s) return;
    cudaFree(s->rec);
    cudaFree(s->rect);
    cudaFree(s->depth);
    cudaFree(s->tcount);
    cudaFree(s->toff);
    cudaFree(s->tfill);
    cudaFree(s->keys);
    cudaFree(s->keys2);
    delete s;
    c->splat = nullptr;
}

int splat_render(fs_ctx *c, int n, const float *x, const float *op, const float *A, const float *col,
                 const float *sh, int deg, const fs_camera *camh, float *rgb, float *T)
{
    SplatState *s = static_cast<SplatState *>(c->splat);
    if (!s) {
        s = new (std::nothrow) SplatState();
        if (!s) return set_error(FS_ENOMEM, "host allocation failed");
        c->splat = s;
    }
    Cam cam;
    for (int k = 0; k < 9; k++) cam.R[k] = (float)camh->R[k];
    for (int k = 0; k < 3; k++) {
        cam.t[k] = (float)camh->t[k];
        cam.bg[k] = (float)camh->bg[k];
    }
    cam.fx = (float)camh->fx;
    cam.fy = (float)camh->fy;
    cam.cx = (float)camh->cx;
    cam.cy = (float)camh->cy;
    cam.w = camh->width;
    cam.h = camh->height;
    cam.znear = (float)camh->znear;
    const int ntx = (cam.w + SP_TILE - 1) / SP_TILE, nty = (cam.h + SP_TILE - 1) / SP_TILE, nt = ntx * nty;
    int rc;
    if (n > s->cap_n || !s->rec) {  // per-Gaussian arrays, grown together
        long long c0 = 0, c1 = 0, c2 = 0;
        if ((rc = grow(&s->rec, c0, n)) || (rc = grow(&s->rect, c1, n)) || (rc = grow(&s->depth, c2, n))) return rc;
        s->cap_n = n > 0 ? n : 1;
    }
    if (nt > s->cap_t || !s->tcount) {  // per-tile arrays
        long long c0 = 0, c1 = 0, c2 = 0;
        if ((rc = grow(&s->tcount, c0, nt)) || (rc = grow(&s->toff, c1, nt)) || (rc = grow(&s->tfill, c2, nt)))
            return rc;
        s->cap_t = nt;
    }
    FS_CUDA(cudaMemsetAsync(s->tcount, 0, (size_t)nt * 4, c->stream));
    FS_CUDA(cudaMemsetAsync(s->tfill, 0, (size_t)nt * 4, c->stream));
    const int gb = grid_blocks(c, n > 0 ? n : 1, 256);
    if (n > 0)
        k_sp_project<<<gb, 256, 0, c->stream>>>(n, x, op, A, col, sh, deg, cam, s->rec, s->rect, s->depth,
                                                s->tcount, ntx, nty);
    unsigned long long *total_d = reinterpret_cast<unsigned long long *>(c->partials);
    k_sp_scan<<<1, 1024, 0, c->stream>>>(s->tcount, s->toff, nt, total_d);
    c->n_launches += 2;
    FS_CUDA(cudaGetLastError());
    unsigned long long tot[2] = {0, 0};
    FS_CUDA(cudaMemcpyAsync(tot, total_d, sizeof(tot), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    s->last_entries = tot[0];
    s->last_max = tot[1];
    if (tot[0] > 0xffffffffull) return set_error(FS_EINVAL, "more than 2^32 tile entries");
    if ((rc = grow(&s->keys, s->cap_k, (long long)tot[0]))) return rc;
    if (n > 0) {
        k_sp_fill<<<gb, 256, 0, c->stream>>>(n, s->rect, s->depth, s->toff, s->tfill, s->keys, ntx);
        c->n_launches += 1;
    }
    if (tot[1] > (unsigned long long)SP_CAP) {
        if ((rc = grow(&s->keys2, s->cap_k2, (long long)tot[0]))) return rc;
        const int idx_digits = n <= (1 << 8) ? 1 : n <= (1 << 16) ? 2 : n <= (1 << 24) ? 3 : 4;
        k_sp_bigsort<<<nt, 256, 0, c->stream>>>(s->keys, s->keys2, s->toff, s->tcount, idx_digits);
        c->n_launches += 1;
    }
    k_sp_render<<<nt, 256, 0, c->stream>>>(s->keys, s->toff, s->tcount, s->rec, cam, ntx, rgb, T);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

void splat_stats(const fs_ctx *c, unsigned long long *entries, unsigned long long *max_tile)
{
    const SplatState *s = static_cast<const SplatState *>(c->splat);
    *entries = s ? s->last_entries : 0;
    *max_tile = s ? s->last_max : 0;
}

}  // namespace fs
