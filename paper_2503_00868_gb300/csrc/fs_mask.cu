// fs_mask.cu -- grid-type mask set-up: cell and face flag bytes, prescribed
// face values, Dirichlet sums of the viscosity operator, band and singularity
// counts. Runs once per mask (Sec. 3.4.2: the loss is restricted by a mask
// derived from the cell types of the grid).
#include <algorithm>
#include <cstring>
#include <vector>

#include <cudaTypedefs.h>

#include "fs_internal.cuh"

namespace fs {
namespace {

// Decode a public-layout index into (i, j, k).
__device__ __forceinline__ void decode(const Layout &L, int idx, int &i, int &j, int &k)
{
    i = idx % L.P;
    int row = idx / L.P;
    j = row % L.R;
    k = row / L.R;
}

__global__ void k_cell_types(Layout L, const uint8_t *__restrict__ types, uint8_t *cflag,
                             unsigned *err)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nC; t += gridDim.x * blockDim.x) {
        int idx = t - L.PL;
        uint8_t f = 0;
        if (idx >= 0 && idx < L.S) {
            int i, j, k;
            decode(L, idx, i, j, k);
            if (i < L.nx && j < L.ny && k < L.nz) {
                uint8_t ty = types[((size_t)k * L.ny + j) * L.nx + i];
                if (ty == FS_LIQUID) f = CF_LIQ;
                else if (ty == FS_AIR) f = CF_AIR;
                else if (ty == FS_SOLID) f = CF_SOLID;
                else { atomicOr(err, 1u); f = CF_SOLID; }
            }
        }
        cflag[t] = f;
    }
}

// Number of non-solid neighbours and the surface band bit. Out-of-grid
// neighbours read flag 0 (guard or padding), i.e. solid.
__global__ void k_cell_flags(Layout L, uint8_t *cflag)
{
    for (int t = L.PL + blockIdx.x * blockDim.x + threadIdx.x; t < L.PL + L.S;
         t += gridDim.x * blockDim.x) {
        uint8_t f = cflag[t];
        if (!(f & (CF_LIQ | CF_AIR | CF_SOLID))) continue;
        const int off[6] = {-1, 1, -L.P, L.P, -L.PL, L.PL};
        int d = 0, air = 0;
        for (int m = 0; m < 6; m++) {
            uint8_t g = cflag[t + off[m]];
            d += (g & (CF_LIQ | CF_AIR)) ? 1 : 0;
            air |= (g & CF_AIR) ? 1 : 0;
        }
        uint8_t base = f & (CF_LIQ | CF_AIR | CF_SOLID);
        uint8_t band = ((f & CF_LIQ) && air) ? CF_BAND : 0;
        cflag[t] = base | (uint8_t)d | band;
    }
}

__device__ __forceinline__ bool solid_like(uint8_t f) { return (f & CF_SOLID) || !(f & (CF_LIQ | CF_AIR)); }

__global__ void k_face_class(Layout L, const uint8_t *__restrict__ cflag, uint8_t *fflag)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nF; t += gridDim.x * blockDim.x) {
        uint8_t out = 0;
        int seg = t - L.PL;
        int c = seg >= 0 ? seg / (L.S + L.PL) : -1;
        int idx = seg - c * (L.S + L.PL);
        if (c >= 0 && c < 3 && idx >= 0 && idx < L.S) {
            int i, j, k;
            decode(L, idx, i, j, k);
            int dims[3] = {L.nx, L.ny, L.nz};
            dims[c] += 1;
            if (i < dims[0] && j < dims[1] && k < dims[2]) {
                int off = c == 0 ? 1 : (c == 1 ? L.P : L.PL);
                uint8_t fr = cflag[L.PL + idx], fl = cflag[L.PL + idx - off];
                if (solid_like(fl) || solid_like(fr)) out = FF_FIXED;
                else if ((fl & CF_LIQ) || (fr & CF_LIQ)) out = FF_FLUID;
                else out = FF_AIR;
            }
        }
        fflag[t] = out;
    }
}

// Viscosity neighbour count of fluid faces and the Dirichlet sums; copies the
// prescribed values of fixed faces into face space.
__global__ void k_face_count(Layout L, uint8_t *fflag, CF3 bc_user, float *bc, float *dsum)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nF; t += gridDim.x * blockDim.x) {
        uint8_t f = fflag[t];
        int seg = t - L.PL;
        int c = seg >= 0 ? seg / (L.S + L.PL) : -1;
        int idx = seg - c * (L.S + L.PL);
        float bv = 0.f;
        if ((f & FF_FIXED) && bc_user.c[0]) bv = bc_user.c[c][idx];
        bc[t] = bv;
        if (!(f & FF_FLUID)) continue;
        const int off[6] = {-1, 1, -L.P, L.P, -L.PL, L.PL};
        int n = 0;
        float ds = 0.f;
        for (int m = 0; m < 6; m++) {
            uint8_t g = fflag[t + off[m]];
            if (g & (FF_FLUID | FF_FIXED)) n++;
            if ((g & FF_FIXED) && bc_user.c[0]) ds += bc_user.c[c][idx + off[m]];
        }
        fflag[t] = (uint8_t)(f | n);
        if (dsum) dsum[t] = ds;
    }
}

// counts: 0 liquid cells, 1 surface band cells, 2 surface band faces, 3 occupied
// band faces (= fluid faces)
__global__ void k_counts(Layout L, const uint8_t *__restrict__ cflag, const uint8_t *__restrict__ fflag,
                         unsigned long long *cnt)
{
    unsigned long long a = 0, b = 0, cs = 0, co = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nF; t += gridDim.x * blockDim.x) {
        if (t < L.nC) {
            uint8_t f = cflag[t];
            a += (f & CF_LIQ) ? 1 : 0;
            b += (f & CF_BAND) ? 1 : 0;
        }
        uint8_t g = fflag[t];
        if (g & FF_FLUID) {
            int seg = t - L.PL;
            int c = seg / (L.S + L.PL);
            int idx = seg - c * (L.S + L.PL);
            int off = c == 0 ? 1 : (c == 1 ? L.P : L.PL);
            uint8_t fr = cflag[L.PL + idx], fl = cflag[L.PL + idx - off];
            cs += ((fr | fl) & CF_BAND) ? 1 : 0;
            co += ((fr | fl) & CF_LIQ) ? 1 : 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        cs += __shfl_down_sync(0xffffffffu, cs, o);
        co += __shfl_down_sync(0xffffffffu, co, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt[0], a);
        atomicAdd(&cnt[1], b);
        atomicAdd(&cnt[2], cs);
        atomicAdd(&cnt[3], co);
    }
}

// act[b] = 1 for every tile block of `m` that holds an element with a bit of
// `mask` set in its flag byte.
__global__ void k_tile_activity(const uint8_t *__restrict__ fl, uint8_t mask, TileMap m, uint8_t *act)
{
    const long long per_vol = (long long)m.PL * m.Z;
    const long long total = per_vol * m.nvol;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(t / per_vol);
        const int idx = (int)(t - (long long)v * per_vol);
        if (!(fl[m.origin0 + (long long)v * m.vstride + idx] & mask)) continue;
        const int i = idx % m.P, row = idx / m.P, j = row % m.R, k = row / m.R;
        const int b = ((v * m.nch + k / m.tz) * m.nty + j / TILE_Y) * m.ntx + i / TILE_X;
        act[b] = 1;
    }
}

// Quad-activity words of the listed tiles: block = one listed tile, thread
// (x, y) = quad x of tile row y; word y of the tile is the ballot of row y.
__global__ void k_quad_mask(const uint8_t *__restrict__ fl, uint8_t mask, const int *__restrict__ list, TileMap m,
                            unsigned *qmask)
{
    int v, k, tyi, txi;
    m.decode(list[blockIdx.x], v, k, tyi, txi);
    const int i = txi * TILE_X + 4 * threadIdx.x, j = tyi * TILE_Y + threadIdx.y;
    bool act = false;
    if (i < m.P && j < m.R) {
        const uchar4 f = *reinterpret_cast<const uchar4 *>(fl + m.origin0 + v * m.vstride + k * m.PL + j * m.P + i);
        act = ((f.x | f.y | f.z | f.w) & mask) != 0;
    }
    const unsigned w = __ballot_sync(0xffffffffu, act);
    if (threadIdx.x == 0) qmask[(size_t)blockIdx.x * TILE_Y + threadIdx.y] = w;
}

}  // namespace

// The driver's tensor-map encoder, found through the runtime (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// A guarded space as a 3-D FP32 tensor: x = pitch, y = rows, z = planes (guard
// planes included), with a box of bx x by x 1 elements. Out-of-range elements
// of a box read as zero.
static int encode_map(CUtensorMap *m, float *base, const Layout &L, long long len, int bx, int by)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return set_error(FS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)L.P, (cuuint64_t)L.R, (cuuint64_t)(len / L.PL)};
    const cuuint64_t strides[2] = {(cuuint64_t)L.P * 4, (cuuint64_t)L.PL * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FS_OK;
}

int make_tensor_maps(fs_ctx *c)
{
    const Layout &L = c->L;
    const int zx = TILE_X + 8, zy = TILE_Y + 2;  // the operator apply's halo box
    struct M { CUtensorMap *m; float *p; long long len; int bx, by; } maps[] = {
        {&c->tmz_pr, c->pr, L.nC, zx, zy},         {&c->tmz_pz, c->pz, L.nC, zx, zy},
        {&c->tmz_pp[0], c->pp[0], L.nC, zx, zy},   {&c->tmz_pp[1], c->pp[1], L.nC, zx, zy},
        {&c->tmz_vr, c->vr, L.nF, zx, zy},         {&c->tmz_vp[0], c->vp[0], L.nF, zx, zy},
        {&c->tmz_vp[1], c->vp[1], L.nF, zx, zy},   {&c->tmz_vz, c->vz, L.nF, zx, zy}};
    for (auto &e : maps) {
        int rc = encode_map(e.m, e.p, L, e.len, e.bx, e.by);
        if (rc) return rc;
    }
    return FS_OK;
}

// Work of the z-marching operator apply: for every column (volume, tile row,
// tile column) the runs of planes whose tile holds an active element (gaps of
// up to two planes are bridged), cut into chunks of at most zc planes, in
// column order so that neighbouring chunks run at about the same time.
static std::vector<int4> zmarch_items(const std::vector<uint8_t> &act, const TileMap &m, int zc)
{
    std::vector<int4> items;
    const int ncol = m.ntx * m.nty * m.nvol;
    for (int col = 0; col < ncol; col++) {
        const int txi = col % m.ntx, tyi = (col / m.ntx) % m.nty, v = col / (m.ntx * m.nty);
        auto active = [&](int k) { return act[(size_t)(((v * m.nch + k) * m.nty + tyi) * m.ntx + txi)] != 0; };
        int k = 0;
        while (k < m.Z) {
            while (k < m.Z && !active(k)) k++;
            if (k >= m.Z) break;
            int e = k + 1, last = k;
            while (e < m.Z && e - last <= 3) {
                if (active(e)) last = e;
                e++;
            }
            const int k1 = last + 1;  // run [k, k1), cut into chunks of at most zc planes
            const int len = k1 - k, nch = (len + zc - 1) / zc;
            for (int c = 0; c < nch; c++)  // equal lengths (within one plane): no short tail chunk
                items.push_back(make_int4(col, k + (int)((long long)len * c / nch),
                                          k + (int)((long long)len * (c + 1) / nch), 0));
            k = k1;
        }
    }
    return items;
}

TileMap make_tilemap(const Layout &L, int nvol, int num_sms)
{
    TileMap m;
    m.P = L.P;
    m.R = L.R;
    m.Z = L.Z;
    m.PL = L.PL;
    m.nvol = nvol;
    m.origin0 = L.PL;
    m.vstride = L.S + L.PL;
    m.ntx = (L.P + TILE_X - 1) / TILE_X;
    m.nty = (L.R + TILE_Y - 1) / TILE_Y;
    // one plane per block: many small independent blocks
    (void)num_sms;
    const long long cols = (long long)m.ntx * m.nty * nvol;
    m.tz = 1;
    m.nch = L.Z;
    m.nblocks = (int)(cols * m.nch);
    return m;
}

int build_mask(fs_ctx *c, const uint8_t *types_dense, const fs_mac *bc)
{
    const Layout &L = c->L;
    const int th = 256;
    CF3 bcu{{nullptr, nullptr, nullptr}};
    if (bc) {
        bcu.c[0] = bc->u;
        bcu.c[1] = bc->v;
        bcu.c[2] = bc->w;
    }
    c->has_bc = bc ? 1 : 0;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c->partials);
    FS_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(unsigned), c->stream));
    FS_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), c->stream));
    // the buffers the multigrid V-cycle writes its result into start from zero
    // off the unknowns of the new mask: it writes them only on quads that hold an
    // unknown, and every other writer leaves them zero off the unknowns
    if (c->pz) FS_CUDA(cudaMemsetAsync(c->pz, 0, (size_t)L.nC * sizeof(float), c->stream));
    if (c->pbr) FS_CUDA(cudaMemsetAsync(c->pbr, 0, (size_t)L.nC * sizeof(float), c->stream));
    if (c->vz) FS_CUDA(cudaMemsetAsync(c->vz, 0, (size_t)L.nF * sizeof(float), c->stream));
    k_cell_types<<<grid_blocks(c, L.nC, th), th, 0, c->stream>>>(L, types_dense, c->cflag, c->err_word);
    k_cell_flags<<<grid_blocks(c, L.S, th), th, 0, c->stream>>>(L, c->cflag);
    k_face_class<<<grid_blocks(c, L.nF, th), th, 0, c->stream>>>(L, c->cflag, c->fflag);
    k_face_count<<<grid_blocks(c, L.nF, th), th, 0, c->stream>>>(L, c->fflag, bcu, c->bc,
                                                                  bc ? c->dsum : nullptr);
    k_counts<<<grid_blocks(c, L.nF, th), th, 0, c->stream>>>(L, c->cflag, c->fflag, cnt);
    if (c->act_cell && c->act_face) {
        FS_CUDA(cudaMemsetAsync(c->act_cell, 0, (size_t)c->tm_cell.nblocks, c->stream));
        FS_CUDA(cudaMemsetAsync(c->act_face, 0, (size_t)c->tm_face.nblocks, c->stream));
        k_tile_activity<<<grid_blocks(c, L.S, th), th, 0, c->stream>>>(c->cflag, CF_LIQ, c->tm_cell, c->act_cell);
        k_tile_activity<<<grid_blocks(c, 3LL * L.S, th), th, 0, c->stream>>>(c->fflag, FF_FLUID, c->tm_face,
                                                                             c->act_face);
    }
    FS_CUDA(cudaGetLastError());
    unsigned long long h[4];
    unsigned herr = 0;
    FS_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaMemcpyAsync(&herr, c->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    if (herr) return set_error(FS_EINVAL, "fs_set_mask: a cell type is not 0 (air), 1 (liquid) or 2 (solid)");
    if (c->act_cell && c->act_face) {
        // ordered lists of the active tiles (set-up work, on the host)
        struct Space { const uint8_t *act; int *list; int n; int *nact; } sp[2] = {
            {c->act_cell, c->list_cell, c->tm_cell.nblocks, &c->nact_cell},
            {c->act_face, c->list_face, c->tm_face.nblocks, &c->nact_face}};
        int4 *items_dev[2] = {c->items_cell, c->items_face};
        int *nitems[2] = {&c->nitems_cell, &c->nitems_face};
        const TileMap *tms[2] = {&c->tm_cell, &c->tm_face};
        for (int si = 0; si < 2; si++) {
            auto &s = sp[si];
            std::vector<uint8_t> act((size_t)s.n);
            FS_CUDA(cudaMemcpy(act.data(), s.act, (size_t)s.n, cudaMemcpyDeviceToHost));
            std::vector<int> list;
            list.reserve((size_t)s.n);
            for (int b = 0; b < s.n; b++)
                if (act[(size_t)b]) list.push_back(b);
            *s.nact = (int)list.size();
            if (!list.empty()) {
                FS_CUDA(cudaMemcpy(s.list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice));
                k_quad_mask<<<(unsigned)list.size(), dim3(TILE_X / 4, TILE_Y), 0, c->stream>>>(
                    si == 0 ? c->cflag : c->fflag, si == 0 ? CF_LIQ : FF_FLUID, s.list, *tms[si],
                    si == 0 ? c->qmask_cell : c->qmask_face);
                FS_CUDA(cudaGetLastError());
            }
            // at most one chunk per resident block of the operator apply (a second
            // chunk on some blocks would double the launch), 8 planes at least
            const long long slots = (long long)zmarch_slots(c, si == 1);
            int zc = (int)std::max<long long>(8, ((long long)list.size() + slots - 1) / slots);
            std::vector<int4> items = zmarch_items(act, *tms[si], zc);
            while ((long long)items.size() > slots && zc < c->L.Z) {
                zc += std::max(1, zc / 8);
                items = zmarch_items(act, *tms[si], zc);
            }
            *nitems[si] = (int)items.size();
            if (!items.empty())
                FS_CUDA(cudaMemcpy(items_dev[si], items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
        }
    }
    c->n_liquid = (long long)h[0];
    c->n_band_cells[FS_MASK_SURFACE] = (long long)h[1];
    c->n_band_cells[FS_MASK_OCCUPIED] = (long long)h[0];
    c->n_band_faces[FS_MASK_SURFACE] = (long long)h[2];
    c->n_band_faces[FS_MASK_OCCUPIED] = (long long)h[3];
    c->n_fluid = (long long)h[3];
    // The pressure operator has the constant on the liquid as null vector when no
    // liquid cell touches air (a closed box full of liquid).
    c->singular = (h[0] > 0 && h[1] == 0) ? 1 : 0;
    c->mask_set = 1;
    c->mask_epoch += 1;
    c->pw_valid[0] = c->pw_valid[1] = 0;
    c->p_floor2[0] = c->p_floor2[1] = 0.0;
    std::memset(c->it_last_p, 0, sizeof(c->it_last_p));
    std::memset(c->it_last_v, 0, sizeof(c->it_last_v));
    c->mic_ready = 0;
    c->mic_sched_ready = 0;
    return FS_OK;
}

}  // namespace fs
