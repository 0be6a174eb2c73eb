// fs_mic0.cu -- MIC(0) preconditioner of the pressure solve (the modified
// incomplete Cholesky of Bridson's "Fluid Simulation for Computer Graphics",
// which the paper cites for its pressure projection, Sec. 3.2.2): factor, forward
// and backward substitution in LEXICOGRAPHIC order (x fastest), exactly the
// recurrences of the sequential algorithm, run as a tile wavefront.
//
// Recurrences (A = 7-point pressure operator, -1 between liquid neighbours,
// prec = 1/sqrt(e), "lower" = the -x, -y, -z neighbours that are liquid):
//   factor:   e_i = d_i - sum_lower prec_m^2 (1 + tau * n_m),  n_m = number of
//             liquid +neighbours of m in the other two directions;
//             e_i < sigma d_i  =>  e_i = d_i
//   forward:  y_i = prec_i (r_i + sum_lower prec_m y_m)
//   backward: z_i = prec_i (y_i + prec_i sum_upper z_m)
//
// Schedule. The grid is cut into 8x8x8 tiles; a tile depends on its -x, -y, -z
// neighbour tiles (forward, factor) or its +x, +y, +z neighbours (backward).
// Tiles holding liquid are listed by tile level (tx + ty + tz). Persistent blocks
// take the next tile from an atomic counter, so every predecessor of a tile was
// taken earlier by a block that is already running: waiting on it always ends.
// A block waits (bounded spin) until each predecessor's flag reaches this
// sweep's epoch, loads the tile and its one-cell halo into shared memory, walks
// the 22 intra-tile diagonal levels (x + y + z = const) with a barrier between
// levels, writes the tile, and publishes its flag. A spin that runs out sets an
// error word; every other wait sees it and gives up, so the launch always ends.
// Values that other blocks of the same launch wrote (halo cells of predecessor
// tiles) are read through L2 (ld.global.cg), never from a possibly stale L1 line.
#include <algorithm>
#include <vector>

#include "fs_internal.cuh"

namespace fs {
namespace {

constexpr int MT = 8;                  // tile edge
constexpr int MTH = MT * MT * MT;      // threads per block, one per cell
enum { MIC_FACTOR = 0, MIC_FORWARD = 1, MIC_BACKWARD = 2 };

struct MicGrid {
    int ntx, nty, ntz;
    int nx, ny, nz;
    int P, PL;      // layout pitch and plane
    int origin;     // cell-space offset of cell (0, 0, 0)
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool liquid(const uint8_t *cf, int t) { return (cf[t] & CF_LIQ) != 0; }

template <int MODE>
__global__ void __launch_bounds__(MTH) k_mic_sweep(MicGrid G, const uint8_t *__restrict__ cf, float *prec,
                                                   const float *in, float *out, const int *__restrict__ order,
                                                   int n, const uint8_t *__restrict__ tact, int *tflag, int *next,
                                                   int epoch, int spin_limit, unsigned *err, float tau,
                                                   float sigma)
{
    // values of the tile with a one-cell halo: cell (x, y, z) at [z+1][y+1][x+1]
    __shared__ float sv[MT + 2][MT + 2][MT + 2];
    __shared__ float sp[MT + 2][MT + 2][MT + 2];  // prec (forward: with the lower halo)
    __shared__ int s_tile;
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int x = tid % MT, y = (tid / MT) % MT, z = tid / (MT * MT);
    const int dir = MODE == MIC_BACKWARD ? 1 : -1;
    for (;;) {
        if (tid == 0) {
            const int w = atomicAdd(next, 1);
            s_tile = w < n ? order[MODE == MIC_BACKWARD ? n - 1 - w : w] : -1;
            s_abort = 0;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile < 0) break;
        const int ti = tile % G.ntx, tj = (tile / G.ntx) % G.nty, tk = tile / (G.ntx * G.nty);
        // wait for the three predecessor tiles
        if (tid < 3) {
            int pi = ti, pj = tj, pk = tk;
            if (tid == 0) pi += dir;
            else if (tid == 1) pj += dir;
            else pk += dir;
            if (pi >= 0 && pj >= 0 && pk >= 0 && pi < G.ntx && pj < G.nty && pk < G.ntz) {
                const int pt = (pk * G.nty + pj) * G.ntx + pi;
                if (tact[pt]) {
                    int spins = 0;
                    while (ld_acquire(tflag + pt) < epoch) {
                        if (ld_acquire(reinterpret_cast<const int *>(err)) != 0 || ++spins > spin_limit) {
                            atomicOr(err, 1u);
                            s_abort = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            // give up on this sweep: publish nothing, drain the remaining tiles
            __syncthreads();
            continue;
        }
        const int gi = ti * MT + x, gj = tj * MT + y, gk = tk * MT + z;
        const bool valid = gi < G.nx && gj < G.ny && gk < G.nz;
        const int t = G.origin + gk * G.PL + gj * G.P + gi;
        const bool liq = valid && liquid(cf, t);
        // own input values, and the halo of already final neighbours
        if (MODE == MIC_FORWARD) {
            sv[z + 1][y + 1][x + 1] = 0.f;
            sp[z + 1][y + 1][x + 1] = liq ? prec[t] : 0.f;
        } else if (MODE == MIC_BACKWARD) {
            sv[z + 1][y + 1][x + 1] = 0.f;
        } else {
            sp[z + 1][y + 1][x + 1] = 0.f;
        }
        // halo faces: threads of the face adjacent to a predecessor load one cell
        if (MODE != MIC_BACKWARD) {
            // lower faces: x = -1, y = -1, z = -1 (cells outside the grid read as non-liquid)
            if (x == 0) {
                const bool ok = gi - 1 >= 0 && gj < G.ny && gk < G.nz && liquid(cf, t - 1);
                sv[z + 1][y + 1][0] = (MODE == MIC_FORWARD && ok) ? __ldcg(out + (t - 1)) : 0.f;
                sp[z + 1][y + 1][0] = ok ? __ldcg(prec + (t - 1)) : 0.f;
            }
            if (y == 0) {
                const bool ok = gj - 1 >= 0 && gi < G.nx && gk < G.nz && liquid(cf, t - G.P);
                sv[z + 1][0][x + 1] = (MODE == MIC_FORWARD && ok) ? __ldcg(out + (t - G.P)) : 0.f;
                sp[z + 1][0][x + 1] = ok ? __ldcg(prec + (t - G.P)) : 0.f;
            }
            if (z == 0) {
                const bool ok = gk - 1 >= 0 && gi < G.nx && gj < G.ny && liquid(cf, t - G.PL);
                sv[0][y + 1][x + 1] = (MODE == MIC_FORWARD && ok) ? __ldcg(out + (t - G.PL)) : 0.f;
                sp[0][y + 1][x + 1] = ok ? __ldcg(prec + (t - G.PL)) : 0.f;
            }
        } else {
            // upper faces: x = 8, y = 8, z = 8
            if (x == MT - 1) {
                const bool ok = gi + 1 < G.nx && gj < G.ny && gk < G.nz && liquid(cf, t + 1);
                sv[z + 1][y + 1][MT + 1] = ok ? __ldcg(out + (t + 1)) : 0.f;
            }
            if (y == MT - 1) {
                const bool ok = gj + 1 < G.ny && gi < G.nx && gk < G.nz && liquid(cf, t + G.P);
                sv[z + 1][MT + 1][x + 1] = ok ? __ldcg(out + (t + G.P)) : 0.f;
            }
            if (z == MT - 1) {
                const bool ok = gk + 1 < G.nz && gi < G.nx && gj < G.ny && liquid(cf, t + G.PL);
                sv[MT + 1][y + 1][x + 1] = ok ? __ldcg(out + (t + G.PL)) : 0.f;
            }
        }
        float own_in = 0.f, own_prec = 0.f, diag = 0.f;
        int nlow = 0;  // bit mask of liquid lower (or upper) neighbours
        if (liq) {
            if (MODE != MIC_FACTOR) own_in = in[t];
            if (MODE == MIC_BACKWARD) own_prec = prec[t];
            diag = (float)(cf[t] & CF_D);
            const int off[3] = {1, G.P, G.PL};
            const int pos[3] = {gi, gj, gk};
            const int lim[3] = {G.nx, G.ny, G.nz};
            for (int a = 0; a < 3; a++) {
                const int q = pos[a] + dir;
                if (q >= 0 && q < lim[a] && liquid(cf, t + dir * off[a])) nlow |= 1 << a;
            }
        }
        __syncthreads();
        // the 22 diagonal levels of the tile (reversed for the backward sweep)
        const int lvl = x + y + z;
        for (int l = 0; l <= 3 * (MT - 1); l++) {
            const int want = MODE == MIC_BACKWARD ? 3 * (MT - 1) - l : l;
            if (lvl == want && liq) {
                if (MODE == MIC_FACTOR) {
                    float e = diag;
                    const int off[3] = {1, G.P, G.PL};
                    for (int a = 0; a < 3; a++) {
                        if (!(nlow & (1 << a))) continue;
                        const float pm = a == 0 ? sp[z + 1][y + 1][x] : (a == 1 ? sp[z + 1][y][x + 1] : sp[z][y + 1][x + 1]);
                        // n_m: liquid +neighbours of m in the other two directions
                        const int m = t - off[a];
                        int nm = 0;
                        for (int b = 0; b < 3; b++) {
                            if (b == a) continue;
                            const int mp[3] = {gi - (a == 0), gj - (a == 1), gk - (a == 2)};
                            const int qb = (b == 0 ? mp[0] : (b == 1 ? mp[1] : mp[2])) + 1;
                            if (qb < (b == 0 ? G.nx : (b == 1 ? G.ny : G.nz)) && liquid(cf, m + off[b])) nm++;
                        }
                        e -= pm * pm * (1.f + tau * (float)nm);
                    }
                    if (e < sigma * diag) e = diag;
                    sp[z + 1][y + 1][x + 1] = diag > 0.f ? 1.f / sqrtf(e) : 0.f;
                } else if (MODE == MIC_FORWARD) {
                    float acc = own_in;
                    if (nlow & 1) acc += sp[z + 1][y + 1][x] * sv[z + 1][y + 1][x];
                    if (nlow & 2) acc += sp[z + 1][y][x + 1] * sv[z + 1][y][x + 1];
                    if (nlow & 4) acc += sp[z][y + 1][x + 1] * sv[z][y + 1][x + 1];
                    sv[z + 1][y + 1][x + 1] = acc * sp[z + 1][y + 1][x + 1];
                } else {
                    float acc = 0.f;
                    if (nlow & 1) acc += sv[z + 1][y + 1][x + 2];
                    if (nlow & 2) acc += sv[z + 1][y + 2][x + 1];
                    if (nlow & 4) acc += sv[z + 2][y + 1][x + 1];
                    sv[z + 1][y + 1][x + 1] = own_prec * (own_in + own_prec * acc);
                }
            }
            __syncthreads();
        }
        if (valid) {
            if (MODE == MIC_FACTOR) prec[t] = liq ? sp[z + 1][y + 1][x + 1] : 0.f;
            else out[t] = liq ? sv[z + 1][y + 1][x + 1] : 0.f;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_release(tflag + tile, epoch);
    }
}

}  // namespace

static MicGrid mic_grid(const fs_ctx *c)
{
    MicGrid g;
    g.nx = c->L.nx;
    g.ny = c->L.ny;
    g.nz = c->L.nz;
    g.ntx = (g.nx + MT - 1) / MT;
    g.nty = (g.ny + MT - 1) / MT;
    g.ntz = (g.nz + MT - 1) / MT;
    g.P = c->L.P;
    g.PL = c->L.PL;
    g.origin = c->L.PL;
    return g;
}

// Tile order by level and the per-tile liquid flag (set-up work, on the host).
static int mic_schedule(fs_ctx *c)
{
    const MicGrid g = mic_grid(c);
    const int ntiles = g.ntx * g.nty * g.ntz;
    std::vector<uint8_t> cf((size_t)c->L.nC);
    FS_CUDA(cudaMemcpy(cf.data(), c->cflag, cf.size(), cudaMemcpyDeviceToHost));
    std::vector<uint8_t> act((size_t)ntiles, 0);
    for (int k = 0; k < g.nz; k++)
        for (int j = 0; j < g.ny; j++)
            for (int i = 0; i < g.nx; i++)
                if (cf[(size_t)g.origin + (size_t)k * g.PL + (size_t)j * g.P + i] & CF_LIQ)
                    act[(size_t)((k / MT) * g.nty + j / MT) * g.ntx + i / MT] = 1;
    std::vector<int> order;
    for (int t = 0; t < ntiles; t++)
        if (act[(size_t)t]) order.push_back(t);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int la = a % g.ntx + (a / g.ntx) % g.nty + a / (g.ntx * g.nty);
        const int lb = b % g.ntx + (b / g.ntx) % g.nty + b / (g.ntx * g.nty);
        return la < lb;
    });
    c->mic_n = (int)order.size();
    if (!order.empty())
        FS_CUDA(cudaMemcpy(c->mic_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->mic_tact, act.data(), act.size(), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemset(c->mic_tflag, 0, (size_t)ntiles * sizeof(int)));
    c->mic_epoch = 0;
    c->mic_sched_ready = 1;
    return FS_OK;
}

template <int MODE>
static int mic_launch(fs_ctx *c, const float *in, float *out)
{
    const MicGrid g = mic_grid(c);
    c->mic_epoch += 1;
    FS_CUDA(cudaMemsetAsync(c->mic_next, 0, sizeof(int), c->stream));
    const int grid = std::max(1, std::min(c->mic_n, 2 * c->num_sms));
    k_mic_sweep<MODE><<<grid, MTH, 0, c->stream>>>(g, c->cflag, c->mic_prec, in, out, c->mic_order, c->mic_n,
                                                   c->mic_tact, c->mic_tflag, c->mic_next, c->mic_epoch,
                                                   c->prm.spin_limit, c->err_word, (float)c->prm.mic_tau,
                                                   (float)c->prm.mic_sigma);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int mic0_factor(fs_ctx *c)
{
    if (!c->mic_sched_ready) {
        int rc = mic_schedule(c);
        if (rc) return rc;
    }
    FS_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(unsigned), c->stream));
    int rc = mic_launch<MIC_FACTOR>(c, nullptr, nullptr);
    if (rc) return rc;
    c->mic_ready = 1;
    return FS_OK;
}

int mic0_apply(fs_ctx *c, const float *r, float *z)
{
    cudaEvent_t e0 = prof_mark(c);
    int rc = mic_launch<MIC_FORWARD>(c, r, c->py);
    if (rc) return rc;
    rc = mic_launch<MIC_BACKWARD>(c, c->py, z);
    if (rc) return rc;
    prof_add(c, K_MIC_APPLY, e0, prof_mark(c), 0.0);
    return FS_OK;
}

}  // namespace fs
