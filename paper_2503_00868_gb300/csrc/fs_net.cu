// fs_net.cu -- the learned pressure preconditioner (arXiv 2503.00868, Sec. 3.4.1,
// Fig. percnn_str_fit: a convolutional network with fitted 3x3x3 kernels that
// maps a pressure right-hand side to a pressure, fitted to solver output).
//
// Network: five 3x3x3 convolutions, channels 2 -> 16 -> 16 -> 16 -> 16 -> 1, zero
// padding at the grid boundary, ReLU after the first four. Input channel 0 is
// r / s on liquid cells rounded to bf16 (s = max |r| over the liquid), channel 1
// the cell type code (liquid 1, air 0, solid -1). Output z = s * y on liquid
// cells. Weights are bf16 (FP32 master copies for training), every hidden
// activation is stored as bf16, every sum accumulates in FP32.
//
// Kernels:
//   k_conv<IN, OUT>  every layer as an implicit GEMM per 3x3x3 tap on the tensor
//                  cores (mma.sync m16n8k16 bf16 x bf16 -> f32, operands via
//                  ldmatrix from a swizzled shared-memory tile); layer 1 builds
//                  its (r/s, cell type) input tile on the fly with the weights
//                  zero-padded to 16 input channels, layer 5 uses one 8-wide
//                  n-tile and writes z = s y on liquid cells; the same kernel
//                  runs the backward-data pass of layers 2-4 with flipped,
//                  transposed weights and a ReLU-derivative epilogue. For
//                  inference layer l visits only the conv tiles within 5 - l
//                  cells of the liquid (the output on liquid cells depends on
//                  nothing farther), from a tile list sorted by that distance;
//   k_bwd_last     gradient through layer 5 to its input;
//   k_wgrad<CIN,COUT>  weight and bias gradients (FP32 CUDA cores, per-block
//                  partial sums, one atomicAdd per weight per block);
//   k_adam         Adam on the FP32 master weights, then the bf16 copies.
// Layout: activations are channel-last, [cell][16] bf16 (32 bytes per cell) in
// cell space; a neighbour outside the grid reads zero (checked per cell).
#include <cuda_bf16.h>

#include <new>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fs_internal.cuh"

namespace fs {

// parameter offsets in the flat FP32 vector (PyTorch conv3d layout [co][ci][kd][kh][kw])
constexpr int NW1 = 16 * 2 * 27, NB1 = 16, NWM = 16 * 16 * 27, NBM = 16, NW5 = 16 * 27, NB5 = 1;
constexpr int OW1 = 0, OB1 = OW1 + NW1;
constexpr int OW2 = OB1 + NB1, OB2 = OW2 + NWM;
constexpr int OW3 = OB2 + NBM, OB3 = OW3 + NWM;
constexpr int OW4 = OB3 + NBM, OB4 = OW4 + NWM;
constexpr int OW5 = OB4 + NBM, OB5 = OW5 + NW5;
constexpr int NPARAM = OB5 + NB5;

struct NetState {
    float *master;        // FP32 parameters, flat
    float *grad;          // FP32 gradient accumulator, flat
    float *m, *v;         // Adam moments
    float *w1f, *w5f;     // bf16-rounded layer-1 / layer-5 weights as float
    __nv_bfloat16 *wf;    // layers 2-4 forward: [3][27 tap][16 co][16 ci]
    __nv_bfloat16 *wf1;   // layer 1 forward: [27 tap][16 co][16 ci], ci >= 2 zero
    __nv_bfloat16 *wf5;   // layer 5 forward: [27 tap][16 co][16 ci], co >= 1 zero
    int *tlist;           // conv tiles sorted by distance to the liquid (0 .. 5 = farther)
    uint8_t *tdist;       // per conv tile: Chebyshev distance to the nearest liquid cell, capped at 5
    int tcount[6];        // tiles within distance d of the liquid
    int *tlist_tc;        // tiles of the tensor-core layer (TC_M x TC_NY of one plane), sorted the same way
    int tcount_tc[6];
    int kernel;           // inference layers: 0 mma.sync (k_conv), 1 tcgen05 (k_conv_tc)
    double last_flops;    // useful flops of the last inference, on the tiles it visited
    long long tlist_epoch;  // mask epoch the list was built for (-1: none)
    __nv_bfloat16 *wt;    // layers 2-4 backward-data: [3][27 tap][16 ci][16 co], tap flipped
    __nv_bfloat16 *act;   // [6][nC][16]: x (2 ch used), a1, a2, a3, a4, spare
    __nv_bfloat16 *gact;  // [2][nC][16] gradient ping-pong
    float *y;             // [nC] network output (training) / scratch
    float *gy;            // [nC] dL/dy
    unsigned *smax;       // device max |r| (float bits)
    int loaded;
};

namespace {

constexpr int NT_X = 32, NT_Y = 8;  // conv tile: 32 x 8 cells of one plane

__device__ __forceinline__ int tap_index(int dz, int dy, int dx) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

__device__ __forceinline__ bool in_grid(const Layout &L, int i, int j, int k)
{
    return i >= 0 && j >= 0 && k >= 0 && i < L.nx && j < L.ny && k < L.nz;
}

__device__ __forceinline__ int cell_t(const Layout &L, int i, int j, int k) { return L.PL + (k * L.R + j) * L.P + i; }

__device__ __forceinline__ float type_code(uint8_t f) { return (f & CF_LIQ) ? 1.f : ((f & CF_AIR) ? 0.f : -1.f); }

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16(x)); }

// ---- layers 2-4 (16 -> 16), tensor cores ------------------------------------------
// Shared tile: 3 planes x (NT_Y + 2) rows x (NT_X + 2) cells x 16 bf16. The two
// 16-byte halves of a cell are swapped when bit 2 of its tile index is set, so
// the 8 rows of an ldmatrix phase fall in distinct banks.
constexpr int TZ3 = 3, TYH = NT_Y + 2, TXH = NT_X + 2;
constexpr int TCELLS = TZ3 * TYH * TXH;

__device__ __forceinline__ uint32_t swz_off(int cidx, int half)  // byte offset of a cell half
{
    return (uint32_t)(cidx * 32 + ((half ^ ((cidx >> 2) & 1)) << 4));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

enum : int { IN_ACT = 0, IN_R = 1 };                  // input: bf16 activations / built from r
enum : int { OUT_RELU = 0, OUT_BWD = 1, OUT_Z = 2 };  // epilogue

struct ConvArgs {
    const __nv_bfloat16 *in;    // IN_ACT: [cell][16]
    const float *r;             // IN_R: right-hand side (cell space)
    const uint8_t *cf;          // cell flags
    const unsigned *smax;       // max |r| over the liquid (float bits)
    const __nv_bfloat16 *wts;   // [27 tap][16 n][16 k]
    const float *bias;          // OUT_RELU: [16]; OUT_Z: [1]
    const __nv_bfloat16 *aref;  // OUT_BWD: the layer input whose ReLU derivative masks
    __nv_bfloat16 *out;         // OUT_RELU, OUT_BWD: [cell][16]
    __nv_bfloat16 *xin;         // IN_R (optional): the bf16 input, channels 0 and 1
    float *y, *z;               // OUT_Z (each optional): network output; z = s y on liquid, else 0
    const int *tiles;           // optional list of conv tiles (else every tile)
    int ntiles;                 // entries of `tiles`
    Layout L;
};

// IN_ACT/OUT_RELU: out = relu(conv(in) + bias). OUT_BWD (backward data):
// out = conv(in) * [aref > 0]. OUT_Z: y = conv(in) + bias, z = s y on liquid
// cells. IN_R: the input is (bf16(r/s) on liquid, cell-type code), channels 2-15
// zero. Outputs only on grid cells.
template <int IN, int OUT>
__global__ void __launch_bounds__(256) k_conv(ConvArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char *tile = smem;                          // TCELLS * 32 bytes
    unsigned char *wsm = smem + TCELLS * 32;             // 27 * 16 rows * 32 bytes
    const Layout &L = a.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // weights once per block (rows n = tap * 16 + co, swizzled like the tile)
    for (int e = tid; e < 27 * 16 * 2; e += blockDim.x) {
        const int row = e >> 1, half = e & 1;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.wts) + row * 2 + half);
        *reinterpret_cast<uint4 *>(wsm + swz_off(row, half)) = v;
    }
    float bv[4] = {0.f, 0.f, 0.f, 0.f};  // bias of this lane's output channels
    if (OUT == OUT_RELU) {
        const int co = (lane & 3) * 2;
        bv[0] = a.bias[co];
        bv[1] = a.bias[co + 1];
        bv[2] = a.bias[8 + co];
        bv[3] = a.bias[8 + co + 1];
    } else if (OUT == OUT_Z) {
        bv[0] = a.bias[0];
    }
    float sc = 1.f, inv = 0.f;
    if (IN == IN_R || OUT == OUT_Z) {
        sc = __uint_as_float(*a.smax);
        inv = sc > 0.f ? 1.f / sc : 0.f;
    }
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile);
    const uint32_t w_s = (uint32_t)__cvta_generic_to_shared(wsm);
    const int ntx = (L.nx + NT_X - 1) / NT_X, nty = (L.ny + NT_Y - 1) / NT_Y;
    const int total = a.tiles ? a.ntiles : ntx * nty * L.nz;
    for (int idx = blockIdx.x; idx < total; idx += gridDim.x) {
        const int tb = a.tiles ? __ldg(a.tiles + idx) : idx;
        const int tx = tb % ntx, ty = (tb / ntx) % nty, tk = tb / (ntx * nty);
        const int i0 = tx * NT_X, j0 = ty * NT_Y;
        __syncthreads();  // previous tile done with the shared tile (and weights stored)
        for (int e = tid; e < TCELLS * 2; e += blockDim.x) {
            const int cidx = e >> 1, half = e & 1;
            const int xx = cidx % TXH, yy = (cidx / TXH) % TYH, zz = cidx / (TXH * TYH);
            const int gi = i0 - 1 + xx, gj = j0 - 1 + yy, gk = tk - 1 + zz;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (in_grid(L, gi, gj, gk)) {
                const int t = cell_t(L, gi, gj, gk);
                if (IN == IN_ACT) {
                    v = __ldg(reinterpret_cast<const uint4 *>(a.in + (size_t)t * 16) + half);
                } else if (half == 0) {
                    const uint8_t f = a.cf[t];
                    const __nv_bfloat162 x = __floats2bfloat162_rn((f & CF_LIQ) ? a.r[t] * inv : 0.f, type_code(f));
                    v.x = *reinterpret_cast<const uint32_t *>(&x);
                }
            }
            *reinterpret_cast<uint4 *>(tile + swz_off(cidx, half)) = v;
        }
        __syncthreads();
        // warp w: row y = w of the tile, two M-tiles of 16 cells (x 0-15, 16-31)
        for (int mt = 0; mt < 2; mt++) {
            float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
            const int row = lane & 15, khalf = lane >> 4;
            for (int dz = 0; dz < 3; dz++)
                for (int dy = 0; dy < 3; dy++)
                    for (int dx = 0; dx < 3; dx++) {
                        const int cidx = (dz * TYH + warp + dy) * TXH + mt * 16 + dx + row;
                        uint32_t a0, a1, a2, a3;
                        ldsm_x4(tile_s + swz_off(cidx, khalf), a0, a1, a2, a3);
                        const int tp = dz * 9 + dy * 3 + dx;
                        const int wrow = tp * 16 + (lane & 7) + ((lane >> 4) << 3);
                        const int wh = (lane >> 3) & 1;
                        uint32_t b0, b1, b2, b3;
                        ldsm_x4(w_s + swz_off(wrow, wh), b0, b1, b2, b3);
                        mma_bf16(acc0, a0, a1, a2, a3, b0, b1);
                        if (OUT != OUT_Z) mma_bf16(acc1, a0, a1, a2, a3, b2, b3);
                    }
            // epilogue: cells (lane/4) and (lane/4 + 8); channels (lane%4)*2 (+1), +8
            const int gj = j0 + warp;
            for (int hr = 0; hr < 2; hr++) {
                const int gi = i0 + mt * 16 + (lane >> 2) + hr * 8;
                if (gi >= L.nx || gj >= L.ny) continue;
                const size_t t = (size_t)cell_t(L, gi, gj, tk);
                const int co = (lane & 3) * 2;
                if (OUT == OUT_Z) {
                    if (co == 0) {
                        const float yv = acc0[hr * 2] + bv[0];
                        if (a.y) a.y[t] = yv;
                        if (a.z) a.z[t] = (a.cf[t] & CF_LIQ) ? sc * yv : 0.f;
                    }
                    continue;
                }
                if (IN == IN_R && a.xin && co == 0) {
                    const uint8_t f = a.cf[t];
                    *reinterpret_cast<__nv_bfloat162 *>(a.xin + t * 16) =
                        __floats2bfloat162_rn((f & CF_LIQ) ? a.r[t] * inv : 0.f, type_code(f));
                }
                float v0 = acc0[hr * 2], v1 = acc0[hr * 2 + 1], v2 = acc1[hr * 2], v3 = acc1[hr * 2 + 1];
                if (OUT == OUT_RELU) {
                    v0 = fmaxf(v0 + bv[0], 0.f);
                    v1 = fmaxf(v1 + bv[1], 0.f);
                    v2 = fmaxf(v2 + bv[2], 0.f);
                    v3 = fmaxf(v3 + bv[3], 0.f);
                } else {
                    const __nv_bfloat162 r0 = *reinterpret_cast<const __nv_bfloat162 *>(a.aref + t * 16 + co);
                    const __nv_bfloat162 r1 = *reinterpret_cast<const __nv_bfloat162 *>(a.aref + t * 16 + 8 + co);
                    v0 = __bfloat162float(r0.x) > 0.f ? v0 : 0.f;
                    v1 = __bfloat162float(r0.y) > 0.f ? v1 : 0.f;
                    v2 = __bfloat162float(r1.x) > 0.f ? v2 : 0.f;
                    v3 = __bfloat162float(r1.y) > 0.f ? v3 : 0.f;
                }
                *reinterpret_cast<__nv_bfloat162 *>(a.out + t * 16 + co) = __floats2bfloat162_rn(v0, v1);
                *reinterpret_cast<__nv_bfloat162 *>(a.out + t * 16 + 8 + co) = __floats2bfloat162_rn(v2, v3);
            }
        }
    }
}

// ---- the same layer on the fifth-generation tensor cores (tcgen05, TMEM) ----------
// Inference only. A tile is TC_NY = 2 rows of TC_M = 128 cells along x of one
// plane; each row is one M = 128, N = 16 GEMM over K = 27 taps x 16 channels,
// issued as 27 tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulators in tensor
// memory, one 16-column accumulator per row) by one thread. The input tile (3
// planes x TC_NY + 2 rows x TC_M + 2 cells, 16 channels) is staged in shared
// memory split by channel half: region [plane][row][half][x][8 channels], so that
// a tap's A operand is the same region read from a start shifted by the tap's
// offset, in the canonical K-major layout without swizzling (8-row core matrices
// of 16 bytes per row, 128 bytes apart along M; the second 8 channels TC_HALF
// bytes further along K). The weights of a tap are [half][out channel][8 in
// channels], 512 bytes. Two input buffers alternate: all threads stage the next
// tile while the tensor core works on the current one. The accumulators are read
// back with tcgen05.ld (warp w owns lanes 32 (w % 4) .. + 31 of row w / 4, one
// cell per lane) for the bias, ReLU and bf16 store. Every wait on the MMAs'
// completion is bounded: on timeout the block records an error bit, waits
// (bounded) for its MMAs in flight, frees its tensor memory and stops.
constexpr int TC_M = 128, TC_NY = 2, TC_XW = TC_M + 2, TC_ROWS = TC_NY + 2, TC_THREADS = 256;
constexpr int TC_HALF = TC_XW * 16;                          // 2080 bytes: one channel half of a row
constexpr int TC_ROWB = 2 * TC_HALF;                         // 4160 bytes per (plane, row)
constexpr int TC_A_BYTES = 3 * TC_ROWS * TC_ROWB;            // 49920 per buffer
constexpr int TC_B_BYTES = 27 * 512;                         // 13824
constexpr size_t TC_SMEM = 128 + 2 * (size_t)TC_A_BYTES + TC_B_BYTES;
constexpr unsigned TC_SPIN = 1u << 24;
constexpr unsigned ERR_TC = 8u;
static_assert(TC_THREADS == 2 * TC_M, "one thread per accumulator row lane in the epilogue");

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in units of 16 bytes, descriptor version 1, no swizzling
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulate (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(16 >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ bool tc_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// 16 FP32 columns of the warp's lane quarter, one lane per thread
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

// tiles of the tensor-core layer: TC_M x TC_NY cells of one plane, index
// (k * ntyc + ty) * ntxc + tx
__device__ __forceinline__ void tc_tile(int tb, const Layout &L, int &i0, int &j0, int &k)
{
    const int ntxc = (L.nx + TC_M - 1) / TC_M, ntyc = (L.ny + TC_NY - 1) / TC_NY;
    i0 = (tb % ntxc) * TC_M;
    j0 = ((tb / ntxc) % ntyc) * TC_NY;
    k = tb / (ntxc * ntyc);
}

// stage the input tile of tile tb into sa: plane kz - 1 + pz, row j0 - 1 + ry,
// cell i0 - 1 + x, both channel halves
template <int IN>
__device__ __forceinline__ void tc_stage(const ConvArgs &a, int tb, unsigned char *sa, float inv)
{
    const Layout &L = a.L;
    int i0, j0, kz;
    tc_tile(tb, L, i0, j0, kz);
    for (int e = threadIdx.x; e < 3 * TC_ROWS * TC_XW; e += blockDim.x) {
        const int x = e % TC_XW, ry = (e / TC_XW) % TC_ROWS, pz = e / (TC_XW * TC_ROWS);
        const int gi = i0 - 1 + x, gj = j0 - 1 + ry, gk = kz - 1 + pz;
        uint4 h0 = make_uint4(0u, 0u, 0u, 0u), h1 = h0;
        if (in_grid(L, gi, gj, gk)) {
            const int t = cell_t(L, gi, gj, gk);
            if (IN == IN_ACT) {
                h0 = __ldg(reinterpret_cast<const uint4 *>(a.in + (size_t)t * 16));
                h1 = __ldg(reinterpret_cast<const uint4 *>(a.in + (size_t)t * 16) + 1);
            } else {
                const uint8_t f = a.cf[t];
                const __nv_bfloat162 xv = __floats2bfloat162_rn((f & CF_LIQ) ? a.r[t] * inv : 0.f, type_code(f));
                h0.x = *reinterpret_cast<const uint32_t *>(&xv);
            }
        }
        unsigned char *row = sa + (pz * TC_ROWS + ry) * TC_ROWB + x * 16;
        *reinterpret_cast<uint4 *>(row) = h0;
        *reinterpret_cast<uint4 *>(row + TC_HALF) = h1;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
}

template <int IN, int OUT>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(ConvArgs a, unsigned *err)
{
    extern __shared__ __align__(128) unsigned char smem_tc[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_tc) + 127) & ~(uintptr_t)127);
    unsigned char *sa[2] = {base, base + TC_A_BYTES};  // input tiles, alternating
    unsigned char *sb = base + 2 * TC_A_BYTES;          // weights
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int stop;
    const Layout &L = a.L;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // weights: [tap][half][co][8 ci] from [tap][co][16 ci]
    for (int e = tid; e < 27 * 16 * 2; e += blockDim.x) {
        const int tap = e >> 5, co = (e >> 1) & 15, half = e & 1;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(a.wts) + (tap * 16 + co) * 2 + half);
        *reinterpret_cast<uint4 *>(sb + tap * 512 + half * 256 + co * 16) = v;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_base)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stop = 0;
    }
    float bv[16];
#pragma unroll
    for (int k = 0; k < 16; k++) bv[k] = 0.f;
    if (OUT == OUT_RELU) {
#pragma unroll
        for (int k = 0; k < 16; k++) bv[k] = a.bias[k];
    } else {
        bv[0] = a.bias[0];
    }
    float sc = 1.f, inv = 0.f;
    if (IN == IN_R || OUT == OUT_Z) {
        sc = __uint_as_float(*a.smax);
        inv = sc > 0.f ? 1.f / sc : 0.f;
    }
    const int ntxc = (L.nx + TC_M - 1) / TC_M, ntyc = (L.ny + TC_NY - 1) / TC_NY;
    const int total = a.tiles ? a.ntiles : ntxc * ntyc * L.nz;
    auto tile_at = [&](int idx) { return a.tiles ? __ldg(a.tiles + idx) : idx; };
    if ((int)blockIdx.x < total) tc_stage<IN>(a, tile_at(blockIdx.x), sa[0], inv);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t sb_u = tc_smem(sb), bar_u = tc_smem(&mbar);
    uint32_t phase = 0;
    int buf = 0;
    for (int idx = blockIdx.x; idx < total; idx += gridDim.x, buf ^= 1) {
        int i0, j0, kz;
        tc_tile(tile_at(idx), L, i0, j0, kz);
        if (tid == 0) {
            const uint32_t sa_u = tc_smem(sa[buf]);
#pragma unroll 1
            for (int yr = 0; yr < TC_NY; yr++) {
#pragma unroll 1
                for (int tap = 0; tap < 27; tap++) {
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                    const uint32_t aaddr = sa_u + (uint32_t)((dz * TC_ROWS + yr + dy) * TC_ROWB + dx * 16);
                    tc_mma(tmem + (uint32_t)(16 * yr), tc_desc(aaddr, TC_HALF, 128), tc_desc(sb_u + tap * 512, 256, 128),
                           tap > 0 ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_u)
                         : "memory");
        }
        // the next tile into the other buffer while the tensor core works
        if (idx + (int)gridDim.x < total) tc_stage<IN>(a, tile_at(idx + gridDim.x), sa[buf ^ 1], inv);
        bool ok = false;
        for (unsigned n = 0; n < TC_SPIN && !ok; n++) ok = tc_try_wait(bar_u, phase);
        if (!ok) {
            if (lane == 0) atomicOr(err, ERR_TC);
            stop = 1;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (stop) break;
        // epilogue: warp w reads lanes 32 (w % 4) .. + 31 of row w / 4
        {
            const int yr = warp >> 2, q = warp & 3;
            float acc[16];
            tc_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * yr), acc);
            const int gi = i0 + 32 * q + lane, gj = j0 + yr;
            if (gi < L.nx && gj < L.ny) {
                const size_t t = (size_t)cell_t(L, gi, gj, kz);
                if (OUT == OUT_Z) {
                    const float yv = acc[0] + bv[0];
                    if (a.y) a.y[t] = yv;
                    if (a.z) a.z[t] = (a.cf[t] & CF_LIQ) ? sc * yv : 0.f;
                } else {
                    uint32_t pk[8];
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(fmaxf(acc[2 * k] + bv[2 * k], 0.f),
                                                                        fmaxf(acc[2 * k + 1] + bv[2 * k + 1], 0.f));
                        pk[k] = *reinterpret_cast<const uint32_t *>(&b2);
                    }
                    uint4 *o = reinterpret_cast<uint4 *>(a.out + t * 16);
                    o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
        }
        // the accumulators read and the next buffer staged before the next MMAs
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (stop) {  // the MMAs of a timed-out tile may still run: wait for them again (bounded) before freeing
        bool ok = false;
        for (unsigned n = 0; n < TC_SPIN && !ok; n++) ok = tc_try_wait(bar_u, phase ^ 1u);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

// Chebyshev distance from each conv tile (32 x 8 cells of one plane) to the
// nearest liquid cell, capped at 5: one block per tile scans the tile grown by 5.
__global__ void __launch_bounds__(256) k_conv_tile_dist(const uint8_t *__restrict__ cf, Layout L, uint8_t *dist)
{
    __shared__ int best;
    const int ntx = (L.nx + NT_X - 1) / NT_X, nty = (L.ny + NT_Y - 1) / NT_Y;
    const int tb = blockIdx.x;
    const int tx = tb % ntx, ty = (tb / ntx) % nty, tk = tb / (ntx * nty);
    const int i0 = tx * NT_X, j0 = ty * NT_Y;
    if (threadIdx.x == 0) best = 5;
    __syncthreads();
    const int bx = NT_X + 10, by = NT_Y + 10, bz = 11;
    int d = 5;
    for (int e = threadIdx.x; e < bx * by * bz; e += blockDim.x) {
        const int gi = i0 - 5 + e % bx, gj = j0 - 5 + (e / bx) % by, gk = tk - 5 + e / (bx * by);
        if (!in_grid(L, gi, gj, gk) || !(cf[cell_t(L, gi, gj, gk)] & CF_LIQ)) continue;
        const int dx = max(0, max(i0 - gi, gi - (i0 + NT_X - 1)));
        const int dy = max(0, max(j0 - gj, gj - (j0 + NT_Y - 1)));
        const int dz = abs(gk - tk);
        d = min(d, max(dx, max(dy, dz)));
    }
    if (d < 5) atomicMin(&best, d);
    __syncthreads();
    if (threadIdx.x == 0) dist[tb] = (uint8_t)best;
}

// max |r| over the liquid, as float bits (non-negative floats order like ints)
__global__ void k_absmax(const float *__restrict__ r, const uint8_t *__restrict__ cf, int n, unsigned *smax)
{
    float m = 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        if (cf[t] & CF_LIQ) m = fmaxf(m, fabsf(r[t]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(smax, __float_as_uint(m));
}

// s is rounded to bf16 (the oracle rounds x = r/s, not s; keep s exact)
// ---- training: loss, gradients -----------------------------------------------------

// Energy-norm loss (y - q/s)^T A (y - q/s) / ((q/s)^T A (q/s)), A the pressure
// operator. Pass 1: e = y - q/s and t = q/s on liquid cells (zero elsewhere).
__global__ void k_net_err(const float *__restrict__ y, const float *__restrict__ q, const uint8_t *__restrict__ cf,
                          const unsigned *__restrict__ smax, float *e, float *tq, int n)
{
    const float sc = __uint_as_float(*smax);
    const float inv = sc > 0.f ? 1.f / sc : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const bool liq = (cf[t] & CF_LIQ) != 0;
        const float tv = liq ? q[t] * inv : 0.f;
        tq[t] = tv;
        e[t] = liq ? y[t] - tv : 0.f;
    }
}

// Pass 2: Ae (kept for the gradient), e.Ae and t.At -> aux[0], aux[1].
__global__ void __launch_bounds__(256) k_net_energy(const float *__restrict__ e, const float *__restrict__ tq,
                                                    float *ae, const uint8_t *__restrict__ cf, Layout L,
                                                    SolveScal *s, double *partials)
{
    double num = 0.0, den = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nC; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        if (!(f & CF_LIQ)) continue;
        const float d = (float)(f & CF_D);
        const float av = d * e[t] - ((e[t - 1] + e[t + 1]) + (e[t - L.P] + e[t + L.P]) + (e[t - L.PL] + e[t + L.PL]));
        const float at = d * tq[t] - ((tq[t - 1] + tq[t + 1]) + (tq[t - L.P] + tq[t + L.P]) +
                                      (tq[t - L.PL] + tq[t + L.PL]));
        ae[t] = av;
        num += (double)e[t] * av;
        den += (double)tq[t] * at;
    }
    double v[2] = {num, den}, tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->aux[0] = tot[0];
        s->aux[1] = tot[1];
    }
}

// Pass 3: dloss/dy = 2 A e / den on liquid cells.
__global__ void k_net_gy(const float *__restrict__ ae, const uint8_t *__restrict__ cf, const SolveScal *s, float *gy,
                         int n)
{
    const double den = s->aux[1];
    const float g = den > 0.0 ? (float)(2.0 / den) : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        gy[t] = (cf[t] & CF_LIQ) ? g * ae[t] : 0.f;
}

// ---- the loss of the network followed by the V-cycle (FS_PRECOND_LEARNED_MG) ----
// With y the network output (masked to the liquid), b/s and q/s the scaled pair
// and M the V-cycle: w = q/s - y - M(b/s - A y), loss = w.A w / (q/s).A (q/s).
// w = (I - M A)(q/s - y), so dloss/dy = -2 (I - A M) A w / den, M and A symmetric.

// ym = y on liquid cells, 0 elsewhere
__global__ void k_net_mask_y(const float *__restrict__ y, const uint8_t *__restrict__ cf, float *ym, int n)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        ym[t] = (cf[t] & CF_LIQ) ? y[t] : 0.f;
}

// t1 = b/s - A ym on liquid cells (the residual the network leaves), 0 elsewhere
__global__ void __launch_bounds__(256) k_netmg_res(const float *__restrict__ b, const float *__restrict__ ym,
                                                   const uint8_t *__restrict__ cf, const unsigned *__restrict__ smax,
                                                   Layout L, float *t1)
{
    const float sc = __uint_as_float(*smax);
    const float inv = sc > 0.f ? 1.f / sc : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nC; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        float v = 0.f;
        if (f & CF_LIQ) {
            const float ay = (float)(f & CF_D) * ym[t] -
                             ((ym[t - 1] + ym[t + 1]) + (ym[t - L.P] + ym[t + L.P]) + (ym[t - L.PL] + ym[t + L.PL]));
            v = b[t] * inv - ay;
        }
        t1[t] = v;
    }
}

// w = q/s - ym - m and tq = q/s on liquid cells, 0 elsewhere
__global__ void k_netmg_err(const float *__restrict__ q, const float *__restrict__ ym, const float *__restrict__ m,
                            const uint8_t *__restrict__ cf, const unsigned *__restrict__ smax, float *w, float *tq,
                            int n)
{
    const float sc = __uint_as_float(*smax);
    const float inv = sc > 0.f ? 1.f / sc : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const bool liq = (cf[t] & CF_LIQ) != 0;
        const float tv = liq ? q[t] * inv : 0.f;
        tq[t] = tv;
        w[t] = liq ? tv - ym[t] - m[t] : 0.f;
    }
}

// dloss/dy = -2 (v - A u) / den on liquid cells, v = A w, u = M v
__global__ void __launch_bounds__(256) k_netmg_gy(const float *__restrict__ v, const float *__restrict__ u,
                                                  const uint8_t *__restrict__ cf, const SolveScal *s, Layout L,
                                                  float *gy)
{
    const double den = s->aux[1];
    const float g = den > 0.0 ? (float)(-2.0 / den) : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nC; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        float o = 0.f;
        if (f & CF_LIQ) {
            const float au = (float)(f & CF_D) * u[t] -
                             ((u[t - 1] + u[t + 1]) + (u[t - L.P] + u[t + L.P]) + (u[t - L.PL] + u[t + L.PL]));
            o = g * (v[t] - au);
        }
        gy[t] = o;
    }
}

// dL/d(layer-5 input) = sum_tap w5[ci][tap] gy[cell - tap], times [a4 > 0]
__global__ void __launch_bounds__(256) k_bwd_last(const float *__restrict__ gy, const float *__restrict__ w5f,
                                                  const __nv_bfloat16 *__restrict__ a4, __nv_bfloat16 *g4, Layout L)
{
    __shared__ float w[NW5];
    for (int t = threadIdx.x; t < NW5; t += blockDim.x) w[t] = w5f[t];
    __syncthreads();
    const int ncell = L.nx * L.ny * L.nz;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
        float acc[16];
#pragma unroll
        for (int o = 0; o < 16; o++) acc[o] = 0.f;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    // output cell (i - d) saw this cell through tap d
                    if (!in_grid(L, i - dx, j - dy, k - dz)) continue;
                    const float g = gy[cell_t(L, i - dx, j - dy, k - dz)];
                    if (g == 0.f) continue;
                    const int tp = tap_index(dz, dy, dx);
#pragma unroll
                    for (int o = 0; o < 16; o++) acc[o] += w[o * 27 + tp] * g;
                }
        const size_t t = (size_t)cell_t(L, i, j, k);
        const __nv_bfloat162 *a = reinterpret_cast<const __nv_bfloat162 *>(a4 + t * 16);
        __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(g4 + t * 16);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float2 av = __bfloat1622float2(a[q]);
            o2[q] = __floats2bfloat162_rn(av.x > 0.f ? acc[2 * q] : 0.f, av.y > 0.f ? acc[2 * q + 1] : 0.f);
        }
    }
}

// Weight and bias gradients of one layer: gW[co][ci][tap] += sum_cells
// g[cell][co] * a[cell + tap][ci]; gB[co] += sum_cells g[cell][co]. g is bf16
// [cell][16] (COUT = 16) or FP32 [cell] (COUT = 1); a is bf16 [cell][16].
template <int CIN, int COUT, bool GF32>
__global__ void __launch_bounds__(256) k_wgrad(const void *__restrict__ gptr, const __nv_bfloat16 *__restrict__ a,
                                               float *gW, float *gB, Layout L)
{
    constexpr int NOUT = COUT * CIN * 27;
    extern __shared__ float wg_smem[];
    float(*sg)[COUT] = reinterpret_cast<float(*)[COUT]>(wg_smem);
    float(*sa)[CIN] = reinterpret_cast<float(*)[CIN]>(wg_smem + NT_X * NT_Y * COUT);
    float part[(NOUT + 255) / 256];
    float bpart = 0.f;
#pragma unroll
    for (int u = 0; u < (NOUT + 255) / 256; u++) part[u] = 0.f;
    const int tid = threadIdx.x;
    const int ntx = (L.nx + NT_X - 1) / NT_X, nty = (L.ny + NT_Y - 1) / NT_Y;
    const int ntiles = ntx * nty * L.nz;
    for (int tb = blockIdx.x; tb < ntiles; tb += gridDim.x) {
        const int tx = tb % ntx, ty = (tb / ntx) % nty, tk = tb / (ntx * nty);
        const int i0 = tx * NT_X, j0 = ty * NT_Y;
        __syncthreads();
        for (int e = tid; e < NT_X * NT_Y * COUT; e += blockDim.x) {
            const int cl = e / COUT, o = e % COUT;
            const int gi = i0 + cl % NT_X, gj = j0 + cl / NT_X;
            float v = 0.f;
            if (gi < L.nx && gj < L.ny) {
                const size_t t = (size_t)cell_t(L, gi, gj, tk);
                v = GF32 ? static_cast<const float *>(gptr)[t]
                         : __bfloat162float(static_cast<const __nv_bfloat16 *>(gptr)[t * 16 + o]);
            }
            sg[cl][o] = v;
        }
        for (int e = tid; e < TCELLS * CIN; e += blockDim.x) {
            const int cidx = e / CIN, ci = e % CIN;
            const int xx = cidx % TXH, yy = (cidx / TXH) % TYH, zz = cidx / (TXH * TYH);
            const int gi = i0 - 1 + xx, gj = j0 - 1 + yy, gk = tk - 1 + zz;
            sa[cidx][ci] = in_grid(L, gi, gj, gk) ? __bfloat162float(a[(size_t)cell_t(L, gi, gj, gk) * 16 + ci]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < (NOUT + 255) / 256; u++) {
            const int o = tid + u * 256;
            if (o >= NOUT) break;
            const int tp = o % 27, ci = (o / 27) % CIN, co = o / (27 * CIN);
            const int dz = tp / 9, dy = (tp / 3) % 3, dx = tp % 3;
            float acc = 0.f;
            for (int cl = 0; cl < NT_X * NT_Y; cl++) {
                const float g = sg[cl][co];
                const int cx = cl % NT_X, cy = cl / NT_X;
                acc += g * sa[(dz * TYH + cy + dy) * TXH + cx + dx][ci];
            }
            part[u] += acc;
        }
        if (tid < COUT)
            for (int cl = 0; cl < NT_X * NT_Y; cl++) bpart += sg[cl][tid];
    }
#pragma unroll
    for (int u = 0; u < (NOUT + 255) / 256; u++) {
        const int o = tid + u * 256;
        if (o < NOUT) atomicAdd(gW + o, part[u]);
    }
    if (tid < COUT) atomicAdd(gB + tid, bpart);
}

// A parameter that does not depend on the residual: a bias, or a weight of the
// cell-type input channel (W1[co][1][tap]).
__device__ __forceinline__ bool offset_param(int t)
{
    if (t < OB1) return (t / 27) % 2 == 1;
    return (t >= OB1 && t < OW2) || (t >= OB2 && t < OW3) || (t >= OB3 && t < OW4) || (t >= OB4 && t < OW5) ||
           t >= OB5;
}

// Adam on the FP32 master copy; the gradient buffer is cleared. With
// `fix_offsets` the offset parameters keep their values.
__global__ void k_adam(float *p, float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, float gscale, int fix_offsets)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (fix_offsets && offset_param(t)) {
            g[t] = 0.f;
            continue;
        }
        const float gr = g[t] * gscale;
        const float mm = b1 * m[t] + (1.f - b1) * gr;
        const float vv = b2 * v[t] + (1.f - b2) * gr * gr;
        m[t] = mm;
        v[t] = vv;
        p[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        g[t] = 0.f;
    }
}

// bf16 working copies from the master copy
__global__ void k_net_refresh(const float *__restrict__ p, float *w1f, float *w5f, __nv_bfloat16 *wf,
                              __nv_bfloat16 *wt, __nv_bfloat16 *wf1, __nv_bfloat16 *wf5)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < NPARAM; t += gridDim.x * blockDim.x) {
        if (t < OB1) {
            w1f[t] = bfr(p[t]);
            const int tp = t % 27, ci = (t / 27) % 2, co = t / 54;  // [co][ci][tap]
            wf1[(tp * 16 + co) * 16 + ci] = __float2bfloat16(p[t]);
        }
        if (t >= OW5 && t < OB5) {
            w5f[t - OW5] = bfr(p[t]);
            const int tp = (t - OW5) % 27, ci = (t - OW5) / 27;    // [1][ci][tap]
            wf5[(tp * 16 + 0) * 16 + ci] = __float2bfloat16(p[t]);
        }
        const int offs[3] = {OW2, OW3, OW4};
        for (int l = 0; l < 3; l++) {
            if (t < offs[l] || t >= offs[l] + NWM) continue;
            const int e = t - offs[l];
            const int tp = e % 27, ci = (e / 27) % 16, co = e / (27 * 16);
            const __nv_bfloat16 v = __float2bfloat16(p[t]);
            wf[(size_t)l * NWM + (tp * 16 + co) * 16 + ci] = v;            // [tap][n = co][k = ci]
            wt[(size_t)l * NWM + ((26 - tp) * 16 + ci) * 16 + co] = v;     // [tap'][n = ci][k = co]
        }
    }
}

__global__ void k_fill_zero(float *p, int n)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) p[t] = 0.f;
}

}  // namespace

static NetState *net(fs_ctx *c) { return static_cast<NetState *>(c->net); }

static size_t conv_smem() { return (size_t)TCELLS * 32 + 27 * 16 * 32; }

static int conv_tiles(const Layout &L) { return ((L.nx + NT_X - 1) / NT_X) * ((L.ny + NT_Y - 1) / NT_Y) * L.nz; }

template <int CIN, int COUT>
static size_t wgrad_smem() { return ((size_t)NT_X * NT_Y * COUT + (size_t)TCELLS * CIN) * 4; }

static int conv_tiles_tc(const Layout &L)
{
    return ((L.nx + TC_M - 1) / TC_M) * ((L.ny + TC_NY - 1) / TC_NY) * L.nz;
}

int net_alloc(fs_ctx *c, bool training)
{
    if (c->net && (!training || net(c)->gact)) return FS_OK;
    NetState *n = net(c);
    if (!n) {
        n = new (std::nothrow) NetState();
        if (!n) return set_error(FS_ENOMEM, "host allocation failed");
        n->tlist_epoch = -1;
        c->net = n;
    }
    auto alloc = [&](void **p, size_t bytes) -> int {
        if (*p) return FS_OK;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            return set_error(FS_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        }
        return check_cuda(cudaMemset(*p, 0, bytes), "cudaMemset");
    };
    const size_t nC = (size_t)c->L.nC;
    int rc;
    if ((rc = alloc((void **)&n->master, NPARAM * 4)) || (rc = alloc((void **)&n->grad, NPARAM * 4)) ||
        (rc = alloc((void **)&n->m, NPARAM * 4)) || (rc = alloc((void **)&n->v, NPARAM * 4)) ||
        (rc = alloc((void **)&n->w1f, NW1 * 4)) || (rc = alloc((void **)&n->w5f, NW5 * 4)) ||
        (rc = alloc((void **)&n->wf, 3 * NWM * 2)) || (rc = alloc((void **)&n->wt, 3 * NWM * 2)) ||
        (rc = alloc((void **)&n->smax, 16)) || (rc = alloc((void **)&n->y, nC * 4)) ||
        (rc = alloc((void **)&n->wf1, 27 * 16 * 16 * 2)) || (rc = alloc((void **)&n->wf5, 27 * 16 * 16 * 2)) ||
        (rc = alloc((void **)&n->tdist, (size_t)conv_tiles(c->L))) ||
        (rc = alloc((void **)&n->tlist, (size_t)conv_tiles(c->L) * sizeof(int))) ||
        (rc = alloc((void **)&n->tlist_tc, (size_t)conv_tiles_tc(c->L) * sizeof(int))))
        return rc;
    // inference needs two activation buffers; training keeps all five layer inputs
    const int nact = training ? 6 : 2;
    if (training && n->act && !n->gact) {
        cudaFree(n->act);
        n->act = nullptr;
    }
    if ((rc = alloc((void **)&n->act, nact * nC * 32))) return rc;
    if (training) {
        if ((rc = alloc((void **)&n->gact, 2 * nC * 32)) || (rc = alloc((void **)&n->gy, nC * 4))) return rc;
    }
    static bool attr_done = false;
    if (!attr_done) {
        const int cs = (int)conv_smem();
        FS_CUDA(cudaFuncSetAttribute(k_conv<IN_R, OUT_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
        FS_CUDA(cudaFuncSetAttribute(k_conv<IN_ACT, OUT_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
        FS_CUDA(cudaFuncSetAttribute(k_conv<IN_ACT, OUT_Z>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
        FS_CUDA(cudaFuncSetAttribute(k_conv<IN_ACT, OUT_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
        FS_CUDA(cudaFuncSetAttribute(k_conv_tc<IN_R, OUT_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TC_SMEM));
        FS_CUDA(cudaFuncSetAttribute(k_conv_tc<IN_ACT, OUT_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TC_SMEM));
        FS_CUDA(cudaFuncSetAttribute(k_conv_tc<IN_ACT, OUT_Z>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TC_SMEM));
        FS_CUDA(cudaFuncSetAttribute(k_wgrad<16, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wgrad_smem<16, 16>()));
        FS_CUDA(cudaFuncSetAttribute(k_wgrad<16, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wgrad_smem<16, 1>()));
        FS_CUDA(cudaFuncSetAttribute(k_wgrad<2, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wgrad_smem<2, 16>()));
        attr_done = true;
    }
    return FS_OK;
}

void net_free(fs_ctx *c)
{
    NetState *n = net(c);
    if (!n) return;
    void *ptrs[] = {n->master, n->grad, n->m, n->v, n->w1f, n->w5f, n->wf, n->wt, n->act, n->gact,
                    n->y, n->gy, n->smax, n->wf1, n->wf5, n->tdist, n->tlist, n->tlist_tc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete n;
    c->net = nullptr;
}

int net_load(fs_ctx *c, const float *params, int count, bool host)
{
    if (count != NPARAM) return set_error(FS_EINVAL, "the network has %d parameters, got %d", NPARAM, count);
    int rc = net_alloc(c, false);
    if (rc) return rc;
    NetState *n = net(c);
    FS_CUDA(cudaMemcpyAsync(n->master, params, NPARAM * 4, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            c->stream));
    k_net_refresh<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(n->master, n->w1f, n->w5f, n->wf, n->wt, n->wf1,
                                                                n->wf5);
    FS_CUDA(cudaGetLastError());
    FS_CUDA(cudaStreamSynchronize(c->stream));
    n->loaded = 1;
    return FS_OK;
}

int net_read(fs_ctx *c, float *params_host)
{
    NetState *n = net(c);
    if (!n || !n->loaded) return set_error(FS_ESTATE, "no network loaded");
    FS_CUDA(cudaMemcpyAsync(params_host, n->master, NPARAM * 4, cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

// Persistent grid of the conv kernel: as many blocks as fit on the SMs.
static int conv_grid(const fs_ctx *c, int tiles)
{
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv<IN_ACT, OUT_RELU>, 256, conv_smem()) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
    }
    return std::max(1, std::min(tiles, c->num_sms * per_sm));
}

// The conv tiles sorted by their distance to the liquid, for the current mask.
static int net_tile_list(fs_ctx *c)
{
    NetState *n = net(c);
    if (n->tlist_epoch == c->mask_epoch) return FS_OK;
    const Layout &L = c->L;
    const int nt = conv_tiles(L);
    k_conv_tile_dist<<<nt, 256, 0, c->stream>>>(c->cflag, L, n->tdist);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    std::vector<uint8_t> d((size_t)nt);
    FS_CUDA(cudaMemcpyAsync(d.data(), n->tdist, (size_t)nt, cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int> list;
    list.reserve((size_t)nt);
    for (int dd = 0; dd <= 5; dd++) {
        for (int t = 0; t < nt; t++)
            if (d[(size_t)t] == dd) list.push_back(t);
        n->tcount[dd] = (int)list.size();
    }
    FS_CUDA(cudaMemcpy(n->tlist, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice));
    // the tensor-core layer's tiles (TC_M x TC_NY of one plane, inside one row of
    // conv tiles since NT_Y is a multiple of TC_NY): the distance of the nearest
    // conv tile they overlap
    const int ntx = (L.nx + NT_X - 1) / NT_X, nty = (L.ny + NT_Y - 1) / NT_Y;
    const int ntxc = (L.nx + TC_M - 1) / TC_M, ntyc = (L.ny + TC_NY - 1) / TC_NY, ntc = conv_tiles_tc(L);
    std::vector<uint8_t> dc((size_t)ntc, 5);
    for (int t = 0; t < ntc; t++) {
        const int i0 = (t % ntxc) * TC_M, j0 = ((t / ntxc) % ntyc) * TC_NY, k = t / (ntxc * ntyc);
        const int ty = j0 / NT_Y;
        uint8_t m = 5;
        for (int tx = i0 / NT_X; tx <= std::min(ntx - 1, (i0 + TC_M - 1) / NT_X); tx++)
            m = std::min(m, d[(size_t)((k * nty + ty) * ntx + tx)]);
        dc[(size_t)t] = m;
    }
    std::vector<int> lc;
    lc.reserve((size_t)ntc);
    for (int dd = 0; dd <= 5; dd++) {
        for (int t = 0; t < ntc; t++)
            if (dc[(size_t)t] == dd) lc.push_back(t);
        n->tcount_tc[dd] = (int)lc.size();
    }
    FS_CUDA(cudaMemcpy(n->tlist_tc, lc.data(), lc.size() * sizeof(int), cudaMemcpyHostToDevice));
    n->tlist_epoch = c->mask_epoch;
    return FS_OK;
}

static void conv_launch(fs_ctx *c, int in, int out, const ConvArgs &a, int tiles)
{
    const int g = conv_grid(c, tiles);
    const size_t sm = conv_smem();
    if (in == IN_R)
        k_conv<IN_R, OUT_RELU><<<g, 256, sm, c->stream>>>(a);
    else if (out == OUT_RELU)
        k_conv<IN_ACT, OUT_RELU><<<g, 256, sm, c->stream>>>(a);
    else if (out == OUT_Z)
        k_conv<IN_ACT, OUT_Z><<<g, 256, sm, c->stream>>>(a);
    else
        k_conv<IN_ACT, OUT_BWD><<<g, 256, sm, c->stream>>>(a);
    c->n_launches += 1;
}

// The tensor-core layer: two blocks per SM (two input tiles and the weights each).
static void conv_launch_tc(fs_ctx *c, int in, int out, const ConvArgs &a, int tiles)
{
    const int g = std::max(1, std::min(tiles, c->num_sms * 2));
    if (in == IN_R)
        k_conv_tc<IN_R, OUT_RELU><<<g, TC_THREADS, TC_SMEM, c->stream>>>(a, c->err_word);
    else if (out == OUT_RELU)
        k_conv_tc<IN_ACT, OUT_RELU><<<g, TC_THREADS, TC_SMEM, c->stream>>>(a, c->err_word);
    else
        k_conv_tc<IN_ACT, OUT_Z><<<g, TC_THREADS, TC_SMEM, c->stream>>>(a, c->err_word);
    c->n_launches += 1;
}

// z = s Net(r / s) on liquid cells, 0 elsewhere (cell space). Training (`keep`)
// runs every layer on every tile and keeps the layer inputs in act[0..4] and the
// output in y; inference runs layer l on the tiles within 5 - l cells of the
// liquid, with activations ping-ponging in act[0..1].
static int net_forward(fs_ctx *c, const float *r, float *z, float *y, bool keep)
{
    NetState *n = net(c);
    const Layout &L = c->L;
    const size_t nC = (size_t)L.nC;
    int rc;
    if (!keep && (rc = net_tile_list(c))) return rc;
    FS_CUDA(cudaMemsetAsync(n->smax, 0, sizeof(unsigned), c->stream));
    k_absmax<<<grid_blocks(c, L.nC, 256), 256, 0, c->stream>>>(r, c->cflag, L.nC, n->smax);
    c->n_launches += 1;
    if (z) FS_CUDA(cudaMemsetAsync(z, 0, nC * sizeof(float), c->stream));
    __nv_bfloat16 *A[6];
    for (int l = 0; l < 6; l++) A[l] = n->act + (keep ? (size_t)l : (size_t)(l & 1)) * nC * 16;
    const int all = conv_tiles(L);
    const bool tc = !keep && n->kernel == 1;  // inference on the tcgen05 layer
    auto tiles_for = [&](int layer) {         // layer 1 .. 5
        return keep ? all : (tc ? n->tcount_tc[5 - layer] : n->tcount[5 - layer]);
    };
    auto launch = [&](int in, int out, const ConvArgs &ca) {
        if (tc)
            conv_launch_tc(c, in, out, ca, ca.ntiles);
        else
            conv_launch(c, in, out, ca, ca.ntiles);
    };
    ConvArgs a{};
    a.cf = c->cflag;
    a.smax = n->smax;
    a.tiles = keep ? nullptr : (tc ? n->tlist_tc : n->tlist);
    a.L = L;
    // layer 1: input built from r; keep: x -> A[0], a1 -> A[1]
    a.r = r;
    a.wts = n->wf1;
    a.bias = n->master + OB1;
    a.xin = keep ? A[0] : nullptr;
    a.out = keep ? A[1] : A[0];
    a.ntiles = tiles_for(1);
    launch(IN_R, OUT_RELU, a);
    __nv_bfloat16 *cur = a.out;
    a.xin = nullptr;
    a.r = nullptr;
    const int bias_off[3] = {OB2, OB3, OB4};
    for (int l = 0; l < 3; l++) {
        __nv_bfloat16 *nxt = keep ? A[2 + l] : (cur == A[0] ? A[1] : A[0]);
        a.in = cur;
        a.wts = n->wf + (size_t)l * NWM;
        a.bias = n->master + bias_off[l];
        a.out = nxt;
        a.ntiles = tiles_for(2 + l);
        launch(IN_ACT, OUT_RELU, a);
        cur = nxt;
    }
    a.in = cur;
    a.wts = n->wf5;
    a.bias = n->master + OB5;
    a.out = nullptr;
    a.y = y;
    a.z = z;
    a.ntiles = tiles_for(5);
    launch(IN_ACT, OUT_Z, a);
    FS_CUDA(cudaGetLastError());
    // the useful flops of the layers, on the cells of the tiles they visit (both
    // tilings hold 256 cells a tile): 2 x 27 x (2 x 16 + 3 x 16 x 16 + 16 x 1) per cell
    n->last_flops = 0.0;
    const double fl[5] = {2.0 * 27 * 2 * 16, 2.0 * 27 * 16 * 16, 2.0 * 27 * 16 * 16, 2.0 * 27 * 16 * 16, 2.0 * 27 * 16};
    for (int l = 1; l <= 5; l++) n->last_flops += fl[l - 1] * 256.0 * (double)tiles_for(l);
    return FS_OK;
}

int net_apply(fs_ctx *c, const float *r, float *z)
{
    NetState *n = net(c);
    if (!n || !n->loaded) return set_error(FS_ESTATE, "the learned preconditioner has no network loaded");
    cudaEvent_t e0 = prof_mark(c);
    int rc = net_forward(c, r, z, nullptr, false);
    prof_add(c, K_NET_APPLY, e0, prof_mark(c), n->last_flops);  // flops, not bytes: a tensor-core entry
    return rc;
}

int net_kernel(fs_ctx *c, int which)
{
    int rc = net_alloc(c, false);
    if (rc) return rc;
    net(c)->kernel = which;
    return FS_OK;
}

// Forward + backward for one (b, q) pair (public-layout cell arrays); adds the
// gradient to the accumulator and the loss to *loss.
int net_grad(fs_ctx *c, const float *b, const float *q, double *loss)
{
    int rc = net_alloc(c, true);
    if (rc) return rc;
    NetState *n = net(c);
    if (!n->loaded) return set_error(FS_ESTATE, "load initial network parameters first");
    const Layout &L = c->L;
    const size_t nC = (size_t)L.nC;
    const int ncell = L.nx * L.ny * L.nz;
    const int gb = std::max(1, std::min((ncell + 255) / 256, c->num_sms * 8));
    // b, q into cell space (zero off liquid): pb <- b, px <- q
    if ((rc = cell_in(c, b, c->pb)) || (rc = cell_in(c, q, c->px))) return rc;
    if ((rc = net_forward(c, c->pb, nullptr, n->y, true))) return rc;
    __nv_bfloat16 *A[5];
    for (int l = 0; l < 5; l++) A[l] = n->act + (size_t)l * nC * 16;
    SolveScal *s = c->scal + 3;
    const int bsn = grid_blocks(c, L.nC, 256);
    if (c->prm.precond == FS_PRECOND_LEARNED_MG) {
        // the network followed by the V-cycle; scratch (no solve runs meanwhile):
        // pxh = ym, pr = b/s - A ym, pz = M pr, pp0 = w, pp1 = q/s, pq = A w, pbr = M A w
        k_net_mask_y<<<bsn, 256, 0, c->stream>>>(n->y, c->cflag, c->pxh, L.nC);
        k_netmg_res<<<bsn, 256, 0, c->stream>>>(c->pb, c->pxh, c->cflag, n->smax, L, c->pr);
        c->n_launches += 2;
        if ((rc = mg_apply(c, c->pr, c->pz, nullptr))) return rc;
        k_netmg_err<<<bsn, 256, 0, c->stream>>>(c->px, c->pxh, c->pz, c->cflag, n->smax, c->pp[0], c->pp[1], L.nC);
        k_net_energy<<<bsn, 256, 0, c->stream>>>(c->pp[0], c->pp[1], c->pq, c->cflag, L, s, c->partials);
        c->n_launches += 2;
        if ((rc = mg_apply(c, c->pq, c->pbr, nullptr))) return rc;
        k_netmg_gy<<<bsn, 256, 0, c->stream>>>(c->pq, c->pbr, c->cflag, s, L, n->gy);
        c->n_launches += 1;
    } else {
        // energy-norm loss; scratch: pr = e, pz = q/s, pq = A e (no solve runs meanwhile)
        k_net_err<<<bsn, 256, 0, c->stream>>>(n->y, c->px, c->cflag, n->smax, c->pr, c->pz, L.nC);
        k_net_energy<<<bsn, 256, 0, c->stream>>>(c->pr, c->pz, c->pq, c->cflag, L, s, c->partials);
        k_net_gy<<<bsn, 256, 0, c->stream>>>(c->pq, c->cflag, s, n->gy, L.nC);
        c->n_launches += 3;
    }
    // layer 5
    const int wg = std::max(1, std::min(((L.nx + NT_X - 1) / NT_X) * ((L.ny + NT_Y - 1) / NT_Y) * L.nz, c->num_sms * 2));
    k_wgrad<16, 1, true><<<wg, 256, wgrad_smem<16, 1>(), c->stream>>>(n->gy, A[4], n->grad + OW5, n->grad + OB5, L);
    __nv_bfloat16 *G[2] = {n->gact, n->gact + nC * 16};
    k_bwd_last<<<gb, 256, 0, c->stream>>>(n->gy, n->w5f, A[4], G[0], L);
    // layers 4, 3, 2: weight gradient, then the gradient of the layer input
    const int woff[3] = {OW2, OW3, OW4}, boff[3] = {OB2, OB3, OB4};
    int gi = 0;
    for (int l = 2; l >= 0; l--) {
        // G[gi] = dL/d(output of layer l+2) (post-ReLU mask applied); input = A[l+1]
        k_wgrad<16, 16, false><<<wg, 256, wgrad_smem<16, 16>(), c->stream>>>(G[gi], A[l + 1], n->grad + woff[l], n->grad + boff[l], L);
        ConvArgs bw{};
        bw.in = G[gi];
        bw.wts = n->wt + (size_t)l * NWM;
        bw.aref = A[l + 1];
        bw.out = G[gi ^ 1];
        bw.L = L;
        conv_launch(c, IN_ACT, OUT_BWD, bw, conv_tiles(L));
        gi ^= 1;
    }
    // layer 1: gradient w.r.t. W1 from the stored input x (2 channels used)
    k_wgrad<2, 16, false><<<wg, 256, wgrad_smem<2, 16>(), c->stream>>>(G[gi], A[0], n->grad + OW1, n->grad + OB1, L);
    c->n_launches += 2 + 6 + 1;
    FS_CUDA(cudaGetLastError());
    SolveScal h;
    if ((rc = read_scal(c, 3, &h))) return rc;
    if (loss) *loss += h.aux[1] > 0.0 ? h.aux[0] / h.aux[1] : 0.0;
    return FS_OK;
}

int net_adam(fs_ctx *c, double lr, double beta1, double beta2, double eps, int step, double gscale, int fix_offsets)
{
    NetState *n = net(c);
    if (!n || !n->loaded || !n->gact) return set_error(FS_ESTATE, "no gradients accumulated");
    if (step < 1) return set_error(FS_EINVAL, "step must be >= 1");
    const float c1 = (float)(1.0 - std::pow(beta1, step)), c2 = (float)(1.0 - std::pow(beta2, step));
    k_adam<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(n->master, n->grad, n->m, n->v, NPARAM, (float)lr,
                                                        (float)beta1, (float)beta2, (float)eps, c1, c2,
                                                        (float)gscale, fix_offsets);
    k_net_refresh<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(n->master, n->w1f, n->w5f, n->wf, n->wt, n->wf1,
                                                                n->wf5);
    c->n_launches += 2;
    FS_CUDA(cudaGetLastError());
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

int net_grad_read(fs_ctx *c, float *grad_host)
{
    NetState *n = net(c);
    if (!n || !n->gact) return set_error(FS_ESTATE, "no gradients accumulated");
    FS_CUDA(cudaMemcpyAsync(grad_host, n->grad, NPARAM * 4, cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

int net_grad_clear(fs_ctx *c)
{
    NetState *n = net(c);
    if (!n) return FS_OK;
    k_fill_zero<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(n->grad, NPARAM);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int net_param_count() { return NPARAM; }

bool net_loaded(const fs_ctx *c) { return c->net && static_cast<const NetState *>(c->net)->loaded; }

}  // namespace fs
