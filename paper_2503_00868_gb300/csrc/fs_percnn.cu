// fs_percnn.cu -- recurrent convolutional pressure solver (arXiv 2503.00868,
// Sec. 3.4.1: the PeRCNN layer that replaces the implicit pressure solve during
// the optimisation, with a fitted convolution kernel and ~100 recurrent
// sub-steps per simulation step).
//
// Reading: the physics operator is the scheme's own 7-point L_p with the
// cell-type boundary conditions (air p = 0, solid walls zero flux), the fitted
// part a 3x3x3 kernel W on the residual, and the recurrent layer emulates an
// implicit solver's iteration:
//   p_0 = 0,  r_k = m (b - L_p p_k),  p_{k+1} = p_k + m (W * r_k),  k < K,
// m the liquid mask, * the 27-tap correlation (taps [dz][dy][dx]). Fixed points
// solve L_p p = b. The kernel is stored point-symmetric (W[t] = W[26 - t]), which
// makes the map b -> p_K symmetric and the projection built on it self-adjoint,
// so the step's adjoint applies the same projection to the cotangent.
// Per sub-step: one residual pass and one 27-point correlation pass (cell space).
//
// Training (fs_percnn_grad): the energy-norm loss of Sec. 3.4.1's fit,
//   e = p_K - q, loss = e^T L_p e / q^T L_p q,
// and dloss/dW by the backward recurrence over the stored residuals:
//   g_K = 2 L_p e / q^T L_p q;  for k = K-1 .. 0:
//   dW[t] += sum_i g_{k+1,i} r_k(i + t);  g_k = g_{k+1} - L_p (m W^T * g_{k+1}).
#include <cmath>
#include <new>

#include "fs_internal.cuh"

namespace fs {

struct PercnnW {
    float w[27];
};

struct PercnnState {
    PercnnW w;
    int K = 0;
    int loaded = 0;
    float *rstack = nullptr;  // K residuals (training)
    int rstack_k = 0;
    float *gk = nullptr, *t1 = nullptr;  // cell space
    double *dw = nullptr;     // device [27]
};

namespace {

constexpr int TH = 256;

__device__ __forceinline__ int tap_offset(const Layout &L, int t)
{
    return (t / 9 - 1) * L.PL + ((t / 3) % 3 - 1) * L.P + (t % 3 - 1);
}

// r = m (b - L_p p)
__global__ void __launch_bounds__(TH) k_pc_res(const float *__restrict__ b, const float *__restrict__ p,
                                               float *__restrict__ r, const uint8_t *__restrict__ cf, int n, int P,
                                               int PL)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        float v = 0.f;
        if (f & CF_LIQ) {
            const float nb = (p[t - 1] + p[t + 1]) + (p[t - P] + p[t + P]) + (p[t - PL] + p[t + PL]);
            v = b[t] - ((float)(f & CF_D) * p[t] - nb);
        }
        r[t] = v;
    }
}

// out = m (W * x) (+ base when base != null): 27-tap correlation on liquid cells
__global__ void __launch_bounds__(TH) k_pc_conv(const float *__restrict__ x, const float *base, float *out,
                                                const uint8_t *__restrict__ cf, Layout L, PercnnW W)
{
    __shared__ int off[27];
    if (threadIdx.x < 27) off[threadIdx.x] = tap_offset(L, threadIdx.x);
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nC; t += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (cf[t] & CF_LIQ) {
#pragma unroll
            for (int q = 0; q < 27; q++) v += W.w[q] * x[t + off[q]];
        }
        out[t] = (base ? base[t] : 0.f) + v;
    }
}

// g = m (g - L_p s)
__global__ void __launch_bounds__(TH) k_pc_lapsub(float *g, const float *__restrict__ s,
                                                  const uint8_t *__restrict__ cf, int n, int P, int PL)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        if (f & CF_LIQ) {
            const float nb = (s[t - 1] + s[t + 1]) + (s[t - P] + s[t + P]) + (s[t - PL] + s[t + PL]);
            g[t] -= (float)(f & CF_D) * s[t] - nb;
        } else {
            g[t] = 0.f;
        }
    }
}

// dw[q] += sum over liquid cells of g_i r(i + o_q)
__global__ void __launch_bounds__(TH) k_pc_wgrad(const float *__restrict__ g, const float *__restrict__ r,
                                                 const uint8_t *__restrict__ cf, Layout L, double *dw)
{
    __shared__ double sh[TH / 32][27];
    int off[27];
#pragma unroll
    for (int q = 0; q < 27; q++) off[q] = tap_offset(L, q);
    double acc[27];
#pragma unroll
    for (int q = 0; q < 27; q++) acc[q] = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L.nC; t += gridDim.x * blockDim.x) {
        if (!(cf[t] & CF_LIQ)) continue;
        const float gv = g[t];
        if (gv == 0.f) continue;
#pragma unroll
        for (int q = 0; q < 27; q++) acc[q] += (double)(gv * r[t + off[q]]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 27; q++) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 27) {
        double s = 0.0;
        for (int w = 0; w < TH / 32; w++) s += sh[w][threadIdx.x];
        atomicAdd(dw + threadIdx.x, s);
    }
}

// e = m (p - q)
__global__ void __launch_bounds__(TH) k_pc_energy(const float *__restrict__ p, const float *__restrict__ q,
                                                  float *e, const uint8_t *__restrict__ cf, int n)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        e[t] = (cf[t] & CF_LIQ) ? p[t] - q[t] : 0.f;
}

// e.Ae and q.Aq over the liquid -> aux[0], aux[1]; Ae kept in ae
__global__ void __launch_bounds__(TH) k_pc_quad(const float *__restrict__ e, const float *__restrict__ q,
                                                float *ae, const uint8_t *__restrict__ cf, int n, int P, int PL,
                                                SolveScal *s, double *partials)
{
    KSum ee, qq;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        float a = 0.f;
        if (f & CF_LIQ) {
            const float d = (float)(f & CF_D);
            a = d * e[t] - ((e[t - 1] + e[t + 1]) + (e[t - P] + e[t + P]) + (e[t - PL] + e[t + PL]));
            const float aq = d * q[t] - ((q[t - 1] + q[t + 1]) + (q[t - P] + q[t + P]) + (q[t - PL] + q[t + PL]));
            ee.add(e[t] * a);
            qq.add(q[t] * aq);
        }
        ae[t] = a;
    }
    double v[2] = {ee.value(), qq.value()}, tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->aux[0] = tot[0];
        s->aux[1] = tot[1];
    }
}

__global__ void k_pc_scale(float *g, const SolveScal *s, int n)
{
    const double den = s->aux[1];
    const float sc = den > 0.0 ? (float)(2.0 / den) : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) g[t] *= sc;
}

// |r|^2 and |b|^2 over the liquid into the scalars of a finished solve of K sub-steps
__global__ void __launch_bounds__(TH) k_pc_finish(const float *__restrict__ b, const float *__restrict__ r,
                                                  const uint8_t *__restrict__ cf, int n, int K, SolveScal *s,
                                                  double *partials)
{
    KSum rr, bb;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        if (cf[t] & CF_LIQ) {
            rr.add(r[t] * r[t]);
            bb.add(b[t] * b[t]);
        }
    double v[2] = {rr.value(), bb.value()}, tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->rr = tot[0];
        s->bb = tot[1];
        s->iter = K;
        s->done = 1;
        s->status = (isfinite(tot[0]) && isfinite(tot[1])) ? FS_OK : FS_ENONFINITE;
    }
}

PercnnState *pcs(fs_ctx *c) { return static_cast<PercnnState *>(c->percnn); }

}  // namespace

void percnn_free(fs_ctx *c)
{
    PercnnState *s = pcs(c);
    if (!s) return;
    cudaFree(s->rstack);
    cudaFree(s->gk);
    cudaFree(s->t1);
    cudaFree(s->dw);
    delete s;
    c->percnn = nullptr;
}

bool percnn_loaded(const fs_ctx *c) { return c->percnn && static_cast<const PercnnState *>(c->percnn)->loaded; }

int percnn_load(fs_ctx *c, const float *w27, int K)
{
    if (!w27) return set_error(FS_EINVAL, "the kernel is NULL");
    if (K < 1 || K > 100000) return set_error(FS_EINVAL, "substeps must be in [1, 100000]");
    for (int t = 0; t < 27; t++)
        if (!std::isfinite(w27[t])) return set_error(FS_EINVAL, "kernel tap %d is not finite", t);
    PercnnState *s = pcs(c);
    if (!s) {
        s = new (std::nothrow) PercnnState();
        if (!s) return set_error(FS_ENOMEM, "host allocation failed");
        c->percnn = s;
    }
    for (int t = 0; t < 27; t++) s->w.w[t] = 0.5f * (w27[t] + w27[26 - t]);  // point-symmetric
    s->K = K;
    s->loaded = 1;
    return FS_OK;
}

int percnn_read(fs_ctx *c, float *w27, int *K)
{
    PercnnState *s = pcs(c);
    if (!s || !s->loaded) return set_error(FS_ESTATE, "no recurrent-solver kernel loaded");
    for (int t = 0; t < 27; t++) w27[t] = s->w.w[t];
    if (K) *K = s->K;
    return FS_OK;
}

// pb -> px by K sub-steps (pr scratch); h gets K and the scalars of the true residual
int solve_pressure_percnn(fs_ctx *c, SolveScal *h)
{
    PercnnState *s = pcs(c);
    if (!s || !s->loaded) return set_error(FS_ESTATE, "the recurrent pressure solver has no kernel loaded");
    const Layout &L = c->L;
    const int bs = grid_blocks(c, L.nC, TH);
    FS_CUDA(cudaMemsetAsync(c->px, 0, (size_t)L.nC * sizeof(float), c->stream));
    for (int k = 0; k < s->K; k++) {
        k_pc_res<<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->pr, c->cflag, L.nC, L.P, L.PL);
        k_pc_conv<<<bs, TH, 0, c->stream>>>(c->pr, c->px, c->px, c->cflag, L, s->w);
        c->n_launches += 2;
    }
    FS_CUDA(cudaGetLastError());
    if (c->singular) {
        int rc = remove_null_mode(c, c->px);
        if (rc) return rc;
    }
    k_pc_res<<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->pr, c->cflag, L.nC, L.P, L.PL);
    k_pc_finish<<<bs, TH, 0, c->stream>>>(c->pb, c->pr, c->cflag, L.nC, s->K, c->scal + 0, c->partials);
    c->n_launches += 2;
    FS_CUDA(cudaGetLastError());
    return read_scal(c, 0, h);
}

int percnn_grad(fs_ctx *c, const float *b, const float *q, double *loss, float *dw_host)
{
    PercnnState *s = pcs(c);
    if (!s || !s->loaded) return set_error(FS_ESTATE, "no recurrent-solver kernel loaded");
    const Layout &L = c->L;
    const size_t nC = (size_t)L.nC;
    const int K = s->K;
    if ((double)K * nC * 4.0 > 8e9) return set_error(FS_EINVAL, "K x grid too large for the residual stack");
    if (s->rstack_k < K) {
        cudaFree(s->rstack);
        s->rstack = nullptr;
        s->rstack_k = 0;
        if (cudaMalloc(&s->rstack, (size_t)K * nC * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FS_ENOMEM, "residual stack of %d x %zu floats", K, nC);
        }
        s->rstack_k = K;
    }
    if (!s->gk) {
        if (cudaMalloc(&s->gk, nC * 4) != cudaSuccess || cudaMalloc(&s->t1, nC * 4) != cudaSuccess ||
            cudaMalloc(&s->dw, 27 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FS_ENOMEM, "recurrent-solver training buffers");
        }
        FS_CUDA(cudaMemset(s->gk, 0, nC * 4));
        FS_CUDA(cudaMemset(s->t1, 0, nC * 4));
    }
    int rc;
    if ((rc = cell_in(c, b, c->pb)) || (rc = cell_in(c, q, c->pz))) return rc;
    const int bs = grid_blocks(c, L.nC, TH);
    FS_CUDA(cudaMemsetAsync(c->px, 0, nC * 4, c->stream));
    for (int k = 0; k < K; k++) {
        float *r = s->rstack + (size_t)k * nC;
        k_pc_res<<<bs, TH, 0, c->stream>>>(c->pb, c->px, r, c->cflag, L.nC, L.P, L.PL);
        k_pc_conv<<<bs, TH, 0, c->stream>>>(r, c->px, c->px, c->cflag, L, s->w);
    }
    // loss and g_K = 2 L e / q.Lq
    SolveScal *sc = c->scal + 3;
    k_pc_energy<<<bs, TH, 0, c->stream>>>(c->px, c->pz, c->pr, c->cflag, L.nC);
    k_pc_quad<<<bs, TH, 0, c->stream>>>(c->pr, c->pz, s->gk, c->cflag, L.nC, L.P, L.PL, sc, c->partials);
    k_pc_scale<<<bs, TH, 0, c->stream>>>(s->gk, sc, L.nC);
    FS_CUDA(cudaMemsetAsync(s->dw, 0, 27 * sizeof(double), c->stream));
    for (int k = K - 1; k >= 0; k--) {
        const float *r = s->rstack + (size_t)k * nC;
        k_pc_wgrad<<<bs, TH, 0, c->stream>>>(s->gk, r, c->cflag, L, s->dw);
        k_pc_conv<<<bs, TH, 0, c->stream>>>(s->gk, nullptr, s->t1, c->cflag, L, s->w);  // W symmetric: W^T = W
        k_pc_lapsub<<<bs, TH, 0, c->stream>>>(s->gk, s->t1, c->cflag, L.nC, L.P, L.PL);
    }
    c->n_launches += 2 * K + 3 + 3 * K;
    FS_CUDA(cudaGetLastError());
    double dw[27];
    FS_CUDA(cudaMemcpyAsync(dw, s->dw, sizeof(dw), cudaMemcpyDeviceToHost, c->stream));
    SolveScal h;
    if ((rc = read_scal(c, 3, &h))) return rc;
    if (loss) *loss += h.aux[1] > 0.0 ? h.aux[0] / h.aux[1] : 0.0;
    if (dw_host)
        for (int t = 0; t < 27; t++) dw_host[t] += (float)dw[t];
    return FS_OK;
}

}  // namespace fs
