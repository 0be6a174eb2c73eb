// fs_fcg.cu -- truncated flexible CG for the pressure solve with the learned
// (nonlinear) preconditioner (the network that stands in for the implicit
// pressure solve, Sec. 3.4.1).
//
// With a preconditioner that changes from one application to the next, plain
// CG loses the conjugacy of its directions. Flexible CG (Notay, "Flexible
// conjugate gradients", SIAM J. Sci. Comput. 22(4), 2000) restores it by
// A-orthogonalising each new direction explicitly against the last M ones:
//   z_k = Net(r_k)
//   p_k = z_k - sum_{j=1..min(k,M)} (z_k . A p_{k-j} / p_{k-j} . A p_{k-j}) p_{k-j}
//   alpha_k = r_k . z_k / p_k . A p_k,   x += alpha_k p_k,   r -= alpha_k A p_k.
// The M most recent (p, A p, p.Ap) triples live in a ring of cell-space vectors.
// Per iteration: the network, then four HBM-bound kernels (dots, direction,
// operator + p.Ap, update); every decision is taken on the device, the host
// reads the scalars every check_every iterations.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "fs_internal.cuh"

namespace fs {
namespace {

constexpr int TH = 256;
constexpr int FCG_M = 4;

// The j-th most recent direction (j = 0 newest), its A p and its p.Ap.
struct Ring {
    const float *p[FCG_M];
    const float *q[FCG_M];
    const double *pq[FCG_M];
};

// beta_j = -z . A p_j / p_j . A p_j (j < nvalid) and r.z -> s->rz
__global__ void __launch_bounds__(TH) k_fcg_dots(const float *__restrict__ z, const float *__restrict__ r, Ring ring,
                                                 int nvalid, int n4, SolveScal *s, double *beta, double *partials)
{
    if (s->done) return;
    KSum acc[FCG_M + 1];
    const float4 *z4 = reinterpret_cast<const float4 *>(z);
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 a = __ldg(z4 + t);
        const float4 b = __ldg(r4 + t);
        acc[FCG_M].add(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w);
#pragma unroll
        for (int j = 0; j < FCG_M; j++) {
            if (j < nvalid) {
                const float4 c = __ldg(reinterpret_cast<const float4 *>(ring.q[j]) + t);
                acc[j].add(a.x * c.x + a.y * c.y + a.z * c.z + a.w * c.w);
            }
        }
    }
    KSum v[FCG_M + 1];
    double tot[FCG_M + 1];
#pragma unroll
    for (int j = 0; j <= FCG_M; j++) v[j] = acc[j];
    if (grid_reduce<FCG_M + 1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        bool ok = isfinite(tot[FCG_M]);
        for (int j = 0; j < FCG_M; j++) {
            const double pq = j < nvalid ? *ring.pq[j] : 0.0;
            beta[j] = (j < nvalid && pq > 0.0) ? -tot[j] / pq : 0.0;
            ok = ok && isfinite(beta[j]);
        }
        if (!ok) { s->done = 1; s->status = FS_ENONFINITE; return; }
        s->rz = tot[FCG_M];
    }
}

// p = z + sum_j beta_j p_j
__global__ void __launch_bounds__(TH) k_fcg_dir(const float *__restrict__ z, Ring ring, int nvalid,
                                                float *__restrict__ p, int n4, const SolveScal *s,
                                                const double *__restrict__ beta)
{
    if (s->done) return;
    float b[FCG_M];
#pragma unroll
    for (int j = 0; j < FCG_M; j++) b[j] = j < nvalid ? (float)beta[j] : 0.f;
    float4 *p4 = reinterpret_cast<float4 *>(p);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(z) + t);
#pragma unroll
        for (int j = 0; j < FCG_M; j++) {
            if (j < nvalid) {
                const float4 w = __ldg(reinterpret_cast<const float4 *>(ring.p[j]) + t);
                v.x += b[j] * w.x; v.y += b[j] * w.y; v.z += b[j] * w.z; v.w += b[j] * w.w;
            }
        }
        p4[t] = v;
    }
}

// q = L_p p (7-point pressure operator on liquid cells), p.q -> *pq_out,
// alpha = r.z / p.q
__global__ void __launch_bounds__(TH) k_fcg_apply(const float *__restrict__ p, float *__restrict__ q,
                                                  const uint8_t *__restrict__ cf, int n, int P, int PL, SolveScal *s,
                                                  double *pq_out, double *partials)
{
    if (s->done) return;
    KSum acc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = cf[t];
        float qv = 0.f;
        if (f & CF_LIQ) {
            const float nb = (p[t - 1] + p[t + 1]) + (p[t - P] + p[t + P]) + (p[t - PL] + p[t + PL]);
            qv = (float)(f & CF_D) * p[t] - nb;
            acc.add(p[t] * qv);
        }
        q[t] = qv;
    }
    KSum v[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        *pq_out = pq;
        s->pq = pq;
        if (!isfinite(pq)) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (!(pq > 0.0)) { s->done = 1; s->status = FS_EBREAKDOWN; }
        else s->alpha = s->rz / pq;
    }
}

// x += alpha p, r -= alpha q; r.r and the convergence decision
__global__ void __launch_bounds__(TH) k_fcg_update(float *__restrict__ x, float *__restrict__ r,
                                                   const float *__restrict__ p, const float *__restrict__ q, int n4,
                                                   SolveScal *s, double *partials)
{
    if (s->done) return;
    const float alpha = (float)s->alpha;
    KSum rr;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    float4 *r4 = reinterpret_cast<float4 *>(r);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 pv = __ldg(reinterpret_cast<const float4 *>(p) + t);
        const float4 qv = __ldg(reinterpret_cast<const float4 *>(q) + t);
        float4 xv = x4[t], rv = r4[t];
        xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
        rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
        x4[t] = xv;
        r4[t] = rv;
        rr.add(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
    }
    KSum v[1] = {rr};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->iter += 1;
        s->rr = tot[0];
        if (!isfinite(tot[0])) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (tot[0] <= s->tol2 * s->bb) { s->done = 1; s->status = FS_OK; }
        else if (s->iter >= s->maxit) { s->done = 1; s->status = FS_ENOCONV; }
    }
}

// x = 0, r = b; b.b and the scalars of a fresh solve
__global__ void __launch_bounds__(TH) k_fcg_init(const float *__restrict__ b, float *__restrict__ x,
                                                 float *__restrict__ r, int n4, double tol2, int maxit, SolveScal *s,
                                                 double *partials)
{
    KSum bb;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(b) + t);
        reinterpret_cast<float4 *>(r)[t] = v;
        reinterpret_cast<float4 *>(x)[t] = zero;
        bb.add(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
    }
    KSum v[1] = {bb};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->bb = tot[0];
        s->rr = tot[0];
        s->rz = 0.0;
        s->pq = 0.0;
        s->alpha = 0.0;
        s->beta = 0.0;
        s->tol2 = tol2;
        s->iter = 0;
        s->maxit = maxit;
        s->status = FS_OK;
        s->done = 0;
        if (!isfinite(tot[0])) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (tot[0] == 0.0) s->done = 1;
    }
}

struct FcgState {
    float *p[FCG_M] = {};
    float *q[FCG_M] = {};
    double *beta = nullptr;  // device [FCG_M]
    double *pq = nullptr;    // device [FCG_M], per ring slot
};

void fcg_free_state(FcgState *f)
{
    if (!f) return;
    for (int j = 0; j < FCG_M; j++) {
        cudaFree(f->p[j]);
        cudaFree(f->q[j]);
    }
    cudaFree(f->beta);
    cudaFree(f->pq);
    delete f;
}

int fcg_alloc(fs_ctx *c)
{
    if (c->fcg) return FS_OK;
    FcgState *f = new (std::nothrow) FcgState();
    if (!f) return set_error(FS_ENOMEM, "flexible CG: host allocation failed");
    const size_t cb = (size_t)c->L.nC * sizeof(float);
    bool ok = true;
    for (int j = 0; j < FCG_M && ok; j++)
        ok = cudaMalloc(&f->p[j], cb) == cudaSuccess && cudaMemset(f->p[j], 0, cb) == cudaSuccess &&
             cudaMalloc(&f->q[j], cb) == cudaSuccess && cudaMemset(f->q[j], 0, cb) == cudaSuccess;
    ok = ok && cudaMalloc(&f->beta, FCG_M * sizeof(double)) == cudaSuccess &&
         cudaMalloc(&f->pq, FCG_M * sizeof(double)) == cudaSuccess &&
         cudaMemset(f->pq, 0, FCG_M * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        fcg_free_state(f);
        return set_error(FS_ENOMEM, "flexible CG: device allocation of %d direction pairs failed", FCG_M);
    }
    c->fcg = f;
    return FS_OK;
}

}  // namespace

void fcg_release(fs_ctx *c)
{
    fcg_free_state(static_cast<FcgState *>(c->fcg));
    c->fcg = nullptr;
}

// Flexible CG on pb -> px with the loaded network, from x = 0 or (warm) from
// the current x with the true residual. Leaves the final scalars in *h (status
// FS_ENOCONV also when |r| stagnates: no tenfold drop over 200 iterations); the
// caller computes the true residual.
int solve_pressure_fcg(fs_ctx *c, SolveScal *h, bool warm)
{
    int rc = fcg_alloc(c);
    if (rc) return rc;
    FcgState *f = static_cast<FcgState *>(c->fcg);
    const Layout &L = c->L;
    SolveScal *s = c->scal + 0;
    const int n4 = L.nC / 4;
    const int b4 = grid_blocks(c, n4, TH), bs = grid_blocks(c, L.nC, TH);
    const double tol2 = c->prm.tol_p * c->prm.tol_p * (c->tol2_scale > 0.0 ? c->tol2_scale : 1.0);
    const double by_vec = (double)L.nC * 4.0;
    if (warm) {
        if ((rc = pressure_restart(c))) return rc;  // r = b - A x, iteration count kept
    } else {
        k_fcg_init<<<b4, TH, 0, c->stream>>>(c->pb, c->px, c->pr, n4, tol2, c->prm.maxit_p, s, c->partials);
        c->n_launches += 1;
    }
    FS_CUDA(cudaGetLastError());
    long long k = 0;
    std::vector<std::pair<int, double>> hist;  // (iteration, r.r) at the host checks
    for (;;) {
        if ((rc = read_scal(c, 0, h))) return rc;
        if (h->done) break;
        if (k > (long long)c->prm.maxit_p + c->prm.check_every)
            return set_error(FS_ECUDA, "flexible CG: iteration flag never set");
        hist.push_back({h->iter, h->rr});
        size_t m = hist.size();
        while (m > 0 && hist[m - 1].first > h->iter - 200) m--;
        if (m > 0 && h->iter >= 200 && h->rr > 1e-2 * hist[m - 1].second) {
            h->status = FS_ENOCONV;
            break;
        }
        for (int b = 0; b < c->prm.check_every; b++, k++) {
            const int slot = (int)(k % FCG_M);
            const int nvalid = (int)std::min<long long>(k, FCG_M);
            Ring ring;
            for (int j = 0; j < FCG_M; j++) {
                const int sj = (int)(((k - 1 - j) % FCG_M + FCG_M) % FCG_M);
                ring.p[j] = f->p[sj];
                ring.q[j] = f->q[sj];
                ring.pq[j] = f->pq + sj;
            }
            if ((rc = learned_apply(c, c->pr, c->pz, &s->done))) return rc;
            if ((rc = remove_null_mode(c, c->pz))) return rc;
            const bool samp = c->prof_on && (b % c->prof_period) == 0;
            cudaEvent_t e0 = samp ? prof_mark(c) : nullptr;
            k_fcg_dots<<<b4, TH, 0, c->stream>>>(c->pz, c->pr, ring, nvalid, n4, s, f->beta, c->partials);
            k_fcg_dir<<<b4, TH, 0, c->stream>>>(c->pz, ring, nvalid, f->p[slot], n4, s, f->beta);
            k_fcg_apply<<<bs, TH, 0, c->stream>>>(f->p[slot], f->q[slot], c->cflag, L.nC, L.P, L.PL, s,
                                                  f->pq + slot, c->partials);
            k_fcg_update<<<b4, TH, 0, c->stream>>>(c->px, c->pr, f->p[slot], f->q[slot], n4, s, c->partials);
            cudaEvent_t e1 = samp ? prof_mark(c) : nullptr;
            // vectors streamed: dots 2 + nvalid, direction 2 + nvalid, operator ~3, update 6
            prof_add(c, K_FCG_VEC, e0, e1, by_vec * (13.0 + 2.0 * nvalid));
            c->n_launches += 4;
        }
        FS_CUDA(cudaGetLastError());
    }
    return check_wait_error(c, "flexible CG");
}

}  // namespace fs
