// fs_pcg.cu -- the two linear solves of the step and the field kernels around
// them (arXiv 2503.00868, Eq. eq::v split as in Sec. 3.2.2):
//   * pressure: L_p q = b on liquid cells (7-point, p = 0 in air), PCG;
//   * viscosity: (I + nu dt L_f) u = rhs on fluid faces, Jacobi-PCG;
//   * divergence, pressure-gradient subtraction, the nu-gradient of the
//     viscosity solve and the loss of Eq. eq::optLoss (Sec. 3.4.2).
//
// The CG scalars (alpha, beta, r.z, r.r) stay on the device: the last block of
// each reducing kernel updates them, so a batch of iterations runs without a
// host round trip; the host reads the convergence flag every `check_every`
// iterations. Once `done` is set every later kernel of the batch returns at once.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "fs_internal.cuh"

namespace fs {
namespace {

constexpr int TH = 256;

struct PoisOp {
    static constexpr uint8_t ACTIVE = CF_LIQ;
    __device__ static __forceinline__ float diag(uint8_t f, float) { return (float)(f & CF_D); }
    __device__ static __forceinline__ float offc(float) { return 1.f; }
};

struct HelmOp {
    static constexpr uint8_t ACTIVE = FF_FLUID;
    __device__ static __forceinline__ float diag(uint8_t f, float cc) { return 1.f + cc * (float)(f & FF_N); }
    __device__ static __forceinline__ float offc(float cc) { return cc; }
};

template <class Op>
__device__ __forceinline__ float inv_diag(uint8_t f, float cc)
{
    if (!(f & Op::ACTIVE)) return 0.f;
    float d = Op::diag(f, cc);
    return d > 0.f ? __frcp_rn(d) : 0.f;
}

// The operator apply over lists of active quads (those holding an unknown; the
// multigrid hierarchy's level-0 lists, one per volume, volume v from element
// base[v]): per quad, p_new = z + beta p_old on the quad and its six neighbours
// (inactive elements hold z = p_old = 0, so p_new = 0 there), q = A p_new on the
// quad, both written whole, and p_new . q. A thread strides through the lists
// with the next entry fetched a step ahead, so only quads with an unknown are
// read or written, where a 128 x 8 tile carries many without.
struct QuadLists {
    const int *ql[3];
    int n[3];
    long long base[3];
    int nv;
};

template <class Op>
__global__ void __launch_bounds__(TH) k_spmv_list(QuadLists Ls, const float *__restrict__ src,
                                                  const float *__restrict__ pold, float *__restrict__ pnew,
                                                  float *__restrict__ q, const uint8_t *__restrict__ fl, int P,
                                                  int PL, float cc, SolveScal *s, double *partials)
{
    if (s->done) return;
    const float beta = (float)s->beta;
    const float off = Op::offc(cc);
    KSum acc;
    const int st = gridDim.x * blockDim.x;
    for (int v = 0; v < Ls.nv; v++) {
        const long long base = Ls.base[v];
        const int *ql = Ls.ql[v];
        const int na = Ls.n[v];
        int i = blockIdx.x * blockDim.x + threadIdx.x;
        int qn = i < na ? __ldg(ql + i) : 0;
        for (; i < na; i += st) {
            const long long t = base + 4LL * qn;
            qn = i + st < na ? __ldg(ql + i + st) : 0;
            const uchar4 f = __ldg(reinterpret_cast<const uchar4 *>(fl + t));
            auto pn4 = [&](long long u) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(src + u));
                const float4 b = __ldg(reinterpret_cast<const float4 *>(pold + u));
                return make_float4(a.x + beta * b.x, a.y + beta * b.y, a.z + beta * b.z, a.w + beta * b.w);
            };
            auto pn1 = [&](long long u) { return __ldg(src + u) + beta * __ldg(pold + u); };
            const float4 c = pn4(t), dn = pn4(t - P), up = pn4(t + P), bk = pn4(t - PL), fw = pn4(t + PL);
            const float lf = pn1(t - 1), rt = pn1(t + 4);
            auto one = [&](uint8_t fe, float ce, float nb) {
                return (fe & Op::ACTIVE) ? Op::diag(fe, cc) * ce - off * nb : 0.f;
            };
            float4 qv;
            qv.x = one(f.x, c.x, (lf + c.y) + (dn.x + up.x) + (bk.x + fw.x));
            qv.y = one(f.y, c.y, (c.x + c.z) + (dn.y + up.y) + (bk.y + fw.y));
            qv.z = one(f.z, c.z, (c.y + c.w) + (dn.z + up.z) + (bk.z + fw.z));
            qv.w = one(f.w, c.w, (c.z + rt) + (dn.w + up.w) + (bk.w + fw.w));
            acc.add(c.x * qv.x + c.y * qv.y + c.z * qv.z + c.w * qv.w);
            *reinterpret_cast<float4 *>(pnew + t) = c;
            *reinterpret_cast<float4 *>(q + t) = qv;
        }
    }
    KSum vv[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(vv, partials, &s->ticket, tot) && threadIdx.x == 0) {
        double pq = tot[0];
        s->pq = pq;
        if (!isfinite(pq)) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (!(pq > 0.0)) { s->done = 1; s->status = FS_EBREAKDOWN; }
        else s->alpha = s->rz / pq;
    }
}

// Flat versions of the two CG kernels, for a context without tile maps.
// p_new = z + beta p_old (z the stored preconditioned residual; for Jacobi the
// solver keeps z = D^-1 r itself), then q = A p_new and the partial sums of
// p_new . q. alpha = r.z / p.q at the end.
template <class Op>
__global__ void __launch_bounds__(TH) k_spmv(const float *__restrict__ src, const float *__restrict__ pold,
                                             float *__restrict__ pnew, float *__restrict__ q,
                                             const uint8_t *__restrict__ fl, int n, int P, int PL, float cc,
                                             SolveScal *s, double *partials)
{
    if (s->done) return;
    const float beta = (float)s->beta;
    KSum acc;
    // Inactive elements keep p = q = 0 (set when the solve starts), so they are
    // neither read nor written here: only their flag byte is touched.
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = fl[t];
        if (!(f & Op::ACTIVE)) continue;
        auto pn = [&](int u) -> float { return __ldg(src + u) + beta * __ldg(pold + u); };
        const float pc = pn(t);
        const float nb = (pn(t - 1) + pn(t + 1)) + (pn(t - P) + pn(t + P)) + (pn(t - PL) + pn(t + PL));
        const float qv = Op::diag(f, cc) * pc - Op::offc(cc) * nb;
        acc.add(pc * qv);
        pnew[t] = pc;
        q[t] = qv;
    }
    KSum v[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        double pq = tot[0];
        s->pq = pq;
        if (!isfinite(pq)) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (!(pq > 0.0)) { s->done = 1; s->status = FS_EBREAKDOWN; }
        else s->alpha = s->rz / pq;
    }
}

// x += alpha p, r -= alpha q; partial sums of r.r (and r.z for Jacobi); the
// last block counts the iteration and decides convergence.
template <class Op, bool JAC>
__global__ void __launch_bounds__(TH) k_update(float *__restrict__ x, float *__restrict__ r,
                                               const float *__restrict__ p, const float *__restrict__ q,
                                               const uint8_t *__restrict__ fl, int n4, float cc,
                                               SolveScal *s, double *partials)
{
    if (s->done) return;
    const float alpha = (float)s->alpha;
    KSum rz, rr;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    float4 *r4 = reinterpret_cast<float4 *>(r);
    const float4 *p4 = reinterpret_cast<const float4 *>(p);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    const uchar4 *f4 = reinterpret_cast<const uchar4 *>(fl);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const uchar4 fv = f4[t];
        // four inactive elements: p = q = 0 there, nothing changes
        if (!((fv.x | fv.y | fv.z | fv.w) & Op::ACTIVE)) continue;
        float4 xv = x4[t], rv = r4[t];
        const float4 pv = __ldg(p4 + t), qv = __ldg(q4 + t);
        xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z; xv.w += alpha * pv.w;
        if (JAC) {
            // scaled residual z = D^-1 r: z -= alpha D^-1 Ap; r.z = sum d z^2, r.r = sum (d z)^2
            rv.x -= alpha * inv_diag<Op>(fv.x, cc) * qv.x; rv.y -= alpha * inv_diag<Op>(fv.y, cc) * qv.y;
            rv.z -= alpha * inv_diag<Op>(fv.z, cc) * qv.z; rv.w -= alpha * inv_diag<Op>(fv.w, cc) * qv.w;
            const float ax = Op::diag(fv.x, cc) * rv.x, ay = Op::diag(fv.y, cc) * rv.y;
            const float az = Op::diag(fv.z, cc) * rv.z, aw = Op::diag(fv.w, cc) * rv.w;
            rz.add(ax * rv.x + ay * rv.y + az * rv.z + aw * rv.w);
            rr.add(ax * ax + ay * ay + az * az + aw * aw);
        } else {
            rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
            rr.add(rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
        }
        x4[t] = xv;
        r4[t] = rv;
    }
    KSum v[2] = {rr, rz};
    double tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->iter += 1;
        s->rr = tot[0];
        if (!isfinite(tot[0]) || !isfinite(tot[1])) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (tot[0] <= s->tol2 * s->bb) { s->done = 1; s->status = FS_OK; }
        else if (s->iter >= s->maxit) { s->done = 1; s->status = FS_ENOCONV; }
        else if (JAC) {
            s->beta = tot[1] / s->rz;
            s->rz = tot[1];
        }
    }
}

// r.z for a stored z (MIC(0) / learned): beta = rz_new / rz (first: beta = 0).
__global__ void __launch_bounds__(TH) k_rz(const float *__restrict__ r, const float *__restrict__ z, int n4,
                                           int first, SolveScal *s, double *partials)
{
    if (s->done) return;
    KSum acc;
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
    const float4 *z4 = reinterpret_cast<const float4 *>(z);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 a = __ldg(r4 + t), b = __ldg(z4 + t);
        acc.add(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w);
    }
    KSum v[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        if (!isfinite(tot[0])) { s->done = 1; s->status = FS_ENONFINITE; return; }
        s->beta = first ? 0.0 : tot[0] / s->rz;
        s->rz = tot[0];
    }
}

__device__ __forceinline__ void init_scalars(SolveScal *s, double bb, double rr, double rz, double tol2,
                                             int maxit)
{
    s->bb = bb;
    s->rr = rr;
    s->rz = rz;
    s->tol2 = tol2;
    s->alpha = 0.0;
    s->beta = 0.0;
    s->pq = 0.0;
    s->iter = 0;
    s->maxit = maxit;
    s->status = FS_OK;
    s->done = 0;
    if (!isfinite(bb) || !isfinite(rr)) { s->done = 1; s->status = FS_ENONFINITE; }
    else if (bb == 0.0 || rr <= tol2 * bb) s->done = 1;
}

// Pressure start: x = 0, r = b, both p buffers 0.
template <bool JAC>
__global__ void __launch_bounds__(TH) k_pois_init(const float *__restrict__ b, float *__restrict__ x,
                                                  float *__restrict__ r, float *__restrict__ p0,
                                                  float *__restrict__ p1, const uint8_t *__restrict__ fl,
                                                  int n4, double tol2, int maxit, SolveScal *s,
                                                  double *partials)
{
    KSum bb, rz;
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    const uchar4 *f4 = reinterpret_cast<const uchar4 *>(fl);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 v = __ldg(b4 + t);
        reinterpret_cast<float4 *>(x)[t] = zero;
        reinterpret_cast<float4 *>(p0)[t] = zero;
        reinterpret_cast<float4 *>(p1)[t] = zero;
        bb.add(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
        if (JAC) {
            // Jacobi keeps the scaled residual z = D^-1 r
            const uchar4 fv = f4[t];
            const float4 z = make_float4(v.x * inv_diag<PoisOp>(fv.x, 0.f), v.y * inv_diag<PoisOp>(fv.y, 0.f),
                                         v.z * inv_diag<PoisOp>(fv.z, 0.f), v.w * inv_diag<PoisOp>(fv.w, 0.f));
            reinterpret_cast<float4 *>(r)[t] = z;
            rz.add(v.x * z.x + v.y * z.y + v.z * z.z + v.w * z.w);
        } else {
            reinterpret_cast<float4 *>(r)[t] = v;
        }
    }
    KSum v[2] = {bb, rz};
    double tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0)
        init_scalars(s, tot[0], tot[0], tot[1], tol2, maxit);
}

// Viscosity start from the guess x (fluid faces): rhs = x + cc * dsum (forward,
// Dirichlet values) or rhs = x (adjoint); r = rhs - A x. Jacobi (JAC) keeps the
// scaled residual D^-1 r and forms r.z here; otherwise r itself is stored and r.z
// comes after the preconditioner.
template <bool JAC>
__global__ void __launch_bounds__(TH) k_helm_init(const float *__restrict__ x, const float *__restrict__ dsum,
                                                  float *__restrict__ r, float *__restrict__ p0,
                                                  float *__restrict__ p1, const uint8_t *__restrict__ fl,
                                                  int n, int P, int PL, float cc, double tol2, int maxit,
                                                  SolveScal *s, double *partials)
{
    KSum bb, rr, rz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = fl[t];
        float rv = 0.f;
        if (f & FF_FLUID) {
            const float xc = x[t];
            const float rhs = dsum ? xc + cc * dsum[t] : xc;
            const float nb = (x[t - 1] + x[t + 1]) + (x[t - P] + x[t + P]) + (x[t - PL] + x[t + PL]);
            const float ax = HelmOp::diag(f, cc) * xc - cc * nb;
            rv = rhs - ax;
            bb.add(rhs * rhs);
            rr.add(rv * rv);
            rz.add(rv * rv * inv_diag<HelmOp>(f, cc));
        }
        r[t] = JAC ? rv * inv_diag<HelmOp>(f, cc) : rv;
        p0[t] = 0.f;
        p1[t] = 0.f;
    }
    KSum v[3] = {bb, rr, rz};
    double tot[3];
    if (grid_reduce<3>(v, partials, &s->ticket, tot) && threadIdx.x == 0)
        init_scalars(s, tot[0], tot[1], tot[2], tol2, maxit);
}

// A running sum carried as hi + lo + rest: each term enters by TwoSum into hi,
// its error by TwoSum into lo, and that error into rest (cascaded summation, as
// accurate as about three times the FP32 precision).
struct Sum3 {
    float hi = 0.f, lo = 0.f, rest = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float e1, e2;
        hi = two_sum(hi, v, e1);
        lo = two_sum(lo, e1, e2);
        rest += e2;
    }
};

// A compensated sum of non-negligible terms given as pairs (h, l): h by TwoSum
// into s, the errors and l into c.
struct Sum2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float h, float l)
    {
        float e;
        s = two_sum(s, h, e);
        c += e + l;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// |b - A x|^2 over the liquid -> s->aux[0] and |b|^2 -> s->aux[1], the final
// convergence check, to FP64 accuracy without FP64 arithmetic per element (this
// GPU runs FP64 at a small fraction of its FP32 rate). The residual of the FP32
// iterate, e = b - d x + sum of the six neighbours, is summed from its eight
// exact terms (d x as a product and its FMA error) by cascaded error-free sums
// (Sum3), so it is known to about 2^-70 of the terms' size, where FP64 would
// round at 2^-53; it is then held as a pair e_hi + e_lo (48 significant bits of
// e itself), squared as a pair (the product and its FMA error), and e^2, e and
// b^2 are summed per thread in compensated pairs (Sum2), converted to FP64 and
// merged in FP64 across the grid. For a singular operator (liquid touching no
// air) the component along the null vector (the constant), which no iterate can
// change, is left out: sum e^2 - (sum e)^2 / N. With r_out, the residual is also
// stored, rounded once to FP32, on the liquid (zero elsewhere, guard planes
// included): the right-hand side of a refinement step. r_out may alias b: every
// thread reads b only at the element it writes.
__global__ void __launch_bounds__(TH) k_pois_true_res(const float *b, const float *__restrict__ x,
                                                      const uint8_t *__restrict__ fl, int n, int P, int PL,
                                                      int singular, SolveScal *s, double *partials, float *r_out)
{
    Sum2 acc, sum, bsq;
    int cnt = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = fl[t];
        if (!(f & CF_LIQ)) {
            if (r_out) r_out[t] = 0.f;
            continue;
        }
        const float d = PoisOp::diag(f, 0.f), xc = x[t], bv = b[t];
        const float dx = d * xc, dxe = fmaf(d, xc, -dx);  // d x = dx + dxe exactly
        Sum3 r;
        r.add(bv);
        r.add(-dx);
        r.add(-dxe);
        r.add(x[t - 1]);
        r.add(x[t + 1]);
        r.add(x[t - P]);
        r.add(x[t + P]);
        r.add(x[t - PL]);
        r.add(x[t + PL]);
        float el;
        const float eh = two_sum(r.hi, r.lo, el);
        el += r.rest;  // e = eh + el
        if (r_out) r_out[t] = eh + el;
        const float sq = eh * eh;
        acc.add(sq, fmaf(eh, eh, -sq) + 2.f * eh * el);
        sum.add(eh, el);
        const float bb = bv * bv;
        bsq.add(bb, fmaf(bv, bv, -bb));
        cnt += 1;
    }
    double v[4] = {acc.value(), sum.value(), (double)cnt, bsq.value()}, tot[4];
    if (grid_reduce<4>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->aux[0] = (singular && tot[2] > 0.0) ? fmax(0.0, tot[0] - tot[1] * tot[1] / tot[2]) : tot[0];
        s->aux[1] = tot[3];
    }
}

// res = r - A e on the liquid, zero elsewhere (guard planes included); e is zero
// off the liquid
__global__ void __launch_bounds__(TH) k_pois_resid(const float *__restrict__ r, const float *__restrict__ e,
                                                   const uint8_t *__restrict__ fl, int n, int P, int PL, float *res)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = fl[t];
        float v = 0.f;
        if (f & CF_LIQ) {
            const float nb = (e[t - 1] + e[t + 1]) + (e[t - P] + e[t + P]) + (e[t - PL] + e[t + PL]);
            v = r[t] - (PoisOp::diag(f, 0.f) * e[t] - nb);
        }
        res[t] = v;
    }
}

// a += b over n elements (n a multiple of 4)
__global__ void __launch_bounds__(TH) k_add4(float *a, const float *__restrict__ b, int n4)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        float4 u = reinterpret_cast<float4 *>(a)[t];
        const float4 v = __ldg(reinterpret_cast<const float4 *>(b) + t);
        u.x += v.x;
        u.y += v.y;
        u.z += v.z;
        u.w += v.w;
        reinterpret_cast<float4 *>(a)[t] = u;
    }
}

// out = a + b over n elements (n a multiple of 4)
__global__ void __launch_bounds__(TH) k_sum4(float *out, const float *__restrict__ a, const float *__restrict__ b,
                                             int n4)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        const float4 u = __ldg(reinterpret_cast<const float4 *>(a) + t);
        const float4 v = __ldg(reinterpret_cast<const float4 *>(b) + t);
        reinterpret_cast<float4 *>(out)[t] = make_float4(u.x + v.x, u.y + v.y, u.z + v.z, u.w + v.w);
    }
}

// Residual replacement: restart CG from the current x with the true residual
// r = b - A x (Jacobi: stored as z = D^-1 r), both p buffers zero; r.r (and
// for Jacobi r.z) recomputed, the iteration count kept.
template <bool JAC>
__global__ void __launch_bounds__(TH) k_pois_restart(const float *__restrict__ b, const float *__restrict__ x,
                                                     float *__restrict__ r, float *__restrict__ p0,
                                                     float *__restrict__ p1, const uint8_t *__restrict__ fl, int n,
                                                     int P, int PL, SolveScal *s, double *partials)
{
    KSum rr, rz;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint8_t f = fl[t];
        float v = 0.f;
        if (f & CF_LIQ) {
            const float nb = (x[t - 1] + x[t + 1]) + (x[t - P] + x[t + P]) + (x[t - PL] + x[t + PL]);
            const float res = b[t] - (PoisOp::diag(f, 0.f) * x[t] - nb);
            v = JAC ? res * inv_diag<PoisOp>(f, 0.f) : res;
            rr.add(res * res);
            rz.add(res * v);
        }
        r[t] = v;
        p0[t] = 0.f;
        p1[t] = 0.f;
    }
    KSum v[2] = {rr, rz};
    double tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->rr = tot[0];
        s->rz = tot[1];
        s->alpha = 0.0;
        s->beta = 0.0;
        s->pq = 0.0;
        s->status = FS_OK;
        s->done = 0;
        if (!isfinite(tot[0])) { s->done = 1; s->status = FS_ENONFINITE; }
        else if (tot[0] <= s->tol2 * s->bb) s->done = 1;
    }
}

// Sum and count of a cell vector over the liquid -> s->aux[0], s->aux[1].
__global__ void __launch_bounds__(TH) k_liquid_sum(const float *__restrict__ x, const uint8_t *__restrict__ fl,
                                                   int n, SolveScal *s, double *partials)
{
    double a = 0.0, c = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        if (fl[t] & CF_LIQ) { a += x[t]; c += 1.0; }
    double v[2] = {a, c}, tot[2];
    if (grid_reduce<2>(v, partials, &s->ticket, tot) && threadIdx.x == 0) {
        s->aux[0] = tot[0];
        s->aux[1] = tot[1];
    }
}

__global__ void k_sub_liquid_mean(float *x, const uint8_t *__restrict__ fl, int n, const SolveScal *s)
{
    const float mean = s->aux[1] > 0.0 ? (float)(s->aux[0] / s->aux[1]) : 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        if (fl[t] & CF_LIQ) x[t] -= mean;
}

// b = -dx * div(u) on liquid cells (cell space), u a public-layout field.
__global__ void __launch_bounds__(TH) k_divergence(CF3 u, float *__restrict__ b, const uint8_t *__restrict__ cf,
                                                   Layout L, float dx)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
        const int t = L.PL + idx;
        float v = 0.f;
        if (cf[t] & CF_LIQ) {
            const float div = (__ldg(u.c[0] + idx + 1) - __ldg(u.c[0] + idx)) +
                              (__ldg(u.c[1] + idx + L.P) - __ldg(u.c[1] + idx)) +
                              (__ldg(u.c[2] + idx + L.PL) - __ldg(u.c[2] + idx));
            v = -dx * div;
        }
        b[t] = v;
    }
}

// out = in - grad q / dx on fluid faces, in elsewhere, 0 in padding; the
// y = 3 slice copies q to q_out (public layout). After a refined solve the
// pressure is the pair q + q2 (q2 nullable), whose differences are taken term
// by term, so it is never rounded to one FP32 value on the way to the velocity.
__global__ void __launch_bounds__(TH) k_grad_subtract(CF3 in, F3 out, const float *__restrict__ q,
                                                      const float *__restrict__ q2, float *q_out,
                                                      const uint8_t *__restrict__ ff, Layout L, float inv_dx)
{
    const int c = blockIdx.y;
    if (c == 3) {
        if (!q_out) return;
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x)
            q_out[idx] = q2 ? q[L.PL + idx] + q2[L.PL + idx] : q[L.PL + idx];
        return;
    }
    const int off = c == 0 ? 1 : (c == 1 ? L.P : L.PL);
    const uint8_t *fc = ff + L.face_origin(c);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
        const uint8_t f = fc[idx];
        float v = 0.f;
        if (f) {
            v = in.c[c][idx];
            if (f & FF_FLUID) {
                float dq = q[L.PL + idx] - q[L.PL + idx - off];
                if (q2) dq += q2[L.PL + idx] - q2[L.PL + idx - off];
                v -= dq * inv_dx;
            }
        }
        out.c[c][idx] = v;
    }
}

// Full field from the viscosity solution: fluid faces from face space, fixed
// faces their prescribed values, zero elsewhere.
__global__ void __launch_bounds__(TH) k_compose(const float *__restrict__ vx, const float *__restrict__ bc,
                                                const uint8_t *__restrict__ ff, F3 out, Layout L)
{
    const int c = blockIdx.y;
    const int o = L.face_origin(c);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
        const uint8_t f = ff[o + idx];
        out.c[c][idx] = (f & FF_FLUID) ? vx[o + idx] : ((f & FF_FIXED) ? bc[o + idx] : 0.f);
    }
}

__global__ void __launch_bounds__(TH) k_mask_fluid(CF3 in, F3 out, const uint8_t *__restrict__ ff, Layout L)
{
    const int c = blockIdx.y;
    const int o = L.face_origin(c);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x)
        out.c[c][idx] = (ff[o + idx] & FF_FLUID) ? in.c[c][idx] : 0.f;
}

__global__ void __launch_bounds__(TH) k_to_face_space(CF3 in, float *__restrict__ vx,
                                                      const uint8_t *__restrict__ ff, Layout L)
{
    const int c = blockIdx.y;
    const int o = L.face_origin(c);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x)
        vx[o + idx] = (ff[o + idx] & FF_FLUID) ? in.c[c][idx] : 0.f;
}

// <x, L~ uv> over fluid faces, L~ u = n_f u_f - sum of fluid/fixed neighbours
// (the 1/dx^2 is applied by the host) -> s->aux[0].
__global__ void __launch_bounds__(TH) k_nu_grad(const float *__restrict__ vx, CF3 uv,
                                                const uint8_t *__restrict__ ff, Layout L, SolveScal *s,
                                                double *partials)
{
    KSum acc;
    const int off[6] = {-1, 1, -L.P, L.P, -L.PL, L.PL};
    for (int c = 0; c < 3; c++) {
        const int o = L.face_origin(c);
        const float *u = uv.c[c];
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
            const uint8_t f = ff[o + idx];
            if (!(f & FF_FLUID)) continue;
            float nb = 0.f;
#pragma unroll
            for (int m = 0; m < 6; m++)
                if (ff[o + idx + off[m]] & (FF_FLUID | FF_FIXED)) nb += u[idx + off[m]];
            const float lu = (float)(f & FF_N) * u[idx] - nb;
            acc.add(vx[o + idx] * lu);
        }
    }
    KSum v[1] = {acc};
    double tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) s->aux[0] = tot[0];
}

// Cosine term of the loss on band cells: writes the per-cell gradient w.r.t.
// the cell-centred velocity (scaled by -alpha/|Bc|) and sums 1 - cos.
__global__ void __launch_bounds__(TH) k_loss_cell(CF3 u, CF3 tg, const uint8_t *__restrict__ cf, uint8_t bandbit,
                                                  F3 gc, Layout L, float scale, SolveScal *s,
                                                  double *partials)
{
    double acc = 0.0;
    const float eps2 = 1e-16f;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
        const int t = L.PL + idx;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (cf[t] & bandbit) {
            const float a0 = 0.5f * (u.c[0][idx] + u.c[0][idx + 1]);
            const float a1 = 0.5f * (u.c[1][idx] + u.c[1][idx + L.P]);
            const float a2 = 0.5f * (u.c[2][idx] + u.c[2][idx + L.PL]);
            const float b0 = 0.5f * (tg.c[0][idx] + tg.c[0][idx + 1]);
            const float b1 = 0.5f * (tg.c[1][idx] + tg.c[1][idx + L.P]);
            const float b2 = 0.5f * (tg.c[2][idx] + tg.c[2][idx + L.PL]);
            const float ab = a0 * b0 + a1 * b1 + a2 * b2;
            const float na = sqrtf(a0 * a0 + a1 * a1 + a2 * a2 + eps2);
            const float nbv = sqrtf(b0 * b0 + b1 * b1 + b2 * b2 + eps2);
            const float inv = 1.f / (na * nbv);
            const float cs = ab * inv;
            acc += 1.0 - (double)cs;
            const float k2 = cs / (na * na);
            g0 = -scale * (b0 * inv - k2 * a0);
            g1 = -scale * (b1 * inv - k2 * a1);
            g2 = -scale * (b2 * inv - k2 * a2);
        }
        gc.c[0][t] = g0;
        gc.c[1][t] = g1;
        gc.c[2][t] = g2;
    }
    double v[1] = {acc}, tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) s->aux[1] = tot[0];
}

// L2 term on band faces plus the gather of the cosine gradient onto faces:
// g += beta (u - t)/|B| on band faces + (gc(L) + gc(R))/2 on every face.
__global__ void __launch_bounds__(TH) k_loss_face(CF3 u, CF3 tg, const uint8_t *__restrict__ cf,
                                                  const uint8_t *__restrict__ ff, uint8_t bandbit, CF3 gc,
                                                  int use_gc, F3 g, Layout L, float beta_over_B,
                                                  SolveScal *s, double *partials)
{
    double acc = 0.0;
    for (int c = 0; c < 3; c++) {
        const int o = L.face_origin(c);
        const int off = c == 0 ? 1 : (c == 1 ? L.P : L.PL);
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
            const uint8_t f = ff[o + idx];
            if (!f) continue;
            float gv = 0.f;
            const uint8_t fr = cf[L.PL + idx], fl = cf[L.PL + idx - off];
            if ((f & FF_FLUID) && ((fr | fl) & bandbit)) {
                const float e = u.c[c][idx] - tg.c[c][idx];
                acc += 0.5 * (double)e * (double)e;
                gv += beta_over_B * e;
            }
            if (use_gc) gv += 0.5f * (gc.c[c][L.PL + idx] + gc.c[c][L.PL + idx - off]);
            if (g.c[0] && gv != 0.f) g.c[c][idx] += gv;
        }
    }
    double v[1] = {acc}, tot[1];
    if (grid_reduce<1>(v, partials, &s->ticket, tot) && threadIdx.x == 0) s->aux[0] = tot[0];
}

}  // namespace
}  // namespace fs

#include "fs_stencil.cuh"
#include "fs_tma.cuh"

namespace fs {

// Persistent grid sizes of the two CG kernels for one operator.
template <class Op>
struct TmaGrids {
    int spmv, upd;
    TmaGrids(const fs_ctx *c, int nitems, int nact)
    {
        static const int rs = resident_blocks((const void *)k_spmv_z<Op>, zmarch_smem());
        static const int ru = resident_blocks((const void *)k_update_q<Op, true>, 0);
        static const int ru2 = resident_blocks((const void *)k_update_q<Op, false>, 0);
        spmv = std::max(1, std::min(nitems, c->num_sms * rs));
        upd = std::max(1, std::min(nact, c->num_sms * std::min(ru, ru2)));
    }
};

// Iterations launched before each read of the convergence flag. A read costs a
// host round trip with the GPU idle, and every iteration launched after
// convergence costs its launches (each returns at once). With the count of the
// last pass of the same kind known, the first batch runs one fewer than it and
// later batches two at a time; otherwise `check` at a time.
struct CgBatches {
    int first, later;
    CgBatches(int last, int check, long long maxit)
    {
        const long long f = std::min<long long>((long long)last - 1, maxit);
        first = last > 1 ? (int)std::max<long long>(f, 1) : check;
        later = last > 1 ? std::min(check, 2) : check;
    }
    int size(long long launched) const { return launched == 0 ? first : later; }
};

int zmarch_slots(const fs_ctx *c, bool face)
{
    const int r = face ? resident_blocks((const void *)k_spmv_z<HelmOp>, zmarch_smem())
                       : resident_blocks((const void *)k_spmv_z<PoisOp>, zmarch_smem());
    return c->num_sms * r;
}

// A bounded wait of a TMA-fed kernel or of the MIC(0) wavefront that ran out
// leaves a bit in the error word.
int check_wait_error(fs_ctx *c, const char *what)
{
    unsigned herr = 0;
    FS_CUDA(cudaMemcpyAsync(&herr, c->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    if (herr & 1u) {
        c->mic_ready = 0;  // the factor may be incomplete: refactor on the next use
        return set_error(FS_ETIMEOUT, "MIC(0) sweep: a wait on a predecessor tile ran out (spin_limit %d)",
                         c->prm.spin_limit);
    }
    if (herr & ERR_TMA) return set_error(FS_ETIMEOUT, "%s: a wait for a tensor copy ran out", what);
    if (herr & 8u)  // the bit of the tensor-core network layer
        return set_error(FS_ETIMEOUT, "%s: a wait for the network's tensor-core MMAs ran out", what);
    return FS_OK;
}

int read_scal(fs_ctx *c, int which, SolveScal *out)
{
    FS_CUDA(cudaMemcpyAsync(c->scal_host + which, c->scal + which, sizeof(SolveScal), cudaMemcpyDeviceToHost,
                            c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    *out = c->scal_host[which];
    return FS_OK;
}

static int finish_status(int st)
{
    return st == FS_OK ? FS_OK : st;
}

int launch_divergence(fs_ctx *c, CF3 u)
{
    const Layout &L = c->L;
    k_divergence<<<grid_blocks(c, L.S, TH), TH, 0, c->stream>>>(u, c->pb, c->cflag, L, (float)c->prm.dx);
    if (c->singular) {
        // the right-hand side must lie in the range of the singular operator
        k_liquid_sum<<<grid_blocks(c, L.nC, TH), TH, 0, c->stream>>>(c->pb, c->cflag, L.nC, c->scal + 2,
                                                                     c->partials);
        k_sub_liquid_mean<<<grid_blocks(c, L.nC, TH), TH, 0, c->stream>>>(c->pb, c->cflag, L.nC, c->scal + 2);
        c->n_launches += 2;
    }
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

// When the pressure operator is singular (liquid touching no air), the
// preconditioned residual is made mean-free over the liquid, so every search
// direction stays in the range of the operator (the preconditioner becomes
// P M^-1 P with P the mean-removing projector, still SPD on that range).
int remove_null_mode(fs_ctx *c, float *z)
{
    if (!c->singular) return FS_OK;
    const Layout &L = c->L;
    const int bs = grid_blocks(c, L.nC, TH);
    k_liquid_sum<<<bs, TH, 0, c->stream>>>(z, c->cflag, L.nC, c->scal + 3, c->partials);
    k_sub_liquid_mean<<<bs, TH, 0, c->stream>>>(z, c->cflag, L.nC, c->scal + 3);
    c->n_launches += 2;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

// The learned preconditioner of flexible CG: the network alone
// (FS_PRECOND_LEARNED), or the network followed by one V-cycle on the residual it
// leaves (FS_PRECOND_LEARNED_MG): z = e + M(r - A e), e = s Net(r/s). The network
// smooths, the V-cycle corrects the error it cannot reach. pp[0] and pp[1] are
// free while flexible CG runs (it keeps its directions in its own ring).
int learned_apply(fs_ctx *c, const float *r, float *z, const int *done)
{
    if (c->prm.precond != FS_PRECOND_LEARNED_MG) return net_apply(c, r, z);
    const Layout &L = c->L;
    float *e = c->pp[0], *res = c->pp[1];
    if (int rc = net_apply(c, r, e)) return rc;
    k_pois_resid<<<grid_blocks(c, L.nC, TH), TH, 0, c->stream>>>(r, e, c->cflag, L.nC, L.P, L.PL, res);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    if (int rc = mg_apply(c, res, z, done)) return rc;
    k_add4<<<grid_blocks(c, L.nC / 4, TH), TH, 0, c->stream>>>(z, e, L.nC / 4);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

static int pressure_tail(fs_ctx *c, const SolveScal &h, long long iters, double bb0, const SolveScal *known,
                         fs_stats *st);

// Warm start (fs_params.warm_start): after the x = 0 initialisation, start
// instead from the last converged pressure of the same kind of projection when
// its residual is below half of |b|^2; r = b - A x, p = 0, iteration count 0.
static int try_warm_start(fs_ctx *c, bool jac)
{
    const int k = c->solve_kind;
    if (!c->prm.warm_start || !c->pw_valid[k] || !c->pw[k]) return FS_OK;
    const Layout &L = c->L;
    const int bs = grid_blocks(c, L.nC, TH);
    k_pois_true_res<<<bs, TH, 0, c->stream>>>(c->pb, c->pw[k], c->cflag, L.nC, L.P, L.PL, c->singular,
                                              c->scal + 2, c->partials, nullptr);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    SolveScal m, h0;
    int rc;
    if ((rc = read_scal(c, 2, &m)) || (rc = read_scal(c, 0, &h0))) return rc;
    if (h0.done || !(m.aux[0] < 0.5 * m.aux[1])) return FS_OK;
    FS_CUDA(cudaMemcpyAsync(c->px, c->pw[k], (size_t)L.nC * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    if (jac)
        k_pois_restart<true><<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->pr, c->pp[0], c->pp[1], c->cflag, L.nC,
                                                       L.P, L.PL, c->scal + 0, c->partials);
    else
        k_pois_restart<false><<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->pr, c->pp[0], c->pp[1], c->cflag, L.nC,
                                                        L.P, L.PL, c->scal + 0, c->partials);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

// Keep the converged pressure for the next warm start of this kind.
static int save_warm_start(fs_ctx *c)
{
    const int k = c->solve_kind;
    if (!c->prm.warm_start) return FS_OK;
    const size_t bytes = (size_t)c->L.nC * sizeof(float);
    if (!c->pw[k]) {
        if (cudaMalloc(&c->pw[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            c->pw[k] = nullptr;
            return FS_OK;  // no warm start then; not an error of the solve
        }
    }
    if (c->q_head) {
        const int n4 = c->L.nC / 4;
        k_sum4<<<grid_blocks(c, n4, TH), TH, 0, c->stream>>>(c->pw[k], c->q_head, c->px, n4);
        c->n_launches += 1;
        FS_CUDA(cudaGetLastError());
    } else {
        FS_CUDA(cudaMemcpyAsync(c->pw[k], c->px, bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    c->pw_valid[k] = 1;
    return FS_OK;
}

// r = b - A x in pr (unscaled) for a warm restart of flexible CG.
int pressure_restart(fs_ctx *c)
{
    const Layout &L = c->L;
    k_pois_restart<false><<<grid_blocks(c, L.nC, TH), TH, 0, c->stream>>>(
        c->pb, c->px, c->pr, c->pp[0], c->pp[1], c->cflag, L.nC, L.P, L.PL, c->scal + 0, c->partials);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

// Jacobi-, MIC(0)- or multigrid-PCG on pb -> px from x = 0 (or from the last
// converged pressure, with fs_params.warm_start). Final scalars in h.
static int pcg_iterate(fs_ctx *c, SolveScal &h)
{
    const Layout &L = c->L;
    SolveScal *s = c->scal + 0;
    const bool jac = c->prm.precond == FS_PRECOND_JACOBI;
    const int n4 = L.nC / 4;
    const double tol2 = c->prm.tol_p * c->prm.tol_p * (c->tol2_scale > 0.0 ? c->tol2_scale : 1.0);
    // z = M r for MIC(0) or the multigrid V-cycle (the stored-z preconditioners)
    auto apply_m = [&]() -> int {
        return c->prm.precond == FS_PRECOND_MG ? mg_apply(c, c->pr, c->pz, &s->done) : mic0_apply(c, c->pr, c->pz);
    };
    // r.z: over the V-cycle's active quads with multigrid, else a dense pass
    auto rz = [&](int first) {
        if (!(c->prm.precond == FS_PRECOND_MG && mg_rz(c, false, c->pr, c->pz, first, s)))
            k_rz<<<grid_blocks(c, n4, TH), TH, 0, c->stream>>>(c->pr, c->pz, n4, first, s, c->partials);
        c->n_launches += 1;
    };
    // z = M r and r.z: with multigrid (and no null mode to remove from z) r.z is
    // formed in the V-cycle's last sweep
    auto precondition = [&](int first) -> int {
        int rc = FS_OK;
        if (c->prm.precond == FS_PRECOND_MG && !c->singular) {
            if (mg_apply_rz(c, c->pr, c->pz, &s->done, s, first, rc) || rc) return rc;
        } else {
            if ((rc = apply_m())) return rc;
            if ((rc = remove_null_mode(c, c->pz))) return rc;
        }
        rz(first);
        return FS_OK;
    };
    if (jac)
        k_pois_init<true><<<grid_blocks(c, n4, TH), TH, 0, c->stream>>>(
            c->pb, c->px, c->pr, c->pp[0], c->pp[1], c->cflag, n4, tol2, c->prm.maxit_p, s, c->partials);
    else
        k_pois_init<false><<<grid_blocks(c, n4, TH), TH, 0, c->stream>>>(
            c->pb, c->px, c->pr, c->pp[0], c->pp[1], c->cflag, n4, tol2, c->prm.maxit_p, s, c->partials);
    if (!c->refining)
        if (int rc = try_warm_start(c, jac)) return rc;
    if (!jac)
        if (int rc = precondition(1)) return rc;
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    const int bs = grid_blocks(c, L.nC, TH);
    const int b4 = grid_blocks(c, n4, TH);
    int cur = 0;
    long long launched = 0;
    double by_spmv = (double)L.nC + 16.0 * (double)c->n_liquid;
    const double by_upd = (double)L.nC + 24.0 * (double)c->n_liquid;
    const bool tiled = c->act_cell != nullptr;
    // with multigrid, the operator apply walks the V-cycle's lists of active quads
    QuadLists qls{};
    qls.nv = 1;
    const bool listed = c->prm.precond == FS_PRECOND_MG && mg_level0_lists(c, false, qls.ql, qls.n, qls.base);
    const long long nlisted = listed ? qls.n[0] : 0;
    static const int rl = resident_blocks((const void *)k_spmv_list<PoisOp>, 0);  // one wave of the list apply
    if (listed) by_spmv = 8.0 * (double)nlisted + 16.0 * (double)c->n_liquid;  // list entry and flags per quad
    const TileMap &tm = c->tm_cell;
    const dim3 tdim(TILE_X / 4, TILE_Y);
    const TmaGrids<PoisOp> tg(c, c->nitems_cell, c->nact_cell);
    // a multigrid iteration costs several operator applies: check convergence more often
    const int check = c->prm.precond == FS_PRECOND_MG ? std::min(c->prm.check_every, 4) : c->prm.check_every;
    int &last = c->it_last_p[c->solve_kind & 1][c->refining ? 1 : 0];
    const CgBatches batches(last, check, c->prm.maxit_p);
    for (;;) {
        const int nb = batches.size(launched);
        for (int b = 0; b < nb; b++) {
            const bool samp = c->prof_on && ((launched + b) % c->prof_period) == 0;  // every prof_period-th
            cudaEvent_t e0 = samp ? prof_mark(c) : nullptr;
            const float *zsrc = jac ? c->pr : c->pz;
            if (listed)
                k_spmv_list<PoisOp><<<wave_blocks(c, nlisted, rl), TH, 0, c->stream>>>(
                    qls, c->pz, c->pp[cur], c->pp[cur ^ 1], c->pq, c->cflag, L.P, L.PL, 0.f, s, c->partials);
            else if (tiled)
                k_spmv_z<PoisOp><<<tg.spmv, tdim, zmarch_smem(), c->stream>>>(
                    jac ? c->tmz_pr : c->tmz_pz, c->tmz_pp[cur], c->pp[cur ^ 1], c->pq, c->cflag, c->items_cell,
                    c->nitems_cell, tm, 0.f, s, c->partials, c->err_word);
            else
                k_spmv<PoisOp><<<bs, TH, 0, c->stream>>>(zsrc, c->pp[cur], c->pp[cur ^ 1], c->pq, c->cflag, L.nC,
                                                         L.P, L.PL, 0.f, s, c->partials);
            cudaEvent_t e1 = samp ? prof_mark(c) : nullptr, e2 = samp ? prof_mark(c) : nullptr;
            if (tiled) {
                if (jac)
                    k_update_q<PoisOp, true><<<tg.upd, tdim, 0, c->stream>>>(
                        c->px, c->pr, c->pp[cur ^ 1], c->pq, c->cflag, c->list_cell, c->qmask_cell, c->nact_cell, tm,
                        0.f, s, c->partials);
                else
                    k_update_q<PoisOp, false><<<tg.upd, tdim, 0, c->stream>>>(
                        c->px, c->pr, c->pp[cur ^ 1], c->pq, c->cflag, c->list_cell, c->qmask_cell, c->nact_cell, tm,
                        0.f, s, c->partials);
            } else if (jac)
                k_update<PoisOp, true><<<b4, TH, 0, c->stream>>>(c->px, c->pr, c->pp[cur ^ 1], c->pq, c->cflag,
                                                                 n4, 0.f, s, c->partials);
            else
                k_update<PoisOp, false><<<b4, TH, 0, c->stream>>>(c->px, c->pr, c->pp[cur ^ 1], c->pq, c->cflag,
                                                                  n4, 0.f, s, c->partials);
            cudaEvent_t e3 = samp ? prof_mark(c) : nullptr;
            prof_add(c, K_P_SPMV, e0, e1, by_spmv);
            prof_add(c, K_P_UPDATE, e2, e3, by_upd);
            c->n_launches += 2;
            if (!jac)
                if (int rc = precondition(0)) return rc;
            cur ^= 1;
        }
        launched += nb;
        FS_CUDA(cudaGetLastError());
        int rc = read_scal(c, 0, &h);
        if (rc) return rc;
        if (h.done) break;
        if (launched > (long long)c->prm.maxit_p + c->prm.check_every)
            return set_error(FS_ECUDA, "pressure solve: iteration flag never set");
    }
    last = h.status == FS_OK ? (int)std::min<long long>(h.iter, 1 << 20) : 0;
    prof_count(c, K_P_SPMV, h.iter);
    prof_count(c, K_P_UPDATE, h.iter);
    if (c->prm.precond == FS_PRECOND_MG) mg_count(c, h.iter, false);
    return check_wait_error(c, "pressure solve");
}

// At most this many refinement steps per solve (one suffices unless CG itself
// stalled on the first pass).
constexpr int kMaxRefine = 2;

static int solve_pressure_once(fs_ctx *c, fs_stats *st)
{
    c->q_head = nullptr;
    if (c->prm.pressure_solver == FS_SOLVER_PERCNN) {
        // K recurrent sub-steps: no convergence test, the true residual is reported
        SolveScal h;
        int rc = solve_pressure_percnn(c, &h);
        if (rc) return rc;
        return pressure_tail(c, h, h.iter, 0.0, nullptr, st);
    }
    const bool learned = c->prm.precond == FS_PRECOND_LEARNED || c->prm.precond == FS_PRECOND_LEARNED_MG;
    if (learned && !net_loaded(c))
        return set_error(FS_ESTATE, "the learned preconditioner has no network loaded");
    FS_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(unsigned), c->stream));
    if (c->prm.precond == FS_PRECOND_MIC0 && !c->mic_ready) {
        int rc = mic0_factor(c);
        if (rc) return rc;
    }
    const Layout &L = c->L;
    const int bs = grid_blocks(c, L.nC, TH);
    // Mixed-precision iterative refinement. CG runs on FP32 vectors, so its
    // recursively updated residual drifts from b - A x, and the rounding of the
    // FP32 iterate alone leaves |b - A x| ~ 2e-7 |A x| |x| / |x|: with a smooth
    // right-hand side (|x| >> |b|) that is above the tolerance (7.9e-6 |b| on a
    // 256^3 blob). When the FP64-evaluated residual of x is above tol |b|, the
    // solve runs again on the correction system A d = b - A x, whose right-hand
    // side is that FP64 residual rounded once to FP32, to an absolute target of
    // tol |b| / 2. The pressure is then kept as the FP32 pair (x, d): the gradient
    // subtract and the warm start read both terms, so it is never rounded to a
    // single FP32 vector on the solver's path.
    float *const b0 = c->pb;
    SolveScal h, m;
    double bb0 = 0.0;
    long long iters = 0;
    bool checked = false;  // m holds the FP64 residual of the pass that ended the loop
    int rc = FS_OK, nref = 0;
    const int kind = c->solve_kind & 1;
    const double tol2 = c->prm.tol_p * c->prm.tol_p;
    // Where the first pass of the last solve of this kind left a true residual
    // above the tolerance, this one stops at half that residual: far above the
    // tolerance (the rounding floor of the FP32 iterate) the refinement runs
    // anyway and the iterations below the floor are saved; just above it (a
    // recursive residual that drifted) the deeper first pass often makes the
    // refinement unnecessary.
    if (c->p_floor2[kind] > tol2) c->tol2_scale = std::min(0.25 * c->p_floor2[kind] / tol2, 1e4);
    for (int pass = 0;; pass++) {
        checked = false;
        rc = learned ? solve_pressure_fcg(c, &h, false) : pcg_iterate(c, h);
        if (rc) break;
        iters += h.iter;
        if (h.status != FS_OK) break;
        // the check of this pass's system (b0 and x, then each correction's); its
        // residual, rounded once to FP32, is the next correction's right-hand side,
        // stored in pbr (in place from the second pass on)
        k_pois_true_res<<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->cflag, L.nC, L.P, L.PL, c->singular,
                                                  c->scal + 2, c->partials, c->pbr);
        c->n_launches += 1;
        if ((rc = check_cuda(cudaGetLastError(), "k_pois_true_res")) || (rc = read_scal(c, 2, &m))) break;
        checked = true;
        if (pass == 0) {
            bb0 = m.aux[1];
            c->p_floor2[kind] = bb0 > 0.0 && m.aux[0] > tol2 * bb0 ? m.aux[0] / bb0 : 0.0;
        }
        if (pass == kMaxRefine || !(bb0 > 0.0) || !(m.aux[0] > tol2 * bb0)) break;
        // the next correction: the terms solved so far kept in the head and the tail
        if (pass == 0) {
            if ((rc = check_cuda(cudaMemcpyAsync(c->pxh, c->px, (size_t)L.nC * sizeof(float),
                                                 cudaMemcpyDeviceToDevice, c->stream),
                                 "cudaMemcpyAsync")) ||
                (rc = remove_null_mode(c, c->pxh)))
                break;
            c->q_head = c->pxh;
            c->pb = c->pbr;
        } else if (pass == 1) {
            if ((rc = check_cuda(cudaMemcpyAsync(c->pxt, c->px, (size_t)L.nC * sizeof(float),
                                                 cudaMemcpyDeviceToDevice, c->stream),
                                 "cudaMemcpyAsync")))
                break;
        } else {
            k_add4<<<grid_blocks(c, L.nC / 4, TH), TH, 0, c->stream>>>(c->pxt, c->px, L.nC / 4);
            c->n_launches += 1;
        }
        if ((rc = remove_null_mode(c, c->pbr))) break;
        c->tol2_scale = 0.25 * bb0 / m.aux[0];
        c->refining = 1;
        nref += 1;
        if (st) st->restarts_p += 1;
    }
    c->refining = 0;
    c->tol2_scale = 1.0;
    if (rc) {
        c->pb = b0;
        return rc;
    }
    if (!checked) {  // a pass that did not converge: the residual of its own system
        k_pois_true_res<<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->cflag, L.nC, L.P, L.PL, c->singular,
                                                  c->scal + 2, c->partials, nullptr);
        c->n_launches += 1;
        if ((rc = check_cuda(cudaGetLastError(), "k_pois_true_res")) || (rc = read_scal(c, 2, &m))) {
            c->pb = b0;
            return rc;
        }
    }
    c->pb = b0;
    if (nref >= 2) {  // fold the earlier corrections into the tail
        k_add4<<<grid_blocks(c, L.nC / 4, TH), TH, 0, c->stream>>>(c->px, c->pxt, L.nC / 4);
        c->n_launches += 1;
    }
    rc = pressure_tail(c, h, iters, bb0, &m, st);
    if (rc == FS_OK) rc = save_warm_start(c);
    return rc;
}

// After the iterations: the true residual (FP64) of the system in pb and px, or
// the one the caller already has (`known`), relative to |b0|^2 when bb0 > 0 (the
// original right-hand side of a refined solve), else to |b|^2; the mean-free
// representative of a singular solve; the statistics.
static int pressure_tail(fs_ctx *c, const SolveScal &h, long long iters, double bb0, const SolveScal *known,
                         fs_stats *st)
{
    const Layout &L = c->L;
    const int bs = grid_blocks(c, L.nC, TH);
    if (!known) {
        k_pois_true_res<<<bs, TH, 0, c->stream>>>(c->pb, c->px, c->cflag, L.nC, L.P, L.PL, c->singular,
                                                  c->scal + 2, c->partials, nullptr);
        c->n_launches += 1;
    }
    if (c->singular) {  // the mean-free representative
        k_liquid_sum<<<bs, TH, 0, c->stream>>>(c->px, c->cflag, L.nC, c->scal + 3, c->partials);
        k_sub_liquid_mean<<<bs, TH, 0, c->stream>>>(c->px, c->cflag, L.nC, c->scal + 3);
        c->n_launches += 2;
    }
    FS_CUDA(cudaGetLastError());
    SolveScal m;
    if (known) {
        m = *known;
    } else {
        int rc = read_scal(c, 2, &m);
        if (rc) return rc;
    }
    const double bb = bb0 > 0.0 ? bb0 : m.aux[1];
    if (st) {
        st->iters_p += (int)iters;
        st->relres_p = bb > 0 ? std::sqrt(h.rr / bb) : 0.0;
        st->true_relres_p = bb > 0 ? std::sqrt(m.aux[0] / bb) : 0.0;
        if (h.status != FS_OK && st->status == FS_OK) st->status = h.status;
    }
    return finish_status(h.status);
}

// The learned preconditioner is judged by the true residual: if flexible CG with
// it does not reach the tolerance (or breaks down), the solve is redone from
// scratch with MIC(0)-PCG.
int solve_pressure(fs_ctx *c, fs_stats *st)
{
    int rc = solve_pressure_once(c, st);
    const int pc = c->prm.precond;
    if ((pc != FS_PRECOND_LEARNED && pc != FS_PRECOND_LEARNED_MG) || rc == FS_OK || rc == FS_ECUDA ||
        rc == FS_EINVAL || rc == FS_ESTATE || rc == FS_ETIMEOUT)
        return rc;
    c->prm.precond = FS_PRECOND_MIC0;
    if (st) {
        st->status = FS_OK;
        st->fallbacks += 1;
    }
    rc = solve_pressure_once(c, st);
    c->prm.precond = pc;
    return rc;
}

int solve_viscosity(fs_ctx *c, bool dirichlet, fs_stats *st)
{
    const Layout &L = c->L;
    SolveScal *s = c->scal + 1;
    const float cc = (float)(c->prm.nu * c->prm.dt / (c->prm.dx * c->prm.dx));
    const int n4 = L.nF / 4;
    const double tol2 = c->prm.tol_v * c->prm.tol_v;
    const int bs = grid_blocks(c, L.nF, TH);
    const int b4 = grid_blocks(c, n4, TH);
    FS_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(unsigned), c->stream));
    // the multigrid preconditioner serves both solves; otherwise Jacobi
    const bool mg = c->prm.precond == FS_PRECOND_MG || c->prm.precond == FS_PRECOND_LEARNED_MG;
    const float *dsum = (dirichlet && c->has_bc) ? c->dsum : nullptr;
    if (mg)
        k_helm_init<false><<<bs, TH, 0, c->stream>>>(c->vx, dsum, c->vr, c->vp[0], c->vp[1], c->fflag, L.nF, L.P, L.PL,
                                                     cc, tol2, c->prm.maxit_v, s, c->partials);
    else
        k_helm_init<true><<<bs, TH, 0, c->stream>>>(c->vx, dsum, c->vr, c->vp[0], c->vp[1], c->fflag, L.nF, L.P, L.PL,
                                                    cc, tol2, c->prm.maxit_v, s, c->partials);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    // z = M r and r.z (first: beta = 0)
    auto precondition = [&](int first) -> int {
        int rc = FS_OK;
        if (mg_apply_faces_rz(c, c->vr, c->vz, cc, &s->done, s, first, rc) || rc) return rc;  // r.z in the V-cycle
        if (!mg_rz(c, true, c->vr, c->vz, first, s))  // over the active quads, else a dense pass
            k_rz<<<b4, TH, 0, c->stream>>>(c->vr, c->vz, n4, first, s, c->partials);
        c->n_launches += 1;
        FS_CUDA(cudaGetLastError());
        return FS_OK;
    };
    if (mg)
        if (int rc = precondition(1)) return rc;
    // a multigrid iteration costs several operator applies: check convergence more often
    const int check = mg ? std::min(c->prm.check_every, 4) : c->prm.check_every;
    int cur = 0;
    long long launched = 0;
    SolveScal h;
    double by_spmv = (double)L.nF + 16.0 * (double)c->n_fluid;
    const double by_upd = (double)L.nF + 24.0 * (double)c->n_fluid;
    const bool tiled = c->act_face != nullptr;
    // with multigrid, the operator apply walks the V-cycles' lists of active quads
    QuadLists qls{};
    qls.nv = 3;
    const bool listed = mg && mg_level0_lists(c, true, qls.ql, qls.n, qls.base);
    const long long nlisted = listed ? (long long)qls.n[0] + qls.n[1] + qls.n[2] : 0;
    static const int rl = resident_blocks((const void *)k_spmv_list<HelmOp>, 0);  // one wave of the list apply
    if (listed) by_spmv = 8.0 * (double)nlisted + 16.0 * (double)c->n_fluid;  // list entry and flags per quad
    const TileMap &tm = c->tm_face;
    const dim3 tdim(TILE_X / 4, TILE_Y);
    const TmaGrids<HelmOp> tg(c, c->nitems_face, c->nact_face);
    int &last = c->it_last_v[dirichlet ? 1 : 0];
    const CgBatches batches(last, check, c->prm.maxit_v);
    for (;;) {
        const int nb = batches.size(launched);
        for (int b = 0; b < nb; b++) {
            const bool samp = c->prof_on && ((launched + b) % c->prof_period) == 0;  // every prof_period-th
            cudaEvent_t e0 = samp ? prof_mark(c) : nullptr;
            if (listed)
                k_spmv_list<HelmOp><<<wave_blocks(c, nlisted, rl), TH, 0, c->stream>>>(
                    qls, c->vz, c->vp[cur], c->vp[cur ^ 1], c->vq, c->fflag, L.P, L.PL, cc, s, c->partials);
            else if (tiled)
                k_spmv_z<HelmOp><<<tg.spmv, tdim, zmarch_smem(), c->stream>>>(
                    mg ? c->tmz_vz : c->tmz_vr, c->tmz_vp[cur], c->vp[cur ^ 1], c->vq, c->fflag, c->items_face,
                    c->nitems_face, tm, cc, s, c->partials, c->err_word);
            else
                k_spmv<HelmOp><<<bs, TH, 0, c->stream>>>(mg ? c->vz : c->vr, c->vp[cur], c->vp[cur ^ 1], c->vq,
                                                         c->fflag, L.nF, L.P, L.PL, cc, s, c->partials);
            cudaEvent_t e1 = samp ? prof_mark(c) : nullptr, e2 = samp ? prof_mark(c) : nullptr;
            if (tiled) {
                if (mg)
                    k_update_q<HelmOp, false><<<tg.upd, tdim, 0, c->stream>>>(
                        c->vx, c->vr, c->vp[cur ^ 1], c->vq, c->fflag, c->list_face, c->qmask_face, c->nact_face, tm,
                        cc, s, c->partials);
                else
                    k_update_q<HelmOp, true><<<tg.upd, tdim, 0, c->stream>>>(
                        c->vx, c->vr, c->vp[cur ^ 1], c->vq, c->fflag, c->list_face, c->qmask_face, c->nact_face, tm,
                        cc, s, c->partials);
            } else if (mg) {
                k_update<HelmOp, false><<<b4, TH, 0, c->stream>>>(c->vx, c->vr, c->vp[cur ^ 1], c->vq, c->fflag, n4,
                                                                  cc, s, c->partials);
            } else {
                k_update<HelmOp, true><<<b4, TH, 0, c->stream>>>(c->vx, c->vr, c->vp[cur ^ 1], c->vq, c->fflag, n4,
                                                                 cc, s, c->partials);
            }
            cudaEvent_t e3 = samp ? prof_mark(c) : nullptr;
            prof_add(c, K_V_SPMV, e0, e1, by_spmv);
            prof_add(c, K_V_UPDATE, e2, e3, by_upd);
            c->n_launches += 2;
            if (mg)
                if (int rc = precondition(0)) return rc;
            cur ^= 1;
        }
        launched += nb;
        FS_CUDA(cudaGetLastError());
        int rc = read_scal(c, 1, &h);
        if (rc) return rc;
        if (h.done) break;
        if (launched > (long long)c->prm.maxit_v + c->prm.check_every)
            return set_error(FS_ECUDA, "viscosity solve: iteration flag never set");
    }
    last = h.status == FS_OK ? (int)std::min<long long>(h.iter, 1 << 20) : 0;
    if (int rc = check_wait_error(c, "viscosity solve")) return rc;
    prof_count(c, K_V_SPMV, h.iter);
    prof_count(c, K_V_UPDATE, h.iter);
    if (mg) mg_count(c, h.iter, true);
    if (st) {
        st->iters_v += h.iter;
        st->relres_v = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
        if (h.status != FS_OK && st->status == FS_OK) st->status = h.status;
    }
    return finish_status(h.status);
}

namespace {
// public cell array -> cell space (zero off liquid), and back
__global__ void k_cell_in(const float *__restrict__ src, float *dst, const uint8_t *__restrict__ cf, Layout L)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x)
        dst[L.PL + idx] = (cf[L.PL + idx] & CF_LIQ) ? src[idx] : 0.f;
}
__global__ void k_cell_out(const float *__restrict__ src, float *dst, Layout L)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x)
        dst[idx] = src[L.PL + idx];
}
__global__ void k_jacobi(const float *__restrict__ r, float *z, const uint8_t *__restrict__ cf, int n)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        z[t] = r[t] * inv_diag<PoisOp>(cf[t], 0.f);
}
}  // namespace

int cell_in(fs_ctx *c, const float *src, float *dst)
{
    k_cell_in<<<grid_blocks(c, c->L.S, TH), TH, 0, c->stream>>>(src, dst, c->cflag, c->L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int cell_out(fs_ctx *c, const float *src, float *dst)
{
    k_cell_out<<<grid_blocks(c, c->L.S, TH), TH, 0, c->stream>>>(src, dst, c->L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int precond_apply_public(fs_ctx *c, const float *r, float *z)
{
    const Layout &L = c->L;
    const int bs = grid_blocks(c, L.S, TH);
    k_cell_in<<<bs, TH, 0, c->stream>>>(r, c->pr, c->cflag, L);
    c->n_launches += 1;
    FS_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(unsigned), c->stream));
    if (c->prm.precond == FS_PRECOND_JACOBI) {
        k_jacobi<<<grid_blocks(c, L.nC, TH), TH, 0, c->stream>>>(c->pr, c->pz, c->cflag, L.nC);
        c->n_launches += 1;
    } else if (c->prm.precond == FS_PRECOND_MG) {
        int rc = mg_apply(c, c->pr, c->pz, nullptr);
        if (rc) return rc;
    } else if (c->prm.precond == FS_PRECOND_MIC0) {
        FS_CUDA(cudaMemsetAsync(c->err_word, 0, sizeof(unsigned), c->stream));
        if (!c->mic_ready) {
            int rc = mic0_factor(c);
            if (rc) return rc;
        }
        int rc = mic0_apply(c, c->pr, c->pz);
        if (rc) return rc;
    } else {
        int rc = learned_apply(c, c->pr, c->pz, nullptr);
        if (rc) return rc;
    }
    k_cell_out<<<bs, TH, 0, c->stream>>>(c->pz, z, L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    unsigned herr = 0;
    FS_CUDA(cudaMemcpyAsync(&herr, c->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    if (c->prm.precond == FS_PRECOND_MIC0 && herr) {
        c->mic_ready = 0;  // the factor may be incomplete: refactor on the next use
        return set_error(FS_ETIMEOUT, "MIC(0) sweep: a wait on a predecessor tile ran out");
    }
    if (herr & 8u) return set_error(FS_ETIMEOUT, "network: a wait for the tensor-core MMAs ran out");
    return FS_OK;
}

// the pressure as its two FP32 terms, public layout (q2 nullable: zeros)
__global__ void __launch_bounds__(TH) k_pair_out(const float *__restrict__ q, const float *__restrict__ q2, float *hi,
                                                 float *lo, Layout L)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.S; idx += gridDim.x * blockDim.x) {
        hi[idx] = q[L.PL + idx];
        lo[idx] = q2 ? q2[L.PL + idx] : 0.f;
    }
}

int pressure_pair(fs_ctx *c, float *q_hi, float *q_lo)
{
    const Layout &L = c->L;
    k_pair_out<<<grid_blocks(c, L.S, TH), TH, 0, c->stream>>>(c->px, c->q_head, q_hi, q_lo, L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_grad_subtract(fs_ctx *c, CF3 in, F3 out, float *q_out)
{
    const Layout &L = c->L;
    dim3 grid(grid_blocks(c, L.S, TH), 4);
    k_grad_subtract<<<grid, TH, 0, c->stream>>>(in, out, c->px, c->q_head, q_out, c->fflag, L,
                                                (float)(1.0 / c->prm.dx));
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_compose(fs_ctx *c, F3 out)
{
    const Layout &L = c->L;
    dim3 grid(grid_blocks(c, L.S, TH), 3);
    k_compose<<<grid, TH, 0, c->stream>>>(c->vx, c->bc, c->fflag, out, L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_mask_fluid(fs_ctx *c, CF3 in, F3 out)
{
    const Layout &L = c->L;
    dim3 grid(grid_blocks(c, L.S, TH), 3);
    k_mask_fluid<<<grid, TH, 0, c->stream>>>(in, out, c->fflag, L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_to_face_space(fs_ctx *c, CF3 in)
{
    const Layout &L = c->L;
    dim3 grid(grid_blocks(c, L.S, TH), 3);
    k_to_face_space<<<grid, TH, 0, c->stream>>>(in, c->vx, c->fflag, L);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

int launch_nu_grad(fs_ctx *c, CF3 uv, double *dot)
{
    const Layout &L = c->L;
    k_nu_grad<<<grid_blocks(c, L.S, TH), TH, 0, c->stream>>>(c->vx, uv, c->fflag, L, c->scal + 3, c->partials);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    SolveScal m;
    int rc = read_scal(c, 3, &m);
    if (rc) return rc;
    *dot = m.aux[0] / (c->prm.dx * c->prm.dx);
    return FS_OK;
}

int launch_loss(fs_ctx *c, CF3 u, CF3 t, int kind, double alpha, double beta, F3 g, double *loss)
{
    const Layout &L = c->L;
    const uint8_t bandbit = kind == FS_MASK_SURFACE ? CF_BAND : CF_LIQ;
    const long long nbc = c->n_band_cells[kind], nbf = c->n_band_faces[kind];
    const bool use_cos = alpha != 0.0 && nbc > 0;
    const int bs = grid_blocks(c, L.S, TH);
    F3 gcw{{c->gc[0], c->gc[1], c->gc[2]}};
    CF3 gcr{{c->gc[0], c->gc[1], c->gc[2]}};
    if (use_cos)
        k_loss_cell<<<bs, TH, 0, c->stream>>>(u, t, c->cflag, bandbit, gcw, L, (float)(alpha / (double)nbc),
                                             c->scal + 3, c->partials);
    const float bo = nbf > 0 ? (float)(beta / (double)nbf) : 0.f;
    k_loss_face<<<bs, TH, 0, c->stream>>>(u, t, c->cflag, c->fflag, bandbit, gcr, use_cos ? 1 : 0, g, L, bo,
                                         c->scal + 2, c->partials);
    c->n_launches += use_cos ? 2 : 1;
    FS_CUDA(cudaGetLastError());
    SolveScal a, b;
    int rc = read_scal(c, 2, &a);
    if (rc) return rc;
    double l = nbf > 0 ? beta * a.aux[0] / (double)nbf : 0.0;
    if (use_cos) {
        rc = read_scal(c, 3, &b);
        if (rc) return rc;
        l += alpha * b.aux[1] / (double)nbc;
    }
    *loss += l;
    return FS_OK;
}

}  // namespace fs
