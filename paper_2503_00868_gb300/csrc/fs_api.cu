// fs_api.cu -- the C ABI declared in include/fluidstep.h: argument checks,
// context memory and the order of kernels for one step, its adjoint and the loss
// (arXiv 2503.00868: Eq. eq::v split as in Sec. 3.2.2, back-traced convection of
// Sec. 3.4.1, loss of Eq. eq::optLoss in Sec. 3.4.2).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fs_internal.cuh"

namespace fs {

static thread_local char g_err[512] = "";

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return 0;
    return set_error(FS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static int check_params(const fs_params *p)
{
    if (!p) return set_error(FS_EINVAL, "params is NULL");
    if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return set_error(FS_EINVAL, "dx must be > 0");
    if (!(p->dt >= 0.0) || !std::isfinite(p->dt)) return set_error(FS_EINVAL, "dt must be >= 0");
    if (!(p->nu >= 0.0) || !std::isfinite(p->nu)) return set_error(FS_EINVAL, "nu must be >= 0");
    if (!(p->rho > 0.0) || !std::isfinite(p->rho)) return set_error(FS_EINVAL, "rho must be > 0");
    for (int c = 0; c < 3; c++)
        if (!std::isfinite(p->g[c])) return set_error(FS_EINVAL, "g must be finite");
    if (p->precond < FS_PRECOND_JACOBI || p->precond > FS_PRECOND_LEARNED_MG)
        return set_error(FS_EINVAL, "unknown preconditioner %d", p->precond);
    if (p->maxit_p < 1 || p->maxit_v < 1) return set_error(FS_EINVAL, "iteration caps must be >= 1");
    if (!(p->tol_p > 0.0) || !(p->tol_v > 0.0)) return set_error(FS_EINVAL, "tolerances must be > 0");
    if (p->check_every < 1 || p->check_every > 4096) return set_error(FS_EINVAL, "check_every must be in [1, 4096]");
    if (p->spin_limit < 1) return set_error(FS_EINVAL, "spin_limit must be >= 1");
    if (!(p->mic_tau >= 0.0 && p->mic_tau <= 1.0)) return set_error(FS_EINVAL, "mic_tau must be in [0, 1]");
    if (!(p->mic_sigma >= 0.0 && p->mic_sigma < 1.0)) return set_error(FS_EINVAL, "mic_sigma must be in [0, 1)");
    if (p->warm_start != 0 && p->warm_start != 1) return set_error(FS_EINVAL, "warm_start must be 0 or 1");
    if (p->advect_grad != FS_ADVECT_GRAD_EXACT && p->advect_grad != FS_ADVECT_GRAD_UPWIND)
        return set_error(FS_EINVAL, "unknown advect_grad %d", p->advect_grad);
    if (p->pressure_solver != FS_SOLVER_PCG && p->pressure_solver != FS_SOLVER_PERCNN)
        return set_error(FS_EINVAL, "unknown pressure solver %d", p->pressure_solver);
    return FS_OK;
}

static int check_field(const fs_mac *m, const char *name, bool nullable)
{
    if (!m) return nullable ? FS_OK : set_error(FS_EINVAL, "%s is NULL", name);
    const float *p[3] = {m->u, m->v, m->w};
    for (int c = 0; c < 3; c++) {
        if (!p[c]) return set_error(FS_EINVAL, "%s component %d is NULL", name, c);
        if (reinterpret_cast<uintptr_t>(p[c]) % 16) return set_error(FS_EINVAL, "%s component %d is not 16-byte aligned", name, c);
    }
    return FS_OK;
}

static bool same_field(const fs_mac *a, const fs_mac *b)
{
    if (!a || !b) return false;
    return a->u == b->u || a->v == b->v || a->w == b->w;
}

static CF3 cf3(const fs_mac *m) { return CF3{{m->u, m->v, m->w}}; }
static F3 f3(fs_mac *m) { return F3{{m->u, m->v, m->w}}; }

static int alloc_zero(void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(FS_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return check_cuda(cudaMemset(*p, 0, bytes), "cudaMemset");
}

// ---- per-kernel timing ---------------------------------------------------------
static const char *kKernelNames[K_COUNT] = {"pressure_spmv", "pressure_update", "visc_spmv", "visc_update",
                                            "advect", "advect_adjoint", "mic0_apply", "net_apply", "fcg_vectors",
                                            "mg_vcycle_p", "mg_vcycle_v", "mg0_smooth2", "mg0_residual",
                                            "mg0_restrict", "mg0_prolong", "mg0_smooth", "mg0_smooth_z",
                                            "mg_coarse"};

struct Prof {
    std::vector<cudaEvent_t> free_ev, all_ev;
    struct Pending { int id; cudaEvent_t a, b; double bytes; };
    std::vector<Pending> pending;
    double ms[K_COUNT] = {};
    double bytes[K_COUNT] = {};
    long long n[K_COUNT] = {};
    long long all[K_COUNT] = {};  // launches that did work, timed or not
};

cudaEvent_t prof_mark(fs_ctx *c)
{
    if (!c->prof_on) return nullptr;
    Prof *p = static_cast<Prof *>(c->prof);
    if (p->free_ev.empty()) return nullptr;
    cudaEvent_t e = p->free_ev.back();
    p->free_ev.pop_back();
    cudaEventRecord(e, c->stream);
    return e;
}

void prof_add(fs_ctx *c, int id, cudaEvent_t a, cudaEvent_t b, double bytes)
{
    if (!c->prof_on) return;
    Prof *p = static_cast<Prof *>(c->prof);
    if (!a || !b) {
        if (a) p->free_ev.push_back(a);
        if (b) p->free_ev.push_back(b);
        return;
    }
    p->pending.push_back({id, a, b, bytes});
}

void prof_count(fs_ctx *c, int id, long long launches)
{
    if (!c->prof_on || !c->prof) return;
    static_cast<Prof *>(c->prof)->all[id] += launches;
}

void prof_flush(fs_ctx *c)
{
    if (!c->prof) return;
    Prof *p = static_cast<Prof *>(c->prof);
    for (auto &q : p->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            p->ms[q.id] += ms;
            p->bytes[q.id] += q.bytes;
            p->n[q.id] += 1;
        } else {
            cudaGetLastError();
        }
        p->free_ev.push_back(q.a);
        p->free_ev.push_back(q.b);
    }
    p->pending.clear();
}

static void prof_destroy(fs_ctx *c)
{
    if (!c->prof) return;
    Prof *p = static_cast<Prof *>(c->prof);
    for (cudaEvent_t e : p->all_ev) cudaEventDestroy(e);
    delete p;
    c->prof = nullptr;
}

static void free_ctx(fs_ctx *c)
{
    if (!c) return;
    prof_destroy(c);
    net_free(c);
    fcg_release(c);
    percnn_free(c);
    splat_free(c);
    mg_free(c);
    void *ptrs[] = {c->cflag, c->fflag, c->bc, c->dsum, c->pb, c->pr, c->pp[0], c->pp[1], c->pq, c->px, c->pz,
                    c->pxh, c->pxt, c->pbr, c->vx, c->vr, c->vp[0], c->vp[1], c->vq, c->vz, c->fu[0], c->fu[1], c->fu[2], c->fg[0], c->fg[1],
                    c->fg[2], c->gc[0], c->gc[1], c->gc[2], c->mic_prec, c->scal, c->partials, c->err_word, c->pw[0], c->pw[1],
                    c->act_cell, c->act_face, c->list_cell, c->list_face, c->items_cell, c->items_face, c->qmask_cell, c->qmask_face,
                    c->py, c->mic_order,
                    c->mic_tact, c->mic_tflag, c->mic_next};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->scal_host) cudaFreeHost(c->scal_host);
    delete c;
}

}  // namespace fs

using namespace fs;

extern "C" {

void fs_default_params(fs_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dx = 1.0;
    p->dt = 1.0 / 30.0;
    p->nu = 0.01;
    p->rho = 1000.0;
    p->precond = FS_PRECOND_JACOBI;
    p->maxit_p = 20000;
    p->maxit_v = 2000;
    p->tol_p = 1e-6;
    p->tol_v = 1e-6;
    p->check_every = 8;
    p->spin_limit = 1 << 22;
    p->mic_tau = 0.97;
    p->mic_sigma = 0.25;
    p->warm_start = 0;
    p->advect_grad = FS_ADVECT_GRAD_EXACT;
    p->pressure_solver = FS_SOLVER_PCG;
}

const char *fs_last_error(void) { return g_err; }

int fs_profile(fs_ctx *c, int enable)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    FS_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    if (enable && !c->prof) {
        Prof *p = new (std::nothrow) Prof();
        if (!p) return set_error(FS_ENOMEM, "host allocation failed");
        for (int k = 0; k < 8192; k++) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            p->all_ev.push_back(e);
            p->free_ev.push_back(e);
        }
        c->prof = p;
    }
    if (c->prof) {
        Prof *p = static_cast<Prof *>(c->prof);
        for (int k = 0; k < K_COUNT; k++) {
            p->ms[k] = 0.0;
            p->bytes[k] = 0.0;
            p->n[k] = 0;
            p->all[k] = 0;
        }
    }
    c->prof_on = enable > 0 ? 1 : 0;
    c->prof_period = enable > 0 ? enable : 1;
    c->n_launches = 0;
    return FS_OK;
}

int fs_profile_read(fs_ctx *c, fs_kernel_time *out, int max, int *count)
{
    if (!c || !count || (max > 0 && !out)) return set_error(FS_EINVAL, "NULL argument");
    FS_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    *count = 0;
    if (!c->prof) return FS_OK;
    Prof *p = static_cast<Prof *>(c->prof);
    for (int k = 0; k < K_COUNT && *count < max; k++) {
        if (!p->n[k]) continue;
        fs_kernel_time &e = out[(*count)++];
        std::memset(&e, 0, sizeof(e));
        std::snprintf(e.name, sizeof(e.name), "%s", kKernelNames[k]);
        e.launches = p->n[k];
        e.total_ms = p->ms[k];
        e.bytes = p->bytes[k];
        e.all_launches = std::max(p->all[k], p->n[k]);
    }
    if (*count < max) {
        fs_kernel_time &e = out[(*count)++];
        std::memset(&e, 0, sizeof(e));
        std::snprintf(e.name, sizeof(e.name), "all_kernels");
        e.launches = c->n_launches;
    }
    return FS_OK;
}

int fs_init_grid(fs_ctx **out, int nx, int ny, int nz, const fs_params *p, void *cuda_stream)
{
    g_err[0] = 0;
    if (!out) return set_error(FS_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2 || nz < 2) return set_error(FS_EINVAL, "grid sizes must be >= 2 (got %d %d %d)", nx, ny, nz);
    int rc = check_params(p);
    if (rc) return rc;
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.P = (nx + 1 + 3) / 4 * 4;
    L.R = ny + 1;
    L.Z = nz + 1;
    const long long PL = (long long)L.P * L.R, S = PL * L.Z;
    const long long nF = 3 * (S + PL) + PL;
    if (nF + 8 >= (1LL << 31)) return set_error(FS_EINVAL, "grid too large for 32-bit indexing");
    L.PL = (int)PL;
    L.S = (int)S;
    L.nC = (int)(S + 2 * PL);
    L.nF = (int)nF;

    fs_ctx *c = new (std::nothrow) fs_ctx();
    if (!c) return set_error(FS_ENOMEM, "host allocation failed");
    c->L = L;
    c->prm = *p;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    if ((rc = check_cuda(cudaGetDevice(&c->device), "cudaGetDevice"))) { free_ctx(c); return rc; }
    if ((rc = check_cuda(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device),
                         "cudaDeviceGetAttribute"))) { free_ctx(c); return rc; }
    c->max_blocks = c->num_sms * 8;
    const size_t cb = (size_t)L.nC * sizeof(float), fb = (size_t)L.nF * sizeof(float), sb = (size_t)L.S * sizeof(float);
#define ALLOC(ptr, bytes)                                                   \
    do {                                                                    \
        if ((rc = alloc_zero((void **)&(ptr), (bytes)))) { free_ctx(c); return rc; } \
    } while (0)
    ALLOC(c->cflag, (size_t)L.nC);
    ALLOC(c->fflag, (size_t)L.nF);
    ALLOC(c->bc, fb);
    ALLOC(c->dsum, fb);
    ALLOC(c->pb, cb);
    ALLOC(c->pr, cb);
    ALLOC(c->pp[0], cb);
    ALLOC(c->pp[1], cb);
    ALLOC(c->pq, cb);
    ALLOC(c->px, cb);
    ALLOC(c->pxh, cb);
    ALLOC(c->pxt, cb);
    ALLOC(c->pbr, cb);
    ALLOC(c->pz, cb);
    ALLOC(c->vx, fb);
    ALLOC(c->vr, fb);
    ALLOC(c->vp[0], fb);
    ALLOC(c->vp[1], fb);
    ALLOC(c->vq, fb);
    ALLOC(c->vz, fb);
    for (int k = 0; k < 3; k++) {
        ALLOC(c->fu[k], sb);
        ALLOC(c->fg[k], sb);
        ALLOC(c->gc[k], cb);
    }
    ALLOC(c->mic_prec, cb);
    ALLOC(c->py, cb);
    c->mic_ntiles = ((nx + 7) / 8) * ((ny + 7) / 8) * ((nz + 7) / 8);
    ALLOC(c->mic_order, (size_t)c->mic_ntiles * sizeof(int));
    ALLOC(c->mic_tact, (size_t)c->mic_ntiles);
    ALLOC(c->mic_tflag, (size_t)c->mic_ntiles * sizeof(int));
    ALLOC(c->mic_next, 16);
    c->tm_cell = make_tilemap(L, 1, c->num_sms);
    c->tm_face = make_tilemap(L, 3, c->num_sms);
    ALLOC(c->act_cell, (size_t)c->tm_cell.nblocks);
    ALLOC(c->act_face, (size_t)c->tm_face.nblocks);
    ALLOC(c->list_cell, (size_t)c->tm_cell.nblocks * sizeof(int));
    ALLOC(c->list_face, (size_t)c->tm_face.nblocks * sizeof(int));
    ALLOC(c->qmask_cell, (size_t)c->tm_cell.nblocks * 8 * sizeof(unsigned));
    ALLOC(c->qmask_face, (size_t)c->tm_face.nblocks * 8 * sizeof(unsigned));
    ALLOC(c->items_cell, (size_t)c->tm_cell.nblocks * sizeof(int4));
    ALLOC(c->items_face, (size_t)c->tm_face.nblocks * sizeof(int4));
    const int red_blocks = std::max(c->max_blocks, std::max(c->tm_cell.nblocks, c->tm_face.nblocks));
    ALLOC(c->scal, 4 * sizeof(SolveScal));
    ALLOC(c->partials, (size_t)red_blocks * 8 * sizeof(double));
    ALLOC(c->err_word, 16);
#undef ALLOC
    if (cudaHostAlloc((void **)&c->scal_host, 4 * sizeof(SolveScal), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->scal_host = nullptr;
        free_ctx(c);
        return set_error(FS_ENOMEM, "pinned allocation failed");
    }
    if (int rc = make_tensor_maps(c)) {
        free_ctx(c);
        return rc;
    }
    *out = c;
    return FS_OK;
}

int fs_destroy(fs_ctx *c)
{
    if (!c) return FS_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return FS_OK;
}

int fs_layout(const fs_ctx *c, fs_layout_t *out)
{
    if (!c || !out) return set_error(FS_EINVAL, "NULL argument");
    out->nx = c->L.nx;
    out->ny = c->L.ny;
    out->nz = c->L.nz;
    out->pitch = c->L.P;
    out->rows = c->L.R;
    out->planes = c->L.Z;
    out->nelems = c->L.S;
    return FS_OK;
}

int fs_set_stream(fs_ctx *c, void *cuda_stream)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return FS_OK;
}

int fs_set_params(fs_ctx *c, const fs_params *p)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->mic_tau != c->prm.mic_tau || p->mic_sigma != c->prm.mic_sigma) c->mic_ready = 0;
    c->prm = *p;
    // a new problem: no warm start from earlier solves (the floor of the first
    // CG pass stays: it depends on the mask and the scale of the pressure, and a
    // wrong one costs one refinement step and is then measured again)
    c->pw_valid[0] = c->pw_valid[1] = 0;
    return FS_OK;
}

int fs_set_mask(fs_ctx *c, const uint8_t *cell_type_dense, const fs_mac *bc)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    g_err[0] = 0;
    if (!cell_type_dense) return set_error(FS_EINVAL, "cell_type_dense is NULL");
    int rc = check_field(bc, "bc", true);
    if (rc) return rc;
    c->mask_set = 0;
    return build_mask(c, cell_type_dense, bc);
}

static int need_mask(const fs_ctx *c)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    if (!c->mask_set) return set_error(FS_ESTATE, "fs_set_mask has not been called");
    return FS_OK;
}

int fs_step(fs_ctx *c, const fs_mac *u_in, fs_mac *u_out, fs_mac *u_visc, fs_stats *st)
{
    int rc = need_mask(c);
    if (rc) return rc;
    g_err[0] = 0;
    if ((rc = check_field(u_in, "u_in", false)) || (rc = check_field(u_out, "u_out", false)) ||
        (rc = check_field(u_visc, "u_visc", true)))
        return rc;
    if (same_field(u_visc, u_out)) return set_error(FS_EINVAL, "u_visc must not alias u_out");
    fs_stats local{};
    fs_stats *s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    // advection + body force -> face space; implicit viscosity in place
    if ((rc = launch_advect(c, cf3(u_in)))) return rc;
    int rv = solve_viscosity(c, true, s);
    if (rv == FS_ECUDA) return rv;
    // full field after viscosity, then the projection
    fs_mac *uv = u_visc ? u_visc : u_out;
    if ((rc = launch_compose(c, f3(uv)))) return rc;
    if ((rc = launch_divergence(c, cf3(uv)))) return rc;
    c->solve_kind = 0;
    int rp = solve_pressure(c, s);
    if (rp == FS_ECUDA || rp == FS_EINVAL) return rp;
    if ((rc = launch_grad_subtract(c, cf3(uv), f3(u_out), nullptr))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    return s->status;
}

int fs_project(fs_ctx *c, fs_mac *u, float *q_out, fs_stats *st)
{
    int rc = need_mask(c);
    if (rc) return rc;
    g_err[0] = 0;
    if ((rc = check_field(u, "u", false))) return rc;
    fs_stats local{};
    fs_stats *s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    if ((rc = launch_divergence(c, cf3(u)))) return rc;
    c->solve_kind = 0;
    int rp = solve_pressure(c, s);
    if (rp == FS_ECUDA || rp == FS_EINVAL) return rp;
    if ((rc = launch_grad_subtract(c, cf3(u), f3(u), q_out))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    return s->status;
}

int fs_adjoint_step(fs_ctx *c, const fs_mac *u_in, const fs_mac *u_visc, const fs_mac *g_out, fs_mac *g_in,
                    double *g_nu, fs_stats *st)
{
    int rc = need_mask(c);
    if (rc) return rc;
    g_err[0] = 0;
    if ((rc = check_field(u_in, "u_in", false)) || (rc = check_field(u_visc, "u_visc", true)) ||
        (rc = check_field(g_out, "g_out", false)) || (rc = check_field(g_in, "g_in", false)))
        return rc;
    if (same_field(g_in, u_in) || same_field(g_in, u_visc))
        return set_error(FS_EINVAL, "g_in must not alias u_in or u_visc");
    fs_stats local{};
    fs_stats *s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    // the field after viscosity: given, or recomputed from u_in
    CF3 uv;
    if (u_visc) {
        uv = cf3(u_visc);
    } else {
        if ((rc = launch_advect(c, cf3(u_in)))) return rc;
        int rv = solve_viscosity(c, true, s);
        if (rv == FS_ECUDA) return rv;
        F3 fu{{c->fu[0], c->fu[1], c->fu[2]}};
        if ((rc = launch_compose(c, fu))) return rc;
        uv = CF3{{c->fu[0], c->fu[1], c->fu[2]}};
    }
    // projection adjoint: the cotangent of fixed and air faces is dropped, then P
    F3 fg{{c->fg[0], c->fg[1], c->fg[2]}};
    CF3 fgc{{c->fg[0], c->fg[1], c->fg[2]}};
    if ((rc = launch_mask_fluid(c, cf3(g_out), fg))) return rc;
    if ((rc = launch_divergence(c, fgc))) return rc;
    c->solve_kind = 1;
    int rp = solve_pressure(c, s);
    if (rp == FS_ECUDA || rp == FS_EINVAL) return rp;
    if ((rc = launch_grad_subtract(c, fgc, fg, nullptr))) return rc;
    // viscosity adjoint: one more solve with the same operator, no Dirichlet part
    if ((rc = launch_to_face_space(c, fgc))) return rc;
    int rv = solve_viscosity(c, false, s);
    if (rv == FS_ECUDA) return rv;
    if (g_nu) {
        double dot = 0.0;
        if ((rc = launch_nu_grad(c, uv, &dot))) return rc;
        *g_nu += -c->prm.dt * dot;
    }
    // advection adjoint (the body force adds a constant)
    if ((rc = launch_advect_adjoint(c, cf3(u_in), f3(g_in)))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    return s->status;
}

int fs_divergence(fs_ctx *c, const fs_mac *u, float *b_out)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if ((rc = check_field(u, "u", false))) return rc;
    if (!b_out) return set_error(FS_EINVAL, "b_out is NULL");
    if ((rc = launch_divergence(c, cf3(u)))) return rc;
    if ((rc = cell_out(c, c->pb, b_out))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

int fs_wall_profile(fs_ctx *c, const double dir[3], const float *vinf, double delta, fs_mac *u_out)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if (!dir || !vinf) return set_error(FS_EINVAL, "dir / vinf is NULL");
    if (!std::isfinite(dir[0]) || !std::isfinite(dir[1]) || !std::isfinite(dir[2]))
        return set_error(FS_EINVAL, "dir must be finite");
    if (!(delta >= 0.0) || !std::isfinite(delta)) return set_error(FS_EINVAL, "delta must be finite and >= 0");
    if ((rc = check_field(u_out, "u_out", false))) return rc;
    if ((rc = launch_wall_profile(c, dir, vinf, delta, f3(u_out)))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

int fs_pbd_project(fs_ctx *c, fs_mac *u, int hold_surface, int iters, double eps, double *div_norm)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if ((rc = check_field(u, "u", false))) return rc;
    if (iters < 0 || iters > 10000000) return set_error(FS_EINVAL, "iters must be in [0, 1e7]");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return set_error(FS_EINVAL, "eps must be finite and >= 0");
    return launch_pbd_project(c, f3(u), hold_surface ? 1 : 0, iters, eps, div_norm);
}

static int check_camera(const fs_camera *cam)
{
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return set_error(FS_EINVAL, "image size must be in [1, 16384]");
    const double *vals[] = {cam->R, cam->t, &cam->fx, &cam->fy, &cam->cx, &cam->cy, &cam->znear, cam->bg};
    const int cnt[] = {9, 3, 1, 1, 1, 1, 1, 3};
    for (int a = 0; a < 8; a++)
        for (int k = 0; k < cnt[a]; k++)
            if (!std::isfinite(vals[a][k])) return set_error(FS_EINVAL, "camera parameters must be finite");
    if (!(cam->znear > 0.0)) return set_error(FS_EINVAL, "znear must be > 0");
    return FS_OK;
}

int fs_splat_render_sh(fs_ctx *c, int n, const float *x, const float *opacity, const float *A, const float *sh,
                       int sh_degree, const fs_camera *cam, float *rgb_out, float *T_out)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    g_err[0] = 0;
    if (n < 0) return set_error(FS_EINVAL, "n must be >= 0");
    if (sh_degree < 0 || sh_degree > 3) return set_error(FS_EINVAL, "sh_degree must be in [0, 3]");
    if (n > 0 && (!x || !opacity || !A || !sh)) return set_error(FS_EINVAL, "Gaussian array is NULL");
    if (!cam || !rgb_out) return set_error(FS_EINVAL, "cam / rgb_out is NULL");
    if (int rc = check_camera(cam)) return rc;
    return splat_render(c, n, x, opacity, A, nullptr, sh, sh_degree, cam, rgb_out, T_out);
}

int fs_splat_render(fs_ctx *c, int n, const float *x, const float *opacity, const float *A, const float *color,
                    const fs_camera *cam, float *rgb_out, float *T_out)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    g_err[0] = 0;
    if (n < 0) return set_error(FS_EINVAL, "n must be >= 0");
    if (n > 0 && (!x || !opacity || !A || !color)) return set_error(FS_EINVAL, "Gaussian array is NULL");
    if (!cam || !rgb_out) return set_error(FS_EINVAL, "cam / rgb_out is NULL");
    if (int rc = check_camera(cam)) return rc;
    return splat_render(c, n, x, opacity, A, color, nullptr, 0, cam, rgb_out, T_out);
}

int fs_splat_stats(const fs_ctx *c, unsigned long long *entries, unsigned long long *max_tile)
{
    if (!c || !entries || !max_tile) return set_error(FS_EINVAL, "NULL argument");
    splat_stats(c, entries, max_tile);
    return FS_OK;
}

int fs_p2g(fs_ctx *c, int np, const float *x, const float *v, const float *C, const float *m, fs_mac *u_out,
           fs_mac *mass_out)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    g_err[0] = 0;
    if (np < 0) return set_error(FS_EINVAL, "np must be >= 0");
    if (np > 0 && (!x || !v || !C || !m)) return set_error(FS_EINVAL, "particle array is NULL");
    int rc;
    if ((rc = check_field(u_out, "u_out", false)) || (rc = check_field(mass_out, "mass_out", true))) return rc;
    F3 mass{{nullptr, nullptr, nullptr}};
    if (mass_out) mass = f3(mass_out);
    if ((rc = launch_p2g(c, np, x, v, C, m, f3(u_out), mass))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

int fs_g2p(fs_ctx *c, int np, float *x, float *v_out, float *C_out, float *F, const float *A0, float *A_out,
           const fs_mac *u, double dt, int advance, double lo, double hi)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    g_err[0] = 0;
    if (np < 0) return set_error(FS_EINVAL, "np must be >= 0");
    if (np > 0 && (!x || !v_out || !C_out)) return set_error(FS_EINVAL, "particle array is NULL");
    if (!std::isfinite(dt) || !std::isfinite(lo) || !std::isfinite(hi)) return set_error(FS_EINVAL, "dt, lo, hi must be finite");
    int rc;
    if ((rc = check_field(u, "u", false))) return rc;
    if ((rc = launch_g2p(c, np, x, v_out, C_out, F, A0, A_out, cf3(u), dt, advance, lo, hi))) return rc;
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

int fs_percnn_load(fs_ctx *c, const float *w27, int substeps)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    return percnn_load(c, w27, substeps);
}

int fs_percnn_read(fs_ctx *c, float *w27, int *substeps)
{
    if (!c || !w27) return set_error(FS_EINVAL, "NULL argument");
    return percnn_read(c, w27, substeps);
}

int fs_percnn_grad(fs_ctx *c, const float *b, const float *q, double *loss, float *dw27)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if (!b || !q || !loss || !dw27) return set_error(FS_EINVAL, "NULL argument");
    return percnn_grad(c, b, q, loss, dw27);
}

int fs_net_param_count(void) { return net_param_count(); }

int fs_net_load(fs_ctx *c, const float *params, int count, int params_on_host)
{
    if (!c || !params) return set_error(FS_EINVAL, "NULL argument");
    g_err[0] = 0;
    return net_load(c, params, count, params_on_host != 0);
}

int fs_net_read(fs_ctx *c, float *params_host, int count)
{
    if (!c || !params_host) return set_error(FS_EINVAL, "NULL argument");
    if (count != net_param_count()) return set_error(FS_EINVAL, "expected %d values", net_param_count());
    return net_read(c, params_host);
}

int fs_net_kernel(fs_ctx *c, int which)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    g_err[0] = 0;
    if (which != 0 && which != 1) return set_error(FS_EINVAL, "which must be 0 (mma.sync) or 1 (tcgen05)");
    return net_kernel(c, which);
}

int fs_net_forward(fs_ctx *c, const float *r, float *z)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if (!r || !z || r == z) return set_error(FS_EINVAL, "bad r / z");
    if (!net_loaded(c)) return set_error(FS_ESTATE, "no network loaded");
    const int saved = c->prm.precond;
    c->prm.precond = FS_PRECOND_LEARNED;
    rc = precond_apply_public(c, r, z);
    c->prm.precond = saved;
    return rc;
}

int fs_net_grad(fs_ctx *c, const float *b, const float *q, double *loss)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if (!b || !q) return set_error(FS_EINVAL, "NULL argument");
    g_err[0] = 0;
    return net_grad(c, b, q, loss);
}

int fs_net_grad_read(fs_ctx *c, float *grad_host, int count)
{
    if (!c || !grad_host) return set_error(FS_EINVAL, "NULL argument");
    if (count != net_param_count()) return set_error(FS_EINVAL, "expected %d values", net_param_count());
    return net_grad_read(c, grad_host);
}

int fs_net_adam(fs_ctx *c, double lr, double beta1, double beta2, double eps, int step, double grad_scale,
                int fix_offsets)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return set_error(FS_EINVAL, "bad Adam hyper-parameters");
    return net_adam(c, lr, beta1, beta2, eps, step, grad_scale, fix_offsets);
}

int fs_pressure_pair(fs_ctx *c, float *q_hi, float *q_lo)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if (!q_hi || !q_lo) return set_error(FS_EINVAL, "NULL argument");
    if (q_hi == q_lo) return set_error(FS_EINVAL, "q_hi and q_lo must not alias");
    return pressure_pair(c, q_hi, q_lo);
}

int fs_adam_update(fs_ctx *c, float *p, const float *g, float *m, float *v, long long n, double lr, double beta1,
                   double beta2, double eps, int step, double grad_scale)
{
    if (!c) return set_error(FS_EINVAL, "NULL context");
    if (n < 0 || (n > 0 && (!p || !g || !m || !v))) return set_error(FS_EINVAL, "bad parameter arrays");
    if (step < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
        !(eps > 0.0) || !std::isfinite(lr) || !std::isfinite(grad_scale))
        return set_error(FS_EINVAL, "bad Adam hyper-parameters");
    return adam_update(c, p, g, m, v, n, lr, beta1, beta2, eps, step, grad_scale);
}

int fs_net_train_step(fs_ctx *c, const float *b_batch, const float *q_batch, int batch, double lr, int step,
                      double *loss)
{
    int rc = need_mask(c);
    if (rc) return rc;
    if (!b_batch || !q_batch || batch < 1) return set_error(FS_EINVAL, "bad batch");
    double l = 0.0;
    for (int k = 0; k < batch; k++) {
        rc = net_grad(c, b_batch + (size_t)k * c->L.S, q_batch + (size_t)k * c->L.S, &l);
        if (rc) return rc;
    }
    rc = net_adam(c, lr, 0.9, 0.999, 1e-8, step, 1.0 / batch, 1);
    if (loss) *loss = l / batch;
    return rc;
}

int fs_precond_apply(fs_ctx *c, const float *r, float *z)
{
    int rc = need_mask(c);
    if (rc) return rc;
    g_err[0] = 0;
    if (!r || !z) return set_error(FS_EINVAL, "NULL argument");
    if (r == z) return set_error(FS_EINVAL, "r and z must not alias");
    return precond_apply_public(c, r, z);
}

int fs_loss_grad(fs_ctx *c, const fs_mac *u, const fs_mac *target, int mask_kind, double alpha, double beta,
                 double *loss, fs_mac *g)
{
    int rc = need_mask(c);
    if (rc) return rc;
    g_err[0] = 0;
    if ((rc = check_field(u, "u", false)) || (rc = check_field(target, "target", false)) ||
        (rc = check_field(g, "g", true)))
        return rc;
    if (!loss) return set_error(FS_EINVAL, "loss is NULL");
    if (mask_kind != FS_MASK_SURFACE && mask_kind != FS_MASK_OCCUPIED)
        return set_error(FS_EINVAL, "unknown mask kind %d", mask_kind);
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return set_error(FS_EINVAL, "alpha, beta must be finite");
    F3 gg = g ? f3(g) : F3{{nullptr, nullptr, nullptr}};
    return launch_loss(c, cf3(u), cf3(target), mask_kind, alpha, beta, gg, loss);
}

}  // extern "C"
