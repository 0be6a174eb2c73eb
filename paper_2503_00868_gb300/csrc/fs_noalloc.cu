// fs_noalloc.cu -- a pressure projection that allocates nothing.
//
// Some callers cannot allocate device memory: code that runs where a CUDA
// allocation is forbidden or would break a fixed memory budget (a plugin inside
// a host application that owns the device allocator, a real-time loop that must
// not call cudaMalloc after start-up). fs_project_noalloc serves them: it runs
// the same Jacobi-PCG projection as fs_project, but every scratch buffer (flag
// bytes, the CG vectors, the reduction partials and scalars) is carved out of
// one file-scope device array of fixed size, so it needs no context and calls
// no allocating routine.
//
// The array is a module-scope __device__ variable: every GPU that loads this
// library holds it until the process exits. In host code the array's name is
// only a host-side stand-in, so every call looks up its device address with
// cudaGetSymbolAddress, with the caller's device current, and passes that to the
// kernels. The lookup is cheap and is not cached: an address kept from before a
// reset of the device's primary context would be stale.
#include <cstring>

#include "fs_internal.cuh"

namespace fs {
namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB: every grid up to 64^3 fits

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array in the current device's context.
int scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(noalloc scratch)");
    *out = p;
    return FS_OK;
}

}  // namespace
}  // namespace fs

using namespace fs;

extern "C" int fs_project_noalloc(int nx, int ny, int nz, const uint8_t *cell_type_dense, fs_mac *u, float *q_out,
                                  double dx, double tol, int maxit, void *cuda_stream, fs_stats *st)
{
    if (nx < 2 || ny < 2 || nz < 2) return set_error(FS_EINVAL, "grid sizes must be >= 2 (got %d %d %d)", nx, ny, nz);
    if (!cell_type_dense) return set_error(FS_EINVAL, "cell_type_dense is NULL");
    if (!u || !u->u || !u->v || !u->w) return set_error(FS_EINVAL, "u is NULL");
    const float *comps[3] = {u->u, u->v, u->w};
    for (int k = 0; k < 3; k++)
        if (reinterpret_cast<uintptr_t>(comps[k]) % 16) return set_error(FS_EINVAL, "u component %d is not 16-byte aligned", k);
    if (!(dx > 0.0) || !(tol > 0.0) || maxit < 1) return set_error(FS_EINVAL, "need dx > 0, tol > 0, maxit >= 1");

    // the layout of fs_init_grid for this size
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.P = (nx + 1 + 3) / 4 * 4;
    L.R = ny + 1;
    L.Z = nz + 1;
    const long long PL = (long long)L.P * L.R, S = PL * L.Z;
    const long long nC = S + 2 * PL, nF = 3 * (S + PL) + PL;
    if (nF + 8 >= (1LL << 31)) return set_error(FS_EINVAL, "grid too large");
    L.PL = (int)PL;
    L.S = (int)S;
    L.nC = (int)nC;
    L.nF = (int)nF;

    fs_ctx c{};
    c.L = L;
    c.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    int rc;
    if ((rc = check_cuda(cudaGetDevice(&c.device), "cudaGetDevice"))) return rc;
    if ((rc = check_cuda(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device),
                         "cudaDeviceGetAttribute")))
        return rc;
    c.max_blocks = c.num_sms * 8;

    // carve the scratch: flags, the Jacobi-PCG vectors, scalars, partials
    const size_t cb = round256((size_t)nC * sizeof(float));
    const size_t need = round256((size_t)nC) + round256((size_t)nF) + round256((size_t)nF * sizeof(float)) + 9 * cb +
                        round256(4 * sizeof(SolveScal)) + round256((size_t)c.max_blocks * 8 * sizeof(double)) + 256;
    if (need > kNoAllocScratchBytes)
        return set_error(FS_EINVAL,
                         "fs_project_noalloc: a %dx%dx%d grid needs %zu bytes of scratch; the static scratch holds "
                         "%zu bytes (every grid up to 64x64x64 fits)",
                         nx, ny, nz, need, kNoAllocScratchBytes);
    void *base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
    unsigned char *p = static_cast<unsigned char *>(base);
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += round256(bytes);
        return q;
    };
    c.cflag = take((size_t)nC);
    c.fflag = take((size_t)nF);
    c.bc = reinterpret_cast<float *>(take((size_t)nF * sizeof(float)));
    c.pb = reinterpret_cast<float *>(take(cb));
    c.pr = reinterpret_cast<float *>(take(cb));
    c.pp[0] = reinterpret_cast<float *>(take(cb));
    c.pp[1] = reinterpret_cast<float *>(take(cb));
    c.pq = reinterpret_cast<float *>(take(cb));
    c.px = reinterpret_cast<float *>(take(cb));
    c.pxh = reinterpret_cast<float *>(take(cb));
    c.pxt = reinterpret_cast<float *>(take(cb));
    c.pbr = reinterpret_cast<float *>(take(cb));
    c.scal = reinterpret_cast<SolveScal *>(take(4 * sizeof(SolveScal)));
    c.partials = reinterpret_cast<double *>(take((size_t)c.max_blocks * 8 * sizeof(double)));
    c.err_word = reinterpret_cast<unsigned *>(take(16));
    SolveScal host_scal[4];
    c.scal_host = host_scal;

    fs_default_params(&c.prm);
    c.prm.dx = dx;
    c.prm.tol_p = tol;
    c.prm.maxit_p = maxit;
    c.prm.precond = FS_PRECOND_JACOBI;

    // The array keeps the previous call's contents. The right-hand side and A p
    // are only written on liquid cells and must read zero elsewhere (including
    // the guard planes), and the reduction tickets must start at zero.
    if ((rc = check_cuda(cudaMemsetAsync(c.pb, 0, (size_t)nC * sizeof(float), c.stream), "cudaMemsetAsync")) ||
        (rc = check_cuda(cudaMemsetAsync(c.pq, 0, (size_t)nC * sizeof(float), c.stream), "cudaMemsetAsync")) ||
        (rc = check_cuda(cudaMemsetAsync(c.scal, 0, 4 * sizeof(SolveScal), c.stream), "cudaMemsetAsync")))
        return rc;

    fs_stats local{};
    fs_stats *s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    if ((rc = build_mask(&c, cell_type_dense, nullptr))) return rc;
    CF3 uc{{u->u, u->v, u->w}};
    F3 uf{{u->u, u->v, u->w}};
    if ((rc = launch_divergence(&c, uc))) return rc;
    int rp = solve_pressure(&c, s);
    if (rp == FS_ECUDA || rp == FS_EINVAL) return rp;
    if ((rc = launch_grad_subtract(&c, uc, uf, q_out))) return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(c.stream), "cudaStreamSynchronize"))) return rc;
    return s->status;
}
