// fs_optim.cu -- the optimiser of the parameter fit (Sec. 3.4.2 fits the
// viscosity, through theta = log nu, and a correction of the initial velocity
// by gradient descent on the loss): one Adam step (Kingma and Ba, 2015, with the
// bias corrections) on a device array of FP32 parameters, elementwise, four
// elements per thread where the pointers allow it.
#include <cmath>

#include "fs_internal.cuh"

namespace fs {

namespace {

constexpr int TH = 256;

// a1 = 1 - beta1 and a2 = 1 - beta2 come from the host, formed in double: 1 - b2
// taken in FP32 from a rounded 0.999 is off by 1.3e-5 relative
__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, float lr, float b1, float b2, float a1,
                                      float a2, float eps, float c1, float c2, float gs)
{
    const float gr = g * gs;
    m = b1 * m + a1 * gr;
    v = b2 * v + a2 * gr * gr;
    p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// n4 quads, then the n - 4 n4 tail elements by the first threads
__global__ void __launch_bounds__(TH) k_adam_vec(float *p, const float *__restrict__ g, float *m, float *v,
                                                 long long n, int vec, float lr, float b1, float b2, float a1, float a2, float eps,
                                                 float c1, float c2, float gs)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = n >> 2;
        for (long long q = t0; q < n4; q += stride) {
            float4 pp = reinterpret_cast<float4 *>(p)[q], mm = reinterpret_cast<float4 *>(m)[q];
            float4 vv = reinterpret_cast<float4 *>(v)[q];
            const float4 gg = __ldg(reinterpret_cast<const float4 *>(g) + q);
            adam1(pp.x, gg.x, mm.x, vv.x, lr, b1, b2, a1, a2, eps, c1, c2, gs);
            adam1(pp.y, gg.y, mm.y, vv.y, lr, b1, b2, a1, a2, eps, c1, c2, gs);
            adam1(pp.z, gg.z, mm.z, vv.z, lr, b1, b2, a1, a2, eps, c1, c2, gs);
            adam1(pp.w, gg.w, mm.w, vv.w, lr, b1, b2, a1, a2, eps, c1, c2, gs);
            reinterpret_cast<float4 *>(p)[q] = pp;
            reinterpret_cast<float4 *>(m)[q] = mm;
            reinterpret_cast<float4 *>(v)[q] = vv;
        }
        done = n4 << 2;
    }
    for (long long t = done + t0; t < n; t += stride) adam1(p[t], g[t], m[t], v[t], lr, b1, b2, a1, a2, eps, c1, c2, gs);
}

}  // namespace

int adam_update(fs_ctx *c, float *p, const float *g, float *m, float *v, long long n, double lr, double beta1,
                double beta2, double eps, int step, double grad_scale)
{
    if (n == 0) return FS_OK;
    const double c1 = 1.0 - std::pow(beta1, (double)step), c2 = 1.0 - std::pow(beta2, (double)step);
    auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    const int vec = al16(p) && al16(g) && al16(m) && al16(v) ? 1 : 0;
    const long long items = vec ? (n + 3) / 4 : n;
    k_adam_vec<<<grid_blocks(c, items, TH), TH, 0, c->stream>>>(p, g, m, v, n, vec, (float)lr, (float)beta1,
                                                                (float)beta2, (float)(1.0 - beta1),
                                                                (float)(1.0 - beta2), (float)eps, (float)c1,
                                                                (float)c2, (float)grad_scale);
    c->n_launches += 1;
    FS_CUDA(cudaGetLastError());
    return FS_OK;
}

}  // namespace fs
