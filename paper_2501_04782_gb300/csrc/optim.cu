// optim.cu -- the L2 reconstruction loss and the optimiser step (Sec. 4.1: "standard L2
// reconstruction loss"; the paper's optimiser is Adan, the fused step here is Adam with
// bias correction).  Both are elementwise and HBM-bound: float4 vector loads where the
// pointers allow, grid-stride loops sized to the SM count.
#include "gv_internal.cuh"

namespace gvk {

namespace {

__global__ void __launch_bounds__(256) l2_loss_kernel(const float *img, const float *tgt, long long n, float scale,
                                                      float *dL, float *loss) {
    float acc = 0.f;
    const float two_s = 2.f * scale;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        float d = img[i] - tgt[i];
        if (dL) dL[i] = two_s * d;
        acc = fmaf(d, d, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        float t = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += s_w[i];
        atomicAdd(loss, scale * t);
    }
}

__global__ void __launch_bounds__(256) adam_kernel(float *p, float *g, float *m, float *v, long long n, float lr,
                                                   float b1, float b2, float eps, float bc1, float bc2,
                                                   int zero_grad) {
    long long stride = (long long)gridDim.x * blockDim.x;
    const float ib1 = 1.f - b1, ib2 = 1.f - b2;
    const float rbc1 = 1.f / bc1, rbc2 = 1.f / bc2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        float gi = g[i];
        float mi = fmaf(b1, m[i], ib1 * gi);
        float vi = fmaf(b2, v[i], ib2 * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * rbc1) / (sqrtf(vi * rbc2) + eps);
        if (zero_grad) g[i] = 0.f;
    }
}

__global__ void grad2d_debug_kernel(Work w, float *out) {
    unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned P = w.L.P;
    if (p >= P) return;
    float4 a = w.g0[p], b = w.g1[p];
    // staged basis (du, dv, da', db', dc', dlog2o, ...) -> (du, dv, dA, dB, dC, do, ...)
    const float o = exp2f(w.feat1[p].y);
    float vals[9] = {a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w, -0.5f * kLog2e * b.x,
                     o > 0.f ? b.y * kLog2e / o : 0.f, b.z, b.w, w.g2[p]};
    for (int k = 0; k < 9; k++) out[(size_t)k * P + p] = vals[k];
}

int grid_for(long long n, int per_block = 256) {
    long long b = (n + per_block - 1) / per_block;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t launch_l2_loss(const float *image, const float *target, long long n, float scale, float *dL, float *loss,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    l2_loss_kernel<<<grid_for(n), 256, 0, s>>>(image, target, n, scale, dL, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                        float bc1, float bc2, int zero_grad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    adam_kernel<<<grid_for(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, zero_grad);
    return cudaGetLastError();
}

cudaError_t launch_grad2d_debug(const Work &w, float *out, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    grad2d_debug_kernel<<<(w.L.P + 255) / 256, 256, 0, s>>>(w, out);
    return cudaGetLastError();
}

}  // namespace gvk
