// optim.cu -- the L2 reconstruction loss and the optimiser steps (Sec. 4.1: the L2
// reconstruction loss; the paper's optimiser is Adan, fused here, beside a fused Adam with
// bias correction).  Both are elementwise and HBM-bound: float4 vector loads where the
// pointers allow, grid-stride loops of at most 4096 blocks.
#include <cmath>
#include <cstdint>
#include <initializer_list>

#include "gv_internal.cuh"

namespace gvk {

namespace {

__global__ void __launch_bounds__(256) l2_loss_kernel(const float *img, const float *tgt, long long n, float scale,
                                                      float *dL, float *loss) {
    pdl_prologue();
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

// Elementwise optimiser kernels: VEC = every array 16-byte aligned, so a thread moves float4
// vectors (four parameters per load of each array); the n % 4 tail goes element by element.
template <class Op, bool VEC>
__device__ __forceinline__ void elementwise(const Op &op, long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long done = 0;
    if (VEC) {
        const long long n4 = n >> 2;
        for (long long i = tid; i < n4; i += stride) op.vec4(i);
        done = n4 << 2;
    }
    for (long long i = done + tid; i < n; i += stride) op.one(i);
}

struct AdamOp {
    float *p, *g, *m, *v;
    float lr, b1, b2, ib1, ib2, eps, rbc1, rbc2;
    int zero_grad;
    __device__ __forceinline__ void upd(float &pi, float gi, float &mi, float &vi) const {
        mi = fmaf(b1, mi, ib1 * gi);
        vi = fmaf(b2, vi, ib2 * gi * gi);
        pi -= lr * (mi * rbc1) / (sqrtf(vi * rbc2) + eps);
    }
    __device__ __forceinline__ void one(long long i) const {
        float pi = p[i], mi = m[i], vi = v[i];
        upd(pi, g[i], mi, vi);
        p[i] = pi;
        m[i] = mi;
        v[i] = vi;
        if (zero_grad) g[i] = 0.f;
    }
    __device__ __forceinline__ void vec4(long long i) const {
        float4 P = reinterpret_cast<float4 *>(p)[i], G = reinterpret_cast<const float4 *>(g)[i];
        float4 M = reinterpret_cast<float4 *>(m)[i], V = reinterpret_cast<float4 *>(v)[i];
        upd(P.x, G.x, M.x, V.x);
        upd(P.y, G.y, M.y, V.y);
        upd(P.z, G.z, M.z, V.z);
        upd(P.w, G.w, M.w, V.w);
        reinterpret_cast<float4 *>(p)[i] = P;
        reinterpret_cast<float4 *>(m)[i] = M;
        reinterpret_cast<float4 *>(v)[i] = V;
        if (zero_grad) reinterpret_cast<float4 *>(g)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
};

// Adan (Sec. 4.1's optimiser; Algorithm 1 of Xie et al.), betas as weights of the new
// term: with d = g - g_prev, m = (1-b1) m + b1 g, v = (1-b2) v + b2 d,
// n = (1-b3) n + b3 (g + (1-b2) d)^2, p = (p - lr (c1 m + c2 v) / (c3 sqrt(n) + eps)) / (1 + wd lr).
// Algorithm 1: c1 = 1, c2 = 1-b2, c3 = 1, and the first step starts the moments from g
// (f1 = f3 = 1: m = g, v = 0, n = g^2).  Debiased form: moments from zero with d = 0 on the
// first step (f1 = b1, f3 = b3), c1 = 1/(1-(1-b1)^k), c2 = (1-b2)/(1-(1-b2)^k),
// c3 = 1/sqrt(1-(1-b3)^k).  g_prev keeps g.  The first step reads neither the moments nor
// g_prev.
struct AdanOp {
    float *p, *g, *m, *v, *nn, *gp;
    float lr, b1, b2, b3, ib1, ib2, ib3, eps, shrink, c1, c2, c3, f1, f3;
    int first, zero_grad;
    __device__ __forceinline__ void upd(float &pi, float gi, float &mi, float &vi, float &ni, float gpi) const {
        if (first) {
            mi = f1 * gi;
            vi = 0.f;
            ni = f3 * (gi * gi);
        } else {
            const float d = gi - gpi;
            mi = fmaf(ib1, mi, b1 * gi);
            vi = fmaf(ib2, vi, b2 * d);
            const float q = fmaf(ib2, d, gi);
            ni = fmaf(ib3, ni, b3 * q * q);
        }
        pi = (pi - lr * fmaf(c2, vi, c1 * mi) / fmaf(c3, sqrtf(ni), eps)) * shrink;
    }
    __device__ __forceinline__ void one(long long i) const {
        const float gi = g[i];
        float pi = p[i], mi = 0.f, vi = 0.f, ni = 0.f, gpi = 0.f;
        if (!first) {
            mi = m[i];
            vi = v[i];
            ni = nn[i];
            gpi = gp[i];
        }
        upd(pi, gi, mi, vi, ni, gpi);
        p[i] = pi;
        m[i] = mi;
        v[i] = vi;
        nn[i] = ni;
        gp[i] = gi;
        if (zero_grad) g[i] = 0.f;
    }
    __device__ __forceinline__ void vec4(long long i) const {
        const float4 G = reinterpret_cast<const float4 *>(g)[i];
        float4 P = reinterpret_cast<float4 *>(p)[i];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 M = z, V = z, N = z, Q = z;
        if (!first) {
            M = reinterpret_cast<float4 *>(m)[i];
            V = reinterpret_cast<float4 *>(v)[i];
            N = reinterpret_cast<float4 *>(nn)[i];
            Q = reinterpret_cast<float4 *>(gp)[i];
        }
        upd(P.x, G.x, M.x, V.x, N.x, Q.x);
        upd(P.y, G.y, M.y, V.y, N.y, Q.y);
        upd(P.z, G.z, M.z, V.z, N.z, Q.z);
        upd(P.w, G.w, M.w, V.w, N.w, Q.w);
        reinterpret_cast<float4 *>(p)[i] = P;
        reinterpret_cast<float4 *>(m)[i] = M;
        reinterpret_cast<float4 *>(v)[i] = V;
        reinterpret_cast<float4 *>(nn)[i] = N;
        reinterpret_cast<float4 *>(gp)[i] = G;
        if (zero_grad) reinterpret_cast<float4 *>(g)[i] = z;
    }
};

template <class Op, bool VEC>
__global__ void __launch_bounds__(256) optim_kernel(Op op, long long n) {
    pdl_prologue();
    elementwise<Op, VEC>(op, n);
}

bool aligned16(std::initializer_list<const void *> ptrs) {
    for (const void *q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) & 15u) return false;
    return true;
}

__global__ void grad2d_debug_kernel(Work w, float *out) {
    pdl_prologue();
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

// acc |= the device error word of the workspace's last render call (one thread).
__global__ void status_or_kernel(const DevHeader *hdr, int *acc) {
    pdl_prologue();
    const unsigned e = *(volatile const unsigned *)&hdr->err;
    if (e) atomicOr(acc, (int)e);
}

int grid_for(long long n, int per_block = 256) {
    long long b = (n + per_block - 1) / per_block;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t launch_l2_loss(const float *image, const float *target, long long n, float scale, float *dL, float *loss,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    launch_pdl(l2_loss_kernel, grid_for(n), 256, 0, s, image, target, n, scale, dL, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                        float bc1, float bc2, int zero_grad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    AdamOp op{p, g, m, v, lr, b1, b2, 1.f - b1, 1.f - b2, eps, 1.f / bc1, 1.f / bc2, zero_grad};
    const int grid = grid_for((n + 3) / 4);
    if (aligned16({p, g, m, v})) launch_pdl(optim_kernel<AdamOp, true>, grid, 256, 0, s, op, n);
    else launch_pdl(optim_kernel<AdamOp, false>, grid, 256, 0, s, op, n);
    return cudaGetLastError();
}

cudaError_t launch_adan(float *p, float *g, float *m, float *v, float *nn, float *g_prev, long long n, float lr,
                        float b1, float b2, float b3, float eps, float wd, long long step, bool debias, int zero_grad,
                        cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    float c1 = 1.f, c2 = 1.f - b2, c3 = 1.f, f1 = 1.f, f3 = 1.f;
    if (debias) {
        const double k = (double)step;
        c1 = (float)(1.0 / (1.0 - std::pow(1.0 - (double)b1, k)));
        c2 = (float)((1.0 - (double)b2) / (1.0 - std::pow(1.0 - (double)b2, k)));
        c3 = (float)(1.0 / std::sqrt(1.0 - std::pow(1.0 - (double)b3, k)));
        f1 = b1;
        f3 = b3;
    }
    AdanOp op{p, g, m, v, nn, g_prev, lr, b1, b2, b3, 1.f - b1, 1.f - b2, 1.f - b3, eps, 1.f / (1.f + wd * lr),
              c1, c2, c3, f1, f3, step == 1 ? 1 : 0, zero_grad};
    const int grid = grid_for((n + 3) / 4);
    if (aligned16({p, g, m, v, nn, g_prev})) launch_pdl(optim_kernel<AdanOp, true>, grid, 256, 0, s, op, n);
    else launch_pdl(optim_kernel<AdanOp, false>, grid, 256, 0, s, op, n);
    return cudaGetLastError();
}

cudaError_t launch_status_or(const void *workspace, int *acc, cudaStream_t s) {
    launch_pdl(status_or_kernel, 1, 1, 0, s, reinterpret_cast<const DevHeader *>(workspace), acc);
    return cudaGetLastError();
}

cudaError_t launch_grad2d_debug(const Work &w, float *out, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    launch_pdl(grad2d_debug_kernel, (w.L.P + 255) / 256, 256, 0, s, w, out);
    return cudaGetLastError();
}

}  // namespace gvk
