// composite.cu -- per-tile front-to-back alpha compositing (forward) and its back-to-front
// replay (backward).
//
// Sec. 3.1: the projected Gaussians are "rasterized onto the observed image planes"; the
// rasterizer is the tile-based alpha compositing of prior 3DGS work: per pixel, over the
// Gaussians in depth order, alpha_i = min(0.99, o_i exp(-power_i)), skipped if below 1/255,
// C += c_i alpha_i T, T *= (1 - alpha_i), stop once T < 1e-4 (after compositing).
//
// Design (GB300): persistent blocks pull tiles from an atomic queue covering every tile of
// every frame of the batch, so uneven frames and uneven tiles balance across the 152 SMs.
// A block is one tile, one thread per pixel, warps laid out as 8x4 pixel blocks so a warp
// covers a compact footprint (more warps skip a Gaussian entirely in the backward).
// Gaussians are staged through shared memory in batches of DEPTH (the stage depth); every
// lane then reads the same staged Gaussian (broadcast).  The forward stops a tile once
// every pixel is done (__syncthreads_and).  The backward keeps per-pixel state in
// registers, recovers T_i = T_{i+1} / (1 - alpha_i) (alpha recomputed bit-identically),
// reduces the nine per-Gaussian gradients of a warp with shuffles, and adds them with one
// lane's vector atomics.  Nothing here is a dense contraction: no tensor cores.
#include "gv_internal.cuh"

namespace gvk {

namespace {

// Work counters: per-warp sums, one 64-bit atomic pair per warp and tile.
__device__ __forceinline__ void add_work(unsigned long long *ctr, unsigned n_eval, unsigned n_comp) {
    unsigned e = __reduce_add_sync(0xffffffffu, n_eval);
    unsigned c = __reduce_add_sync(0xffffffffu, n_comp);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(ctr, (unsigned long long)e);
        atomicAdd(ctr + 1, (unsigned long long)c);
    }
}

template <int TW, int TH>
__device__ __forceinline__ void pixel_of_thread(int t, int &lx, int &ly) {
    constexpr int WX = TW / 8;
    int wq = t >> 5, l = t & 31;
    lx = (wq % WX) * 8 + (l & 7);
    ly = (wq / WX) * 4 + (l >> 3);
}

template <int TW, int TH, int DEPTH>
__global__ void __launch_bounds__(TW *TH) composite_fwd_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                               float bg2, float *image, float *final_T,
                                                               int32_t *last_idx) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_a[DEPTH];
    __shared__ float4 s_b[DEPTH];
    __shared__ float s_c[DEPTH];
    __shared__ unsigned s_tile;
    int lx, ly;
    pixel_of_thread<TW, TH>(threadIdx.x, lx, ly);
    const unsigned ntiles = w.L.tiles;
    const int F = (int)w.L.F;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&w.hdr->queue[0], 1u);
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        const DevFrame &fr = w.frames[find_frame_by_tile(w.frames, F, tile)];
        const int W = fr.W, H = fr.H;
        const unsigned lt = tile - fr.tile_offset;
        const int x = (int)(lt % fr.tiles_x) * TW + lx;
        const int y = (int)(lt / fr.tiles_x) * TH + ly;
        const bool inside = x < W && y < H;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const uint2 rg = w.ranges[tile];
        float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
        int last = -1;
        bool done = !inside;
        unsigned n_eval = 0, n_comp = 0;
        for (unsigned start = rg.x; start < rg.y; start += DEPTH) {
            if (__syncthreads_and(done)) break;
            const int n = (int)min((unsigned)DEPTH, rg.y - start);
            for (int i = threadIdx.x; i < n; i += NT) {
                const unsigned p = min(ids[start + i], w.L.P - 1u);  // in range unless a wait gave up
                s_a[i] = w.feat0[p];
                s_b[i] = w.feat1[p];
                s_c[i] = w.feat2[p];
            }
            __syncthreads();
            if (!done) {
                int j = 0;
                for (; j < n; j++) {
                    const float4 a = s_a[j], b = s_b[j];
                    float dx, dy, G;
                    const float alpha = splat_alpha(a.x, a.y, a.z, a.w, b.x, b.y, px, py, dx, dy, G);
                    if (alpha < kAlphaMin) continue;
                    n_comp++;
                    const float wgt = __fmul_rn(alpha, T);
                    c0 = fmaf(b.z, wgt, c0);
                    c1 = fmaf(b.w, wgt, c1);
                    c2 = fmaf(s_c[j], wgt, c2);
                    T = __fmul_rn(T, __fsub_rn(1.f, alpha));
                    last = (int)(start + j);
                    if (T < kTStop) { done = true; j++; break; }
                }
                n_eval += (unsigned)j;
            }
        }
        add_work(w.hdr->work, n_eval, n_comp);
        if (inside) {
            const size_t plane = (size_t)W * H;
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y * W + x;
            image[img] = fmaf(T, bg0, c0);
            image[img + plane] = fmaf(T, bg1, c1);
            image[img + 2 * plane] = fmaf(T, bg2, c2);
            final_T[pix] = T;
            last_idx[pix] = last;
        }
        __syncthreads();
    }
}

template <int TW, int TH, int DEPTH>
__global__ void __launch_bounds__(TW *TH) composite_bwd_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                               float bg2, const float *final_T,
                                                               const int32_t *last_idx, const float *dL) {
    constexpr int NT = TW * TH;
    __shared__ float4 s_a[DEPTH];
    __shared__ float4 s_b[DEPTH];
    __shared__ float s_c[DEPTH];
    __shared__ unsigned s_p[DEPTH];
    __shared__ unsigned s_tile;
    __shared__ int s_max;
    int lx, ly;
    pixel_of_thread<TW, TH>(threadIdx.x, lx, ly);
    const int lane = threadIdx.x & 31;
    const unsigned ntiles = w.L.tiles;
    const int F = (int)w.L.F;
    for (;;) {
        if (threadIdx.x == 0) { s_tile = atomicAdd(&w.hdr->queue[1], 1u); s_max = -1; }
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        const DevFrame &fr = w.frames[find_frame_by_tile(w.frames, F, tile)];
        const int W = fr.W, H = fr.H;
        const unsigned lt = tile - fr.tile_offset;
        const int x = (int)(lt % fr.tiles_x) * TW + lx;
        const int y = (int)(lt / fr.tiles_x) * TH + ly;
        const bool inside = x < W && y < H;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const uint2 rg = w.ranges[tile];
        float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        int last = -1;
        if (inside) {
            const size_t plane = (size_t)W * H;
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y * W + x;
            T = final_T[pix];
            last = last_idx[pix];
            g0 = dL[img];
            g1 = dL[img + plane];
            g2 = dL[img + 2 * plane];
        }
        float S0 = T * bg0, S1 = T * bg1, S2 = T * bg2;  // colour behind the current Gaussian
        int wmax = __reduce_max_sync(0xffffffffu, last);
        if (lane == 0) atomicMax(&s_max, wmax);
        __syncthreads();
        const int end = min(s_max + 1, (int)rg.y);  // last_idx from the forward lies in [rg.x, rg.y)
        unsigned n_comp = 0;
        const unsigned n_eval = (last >= (int)rg.x) ? (unsigned)(min(last + 1, (int)rg.y) - (int)rg.x) : 0u;
        for (int bend = end; bend > (int)rg.x; bend -= DEPTH) {
            const int bstart = max((int)rg.x, bend - DEPTH);
            const int n = bend - bstart;
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += NT) {
                const unsigned p = min(ids[bstart + i], w.L.P - 1u);
                s_p[i] = p;
                s_a[i] = w.feat0[p];
                s_b[i] = w.feat1[p];
                s_c[i] = w.feat2[p];
            }
            __syncthreads();
            for (int j = n - 1; j >= 0; j--) {
                const int pos = bstart + j;
                float du = 0.f, dv = 0.f, dA = 0.f, dB = 0.f, dC = 0.f, dop = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
                bool contrib = false;
                if (pos <= last) {
                    const float4 a = s_a[j], b = s_b[j];
                    const float cb = s_c[j];
                    float dx, dy, G;
                    const float alpha = splat_alpha(a.x, a.y, a.z, a.w, b.x, b.y, px, py, dx, dy, G);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        n_comp++;
                        const float ra = __frcp_rn(__fsub_rn(1.f, alpha));
                        const float Tin = T * ra;
                        const float wgt = alpha * Tin;
                        dr = wgt * g0;
                        dg = wgt * g1;
                        db = wgt * g2;
                        const float dal = g0 * (b.z * Tin - S0 * ra) + g1 * (b.w * Tin - S1 * ra) +
                                          g2 * (cb * Tin - S2 * ra);
                        S0 = fmaf(b.z, wgt, S0);
                        S1 = fmaf(b.w, wgt, S1);
                        S2 = fmaf(cb, wgt, S2);
                        T = Tin;
                        if (__fmul_rn(b.y, G) < kAlphaMax) {
                            dop = dal * G;
                            const float dpow = -dal * alpha;
                            dA = 0.5f * dpow * dx * dx;
                            dB = dpow * dx * dy;
                            dC = 0.5f * dpow * dy * dy;
                            du = dpow * (a.z * dx + a.w * dy);
                            dv = dpow * (a.w * dx + b.x * dy);
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        du += __shfl_xor_sync(0xffffffffu, du, o);
                        dv += __shfl_xor_sync(0xffffffffu, dv, o);
                        dA += __shfl_xor_sync(0xffffffffu, dA, o);
                        dB += __shfl_xor_sync(0xffffffffu, dB, o);
                        dC += __shfl_xor_sync(0xffffffffu, dC, o);
                        dop += __shfl_xor_sync(0xffffffffu, dop, o);
                        dr += __shfl_xor_sync(0xffffffffu, dr, o);
                        dg += __shfl_xor_sync(0xffffffffu, dg, o);
                        db += __shfl_xor_sync(0xffffffffu, db, o);
                    }
                    if (lane == 0) {
                        const unsigned p = s_p[j];
                        atomicAdd(w.g0 + p, make_float4(du, dv, dA, dB));
                        atomicAdd(w.g1 + p, make_float4(dC, dop, dr, dg));
                        atomicAdd(w.g2 + p, db);
                    }
                }
            }
        }
        add_work(w.hdr->work + 2, n_eval, n_comp);
        __syncthreads();
    }
}

template <int TW, int TH, int DEPTH>
int occupancy_fwd() {
    static int blocks = 0;
    if (!blocks) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_fwd_kernel<TW, TH, DEPTH>, TW * TH, 0);
    return blocks > 0 ? blocks : 1;
}

template <int TW, int TH, int DEPTH>
int occupancy_bwd() {
    static int blocks = 0;
    if (!blocks) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_bwd_kernel<TW, TH, DEPTH>, TW * TH, 0);
    return blocks > 0 ? blocks : 1;
}

template <int TW, int TH, int DEPTH>
cudaError_t run_fwd(const Work &w, const unsigned *ids, float bg0, float bg1, float bg2, float *image, float *T,
                    int32_t *idx, int num_sms, cudaStream_t s) {
    unsigned grid = min(w.L.tiles, (unsigned)(num_sms * occupancy_fwd<TW, TH, DEPTH>()));
    if (grid == 0) return cudaSuccess;
    composite_fwd_kernel<TW, TH, DEPTH><<<grid, TW * TH, 0, s>>>(w, ids, bg0, bg1, bg2, image, T, idx);
    return cudaGetLastError();
}

template <int TW, int TH, int DEPTH>
cudaError_t run_bwd(const Work &w, const unsigned *ids, float bg0, float bg1, float bg2, const float *T,
                    const int32_t *idx, const float *dL, int num_sms, cudaStream_t s) {
    unsigned grid = min(w.L.tiles, (unsigned)(num_sms * occupancy_bwd<TW, TH, DEPTH>()));
    if (grid == 0) return cudaSuccess;
    composite_bwd_kernel<TW, TH, DEPTH><<<grid, TW * TH, 0, s>>>(w, ids, bg0, bg1, bg2, T, idx, dL);
    return cudaGetLastError();
}

#define GV_DISPATCH(FN, ...)                                                                     \
    switch (tile_w * 1000 + tile_h) {                                                            \
        case 8008:                                                                               \
            switch (depth) {                                                                     \
                case 32: return FN<8, 8, 32>(__VA_ARGS__);                                       \
                case 64: return FN<8, 8, 64>(__VA_ARGS__);                                       \
                case 128: return FN<8, 8, 128>(__VA_ARGS__);                                     \
                case 256: return FN<8, 8, 256>(__VA_ARGS__);                                     \
            }                                                                                    \
            break;                                                                               \
        case 16008:                                                                              \
            switch (depth) {                                                                     \
                case 32: return FN<16, 8, 32>(__VA_ARGS__);                                      \
                case 64: return FN<16, 8, 64>(__VA_ARGS__);                                      \
                case 128: return FN<16, 8, 128>(__VA_ARGS__);                                    \
                case 256: return FN<16, 8, 256>(__VA_ARGS__);                                    \
            }                                                                                    \
            break;                                                                               \
        case 16016:                                                                              \
            switch (depth) {                                                                     \
                case 32: return FN<16, 16, 32>(__VA_ARGS__);                                     \
                case 64: return FN<16, 16, 64>(__VA_ARGS__);                                     \
                case 128: return FN<16, 16, 128>(__VA_ARGS__);                                   \
                case 256: return FN<16, 16, 256>(__VA_ARGS__);                                   \
            }                                                                                    \
            break;                                                                               \
    }                                                                                            \
    return cudaErrorInvalidValue;

}  // namespace

cudaError_t launch_composite_fwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf, float bg0,
                                 float bg1, float bg2, float *image, float *final_T, int32_t *last_idx,
                                 int num_sms, cudaStream_t s) {
    const unsigned *ids = w.tval[tile_buf];
    GV_DISPATCH(run_fwd, w, ids, bg0, bg1, bg2, image, final_T, last_idx, num_sms, s)
}

cudaError_t launch_composite_bwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf, float bg0,
                                 float bg1, float bg2, const float *final_T, const int32_t *last_idx,
                                 const float *dL_dimage, int num_sms, cudaStream_t s) {
    const unsigned *ids = w.tval[tile_buf];
    GV_DISPATCH(run_bwd, w, ids, bg0, bg1, bg2, final_T, last_idx, dL_dimage, num_sms, s)
}

}  // namespace gvk
