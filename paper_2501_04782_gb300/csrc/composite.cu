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
// A block is one tile, two pixels per thread, each warp an 8x8 pixel block so a warp
// covers a compact footprint (more warps skip a Gaussian entirely in the backward).
// Gaussians are staged through shared memory in batches of DEPTH (the stage depth); every
// lane then reads the same staged Gaussian (broadcast).  The forward stops a tile once
// every pixel is done (__syncthreads_and).  The backward keeps per-pixel state in
// registers, recovers T_i = T_{i+1} / (1 - alpha_i) (alpha recomputed bit-identically),
// reduces the nine per-Gaussian gradients of a warp with a transposed shuffle reduction,
// and adds them with one atomic instruction (nine lanes, nine addresses).  Nothing here
// is a dense contraction: no tensor cores.
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

// Thread -> pixels.  A warp owns an 8x8 pixel block of the tile; lane l owns pixel
// (l & 7, l >> 3) of the block and the pixel four rows below it.
template <int TW, int TH>
__device__ __forceinline__ void pixels_of_thread(int t, int &lx, int &ly) {
    constexpr int WX = TW / 8;
    int wq = t >> 5, l = t & 31;
    lx = (wq % WX) * 8 + (l & 7);
    ly = (wq / WX) * 8 + (l >> 3);
}

// Transposed warp reduction of nine values.  At each of the five shuffle levels a lane
// keeps one half of its vector and adds the partner's copy of that half, so the vector
// halves every level (10 -> 5 -> 3 -> 2 -> 1 values, padded) and the nine warp sums end
// up spread over the lanes: 12 shuffles instead of 45 for a plain butterfly.  Returns the
// warp sum of slot `slot` (valid when slot < 9; lanes l and l ^ 1 hold the same slot).
__device__ __forceinline__ float warp_reduce9(const float v[9], int lane, int &slot) {
    const unsigned FULL = 0xffffffffu;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float lo = v[i], up = (i + 5 < 9) ? v[i + 5] : 0.f;
        a[i] = (h4 ? up : lo) + __shfl_xor_sync(FULL, h4 ? lo : up, 16);
    }
    float b[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float lo = a[i], up = (i + 3 < 5) ? a[i + 3] : 0.f;
        b[i] = (h3 ? up : lo) + __shfl_xor_sync(FULL, h3 ? lo : up, 8);
    }
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float lo = b[i], up = (i + 2 < 3) ? b[i + 2] : 0.f;
        c[i] = (h2 ? up : lo) + __shfl_xor_sync(FULL, h2 ? lo : up, 4);
    }
    float d = (h1 ? c[1] : c[0]) + __shfl_xor_sync(FULL, h1 ? c[0] : c[1], 2);
    d += __shfl_xor_sync(FULL, d, 1);
    const int ic = h1 ? 1 : 0;
    const int ib = h2 ? 2 + ic : ic;  // valid < 3
    const int ia = h3 ? 3 + ib : ib;  // valid < 5
    slot = (ib < 3 && ia < 5) ? (h4 ? 5 : 0) + ia : 99;
    return d;
}

// One pixel's front-to-back step over a staged Gaussian (forward).
__device__ __forceinline__ void fwd_pixel(const float4 &a, const float4 &b, float cb, float px, float py, int pos,
                                          float &T, float &c0, float &c1, float &c2, int &last, bool &done,
                                          unsigned &n_comp) {
    if (done) return;
    float dx, dy, G;
    const float alpha = splat_alpha(a.x, a.y, a.z, a.w, b.x, b.y, px, py, dx, dy, G);
    if (alpha < kAlphaMin) return;
    n_comp++;
    const float wgt = __fmul_rn(alpha, T);
    c0 = fmaf(b.z, wgt, c0);
    c1 = fmaf(b.w, wgt, c1);
    c2 = fmaf(cb, wgt, c2);
    T = __fmul_rn(T, __fsub_rn(1.f, alpha));
    last = pos;
    if (T < kTStop) done = true;
}

template <int TW, int TH, int DEPTH>
__global__ void __launch_bounds__(TW *TH / 2) composite_fwd_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                                   float bg2, float *image, float *final_T,
                                                                   int32_t *last_idx) {
    constexpr int NT = TW * TH / 2;
    __shared__ float4 s_a[DEPTH];
    __shared__ float4 s_b[DEPTH];
    __shared__ float s_c[DEPTH];
    __shared__ unsigned s_tile;
    int lx, ly;
    pixels_of_thread<TW, TH>(threadIdx.x, lx, ly);
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
        const int y0 = (int)(lt / fr.tiles_x) * TH + ly, y1 = y0 + 4;
        const bool in0 = x < W && y0 < H, in1 = x < W && y1 < H;
        const float px = (float)x + 0.5f, py0 = (float)y0 + 0.5f, py1 = (float)y1 + 0.5f;
        const uint2 rg = w.ranges[tile];
        float T0 = 1.f, r0 = 0.f, g0 = 0.f, b0 = 0.f, T1 = 1.f, r1 = 0.f, g1 = 0.f, b1 = 0.f;
        int last0 = -1, last1 = -1;
        bool done0 = !in0, done1 = !in1;
        unsigned n_comp = 0;
        for (unsigned start = rg.x; start < rg.y; start += DEPTH) {
            if (__syncthreads_and(done0 && done1)) break;
            const int n = (int)min((unsigned)DEPTH, rg.y - start);
            for (int i = threadIdx.x; i < n; i += NT) {
                const unsigned p = min(ids[start + i], w.L.P - 1u);  // in range unless a wait gave up
                s_a[i] = w.feat0[p];
                s_b[i] = w.feat1[p];
                s_c[i] = w.feat2[p];
            }
            __syncthreads();
            for (int j = 0; j < n && !(done0 && done1); j++) {
                const float4 a = s_a[j], b = s_b[j];
                const float cb = s_c[j];
                const int pos = (int)(start + j);
                fwd_pixel(a, b, cb, px, py0, pos, T0, r0, g0, b0, last0, done0, n_comp);
                fwd_pixel(a, b, cb, px, py1, pos, T1, r1, g1, b1, last1, done1, n_comp);
            }
        }
        // evaluated entries: up to the stop, or the whole list
        unsigned n_eval = 0;
        if (in0) n_eval += (T0 < kTStop) ? (unsigned)(last0 + 1 - (int)rg.x) : rg.y - rg.x;
        if (in1) n_eval += (T1 < kTStop) ? (unsigned)(last1 + 1 - (int)rg.x) : rg.y - rg.x;
        add_work(w.hdr->work, n_eval, n_comp);
        const size_t plane = (size_t)W * H;
        if (in0) {
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y0 * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y0 * W + x;
            image[img] = fmaf(T0, bg0, r0);
            image[img + plane] = fmaf(T0, bg1, g0);
            image[img + 2 * plane] = fmaf(T0, bg2, b0);
            final_T[pix] = T0;
            last_idx[pix] = last0;
        }
        if (in1) {
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y1 * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y1 * W + x;
            image[img] = fmaf(T1, bg0, r1);
            image[img + plane] = fmaf(T1, bg1, g1);
            image[img + 2 * plane] = fmaf(T1, bg2, b1);
            final_T[pix] = T1;
            last_idx[pix] = last1;
        }
        __syncthreads();
    }
}

// Per-pixel replay state of the backward.
struct BwdPixel {
    float px, py;
    float T;               // transmittance behind the current Gaussian
    float g0, g1, g2;      // dL/dC
    float S0, S1, S2;      // colour composited behind the current Gaussian (incl. background)
    int last;
};

// One pixel's back-to-front step over a staged Gaussian: adds its nine screen-space
// gradient contributions (du, dv, dA, dB, dC, do, dr, dg, db) to acc.
__device__ __forceinline__ bool bwd_pixel(const float4 &a, const float4 &b, float cb, int pos, BwdPixel &q,
                                          float acc[9]) {
    if (pos > q.last) return false;
    float dx, dy, G;
    const float alpha = splat_alpha(a.x, a.y, a.z, a.w, b.x, b.y, q.px, q.py, dx, dy, G);
    if (alpha < kAlphaMin) return false;
    const float ra = __frcp_rn(__fsub_rn(1.f, alpha));
    const float Tin = q.T * ra;
    const float wgt = alpha * Tin;
    acc[6] = fmaf(wgt, q.g0, acc[6]);
    acc[7] = fmaf(wgt, q.g1, acc[7]);
    acc[8] = fmaf(wgt, q.g2, acc[8]);
    const float dal = q.g0 * (b.z * Tin - q.S0 * ra) + q.g1 * (b.w * Tin - q.S1 * ra) + q.g2 * (cb * Tin - q.S2 * ra);
    q.S0 = fmaf(b.z, wgt, q.S0);
    q.S1 = fmaf(b.w, wgt, q.S1);
    q.S2 = fmaf(cb, wgt, q.S2);
    q.T = Tin;
    if (__fmul_rn(b.y, G) < kAlphaMax) {
        acc[5] = fmaf(dal, G, acc[5]);
        const float dpow = -dal * alpha;
        const float hp = 0.5f * dpow;
        acc[2] = fmaf(hp * dx, dx, acc[2]);
        acc[3] = fmaf(dpow * dx, dy, acc[3]);
        acc[4] = fmaf(hp * dy, dy, acc[4]);
        acc[0] = fmaf(dpow, a.z * dx + a.w * dy, acc[0]);
        acc[1] = fmaf(dpow, a.w * dx + b.x * dy, acc[1]);
    }
    return true;
}

template <int TW, int TH, int DEPTH>
__global__ void __launch_bounds__(TW *TH / 2) composite_bwd_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                                   float bg2, const float *final_T,
                                                                   const int32_t *last_idx, const float *dL) {
    constexpr int NT = TW * TH / 2;
    __shared__ float4 s_a[DEPTH];
    __shared__ float4 s_b[DEPTH];
    __shared__ float s_c[DEPTH];
    __shared__ unsigned s_p[DEPTH];
    __shared__ unsigned s_tile;
    __shared__ int s_max;
    int lx, ly;
    pixels_of_thread<TW, TH>(threadIdx.x, lx, ly);
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
        const int ybase = (int)(lt / fr.tiles_x) * TH + ly;
        const uint2 rg = w.ranges[tile];
        BwdPixel q[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int y = ybase + 4 * k;
            q[k].px = (float)x + 0.5f;
            q[k].py = (float)y + 0.5f;
            q[k].T = 1.f;
            q[k].g0 = q[k].g1 = q[k].g2 = 0.f;
            q[k].last = -1;
            if (x < W && y < H) {
                const size_t plane = (size_t)W * H;
                const size_t pix = (size_t)fr.pixel_offset + (size_t)y * W + x;
                const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y * W + x;
                q[k].T = final_T[pix];
                q[k].last = min(last_idx[pix], (int)rg.y - 1);  // from the forward: in [rg.x, rg.y)
                q[k].g0 = dL[img];
                q[k].g1 = dL[img + plane];
                q[k].g2 = dL[img + 2 * plane];
            }
            q[k].S0 = q[k].T * bg0;
            q[k].S1 = q[k].T * bg1;
            q[k].S2 = q[k].T * bg2;
        }
        unsigned n_comp = 0;
        unsigned n_eval = 0;
#pragma unroll
        for (int k = 0; k < 2; k++)
            if (q[k].last >= (int)rg.x) n_eval += (unsigned)(q[k].last + 1 - (int)rg.x);
        const int wmax = __reduce_max_sync(0xffffffffu, max(q[0].last, q[1].last));
        if (lane == 0) atomicMax(&s_max, wmax);
        __syncthreads();
        const int end = min(s_max + 1, (int)rg.y);
        const int wlast = wmax;  // this warp's last position: earlier entries only
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
            const int jtop = min(n - 1, wlast - bstart);
            for (int j = jtop; j >= 0; j--) {
                const float4 a = s_a[j], b = s_b[j];
                const float cb = s_c[j];
                const int pos = bstart + j;
                float acc[9];
#pragma unroll
                for (int k = 0; k < 9; k++) acc[k] = 0.f;
                const bool c0 = bwd_pixel(a, b, cb, pos, q[0], acc);
                const bool c1 = bwd_pixel(a, b, cb, pos, q[1], acc);
                n_comp += (unsigned)c0 + (unsigned)c1;
                if (!__any_sync(0xffffffffu, c0 || c1)) continue;
                int slot;
                const float sum = warp_reduce9(acc, lane, slot);
                if (slot < 9 && !(lane & 1)) {
                    const unsigned p = s_p[j];
                    float *dst = slot < 4 ? &w.g0[p].x + slot : (slot < 8 ? &w.g1[p].x + (slot - 4) : w.g2 + p);
                    atomicAdd(dst, sum);
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
    if (!blocks) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_fwd_kernel<TW, TH, DEPTH>, TW * TH / 2, 0);
    return blocks > 0 ? blocks : 1;
}

template <int TW, int TH, int DEPTH>
int occupancy_bwd() {
    static int blocks = 0;
    if (!blocks) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_bwd_kernel<TW, TH, DEPTH>, TW * TH / 2, 0);
    return blocks > 0 ? blocks : 1;
}

template <int TW, int TH, int DEPTH>
cudaError_t run_fwd(const Work &w, const unsigned *ids, float bg0, float bg1, float bg2, float *image, float *T,
                    int32_t *idx, int num_sms, cudaStream_t s) {
    unsigned grid = min(w.L.tiles, (unsigned)(num_sms * occupancy_fwd<TW, TH, DEPTH>()));
    if (grid == 0) return cudaSuccess;
    composite_fwd_kernel<TW, TH, DEPTH><<<grid, TW * TH / 2, 0, s>>>(w, ids, bg0, bg1, bg2, image, T, idx);
    return cudaGetLastError();
}

template <int TW, int TH, int DEPTH>
cudaError_t run_bwd(const Work &w, const unsigned *ids, float bg0, float bg1, float bg2, const float *T,
                    const int32_t *idx, const float *dL, int num_sms, cudaStream_t s) {
    unsigned grid = min(w.L.tiles, (unsigned)(num_sms * occupancy_bwd<TW, TH, DEPTH>()));
    if (grid == 0) return cudaSuccess;
    composite_bwd_kernel<TW, TH, DEPTH><<<grid, TW * TH / 2, 0, s>>>(w, ids, bg0, bg1, bg2, T, idx, dL);
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
