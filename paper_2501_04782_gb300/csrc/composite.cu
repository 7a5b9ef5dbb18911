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
// A block is one tile.  The forward runs two pixels per thread, each warp an 8x8 pixel
// block (a compact footprint: the warp stops early), or four on 32x32 tiles; the backward
// runs four pixels of one column per thread on tiles 16 or 32 wide (8x16 or 16x8 per
// warp), two on 8x8 tiles.
// Gaussians are staged through shared memory in batches of DEPTH (the stage depth); every
// lane then reads the same staged Gaussian (broadcast).  The backward double-buffers its
// stages: the next stage's records arrive by cp.async while one is replayed.  The forward takes two Gaussians
// per round; a pixel's cutoff test compares alpha with a per-pixel threshold (1/255, or 2
// once the pixel is done), so the stop rule costs no extra test per Gaussian; a warp
// leaves the tile once all its pixels are done and a block once every pixel is
// (__syncthreads_and).  The backward keeps per-pixel state in registers, recovers
// T_i = T_{i+1} / (1 - alpha_i) (alpha recomputed bit-identically), reduces the nine
// per-Gaussian gradients of a warp with a transposed shuffle reduction and adds them with
// one atomic instruction (nine lanes, nine addresses), or, when few lanes contribute, adds
// each lane's values directly.  Nothing here is a dense contraction: no tensor cores.
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

// A replayed Gaussian with at most this many lanes of the warp contributing adds each
// lane's nine values with its own atomics; denser ones go through warp_reduce9 (one
// atomic per value).  Many lanes adding to one address contend, so the direct path
// is for sparse warps only.
constexpr int kSparseLanes = 8;

// A block leaving the persistent loop counts itself done; the last one resets the work
// queue and the done count, so the next launch on this workspace starts from zero.
__device__ __forceinline__ void queue_done(unsigned *queue, unsigned *done) {
    if (threadIdx.x == 0 && atomicAdd(done, 1u) == gridDim.x - 1) {
        *queue = 0u;
        *done = 0u;
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

// Thread -> pixels: PX pixels per lane, all in one column, so the Gaussian's dx and the
// terms that depend on it alone are shared.  A warp owns a block WBW pixels wide: lane l
// takes column l % WBW and rows l / WBW + RS k (k < PX), RS = 32 / WBW.  Four pixels per
// lane halve the per-pixel cost of a staged Gaussian's loads and, in the backward, of the
// warp reductions and atomics, against two.
template <int TW, int TH, int PX>
struct PixMap {
    static constexpr int WBW = (PX == 4 && TH < 16) ? 16 : 8;
    static constexpr int RS = 32 / WBW;
    static constexpr int WBH = RS * PX;
    static constexpr int WX = TW / WBW;
    static constexpr int NT = TW * TH / PX;
    static_assert(TW % WBW == 0 && TH % WBH == 0, "tile not covered by whole warps");
};

// Double-buffered stages of a tile's list (the backward's).  The ids of a stage are
// copied two stages ahead and its Gaussians' records one stage ahead (cp.async), so the
// replay of one stage overlaps the loads of the next two.  Thread t copies entries t,
// t + NT, ... of both, so it reads back only id slots it copied itself (its own cp.async
// wait suffices); the records need the block barrier.
template <int NT>
__device__ __forceinline__ void stage_copy_ids(unsigned *slot, const unsigned *ids, unsigned first, int n) {
    for (int i = threadIdx.x; i < n; i += NT) cp_async4(slot + i, ids + first + i);
}

template <int NT>
__device__ __forceinline__ void stage_copy_records(const Work &w, const unsigned *slot, int n, float4 *a, float4 *b,
                                                   float *c, unsigned *pair) {
    for (int i = threadIdx.x; i < n; i += NT) {
        const unsigned p = min(slot[i], w.L.P - 1u);  // in range unless a wait gave up
        if (pair) pair[i] = p;
        cp_async16(a + i, w.feat0 + p);
        cp_async16(b + i, w.feat1 + p);
        cp_async4(c + i, w.feat2 + p);
    }
}

// One pixel's colour out of the forward, and with a loss target its L2 terms: dL =
// 2 scale (c - target) per channel, the squared differences added to acc.
__device__ __forceinline__ void write_pixel(float *image, size_t img, size_t plane, float c0, float c1, float c2,
                                            const LossArgs &ls, float &acc) {
    image[img] = c0;
    image[img + plane] = c1;
    image[img + 2 * plane] = c2;
    if (ls.target) {
        const float d0 = c0 - ls.target[img], d1 = c1 - ls.target[img + plane], d2 = c2 - ls.target[img + 2 * plane];
        if (ls.dL) {
            const float two_s = 2.f * ls.scale;
            ls.dL[img] = two_s * d0;
            ls.dL[img + plane] = two_s * d1;
            ls.dL[img + 2 * plane] = two_s * d2;
        }
        acc = fmaf(d0, d0, acc);
        acc = fmaf(d1, d1, acc);
        acc = fmaf(d2, d2, acc);
    }
}

// The block's loss terms into *loss (scaled), one atomic per block; every thread calls it.
template <int NT>
__device__ __forceinline__ void flush_loss(const LossArgs &ls, float acc) {
    if (!ls.target || !ls.loss) return;
    __shared__ float s_l[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_l[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < NT / 32; i++) t += s_l[i];
        atomicAdd(ls.loss, ls.scale * t);
    }
}

template <int TW, int TH, int DEPTH>
__global__ void __launch_bounds__(TW *TH / 2) composite_fwd_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                                   float bg2, float *image, float *final_T,
                                                                   int32_t *last_idx, LossArgs ls) {
    pdl_prologue();
    constexpr int NT = TW * TH / 2;
    __shared__ float4 s_a[DEPTH + 1];
    __shared__ float4 s_b[DEPTH + 1];
    __shared__ float s_c[DEPTH + 1];
    __shared__ unsigned s_tile;
    int lx, ly;
    pixels_of_thread<TW, TH>(threadIdx.x, lx, ly);
    const unsigned ntiles = w.L.tiles;
    const int F = (int)w.L.F;
    const bool failed = w.hdr->err != 0u;  // lists incomplete: every tile renders empty
    float lacc = 0.f;  // this thread's squared loss terms
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&w.hdr->queue[0], 1u);
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) {
            queue_done(w.hdr->queue + 0, w.hdr->queue + 2);
            break;
        }
        const DevFrame &fr = w.frames[find_frame_by_tile(w.frames, F, tile)];
        const int W = fr.W, H = fr.H;
        const unsigned lt = tile - fr.tile_offset;
        const int x = (int)(lt % fr.tiles_x) * TW + lx;
        const int y0 = (int)(lt / fr.tiles_x) * TH + ly, y1 = y0 + 4;
        const bool in0 = x < W && y0 < H, in1 = x < W && y1 < H;
        const float px = (float)x + 0.5f;
        const float2 npy = make_float2(-((float)y0 + 0.5f), -((float)y1 + 0.5f));
        uint2 rg = failed ? make_uint2(0u, 0u) : w.ranges[tile];
        if (rg.x >= rg.y) rg = make_uint2(0u, 0u);  // an empty tile (no key recorded a range)
        float2 T = make_float2(1.f, 1.f), cr = make_float2(0.f, 0.f), cg = cr, cb = cr;
        int last0 = -1, last1 = -1;
        // per-pixel alpha threshold: 1/255, or 2 (above any alpha) once the pixel is done
        float2 thr = make_float2(in0 ? kAlphaMin : 2.f, in1 ? kAlphaMin : 2.f);
        for (unsigned start = rg.x; start < rg.y; start += DEPTH) {
            if (__syncthreads_and(thr.x > 1.f && thr.y > 1.f)) break;
            const int n = (int)min((unsigned)DEPTH, rg.y - start);
            for (int i = threadIdx.x; i < n; i += NT) {
                const unsigned p = min(ids[start + i], w.L.P - 1u);  // in range unless a wait gave up
                s_a[i] = w.feat0[p];
                s_b[i] = w.feat1[p];
                s_c[i] = w.feat2[p];
            }
            if (threadIdx.x == 0 && (n & 1)) {  // pad to pairs: a Gaussian of opacity 0 (2^-inf)
                s_a[n] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_b[n] = make_float4(0.f, -__int_as_float(0x7f800000), 0.f, 0.f);
                s_c[n] = 0.f;
            }
            __syncthreads();
            // two staged Gaussians per round: their exponents are independent of the pixel
            // state, so both are evaluated before the two (sequential) compositing updates
            for (int j = 0; j < n; j += 2) {
                if (!__any_sync(0xffffffffu, thr.x < 1.f || thr.y < 1.f)) break;
                const float4 fa0 = s_a[j], fa1 = s_b[j];
                const float4 fb0 = s_a[j + 1], fb1 = s_b[j + 1];
                float dxa, dxb;
                float2 dya, dyb;
                const float2 ea = splat_exponent2(fa0, fa1, px, npy, dxa, dya);
                const float2 eb = splat_exponent2(fb0, fb1, px, npy, dxb, dyb);
                const float2 ra = make_float2(fminf(ex2_approx(ea.x), kAlphaMax), fminf(ex2_approx(ea.y), kAlphaMax));
                const float2 rb = make_float2(fminf(ex2_approx(eb.x), kAlphaMax), fminf(ex2_approx(eb.y), kAlphaMax));
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    const float2 rr = k ? rb : ra;
                    const float4 f1 = k ? fb1 : fa1;
                    // a pixel that is done, or below the cutoff, takes alpha 0: T and colour unchanged
                    const bool c0 = rr.x >= thr.x, c1 = rr.y >= thr.y;
                    if (!__any_sync(0xffffffffu, c0 || c1)) continue;  // no lane composites it
                    const float a0 = c0 ? rr.x : 0.f, a1 = c1 ? rr.y : 0.f;
                    const float2 wg = __fmul2_rn(make_float2(a0, a1), T);
                    cr = __ffma2_rn(dup2(f1.z), wg, cr);
                    cg = __ffma2_rn(dup2(f1.w), wg, cg);
                    cb = __ffma2_rn(dup2(s_c[j + k]), wg, cb);
                    T = __fmul2_rn(T, __fadd2_rn(make_float2(1.f, 1.f), make_float2(-a0, -a1)));
                    const int pos = (int)(start + j + k);
                    if (c0) { last0 = pos; if (T.x < kTStop) thr.x = 2.f; }
                    if (c1) { last1 = pos; if (T.y < kTStop) thr.y = 2.f; }
                }
            }
        }
        // evaluated entries: up to the stop, or the whole list (composited pairs are
        // counted by the backward, which replays exactly those)
        unsigned n_eval = 0;
        if (in0) n_eval += (T.x < kTStop) ? (unsigned)(last0 + 1 - (int)rg.x) : rg.y - rg.x;
        if (in1) n_eval += (T.y < kTStop) ? (unsigned)(last1 + 1 - (int)rg.x) : rg.y - rg.x;
        add_work(w.hdr->work, n_eval, 0u);
        const size_t plane = (size_t)W * H;
        if (in0) {
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y0 * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y0 * W + x;
            write_pixel(image, img, plane, fmaf(T.x, bg0, cr.x), fmaf(T.x, bg1, cg.x), fmaf(T.x, bg2, cb.x), ls,
                        lacc);
            final_T[pix] = T.x;
            last_idx[pix] = last0;
        }
        if (in1) {
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y1 * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y1 * W + x;
            write_pixel(image, img, plane, fmaf(T.y, bg0, cr.y), fmaf(T.y, bg1, cg.y), fmaf(T.y, bg2, cb.y), ls,
                        lacc);
            final_T[pix] = T.y;
            last_idx[pix] = last1;
        }
        __syncthreads();
    }
    flush_loss<NT>(ls, lacc);
}

// The forward with PX (four) pixels per lane; same arithmetic and decisions as
// composite_fwd_kernel, pixel by pixel.
template <int TW, int TH, int DEPTH, int PX>
__global__ void __launch_bounds__(TW *TH / PX) composite_fwd4_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                                     float bg2, float *image, float *final_T,
                                                                     int32_t *last_idx, LossArgs ls) {
    pdl_prologue();
    using M = PixMap<TW, TH, PX>;
    constexpr int NT = M::NT, NP = PX / 2;
    __shared__ float4 s_a[DEPTH + 1];
    __shared__ float4 s_b[DEPTH + 1];
    __shared__ float s_c[DEPTH + 1];
    __shared__ unsigned s_tile;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int lx = (wq % M::WX) * M::WBW + lane % M::WBW;
    const int ly = (wq / M::WX) * M::WBH + lane / M::WBW;
    const unsigned ntiles = w.L.tiles;
    const int F = (int)w.L.F;
    const bool failed = w.hdr->err != 0u;  // lists incomplete: every tile renders empty
    float lacc = 0.f;  // this thread's squared loss terms
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&w.hdr->queue[0], 1u);
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) {
            queue_done(w.hdr->queue + 0, w.hdr->queue + 2);
            break;
        }
        const DevFrame &fr = w.frames[find_frame_by_tile(w.frames, F, tile)];
        const int W = fr.W, H = fr.H;
        const unsigned lt = tile - fr.tile_offset;
        const int x = (int)(lt % fr.tiles_x) * TW + lx;
        const int ybase = (int)(lt / fr.tiles_x) * TH + ly;
        const float px = (float)x + 0.5f;
        uint2 rg = failed ? make_uint2(0u, 0u) : w.ranges[tile];
        if (rg.x >= rg.y) rg = make_uint2(0u, 0u);  // an empty tile (no key recorded a range)
        // pixel 2k + h of the thread is row ybase + RS (2k + h); packed over pixel pairs
        float2 npy[NP], T[NP], cr[NP], cg[NP], cb[NP], thr[NP];
        int last[PX];
#pragma unroll
        for (int k = 0; k < NP; k++) {
            const int ya = ybase + M::RS * (2 * k), yb = ya + M::RS;
            npy[k] = make_float2(-((float)ya + 0.5f), -((float)yb + 0.5f));
            T[k] = make_float2(1.f, 1.f);
            cr[k] = cg[k] = cb[k] = make_float2(0.f, 0.f);
            // per-pixel alpha threshold: 1/255, or 2 (above any alpha) once the pixel is done
            thr[k] = make_float2(x < W && ya < H ? kAlphaMin : 2.f, x < W && yb < H ? kAlphaMin : 2.f);
            last[2 * k] = last[2 * k + 1] = -1;
        }
        auto live = [&]() {
            bool a = false;
#pragma unroll
            for (int k = 0; k < NP; k++) a = a || thr[k].x < 1.f || thr[k].y < 1.f;
            return a;
        };
        for (unsigned start = rg.x; start < rg.y; start += DEPTH) {
            if (__syncthreads_and(!live())) break;
            const int n = (int)min((unsigned)DEPTH, rg.y - start);
            for (int i = threadIdx.x; i < n; i += NT) {
                const unsigned p = min(ids[start + i], w.L.P - 1u);  // in range unless a wait gave up
                s_a[i] = w.feat0[p];
                s_b[i] = w.feat1[p];
                s_c[i] = w.feat2[p];
            }
            if (threadIdx.x == 0 && (n & 1)) {  // pad to pairs: a Gaussian of opacity 0 (2^-inf)
                s_a[n] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_b[n] = make_float4(0.f, -__int_as_float(0x7f800000), 0.f, 0.f);
                s_c[n] = 0.f;
            }
            __syncthreads();
            // two staged Gaussians per round: their exponents are independent of the pixel
            // state, so both are evaluated before the two (sequential) compositing updates
            for (int j = 0; j < n; j += 2) {
                if (!__any_sync(0xffffffffu, live())) break;
                float2 rr[2][NP];
                float4 f1s[2];
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    const float4 f0 = s_a[j + g], f1 = s_b[j + g];
                    f1s[g] = f1;
                    // e = a' dx^2 + b' dx dy + c' dy^2 + log2 o, rounded as the backward's
                    const float dx = __fsub_rn(f0.x, px);
                    const float s0 = __fmaf_rn(__fmul_rn(f0.z, dx), dx, f1.y);
                    const float bdx = __fmul_rn(f0.w, dx);
#pragma unroll
                    for (int k = 0; k < NP; k++) {
                        const float2 dy = __fadd2_rn(dup2(f0.y), npy[k]);
                        const float2 t = __ffma2_rn(dup2(bdx), dy, dup2(s0));
                        const float2 e = __ffma2_rn(__fmul2_rn(dup2(f1.x), dy), dy, t);
                        rr[g][k] = make_float2(fminf(ex2_approx(e.x), kAlphaMax), fminf(ex2_approx(e.y), kAlphaMax));
                    }
                }
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    const float4 f1 = f1s[g];
                    // a pixel that is done, or below the cutoff, takes alpha 0: T and colour unchanged
                    bool c[PX], any = false;
#pragma unroll
                    for (int k = 0; k < NP; k++) {
                        c[2 * k] = rr[g][k].x >= thr[k].x;
                        c[2 * k + 1] = rr[g][k].y >= thr[k].y;
                        any = any || c[2 * k] || c[2 * k + 1];
                    }
                    if (!__any_sync(0xffffffffu, any)) continue;  // no lane composites it
                    const float cbg = s_c[j + g];
                    const int pos = (int)(start + j + g);
#pragma unroll
                    for (int k = 0; k < NP; k++) {
                        const float a0 = c[2 * k] ? rr[g][k].x : 0.f, a1 = c[2 * k + 1] ? rr[g][k].y : 0.f;
                        const float2 wg = __fmul2_rn(make_float2(a0, a1), T[k]);
                        cr[k] = __ffma2_rn(dup2(f1.z), wg, cr[k]);
                        cg[k] = __ffma2_rn(dup2(f1.w), wg, cg[k]);
                        cb[k] = __ffma2_rn(dup2(cbg), wg, cb[k]);
                        T[k] = __fmul2_rn(T[k], __fadd2_rn(make_float2(1.f, 1.f), make_float2(-a0, -a1)));
                        if (c[2 * k]) { last[2 * k] = pos; if (T[k].x < kTStop) thr[k].x = 2.f; }
                        if (c[2 * k + 1]) { last[2 * k + 1] = pos; if (T[k].y < kTStop) thr[k].y = 2.f; }
                    }
                }
            }
        }
        // evaluated entries: up to the stop, or the whole list (composited pairs are
        // counted by the backward, which replays exactly those)
        unsigned n_eval = 0;
        const size_t plane = (size_t)W * H;
#pragma unroll
        for (int q = 0; q < PX; q++) {
            const int y = ybase + M::RS * q;
            if (!(x < W && y < H)) continue;
            const float Tq = (q & 1) ? T[q >> 1].y : T[q >> 1].x;
            const float rq = (q & 1) ? cr[q >> 1].y : cr[q >> 1].x;
            const float gq = (q & 1) ? cg[q >> 1].y : cg[q >> 1].x;
            const float bq = (q & 1) ? cb[q >> 1].y : cb[q >> 1].x;
            n_eval += (Tq < kTStop) ? (unsigned)(last[q] + 1 - (int)rg.x) : rg.y - rg.x;
            const size_t pix = (size_t)fr.pixel_offset + (size_t)y * W + x;
            const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y * W + x;
            write_pixel(image, img, plane, fmaf(Tq, bg0, rq), fmaf(Tq, bg1, gq), fmaf(Tq, bg2, bq), ls, lacc);
            final_T[pix] = Tq;
            last_idx[pix] = last[q];
        }
        add_work(w.hdr->work, n_eval, 0u);
        __syncthreads();
    }
    flush_loss<NT>(ls, lacc);
}

// Pixels per lane of the forward for a tile shape (measured: four on 32x32 tiles, 17 %
// faster on 8 x 1920x1080 / 1M; two elsewhere, where a warp's 8x8 block stops earlier
// than an 8x16 one: four were 12-14 % slower at 960x540 / 200k).
template <int TW, int TH>
constexpr int fwd_px() { return TH >= 32 ? 4 : 2; }

// COUNT: also count the replayed (composited) pairs into work[3] (only while per-stage
// profiling is on: the count costs instructions in the inner loop).
template <int TW, int TH, int DEPTH, int PX, bool COUNT>
__global__ void __launch_bounds__(TW *TH / PX) composite_bwd_kernel(Work w, const unsigned *ids, float bg0, float bg1,
                                                                    float bg2, const float *final_T,
                                                                    const int32_t *last_idx, const float *dL) {
    pdl_prologue();
    using M = PixMap<TW, TH, PX>;
    constexpr int NT = M::NT, NP = PX / 2;
    // two stage buffers: the copies of the next stage land while this one is replayed
    __shared__ float4 s_a[2][DEPTH];
    __shared__ float4 s_b[2][DEPTH];
    __shared__ float s_c[2][DEPTH];
    __shared__ unsigned s_p[2][DEPTH];
    __shared__ unsigned s_id[2][DEPTH];
    __shared__ unsigned s_tile;
    __shared__ int s_max;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int lx = (wq % M::WX) * M::WBW + lane % M::WBW;
    const int ly = (wq / M::WX) * M::WBH + lane / M::WBW;
    const unsigned ntiles = w.L.tiles;
    const int F = (int)w.L.F;
    const bool failed = w.hdr->err != 0u;  // lists incomplete: every tile renders empty
    for (;;) {
        if (threadIdx.x == 0) { s_tile = atomicAdd(&w.hdr->queue[1], 1u); s_max = -1; }
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) {
            queue_done(w.hdr->queue + 1, w.hdr->queue + 3);
            break;
        }
        const DevFrame &fr = w.frames[find_frame_by_tile(w.frames, F, tile)];
        const int W = fr.W, H = fr.H;
        const unsigned lt = tile - fr.tile_offset;
        const int x = (int)(lt % fr.tiles_x) * TW + lx;
        const int ybase = (int)(lt / fr.tiles_x) * TH + ly;
        const float px = (float)x + 0.5f;
        uint2 rg = failed ? make_uint2(0u, 0u) : w.ranges[tile];
        if (rg.x >= rg.y) rg = make_uint2(0u, 0u);  // an empty tile (no key recorded a range)
        const size_t plane = (size_t)W * H;
        // per-pixel replay state, packed over pixel pairs: pixel 2k + h is row ybase + RS (2k + h)
        float2 npy[NP], T[NP], g0[NP], g1[NP], g2[NP], gS[NP];
        int last[PX];
        unsigned n_comp = 0, n_eval = 0;
        int lmax = -1;
#pragma unroll
        for (int q = 0; q < PX; q++) {
            const int y = ybase + M::RS * q;
            float Tq = 1.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
            int lq = -1;
            if (x < W && y < H) {
                const size_t pix = (size_t)fr.pixel_offset + (size_t)y * W + x;
                const size_t img = 3 * (size_t)fr.pixel_offset + (size_t)y * W + x;
                Tq = final_T[pix];
                lq = min(last_idx[pix], (int)rg.y - 1);  // from the forward: in [rg.x, rg.y)
                d0 = dL[img];
                d1 = dL[img + plane];
                d2 = dL[img + 2 * plane];
            }
            last[q] = lq;
            lmax = max(lmax, lq);
            if (lq >= (int)rg.x) n_eval += (unsigned)(lq + 1 - (int)rg.x);
            const float ny = -((float)y + 0.5f);
            if (q & 1) {
                npy[q >> 1].y = ny; T[q >> 1].y = Tq; g0[q >> 1].y = d0; g1[q >> 1].y = d1; g2[q >> 1].y = d2;
            } else {
                npy[q >> 1].x = ny; T[q >> 1].x = Tq; g0[q >> 1].x = d0; g1[q >> 1].x = d1; g2[q >> 1].x = d2;
            }
        }
#pragma unroll
        for (int k = 0; k < NP; k++) {
            // gS = -(sum_ch g_ch S_ch), S_ch the colour composited behind the current
            // Gaussian (the background term to start with): only its dot product with the
            // pixel's upstream gradient g enters dL/dalpha
            const float2 gbg = __ffma2_rn(g2[k], dup2(bg2), __ffma2_rn(g1[k], dup2(bg1), __fmul2_rn(g0[k], dup2(bg0))));
            gS[k] = __fmul2_rn(T[k], make_float2(-gbg.x, -gbg.y));
        }
        const int wmax = __reduce_max_sync(0xffffffffu, lmax);
        if (lane == 0) atomicMax(&s_max, wmax);
        __syncthreads();
        const int end = min(s_max + 1, (int)rg.y), lo = (int)rg.x;
        // stage s holds the Gaussians [max(lo, end - (s + 1) DEPTH), end - s DEPTH), replayed
        // back to front from buffer s & 1
        auto stage_n = [&](int bend) { return bend > lo ? bend - max(lo, bend - DEPTH) : 0; };
        auto stage_first = [&](int bend) { return (unsigned)max(lo, bend - DEPTH); };
        stage_copy_ids<NT>(s_id[0], ids, stage_first(end), stage_n(end));
        cp_async_commit();
        cp_async_wait_all();
        stage_copy_records<NT>(w, s_id[0], stage_n(end), s_a[0], s_b[0], s_c[0], s_p[0]);
        stage_copy_ids<NT>(s_id[1], ids, stage_first(end - DEPTH), stage_n(end - DEPTH));
        cp_async_commit();
        int buf = 0;
        for (int bend = end; bend > lo; bend -= DEPTH, buf ^= 1) {
            const int bstart = max(lo, bend - DEPTH);
            const int n = bend - bstart;
            cp_async_wait_all();
            __syncthreads();  // stage in buffer buf complete; the other buffer's stage replayed
            stage_copy_records<NT>(w, s_id[buf ^ 1], stage_n(bend - DEPTH), s_a[buf ^ 1], s_b[buf ^ 1], s_c[buf ^ 1],
                                   s_p[buf ^ 1]);
            stage_copy_ids<NT>(s_id[buf], ids, stage_first(bend - 2 * DEPTH), stage_n(bend - 2 * DEPTH));
            cp_async_commit();
            const float4 *sa = s_a[buf], *sb = s_b[buf];
            const float *sc = s_c[buf];
            const unsigned *sp = s_p[buf];
            const int jtop = min(n - 1, wmax - bstart);  // this warp's pixels stop before the rest
            for (int j = jtop; j >= 0; j--) {
                const float4 f0 = sa[j], f1 = sb[j];
                const int pos = bstart + j;
                // exponents e = a' dx^2 + b' dx dy + c' dy^2 + log2 o, rounded exactly as the
                // forward's (the replay divides its transmittance back)
                const float dx = __fsub_rn(f0.x, px);
                const float s0 = __fmaf_rn(__fmul_rn(f0.z, dx), dx, f1.y);
                const float bdx = __fmul_rn(f0.w, dx);
                float2 dy[NP], r[NP];
                bool v[PX];
                bool any = false;
#pragma unroll
                for (int k = 0; k < NP; k++) {
                    dy[k] = __fadd2_rn(dup2(f0.y), npy[k]);
                    const float2 t = __ffma2_rn(dup2(bdx), dy[k], dup2(s0));
                    const float2 e = __ffma2_rn(__fmul2_rn(dup2(f1.x), dy[k]), dy[k], t);
                    r[k] = make_float2(ex2_approx(e.x), ex2_approx(e.y));  // o exp(-power), unclamped
                    // the forward's cutoff test min(r, 0.99) >= 1/255 is r >= 1/255 (r = 2^e is
                    // finite and non-negative): the same decision without the clamp
                    v[2 * k] = pos <= last[2 * k] && r[k].x >= kAlphaMin;
                    v[2 * k + 1] = pos <= last[2 * k + 1] && r[k].y >= kAlphaMin;
                    any = any || v[2 * k] || v[2 * k + 1];
                }
                const unsigned act = __ballot_sync(0xffffffffu, any);
                if (!act) continue;
                const float cb = sc[j];
                // Per-lane sums over the thread's pixels (one column: dx is the lane's):
                // S0 = sum dL/de, S1 = sum dL/de dy, S2 = sum dL/de dy^2 and the colour terms;
                // the screen-space gradients follow by the chain rule of e: du = (2a'dx) S0 +
                // b' S1, dv = (b'dx) S0 + 2c' S1, da' = dx^2 S0, db' = dx S1, dc' = S2, and
                // dlog2o = S0 (alpha = 2^e, so dL/de carries the factor ln 2, applied per term).
                float2 A0, A1, A2, Cr, Cg, Cb;
#pragma unroll
                for (int k = 0; k < NP; k++) {
                    const bool va = v[2 * k], vb = v[2 * k + 1];
                    if (COUNT) n_comp += (unsigned)va + (unsigned)vb;
                    const float a0 = va ? fminf(r[k].x, kAlphaMax) : 0.f, a1 = vb ? fminf(r[k].y, kAlphaMax) : 0.f;
                    const float2 al = make_float2(a0, a1);
                    // a pixel that does not composite this Gaussian has alpha 0: 1 / (1 - 0) is
                    // exactly 1 (the hardware reciprocal is exact on powers of two), so T stays
                    const float2 om = __fadd2_rn(make_float2(1.f, 1.f), make_float2(-a0, -a1));
                    const float2 ra = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                    const float2 Tin = __fmul2_rn(T[k], ra);
                    const float2 wg = __fmul2_rn(al, Tin);
                    // dL/dalpha = sum_ch g_ch (c_ch Tin - S_ch / (1 - alpha)) = gc Tin + gS / (1 - alpha)
                    const float2 gc = __ffma2_rn(g2[k], dup2(cb), __ffma2_rn(g1[k], dup2(f1.w), __fmul2_rn(g0[k], dup2(f1.z))));
                    const float2 dal = __ffma2_rn(gS[k], ra, __fmul2_rn(gc, Tin));
                    gS[k] = __ffma2_rn(make_float2(-gc.x, -gc.y), wg, gS[k]);
                    T[k] = Tin;
                    // dL/de for the exponent e: alpha = 2^e unless clamped at 0.99, so dalpha/de
                    // is alpha ln 2 where composited below the clamp, else 0
                    const float2 kk = __fmul2_rn(make_float2(a0 < kAlphaMax ? a0 : 0.f, a1 < kAlphaMax ? a1 : 0.f),
                                                 dup2(kLn2));
                    const float2 de = __fmul2_rn(dal, kk);
                    const float2 ddy = __fmul2_rn(de, dy[k]);
                    // the moments and colour sums accumulate over the thread's pixels by fused
                    // multiply-adds (one rounding per term)
                    if (k == 0) {
                        A0 = de; A1 = ddy; A2 = __fmul2_rn(ddy, dy[k]);
                        Cr = __fmul2_rn(wg, g0[k]); Cg = __fmul2_rn(wg, g1[k]); Cb = __fmul2_rn(wg, g2[k]);
                    } else {
                        A0 = __fadd2_rn(A0, de); A1 = __fadd2_rn(A1, ddy); A2 = __ffma2_rn(ddy, dy[k], A2);
                        Cr = __ffma2_rn(wg, g0[k], Cr); Cg = __ffma2_rn(wg, g1[k], Cg); Cb = __ffma2_rn(wg, g2[k], Cb);
                    }
                }
                const float S0 = A0.x + A0.y, S1 = A1.x + A1.y, S2 = A2.x + A2.y;
                const float vs[9] = {fmaf(f0.w, S1, 2.f * f0.z * dx * S0), fmaf(2.f * f1.x, S1, f0.w * dx * S0),
                                     dx * dx * S0, dx * S1, S2, S0, Cr.x + Cr.y, Cg.x + Cg.y, Cb.x + Cb.y};
                if (__popc(act) <= kSparseLanes) {
                    if (any) {
                        const unsigned p = sp[j];
                        float *a = &w.g0[p].x, *b = &w.g1[p].x;
                        atomicAdd(a, vs[0]); atomicAdd(a + 1, vs[1]); atomicAdd(a + 2, vs[2]); atomicAdd(a + 3, vs[3]);
                        atomicAdd(b, vs[4]); atomicAdd(b + 1, vs[5]); atomicAdd(b + 2, vs[6]); atomicAdd(b + 3, vs[7]);
                        atomicAdd(w.g2 + p, vs[8]);
                    }
                } else {
                    int slot;
                    const float sum = warp_reduce9(vs, lane, slot);
                    if (slot < 9 && !(lane & 1)) {
                        const unsigned p = sp[j];
                        float *dst = slot < 4 ? &w.g0[p].x + slot : (slot < 8 ? &w.g1[p].x + (slot - 4) : w.g2 + p);
                        atomicAdd(dst, sum);
                    }
                }
            }
        }
        add_work(w.hdr->work + 2, n_eval, n_comp);
        __syncthreads();
    }
}

// Pixels per lane of the backward for a tile shape: four where a warp still covers whole
// rows of the tile (16-wide tiles), else two.
template <int TW, int TH>
constexpr int bwd_px() { return TW >= 16 ? 4 : 2; }

template <int TW, int TH, int DEPTH>
int occupancy_fwd() {
    constexpr int PX = fwd_px<TW, TH>();
    static int blocks = 0;
    if (!blocks) {
        if constexpr (PX == 4)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_fwd4_kernel<TW, TH, DEPTH, 4>, TW * TH / 4, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_fwd_kernel<TW, TH, DEPTH>, TW * TH / 2, 0);
    }
    return blocks > 0 ? blocks : 1;
}

template <int TW, int TH, int DEPTH>
int occupancy_bwd() {
    constexpr int PX = bwd_px<TW, TH>();
    static int blocks = 0;
    if (!blocks)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, composite_bwd_kernel<TW, TH, DEPTH, PX, false>,
                                                      TW * TH / PX, 0);
    return blocks > 0 ? blocks : 1;
}

template <int TW, int TH, int DEPTH>
cudaError_t run_fwd(const Work &w, const unsigned *ids, float bg0, float bg1, float bg2, float *image, float *T,
                    int32_t *idx, const LossArgs &ls, int num_sms, cudaStream_t s) {
    unsigned grid = min(w.L.tiles, (unsigned)(num_sms * occupancy_fwd<TW, TH, DEPTH>()));
    if (grid == 0) return cudaSuccess;
    if constexpr (fwd_px<TW, TH>() == 4)
        launch_pdl(composite_fwd4_kernel<TW, TH, DEPTH, 4>, grid, TW * TH / 4, 0, s, w, ids, bg0, bg1, bg2, image, T, idx,
                   ls);
    else
        launch_pdl(composite_fwd_kernel<TW, TH, DEPTH>, grid, TW * TH / 2, 0, s, w, ids, bg0, bg1, bg2, image, T, idx,
                   ls);
    return cudaGetLastError();
}

template <int TW, int TH, int DEPTH>
cudaError_t run_bwd(const Work &w, const unsigned *ids, float bg0, float bg1, float bg2, const float *T,
                    const int32_t *idx, const float *dL, bool count, int num_sms, cudaStream_t s) {
    unsigned grid = min(w.L.tiles, (unsigned)(num_sms * occupancy_bwd<TW, TH, DEPTH>()));
    if (grid == 0) return cudaSuccess;
    constexpr int PX = bwd_px<TW, TH>();
    if (count)
        launch_pdl(composite_bwd_kernel<TW, TH, DEPTH, PX, true>, grid, TW * TH / PX, 0, s, w, ids, bg0, bg1, bg2, T,
                   idx, dL);
    else
        launch_pdl(composite_bwd_kernel<TW, TH, DEPTH, PX, false>, grid, TW * TH / PX, 0, s, w, ids, bg0, bg1, bg2, T,
                   idx, dL);
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
        case 32016:                                                                              \
            switch (depth) {                                                                     \
                case 32: return FN<32, 16, 32>(__VA_ARGS__);                                     \
                case 64: return FN<32, 16, 64>(__VA_ARGS__);                                     \
                case 128: return FN<32, 16, 128>(__VA_ARGS__);                                   \
                case 256: return FN<32, 16, 256>(__VA_ARGS__);                                   \
            }                                                                                    \
            break;                                                                               \
        case 32032:                                                                              \
            switch (depth) {                                                                     \
                case 32: return FN<32, 32, 32>(__VA_ARGS__);                                     \
                case 64: return FN<32, 32, 64>(__VA_ARGS__);                                     \
                case 128: return FN<32, 32, 128>(__VA_ARGS__);                                   \
                case 256: return FN<32, 32, 256>(__VA_ARGS__);                                   \
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
                                 const LossArgs &loss, int num_sms, cudaStream_t s) {
    const unsigned *ids = w.tval[tile_buf];
    GV_DISPATCH(run_fwd, w, ids, bg0, bg1, bg2, image, final_T, last_idx, loss, num_sms, s)
}

cudaError_t launch_composite_bwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf, float bg0,
                                 float bg1, float bg2, const float *final_T, const int32_t *last_idx,
                                 const float *dL_dimage, bool count_replayed, int num_sms, cudaStream_t s) {
    const unsigned *ids = w.tval[tile_buf];
    GV_DISPATCH(run_bwd, w, ids, bg0, bg1, bg2, final_T, last_idx, dL_dimage, count_replayed, num_sms, s)
}

}  // namespace gvk
