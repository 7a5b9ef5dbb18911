// gv_internal.cuh -- definitions shared by the libgv kernels and the host ABI layer.
//
// Device data layout of one render call (all in the caller's workspace, see plan_layout):
//   header      DevHeader: error word, key count, work-queue and sort counters
//   frames      DevFrame[F]: camera and offsets of each frame
//   per pair    (frame, Gaussian) pairs, P = sum of per-frame Gaussian counts:
//               feat0 float4 (u, v, a', b'), feat1 float4 (c', log2 o, r, g), feat2 float
//               (b) (the staged record, below), rect uint4 (pixel box of the extent, cell
//               count, frame), ell float4 (the culling record), depth keys and pair ids
//               (double-buffered for the depth sort), grad2d (two float4 + float)
//   per key     tile ids and pair ids, double-buffered for the tile sort
//   per chunk   the depth-ordered pair owning the chunk's first cell (key emission)
//   per tile    [start, end) ranges into the sorted key list
//   sort        digit histograms and decoupled look-back status words
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gv.h"

namespace gvk {
// Programmatic dependent launch (every kernel of the library is launched with it): the
// next kernel of the stream may be scheduled while this one runs, so launch latency and
// the previous grid's tail overlap.  Every kernel starts with pdl_prologue(): it first
// waits until the preceding grid has completed and its memory is visible (so nothing is
// read or written early), then allows its own dependents to launch.
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches kernel k with the programmatic-stream-serialisation attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}


// Rendering constants (Sec. 3.1 conventions; see include/gv.h).
constexpr float kAlphaMin = 0.003921568859368563f;  // 1/255
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kEps2d = 0.3f;
constexpr float kZNear = 0.2f;
constexpr float kExtK = 3.329042911529541f;          // sqrt(2 ln 255), rounded to FP32
constexpr float kLn255 = 5.541263545158426f;         // ln 255

// Device error bits (DevHeader::err).
enum : unsigned { ERR_CAPACITY = 1u, ERR_TIMEOUT = 2u };

constexpr int kMaxFramesPerSetup = 96;  // frames per setup launch (kernel parameter space)

struct DevFrame {
    int W, H;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float time;
    long long gauss_offset;
    long long pixel_offset;
    unsigned pair_offset, gauss_count;
    unsigned tile_offset, tiles_x, tiles_y, pad;
    // time-parameterised means: the four control points ctrl[spline_lo .. + 3] carry the
    // non-zero cubic B-spline weights spline_w at this frame's time (host-computed)
    int spline_lo;
    float spline_w[4];
    float campos[3];  // camera centre -R^T t (view direction of the spherical harmonics)
};

struct DevHeader {
    unsigned err;
    unsigned keys_used;             // min(keys_total, capacity)
    unsigned long long keys_total;  // keys (after culling) the call emits; on a capacity error,
                                    // the key capacity it needs
    unsigned n_pairs;               // P, read by the depth sort's first pass
    unsigned n_drawn;               // pairs with a depth key (a non-empty extent box): the
                                    // depth-sorted list holds only these, in its first n_drawn slots
    unsigned sort_ctr[16];          // tile-acquisition counters: sort passes 0-7, cell-offset scan 12
    unsigned queue[4];              // persistent work-queue counters
    long long spin_limit;           // iteration limit of every device-side wait
    int drop_signal;                // test hook: first look-back block never publishes
    int pad;
    unsigned long long work[4];     // pairs evaluated / composited: fwd 0-1, bwd 2-3
    unsigned fp64_count;            // ill-conditioned pairs listed by the projection (FP64 chain rule)
    unsigned n_chunks;              // emission chunks of kEmitBlock cells
    unsigned long long cells;       // cells: tiles of the pairs' extent boxes, before culling
};

// rect.w of a pair: frame index, bit 31 set when the backward runs its geometric chain
// rule in FP64 (ill-conditioned footprint)
constexpr unsigned kRectFp64 = 1u << 31;
constexpr unsigned kRectFrame = kRectFp64 - 1u;

// Radix sort geometry (one onesweep pass = one 8-bit digit): keys per thread by sort size.
// Up to 2^18 keys 2048-key block tiles (few tiles: a short look-back chain), up to 2^20
// 1024-key tiles (more blocks in flight), above 3072-key tiles (fewer look-back steps).
constexpr int kSortThreads = 256;
constexpr int kRadix = 256;
constexpr unsigned kSortSmallN = 1u << 20;
__host__ __device__ constexpr int sort_items(unsigned n_cap) {
    return n_cap <= (1u << 18) ? 8 : (n_cap <= kSortSmallN ? 4 : 12);
}
__host__ __device__ constexpr unsigned sort_tile_keys(unsigned n_cap) {
    return (unsigned)(kSortThreads * sort_items(n_cap));
}
__host__ __device__ constexpr unsigned sort_tiles(unsigned n, unsigned n_cap) {
    return (n + sort_tile_keys(n_cap) - 1) / sort_tile_keys(n_cap);
}

// Emission block geometry (count scan + load-balanced key emission).  The emission walks
// cells (the tiles of each pair's extent box) and keeps those the cull keeps; the chunk
// table holds up to kCellsPerKey cells per key of capacity.
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitBlock = kEmitThreads * kEmitItems;  // 2048 pairs (or cells) per block
constexpr unsigned kCellsPerKey = 2;
__host__ __device__ constexpr unsigned emit_chunk_cap(unsigned key_cap) {
    return (unsigned)(((unsigned long long)key_cap * kCellsPerKey + kEmitBlock - 1) / kEmitBlock) + 1u;
}

// Workspace layout (byte offsets), computed on the host.
struct Layout {
    size_t hdr, frames;
    size_t feat0, feat1, feat2, rect, ell, dkey[2], dval[2];
    size_t scan_look, offsets, chunk_first;
    size_t g0, g1, g2;
    size_t fp64_list;
    size_t ranges;
    size_t tkey[2], tval[2];
    size_t hist, look;
    size_t total;
    unsigned P, tiles, F;
    unsigned tiles_alloc;  // ranges capacity (tile count of the finest tiling, 8x8)
    unsigned key_cap;
    unsigned chunk_cap;    // emission chunks (emit_chunk_cap(key_cap))
    unsigned look_tiles;   // look-back tiles per buffer (sort tiles or emission chunks)
    unsigned emit_blocks;
    int tile_bits;         // live bits of the global tile id
};

// Pointers into one workspace.
struct Work {
    DevHeader *hdr;
    DevFrame *frames;
    float4 *feat0, *feat1;
    float *feat2;
    uint4 *rect;   // (x0 | y0 << 16, x1 | y1 << 16, cells, frame | kRectFp64): pixel box of the extent
    float4 *ell;   // culling record (kx, ds, tc, dn), see cull_record
    unsigned *dkey[2], *dval[2];
    unsigned long long *scan_look;  // [emit_blocks] status words of the cell-offset scan
    unsigned *offsets;      // [P + 1] exclusive cell offsets of the pairs in depth order
    unsigned *chunk_first;  // [chunk_cap] depth-ordered pair owning a chunk's first cell
    float4 *g0, *g1;
    float *g2;
    unsigned *fp64_list;  // [P] pairs whose geometric chain rule runs in FP64
    uint2 *ranges;
    unsigned *tkey[2], *tval[2];
    unsigned *hist;   // [8][256]: depth-sort passes 0-3, tile-sort passes 4-7
    unsigned *look;   // [2][look_tiles][256]
    Layout L;
};

struct GaussPtrs {
    const float *mean, *vel, *log_scale, *quat, *logit, *rgb;
    long long N;
    int n_ctrl;  // > 0: means on the B-spline over ctrl; log_scale_t / quat_t: cubic terms (or NULL)
    const float *ctrl, *log_scale_t, *quat_t;
    int sh_degree;     // 0..3; > 0: colour = rgb + sum_k Y_k(dir) sh[ch][k]
    const float *sh;   // [3][(sh_degree + 1)^2 - 1][N]
    uint8_t *visible;  // [N] or NULL: set to 1 for Gaussians with a kept key (forward)
};

struct GradPtrs {
    float *mean, *vel, *log_scale, *quat, *logit, *rgb;
    float *cam;  // [F][kCamGrad] or NULL
    float *ctrl, *log_scale_t, *quat_t;  // time-parameterised form
    float *sh;                           // spherical-harmonic coefficients or NULL
};

// Camera gradient per frame: dR (9, row-major), dt (3), dfx, dfy, dcx, dcy.
constexpr int kCamGrad = 16;

struct FrameChunk {
    DevFrame f[kMaxFramesPerSetup];
};

// ---- host launchers (stream-ordered, no allocation) --------------------------------

// setup.cu
cudaError_t launch_setup(const Work &w, const FrameChunk &chunk, int first, int count, bool zero_all,
                         long long spin_limit, int drop_signal, cudaStream_t s);
const void *setup_kernel_ptr();
// project.cu
// shared_set: every frame draws the same Gaussian range (one thread per Gaussian then loops
// over the frames, for the plain form)
cudaError_t launch_project_fwd(const Work &w, const GaussPtrs &g, int tile_w, int tile_h, bool shared_set,
                               int num_sms, cudaStream_t s);
cudaError_t launch_bin_from_screen(const Work &w, long long n, const float *u, const float *v,
                                   const float *sxx, const float *sxy, const float *syy, const float *tau,
                                   const float *depth, const uint8_t *valid, int tile_w, int tile_h,
                                   int32_t *counts, int num_sms, cudaStream_t s);
cudaError_t launch_project_bwd(const Work &w, const GaussPtrs &g, const GradPtrs &gr, int mode, int num_sms,
                               cudaStream_t s);
// FP64 chain rule of the pairs the projection flagged (may run concurrently with the above)
cudaError_t launch_project_bwd_fp64(const Work &w, const GaussPtrs &g, const GradPtrs &gr, int num_sms,
                                    cudaStream_t s);
// sort.cu
// Key 0xFFFFFFFF means "no key": every pass drops it (neither ranked, counted nor written),
// so a pass writes only the live keys, compacted; digit histograms count live keys only.
constexpr unsigned kNoKey = 0xFFFFFFFFu;
int sort_passes(int bits);
// n_dev: keys read by the first pass; n_dev_later (or n_dev when NULL): by the later passes
// (the live keys the first pass kept).
cudaError_t launch_radix_sort(const Work &w, unsigned *keys[2], unsigned *vals[2], const unsigned *n_dev,
                              unsigned n_cap, int bits, bool vals_identity, bool prepared, int hist_slot,
                              int ctr_slot, int num_sms, cudaStream_t s, int *result_buf, int first_pass = 0,
                              const unsigned *n_dev_later = nullptr, uint2 *final_ranges = nullptr,
                              unsigned n_tiles = 0);
// Warp-aggregated count of one 8-bit digit per lane into a shared histogram row.
__device__ __forceinline__ void count_digit(unsigned *row, unsigned d, unsigned active) {
    const unsigned peers = __match_any_sync(active, d);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(row + d, (unsigned)__popc(peers));
}
// binning.cu
// Cell offsets, then key emission fused with the first tile-sort pass: the kept keys land
// in tkey[1] / tval[1] sorted by their low tile digit.
cudaError_t launch_emit(const Work &w, int depth_buf, int tile_w, int tile_h, int num_sms, cudaStream_t s);
// Each tile's [start, end) of the final list.  setup starts every tile empty (start >= end
// reads as empty).  Lists of up to kFusedRangesKeys keys of capacity get them from the kernel
// that writes the list (the last tile-sort pass, or the emission when the tile ids fit one
// digit): one atomic min / max per run of equal ids it writes, which saves a launch.  Larger
// lists -- where those atomics cost more than a separate pass (8 x 1920x1080 / 1M: 46M keys,
// 64 runs per sort tile) -- from ranges_kernel (launch_ranges).  launch_debug_ranges copies
// them out with empty tiles as (0, 0).
constexpr unsigned kFusedRangesKeys = 1u << 22;
cudaError_t launch_ranges(const Work &w, int tile_buf, int num_sms, cudaStream_t s);
cudaError_t launch_debug_ranges(const Work &w, uint2 *out, cudaStream_t s);
// composite.cu
// The L2 loss fused into the compositing forward (Sec. 4.1); target == nullptr: none.
// dL (if not null) = 2 scale (image - target), loss (if not null) += scale sum (image -
// target)^2 -- the same expressions as the separate loss kernel.
struct LossArgs {
    const float *target = nullptr;
    float *dL = nullptr;
    float *loss = nullptr;
    float scale = 0.f;
};
cudaError_t launch_composite_fwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf,
                                 float bg0, float bg1, float bg2, float *image, float *final_T,
                                 int32_t *last_idx, const LossArgs &loss, int num_sms, cudaStream_t s);
// count_replayed: also count the replayed pairs (work[3]; costs inner-loop instructions)
cudaError_t launch_composite_bwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf,
                                 float bg0, float bg1, float bg2, const float *final_T,
                                 const int32_t *last_idx, const float *dL_dimage, bool count_replayed,
                                 int num_sms, cudaStream_t s);
// optim.cu
cudaError_t launch_l2_loss(const float *image, const float *target, long long n, float scale,
                           float *dL, float *loss, cudaStream_t s);
cudaError_t launch_adam(float *p, float *g, float *m, float *v, long long n, float lr, float b1,
                        float b2, float eps, float bc1, float bc2, int zero_grad, cudaStream_t s);
cudaError_t launch_adan(float *p, float *g, float *m, float *v, float *nn, float *g_prev, long long n, float lr,
                        float b1, float b2, float b3, float eps, float wd, long long step, bool debias, int zero_grad,
                        cudaStream_t s);
// acc |= the error word of the render call that last used `workspace` (header at offset 0)
cudaError_t launch_status_or(const void *workspace, int *acc, cudaStream_t s);
cudaError_t launch_gather_debug(const Work &w, float *mean2d, float *conic, float *opacity,
                                float *depth, int32_t *counts, int depth_buf, cudaStream_t s);
cudaError_t launch_grad2d_debug(const Work &w, float *out, cudaStream_t s);

// ---- small device helpers ----------------------------------------------------------

__device__ __forceinline__ int find_frame_by_pair(const DevFrame *fr, int F, unsigned p) {
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (fr[mid].pair_offset <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_frame_by_tile(const DevFrame *fr, int F, unsigned t) {
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (fr[mid].tile_offset <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Staged splat record.  The compositing kernels read, per (frame, Gaussian) pair,
// feat0 = (u, v, a', b') and feat1 = (c', log2 o, r, g), feat2 = b, where
//   a' = -log2(e) A / 2,  b' = -log2(e) B,  c' = -log2(e) C / 2
// for the conic (A, B, C), so that o exp(-1/2 (A dx^2 + 2 B dx dy + C dy^2)) =
// 2^(a' dx^2 + b' dx dy + c' dy^2 + log2 o): one exponent, no separate opacity product.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float ex2_approx(float x) {  // hardware 2^x (MUFU), flush-to-zero
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {  // hardware 1/x (MUFU), flush-to-zero
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Asynchronous global -> shared copies (cp.async): the copy needs no register and lands
// while the thread computes; cp_async_wait_all() then a block barrier make it visible.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {  // both 16-byte aligned
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Exponents of one staged Gaussian at the two pixels (px, py.x) and (px, py.y) a thread
// owns: e = a' dx^2 + b' dx dy + c' dy^2 + log2 o, with dx shared.  Written with explicit
// round-to-nearest (packed) operations so the forward and the backward compute
// bit-identical values (the backward replays the forward's decisions and divides its
// transmittance back).  Also returns dx, dy (packed) for the gradients.
__device__ __forceinline__ float2 splat_exponent2(float4 f0, float4 f1, float px, float2 npy, float &dx,
                                                  float2 &dy) {
    dx = __fsub_rn(f0.x, px);
    dy = __fadd2_rn(dup2(f0.y), npy);                       // v - py, both pixels
    const float s0 = __fmaf_rn(__fmul_rn(f0.z, dx), dx, f1.y);  // a' dx^2 + log2 o
    const float bdx = __fmul_rn(f0.w, dx);                  // b' dx
    const float2 t = __ffma2_rn(dup2(bdx), dy, dup2(s0));   // + b' dx dy
    return __ffma2_rn(__fmul2_rn(dup2(f1.x), dy), dy, t);   // + c' dy^2
}

// ---- onesweep building blocks (256-thread blocks; thread t owns digit t) ---------------

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread block; returns the total.
// s_warp: 17 words of shared memory.
__device__ __forceinline__ unsigned block_excl_scan_256(unsigned x, unsigned *s_warp, unsigned &excl) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        unsigned t = lane < 8 ? s_warp[lane] : 0u;
        unsigned ti = t;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < 8) s_warp[8 + lane] = ti - t;
        if (lane == 7) s_warp[16] = ti;
    }
    __syncthreads();
    excl = s_warp[8 + wid] + inc - x;
    unsigned total = s_warp[16];
    __syncthreads();
    return total;
}

// Status word of one (tile, digit) in a look-back buffer: flag in the top two bits, count
// below.  Buffers are zeroed (no flag) before a pass uses them.
constexpr unsigned kFlagAgg = 1u << 30;
constexpr unsigned kFlagInc = 2u << 30;
constexpr unsigned kValMask = (1u << 30) - 1u;

// Decoupled look-back of one digit d of `tile` in a pass over look[tile][256], in two
// steps so that a block can publish its counts as soon as it has them and walk its
// predecessors only when it needs their sum (after its own shared-memory work, which gives
// the predecessors that much longer to publish their inclusive prefixes):
// - lookback_publish: the tile's own count of d (tile 0: directly as its inclusive prefix;
//   others: as an aggregate).  drop (test hook): tile 0 never publishes.
// - lookback_walk<WIN>: the sum of the counts of all earlier tiles.  The predecessors are
//   read WIN at a time (independent loads in flight), their aggregates summed until an
//   inclusive prefix is found; an unpublished predecessor is polled again.  Then the
//   tile's inclusive prefix is published.  Every wait is bounded by `limit` polls without
//   progress; a wait that gives up (or finds ERR_TIMEOUT already set) sets ERR_TIMEOUT and
//   gave_up, publishes anyway and returns a partial sum: the caller then writes nothing.
constexpr int kLookWindow = 4;

__device__ __forceinline__ void lookback_publish(unsigned *look, unsigned tile, unsigned d, unsigned mine, bool drop) {
    if (tile == 0) {
        if (!drop) atomicExch(look + d, kFlagInc | mine);
    } else {
        atomicExch(look + (size_t)tile * kRadix + d, kFlagAgg | mine);
    }
}

template <int WIN>
__device__ __forceinline__ unsigned lookback_walk(unsigned *look, unsigned tile, unsigned d, unsigned mine,
                                                  DevHeader *hdr, long long limit, bool &gave_up) {
    unsigned excl = 0;
    gave_up = false;
    if (tile == 0) return 0u;
    long long spins = 0;
    int j = (int)tile - 1;
    bool found = false;
    while (!found) {
        unsigned st[WIN];
#pragma unroll
        for (int k = 0; k < WIN; k++)
            st[k] = j - k >= 0 ? *((volatile unsigned *)(look + (size_t)(j - k) * kRadix + d)) : 0u;
        int adv = 0;
#pragma unroll
        for (int k = 0; k < WIN; k++) {
            if (found || adv < k || j - k < 0) continue;  // stop at the first unpublished status
            const unsigned fl = st[k] & ~kValMask;
            if (fl == kFlagInc) {
                excl += st[k] & kValMask;
                found = true;
            } else if (fl == kFlagAgg) {
                excl += st[k] & kValMask;
                adv = k + 1;
            }
        }
        if (found) break;
        j -= adv;
        if (adv > 0) {
            spins = 0;
            continue;
        }
        if (++spins > limit || (*((volatile unsigned *)&hdr->err) & ERR_TIMEOUT)) {
            gave_up = true;
            break;
        }
        __nanosleep(32);
    }
    if (gave_up) atomicOr(&hdr->err, ERR_TIMEOUT);
    atomicExch(look + (size_t)tile * kRadix + d, kFlagInc | ((excl + mine) & kValMask));
    return excl;
}

// lookback_walk of digit d by a group of G consecutive lanes of one warp (G a power of two
// up to 32; member m = lane % G, gmask the group's lanes), after lookback_publish: member m
// reads predecessors j - 4m .. j - 4m - 3, so one poll covers 4G predecessors.  The group
// takes the nearest member whose window ends the walk (an inclusive prefix, or an
// unpublished status) and sums the counts up to it; every member returns the same sum.
// Member 0 publishes the inclusive prefix.  Used by passes whose digit has fewer than 8 live
// bits, where the block has 256 / 2^bits threads per digit.
__device__ __forceinline__ unsigned lookback_walk_group(unsigned *look, unsigned tile, unsigned d, unsigned mine,
                                                        int G, int m, unsigned gmask, DevHeader *hdr,
                                                        long long limit, bool &gave_up) {
    const int base = (int)(threadIdx.x & 31u) - m;  // the group's first lane
    gave_up = false;
    if (tile == 0) return 0u;
    unsigned excl = 0;
    long long spins = 0;
    int j = (int)tile - 1;
    for (;;) {
        unsigned st[kLookWindow];
#pragma unroll
        for (int k = 0; k < kLookWindow; k++) {
            const int idx = j - kLookWindow * m - k;
            const unsigned past = kFlagInc;  // before tile 0: an empty inclusive prefix
            st[k] = idx >= 0 ? *((volatile unsigned *)(look + (size_t)idx * kRadix + d)) : past;
        }
        // this member's window, nearest first: 0 all aggregates, 1 an inclusive prefix ends it,
        // 2 an unpublished status stops it (len: the entries taken)
        unsigned sum = 0;
        int term = 0, len = kLookWindow;
#pragma unroll
        for (int k = 0; k < kLookWindow; k++) {
            if (term) continue;
            const unsigned fl = st[k] & ~kValMask;
            if (fl == kFlagInc) { sum += st[k] & kValMask; term = 1; len = k + 1; }
            else if (fl == kFlagAgg) sum += st[k] & kValMask;
            else { term = 2; len = k; }
        }
        const unsigned ended = (__ballot_sync(gmask, term != 0) >> base) & (G == 32 ? 0xffffffffu : (1u << G) - 1u);
        const int ms = ended ? __ffs(ended) - 1 : G;  // nearest member whose window ends the walk
        unsigned c = m <= ms ? sum : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            if (o < G) c += __shfl_xor_sync(gmask, c, o, G);
        excl += c;
        const int ts = __shfl_sync(gmask, term, ms < G ? ms : 0, G);
        const int ls = __shfl_sync(gmask, len, ms < G ? ms : 0, G);
        if (ms < G && ts == 1) break;
        const int taken = ms < G ? kLookWindow * ms + ls : kLookWindow * G;
        j -= taken;
        if (taken > 0) {
            spins = 0;
            continue;
        }
        bool quit = ++spins > limit || (*((volatile unsigned *)&hdr->err) & ERR_TIMEOUT);
        quit = __shfl_sync(gmask, quit, 0, G);
        if (quit) {
            gave_up = true;
            break;
        }
        __nanosleep(32);
    }
    if (m == 0) {
        if (gave_up) atomicOr(&hdr->err, ERR_TIMEOUT);
        atomicExch(look + (size_t)tile * kRadix + d, kFlagInc | ((excl + mine) & kValMask));
    }
    return excl;
}

// ---- culled tile binning (integer decisions, every FP32 operation explicitly rounded) --
//
// A pair is binned from the extent box of its alpha >= 1/255 ellipse d^T Sigma2^-1 d <= tau
// (half-widths ex = sqrt(tau a), ey = sqrt(tau c) for Sigma2 = [[a, b], [b, c]]): pixel
// centres x + 0.5 in [u - ex, u + ex], x0 = ceil((u - ex) - 0.5), x1 = floor((u + ex) - 0.5),
// clipped to the image (same in y).  Its cells are the tiles of that box; a cell is kept
// when one of its pixel columns has its centre between the two ends of the ellipse over
// the band of pixel-centre rows of the cell's tile row (clipped to the box).  At offset dy
// the ellipse spans dx = kx dy +- sqrt((tc - dy^2) dn) with kx = b / c, tc = tau c,
// dn = det / c^2; over a band [d0, d1] the right end peaks at dy = clamp(ds, d0, d1) and
// the left end at clamp(-ds, d0, d1), ds = b ex / a (the height of the rightmost point).
// A near-singular footprint (a c > 64 det) keeps its whole box.  Fixed operation order and
// rounding, so the FP32 CPU reference reproduces every decision.

struct PixBox {
    int x0, y0, x1, y1;
};

// Extent box; false when empty (or tau <= 0: the Gaussian never reaches alpha 1/255).
__device__ __forceinline__ bool extent_box(float u, float v, float a, float c, float tau, int W, int H, float &ex,
                                           PixBox &b) {
    if (!(tau > 0.f)) return false;
    ex = __fsqrt_rn(__fmul_rn(tau, a));
    const float ey = __fsqrt_rn(__fmul_rn(tau, c));
    float x0 = ceilf(__fsub_rn(__fsub_rn(u, ex), 0.5f));
    float x1 = floorf(__fsub_rn(__fadd_rn(u, ex), 0.5f));
    float y0 = ceilf(__fsub_rn(__fsub_rn(v, ey), 0.5f));
    float y1 = floorf(__fsub_rn(__fadd_rn(v, ey), 0.5f));
    if (x0 < 0.f) x0 = 0.f;
    if (y0 < 0.f) y0 = 0.f;
    if (x1 > (float)(W - 1)) x1 = (float)(W - 1);
    if (y1 > (float)(H - 1)) y1 = (float)(H - 1);
    if (!(x0 <= x1) || !(y0 <= y1)) return false;
    b.x0 = (int)x0; b.y0 = (int)y0; b.x1 = (int)x1; b.y1 = (int)y1;
    return true;
}

__device__ __forceinline__ float4 cull_record(float a, float b, float c, float tau, float ex) {
    const float ac = __fmul_rn(a, c), det = __fsub_rn(ac, __fmul_rn(b, b));
    if (!(a > 0.f) || !(c > 0.f) || ac > __fmul_rn(64.f, det))
        return make_float4(0.f, 0.f, __int_as_float(0x7f800000), __int_as_float(0x7f800000));
    return make_float4(__fdiv_rn(b, c), __fdiv_rn(__fmul_rn(b, ex), a), __fmul_rn(tau, c),
                       __fdiv_rn(det, __fmul_rn(c, c)));
}

// Pixel columns [i0, i1] of the band of pixel rows [ylo, yhi]; false when none.
__device__ __forceinline__ bool cull_row(float u, float v, float4 e, int ylo, int yhi, int x0, int x1, int &i0,
                                         int &i1) {
    const float d0 = __fsub_rn(__fadd_rn((float)ylo, 0.5f), v), d1 = __fsub_rn(__fadd_rn((float)yhi, 0.5f), v);
    const float dr = fminf(fmaxf(e.y, d0), d1), dl = fminf(fmaxf(-e.y, d0), d1);
    const float hr = __fsqrt_rn(fmaxf(__fmul_rn(__fsub_rn(e.z, __fmul_rn(dr, dr)), e.w), 0.f));
    const float hl = __fsqrt_rn(fmaxf(__fmul_rn(__fsub_rn(e.z, __fmul_rn(dl, dl)), e.w), 0.f));
    const float xr = __fadd_rn(__fmul_rn(e.x, dr), hr), xl = __fsub_rn(__fmul_rn(e.x, dl), hl);
    const float f0 = fmaxf(ceilf(__fsub_rn(__fadd_rn(u, xl), 0.5f)), (float)x0);
    const float f1 = fminf(floorf(__fsub_rn(__fadd_rn(u, xr), 0.5f)), (float)x1);
    if (!(f0 <= f1)) return false;
    i0 = (int)f0;
    i1 = (int)f1;
    return true;
}

// Kept tile columns [t0, t1] of tile row ty of a box; false when none.
__device__ __forceinline__ bool cull_tiles(float u, float v, float4 e, const PixBox &b, int ty, int lw, int lh,
                                           int &t0, int &t1) {
    const int ylo = max(ty << lh, b.y0), yhi = min((ty << lh) + (1 << lh) - 1, b.y1);
    int i0, i1;
    if (!cull_row(u, v, e, ylo, yhi, b.x0, b.x1, i0, i1)) return false;
    t0 = i0 >> lw;
    t1 = i1 >> lw;
    return true;
}

__device__ __forceinline__ uint2 pack_box(const PixBox &b) {
    return make_uint2((unsigned)b.x0 | ((unsigned)b.y0 << 16), (unsigned)b.x1 | ((unsigned)b.y1 << 16));
}

__device__ __forceinline__ PixBox unpack_box(uint4 r) {
    PixBox b;
    b.x0 = (int)(r.x & 0xFFFFu); b.y0 = (int)(r.x >> 16);
    b.x1 = (int)(r.y & 0xFFFFu); b.y1 = (int)(r.y >> 16);
    return b;
}

// Tile-sort digit counts of one tile-id range [t0, t0 + len) (a row run of a pair's kept
// tiles): digit 0 through a difference array over its 256 values (the range wraps around
// len >> 8 times plus a partial run), higher digits directly (a run spans one or two of
// their values).
__device__ __forceinline__ void count_tile_run(unsigned t0, unsigned len, int passes, int *s_diff, unsigned *s_full,
                                               unsigned (*s_h)[kRadix]) {
    const unsigned full = len >> 8, rem = len & 255u;
    if (full) atomicAdd(s_full, full);
    if (rem) {
        const unsigned a = t0 & 255u, e = a + rem;
        atomicAdd(s_diff + a, 1);
        if (e <= 256u) {
            atomicAdd(s_diff + e, -1);
        } else {
            atomicAdd(s_diff + 256, -1);
            atomicAdd(s_diff + 0, 1);
            atomicAdd(s_diff + (e - 256u), -1);
        }
    }
    const unsigned t1 = t0 + len - 1u;
    for (int ps = 1; ps < passes; ps++) {
        const int sh = 8 * ps;
        for (unsigned h = t0 >> sh; h <= (t1 >> sh); h++) {
            const unsigned lo = max(t0, h << sh), hi = min(t1, ((h + 1u) << sh) - 1u);
            atomicAdd(&s_h[ps][h & 255u], hi - lo + 1u);
        }
    }
}

// Flush a block's tile-sort digit counts: digit 0 from its difference array (prefix sum
// plus the full wraps), higher digits as counted.  Every thread of the block calls it.
__device__ __forceinline__ void flush_tile_hist(int passes, int *s_diff, unsigned s_full, unsigned (*s_h)[kRadix],
                                                unsigned *tile_hist) {
    const int t = threadIdx.x, lane = t & 31;
    if (t < 32) {
        int carry = 0;
        for (int base8 = 0; base8 < 256; base8 += 32) {
            int x = s_diff[base8 + lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            s_h[0][base8 + lane] = (unsigned)(x + carry) + s_full;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
    for (int i = t; i < passes * kRadix; i += blockDim.x) {
        const unsigned v = (&s_h[0][0])[i];
        if (v) atomicAdd(tile_hist + i, v);
    }
}

}  // namespace gvk
