// gv_internal.cuh -- definitions shared by the libgv kernels and the host ABI layer.
//
// Device data layout of one render call (all in the caller's workspace, see plan_layout):
//   header      DevHeader: error word, key count, work-queue and sort counters
//   frames      DevFrame[F]: camera and offsets of each frame
//   per pair    (frame, Gaussian) pairs, P = sum of per-frame Gaussian counts:
//               feat0 float4 (u, v, conic A, conic B), feat1 float4 (conic C, opacity, r, g),
//               feat2 float (b), rect uint4 (tile rect + frame tile base), depth keys and
//               pair ids (double-buffered for the depth sort), grad2d (two float4 + float)
//   per key     tile ids and pair ids, double-buffered for the tile sort
//   per tile    [start, end) ranges into the sorted key list
//   sort        digit histograms and decoupled look-back status words
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gv.h"

namespace gvk {

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
};

struct DevHeader {
    unsigned err;
    unsigned keys_used;             // min(keys_total, capacity)
    unsigned long long keys_total;  // keys the call needed
    unsigned n_pairs;               // P, read by the depth sort
    unsigned pad0;
    unsigned sort_ctr[16];          // tile-acquisition counters of the sort passes
    unsigned queue[4];              // persistent work-queue counters
    long long spin_limit;           // iteration limit of every device-side wait
    int drop_signal;                // test hook: first look-back block never publishes
    int pad;
    unsigned long long work[4];     // pairs evaluated / composited: fwd 0-1, bwd 2-3
    unsigned fp64_count;            // ill-conditioned pairs listed by the projection (FP64 chain rule)
    unsigned pad1;
};

// Radix sort geometry (one onesweep pass = one 8-bit digit).  Small sorts use 1024-key
// block tiles (more blocks in flight), large ones 3840-key tiles (fewer look-back steps).
// rect.w of a pair: frame index, bit 31 set when the backward runs its geometric chain
// rule in FP64 (ill-conditioned footprint)
constexpr unsigned kRectFp64 = 1u << 31;
constexpr unsigned kRectFrame = kRectFp64 - 1u;

constexpr int kSortThreads = 256;
constexpr int kRadix = 256;
constexpr unsigned kSortSmallN = 1u << 20;
__host__ __device__ constexpr int sort_items(unsigned n_cap) { return n_cap <= kSortSmallN ? 4 : 15; }
__host__ __device__ constexpr unsigned sort_tile_keys(unsigned n_cap) {
    return (unsigned)(kSortThreads * sort_items(n_cap));
}
__host__ __device__ constexpr unsigned sort_tiles(unsigned n, unsigned n_cap) {
    return (n + sort_tile_keys(n_cap) - 1) / sort_tile_keys(n_cap);
}

// Emission block geometry (count scan + load-balanced key emission).
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitBlock = kEmitThreads * kEmitItems;  // 2048 pairs per block

// Workspace layout (byte offsets), computed on the host.
struct Layout {
    size_t hdr, frames;
    size_t feat0, feat1, feat2, rect, dkey[2], dval[2];
    size_t blocksum, blockprefix, offsets, chunk_first;
    size_t g0, g1, g2;
    size_t fp64_list;
    size_t ranges;
    size_t tkey[2], tval[2];
    size_t hist, look;
    size_t total;
    unsigned P, tiles, F;
    unsigned tiles_alloc;  // ranges capacity (tile count of the finest tiling, 8x8)
    unsigned key_cap;
    unsigned look_tiles;   // look-back tiles per buffer
    unsigned emit_blocks;
    int tile_bits;         // live bits of the global tile id
};

// Pointers into one workspace.
struct Work {
    DevHeader *hdr;
    DevFrame *frames;
    float4 *feat0, *feat1;
    float *feat2;
    uint4 *rect;
    unsigned *dkey[2], *dval[2];
    unsigned *blocksum, *blockprefix;
    unsigned *offsets;  // [P + 1] exclusive key offsets of the pairs in depth order
    unsigned *chunk_first;  // [key_cap / kEmitBlock + 1] depth-ordered pair owning a chunk's first key
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
};

struct GradPtrs {
    float *mean, *vel, *log_scale, *quat, *logit, *rgb;
};

struct FrameChunk {
    DevFrame f[kMaxFramesPerSetup];
};

// ---- host launchers (stream-ordered, no allocation) --------------------------------

// setup.cu
cudaError_t launch_setup(const Work &w, const FrameChunk &chunk, int first, int count, bool zero_all,
                         long long spin_limit, int drop_signal, cudaStream_t s);
const void *setup_kernel_ptr();
// project.cu
cudaError_t launch_project_fwd(const Work &w, const GaussPtrs &g, int tile_w, int tile_h, int num_sms,
                               cudaStream_t s);
cudaError_t launch_bin_from_screen(const Work &w, long long n, const float *u, const float *v,
                                   const float *ex, const float *ey, const float *depth,
                                   const uint8_t *valid, int tile_w, int tile_h, int32_t *counts,
                                   cudaStream_t s);
cudaError_t launch_project_bwd(const Work &w, const GaussPtrs &g, const GradPtrs &gr, int mode, int num_sms,
                               cudaStream_t s);
// FP64 chain rule of the pairs the projection flagged (may run concurrently with the above)
cudaError_t launch_project_bwd_fp64(const Work &w, const GaussPtrs &g, const GradPtrs &gr, int num_sms,
                                    cudaStream_t s);
// sort.cu
int sort_passes(int bits);
cudaError_t launch_radix_sort(const Work &w, unsigned *keys[2], unsigned *vals[2], const unsigned *n_dev,
                              unsigned n_cap, int bits, bool vals_identity, bool prepared, int hist_slot,
                              int ctr_slot, int num_sms, cudaStream_t s, int *result_buf);
// Warp-aggregated count of one 8-bit digit per lane into a shared histogram row.
__device__ __forceinline__ void count_digit(unsigned *row, unsigned d, unsigned active) {
    const unsigned peers = __match_any_sync(active, d);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(row + d, (unsigned)__popc(peers));
}
// binning.cu
cudaError_t launch_emit(const Work &w, int depth_buf, int tile_bits, int tile_hist_slot, int num_sms,
                        cudaStream_t s);
cudaError_t launch_ranges(const Work &w, int tile_buf, int num_sms, cudaStream_t s);
// composite.cu
cudaError_t launch_composite_fwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf,
                                 float bg0, float bg1, float bg2, float *image, float *final_T,
                                 int32_t *last_idx, int num_sms, cudaStream_t s);
cudaError_t launch_composite_bwd(const Work &w, int tile_w, int tile_h, int depth, int tile_buf,
                                 float bg0, float bg1, float bg2, const float *final_T,
                                 const int32_t *last_idx, const float *dL_dimage, int num_sms,
                                 cudaStream_t s);
// optim.cu
cudaError_t launch_l2_loss(const float *image, const float *target, long long n, float scale,
                           float *dL, float *loss, cudaStream_t s);
cudaError_t launch_adam(float *p, float *g, float *m, float *v, long long n, float lr, float b1,
                        float b2, float eps, float bc1, float bc2, int zero_grad, cudaStream_t s);
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

}  // namespace gvk
