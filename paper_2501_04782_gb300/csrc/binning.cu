// binning.cu -- per-call setup, tile-count prefix scan, key emission and tile ranges.
//
// Binning is two-level.  The pairs are first sorted by camera depth (one 32-bit radix
// sort over the P pairs), then each pair, in depth order, emits one key per tile its
// extent rectangle covers (row-major), and the keys are sorted stably by tile id only.
// The result is the unique list a stable sort of (tile << 32 | depth bits) keys emitted in
// pair order would give -- ordered by tile, then depth, then pair index -- but the
// expensive per-key sort touches only the live tile-id bits (one or two 8-bit passes
// instead of five or six).
#include <algorithm>

#include "gv_internal.cuh"

namespace gvk {

namespace {

__global__ void setup_kernel(Work w, FrameChunk chunk, int first, int count, int zero_all,
                             long long spin_limit, int drop_signal) {
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    int stride = gridDim.x * blockDim.x;
    for (int i = tid; i < count; i += stride) w.frames[first + i] = chunk.f[i];
    if (!zero_all) return;
    if (tid == 0) {
        DevHeader h = {};
        h.spin_limit = spin_limit;
        h.drop_signal = drop_signal;
        h.n_pairs = w.L.P;
        *w.hdr = h;
    }
    for (int i = tid; i < 8 * kRadix; i += stride) w.hist[i] = 0u;
    for (unsigned i = tid; i < w.L.tiles; i += stride) w.ranges[i] = make_uint2(0u, 0u);
    // look-back buffer 0 of the depth sort (its digits are counted by the projection)
    const unsigned nlook = sort_tiles(w.L.P, w.L.P) * kRadix;
    for (unsigned i = tid; i < nlook; i += stride) w.look[i] = 0u;
}

// Sum of the tile counts of each block of kEmitBlock pairs taken in depth order.
__global__ void __launch_bounds__(kEmitThreads) count_reduce_kernel(Work w, const unsigned *order) {
    __shared__ unsigned s_w[8];
    unsigned b = blockIdx.x;
    unsigned base = b * kEmitBlock;
    unsigned sum = 0;
    for (int i = 0; i < kEmitItems; i++) {
        unsigned idx = base + i * kEmitThreads + threadIdx.x;
        if (idx < w.L.P) {
            unsigned p = order[idx];
            if (p < w.L.P) sum += w.rect[p].z;  // ids are in range unless a bounded wait gave up
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        for (int i = 0; i < kEmitThreads / 32; i++) tot += s_w[i];
        w.blocksum[b] = tot;
    }
}

// Exclusive scan of the block sums (single block), total key count and capacity check.
__global__ void __launch_bounds__(1024) count_scan_kernel(Work w) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const unsigned nb = w.L.emit_blocks;
    for (unsigned base = 0; base < nb; base += 1024) {
        unsigned i = base + threadIdx.x;
        unsigned long long x = i < nb ? w.blocksum[i] : 0ull;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            unsigned long long t = s_w[lane], ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= o) ti += y;
            }
            s_w[lane] = ti - t;
        }
        __syncthreads();
        unsigned long long ex = s_carry + s_w[wid] + inc - x;
        // prefixes beyond the capacity are clamped: those blocks emit nothing
        if (i < nb) w.blockprefix[i] = (unsigned)min(ex, (unsigned long long)w.L.key_cap);
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = ex + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        unsigned long long K = s_carry;
        w.hdr->keys_total = K;
        w.hdr->keys_used = (unsigned)min(K, (unsigned long long)w.L.key_cap);
        if (K > w.L.key_cap) atomicOr(&w.hdr->err, ERR_CAPACITY);
    }
}

// Tile-sort digit counts of one tile-id range [t0, t0 + len) (a row of a pair's tile
// rectangle): digit 0 through a difference array over its 256 values (the range wraps
// around len >> 8 times plus a partial run), higher digits directly (a row spans one or two
// of their values).
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

// Exclusive key offsets of every pair in depth order: off[i] for i < P, off[P] = K.
// Block b scans its kEmitBlock pairs and adds the block prefix.  Each pair also records
// the emission chunks whose first key it owns.
__global__ void __launch_bounds__(kEmitThreads) offsets_kernel(Work w, const unsigned *order) {
    __shared__ unsigned s_w[8];
    const unsigned b = blockIdx.x, base = b * kEmitBlock;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    // blocked: thread t owns pairs base + t*8 .. +7
    unsigned c[kEmitItems], sum = 0;
#pragma unroll
    for (int i = 0; i < kEmitItems; i++) {
        unsigned idx = base + t * kEmitItems + i;
        unsigned p = idx < w.L.P ? order[idx] : 0u;
        if (p >= w.L.P) p = 0u;  // ids are in range unless a bounded wait gave up
        c[i] = idx < w.L.P ? w.rect[p].z : 0u;
        sum += c[i];
    }
    unsigned inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    unsigned run = w.blockprefix[b] + inc - sum;
    for (int q = 0; q < wid; q++) run += s_w[q];
    const unsigned cap = w.L.key_cap;
#pragma unroll
    for (int i = 0; i < kEmitItems; i++) {
        unsigned idx = base + t * kEmitItems + i;
        if (idx < w.L.P) {
            const unsigned lo = min(run, cap), hi = min(run + c[i], cap);
            w.offsets[idx] = lo;
            // this pair owns the first key of every emission chunk starting in [lo, hi)
            for (unsigned ch = (lo + kEmitBlock - 1) / kEmitBlock; ch * kEmitBlock < hi; ch++) w.chunk_first[ch] = idx;
        }
        run += c[i];
    }
    if (b == 0 && t == 0) w.offsets[w.L.P] = w.hdr->keys_used;
}

// Flush a block's tile-sort digit counts: digit 0 from its difference array (prefix sum
// plus the full wraps), higher digits as counted.
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

// Key emission balanced over keys: each block iteration takes kEmitBlock consecutive
// keys and finds the pair owning every key with a load-balancing search: the pairs whose
// keys fall in the chunk (a window of the depth-ordered offsets starting at the chunk's
// owner recorded by offsets_kernel; every pair in it owns at least one key, pairs with no
// key sort last) mark their first key, and an inclusive max scan over the chunk carries
// each mark forward.  Keys are written coalesced as (tile id,
// pair id), the tiles of a pair in row-major order.  Also counts the tile-sort digit
// histograms.
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(Work w, const unsigned *order, int tile_passes,
                                                            unsigned *tile_hist) {
    __shared__ int s_owner[kEmitBlock];
    __shared__ unsigned s_off[kEmitBlock + 1];
    __shared__ unsigned s_pair[kEmitBlock];
    __shared__ int s_wmax[kEmitThreads / 32];
    __shared__ unsigned s_lo, s_n;
    __shared__ int s_diff[257];
    __shared__ unsigned s_full;
    __shared__ unsigned s_h[4][kRadix];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < 257; i += kEmitThreads) s_diff[i] = 0;
    for (int i = t; i < 4 * kRadix; i += kEmitThreads) (&s_h[0][0])[i] = 0u;
    if (t == 0) s_full = 0u;
    const unsigned K = w.hdr->keys_used;
    const unsigned P = w.L.P;
    const unsigned *off = w.offsets;
    const unsigned nchunks = (K + kEmitBlock - 1) / kEmitBlock;
    {   // look-back buffer 0 of the tile sort (the depth sort is finished with it)
        const unsigned nlook = sort_tiles(K, w.L.key_cap) * kRadix;
        for (unsigned i = blockIdx.x * blockDim.x + t; i < nlook; i += gridDim.x * blockDim.x) w.look[i] = 0u;
    }
    for (unsigned chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const unsigned k0 = chunk * kEmitBlock;
        const unsigned kb = min(K - k0, (unsigned)kEmitBlock);
        __syncthreads();
        if (t == 0) {
            // the pairs owning this chunk's keys run from the owner of its first key to the
            // owner of the next chunk's first key (pairs after the last key own nothing here)
            const unsigned lo = min(w.chunk_first[chunk], P - 1u);
            const unsigned hi = chunk + 1 < nchunks ? min(w.chunk_first[chunk + 1], P - 1u) : P - 1u;
            s_lo = lo;
            s_n = min(hi >= lo ? hi - lo + 1 : 1u, (unsigned)kEmitBlock);
        }
        for (int i = t; i < kEmitBlock; i += kEmitThreads) s_owner[i] = -1;
        __syncthreads();
        const unsigned plo = s_lo, np = s_n;
        for (unsigned i = t; i <= np; i += kEmitThreads) {
            const unsigned o = off[plo + i];  // plo + np <= P: off[P] = K
            s_off[i] = o;
            if (i == np) break;
            const unsigned p = order[plo + i];
            s_pair[i] = p < P ? p : 0u;  // in range unless a bounded wait gave up
            const unsigned first = o > k0 ? o - k0 : 0u;
            if (first < kb) s_owner[first] = (int)i;
        }
        __syncthreads();
        // inclusive max scan of s_owner: thread t owns entries t*8 .. t*8+7
        int run = -1;
        int v[kEmitItems];
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            v[i] = s_owner[t * kEmitItems + i];
            run = max(run, v[i]);
            v[i] = run;
        }
        int incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = max(incl, y);
        }
        if (lane == 31) s_wmax[wid] = incl;
        __syncthreads();
        int carry = -1;
        for (int q = 0; q < wid; q++) carry = max(carry, s_wmax[q]);
        int excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = -1;
        carry = max(carry, excl);
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) s_owner[t * kEmitItems + i] = max(carry, v[i]);
        __syncthreads();
        for (unsigned r0 = 0; r0 < (unsigned)kEmitBlock; r0 += kEmitThreads) {
            const unsigned e = r0 + t;
            if (e < kb) {
                const int i = max(s_owner[e], 0);
                const unsigned j = k0 + e - s_off[i];
                const unsigned p = s_pair[i];
                const uint4 r = w.rect[p];  // consecutive keys mostly share a pair: L1 hits
                const DevFrame &fr = w.frames[min(r.w & kRectFrame, w.L.F - 1u)];
                const unsigned tx0 = r.x & 0xFFFFu, ty0 = r.x >> 16, tx1 = r.y & 0xFFFFu;
                const unsigned wr = tx1 - tx0 + 1u;
                // j / wr through the FP32 reciprocal, corrected to the exact quotient (j < 2^24)
                unsigned q = (unsigned)((float)j * __frcp_rn((float)wr));
                int rem = (int)j - (int)(q * wr);
                if (rem < 0) { q--; rem += (int)wr; }
                else if (rem >= (int)wr) { q++; rem -= (int)wr; }
                const unsigned tile = min(fr.tile_offset + (ty0 + q) * fr.tiles_x + tx0 + (unsigned)rem, w.L.tiles - 1u);
                w.tkey[0][k0 + e] = tile;
                w.tval[0][k0 + e] = p;
                // the key starting a row run (in this chunk) counts the run's tile digits
                if (tile_passes > 0 && (rem == 0 || e == 0)) {
                    const unsigned pair_end = min(s_off[i + 1], k0 + kb);  // this pair's keys end here
                    const unsigned len = min(wr - (unsigned)rem, pair_end - (k0 + e));
                    count_tile_run(tile, len, tile_passes, s_diff, &s_full, s_h);
                }
            }
        }
    }
    if (tile_passes == 0) return;
    __syncthreads();
    flush_tile_hist(tile_passes, s_diff, s_full, s_h, tile_hist);
}

// Per-tile [start, end) of the sorted keys.  A warp takes 32 * kRangeItems consecutive keys
// per round (lane l holds keys l, l + 32, ...: independent coalesced loads in flight) and
// gets each key's neighbours by shuffles; only the round's two outer neighbours are loaded.
constexpr int kRangeItems = 8;

__global__ void __launch_bounds__(256) ranges_kernel(Work w, const unsigned *keys) {
    const unsigned n = w.hdr->keys_used;
    const int lane = threadIdx.x & 31;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    const unsigned span = 32u * kRangeItems;
    for (unsigned base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * span; base < n;
         base += warps * span) {
        unsigned k[kRangeItems];
#pragma unroll
        for (int j = 0; j < kRangeItems; j++) {
            const unsigned i = base + 32u * j + lane;
            k[j] = i < n ? keys[i] : 0xFFFFFFFFu;
        }
        const unsigned before = base > 0 ? keys[base - 1] : 0xFFFFFFFFu;  // same address for all lanes
        const unsigned after = base + span < n ? keys[base + span] : 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < kRangeItems; j++) {
            const unsigned i = base + 32u * j + lane;
            unsigned prev = __shfl_up_sync(0xffffffffu, k[j], 1);
            const unsigned prev_row = __shfl_sync(0xffffffffu, j > 0 ? k[j > 0 ? j - 1 : 0] : before, 31);
            if (lane == 0) prev = j > 0 ? prev_row : before;
            unsigned next = __shfl_down_sync(0xffffffffu, k[j], 1);
            const unsigned next_row = __shfl_sync(0xffffffffu, j + 1 < kRangeItems ? k[j + 1 < kRangeItems ? j + 1 : j] : after, 0);
            if (lane == 31) next = j + 1 < kRangeItems ? next_row : after;
            const unsigned t = k[j];
            if (i >= n || t >= w.L.tiles) continue;  // tile ids are in range unless a wait gave up
            if (i == 0 || prev != t) w.ranges[t].x = i;
            if (i == n - 1 || next != t) w.ranges[t].y = i + 1;
        }
    }
}

__global__ void gather_debug_kernel(Work w, float *mean2d, float *conic, float *opacity, float *depth,
                                    int32_t *counts, int depth_buf) {
    unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned P = w.L.P;
    if (p >= P) return;
    float4 a = w.feat0[p], b = w.feat1[p];
    if (mean2d) { mean2d[p] = a.x; mean2d[P + p] = a.y; }
    if (conic) {  // the staged record holds -log2(e) (A/2, B, C/2)
        conic[p] = -2.f * kLn2 * a.z;
        conic[P + p] = -kLn2 * a.w;
        conic[2 * P + p] = -2.f * kLn2 * b.x;
    }
    if (opacity) opacity[p] = exp2f(b.y);
    if (counts) counts[p] = (int32_t)w.rect[p].z;
    // position p of the depth-sorted list holds (depth key, pair id); culled pairs: NaN
    if (depth) depth[w.dval[depth_buf][p]] = __uint_as_float(w.dkey[depth_buf][p]);
}

}  // namespace

const void *setup_kernel_ptr() { return (const void *)setup_kernel; }

cudaError_t launch_setup(const Work &w, const FrameChunk &chunk, int first, int count, bool zero_all,
                         long long spin_limit, int drop_signal, cudaStream_t s) {
    unsigned work = zero_all ? max(max(w.L.tiles, (unsigned)(8 * kRadix)), sort_tiles(w.L.P, w.L.P) * kRadix)
                             : (unsigned)count;
    unsigned blocks = min((work + 255u) / 256u, 1024u);
    if (blocks == 0) blocks = 1;
    setup_kernel<<<blocks, 256, 0, s>>>(w, chunk, first, count, zero_all ? 1 : 0, spin_limit, drop_signal);
    return cudaGetLastError();
}

cudaError_t launch_emit(const Work &w, int depth_buf, int tile_bits, int tile_hist_slot, int num_sms, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    const unsigned *order = w.dval[depth_buf];
    count_reduce_kernel<<<w.L.emit_blocks, kEmitThreads, 0, s>>>(w, order);
    count_scan_kernel<<<1, 1024, 0, s>>>(w);
    int passes = tile_bits <= 0 ? 0 : (tile_bits + 7) / 8;
    offsets_kernel<<<w.L.emit_blocks, kEmitThreads, 0, s>>>(w, order);
    unsigned chunks = (w.L.key_cap + kEmitBlock - 1) / kEmitBlock;
    unsigned grid = std::max(1u, std::min(chunks, (unsigned)num_sms * 8u));
    emit_kernel<<<grid, kEmitThreads, 0, s>>>(w, order, passes, w.hist + (size_t)tile_hist_slot * kRadix);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const Work &w, int tile_buf, int num_sms, cudaStream_t s) {
    ranges_kernel<<<num_sms * 8, 256, 0, s>>>(w, w.tkey[tile_buf]);
    return cudaGetLastError();
}

cudaError_t launch_gather_debug(const Work &w, float *mean2d, float *conic, float *opacity, float *depth,
                                int32_t *counts, int depth_buf, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    gather_debug_kernel<<<(w.L.P + 255) / 256, 256, 0, s>>>(w, mean2d, conic, opacity, depth, counts, depth_buf);
    return cudaGetLastError();
}

}  // namespace gvk
