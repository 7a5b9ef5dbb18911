// binning.cu -- per-call setup, cell offsets, key emission fused with the first pass of
// the tile sort, and tile ranges.
//
// Binning is two-level.  The pairs are first sorted by camera depth (one 32-bit radix
// sort over the P pairs), then each pair, in depth order, enumerates its cells (the tiles
// of its extent box, row-major) and emits a key for every cell the cull keeps, and the
// keys are sorted stably by tile id only.  The result is the unique list a stable sort of
// (tile << 32 | depth bits) keys emitted in pair order would give -- ordered by tile, then
// depth, then pair index -- but the per-key sort touches only the live tile-id bits, and
// its first 8-bit pass happens during emission: the emitted keys are ranked by their low
// tile digit inside each chunk and scattered straight to their first-pass positions.
#include <algorithm>
#include <cstddef>

#include "gv_internal.cuh"

namespace gvk {

namespace {

__global__ void setup_kernel(Work w, FrameChunk chunk, int first, int count, int zero_all,
                             long long spin_limit, int drop_signal) {
    pdl_prologue();
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
    // each tile's [start, end) is recorded by min / max over the runs of its id in the final
    // list (start >= end: an empty tile)
    for (unsigned i = tid; i < w.L.tiles; i += stride) w.ranges[i] = make_uint2(0xFFFFFFFFu, 0u);
    for (unsigned i = tid; i < w.L.emit_blocks; i += stride) w.scan_look[i] = 0ull;
    // look-back buffer 0 of the depth sort (its digits are counted by the projection)
    const unsigned nlook = sort_tiles(w.L.P, w.L.P) * kRadix;
    for (unsigned i = tid; i < nlook; i += stride) w.look[i] = 0u;
}

// Cell offsets in one pass.  Each block takes the next run of kEmitBlock depth-ordered
// drawn pairs from a ticket counter, scans their cell counts (the tiles of their extent
// boxes), gets the cells of all earlier runs by decoupled look-back over 64-bit status words
// (flag in the top two bits), and writes every pair's exclusive offset: off[i] for
// i < n_drawn, off[n_drawn] = cells.  Each pair records the emission chunks whose first cell
// it owns, and each block clears the emission's look-back words of the chunks that start in
// its cells (warp 0 walks the look-back, 32 predecessors per poll).  The block holding the
// last run checks the capacities: the kept keys (counted
// by the projection) against the key capacity, the cells against the chunk table; on
// overflow keys_total reports the key capacity the call needs.  Every wait is bounded: a
// look-back that gives up sets ERR_TIMEOUT (the offsets are then wrong but every write
// stays in bounds).
constexpr unsigned long long kScanAgg = 1ull << 62, kScanInc = 2ull << 62, kScanVal = (1ull << 62) - 1ull;
constexpr int kScanCtr = 12;

__device__ __forceinline__ void finish_cells(Work &w, unsigned long long cells) {
    const unsigned long long K = w.hdr->keys_total;
    const unsigned long long chunks = (cells + kEmitBlock - 1) / kEmitBlock;
    bool over = K > w.L.key_cap;
    const bool table = chunks > w.L.chunk_cap || cells > 0xFFFFFFFFull;
    if (table) {
        over = true;
        const unsigned long long need = (cells + kCellsPerKey - 1) / kCellsPerKey + kEmitBlock;
        w.hdr->keys_total = max(K, need);
    }
    w.hdr->cells = cells;
    w.hdr->keys_used = (unsigned)min(K, (unsigned long long)w.L.key_cap);
    w.hdr->n_chunks = table ? 0u : (unsigned)chunks;
    if (over) atomicOr(&w.hdr->err, ERR_CAPACITY);
}

__global__ void __launch_bounds__(kEmitThreads) cell_offsets_kernel(Work w, const unsigned *order) {
    pdl_prologue();
    __shared__ unsigned long long s_w[kEmitThreads / 32];
    __shared__ unsigned long long s_excl;
    __shared__ unsigned s_blk;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned P = w.L.P, nd = min(w.hdr->n_drawn, P);
    const unsigned nblk = (nd + kEmitBlock - 1) / kEmitBlock;
    const long long limit = w.hdr->spin_limit;
    unsigned *look0 = w.look;  // the emission's look-back words (buffer 0)
    if (nblk == 0) {
        if (blockIdx.x == 0 && t == 0) {
            w.offsets[0] = 0u;
            finish_cells(w, 0ull);
        }
        return;
    }
    for (;;) {
        if (t == 0) s_blk = atomicAdd(&w.hdr->sort_ctr[kScanCtr], 1u);
        __syncthreads();
        const unsigned b = s_blk;
        if (b >= nblk) break;
        const unsigned base = b * kEmitBlock;
        // blocked: thread t owns the pairs base + 8t .. base + 8t + 7
        unsigned c[kEmitItems];
        unsigned long long sum = 0;
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            const unsigned idx = base + t * kEmitItems + i;
            unsigned p = idx < nd ? order[idx] : 0u;
            if (p >= P) p = 0u;  // ids are in range unless a bounded wait gave up
            c[i] = idx < nd ? w.rect[p].z : 0u;
            sum += c[i];
        }
        unsigned long long inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[wid] = inc;
        __syncthreads();
        if (wid == 0) {  // warp 0 publishes this run's cells and finds the cells before it
            unsigned long long total = 0;
            for (int q = 0; q < kEmitThreads / 32; q++) total += s_w[q];
            unsigned long long excl = 0;
            if (b == 0) {
                if (lane == 0) atomicExch(&w.scan_look[0], kScanInc | (total & kScanVal));
            } else {
                if (lane == 0) atomicExch(&w.scan_look[b], kScanAgg | (total & kScanVal));
                // lane l reads predecessor j - l: one poll covers 32 runs; the walk ends at the
                // nearest inclusive prefix, and waits at the nearest unpublished status
                long long spins = 0;
                int j = (int)b - 1;
                for (;;) {
                    const int idx = j - lane;
                    const unsigned long long past = kScanInc;  // before run 0: an empty prefix
                    const unsigned long long st =
                        idx >= 0 ? *((volatile unsigned long long *)&w.scan_look[idx]) : past;
                    const unsigned long long fl = st & ~kScanVal;
                    const unsigned stop = __ballot_sync(0xffffffffu, fl != kScanAgg);
                    const int first = stop ? __ffs(stop) - 1 : 32;
                    unsigned long long v = (lane < first || (lane == first && fl == kScanInc)) ? (st & kScanVal) : 0ull;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    excl += v;
                    if (first == 32) {
                        j -= 32;
                        spins = 0;
                        continue;
                    }
                    const bool inc = __shfl_sync(0xffffffffu, fl == kScanInc, first);
                    if (inc) break;
                    j -= first;  // the aggregates before the unpublished status are taken
                    if (first > 0) {
                        spins = 0;
                        continue;
                    }
                    bool quit = ++spins > limit || (*((volatile unsigned *)&w.hdr->err) & ERR_TIMEOUT);
                    quit = __shfl_sync(0xffffffffu, quit, 0);
                    if (quit) {
                        if (lane == 0) atomicOr(&w.hdr->err, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                }
                if (lane == 0) atomicExch(&w.scan_look[b], kScanInc | ((excl + total) & kScanVal));
            }
            if (lane == 0) {
                s_excl = excl;
                if (b == nblk - 1) {
                    w.offsets[nd] = (unsigned)min(excl + total, 0xFFFFFFFFull);
                    finish_cells(w, excl + total);
                }
            }
        }
        __syncthreads();
        unsigned long long run = s_excl + inc - sum;
        for (int q = 0; q < wid; q++) run += s_w[q];
        const unsigned long long blk_lo = s_excl;
        unsigned long long blk_hi = s_excl;
        for (int q = 0; q < kEmitThreads / 32; q++) blk_hi += s_w[q];
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            const unsigned idx = base + t * kEmitItems + i;
            if (idx < nd) {
                const unsigned long long lo = run, hi = run + c[i];
                w.offsets[idx] = (unsigned)min(lo, 0xFFFFFFFFull);
                // this pair owns the first cell of every emission chunk starting in [lo, hi)
                for (unsigned long long ch = (lo + kEmitBlock - 1) / kEmitBlock;
                     ch < w.L.chunk_cap && ch * kEmitBlock < hi; ch++)
                    w.chunk_first[ch] = idx;
            }
            run += c[i];
        }
        // the emission chunks starting in this block's cells: clear their look-back words
        const unsigned long long ch0 = (blk_lo + kEmitBlock - 1) / kEmitBlock;
        const unsigned long long ch1 = min((blk_hi + kEmitBlock - 1) / kEmitBlock, (unsigned long long)w.L.chunk_cap);
        for (unsigned long long i = ch0 * kRadix + t; i < ch1 * kRadix; i += kEmitThreads) look0[i] = 0u;
        __syncthreads();
    }
}

// Key emission fused with the first pass of the tile sort, balanced over cells.  Each
// block iteration takes the next chunk of kEmitBlock consecutive cells (in the order the
// offsets define: pairs by depth, each pair's extent-box tiles row-major) from an atomic
// counter and finds the pair owning every cell with a load-balancing search: the pairs
// whose cells fall in the chunk (a window of the depth-ordered offsets starting at the
// chunk's owner recorded by cell_offsets_kernel) mark their first cell, and an inclusive max
// scan over the chunk carries each mark forward.  While the window is read, the records of
// its first kEmitStage pairs (pixel box, frame, screen mean, cull record) are staged in
// shared memory, so the cells read them there instead of gathering them from L2 cell by
// cell (8 x 1920x1080 / 1M: emission 1.22 -> 1.09 ms).  A cell is a key when the cull keeps its
// tile (cull_tiles, as the projection counted).  The keys are ranked stably by their low
// tile digit inside the chunk (warp match + per-warp histograms, in cell order) and staged
// in shared memory in digit order; then the per-digit counts of all earlier chunks come
// from decoupled look-back (walked after the staging, which gives the earlier chunks that
// much longer to publish: 8 x 1920x1080 / 1M emission 1.093 -> 1.065 ms), and (tile id, pair
// id) is scattered to its first-pass position: out of this kernel the kept keys are
// compacted and sorted by the low tile digit, in depth order within a digit.  The global
// digit offsets come from the projection's counts of the kept keys.
constexpr int kEmitSmemFrames = 64;
// pairs of a chunk whose records are staged in shared memory (8 x 1920x1080 / 1M: emission
// 1.060 ms with 128, 1.034 ms with 256)
constexpr int kEmitStage = 256;
constexpr int kEmitLookWindow = 4;  // predecessors read per poll of the emission's look-back

struct EmitSortArgs {
    const unsigned *order;  // depth-sorted pair ids
    unsigned *keys_out, *vals_out;
    const unsigned *hist;   // low-digit counts of all kept keys
    unsigned *ctr;          // chunk counter
    unsigned *look_next;    // look-back buffer of the next tile-sort pass (cleared here)
    uint2 *ranges;          // tile ids of one digit: this pass is the whole sort, so it also
                            // records each tile's [start, end) (RANGES)
    int lw, lh;
};

template <bool RANGES>
__global__ void __launch_bounds__(kEmitThreads, 4) emit_sort_kernel(Work w, EmitSortArgs a) {
    pdl_prologue();
    __shared__ int s_owner[kEmitBlock];          // later: the chunk's keys, reordered by digit
    __shared__ unsigned s_off[kEmitBlock + 1];
    __shared__ unsigned s_pair[kEmitBlock];      // later: their pair ids
    __shared__ unsigned s_whist[8][kRadix];
    __shared__ unsigned s_gexcl[kRadix], s_dstart[kRadix], s_gbase[kRadix];
    __shared__ unsigned s_scan[24];
    __shared__ int s_wmax[kEmitThreads / 32];
    __shared__ unsigned s_chunk, s_lo, s_n;
    __shared__ int s_abort;
    __shared__ uint2 s_frames[kEmitSmemFrames];  // (tile_offset, tiles_x) of the first frames
    // records of the chunk's first kEmitStage pairs: pixel box, frame (tile_offset, tiles_x),
    // screen mean, cull record (the cells of later pairs read them from global memory)
    __shared__ uint2 s_pbox[kEmitStage], s_pfg[kEmitStage];
    __shared__ float2 s_puv[kEmitStage];
    __shared__ float4 s_pell[kEmitStage];
    unsigned *s_keys = reinterpret_cast<unsigned *>(s_owner);
    unsigned *s_vals = s_pair;
    // a call whose capacity check failed keeps no list: nothing to emit (the decision is the
    // block's, as a wait of another block may set a timeout meanwhile)
    if (__syncthreads_or(*((volatile unsigned *)&w.hdr->err) != 0u)) return;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned P = w.L.P, nchunks = w.hdr->n_chunks, nd = min(w.hdr->n_drawn, P);
    const unsigned cells = (unsigned)min(w.hdr->cells, 0xFFFFFFFFull);
    const unsigned *off = w.offsets;
    const long long limit = w.hdr->spin_limit;
    const unsigned next_tiles = sort_tiles(w.hdr->keys_used, w.L.key_cap);
    for (unsigned i = blockIdx.x * kEmitThreads + t; i < next_tiles * kRadix; i += gridDim.x * kEmitThreads)
        a.look_next[i] = 0u;
    for (int i = t; i < (int)min(w.L.F, (unsigned)kEmitSmemFrames); i += kEmitThreads)
        s_frames[i] = make_uint2(w.frames[i].tile_offset, w.frames[i].tiles_x);
    {
        unsigned ex;
        block_excl_scan_256(a.hist[t], s_scan, ex);
        s_gexcl[t] = ex;
    }
    for (;;) {
        if (t == 0) { s_chunk = atomicAdd(a.ctr, 1u); s_abort = 0; }
        for (int i = t; i < 8 * kRadix; i += kEmitThreads) (&s_whist[0][0])[i] = 0u;
        for (int i = t; i < kEmitBlock; i += kEmitThreads) s_owner[i] = -1;
        __syncthreads();
        const unsigned chunk = s_chunk;
        if (chunk >= nchunks) break;
        const unsigned k0 = chunk * kEmitBlock;
        const unsigned kb = min(cells - k0, (unsigned)kEmitBlock);
        if (t == 0) {
            // the pairs owning this chunk's cells run from the owner of its first cell to the
            // owner of the next chunk's first cell (pairs after the last cell own nothing here)
            const unsigned lo = min(w.chunk_first[chunk], nd - 1u);  // chunks exist only when nd > 0
            const unsigned hi = chunk + 1 < nchunks ? min(w.chunk_first[chunk + 1], nd - 1u) : nd - 1u;
            s_lo = lo;
            s_n = min(hi >= lo ? hi - lo + 1 : 1u, (unsigned)kEmitBlock);
        }
        __syncthreads();
        const unsigned plo = s_lo, np = s_n;
        for (unsigned i = t; i <= np; i += kEmitThreads) {
            const unsigned o = off[plo + i];  // plo + np <= nd: off[nd] = cells
            s_off[i] = o;
            if (i == np) break;
            const unsigned p = min(a.order[plo + i], P - 1u);  // in range unless a bounded wait gave up
            s_pair[i] = p;
            const unsigned first = o > k0 ? o - k0 : 0u;
            if (first < kb) s_owner[first] = (int)i;
            if (i < (unsigned)kEmitStage) {
                const uint4 r = w.rect[p];
                const float4 f0 = w.feat0[p];
                const unsigned fi = min(r.w & kRectFrame, w.L.F - 1u);
                s_pbox[i] = make_uint2(r.x, r.y);
                s_pfg[i] = fi < (unsigned)kEmitSmemFrames ? s_frames[fi]
                                                          : make_uint2(w.frames[fi].tile_offset, w.frames[fi].tiles_x);
                s_puv[i] = make_float2(f0.x, f0.y);
                s_pell[i] = w.ell[p];
            }
        }
        __syncthreads();
        {   // inclusive max scan of s_owner: thread t owns entries t*8 .. t*8+7
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
        }
        __syncthreads();
        // cells of this thread: warp w owns cells [256 w, 256 w + 256), lane l cells l, l + 32, ...
        unsigned key[kEmitItems], val[kEmitItems], rank[kEmitItems];
        unsigned kept = 0;  // bit i: cell i is a key
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            const unsigned e = wid * (32 * kEmitItems) + i * 32 + lane;
            key[i] = 0u;
            val[i] = 0u;
            if (e < kb) {
                const int oi = max(s_owner[e], 0);
                const unsigned j = k0 + e - s_off[oi];
                const unsigned p = s_pair[oi];
                uint2 box, fg;
                float2 uv;
                float4 el;
                if (oi < kEmitStage) {
                    box = s_pbox[oi];
                    fg = s_pfg[oi];
                    uv = s_puv[oi];
                    el = s_pell[oi];
                } else {
                    const uint4 r = w.rect[p];
                    const unsigned fi = min(r.w & kRectFrame, w.L.F - 1u);
                    box = make_uint2(r.x, r.y);
                    fg = fi < (unsigned)kEmitSmemFrames ? s_frames[fi]
                                                        : make_uint2(w.frames[fi].tile_offset, w.frames[fi].tiles_x);
                    const float4 f0 = w.feat0[p];
                    uv = make_float2(f0.x, f0.y);
                    el = w.ell[p];
                }
                const PixBox bx = unpack_box(make_uint4(box.x, box.y, 0u, 0u));
                const unsigned tx0 = (unsigned)bx.x0 >> a.lw, ty0 = (unsigned)bx.y0 >> a.lh;
                const unsigned wr = ((unsigned)bx.x1 >> a.lw) - tx0 + 1u;
                // j / wr through the FP32 reciprocal, corrected to the exact quotient (j < 2^24)
                unsigned q = (unsigned)((float)j * __frcp_rn((float)wr));
                int rem = (int)j - (int)(q * wr);
                if (rem < 0) { q--; rem += (int)wr; }
                else if (rem >= (int)wr) { q++; rem -= (int)wr; }
                const int tx = (int)tx0 + rem, ty = (int)(ty0 + q);
                int t0, t1;
                if (cull_tiles(uv.x, uv.y, el, bx, ty, a.lw, a.lh, t0, t1) && tx >= t0 && tx <= t1) {
                    key[i] = min(fg.x + (unsigned)ty * fg.y + (unsigned)tx, w.L.tiles - 1u);
                    val[i] = p;
                    kept |= 1u << i;
                }
            }
        }
        // stable rank of the keys inside the warp (by item, then by lane); a cell that is not
        // a key matches no lane but itself and is not counted
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            const bool live = (kept >> i) & 1u;
            const unsigned d = key[i] & 255u;
            const unsigned peers = __match_any_sync(0xffffffffu, live ? d : 0x100u + (unsigned)lane);
            unsigned before = 0;
            if (live) before = s_whist[wid][d];
            rank[i] = before + __popc(peers & lanemask_lt());
            __syncwarp();
            if (live && lane == __ffs(peers) - 1) s_whist[wid][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread t owns digit t: exclusive offsets over warps, chunk total
        unsigned total = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const unsigned c = s_whist[q][t];
            s_whist[q][t] = total;
            total += c;
        }
        // the chunk's counts are published at once (digits above the tile ids' live bits hold
        // no key: no look-back for them); its keys go to shared memory in digit order before
        // it walks its predecessors
        const bool dig = t < (1 << min(8, w.L.tile_bits));
        if (dig) lookback_publish(w.look, chunk, (unsigned)t, total, false);
        unsigned dex;
        const unsigned nkeys = block_excl_scan_256(total, s_scan, dex);
        s_dstart[t] = dex;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            if (!((kept >> i) & 1u)) continue;
            const unsigned d = key[i] & 255u;
            const unsigned pos = s_dstart[d] + s_whist[wid][d] + rank[i];
            s_keys[pos] = key[i];
            s_vals[pos] = val[i];
        }
        bool gave_up = false;
        const unsigned excl =
            dig ? lookback_walk<kEmitLookWindow>(w.look, chunk, (unsigned)t, total, w.hdr, limit, gave_up) : 0u;
        if (gave_up) s_abort = 1;
        s_gbase[t] = s_gexcl[t] + excl;
        __syncthreads();
        if (!s_abort) {
            for (unsigned pos = t; pos < nkeys; pos += kEmitThreads) {
                const unsigned k = s_keys[pos];
                const unsigned d = k & 255u;
                const unsigned gpos = s_gbase[d] + pos - s_dstart[d];
                if (gpos < w.L.key_cap) {
                    a.keys_out[gpos] = k;
                    a.vals_out[gpos] = s_vals[pos];
                    if (RANGES) {  // runs of equal tile ids are contiguous in the chunk's order
                        if (pos == 0 || s_keys[pos - 1] != k) atomicMin(&a.ranges[k].x, gpos);
                        if (pos + 1 == nkeys || s_keys[pos + 1] != k) atomicMax(&a.ranges[k].y, gpos + 1u);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Per-tile [start, end) of the sorted keys, for lists of more than kFusedRangesKeys keys of
// capacity (the kernel that writes a smaller final list records them itself).  A warp takes 32 * kRangeItems consecutive keys
// per round (lane l holds keys l, l + 32, ...: independent coalesced loads in flight) and
// gets each key's neighbours by shuffles; only the round's two outer neighbours are loaded.
constexpr int kRangeItems = 8;

__global__ void __launch_bounds__(256) ranges_kernel(Work w, const unsigned *keys) {
    pdl_prologue();
    const unsigned n = w.hdr->err != 0u ? 0u : w.hdr->keys_used;  // a failed call's tiles stay empty
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

// The tile ranges for the debug read: an empty tile (start >= end) reads as (0, 0).
__global__ void debug_ranges_kernel(Work w, uint2 *out) {
    pdl_prologue();
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < w.L.tiles; t += gridDim.x * blockDim.x) {
        const uint2 r = w.ranges[t];
        out[t] = r.x < r.y ? r : make_uint2(0u, 0u);
    }
}

__global__ void gather_debug_kernel(Work w, float *mean2d, float *conic, float *opacity, float *depth,
                                    int32_t *counts, int depth_buf) {
    pdl_prologue();
    unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned P = w.L.P;
    if (p >= P) return;
    const unsigned nd = min(w.hdr->n_drawn, P);
    float4 a = w.feat0[p], b = w.feat1[p];
    if (mean2d) { mean2d[p] = a.x; mean2d[P + p] = a.y; }
    if (conic) {  // the staged record holds -log2(e) (A/2, B, C/2)
        conic[p] = -2.f * kLn2 * a.z;
        conic[P + p] = -kLn2 * a.w;
        conic[2 * P + p] = -2.f * kLn2 * b.x;
    }
    if (opacity) opacity[p] = exp2f(b.y);
    if (counts) counts[p] = (int32_t)w.rect[p].z;
    // position p < n_drawn of the depth-sorted list holds (depth key, pair id); culled pairs
    // are not in it (the caller's initial value stays)
    if (depth && p < nd) depth[min(w.dval[depth_buf][p], P - 1u)] = __uint_as_float(w.dkey[depth_buf][p]);
}

}  // namespace

const void *setup_kernel_ptr() { return (const void *)setup_kernel; }

cudaError_t launch_setup(const Work &w, const FrameChunk &chunk, int first, int count, bool zero_all,
                         long long spin_limit, int drop_signal, cudaStream_t s) {
    unsigned work = zero_all ? max(max(w.L.tiles, (unsigned)(8 * kRadix)), sort_tiles(w.L.P, w.L.P) * kRadix)
                             : (unsigned)count;
    unsigned blocks = min((work + 255u) / 256u, 1024u);
    if (blocks == 0) blocks = 1;
    launch_pdl(setup_kernel, blocks, 256, 0, s, w, chunk, first, count, zero_all ? 1 : 0, spin_limit, drop_signal);
    return cudaGetLastError();
}

cudaError_t launch_emit(const Work &w, int depth_buf, int tile_w, int tile_h, int num_sms, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    const unsigned *order = w.dval[depth_buf];
    launch_pdl(cell_offsets_kernel, std::max(1u, std::min(w.L.emit_blocks, (unsigned)num_sms * 4u)), kEmitThreads,
               0, s, w, order);
    EmitSortArgs a;
    a.order = order;
    a.keys_out = w.tkey[1];
    a.vals_out = w.tval[1];
    a.hist = w.hist + 4 * kRadix;
    a.ctr = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(w.hdr) + offsetof(DevHeader, sort_ctr)) + 4;
    a.look_next = w.look + (size_t)w.L.look_tiles * kRadix;
    a.ranges = w.ranges;
    a.lw = __builtin_ctz(tile_w);
    a.lh = __builtin_ctz(tile_h);
    const unsigned grid = std::max(1u, std::min(w.L.chunk_cap, (unsigned)num_sms * 4u));
    if (sort_passes(w.L.tile_bits) <= 1 && w.L.key_cap <= kFusedRangesKeys)
        launch_pdl(emit_sort_kernel<true>, grid, kEmitThreads, 0, s, w, a);
    else launch_pdl(emit_sort_kernel<false>, grid, kEmitThreads, 0, s, w, a);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const Work &w, int tile_buf, int num_sms, cudaStream_t s) {
    launch_pdl(ranges_kernel, num_sms * 8, 256, 0, s, w, w.tkey[tile_buf]);
    return cudaGetLastError();
}
cudaError_t launch_debug_ranges(const Work &w, uint2 *out, cudaStream_t s) {
    if (w.L.tiles == 0) return cudaSuccess;
    launch_pdl(debug_ranges_kernel, (w.L.tiles + 255) / 256, 256, 0, s, w, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_debug(const Work &w, float *mean2d, float *conic, float *opacity, float *depth,
                                int32_t *counts, int depth_buf, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    launch_pdl(gather_debug_kernel, (w.L.P + 255) / 256, 256, 0, s, w, mean2d, conic, opacity, depth, counts, depth_buf);
    return cudaGetLastError();
}

}  // namespace gvk
