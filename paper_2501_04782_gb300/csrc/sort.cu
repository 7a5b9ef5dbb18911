// sort.cu -- stable LSD radix sort of (32-bit key, 32-bit value) pairs, 8 bits per pass.
//
// One pass is a single "onesweep" kernel: each block takes the next tile (256 x 4, 8 or 12
// keys by the key count) from an atomic counter, ranks its keys stably per digit (warp
// match or bit ballots + per-warp histograms), publishes its per-digit counts, stages its
// keys in shared memory in digit order, obtains the exclusive prefix of all earlier tiles
// by decoupled look-back (for a full 8-bit digit only after the staging), and scatters.
// The per-digit global offsets come from one histogram kernel that counts every pass's
// digits up front.  Keys and values are read
// once and written once per pass (the HBM roofline of the sort).
//
// Bounded waits: a look-back spin gives up after DevHeader::spin_limit polls, sets
// ERR_TIMEOUT and publishes anyway; a block that gave up writes nothing (its output is
// undefined but every write stays in bounds).
#include <algorithm>
#include <type_traits>
#include <cstddef>

#include "gv_internal.cuh"

namespace gvk {

namespace {

// Per-pass digit histograms of the live keys among n (passes of 8 bits starting at bit 0);
// also clears look-back buffer 0 for the tiles this sort will use.
// passes == 0: the histograms were counted by the producer of the keys; only clear.
__global__ void __launch_bounds__(256) sort_hist_kernel(const unsigned *keys, const unsigned *n_dev, unsigned n_cap,
                                                        int passes, unsigned *hist, unsigned *look0) {
    pdl_prologue();
    __shared__ unsigned s_h[4][kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0u;
    __syncthreads();
    unsigned n = min(*n_dev, n_cap);
    unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = blockIdx.x * blockDim.x; base < n; base += stride) {
        unsigned i = base + threadIdx.x;
        unsigned k = i < n ? keys[i] : kNoKey;
        bool ok = k != kNoKey;
        unsigned active = __ballot_sync(0xffffffffu, ok);
        if (!ok) continue;
        for (int ps = 0; ps < passes; ps++) count_digit(s_h[ps], (k >> (8 * ps)) & 255u, active);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
        unsigned c = (&s_h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
    unsigned ntiles = sort_tiles(n, n_cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ntiles * kRadix; i += stride) look0[i] = 0u;
}

struct PassArgs {
    const unsigned *keys_in, *vals_in;  // vals_in == nullptr: value = input position
    unsigned *keys_out, *vals_out;
    const unsigned *n_dev;  // keys this pass reads
    unsigned n_cap;
    int shift;
    int dbits;              // live bits of this pass's digit (the last pass of a sort may have fewer than 8)
    const unsigned *hist;   // this pass's 256 digit counts
    unsigned *look_cur;     // [tiles][256] status words of this pass
    unsigned *look_next;    // cleared for the next pass
    unsigned *ctr;          // tile counter of this pass
    DevHeader *hdr;
    uint2 *ranges;          // the last pass of the tile sort: each tile's [start, end) of the
    unsigned n_tiles;       // final list, from the runs of equal keys it writes (else null)
};

// RANGES: the last pass of a tile sort whose final list also gets each tile's range.
// GROUPED: a digit of at most 4 live bits, its look-back walked by a group of threads.
template <int ITEMS, bool BALLOT, bool RANGES, bool GROUPED>
__global__ void __launch_bounds__(kSortThreads, 4) sort_pass_kernel(PassArgs a) {
    pdl_prologue();
    constexpr int TILE = kSortThreads * ITEMS;
    __shared__ unsigned s_keys[TILE];
    __shared__ unsigned s_vals[TILE];
    __shared__ unsigned s_whist[8][kRadix];
    __shared__ unsigned s_gexcl[kRadix];    // exclusive global digit offsets
    __shared__ unsigned s_dstart[kRadix];   // exclusive digit offsets inside the tile
    __shared__ unsigned s_gbase[kRadix];    // global position of this tile's first key of a digit
    __shared__ unsigned s_scan[24];
    __shared__ unsigned s_tile;
    __shared__ int s_abort;

    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const unsigned n = min(*a.n_dev, a.n_cap);
    const unsigned ntiles = (n + TILE - 1) / TILE;
    // every key's digit is taken to the pass's live bits, so ranking, histogram, offsets and
    // scatter agree on it for any key (a key with bits above them cannot index past a digit)
    const unsigned dmask = (1u << a.dbits) - 1u;
    const long long limit = a.hdr->spin_limit;
    const bool drop = a.hdr->drop_signal != 0;
    // A call that already failed (key capacity exceeded, or a wait that gave up) has
    // incomplete input here -- the emission kept only the first key_cap keys while the
    // digit counts cover all of them, and a block that gave up wrote nothing -- and its
    // lists are discarded: the pass does nothing (the block takes no tile; the decision is
    // the block's, as a wait of another block may set the error meanwhile).
    if (__syncthreads_or(*((volatile unsigned *)&a.hdr->err) != 0u)) return;
    {
        unsigned ex;
        block_excl_scan_256(a.hist[t], s_scan, ex);
        s_gexcl[t] = ex;
    }
    for (;;) {
        if (t == 0) { s_tile = atomicAdd(a.ctr, 1u); s_abort = 0; }
        for (int i = t; i < 8 * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
        __syncthreads();
        const unsigned tile = s_tile;
        if (tile >= ntiles) break;
        const unsigned base = tile * TILE;
        unsigned k[ITEMS], v[ITEMS], r[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            unsigned idx = base + wid * (32 * ITEMS) + i * 32 + lane;
            if (idx < n) {
                k[i] = a.keys_in[idx];
                v[i] = a.vals_in ? a.vals_in[idx] : idx;
            } else {
                k[i] = kNoKey;  // past the end: dropped like any absent key
                v[i] = 0u;
            }
        }
        // stable rank of the live keys inside the warp: by item, then by lane.  The lanes
        // holding the same digit come from a warp match or (BALLOT, faster on sorts of many
        // millions of keys) from eight ballots, one per digit bit; absent keys match nothing.
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            const bool live = k[i] != kNoKey;
            unsigned d = (k[i] >> a.shift) & dmask;
            unsigned peers;
            if (BALLOT) {
                peers = __ballot_sync(0xffffffffu, live);
#pragma unroll
                for (int b = 0; b < 8; b++) {
                    if (b >= a.dbits) break;  // the digit has dbits bits
                    const bool bit = (d >> b) & 1u;
                    const unsigned m = __ballot_sync(0xffffffffu, bit);
                    peers &= bit ? m : ~m;
                }
            } else {
                peers = __match_any_sync(0xffffffffu, live ? d : 0x100u + (unsigned)lane);
            }
            unsigned before = live ? s_whist[wid][d] : 0u;
            r[i] = before + __popc(peers & lanemask_lt());
            __syncwarp();
            if (live && lane == __ffs(peers) - 1) s_whist[wid][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread t owns digit t: exclusive offsets over warps, tile total
        unsigned total = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            unsigned c = s_whist[q][t];
            s_whist[q][t] = total;
            total += c;
        }
        // this tile's counts are published at once (digits above the pass's live bits hold no
        // key).  With a full 8-bit digit the tile's keys go to shared memory in digit order
        // before it walks its predecessors, which have that much longer to publish their
        // inclusive prefixes (8 x 1080p depth sort 0.238 -> 0.220 ms); a digit of 5-7 bits walks
        // at once, as its later inclusive prefix would lengthen its successors' walks more
        // (tile pass 0.379 -> 0.389 ms when late).  With at most 4 live bits, a group of
        // G = 256 / 2^bits threads (16, or a warp) walks each digit's chain, G times as many
        // predecessors per poll (960x540 tile pass, 2 bits: 22 -> 20 us; with 6 bits, groups of
        // 4 were slower than one thread per digit).
        const unsigned ndig = 1u << a.dbits;
        if ((unsigned)t < ndig) lookback_publish(a.look_cur, tile, (unsigned)t, total, drop);
        if (GROUPED) s_gbase[t] = total;  // this tile's count of digit t, for its group
        const bool early = !GROUPED && a.dbits < 8;
        bool gave_up = false;
        unsigned excl = 0;
        if (early && (unsigned)t < ndig)
            excl = lookback_walk<kLookWindow>(a.look_cur, tile, (unsigned)t, total, a.hdr, limit, gave_up);
        unsigned dex;
        const unsigned nlive = block_excl_scan_256(total, s_scan, dex);
        s_dstart[t] = dex;
        a.look_next[(size_t)tile * kRadix + t] = 0u;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; i++) {
            if (k[i] == kNoKey) continue;
            unsigned d = (k[i] >> a.shift) & dmask;
            unsigned pos = s_dstart[d] + s_whist[wid][d] + r[i];
            s_keys[pos] = k[i];
            s_vals[pos] = v[i];
        }
        if (!GROUPED) {
            if (!early && (unsigned)t < ndig)
                excl = lookback_walk<kLookWindow>(a.look_cur, tile, (unsigned)t, total, a.hdr, limit, gave_up);
        } else {
            const int G = min(32, kRadix >> a.dbits), m = t % G;
            const unsigned dg = (unsigned)(t / G);
            const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << ((t & 31) - m);
            unsigned ex = 0;
            if (dg < ndig)
                ex = lookback_walk_group(a.look_cur, tile, dg, s_gbase[dg], G, m, gmask, a.hdr, limit, gave_up);
            __syncthreads();  // every group has read its count
            if (m == 0 && dg < ndig) s_gbase[dg] = ex;
            __syncthreads();
            excl = (unsigned)t < ndig ? s_gbase[t] : 0u;
        }
        if (gave_up) s_abort = 1;
        s_gbase[t] = s_gexcl[t] + excl;
        __syncthreads();
        if (!s_abort) {
            for (int pos = t; pos < (int)nlive; pos += kSortThreads) {
                unsigned key = s_keys[pos];
                unsigned d = (key >> a.shift) & dmask;
                unsigned gpos = s_gbase[d] + (unsigned)pos - s_dstart[d];
                if (gpos < n) {
                    a.keys_out[gpos] = key;
                    a.vals_out[gpos] = s_vals[pos];
                    // the output is the final list: equal keys are contiguous here (stable, and
                    // sorted by the lower bits before this pass), so each run's ends bound the
                    // tile's range; other blocks' runs of the same key combine by min / max
                    if (RANGES && key < a.n_tiles) {
                        if (pos == 0 || s_keys[pos - 1] != key) atomicMin(&a.ranges[key].x, gpos);
                        if (pos + 1 == (int)nlive || s_keys[pos + 1] != key) atomicMax(&a.ranges[key].y, gpos + 1u);
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

int sort_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

// Key capacity from which the passes rank by ballots (measured: 15 % faster on 34M keys,
// slower on 1M).
constexpr unsigned kSortBallotN = 1u << 22;

// Sorts keys[0]/vals[0] by their low `bits` bits.  *result_buf receives the buffer index
// (0 or 1) that holds the sorted output.  hist_slot selects 4 histogram rows of the
// workspace (0 or 4), ctr_slot 4 tile counters (both zero on entry: the setup kernel
// clears them).  prepared: the producer of the keys already counted every pass's digits
// into those rows and cleared look-back buffer 0 for sort_tiles(n, n_cap) tiles;
// otherwise a histogram kernel does both first.  first_pass > 0: the first passes were
// done by the producer (the keys sorted by their low 8 * first_pass bits are in buffer
// first_pass & 1, and the look-back buffer of pass first_pass is cleared).
cudaError_t launch_radix_sort(const Work &w, unsigned *keys[2], unsigned *vals[2], const unsigned *n_dev,
                              unsigned n_cap, int bits, bool vals_identity, bool prepared, int hist_slot,
                              int ctr_slot, int num_sms, cudaStream_t s, int *result_buf, int first_pass,
                              const unsigned *n_dev_later, uint2 *final_ranges, unsigned n_tiles) {
    int passes = sort_passes(bits);
    *result_buf = first_pass & 1;
    if (passes <= first_pass || n_cap == 0) return cudaSuccess;
    unsigned *hist = w.hist + (size_t)hist_slot * kRadix;
    const unsigned max_tiles = sort_tiles(n_cap, n_cap);
    unsigned *look[2] = {w.look, w.look + (size_t)w.L.look_tiles * kRadix};
    cudaError_t e;
    if (!prepared && first_pass == 0) {
        int hist_blocks = (int)std::min<unsigned>((n_cap + 255) / 256, (unsigned)num_sms * 4u);
        launch_pdl(sort_hist_kernel, hist_blocks, 256, 0, s, keys[0], n_dev, n_cap, passes, hist, look[0]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int items = sort_items(n_cap);
    const int per_sm = 4;  // resident blocks per SM (launch bounds)
    int grid = (int)std::min<unsigned>(max_tiles, (unsigned)num_sms * per_sm);
    int cur = first_pass & 1;
    for (int ps = first_pass; ps < passes; ps++) {
        PassArgs a;
        a.keys_in = keys[cur];
        a.vals_in = (ps == 0 && vals_identity) ? nullptr : vals[cur];
        a.keys_out = keys[cur ^ 1];
        a.vals_out = vals[cur ^ 1];
        a.n_dev = ps > 0 && n_dev_later ? n_dev_later : n_dev;
        a.n_cap = n_cap;
        a.shift = 8 * ps;
        a.dbits = std::min(8, bits - 8 * ps);
        a.hist = hist + (size_t)ps * kRadix;
        a.look_cur = look[ps & 1];
        a.look_next = look[(ps & 1) ^ 1];
        a.ctr = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(w.hdr) + offsetof(DevHeader, sort_ctr)) +
                ctr_slot + ps;
        a.hdr = w.hdr;
        a.ranges = ps == passes - 1 ? final_ranges : nullptr;
        a.n_tiles = n_tiles;
        // the kernel for this pass: keys per thread, ranking, range recording, grouped look-back
        auto pick = [&](auto R, auto Gp) -> void (*)(PassArgs) {
            constexpr bool RR = decltype(R)::value, GG = decltype(Gp)::value;
            if (items == 8) return sort_pass_kernel<8, false, RR, GG>;
            if (items == 4) return sort_pass_kernel<4, false, RR, GG>;
            if (n_cap < kSortBallotN) return sort_pass_kernel<12, false, RR, GG>;
            return sort_pass_kernel<12, true, RR, GG>;
        };
        const bool grouped = a.dbits <= 4;
        void (*kern)(PassArgs) = a.ranges ? (grouped ? pick(std::true_type{}, std::true_type{})
                                                     : pick(std::true_type{}, std::false_type{}))
                                          : (grouped ? pick(std::false_type{}, std::true_type{})
                                                     : pick(std::false_type{}, std::false_type{}));
        launch_pdl(kern, grid, kSortThreads, 0, s, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *result_buf = cur;
    return cudaSuccess;
}

}  // namespace gvk
