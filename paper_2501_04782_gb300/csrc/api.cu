// api.cu -- the C ABI of libgv (include/gv.h): argument validation, workspace layout,
// stage sequencing on the caller's stream, device status read-back, the autotuner and
// the CUDA-graph form.  Host code only; every stage runs in the kernels of the other
// translation units.  No call here allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gv_internal.cuh"

using namespace gvk;

struct gv_ctx {
    int device = 0;
    int num_sms = 1;
    gv_options opt{};
    std::string err;
    long long spin_limit = 1 << 20;
    int drop_signal = 0;
    // per-stage timing (gv_profile_enable): an event pair per stage, recorded on the
    // call's stream, and the kernels the stage launched
    bool profile = false;
    bool count_replayed = false;  // the backward counts its replayed pairs (profile mode 2)
    bool capturing = false;
    cudaEvent_t ev[GV_NUM_STAGES][2] = {};
    bool ev_used[GV_NUM_STAGES] = {};
    int launches[GV_NUM_STAGES] = {};
    // side stream of the backward: the FP64 chain rule of flagged pairs runs beside the
    // FP32 pass (fork and join by events; also valid inside a stream capture)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

namespace {

// RAII stage marker: records the start event on construction, the end on destruction.
struct StageTimer {
    gv_ctx *c;
    int st;
    cudaStream_t s;
    StageTimer(gv_ctx *c_, int st_, cudaStream_t s_, int kernels) : c(c_), st(st_), s(s_) {
        c->launches[st] = kernels;
        if (c->profile && !c->capturing) {
            cudaEventRecord(c->ev[st][0], s);
            c->ev_used[st] = true;
        }
    }
    ~StageTimer() {
        if (c->profile && !c->capturing) cudaEventRecord(c->ev[st][1], s);
    }
};

}  // namespace

namespace {

constexpr long long kDefaultSpin = 1 << 20;

gv_status fail(gv_ctx *c, gv_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define GV_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, GV_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

bool valid_options(const gv_options &o) {
    bool tile_ok = (o.tile_w == 8 && o.tile_h == 8) || (o.tile_w == 16 && o.tile_h == 8) ||
                   (o.tile_w == 16 && o.tile_h == 16) || (o.tile_w == 32 && o.tile_h == 16) ||
                   (o.tile_w == 32 && o.tile_h == 32);
    bool depth_ok = o.stage_depth == 32 || o.stage_depth == 64 || o.stage_depth == 128 || o.stage_depth == 256;
    return tile_ok && depth_ok && std::isfinite(o.bg[0]) && std::isfinite(o.bg[1]) && std::isfinite(o.bg[2]);
}

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

struct Plan {
    Layout L;
    std::vector<DevFrame> frames;
    int bwd_mode = 0;  // 0 disjoint sets, 1 one shared set, 2 overlapping sets
};

// Frame table, sizes and byte offsets of one call.  key_cap_req > 0 fixes the key
// capacity; otherwise it is the largest that fits in ws_bytes.
// The four non-zero cubic B-spline weights at t of the clamped, uniformly knotted spline
// over n_ctrl control points (Sec. 3.2, Eq. 2), by the Cox-de Boor recursion on the span
// [u_k, u_{k+1}) holding t (t = 1: the last span); lo = k - 3 is the first control point.
void spline_weights(int n_ctrl, double t, int &lo, float w[4]) {
    auto u = [n_ctrl](int i) {
        return i < 4 ? 0.0 : (i >= n_ctrl ? 1.0 : (double)(i - 3) / (double)(n_ctrl - 3));
    };
    t = std::min(1.0, std::max(0.0, t));
    int k = 3;
    while (k < n_ctrl - 1 && !(t < u(k + 1))) k++;
    double N[4] = {1.0, 0.0, 0.0, 0.0};  // N[j] = N_{k-p+j, p} for the current degree p
    for (int p = 1; p <= 3; p++) {
        double nx[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j <= p; j++) {
            const int i = k - p + j;
            double a = 0.0, b = 0.0;
            if (j >= 1 && u(i + p) > u(i)) a = (t - u(i)) / (u(i + p) - u(i)) * N[j - 1];
            if (j < p && u(i + p + 1) > u(i + 1)) b = (u(i + p + 1) - t) / (u(i + p + 1) - u(i + 1)) * N[j];
            nx[j] = a + b;
        }
        for (int j = 0; j < 4; j++) N[j] = nx[j];
    }
    lo = k - 3;
    for (int j = 0; j < 4; j++) w[j] = (float)N[j];
}

gv_status make_plan(gv_ctx *ctx, const gv_options &o, long long N, const gv_frame_desc *fd, int F,
                    long long key_cap_req, size_t ws_bytes, Plan &pl, int n_ctrl = 0) {
    if (F < 1 || F > GV_MAX_FRAMES) return fail(ctx, GV_ERR_INVALID_ARG, "frame count %d out of [1, %d]", F, GV_MAX_FRAMES);
    if (!fd) return fail(ctx, GV_ERR_INVALID_ARG, "frames is NULL");
    pl.frames.resize(F);
    unsigned long long P = 0, tiles = 0, tiles88 = 0;
    for (int f = 0; f < F; f++) {
        const gv_frame_desc &d = fd[f];
        const gv_camera &c = d.cam;
        if (c.W <= 0 || c.H <= 0 || c.W > 32768 || c.H > 32768)
            return fail(ctx, GV_ERR_INVALID_ARG, "frame %d: bad size %dx%d", f, c.W, c.H);
        if (d.gauss_offset < 0 || d.gauss_count < 0 || d.gauss_offset + d.gauss_count > N)
            return fail(ctx, GV_ERR_INVALID_ARG, "frame %d: Gaussian range [%lld, +%lld) outside [0, %lld)", f,
                        (long long)d.gauss_offset, (long long)d.gauss_count, N);
        if (d.pixel_offset < 0) return fail(ctx, GV_ERR_INVALID_ARG, "frame %d: negative pixel offset", f);
        DevFrame &x = pl.frames[f];
        memset(&x, 0, sizeof(x));
        x.W = c.W; x.H = c.H;
        x.fx = c.fx; x.fy = c.fy; x.cx = c.cx; x.cy = c.cy;
        for (int i = 0; i < 9; i++) x.R[i] = c.R[i];
        for (int i = 0; i < 3; i++) x.t[i] = c.t[i];
        for (int j = 0; j < 3; j++)
            x.campos[j] = (float)-((double)c.R[j] * c.t[0] + (double)c.R[3 + j] * c.t[1] + (double)c.R[6 + j] * c.t[2]);
        x.time = c.time;
        if (n_ctrl > 0) {
            x.time = std::min(1.f, std::max(0.f, c.time));
            spline_weights(n_ctrl, c.time, x.spline_lo, x.spline_w);
        }
        x.gauss_offset = d.gauss_offset;
        x.gauss_count = (unsigned)d.gauss_count;
        x.pixel_offset = d.pixel_offset;
        x.pair_offset = (unsigned)P;
        x.tiles_x = (unsigned)((c.W + o.tile_w - 1) / o.tile_w);
        x.tiles_y = (unsigned)((c.H + o.tile_h - 1) / o.tile_h);
        x.tile_offset = (unsigned)tiles;
        P += (unsigned long long)d.gauss_count;
        tiles += (unsigned long long)x.tiles_x * x.tiles_y;
        tiles88 += (unsigned long long)((c.W + 7) / 8) * ((c.H + 7) / 8);
    }
    if (P >= (1ull << 30)) return fail(ctx, GV_ERR_INVALID_ARG, "too many (frame, Gaussian) pairs: %llu", P);
    if (tiles88 >= (1ull << 30)) return fail(ctx, GV_ERR_INVALID_ARG, "too many tiles: %llu", tiles88);
    // backward mode: identical sets, disjoint sets, or overlapping
    bool same = true;
    for (int f = 1; f < F; f++)
        same = same && fd[f].gauss_offset == fd[0].gauss_offset && fd[f].gauss_count == fd[0].gauss_count;
    if (F > 1 && same) {
        pl.bwd_mode = 1;
    } else {
        std::vector<std::pair<long long, long long>> iv;
        for (int f = 0; f < F; f++)
            if (fd[f].gauss_count > 0) iv.push_back({(long long)fd[f].gauss_offset, (long long)fd[f].gauss_count});
        std::sort(iv.begin(), iv.end());
        bool disjoint = true;
        for (size_t i = 1; i < iv.size(); i++) disjoint = disjoint && iv[i].first >= iv[i - 1].first + iv[i - 1].second;
        pl.bwd_mode = disjoint ? 0 : 2;
    }
    Layout &L = pl.L;
    memset(&L, 0, sizeof(L));
    L.P = (unsigned)P;
    L.tiles = (unsigned)tiles;
    L.tiles_alloc = (unsigned)std::max(tiles88, tiles);
    L.F = (unsigned)F;
    L.emit_blocks = (unsigned)((P + kEmitBlock - 1) / kEmitBlock);
    int bits = 1;
    while ((1ull << bits) < tiles) bits++;
    L.tile_bits = bits;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off = align_up(off + bytes); return r; };
    L.hdr = take(sizeof(DevHeader));
    L.frames = take(sizeof(DevFrame) * F);
    size_t Pn = std::max<size_t>(P, 1);
    L.feat0 = take(16 * Pn);
    L.feat1 = take(16 * Pn);
    L.feat2 = take(4 * Pn);
    L.rect = take(16 * Pn);
    L.ell = take(16 * Pn);
    L.dkey[0] = take(4 * Pn);
    L.dkey[1] = take(4 * Pn);
    L.dval[0] = take(4 * Pn);
    L.dval[1] = take(4 * Pn);
    L.scan_look = take(8 * std::max<size_t>(L.emit_blocks, 1));
    L.offsets = take(4 * (Pn + 1));
    L.g0 = take(16 * Pn);
    L.g1 = take(16 * Pn);
    L.g2 = take(4 * Pn);
    L.fp64_list = take(4 * Pn);
    L.ranges = take(8 * (size_t)L.tiles_alloc);
    L.hist = take(4 * 8 * kRadix);
    const size_t fixed = off;
    // look-back tiles: those of the sorts, and the emission chunks (which share buffer 0)
    auto look_tiles_for = [&](unsigned cap) {
        return std::max(std::max(std::max(sort_tiles(cap, cap), sort_tiles((unsigned)P, (unsigned)P)),
                                 emit_chunk_cap(cap)), 1u);
    };
    auto total_for = [&](unsigned long long cap) {
        const unsigned c = (unsigned)std::min<unsigned long long>(std::max<unsigned long long>(cap, 1), 1ull << 30);
        size_t t = fixed;
        t += 4 * align_up(4 * (size_t)c);
        t += align_up(4 * (size_t)emit_chunk_cap(c));
        t += align_up(2 * 4 * (size_t)look_tiles_for(c) * kRadix);
        return t;
    };
    unsigned long long cap;
    if (key_cap_req > 0) {
        cap = (unsigned long long)key_cap_req;
    } else {
        if (ws_bytes < total_for(1)) return fail(ctx, GV_ERR_INVALID_ARG, "workspace of %zu bytes is too small (need > %zu)",
                                                 ws_bytes, total_for(1));
        unsigned long long lo = 1, hi = (1ull << 30) - 1;
        while (lo < hi) {
            unsigned long long mid = (lo + hi + 1) / 2;
            if (total_for(mid) <= ws_bytes) lo = mid; else hi = mid - 1;
        }
        cap = lo;
    }
    if (cap >= (1ull << 30)) return fail(ctx, GV_ERR_INVALID_ARG, "key capacity %llu >= 2^30", cap);
    L.key_cap = (unsigned)cap;
    size_t kc = std::max<size_t>(cap, 1);
    L.chunk_cap = emit_chunk_cap((unsigned)kc);
    L.look_tiles = look_tiles_for((unsigned)kc);
    L.tkey[0] = take(4 * kc);
    L.tkey[1] = take(4 * kc);
    L.tval[0] = take(4 * kc);
    L.tval[1] = take(4 * kc);
    L.chunk_first = take(4 * (size_t)L.chunk_cap);
    L.look = take((size_t)2 * 4 * L.look_tiles * kRadix);
    L.total = off;
    if (key_cap_req <= 0 && L.total > ws_bytes)
        return fail(ctx, GV_ERR_INVALID_ARG, "workspace layout (%zu) exceeds %zu bytes", L.total, ws_bytes);
    return GV_OK;
}

Work make_work(void *ws, const Layout &L) {
    char *b = (char *)ws;
    Work w;
    w.hdr = (DevHeader *)(b + L.hdr);
    w.frames = (DevFrame *)(b + L.frames);
    w.feat0 = (float4 *)(b + L.feat0);
    w.feat1 = (float4 *)(b + L.feat1);
    w.feat2 = (float *)(b + L.feat2);
    w.rect = (uint4 *)(b + L.rect);
    w.ell = (float4 *)(b + L.ell);
    for (int i = 0; i < 2; i++) {
        w.dkey[i] = (unsigned *)(b + L.dkey[i]);
        w.dval[i] = (unsigned *)(b + L.dval[i]);
        w.tkey[i] = (unsigned *)(b + L.tkey[i]);
        w.tval[i] = (unsigned *)(b + L.tval[i]);
    }
    w.scan_look = (unsigned long long *)(b + L.scan_look);
    w.offsets = (unsigned *)(b + L.offsets);
    w.chunk_first = (unsigned *)(b + L.chunk_first);
    w.g0 = (float4 *)(b + L.g0);
    w.g1 = (float4 *)(b + L.g1);
    w.g2 = (float *)(b + L.g2);
    w.fp64_list = (unsigned *)(b + L.fp64_list);
    w.ranges = (uint2 *)(b + L.ranges);
    w.hist = (unsigned *)(b + L.hist);
    w.look = (unsigned *)(b + L.look);
    w.L = L;
    return w;
}

GaussPtrs gauss_ptrs(const gv_gaussians *g) {
    GaussPtrs p;
    p.mean = g->mean; p.vel = g->vel; p.log_scale = g->log_scale;
    p.quat = g->quat; p.logit = g->opacity_logit; p.rgb = g->rgb;
    p.N = g->N;
    p.n_ctrl = g->n_ctrl;
    p.ctrl = g->ctrl; p.log_scale_t = g->log_scale_t; p.quat_t = g->quat_t;
    p.sh_degree = g->sh_degree;
    p.sh = g->sh_degree > 0 ? g->sh : nullptr;
    p.visible = g->visible;
    if (p.n_ctrl > 0) p.vel = nullptr;
    return p;
}

gv_status check_gaussians(gv_ctx *ctx, const gv_gaussians *g) {
    if (!g) return fail(ctx, GV_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->N < 0) return fail(ctx, GV_ERR_INVALID_ARG, "negative Gaussian count");
    if (g->n_ctrl != 0 && (g->n_ctrl < 4 || g->n_ctrl > 64))
        return fail(ctx, GV_ERR_INVALID_ARG, "n_ctrl %d outside [4, 64]", g->n_ctrl);
    if (g->N > 0 && ((g->n_ctrl ? !g->ctrl : !g->mean) || !g->log_scale || !g->quat || !g->opacity_logit || !g->rgb))
        return fail(ctx, GV_ERR_INVALID_ARG, "a required Gaussian parameter plane is NULL");
    if (g->sh_degree < 0 || g->sh_degree > 3)
        return fail(ctx, GV_ERR_INVALID_ARG, "sh_degree %d outside [0, 3]", g->sh_degree);
    if (g->N > 0 && g->sh_degree > 0 && !g->sh)
        return fail(ctx, GV_ERR_INVALID_ARG, "sh_degree %d with NULL sh", g->sh_degree);
    return GV_OK;
}

// Upload the frame table and clear the per-call state (setup kernels, captured by value).
gv_status run_setup(gv_ctx *ctx, const Work &w, const Plan &pl, cudaStream_t s) {
    int F = (int)pl.frames.size();
    for (int first = 0; first < F; first += kMaxFramesPerSetup) {
        FrameChunk ch;
        memset(&ch, 0, sizeof(ch));
        int cnt = std::min(kMaxFramesPerSetup, F - first);
        for (int i = 0; i < cnt; i++) ch.f[i] = pl.frames[first + i];
        GV_CUDA(launch_setup(w, ch, first, cnt, first == 0, ctx->spin_limit, ctx->drop_signal, s));
    }
    return GV_OK;
}

int depth_result_buf() { return sort_passes(32) & 1; }
int tile_result_buf(const Layout &L) { return sort_passes(L.tile_bits) & 1; }

// The tile-sort passes after the first (which the emission does): buffer 1 onwards.
cudaError_t tile_sort_rest(gv_ctx *ctx, const Work &w, cudaStream_t s, int *tres) {
    const unsigned *n_keys =
        reinterpret_cast<const unsigned *>(reinterpret_cast<const char *>(w.hdr) + offsetof(DevHeader, keys_used));
    unsigned *tk[2] = {w.tkey[0], w.tkey[1]}, *tv[2] = {w.tval[0], w.tval[1]};
    return launch_radix_sort(w, tk, tv, n_keys, w.L.key_cap, w.L.tile_bits, false, true, 4, 4, ctx->num_sms, s, tres,
                             1, nullptr, w.L.key_cap <= kFusedRangesKeys ? w.ranges : nullptr, w.L.tiles);
}

// loss: the L2 loss fused into the compositing forward (target == nullptr: none)
gv_status forward_stages(gv_ctx *ctx, const gv_gaussians *g, const Plan &pl, const Work &w, float *image,
                         float *final_T, int32_t *last_idx, cudaStream_t s, const LossArgs &loss = LossArgs()) {
    const gv_options &o = ctx->opt;
    for (int i = 0; i < GV_NUM_STAGES; i++) ctx->launches[i] = 0;
    {
        StageTimer tm(ctx, GV_STAGE_SETUP, s, (int)((pl.frames.size() + kMaxFramesPerSetup - 1) / kMaxFramesPerSetup));
        gv_status st = run_setup(ctx, w, pl, s);
        if (st != GV_OK) return st;
    }
    if (w.L.P > 0) {
        {
            StageTimer tm(ctx, GV_STAGE_PROJECT, s, 1);
            GV_CUDA(launch_project_fwd(w, gauss_ptrs(g), o.tile_w, o.tile_h, pl.bwd_mode == 1, ctx->num_sms, s));
        }
        int dres = 0;
        {
            StageTimer tm(ctx, GV_STAGE_DEPTH_SORT, s, sort_passes(32));
            const unsigned *n_pairs = reinterpret_cast<const unsigned *>(reinterpret_cast<const char *>(w.hdr) +
                                                                           offsetof(DevHeader, n_pairs));
            const unsigned *n_drawn = reinterpret_cast<const unsigned *>(reinterpret_cast<const char *>(w.hdr) +
                                                                           offsetof(DevHeader, n_drawn));
            unsigned *dk[2] = {w.dkey[0], w.dkey[1]}, *dv[2] = {w.dval[0], w.dval[1]};
            // the first pass drops the culled pairs (no depth key); the others sort the rest
            GV_CUDA(launch_radix_sort(w, dk, dv, n_pairs, w.L.P, 32, true, true, 0, 0, ctx->num_sms, s, &dres, 0,
                                      n_drawn));
        }
        {
            StageTimer tm(ctx, GV_STAGE_EMIT, s, 2);
            GV_CUDA(launch_emit(w, dres, o.tile_w, o.tile_h, ctx->num_sms, s));
        }
        int tres = 0;
        {
            StageTimer tm(ctx, GV_STAGE_TILE_SORT, s, sort_passes(w.L.tile_bits) - 1);
            GV_CUDA(tile_sort_rest(ctx, w, s, &tres));
        }
        if (w.L.key_cap > kFusedRangesKeys) {  // else recorded by the kernel that wrote the list
            StageTimer tm(ctx, GV_STAGE_RANGES, s, 1);
            GV_CUDA(launch_ranges(w, tres, ctx->num_sms, s));
        }
    }
    {
        StageTimer tm(ctx, GV_STAGE_COMPOSITE_FWD, s, 1);
        GV_CUDA(launch_composite_fwd(w, o.tile_w, o.tile_h, o.stage_depth, tile_result_buf(w.L), o.bg[0], o.bg[1],
                                     o.bg[2], image, final_T, last_idx, loss, ctx->num_sms, s));
    }
    return GV_OK;
}

gv_status backward_stages(gv_ctx *ctx, const gv_gaussians *g, const Plan &pl, const Work &w, const float *final_T,
                          const int32_t *last_idx, const float *dL, const gv_gaussians_grad *grad, cudaStream_t s) {
    const gv_options &o = ctx->opt;
    ctx->launches[GV_STAGE_COMPOSITE_BWD] = ctx->launches[GV_STAGE_PROJECT_BWD] = 0;
    if (w.L.P == 0) return GV_OK;
    // the three screen-space gradient planes are adjacent in the workspace: one memset; the
    // backward work queue is reset by the last block of the previous backward (or by setup)
    GV_CUDA(cudaMemsetAsync(w.g0, 0, (size_t)(reinterpret_cast<char *>(w.g2 + w.L.P) - reinterpret_cast<char *>(w.g0)),
                            s));
    {
        StageTimer tm(ctx, GV_STAGE_COMPOSITE_BWD, s, 1);
        // the replayed pairs are counted only in profile mode 2
        GV_CUDA(launch_composite_bwd(w, o.tile_w, o.tile_h, o.stage_depth, tile_result_buf(w.L), o.bg[0], o.bg[1],
                                     o.bg[2], final_T, last_idx, dL, ctx->count_replayed, ctx->num_sms, s));
    }
    GradPtrs gp;
    gp.mean = grad->mean; gp.vel = grad->vel; gp.log_scale = grad->log_scale;
    gp.quat = grad->quat; gp.logit = grad->opacity_logit; gp.rgb = grad->rgb;
    gp.cam = grad->camera;
    gp.ctrl = grad->ctrl; gp.log_scale_t = grad->log_scale_t; gp.quat_t = grad->quat_t;
    gp.sh = g->sh_degree > 0 ? grad->sh : nullptr;
    {
        StageTimer tm(ctx, GV_STAGE_PROJECT_BWD, s, 2);
        const GaussPtrs gptr = gauss_ptrs(g);
        int dev = -1;
        GV_CUDA(cudaGetDevice(&dev));
        if (dev == ctx->device) {  // the side stream belongs to the context's device
            GV_CUDA(cudaEventRecord(ctx->fork, s));
            GV_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
            GV_CUDA(launch_project_bwd_fp64(w, gptr, gp, ctx->num_sms, ctx->side));
            GV_CUDA(cudaEventRecord(ctx->join, ctx->side));
            GV_CUDA(launch_project_bwd(w, gptr, gp, pl.bwd_mode, ctx->num_sms, s));
            GV_CUDA(cudaStreamWaitEvent(s, ctx->join, 0));
        } else {
            GV_CUDA(launch_project_bwd(w, gptr, gp, pl.bwd_mode, ctx->num_sms, s));
            GV_CUDA(launch_project_bwd_fp64(w, gptr, gp, ctx->num_sms, s));
        }
    }
    return GV_OK;
}

// The time-parameterised form needs the control-point plane instead of the mean plane.
gv_status check_grad(gv_ctx *ctx, const gv_gaussians_grad *grad, const gv_gaussians *g) {
    const bool spline = g && g->n_ctrl > 0;
    if (!grad || (spline ? !grad->ctrl : !grad->mean) || !grad->log_scale || !grad->quat || !grad->opacity_logit ||
        !grad->rgb)
        return fail(ctx, GV_ERR_INVALID_ARG, "a required gradient plane is NULL");
    return GV_OK;
}

gv_frame_desc single_frame(const gv_camera *cam, long long N) {
    gv_frame_desc d;
    memset(&d, 0, sizeof(d));
    d.cam = *cam;
    d.gauss_offset = 0;
    d.gauss_count = N;
    d.pixel_offset = 0;
    return d;
}

}  // namespace

// Scratch of gv_render_fwd_noalloc: one device array per GPU that loads the library, held
// until exit.  Host code needs the array's device address: the name is only a host-side
// stand-in for it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GV_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch in the current context (the current device's), looked
// up on every call: an address kept from an earlier call would belong to whatever context
// was current then (a cudaDeviceReset, or another context made current on the device,
// makes it stale).  The lookup does not allocate; the first one on a device also loads the
// library's module there.
cudaError_t noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

struct gv_graph {
    gv_ctx *ctx = nullptr;
    gv_options opt{};  // the context's options at capture (tile shape of the captured kernels)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> setup_nodes;  // in launch order, one per frame chunk
    Plan plan;
    int n_ctrl = 0;  // time-parameterised means: the frames' spline weights follow their times
    Work work;
    std::vector<gv_frame_desc> frames;
};

extern "C" {

const char *gv_status_string(gv_status s) {
    switch (s) {
        case GV_OK: return "ok";
        case GV_ERR_INVALID_ARG: return "invalid argument";
        case GV_ERR_CAPACITY: return "key capacity exceeded";
        case GV_ERR_TIMEOUT: return "device wait timed out";
        case GV_ERR_CUDA: return "CUDA error";
        case GV_ERR_UNIMPLEMENTED: return "unimplemented";
    }
    return "unknown status";
}

gv_status gv_create(gv_ctx **out, const gv_options *opt) {
    if (!out) return GV_ERR_INVALID_ARG;
    *out = nullptr;
    gv_ctx *c = new (std::nothrow) gv_ctx();
    if (!c) return GV_ERR_INVALID_ARG;
    c->opt.tile_w = 16; c->opt.tile_h = 16; c->opt.stage_depth = 256;
    c->opt.bg[0] = c->opt.bg[1] = c->opt.bg[2] = 0.f;
    if (opt) {
        if (!valid_options(*opt)) { delete c; return GV_ERR_INVALID_ARG; }
        c->opt = *opt;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GV_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        gv_destroy(c);
        return GV_ERR_CUDA;
    }
    *out = c;
    return GV_OK;
}

gv_status gv_destroy(gv_ctx *ctx) {
    if (!ctx) return GV_OK;
    for (int i = 0; i < GV_NUM_STAGES; i++)
        for (int j = 0; j < 2; j++)
            if (ctx->ev[i][j]) cudaEventDestroy(ctx->ev[i][j]);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    delete ctx;
    return GV_OK;
}

gv_status gv_profile_enable(gv_ctx *ctx, int32_t on) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    if (on && !ctx->ev[0][0]) {
        for (int i = 0; i < GV_NUM_STAGES; i++)
            for (int j = 0; j < 2; j++) GV_CUDA(cudaEventCreate(&ctx->ev[i][j]));
    }
    ctx->profile = on != 0;
    ctx->count_replayed = on == 2;
    for (int i = 0; i < GV_NUM_STAGES; i++) ctx->ev_used[i] = false;
    return GV_OK;
}

gv_status gv_profile_read(gv_ctx *ctx, float *ms, int32_t *launches) {
    if (!ctx || !ms) return GV_ERR_INVALID_ARG;
    for (int i = 0; i < GV_NUM_STAGES; i++) {
        ms[i] = -1.f;
        if (launches) launches[i] = ctx->launches[i];
        if (!ctx->profile || !ctx->ev_used[i]) continue;
        GV_CUDA(cudaEventSynchronize(ctx->ev[i][1]));
        float t = 0.f;
        GV_CUDA(cudaEventElapsedTime(&t, ctx->ev[i][0], ctx->ev[i][1]));
        ms[i] = t;
    }
    return GV_OK;
}

gv_status gv_get_options(const gv_ctx *ctx, gv_options *opt) {
    if (!ctx || !opt) return GV_ERR_INVALID_ARG;
    *opt = ctx->opt;
    return GV_OK;
}

gv_status gv_set_options(gv_ctx *ctx, const gv_options *opt) {
    if (!ctx || !opt) return GV_ERR_INVALID_ARG;
    if (!valid_options(*opt))
        return fail(ctx, GV_ERR_INVALID_ARG, "invalid options: tile %dx%d, stage depth %d", opt->tile_w, opt->tile_h,
                    opt->stage_depth);
    ctx->opt = *opt;
    return GV_OK;
}

const char *gv_last_error(const gv_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

gv_status gv_workspace_size(const gv_ctx *cctx, const gv_frame_desc *frames, int32_t F, int64_t key_capacity,
                            size_t *bytes) {
    gv_ctx *ctx = const_cast<gv_ctx *>(cctx);
    if (!ctx || !bytes) return GV_ERR_INVALID_ARG;
    long long N = 0;
    for (int f = 0; frames && f < F; f++) N = std::max<long long>(N, frames[f].gauss_offset + frames[f].gauss_count);
    long long P = 0;
    for (int f = 0; frames && f < F; f++) P += frames[f].gauss_count;
    long long cap = key_capacity > 0 ? key_capacity : 16 * P + 65536;
    Plan pl;
    gv_status st = make_plan(ctx, ctx->opt, N, frames, F, cap, 0, pl);
    if (st != GV_OK) return st;
    *bytes = pl.L.total;
    return GV_OK;
}

gv_status gv_render_batch_fwd(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames, int32_t F,
                              void *workspace, size_t ws_bytes, float *image, float *final_T, int32_t *last_idx,
                              gv_stream stream) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    gv_status st = check_gaussians(ctx, g);
    if (st != GV_OK) return st;
    if (!workspace || !image || !final_T || !last_idx) return fail(ctx, GV_ERR_INVALID_ARG, "NULL buffer");
    Plan pl;
    st = make_plan(ctx, ctx->opt, g->N, frames, F, 0, ws_bytes, pl, g->n_ctrl);
    if (st != GV_OK) return st;
    Work w = make_work(workspace, pl.L);
    return forward_stages(ctx, g, pl, w, image, final_T, last_idx, (cudaStream_t)stream);
}

gv_status gv_render_batch_fwd_l2(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames, int32_t F,
                                 void *workspace, size_t ws_bytes, float *image, float *final_T, int32_t *last_idx,
                                 const float *target, float scale, float *dL_dimage, float *loss, gv_stream stream) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    gv_status st = check_gaussians(ctx, g);
    if (st != GV_OK) return st;
    if (!workspace || !image || !final_T || !last_idx || !target) return fail(ctx, GV_ERR_INVALID_ARG, "NULL buffer");
    Plan pl;
    st = make_plan(ctx, ctx->opt, g->N, frames, F, 0, ws_bytes, pl, g->n_ctrl);
    if (st != GV_OK) return st;
    Work w = make_work(workspace, pl.L);
    LossArgs la;
    la.target = target;
    la.dL = dL_dimage;
    la.loss = loss;
    la.scale = scale;
    return forward_stages(ctx, g, pl, w, image, final_T, last_idx, (cudaStream_t)stream, la);
}

gv_status gv_render_batch_bwd(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames, int32_t F,
                              void *workspace, size_t ws_bytes, const float *final_T, const int32_t *last_idx,
                              const float *dL_dimage, gv_gaussians_grad *grad, gv_stream stream) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    gv_status st = check_gaussians(ctx, g);
    if (st != GV_OK) return st;
    st = check_grad(ctx, grad, g);
    if (st != GV_OK) return st;
    if (!workspace || !final_T || !last_idx || !dL_dimage) return fail(ctx, GV_ERR_INVALID_ARG, "NULL buffer");
    Plan pl;
    st = make_plan(ctx, ctx->opt, g->N, frames, F, 0, ws_bytes, pl, g->n_ctrl);
    if (st != GV_OK) return st;
    Work w = make_work(workspace, pl.L);
    return backward_stages(ctx, g, pl, w, final_T, last_idx, dL_dimage, grad, (cudaStream_t)stream);
}

gv_status gv_render_fwd(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, void *workspace, size_t ws_bytes,
                        float *image, float *final_T, int32_t *last_idx, gv_stream stream) {
    if (!ctx || !g || !cam) return ctx ? fail(ctx, GV_ERR_INVALID_ARG, "NULL argument") : GV_ERR_INVALID_ARG;
    gv_frame_desc d = single_frame(cam, g->N);
    return gv_render_batch_fwd(ctx, g, &d, 1, workspace, ws_bytes, image, final_T, last_idx, stream);
}

gv_status gv_render_fwd_l2(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, void *workspace,
                           size_t ws_bytes, float *image, float *final_T, int32_t *last_idx, const float *target,
                           float scale, float *dL_dimage, float *loss, gv_stream stream) {
    if (!ctx || !g || !cam) return ctx ? fail(ctx, GV_ERR_INVALID_ARG, "NULL argument") : GV_ERR_INVALID_ARG;
    gv_frame_desc d = single_frame(cam, g->N);
    return gv_render_batch_fwd_l2(ctx, g, &d, 1, workspace, ws_bytes, image, final_T, last_idx, target, scale,
                                  dL_dimage, loss, stream);
}

gv_status gv_render_bwd(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, void *workspace, size_t ws_bytes,
                        const float *final_T, const int32_t *last_idx, const float *dL_dimage,
                        gv_gaussians_grad *grad, gv_stream stream) {
    if (!ctx || !g || !cam) return ctx ? fail(ctx, GV_ERR_INVALID_ARG, "NULL argument") : GV_ERR_INVALID_ARG;
    gv_frame_desc d = single_frame(cam, g->N);
    return gv_render_batch_bwd(ctx, g, &d, 1, workspace, ws_bytes, final_T, last_idx, dL_dimage, grad, stream);
}

// The forward for callers that cannot allocate device memory: a plug-in whose host
// application owns every device allocation (it may not call cudaMalloc itself), or a
// real-time loop that must not let cudaMalloc / cudaFree synchronise the device in the
// middle of a frame.  Its workspace is g_noalloc_scratch; the kernels are gv_render_fwd's.
gv_status gv_render_fwd_noalloc(gv_ctx *ctx, const gv_gaussians *g, const gv_camera *cam, float *image,
                                float *final_T, int32_t *last_idx, gv_stream stream) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    if (!cam) return fail(ctx, GV_ERR_INVALID_ARG, "NULL camera");
    gv_status st = check_gaussians(ctx, g);
    if (st != GV_OK) return st;
    if (!image || !final_T || !last_idx) return fail(ctx, GV_ERR_INVALID_ARG, "NULL buffer");
    void *scratch = nullptr;
    GV_CUDA(noalloc_scratch(&scratch));
    gv_frame_desc d = single_frame(cam, g->N);
    Plan pl;
    // the frame itself first (sizes, ranges: errors passed through), then its fit
    st = make_plan(ctx, ctx->opt, g->N, &d, 1, 1, 0, pl, g->n_ctrl);
    if (st != GV_OK) return st;
    if (pl.L.total > GV_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, GV_ERR_INVALID_ARG,
                    "%lld Gaussians on a %dx%d frame need %zu bytes before any key, more than the %u-byte static "
                    "scratch", (long long)g->N, cam->W, cam->H, pl.L.total, (unsigned)GV_NOALLOC_SCRATCH_BYTES);
    st = make_plan(ctx, ctx->opt, g->N, &d, 1, 0, GV_NOALLOC_SCRATCH_BYTES, pl, g->n_ctrl);
    if (st != GV_OK) return st;
    Work w = make_work(scratch, pl.L);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the forward's own setup kernel clears
    // the header, counters, histograms and tile ranges, and each sort clears its look-back
    // words, exactly as for a reused caller workspace
    st = forward_stages(ctx, g, pl, w, image, final_T, last_idx, s);
    if (st != GV_OK) return st;
    DevHeader h;
    GV_CUDA(cudaMemcpyAsync(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaStreamSynchronize(s));
    if (h.err & ERR_TIMEOUT) return fail(ctx, GV_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    if (h.err & ERR_CAPACITY)
        return fail(ctx, GV_ERR_CAPACITY, "the frame needs %llu keys; the %u-byte static scratch holds %u",
                    (unsigned long long)h.keys_total, (unsigned)GV_NOALLOC_SCRATCH_BYTES, pl.L.key_cap);
    return GV_OK;
}

gv_status gv_read_status(gv_ctx *ctx, const void *workspace, size_t ws_bytes, gv_stream stream,
                         int64_t *keys_needed) {
    (void)ws_bytes;
    if (!ctx || !workspace) return GV_ERR_INVALID_ARG;
    DevHeader h;
    GV_CUDA(cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    GV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (keys_needed) *keys_needed = (int64_t)h.keys_total;
    if (h.err & ERR_TIMEOUT) return fail(ctx, GV_ERR_TIMEOUT, "a device-side wait exceeded its limit");
    if (h.err & ERR_CAPACITY)
        return fail(ctx, GV_ERR_CAPACITY, "the call needed %llu keys, more than the workspace holds",
                    (unsigned long long)h.keys_total);
    return GV_OK;
}

gv_status gv_status_accumulate(gv_ctx *ctx, const void *workspace, int32_t *acc, gv_stream stream) {
    if (!ctx || !workspace || !acc) return GV_ERR_INVALID_ARG;
    GV_CUDA(launch_status_or(workspace, acc, (cudaStream_t)stream));
    return GV_OK;
}

gv_status gv_read_counters(gv_ctx *ctx, const void *workspace, gv_stream stream, int64_t *out) {
    if (!ctx || !workspace || !out) return GV_ERR_INVALID_ARG;
    DevHeader h;
    GV_CUDA(cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    GV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    out[0] = (int64_t)h.keys_used;
    out[1] = (int64_t)h.n_pairs;
    for (int i = 0; i < 4; i++) out[2 + i] = (int64_t)h.work[i];
    out[3] = (int64_t)h.n_drawn;  // the forward does not count composited pairs (work[1] is 0)
    return GV_OK;
}

gv_status gv_l2_loss_grad(gv_ctx *ctx, const float *image, const float *target, int64_t n, float scale,
                          float *dL_dimage, float *loss, gv_stream stream) {
    if (!ctx || !image || !target || n < 0) return GV_ERR_INVALID_ARG;
    GV_CUDA(launch_l2_loss(image, target, n, scale, dL_dimage, loss, (cudaStream_t)stream));
    return GV_OK;
}

gv_status gv_adam_step(gv_ctx *ctx, float *param, float *grad, float *m, float *v, int64_t n, int64_t step, float lr,
                       float beta1, float beta2, float eps, int32_t zero_grad, gv_stream stream) {
    if (!ctx || !param || !grad || !m || !v || n < 0 || step < 1) return GV_ERR_INVALID_ARG;
    float bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
    float bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
    GV_CUDA(launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, bc1, bc2, zero_grad, (cudaStream_t)stream));
    return GV_OK;
}

gv_status gv_adan_step(gv_ctx *ctx, float *param, float *grad, float *m, float *v, float *nsq, float *g_prev,
                       int64_t n, int64_t step, float lr, float beta1, float beta2, float beta3, float eps,
                       float weight_decay, int32_t bias_correction, int32_t zero_grad, gv_stream stream) {
    if (!ctx || !param || !grad || !m || !v || !nsq || !g_prev || n < 0 || step < 1) return GV_ERR_INVALID_ARG;
    if (bias_correction && !(beta1 > 0.f && beta2 > 0.f && beta3 > 0.f)) return GV_ERR_INVALID_ARG;
    GV_CUDA(launch_adan(param, grad, m, v, nsq, g_prev, n, lr, beta1, beta2, beta3, eps, weight_decay, step,
                        bias_correction != 0, zero_grad, (cudaStream_t)stream));
    return GV_OK;
}

gv_status gv_autotune(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames, int32_t F, void *workspace,
                      size_t ws_bytes, float *image, float *final_T, int32_t *last_idx, const float *dL_dimage,
                      gv_gaussians_grad *grad, int32_t reps, gv_options *best, float *ms_out, gv_stream stream) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    if (reps < 1) reps = 1;
    constexpr int kShapes = 5;
    const int shapes[kShapes][2] = {{8, 8}, {16, 8}, {16, 16}, {32, 16}, {32, 32}};
    const int depths[3] = {64, 128, 256};
    gv_options keep = ctx->opt, found = ctx->opt;
    float best_ms = INFINITY;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    GV_CUDA(cudaEventCreate(&e0));
    GV_CUDA(cudaEventCreate(&e1));
    gv_status result = GV_OK;
    int k = 0;
    for (int si = 0; si < kShapes && result == GV_OK; si++) {
        for (int di = 0; di < 3 && result == GV_OK; di++, k++) {
            gv_options o = keep;
            o.tile_w = shapes[si][0];
            o.tile_h = shapes[si][1];
            o.stage_depth = depths[di];
            ctx->opt = o;
            float ms = INFINITY;
            gv_status st = gv_render_batch_fwd(ctx, g, frames, F, workspace, ws_bytes, image, final_T, last_idx, stream);
            if (st == GV_OK)
                st = gv_render_batch_bwd(ctx, g, frames, F, workspace, ws_bytes, final_T, last_idx, dL_dimage, grad,
                                         stream);
            if (st == GV_OK) st = gv_read_status(ctx, workspace, ws_bytes, stream, nullptr);
            if (st == GV_OK) {
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && st == GV_OK; r++) {
                    st = gv_render_batch_fwd(ctx, g, frames, F, workspace, ws_bytes, image, final_T, last_idx, stream);
                    if (st == GV_OK)
                        st = gv_render_batch_bwd(ctx, g, frames, F, workspace, ws_bytes, final_T, last_idx, dL_dimage,
                                                 grad, stream);
                }
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) == cudaSuccess) {
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = t / reps;
                }
            }
            if (st == GV_ERR_CUDA) result = st;  // a CUDA failure ends the search
            if (ms_out) ms_out[k] = ms;
            if (st == GV_OK && ms < best_ms) { best_ms = ms; found = o; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != GV_OK) { ctx->opt = keep; return result; }
    if (!std::isfinite(best_ms)) { ctx->opt = keep; return fail(ctx, GV_ERR_CAPACITY, "no configuration fits the workspace"); }
    ctx->opt = found;
    if (best) *best = found;
    return GV_OK;
}

gv_status gv_graph_capture(gv_ctx *ctx, const gv_gaussians *g, const gv_frame_desc *frames, int32_t F,
                           void *workspace, size_t ws_bytes, float *image, float *final_T, int32_t *last_idx,
                           const float *target, float loss_scale, float *loss, float *dL_dimage,
                           gv_gaussians_grad *grad, gv_stream stream, gv_graph **out) {
    if (!ctx || !out) return GV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!stream) return fail(ctx, GV_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    gv_status st = check_gaussians(ctx, g);
    if (st != GV_OK) return st;
    if (dL_dimage) {
        st = check_grad(ctx, grad, g);
        if (st != GV_OK) return st;
    }
    gv_graph *G = new (std::nothrow) gv_graph();
    if (!G) return fail(ctx, GV_ERR_INVALID_ARG, "out of host memory");
    G->ctx = ctx;
    G->opt = ctx->opt;
    st = make_plan(ctx, ctx->opt, g->N, frames, F, 0, ws_bytes, G->plan, g->n_ctrl);
    G->n_ctrl = g->n_ctrl;
    if (st != GV_OK) { delete G; return st; }
    G->work = make_work(workspace, G->plan.L);
    G->frames.assign(frames, frames + F);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { delete G; return fail(ctx, GV_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e)); }
    ctx->capturing = true;
    // with a target, the L2 loss is fused into the compositing forward
    LossArgs la;
    if (target) {
        la.target = target;
        la.dL = dL_dimage;
        la.loss = loss;
        la.scale = loss_scale;
        if (loss) {
            const cudaError_t e2 = cudaMemsetAsync(loss, 0, sizeof(float), s);
            if (e2 != cudaSuccess) st = fail(ctx, GV_ERR_CUDA, "loss in capture: %s", cudaGetErrorString(e2));
        }
    }
    if (st == GV_OK) st = forward_stages(ctx, g, G->plan, G->work, image, final_T, last_idx, s, la);
    if (st == GV_OK && dL_dimage)
        st = backward_stages(ctx, g, G->plan, G->work, final_T, last_idx, dL_dimage, grad, s);
    ctx->capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (st != GV_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete G;
        return st != GV_OK ? st : fail(ctx, GV_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    }
    G->graph = graph;
    // locate the setup kernel nodes (frame table upload) for gv_graph_set_frames
    size_t n = 0;
    cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(graph, nodes.data(), &n);
    std::vector<std::pair<int, cudaGraphNode_t>> found;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        if (kp.func != setup_kernel_ptr()) continue;
        int first = *(int *)kp.kernelParams[2];
        found.push_back({first, nd});
    }
    std::sort(found.begin(), found.end(), [](auto &a, auto &b) { return a.first < b.first; });
    for (auto &f : found) G->setup_nodes.push_back(f.second);
    e = cudaGraphInstantiate(&G->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete G;
        return fail(ctx, GV_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    *out = G;
    return GV_OK;
}

gv_status gv_graph_set_frames(gv_graph *G, const gv_frame_desc *frames, int32_t F) {
    if (!G) return GV_ERR_INVALID_ARG;
    gv_ctx *ctx = G->ctx;
    if (F != (int32_t)G->frames.size() || !frames) return fail(ctx, GV_ERR_INVALID_ARG, "frame count differs from capture");
    for (int f = 0; f < F; f++) {
        const gv_frame_desc &a = frames[f], &b = G->frames[f];
        if (a.cam.W != b.cam.W || a.cam.H != b.cam.H || a.gauss_offset != b.gauss_offset ||
            a.gauss_count != b.gauss_count || a.pixel_offset != b.pixel_offset)
            return fail(ctx, GV_ERR_INVALID_ARG, "frame %d: size, Gaussian range or pixel offset differs from capture", f);
    }
    Plan pl;
    long long N = 0;
    for (int f = 0; f < F; f++) N = std::max<long long>(N, frames[f].gauss_offset + frames[f].gauss_count);
    gv_status st = make_plan(ctx, G->opt, N, frames, F, G->plan.L.key_cap, 0, pl, G->n_ctrl);
    if (st != GV_OK) return st;
    int ci = 0;
    for (int first = 0; first < F; first += kMaxFramesPerSetup, ci++) {
        if (ci >= (int)G->setup_nodes.size()) return fail(ctx, GV_ERR_INVALID_ARG, "graph has no setup node %d", ci);
        FrameChunk ch;
        memset(&ch, 0, sizeof(ch));
        int cnt = std::min(kMaxFramesPerSetup, F - first);
        for (int i = 0; i < cnt; i++) ch.f[i] = pl.frames[first + i];
        cudaKernelNodeParams kp;
        GV_CUDA(cudaGraphKernelNodeGetParams(G->setup_nodes[ci], &kp));
        Work w = G->work;
        int zero_all = first == 0 ? 1 : 0;
        long long spin = ctx->spin_limit;
        int drop = ctx->drop_signal;
        void *args[] = {&w, &ch, &first, &cnt, &zero_all, &spin, &drop};
        kp.kernelParams = args;
        kp.extra = nullptr;
        GV_CUDA(cudaGraphExecKernelNodeSetParams(G->exec, G->setup_nodes[ci], &kp));
    }
    G->frames.assign(frames, frames + F);
    return GV_OK;
}

gv_status gv_graph_launch(gv_graph *G, gv_stream stream) {
    if (!G) return GV_ERR_INVALID_ARG;
    gv_ctx *ctx = G->ctx;
    GV_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
    return GV_OK;
}

gv_status gv_graph_destroy(gv_graph *G) {
    if (!G) return GV_OK;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
    return GV_OK;
}

gv_status gv_debug_bin_sort(gv_ctx *ctx, int64_t n, const float *u, const float *v, const float *sxx, const float *sxy,
                            const float *syy, const float *tau, const float *depth, const uint8_t *valid, int32_t W,
                            int32_t H, void *workspace, size_t ws_bytes, int32_t *counts, uint32_t *sorted_tile,
                            uint32_t *sorted_id, int64_t cap, int64_t *K, gv_stream stream) {
    if (!ctx || n < 0 || !workspace || !K) return GV_ERR_INVALID_ARG;
    if (n > 0 && (!u || !v || !sxx || !sxy || !syy || !tau || !depth || !valid))
        return fail(ctx, GV_ERR_INVALID_ARG, "NULL input");
    gv_frame_desc d;
    memset(&d, 0, sizeof(d));
    d.cam.W = W; d.cam.H = H; d.cam.fx = d.cam.fy = 1.f;
    d.gauss_count = n;
    Plan pl;
    gv_status st = make_plan(ctx, ctx->opt, n, &d, 1, 0, ws_bytes, pl);
    if (st != GV_OK) return st;
    Work w = make_work(workspace, pl.L);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_setup(ctx, w, pl, s);
    if (st != GV_OK) return st;
    GV_CUDA(launch_bin_from_screen(w, n, u, v, sxx, sxy, syy, tau, depth, valid, ctx->opt.tile_w, ctx->opt.tile_h,
                                   counts, ctx->num_sms, s));
    int tres = 0;
    if (n > 0) {
        int dres = 0;
        const unsigned *n_pairs = reinterpret_cast<const unsigned *>(reinterpret_cast<const char *>(w.hdr) +
                                                                       offsetof(DevHeader, n_pairs));
        const unsigned *n_drawn = reinterpret_cast<const unsigned *>(reinterpret_cast<const char *>(w.hdr) +
                                                                       offsetof(DevHeader, n_drawn));
        unsigned *dk[2] = {w.dkey[0], w.dkey[1]}, *dv[2] = {w.dval[0], w.dval[1]};
        GV_CUDA(launch_radix_sort(w, dk, dv, n_pairs, w.L.P, 32, true, true, 0, 0, ctx->num_sms, s, &dres, 0,
                                  n_drawn));
        GV_CUDA(launch_emit(w, dres, ctx->opt.tile_w, ctx->opt.tile_h, ctx->num_sms, s));
        GV_CUDA(tile_sort_rest(ctx, w, s, &tres));
    }
    int64_t needed = 0;
    st = gv_read_status(ctx, workspace, ws_bytes, stream, &needed);
    *K = needed;
    if (st != GV_OK) return st;
    if (needed > cap) return fail(ctx, GV_ERR_CAPACITY, "output capacity %lld < %lld keys", (long long)cap, (long long)needed);
    if (needed > 0) {
        if (sorted_tile) GV_CUDA(cudaMemcpyAsync(sorted_tile, w.tkey[tres], 4 * (size_t)needed, cudaMemcpyDeviceToDevice, s));
        if (sorted_id) GV_CUDA(cudaMemcpyAsync(sorted_id, w.tval[tres], 4 * (size_t)needed, cudaMemcpyDeviceToDevice, s));
    }
    GV_CUDA(cudaStreamSynchronize(s));
    return GV_OK;
}

gv_status gv_debug_read(gv_ctx *ctx, const gv_frame_desc *frames, int32_t F, const void *workspace, size_t ws_bytes,
                        float *mean2d, float *conic, float *opacity, float *depth, int32_t *counts, uint32_t *sorted_id,
                        uint32_t *sorted_tile, uint32_t *ranges, int64_t *P, int64_t *K, int64_t *tiles,
                        gv_stream stream) {
    if (!ctx || !workspace) return GV_ERR_INVALID_ARG;
    long long N = 0;
    for (int f = 0; frames && f < F; f++) N = std::max<long long>(N, frames[f].gauss_offset + frames[f].gauss_count);
    Plan pl;
    gv_status st = make_plan(ctx, ctx->opt, N, frames, F, 0, ws_bytes, pl);
    if (st != GV_OK) return st;
    Work w = make_work(const_cast<void *>(workspace), pl.L);
    cudaStream_t s = (cudaStream_t)stream;
    GV_CUDA(launch_gather_debug(w, mean2d, conic, opacity, depth, counts, depth_result_buf(), s));
    DevHeader h;
    GV_CUDA(cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s));
    GV_CUDA(cudaStreamSynchronize(s));
    int tres = tile_result_buf(pl.L);
    if (sorted_id && h.keys_used)
        GV_CUDA(cudaMemcpyAsync(sorted_id, w.tval[tres], 4 * (size_t)h.keys_used, cudaMemcpyDeviceToDevice, s));
    if (sorted_tile && h.keys_used)
        GV_CUDA(cudaMemcpyAsync(sorted_tile, w.tkey[tres], 4 * (size_t)h.keys_used, cudaMemcpyDeviceToDevice, s));
    if (ranges) GV_CUDA(launch_debug_ranges(w, reinterpret_cast<uint2 *>(ranges), s));
    GV_CUDA(cudaStreamSynchronize(s));
    if (P) *P = pl.L.P;
    if (K) *K = h.keys_used;
    if (tiles) *tiles = pl.L.tiles;
    return GV_OK;
}

gv_status gv_debug_set_wait(gv_ctx *ctx, int64_t spin_limit, int32_t drop_signal) {
    if (!ctx) return GV_ERR_INVALID_ARG;
    ctx->spin_limit = spin_limit > 0 ? spin_limit : kDefaultSpin;
    ctx->drop_signal = drop_signal ? 1 : 0;
    return GV_OK;
}

gv_status gv_debug_read_grad2d(gv_ctx *ctx, const gv_frame_desc *frames, int32_t F, const void *workspace,
                               size_t ws_bytes, float *out, gv_stream stream) {
    if (!ctx || !workspace || !out) return GV_ERR_INVALID_ARG;
    long long N = 0;
    for (int f = 0; frames && f < F; f++) N = std::max<long long>(N, frames[f].gauss_offset + frames[f].gauss_count);
    Plan pl;
    gv_status st = make_plan(ctx, ctx->opt, N, frames, F, 0, ws_bytes, pl);
    if (st != GV_OK) return st;
    Work w = make_work(const_cast<void *>(workspace), pl.L);
    GV_CUDA(launch_grad2d_debug(w, out, (cudaStream_t)stream));
    GV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return GV_OK;
}

}  // extern "C"
