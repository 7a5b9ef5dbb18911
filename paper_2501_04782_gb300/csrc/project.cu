// project.cu -- projection of (frame, Gaussian) pairs to screen space (forward) and the
// chain rule from screen-space gradients back to the raw parameters (backward).
//
// Sec. 3.1: Sigma = (R S)(R S)^T from a quaternion and log-scales; the Gaussian is
// projected onto the image plane of the frame's pinhole camera (Sec. 3.4: intrinsics
// fx, fy, cx, cy; extrinsics R, t).  The 2D covariance is the local-affine (EWA)
// approximation J W Sigma W^T J^T plus a 0.3 px^2 low-pass, its inverse the conic.
// Sec. 3.2: the mean moves with time, colour and opacity do not -- a linear drift
// mu_t = mu_0 + t vel, or Eq. 2's clamped cubic B-spline over control points with Eq. 3's
// cubic log-scale and quaternion terms (SPLINE).  Sec. 3.1's view-dependent colour adds
// real spherical harmonics of degree 1-3 at the direction from the camera centre (SH).
// The forward also culls each pair's extent box per tile row against the ellipse, counts
// the digits of the depth sort and of the tile sort's kept keys, and sets the "drawn on
// some frame" flag (Sec. 4.1); the backward also accumulates the camera adjoint
// (Sec. 3.4, CAM) and runs ill-conditioned pairs' geometry in FP64.  The kernels are
// HBM-bound: one thread per pair, coalesced SoA plane reads.
#include <algorithm>

#include <type_traits>

#include "gv_internal.cuh"

namespace gvk {

namespace {

// Scalar helpers so the projection and its chain rule can run in FP32 (the default) or
// FP64 (ill-conditioned pairs in the backward).
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

template <typename F>
struct PairState {
    F mx, my, mz;        // world mean at the frame's time
    F xc, yc, zc;        // camera-space mean
    F s0, s1, s2;        // scales
    F qw, qx, qy, qz;    // normalised quaternion
    F inv_qn;            // 1 / |q|
    F R[9];              // Gaussian rotation
    F S3[6];             // world covariance xx, xy, xz, yy, yz, zz
    F T0[3], T1[3];      // rows of J W
    F a, b, c;           // Sigma2 (with low-pass)
    F A, B, C;           // conic
    F u, v;
    F o;
    bool valid;
};

// The projection of one (frame, Gaussian) pair in three parts: the mean at the frame's time
// (load_mean), the Gaussian's own shape -- scales, rotation, 3D covariance, opacity --
// (load_shape: frame-independent unless SPLINE), and the camera part (project_camera).
// SPLINE: the time-parameterised form (g.n_ctrl > 0: B-spline means, cubic log-scale and
// quaternion); otherwise mean + t vel and constant log-scale and quaternion.
template <typename F, bool SPLINE = false>
__device__ __forceinline__ void load_mean(const GaussPtrs &g, long long gi, const DevFrame &fr, PairState<F> &st) {
    const long long N = g.N;
    const F time = (F)fr.time;
    if constexpr (SPLINE) {  // Eq. 2: mu(t) = sum_i N_{i,3}(t) P_i over the four non-zero weights
        const long long C = g.n_ctrl;
        F m[3] = {(F)0, (F)0, (F)0};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const F wj = (F)fr.spline_w[j];
            const long long c = fr.spline_lo + j;
#pragma unroll
            for (int k = 0; k < 3; k++) m[k] = fma_(wj, (F)g.ctrl[(k * C + c) * N + gi], m[k]);
        }
        st.mx = m[0]; st.my = m[1]; st.mz = m[2];
    } else {
        st.mx = (F)g.mean[gi];
        st.my = (F)g.mean[N + gi];
        st.mz = (F)g.mean[2 * N + gi];
        if (g.vel) {
            st.mx = fma_(time, (F)g.vel[gi], st.mx);
            st.my = fma_(time, (F)g.vel[N + gi], st.my);
            st.mz = fma_(time, (F)g.vel[2 * N + gi], st.mz);
        }
    }
}

template <typename F, bool SPLINE = false>
__device__ __forceinline__ void load_shape(const GaussPtrs &g, long long gi, const DevFrame &fr, PairState<F> &st) {
    const long long N = g.N;
    const F time = (F)fr.time;
    // Eq. 3: log-scale and quaternion as cubic polynomials of t (t^0 term: the plain plane)
    auto cubic = [&](const float *base, const float *terms, int rows, int k) -> F {
        F v = (F)base[k * N + gi];
        if (SPLINE && terms) {
            const F a1 = (F)terms[(0 * rows + k) * N + gi], a2 = (F)terms[(1 * rows + k) * N + gi],
                    a3 = (F)terms[(2 * rows + k) * N + gi];
            v = fma_(time, fma_(time, fma_(time, a3, a2), a1), v);
        }
        return v;
    };
    st.s0 = exp_(cubic(g.log_scale, g.log_scale_t, 3, 0));
    st.s1 = exp_(cubic(g.log_scale, g.log_scale_t, 3, 1));
    st.s2 = exp_(cubic(g.log_scale, g.log_scale_t, 3, 2));
    F qw = cubic(g.quat, g.quat_t, 4, 0), qx = cubic(g.quat, g.quat_t, 4, 1), qy = cubic(g.quat, g.quat_t, 4, 2),
      qz = cubic(g.quat, g.quat_t, 4, 3);
    F inv = rsqrt_(qw * qw + qx * qx + qy * qy + qz * qz);
    st.inv_qn = inv;
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    st.qw = qw; st.qx = qx; st.qy = qy; st.qz = qz;
    F *R = st.R;
    const F one = (F)1, two = (F)2;
    R[0] = one - two * (qy * qy + qz * qz); R[1] = two * (qx * qy - qw * qz); R[2] = two * (qx * qz + qw * qy);
    R[3] = two * (qx * qy + qw * qz); R[4] = one - two * (qx * qx + qz * qz); R[5] = two * (qy * qz - qw * qx);
    R[6] = two * (qx * qz - qw * qy); R[7] = two * (qy * qz + qw * qx); R[8] = one - two * (qx * qx + qy * qy);
    F s0q = st.s0 * st.s0, s1q = st.s1 * st.s1, s2q = st.s2 * st.s2;
    // Sigma3_ij = sum_k R_ik R_jk s_k^2
    st.S3[0] = R[0] * R[0] * s0q + R[1] * R[1] * s1q + R[2] * R[2] * s2q;
    st.S3[1] = R[0] * R[3] * s0q + R[1] * R[4] * s1q + R[2] * R[5] * s2q;
    st.S3[2] = R[0] * R[6] * s0q + R[1] * R[7] * s1q + R[2] * R[8] * s2q;
    st.S3[3] = R[3] * R[3] * s0q + R[4] * R[4] * s1q + R[5] * R[5] * s2q;
    st.S3[4] = R[3] * R[6] * s0q + R[4] * R[7] * s1q + R[5] * R[8] * s2q;
    st.S3[5] = R[6] * R[6] * s0q + R[7] * R[7] * s1q + R[8] * R[8] * s2q;
    st.o = one / (one + exp_(-(F)g.logit[gi]));
}

// The camera part: camera-space mean, near cull, J W, Sigma2 (with the low-pass), conic,
// screen mean; st.valid false when culled.
template <typename F>
__device__ __forceinline__ void project_camera(const DevFrame &fr, PairState<F> &st) {
    const F one = (F)1;
    F W[9];
    for (int i = 0; i < 9; i++) W[i] = (F)fr.R[i];
    st.xc = W[0] * st.mx + W[1] * st.my + W[2] * st.mz + (F)fr.t[0];
    st.yc = W[3] * st.mx + W[4] * st.my + W[5] * st.mz + (F)fr.t[1];
    st.zc = W[6] * st.mx + W[7] * st.my + W[8] * st.mz + (F)fr.t[2];
    st.valid = st.zc > (F)kZNear;
    if (!st.valid) return;
    F iz = one / st.zc;
    F rx = st.xc * iz, ry = st.yc * iz;
    F jx = (F)fr.fx * iz, jy = (F)fr.fy * iz;
    // rows of T = J W with J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]]
    for (int j = 0; j < 3; j++) {
        st.T0[j] = jx * (W[j] - rx * W[6 + j]);
        st.T1[j] = jy * (W[3 + j] - ry * W[6 + j]);
    }
    const F *S = st.S3;
    F v0x = S[0] * st.T0[0] + S[1] * st.T0[1] + S[2] * st.T0[2];
    F v0y = S[1] * st.T0[0] + S[3] * st.T0[1] + S[4] * st.T0[2];
    F v0z = S[2] * st.T0[0] + S[4] * st.T0[1] + S[5] * st.T0[2];
    F v1x = S[0] * st.T1[0] + S[1] * st.T1[1] + S[2] * st.T1[2];
    F v1y = S[1] * st.T1[0] + S[3] * st.T1[1] + S[4] * st.T1[2];
    F v1z = S[2] * st.T1[0] + S[4] * st.T1[1] + S[5] * st.T1[2];
    st.a = st.T0[0] * v0x + st.T0[1] * v0y + st.T0[2] * v0z + (F)kEps2d;
    st.b = st.T0[0] * v1x + st.T0[1] * v1y + st.T0[2] * v1z;
    st.c = st.T1[0] * v1x + st.T1[1] * v1y + st.T1[2] * v1z + (F)kEps2d;
    F det = st.a * st.c - st.b * st.b;
    if (!(det > (F)0)) { st.valid = false; return; }
    F idet = one / det;
    st.A = st.c * idet;
    st.B = -st.b * idet;
    st.C = st.a * idet;
    st.u = fma_((F)fr.fx, rx, (F)fr.cx);
    st.v = fma_((F)fr.fy, ry, (F)fr.cy);
    if (!(isfinite(st.u) && isfinite(st.v) && isfinite(st.A) && isfinite(st.B) && isfinite(st.C)))
        st.valid = false;
}

template <typename F, bool SPLINE = false>
__device__ __forceinline__ void load_and_project(const GaussPtrs &g, long long gi, const DevFrame &fr,
                                                 PairState<F> &st) {
    load_mean<F, SPLINE>(g, gi, fr, st);
    load_shape<F, SPLINE>(g, gi, fr, st);
    project_camera<F>(fr, st);
}

// Per-block binning counters of the projection: depth-sort digits (4 passes), tile-sort
// digits of the kept keys (digit 0 through a difference array), kept-key total.
struct BinShared {
    unsigned depth[4][kRadix];
    unsigned tile[4][kRadix];
    int diff[257];
    unsigned full;
    unsigned drawn;  // pairs with a depth key
    unsigned long long live;
};

__device__ __forceinline__ void bin_shared_init(BinShared &sb) {
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
        (&sb.depth[0][0])[i] = 0u;
        (&sb.tile[0][0])[i] = 0u;
    }
    for (int i = threadIdx.x; i < 257; i += blockDim.x) sb.diff[i] = 0;
    if (threadIdx.x == 0) { sb.full = 0u; sb.drawn = 0u; sb.live = 0ull; }
}

// View-dependent colour (Sec. 3.1: colour as spherical harmonics of order d_c <= 3; the
// degree-0 term is the plain colour plane): colour = rgb + sum_k Y_k(d) sh[ch][k], Y_k the
// real spherical harmonics of degrees 1..d_c in the order (l, m = -l..l) with the
// Condon-Shortley phase, written out as Cartesian polynomials of the unit direction d from
// the camera centre to the mean (world frame).  Normalisations sqrt((2l+1)/(4 pi) ...):
constexpr float kSh1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kSh2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float kSh20 = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float kSh22 = 0.54627421529603959f;  // sqrt(15/(16 pi))
constexpr float kSh33 = 0.59004358992664352f;  // sqrt(35/(32 pi))
constexpr float kSh32a = 2.8906114426405538f;  // sqrt(105/(4 pi))
constexpr float kSh31 = 0.45704579946446572f;  // sqrt(21/(32 pi))
constexpr float kSh30 = 0.37317633259011540f;  // sqrt(7/(16 pi))
constexpr float kSh32 = 1.4453057213202769f;   // sqrt(105/(16 pi))
constexpr int kShMax = 15;                      // terms above degree 0 at degree 3

__device__ __forceinline__ int sh_terms(int deg) { return (deg + 1) * (deg + 1) - 1; }

__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float Y[kShMax]) {
    Y[0] = -kSh1 * y;
    Y[1] = kSh1 * z;
    Y[2] = -kSh1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[3] = kSh2a * x * y;
    Y[4] = -kSh2a * y * z;
    Y[5] = kSh20 * (3.f * zz - 1.f);
    Y[6] = -kSh2a * x * z;
    Y[7] = kSh22 * (xx - yy);
    if (deg < 3) return;
    Y[8] = -kSh33 * y * (3.f * xx - yy);
    Y[9] = kSh32a * x * y * z;
    Y[10] = -kSh31 * y * (5.f * zz - 1.f);
    Y[11] = kSh30 * z * (5.f * zz - 3.f);
    Y[12] = -kSh31 * x * (5.f * zz - 1.f);
    Y[13] = kSh32 * z * (xx - yy);
    Y[14] = -kSh33 * x * (xx - 3.f * yy);
}

// sum_k s_k grad Y_k at (x, y, z), the polynomials taken as functions of three variables.
__device__ __forceinline__ void sh_dir_grad(int deg, float x, float y, float z, const float s[kShMax], float g[3]) {
    float gx = -kSh1 * s[2], gy = -kSh1 * s[0], gz = kSh1 * s[1];
    if (deg >= 2) {
        gx += kSh2a * (y * s[3] - z * s[6]) + 2.f * kSh22 * x * s[7];
        gy += kSh2a * (x * s[3] - z * s[4]) - 2.f * kSh22 * y * s[7];
        gz += -kSh2a * (y * s[4] + x * s[6]) + 6.f * kSh20 * z * s[5];
    }
    if (deg >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z, q = 5.f * zz - 1.f;
        gx += -6.f * kSh33 * x * y * s[8] + kSh32a * y * z * s[9] - kSh31 * q * s[12] + 2.f * kSh32 * x * z * s[13] -
              3.f * kSh33 * (xx - yy) * s[14];
        gy += -3.f * kSh33 * (xx - yy) * s[8] + kSh32a * x * z * s[9] - kSh31 * q * s[10] - 2.f * kSh32 * y * z * s[13] +
              6.f * kSh33 * x * y * s[14];
        gz += kSh32a * x * y * s[9] - 10.f * kSh31 * y * z * s[10] + kSh30 * (15.f * zz - 3.f) * s[11] -
              10.f * kSh31 * x * z * s[12] + kSh32 * (xx - yy) * s[13];
    }
    g[0] = gx;
    g[1] = gy;
    g[2] = gz;
}

// Unit view direction d = (mu - c) / |mu - c| from the frame's camera centre c, and 1/|mu - c|.
__device__ __forceinline__ void view_dir(const PairState<float> &st, const DevFrame &fr, float d[3], float &rn) {
    const float vx = st.mx - fr.campos[0], vy = st.my - fr.campos[1], vz = st.mz - fr.campos[2];
    rn = rsqrtf(vx * vx + vy * vy + vz * vz);
    d[0] = vx * rn;
    d[1] = vy * rn;
    d[2] = vz * rn;
}

// The pair's colour: rgb, plus the spherical-harmonic terms when SH (valid pairs only: a
// culled pair's colour is never read).
template <bool SH>
__device__ __forceinline__ void pair_colour(const GaussPtrs &g, long long gi, const PairState<float> &st,
                                            const DevFrame &fr, float col[3]) {
    const long long N = g.N;
    col[0] = g.rgb[gi];
    col[1] = g.rgb[N + gi];
    col[2] = g.rgb[2 * N + gi];
    if constexpr (SH) {
        if (!st.valid) return;
        float d[3], rn, Y[kShMax];
        view_dir(st, fr, d, rn);
        sh_eval(g.sh_degree, d[0], d[1], d[2], Y);
        const int K = sh_terms(g.sh_degree);
#pragma unroll
        for (int k = 0; k < kShMax; k++) {
            if (k >= K) break;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) col[ch] = fmaf(Y[k], g.sh[((long long)ch * K + k) * N + gi], col[ch]);
        }
    }
}

// Bins one pair (culled rule, see gv_internal.cuh), the per-pair part: extent box, cells,
// cull record (rect and ell written).  Returns the number of tile rows of its box (0 when
// it bins nothing); the rows are culled by warp_cull_rows.
struct PairBin {
    float u, v;
    float4 e;
    uint2 box;
    unsigned tile_offset, tiles_x;
    int rows;
};

__device__ __forceinline__ unsigned bin_pair(const Work &w, unsigned p, float u, float v, float a, float b, float c,
                                             float tau, const DevFrame &fr, unsigned frame_word, int lw, int lh,
                                             PairBin &pb) {
    float ex;
    PixBox bx;
    pb.u = u; pb.v = v; pb.rows = 0;
    pb.tile_offset = fr.tile_offset; pb.tiles_x = fr.tiles_x;
    if (!extent_box(u, v, a, c, tau, fr.W, fr.H, ex, bx)) {
        w.rect[p] = make_uint4(0u, 0u, 0u, frame_word);
        pb.box = make_uint2(0u, 0u);
        pb.e = make_float4(0.f, 0.f, 0.f, 0.f);
        return 0u;
    }
    const int tx0 = bx.x0 >> lw, tx1 = bx.x1 >> lw, ty0 = bx.y0 >> lh, ty1 = bx.y1 >> lh;
    const unsigned cells = (unsigned)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
    pb.e = cull_record(a, b, c, tau, ex);
    pb.box = pack_box(bx);
    pb.rows = ty1 - ty0 + 1;
    w.rect[p] = make_uint4(pb.box.x, pb.box.y, cells, frame_word);
    w.ell[p] = pb.e;
    return cells;
}

// The rows of the warp's 32 pairs, culled by the warp together (lane l takes rows l,
// l + 32, ... of the concatenated row list, so a pair with many tile rows does not hold
// the other lanes back): counts the tile-sort digits of the kept row runs.  Returns the
// kept keys of the rows this lane processed; with PER_PAIR, also adds each row's kept
// keys to s_pair_live[owner lane].  kept_lanes receives (in every lane) the mask of the
// lanes whose pair kept at least one key.  Every lane of the warp calls it.
template <bool PER_PAIR>
__device__ __forceinline__ unsigned warp_cull_rows(const PairBin &pb, int lw, int lh, int tile_passes, BinShared &sb,
                                                   unsigned *s_pair_live, unsigned &kept_lanes) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int inc = pb.rows;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    const int start = inc - pb.rows, R = __shfl_sync(FULL, inc, 31);
    unsigned live = 0, owners = 0;
    for (int base = 0; base < R; base += 32) {
        const int r = base + lane;
        int lo = 0, hi = 31;  // owner: the last lane whose rows start at or before r
#pragma unroll
        for (int it = 0; it < 5; it++) {
            const int mid = (lo + hi + 1) >> 1;
            if (__shfl_sync(FULL, start, mid) <= r) lo = mid; else hi = mid - 1;
        }
        const float u = __shfl_sync(FULL, pb.u, lo), v = __shfl_sync(FULL, pb.v, lo);
        const float4 e = make_float4(__shfl_sync(FULL, pb.e.x, lo), __shfl_sync(FULL, pb.e.y, lo),
                                     __shfl_sync(FULL, pb.e.z, lo), __shfl_sync(FULL, pb.e.w, lo));
        const uint4 rb = make_uint4(__shfl_sync(FULL, pb.box.x, lo), __shfl_sync(FULL, pb.box.y, lo), 0u, 0u);
        const unsigned toff = __shfl_sync(FULL, pb.tile_offset, lo), tx = __shfl_sync(FULL, pb.tiles_x, lo);
        const int ostart = __shfl_sync(FULL, start, lo);
        if (r < R) {
            const PixBox bx = unpack_box(rb);
            const int ty = (bx.y0 >> lh) + (r - ostart);
            int t0, t1;
            if (cull_tiles(u, v, e, bx, ty, lw, lh, t0, t1)) {
                const unsigned len = (unsigned)(t1 - t0 + 1);
                live += len;
                owners |= 1u << lo;
                count_tile_run(toff + (unsigned)ty * tx + (unsigned)t0, len, tile_passes, sb.diff, &sb.full, sb.tile);
                if (PER_PAIR) atomicAdd(s_pair_live + lo, len);
            }
        }
    }
    kept_lanes = __reduce_or_sync(FULL, owners);
    return live;
}

// Adds a block's binning counters to the workspace: depth digits to histogram rows 0-3,
// tile digits to rows 4.., the kept-key total to keys_total.  Every thread calls it.
__device__ __forceinline__ void bin_shared_flush(const Work &w, BinShared &sb, unsigned live, int tile_passes) {
    const unsigned long long lsum = __reduce_add_sync(0xffffffffu, live);
    if ((threadIdx.x & 31) == 0 && lsum) atomicAdd(&sb.live, lsum);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
        const unsigned c = (&sb.depth[0][0])[i];
        if (c) atomicAdd(w.hist + i, c);
    }
    if (threadIdx.x == 0 && sb.live) atomicAdd(&w.hdr->keys_total, sb.live);
    if (threadIdx.x == 0 && sb.drawn) atomicAdd(&w.hdr->n_drawn, sb.drawn);
    flush_tile_hist(tile_passes, sb.diff, sb.full, sb.tile, w.hist + 4 * kRadix);
}

// Ill-conditioned pairs: when Sigma2 is close to singular (a c / det > 64, a Gaussian
// stretched by the perspective, typically near the camera and far off axis) the FP32
// inverse and -Q G Q lose digits.  The projection lists such pairs (and flags them in
// rect.w); the backward skips their geometric chain rule in FP32 and a small FP64 kernel
// redoes it, concurrently with the FP32 pass (keeping FP64 registers out of the common
// FP32 kernel).
constexpr float kFp64Condition = 64.f;

__device__ __forceinline__ bool ill_conditioned(const PairState<float> &st) {
    const float det = st.a * st.c - st.b * st.b;
    return st.a * st.c > kFp64Condition * det;
}

// alpha >= 1/255 needs d^T conic d <= tau = 2 ln(255 o) (capped at 2 ln 255 by the clamp)
__device__ __forceinline__ float tau_of(float o) { return fminf(2.f * (kLn255 + logf(o)), kExtK * kExtK); }

// The records of one projected pair: binning box and cull record (bin_pair; nothing binned
// when the pair is culled), the FP64 list entry of an ill-conditioned binned pair, the
// staged compositing record and the depth key.  Returns the key (kNoKey: bins nothing).
__device__ __forceinline__ unsigned write_pair(const Work &w, unsigned p, int f, const DevFrame &fr,
                                               const PairState<float> &st, float tau, float log2o, const float col[3],
                                               int lw, int lh, PairBin &pb) {
    const unsigned cells =
        bin_pair(w, p, st.u, st.v, st.a, st.b, st.c, st.valid ? tau : 0.f, fr, (unsigned)f, lw, lh, pb);
    if (cells && ill_conditioned(st)) {  // only binned pairs get a gradient
        w.fp64_list[atomicAdd(&w.hdr->fp64_count, 1u)] = p;
        w.rect[p].w = (unsigned)f | kRectFp64;
    }
    w.feat0[p] = make_float4(st.u, st.v, -0.5f * kLog2e * st.A, -kLog2e * st.B);
    w.feat1[p] = make_float4(-0.5f * kLog2e * st.C, log2o, col[0], col[1]);
    w.feat2[p] = col[2];
    const unsigned key = cells ? __float_as_uint(st.zc) : kNoKey;
    w.dkey[0][p] = key;
    return key;
}

// Counters of one round of pairs (every lane of the warp calls it): the kept keys' tile
// digits (warp_cull_rows), the drawn flag, the drawn pairs and their depth digits (the sort
// drops the others).  Returns the round's kept keys of this lane's rows.
__device__ __forceinline__ unsigned count_round(const GaussPtrs &g, long long gi, bool in, unsigned key,
                                                const PairBin &pb, int lw, int lh, int tile_passes, BinShared &sb,
                                                unsigned &kept) {
    unsigned kept_lanes;
    const unsigned live = warp_cull_rows<false>(pb, lw, lh, tile_passes, sb, nullptr, kept_lanes);
    kept = (kept_lanes >> (threadIdx.x & 31)) & 1u;
    const unsigned active = __ballot_sync(0xffffffffu, in && key != kNoKey);
    if ((threadIdx.x & 31) == 0 && active) atomicAdd(&sb.drawn, (unsigned)__popc(active));
    if (in && key != kNoKey)
        for (int ps = 0; ps < 4; ps++) count_digit(sb.depth[ps], (key >> (8 * ps)) & 255u, active);
    return live;
}

// Grid-stride over the pairs so each block flushes its counters once.
template <bool SPLINE, bool SH>
__global__ void __launch_bounds__(256) project_fwd_kernel(Work w, GaussPtrs g, int lw, int lh, int tile_passes) {
    pdl_prologue();
    __shared__ BinShared sb;
    bin_shared_init(sb);
    __syncthreads();
    const unsigned stride = gridDim.x * blockDim.x;
    unsigned live_sum = 0;
    // every thread of a block runs the same number of rounds (the warp votes see full warps)
    for (unsigned base = blockIdx.x * blockDim.x; base < w.L.P; base += stride) {
        const unsigned p = base + threadIdx.x;
        const bool in = p < w.L.P;
        unsigned key = 0xFFFFFFFFu;
        PairBin pb;
        pb.rows = 0;
        long long gi = 0;
        if (in) {
            int f = find_frame_by_pair(w.frames, (int)w.L.F, p);
            const DevFrame &fr = w.frames[f];
            gi = fr.gauss_offset + (long long)(p - fr.pair_offset);
            PairState<float> st;
            load_and_project<float, SPLINE>(g, gi, fr, st);
            float col[3];
            pair_colour<SH>(g, gi, st, fr, col);
            key = write_pair(w, p, f, fr, st, tau_of(st.o), log2f(st.o), col, lw, lh, pb);
        }
        unsigned kept;
        live_sum += count_round(g, gi, in, key, pb, lw, lh, tile_passes, sb, kept);
        if (g.visible && kept) g.visible[gi] = 1;  // benign same-value race
    }
    bin_shared_flush(w, sb, live_sum, tile_passes);
}

// A shared set (every frame of the call draws the same Gaussian range; plain colour, means
// constant or drifting linearly): one thread per Gaussian loops over the frames, so its
// parameters are read once and the frame-independent part of the projection (scales,
// rotation, 3D covariance, opacity, colour, the cutoff level tau) is computed once instead
// of once per frame.  Records and counters are project_fwd_kernel's, pair by pair (the
// same expressions on the same values).
__global__ void __launch_bounds__(256, 4) project_fwd_shared_kernel(Work w, GaussPtrs g, int lw, int lh,
                                                                 int tile_passes) {
    pdl_prologue();
    __shared__ BinShared sb;
    bin_shared_init(sb);
    __syncthreads();
    const DevFrame &f0 = w.frames[0];
    const unsigned n = f0.gauss_count;
    const int F = (int)w.L.F;
    const long long N = g.N;
    const unsigned stride = gridDim.x * blockDim.x;
    unsigned live_sum = 0;
    // every thread of a block runs the same rounds (the warp votes see full warps)
    for (unsigned base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const unsigned j = base + threadIdx.x;
        const bool in = j < n;
        const long long gi = f0.gauss_offset + (long long)(in ? j : 0u);
        PairState<float> st;
        float m[3] = {0.f, 0.f, 0.f}, vel[3] = {0.f, 0.f, 0.f}, col[3] = {0.f, 0.f, 0.f};
        float tau = 0.f, log2o = 0.f;
        if (in) {
            for (int k = 0; k < 3; k++) {
                m[k] = g.mean[k * N + gi];
                if (g.vel) vel[k] = g.vel[k * N + gi];
                col[k] = g.rgb[k * N + gi];
            }
            load_shape<float, false>(g, gi, f0, st);
            tau = tau_of(st.o);
            log2o = log2f(st.o);
        }
        unsigned drawn = 0;
        for (int f = 0; f < F; f++) {
            const DevFrame &fr = w.frames[f];
            const unsigned p = fr.pair_offset + j;
            unsigned key = kNoKey;
            PairBin pb;
            pb.rows = 0;
            if (in) {
                if (g.vel) {
                    const float time = fr.time;
                    st.mx = fmaf(time, vel[0], m[0]);
                    st.my = fmaf(time, vel[1], m[1]);
                    st.mz = fmaf(time, vel[2], m[2]);
                } else {
                    st.mx = m[0]; st.my = m[1]; st.mz = m[2];
                }
                project_camera<float>(fr, st);
                key = write_pair(w, p, f, fr, st, tau, log2o, col, lw, lh, pb);
            }
            unsigned kept;
            live_sum += count_round(g, gi, in, key, pb, lw, lh, tile_passes, sb, kept);
            drawn |= kept;
        }
        if (g.visible && in && drawn) g.visible[gi] = 1;
    }
    bin_shared_flush(w, sb, live_sum, tile_passes);
}

// Stage-isolated binning: screen-space inputs of one frame given by the caller (mean,
// Sigma2, tau, depth); counts[p] receives the kept-key count.
__global__ void __launch_bounds__(256) bin_from_screen_kernel(Work w, long long n, const float *u, const float *v,
                                                              const float *sxx, const float *sxy, const float *syy,
                                                              const float *tau, const float *depth,
                                                              const uint8_t *valid, int lw, int lh, int tile_passes,
                                                              int32_t *counts) {
    pdl_prologue();
    __shared__ BinShared sb;
    __shared__ unsigned s_live[256];
    bin_shared_init(sb);
    __syncthreads();
    const unsigned stride = gridDim.x * blockDim.x;
    unsigned live_sum = 0;
    const DevFrame &fr = w.frames[0];
    unsigned *s_warp_live = s_live + (threadIdx.x & ~31u);
    for (unsigned base = blockIdx.x * blockDim.x; base < (unsigned)n; base += stride) {
        const unsigned p = base + threadIdx.x;
        const bool in = p < (unsigned)n;
        unsigned key = 0xFFFFFFFFu;
        PairBin pb;
        pb.rows = 0;
        s_live[threadIdx.x] = 0u;
        if (in) {
            unsigned cells = 0;
            if (valid[p]) cells = bin_pair(w, p, u[p], v[p], sxx[p], sxy[p], syy[p], tau[p], fr, 0u, lw, lh, pb);
            else w.rect[p] = make_uint4(0u, 0u, 0u, 0u);
            w.feat0[p] = make_float4(u[p], v[p], 0.f, 0.f);
            key = cells ? __float_as_uint(depth[p]) : 0xFFFFFFFFu;
            w.dkey[0][p] = key;
        }
        __syncwarp();
        unsigned kept_lanes;
        live_sum += warp_cull_rows<true>(pb, lw, lh, tile_passes, sb, s_warp_live, kept_lanes);
        __syncwarp();
        if (in && counts) counts[p] = (int32_t)s_live[threadIdx.x];
        // depth digits of the pairs with a key (the sort drops the others)
        const unsigned active = __ballot_sync(0xffffffffu, in && key != kNoKey);
        if ((threadIdx.x & 31) == 0 && active) atomicAdd(&sb.drawn, (unsigned)__popc(active));
        if (in && key != kNoKey)
            for (int ps = 0; ps < 4; ps++) count_digit(sb.depth[ps], (key >> (8 * ps)) & 255u, active);
    }
    bin_shared_flush(w, sb, live_sum, tile_passes);
}

// Chain rule of the geometric part of one pair: gradients w.r.t. the screen mean (du, dv)
// and the conic (dA, dB, dC) to mean, velocity, log-scale and quaternion, added into acc
// (rows 0-12 of the 17-row layout: mean 3, vel 3, log_scale 3, quat 4), and, when cam is
// not NULL, to the frame's camera (Sec. 3.4), added into cam[kCamGrad]: x_c = R mu + t
// gives dR += dx_c mu^T and dt += dx_c, T = J R gives dR += J^T dT, and u = fx x/z + cx,
// J00 = fx/z, J02 = -fx x/z^2 give dfx (likewise fy, cy).
template <typename F>
__device__ __forceinline__ void geometry_backward(const PairState<F> &st, const DevFrame &fr, F du, F dv, F dA,
                                                  F dB, F dC, float acc[17], float *cam = nullptr) {
    const F half = (F)0.5, two = (F)2;
    // conic Q = Sigma2^{-1}: dL/dSigma2 = -Q G Q with G = [[dA, dB/2], [dB/2, dC]]
    F X00 = st.A * dA + half * st.B * dB, X01 = half * st.A * dB + st.B * dC;
    F X10 = st.B * dA + half * st.C * dB, X11 = half * st.B * dB + st.C * dC;
    F ga = -(X00 * st.A + X01 * st.B);
    F gb = -(X00 * st.B + X01 * st.C);
    F gc = -(X10 * st.B + X11 * st.C);
    // Sigma2 = T Sigma3 T^T: dSigma3 = T^T G T, dT = 2 G T Sigma3
    const F *S = st.S3;
    F v0[3], v1[3];
    v0[0] = S[0] * st.T0[0] + S[1] * st.T0[1] + S[2] * st.T0[2];
    v0[1] = S[1] * st.T0[0] + S[3] * st.T0[1] + S[4] * st.T0[2];
    v0[2] = S[2] * st.T0[0] + S[4] * st.T0[1] + S[5] * st.T0[2];
    v1[0] = S[0] * st.T1[0] + S[1] * st.T1[1] + S[2] * st.T1[2];
    v1[1] = S[1] * st.T1[0] + S[3] * st.T1[1] + S[4] * st.T1[2];
    v1[2] = S[2] * st.T1[0] + S[4] * st.T1[1] + S[5] * st.T1[2];
    F dT0[3], dT1[3];
    for (int j = 0; j < 3; j++) {
        dT0[j] = two * (ga * v0[j] + gb * v1[j]);
        dT1[j] = two * (gb * v0[j] + gc * v1[j]);
    }
    F dS[3][3];
    for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++)
            dS[k][l] = ga * st.T0[k] * st.T0[l] + gb * (st.T0[k] * st.T1[l] + st.T1[k] * st.T0[l]) +
                       gc * st.T1[k] * st.T1[l];
    // T = J W
    F W[9];
    for (int i = 0; i < 9; i++) W[i] = (F)fr.R[i];
    F dJ00 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
    F dJ02 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
    F dJ11 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
    F dJ12 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
    F iz = (F)1 / st.zc, iz2 = iz * iz, iz3 = iz2 * iz;
    F fx = (F)fr.fx, fy = (F)fr.fy;
    F dxc = du * fx * iz - dJ02 * fx * iz2;
    F dyc = dv * fy * iz - dJ12 * fy * iz2;
    F dzc = -du * fx * st.xc * iz2 - dv * fy * st.yc * iz2 - dJ00 * fx * iz2 - dJ11 * fy * iz2 +
            two * (dJ02 * fx * st.xc + dJ12 * fy * st.yc) * iz3;
    if (cam) {
        const F J00 = fx * iz, J02 = -fx * st.xc * iz2, J11 = fy * iz, J12 = -fy * st.yc * iz2;
        const F m[3] = {st.mx, st.my, st.mz}, dx3[3] = {dxc, dyc, dzc};
#pragma unroll
        for (int r = 0; r < 3; r++) {
#pragma unroll
            for (int k = 0; k < 3; k++) cam[r * 3 + k] += (float)(dx3[r] * m[k]);
            cam[9 + r] += (float)dx3[r];
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            cam[c] += (float)(J00 * dT0[c]);
            cam[3 + c] += (float)(J11 * dT1[c]);
            cam[6 + c] += (float)(J02 * dT0[c] + J12 * dT1[c]);
        }
        cam[12] += (float)(du * st.xc * iz + dJ00 * iz - dJ02 * st.xc * iz2);
        cam[13] += (float)(dv * st.yc * iz + dJ11 * iz - dJ12 * st.yc * iz2);
        cam[14] += (float)du;
        cam[15] += (float)dv;
    }
    // x_c = W mu + t
    F dmx = W[0] * dxc + W[3] * dyc + W[6] * dzc;
    F dmy = W[1] * dxc + W[4] * dyc + W[7] * dzc;
    F dmz = W[2] * dxc + W[5] * dyc + W[8] * dzc;
    const F time = (F)fr.time;
    acc[0] += (float)dmx; acc[1] += (float)dmy; acc[2] += (float)dmz;
    acc[3] += (float)(time * dmx); acc[4] += (float)(time * dmy); acc[5] += (float)(time * dmz);
    // Sigma3 = M M^T, M = R diag(s): dM = 2 dSigma3 M
    const F *R = st.R;
    F s[3] = {st.s0, st.s1, st.s2};
    F G[9];
    for (int j = 0; j < 3; j++) {
        F dsj = (F)0;
        for (int k = 0; k < 3; k++) {
            F dMkj = two * s[j] * (dS[k][0] * R[j] + dS[k][1] * R[3 + j] + dS[k][2] * R[6 + j]);
            G[k * 3 + j] = dMkj * s[j];
            dsj += dMkj * R[k * 3 + j];
        }
        acc[6 + j] += (float)(dsj * s[j]);
    }
    // R(q): gradient w.r.t. the normalised quaternion, then through the normalisation
    F w = st.qw, x = st.qx, y = st.qy, z = st.qz;
    F S01 = G[1] + G[3], S02 = G[2] + G[6], S12 = G[5] + G[7];
    F A10 = G[3] - G[1], A02 = G[2] - G[6], A21 = G[7] - G[5];
    F dw = two * (z * A10 + y * A02 + x * A21);
    F dx = two * (y * S01 + z * S02 + w * A21 - two * x * (G[4] + G[8]));
    F dy = two * (x * S01 + z * S12 + w * A02 - two * y * (G[0] + G[8]));
    F dz = two * (x * S02 + y * S12 + w * A10 - two * z * (G[0] + G[4]));
    F dot = dw * w + dx * x + dy * y + dz * z;
    acc[9] += (float)((dw - w * dot) * st.inv_qn);
    acc[10] += (float)((dx - x * dot) * st.inv_qn);
    acc[11] += (float)((dy - y * dot) * st.inv_qn);
    acc[12] += (float)((dz - z * dot) * st.inv_qn);
}

// Chain rule of one pair: screen-space gradient to the raw-parameter gradients, added
// into acc[17] (mean 3, vel 3, log_scale 3, quat 4, logit 1, rgb 3).  The compositing
// backward accumulates (du, dv, da', db', dc', dlog2o, dr, dg, db) for the staged record
// (a', b', c') = -log2(e) (A/2, B, C/2) and log2 o; converted here to the conic and opacity.
// The geometric part of a pair the projection listed as ill-conditioned is left to the
// FP64 kernel.
// SH: the colour's spherical-harmonic terms.  Returns true when the pair has a colour
// gradient, then shY[k] = Y_k(d) (the coefficients' gradient is dsh[ch][k] = Y_k dc_ch,
// added by the caller); through the direction d = v / |v|, v = mu - c: dv = (I - d d^T) dd
// / |v| adds to the mean and, c = -R^T t being the camera centre, to the camera
// (dR_rj += t_r dv_j, dt_r += sum_j R_rj dv_j).  Done in FP32 for deferred pairs too.
template <bool SH = false>
__device__ __forceinline__ bool pair_backward(const PairState<float> &st, bool deferred, const DevFrame &fr,
                                              float4 g0, float4 g1, float g2, float acc[17],
                                              float *cam = nullptr, const GaussPtrs *gp = nullptr,
                                              long long gi = 0, float *shY = nullptr) {
    bool sh_live = false;
    acc[14] += g1.z;
    acc[15] += g1.w;
    acc[16] += g2;
    // d log2(o) / d logit = (1 - o) / ln 2
    acc[13] += g1.y * (1.f - st.o) * kLog2e;
    if constexpr (SH) {
        if (st.valid && (g1.z != 0.f || g1.w != 0.f || g2 != 0.f)) {
            sh_live = true;
            const GaussPtrs &g = *gp;
            const long long N = g.N;
            const int K = sh_terms(g.sh_degree);
            float d[3], rn, sk[kShMax];
            view_dir(st, fr, d, rn);
            sh_eval(g.sh_degree, d[0], d[1], d[2], shY);
            const float dc[3] = {g1.z, g1.w, g2};
#pragma unroll
            for (int k = 0; k < kShMax; k++) {
                sk[k] = 0.f;
                if (k >= K) continue;
#pragma unroll
                for (int ch = 0; ch < 3; ch++) sk[k] = fmaf(dc[ch], g.sh[((long long)ch * K + k) * N + gi], sk[k]);
            }
            float dd[3];
            sh_dir_grad(g.sh_degree, d[0], d[1], d[2], sk, dd);
            const float along = dd[0] * d[0] + dd[1] * d[1] + dd[2] * d[2];
            float dv[3];
#pragma unroll
            for (int j = 0; j < 3; j++) dv[j] = (dd[j] - d[j] * along) * rn;
            const float time = fr.time;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                acc[j] += dv[j];
                acc[3 + j] += time * dv[j];
            }
            if (cam) {
#pragma unroll
                for (int r = 0; r < 3; r++) {
#pragma unroll
                    for (int j = 0; j < 3; j++) {
                        cam[r * 3 + j] += fr.t[r] * dv[j];
                        cam[9 + r] += fr.R[r * 3 + j] * dv[j];
                    }
                }
            }
        }
    }
    if (!st.valid || deferred) return sh_live;
    const float dA = -0.5f * kLog2e * g0.z, dB = -kLog2e * g0.w, dC = -0.5f * kLog2e * g1.x;
    geometry_backward<float>(st, fr, g0.x, g0.y, dA, dB, dC, acc, cam);
    return sh_live;
}

// Adds acc into the gradient planes: rows [0, 13) (geometry) atomically when geo_atomic
// (the FP64 kernel may add into them concurrently), or left alone when skip_geo; rows
// [13, 17) (opacity, colour) atomically when atomic.
__device__ __forceinline__ void store_grad(const GradPtrs &gr, long long N, long long gi, const float acc[17],
                                           bool atomic, bool geo_atomic = false, bool skip_geo = false,
                                           bool spline = false) {
    float *mean = spline ? nullptr : gr.mean, *vel = spline ? nullptr : gr.vel;
    float *rows[17] = {mean, mean ? mean + N : nullptr, mean ? mean + 2 * N : nullptr,
                       vel, vel ? vel + N : nullptr, vel ? vel + 2 * N : nullptr,
                       gr.log_scale, gr.log_scale + N, gr.log_scale + 2 * N,
                       gr.quat, gr.quat + N, gr.quat + 2 * N, gr.quat + 3 * N,
                       gr.logit, gr.rgb, gr.rgb + N, gr.rgb + 2 * N};
#pragma unroll
    for (int k = 0; k < 17; k++) {
        if (!rows[k] || (k < 13 && skip_geo)) continue;
        if (atomic || (k < 13 && geo_atomic)) atomicAdd(rows[k] + gi, acc[k]);
        else rows[k][gi] += acc[k];
    }
}

// The time-parameterised planes of one pair's geometric gradient (rows 0-2: d mu(t), rows
// 6-8: d log_scale(t), rows 9-12: d quat(t)): dP_{lo+j} += w_j d mu for the frame's four
// spline weights, and the t, t^2, t^3 coefficients get t^p times the log-scale and
// quaternion gradients (their t^0 terms are the plain planes, written by store_grad).
__device__ __forceinline__ void store_grad_time(const GradPtrs &gr, const GaussPtrs &g, const DevFrame &fr,
                                                long long gi, const float acc[17], bool atomic) {
    const long long N = g.N, C = g.n_ctrl;
    auto add = [atomic](float *dst, float v) {
        if (atomic) atomicAdd(dst, v);
        else *dst += v;
    };
    if (gr.ctrl)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int k = 0; k < 3; k++) add(gr.ctrl + (k * C + fr.spline_lo + j) * N + gi, fr.spline_w[j] * acc[k]);
    const float t = fr.time;
    float tp = t;
#pragma unroll
    for (int p = 0; p < 3; p++, tp *= t) {
        if (gr.log_scale_t && g.log_scale_t)
#pragma unroll
            for (int k = 0; k < 3; k++) add(gr.log_scale_t + (p * 3 + k) * N + gi, tp * acc[6 + k]);
        if (gr.quat_t && g.quat_t)
#pragma unroll
            for (int k = 0; k < 4; k++) add(gr.quat_t + (p * 4 + k) * N + gi, tp * acc[9 + k]);
    }
}

// Adds the spherical-harmonic coefficient gradients dsh[ch][k] = Y[k] c[ch] of one
// Gaussian (c: one pair's colour gradient), or acc[(ch * kShMax + k) * stride] when Y is NULL.
__device__ __forceinline__ void store_grad_sh(const GradPtrs &gr, const GaussPtrs &g, long long gi, const float *Y,
                                              const float c[3], const float *acc, bool atomic, int stride = 1) {
    if (!gr.sh) return;
    const long long N = g.N;
    const int K = sh_terms(g.sh_degree);
    if (atomic) {
#pragma unroll
        for (int k = 0; k < kShMax; k++) {
            if (k >= K) break;
#pragma unroll
            for (int ch = 0; ch < 3; ch++)
                atomicAdd(gr.sh + ((long long)ch * K + k) * N + gi, Y ? Y[k] * c[ch] : acc[(ch * kShMax + k) * stride]);
        }
        return;
    }
    // read-modify-write one channel at a time in two phases: the channel's old values are
    // all loaded before any is stored, so those loads are in flight together
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float *row = gr.sh + (long long)ch * K * N + gi;
        float old[kShMax];
#pragma unroll
        for (int k = 0; k < kShMax; k++)
            if (k < K) old[k] = row[(long long)k * N];
#pragma unroll
        for (int k = 0; k < kShMax; k++)
            if (k < K) row[(long long)k * N] = old[k] + (Y ? Y[k] * c[ch] : acc[(ch * kShMax + k) * stride]);
    }
}

// Camera gradients: per block, one slot of kCamGrad floats per frame in shared memory for
// the first kCamSmemFrames frames (global atomics beyond), added to gr.cam once per block.
constexpr int kCamSmemFrames = 32;

// Transposed warp sum of 16 values: returns the sum of slot lane >> 1 (lanes 2s and 2s + 1
// hold slot s).
__device__ __forceinline__ float warp_reduce16(const float v[16], int lane) {
    const unsigned FULL = 0xffffffffu;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
    float a[8], b[4], c[2];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = (h4 ? v[i + 8] : v[i]) + __shfl_xor_sync(FULL, h4 ? v[i] : v[i + 8], 16);
#pragma unroll
    for (int i = 0; i < 4; i++) b[i] = (h3 ? a[i + 4] : a[i]) + __shfl_xor_sync(FULL, h3 ? a[i] : a[i + 4], 8);
#pragma unroll
    for (int i = 0; i < 2; i++) c[i] = (h2 ? b[i + 2] : b[i]) + __shfl_xor_sync(FULL, h2 ? b[i] : b[i + 2], 4);
    float d = (h1 ? c[1] : c[0]) + __shfl_xor_sync(FULL, h1 ? c[0] : c[1], 2);
    return d + __shfl_xor_sync(FULL, d, 1);
}

// Adds each lane's camera gradient cam (of frame f) to the block's slots: a warp whose
// lanes share one frame sums first; a warp that straddles frames adds lane by lane.
// Every lane of the warp calls it.
__device__ __forceinline__ void cam_add(const float cam[kCamGrad], int f, float (*s_cam)[kCamGrad], float *gcam) {
    const int lane = threadIdx.x & 31;
    const int f0 = __shfl_sync(0xffffffffu, f, 0);
    if (__all_sync(0xffffffffu, f == f0)) {
        const float sum = warp_reduce16(cam, lane);
        if (!(lane & 1)) {
            const int slot = lane >> 1;
            if (f0 < kCamSmemFrames) atomicAdd(&s_cam[f0][slot], sum);
            else atomicAdd(gcam + (size_t)f0 * kCamGrad + slot, sum);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kCamGrad; k++) {
            if (f < kCamSmemFrames) atomicAdd(&s_cam[f][k], cam[k]);
            else atomicAdd(gcam + (size_t)f * kCamGrad + k, cam[k]);
        }
    }
}

__device__ __forceinline__ void cam_block_init(float (*s_cam)[kCamGrad], int F) {
    for (int i = threadIdx.x; i < min(F, kCamSmemFrames) * kCamGrad; i += blockDim.x) (&s_cam[0][0])[i] = 0.f;
    __syncthreads();
}

__device__ __forceinline__ void cam_block_flush(float (*s_cam)[kCamGrad], int F, float *gcam) {
    __syncthreads();
    for (int i = threadIdx.x; i < min(F, kCamSmemFrames) * kCamGrad; i += blockDim.x) {
        const float v = (&s_cam[0][0])[i];
        if (v != 0.f) atomicAdd(gcam + i, v);
    }
}

// acc[(ch * kShMax + k) * stride] += Y[k] dc_ch (the coefficient gradients of one pair,
// summed over the frames of a shared set; K terms).
template <bool SH>
__device__ __forceinline__ void sh_accumulate(const float *Y, int K, float4 g1, float g2, float *acc, int stride) {
    if constexpr (SH) {
        const float dc[3] = {g1.z, g1.w, g2};
#pragma unroll
        for (int k = 0; k < kShMax; k++) {
            if (k >= K) break;
#pragma unroll
            for (int ch = 0; ch < 3; ch++) acc[(ch * kShMax + k) * stride] += Y[k] * dc[ch];
        }
    }
}

// mode 0: one thread per pair, each Gaussian in at most one frame (plain +=)
// mode 2: one thread per pair, overlapping sets (atomicAdd)
// A pair that binned nothing (no cell: culled, or its extent box off the frame) has a zero
// screen-space gradient and adds exactly zero, so it is skipped: each warp takes a window
// of consecutive pairs, lists the ones that binned cells (in order, in shared memory) and
// maps them 32 at a time.  When at most half the pairs binned cells (960x540 / 200k: 93k
// of 200k) a window is 64 pairs, whose live ones mostly fill one round of the warp's lanes;
// otherwise 32, one round per window as with a thread per pair.  Grid-stride over the
// windows; CAM: also the camera gradients of the frames; SPLINE: the time-parameterised form.
// Without SH or CAM the kernel keeps six blocks per SM (80 registers; uncapped, the
// time-parameterised form took 94 and ran 0.051 -> 0.071 ms at 960x540 / 200k).
constexpr int kBwdPairThreads = 128, kBwdPairWindow = 64;

template <bool CAM, bool SPLINE, bool SH>
__global__ void __launch_bounds__(kBwdPairThreads, (SH || CAM) ? 0 : 6)
    project_bwd_pairs_kernel(Work w, GaussPtrs g, GradPtrs gr, int atomic) {
    pdl_prologue();
    __shared__ float s_cam[CAM ? kCamSmemFrames : 1][kCamGrad];
    __shared__ unsigned s_live[kBwdPairThreads / 32][kBwdPairWindow];
    const int F = (int)w.L.F;
    if (CAM) cam_block_init(s_cam, F);
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const unsigned P = w.L.P;
    const unsigned win_pairs = 2u * min(w.hdr->n_drawn, P) <= P ? (unsigned)kBwdPairWindow : 32u;
    const unsigned nwin = (P + win_pairs - 1) / win_pairs;
    const unsigned nwarps = gridDim.x * (kBwdPairThreads / 32);
    for (unsigned win = blockIdx.x * (kBwdPairThreads / 32) + wq; win < nwin; win += nwarps) {
        const unsigned pa = win * win_pairs + lane, pb = pa + 32u;
        const bool la = pa < P && w.rect[pa].z != 0u;
        const bool lb = win_pairs > 32u && pb < P && w.rect[pb].z != 0u;
        const unsigned ma = __ballot_sync(0xffffffffu, la), mb = __ballot_sync(0xffffffffu, lb);
        const unsigned lt = lanemask_lt();
        if (la) s_live[wq][__popc(ma & lt)] = pa;
        if (lb) s_live[wq][__popc(ma) + __popc(mb & lt)] = pb;
        __syncwarp();
        const int n = __popc(ma) + __popc(mb);
        for (int r = 0; r < n; r += 32) {
            const bool live = r + lane < n;
            float cam[kCamGrad];
#pragma unroll
            for (int k = 0; k < kCamGrad; k++) cam[k] = 0.f;
            int f = F - 1;
            if (live) {
                const unsigned p = s_live[wq][r + lane];
                f = find_frame_by_pair(w.frames, F, p);
                const DevFrame &fr = w.frames[f];
                long long gi = fr.gauss_offset + (long long)(p - fr.pair_offset);
                PairState<float> st;
                load_and_project<float, SPLINE>(g, gi, fr, st);
                float acc[17];
#pragma unroll
                for (int k = 0; k < 17; k++) acc[k] = 0.f;
                const bool deferred = (w.rect[p].w & kRectFp64) != 0u;
                float shY[SH ? kShMax : 1];
                const float4 g1 = w.g1[p];
                const float g2 = w.g2[p];
                const bool sh_live = pair_backward<SH>(st, deferred, fr, w.g0[p], g1, g2, acc, CAM ? cam : nullptr, &g,
                                                       gi, shY);
                if (SH) {
                    // a deferred pair's mean rows hold the direction term only; the FP64 kernel
                    // adds the geometric part to the same planes concurrently
                    store_grad(gr, g.N, gi, acc, atomic != 0, deferred, false, SPLINE);
                    if (SPLINE) store_grad_time(gr, g, fr, gi, acc, atomic != 0 || deferred);
                    const float dc[3] = {g1.z, g1.w, g2};
                    if (sh_live) store_grad_sh(gr, g, gi, shY, dc, nullptr, atomic != 0);
                } else {
                    store_grad(gr, g.N, gi, acc, atomic != 0, false, deferred, SPLINE);
                    if (SPLINE && !deferred) store_grad_time(gr, g, fr, gi, acc, atomic != 0);
                }
            }
            if (CAM) {  // an idle lane (zero gradient) takes lane 0's frame
                const int fl = __shfl_sync(0xffffffffu, f, 0);
                cam_add(cam, live ? f : fl, s_cam, gr.cam);
            }
        }
        __syncwarp();  // the window's list is read before the next one overwrites it
    }
    if (CAM) cam_block_flush(s_cam, F, gr.cam);
}

// mode 1: one shared Gaussian set; one thread per Gaussian sums over all frames (grid-stride).
// SPLINE: the time-parameterised form (g.n_ctrl > 0).  The kernel is bound by memory
// latency at four blocks per SM, so each frame's screen-space gradient and flags are loaded
// one frame ahead, and (without spline or SH) the frame-independent shape is loaded and
// computed once per Gaussian, as the forward does (8 x 1920x1080 / 1M: 0.34 -> 0.23 ms).
// The SH variants cap their registers at three blocks per SM; the others take no minimum
// (a minimum of one block made the compiler's code 30 % slower on 1M-Gaussian sets).
template <bool CAM, bool SPLINE, bool SH>
__global__ void __launch_bounds__(128, SH ? 3 : 0) project_bwd_shared_kernel(Work w, GaussPtrs g, GradPtrs gr) {
    pdl_prologue();
    __shared__ float s_cam[CAM ? kCamSmemFrames : 1][kCamGrad];
    // each thread's coefficient-gradient sums over the frames, a column of its own
    __shared__ float s_acc_sh[SH ? 3 * kShMax : 1][SH ? 128 : 1];
    float *acc_sh = &s_acc_sh[0][SH ? threadIdx.x : 0];
    const int Ksh = SH ? sh_terms(g.sh_degree) : 0;
    const int F = (int)w.L.F;
    if (CAM) cam_block_init(s_cam, F);
    const DevFrame &f0 = w.frames[0];
    for (unsigned base = blockIdx.x * blockDim.x; base < f0.gauss_count; base += gridDim.x * blockDim.x) {
        const unsigned j = base + threadIdx.x;
        const bool in = j < f0.gauss_count;
        const long long gi = f0.gauss_offset + j;
        float acc[17];
#pragma unroll
        for (int k = 0; k < 17; k++) acc[k] = 0.f;
        if (SH)
            for (int k = 0; k < 3 * kShMax; k++) acc_sh[k * 128] = 0.f;
        bool any_deferred = false;
        // frame f + 1's screen-space gradient and flags load while frame f is mapped
        float4 pg0 = make_float4(0.f, 0.f, 0.f, 0.f), pg1 = pg0;
        float pg2 = 0.f;
        unsigned pw = 0u;
        auto fetch = [&](int f) {
            const unsigned p = w.frames[f].pair_offset + j;
            pw = w.rect[p].w;
            pg0 = w.g0[p];
            pg1 = w.g1[p];
            pg2 = w.g2[p];
        };
        if (in && F > 0) fetch(0);
        PairState<float> st;
        float m0[3] = {0.f, 0.f, 0.f}, v0[3] = {0.f, 0.f, 0.f};
        // without a spline (and without SH, whose registers do not allow it) the shape does
        // not depend on the frame: loaded and computed once per Gaussian
        constexpr bool kHoist = !SPLINE && !SH;
        if (kHoist && in) {
            const long long N = g.N;
            for (int k = 0; k < 3; k++) {
                m0[k] = g.mean[k * N + gi];
                if (g.vel) v0[k] = g.vel[k * N + gi];
            }
            load_shape<float, false>(g, gi, f0, st);
        }
        for (int f = 0; f < F; f++) {
            float cam[kCamGrad];
#pragma unroll
            for (int k = 0; k < kCamGrad; k++) cam[k] = 0.f;
            const float4 cg0 = pg0, cg1 = pg1;
            const float cg2 = pg2;
            const unsigned cw = pw;
            if (in && f + 1 < F) fetch(f + 1);
            if (in) {
                const DevFrame &fr = w.frames[f];
                if (kHoist) {
                    if (g.vel) {
                        st.mx = fmaf(fr.time, v0[0], m0[0]);
                        st.my = fmaf(fr.time, v0[1], m0[1]);
                        st.mz = fmaf(fr.time, v0[2], m0[2]);
                    } else {
                        st.mx = m0[0]; st.my = m0[1]; st.mz = m0[2];
                    }
                    project_camera<float>(fr, st);
                } else {
                    load_and_project<float, SPLINE>(g, gi, fr, st);
                }
                const bool deferred = (cw & kRectFp64) != 0u;
                any_deferred |= deferred;
                if (SPLINE) {
                    // the frame's spline weights and powers of t differ: map this frame's
                    // geometric gradient now (the FP64 kernel adds atomically to the same
                    // planes when any frame of this Gaussian was deferred)
                    float accf[17];
#pragma unroll
                    for (int k = 0; k < 17; k++) accf[k] = 0.f;
                    float shY[SH ? kShMax : 1];
                    if (pair_backward<SH>(st, deferred, fr, cg0, cg1, cg2, accf, CAM ? cam : nullptr, &g, gi, shY))
                        sh_accumulate<SH>(shY, Ksh, cg1, cg2, acc_sh, 128);
                    if (!deferred || SH) store_grad_time(gr, g, fr, gi, accf, true);
#pragma unroll
                    for (int k = 6; k < 17; k++) acc[k] += accf[k];
                } else {
                    float shY[SH ? kShMax : 1];
                    if (pair_backward<SH>(st, deferred, fr, cg0, cg1, cg2, acc, CAM ? cam : nullptr, &g, gi, shY))
                        sh_accumulate<SH>(shY, Ksh, cg1, cg2, acc_sh, 128);
                }
            }
            if (CAM) cam_add(cam, f, s_cam, gr.cam);
        }
        if (in) store_grad(gr, g.N, gi, acc, false, any_deferred, false, SPLINE);
        if (SH && in) store_grad_sh(gr, g, gi, nullptr, nullptr, acc_sh, false, 128);
    }
    if (CAM) cam_block_flush(s_cam, F, gr.cam);
}

// FP64 geometric chain rule of the pairs the projection listed as ill-conditioned; atomic
// because several frames of a shared set may list the same Gaussian, and because the FP32
// pass runs concurrently.  The list lives until the next forward's setup clears it, so a
// backward can be repeated.
__global__ void __launch_bounds__(128) project_bwd_fp64_kernel(Work w, GaussPtrs g, GradPtrs gr) {
    pdl_prologue();
    const unsigned n = min(w.hdr->fp64_count, w.L.P);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned p = min(w.fp64_list[i], w.L.P - 1u);
        const DevFrame &fr = w.frames[find_frame_by_pair(w.frames, (int)w.L.F, p)];
        const long long gi = fr.gauss_offset + (long long)(p - fr.pair_offset);
        PairState<double> sd;
        if (g.n_ctrl > 0) load_and_project<double, true>(g, gi, fr, sd);
        else load_and_project<double, false>(g, gi, fr, sd);
        if (!sd.valid) continue;
        const float4 g0 = w.g0[p], g1 = w.g1[p];
        float acc[17];
#pragma unroll
        for (int k = 0; k < 17; k++) acc[k] = 0.f;
        float cam[kCamGrad];
#pragma unroll
        for (int k = 0; k < kCamGrad; k++) cam[k] = 0.f;
        geometry_backward<double>(sd, fr, (double)g0.x, (double)g0.y, -0.5 * (double)kLog2e * g0.z,
                                  -(double)kLog2e * g0.w, -0.5 * (double)kLog2e * g1.x, acc,
                                  gr.cam ? cam : nullptr);
        acc[13] = acc[14] = acc[15] = acc[16] = 0.f;  // colour and opacity were done in FP32
        store_grad(gr, g.N, gi, acc, true, false, false, g.n_ctrl > 0);
        if (g.n_ctrl > 0) store_grad_time(gr, g, fr, gi, acc, true);
        if (gr.cam) {
            const int f = find_frame_by_pair(w.frames, (int)w.L.F, p);
            for (int k = 0; k < kCamGrad; k++) atomicAdd(gr.cam + (size_t)f * kCamGrad + k, cam[k]);
        }
    }
}

}  // namespace

int tile_sort_passes(const Work &w) { return std::max(1, (w.L.tile_bits + 7) / 8); }

cudaError_t launch_project_fwd(const Work &w, const GaussPtrs &g, int tile_w, int tile_h, bool shared_set,
                               int num_sms, cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    int lw = __builtin_ctz(tile_w), lh = __builtin_ctz(tile_h);
    if (shared_set && w.L.F > 1 && g.n_ctrl == 0 && g.sh_degree == 0) {
        const unsigned n = w.L.P / w.L.F;
        const unsigned blocks = std::max(1u, std::min((n + 255u) / 256u, (unsigned)num_sms * 4u));
        launch_pdl(project_fwd_shared_kernel, blocks, 256, 0, s, w, g, lw, lh, tile_sort_passes(w));
        return cudaGetLastError();
    }
    // four blocks per SM: fewer per-block histogram flushes (measured at 960x540 / 200k: 24.7 -> 20.7 us;
    // unchanged on 8 x 1920x1080 / 1M)
    unsigned blocks = std::min((w.L.P + 255u) / 256u, (unsigned)num_sms * 4u);
    const int tp = tile_sort_passes(w);
    const bool spline = g.n_ctrl > 0, sh = g.sh_degree > 0;
    if (spline && sh) launch_pdl(project_fwd_kernel<true, true>, blocks, 256, 0, s, w, g, lw, lh, tp);
    else if (spline) launch_pdl(project_fwd_kernel<true, false>, blocks, 256, 0, s, w, g, lw, lh, tp);
    else if (sh) launch_pdl(project_fwd_kernel<false, true>, blocks, 256, 0, s, w, g, lw, lh, tp);
    else launch_pdl(project_fwd_kernel<false, false>, blocks, 256, 0, s, w, g, lw, lh, tp);
    return cudaGetLastError();
}

cudaError_t launch_bin_from_screen(const Work &w, long long n, const float *u, const float *v, const float *sxx,
                                   const float *sxy, const float *syy, const float *tau, const float *depth,
                                   const uint8_t *valid, int tile_w, int tile_h, int32_t *counts, int num_sms,
                                   cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int lw = __builtin_ctz(tile_w), lh = __builtin_ctz(tile_h);
    unsigned blocks = std::min((unsigned)((n + 255) / 256), (unsigned)num_sms * 8u);
    launch_pdl(bin_from_screen_kernel, blocks, 256, 0, s, w, n, u, v, sxx, sxy, syy, tau, depth, valid, lw, lh,
                                                   tile_sort_passes(w), counts);
    return cudaGetLastError();
}

// Calls fn(CAM, SPLINE, SH) with the three flags as std::integral_constant<bool, .>.
template <class Fn>
void dispatch_bwd(bool cam, bool spline, bool sh, Fn &&fn) {
    auto with_sh = [&](auto C, auto S) {
        if (sh) fn(C, S, std::true_type{});
        else fn(C, S, std::false_type{});
    };
    auto with_spline = [&](auto C) {
        if (spline) with_sh(C, std::true_type{});
        else with_sh(C, std::false_type{});
    };
    if (cam) with_spline(std::true_type{});
    else with_spline(std::false_type{});
}

cudaError_t launch_project_bwd(const Work &w, const GaussPtrs &g, const GradPtrs &gr, int mode, int num_sms,
                               cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    if (mode == 1) {
        // all frames share one set; its size is the first frame's count
        unsigned n = w.L.P / w.L.F;
        unsigned blocks = std::min((n + 127) / 128, (unsigned)num_sms * 16u);
        dispatch_bwd(gr.cam != nullptr, g.n_ctrl > 0, g.sh_degree > 0, [&](auto C, auto S, auto H) {
            launch_pdl(project_bwd_shared_kernel<decltype(C)::value, decltype(S)::value, decltype(H)::value>, blocks,
                       128, 0, s, w, g, gr);
        });
    } else {
        // one 32-pair window per warp (the 64-pair windows leave half the warps without one)
        unsigned blocks = std::min((w.L.P + kBwdPairThreads - 1) / kBwdPairThreads, (unsigned)num_sms * 16u);
        const int at = mode == 2 ? 1 : 0;
        dispatch_bwd(gr.cam != nullptr, g.n_ctrl > 0, g.sh_degree > 0, [&](auto C, auto S, auto H) {
            launch_pdl(project_bwd_pairs_kernel<decltype(C)::value, decltype(S)::value, decltype(H)::value>, blocks,
                       kBwdPairThreads, 0, s, w, g, gr, at);
        });
    }
    return cudaGetLastError();
}

cudaError_t launch_project_bwd_fp64(const Work &w, const GaussPtrs &g, const GradPtrs &gr, int num_sms,
                                    cudaStream_t s) {
    if (w.L.P == 0) return cudaSuccess;
    launch_pdl(project_bwd_fp64_kernel, num_sms, 128, 0, s, w, g, gr);
    return cudaGetLastError();
}

}  // namespace gvk
