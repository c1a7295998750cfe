// cvx_scan_lanes.cu -- the line scan of the damage energy with one line per
// lane: the FP32 screening pass of the per-point convexification (Eqs. 4.3,
// 4.4 restated per point, Algorithm 1 read at t = 0), without an exact FP32
// hull.
//
// A warp takes a work item (a node and up to 256 of its directions) and each
// lane samples its own line, two samples per paired FP32 instruction, without
// storing it.  For the hull at t = 0 of the left set {x < 0} and the right set
// {x > 0} of the samples (x = m - m0) the pass at a slope s yields
//   e_L = min over the left of (v - s x),  e_R = min over the right,
// and their minimisers a < 0 < b.  For any s, min(e_L, e_R) is a lower bound
// of the hull value at 0 (an affine minorant read at 0), and the chord of
// (a, b) at 0, a convex combination of e_L and e_R, is an upper bound.  The
// first pass takes the line's tangent slope at t = 0; later passes take the
// slope of the last pair (the supporting-slope iteration of a bridge search),
// which converges to the bridge, where both bounds meet.  A line is dropped
// as soon as its lower bound exceeds m + eps(m), m = min(W(F), the smallest
// upper bound of any line of the node) -- the node's smallest upper bound is
// shared by all items of the node through one word in global memory -- and
// only lines that are still candidates take further passes: many of them
// lane by lane, a few of them with the whole warp on one line.  No decision
// is taken here: the item's best directions by lower bound go to k_select,
// and the node is decided on FP64 samples by k_refine / k_commit, exactly as
// after the warp-per-line scan.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdlib.h>
#include <string.h>

#include "cvx_line.cuh"

namespace cvx {

namespace {

constexpr int kLaneWarps = 8;
constexpr int kLaneRounds = 4;  // passes per line at most
// fewer live lines than this in a later pass: the whole warp on each line
// (64 samples per lane and a warp reduction) instead of one line per lane
#ifndef CVX_LANE_COOP
#define CVX_LANE_COOP 6
#endif
constexpr int kLaneCoop = CVX_LANE_COOP;

constexpr int kConv = 1 << 28;    // bounds settled (pair repeated or within eps/4): no further pass
constexpr int kDrop = 1 << 29;    // lower bound above the node's reference value
constexpr int kNoPair = 1 << 30;  // a side without a finite sample: no bridge pair
constexpr int kCert = 1 << 27;    // certified: no sample lies on or below the tangent line at the
                                  // centre, so the line cannot split the node
constexpr int kTan = 1 << 26;     // the first pass took the line's tangent slope

// One line of a warp's item.
struct LaneState {
    float q_lo, q_hi;  // bounds of the hull value at 0 of the left and right sets
    float s;           // slope of the next pass (chord slope of the last pair)
    int ab;            // a (bits 0-11), b (bits 12-23) sample indices, kConv, kDrop
};

// Node constants of a warp's item.
struct LaneNode {
    NodeLine nl;
    float C, sa, cb, w0;  // sample shift, tangent-slope constants, FP32 centre sample
    // centre expansion of the line function for the no-split certificate:
    // d0 = d(0), B1p = B1 + 2 B2 lg0 (lg0 = log2 J0), gp = dv/dd at d0,
    // k1e = K1 2^{-d0} (d0 > 0, else 0), invJ0 = 1 / J0
    float d0, B1p, gp, k1e, invJ0;
    float d0abs;  // |A0| + |lg0| (|B1| + B2 |lg0|): magnitude of the terms of d0
    int e;        // the node's window exponent (line spacing h 2^e)
};

struct SideMin {
    float eL, eR;    // minima of v - s x over the left and the right samples
    int kL, kR;      // pair index of each minimum, -1 if the side has no finite sample
    float eLf, eRf;  // the same minima over the far samples only (outside the near
                     // region [2 kf - m0, 2 kn], see line_pass)
};

__device__ __forceinline__ void side_update(f32x2 B, int k, float &e, int &kk) {
    float b0, b1;
    upk2(B, b0, b1);
    const float m = fminf(b0, b1);
    if (m < e) {
        e = m;
        kk = k;
    }
}

// Pass over a line at slope s = -ns.  Pairs (x, x + 1): left x = 2k - m0,
// right x = 2k + 1, for k = k0, k0 + kstep, ... < m0 / 2; with m0 odd the
// lane with k0 = 0 also takes the sample next to the centre on the left
// (x = -1) and the last one on the right (x = m0) as pair m0 / 2.  The
// samples are those of sample_w (each half of a paired instruction rounds
// as the scalar one), at t = fl(x h).  Left pairs k >= kf and right pairs
// k < kn form the near region (x in [2 kf - m0, -1] and [1, 2 kn]); the far
// minima leave it out.
__device__ __forceinline__ SideMin line_pass(const NHPair &c, f32x2 H, float ns, int m0, int k0,
                                             int kstep, int kf = 0, int kn = 0) {
    SideMin r;
    r.eL = r.eR = INFINITY;
    r.kL = r.kR = -1;
    const int np = m0 >> 1;
    const f32x2 NS = pk2(ns, ns);
    const float st = 2.0f * (float)kstep;
    const f32x2 STEP = pk2(st, st);
    f32x2 X = pk2((float)(2 * k0 - m0), (float)(2 * k0 - m0 + 1));
    int k = k0;
#pragma unroll 2
    for (; k < kf; k += kstep) {
        side_update(fma2(NS, X, sample_nh2(c, mul2(X, H))), k, r.eL, r.kL);
        X = add2(X, STEP);
    }
    r.eLf = r.eL;
#pragma unroll 2
    for (; k < np; k += kstep) {
        side_update(fma2(NS, X, sample_nh2(c, mul2(X, H))), k, r.eL, r.kL);
        X = add2(X, STEP);
    }
    X = pk2((float)(2 * k0 + 1), (float)(2 * k0 + 2));
    k = k0;
#pragma unroll 2
    for (; k < kn; k += kstep) {
        side_update(fma2(NS, X, sample_nh2(c, mul2(X, H))), k, r.eR, r.kR);
        X = add2(X, STEP);
    }
    float ef = INFINITY;
    int kk = -1;
#pragma unroll 2
    for (; k < np; k += kstep) {
        side_update(fma2(NS, X, sample_nh2(c, mul2(X, H))), k, ef, kk);
        X = add2(X, STEP);
    }
    if ((m0 & 1) && k0 == 0) {
        X = pk2(-1.0f, -1.0f);
        side_update(fma2(NS, X, sample_nh2(c, mul2(X, H))), np, r.eL, r.kL);
        X = pk2((float)m0, (float)m0);
        side_update(fma2(NS, X, sample_nh2(c, mul2(X, H))), np, ef, kk);
    }
    r.eRf = ef;
    if (ef < r.eR) {
        r.eR = ef;
        r.kR = kk;
    }
    return r;
}

// Certificate that a line cannot split its node: with s0 = the line's
// tangent slope at the centre (the slope of the first pass), every sample
// m != m0 satisfies v(t_m) - v(0) - s0 x_m > 0 for the FP64 line function,
// i.e. the tangent line at the centre supports the whole line strictly, so
// the centre is a strict vertex of the lower hull (Algorithm 1).
//  - far samples (outside the near region): from the pass's far minimum at
//    s0 less its rounding bound and the FP32 sample error bound eps, against
//    the centre sample plus eps;
//  - near samples (x in [xl, -1] and [1, xr]): the second-order remainder
//    computed from the centre expansion, so that its error scales with t
//    instead of with |v|: with u = t cof F:R / J0, ell = log2(1 + u),
//      d(t) - d0 - d'(0) t = A2 t^2 + B1p (ell - u / ln 2) + B2 ell^2 = Dd,
//    log1p(u) - u from the series of 2 atanh(u / (2 + u)), and for d0 > 0
//      v(t) - v(0) - v'(0) t = gp Dd - K1 2^{-d0} (e^{-y} - 1 + y),
//    y = (d - d0) ln 2 (series), for d0 <= 0 it is (1 + K2) Dd.  A sample is
//    certified when that value exceeds 16 u ((S1 + |s0|) |x| + (1 + |d0|_abs)
//    S2 x^2), S1 and S2 the magnitudes of the first- and second-order terms
//    per sample, built from the absolute sums sum |F_i R_i| and
//    sum |cof F_i R_i| (so that a cancellation in F:R or cof F:R does not hide
//    the rounding of its terms): the rounding of the FP32 line constants, of t
//    and of the FP32 arithmetic, all first- or second-order in t.  Samples
//    where d changes sign, or |u| or |y| leave the series' range, are not
//    certified.
__device__ bool flat_certificate(const LaneNode &N, const DirLine &dl, float4 d32, float h, int m0,
                                 int xl, int xr, float s0, float eFar, float kap) {
    const float C = N.C, w0 = N.w0;
    const float kLn2f = 0.693147180559945309f, kInvLn2 = 1.442695040888963407f;
    // far samples: every far m has b_m = v_m - s0 x_m >= qf, and its sample
    // error is at most kEps32 max(kappa', |b_m| + |s0| m0 + C), so the FP64
    // value exceeds the tangent line at the centre if qf less that bound at
    // b_m = qf (the worst case) exceeds the centre sample plus its bound
    if (eFar < INFINITY) {
        const float qf = eFar - 3.2f * kU32 * (fabsf(eFar) + 2.0f * fabsf(s0) * (float)m0) - 1e-30f;
        const float ef = kEps32 * fmaxf(kap, fabsf(qf) + fabsf(s0) * (float)m0 + C);
        if (!(qf - ef > w0 + eps32_at(w0, kap, C))) return false;
    }
    const float rJ = dl.cJ * N.invJ0;
    const float xm = (float)max(-xl, xr);
    if (!(fabsf(rJ) * xm * h <= 0.25f)) return false;
    const float dprime = dl.A1 + N.B1p * rJ * kInvLn2;
    if (!(fabsf(dprime) * xm * h * kLn2f <= 0.5f)) return false;
    const float A2 = dl.A2, B2 = N.nl.B2, B1p = N.B1p, gp = N.gp, k1e = N.k1e, d0 = N.d0;
    // absolute sums of the terms of F:R and cof F:R
    const float R0 = d32.x * d32.z, R1 = d32.x * d32.w, R2 = d32.y * d32.z, R3 = d32.y * d32.w;
    const float cA = fabsf(N.nl.F[0] * R0) + fabsf(N.nl.F[1] * R1) + fabsf(N.nl.F[2] * R2) +
                     fabsf(N.nl.F[3] * R3);
    const float cJA = fabsf(N.nl.cof[0] * R0) + fabsf(N.nl.cof[1] * R1) +
                      fabsf(N.nl.cof[2] * R2) + fabsf(N.nl.cof[3] * R3);
    const float rJa = cJA * fabsf(N.invJ0);
    const float dpa = N.nl.mu * cA + fabsf(B1p) * rJa * kInvLn2;
    const float S1 = h * gp * dpa;
    const float S2 = h * h * (gp * (A2 + fabsf(B1p) * rJa * rJa * 0.5f * kInvLn2 +
                                    B2 * rJa * rJa * kInvLn2 * kInvLn2) +
                              k1e * kLn2f * kLn2f * dpa * dpa * 0.5f);
    const float c1 = 16.0f * kU32 * (S1 + fabsf(s0));
    const float c2 = 16.0f * kU32 * (1.0f + N.d0abs) * S2;
    bool ok = true;
    for (int x = xl; x <= xr && ok; ++x) {
        if (x == 0) continue;
        const float t = __fmul_rn((float)x, h);
        const float u = rJ * t;
        const float z = __fdividef(u, 2.0f + u);
        const float z2 = z * z;
        // log1p(u) - u = -u z + 2 z^3 (1/3 + z^2/5 + z^4/7 + z^6/9 + ...)
        const float lm =
            __fmaf_rn(2.0f * z * z2,
                      __fmaf_rn(z2, __fmaf_rn(z2, __fmaf_rn(z2, 1.0f / 9.0f, 1.0f / 7.0f), 0.2f),
                                1.0f / 3.0f),
                      -u * z);
        const float ell = (u + lm) * kInvLn2;
        const float Dd = __fmaf_rn(A2 * t, t, __fmaf_rn(B1p, lm * kInvLn2, B2 * ell * ell));
        const float dd = __fmaf_rn(dprime, t, Dd);
        float rem;
        if (d0 > 0.0f) {
            if (!(d0 + dd > 0.0f)) return false;
            const float y = dd * kLn2f;
            // e^{-y} - 1 + y = y^2 (1/2 - y/6 + y^2/24 - y^3/120 + y^4/720 - y^5/5040)
            const float ph =
                y * y *
                __fmaf_rn(-y,
                          __fmaf_rn(-y,
                                    __fmaf_rn(-y, __fmaf_rn(-y, __fmaf_rn(y, 1.0f / 5040.0f,
                                                                          -1.0f / 720.0f),
                                                            1.0f / 120.0f),
                                              -1.0f / 24.0f),
                                    1.0f / 6.0f),
                          0.5f);
            rem = __fmaf_rn(gp, Dd, -k1e * ph);
        } else {
            if (!(d0 + dd <= 0.0f)) return false;
            rem = gp * Dd;
        }
        const float ax = fabsf((float)x);
        ok = rem > ax * __fmaf_rn(c2, ax, c1);
    }
    return ok;
}

// Warp-wide minimum of one side over the lanes' partial passes.
__device__ __forceinline__ void warp_side(float &e, int &k) {
    const float m = warp_min_f32(e);
    const unsigned bal = __ballot_sync(kFull, k >= 0 && e == m);
    k = bal ? __shfl_sync(kFull, k, __ffs(bal) - 1) : -1;
    e = m;
}

// The sample of a side's minimum pair: index m and FP32 value v, recomputed
// bit for bit (the pass kept fminf(b0, b1): b1 if b1 < b0 or b0 is NaN).
__device__ __forceinline__ void side_pick(const NHPair &c, f32x2 H, float ns, int m0, int k,
                                          bool left, int &m, float &v) {
    const int np = m0 >> 1;
    float x0, x1;
    if (k < np) {
        x0 = left ? (float)(2 * k - m0) : (float)(2 * k + 1);
        x1 = x0 + 1.0f;
    } else {
        x0 = x1 = left ? -1.0f : (float)m0;
    }
    const f32x2 X = pk2(x0, x1);
    const f32x2 V = sample_nh2(c, mul2(X, H));
    float v0, v1, b0, b1;
    upk2(V, v0, v1);
    upk2(fma2(pk2(ns, ns), X, V), b0, b1);
    const bool second = b1 < b0 || b0 != b0;
    m = (int)(second ? x1 : x0) + m0;
    v = second ? v1 : v0;
}

struct Bounds {
    float q_lo, q_hi, s;
    int a, b;
};

// Bounds of a pass at slope s: q_lo = min(e_L, e_R) less the rounding bound
// of the computed v - s x, q_hi = the chord of the minimisers at 0 plus its
// rounding bound, and the chord's slope for the next pass.  A side without a
// finite sample leaves the centre alone on its hull: no bound below it.
__device__ __forceinline__ Bounds pass_bounds(const NHPair &c, f32x2 H, float s, int m0,
                                              const SideMin &r) {
    Bounds o;
    if (r.kL < 0 || r.kR < 0) {
        o.q_lo = o.q_hi = INFINITY;
        o.s = s;
        o.a = o.b = -1;
        return o;
    }
    float va, vb;
    side_pick(c, H, -s, m0, r.kL, true, o.a, va);
    side_pick(c, H, -s, m0, r.kR, false, o.b, vb);
    const float e = fminf(r.eL, r.eR);
    const float xa = (float)(o.a - m0), xb = (float)(o.b - m0);
    const float chord = va + (vb - va) * __fdiv_rn(-xa, xb - xa);
    o.q_hi = chord + 4.0f * kU32 * (fabsf(va) + fabsf(vb) + fabsf(chord)) + 1e-30f;
    o.q_lo = fminf(e - 3.2f * kU32 * (fabsf(e) + 2.0f * fabsf(s) * (float)m0) - 1e-30f, o.q_hi);
    o.s = __fdividef(vb - va, xb - xa);
    return o;
}

__device__ __forceinline__ int enc_ab(int a, int b) {
    return a < 0 ? (kConv | kNoPair) : (a | (b << 12));
}

__device__ __forceinline__ float key2f(int k) { return __int_as_float(f2key(__int_as_float(k))); }

// Line constants of one direction in register pairs.
__device__ __forceinline__ NHPair line_pair(const NHPair &node, const DirLine &dl) {
    NHPair c = node;
    c.A1 = pk2(dl.A1, dl.A1);
    c.A2 = pk2(dl.A2, dl.A2);
    c.CJ = pk2(dl.cJ, dl.cJ);
    return c;
}

// Global direction index of entry j of a node's proposal window (row-major
// over (da, db) in [-w, w]^2 around the centre cell, indices wrapping).
__device__ __forceinline__ int lane_window_dir(const ProbDesc &pd, int2 c, int j) {
    const int s = 2 * pd.window + 1;
    int i = (c.x + j / s - pd.window) % pd.Na;
    int k = (c.y + j % s - pd.window) % pd.Nb;
    if (i < 0) i += pd.Na;
    if (k < 0) k += pd.Nb;
    return i * pd.Nb + k;
}

}  // namespace

#ifndef CVX_LANE_MIN_BLOCKS
#define CVX_LANE_MIN_BLOCKS 4  // CTAs of 256 threads per SM the registers target
#endif

__global__ void __launch_bounds__(32 * kLaneWarps, CVX_LANE_MIN_BLOCKS)
    k_scan_lanes(const Pipe P, int level) {
    __shared__ LaneState s_st[kLaneWarps][kLaneItemMax];
    __shared__ float s_ef[kLaneWarps][kLaneItemMax];  // far minimum of the first pass
    __shared__ unsigned short s_live[kLaneWarps][kLaneItemMax];
    __shared__ LaneNode s_nd[kLaneWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool win = P.pass == PASS_WINDOW;
    const int n_nodes = P.cnt[level];
    const long long n_items = (long long)n_nodes * P.C;
    const int32_t *qp = P.qp[level], *qh = P.qh[level];
    LaneState *st = s_st[warp];
    float *efl = s_ef[warp];
    unsigned short *live = s_live[warp];
    LaneNode &N = s_nd[warp];
    unsigned long long n_valid = 0;
    unsigned n_lines = 0, n_drop = 0, n_flat = 0, n_extra = 0, n_cert = 0;

    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(P.item_ctr + level, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        const int qi = (int)(item / P.C), ch = (int)(item % P.C);
        const int p = qp[qi];
        const ProbDesc &pd = P.probs[P.pid[p]];
        const int chunks = win ? pd.wchunks : pd.chunks;
        if (ch >= chunks) continue;
        if (lane == 0) {
            const cvx_node *nd = node_ptr(pd, p, qh[qi]);
            const double F[4] = {nd->F[0], nd->F[1], nd->F[2], nd->F[3]};
            const double beta = pd.beta[p - pd.point_off];
            N.nl = make_node_line(F, beta, pd.mat);
            N.C = (float)line_shift(pd.mat, beta);
            N.e = nd->window_exp;
            center_slope_consts(N.nl, scaled_line(pd.line, N.e).h64, N.sa, N.cb);
            DirLine d0;
            d0.A1 = d0.A2 = d0.cJ = 0.0f;
            d0.J0 = N.nl.J0;
            N.w0 = sample_w<CVX_ENERGY_NH_DAMAGE>(N.nl, d0, 0.0f);
            {
                const double J0 = N.nl.J0, lg0 = J0 > 0.0 ? log2(J0) : 0.0;
                const double dc = (double)N.nl.A0 + lg0 * ((double)N.nl.B1 + (double)N.nl.B2 * lg0);
                const double e2 = exp2(-dc);
                N.d0 = (float)dc;
                N.B1p = (float)((double)N.nl.B1 + 2.0 * (double)N.nl.B2 * lg0);
                N.gp = (float)(dc < 0.0 ? 1.0 + (double)N.nl.K2 : 1.0 + (double)N.nl.K1 * kLn2d * e2);
                N.k1e = dc > 0.0 ? (float)((double)N.nl.K1 * e2) : 0.0f;
                N.invJ0 = J0 > 0.0 ? (float)(1.0 / J0) : 0.0f;
                N.d0abs = (float)(fabs((double)N.nl.A0) +
                                  fabs(lg0) * (fabs((double)N.nl.B1) + (double)N.nl.B2 * fabs(lg0)));
            }
        }
        __syncwarp();
        const LineSpec ln = scaled_line(pd.line, N.e);
        const int m0 = ln.m0;
        const int D = win ? pd.wD : pd.D, dpi = win ? pd.wdpi : pd.dpi, doff = pd.dir_off;
        const int d0 = ch * dpi, nl_item = min(D, d0 + dpi) - d0;
        const int2 cen = win ? P.center[qi] : make_int2(0, 0);
        const float kap = pd.kappa_f, C = N.C, w0 = N.w0, sa = N.sa, cb = N.cb;
        const float epsc = eps32_at(w0, kap, C);
        // global direction of line j of block blk of this item
        auto gdir = [&](int blk, int j) {
            return win ? lane_window_dir(pd, cen, d0 + blk + j) : d0 + blk + j;
        };
        const f32x2 H = pk2(ln.h32, ln.h32);
        NHPair node = nh_pair_node(N.nl);
        node.J0 = pk2(N.nl.J0, N.nl.J0);
        // the item's best directions so far: lane i < kItemTop holds entry i
        float tq = INFINITY;
        int td = INT_MAX, tab = -1;
        float drop = INFINITY, qhi = INFINITY;
        float U = INFINITY;  // smallest upper bound of the node seen by this warp

        for (int blk = 0; blk < nl_item; blk += kLaneItemMax) {
            const int nb = min(kLaneItemMax, nl_item - blk);
            // ---- first pass: lane l takes the contiguous run of lines
            // j = l P + p, so each line after the first starts from its
            // neighbour's bridge slope when that neighbour splits clearly
            // (else from its own tangent slope at t = 0)
            const int Pn = (nb + 31) >> 5;
            float umin = INFINITY, s_prev = 0.0f;
            bool warm = false;
            // near region of the no-split certificate: |x| up to Xn samples
            // (even, at most 0.04 in t and 32 samples)
            const int np = m0 >> 1;
            const int Xn = min(min(32, (int)(0.04f / ln.h32)), m0) & ~1;
            const int kf = max(0, np - Xn / 2), kn = min(np, Xn / 2);
            for (int q = 0; q < Pn; ++q) {
                const int j = lane * Pn + q;
                if (j >= nb) break;
                const int gd = gdir(blk, j);
                const DirLine dl = make_dir_line<CVX_ENERGY_NH_DAMAGE>(N.nl, P.dir32[doff + gd]);
                const NHPair c = line_pair(node, dl);
                const bool tangent = !warm;
                const float s0 = warm ? s_prev : sa * __fmaf_rn(cb, dl.cJ, dl.A1);
                const SideMin sm = line_pass(c, H, -s0, m0, 0, 1, kf, kn);
                const Bounds b = pass_bounds(c, H, s0, m0, sm);
                LaneState t;
                t.q_lo = b.q_lo;
                t.q_hi = b.q_hi;
                t.s = b.s;
                t.ab = enc_ab(b.a, b.b);
                if (b.q_hi - b.q_lo <= 0.25f * eps32_at(b.q_lo, kap, C)) t.ab |= kConv;
                if (tangent) t.ab |= kTan;
                st[j] = t;
                efl[j] = fminf(sm.eLf, sm.eRf);
                umin = fminf(umin, b.q_hi);
                warm = b.a >= 0 && b.q_hi < w0 - epsc;
                s_prev = b.s;
                n_valid += valid_samples(dl, ln, CVX_ENERGY_NH_DAMAGE);
            }
            n_lines += nb;
            // the node's smallest upper bound, shared with its other items
            {
                const float um = warp_min_f32(umin);
                int old = 0;
                if (lane == 0) old = atomicMin(P.node_u + qi, f2key(um));
                U = fminf(U, fminf(um, key2f(__shfl_sync(kFull, old, 0))));
            }
            __syncwarp();

            // ---- further passes over the lines that are still candidates
            for (int r = 1; r < kLaneRounds; ++r) {
                const float mref = fminf(w0, U);
                const float thr = mref + eps32_at(mref, kap, C);
                int n_live = 0;
                for (int base = 0; base < nb; base += 32) {
                    const int j = base + lane;
                    bool lv = false;
                    if (j < nb && !(st[j].ab & (kConv | kDrop))) {
                        const float q = st[j].q_lo;
                        if (q - eps32_at(q, kap, C) > thr) st[j].ab |= kDrop;
                        else lv = true;
                    }
                    const unsigned bal = __ballot_sync(kFull, lv);
                    if (lv) live[n_live + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)j;
                    n_live += __popc(bal);
                }
                __syncwarp();
                if (n_live == 0) break;
                n_extra += n_live;
                float um = INFINITY;
                if (n_live >= kLaneCoop) {
                    // lane by lane
                    for (int i = lane; i < n_live; i += 32) {
                        const int j = live[i];
                        const DirLine dl =
                            make_dir_line<CVX_ENERGY_NH_DAMAGE>(N.nl, P.dir32[doff + gdir(blk, j)]);
                        const NHPair c = line_pair(node, dl);
                        LaneState t = st[j];
                        const Bounds b = pass_bounds(c, H, t.s, m0, line_pass(c, H, -t.s, m0, 0, 1));
                        const int ab = enc_ab(b.a, b.b);
                        const bool same = ab == (t.ab & ~kTan);
                        t.q_lo = fmaxf(t.q_lo, b.q_lo);
                        t.q_hi = fminf(t.q_hi, b.q_hi);
                        t.s = b.s;
                        t.ab = ab | (t.ab & kTan);
                        if (same || t.q_hi - t.q_lo <= 0.25f * eps32_at(t.q_lo, kap, C)) t.ab |= kConv;
                        st[j] = t;
                        um = fminf(um, b.q_hi);
                    }
                } else {
                    // the whole warp on each line
                    for (int i = 0; i < n_live; ++i) {
                        const int j = live[i];
                        const DirLine dl =
                            make_dir_line<CVX_ENERGY_NH_DAMAGE>(N.nl, P.dir32[doff + gdir(blk, j)]);
                        const NHPair c = line_pair(node, dl);
                        LaneState t = st[j];
                        SideMin sm = line_pass(c, H, -t.s, m0, lane, 32);
                        warp_side(sm.eL, sm.kL);
                        warp_side(sm.eR, sm.kR);
                        const Bounds b = pass_bounds(c, H, t.s, m0, sm);
                        const int ab = enc_ab(b.a, b.b);
                        const bool same = ab == (t.ab & ~kTan);
                        t.q_lo = fmaxf(t.q_lo, b.q_lo);
                        t.q_hi = fminf(t.q_hi, b.q_hi);
                        t.s = b.s;
                        t.ab = ab | (t.ab & kTan);
                        if (same || t.q_hi - t.q_lo <= 0.25f * eps32_at(t.q_lo, kap, C)) t.ab |= kConv;
                        __syncwarp();
                        if (lane == 0) st[j] = t;
                        um = fminf(um, b.q_hi);
                    }
                }
                um = warp_min_f32(um);
                int old = 0;
                if (lane == 0) old = atomicMin(P.node_u + qi, f2key(um));
                U = fminf(U, fminf(um, key2f(__shfl_sync(kFull, old, 0))));
                __syncwarp();
            }

            // ---- merge the block's candidates into the item's best list
            {
                int old = 0;
                if (lane == 0) old = atomicMin(P.node_u + qi, f2key(INFINITY));
                U = fminf(U, key2f(__shfl_sync(kFull, old, 0)));
            }
            const float mref = fminf(w0, U);
            const float thr = mref + eps32_at(mref, kap, C);
            // lines that would be candidates although they do not split
            // clearly (their bound does not clear the reference value): try
            // to certify that they cannot split, so that they need no FP64
            // refinement.  Only lines whose first pass took the tangent slope
            // have the far minimum the certificate needs.
            {
                int n_try = 0;
                for (int base = 0; base < nb; base += 32) {
                    const int j = base + lane;
                    bool tr = false;
                    if (j < nb) {
                        const LaneState s = st[j];
                        tr = (s.ab & kTan) && !(s.ab & (kDrop | kNoPair)) && !(s.q_hi < w0 - epsc) &&
                             s.q_lo - eps32_at(s.q_lo, kap, C) <= thr;
                    }
                    const unsigned bal = __ballot_sync(kFull, tr);
                    if (tr) live[n_try + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)j;
                    n_try += __popc(bal);
                }
                __syncwarp();
                for (int i = lane; i < n_try; i += 32) {
                    const int j = live[i];
                    const float4 d32 = P.dir32[doff + gdir(blk, j)];
                    const DirLine dl = make_dir_line<CVX_ENERGY_NH_DAMAGE>(N.nl, d32);
                    const float s0 = sa * __fmaf_rn(cb, dl.cJ, dl.A1);
                    if (flat_certificate(N, dl, d32, ln.h32, m0, 2 * kf - m0, 2 * kn, s0, efl[j], kap))
                        st[j].ab |= kCert;
                }
                __syncwarp();
            }
            unsigned taken = 0;  // bit t: line lane + 32 t of the block
            unsigned dropm = 0;  // bit t: that line is dropped
            unsigned certm = 0;  // bit t: that line is certified not to split
            for (int t = 0, j = lane; j < nb; ++t, j += 32) {
                const LaneState s = st[j];
                const bool ce = (s.ab & kCert) != 0;
                const bool dr = !ce && ((s.ab & kDrop) || s.q_lo - eps32_at(s.q_lo, kap, C) > thr);
                dropm |= (dr || ce) ? 1u << t : 0u;
                certm |= ce ? 1u << t : 0u;
                qhi = fminf(qhi, s.q_hi);
                n_drop += dr ? 1u : 0u;
                n_cert += ce ? 1u : 0u;
                n_flat += (!dr && !ce && s.q_lo >= w0 - epsc) ? 1u : 0u;
            }
            bool held_taken = false;
            float nq = INFINITY;
            int nd = INT_MAX, nab = -1;
            for (int n = 0; n < kItemTop; ++n) {
                float bq = INFINITY;
                int bd = INT_MAX, bt = -1, bab = -1;
                for (int t = 0, j = lane; j < nb; ++t, j += 32) {
                    if (((taken | dropm) >> t) & 1u) continue;
                    const float q = st[j].q_lo;
                    const int gd = gdir(blk, j);
                    if (q < bq || (q == bq && gd < bd)) {
                        bq = q;
                        bd = gd;
                        bt = t;
                        bab = st[j].ab;
                    }
                }
                if (lane < kItemTop && !held_taken && (tq < bq || (tq == bq && td < bd))) {
                    bq = tq;
                    bd = td;
                    bt = 32;  // the held entry
                    bab = tab;
                }
                const float m = warp_min_f32(bq);
                if (!(m < INFINITY)) break;
                const int dm = __reduce_min_sync(kFull, bq == m ? bd : INT_MAX);
                const unsigned win_l = __ballot_sync(kFull, bq == m && bd == dm);
                const int src = __ffs(win_l) - 1;
                const int wab = __shfl_sync(kFull, bab, src);
                if (lane == src) {
                    if (bt == 32) held_taken = true;
                    else taken |= 1u << bt;
                }
                if (lane == n) {
                    nq = m;
                    nd = dm;
                    nab = wab;
                }
            }
            // what was not kept: the smallest lower bound of the rest
            // (a certified line cannot split the node nor lower its value
            // below W(F): it bounds nothing the decision needs)
            for (int t = 0, j = lane; j < nb; ++t, j += 32)
                if (!(((taken | certm) >> t) & 1u)) drop = fminf(drop, st[j].q_lo);
            if (lane < kItemTop && !held_taken) drop = fminf(drop, tq);
            tq = nq;
            td = nd;
            tab = nab;
            __syncwarp();
        }

        // ---- the item's record
        drop = warp_min_f32(drop);
        qhi = warp_min_f32(qhi);
        ItemCands *out = P.items + item;
        if (lane < kItemTop) {
            const bool has = tq < INFINITY;
            out->q[lane] = has ? tq : INFINITY;
            out->dir[lane] = has ? td : -1;
            // the FP32 bridge pair of a kept line, a | b << 16
            out->ab[lane] = has && !(tab & kNoPair) ? ((tab & 0xfff) | (((tab >> 12) & 0xfff) << 16)) : -1;
        }
        const unsigned nk = __ballot_sync(kFull, lane < kItemTop && tq < INFINITY);
        if (lane == 0) {
            out->n = __popc(nk);
            out->w0 = w0;
            out->dropped = drop;
            out->qhi_min = qhi;
            out->flags = 0;
            out->pad = 0;
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) n_valid += __shfl_xor_sync(kFull, n_valid, o);
    n_drop = __reduce_add_sync(kFull, n_drop);
    n_flat = __reduce_add_sync(kFull, n_flat);
    n_cert = __reduce_add_sync(kFull, n_cert);
    if (lane == 0) {
        if (n_cert) atomicAdd(P.counters + C_CERT, (unsigned long long)n_cert);
        if (n_lines) atomicAdd(P.counters + C_LINES, (unsigned long long)n_lines);
        if (n_drop) atomicAdd(P.counters + C_BOUNDED, (unsigned long long)n_drop);
        if (n_flat) atomicAdd(P.counters + C_FLAT, (unsigned long long)n_flat);
        if (n_extra) atomicAdd(P.counters + C_ROUNDS, (unsigned long long)n_extra);
        if (n_valid) atomicAdd(P.counters + C_VALID, n_valid);
    }
}

int lane_scan_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan_lanes, 32 * kLaneWarps, 0) !=
        cudaSuccess)
        return 0;
    return nb;
}

bool lane_scan_enabled(int energy) {
    static int env = -1;
    if (env < 0) {
        const char *v = getenv("CVX_SCAN_KERNEL");
        env = (v && strcmp(v, "warp") == 0) ? 0 : 1;
    }
    return energy == CVX_ENERGY_NH_DAMAGE && env == 1;
}

cudaError_t launch_scan_lanes(const Pipe &p, int level, int sms, cudaStream_t s) {
    static int bpsm = 0;
    if (!bpsm) bpsm = lane_scan_blocks_per_sm();
    if (bpsm < 1) return cudaErrorInvalidConfiguration;
    k_scan_lanes<<<sms * bpsm, 32 * kLaneWarps, 0, s>>>(p, level);
    return cudaGetLastError();
}

}  // namespace cvx
