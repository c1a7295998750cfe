// cvx_bridge.cuh -- warp-cooperative exact lower-hull bridge of one sampled
// rank-one line, read at the line's centre (Algorithm 1 + "interpolation at
// l = 0", Sec. 4.2).
//
// One warp owns one line of L FP32 samples at integer abscissae x = m - m0.
// Sample m lives in register slot j = m / 32 of lane m % 32 (so a slot is a
// contiguous run of 32 samples) and in the warp's shared-memory copy sw[m].
// NaN marks excluded samples (det <= 0 or m >= L); they are contiguous at the
// line ends, so the left set {m < m0} and right set {m > m0} are intervals.
//
// The value of the lower hull at x = 0 is min(w_m0, min over a < m0 < b of
// the chord (a, b) at 0).  The minimising pair of the left/right sets (the
// "bridge") is the pair whose chord supports every sample; the centre is a
// strict hull vertex iff it lies strictly below that chord (Algorithm 1 pops
// points on a chord, so its vertices are strict).
//
// Search (all exact in the end):
//  1. start pair: the previous direction's bridge (neighbouring directions
//     have neighbouring tangent points) or, cold, the argmins at slope 0;
//  2. supporting-slope iteration in 32-sample windows around a and b: with
//     s = slope(a, b), move a (b) to the window's argmin of w - s x; each move
//     lowers the chord at 0;
//  3. exact check of the window samples against the chord: FP32 anchor-
//     relative residual with a rigorous rounding bound, FP64 (exact for FP32
//     inputs and integer abscissae) only inside the bound;
//  4. one certifying pass over the whole line: count samples with
//     w - s x < H + Delta (Delta bounds all FP32 rounding); if every such
//     sample lies in a window (already exactly checked) the bridge is exact;
//     otherwise the outside candidates are checked exactly (rare path).
#pragma once

#include "cvx_device.cuh"

namespace cvx {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHullCap = 96;  // rounds of the search before it gives up (flagged)

struct LineGeom {
    int L, m0, j0, c0;  // samples, centre index, centre slot and lane
};

struct HullCounters {
    unsigned fp64, full_passes, rare, caps;   // fp64: per lane; others: lane 0
    unsigned wsteps, rounds, fp64r, fp64c;    // wsteps/rounds/fp64c: lane 0; fp64r: per lane
};

struct BridgeOut {
    int a, b;   // left/right bridge vertices, -1 if a side is empty
    int lam;    // 1: the centre is not a strict vertex (the point splits)
    float wa, wb, w0;
};

// order-preserving float -> int (NaN -> INT_MAX)
__device__ __forceinline__ int f2key(float e) {
    int i = __float_as_int(e);
    i ^= (i >> 31) & 0x7fffffff;
    return (e == e) ? i : 0x7fffffff;
}

// Side of sample (x_i, w_i) with respect to the line through (x_a, w_a) and
// (x_b, w_b): +1 above, -1 below, 0 on it.  s is the FP32 slope
// fl(fl(w_b - w_a) / (x_b - x_a)); (x_n, w_n) is the endpoint used as anchor
// (the nearer one keeps the FP32 residual small).  The FP32 residual
// r = fl(fl(w_i - w_n) - s (x_i - x_n)) differs from the exact one by at most
// u (|r| + |w_i - w_n| + 2 |s (x_i - x_n)|) (first order); inside that bound
// the sign is taken from the FP64 orientation determinant, which is exact for
// FP32 samples and integer abscissae below 2^12.
__device__ __forceinline__ int side_exact(float wi, int xi, float wa, int xa, float wb, int xb,
                                          float s, float wn, int xn, unsigned &fp64) {
    if (!(wi < INFINITY)) return 1;
    float dw = __fsub_rn(wi, wn);
    float dx = (float)(xi - xn);
    float r = __fmaf_rn(-s, dx, dw);
    float bound = 1.01f * kU32 * (fabsf(r) + fabsf(dw) + 2.0f * fabsf(s * dx)) + 1e-30f;
    if (r > bound) return 1;
    if (r < -bound) return -1;
    ++fp64;
    double sg = ((double)wi - (double)wa) * (double)(xb - xa) -
                ((double)wb - (double)wa) * (double)(xi - xa);
    return sg > 0.0 ? 1 : (sg < 0.0 ? -1 : 0);
}

__device__ __forceinline__ float slope_of(float wa, int a, float wb, int b) {
    return __fdiv_rn(__fsub_rn(wb, wa), (float)(b - a));
}

// Full pass: argmin over the left and right sets of w - s x (FP32).
template <int NS>
__device__ __forceinline__ void full_argmin(const float (&w)[NS], const LineGeom &g, int lane,
                                            float s, int &a, int &b) {
    const float ns32 = -32.0f * s;
    float bl = INFINITY, br = INFINITY;
    int jl = -1, jr = -1;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        if (32 * j >= g.L) break;
        float c = __fmaf_rn(ns32, (float)j, w[j]);
        bool isl = (j < g.j0) || (j == g.j0 && lane < g.c0);
        bool isr = (j > g.j0) || (j == g.j0 && lane > g.c0);
        if (isl && c < bl) { bl = c; jl = j; }
        if (isr && c < br) { br = c; jr = j; }
    }
    const float off = -s * (float)(lane - g.m0);
    float vl = (jl >= 0) ? bl + off : INFINITY;
    float vr = (jr >= 0) ? br + off : INFINITY;
    int kl = f2key(vl), kr = f2key(vr);
    int ml = __reduce_min_sync(kFull, kl), mr = __reduce_min_sync(kFull, kr);
    unsigned bal = __ballot_sync(kFull, kl == ml), bar = __ballot_sync(kFull, kr == mr);
    int sl = __ffs(bal) - 1, sr = __ffs(bar) - 1;
    int ia = __shfl_sync(kFull, 32 * jl + lane, sl);
    int ib = __shfl_sync(kFull, 32 * jr + lane, sr);
    a = (ml == f2key(INFINITY) || ml == 0x7fffffff) ? -1 : ia;
    b = (mr == f2key(INFINITY) || mr == 0x7fffffff) ? -1 : ib;
}

// Window of 32 samples around the left vertex a (inside [0, m0)) and the right
// vertex b (inside (m0, L)).
__device__ __forceinline__ int win_lo_a(int a, int m0) { return max(0, min(a - 16, m0 - 32)); }
__device__ __forceinline__ int win_lo_b(int b, int m0, int L) {
    return min(max(b - 15, m0 + 1), max(m0 + 1, L - 32));
}

template <int NS>
__device__ BridgeOut warp_bridge(const float (&w)[NS], const float *sw, const LineGeom &g,
                                 int lane, int warm_a, int warm_b, HullCounters &hc) {
    BridgeOut out;
    const int m0 = g.m0, L = g.L;
    out.w0 = sw[m0];
    out.a = out.b = -1;
    out.lam = 0;
    out.wa = out.wb = out.w0;
    if (m0 < 1 || !(sw[m0 - 1] < INFINITY) || !(sw[m0 + 1] < INFINITY)) return out;

    int a, b;
    bool warm = warm_a >= 0 && warm_a < m0 && warm_b > m0 && warm_b < L &&
                sw[warm_a] < INFINITY && sw[warm_b] < INFINITY;
    if (warm) {
        a = warm_a;
        b = warm_b;
    } else {
        full_argmin<NS>(w, g, lane, 0.0f, a, b);
        if (lane == 0) ++hc.full_passes;
        if (a < 0 || b < 0) return out;
    }

    bool fp32_steps = true;
    bool done = false;
    int round = 0;
    for (; round < kHullCap && !done; ++round) {
        if (lane == 0) ++hc.rounds;
        // ---- 2. supporting-slope iteration inside the windows (FP32) -------
        if (fp32_steps) {
            for (int it = 0; it < 32; ++it) {
                float wa = sw[a], wb = sw[b];
                float s = slope_of(wa, a, wb, b);
                int loA = win_lo_a(a, m0), loB = win_lo_b(b, m0, L);
                int kA = loA + lane, kB = loB + lane;
                float vA = kA < m0 ? sw[kA] : __int_as_float(0x7fffffff);
                float vB = kB < L ? sw[kB] : __int_as_float(0x7fffffff);
                int keyA = f2key(__fmaf_rn(-s, (float)(kA - m0), vA));
                int keyB = f2key(__fmaf_rn(-s, (float)(kB - m0), vB));
                int mA = __reduce_min_sync(kFull, keyA), mB = __reduce_min_sync(kFull, keyB);
                unsigned bA = __ballot_sync(kFull, keyA == mA), bB = __ballot_sync(kFull, keyB == mB);
                int na = ((bA >> (a - loA)) & 1u) ? a : loA + __ffs(bA) - 1;
                int nb = ((bB >> (b - loB)) & 1u) ? b : loB + __ffs(bB) - 1;
                if (lane == 0) ++hc.wsteps;
                if (na == a && nb == b) break;
                a = na;
                b = nb;
            }
        }
        float wa = sw[a], wb = sw[b];
        float s = slope_of(wa, a, wb, b);
        int loA = win_lo_a(a, m0), loB = win_lo_b(b, m0, L);
        int kA = loA + lane, kB = loB + lane;
        bool inA = kA < m0, inB = kB < L;
        float vA = inA ? sw[kA] : __int_as_float(0x7fffffff);
        float vB = inB ? sw[kB] : __int_as_float(0x7fffffff);

        // ---- 3. exact check of the windows --------------------------------
        int sA = (inA && kA != a) ? side_exact(vA, kA, wa, a, wb, b, s, wa, a, hc.fp64) : 1;
        int sB = (inB && kB != b) ? side_exact(vB, kB, wa, a, wb, b, s, wb, b, hc.fp64) : 1;
        unsigned belowA = __ballot_sync(kFull, sA < 0), belowB = __ballot_sync(kFull, sB < 0);
        if (belowA | belowB) {
            // move to the violating sample with the lowest FP32 w - s x
            int keyA = sA < 0 ? f2key(__fmaf_rn(-s, (float)(kA - m0), vA)) : 0x7fffffff;
            int keyB = sB < 0 ? f2key(__fmaf_rn(-s, (float)(kB - m0), vB)) : 0x7fffffff;
            int mA = __reduce_min_sync(kFull, keyA), mB = __reduce_min_sync(kFull, keyB);
            unsigned bA = __ballot_sync(kFull, keyA == mA && sA < 0);
            unsigned bB = __ballot_sync(kFull, keyB == mB && sB < 0);
            if (belowA) a = loA + __ffs(bA) - 1;
            if (belowB) b = loB + __ffs(bB) - 1;
            if (round >= 1) fp32_steps = false;
            continue;
        }
        unsigned onA = __ballot_sync(kFull, sA == 0 && kA < a);
        unsigned onB = __ballot_sync(kFull, sB == 0 && kB > b);
        if (onA | onB) {
            // collinear samples farther out: Algorithm 1 keeps the outermost
            if (onA) a = loA + __ffs(onA) - 1;
            if (onB) b = loB + 31 - __clz(onB);
            fp32_steps = false;
            continue;
        }

        // ---- 4. certifying pass over the whole line ------------------------
        const float ns32 = -32.0f * s;
        const float Hp = __fmaf_rn(-s, (float)(a - m0), wa);
        const float Delta = 8.0f * kU32 * (fabsf(Hp) + 2.0f * fabsf(s) * (float)L) + 1e-30f;
        const float T = __fadd_rn(Hp, Delta);
        const float Tl = __fmaf_rn(s, (float)(lane - m0), T);
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            if (32 * j >= L) break;
            cnt += (__fmaf_rn(ns32, (float)j, w[j]) < Tl) ? 1 : 0;
        }
        auto cand = [&](int k, float v) -> int {
            float Tk = __fmaf_rn(s, (float)((k & 31) - m0), T);
            return (__fmaf_rn(ns32, (float)(k >> 5), v) < Tk) ? 1 : 0;
        };
        int cw = (inA ? cand(kA, vA) : 0) + (inB ? cand(kB, vB) : 0) +
                 (lane == 0 ? cand(m0, out.w0) : 0);
        int C = __reduce_add_sync(kFull, cnt);
        int Cw = __reduce_add_sync(kFull, cw);
        if (C == Cw) {
            done = true;
            break;
        }

        // ---- rare path: exact check of the candidates outside the windows --
        if (lane == 0) ++hc.rare;
        int bestKeyL = 0x7fffffff, bestKL = -1, bestKeyR = 0x7fffffff, bestKR = -1;
        int outL = 0x7fffffff, outR = -1;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            if (32 * j >= L) break;
            const int k = 32 * j + lane;
            const float v = w[j];
            const float c = __fmaf_rn(ns32, (float)j, v);
            bool inwin = (k >= loA && k < loA + 32 && k < m0) || (k >= loB && k < loB + 32 && k < L);
            bool cnd = k < L && k != m0 && !inwin && (c < Tl);
            if (__any_sync(kFull, cnd)) {
                int sd = 1;
                if (cnd) {
                    if (k < m0) sd = side_exact(v, k, wa, a, wb, b, s, wa, a, hc.fp64r);
                    else sd = side_exact(v, k, wa, a, wb, b, s, wb, b, hc.fp64r);
                }
                int key = f2key(c - s * (float)(lane - m0));
                if (sd < 0 && k < m0 && key < bestKeyL) { bestKeyL = key; bestKL = k; }
                if (sd < 0 && k > m0 && key < bestKeyR) { bestKeyR = key; bestKR = k; }
                if (sd == 0 && k < a && k < outL) outL = k;
                if (sd == 0 && k > b && k > outR) outR = k;
            }
        }
        int mL = __reduce_min_sync(kFull, bestKeyL), mR = __reduce_min_sync(kFull, bestKeyR);
        unsigned bl = __ballot_sync(kFull, bestKL >= 0 && bestKeyL == mL);
        unsigned br = __ballot_sync(kFull, bestKR >= 0 && bestKeyR == mR);
        int ol = __reduce_min_sync(kFull, outL), orr = __reduce_max_sync(kFull, outR);
        if (bl | br) {
            if (bl) a = __shfl_sync(kFull, bestKL, __ffs(bl) - 1);
            if (br) b = __shfl_sync(kFull, bestKR, __ffs(br) - 1);
            if (round >= 1) fp32_steps = false;
            continue;
        }
        if (ol != 0x7fffffff || orr >= 0) {
            if (ol != 0x7fffffff) a = ol;
            if (orr >= 0) b = orr;
            fp32_steps = false;
            continue;
        }
        done = true;  // every candidate lies exactly on or above the chord
    }
    if (!done && lane == 0) ++hc.caps;

    // ---- centre: strict vertex iff strictly below the bridge chord ---------
    const float wa = sw[a], wb = sw[b];
    const float s = slope_of(wa, a, wb, b);
    unsigned c64 = 0;
    int sc = side_exact(out.w0, m0, wa, a, wb, b, s, wa, a, c64);
    if (lane == 0) hc.fp64c += c64;
    out.a = a;
    out.b = b;
    out.wa = wa;
    out.wb = wb;
    out.lam = sc >= 0 ? 1 : 0;
    return out;
}

// Hull value at 0 of a bridge in FP64: (x_b w_a - x_a w_b) / (x_b - x_a),
// or w_m0 when the centre is a vertex.
__device__ __forceinline__ double bridge_h64(const BridgeOut &o, int m0) {
    if (!o.lam) return (double)o.w0;
    double xa = (double)(o.a - m0), xb = (double)(o.b - m0);
    return (xb * (double)o.wa - xa * (double)o.wb) / (xb - xa);
}

}  // namespace cvx
