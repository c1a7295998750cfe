// cvx_bridge.cuh -- warp-cooperative exact lower-hull bridge of one sampled
// rank-one line, read at the line's centre (Algorithm 1 + "interpolation at
// l = 0", Sec. 4.2).
//
// One warp owns one line of L FP32 samples at integer abscissae x = m - m0,
// stored in the warp's shared-memory buffer sw[0, L).  The line is processed
// in chunks of 128 samples: in chunk q lane l owns samples 128 q + 4 l + i,
// i = 0..3 (one 16-byte shared access).  Samples past the last full chunk
// (the tail) are owned one per lane.  NaN and +inf mark excluded samples
// (det <= 0); they are contiguous at the line ends, so the left set
// {m < m0} and the right set {m > m0} are intervals.
//
// The value of the lower hull at x = 0 is min(w_m0, min over a < m0 < b of
// the chord (a, b) at 0).  The minimising pair of the left/right sets (the
// "bridge") is the pair whose chord supports every sample; the centre is a
// strict hull vertex iff it lies strictly below that chord (Algorithm 1 pops
// points lying on a chord, so its vertices are strict).
//
// Search (exact in the end):
//  1. start pair: the previous direction's bridge (neighbouring directions
//     have neighbouring tangent points) or, cold, the argmins at slope 0;
//  2. supporting-slope iteration in 32-sample windows around a and b: with
//     s = slope(a, b), move a (b) to the window's argmin of w - s x; every
//     move lowers the chord at 0;
//  3. exact check of the window samples against the chord: FP32 residual
//     relative to the nearer endpoint with a rigorous rounding bound, and the
//     FP64 orientation determinant (exact for FP32 samples and integer
//     abscissae below 2^12) only inside that bound;
//  4. one certifying pass over the whole line: count samples with
//     w - s x < H + Delta (Delta bounds all FP32 rounding of that test); if
//     every such sample lies in a window (already checked exactly) or is the
//     centre, the bridge is exact; otherwise the outside candidates are
//     checked exactly (rare path) and the search continues.
#pragma once

#include "cvx_device.cuh"

namespace cvx {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHullCap = 96;  // rounds of the search before it gives up (flagged)
// rounds of the screening search: a search that stops before its pair is
// global leaves a rigorous but loose lower bound, and loose bounds can push
// the best directions out of the FP64 refinement
constexpr int kScreenRounds = 4;

struct LineGeom {
    int L, m0, nfull;  // samples, centre index, number of full 128-sample chunks
};

// Per-warp event counters in shared memory, written by lane 0 only.
enum { HC_FP64W, HC_FP64R, HC_FP64C, HC_FULL, HC_RARE, HC_CAPS, HC_WSTEPS, HC_ROUNDS, HC_N };
struct HullCounters {
    unsigned *c;
};

struct BridgeOut {
    int a, b;   // left/right bridge vertices, -1 if a side is empty
    int lam;    // 1: the centre is not a strict vertex (the point splits)
    float wa, wb, w0;
};

// order-preserving float -> int for non-NaN values
__device__ __forceinline__ int f2key(float e) {
    int i = __float_as_int(e);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float nan_to_inf(float v) { return v == v ? v : INFINITY; }

// Side of sample (x_i, w_i) with respect to the line through (x_a, w_a) and
// (x_b, w_b): +1 above, -1 below, 0 on it.  s = fl(fl(w_b - w_a) / (x_b - x_a))
// (IEEE division); (x_n, w_n) is the endpoint used as anchor.  The FP32
// residual r = fl(fl(w_i - w_n) - s (x_i - x_n)) differs from the exact one by
// at most u (|r| + |w_i - w_n| + 2 |s (x_i - x_n)|) to first order; inside
// 1.01 times that bound the sign comes from the FP64 determinant.
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

__device__ __forceinline__ float slope_exact(float wa, int a, float wb, int b) {
    return __fdiv_rn(__fsub_rn(wb, wa), (float)(b - a));
}

// Certifying-pass predicate for sample k, computed identically wherever it is
// evaluated: fl(w_k - s 128 floor(k/128)) < fl(T + s ((k mod 128) - m0)).
__device__ __forceinline__ int cand_pred(int k, float v, float ns, float s, float T, int m0) {
    const float c = __fmaf_rn(ns, (float)(k & ~127), v);
    const float Tk = __fmaf_rn(s, (float)((k & 127) - m0), T);
    return c < Tk ? 1 : 0;
}

// Full pass over the line: argmin of w - s x over the left and right sets
// (FP32, approximate; exactness comes from the later checks).
static __device__ __noinline__ void full_argmin(const float *sw, const LineGeom g, int lane, float s,
                                         int &a, int &b) {
    float bl = INFINITY, br = INFINITY;
    int kl = -1, kr = -1;
    for (int k = lane; k < g.L; k += 32) {
        if (k == g.m0) continue;
        const float e = __fmaf_rn(-s, (float)(k - g.m0), sw[k]);
        if (k < g.m0) {
            if (e < bl) { bl = e; kl = k; }
        } else if (e < br) {
            br = e;
            kr = k;
        }
    }
    int keyl = kl >= 0 ? f2key(bl) : 0x7fffffff, keyr = kr >= 0 ? f2key(br) : 0x7fffffff;
    int ml = __reduce_min_sync(kFull, keyl), mr = __reduce_min_sync(kFull, keyr);
    unsigned bal = __ballot_sync(kFull, keyl == ml), bar = __ballot_sync(kFull, keyr == mr);
    int ia = __shfl_sync(kFull, kl, __ffs(bal) - 1), ib = __shfl_sync(kFull, kr, __ffs(bar) - 1);
    const int kinf = f2key(INFINITY);
    a = (ml >= kinf) ? -1 : ia;
    b = (mr >= kinf) ? -1 : ib;
}

// Window of 32 samples around the left vertex a (inside [0, m0)) and the right
// vertex b (inside (m0, L)).
__device__ __forceinline__ int win_lo_a(int a, int m0) { return max(0, min(a - 16, m0 - 32)); }
__device__ __forceinline__ int win_lo_b(int b, int m0, int L) {
    return min(max(b - 15, m0 + 1), max(m0 + 1, L - 32));
}

// Rare path: exact check of every certifying-pass candidate outside the
// windows and the centre.  Returns 1 if the pair changed (a sample strictly
// below the chord, or a collinear sample farther out).
static __device__ __noinline__ int rare_path(const float *sw, const LineGeom g, int lane, int &a, int &b,
                                      float wa, float wb, float s, float ns, float T, int loA,
                                      int loB, unsigned &fp64_total) {
    unsigned fp64 = 0;
    int bestKeyL = 0x7fffffff, bestKL = -1, bestKeyR = 0x7fffffff, bestKR = -1;
    int outL = 0x7fffffff, outR = -1;
    for (int k0 = 0; k0 < g.L; k0 += 32) {
        const int k = k0 + lane;
        const float v = k < g.L ? sw[k] : INFINITY;
        bool inwin = (k >= loA && k < loA + 32 && k < g.m0) || (k >= loB && k < loB + 32);
        bool cnd = k < g.L && k != g.m0 && !inwin && cand_pred(k, v, ns, s, T, g.m0);
        if (__any_sync(kFull, cnd)) {
            int sd = 1;
            if (cnd) {
                if (k < g.m0) sd = side_exact(v, k, wa, a, wb, b, s, wa, a, fp64);
                else sd = side_exact(v, k, wa, a, wb, b, s, wb, b, fp64);
            }
            const int key = f2key(__fmaf_rn(-s, (float)(k - g.m0), v));
            if (sd < 0 && k < g.m0 && key < bestKeyL) { bestKeyL = key; bestKL = k; }
            if (sd < 0 && k > g.m0 && key < bestKeyR) { bestKeyR = key; bestKR = k; }
            if (sd == 0 && k < a && k < outL) outL = k;
            if (sd == 0 && k > b && k > outR) outR = k;
        }
    }
    fp64_total = __reduce_add_sync(kFull, fp64);
    int mL = __reduce_min_sync(kFull, bestKeyL), mR = __reduce_min_sync(kFull, bestKeyR);
    unsigned bl = __ballot_sync(kFull, bestKL >= 0 && bestKeyL == mL);
    unsigned br = __ballot_sync(kFull, bestKR >= 0 && bestKeyR == mR);
    int ol = __reduce_min_sync(kFull, outL), orr = __reduce_max_sync(kFull, outR);
    if (bl | br) {
        if (bl) a = __shfl_sync(kFull, bestKL, __ffs(bl) - 1);
        if (br) b = __shfl_sync(kFull, bestKR, __ffs(br) - 1);
        return 1;
    }
    if (ol != 0x7fffffff || orr >= 0) {
        if (ol != 0x7fffffff) a = ol;
        if (orr >= 0) b = orr;
        return 1;
    }
    return 0;
}

__device__ __forceinline__ BridgeOut warp_bridge(float *sw, const LineGeom g, int lane,
                                                 int warm_a, int warm_b, HullCounters &hc) {
    BridgeOut out;
    const int m0 = g.m0, L = g.L;
    out.w0 = sw[m0];
    out.a = out.b = -1;
    out.lam = 0;
    out.wa = out.wb = out.w0;
    if (m0 < 1 || !(sw[m0 - 1] < INFINITY) || !(sw[m0 + 1] < INFINITY)) return out;

    int a, b;
    if (warm_a >= 0 && warm_a < m0 && warm_b > m0 && warm_b < L && sw[warm_a] < INFINITY &&
        sw[warm_b] < INFINITY) {
        a = warm_a;
        b = warm_b;
    } else {
        full_argmin(sw, g, lane, 0.0f, a, b);
        if (lane == 0) ++hc.c[HC_FULL];
        if (a < 0 || b < 0) return out;
    }

    bool fp32_steps = true;
    bool done = false;
    int round = 0;
    float wa = sw[a], wb = sw[b];
    float s_fin = 0.0f;
    for (; round < kHullCap && !done; ++round) {
        if (lane == 0) ++hc.c[HC_ROUNDS];
        int loA = win_lo_a(a, m0), loB = win_lo_b(b, m0, L);
        int kA = loA + lane, kB = loB + lane;
        float vA = kA < m0 ? nan_to_inf(sw[kA]) : INFINITY;
        float vB = kB < L ? nan_to_inf(sw[kB]) : INFINITY;
        // ---- 2. supporting-slope iteration inside the windows (FP32) -------
        if (fp32_steps) {
            float XA = (float)(kA - m0), XB = (float)(kB - m0);
            for (int it = 0; it < 32; ++it) {
                const float s = __fdividef(wb - wa, (float)(b - a));
                const int keyA = f2key(__fmaf_rn(-s, XA, vA));
                const int keyB = f2key(__fmaf_rn(-s, XB, vB));
                const int mA = __reduce_min_sync(kFull, keyA), mB = __reduce_min_sync(kFull, keyB);
                const unsigned bA = __ballot_sync(kFull, keyA == mA);
                const unsigned bB = __ballot_sync(kFull, keyB == mB);
                const int na = ((bA >> (a - loA)) & 1u) ? a : loA + __ffs(bA) - 1;
                const int nb = ((bB >> (b - loB)) & 1u) ? b : loB + __ffs(bB) - 1;
                if (lane == 0) ++hc.c[HC_WSTEPS];
                if (na == a && nb == b) break;
                wa = __shfl_sync(kFull, vA, na - loA);
                wb = __shfl_sync(kFull, vB, nb - loB);
                a = na;
                b = nb;
                const int nloA = win_lo_a(a, m0), nloB = win_lo_b(b, m0, L);
                if (nloA != loA && (a - loA < 4 || a - loA > 27)) {
                    loA = nloA;
                    kA = loA + lane;
                    vA = kA < m0 ? nan_to_inf(sw[kA]) : INFINITY;
                    XA = (float)(kA - m0);
                }
                if (nloB != loB && (b - loB < 4 || b - loB > 27)) {
                    loB = nloB;
                    kB = loB + lane;
                    vB = kB < L ? nan_to_inf(sw[kB]) : INFINITY;
                    XB = (float)(kB - m0);
                }
            }
            // windows centred on the final pair for the checks below
            const int nloA = win_lo_a(a, m0), nloB = win_lo_b(b, m0, L);
            if (nloA != loA) {
                loA = nloA;
                kA = loA + lane;
                vA = kA < m0 ? nan_to_inf(sw[kA]) : INFINITY;
            }
            if (nloB != loB) {
                loB = nloB;
                kB = loB + lane;
                vB = kB < L ? nan_to_inf(sw[kB]) : INFINITY;
            }
        }
        const bool inA = kA < m0, inB = kB < L;
        const float s = slope_exact(wa, a, wb, b);

        // ---- 3. exact check of the windows --------------------------------
        unsigned uA = 0, uB = 0;
        const int sA = (inA && kA != a) ? side_exact(vA, kA, wa, a, wb, b, s, wa, a, uA) : 1;
        const int sB = (inB && kB != b) ? side_exact(vB, kB, wa, a, wb, b, s, wb, b, uB) : 1;
        {
            const unsigned n64 = __popc(__ballot_sync(kFull, uA != 0)) + __popc(__ballot_sync(kFull, uB != 0));
            if (lane == 0) hc.c[HC_FP64W] += n64;
        }
        const unsigned belowA = __ballot_sync(kFull, sA < 0), belowB = __ballot_sync(kFull, sB < 0);
        if (belowA | belowB) {
            // move to the violating sample with the lowest FP32 w - s x
            const int keyA = sA < 0 ? f2key(__fmaf_rn(-s, (float)(kA - m0), vA)) : 0x7fffffff;
            const int keyB = sB < 0 ? f2key(__fmaf_rn(-s, (float)(kB - m0), vB)) : 0x7fffffff;
            const int mA = __reduce_min_sync(kFull, keyA), mB = __reduce_min_sync(kFull, keyB);
            const unsigned bA = __ballot_sync(kFull, keyA == mA && sA < 0);
            const unsigned bB = __ballot_sync(kFull, keyB == mB && sB < 0);
            if (belowA) a = loA + __ffs(bA) - 1;
            if (belowB) b = loB + __ffs(bB) - 1;
            wa = sw[a];
            wb = sw[b];
            if (round >= 1) fp32_steps = false;
            continue;
        }
        const unsigned onA = __ballot_sync(kFull, sA == 0 && kA < a);
        const unsigned onB = __ballot_sync(kFull, sB == 0 && kB > b);
        if (onA | onB) {
            // collinear samples farther out: Algorithm 1 keeps the outermost
            if (onA) a = loA + __ffs(onA) - 1;
            if (onB) b = loB + 31 - __clz(onB);
            wa = sw[a];
            wb = sw[b];
            fp32_steps = false;
            continue;
        }

        // ---- 4. certifying pass over the whole line ------------------------
        // The window samples (checked exactly above) and the centre are
        // masked with +inf; any other sample with w - s x < H + Delta is a
        // candidate that needs the exact check of the rare path.
        const float ns = -s;
        const float Hp = __fmaf_rn(-s, (float)(a - m0), wa);
        const float Delta = 8.0f * kU32 * (fabsf(Hp) + 2.0f * fabsf(s) * (float)L) + 1e-30f;
        const float T = __fadd_rn(Hp, Delta);
        if (inA) sw[kA] = INFINITY;
        if (inB) sw[kB] = INFINITY;
        if (lane == 0) sw[m0] = INFINITY;
        __syncwarp();
        float Tl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) Tl[i] = __fmaf_rn(s, (float)(4 * lane + i - m0), T);
        bool any = false;
        float fq = 0.0f;
#pragma unroll 4
        for (int q = 0; q < g.nfull; ++q, fq += 128.0f) {
            const float4 v = *reinterpret_cast<const float4 *>(sw + 128 * q + 4 * lane);
            any |= __fmaf_rn(ns, fq, v.x) < Tl[0];
            any |= __fmaf_rn(ns, fq, v.y) < Tl[1];
            any |= __fmaf_rn(ns, fq, v.z) < Tl[2];
            any |= __fmaf_rn(ns, fq, v.w) < Tl[3];
        }
        for (int k = 128 * g.nfull + lane; k < L; k += 32) any |= cand_pred(k, sw[k], ns, s, T, m0);
        int moved = 0;
        if (__any_sync(kFull, any)) {
            // ---- rare path (windows and centre still masked) ----------------
            unsigned r64 = 0;
            moved = rare_path(sw, g, lane, a, b, wa, wb, s, ns, T, loA, loB, r64);
            if (lane == 0) {
                ++hc.c[HC_RARE];
                hc.c[HC_FP64R] += r64;
            }
        }
        __syncwarp();
        if (inA) sw[kA] = vA;  // excluded samples come back as +inf
        if (inB) sw[kB] = vB;
        if (lane == 0) sw[m0] = out.w0;
        __syncwarp();
        if (moved) {
            wa = sw[a];
            wb = sw[b];
            if (round >= 1) fp32_steps = false;
            continue;
        }
        s_fin = s;
        done = true;  // every candidate lies exactly on or above the chord
    }
    if (!done && lane == 0) ++hc.c[HC_CAPS];

    // ---- centre: strict vertex iff strictly below the bridge chord ---------
    const float s = done ? s_fin : slope_exact(wa, a, wb, b);
    unsigned c64 = 0;
    const int sc = side_exact(out.w0, m0, wa, a, wb, b, s, wa, a, c64);
    if (lane == 0) hc.c[HC_FP64C] += c64;
    out.a = a;
    out.b = b;
    out.wa = wa;
    out.wb = wb;
    out.lam = sc >= 0 ? 1 : 0;
    return out;
}

// -------------------------------------------------------------------------
// Screening form (used by the line scan, whose decisions are taken later in
// FP64): rigorous bounds on the value at 0 of the lower hull of the left and
// right sets instead of the exact bridge.  For ANY slope s,
//   hull(0) >= min_i (w_i - s x_i)                  (an affine minorant)
// and for any pair a < 0 < b,
//   hull(0) <= chord(a, b)(0).
// The window iteration makes both sides meet up to rounding; the min pass
// costs one FMA and one min per sample.
// -------------------------------------------------------------------------
struct ScreenOut {
    int a, b;          // approximate bridge (for the next direction's warm start), -1 if none
    float q_lo, q_hi;  // q_lo <= value at 0 of the hull of the FP32 left/right samples <= q_hi
    float w0;          // FP32 centre sample
};

// Min over the line of w - s x, the centre excluded (set to +inf by the
// caller); per lane four independent running minima per chunk component.
__device__ __forceinline__ float min_pass(const float *sw, const LineGeom &g, int lane, float s) {
    const float ns = -s;
    const f32x2 NS = pk2(ns, ns);
    float m[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
    float fq = 0.0f;
#pragma unroll 4
    for (int q = 0; q < g.nfull; ++q, fq += 128.0f) {
        const float4 v = *reinterpret_cast<const float4 *>(sw + 128 * q + 4 * lane);
        const f32x2 FQ = pk2(fq, fq);
        float e0, e1, e2, e3;
        upk2(fma2(NS, FQ, pk2(v.x, v.y)), e0, e1);
        upk2(fma2(NS, FQ, pk2(v.z, v.w)), e2, e3);
        m[0] = fminf(m[0], e0);
        m[1] = fminf(m[1], e1);
        m[2] = fminf(m[2], e2);
        m[3] = fminf(m[3], e3);
    }
    float e = INFINITY;
#pragma unroll
    for (int i = 0; i < 4; ++i) e = fminf(e, __fmaf_rn(ns, (float)(4 * lane + i - g.m0), m[i]));
    for (int k = 128 * g.nfull + lane; k < g.L; k += 32)
        e = fminf(e, __fmaf_rn(ns, (float)(k - g.m0), sw[k]));
    // warp minimum (keys order like floats; NaN never wins against +inf)
    const int mk = __reduce_min_sync(kFull, f2key(nan_to_inf(e)));
    return __int_as_float(f2key(__int_as_float(mk)));  // f2key is its own inverse
}

__device__ __forceinline__ ScreenOut warp_screen(float *sw, const LineGeom g, int lane,
                                                 int warm_a, int warm_b, HullCounters &hc) {
    ScreenOut out;
    const int m0 = g.m0, L = g.L;
    out.w0 = sw[m0];
    out.a = out.b = -1;
    out.q_lo = out.q_hi = INFINITY;
    if (m0 < 1 || !(sw[m0 - 1] < INFINITY) || !(sw[m0 + 1] < INFINITY)) return out;

    int a, b;
    if (warm_a >= 0 && warm_a < m0 && warm_b > m0 && warm_b < L && sw[warm_a] < INFINITY &&
        sw[warm_b] < INFINITY) {
        a = warm_a;
        b = warm_b;
    } else {
        full_argmin(sw, g, lane, 0.0f, a, b);
        if (lane == 0) ++hc.c[HC_FULL];
        if (a < 0 || b < 0) return out;
    }
    float wa = sw[a], wb = sw[b];
    float s = 0.0f, emin = -INFINITY;
    for (int round = 0; round < kScreenRounds; ++round) {
        if (lane == 0) ++hc.c[HC_ROUNDS];
        // supporting-slope iteration inside 32-sample windows around a and b
        int loA = win_lo_a(a, m0), loB = win_lo_b(b, m0, L);
        int kA = loA + lane, kB = loB + lane;
        float vA = kA < m0 ? nan_to_inf(sw[kA]) : INFINITY;
        float vB = kB < L ? nan_to_inf(sw[kB]) : INFINITY;
        float XA = (float)(kA - m0), XB = (float)(kB - m0);
        for (int it = 0; it < 32; ++it) {
            s = __fdividef(wb - wa, (float)(b - a));
            const int keyA = f2key(__fmaf_rn(-s, XA, vA));
            const int keyB = f2key(__fmaf_rn(-s, XB, vB));
            const int mA = __reduce_min_sync(kFull, keyA), mB = __reduce_min_sync(kFull, keyB);
            const unsigned bA = __ballot_sync(kFull, keyA == mA);
            const unsigned bB = __ballot_sync(kFull, keyB == mB);
            const int na = ((bA >> (a - loA)) & 1u) ? a : loA + __ffs(bA) - 1;
            const int nb = ((bB >> (b - loB)) & 1u) ? b : loB + __ffs(bB) - 1;
            if (lane == 0) ++hc.c[HC_WSTEPS];
            if (na == a && nb == b) break;
            wa = __shfl_sync(kFull, vA, na - loA);
            wb = __shfl_sync(kFull, vB, nb - loB);
            a = na;
            b = nb;
            const int nloA = win_lo_a(a, m0), nloB = win_lo_b(b, m0, L);
            if (nloA != loA && (a - loA < 4 || a - loA > 27)) {
                loA = nloA;
                kA = loA + lane;
                vA = kA < m0 ? nan_to_inf(sw[kA]) : INFINITY;
                XA = (float)(kA - m0);
            }
            if (nloB != loB && (b - loB < 4 || b - loB > 27)) {
                loB = nloB;
                kB = loB + lane;
                vB = kB < L ? nan_to_inf(sw[kB]) : INFINITY;
                XB = (float)(kB - m0);
            }
        }
        s = __fdividef(wb - wa, (float)(b - a));
        // min pass with the centre masked
        __syncwarp();
        if (lane == 0) sw[m0] = INFINITY;
        __syncwarp();
        emin = min_pass(sw, g, lane, s);
        __syncwarp();
        if (lane == 0) sw[m0] = out.w0;
        __syncwarp();
        const float H = __fmaf_rn(-s, (float)(a - m0), wa);
        const float M = fabsf(H) + fabsf(s) * (float)m0;
        if (emin >= H - 4.0f * kU32 * M) break;  // the windows' pair is (nearly) global
        if (round == kScreenRounds - 1) break;     // bounds stay rigorous, only looser
        // a sample lies clearly below the chord: restart from the global argmin
        if (lane == 0) ++hc.c[HC_RARE];
        full_argmin(sw, g, lane, s, a, b);
        if (a < 0 || b < 0) return out;
        wa = sw[a];
        wb = sw[b];
    }
    // rigorous bounds (first-order rounding of each computed w - s x is at most
    // 3u (|w - s x| + 2 |s| m0); the chord at 0 is within 4u (|wa|+|wb|+|q|))
    const float xa = (float)(a - m0), xb = (float)(b - m0);
    const float chord = wa + (wb - wa) * __fdividef(-xa, xb - xa);
    out.q_lo = emin - 3.2f * kU32 * (fabsf(emin) + 2.0f * fabsf(s) * (float)m0) - 1e-30f;
    out.q_hi = chord + 4.0f * kU32 * (fabsf(wa) + fabsf(wb) + fabsf(chord)) + 1e-30f;
    out.q_lo = fminf(out.q_lo, out.q_hi);
    out.a = a;
    out.b = b;
    return out;
}

}  // namespace cvx
