// cvx_line.cuh -- sampling one rank-one line into a warp's shared buffer.
#pragma once

#include <type_traits>

#include "cvx_bridge.cuh"
#include "cvx_internal.h"

namespace cvx {

// In chunk q lane l computes samples 128 q + 4 l + i (one 16-byte store); the
// tail past the last full chunk is one sample per lane.  tl[i] = (4 l + i - m0) h.
template <int EK>
__device__ __forceinline__ void sample_line(float *sw, const NodeLine &nl, const DirLine &dl,
                                            const LineSpec &ln, int lane, const float (&tl)[4]) {
    const float h128 = 128.0f * ln.h32;
    float fq = 0.0f;
#pragma unroll 1
    for (int q = 0; q < ln.nfull; ++q, fq += 1.0f) {
        float4 v;
        v.x = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[0]));
        v.y = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[1]));
        v.z = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[2]));
        v.w = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[3]));
        *reinterpret_cast<float4 *>(sw + 128 * q + 4 * lane) = v;
    }
    for (int k = 128 * ln.nfull + lane; k < ln.L; k += 32)
        sw[k] = sample_w<EK>(nl, dl, (float)(k - ln.m0) * ln.h32);
}

// sample_line that also returns this lane's min over its samples of
// v - s x (ns = -s, x = m - m0): with the warp minimum, a lower bound of the
// line's hull value at 0 for any slope s (the centre sample included only
// lowers it).
template <int EK>
__device__ __forceinline__ float sample_line_min(float *sw, const NodeLine &nl, const DirLine &dl,
                                                 const LineSpec &ln, int lane,
                                                 const float (&tl)[4], float ns) {
    const float h128 = 128.0f * ln.h32;
    float fq = 0.0f, fx = 0.0f;
    float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
#pragma unroll 1
    for (int q = 0; q < ln.nfull; ++q, fq += 1.0f, fx += 128.0f) {
        float4 v;
        v.x = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[0]));
        v.y = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[1]));
        v.z = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[2]));
        v.w = sample_w<EK>(nl, dl, __fmaf_rn(h128, fq, tl[3]));
        *reinterpret_cast<float4 *>(sw + 128 * q + 4 * lane) = v;
        m0 = fminf(m0, __fmaf_rn(ns, fx, v.x));
        m1 = fminf(m1, __fmaf_rn(ns, fx, v.y));
        m2 = fminf(m2, __fmaf_rn(ns, fx, v.z));
        m3 = fminf(m3, __fmaf_rn(ns, fx, v.w));
    }
    float e = fminf(fminf(__fmaf_rn(ns, (float)(4 * lane - ln.m0), m0),
                          __fmaf_rn(ns, (float)(4 * lane + 1 - ln.m0), m1)),
                    fminf(__fmaf_rn(ns, (float)(4 * lane + 2 - ln.m0), m2),
                          __fmaf_rn(ns, (float)(4 * lane + 3 - ln.m0), m3)));
    for (int k = 128 * ln.nfull + lane; k < ln.L; k += 32) {
        const float v = sample_w<EK>(nl, dl, (float)(k - ln.m0) * ln.h32);
        sw[k] = v;
        e = fminf(e, __fmaf_rn(ns, (float)(k - ln.m0), v));
    }
    return e;
}

// sample_line_min for the damage energy on paired FP32 arithmetic: the same
// samples bit for bit.  The bound takes v - s x with the sample's own
// abscissa in one FMA (x exact), so each term has a single rounding, and it
// leaves the centre out: the result bounds from below the value at 0 of the
// hull of the left and right sets, which is the quantity the hull search
// bounds.  The chunk holding the centre is peeled so that only it pays for
// the mask.  With tail1 the line has one sample past its full chunks (the
// right end, L = 128 nfull + 1), computed beforehand by the caller (tv).
// c holds the line's constants in register pairs; nl and dl serve
// the scalar samples past the full chunks.
__device__ __forceinline__ float sample_line_min_nh(float *sw, const NodeLine &nl,
                                                    const NHPair &c, const DirLine &dl,
                                                    const LineSpec &ln, int lane,
                                                    const float (&tl)[4], float ns, bool tail1,
                                                    float tv) {
    const float h128 = 128.0f * ln.h32;
    const f32x2 H = pk2(h128, h128), TL01 = pk2(tl[0], tl[1]), TL23 = pk2(tl[2], tl[3]);
    const f32x2 NS = pk2(ns, ns), ONE = pk2(1.0f, 1.0f), STEP = pk2(128.0f, 128.0f);
    const float x0 = (float)(4 * lane - ln.m0);
    f32x2 FQ = pk2(0.0f, 0.0f), X01 = pk2(x0, x0 + 1.0f), X23 = pk2(x0 + 2.0f, x0 + 3.0f);
    float e = INFINITY;
    auto chunk = [&](int q, bool centre, bool lane0 = false) {
        const f32x2 V01 = sample_nh2(c, fma2(H, FQ, TL01));
        const f32x2 V23 = sample_nh2(c, fma2(H, FQ, TL23));
        float4 v;
        upk2(V01, v.x, v.y);
        upk2(V23, v.z, v.w);
        *reinterpret_cast<float4 *>(sw + 128 * q + 4 * lane) = v;
        float b0, b1, b2, b3;
        upk2(fma2(NS, X01, V01), b0, b1);
        upk2(fma2(NS, X23, V23), b2, b3);
        if (centre && lane0) {  // m0 = 128 q: the first sample of lane 0
            b0 = lane == 0 ? INFINITY : b0;
        } else if (centre) {
            const int ic = ln.m0 - 128 * q - 4 * lane;  // in [0, 4) on the lane holding m0
            b0 = ic == 0 ? INFINITY : b0;
            b1 = ic == 1 ? INFINITY : b1;
            b2 = ic == 2 ? INFINITY : b2;
            b3 = ic == 3 ? INFINITY : b3;
        }
        e = fmin3(e, b0, b1);
        e = fmin3(e, b2, b3);
        FQ = add2(FQ, ONE);
        X01 = add2(X01, STEP);
        X23 = add2(X23, STEP);
    };
    // L = 1025 and 2049 (centre in chunk nfull / 2): chunks unrolled at compile
    // time, so no loop counter, branch or address arithmetic per chunk
    auto unrolled = [&](auto nf) {
        constexpr int NF = decltype(nf)::value;
#pragma unroll
        for (int q = 0; q < NF; ++q) chunk(q, q == NF / 2, true);  // m0 = 64 NF
    };
    if (tail1 && ln.nfull == 8) {
        unrolled(std::integral_constant<int, 8>());
    } else if (tail1 && ln.nfull == 16) {
        unrolled(std::integral_constant<int, 16>());
    } else {
        const int qc = min(ln.m0 >> 7, ln.nfull);  // chunk of the centre (nfull: in the tail)
#pragma unroll 1
        for (int q = 0; q < qc; ++q) chunk(q, false);
        if (qc < ln.nfull) {
            chunk(qc, true);
#pragma unroll 1
            for (int q = qc + 1; q < ln.nfull; ++q) chunk(q, false);
        }
    }
    if (tail1) {
        if (lane == 0) sw[ln.L - 1] = tv;
        return fminf(e, __fmaf_rn(ns, (float)(ln.L - 1 - ln.m0), tv));
    }
    for (int k = 128 * ln.nfull + lane; k < ln.L; k += 32) {
        const float v = sample_w<CVX_ENERGY_NH_DAMAGE>(nl, dl, (float)(k - ln.m0) * ln.h32);
        sw[k] = v;
        if (k != ln.m0) e = fminf(e, __fmaf_rn(ns, (float)(k - ln.m0), v));
    }
    return e;
}

// Number of samples with J(t) > 0 on a line (the algorithmic work count).
__device__ __forceinline__ int valid_samples(const DirLine &dl, const LineSpec &ln, int energy) {
    if (energy != CVX_ENERGY_NH_DAMAGE || dl.cJ == 0.0f) return ln.L;
    const float xs = __fdividef(-dl.J0, dl.cJ * ln.h32);  // J = 0 at x = m - m0 = xs
    const float lim = (float)ln.L;
    if (dl.cJ > 0.0f) {  // valid for x > xs
        const float lo = fminf(fmaxf(floorf(xs) + 1.0f, -lim), lim);
        return max(0, min(ln.L, ln.m0 - max((int)lo, -ln.m0) + 1));
    }
    const float hi = fminf(fmaxf(ceilf(xs) - 1.0f, -lim), lim);  // valid for x < xs
    return max(0, min(ln.L, (int)hi + ln.m0 + 1));
}

}  // namespace cvx
