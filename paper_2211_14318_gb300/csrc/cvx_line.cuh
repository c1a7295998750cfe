// cvx_line.cuh -- sampling one rank-one line into a warp's shared buffer.
#pragma once

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
