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
