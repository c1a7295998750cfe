// cvx_kernels.cu -- single steps of the method as their own kernels (the
// pipeline is in cvx_pipeline.cu): FP64 energy and stress (Eqs. 2.9, 2.12),
// history update (Eq. 2.5), the line scan's FP32 samples (Eq. 4.4) and the
// exact lower-hull bridge of given FP32 samples (Algorithm 1 read at t = 0).
#include <cuda_runtime.h>

#include "cvx_line.cuh"

namespace cvx {

// -------------------------------------------------------------------------
// Single steps: energy, history, line samples, hull bridge.
// -------------------------------------------------------------------------
__global__ void k_energy(int64_t n, const double *F, const double *beta, double *W, double *P,
                         Material m) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double G[4] = {F[4 * p], F[4 * p + 1], F[4 * p + 2], F[4 * p + 3]};
    W[p] = energy64(G, beta[p], m);
    if (P) {
        double Q[4];
        stress64(G, beta[p], m, Q);
        for (int k = 0; k < 4; ++k) P[4 * p + k] = Q[k];
    }
}

cudaError_t launch_energy(int64_t n, const double *F, const double *beta, double *W, double *P,
                          Material m, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_energy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, F, beta, W, P, m);
    return cudaGetLastError();
}

__global__ void k_history(int64_t n, const double *F, const double *bin, double *bout,
                          Material m) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double G[4] = {F[4 * p], F[4 * p + 1], F[4 * p + 2], F[4 * p + 3]};
    double lj, J;
    const double s = psi0_nh64(G, m, &lj, &J);
    const double b = bin ? bin[p] : 0.0;
    bout[p] = s > b ? s : b;
}

cudaError_t launch_history(int64_t n, const double *F, const double *bin, double *bout,
                           Material m, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_history<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, F, bin, bout, m);
    return cudaGetLastError();
}

// The kernel's own FP32 samples (kappa W), returned as W = sample / kappa.
template <int EK>
__global__ void __launch_bounds__(128) k_sample_lines(int64_t n, const double *F,
                                                      const double *beta, const int32_t *dir,
                                                      const float4 *dir32, int D, Material m,
                                                      LineSpec ln, float *out) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (line >= n) return;
    float *sw = reinterpret_cast<float *>(smem4) + warp * ln.stride;
    const int dj = dir[line];
    if (dj < 0 || dj >= D) {  // out-of-range direction index: NaN line
        for (int k = lane; k < ln.L; k += 32) out[line * ln.L + k] = __int_as_float(0x7fffffff);
        return;
    }
    double G[4] = {F[4 * line], F[4 * line + 1], F[4 * line + 2], F[4 * line + 3]};
    const NodeLine nl = make_node_line(G, beta[line], m);
    const DirLine dl = make_dir_line<EK>(nl, dir32[dj]);
    if (EK == CVX_ENERGY_NH_DAMAGE) {
        // the lane-per-line scan's samples: t = fl((m - m0) h)
        for (int k = lane; k < ln.L; k += 32)
            sw[k] = sample_w<EK>(nl, dl, __fmul_rn((float)(k - ln.m0), ln.h32));
    } else {
        float tl[4];
        for (int i = 0; i < 4; ++i) tl[i] = (float)(4 * lane + i - ln.m0) * ln.h32;
        sample_line<EK>(sw, nl, dl, ln, lane, tl);
    }
    __syncwarp();
    const double kap = line_kappa(m), shift = line_shift(m, beta[line]);
    for (int k = lane; k < ln.L; k += 32)
        out[line * ln.L + k] = (float)(((double)sw[k] + shift) / kap);
}

cudaError_t launch_sample_lines(int64_t n, const double *F, const double *beta,
                                const int32_t *dir, const float4 *dir32, int D, Material m,
                                LineSpec ln, float *w, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int warps = 4;
    const unsigned grid = (unsigned)((n + warps - 1) / warps);
    const size_t smem = (size_t)warps * ln.stride * sizeof(float);
    if (m.energy == CVX_ENERGY_NH_DAMAGE)
        k_sample_lines<CVX_ENERGY_NH_DAMAGE><<<grid, warps * 32, smem, s>>>(n, F, beta, dir, dir32,
                                                                           D, m, ln, w);
    else
        k_sample_lines<CVX_ENERGY_DOUBLE_WELL><<<grid, warps * 32, smem, s>>>(n, F, beta, dir,
                                                                             dir32, D, m, ln, w);
    return cudaGetLastError();
}

// Tangent of W^R over lamination trees (Algorithm 3 on second derivatives):
// the sum over the leaves of (path weight) d^2W/dFdF(F_leaf).
__global__ void k_tree_tangent(int64_t n, int NT, const cvx_node *tree, const double *beta,
                               Material m, double *A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const cvx_node *tr = tree + p * NT;
    double acc[16];
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    if (!(tr[0].flags & CVX_NODE_EXISTS) || !(tr[0].w == tr[0].w)) {
        for (int k = 0; k < 16; ++k) A[16 * p + k] = nan("");
        return;
    }
    for (int i = 0; i < NT; ++i) {
        const cvx_node &nd = tr[i];
        if (!(nd.flags & CVX_NODE_EXISTS) || (nd.flags & CVX_NODE_LAMINATED)) continue;
        const double F[4] = {nd.F[0], nd.F[1], nd.F[2], nd.F[3]};
        double Al[16];
        tangent64(F, beta[p], m, Al);
        for (int k = 0; k < 16; ++k) acc[k] += nd.weight * Al[k];
    }
    for (int k = 0; k < 16; ++k) A[16 * p + k] = acc[k];
}

cudaError_t launch_tree_tangent(int64_t n, int NT, const cvx_node *tree, const double *beta,
                                Material m, double *A, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_tree_tangent<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, NT, tree, beta, m, A);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128) k_hull(int64_t n, int L, const float *w_in, int32_t *mm,
                                              int32_t *mp, double *hv,
                                              unsigned long long *counters) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (line >= n) return;
    const int stride = line_stride(L);
    float *sw = reinterpret_cast<float *>(smem4) + warp * stride;
    for (int k = lane; k < L; k += 32) sw[k] = w_in[line * L + k];
    __syncwarp();
    const int m0 = (L - 1) / 2;
    const LineGeom g{L, m0, L >> 7};
    __shared__ unsigned s_hc[4][HC_N];
    if (lane == 0)
        for (int i = 0; i < HC_N; ++i) s_hc[warp][i] = 0u;
    __syncwarp();
    HullCounters hc{s_hc[warp]};
    const BridgeOut o = warp_bridge(sw, g, lane, -1, -1, hc);
    if (lane == 0) {
        mm[line] = o.lam ? o.a : m0;
        mp[line] = o.lam ? o.b : m0;
        if (o.lam) {
            const double xa = (double)(o.a - m0), xb = (double)(o.b - m0);
            hv[line] = (xb * (double)o.wa - xa * (double)o.wb) / (xb - xa);
        } else {
            hv[line] = (double)o.w0;
        }
        if (hc.c[HC_CAPS]) atomicAdd(counters + C_CAPS, (unsigned long long)hc.c[HC_CAPS]);
    }
}

cudaError_t launch_hull(int64_t n, int L, const float *w, int32_t *mm, int32_t *mp, double *h,
                        unsigned long long *counters, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int warps = 4;
    k_hull<<<(unsigned)((n + warps - 1) / warps), warps * 32,
             (size_t)warps * line_stride(L) * sizeof(float), s>>>(n, L, w, mm, mp, h, counters);
    return cudaGetLastError();
}

}  // namespace cvx
