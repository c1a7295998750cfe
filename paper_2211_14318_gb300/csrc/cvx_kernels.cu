// cvx_kernels.cu -- kernels of the per-point rank-one convexification.
//
//   k_init          roots of the lamination trees, level-0 node queue
//   k_scan          line sampling + exact hull bridge + min over directions
//                   (the hot loop: Eq. 4.4, Algorithm 1, Eq. 4.3)
//   k_expand        per node: best direction over work items, split into
//                   F+- (Eq. 3.3 / Algorithm 2), next-level node queue
//   k_leaf          W^R and P over the tree leaves (Eq. 5.2, Algorithm 3)
//   k_energy, k_history, k_sample_lines, k_hull   single steps of the method
#include <cuda_runtime.h>

#include "cvx_bridge.cuh"
#include "cvx_internal.h"

namespace cvx {

// -------------------------------------------------------------------------
// Sampling of one line into registers (slot j of lane l = sample 32 j + l)
// and into the warp's shared-memory copy.  Returns (on every lane) the number
// of finite samples.
// -------------------------------------------------------------------------
template <int NS, int EK>
__device__ __forceinline__ int sample_line(float (&w)[NS], float *sw, const NodeLine &nl,
                                           const DirLine &dl, const LineSpec &ln, int lane) {
    const float tl = (float)(lane - ln.m0) * ln.h32;
    const float h32x = 32.0f * ln.h32;
    int valid = 0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int k = 32 * j + lane;
        float v = __int_as_float(0x7fffffff);
        if (32 * j < ln.L) {
            const float t = __fmaf_rn(h32x, (float)j, tl);
            v = sample_w<EK>(nl, dl, t);
            if (k >= ln.L) v = __int_as_float(0x7fffffff);
            valid += __popc(__ballot_sync(kFull, v < INFINITY));
        }
        w[j] = v;
        sw[k] = v;
    }
    return valid;
}

__device__ __forceinline__ float h32_of(const BridgeOut &o, int m0, float *err) {
    if (!o.lam) {
        *err = 0.0f;
        return o.w0;
    }
    float xa = (float)(o.a - m0), xb = (float)(o.b - m0);
    float alpha = -xa / (xb - xa);
    *err = 6.0f * kU32 * (fabsf(o.wa) + fabsf(o.wb)) + 1e-30f;
    return o.wa + (o.wb - o.wa) * alpha;
}

__device__ __forceinline__ double h64_of(int lam, int a, int b, float wa, float wb, float w0,
                                         int m0) {
    if (!lam) return (double)w0;
    double xa = (double)(a - m0), xb = (double)(b - m0);
    return (xb * (double)wa - xa * (double)wb) / (xb - xa);
}

__device__ __forceinline__ void add_counter(unsigned long long *c, int idx, unsigned long long v) {
    if (v) atomicAdd(c + idx, v);
}

// -------------------------------------------------------------------------
// k_scan: persistent over work items (node, block of directions).  Each warp
// scans a contiguous run of directions (warm-starting every hull search from
// the previous direction's bridge), keeps its best line, and the CTA reduces
// the warps' bests in FP64 (ties -> lowest direction index).
// -------------------------------------------------------------------------
template <int NS, int EK>
__global__ void __launch_bounds__(512) k_scan(const ScanArgs A) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *sw = smem + warp * (NS * 32);
    __shared__ NodeLine s_nl;
    __shared__ double s_h[16];
    __shared__ float s_h32[16], s_h2[16];
    __shared__ int s_dir[16], s_mm[16], s_mp[16], s_fl[16];

    const LineSpec ln = A.line;
    const LineGeom g{ln.L, ln.m0, ln.m0 >> 5, ln.m0 & 31};
    const int n_nodes = *A.q_count;
    const long long n_items = (long long)n_nodes * A.chunks;
    HullCounters hc{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    unsigned long long n_valid = 0, n_lines = 0, n_dir64 = 0;

    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int qi = (int)(item / A.chunks), ch = (int)(item % A.chunks);
        const int p = A.q_point[qi], hi = A.q_heap[qi];
        __syncthreads();
        if (threadIdx.x == 0) {
            const cvx_node &nd = A.tree[(long long)p * A.NT + hi];
            double F[4] = {nd.F[0], nd.F[1], nd.F[2], nd.F[3]};
            s_nl = make_node_line(F, A.beta[p], A.mat);
        }
        __syncthreads();
        const NodeLine nl = s_nl;
        const int d0 = ch * A.dirs_per_item, d1 = min(A.D, d0 + A.dirs_per_item);
        const int per = (d1 - d0 + nw - 1) / nw;
        const int jb = d0 + warp * per, je = min(d1, jb + per);

        float b_h32 = INFINITY, b_err = 0.0f, b_h2 = INFINITY, b_wa = 0.0f, b_wb = 0.0f;
        float w0 = 0.0f;
        int b_dir = -1, b_a = ln.m0, b_b = ln.m0, b_lam = 0, b_fl = 0;
        int warm_a = -1, warm_b = -1;
        for (int dj = jb; dj < je; ++dj) {
            const DirLine dl = make_dir_line<EK>(nl, A.dir32[dj]);
            float w[NS];
            n_valid += sample_line<NS, EK>(w, sw, nl, dl, ln, lane);
            __syncwarp();
            const unsigned caps0 = hc.caps;
            const BridgeOut o = warp_bridge<NS>(w, sw, g, lane, warm_a, warm_b, hc);
            __syncwarp();
            ++n_lines;
            w0 = o.w0;
            if (o.a >= 0) {
                warm_a = o.a;
                warm_b = o.b;
            }
            float err;
            const float h32 = h32_of(o, ln.m0, &err);
            bool better;
            if (b_dir < 0) better = true;
            else if (h32 + err < b_h32 - b_err) better = true;
            else if (h32 - err > b_h32 + b_err) better = false;
            else {
                ++n_dir64;
                double hn = h64_of(o.lam, o.a, o.b, o.wa, o.wb, o.w0, ln.m0);
                double hb = h64_of(b_lam, b_a, b_b, b_wa, b_wb, w0, ln.m0);
                better = hn < hb;  // equal -> keep the lower direction index
            }
            const int fl = (__shfl_sync(kFull, hc.caps, 0) != __shfl_sync(kFull, caps0, 0))
                               ? CVX_NODE_ITER_CAP : 0;
            if (better) {
                b_h2 = fminf(b_h2, b_h32);
                b_h32 = h32;
                b_err = err;
                b_dir = dj;
                b_lam = o.lam;
                b_a = o.lam ? o.a : ln.m0;
                b_b = o.lam ? o.b : ln.m0;
                b_wa = o.wa;
                b_wb = o.wb;
                b_fl = fl;
            } else {
                b_h2 = fminf(b_h2, h32);
            }
        }
        if (lane == 0) {
            s_h[warp] = b_dir >= 0 ? h64_of(b_lam, b_a, b_b, b_wa, b_wb, w0, ln.m0) : INFINITY;
            s_h32[warp] = b_h32;
            s_h2[warp] = b_h2;
            s_dir[warp] = b_dir;
            s_mm[warp] = b_a;
            s_mp[warp] = b_b;
            s_fl[warp] = b_fl;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int bw = -1;
            for (int k = 0; k < nw; ++k) {
                if (s_dir[k] < 0) continue;
                if (bw < 0 || s_h[k] < s_h[bw] || (s_h[k] == s_h[bw] && s_dir[k] < s_dir[bw])) bw = k;
            }
            ItemBest r;
            if (bw < 0) {
                r.h = INFINITY;
                r.h32 = INFINITY;
                r.h2 = INFINITY;
                r.dir = -1;
                r.mm = r.mp = ln.m0;
                r.flags = 0;
            } else {
                float sec = s_h2[bw];
                int fl = 0;
                for (int k = 0; k < nw; ++k) {
                    if (s_dir[k] < 0) continue;
                    fl |= s_fl[k];
                    if (k != bw) sec = fminf(sec, fminf(s_h32[k], s_h2[k]));
                }
                r.h = s_h[bw];
                r.h32 = s_h32[bw];
                r.h2 = sec;
                r.dir = s_dir[bw];
                r.mm = s_mm[bw];
                r.mp = s_mp[bw];
                r.flags = fl;
            }
            A.out[item] = r;
        }
    }
    // counters: per-lane FP64 checks summed, warp-uniform ones from lane 0
    unsigned fp64 = __reduce_add_sync(kFull, hc.fp64);
    unsigned fp64r = __reduce_add_sync(kFull, hc.fp64r);
    if (lane == 0) {
        add_counter(A.counters, C_FP64W, fp64);
        add_counter(A.counters, C_FP64R, fp64r);
        add_counter(A.counters, C_FP64C, hc.fp64c);
        add_counter(A.counters, C_WSTEPS, hc.wsteps);
        add_counter(A.counters, C_ROUNDS, hc.rounds);
        add_counter(A.counters, C_DIR64, n_dir64);
        add_counter(A.counters, C_LINES, n_lines);
        add_counter(A.counters, C_VALID, n_valid);
        add_counter(A.counters, C_FP64, fp64 + fp64r + hc.fp64c);
        add_counter(A.counters, C_FULL, hc.full_passes);
        add_counter(A.counters, C_RARE, hc.rare);
        add_counter(A.counters, C_CAPS, hc.caps);
    }
}

template <int NS, int EK>
static cudaError_t launch_scan_t(const ScanArgs &a, int warps, int grid, cudaStream_t s) {
    const size_t smem = (size_t)warps * NS * 32 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_scan<NS, EK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_scan<NS, EK><<<grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NS, int EK>
static int occ_t(int warps) {
    const size_t smem = (size_t)warps * NS * 32 * sizeof(float);
    cudaFuncSetAttribute(k_scan<NS, EK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan<NS, EK>, warps * 32, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_scan(const ScanArgs &a, int energy, int ns, int warps, int grid,
                        cudaStream_t s) {
#define SC(N)                                                                          \
    case N:                                                                            \
        return energy == CVX_ENERGY_NH_DAMAGE                                          \
                   ? launch_scan_t<N, CVX_ENERGY_NH_DAMAGE>(a, warps, grid, s)         \
                   : launch_scan_t<N, CVX_ENERGY_DOUBLE_WELL>(a, warps, grid, s);
    switch (ns) {
        SC(8)
        SC(17)
        SC(33)
        SC(65)
    default: return cudaErrorInvalidValue;
    }
#undef SC
}

int scan_max_blocks_per_sm(int energy, int ns, int warps) {
#define OCC(N)                                                                              \
    case N:                                                                                 \
        return energy == CVX_ENERGY_NH_DAMAGE ? occ_t<N, CVX_ENERGY_NH_DAMAGE>(warps)       \
                                              : occ_t<N, CVX_ENERGY_DOUBLE_WELL>(warps);
    switch (ns) {
        OCC(8)
        OCC(17)
        OCC(33)
        OCC(65)
    default: return 0;
    }
#undef OCC
}

// -------------------------------------------------------------------------
// k_init: one thread per point.
// -------------------------------------------------------------------------
__global__ void k_init(const InitArgs A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x == 0) {
        const int64_t left = A.n - (int64_t)blockIdx.x * blockDim.x;
        atomicAdd(A.counters + C_POINTS,
                  (unsigned long long)(left < (int64_t)blockDim.x ? left : blockDim.x));
    }
    if (p >= A.n) return;
    const double *Fp = A.F + 4 * p;
    double F[4] = {Fp[0], Fp[1], Fp[2], Fp[3]};
    const double J = F[0] * F[3] - F[1] * F[2];
    const bool ok = A.mat.energy == CVX_ENERGY_DOUBLE_WELL || J > 0.0;
    cvx_node &nd = A.tree[p * A.NT];
    for (int k = 0; k < 4; ++k) nd.F[k] = F[k];
    nd.weight = 1.0;
    nd.xi = 0.0;
    nd.dir = -1;
    nd.m_minus = nd.m_plus = A.m0;
    nd.gap = 0.0f;
    nd.pad = 0;
    if (!ok) {
        nd.w = nan("");
        nd.h = nd.w;
        nd.flags = 0;
        A.status[p] = CVX_PT_NONPOS_DET;
        return;
    }
    nd.w = energy64(F, A.beta[p], A.mat);
    nd.h = nd.w;
    A.status[p] = CVX_PT_OK;
    if (A.depth == 0) {
        nd.flags = CVX_NODE_EXISTS | CVX_NODE_LEAF;
    } else {
        nd.flags = CVX_NODE_EXISTS;
        int pos = atomicAdd(A.q_count, 1);
        A.q_point[pos] = (int32_t)p;
        A.q_heap[pos] = 0;
    }
}

cudaError_t launch_init(const InitArgs &a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_init<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// -------------------------------------------------------------------------
// k_expand: one thread per queued node.  Split points in FP64 with explicit
// rounding (no contraction): t = (m - m0) h, F+- = F + t R, xi = (m0-m-)/(m+-m-).
// -------------------------------------------------------------------------
__global__ void k_expand(const ExpandArgs A) {
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= *A.q_count) return;
    const int p = A.q_point[qi], hi = A.q_heap[qi];
    const ItemBest *r = A.items + (long long)qi * A.chunks;
    int bi = -1;
    for (int c = 0; c < A.chunks; ++c) {
        if (r[c].dir < 0) continue;
        if (bi < 0 || r[c].h < r[bi].h || (r[c].h == r[bi].h && r[c].dir < r[bi].dir)) bi = c;
    }
    cvx_node &nd = A.tree[(long long)p * A.NT + hi];
    nd.flags |= CVX_NODE_SCANNED;
    atomicAdd(A.counters + C_NODES, 1ull);
    if (bi < 0) {
        nd.flags |= CVX_NODE_LEAF;
        return;
    }
    const ItemBest b = r[bi];
    float sec = b.h2;
    for (int c = 0; c < A.chunks; ++c)
        if (c != bi && r[c].dir >= 0) sec = fminf(sec, fminf(r[c].h32, r[c].h2));
    const int m0 = A.line.m0;
    nd.dir = b.dir;
    nd.m_minus = b.mm;
    nd.m_plus = b.mp;
    nd.h = b.h;
    nd.gap = sec - b.h32;
    int fl = b.flags & CVX_NODE_ITER_CAP;
    // FP32 sampling error is a few units of 2^-24 relative to |W|: two
    // directions closer than 32 u |W| are reported as a tie (warning only).
    const float tol = 32.0f * kU32 * (fabsf((float)b.h) + fabsf((float)nd.w) + 1e-3f);
    if (nd.gap <= tol) {
        fl |= CVX_NODE_TIE;
        atomicAdd(A.counters + C_TIES, 1ull);
    }
    if (b.mm == m0) {
        nd.flags |= fl | CVX_NODE_LEAF;
        return;
    }
    fl |= CVX_NODE_LAMINATED;
    if (b.mm == 0 || b.mp == A.line.L - 1) fl |= CVX_NODE_EDGE;
    nd.flags |= fl;
    atomicAdd(A.counters + C_LAMINATED, 1ull);
    const double xi = (double)(m0 - b.mm) / (double)(b.mp - b.mm);
    nd.xi = xi;
    const double *d = A.dir64 + 4 * (long long)b.dir;
    const double R[4] = {__dmul_rn(d[0], d[2]), __dmul_rn(d[0], d[3]), __dmul_rn(d[1], d[2]),
                         __dmul_rn(d[1], d[3])};
    const double tm = __dmul_rn((double)(b.mm - m0), A.line.h64);
    const double tp = __dmul_rn((double)(b.mp - m0), A.line.h64);
    const bool leaf_children = A.level + 1 >= A.depth;
    const double beta = A.beta[p];
    for (int side = 0; side < 2; ++side) {
        const int ci = 2 * hi + 1 + side;  // 2i+1: F-, 2i+2: F+
        cvx_node &c = A.tree[(long long)p * A.NT + ci];
        const double t = side ? tp : tm;
        double F[4];
        for (int k = 0; k < 4; ++k) F[k] = __dadd_rn(nd.F[k], __dmul_rn(t, R[k]));
        for (int k = 0; k < 4; ++k) c.F[k] = F[k];
        c.weight = side ? __dmul_rn(nd.weight, xi) : __dmul_rn(nd.weight, __dsub_rn(1.0, xi));
        c.w = energy64(F, beta, A.mat);
        c.h = c.w;
        c.xi = 0.0;
        c.dir = -1;
        c.m_minus = c.m_plus = m0;
        c.gap = 0.0f;
        c.pad = 0;
        c.flags = CVX_NODE_EXISTS | (leaf_children ? CVX_NODE_LEAF : 0);
    }
    if (!leaf_children) {
        int pos = atomicAdd(A.nq_count, 2);
        A.nq_point[pos] = p;
        A.nq_heap[pos] = 2 * hi + 1;
        A.nq_point[pos + 1] = p;
        A.nq_heap[pos + 1] = 2 * hi + 2;
    }
}

cudaError_t launch_expand(const ExpandArgs &a, int64_t max_nodes, cudaStream_t s) {
    if (max_nodes == 0) return cudaSuccess;
    k_expand<<<(unsigned)((max_nodes + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// -------------------------------------------------------------------------
// k_leaf: W^R = sum over leaves of (path weight) W(F_leaf), same for P
// (Algorithm 3 with the recursion unrolled over the heap).
// -------------------------------------------------------------------------
__global__ void k_leaf(const LeafArgs A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.n) return;
    const cvx_node *tr = A.tree + p * A.NT;
    int st = A.status[p];
    if (st & CVX_PT_NONPOS_DET) {
        A.W_R[p] = nan("");
        for (int k = 0; k < 4; ++k) A.P[4 * p + k] = nan("");
        if (A.root) {
            cvx_laminate z = {};
            z.dir = -1;
            A.root[p] = z;
        }
        return;
    }
    const double beta = A.beta[p];
    double W = 0.0, P[4] = {0.0, 0.0, 0.0, 0.0};
    int fl = 0;
    for (int i = 0; i < A.NT; ++i) {
        const cvx_node &nd = tr[i];
        if (!(nd.flags & CVX_NODE_EXISTS)) continue;
        fl |= nd.flags;
        if (nd.flags & CVX_NODE_LAMINATED) continue;
        double F[4] = {nd.F[0], nd.F[1], nd.F[2], nd.F[3]};
        double Pl[4];
        stress64(F, beta, A.mat, Pl);
        W += nd.weight * energy64(F, beta, A.mat);
        for (int k = 0; k < 4; ++k) P[k] += nd.weight * Pl[k];
    }
    A.W_R[p] = W;
    for (int k = 0; k < 4; ++k) A.P[4 * p + k] = P[k];
    if (fl & CVX_NODE_TIE) st |= CVX_PT_TIE;
    if (fl & CVX_NODE_EDGE) st |= CVX_PT_EDGE;
    if (fl & CVX_NODE_ITER_CAP) st |= CVX_PT_ITER_CAP;
    A.status[p] = st;
    if (A.root) {
        cvx_laminate L;
        const cvx_node &r0 = tr[0];
        L.laminated = (r0.flags & CVX_NODE_LAMINATED) ? 1 : 0;
        L.dir = r0.dir;
        L.m_minus = r0.m_minus;
        L.m_plus = r0.m_plus;
        L.xi = r0.xi;
        L.h = r0.h;
        for (int k = 0; k < 4; ++k) {
            L.F_plus[k] = L.laminated ? tr[2].F[k] : r0.F[k];
            L.F_minus[k] = L.laminated ? tr[1].F[k] : r0.F[k];
        }
        A.root[p] = L;
    }
}

cudaError_t launch_leaf(const LeafArgs &a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_leaf<<<(unsigned)((a.n + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

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
    double s = psi0_nh64(G, m, &lj, &J);
    double b = bin ? bin[p] : 0.0;
    bout[p] = s > b ? s : b;
}

cudaError_t launch_history(int64_t n, const double *F, const double *bin, double *bout,
                           Material m, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_history<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, F, bin, bout, m);
    return cudaGetLastError();
}

template <int NS, int EK>
__global__ void __launch_bounds__(128) k_sample_lines(int64_t n, const double *F,
                                                      const double *beta, const int32_t *dir,
                                                      const float4 *dir32, int D, Material m,
                                                      LineSpec ln, float *out) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (line >= n) return;
    float *sw = smem + warp * NS * 32;
    const int dj = dir[line];
    if (dj < 0 || dj >= D) {  // out-of-range direction index: NaN line
        for (int k = lane; k < ln.L; k += 32) out[line * ln.L + k] = __int_as_float(0x7fffffff);
        return;
    }
    double G[4] = {F[4 * line], F[4 * line + 1], F[4 * line + 2], F[4 * line + 3]};
    const NodeLine nl = make_node_line(G, beta[line], m);
    const DirLine dl = make_dir_line<EK>(nl, dir32[dj]);
    float w[NS];
    sample_line<NS, EK>(w, sw, nl, dl, ln, lane);
    for (int k = lane; k < ln.L; k += 32) out[line * ln.L + k] = sw[k];
}

template <int NS, int EK>
static cudaError_t launch_sample_t(int64_t n, const double *F, const double *beta,
                                   const int32_t *dir, const float4 *dir32, int D, Material m,
                                   LineSpec ln, float *w, cudaStream_t s) {
    const int warps = 4;
    k_sample_lines<NS, EK><<<(unsigned)((n + warps - 1) / warps), warps * 32,
                             warps * NS * 32 * sizeof(float), s>>>(n, F, beta, dir, dir32, D, m,
                                                                   ln, w);
    return cudaGetLastError();
}

cudaError_t launch_sample_lines(int64_t n, const double *F, const double *beta,
                                const int32_t *dir, const float4 *dir32, int D, Material m,
                                LineSpec line, int ns, float *w, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
#define SL(N)                                                                                 \
    case N:                                                                                   \
        return m.energy == CVX_ENERGY_NH_DAMAGE                                               \
                   ? launch_sample_t<N, CVX_ENERGY_NH_DAMAGE>(n, F, beta, dir, dir32, D, m, line, \
                                                              w, s)                           \
                   : launch_sample_t<N, CVX_ENERGY_DOUBLE_WELL>(n, F, beta, dir, dir32, D, m,     \
                                                                line, w, s);
    switch (ns) {
        SL(8)
        SL(17)
        SL(33)
        SL(65)
    default: return cudaErrorInvalidValue;
    }
#undef SL
}

template <int NS>
__global__ void __launch_bounds__(128) k_hull(int64_t n, int L, const float *w_in, int32_t *mm,
                                              int32_t *mp, double *hv,
                                              unsigned long long *counters) {
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t line = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (line >= n) return;
    float *sw = smem + warp * NS * 32;
    float w[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int k = 32 * j + lane;
        float v = k < L ? w_in[line * L + k] : __int_as_float(0x7fffffff);
        w[j] = v;
        sw[k] = v;
    }
    __syncwarp();
    const int m0 = (L - 1) / 2;
    const LineGeom g{L, m0, m0 >> 5, m0 & 31};
    HullCounters hc{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    const BridgeOut o = warp_bridge<NS>(w, sw, g, lane, -1, -1, hc);
    if (lane == 0) {
        mm[line] = o.lam ? o.a : m0;
        mp[line] = o.lam ? o.b : m0;
        hv[line] = h64_of(o.lam, o.a, o.b, o.wa, o.wb, o.w0, m0);
        if (hc.caps) atomicAdd(counters + C_CAPS, (unsigned long long)hc.caps);
    }
}

cudaError_t launch_hull(int64_t n, int L, int ns, const float *w, int32_t *mm, int32_t *mp,
                          double *h, unsigned long long *counters, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int warps = 4;
    const unsigned grid = (unsigned)((n + warps - 1) / warps);
#define HL(N)                                                                            \
    case N:                                                                              \
        k_hull<N><<<grid, warps * 32, warps * N * 32 * sizeof(float), s>>>(n, L, w, mm, mp, h, \
                                                                           counters);    \
        return cudaGetLastError();
    switch (ns) {
        HL(8)
        HL(17)
        HL(33)
        HL(65)
    default: return cudaErrorInvalidValue;
    }
#undef HL
}

}  // namespace cvx
