// cvx_kernels.cu -- kernels of the per-point rank-one convexification.
//
// Per lamination level (Eq. 3.3, top-down):
//   k_scan    FP32 screening: every direction's line is sampled (Eq. 4.4),
//             its exact FP32 hull bridge found (Algorithm 1 read at t = 0) and
//             the best directions kept per work item (the hot loop)
//   k_select  per node: the directions whose FP32 value lies within the
//             screening tolerance of the best (any other direction provably
//             loses in FP64), or none if the node provably does not split
//   k_refine  per candidate: the line resampled in FP64 and its bridge found
//             in FP64 -- the decisions whose stability needs it
//   k_commit  per node: minimum over directions in FP64 (Eq. 4.3), split into
//             F+- (Algorithm 2), next-level node queue
// and around them:
//   k_init    roots of the lamination trees, level-0 node queue
//   k_leaf    W^R and P over the tree leaves (Eq. 5.2, Algorithm 3)
//   k_energy, k_history, k_sample_lines, k_hull   single steps of the method
#include <cuda_runtime.h>
#include <limits.h>

#include "cvx_bridge.cuh"
#include "cvx_internal.h"

namespace cvx {

__device__ __forceinline__ void add_counter(unsigned long long *c, int idx, unsigned long long v) {
    if (v) atomicAdd(c + idx, v);
}

// -------------------------------------------------------------------------
// Sampling of one line into the warp's shared buffer: in chunk q lane l
// computes samples 128 q + 4 l + i (one 16-byte store); the tail past the
// last full chunk is one sample per lane.  tl[i] = (4 l + i - m0) h.
// -------------------------------------------------------------------------
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

// Sorted insertion into a warp's best list (uniform across the warp).
__device__ __forceinline__ void top_insert(float (&q)[kWarpTop], int (&d)[kWarpTop],
                                           float &dropped, float v, int dir) {
    if (!(v < q[kWarpTop - 1])) {
        dropped = fminf(dropped, v);
        return;
    }
    dropped = fminf(dropped, q[kWarpTop - 1]);
    int k = kWarpTop - 1;
#pragma unroll
    for (int i = kWarpTop - 1; i > 0; --i) {
        if (v < q[i - 1]) {
            q[i] = q[i - 1];
            d[i] = d[i - 1];
            k = i - 1;
        }
    }
    // place at the first slot whose predecessor is <= v
#pragma unroll
    for (int i = 0; i < kWarpTop; ++i)
        if (i == k) {
            q[i] = v;
            d[i] = dir;
        }
}

// -------------------------------------------------------------------------
// k_scan: persistent over work items (node, block of directions).  Each warp
// scans a contiguous run of directions, warm-starting every hull search from
// the previous direction's bridge, and keeps its best directions by q.
// -------------------------------------------------------------------------
// CTAs of 256 threads resident per SM that the register allocation targets
#ifndef CVX_SCAN_MIN_BLOCKS
#define CVX_SCAN_MIN_BLOCKS 3
#endif

template <int EK>
__global__ void __launch_bounds__(256, CVX_SCAN_MIN_BLOCKS) k_scan(const ScanArgs A) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const LineSpec ln = A.line;
    float *sw = reinterpret_cast<float *>(smem4) + warp * ln.stride;
    __shared__ NodeLine s_nl;
    __shared__ float s_q[16][kWarpTop];
    __shared__ int s_d[16][kWarpTop];
    __shared__ float s_drop[16], s_qhi[16];
    __shared__ int s_fl[16];
    __shared__ float s_w0;
    __shared__ unsigned s_hc[16][HC_N];

    const LineGeom g{ln.L, ln.m0, ln.nfull};
    float tl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tl[i] = (float)(4 * lane + i - ln.m0) * ln.h32;
    const int n_nodes = *A.q_count;
    const long long n_items = (long long)n_nodes * A.chunks;
    if (lane == 0)
        for (int i = 0; i < HC_N; ++i) s_hc[warp][i] = 0u;
    __syncwarp();
    HullCounters hc{s_hc[warp]};
    unsigned long long n_valid = 0, n_lines = 0;

    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int qi = (int)(item / A.chunks), ch = (int)(item % A.chunks);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int p = A.q_point[qi], hi = A.q_heap[qi];
            const cvx_node &nd = A.tree[(long long)p * A.NT + hi];
            double F[4] = {nd.F[0], nd.F[1], nd.F[2], nd.F[3]};
            s_nl = make_node_line(F, A.beta[p], A.mat);
        }
        __syncthreads();
        // the per-sample constants in registers; F and cof F stay in shared
        // memory and are read once per direction
        NodeLine nl;
        nl.A0 = s_nl.A0;
        nl.B1 = s_nl.B1;
        nl.B2 = s_nl.B2;
        nl.a1 = s_nl.a1;
        nl.K1 = s_nl.K1;
        nl.K2 = s_nl.K2;
        const int d0 = ch * A.dirs_per_item, d1 = min(A.D, d0 + A.dirs_per_item);
        const int per = (d1 - d0 + nw - 1) / nw;
        const int jb = d0 + warp * per, je = min(d1, jb + per);

        float tq[kWarpTop];
        int td[kWarpTop];
#pragma unroll
        for (int i = 0; i < kWarpTop; ++i) {
            tq[i] = INFINITY;
            td[i] = -1;
        }
        float dropped = INFINITY, w0 = 0.0f, qhi_min = INFINITY;
        int fl = 0;
        int warm_a = -1, warm_b = -1;
        for (int dj = jb; dj < je; ++dj) {
            const DirLine dl = make_dir_line<EK>(s_nl, A.dir32[dj]);
            sample_line<EK>(sw, nl, dl, ln, lane, tl);
            __syncwarp();
            const ScreenOut o = warp_screen(sw, g, lane, warm_a, warm_b, hc);
            __syncwarp();
            if (lane == 0) {
                ++n_lines;
                n_valid += valid_samples(dl, ln, EK);
            }
            w0 = o.w0;
            if (o.a >= 0) {
                warm_a = o.a;
                warm_b = o.b;
            }
            qhi_min = fminf(qhi_min, o.q_hi);
            top_insert(tq, td, dropped, o.q_lo, dj);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kWarpTop; ++i) {
                s_q[warp][i] = tq[i];
                s_d[warp][i] = td[i];
            }
            s_drop[warp] = dropped;
            s_qhi[warp] = qhi_min;
            s_fl[warp] = fl;
            if (jb < je) s_w0 = w0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // merge the warps' lists (ties -> lower direction index)
            ItemCands r;
            float drop = INFINITY, qhi = INFINITY;
            int f = 0;
            for (int k = 0; k < nw; ++k) {
                drop = fminf(drop, s_drop[k]);
                qhi = fminf(qhi, s_qhi[k]);
                f |= s_fl[k];
            }
            r.qhi_min = qhi;
            r.pad = 0;
            int taken[16];
            for (int k = 0; k < nw; ++k) taken[k] = 0;
            int n = 0;
            for (; n < kItemTop; ++n) {
                int bk = -1;
                for (int k = 0; k < nw; ++k) {
                    if (taken[k] >= kWarpTop || s_d[k][taken[k]] < 0) continue;
                    if (bk < 0 || s_q[k][taken[k]] < s_q[bk][taken[bk]] ||
                        (s_q[k][taken[k]] == s_q[bk][taken[bk]] &&
                         s_d[k][taken[k]] < s_d[bk][taken[bk]]))
                        bk = k;
                }
                if (bk < 0) break;
                r.q[n] = s_q[bk][taken[bk]];
                r.dir[n] = s_d[bk][taken[bk]];
                ++taken[bk];
            }
            for (int k = 0; k < nw; ++k)
                if (taken[k] < kWarpTop && s_d[k][taken[k]] >= 0) drop = fminf(drop, s_q[k][taken[k]]);
            for (int i = n; i < kItemTop; ++i) {
                r.q[i] = INFINITY;
                r.dir[i] = -1;
            }
            r.n = n;
            r.w0 = s_w0;
            r.dropped = drop;
            r.flags = f;
            A.out[item] = r;
        }
    }
    if (lane == 0) {
        const unsigned *c = hc.c;
        add_counter(A.counters, C_LINES, n_lines);
        add_counter(A.counters, C_VALID, n_valid);
        add_counter(A.counters, C_FP64, (unsigned long long)c[HC_FP64W] + c[HC_FP64R] + c[HC_FP64C]);
        add_counter(A.counters, C_FP64W, c[HC_FP64W]);
        add_counter(A.counters, C_FP64R, c[HC_FP64R]);
        add_counter(A.counters, C_FP64C, c[HC_FP64C]);
        add_counter(A.counters, C_FULL, c[HC_FULL]);
        add_counter(A.counters, C_RARE, c[HC_RARE]);
        add_counter(A.counters, C_CAPS, c[HC_CAPS]);
        add_counter(A.counters, C_WSTEPS, c[HC_WSTEPS]);
        add_counter(A.counters, C_ROUNDS, c[HC_ROUNDS]);
    }
}

static size_t scan_smem(int warps, int stride) { return (size_t)warps * stride * sizeof(float); }

template <int EK>
static cudaError_t launch_scan_t(const ScanArgs &a, int warps, int grid, cudaStream_t s) {
    const size_t smem = scan_smem(warps, a.line.stride);
    cudaError_t e = cudaFuncSetAttribute(k_scan<EK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_scan<EK><<<grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(const ScanArgs &a, int warps, int grid, cudaStream_t s) {
    return a.mat.energy == CVX_ENERGY_NH_DAMAGE
               ? launch_scan_t<CVX_ENERGY_NH_DAMAGE>(a, warps, grid, s)
               : launch_scan_t<CVX_ENERGY_DOUBLE_WELL>(a, warps, grid, s);
}

template <int EK>
static int occ_t(int warps, int stride) {
    const size_t smem = scan_smem(warps, stride);
    if (cudaFuncSetAttribute(k_scan<EK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan<EK>, warps * 32, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

int scan_max_blocks_per_sm(int energy, int warps, int stride) {
    return energy == CVX_ENERGY_NH_DAMAGE ? occ_t<CVX_ENERGY_NH_DAMAGE>(warps, stride)
                                          : occ_t<CVX_ENERGY_DOUBLE_WELL>(warps, stride);
}

// -------------------------------------------------------------------------
// k_select: one thread per queued node.  q is the FP32 value at t = 0 of a
// direction's left/right bridge chord and eps bounds |q_FP32 - q_FP64|
// (1-Lipschitz in the samples), q_lo <= q_R^FP32 <= q_hi per direction.  The
// node's FP64 value V = min(W(F), min_R q_R^FP64) is at most
// min(w0, min_R q_hi) + eps, so a direction with q_lo > min(w0, U) + 2 eps
// (U = min q_hi) can neither be the FP64 minimiser nor split the node, and if
// min q_lo > w0 + 2 eps no line splits.  The (at most kNodeCand) directions
// with the smallest q_lo inside that band are refined in FP64; k_commit checks
// that no unrefined direction (q_lo >= qcut) can win.
// -------------------------------------------------------------------------
__global__ void k_select(const SelectArgs A) {
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= *A.q_count) return;
    const ItemCands *r = A.items + (long long)qi * A.chunks;
    float qmin = INFINITY, drop = INFINITY, U = INFINITY;
    int fl = 0;
    const float w0 = r[0].w0;
    for (int c = 0; c < A.chunks; ++c) {
        qmin = fminf(qmin, r[c].q[0]);
        drop = fminf(drop, r[c].dropped);
        U = fminf(U, r[c].qhi_min);
        fl |= r[c].flags;
    }
    NodeCands nc;
    nc.n = 0;
    nc.eps = kEps32 * fmaxf(A.kappa, fmaxf(fabsf(qmin), fabsf(w0)));
    float qcut = drop;
    if (qmin <= w0 + 2.0f * nc.eps) {
        const float lim = fminf(w0, U) + 2.0f * nc.eps;
        // merge the items' sorted lists, smallest q first (ties: lower direction)
        int pos[64];
        const int nch = A.chunks < 64 ? A.chunks : 64;
        for (int c = 0; c < nch; ++c) pos[c] = 0;
        while (true) {
            int bc = -1;
            for (int c = 0; c < nch; ++c) {
                if (pos[c] >= r[c].n) continue;
                if (bc < 0 || r[c].q[pos[c]] < r[bc].q[pos[bc]] ||
                    (r[c].q[pos[c]] == r[bc].q[pos[bc]] && r[c].dir[pos[c]] < r[bc].dir[pos[bc]]))
                    bc = c;
            }
            if (bc < 0) break;
            const float q = r[bc].q[pos[bc]];
            if (!(q <= lim) || nc.n == kNodeCand) {
                qcut = fminf(qcut, q);
                break;
            }
            nc.dir[nc.n++] = r[bc].dir[pos[bc]];
            ++pos[bc];
        }
        for (int c = nch; c < A.chunks; ++c) qcut = fminf(qcut, r[c].q[0]);
    } else {
        qcut = qmin;
    }
    nc.qcut = qcut;
    nc.flags = fl;
    A.cands[qi] = nc;
    if (nc.n) {
        const int pos = atomicAdd(A.work_count, nc.n);
        for (int c = 0; c < nc.n; ++c) A.work[pos + c] = make_int2(qi, c);
        atomicAdd(A.counters + C_REFINED, (unsigned long long)nc.n);
    }
}

cudaError_t launch_select(const SelectArgs &a, int64_t max_nodes, cudaStream_t s) {
    if (max_nodes == 0) return cudaSuccess;
    k_select<<<(unsigned)((max_nodes + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// -------------------------------------------------------------------------
// FP64 bridge of the left and right sets of one line held in shared memory:
// supporting-slope iteration with full passes; ties go to the outermost sample
// (Algorithm 1 keeps the outermost of collinear points).
// -------------------------------------------------------------------------
__device__ __forceinline__ void warp_min_dk(double &v, int &k, bool prefer_low) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const double v2 = __shfl_xor_sync(kFull, v, o);
        const int k2 = __shfl_xor_sync(kFull, k, o);
        if (v2 < v || (v2 == v && (prefer_low ? k2 < k : k2 > k))) {
            v = v2;
            k = k2;
        }
    }
}

__device__ void bridge64(const double *sw, int L, int m0, int lane, int &a, int &b) {
    double s = 0.0;
    a = b = -1;
    for (int it = 0; it < 128; ++it) {
        double bl = INFINITY, br = INFINITY;
        int kl = INT_MAX, kr = -1;
        for (int k = lane; k < L; k += 32) {
            if (k == m0) continue;
            const double v = sw[k];
            if (!(v < INFINITY)) continue;
            const double e = v - s * (double)(k - m0);
            if (k < m0) {
                if (e < bl || (e == bl && k < kl)) { bl = e; kl = k; }
            } else if (e < br || (e == br && k > kr)) {
                br = e;
                kr = k;
            }
        }
        warp_min_dk(bl, kl, true);
        warp_min_dk(br, kr, false);
        if (kl == INT_MAX || kr < 0) {
            a = b = -1;
            return;
        }
        if (kl == a && kr == b) return;
        a = kl;
        b = kr;
        s = (sw[b] - sw[a]) / (double)(b - a);
    }
}

__global__ void __launch_bounds__(128) k_refine(const RefineArgs A) {
    extern __shared__ double sm64[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const LineSpec ln = A.line;
    double *sw = sm64 + warp * ln.stride;
    const int nwork = *A.work_count;
    for (int w = blockIdx.x * (blockDim.x >> 5) + warp; w < nwork;
         w += gridDim.x * (blockDim.x >> 5)) {
    const int2 wk = A.work[w];
    const int qi = wk.x, c = wk.y;
    const int p = A.q_point[qi], hi = A.q_heap[qi];
    const int dir = A.cands[qi].dir[c];
    const cvx_node &nd = A.tree[(long long)p * A.NT + hi];
    const double F[4] = {nd.F[0], nd.F[1], nd.F[2], nd.F[3]};
    const double *d = A.dir64 + 4 * (long long)dir;
    const double R[4] = {__dmul_rn(d[0], d[2]), __dmul_rn(d[0], d[3]), __dmul_rn(d[1], d[2]),
                         __dmul_rn(d[1], d[3])};
    const double beta = A.beta[p];
    for (int k = lane; k < ln.L; k += 32) sw[k] = sample_w64(F, R, k, ln.m0, ln.h64, beta, A.mat);
    __syncwarp();
    int a, b;
    bridge64(sw, ln.L, ln.m0, lane, a, b);
    if (lane == 0) {
        RefineOut o;
        o.a = a;
        o.b = b;
        o.pad = 0;
        if (a >= 0) {
            const double xa = (double)(a - ln.m0), xb = (double)(b - ln.m0);
            o.q = (xb * sw[a] - xa * sw[b]) / (xb - xa);
            o.ok = 1;
        } else {
            o.q = INFINITY;
            o.ok = 0;
        }
        A.out[(long long)qi * kNodeCand + c] = o;
    }
    __syncwarp();
    }
}

cudaError_t launch_refine(const RefineArgs &a, int64_t max_work, cudaStream_t s) {
    if (max_work == 0) return cudaSuccess;
    const int warps = 4;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (max_work + warps - 1) / warps;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    k_refine<<<grid, warps * 32, (size_t)warps * a.line.stride * sizeof(double), s>>>(a);
    return cudaGetLastError();
}

// -------------------------------------------------------------------------
// k_commit: one thread per queued node.  Split points in FP64 with explicit
// rounding (no contraction): t = (m - m0) h, F+- = F + t R, xi = (m0-m-)/(m+-m-).
// -------------------------------------------------------------------------
__global__ void k_commit(const CommitArgs A) {
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= *A.q_count) return;
    const int p = A.q_point[qi], hi = A.q_heap[qi];
    const NodeCands &nc = A.cands[qi];
    cvx_node &nd = A.tree[(long long)p * A.NT + hi];
    nd.flags |= CVX_NODE_SCANNED | (nc.flags & (CVX_NODE_ITER_CAP | CVX_NODE_OVERFLOW));
    atomicAdd(A.counters + C_NODES, 1ull);
    const RefineOut *ro = A.refined + (long long)qi * kNodeCand;
    int bc = -1;
    double second = INFINITY;
    for (int c = 0; c < nc.n; ++c) {
        if (!ro[c].ok) continue;
        if (bc < 0 || ro[c].q < ro[bc].q || (ro[c].q == ro[bc].q && nc.dir[c] < nc.dir[bc])) {
            if (bc >= 0) second = fmin(second, ro[bc].q);
            bc = c;
        } else {
            second = fmin(second, ro[c].q);
        }
    }
    const int m0 = A.line.m0;
    nd.gap = (float)(second - (bc >= 0 ? ro[bc].q : nd.w));
    // FP64 node value among the refined directions; an unrefined direction
    // (FP32 q >= qcut) could only win if qcut - eps reached it
    const double V = (bc >= 0 && ro[bc].q < nd.w) ? ro[bc].q : nd.w;
    if (!(((double)nc.qcut - (double)nc.eps) / A.kappa > V)) {
        nd.flags |= CVX_NODE_OVERFLOW;
        atomicAdd(A.counters + C_OVERFLOW, 1ull);
    }
    // the centre splits off iff the chord lies strictly below W(F) (FP64)
    if (bc < 0 || !(ro[bc].q < nd.w)) {
        nd.dir = bc >= 0 ? nc.dir[bc] : -1;
        nd.flags |= CVX_NODE_LEAF;
        return;
    }
    const RefineOut b = ro[bc];
    int fl = CVX_NODE_LAMINATED;
    if (b.a == 0 || b.b == A.line.L - 1) fl |= CVX_NODE_EDGE;
    if (second == b.q) {
        fl |= CVX_NODE_TIE;
        atomicAdd(A.counters + C_TIES, 1ull);
    }
    nd.flags |= fl;
    nd.dir = nc.dir[bc];
    nd.m_minus = b.a;
    nd.m_plus = b.b;
    nd.h = b.q;
    atomicAdd(A.counters + C_LAMINATED, 1ull);
    const double xi = (double)(m0 - b.a) / (double)(b.b - b.a);
    nd.xi = xi;
    const double *d = A.dir64 + 4 * (long long)nd.dir;
    const double R[4] = {__dmul_rn(d[0], d[2]), __dmul_rn(d[0], d[3]), __dmul_rn(d[1], d[2]),
                         __dmul_rn(d[1], d[3])};
    const double tm = __dmul_rn((double)(b.a - m0), A.line.h64);
    const double tp = __dmul_rn((double)(b.b - m0), A.line.h64);
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
        const int pos = atomicAdd(A.nq_count, 2);
        A.nq_point[pos] = p;
        A.nq_heap[pos] = 2 * hi + 1;
        A.nq_point[pos + 1] = p;
        A.nq_heap[pos + 1] = 2 * hi + 2;
    }
}

cudaError_t launch_commit(const CommitArgs &a, int64_t max_nodes, cudaStream_t s) {
    if (max_nodes == 0) return cudaSuccess;
    k_commit<<<(unsigned)((max_nodes + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
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
        const int pos = atomicAdd(A.q_count, 1);
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
    if (fl & CVX_NODE_OVERFLOW) st |= CVX_PT_OVERFLOW;
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
    float tl[4];
    for (int i = 0; i < 4; ++i) tl[i] = (float)(4 * lane + i - ln.m0) * ln.h32;
    sample_line<EK>(sw, nl, dl, ln, lane, tl);
    __syncwarp();
    const double kap = line_kappa(m);
    for (int k = lane; k < ln.L; k += 32) out[line * ln.L + k] = (float)((double)sw[k] / kap);
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
