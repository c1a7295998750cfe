// cvx_pipeline.cu -- the per-point convexification pipeline over any number
// of problems (convexify_points is a batch of one).
//
// Per lamination level (Eq. 3.3, top-down):
//   k_scan    FP32 screening: every direction's line is sampled (Eq. 4.4),
//             bounds on its hull value at t = 0 (Algorithm 1 read at t = 0)
//             are found and the best directions kept per work item -- the hot
//             loop; work items are handed out by an atomic counter
//   k_select  per node: the directions whose FP32 bound lies within the
//             screening band of the best (any other direction provably loses
//             in FP64), or none if the node provably does not split
//   k_refine  per candidate: the line resampled in FP64 and its bridge found
//             in FP64 -- the decisions whose stability needs it
//   k_commit  per node: minimum over directions in FP64 (Eq. 4.3), split into
//             F+- (Algorithm 2), next-level node queue
// around them:
//   k_init    problem of each point, roots of the lamination trees, level-0 queue
//   k_leaf    W^R and P over the tree leaves (Eq. 5.2, Algorithm 3)
#include <cuda_runtime.h>
#include <limits.h>

#include "cvx_line.cuh"

namespace cvx {

__device__ __forceinline__ void add_counter(unsigned long long *c, int idx, unsigned long long v) {
    if (v) atomicAdd(c + idx, v);
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
#pragma unroll
    for (int i = 0; i < kWarpTop; ++i)
        if (i == k) {
            q[i] = v;
            d[i] = dir;
        }
}

// Global direction index of entry j of a node's proposal window: row-major
// over (da, db) in [-w, w]^2 around the centre (ia, ib) of the Na x Nb grid.
__device__ __forceinline__ int window_dir(const ProbDesc &pd, int2 c, int j) {
    const int s = 2 * pd.window + 1;
    int i = (c.x + j / s - pd.window) % pd.Na;
    int k = (c.y + j % s - pd.window) % pd.Nb;
    if (i < 0) i += pd.Na;
    if (k < 0) k += pd.Nb;
    return i * pd.Nb + k;
}

__device__ __forceinline__ int pass_chunks(const ProbDesc &pd, int pass) {
    return pass == PASS_WINDOW ? pd.wchunks : pd.chunks;
}

// -------------------------------------------------------------------------
// k_init: one thread per point of any problem.
// -------------------------------------------------------------------------
__global__ void k_init(const Pipe P) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x == 0) {
        const long long left = P.N - (long long)blockIdx.x * blockDim.x;
        atomicAdd(P.counters + C_POINTS,
                  (unsigned long long)(left < (long long)blockDim.x ? left : blockDim.x));
    }
    if (p >= P.N) return;
    int lo = 0, hi = P.n_probs - 1;  // problems are sorted by point_off
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.probs[mid].point_off <= p) lo = mid;
        else hi = mid - 1;
    }
    P.pid[p] = lo;
    const ProbDesc &pd = P.probs[lo];
    const long long lp = p - pd.point_off;
    cvx_node *tr = node_ptr(pd, p, 0);
    for (int i = 1; i < pd.NT; ++i) {  // unused nodes read as zero
        cvx_node z = {};
        tr[i] = z;
    }
    const double *Fp = pd.F + 4 * lp;
    double F[4] = {Fp[0], Fp[1], Fp[2], Fp[3]};
    const double J = F[0] * F[3] - F[1] * F[2];
    const bool ok = pd.mat.energy == CVX_ENERGY_DOUBLE_WELL || J > 0.0;
    cvx_node nd = {};
    for (int k = 0; k < 4; ++k) nd.F[k] = F[k];
    nd.weight = 1.0;
    nd.dir = -1;
    nd.m_minus = nd.m_plus = pd.line.m0;
    if (!ok) {
        nd.w = nan("");
        nd.h = nd.w;
        tr[0] = nd;
        pd.status[lp] = CVX_PT_NONPOS_DET;
        return;
    }
    nd.w = energy64(F, pd.beta[lp], pd.mat);
    nd.h = nd.w;
    pd.status[lp] = CVX_PT_OK;
    if (pd.K == 0) {
        nd.flags = CVX_NODE_EXISTS | CVX_NODE_LEAF;
        tr[0] = nd;
    } else {
        nd.flags = CVX_NODE_EXISTS;
        tr[0] = nd;
        const int pos = atomicAdd(P.cnt, 1);
        P.qp[0][pos] = (int32_t)p;
        P.qh[0][pos] = 0;
    }
}

// -------------------------------------------------------------------------
// k_scan: persistent CTAs take work items (node, block of directions) from an
// atomic counter.  Each warp scans a contiguous run of directions,
// warm-starting every hull search from the previous direction's bridge, and
// keeps its best directions by their lower bound.
// -------------------------------------------------------------------------
#ifndef CVX_SCAN_MIN_BLOCKS
#define CVX_SCAN_MIN_BLOCKS 4  // CTAs of 256 threads per SM the registers target
#endif

constexpr int kScanWarps = 8;  // warps per line-scan CTA at most (256 threads)

template <int EK>
__global__ void __launch_bounds__(32 * kScanWarps, CVX_SCAN_MIN_BLOCKS) k_scan(const Pipe P, int level) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float *sw = reinterpret_cast<float *>(smem4) + warp * P.stride32;
    __shared__ NodeLine s_nl;
    __shared__ ProbDesc s_pd;
    __shared__ long long s_item;
    // per-warp arrays: at most kScanWarps warps (the launch bound)
    __shared__ float s_q[kScanWarps][kWarpTop];
    __shared__ int s_d[kScanWarps][kWarpTop];
    __shared__ float s_drop[kScanWarps], s_qhi[kScanWarps];
    __shared__ float s_w0;
    __shared__ float s_shift;  // the point's sample shift C
    __shared__ float s_sa, s_cb;  // centre-slope constants of the node (damage energy)
    __shared__ int s_e;           // the node's window exponent
    __shared__ int s_ukey;     // smallest q_hi screened so far in this item (f2key order)
    __shared__ int2 s_c;
    __shared__ unsigned s_hc[kScanWarps][HC_N];
    // damage energy, a warp's next 32 lines: (A1, A1, A2, A2) and
    // (cof F : R, cof F : R, tangent slope at t = 0, right-end sample)
    __shared__ float4 s_dir[kScanWarps][32][2];
    const bool win = P.pass == PASS_WINDOW;

    const int n_nodes = P.cnt[level];
    const long long n_items = (long long)n_nodes * P.C;
    const int32_t *qp = P.qp[level], *qh = P.qh[level];
    if (lane == 0)
        for (int i = 0; i < HC_N; ++i) s_hc[warp][i] = 0u;
    __syncwarp();
    HullCounters hc{s_hc[warp]};
    unsigned long long n_valid = 0, n_lines = 0;
    unsigned n_bounded = 0, n_flat = 0;  // warp-uniform, reported by lane 0

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long item = (long long)atomicAdd(P.item_ctr + level, 1ull);
            s_item = item;
            if (item < n_items) {
                const int qi = (int)(item / P.C), ch = (int)(item % P.C);
                const int p = qp[qi], hi = qh[qi];
                s_pd = P.probs[P.pid[p]];
                if (win) s_c = P.center[qi];
                if (ch < pass_chunks(s_pd, P.pass)) {
                    const cvx_node *nd = node_ptr(s_pd, p, hi);
                    double F[4] = {nd->F[0], nd->F[1], nd->F[2], nd->F[3]};
                    const double beta = s_pd.beta[p - s_pd.point_off];
                    s_nl = make_node_line(F, beta, s_pd.mat);
                    s_shift = (float)line_shift(s_pd.mat, beta);
                    s_ukey = f2key(INFINITY);
                    s_e = nd->window_exp;
                    if (EK == CVX_ENERGY_NH_DAMAGE)
                        center_slope_consts(s_nl, scaled_line(s_pd.line, s_e).h64, s_sa, s_cb);
                }
            }
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= n_items) break;
        const int ch = (int)(item % P.C);
        if (ch >= pass_chunks(s_pd, P.pass)) continue;
        const LineSpec ln = scaled_line(s_pd.line, s_e);
        const LineGeom g{ln.L, ln.m0, ln.nfull};
        float tl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) tl[i] = (float)(4 * lane + i - ln.m0) * ln.h32;
        // the per-sample constants in registers; F and cof F stay in shared
        // memory and are read once per direction
        NodeLine nl;
        nl.A0 = s_nl.A0;
        nl.B1 = s_nl.B1;
        nl.B2 = s_nl.B2;
        nl.K1 = s_nl.K1;
        nl.K2 = s_nl.K2;
        const int D = win ? s_pd.wD : s_pd.D, doff = s_pd.dir_off;
        const int dpi = win ? s_pd.wdpi : s_pd.dpi;
        const int2 cen = s_c;
        const int d0 = ch * dpi, d1 = min(D, d0 + dpi);
        // the item's directions in segments of up to 16 contiguous ones, dealt
        // to the warps in turn: the lines that need a hull search cluster
        // around the split direction, and this spreads them over the warps
        // (the first search of a segment starts far from its bridge; the
        // search runs until its pair is certified, kScreenRounds)
        const int seg = max(1, min(16, (d1 - d0 + nw - 1) / nw));
        const int nseg = (d1 - d0 + seg - 1) / seg;

        float tq[kWarpTop];
        int td[kWarpTop];
#pragma unroll
        for (int i = 0; i < kWarpTop; ++i) {
            tq[i] = INFINITY;
            td[i] = -1;
        }
        float dropped = INFINITY, w0 = 0.0f, qhi_min = INFINITY;
        int warm_a = -1, warm_b = -1;
        float s_warm = 0.0f;  // slope of the last searched bridge
        // slope of the sampling-pass bound: the line's own tangent at t = 0
        // (damage energy) until a search finds a bridge clearly below the
        // centre, then that bridge's slope until a line is flat again
        bool cmode = EK == CVX_ENERGY_NH_DAMAGE;
        const float sa = s_sa, cb = s_cb;
        NHPair npair = nh_pair_node(nl);
        npair.J0 = pk2(s_nl.J0, s_nl.J0);  // J(0) = det F of the node, every line
        float my_cJ = 0.0f;   // lane k keeps the k-th line of each run of 32 for the work count
        const float kap = s_pd.kappa_f, C = s_shift;
        // L = 128 nfull + 1: the one sample past the full chunks (the right
        // end) is taken in the 32-line setup below, one lane per line
        const bool tail1 = EK == CVX_ENERGY_NH_DAMAGE && ln.nfull > 0 && ln.L == 128 * ln.nfull + 1;
        if (EK == CVX_ENERGY_NH_DAMAGE && d1 - d0 >= 64 * nw) {
            // seed: one line per warp, spread over the item, searched outright,
            // so that the item's smallest upper bound starts near the best value
            // and the bound test drops more lines from the start (the seed lines
            // are scanned again below)
            const int span = (d1 - d0) / nw;
            const int dj = d0 + warp * span + span / 2;
            const int gd = win ? window_dir(s_pd, cen, dj) : dj;
            const DirLine dl = make_dir_line<EK>(s_nl, P.dir32[doff + gd]);
            NHPair c = npair;
            c.A1 = pk2(dl.A1, dl.A1);
            c.A2 = pk2(dl.A2, dl.A2);
            c.CJ = pk2(dl.cJ, dl.cJ);
            const float tv = tail1 ? sample_w<EK>(nl, dl, (float)(ln.L - 1 - ln.m0) * ln.h32) : 0.0f;
            sample_line_min_nh(sw, nl, c, dl, ln, lane, tl, 0.0f, tail1, tv);
            __syncwarp();
            const ScreenOut o = warp_screen(sw, g, lane, -1, -1, hc);
            if (o.a >= 0 && lane == 0) atomicMin(&s_ukey, f2key(o.q_hi));
            __syncthreads();
        }
        for (int sg = warp; sg < nseg; sg += nw) {
            const int jb = d0 + sg * seg, je = min(d1, jb + seg);
            if (EK == CVX_ENERGY_NH_DAMAGE) cmode = true;
            n_lines += (unsigned long long)(je - jb);
            for (int dj = jb; dj < je; ++dj) {
                const int gd = win ? window_dir(s_pd, cen, dj) : dj;
                const int r = (dj - jb) & 31;
                // damage energy: every 32 lines, lane k sets up the k-th next line
                // (its constants, tangent slope, valid-sample count and, with
                // L = 128 nfull + 1, its right-end sample) for the whole warp
                if (EK == CVX_ENERGY_NH_DAMAGE && r == 0) {
                    const int dd = dj + lane;
                    if (dd < je) {
                        const int gd2 = win ? window_dir(s_pd, cen, dd) : dd;
                        const DirLine d2 = make_dir_line<EK>(s_nl, P.dir32[doff + gd2]);
                        const float tv =
                            tail1 ? sample_w<EK>(nl, d2, (float)(ln.L - 1 - ln.m0) * ln.h32) : 0.0f;
                        s_dir[warp][lane][0] = make_float4(d2.A1, d2.A1, d2.A2, d2.A2);
                        s_dir[warp][lane][1] =
                            make_float4(d2.cJ, d2.cJ, sa * __fmaf_rn(cb, d2.cJ, d2.A1), tv);
                        n_valid += valid_samples(d2, ln, EK);
                    }
                    __syncwarp();
                }
                DirLine dl;
                NHPair c;
                float sl, tvr = 0.0f;
                if (EK == CVX_ENERGY_NH_DAMAGE) {
                    const float4 q0 = s_dir[warp][r][0], q1 = s_dir[warp][r][1];
                    c = npair;
                    c.A1 = pk2(q0.x, q0.y);
                    c.A2 = pk2(q0.z, q0.w);
                    c.CJ = pk2(q1.x, q1.y);
                    dl.A1 = q0.x;
                    dl.A2 = q0.z;
                    dl.cJ = q1.x;
                    dl.J0 = s_nl.J0;
                    sl = cmode ? q1.z : s_warm;
                    tvr = q1.w;
                } else {
                    dl = make_dir_line<EK>(s_nl, P.dir32[doff + gd]);
                    sl = s_warm;
                }
                // sampling, with min over the line of v - s x at slope sl: a lower
                // bound qb of the value at 0 of the hull of the left and right sets
                // (any slope gives one; the damage-energy sampler leaves the centre
                // out of the min, the test energy's keeps it, which only lowers qb)
                const float e = EK == CVX_ENERGY_NH_DAMAGE
                                    ? sample_line_min_nh(sw, nl, c, dl, ln, lane, tl, -sl, tail1, tvr)
                                    : sample_line_min<EK>(sw, nl, dl, ln, lane, tl, -sl);
                // (the damage-energy bound starts at +inf and its mins skip NaN,
                // so it is never NaN: a float reduction gives the key order's min)
                float emin;
                if (EK == CVX_ENERGY_NH_DAMAGE) {
                    emin = warp_min_f32(e);
                } else {
                    const int ek = __reduce_min_sync(kFull, f2key(nan_to_inf(e)));
                    emin = __int_as_float(f2key(__int_as_float(ek)));
                }
                const float qb = emin - 3.2f * kU32 * (fabsf(emin) + 2.0f * fabsf(sl) * (float)ln.m0) -
                                 1e-30f;
                __syncwarp();
                // a line whose bound already exceeds m + eps(m), m = min(W(F), the
                // smallest upper bound seen in this item), can neither win nor split
                // (the node-level test in k_select uses the same monotone rule)
                const float wc = sw[ln.m0];
                const int ukey = *(volatile int *)&s_ukey;
                const float mref = fminf(wc, __int_as_float(f2key(__int_as_float(ukey))));
                const bool bounded = qb - eps32_at(qb, kap, C) > mref + eps32_at(mref, kap, C);
                // a flat line: its bound is within the sample error of the centre
                // value, so no bridge of it lies clearly below the centre; the
                // search is skipped and qb stands as its lower bound (its upper
                // bound stays unknown).  Such lines only matter at nodes whose
                // split, if any, is within the FP32 error, where the FP64
                // refinement of the best candidates decides.
                const float epsc = eps32_at(wc, kap, C);
                const bool flat = EK == CVX_ENERGY_NH_DAMAGE && !bounded && qb >= wc - epsc;
                ScreenOut o;
                if (bounded || flat) {
                    o.a = o.b = -1;
                    o.q_lo = qb;
                    o.q_hi = INFINITY;
                    o.w0 = wc;
                    if (flat) cmode = true;
                } else {
                    o = warp_screen(sw, g, lane, warm_a, warm_b, hc);
                    if (o.a >= 0) {
                        s_warm = __fdividef(sw[o.b] - sw[o.a], (float)(o.b - o.a));
                        if (lane == 0) atomicMin(&s_ukey, f2key(o.q_hi));
                    }
                    cmode = EK == CVX_ENERGY_NH_DAMAGE && !(o.a >= 0 && o.q_hi < wc - epsc);
                }
                n_bounded += bounded ? 1u : 0u;
                n_flat += flat ? 1u : 0u;
                __syncwarp();
                if (EK != CVX_ENERGY_NH_DAMAGE && lane == r) my_cJ = dl.cJ;
                if (EK != CVX_ENERGY_NH_DAMAGE && (r == 31 || dj == je - 1)) {
                    if (lane <= r) {
                        DirLine vl = dl;
                        vl.cJ = my_cJ;
                        n_valid += valid_samples(vl, ln, EK);
                    }
                }
                w0 = o.w0;
                if (o.a >= 0) {
                    warm_a = o.a;
                    warm_b = o.b;
                }
                qhi_min = fminf(qhi_min, o.q_hi);
                if (bounded)
                    dropped = fminf(dropped, qb);
                else
                    top_insert(tq, td, dropped, o.q_lo, gd);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kWarpTop; ++i) {
                s_q[warp][i] = tq[i];
                s_d[warp][i] = td[i];
            }
            s_drop[warp] = dropped;
            s_qhi[warp] = qhi_min;
            if (warp < nseg) s_w0 = w0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // merge the warps' lists (ties -> lower direction index)
            ItemCands r;
            float drop = INFINITY, qhi = INFINITY;
            for (int k = 0; k < nw; ++k) {
                drop = fminf(drop, s_drop[k]);
                qhi = fminf(qhi, s_qhi[k]);
            }
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
                r.ab[n] = -1;
                ++taken[bk];
            }
            for (int k = 0; k < nw; ++k)
                if (taken[k] < kWarpTop && s_d[k][taken[k]] >= 0) drop = fminf(drop, s_q[k][taken[k]]);
            for (int i = n; i < kItemTop; ++i) {
                r.q[i] = INFINITY;
                r.dir[i] = -1;
                r.ab[i] = -1;
            }
            r.n = n;
            r.w0 = s_w0;
            r.dropped = drop;
            r.qhi_min = qhi;
            r.flags = 0;
            r.pad = 0;
            P.items[item] = r;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) n_valid += __shfl_xor_sync(kFull, n_valid, o);
    if (lane == 0) {
        const unsigned *c = hc.c;
        add_counter(P.counters, C_LINES, n_lines);
        add_counter(P.counters, C_BOUNDED, n_bounded);
        add_counter(P.counters, C_FLAT, n_flat);
        add_counter(P.counters, C_VALID, n_valid);
        add_counter(P.counters, C_FULL, c[HC_FULL]);
        add_counter(P.counters, C_RARE, c[HC_RARE]);
        add_counter(P.counters, C_WSTEPS, c[HC_WSTEPS]);
        add_counter(P.counters, C_ROUNDS, c[HC_ROUNDS]);
    }
}

static size_t scan_smem(int warps, int stride) { return (size_t)warps * stride * sizeof(float); }

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

// RefineOut.pad of a candidate k_refine did not refine: q holds a lower bound
// of its FP64 value, above the node's minimum.
constexpr int kScreened = 2;

// -------------------------------------------------------------------------
// k_select: one thread per queued node.  eps bounds |q_FP32 - q_FP64|
// (1-Lipschitz in the samples), q_lo <= q_R^FP32 <= q_hi per direction.  The
// node's FP64 value V = min(W(F), min_R q_R^FP64) is at most
// min(w0, min_R q_hi) + eps, so a direction with q_lo > min(w0, U) + 2 eps
// (U = min q_hi) can neither be the FP64 minimiser nor split the node, and if
// min q_lo > w0 + 2 eps no line splits.  The (at most kNodeCand) directions
// with the smallest q_lo inside that band are refined in FP64; k_commit checks
// that no unrefined direction (q_lo >= qcut) can win.
// -------------------------------------------------------------------------
__global__ void k_select(const Pipe P, int level) {
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= P.cnt[level]) return;
    const ProbDesc &pd = P.probs[P.pid[P.qp[level][qi]]];
    const ItemCands *r = P.items + (long long)qi * P.C;
    const int chunks = pass_chunks(pd, P.pass);
    float qmin = INFINITY, drop = INFINITY, U = INFINITY;
    int fl = 0;
    const float w0 = r[0].w0;
    for (int c = 0; c < chunks; ++c) {
        qmin = fminf(qmin, r[c].q[0]);
        drop = fminf(drop, r[c].dropped);
        U = fminf(U, r[c].qhi_min);
        fl |= r[c].flags;
    }
    NodeCands nc;
    nc.n = 0;
    float cq[kNodeCand];  // the candidates' FP32 lower bounds
    const float shift = (float)line_shift(pd.mat, pd.beta[P.qp[level][qi] - pd.point_off]);
    const float kap = pd.kappa_f;
    // a direction is a candidate iff q - eps(q) <= m + eps(m), m = min(W(F), U)
    const float mref = fminf(w0, U);
    const float R = mref + eps32_at(mref, kap, shift);
    float qcut = drop;
    if (qmin - eps32_at(qmin, kap, shift) <= R) {
        // merge the items' sorted lists, smallest q first (ties: lower direction)
        int pos[64];
        const int nch = chunks < 64 ? chunks : 64;
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
            if (!(q - eps32_at(q, kap, shift) <= R) || nc.n == kNodeCand) {
                qcut = fminf(qcut, q);
                break;
            }
            cq[nc.n] = q;
            nc.dir[nc.n] = r[bc].dir[pos[bc]];
            nc.ab[nc.n++] = r[bc].ab[pos[bc]];
            ++pos[bc];
        }
        for (int c = nch; c < chunks; ++c) qcut = fminf(qcut, r[c].q[0]);
    } else {
        qcut = fminf(qcut, qmin);
    }
    nc.qcut = qcut;
    nc.eps = qcut < INFINITY ? eps32_at(qcut, kap, shift) : 0.0f;
    nc.flags = fl;
    if (nc.n) {
        // node constants of the FP64 refinement, once per node
        const cvx_node *nd = node_ptr(pd, P.qp[level][qi], P.qh[level][qi]);
        const double F[4] = {nd->F[0], nd->F[1], nd->F[2], nd->F[3]};
        const double beta = pd.beta[P.qp[level][qi] - pd.point_off];
        nc.nl = make_node_line(F, beta, pd.mat);
        nc.ek = exp(-beta / pd.mat.D0);
        nc.shift = line_shift(pd.mat, beta);
    }
    P.cands[qi] = nc;
    if (nc.n) {
        const int pos = atomicAdd(P.cnt + (P.K + 1) + level, nc.n);
        for (int c = 0; c < nc.n; ++c) P.work[pos + c] = make_int2(qi, c);
        // per candidate, a lower bound of its FP64 value in W units (as for
        // qcut in k_commit): (q - eps(q) + C) / kappa'; k_refine's second
        // phase skips a candidate whose bound exceeds the first one's value
        RefineOut *ro = P.refined + (long long)qi * kNodeCand;
        for (int c = 0; c < nc.n; ++c) {
            const float q = cq[c];
            RefineOut o;
            o.q = ((double)q - (double)eps32_at(q, kap, shift) + nc.shift) / pd.kappa;
            o.a = o.b = -1;
            o.ok = 0;
            o.pad = kScreened;
            ro[c] = o;
        }
    }
}

// -------------------------------------------------------------------------
// FP64 bridge of the left and right sets of one line held in shared memory:
// supporting-slope iteration with full passes; ties go to the outermost sample
// (Algorithm 1 keeps the outermost of collinear points).
//
// The minima of v - s x are compared as order-preserving integer keys of the
// doubles, so that the comparisons run on the integer pipe: the FP64 pipe
// (2 lanes per SM per clock) is what bounds the refinement, and a key compares
// exactly as its double does.
// -------------------------------------------------------------------------

// Integer key of a double that is not NaN: x < y iff dkey(x) < dkey(y), and
// x == y iff the keys are equal (-0 and +0 share the key 0).
__device__ __forceinline__ long long dkey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : -(b & 0x7fffffffffffffffLL);
}

constexpr long long kKeyInf = 0x7ff0000000000000LL;  // dkey(+inf)

// Warp-wide minimum of (key, sample index); ties to the lower index if
// prefer_low, else to the higher.
__device__ __forceinline__ void warp_min_key(long long &v, int &k, bool prefer_low) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const long long v2 = __shfl_xor_sync(kFull, v, o);
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
        long long bl = kKeyInf, br = kKeyInf;
        int kl = INT_MAX, kr = -1;
        for (int k = lane; k < L; k += 32) {
            if (k == m0) continue;
            const double v = sw[k];
            if (!(v < INFINITY)) continue;
            const long long e = dkey(v - s * (double)(k - m0));
            if (k < m0) {
                if (e < bl || (e == bl && k < kl)) {
                    bl = e;
                    kl = k;
                }
            } else if (e < br || (e == br && k > kr)) {
                br = e;
                kr = k;
            }
        }
        warp_min_key(bl, kl, true);
        warp_min_key(br, kr, false);
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

// Windowed FP64 bridge: supporting-slope iteration over two 32-sample
// windows of FP64 samples (vA at kA = loA + lane left of the centre, vB at
// kB = loB + lane right of it), seeded with (a, b).  Ties go to the outermost
// sample, as in bridge64.  false if it does not settle.
__device__ bool window_bridge64(double vA, double vB, int kA, int kB, int m0, int &a, int &b,
                                double &wa, double &wb, int lane, int loA, int loB) {
    const bool okA = vA < INFINITY, okB = vB < INFINITY;
    const double xA = (double)(kA - m0), xB = (double)(kB - m0);
    for (int it = 0; it < 64; ++it) {
        const double s = (wb - wa) / (double)(b - a);
        long long eA = okA ? dkey(vA - s * xA) : kKeyInf;
        long long eB = okB ? dkey(vB - s * xB) : kKeyInf;
        int ka = okA ? kA : INT_MAX, kb = okB ? kB : -1;
        warp_min_key(eA, ka, true);
        warp_min_key(eB, kb, false);
        if (ka == INT_MAX || kb < 0) return false;
        if (ka == a && kb == b) return true;
        a = ka;
        b = kb;
        wa = __shfl_sync(kFull, vA, a - loA);
        wb = __shfl_sync(kFull, vB, b - loB);
    }
    return false;
}

// Half-warp minimum with the sample index (lanes 0-15 and 16-31 reduce
// separately); ties to the lower index if prefer_low, else to the higher.
__device__ __forceinline__ void half_min_key(long long &v, int &k, bool prefer_low) {
#pragma unroll
    for (int o = 8; o; o >>= 1) {
        const long long v2 = __shfl_xor_sync(kFull, v, o);
        const int k2 = __shfl_xor_sync(kFull, k, o);
        if (v2 < v || (v2 == v && (prefer_low ? k2 < k : k2 > k))) {
            v = v2;
            k = k2;
        }
    }
}

// FP64 bridge from the line scan's FP32 pair (a, b) (damage energy): the
// supporting-slope iteration over FP64 samples in two windows around a and
// b (16 samples each, one per lane, for L <= 513; 32 each, two per lane,
// above), then a certificate over the whole line that every sample outside
// the windows lies strictly above the FP64 chord.  Each such sample is first
// tested on its FP32 value, computed on the fly: its FP32 sample less the
// FP32 error bound kEps32 max(kappa', |v| + C) and the rounding bound of the
// chord evaluated in FP32 sample units lies above the chord.  Where that test
// is inconclusive (near the tangent points, or det near 0) the sample is
// taken in FP64 and compared with the chord exactly.  An FP64 sample on or
// below the chord moves the pair to the lowest such sample of its side (at
// the chord's slope) and the windows are taken around the new pair, at most
// 4 times.  Returns false if that does not settle (the caller resamples the
// whole line in FP64); n64 counts the FP64 spot samples.
// Lines up to this many samples take FP64 windows of 16 samples per side in
// the refinement (one sample per lane), longer lines 32 per side (two per
// lane).  A window that misses a tangent point only costs a further round:
// the certificate over the whole line moves it.
#ifndef CVX_REFINE_NARROW_MAX_L
#define CVX_REFINE_NARROW_MAX_L 513
#endif

__device__ bool refine_hinted(const double F[4], const double R[4], double beta, const NodeCands &nc,
                              const ProbDesc &pd, const LineSpec &ln, float4 d32, int hab, int lane,
                              int &a, int &b, double &wa, double &wb, unsigned &n64,
                              int *spot_q) {
    const int m0 = ln.m0, L = ln.L;
    const double ek = nc.ek;
    a = hab & 0xffff;
    b = hab >> 16;
    if (!(a >= 0 && a < m0 && b > m0 && b < L)) return false;
    const bool narrow = L <= CVX_REFINE_NARROW_MAX_L;
    const int W = narrow ? 16 : 32;
    const double kap = pd.kappa, C = nc.shift;
    const float kapf = pd.kappa_f, Cf = (float)C;
    const DirLine dl = make_dir_line<CVX_ENERGY_NH_DAMAGE>(nc.nl, d32);
    for (int round = 0; round < 4; ++round) {
        const int loA = max(0, min(a - W / 2, m0 - W));
        const int loB = max(m0 + 1, min(b - (W / 2 - 1), L - W));
        // window samples: narrow, lane l < 16 holds left loA + l and lane
        // l >= 16 right loB + l - 16; wide, every lane holds left loA + l and
        // right loB + l
        const int kA = narrow ? loA + (lane & 15) : loA + lane;
        const int kB = narrow ? loB + (lane & 15) : loB + lane;
        const bool hasA = narrow ? lane < 16 : true, hasB = narrow ? lane >= 16 : true;
        double vA = INFINITY, vB = INFINITY;
        if (hasA && kA < m0) {
            const double v = sample_w64_ek(F, R, kA, m0, ln.h64, beta, ek, pd.mat);
            vA = v == v ? v : INFINITY;
        }
        if (hasB && kB < L) {
            const double v = sample_w64_ek(F, R, kB, m0, ln.h64, beta, ek, pd.mat);
            vB = v == v ? v : INFINITY;
        }
        auto valA = [&](int k) { return __shfl_sync(kFull, vA, k - loA); };
        auto valB = [&](int k) { return __shfl_sync(kFull, vB, narrow ? 16 + k - loB : k - loB); };
        wa = valA(a);
        wb = valB(b);
        if (!(wa < INFINITY && wb < INFINITY)) return false;
        bool settled = false;
        // per round: which window samples count, and their abscissae
        const bool left = lane < 16;
        const double vN = left ? vA : vB;
        const int kN = left ? kA : kB;
        const bool okA = vA < INFINITY, okB = vB < INFINITY, okN = vN < INFINITY;
        const double xA = (double)(kA - m0), xB = (double)(kB - m0), xN = (double)(kN - m0);
        for (int it = 0; it < 64 && !settled; ++it) {
            const double s = (wb - wa) / (double)(b - a);
            int na, nb;
            if (narrow) {
                long long e = okN ? dkey(vN - s * xN) : kKeyInf;
                int kk = okN ? kN : (left ? INT_MAX : -1);
                half_min_key(e, kk, left);
                na = __shfl_sync(kFull, kk, 0);
                nb = __shfl_sync(kFull, kk, 16);
            } else {
                long long eA = okA ? dkey(vA - s * xA) : kKeyInf;
                long long eB = okB ? dkey(vB - s * xB) : kKeyInf;
                int ka = okA ? kA : INT_MAX, kb = okB ? kB : -1;
                warp_min_key(eA, ka, true);
                warp_min_key(eB, kb, false);
                na = ka;
                nb = kb;
            }
            if (na == INT_MAX || nb < 0) return false;
            settled = na == a && nb == b;
            a = na;
            b = nb;
            wa = valA(a);
            wb = valB(b);
        }
        if (!settled) return false;
        // certificate over the samples outside the windows and the centre
        const double s = (wb - wa) / (double)(b - a);
        const float la = (float)(kap * wa - C), ls = (float)(kap * s);
        const int hiA = min(loA + W, m0), hiB = min(loB + W, L);
        long long eL = kKeyInf, eR = kKeyInf;  // lowest v - s x of FP64 samples on or below
        int kL = INT_MAX, kR = -1;              // the chord, per side (keys)
        unsigned c64 = 0;
        // FP64 spot sample k, compared with the chord exactly
        auto spot = [&](int k) {
            ++c64;
            const double v = sample_w64_ek(F, R, k, m0, ln.h64, beta, ek, pd.mat);
            if (!(v == v)) return;  // det <= 0: excluded
            const double line = wa + s * (double)(k - a);
            if (v > line + 1e-14 * fabs(line)) return;
            const long long e = dkey(v - s * (double)(k - m0));
            if (k < m0) {
                if (e < eL || (e == eL && k < kL)) {
                    eL = e;
                    kL = k;
                }
            } else if (e < eR || (e == eR && k > kR)) {
                eR = e;
                kR = k;
            }
        };
        // samples whose FP32 test is inconclusive queue up in the warp's
        // shared-memory buffer and are taken in FP64 32 at a time, one per
        // lane, so that a few scattered ones do not each cost the whole warp
        // an FP64 sample; the minima do not depend on the order
        int nq = 0;
        for (int base = 0; base < L; base += 32) {
            const int k = base + lane;
            bool need = false;
            if (k < L && k != m0 && !(k >= loA && k < hiA) && !(k >= loB && k < hiB)) {
                const float v32 =
                    sample_w<CVX_ENERGY_NH_DAMAGE>(nc.nl, dl, __fmul_rn((float)(k - m0), ln.h32));
                need = true;
                if (v32 < INFINITY && v32 > -INFINITY) {
                    const float x = (float)(k - a);
                    const float Lv = __fmaf_rn(ls, x, la);
                    const float err = 2.0f * kU32 * (fabsf(la) + fabsf(ls * x) + fabsf(Lv)) +
                                      kEps32 * fmaxf(kapf, fabsf(v32) + Cf) + 1e-30f;
                    need = !(__fsub_rn(v32, Lv) > 1.001f * err);  // else above the chord
                }
            }
            const unsigned bal = __ballot_sync(kFull, need);
            if (need) spot_q[nq + __popc(bal & ((1u << lane) - 1u))] = k;
            nq += __popc(bal);
            __syncwarp();
            if (nq >= 32) {
                spot(spot_q[lane]);
                const int rest = nq - 32;
                __syncwarp();
                if (lane < rest) spot_q[lane] = spot_q[32 + lane];
                nq = rest;
                __syncwarp();
            }
        }
        if (lane < nq) spot(spot_q[lane]);
        __syncwarp();
        n64 += c64;
        warp_min_key(eL, kL, true);
        warp_min_key(eR, kR, false);
        if (kL == INT_MAX && kR < 0) return true;  // certified
        if (kL != INT_MAX) a = kL;
        if (kR >= 0) b = kR;
    }
    return false;
}

// The FP64 refinement of candidate c of queued node qi (one warp): writes
// P.refined[qi][c].
template <int EK>
__device__ __forceinline__ void refine_one(const Pipe &P, int level, int qi, int c, int lane,
                                           double *sw, HullCounters &hc,
                                           unsigned long long &n_full, unsigned &n_spot) {
    float *sw32 = reinterpret_cast<float *>(sw);
    const int32_t *qp = P.qp[level], *qh = P.qh[level];
    const int p = qp[qi], hi = qh[qi];
    const ProbDesc &pd = P.probs[P.pid[p]];
    const cvx_node *nd = node_ptr(pd, p, hi);
    const LineSpec ln = scaled_line(pd.line, nd->window_exp);
    const int m0 = ln.m0;
    const int dir = P.cands[qi].dir[c];
    const double F[4] = {nd->F[0], nd->F[1], nd->F[2], nd->F[3]};
    const double *d = P.dir64 + 4 * ((long long)pd.dir_off + dir);
    const double R[4] = {__dmul_rn(d[0], d[2]), __dmul_rn(d[0], d[3]), __dmul_rn(d[1], d[2]),
                         __dmul_rn(d[1], d[3])};
    const double beta = pd.beta[p - pd.point_off];
    const int hab = P.cands[qi].ab[c];
    if (EK == CVX_ENERGY_NH_DAMAGE && hab >= 0) {
        // the scan's FP32 pair as the start, windows in FP64, FP32 certificate
        int a, b;
        double wa = 0.0, wb = 0.0;
        bool ok = refine_hinted(F, R, beta, P.cands[qi], pd, ln, P.dir32[pd.dir_off + dir], hab,
                                lane, a, b, wa, wb, n_spot, reinterpret_cast<int *>(sw));
        if (!ok) {
            ++n_full;
            const double ek = P.cands[qi].ek;
            for (int k = lane; k < ln.L; k += 32)
                sw[k] = sample_w64_ek(F, R, k, m0, ln.h64, beta, ek, pd.mat);
            __syncwarp();
            bridge64(sw, ln.L, m0, lane, a, b);
            if (a >= 0) {
                wa = sw[a];
                wb = sw[b];
            }
        }
        if (lane == 0) {
            RefineOut o;
            o.a = a;
            o.b = b;
            o.pad = 0;
            if (a >= 0) {
                const double xa = (double)(a - m0), xb = (double)(b - m0);
                o.q = (xb * wa - xa * wb) / (xb - xa);
                o.ok = 1;
            } else {
                o.q = INFINITY;
                o.ok = 0;
            }
            P.refined[(long long)qi * kNodeCand + c] = o;
        }
        __syncwarp();
        return;
    }
    // FP32 line and its approximate bridge
    const NodeLine nl = P.cands[qi].nl;
    const DirLine dl = make_dir_line<EK>(nl, P.dir32[pd.dir_off + dir]);
    float tl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tl[i] = (float)(4 * lane + i - m0) * ln.h32;
    sample_line<EK>(sw32, nl, dl, ln, lane, tl);
    __syncwarp();
    const LineGeom g{ln.L, m0, ln.nfull};
    const ScreenOut so = warp_screen(sw32, g, lane, -1, -1, hc);
    int a = so.a, b = so.b;
    bool ok = a >= 0 && b >= 0;
    double wa = 0.0, wb = 0.0;
    int loA = 0, loB = 0;
    if (ok) {
        loA = max(0, min(a - 16, m0 - 32));
        loB = min(max(m0 + 1, b - 15), ln.L - 32);
        loB = max(loB, m0 + 1);
        const int kA = loA + lane, kB = loB + lane;
        double vA = INFINITY, vB = INFINITY;
        if (kA < m0) {
            const double v = sample_w64(F, R, kA, m0, ln.h64, beta, pd.mat);
            vA = v == v ? v : INFINITY;
        }
        if (kB < ln.L) {
            const double v = sample_w64(F, R, kB, m0, ln.h64, beta, pd.mat);
            vB = v == v ? v : INFINITY;
        }
        wa = __shfl_sync(kFull, vA, a - loA);
        wb = __shfl_sync(kFull, vB, b - loB);
        ok = wa < INFINITY && wb < INFINITY &&
             window_bridge64(vA, vB, kA, kB, m0, a, b, wa, wb, lane, loA, loB);
    }
    if (ok) {
        // certificate over the samples outside the windows
        const double s = (wb - wa) / (double)(b - a);
        const double kap = pd.kappa, shift = P.cands[qi].shift;
        bool good = true;
        for (int k = lane; k < ln.L && good; k += 32) {
            if (k == m0 || (k >= loA && k < loA + 32 && k < m0) || (k >= loB && k < loB + 32))
                continue;
            const double line = wa + s * (double)(k - a);
            const float v32 = sw32[k];
            if (v32 < INFINITY && v32 > -INFINITY) {
                const double e = (double)kEps32 * fmax(kap, fabs((double)v32) + shift);
                const double lb = ((double)v32 - e + shift) / kap;
                good = lb > line + 1e-14 * (fabs(line) + fabs(lb));
            } else {
                const double v = sample_w64(F, R, k, m0, ln.h64, beta, pd.mat);
                good = !(v == v) || v > line + 1e-14 * fabs(line);
            }
        }
        ok = __all_sync(kFull, good);
    }
    __syncwarp();
    if (!ok) {
        // resample the whole line in FP64
        ++n_full;
        for (int k = lane; k < ln.L; k += 32) sw[k] = sample_w64(F, R, k, m0, ln.h64, beta, pd.mat);
        __syncwarp();
        bridge64(sw, ln.L, m0, lane, a, b);
        if (a >= 0) {
            wa = sw[a];
            wb = sw[b];
        }
    }
    if (lane == 0) {
        RefineOut o;
        o.a = a;
        o.b = b;
        o.pad = 0;
        if (a >= 0) {
            const double xa = (double)(a - m0), xb = (double)(b - m0);
            o.q = (xb * wa - xa * wb) / (xb - xa);
            o.ok = 1;
        } else {
            o.q = INFINITY;
            o.ok = 0;
        }
        P.refined[(long long)qi * kNodeCand + c] = o;
    }
    __syncwarp();
}

// k_refine: one warp per screened (node, direction).  The FP64 bridge of the
// left and right sample sets is searched in two 32-sample FP64 windows around
// the FP32 bridge and certified against the whole line with the FP32 samples:
// every sample m outside the windows must satisfy
//   (v32_m - kEps32 max(kappa', |v32_m| + C) + C) / kappa' > the FP64 bridge line at m,
// i.e. its FP64 value lies strictly above the line, so the windows' bridge is
// the bridge of all samples.  Otherwise (and where the FP32 samples are not
// finite) the whole line is resampled in FP64 (bridge64).
//
// Two launches per level.  Phase 0 refines each node's first candidate (the
// smallest FP32 lower bound); its FP64 value gives the node an upper bound
// V0 = min(W(F), q_0) of the FP64 minimum.  Phase 1 refines the others,
// except a candidate whose FP64 value is bounded below by more than V0 (the
// bound k_select stored: its FP32 lower bound less the FP32 error bound), as
// it can neither be the minimiser nor tie with it.  The decisions are those
// of refining every candidate.
template <int EK>
__global__ void __launch_bounds__(128) k_refine(const Pipe P, int level, int phase) {
    extern __shared__ double sm64[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *sw = sm64 + warp * P.stride64;
    __shared__ unsigned s_hc[4][HC_N];  // the screen's event counters (not reported here)
    if (lane == 0)
        for (int i = 0; i < HC_N; ++i) s_hc[warp][i] = 0u;
    __syncwarp();
    HullCounters hc{s_hc[warp]};
    unsigned long long n_full = 0, n_ref = 0;
    unsigned n_spot = 0;  // FP64 spot samples of the certificates (per lane)
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    // the warp's next (node, candidate): phase 0 takes 32 nodes per step and
    // their first candidates one after another, phase 1 the work list
    const int nn = P.cnt[level], nwork = P.cnt[(P.K + 1) + level];
    const int32_t *qp = P.qp[level], *qh = P.qh[level];
    int next = phase == 0 ? gw * 32 : gw, cur = 0;
    unsigned bal = 0;
    for (;;) {
        int qi = -1, c = 0;
        if (phase == 0) {
            while (!bal && next < nn) {
                cur = next;
                bal = __ballot_sync(kFull, cur + lane < nn && P.cands[cur + lane].n > 0);
                next += nwarps * 32;
            }
            if (!bal) break;
            qi = cur + __ffs(bal) - 1;
            bal &= bal - 1;
        } else {
            while (next < nwork) {
                const int2 wk = P.work[next];
                next += nwarps;
                if (wk.y == 0) continue;
                const RefineOut *ro = P.refined + (long long)wk.x * kNodeCand;
                const ProbDesc &pd = P.probs[P.pid[qp[wk.x]]];
                const double w_node = node_ptr(pd, qp[wk.x], qh[wk.x])->w;
                const double V0 = ro[0].ok && ro[0].q < w_node ? ro[0].q : w_node;
                if (ro[wk.y].q > V0) continue;  // the stored lower bound: screened out
                qi = wk.x;
                c = wk.y;
                break;
            }
            if (qi < 0) break;
        }
        refine_one<EK>(P, level, qi, c, lane, sw, hc, n_full, n_spot);
        ++n_ref;
    }
    if (lane == 0) add_counter(P.counters, C_REFFULL, n_full);
    if (lane == 0) add_counter(P.counters, C_REFINED, n_ref);
    n_spot = __reduce_add_sync(kFull, n_spot);
    if (lane == 0) add_counter(P.counters, C_FP64, n_spot);
}

// Offset of grid index i from the centre c on a periodic axis of N cells, in
// (-N/2, N/2].
__device__ __forceinline__ int wrap_offset(int i, int c, int N) {
    int d = (i - c) % N;
    if (d < 0) d += N;
    return d > N / 2 ? d - N : d;
}

// Grid cell nearest to the reflection of direction gd (angles pi i / Na,
// pi j / Nb) about the principal axes of F: theta_a -> 2 phi1 - theta_a,
// theta_b -> 2 phi2 - theta_b, with phi1 (phi2) the angle of the eigenvector
// of F F^T (F^T F) with the larger eigenvalue, 0.5 atan2(2B, A - C) for the
// symmetric [[A, B], [B, C]].  An isotropic W takes the same values on both
// lines (the reflections M1, M2 satisfy M1 F M2 = F and keep |.| and det).
// FP64 with explicit rounding in the order (2 phi) Na / pi - i.
__device__ int2 mirror_cell(const double F[4], int gd, int Na, int Nb) {
    constexpr double kPi = 3.14159265358979323846;
    const double f00 = F[0], f01 = F[1], f10 = F[2], f11 = F[3];
    const double y1 = __dmul_rn(2.0, __dadd_rn(__dmul_rn(f00, f10), __dmul_rn(f01, f11)));
    const double x1 = __dsub_rn(__dadd_rn(__dmul_rn(f00, f00), __dmul_rn(f01, f01)),
                                __dadd_rn(__dmul_rn(f10, f10), __dmul_rn(f11, f11)));
    const double y2 = __dmul_rn(2.0, __dadd_rn(__dmul_rn(f00, f01), __dmul_rn(f10, f11)));
    const double x2 = __dsub_rn(__dadd_rn(__dmul_rn(f00, f00), __dmul_rn(f10, f10)),
                                __dadd_rn(__dmul_rn(f01, f01), __dmul_rn(f11, f11)));
    const double p1 = __dmul_rn(0.5, atan2(y1, x1)), p2 = __dmul_rn(0.5, atan2(y2, x2));
    const double ua = __dsub_rn(__ddiv_rn(__dmul_rn(__dmul_rn(2.0, p1), (double)Na), kPi),
                                (double)(gd / Nb));
    const double ub = __dsub_rn(__ddiv_rn(__dmul_rn(__dmul_rn(2.0, p2), (double)Nb), kPi),
                                (double)(gd % Nb));
    int ma = (int)floor(__dadd_rn(ua, 0.5)) % Na, mb = (int)floor(__dadd_rn(ub, 0.5)) % Nb;
    if (ma < 0) ma += Na;
    if (mb < 0) mb += Nb;
    return make_int2(ma, mb);
}

// -------------------------------------------------------------------------
// k_commit: one thread per queued node.  Split points in FP64 with explicit
// rounding (no contraction): t = (m - m0) h, F+- = F + t R, xi = (m0-m-)/(m+-m-).
// -------------------------------------------------------------------------
__global__ void k_commit(const Pipe P, int level) {
    const int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= P.cnt[level]) return;
    const int p = P.qp[level][qi], hi = P.qh[level][qi];
    const ProbDesc &pd = P.probs[P.pid[p]];
    const NodeCands &nc = P.cands[qi];
    cvx_node &nd = *node_ptr(pd, p, hi);
    const RefineOut *ro = P.refined + (long long)qi * kNodeCand;
    int bc = -1;
    double second = INFINITY;
    for (int c = 0; c < nc.n; ++c) {
        if (!ro[c].ok) {
            // skipped by k_refine: only its lower bound is known (above the
            // node's minimum), which bounds the gap to the second best
            if (ro[c].pad == kScreened) second = fmin(second, ro[c].q);
            continue;
        }
        if (bc < 0 || ro[c].q < ro[bc].q || (ro[c].q == ro[bc].q && nc.dir[c] < nc.dir[bc])) {
            if (bc >= 0) second = fmin(second, ro[bc].q);
            bc = c;
        } else {
            second = fmin(second, ro[c].q);
        }
    }
    const int m0 = pd.line.m0;
    // FP64 node value among the refined directions; an unrefined direction
    // (FP32 q >= qcut) could only win if qcut - eps reached it
    const double V = (bc >= 0 && ro[bc].q < nd.w) ? ro[bc].q : nd.w;
    const double shift = line_shift(pd.mat, pd.beta[p - pd.point_off]);
    const bool overflow = !(((double)nc.qcut - (double)nc.eps + shift) / pd.kappa > V);
    // the node's decision: the best refined direction, or (mirror stage) the
    // main window's when that one holds the lower value
    const bool split = bc >= 0 && ro[bc].q < nd.w;
    RefineOut best = bc >= 0 ? ro[bc] : RefineOut{nd.w, m0, m0, 0, 0};
    int bdir = bc >= 0 ? nc.dir[bc] : -1;
    int xfl = (nc.flags & (CVX_NODE_ITER_CAP | CVX_NODE_OVERFLOW)) |
              (overflow ? CVX_NODE_OVERFLOW : 0);
    if (P.pass == PASS_WINDOW) {
        // fallback test of a proposal window: the window's best direction on
        // its border, or (main stage) an energy gap |E_pred - V| / (1e-8 + |V|)
        // above gap_tol between the proposed laminate and the window's value,
        // defers the node to the full scan
        atomicAdd(P.counters + C_WNODES, 1ull);
        bool border = false;
        const int gd = split ? nc.dir[bc] : -1;
        if (split) {
            const int2 c = P.center[qi];
            border = abs(wrap_offset(gd / pd.Nb, c.x, pd.Na)) >= pd.window ||
                     abs(wrap_offset(gd % pd.Nb, c.y, pd.Nb)) >= pd.window;
        }
        bool gap_fail = false;
        if (!P.mirror) {
            const double gap = ((pd.flags & CVX_FLAG_GAP_ONE_SIDED) ? V - P.e_pred[qi]
                                                                    : fabs(P.e_pred[qi] - V)) /
                               (1e-8 + fabs(V));
            gap_fail = !(gap <= pd.gap_tol);
        }
        if (border && !gap_fail && P.nx_p) {
            // re-centre the window on its border minimum and scan it again
            const int pos = atomicAdd(P.nx_cnt + level, 1);
            P.nx_p[pos] = p;
            P.nx_h[pos] = hi;
            P.nx_cen[pos] = make_int2(gd / pd.Nb, gd % pd.Nb);
            if (P.mirror)
                P.nx_rec[pos] = P.rec[qi];
            else
                P.nx_ep[pos] = P.e_pred[qi];
            atomicAdd(P.counters + C_RECENTRED, 1ull);
            return;
        }
        if (border || gap_fail) {
            const int pos = atomicAdd(P.fcnt + level, 1);
            P.fq_p[level][pos] = p;
            P.fq_h[level][pos] = hi;
            atomicAdd(P.counters + C_FALLBACK, 1ull);
            return;
        }
        if (!P.mirror && P.mirror_on && split) {
            // scan the twin basin: the window around the mirror cell of gd,
            // unless it lies inside this window
            const int2 mc = mirror_cell(nd.F, gd, pd.Na, pd.Nb);
            const int2 c = P.center[qi];
            const bool inside = abs(wrap_offset(mc.x, c.x, pd.Na)) + pd.mwindow <= pd.window &&
                                abs(wrap_offset(mc.y, c.y, pd.Nb)) + pd.mwindow <= pd.window;
            if (!inside) {
                const int pos = atomicAdd(P.mcnt + level, 1);
                P.mq_p[pos] = p;
                P.mq_h[pos] = hi;
                P.mcen[pos] = mc;
                WinRec r;
                r.q = ro[bc].q;
                r.second = second;
                r.dir = gd;
                r.a = ro[bc].a;
                r.b = ro[bc].b;
                r.flags = xfl;
                P.mrec[pos] = r;
                atomicAdd(P.counters + C_MIRROR, 1ull);
                return;
            }
        }
        if (P.mirror) {
            // the lower of the two windows' values; the lower direction index
            // on equal values (a main-window record always splits)
            const WinRec r = P.rec[qi];
            if (split && (ro[bc].q < r.q || (ro[bc].q == r.q && gd < r.dir))) {
                second = fmin(second, r.q);
                atomicAdd(P.counters + C_MIRROR_WON, 1ull);
            } else {
                second = fmin(r.second, bc >= 0 ? ro[bc].q : (double)INFINITY);
                best.q = r.q;
                best.a = r.a;
                best.b = r.b;
                best.ok = 1;
                bdir = r.dir;
            }
            xfl |= r.flags;
        }
    }
    const bool lam = best.q < nd.w && bdir >= 0;
    // adaptive line window: a split with an end on the end of its line is
    // scanned again with the window doubled (Sec. 4.1: r sufficiently large)
    if (P.pass == PASS_FULL && P.nx_p && bc >= 0 && ro[bc].q < nd.w &&
        (ro[bc].a == 0 || ro[bc].b == pd.line.L - 1) &&
        nd.window_exp < CVX_WINDOW_DOUBLINGS_OF(pd.flags)) {
        nd.window_exp += 1;
        const int pos = atomicAdd(P.nx_cnt + level, 1);
        P.nx_p[pos] = p;
        P.nx_h[pos] = hi;
        atomicAdd(P.counters + C_DOUBLED, 1ull);
        return;
    }
    nd.flags |= CVX_NODE_SCANNED | xfl;
    if (P.pass == PASS_FALLBACK) nd.flags |= CVX_NODE_FALLBACK;
    atomicAdd(P.counters + C_NODES, 1ull);
    nd.gap = (float)(second - (bdir >= 0 ? best.q : nd.w));
    if (xfl & CVX_NODE_OVERFLOW) atomicAdd(P.counters + C_OVERFLOW, 1ull);
    // the centre splits off iff the chord lies strictly below W(F) (FP64)
    if (!lam) {
        nd.dir = bdir;
        nd.flags |= CVX_NODE_LEAF;
        return;
    }
    const RefineOut b = best;
    int fl = CVX_NODE_LAMINATED;
    if (b.a == 0 || b.b == pd.line.L - 1) {
        fl |= CVX_NODE_EDGE;
        atomicAdd(P.counters + C_EDGE, 1ull);
    }
    if (second == b.q) {
        fl |= CVX_NODE_TIE;
        atomicAdd(P.counters + C_TIES, 1ull);
    }
    nd.flags |= fl;
    nd.dir = bdir;
    nd.m_minus = b.a;
    nd.m_plus = b.b;
    nd.h = b.q;
    atomicAdd(P.counters + C_LAMINATED, 1ull);
    const double *d = P.dir64 + 4 * ((long long)pd.dir_off + nd.dir);
    const double R[4] = {__dmul_rn(d[0], d[2]), __dmul_rn(d[0], d[3]), __dmul_rn(d[1], d[2]),
                         __dmul_rn(d[1], d[3])};
    const LineSpec lnd = scaled_line(pd.line, nd.window_exp);
    double tm = __dmul_rn((double)(b.a - m0), lnd.h64);
    double tp = __dmul_rn((double)(b.b - m0), lnd.h64);
    const bool leaf_children = level + 1 >= pd.K;
    const double beta = pd.beta[p - pd.point_off];
    double xi = (double)(m0 - b.a) / (double)(b.b - b.a);
    if (pd.flags & CVX_FLAG_REFINE_NEWTON) {
        double hN;
        if (newton_tangent64(nd.F, R, beta, pd.mat, lnd.h64 * m0, b.q, tm, tp, hN)) {
            xi = -tm / (tp - tm);
            nd.h = hN;
            nd.flags |= CVX_NODE_NEWTON;
        }
    }
    nd.xi = xi;
    for (int side = 0; side < 2; ++side) {
        const int ci = 2 * hi + 1 + side;  // 2i+1: F-, 2i+2: F+
        cvx_node &c = *node_ptr(pd, p, ci);
        const double t = side ? tp : tm;
        double F[4];
        for (int k = 0; k < 4; ++k) F[k] = __dadd_rn(nd.F[k], __dmul_rn(t, R[k]));
        for (int k = 0; k < 4; ++k) c.F[k] = F[k];
        c.weight = side ? __dmul_rn(nd.weight, xi) : __dmul_rn(nd.weight, __dsub_rn(1.0, xi));
        c.w = energy64(F, beta, pd.mat);
        c.h = c.w;
        c.xi = 0.0;
        c.dir = -1;
        c.m_minus = c.m_plus = m0;
        c.gap = 0.0f;
        c.window_exp = nd.window_exp;  // children start from their parent's window
        c.flags = CVX_NODE_EXISTS | (leaf_children ? CVX_NODE_LEAF : 0);
    }
    if (!leaf_children) {
        const int pos = atomicAdd(P.ncnt + level + 1, 2);
        P.qp[level + 1][pos] = p;
        P.qh[level + 1][pos] = 2 * hi + 1;
        P.qp[level + 1][pos + 1] = p;
        P.qh[level + 1][pos + 1] = 2 * hi + 2;
    }
}

// -------------------------------------------------------------------------
// k_leaf: W^R = sum over leaves of (path weight) W(F_leaf), same for P
// (Algorithm 3 with the recursion unrolled over the heap).
// -------------------------------------------------------------------------
__global__ void k_leaf(const Pipe P) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.N) return;
    const ProbDesc &pd = P.probs[P.pid[p]];
    const long long lp = p - pd.point_off;
    const cvx_node *tr = node_ptr(pd, p, 0);
    int st = pd.status[lp];
    if (st & CVX_PT_NONPOS_DET) {
        pd.W_R[lp] = nan("");
        for (int k = 0; k < 4; ++k) pd.P[4 * lp + k] = nan("");
        if (pd.root) {
            cvx_laminate z = {};
            z.dir = -1;
            pd.root[lp] = z;
        }
        return;
    }
    const double beta = pd.beta[lp];
    double W = 0.0, Pv[4] = {0.0, 0.0, 0.0, 0.0};
    int fl = 0;
    for (int i = 0; i < pd.NT; ++i) {
        const cvx_node &nd = tr[i];
        if (!(nd.flags & CVX_NODE_EXISTS)) continue;
        fl |= nd.flags;
        if (nd.flags & CVX_NODE_LAMINATED) continue;
        double F[4] = {nd.F[0], nd.F[1], nd.F[2], nd.F[3]};
        double Pl[4];
        stress64(F, beta, pd.mat, Pl);
        W += nd.weight * energy64(F, beta, pd.mat);
        for (int k = 0; k < 4; ++k) Pv[k] += nd.weight * Pl[k];
    }
    pd.W_R[lp] = W;
    for (int k = 0; k < 4; ++k) pd.P[4 * lp + k] = Pv[k];
    if (fl & CVX_NODE_TIE) st |= CVX_PT_TIE;
    if (fl & CVX_NODE_EDGE) st |= CVX_PT_EDGE;
    if (fl & CVX_NODE_ITER_CAP) st |= CVX_PT_ITER_CAP;
    if (fl & CVX_NODE_OVERFLOW) st |= CVX_PT_OVERFLOW;
    if (fl & CVX_NODE_FALLBACK) st |= CVX_PT_FALLBACK;
    pd.status[lp] = st;
    if (pd.root) {
        cvx_laminate Lm;
        const cvx_node &r0 = tr[0];
        Lm.laminated = (r0.flags & CVX_NODE_LAMINATED) ? 1 : 0;
        Lm.dir = r0.dir;
        Lm.m_minus = r0.m_minus;
        Lm.m_plus = r0.m_plus;
        Lm.xi = r0.xi;
        Lm.h = r0.h;
        for (int k = 0; k < 4; ++k) {
            Lm.F_plus[k] = Lm.laminated ? tr[2].F[k] : r0.F[k];
            Lm.F_minus[k] = Lm.laminated ? tr[1].F[k] : r0.F[k];
        }
        pd.root[lp] = Lm;
    }
}

// -------------------------------------------------------------------------
// Workspace layout and the enqueueing of one run.
// -------------------------------------------------------------------------
static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t pipe_carve(Pipe *pp, char *ws, long long N, int K, int C, int n_probs,
                         bool window, bool rescan, bool mirror) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + bytes);
        return o;
    };
    const size_t maxq = K > 0 ? ((size_t)N << (K - 1)) : 0;
    const size_t o_probs = take(sizeof(ProbDesc) * (size_t)n_probs);
    const size_t o_pid = take(sizeof(int32_t) * (size_t)N);
    size_t o_qp[kMaxDepth], o_qh[kMaxDepth];
    for (int l = 0; l < K; ++l) {
        o_qp[l] = take(sizeof(int32_t) * ((size_t)N << l));
        o_qh[l] = take(sizeof(int32_t) * ((size_t)N << l));
    }
    const size_t o_cnt = take(sizeof(int32_t) * 2 * (K + 1));
    const size_t o_ictr = take(sizeof(unsigned long long) * (K + 1));
    const size_t o_items = take(sizeof(ItemCands) * maxq * C);
    const size_t o_cands = take(sizeof(NodeCands) * maxq);
    const size_t o_work = take(sizeof(int2) * maxq * kNodeCand);
    const size_t o_ref = take(sizeof(RefineOut) * maxq * kNodeCand);
    const size_t o_nu = take(sizeof(int) * maxq);
    size_t o_fqp[kMaxDepth], o_fqh[kMaxDepth], o_fcnt = 0, o_fictr = 0, o_cen = 0, o_ep = 0;
    size_t o_rqp[2] = {0, 0}, o_rqh[2] = {0, 0}, o_rcen[2] = {0, 0}, o_rep[2] = {0, 0};
    size_t o_rcnt = 0, o_ritem = 0;
    // the mirror stage's re-centring passes count in a second block
    const int rblocks = kMaxRecentre * (mirror ? 2 : 1);
    if (window) {
        for (int l = 0; l < K; ++l) {
            o_fqp[l] = take(sizeof(int32_t) * ((size_t)N << l));
            o_fqh[l] = take(sizeof(int32_t) * ((size_t)N << l));
        }
        o_fcnt = take(sizeof(int32_t) * 2 * (K + 1));
        o_fictr = take(sizeof(unsigned long long) * (K + 1));
        o_cen = take(sizeof(int2) * maxq);
        o_ep = take(sizeof(double) * maxq);
    }
    if (window || rescan) {
        for (int b = 0; b < 2; ++b) {
            o_rqp[b] = take(sizeof(int32_t) * maxq);
            o_rqh[b] = take(sizeof(int32_t) * maxq);
            o_rcen[b] = take(sizeof(int2) * maxq);
            o_rep[b] = take(sizeof(double) * maxq);
        }
        o_rcnt = take(sizeof(int32_t) * 2 * (K + 1) * rblocks);
        o_ritem = take(sizeof(unsigned long long) * (K + 1) * rblocks);
    }
    size_t o_mprobs = 0, o_mqp = 0, o_mqh = 0, o_mcen = 0, o_mrec = 0, o_mcnt = 0, o_mitem = 0;
    size_t o_rrec[2] = {0, 0};
    if (window && mirror) {
        o_mprobs = take(sizeof(ProbDesc) * (size_t)n_probs);
        o_mqp = take(sizeof(int32_t) * maxq);
        o_mqh = take(sizeof(int32_t) * maxq);
        o_mcen = take(sizeof(int2) * maxq);
        o_mrec = take(sizeof(WinRec) * maxq);
        o_mcnt = take(sizeof(int32_t) * 2 * (K + 1));
        o_mitem = take(sizeof(unsigned long long) * (K + 1));
        for (int b = 0; b < 2; ++b) o_rrec[b] = take(sizeof(WinRec) * maxq);
    }
    if (pp) {
        Pipe &p = *pp;
        p.probs = (const ProbDesc *)(ws + o_probs);
        p.pid = (int32_t *)(ws + o_pid);
        for (int l = 0; l < kMaxDepth; ++l) {
            p.qp[l] = l < K ? (int32_t *)(ws + o_qp[l]) : nullptr;
            p.qh[l] = l < K ? (int32_t *)(ws + o_qh[l]) : nullptr;
        }
        p.cnt = (int32_t *)(ws + o_cnt);
        p.item_ctr = (unsigned long long *)(ws + o_ictr);
        p.items = (ItemCands *)(ws + o_items);
        p.cands = (NodeCands *)(ws + o_cands);
        p.work = (int2 *)(ws + o_work);
        p.refined = (RefineOut *)(ws + o_ref);
        p.node_u = (int *)(ws + o_nu);
        p.ncnt = p.cnt;
        p.pass = window ? PASS_WINDOW : PASS_FULL;
        for (int l = 0; l < kMaxDepth; ++l) {
            p.fq_p[l] = window && l < K ? (int32_t *)(ws + o_fqp[l]) : nullptr;
            p.fq_h[l] = window && l < K ? (int32_t *)(ws + o_fqh[l]) : nullptr;
        }
        p.fcnt = window ? (int32_t *)(ws + o_fcnt) : nullptr;
        p.fitem_ctr = window ? (unsigned long long *)(ws + o_fictr) : nullptr;
        p.center = window ? (int2 *)(ws + o_cen) : nullptr;
        p.e_pred = window ? (double *)(ws + o_ep) : nullptr;
        const bool rq = window || rescan;
        for (int b = 0; b < 2; ++b) {
            p.rq_p[b] = rq ? (int32_t *)(ws + o_rqp[b]) : nullptr;
            p.rq_h[b] = rq ? (int32_t *)(ws + o_rqh[b]) : nullptr;
            p.rcen[b] = rq ? (int2 *)(ws + o_rcen[b]) : nullptr;
            p.rep[b] = rq ? (double *)(ws + o_rep[b]) : nullptr;
        }
        p.rcnt = rq ? (int32_t *)(ws + o_rcnt) : nullptr;
        p.ritem = rq ? (unsigned long long *)(ws + o_ritem) : nullptr;
        p.nx_p = p.nx_h = p.nx_cnt = nullptr;
        p.nx_cen = nullptr;
        p.nx_ep = nullptr;
        const bool mq = window && mirror;
        p.mirror_on = mq ? 1 : 0;
        p.mirror = 0;
        p.mprobs = mq ? (const ProbDesc *)(ws + o_mprobs) : nullptr;
        p.mq_p = mq ? (int32_t *)(ws + o_mqp) : nullptr;
        p.mq_h = mq ? (int32_t *)(ws + o_mqh) : nullptr;
        p.mcen = mq ? (int2 *)(ws + o_mcen) : nullptr;
        p.mrec = mq ? (WinRec *)(ws + o_mrec) : nullptr;
        p.mcnt = mq ? (int32_t *)(ws + o_mcnt) : nullptr;
        p.mitem = mq ? (unsigned long long *)(ws + o_mitem) : nullptr;
        for (int b = 0; b < 2; ++b) p.rrec[b] = mq ? (WinRec *)(ws + o_rrec[b]) : nullptr;
        p.rec = p.nx_rec = nullptr;
    }
    return off;
}

size_t pipe_bytes(long long N, int K, int C, int n_probs, bool window, bool rescan,
                  bool mirror) {
    return pipe_carve(nullptr, nullptr, N, K, C, n_probs, window, rescan, mirror);
}

void pipe_layout(Pipe &p, char *ws) {
    pipe_carve(&p, ws, p.N, p.K, p.C, p.n_probs, p.window != 0, p.adaptive > 0,
               p.mirror_on != 0);
}

Pipe window_pipe(const Pipe &p, int level, int r, int R) {
    Pipe q = p;
    q.pass = PASS_WINDOW;
    if (r > 0) {
        const int b = (r - 1) & 1;
        q.cnt = p.rcnt + (size_t)2 * (p.K + 1) * (r - 1);
        q.item_ctr = p.ritem + (size_t)(p.K + 1) * (r - 1);
        q.qp[level] = p.rq_p[b];
        q.qh[level] = p.rq_h[b];
        q.center = p.rcen[b];
        q.e_pred = p.rep[b];
        q.ncnt = p.cnt;  // children go to the level queue of the next level
    }
    if (r < R) {
        const int b = r & 1;
        q.nx_p = p.rq_p[b];
        q.nx_h = p.rq_h[b];
        q.nx_cen = p.rcen[b];
        q.nx_ep = p.rep[b];
        q.nx_cnt = p.rcnt + (size_t)2 * (p.K + 1) * r;
    } else {
        q.nx_p = q.nx_h = q.nx_cnt = nullptr;
        q.nx_cen = nullptr;
        q.nx_ep = nullptr;
    }
    return q;
}

Pipe mirror_pipe(const Pipe &p, int level, int r, int R) {
    Pipe q = p;
    q.pass = PASS_WINDOW;
    q.mirror = 1;
    q.probs = p.mprobs;
    q.e_pred = nullptr;
    if (r == 0) {
        q.cnt = p.mcnt;
        q.item_ctr = p.mitem;
        q.qp[level] = p.mq_p;
        q.qh[level] = p.mq_h;
        q.center = p.mcen;
        q.rec = p.mrec;
    } else {
        const int b = (r - 1) & 1;
        q.cnt = p.rcnt + (size_t)2 * (p.K + 1) * (kMaxRecentre + r - 1);
        q.item_ctr = p.ritem + (size_t)(p.K + 1) * (kMaxRecentre + r - 1);
        q.qp[level] = p.rq_p[b];
        q.qh[level] = p.rq_h[b];
        q.center = p.rcen[b];
        q.rec = p.rrec[b];
    }
    q.ncnt = p.cnt;  // children go to the level queue of the next level
    if (r < R) {
        const int b = r & 1;
        q.nx_p = p.rq_p[b];
        q.nx_h = p.rq_h[b];
        q.nx_cen = p.rcen[b];
        q.nx_ep = nullptr;
        q.nx_rec = p.rrec[b];
        q.nx_cnt = p.rcnt + (size_t)2 * (p.K + 1) * (kMaxRecentre + r);
    } else {
        q.nx_p = q.nx_h = q.nx_cnt = nullptr;
        q.nx_cen = nullptr;
        q.nx_ep = nullptr;
        q.nx_rec = nullptr;
    }
    return q;
}

Pipe rescan_pipe(const Pipe &p, int level, int r, int A) {
    Pipe q = p;
    q.pass = PASS_FULL;
    if (r > 0) {
        const int b = (r - 1) & 1;
        q.cnt = p.rcnt + (size_t)2 * (p.K + 1) * (r - 1);
        q.item_ctr = p.ritem + (size_t)(p.K + 1) * (r - 1);
        q.qp[level] = p.rq_p[b];
        q.qh[level] = p.rq_h[b];
        q.ncnt = p.cnt;  // children go to the level queue of the next level
    }
    if (r < A) {
        const int b = r & 1;
        q.nx_p = p.rq_p[b];
        q.nx_h = p.rq_h[b];
        q.nx_cen = nullptr;
        q.nx_ep = nullptr;
        q.nx_cnt = p.rcnt + (size_t)2 * (p.K + 1) * r;
    } else {
        q.nx_p = q.nx_h = q.nx_cnt = nullptr;
        q.nx_cen = nullptr;
        q.nx_ep = nullptr;
    }
    return q;
}

Pipe fallback_pipe(const Pipe &p, int level) {
    Pipe q = p;
    q.pass = PASS_FALLBACK;
    q.cnt = p.fcnt;
    q.item_ctr = p.fitem_ctr;
    q.qp[level] = p.fq_p[level];
    q.qh[level] = p.fq_h[level];
    q.ncnt = p.cnt;
    return q;
}

template <int EK>
static cudaError_t launch_scan_t(const Pipe &p, int level, int warps, int grid, cudaStream_t s) {
    const size_t smem = scan_smem(warps, p.stride32);
    cudaError_t e = cudaFuncSetAttribute(k_scan<EK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_scan<EK><<<grid, warps * 32, smem, s>>>(p, level);
    return cudaGetLastError();
}

cudaError_t pipe_begin(const Pipe &p, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(p.cnt, 0, sizeof(int32_t) * 2 * (p.K + 1), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.item_ctr, 0, sizeof(unsigned long long) * (p.K + 1), s)) !=
        cudaSuccess)
        return e;
    if (p.window || p.adaptive) {
        const int rb = kMaxRecentre * (p.mirror_on ? 2 : 1);
        if ((e = cudaMemsetAsync(p.rcnt, 0, sizeof(int32_t) * 2 * (p.K + 1) * rb, s)) !=
            cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(p.ritem, 0, sizeof(unsigned long long) * (p.K + 1) * rb, s)) !=
            cudaSuccess)
            return e;
    }
    if (p.mirror_on) {
        if ((e = cudaMemsetAsync(p.mcnt, 0, sizeof(int32_t) * 2 * (p.K + 1), s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(p.mitem, 0, sizeof(unsigned long long) * (p.K + 1), s)) !=
            cudaSuccess)
            return e;
    }
    if (p.window) {
        if ((e = cudaMemsetAsync(p.fcnt, 0, sizeof(int32_t) * 2 * (p.K + 1), s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(p.fitem_ctr, 0, sizeof(unsigned long long) * (p.K + 1), s)) !=
            cudaSuccess)
            return e;
    }
    k_init<<<(unsigned)((p.N + 255) / 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t pipe_level(const Pipe &p, int l, int warps, int grid, cudaStream_t s,
                       cudaEvent_t *ev) {
    cudaError_t e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long max_nodes = p.N << l;
    if (p.lanes) {
        // the node bounds start at +inf (a huge finite key); reset outside the timed region
        if ((e = cudaMemsetAsync(p.node_u, 0x7f, sizeof(int) * (size_t)max_nodes, s)) != cudaSuccess)
            return e;
    }
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    if (p.lanes)
        e = launch_scan_lanes(p, l, sms, s);
    else
        e = p.energy == CVX_ENERGY_NH_DAMAGE
                ? launch_scan_t<CVX_ENERGY_NH_DAMAGE>(p, l, warps, grid, s)
                : launch_scan_t<CVX_ENERGY_DOUBLE_WELL>(p, l, warps, grid, s);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
    const unsigned nb = (unsigned)((max_nodes + 127) / 128);
    k_select<<<nb, 128, 0, s>>>(p, l);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long want = (max_nodes * kNodeCand + 3) / 4;
    const unsigned rg = (unsigned)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    const size_t rsm = (size_t)4 * p.stride64 * sizeof(double);
    auto kr = p.energy == CVX_ENERGY_NH_DAMAGE ? k_refine<CVX_ENERGY_NH_DAMAGE>
                                               : k_refine<CVX_ENERGY_DOUBLE_WELL>;
    if ((e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm)) !=
        cudaSuccess)
        return e;
    kr<<<rg, 128, rsm, s>>>(p, l, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kr<<<rg, 128, rsm, s>>>(p, l, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_commit<<<nb, 128, 0, s>>>(p, l);
    return cudaGetLastError();
}

cudaError_t pipe_end(const Pipe &p, cudaStream_t s) {
    k_leaf<<<(unsigned)((p.N + 127) / 128), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t pipe_enqueue(const Pipe &p, int warps, int grid, cudaStream_t s, cudaEvent_t *ev) {
    cudaError_t e;
    if (p.N == 0) return cudaSuccess;
    if ((e = pipe_begin(p, s)) != cudaSuccess) return e;
    const int A = p.adaptive;
    for (int l = 0; l < p.K; ++l)
        for (int r = 0; r <= A; ++r) {
            const Pipe q = A ? rescan_pipe(p, l, r, A) : p;
            if ((e = pipe_level(q, l, warps, grid, s, ev ? ev + 2 * (l * (A + 1) + r) : nullptr)) !=
                cudaSuccess)
                return e;
        }
    return pipe_end(p, s);
}

}  // namespace cvx
