// cvx_internal.h -- structures shared by the kernels and the host side of
// libconvexify (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "convexify.h"
#include "cvx_device.cuh"

namespace cvx {

constexpr int kWarpTop = 4;    // best directions kept per warp
constexpr int kItemTop = 16;   // per work item
constexpr int kNodeCand = 16;  // candidates refined in FP64 per node
constexpr int kLaneItemMax = 256;  // lines per block of a work item of the lane-per-line scan
constexpr int kMaxDepth = 8;
constexpr int kMaxRecentre = 8;  // window re-centrings per node at most (surrogate_propose)
// Bound on the FP32 sampling error of v = kappa' W - C in sample units,
// relative to max(kappa', |v| + C) (>= kappa' max(1, |W|)): 3.5 times the
// largest error measured against FP64.
constexpr float kEps32 = 1.1e-6f;

// The FP32 error bound at sample value x (C = the point's sample shift).
__device__ __forceinline__ float eps32_at(float x, float kappa, float C) {
    return kEps32 * fmaxf(kappa, fabsf(x) + C);
}

// Best directions of one work item (a node and a block of its directions),
// ranked by q = a rigorous lower bound on the value at t = 0 of the hull of the
// FP32 samples of the left and right sets (the node's hull value when the
// centre does not lie below it); qhi_min is the smallest upper bound seen.
struct ItemCands {
    float q[kItemTop];
    int dir[kItemTop];
    int ab[kItemTop];  // FP32 bridge pair a | b << 16 of each kept direction, -1 if unknown
    float w0;       // FP32 centre sample
    float dropped;  // smallest q not kept
    float qhi_min;  // smallest upper bound over the item's directions
    int n, flags, pad;
};

struct NodeCands {
    int dir[kNodeCand];
    int ab[kNodeCand];  // FP32 bridge pair hint per candidate (as in ItemCands), -1 if unknown
    int n, flags;
    float qcut;  // smallest FP32 q of a direction not refined (sample units)
    float eps;   // FP32 error bound used at this node (sample units)
    // node constants for the FP64 refinement, computed once per node
    NodeLine nl;  // FP32 line constants (make_node_line)
    double ek;    // exp(-beta_k / D_0)
    double shift; // sample shift C in FP64 (line_shift)
};

// A window decision carried to the node's mirror window (surrogate_propose,
// CVX_FLAG_MIRROR_WINDOW): the FP64 value and bridge of the best direction,
// the second-best value and the node flags (iteration cap, overflow).
struct WinRec {
    double q, second;
    int dir, a, b, flags;
};

struct RefineOut {
    double q;  // FP64 chord value at 0 of the bridge of the left and right sets
    int a, b;
    int ok, pad;
};

enum CounterIdx {
    C_POINTS = 0, C_NODES, C_LINES, C_VALID, C_LAMINATED, C_FP64, C_FULL, C_RARE, C_TIES,
    C_CAPS, C_WSTEPS, C_ROUNDS, C_FP64W, C_FP64R, C_FP64C, C_REFINED, C_OVERFLOW, C_WNODES,
    C_FALLBACK, C_REFFULL, C_BOUNDED, C_FLAT, C_RECENTRED, C_CERT, C_EDGE, C_DOUBLED, C_MIRROR,
    C_MIRROR_WON, C_NUM
};

// Pipeline passes over one level's queue.
enum PassKind {
    PASS_FULL = 0,      // every direction of the problem
    PASS_WINDOW = 1,    // the proposed angular window; failing nodes are deferred
    PASS_FALLBACK = 2   // every direction, over the deferred nodes
};

struct LineSpec {
    int L, m0, nfull, stride;  // samples, centre, full 128-chunks, per-warp buffer floats
    float h32;                 // sample spacing, FP32
    int pad;
    double h64;                // sample spacing, FP64
};

// One problem of a call (convexify_points is a batch of one).  Points of all
// problems share one global index space [point_off, point_off + n).
struct ProbDesc {
    LineSpec line;
    Material mat;
    double kappa;
    float kappa_f;
    int D, dir_off;  // directions [dir_off, dir_off + D) of the call's tables
    int K, NT;       // depth, tree nodes per point
    int chunks, dpi; // work items per node, directions per item
    int flags;       // cvx_params.flags
    // proposal window (surrogate_propose): half-width w on the Na x Nb angle
    // grid, wD = (2w + 1)^2 directions in wchunks items of wdpi; gap_tol of
    // the fallback test
    int window, Na, Nb, wD, wchunks, wdpi;
    int mwindow;  // half-width of the mirror window (0: none)
    double gap_tol;
    long long point_off, n;
    const double *F, *beta;
    double *W_R, *P;
    int32_t *status;
    cvx_laminate *root;
    cvx_node *tree;  // n x NT nodes
};

__device__ __forceinline__ cvx_node *node_ptr(const ProbDesc &pd, long long p, int hi) {
    return pd.tree + (p - pd.point_off) * pd.NT + hi;
}

// Device buffers of one pipeline run (all in one workspace).
struct Pipe {
    const ProbDesc *probs;
    int n_probs;
    long long N;         // points of all problems
    int K;               // largest depth
    int C;               // item stride per node (largest chunks)
    int stride32, stride64;
    int energy;
    int32_t *pid;        // problem of each global point
    int32_t *qp[kMaxDepth], *qh[kMaxDepth];  // node queues per level
    int32_t *cnt;        // node count per level (K + 1) and refine work count per level (K + 1)
    unsigned long long *item_ctr;  // work-item counter per level
    ItemCands *items;
    NodeCands *cands;
    int2 *work;
    RefineOut *refined;
    const float4 *dir32;
    const double *dir64;
    unsigned long long *counters;
    // windowed passes (carved only when window != 0)
    int window;
    int pass;                             // PassKind of the launches this Pipe drives
    int32_t *ncnt;                        // node counts the next level's queue uses
    int32_t *fq_p[kMaxDepth], *fq_h[kMaxDepth];  // nodes deferred to the full scan
    int32_t *fcnt;                        // their counts (as cnt)
    unsigned long long *fitem_ctr;
    int2 *center;                         // proposed window centre per queued node
    double *e_pred;                       // energy of the proposed laminate per queued node
    // window re-centring: two ping-pong queues of nodes whose window minimum
    // lay on the border, with their new centre and E_pred; per pass r a block
    // of 2 (K + 1) counts and K + 1 item counters
    int32_t *rq_p[2], *rq_h[2];
    int2 *rcen[2];
    double *rep[2];
    int32_t *rcnt;
    unsigned long long *ritem;
    // where this window pass sends nodes to re-centre (nullptr: to the full scan)
    int32_t *nx_p, *nx_h, *nx_cnt;
    int2 *nx_cen;
    double *nx_ep;
    // lane-per-line scan (damage energy): 1 selects it for this run's levels
    int lanes;
    // adaptive line window: the largest number of doublings of any problem
    // (the rescan passes use the re-centring queues)
    int adaptive;
    int *node_u;                          // per queued node: smallest FP32 upper bound (f2key)
    // mirror windows (CVX_FLAG_MIRROR_WINDOW): a main-stage window pass sends
    // nodes that split to the mirror queue with the mirror cell of their best
    // direction and that direction's result; the mirror stage's passes read
    // the problem table with the mirror window's geometry (mprobs) and, after
    // its first pass, the re-centring queues with records rrec
    int mirror_on;                        // 1: the run has mirror windows (buffers carved)
    int mirror;                           // 1: a pass of the mirror stage
    const ProbDesc *mprobs;
    int32_t *mq_p, *mq_h;                 // mirror queue of the current level
    int2 *mcen;
    WinRec *mrec;
    int32_t *mcnt;                        // its counts (as cnt)
    unsigned long long *mitem;
    WinRec *rrec[2];
    WinRec *rec;                          // records of the queue a mirror-stage pass reads
    WinRec *nx_rec;                       // where it sends re-centred nodes' records
};

// Bytes of the workspace part that depends on the shape (see pipe_layout).
size_t pipe_bytes(long long N, int K, int C, int n_probs, bool window = false,
                  bool rescan = false, bool mirror = false);
// Carves the workspace into the Pipe's buffers (p.N, K, C, n_probs, window set).
void pipe_layout(Pipe &p, char *ws);
// Enqueues the whole pipeline (zeroing, init, K levels, leaves) on s.
// ev (optional, 2*K events) brackets each line-scan launch.
cudaError_t pipe_enqueue(const Pipe &p, int warps, int grid, cudaStream_t s, cudaEvent_t *ev);
// The same in pieces: zeroing + init, one pass over one level, the leaves.
cudaError_t pipe_begin(const Pipe &p, cudaStream_t s);
cudaError_t pipe_level(const Pipe &p, int level, int warps, int grid, cudaStream_t s,
                       cudaEvent_t *ev);
cudaError_t pipe_end(const Pipe &p, cudaStream_t s);
// The Pipe that runs the full scan over the nodes a window pass deferred.
Pipe fallback_pipe(const Pipe &p, int level);
// The Pipe of window pass r (0: the level queue with the network's centres;
// r >= 1: the nodes re-centred by pass r - 1) with re-centring allowed while
// r < R.
Pipe window_pipe(const Pipe &p, int level, int r, int R);
// The Pipe of mirror-stage pass r (0: the mirror queue; r >= 1: the nodes
// re-centred by pass r - 1) with re-centring allowed while r < R.
Pipe mirror_pipe(const Pipe &p, int level, int r, int R);
// The Pipe of full-scan pass r of a level with adaptive line windows (0: the
// level queue; r >= 1: the nodes pass r - 1 sent back with a doubled window),
// sending nodes back while r < A.
Pipe rescan_pipe(const Pipe &p, int level, int r, int A);

// The line of a node with window exponent e: spacing h 2^e (exact in FP32
// and FP64).
__host__ __device__ inline LineSpec scaled_line(LineSpec l, int e) {
    if (e) {
        l.h32 = ldexpf(l.h32, e);
        l.h64 = ldexp(l.h64, e);
    }
    return l;
}
int scan_max_blocks_per_sm(int energy, int warps, int stride);
// Lane-per-line scan (cvx_scan_lanes.cu): whether it serves this energy (the
// damage energy, unless the environment variable CVX_SCAN_KERNEL is "warp"),
// its resident CTAs per SM, and its launch (node-bound reset included).
bool lane_scan_enabled(int energy);
int lane_scan_blocks_per_sm();
cudaError_t launch_scan_lanes(const Pipe &p, int level, int sms, cudaStream_t s);
// Directions per work item of the lane-per-line scan: whole nodes (a warp
// takes them in blocks of kLaneItemMax lines), smaller items (multiples of
// 32) when the nodes are too few for every warp of the grid to get two items.
inline int lane_dirs_per_item(long long n_nodes, int D, long long total_warps, int cap) {
    int dpi = D;
    if (cap > 0 && cap < dpi) dpi = cap;
    const long long want = total_warps * 2;
    if (n_nodes * ((D + dpi - 1) / dpi) < want) {
        const long long chunks = (want + n_nodes - 1) / n_nodes;
        long long d = (D + chunks - 1) / chunks;
        d = (d + 31) / 32 * 32;
        if (d < dpi) dpi = (int)d;
    }
    return dpi < D ? dpi : D;
}

// single steps
cudaError_t launch_energy(int64_t n, const double *F, const double *beta, double *W, double *P,
                          Material m, cudaStream_t s);
cudaError_t launch_history(int64_t n, const double *F, const double *bin, double *bout,
                           Material m, cudaStream_t s);
cudaError_t launch_sample_lines(int64_t n, const double *F, const double *beta,
                                const int32_t *dir, const float4 *dir32, int D, Material m,
                                LineSpec line, float *w, cudaStream_t s);
cudaError_t launch_hull(int64_t n, int L, const float *w, int32_t *mm, int32_t *mp, double *h,
                        unsigned long long *counters, cudaStream_t s);
cudaError_t launch_tree_tangent(int64_t n, int NT, const cvx_node *tree, const double *beta,
                                Material m, double *A, cudaStream_t s);

// Per-warp shared-memory stride of a line of L samples (16-byte aligned).
__host__ __device__ inline int line_stride(int L) { return (L + 3) & ~3; }

inline LineSpec make_line(int L, double t_half) {
    LineSpec l;
    l.L = L;
    l.m0 = (L - 1) / 2;
    l.h64 = 2.0 * t_half / (double)(L - 1);
    l.h32 = (float)l.h64;
    l.nfull = L >> 7;
    l.stride = line_stride(L);
    l.pad = 0;
    return l;
}

}  // namespace cvx
