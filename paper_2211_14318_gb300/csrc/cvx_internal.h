// cvx_internal.h -- structures shared by the kernels and the host side of
// libconvexify (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "convexify.h"
#include "cvx_device.cuh"

namespace cvx {

enum { CVX_NODE_ITER_CAP = 64, CVX_NODE_OVERFLOW = 128 };

constexpr int kWarpTop = 4;    // best directions kept per warp
constexpr int kItemTop = 8;    // per work item
constexpr int kNodeCand = 16;  // candidates refined in FP64 per node
// Bound on the FP32 sampling error of kappa W (kappa-scaled units, relative to
// max(kappa, |q|)): 3.5 times the largest error measured against FP64.
constexpr float kEps32 = 1.1e-6f;

// Best directions of one work item (a node and a block of its directions),
// ranked by q = a rigorous lower bound on the value at t = 0 of the hull of the
// FP32 samples of the left and right sets (the node's hull value when the
// centre does not lie below it); qhi_min is the smallest upper bound seen.
struct ItemCands {
    float q[kItemTop];
    int dir[kItemTop];
    float w0;       // FP32 centre sample
    float dropped;  // smallest q not kept
    float qhi_min;  // smallest upper bound over the item's directions
    int n, flags, pad;
};

struct NodeCands {
    int dir[kNodeCand];
    int n, flags;
    float qcut;  // smallest FP32 q of a direction not refined (kappa-scaled)
    float eps;   // FP32 error bound used at this node (kappa-scaled)
};

struct RefineOut {
    double q;  // FP64 chord value at 0 of the bridge of the left and right sets
    int a, b;
    int ok, pad;
};

enum CounterIdx {
    C_POINTS = 0, C_NODES, C_LINES, C_VALID, C_LAMINATED, C_FP64, C_FULL, C_RARE, C_TIES,
    C_CAPS, C_WSTEPS, C_ROUNDS, C_FP64W, C_FP64R, C_FP64C, C_REFINED, C_OVERFLOW, C_NUM
};

struct LineSpec {
    int L, m0, nfull, stride;  // samples, centre, full 128-chunks, per-warp buffer floats
    float h32;                 // sample spacing, FP32
    double h64;                // sample spacing, FP64
};

struct ScanArgs {
    const cvx_node *tree;
    int NT;
    const double *beta;
    const int32_t *q_point, *q_heap, *q_count;
    const float4 *dir32;
    int D, chunks, dirs_per_item;
    Material mat;
    LineSpec line;
    ItemCands *out;
    unsigned long long *counters;
};

struct SelectArgs {
    const int32_t *q_count;
    const ItemCands *items;
    int chunks;
    float kappa;
    NodeCands *cands;
    int2 *work;  // (queue index, candidate index)
    int32_t *work_count;
    unsigned long long *counters;
};

struct RefineArgs {
    const cvx_node *tree;
    int NT;
    const double *beta;
    const int32_t *q_point, *q_heap;
    const NodeCands *cands;
    const int2 *work;
    const int32_t *work_count;
    const double *dir64;
    Material mat;
    LineSpec line;
    RefineOut *out;
};

struct CommitArgs {
    cvx_node *tree;
    int NT, level, depth;
    const double *beta;
    const int32_t *q_point, *q_heap, *q_count;
    int32_t *nq_point, *nq_heap, *nq_count;
    const NodeCands *cands;
    const RefineOut *refined;
    const double *dir64;
    double kappa;
    Material mat;
    LineSpec line;
    unsigned long long *counters;
};

struct InitArgs {
    int64_t n;
    const double *F, *beta;
    cvx_node *tree;
    int NT, depth;
    int32_t *q_point, *q_heap, *q_count;
    int32_t *status;
    Material mat;
    int m0;
    unsigned long long *counters;
};

struct LeafArgs {
    int64_t n;
    const cvx_node *tree;
    int NT;
    const double *beta;
    double *W_R, *P;
    int32_t *status;
    cvx_laminate *root;
    Material mat;
};

// kernel launchers (cvx_kernels.cu)
cudaError_t launch_init(const InitArgs &a, cudaStream_t s);
cudaError_t launch_scan(const ScanArgs &a, int warps, int grid, cudaStream_t s);
int scan_max_blocks_per_sm(int energy, int warps, int stride);
cudaError_t launch_select(const SelectArgs &a, int64_t max_nodes, cudaStream_t s);
cudaError_t launch_refine(const RefineArgs &a, int64_t max_work, cudaStream_t s);
cudaError_t launch_commit(const CommitArgs &a, int64_t max_nodes, cudaStream_t s);
cudaError_t launch_leaf(const LeafArgs &a, cudaStream_t s);
cudaError_t launch_energy(int64_t n, const double *F, const double *beta, double *W, double *P,
                          Material m, cudaStream_t s);
cudaError_t launch_history(int64_t n, const double *F, const double *bin, double *bout,
                           Material m, cudaStream_t s);
cudaError_t launch_sample_lines(int64_t n, const double *F, const double *beta,
                                const int32_t *dir, const float4 *dir32, int D, Material m,
                                LineSpec line, float *w, cudaStream_t s);
cudaError_t launch_hull(int64_t n, int L, const float *w, int32_t *mm, int32_t *mp, double *h,
                        unsigned long long *counters, cudaStream_t s);

// Per-warp shared-memory stride of a line of L samples (16-byte aligned).
__host__ __device__ inline int line_stride(int L) { return (L + 3) & ~3; }

}  // namespace cvx
