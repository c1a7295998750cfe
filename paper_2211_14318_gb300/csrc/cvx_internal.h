// cvx_internal.h -- structures shared by the kernels and the host side of
// libconvexify (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "convexify.h"
#include "cvx_device.cuh"

namespace cvx {

enum { CVX_NODE_ITER_CAP = 64 };

// Best line of one work item (a node and a block of its directions).
struct ItemBest {
    double h;    // hull value at 0 (FP64 of the FP32 samples)
    float h32;   // FP32 estimate of h
    float h2;    // FP32 second-best hull value seen in the item
    int32_t dir, mm, mp, flags;
};
static_assert(sizeof(ItemBest) == 32, "ItemBest layout");

enum CounterIdx {
    C_POINTS = 0, C_NODES, C_LINES, C_VALID, C_LAMINATED, C_FP64, C_FULL, C_RARE, C_TIES,
    C_CAPS, C_WSTEPS, C_ROUNDS, C_FP64W, C_FP64R, C_FP64C, C_DIR64, C_NUM
};

struct LineSpec {
    int L, m0;
    float h32;    // sample spacing, FP32
    double h64;   // sample spacing, FP64
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
    ItemBest *out;
    unsigned long long *counters;
};

struct ExpandArgs {
    cvx_node *tree;
    int NT, level, depth;
    const double *beta;
    const int32_t *q_point, *q_heap, *q_count;
    int32_t *nq_point, *nq_heap, *nq_count;
    const ItemBest *items;
    int chunks;
    const double *dir64;
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
cudaError_t launch_scan(const ScanArgs &a, int energy, int ns, int warps, int grid,
                        cudaStream_t s);
int scan_max_blocks_per_sm(int energy, int ns, int warps);
cudaError_t launch_expand(const ExpandArgs &a, int64_t max_nodes, cudaStream_t s);
cudaError_t launch_leaf(const LeafArgs &a, cudaStream_t s);
cudaError_t launch_energy(int64_t n, const double *F, const double *beta, double *W, double *P,
                          Material m, cudaStream_t s);
cudaError_t launch_history(int64_t n, const double *F, const double *bin, double *bout,
                           Material m, cudaStream_t s);
cudaError_t launch_sample_lines(int64_t n, const double *F, const double *beta,
                                const int32_t *dir, const float4 *dir32, int D, Material m,
                                LineSpec line, int ns, float *w, cudaStream_t s);
cudaError_t launch_hull(int64_t n, int L, int ns, const float *w, int32_t *mm, int32_t *mp,
                        double *h, unsigned long long *counters, cudaStream_t s);

inline int slots_for(int L) {
    int ns = (L + 31) / 32;
    if (ns <= 8) return 8;
    if (ns <= 17) return 17;
    if (ns <= 33) return 33;
    if (ns <= 65) return 65;
    return -1;
}

}  // namespace cvx
