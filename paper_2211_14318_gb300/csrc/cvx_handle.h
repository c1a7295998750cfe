// cvx_handle.h -- host-side state behind cvx_handle and helpers shared by the
// entry points (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "convexify.h"
#include "cvx_internal.h"

struct cvx_batch_plan;  // cvx_batch.cu
namespace cvx {
struct Surrogate;  // cvx_surrogate.cu
}

struct cvx_handle {
    int device = 0;
    int sm_count = 0;
    // direction table of the last convexify_points / single-step call
    int dir_na = -1, dir_nb = -1;
    bool dir_custom = false;
    int D = 0;
    size_t dir_cap = 0;
    float4 *d_dir32 = nullptr;
    double *d_dir64 = nullptr;
    // workspace (grown with cudaMalloc; ws_gen counts reallocations)
    char *ws = nullptr;
    size_t ws_cap = 0;
    unsigned ws_gen = 0;
    unsigned long long *d_counters = nullptr;
    int tune_warps = 8;
    int tune_dpi = 0;
    // optional CUDA-event timing of the scan launches
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_pool;
    // batched form: captured graph of the last problem set, autotune cache
    cvx_batch_plan *plan = nullptr;
    std::map<std::string, std::pair<int, int>> tune_cache;
    int last_tune_warps = 0, last_tune_dpi = 0, last_tune_cached = 0;
    // surrogate proposal network (weights, optimiser state, batch buffers)
    cvx::Surrogate *sur = nullptr;
};

namespace cvx {

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *where);
Material material_of(const cvx_params *p);
// allow_stvk: the St. Venant-Kirchhoff energy (global-grid calls only).
int check_params(const cvx_params *p, bool need_line, bool allow_stvk = false);
int ensure_ws(cvx_handle *h, size_t bytes, cudaStream_t s);
// With profiling on: n_launches event pairs (2 per line-scan launch, recorded
// on the launching stream around it), registered for cvx_get_scan_timing.
int scan_events(cvx_handle *h, int n_launches, std::vector<cudaEvent_t> &ev);
// Direction table of the handle for a parameter set (angle grid or custom).
int ensure_dirs(cvx_handle *h, const cvx_params *p, cudaStream_t s);
// Direction rows (a1, a2, b1, b2) of a parameter set, FP64.
void direction_rows(const cvx_params *p, std::vector<double> &rows);
void destroy_batch_plan(cvx_handle *h);
void destroy_surrogate(cvx_handle *h);

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Work items per node: whole nodes when there are enough of them, otherwise
// split the directions so every SM gets work.
inline int dirs_per_item(long long n_nodes, int D, int grid, int warps, int cap) {
    int dpi;
    const long long want_items = (long long)grid * 4;
    if (n_nodes >= want_items) {
        dpi = D;
    } else {
        const long long chunks = (want_items + n_nodes - 1) / n_nodes;
        const long long d = (D + chunks - 1) / chunks;
        dpi = (int)(d > warps * 2 ? d : warps * 2);
    }
    if (cap > 0 && dpi > cap) dpi = cap;
    return dpi < D ? dpi : D;
}

}  // namespace cvx

#define CK(call, where)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cvx::cuda_fail(e_, where); \
    } while (0)
