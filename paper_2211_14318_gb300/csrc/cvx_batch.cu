// cvx_batch.cu -- convexify_batch: many problems in one pipeline run, captured
// as a CUDA graph and replayed; the autotuner that picks its launch shape.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "cvx_handle.h"

using namespace cvx;

struct cvx_batch_plan {
    std::string key;
    unsigned ws_gen = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    ProbDesc *h_table = nullptr;  // pinned: the graph copies it to the device
    float4 *d_dir32 = nullptr;
    double *d_dir64 = nullptr;
};

namespace cvx {

void destroy_batch_plan(cvx_handle *h) {
    cvx_batch_plan *p = h->plan;
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->h_table) cudaFreeHost(p->h_table);
    cudaFree(p->d_dir32);
    cudaFree(p->d_dir64);
    delete p;
    h->plan = nullptr;
}

}  // namespace cvx

namespace {

void append(std::string &k, const void *p, size_t n) { k.append((const char *)p, n); }

// Everything that a captured graph depends on: shapes, parameters, direction
// rows and the caller's pointers.
std::string signature(int np, const cvx_problem *pr) {
    std::string k;
    for (int i = 0; i < np; ++i) {
        const cvx_problem &q = pr[i];
        cvx_params pp = q.params;
        const double *rows = pp.dirs;
        pp.dirs = nullptr;
        append(k, &pp, sizeof pp);
        if (rows) append(k, rows, sizeof(double) * 4 * (size_t)q.params.n_dirs);
        append(k, &q.n, sizeof q.n);
        const void *ptrs[6] = {q.F, q.beta_k, q.W_R, q.P, q.status, q.root};
        append(k, ptrs, sizeof ptrs);
    }
    return k;
}

// What the launch shape depends on: energy and the set of (L, D, K).
std::string tune_key(int np, const cvx_problem *pr) {
    std::set<std::string> s;
    for (int i = 0; i < np; ++i) {
        const cvx_params &p = pr[i].params;
        const int D = p.dirs ? p.n_dirs : p.n_theta_a * p.n_theta_b;
        char b[64];
        snprintf(b, sizeof b, "%d.%d.%d", p.line_points, D, p.depth);
        s.insert(b);
    }
    std::string k = "e" + std::to_string(pr[0].params.energy);
    for (auto &x : s) k += "_" + x;
    return k;
}

void load_tune_file(cvx_handle *h) {
    const char *path = getenv("CVX_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[4096];
    while (fgets(line, sizeof line, f)) {
        char key[3000];
        int w = 0, d = 0;
        // warps 0: the lane-per-line scan; 1..8: the warp-per-line scan
        if (sscanf(line, " \"%2999[^\"]\": [%d, %d]", key, &w, &d) == 3 && w >= 0 && w <= 8)
            h->tune_cache[key] = {w, d};
    }
    fclose(f);
}

void save_tune_file(const cvx_handle *h) {
    const char *path = getenv("CVX_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : h->tune_cache)
        fprintf(f, "  \"%s\": [%d, %d]%s\n", kv.first.c_str(), kv.second.first, kv.second.second,
                ++i < h->tune_cache.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
}

struct Layout {
    Pipe pipe;
    std::vector<ProbDesc> table;
    int grid = 0;
};

// Builds the problem table and carves the workspace for the given problems
// (n_use[i] points of problem i) and launch shape.
int build_layout(cvx_handle *h, int np, const cvx_problem *pr, const std::vector<long long> &n_use,
                 const std::vector<int> &dir_off, const float4 *d32, const double *d64, int warps,
                 int dpi_cap, cudaStream_t s, Layout &lo) {
    int stride = 4;
    int K = 0;
    long long N = 0;
    for (int i = 0; i < np; ++i) {
        stride = std::max(stride, line_stride(pr[i].params.line_points));
        K = std::max(K, pr[i].params.depth);
        N += n_use[i];
    }
    const int energy = pr[0].params.energy;
    const int bpsm = scan_max_blocks_per_sm(energy, warps > 0 ? warps : 8, stride);
    if (bpsm < 1) return fail(CVX_ERR_UNSUPPORTED, "scan kernel cannot launch with %d warps", warps);
    lo.grid = h->sm_count * bpsm;
    // warps == 0: the lane-per-line scan (damage energy)
    const bool lanes = warps == 0;
    if (lanes && !lane_scan_enabled(energy))
        return fail(CVX_ERR_UNSUPPORTED, "lane-per-line scan not available for this energy");
    const long long lane_warps = (long long)h->sm_count * lane_scan_blocks_per_sm() * 8;
    lo.table.assign(np, ProbDesc{});
    int C = 1, A = 0;
    long long off = 0;
    size_t tree_bytes = 0;
    std::vector<size_t> tree_off(np);
    for (int i = 0; i < np; ++i) {
        const cvx_params &p = pr[i].params;
        ProbDesc &pd = lo.table[i];
        pd.line = make_line(p.line_points, p.t_half);
        pd.mat = material_of(&p);
        pd.kappa = line_kappa(pd.mat);
        pd.kappa_f = (float)pd.kappa;
        pd.D = p.dirs ? p.n_dirs : p.n_theta_a * p.n_theta_b;
        pd.dir_off = dir_off[i];
        pd.flags = p.flags;
        A = std::max(A, (int)CVX_WINDOW_DOUBLINGS_OF(p.flags));
        pd.K = p.depth;
        pd.NT = (1 << (p.depth + 1)) - 1;
        pd.dpi = lanes ? lane_dirs_per_item(N, pd.D, lane_warps, dpi_cap)
                       : dirs_per_item(N, pd.D, lo.grid, warps, dpi_cap);
        pd.chunks = (pd.D + pd.dpi - 1) / pd.dpi;
        C = std::max(C, pd.chunks);
        pd.point_off = off;
        pd.n = n_use[i];
        off += n_use[i];
        pd.F = pr[i].F;
        pd.beta = pr[i].beta_k;
        pd.W_R = pr[i].W_R;
        pd.P = pr[i].P;
        pd.status = pr[i].status;
        pd.root = pr[i].root;
        tree_off[i] = tree_bytes;
        tree_bytes += ((sizeof(cvx_node) * (size_t)n_use[i] * pd.NT) + 255) & ~(size_t)255;
    }
    Pipe &pp = lo.pipe;
    pp = Pipe{};
    pp.n_probs = np;
    pp.N = N;
    pp.K = K;
    pp.C = C;
    pp.stride32 = pp.stride64 = stride;
    pp.energy = energy;
    pp.lanes = lanes ? 1 : 0;
    pp.adaptive = A;
    const size_t pipe_sz = (pipe_bytes(N, K, C, np, false, A > 0) + 255) & ~(size_t)255;
    int rc = ensure_ws(h, pipe_sz + tree_bytes, s);
    if (rc) return rc;
    pipe_layout(pp, h->ws);
    for (int i = 0; i < np; ++i) lo.table[i].tree = (cvx_node *)(h->ws + pipe_sz + tree_off[i]);
    pp.dir32 = d32;
    pp.dir64 = d64;
    pp.counters = h->d_counters;
    return CVX_OK;
}

}  // namespace

extern "C" {

int cvx_get_batch_tuning(cvx_handle *h, int *warps_per_cta, int *dirs_per_item_cap,
                         int *from_cache) {
    if (!h || !warps_per_cta || !dirs_per_item_cap || !from_cache)
        return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    *warps_per_cta = h->last_tune_warps;
    *dirs_per_item_cap = h->last_tune_dpi;
    *from_cache = h->last_tune_cached;
    return CVX_OK;
}

int convexify_batch(cvx_handle *h, int np, const cvx_problem *pr, cvx_stream sv) {
    if (np < 1 || np > 65536 || !pr) return fail(CVX_ERR_INVALID_ARG, "need 1 to 65536 problems");
    long long N = 0;
    for (int i = 0; i < np; ++i) {
        int rc = check_params(&pr[i].params, true);
        if (rc) return rc;
        if (pr[i].params.energy != pr[0].params.energy)
            return fail(CVX_ERR_INVALID_ARG, "all problems of a batch must use the same energy");
        if (pr[i].n < 0) return fail(CVX_ERR_INVALID_ARG, "problem %d: n < 0", i);
        if (pr[i].n > 0 && (!pr[i].F || !pr[i].beta_k || !pr[i].W_R || !pr[i].P || !pr[i].status))
            return fail(CVX_ERR_INVALID_ARG, "problem %d: NULL array", i);
        N += pr[i].n;
    }
    if (N > ((long long)1 << 31) / 256) return fail(CVX_ERR_INVALID_ARG, "more than 2^23 points");
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (N == 0) return CVX_OK;
    cudaStream_t s = (cudaStream_t)sv;
    DeviceGuard g(h->device);

    const std::string key = signature(np, pr);
    if (h->plan && h->plan->key == key && h->plan->ws_gen == h->ws_gen) {
        CK(cudaGraphLaunch(h->plan->exec, s), "convexify_batch/replay");
        return CVX_OK;
    }
    destroy_batch_plan(h);
    cvx_batch_plan *plan = new cvx_batch_plan();
    h->plan = plan;
    plan->key = key;

    // direction tables, one copy per distinct direction set
    std::vector<int> dir_off(np);
    std::map<std::string, int> seen;
    std::vector<double> all64, rows;
    for (int i = 0; i < np; ++i) {
        const cvx_params &p = pr[i].params;
        std::string dk;
        if (p.dirs) {
            dk = "c";
            append(dk, p.dirs, sizeof(double) * 4 * (size_t)p.n_dirs);
        } else {
            dk = "g" + std::to_string(p.n_theta_a) + "x" + std::to_string(p.n_theta_b);
        }
        auto it = seen.find(dk);
        if (it != seen.end()) {
            dir_off[i] = it->second;
            continue;
        }
        direction_rows(&p, rows);
        dir_off[i] = (int)(all64.size() / 4);
        seen[dk] = dir_off[i];
        all64.insert(all64.end(), rows.begin(), rows.end());
    }
    const int Dall = (int)(all64.size() / 4);
    std::vector<float4> all32(Dall);
    for (int k = 0; k < Dall; ++k)
        all32[k] = make_float4((float)all64[4 * k], (float)all64[4 * k + 1],
                               (float)all64[4 * k + 2], (float)all64[4 * k + 3]);
    CK(cudaMalloc(&plan->d_dir32, sizeof(float4) * Dall), "convexify_batch/directions");
    CK(cudaMalloc(&plan->d_dir64, sizeof(double) * 4 * Dall), "convexify_batch/directions");
    CK(cudaMemcpy(plan->d_dir32, all32.data(), sizeof(float4) * Dall, cudaMemcpyHostToDevice),
       "convexify_batch/directions");
    CK(cudaMemcpy(plan->d_dir64, all64.data(), sizeof(double) * 4 * Dall, cudaMemcpyHostToDevice),
       "convexify_batch/directions");

    // launch shape: cached, or timed trials on a sample of the points
    if (h->tune_cache.empty()) load_tune_file(h);
    const std::string tk = tune_key(np, pr);
    int warps = 8, dpi_cap = 0;
    auto tc = h->tune_cache.find(tk);
    if (tc != h->tune_cache.end()) {
        warps = tc->second.first;
        dpi_cap = tc->second.second;
        h->last_tune_cached = 1;
    } else {
        std::vector<long long> n_s(np);
        const long long S = 8192;
        for (int i = 0; i < np; ++i)
            n_s[i] = pr[i].n ? std::max(1LL, std::min((long long)pr[i].n, (pr[i].n * S + N - 1) / N))
                             : 0;
        float best = 3.4e38f;
        bool warmed = false;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "autotune");
        CK(cudaEventCreate(&e1), "autotune");
        // launch shapes: the warp-per-line scan with 4 or 8 warps per CTA (it is
        // compiled for at most 256 threads) and three item caps, and (damage
        // energy) the lane-per-line scan (warps 0) with three item caps
        std::vector<std::pair<int, int>> shapes;
        for (int w : {4, 8})
            for (int cap : {256, 1024, 0}) shapes.push_back({w, cap});
        if (lane_scan_enabled(pr[0].params.energy))
            for (int cap : {64, 128, 0}) shapes.push_back({0, cap});
        for (const auto &sh : shapes) {
            const int w = sh.first, cap = sh.second;
            {
                Layout lo;
                int rc = build_layout(h, np, pr, n_s, dir_off, plan->d_dir32, plan->d_dir64, w,
                                      cap, s, lo);
                if (rc) continue;
                CK(cudaMemcpyAsync((void *)lo.pipe.probs, lo.table.data(),
                                   sizeof(ProbDesc) * np, cudaMemcpyHostToDevice, s),
                   "autotune");
                if (!warmed)  // one untimed run before the first timed trial
                    CK(pipe_enqueue(lo.pipe, w, lo.grid, s, nullptr), "autotune");
                warmed = true;
                CK(cudaEventRecord(e0, s), "autotune");
                CK(pipe_enqueue(lo.pipe, w, lo.grid, s, nullptr), "autotune");
                CK(cudaEventRecord(e1, s), "autotune");
                CK(cudaEventSynchronize(e1), "autotune");
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, e0, e1), "autotune");
                if (ms < best) {
                    best = ms;
                    warps = w;
                    dpi_cap = cap;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h->tune_cache[tk] = {warps, dpi_cap};
        save_tune_file(h);
        h->last_tune_cached = 0;
    }
    h->last_tune_warps = warps;
    h->last_tune_dpi = dpi_cap;

    // the real layout, captured once
    std::vector<long long> n_all(np);
    for (int i = 0; i < np; ++i) n_all[i] = pr[i].n;
    Layout lo;
    int rc = build_layout(h, np, pr, n_all, dir_off, plan->d_dir32, plan->d_dir64, warps, dpi_cap,
                          s, lo);
    if (rc) return rc;
    CK(cudaMallocHost(&plan->h_table, sizeof(ProbDesc) * np), "convexify_batch/table");
    memcpy(plan->h_table, lo.table.data(), sizeof(ProbDesc) * np);
    CK(cudaStreamCreateWithFlags(&plan->cap, cudaStreamNonBlocking), "convexify_batch/capture");
    CK(cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeRelaxed), "convexify_batch/capture");
    cudaError_t e = cudaMemcpyAsync((void *)lo.pipe.probs, plan->h_table, sizeof(ProbDesc) * np,
                                    cudaMemcpyHostToDevice, plan->cap);
    if (e == cudaSuccess) e = pipe_enqueue(lo.pipe, warps, lo.grid, plan->cap, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(plan->cap, &graph);
    if (e != cudaSuccess) return cuda_fail(e, "convexify_batch/capture");
    if (e2 != cudaSuccess) return cuda_fail(e2, "convexify_batch/capture");
    plan->graph = graph;
    CK(cudaGraphInstantiate(&plan->exec, graph, 0), "convexify_batch/instantiate");
    plan->ws_gen = h->ws_gen;
    CK(cudaGraphLaunch(plan->exec, s), "convexify_batch/launch");
    return CVX_OK;
}

}  // extern "C"
