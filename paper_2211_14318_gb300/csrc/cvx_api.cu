// cvx_api.cu -- host side of the C ABI declared in include/convexify.h:
// argument validation, the handle (workspace, direction tables, counters),
// and the enqueueing of the per-level kernels on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "convexify.h"
#include "cvx_internal.h"

using namespace cvx;

struct cvx_handle {
    int device = 0;
    int sm_count = 0;
    // direction table cache
    int dir_na = -1, dir_nb = -1;
    bool dir_custom = false;
    int D = 0;
    size_t dir_cap = 0;
    float4 *d_dir32 = nullptr;
    double *d_dir64 = nullptr;
    // workspace
    char *ws = nullptr;
    size_t ws_cap = 0;
    unsigned long long *d_counters = nullptr;
    int tune_warps = 8;
    int tune_dpi = 0;
    // optional CUDA-event timing of the scan launches
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_pool;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(CVX_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    return fail(CVX_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

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

Material material_of(const cvx_params *p) {
    Material m;
    m.mu = p->mu;
    m.lam = p->lambda_L;
    m.Dinf = p->D_inf;
    m.D0 = p->D0;
    m.energy = p->energy;
    return m;
}

int check_params(const cvx_params *p, bool need_line) {
    if (!p) return fail(CVX_ERR_INVALID_ARG, "params is NULL");
    if (p->energy != CVX_ENERGY_NH_DAMAGE && p->energy != CVX_ENERGY_DOUBLE_WELL)
        return fail(CVX_ERR_INVALID_ARG, "unknown energy kind %d", p->energy);
    if (p->energy == CVX_ENERGY_NH_DAMAGE) {
        if (!(p->mu > 0.0) || !(p->lambda_L >= 0.0) || !(p->D_inf >= 0.0 && p->D_inf < 1.0) ||
            !(p->D0 > 0.0))
            return fail(CVX_ERR_INVALID_ARG,
                        "material out of range (mu > 0, lambda >= 0, 0 <= D_inf < 1, D0 > 0)");
    }
    if (p->flags != 0) return fail(CVX_ERR_INVALID_ARG, "flags must be 0");
    if (!need_line) return CVX_OK;
    if (p->line_points < 3 || p->line_points > 2079 || (p->line_points % 2) == 0)
        return fail(CVX_ERR_INVALID_ARG, "line_points must be odd in [3, 2079], got %d",
                    p->line_points);
    if (!(p->t_half > 0.0) || !isfinite(p->t_half))
        return fail(CVX_ERR_INVALID_ARG, "t_half must be positive");
    if (p->depth < 0 || p->depth > 8)
        return fail(CVX_ERR_INVALID_ARG, "depth must be in [0, 8], got %d", p->depth);
    if (p->dirs) {
        if (p->n_dirs < 1 || p->n_dirs > (1 << 20))
            return fail(CVX_ERR_INVALID_ARG, "n_dirs must be in [1, 2^20]");
    } else {
        if (p->n_theta_a < 1 || p->n_theta_b < 1 ||
            (int64_t)p->n_theta_a * p->n_theta_b > (1 << 20))
            return fail(CVX_ERR_INVALID_ARG, "angle grid must be >= 1 x 1 and <= 2^20 directions");
    }
    return CVX_OK;
}

LineSpec line_of(const cvx_params *p) {
    LineSpec l;
    l.L = p->line_points;
    l.m0 = (p->line_points - 1) / 2;
    l.h64 = 2.0 * p->t_half / (double)(p->line_points - 1);
    l.h32 = (float)l.h64;
    l.nfull = l.L >> 7;
    l.stride = line_stride(l.L);
    return l;
}

// Direction table: a_i = (cos pi i/Na, sin pi i/Na), b_j likewise, j_dir = i Nb + j,
// or a copy of the caller's rows.
int ensure_dirs(cvx_handle *h, const cvx_params *p, cudaStream_t s) {
    if (!p->dirs && !h->dir_custom && h->dir_na == p->n_theta_a && h->dir_nb == p->n_theta_b)
        return CVX_OK;
    const int D = p->dirs ? p->n_dirs : p->n_theta_a * p->n_theta_b;
    std::vector<double> d64((size_t)D * 4);
    if (p->dirs) {
        memcpy(d64.data(), p->dirs, sizeof(double) * 4 * (size_t)D);
    } else {
        for (int i = 0; i < p->n_theta_a; ++i) {
            const double ta = M_PI * (double)i / (double)p->n_theta_a;
            for (int j = 0; j < p->n_theta_b; ++j) {
                const double tb = M_PI * (double)j / (double)p->n_theta_b;
                double *r = &d64[4 * ((size_t)i * p->n_theta_b + j)];
                r[0] = cos(ta);
                r[1] = sin(ta);
                r[2] = cos(tb);
                r[3] = sin(tb);
            }
        }
    }
    std::vector<float4> d32(D);
    for (int k = 0; k < D; ++k)
        d32[k] = make_float4((float)d64[4 * k], (float)d64[4 * k + 1], (float)d64[4 * k + 2],
                             (float)d64[4 * k + 3]);
    if ((size_t)D > h->dir_cap) {
        CK(cudaStreamSynchronize(s), "direction table");
        cudaFree(h->d_dir32);
        cudaFree(h->d_dir64);
        h->d_dir32 = nullptr;
        h->d_dir64 = nullptr;
        h->dir_cap = 0;
        CK(cudaMalloc(&h->d_dir32, sizeof(float4) * D), "direction table");
        CK(cudaMalloc(&h->d_dir64, sizeof(double) * 4 * D), "direction table");
        h->dir_cap = D;
    }
    // synchronous copies: the host vectors die at return
    CK(cudaStreamSynchronize(s), "direction table");
    CK(cudaMemcpy(h->d_dir32, d32.data(), sizeof(float4) * D, cudaMemcpyHostToDevice),
       "direction table");
    CK(cudaMemcpy(h->d_dir64, d64.data(), sizeof(double) * 4 * D, cudaMemcpyHostToDevice),
       "direction table");
    h->D = D;
    h->dir_custom = p->dirs != nullptr;
    h->dir_na = p->dirs ? -1 : p->n_theta_a;
    h->dir_nb = p->dirs ? -1 : p->n_theta_b;
    return CVX_OK;
}

int ensure_ws(cvx_handle *h, size_t bytes, cudaStream_t s) {
    if (bytes <= h->ws_cap) return CVX_OK;
    CK(cudaStreamSynchronize(s), "workspace");
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_cap = 0;
    size_t cap = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&h->ws, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CVX_ERR_OOM, "workspace of %zu bytes: %s", cap, cudaGetErrorString(e));
    }
    h->ws_cap = cap;
    return CVX_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace cvx {
// Records the calling thread's last error for entry points in other files.
int set_error_message(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace cvx

extern "C" {

int cvx_last_error(char *buf, size_t len) {
    if (buf && len) {
        size_t n = std::min(len - 1, g_err.size());
        memcpy(buf, g_err.data(), n);
        buf[n] = 0;
    }
    return (int)g_err.size();
}

int cvx_create(cvx_handle **out, int device) {
    if (!out) return fail(CVX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int nd = 0;
    CK(cudaGetDeviceCount(&nd), "cudaGetDeviceCount");
    if (device < 0 || device >= nd)
        return fail(CVX_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, nd);
    DeviceGuard g(device);
    cvx_handle *h = new cvx_handle();
    h->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_counters, sizeof(unsigned long long) * C_NUM);
    if (e == cudaSuccess) e = cudaMemset(h->d_counters, 0, sizeof(unsigned long long) * C_NUM);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cvx_create");
    }
    *out = h;
    return CVX_OK;
}

int cvx_destroy(cvx_handle *h) {
    if (!h) return CVX_OK;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    for (auto *v : {&h->ev_pending, &h->ev_pool})
        for (auto &e : *v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    cudaFree(h->d_dir32);
    cudaFree(h->d_dir64);
    cudaFree(h->ws);
    cudaFree(h->d_counters);
    delete h;
    return CVX_OK;
}

int cvx_get_stats(cvx_handle *h, cvx_stats *out, int reset) {
    if (!h || !out) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(h->device);
    unsigned long long c[C_NUM];
    CK(cudaDeviceSynchronize(), "cvx_get_stats");
    CK(cudaMemcpy(c, h->d_counters, sizeof c, cudaMemcpyDeviceToHost), "cvx_get_stats");
    out->points = (int64_t)c[C_POINTS];
    out->nodes_scanned = (int64_t)c[C_NODES];
    out->lines = (int64_t)c[C_LINES];
    out->valid_samples = (int64_t)c[C_VALID];
    out->laminated = (int64_t)c[C_LAMINATED];
    out->fp64_checks = (int64_t)c[C_FP64];
    out->full_passes = (int64_t)c[C_FULL];
    out->rare_paths = (int64_t)c[C_RARE];
    out->ties = (int64_t)c[C_TIES];
    out->iter_caps = (int64_t)c[C_CAPS];
    out->window_steps = (int64_t)c[C_WSTEPS];
    out->rounds = (int64_t)c[C_ROUNDS];
    out->fp64_window = (int64_t)c[C_FP64W];
    out->fp64_rare = (int64_t)c[C_FP64R];
    out->fp64_center = (int64_t)c[C_FP64C];
    out->refined = (int64_t)c[C_REFINED];
    out->overflow = (int64_t)c[C_OVERFLOW];
    if (reset) CK(cudaMemset(h->d_counters, 0, sizeof c), "cvx_get_stats");
    return CVX_OK;
}

int cvx_set_profiling(cvx_handle *h, int enable) {
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    h->profiling = enable != 0;
    return CVX_OK;
}

int cvx_get_scan_timing(cvx_handle *h, double *ms, int64_t *launches, int reset) {
    if (!h || !ms || !launches) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(h->device);
    double tot = 0.0;
    for (auto &e : h->ev_pending) {
        CK(cudaEventSynchronize(e.second), "cvx_get_scan_timing");
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, e.first, e.second), "cvx_get_scan_timing");
        tot += t;
    }
    *ms = tot;
    *launches = (int64_t)h->ev_pending.size();
    if (reset) {
        for (auto &e : h->ev_pending) h->ev_pool.push_back(e);
        h->ev_pending.clear();
    }
    return CVX_OK;
}

int cvx_struct_size(int which) {
    switch (which) {
    case 0: return (int)sizeof(cvx_params);
    case 1: return (int)sizeof(cvx_node);
    case 2: return (int)sizeof(cvx_laminate);
    case 3: return (int)sizeof(cvx_stats);
    default: return -1;
    }
}

int cvx_set_tuning(cvx_handle *h, int warps_per_cta, int dirs_per_item) {
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (warps_per_cta < 1 || warps_per_cta > 16)
        return fail(CVX_ERR_INVALID_ARG, "warps_per_cta must be in [1, 16]");
    if (dirs_per_item < 0) return fail(CVX_ERR_INVALID_ARG, "dirs_per_item must be >= 0");
    h->tune_warps = warps_per_cta;
    h->tune_dpi = dirs_per_item;
    return CVX_OK;
}

int cvx_energy(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
               const double *beta_k, double *W, double *P, cvx_stream s) {
    int rc = check_params(p, false);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!F || !beta_k || !W)) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    CK(launch_energy(n, F, beta_k, W, P, material_of(p), (cudaStream_t)s), "cvx_energy");
    return CVX_OK;
}

int cvx_history_update(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
                       const double *beta_in, double *beta_out, cvx_stream s) {
    int rc = check_params(p, false);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!F || !beta_out)) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    CK(launch_history(n, F, beta_in, beta_out, material_of(p), (cudaStream_t)s),
       "cvx_history_update");
    return CVX_OK;
}

int cvx_sample_lines(cvx_handle *h, const cvx_params *p, int64_t n_lines, const double *F,
                     const double *beta_k, const int32_t *dir, float *w, cvx_stream s) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n_lines < 0) return fail(CVX_ERR_INVALID_ARG, "n_lines < 0");
    if (n_lines > 0 && (!F || !beta_k || !dir || !w)) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    rc = ensure_dirs(h, p, (cudaStream_t)s);
    if (rc) return rc;
    const LineSpec ln = line_of(p);
    CK(launch_sample_lines(n_lines, F, beta_k, dir, h->d_dir32, h->D, material_of(p), ln, w,
                           (cudaStream_t)s),
       "cvx_sample_lines");
    return CVX_OK;
}

int cvx_hull_bridge(cvx_handle *h, int64_t n_lines, int32_t L, const float *w, int32_t *m_minus,
                    int32_t *m_plus, double *hval, cvx_stream s) {
    if (L < 3 || L > 2079 || (L % 2) == 0)
        return fail(CVX_ERR_INVALID_ARG, "L must be odd in [3, 2079], got %d", L);
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n_lines < 0) return fail(CVX_ERR_INVALID_ARG, "n_lines < 0");
    if (n_lines > 0 && (!w || !m_minus || !m_plus || !hval))
        return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    CK(launch_hull(n_lines, L, w, m_minus, m_plus, hval, h->d_counters,
                   (cudaStream_t)s),
       "cvx_hull_bridge");
    return CVX_OK;
}

int convexify_points(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
                     const double *beta_k, double *W_R, double *P, cvx_laminate *root,
                     cvx_node *tree, int32_t *status, cvx_stream sv) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0 || n > ((int64_t)1 << 31) / 256)
        return fail(CVX_ERR_INVALID_ARG, "n out of range [0, 2^23]");
    if (n > 0 && (!F || !beta_k || !W_R || !P || !status))
        return fail(CVX_ERR_INVALID_ARG, "NULL array (F, beta_k, W_R, P, status are required)");
    if (n == 0) return CVX_OK;
    cudaStream_t s = (cudaStream_t)sv;
    DeviceGuard g(h->device);
    rc = ensure_dirs(h, p, s);
    if (rc) return rc;

    const LineSpec ln = line_of(p);
    const int K = p->depth;
    const int NT = (1 << (K + 1)) - 1;
    const int D = h->D;
    const int warps = h->tune_warps;
    const int bpsm = scan_max_blocks_per_sm(p->energy, warps, ln.stride);
    if (bpsm < 1) return fail(CVX_ERR_UNSUPPORTED, "scan kernel cannot launch with %d warps", warps);
    const int grid = h->sm_count * bpsm;
    // directions per work item: whole nodes when there are enough of them,
    // otherwise split the directions so every SM gets work
    int dpi = h->tune_dpi;
    if (dpi <= 0) {
        const int64_t want_items = (int64_t)grid * 4;
        if (n >= want_items) dpi = D;
        else {
            const int64_t chunks = (want_items + n - 1) / n;
            dpi = (int)std::max<int64_t>(warps * 2, (D + chunks - 1) / chunks);
        }
    }
    dpi = std::min(dpi, D);
    const int chunks = (D + dpi - 1) / dpi;

    // workspace layout (level l holds at most n 2^l nodes)
    const size_t maxq = K > 0 ? ((size_t)n << (K - 1)) : 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t o_tree = tree ? 0 : take(sizeof(cvx_node) * (size_t)n * NT);
    std::vector<size_t> o_qp(K + 1), o_qh(K + 1);
    for (int l = 0; l < K; ++l) {
        o_qp[l] = take(sizeof(int32_t) * ((size_t)n << l));
        o_qh[l] = take(sizeof(int32_t) * ((size_t)n << l));
    }
    const size_t o_cnt = take(sizeof(int32_t) * 2 * (K + 1));
    const size_t o_items = take(sizeof(ItemCands) * maxq * chunks);
    const size_t o_cands = take(sizeof(NodeCands) * maxq);
    const size_t o_work = take(sizeof(int2) * maxq * kNodeCand);
    const size_t o_ref = take(sizeof(RefineOut) * maxq * kNodeCand);
    rc = ensure_ws(h, off, s);
    if (rc) return rc;
    char *ws = h->ws;
    cvx_node *tr = tree ? tree : (cvx_node *)(ws + o_tree);
    int32_t *cnt = (int32_t *)(ws + o_cnt);      // node counts per level
    int32_t *wcnt = cnt + (K + 1);               // refine work counts per level

    CK(cudaMemsetAsync(tr, 0, sizeof(cvx_node) * (size_t)n * NT, s), "convexify_points");
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 2 * (K + 1), s), "convexify_points");

    const Material mat = material_of(p);
    InitArgs ia;
    ia.n = n;
    ia.F = F;
    ia.beta = beta_k;
    ia.tree = tr;
    ia.NT = NT;
    ia.depth = K;
    ia.q_point = K ? (int32_t *)(ws + o_qp[0]) : nullptr;
    ia.q_heap = K ? (int32_t *)(ws + o_qh[0]) : nullptr;
    ia.q_count = cnt;
    ia.status = status;
    ia.mat = mat;
    ia.m0 = ln.m0;
    ia.counters = h->d_counters;
    CK(launch_init(ia, s), "convexify_points/init");

    ItemCands *items = (ItemCands *)(ws + o_items);
    NodeCands *cands = (NodeCands *)(ws + o_cands);
    int2 *work = (int2 *)(ws + o_work);
    RefineOut *refined = (RefineOut *)(ws + o_ref);
    for (int l = 0; l < K; ++l) {
        const int64_t max_nodes = (int64_t)n << l;
        int32_t *qp = (int32_t *)(ws + o_qp[l]), *qh = (int32_t *)(ws + o_qh[l]);
        ScanArgs sa;
        sa.tree = tr;
        sa.NT = NT;
        sa.beta = beta_k;
        sa.q_point = qp;
        sa.q_heap = qh;
        sa.q_count = cnt + l;
        sa.dir32 = h->d_dir32;
        sa.D = D;
        sa.chunks = chunks;
        sa.dirs_per_item = dpi;
        sa.mat = mat;
        sa.line = ln;
        sa.out = items;
        sa.counters = h->d_counters;
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if (h->profiling) {
            if (!h->ev_pool.empty()) {
                ev = h->ev_pool.back();
                h->ev_pool.pop_back();
            } else {
                CK(cudaEventCreate(&ev.first), "profiling");
                CK(cudaEventCreate(&ev.second), "profiling");
            }
            CK(cudaEventRecord(ev.first, s), "profiling");
        }
        CK(launch_scan(sa, warps, grid, s), "convexify_points/scan");
        if (h->profiling) {
            CK(cudaEventRecord(ev.second, s), "profiling");
            h->ev_pending.push_back(ev);
        }

        SelectArgs se;
        se.q_count = cnt + l;
        se.items = items;
        se.chunks = chunks;
        se.kappa = (float)line_kappa(mat);
        se.cands = cands;
        se.work = work;
        se.work_count = wcnt + l;
        se.counters = h->d_counters;
        CK(launch_select(se, max_nodes, s), "convexify_points/select");

        RefineArgs ra;
        ra.tree = tr;
        ra.NT = NT;
        ra.beta = beta_k;
        ra.q_point = qp;
        ra.q_heap = qh;
        ra.cands = cands;
        ra.work = work;
        ra.work_count = wcnt + l;
        ra.dir64 = h->d_dir64;
        ra.mat = mat;
        ra.line = ln;
        ra.out = refined;
        CK(launch_refine(ra, max_nodes * kNodeCand, s), "convexify_points/refine");

        CommitArgs ca;
        ca.tree = tr;
        ca.NT = NT;
        ca.level = l;
        ca.depth = K;
        ca.beta = beta_k;
        ca.q_point = qp;
        ca.q_heap = qh;
        ca.q_count = cnt + l;
        ca.nq_point = l + 1 < K ? (int32_t *)(ws + o_qp[l + 1]) : nullptr;
        ca.nq_heap = l + 1 < K ? (int32_t *)(ws + o_qh[l + 1]) : nullptr;
        ca.nq_count = cnt + l + 1;
        ca.cands = cands;
        ca.refined = refined;
        ca.dir64 = h->d_dir64;
        ca.kappa = line_kappa(mat);
        ca.mat = mat;
        ca.line = ln;
        ca.counters = h->d_counters;
        CK(launch_commit(ca, max_nodes, s), "convexify_points/commit");
    }

    LeafArgs la;
    la.n = n;
    la.tree = tr;
    la.NT = NT;
    la.beta = beta_k;
    la.W_R = W_R;
    la.P = P;
    la.status = status;
    la.root = root;
    la.mat = mat;
    CK(launch_leaf(la, s), "convexify_points/leaf");
    return CVX_OK;
}

}  // extern "C"
