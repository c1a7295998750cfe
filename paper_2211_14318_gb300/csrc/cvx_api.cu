// cvx_api.cu -- host side of the C ABI declared in include/convexify.h:
// argument validation, the handle (workspace, direction tables, counters),
// the single steps and convexify_points (a pipeline run over one problem).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "cvx_handle.h"

using namespace cvx;

namespace {
thread_local std::string g_err;
}  // namespace

namespace cvx {

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

// Records the calling thread's last error for entry points in other files.
int set_error_message(int code, const char *msg) { return fail(code, "%s", msg); }

Material material_of(const cvx_params *p) {
    Material m;
    m.mu = p->mu;
    m.lam = p->lambda_L;
    m.Dinf = p->D_inf;
    m.D0 = p->D0;
    m.energy = p->energy;
    return m;
}

int check_params(const cvx_params *p, bool need_line, bool allow_stvk) {
    if (!p) return fail(CVX_ERR_INVALID_ARG, "params is NULL");
    if (p->energy == CVX_ENERGY_STVK_DAMAGE && !allow_stvk)
        return fail(CVX_ERR_UNSUPPORTED,
                    "the St. Venant-Kirchhoff energy is built for the global-grid calls only");
    if (p->energy != CVX_ENERGY_NH_DAMAGE && p->energy != CVX_ENERGY_DOUBLE_WELL &&
        p->energy != CVX_ENERGY_STVK_DAMAGE)
        return fail(CVX_ERR_INVALID_ARG, "unknown energy kind %d", p->energy);
    if (p->energy != CVX_ENERGY_DOUBLE_WELL) {
        if (!(p->mu > 0.0) || !(p->lambda_L >= 0.0) || !(p->D_inf >= 0.0 && p->D_inf < 1.0) ||
            !(p->D0 > 0.0))
            return fail(CVX_ERR_INVALID_ARG,
                        "material out of range (mu > 0, lambda >= 0, 0 <= D_inf < 1, D0 > 0)");
    }
    if (p->flags & ~(CVX_FLAG_REFINE_NEWTON | CVX_FLAG_GAP_ONE_SIDED | CVX_FLAG_MIRROR_WINDOW |
                     CVX_FLAG_WINDOW_DOUBLINGS(15)))
        return fail(CVX_ERR_INVALID_ARG, "unknown flags");
    if (CVX_WINDOW_DOUBLINGS_OF(p->flags) > kMaxRecentre)
        return fail(CVX_ERR_INVALID_ARG, "window doublings must be in [0, 8]");
    if (p->recentre < 0 || p->recentre > kMaxRecentre)
        return fail(CVX_ERR_INVALID_ARG, "recentre must be in [0, 8], got %d", p->recentre);
    if (!need_line) return CVX_OK;
    if (p->line_points < 3 || p->line_points > 2079 || (p->line_points % 2) == 0)
        return fail(CVX_ERR_INVALID_ARG, "line_points must be odd in [3, 2079], got %d",
                    p->line_points);
    if (!(p->t_half > 0.0) || !isfinite(p->t_half))
        return fail(CVX_ERR_INVALID_ARG, "t_half must be positive");
    if (p->depth < 0 || p->depth > kMaxDepth)
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

// Direction table: a_i = (cos pi i/Na, sin pi i/Na), b_j likewise, j_dir = i Nb + j,
// or a copy of the caller's rows.
void direction_rows(const cvx_params *p, std::vector<double> &d64) {
    const int D = p->dirs ? p->n_dirs : p->n_theta_a * p->n_theta_b;
    d64.resize((size_t)D * 4);
    if (p->dirs) {
        memcpy(d64.data(), p->dirs, sizeof(double) * 4 * (size_t)D);
        return;
    }
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

int scan_events(cvx_handle *h, int n_launches, std::vector<cudaEvent_t> &ev) {
    ev.clear();
    if (!h->profiling) return CVX_OK;
    for (int l = 0; l < n_launches; ++l) {
        std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
        if (!h->ev_pool.empty()) {
            e = h->ev_pool.back();
            h->ev_pool.pop_back();
        } else {
            CK(cudaEventCreate(&e.first), "profiling");
            CK(cudaEventCreate(&e.second), "profiling");
        }
        ev.push_back(e.first);
        ev.push_back(e.second);
        h->ev_pending.push_back(e);
    }
    return CVX_OK;
}

int ensure_ws(cvx_handle *h, size_t bytes, cudaStream_t s) {
    if (bytes <= h->ws_cap) return CVX_OK;
    CK(cudaStreamSynchronize(s), "workspace");
    CK(cudaDeviceSynchronize(), "workspace");
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_cap = 0;
    ++h->ws_gen;
    const size_t cap = std::max(bytes + bytes / 8, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&h->ws, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CVX_ERR_OOM, "workspace of %zu bytes: %s", cap, cudaGetErrorString(e));
    }
    h->ws_cap = cap;
    return CVX_OK;
}

}  // namespace cvx

namespace cvx {

int ensure_dirs(cvx_handle *h, const cvx_params *p, cudaStream_t s) {
    if (!p->dirs && !h->dir_custom && h->dir_na == p->n_theta_a && h->dir_nb == p->n_theta_b)
        return CVX_OK;
    std::vector<double> d64;
    direction_rows(p, d64);
    const int D = (int)(d64.size() / 4);
    std::vector<float4> d32(D);
    for (int k = 0; k < D; ++k)
        d32[k] = make_float4((float)d64[4 * k], (float)d64[4 * k + 1], (float)d64[4 * k + 2],
                             (float)d64[4 * k + 3]);
    CK(cudaStreamSynchronize(s), "direction table");
    if ((size_t)D > h->dir_cap) {
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

}  // namespace cvx

namespace {

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

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
    destroy_batch_plan(h);
    destroy_surrogate(h);
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
    out->window_nodes = (int64_t)c[C_WNODES];
    out->fallbacks = (int64_t)c[C_FALLBACK];
    out->refine_full = (int64_t)c[C_REFFULL];
    out->lines_bounded = (int64_t)c[C_BOUNDED];
    out->lines_flat = (int64_t)c[C_FLAT];
    out->recentred = (int64_t)c[C_RECENTRED];
    out->lines_certified = (int64_t)c[C_CERT];
    out->edge_splits = (int64_t)c[C_EDGE];
    out->window_doublings = (int64_t)c[C_DOUBLED];
    out->mirror_windows = (int64_t)c[C_MIRROR];
    out->mirror_won = (int64_t)c[C_MIRROR_WON];
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
    case 4: return (int)sizeof(cvx_problem);
    case 5: return (int)sizeof(cvx_grid);
    default: return -1;
    }
}

int cvx_set_tuning(cvx_handle *h, int warps_per_cta, int dirs_per_item) {
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (warps_per_cta < 1 || warps_per_cta > 8)
        return fail(CVX_ERR_INVALID_ARG, "warps_per_cta must be in [1, 8]");
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
    const LineSpec ln = make_line(p->line_points, p->t_half);
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
    CK(launch_hull(n_lines, L, w, m_minus, m_plus, hval, h->d_counters, (cudaStream_t)s),
       "cvx_hull_bridge");
    return CVX_OK;
}

int cvx_tree_tangent(cvx_handle *h, const cvx_params *p, int64_t n, const double *beta_k,
                     const cvx_node *tree, double *A, cvx_stream s) {
    int rc = check_params(p, false);
    if (rc) return rc;
    if (p->depth < 0 || p->depth > kMaxDepth)
        return fail(CVX_ERR_INVALID_ARG, "depth must be in [0, 8], got %d", p->depth);
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!beta_k || !tree || !A)) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    CK(launch_tree_tangent(n, (1 << (p->depth + 1)) - 1, tree, beta_k, material_of(p), A,
                           (cudaStream_t)s),
       "cvx_tree_tangent");
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

    const Material mat = material_of(p);
    const int warps = h->tune_warps;
    ProbDesc pd = {};
    pd.line = make_line(p->line_points, p->t_half);
    const int bpsm = scan_max_blocks_per_sm(p->energy, warps, pd.line.stride);
    if (bpsm < 1) return fail(CVX_ERR_UNSUPPORTED, "scan kernel cannot launch with %d warps", warps);
    const int grid = h->sm_count * bpsm;
    pd.mat = mat;
    pd.kappa = line_kappa(mat);
    pd.kappa_f = (float)pd.kappa;
    pd.D = h->D;
    pd.dir_off = 0;
    pd.flags = p->flags;
    pd.K = p->depth;
    pd.NT = (1 << (p->depth + 1)) - 1;
    const bool lanes = lane_scan_enabled(p->energy);
    if (lanes)
        pd.dpi = lane_dirs_per_item(n, pd.D, (long long)h->sm_count * lane_scan_blocks_per_sm() * 8,
                                    h->tune_dpi);
    else
        pd.dpi = h->tune_dpi > 0 ? std::min(h->tune_dpi, pd.D)
                                 : dirs_per_item(n, pd.D, grid, warps, 0);
    pd.chunks = (pd.D + pd.dpi - 1) / pd.dpi;
    pd.point_off = 0;
    pd.n = n;
    pd.F = F;
    pd.beta = beta_k;
    pd.W_R = W_R;
    pd.P = P;
    pd.status = status;
    pd.root = root;

    Pipe pp = {};
    pp.n_probs = 1;
    pp.N = n;
    pp.K = p->depth;
    pp.C = pd.chunks;
    pp.stride32 = pp.stride64 = pd.line.stride;
    pp.energy = p->energy;
    pp.lanes = lanes ? 1 : 0;
    pp.adaptive = CVX_WINDOW_DOUBLINGS_OF(p->flags);
    const size_t pipe_sz = align_up(pipe_bytes(pp.N, pp.K, pp.C, 1, false, pp.adaptive > 0));
    const size_t tree_sz = tree ? 0 : sizeof(cvx_node) * (size_t)n * pd.NT;
    rc = ensure_ws(h, pipe_sz + tree_sz, s);
    if (rc) return rc;
    pipe_layout(pp, h->ws);
    pd.tree = tree ? tree : (cvx_node *)(h->ws + pipe_sz);
    pp.dir32 = h->d_dir32;
    pp.dir64 = h->d_dir64;
    pp.counters = h->d_counters;
    // pageable source: returns once staged, so the stack copy may go away
    CK(cudaMemcpyAsync((void *)pp.probs, &pd, sizeof pd, cudaMemcpyHostToDevice, s),
       "convexify_points/table");

    std::vector<cudaEvent_t> ev;
    rc = scan_events(h, pp.K * (pp.adaptive + 1), ev);
    if (rc) return rc;
    CK(pipe_enqueue(pp, warps, grid, s, ev.empty() ? nullptr : ev.data()), "convexify_points");
    return CVX_OK;
}

}  // extern "C"
