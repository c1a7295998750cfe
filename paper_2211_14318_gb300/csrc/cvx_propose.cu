// cvx_propose.cu -- the surrogate-proposed form of the per-point
// convexification, and training labels from lamination trees.
//
// Per tree level: the network reads every queued node (k_feat -> tensor-core
// forward -> k_decode), which gives a window centre on the angle grid and the
// energy E_pred of the proposed laminate; the line scan then covers only the
// (2w + 1)^2 directions of the window (PASS_WINDOW), and k_commit defers to
// the full scan (PASS_FALLBACK) every node whose window decision fails the
// fallback test: best direction on the window border after the re-centrings,
// or |E_pred - V| / (1e-8 + |V|) > gap_tol.  With CVX_FLAG_MIRROR_WINDOW a
// node whose window split is scanned again around the mirror cell of its
// direction (the twin basin of an isotropic W) and takes the lower value.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "cvx_handle.h"
#include "cvx_surrogate.h"

namespace cvx {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kChunk = 1 << 16;  // nodes per network launch sequence

// Standardised network inputs of queued nodes off .. off + chunk - 1.
__global__ void k_feat(const Pipe P, int level, int off, int chunk, const float *scale,
                       __nv_bfloat16 *X) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= chunk) return;
    const int qi = off + r;
    if (qi >= P.cnt[level]) return;
    const int p = P.qp[level][qi], hi = P.qh[level][qi];
    const ProbDesc &pd = P.probs[P.pid[p]];
    const cvx_node *nd = node_ptr(pd, p, hi);
    const double J = nd->F[0] * nd->F[3] - nd->F[1] * nd->F[2];
    const float x[6] = {(float)nd->F[0], (float)nd->F[1], (float)nd->F[2], (float)nd->F[3],
                        (float)pd.beta[p - pd.point_off], (float)log(J)};
    for (int k = 0; k < 16; ++k)
        X[(long long)r * 16 + k] =
            __float2bfloat16_rn(k < 6 ? (x[k] - scale[k]) * scale[6 + k] : 0.0f);
}

// Window centre (nearest grid cell of the wrapped angles) and E_pred =
// xi W(F+) + (1 - xi) W(F-) of the proposed laminate: R = a (x) b of the
// unrounded angles, amp = jump : R, F+ = F + (1 - xi) amp R, F- = F - xi amp R.
__global__ void k_decode(const Pipe P, int level, int off, int chunk, const float *out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= chunk) return;
    const int qi = off + r;
    if (qi >= P.cnt[level]) return;
    const int p = P.qp[level][qi], hi = P.qh[level][qi];
    const ProbDesc &pd = P.probs[P.pid[p]];
    const cvx_node *nd = node_ptr(pd, p, hi);
    const float *o = out + (long long)r * 7;
    double ta = fmod((double)o[0], kPi), tb = fmod((double)o[1], kPi);
    if (ta < 0.0) ta += kPi;
    if (tb < 0.0) tb += kPi;
    int ia = (int)floor(ta * pd.Na / kPi + 0.5) % pd.Na;
    int ib = (int)floor(tb * pd.Nb / kPi + 0.5) % pd.Nb;
    P.center[qi] = make_int2(ia, ib);
    const double a0 = cos(ta), a1 = sin(ta), b0 = cos(tb), b1 = sin(tb);
    const double R[4] = {a0 * b0, a0 * b1, a1 * b0, a1 * b1};
    const double xi = 1.0 / (1.0 + exp(-(double)o[2]));
    double amp = 0.0;
    for (int k = 0; k < 4; ++k) amp += (double)o[3 + k] * R[k];
    double Fp[4], Fm[4];
    for (int k = 0; k < 4; ++k) {
        Fp[k] = nd->F[k] + (1.0 - xi) * amp * R[k];
        Fm[k] = nd->F[k] - xi * amp * R[k];
    }
    const double beta = pd.beta[p - pd.point_off];
    P.e_pred[qi] = xi * energy64(Fp, beta, pd.mat) + (1.0 - xi) * energy64(Fm, beta, pd.mat);
}

__global__ void k_fell_back(long long n, const int32_t *status, uint8_t *fb) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) fb[i] = (status[i] & CVX_PT_FALLBACK) ? 1 : 0;
}

// Labels: scanned nodes per point, then one sample per scanned node.
__global__ void k_label_count(long long n, int NT, const cvx_node *tree, int32_t *cnt) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c = 0;
    for (int i = 0; i < NT; ++i) c += (tree[p * NT + i].flags & CVX_NODE_SCANNED) ? 1 : 0;
    cnt[p] = c;
}

__global__ void k_label_write(long long n, int NT, int Na, int Nb, const cvx_node *tree,
                              const double *beta, const long long *off, float *X, float *Y) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    long long o = off[p];
    for (int i = 0; i < NT; ++i) {
        const cvx_node &nd = tree[p * NT + i];
        if (!(nd.flags & CVX_NODE_SCANNED)) continue;
        const double J = nd.F[0] * nd.F[3] - nd.F[1] * nd.F[2];
        float *x = X + o * 6, *y = Y + o * 7;
        for (int k = 0; k < 4; ++k) x[k] = (float)nd.F[k];
        x[4] = (float)beta[p];
        x[5] = (float)log(J);
        if (nd.flags & CVX_NODE_LAMINATED) {
            const cvx_node &cm = tree[p * NT + 2 * i + 1], &cp = tree[p * NT + 2 * i + 2];
            y[0] = (float)(kPi * (nd.dir / Nb) / Na);
            y[1] = (float)(kPi * (nd.dir % Nb) / Nb);
            y[2] = (float)nd.xi;
            for (int k = 0; k < 4; ++k) y[3 + k] = (float)(cp.F[k] - cm.F[k]);
        } else {
            y[0] = y[1] = y[2] = nanf("");
            for (int k = 0; k < 4; ++k) y[3 + k] = 0.0f;
        }
        ++o;
    }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace cvx

using namespace cvx;

extern "C" {

int surrogate_labels(cvx_handle *h, const cvx_params *p, int64_t n, const double *beta_k,
                     const cvx_node *tree, float *X, float *Y, int64_t *count, cvx_stream sv) {
    int rc = check_params(p, false);
    if (rc) return rc;
    if (!h || !count) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    if (p->dirs) return fail(CVX_ERR_INVALID_ARG, "labels need the angle grid (dirs == NULL)");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    *count = 0;
    if (n == 0) return CVX_OK;
    if (!beta_k || !tree || !X || !Y) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    const int NT = (1 << (p->depth + 1)) - 1;
    int32_t *cnt = nullptr;
    long long *off = nullptr;
    CK(cudaMalloc(&cnt, sizeof(int32_t) * n), "surrogate_labels");
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_label_count<<<nb, 256, 0, s>>>(n, NT, tree, cnt);
    std::vector<int32_t> c((size_t)n);
    std::vector<long long> o((size_t)n);
    cudaError_t e = cudaMemcpyAsync(c.data(), cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate_labels");
    long long t = 0;
    for (int64_t i = 0; i < n; ++i) {
        o[(size_t)i] = t;
        t += c[(size_t)i];
    }
    CK(cudaMalloc(&off, sizeof(long long) * n), "surrogate_labels");
    e = cudaMemcpyAsync(off, o.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_label_write<<<nb, 256, 0, s>>>(n, NT, p->n_theta_a, p->n_theta_b, tree, beta_k, off, X, Y);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(off);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate_labels");
    *count = t;
    return CVX_OK;
}

int surrogate_propose(cvx_handle *h, const cvx_params *p, int64_t n, const double *F,
                      const double *beta_k, int window, double gap_tol, double *W_R, double *P,
                      cvx_laminate *root, cvx_node *tree, uint8_t *fell_back, int32_t *status,
                      cvx_stream sv) {
    int rc = check_params(p, true);
    if (rc) return rc;
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (p->dirs) return fail(CVX_ERR_INVALID_ARG, "the proposal window needs the angle grid");
    if (CVX_WINDOW_DOUBLINGS_OF(p->flags))
        return fail(CVX_ERR_UNSUPPORTED, "surrogate_propose: adaptive line windows are not supported");
    if (window < 0 || 2 * window + 1 > std::min(p->n_theta_a, p->n_theta_b))
        return fail(CVX_ERR_INVALID_ARG, "window must satisfy 0 <= 2 w + 1 <= min(Na, Nb)");
    if (!(gap_tol >= 0.0)) return fail(CVX_ERR_INVALID_ARG, "gap_tol must be >= 0");
    if (n < 0 || n > ((int64_t)1 << 31) / 256)
        return fail(CVX_ERR_INVALID_ARG, "n out of range [0, 2^23]");
    if (n > 0 && (!F || !beta_k || !W_R || !P || !status))
        return fail(CVX_ERR_INVALID_ARG, "NULL array (F, beta_k, W_R, P, status are required)");
    if (!h->sur || !h->sur->has_weights) return fail(CVX_ERR_NOT_TRAINED, "no surrogate weights");
    if (n == 0) return CVX_OK;
    cudaStream_t s = (cudaStream_t)sv;
    DeviceGuard g(h->device);
    rc = ensure_dirs(h, p, s);
    if (rc) return rc;

    const int warps = h->tune_warps;
    ProbDesc pd = {};
    pd.line = make_line(p->line_points, p->t_half);
    const int bpsm = scan_max_blocks_per_sm(p->energy, warps, pd.line.stride);
    if (bpsm < 1) return fail(CVX_ERR_UNSUPPORTED, "scan kernel cannot launch with %d warps", warps);
    const int grid = h->sm_count * bpsm;
    pd.mat = material_of(p);
    pd.kappa = line_kappa(pd.mat);
    pd.kappa_f = (float)pd.kappa;
    pd.D = h->D;
    pd.dir_off = 0;
    pd.flags = p->flags;
    pd.K = p->depth;
    pd.NT = (1 << (p->depth + 1)) - 1;
    const bool lanes = lane_scan_enabled(p->energy);
    const long long lane_warps = (long long)h->sm_count * lane_scan_blocks_per_sm() * 8;
    pd.dpi = lanes ? lane_dirs_per_item(n, pd.D, lane_warps, 0)
                   : dirs_per_item(n, pd.D, grid, warps, 0);
    pd.chunks = (pd.D + pd.dpi - 1) / pd.dpi;
    pd.window = window;
    pd.Na = p->n_theta_a;
    pd.Nb = p->n_theta_b;
    pd.wD = (2 * window + 1) * (2 * window + 1);
    pd.wdpi = lanes ? lane_dirs_per_item(n, pd.wD, lane_warps, 0)
                    : dirs_per_item(n, pd.wD, grid, warps, 0);
    pd.wchunks = (pd.wD + pd.wdpi - 1) / pd.wdpi;
    const bool mirror = (p->flags & CVX_FLAG_MIRROR_WINDOW) != 0;
    pd.mwindow = mirror ? (window + 1) / 2 : 0;
    pd.gap_tol = gap_tol;
    pd.point_off = 0;
    pd.n = n;
    pd.F = F;
    pd.beta = beta_k;
    pd.W_R = W_R;
    pd.P = P;
    pd.status = status;
    pd.root = root;

    // the mirror window's geometry (the mirror stage's problem table is pd
    // with these, built once pd is complete)
    const int mwD = (2 * pd.mwindow + 1) * (2 * pd.mwindow + 1);
    const int mwdpi = lanes ? lane_dirs_per_item(n, mwD, lane_warps, 0)
                            : dirs_per_item(n, mwD, grid, warps, 0);
    const int mwchunks = (mwD + mwdpi - 1) / mwdpi;

    Pipe pp = {};
    pp.n_probs = 1;
    pp.N = n;
    pp.K = p->depth;
    pp.C = std::max(std::max(pd.chunks, pd.wchunks), mirror ? mwchunks : 0);
    pp.mirror_on = mirror ? 1 : 0;
    pp.stride32 = pp.stride64 = pd.line.stride;
    pp.energy = p->energy;
    pp.window = 1;
    pp.lanes = lanes ? 1 : 0;
    const size_t pipe_sz = up256(pipe_bytes(pp.N, pp.K, pp.C, 1, true, false, mirror));
    const size_t tree_sz = tree ? 0 : sizeof(cvx_node) * (size_t)n * pd.NT;
    rc = ensure_ws(h, pipe_sz + tree_sz, s);
    if (rc) return rc;
    pipe_layout(pp, h->ws);
    pd.tree = tree ? tree : (cvx_node *)(h->ws + pipe_sz);
    pp.dir32 = h->d_dir32;
    pp.dir64 = h->d_dir64;
    pp.counters = h->d_counters;
    const long long maxq = pp.K > 0 ? (n << (pp.K - 1)) : 0;
    const int chunk = (int)std::min<long long>(kChunk, std::max<long long>(maxq, 1));
    rc = sur_batch(h, chunk);
    if (rc) return rc;
    Surrogate &S = *h->sur;
    // pageable source: returns once staged
    CK(cudaMemcpyAsync((void *)pp.probs, &pd, sizeof pd, cudaMemcpyHostToDevice, s),
       "surrogate_propose/table");
    ProbDesc pm = pd;
    pm.window = pd.mwindow;
    pm.wD = mwD;
    pm.wdpi = mwdpi;
    pm.wchunks = mwchunks;
    if (mirror)
        CK(cudaMemcpyAsync((void *)pp.mprobs, &pm, sizeof pm, cudaMemcpyHostToDevice, s),
           "surrogate_propose/table");
    const int R = p->recentre;
    std::vector<cudaEvent_t> ev;  // window passes, mirror passes and fallback scan of every level
    const int per_level = (R + 1) * (mirror ? 2 : 1) + 1;
    rc = scan_events(h, per_level * pp.K, ev);
    if (rc) return rc;
    CK(pipe_begin(pp, s), "surrogate_propose");
    for (int l = 0; l < pp.K; ++l) {
        const long long max_nodes = n << l;
        for (long long off = 0; off < max_nodes; off += chunk) {
            const int m = (int)std::min<long long>(chunk, max_nodes - off);
            k_feat<<<(m + 255) / 256, 256, 0, s>>>(pp, l, (int)off, m, S.scale, S.X);
            CK(cudaGetLastError(), "surrogate_propose/features");
            rc = sur_forward(h, m, false, s, pp.cnt + l, (int)off);
            if (rc) return rc;
            k_decode<<<(m + 255) / 256, 256, 0, s>>>(pp, l, (int)off, m, S.out);
            CK(cudaGetLastError(), "surrogate_propose/decode");
        }
        cudaEvent_t *evl = ev.empty() ? nullptr : &ev[2 * per_level * l];
        int e = 0;
        for (int r = 0; r <= R; ++r, ++e)
            CK(pipe_level(window_pipe(pp, l, r, R), l, warps, grid, s, evl ? evl + 2 * e : nullptr),
               "surrogate_propose/window");
        if (mirror)
            for (int r = 0; r <= R; ++r, ++e)
                CK(pipe_level(mirror_pipe(pp, l, r, R), l, warps, grid, s,
                              evl ? evl + 2 * e : nullptr),
                   "surrogate_propose/mirror");
        CK(pipe_level(fallback_pipe(pp, l), l, warps, grid, s, evl ? evl + 2 * e : nullptr),
           "surrogate_propose/fallback");
    }
    CK(pipe_end(pp, s), "surrogate_propose");
    if (fell_back) {
        k_fell_back<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, status, fell_back);
        CK(cudaGetLastError(), "surrogate_propose");
    }
    return CVX_OK;
}

}  // extern "C"
