// cvx_noalloc.cu -- convexify_points_static: the same per-point
// convexification as convexify_points, for callers that are not allowed to
// allocate device memory.
//
// Typical callers: a material routine plugged into a host finite-element code
// that owns all device memory through its own pool and forbids the plugin to
// call cudaMalloc, or a latency-critical caller for which cudaMalloc's implicit
// device synchronisation is not acceptable.  They pass inputs and outputs; all
// scratch (direction tables, tree, node queues, candidate records, counters)
// lives in one file-scope device array of fixed size.  Nothing here calls
// cudaMalloc, cudaFree or any other allocating routine.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "convexify.h"
#include "cvx_internal.h"

namespace cvx {
int set_error_message(int code, const char *msg);  // cvx_api.cu
int check_params(const cvx_params *p, bool need_line, bool allow_stvk = false);  // cvx_api.cu
}

using namespace cvx;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kStaticMaxDirs = 16384;
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a stand-in: its device address
// is obtained with cudaGetSymbolAddress once per device (see setup()).
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices];
int g_sms[kMaxDevices];
// host staging of the direction tables (static: no host heap either)
float4 g_dir32[kStaticMaxDirs];
double g_dir64[4 * kStaticMaxDirs];
ProbDesc g_desc;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int err(int code, const char *msg) { return set_error_message(code, msg); }

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
int setup(int dev, void **addr, int *sms) {
    if (dev < 0 || dev >= kMaxDevices) return err(CVX_ERR_UNSUPPORTED, "device index too large");
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(CVX_ERR_CUDA, "convexify_points_static: cudaGetSymbolAddress failed");
        }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return err(CVX_ERR_CUDA, "convexify_points_static: device query failed");
        g_addr[dev] = p;
        g_sms[dev] = n;
    }
    *addr = g_addr[dev];
    *sms = g_sms[dev];
    return CVX_OK;
}

}  // namespace

extern "C" int convexify_points_static(const cvx_params *p, int64_t n, const double *F,
                                       const double *beta_k, double *W_R, double *P,
                                       int32_t *status, cvx_stream sv) {
    // the same parameter checks as convexify_points (material, flags, line,
    // depth, direction count in [1, 2^20] computed in 64 bits), then the
    // static limit
    int rc = check_params(p, true);
    if (rc) return rc;
    if (CVX_WINDOW_DOUBLINGS_OF(p->flags))
        return err(CVX_ERR_UNSUPPORTED,
                   "convexify_points_static: adaptive line windows are not supported");
    const int64_t D64 = p->dirs ? (int64_t)p->n_dirs : (int64_t)p->n_theta_a * p->n_theta_b;
    if (D64 < 1 || D64 > kStaticMaxDirs)
        return err(CVX_ERR_INVALID_ARG,
                   "convexify_points_static: more than 16384 directions (use convexify_points)");
    const int D = (int)D64;
    if (n < 0) return err(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!F || !beta_k || !W_R || !P || !status))
        return err(CVX_ERR_INVALID_ARG, "NULL array (F, beta_k, W_R, P, status are required)");
    if (n == 0) return CVX_OK;

    const LineSpec ln = make_line(p->line_points, p->t_half);
    const int K = p->depth;
    const int NT = (1 << (K + 1)) - 1;
    const int warps = 8;
    Material mat;
    mat.mu = p->mu;
    mat.lam = p->lambda_L;
    mat.Dinf = p->D_inf;
    mat.D0 = p->D0;
    mat.energy = p->energy;

    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(CVX_ERR_CUDA, "no current device");
    void *base = nullptr;
    int sms = 0;
    rc = setup(dev, &base, &sms);
    if (rc) return rc;
    const int bpsm = scan_max_blocks_per_sm(p->energy, warps, ln.stride);
    if (bpsm < 1) return err(CVX_ERR_UNSUPPORTED, "scan kernel cannot launch");
    const int grid = sms * bpsm;
    const bool lanes = lane_scan_enabled(p->energy);
    int dpi = D;
    if (lanes) {
        dpi = lane_dirs_per_item(n, D, (long long)sms * lane_scan_blocks_per_sm() * 8, 0);
    } else {
        const int64_t want_items = (int64_t)grid * 4;
        if (n < want_items) {
            const int64_t chunks = (want_items + n - 1) / n;
            const int64_t d = (D + chunks - 1) / chunks;
            dpi = (int)(d > warps * 2 ? d : warps * 2);
        }
        if (dpi > D) dpi = D;
    }
    const int chunks = (D + dpi - 1) / dpi;

    // scratch layout: counters, direction tables, tree, then the pipeline's
    // own buffers (problem table first)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + bytes);
        return o;
    };
    const size_t o_ctr = take(sizeof(unsigned long long) * C_NUM);
    const size_t o_d32 = take(sizeof(float4) * D);
    const size_t o_d64 = take(sizeof(double) * 4 * D);
    const size_t o_tree = take(sizeof(cvx_node) * (size_t)n * NT);
    const size_t o_pipe = take(pipe_bytes(n, K, chunks, 1));
    if (off > kStaticScratchBytes)
        return err(CVX_ERR_INVALID_ARG,
                   "convexify_points_static: problem needs more than the 64 MiB static scratch "
                   "(fewer points per call, or convexify_points)");
    char *ws = (char *)base;
    cudaStream_t s = (cudaStream_t)sv;

    // direction tables (staged in static host arrays, copied while the lock is held)
    if (p->dirs) {
        memcpy(g_dir64, p->dirs, sizeof(double) * 4 * (size_t)D);
    } else {
        for (int i = 0; i < p->n_theta_a; ++i) {
            const double ta = M_PI * (double)i / (double)p->n_theta_a;
            for (int j = 0; j < p->n_theta_b; ++j) {
                const double tb = M_PI * (double)j / (double)p->n_theta_b;
                double *r = g_dir64 + 4 * ((size_t)i * p->n_theta_b + j);
                r[0] = cos(ta);
                r[1] = sin(ta);
                r[2] = cos(tb);
                r[3] = sin(tb);
            }
        }
    }
    for (int k = 0; k < D; ++k)
        g_dir32[k] = make_float4((float)g_dir64[4 * k], (float)g_dir64[4 * k + 1],
                                 (float)g_dir64[4 * k + 2], (float)g_dir64[4 * k + 3]);

    ProbDesc &pd = g_desc;
    pd = ProbDesc{};
    pd.line = ln;
    pd.mat = mat;
    pd.kappa = line_kappa(mat);
    pd.kappa_f = (float)pd.kappa;
    pd.D = D;
    pd.dir_off = 0;
    pd.flags = p->flags;
    pd.K = K;
    pd.NT = NT;
    pd.chunks = chunks;
    pd.dpi = dpi;
    pd.point_off = 0;
    pd.n = n;
    pd.F = F;
    pd.beta = beta_k;
    pd.W_R = W_R;
    pd.P = P;
    pd.status = status;
    pd.root = nullptr;
    pd.tree = (cvx_node *)(ws + o_tree);

    Pipe pp = {};
    pp.n_probs = 1;
    pp.N = n;
    pp.K = K;
    pp.C = chunks;
    pp.stride32 = pp.stride64 = ln.stride;
    pp.energy = p->energy;
    pp.lanes = lanes ? 1 : 0;
    pipe_layout(pp, ws + o_pipe);
    pp.dir32 = (const float4 *)(ws + o_d32);
    pp.dir64 = (const double *)(ws + o_d64);
    pp.counters = (unsigned long long *)(ws + o_ctr);

    // pageable sources: cudaMemcpyAsync returns once the data is staged
    if (cudaMemcpyAsync(ws + o_d32, g_dir32, sizeof(float4) * D, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(ws + o_d64, g_dir64, sizeof(double) * 4 * D, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync((void *)pp.probs, &pd, sizeof pd, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return err(CVX_ERR_CUDA, "convexify_points_static: table copy failed");

    // What must start at zero: the counters here; the queue counts and work
    // counters are cleared, and every tree node written, by the pipeline itself.
    if (cudaMemsetAsync(pp.counters, 0, sizeof(unsigned long long) * C_NUM, s) != cudaSuccess)
        return err(CVX_ERR_CUDA, "convexify_points_static: scratch clear failed");
    if (pipe_enqueue(pp, warps, grid, s, nullptr) != cudaSuccess)
        return err(CVX_ERR_CUDA, "convexify_points_static: pipeline launch failed");
    return CVX_OK;
}
