// cvx_surrogate.cu -- the surrogate proposal network: parameters, BF16
// packing, the forward and backward passes as sequences of tensor-core GEMMs
// (cvx_gemm.cu) with fused epilogues, the loss, Adam, training, save/load.
//
// Network: x = standardised (F11, F12, F21, F22, beta_k, ln det F) ->
// 4 x [256, GELU] -> 7 outputs (two direction angles, the logit of the volume
// fraction, the four entries of the jump F+ - F-).  Weights are kept in FP32
// (master copy, Adam state) and packed to BF16 for the tensor cores, in both
// orientations (W for the forward pass, W^T for back-propagation).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "cvx_handle.h"
#include "cvx_mlp.h"
#include "cvx_surrogate.h"

namespace cvx {

namespace {

constexpr long long kWOff[5] = {0, 1792, 67584, 133376, 199168};
constexpr long long kBOff[5] = {1536, 67328, 133120, 198912, 200960};
constexpr int kOut[5] = {256, 256, 256, 256, 7};
constexpr int kIn[5] = {6, 256, 256, 256, 256};
static_assert(kBOff[4] + 7 == kSurParams, "parameter layout");

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ kernels
// P (rows_pad x cols_pad) = W (out x in) zero-padded; T (cols_pad x rows_pad) = P^T.
__global__ void k_pack(const float *W, int out, int in, int rows_pad, int cols_pad, bf16 *P,
                       bf16 *T) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows_pad * cols_pad) return;
    const int r = idx / cols_pad, c = idx % cols_pad;
    const float v = (r < out && c < in) ? W[(long long)r * in + c] : 0.0f;
    const bf16 b = __float2bfloat16_rn(v);
    if (P) P[(long long)r * cols_pad + c] = b;
    if (T) T[(long long)c * rows_pad + r] = b;
}

// Standardised inputs of rows idx[m] (or m) -> X (n x 16, bf16, zero-padded)
// and its transpose XT (16 x ldt); optional labels gathered the same way.
__global__ void k_input(int n, const int *idx, const float *Xraw, const float *scale, bf16 *X,
                        bf16 *XT, int ldt, const float *Yraw, float *Y) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const long long src = idx ? idx[m] : m;
    for (int k = 0; k < 16; ++k) {
        const float v = k < 6 ? (Xraw[src * 6 + k] - scale[k]) * scale[6 + k] : 0.0f;
        const bf16 b = __float2bfloat16_rn(v);
        X[(long long)m * 16 + k] = b;
        if (XT) XT[(long long)k * ldt + m] = b;
    }
    if (Y)
        for (int k = 0; k < 7; ++k) Y[(long long)m * 7 + k] = Yraw[src * 7 + k];
}

// Loss of the batch (mean over its n samples) and dL/d(out), rounded to bf16
// as the operand of the last layer's back-propagation (dZ, n x 16 and its
// transpose); the output bias gradient from the unrounded values.
__global__ void k_loss(int n, const float *out, const float *Y, bf16 *dZ, bf16 *dZT, int ldt,
                       float *g_b4, float *loss) {
    __shared__ float s_l[8], s_b[8][7];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float inv_n = 1.0f / (float)n;
    float L = 0.0f, g[7] = {0, 0, 0, 0, 0, 0, 0};
    if (m < n) {
        const float *o = out + (long long)m * 7;
        const float *y = Y + (long long)m * 7;
        if (!isnan(y[0])) {
            for (int i = 0; i < 2; ++i) {
                const float d = 2.0f * (o[i] - y[i]);
                L += 1.0f - cosf(d);
                g[i] = 2.0f * sinf(d);
            }
        }
        if (!isnan(y[2])) {
            const float s = 1.0f / (1.0f + expf(-o[2]));
            L += (s - y[2]) * (s - y[2]);
            g[2] = 2.0f * (s - y[2]) * s * (1.0f - s);
        }
        for (int j = 3; j < 7; ++j) {
            const float d = o[j] - y[j];
            L += d * d;
            g[j] = 2.0f * d;
        }
        for (int j = 0; j < 16; ++j) {
            const bf16 b = __float2bfloat16_rn(j < 7 ? g[j] * inv_n : 0.0f);
            dZ[(long long)m * 16 + j] = b;
            dZT[(long long)j * ldt + m] = b;
        }
    }
    for (int o = 16; o; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
    for (int j = 0; j < 7; ++j)
        for (int o = 16; o; o >>= 1) g[j] += __shfl_xor_sync(0xffffffffu, g[j], o);
    if (lane == 0) {
        s_l[warp] = L;
        for (int j = 0; j < 7; ++j) s_b[warp][j] = g[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.0f, b[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s_l[w];
            for (int j = 0; j < 7; ++j) b[j] += s_b[w][j];
        }
        atomicAdd(loss, a * inv_n);
        for (int j = 0; j < 7; ++j) atomicAdd(g_b4 + j, b[j] * inv_n);
    }
}

__global__ void k_adam(long long n, float *w, const float *g, float *m, float *v, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <typename T>
cudaError_t alloc(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * count);
}

}  // namespace

void destroy_surrogate(cvx_handle *h) {
    Surrogate *S = h->sur;
    if (!S) return;
    void *ptrs[] = {S->scale, S->w, S->g, S->m, S->v, S->X, S->XT, S->dZo, S->dZoT, S->out, S->Yb,
                    S->loss, S->err, S->idx};
    for (void *p : ptrs) cudaFree(p);
    for (int l = 0; l < 5; ++l) {
        cudaFree(S->Wp[l]);
        cudaFree(S->Wt[l]);
    }
    for (int l = 0; l < 4; ++l) {
        cudaFree(S->A[l]);
        cudaFree(S->AT[l]);
        cudaFree(S->Z[l]);
    }
    for (int l = 0; l < 2; ++l) {
        cudaFree(S->dZ[l]);
        cudaFree(S->dZT[l]);
    }
    delete S;
    h->sur = nullptr;
}

int sur_params(cvx_handle *h) {
    if (h->sur && h->sur->w) return CVX_OK;
    if (!h->sur) h->sur = new Surrogate();
    Surrogate &S = *h->sur;
    CK(alloc(&S.scale, 12), "surrogate");
    CK(alloc(&S.w, kSurParams), "surrogate");
    CK(alloc(&S.g, kSurParams), "surrogate");
    CK(alloc(&S.m, kSurParams), "surrogate");
    CK(alloc(&S.v, kSurParams), "surrogate");
    CK(alloc(&S.loss, 1), "surrogate");
    CK(alloc(&S.err, 1), "surrogate");
    CK(cudaMemset(S.err, 0, sizeof(int)), "surrogate");
    CK(alloc(&S.Wp[0], 256 * 16), "surrogate");
    for (int l = 1; l < 4; ++l) {
        CK(alloc(&S.Wp[l], 256 * 256), "surrogate");
        CK(alloc(&S.Wt[l], 256 * 256), "surrogate");
    }
    CK(alloc(&S.Wp[4], 16 * 256), "surrogate");
    CK(alloc(&S.Wt[4], 256 * 16), "surrogate");
    return CVX_OK;
}

int sur_batch(cvx_handle *h, int n) {
    Surrogate &S = *h->sur;
    if (n <= S.cap) return CVX_OK;
    const int cap = ((n + 127) / 128) * 128;
    cudaDeviceSynchronize();
    bf16 **b16[] = {&S.X, &S.XT, &S.dZo, &S.dZoT};
    for (auto p : b16) {
        cudaFree(*p);
        *p = nullptr;
    }
    for (int l = 0; l < 4; ++l) {
        cudaFree(S.A[l]);
        cudaFree(S.AT[l]);
        cudaFree(S.Z[l]);
    }
    for (int l = 0; l < 2; ++l) {
        cudaFree(S.dZ[l]);
        cudaFree(S.dZT[l]);
    }
    cudaFree(S.out);
    cudaFree(S.Yb);
    S.cap = 0;
    CK(alloc(&S.X, (size_t)cap * 16), "surrogate batch");
    CK(alloc(&S.XT, (size_t)cap * 16), "surrogate batch");
    CK(alloc(&S.dZo, (size_t)cap * 16), "surrogate batch");
    CK(alloc(&S.dZoT, (size_t)cap * 16), "surrogate batch");
    for (int l = 0; l < 4; ++l) {
        CK(alloc(&S.A[l], (size_t)cap * 256), "surrogate batch");
        CK(alloc(&S.AT[l], (size_t)cap * 256), "surrogate batch");
        CK(alloc(&S.Z[l], (size_t)cap * 256), "surrogate batch");
    }
    for (int l = 0; l < 2; ++l) {
        CK(alloc(&S.dZ[l], (size_t)cap * 256), "surrogate batch");
        CK(alloc(&S.dZT[l], (size_t)cap * 256), "surrogate batch");
    }
    CK(alloc(&S.out, (size_t)cap * 7), "surrogate batch");
    CK(alloc(&S.Yb, (size_t)cap * 7), "surrogate batch");
    S.cap = cap;
    return CVX_OK;
}

namespace {

cudaError_t sur_pack(Surrogate &S, cudaStream_t s) {
    const int rp[5] = {256, 256, 256, 256, 16}, cp[5] = {16, 256, 256, 256, 256};
    for (int l = 0; l < 5; ++l) {
        const int total = rp[l] * cp[l];
        k_pack<<<(total + 255) / 256, 256, 0, s>>>(S.w + kWOff[l], kOut[l], kIn[l], rp[l], cp[l],
                                                   S.Wp[l], l ? S.Wt[l] : nullptr);
    }
    return cudaGetLastError();
}

GemmEpi epi(int mode, int Mv, int *err) {
    GemmEpi e = {};
    e.mode = mode;
    e.M_valid = Mv;
    e.err = err;
    return e;
}

#define TMAP(map, ptr, rows, cols, ld, box)                                           \
    do {                                                                              \
        if (!make_tmap_bf16(&(map), (ptr), (rows), (cols), (ld), (box)))              \
            return fail(CVX_ERR_CUDA, "tensor map for %s failed", #ptr);              \
    } while (0)

}  // namespace

// Forward pass of n <= cap standardised rows in S.X (and S.XT).  train: keep
// Z, A^T for the backward pass (otherwise the activations alternate between
// two buffers).  M_dev (optional): device-side row count, of which rows
// m_off .. m_off + n - 1 are these.
int sur_forward(cvx_handle *h, int n, bool train, cudaStream_t s, const int *M_dev, int m_off) {
    Surrogate &S = *h->sur;
    CUtensorMap tX, tW, tA;
    TMAP(tX, S.X, n, 16, 16, 128);
    TMAP(tW, S.Wp[0], 256, 16, 16, 256);
    GemmEpi e = epi(EPI_HIDDEN, n, S.err);
    e.M_dev = M_dev;
    e.m_off = m_off;
    e.bias = S.w + kBOff[0];
    e.Z = train ? S.Z[0] : nullptr;
    e.ldz = 256;
    e.A = S.A[0];
    e.lda = 256;
    e.AT = train ? S.AT[0] : nullptr;
    e.ldat = S.cap;
    CK(launch_gemm(tX, tW, n, 256, 16, 16, 256, e, s), "surrogate forward");
    for (int l = 1; l < 4; ++l) {
        bf16 *in = train ? S.A[l - 1] : S.A[(l - 1) & 1];
        TMAP(tA, in, n, 256, 256, 128);
        TMAP(tW, S.Wp[l], 256, 256, 256, 256);
        e.bias = S.w + kBOff[l];
        e.Z = train ? S.Z[l] : nullptr;
        e.A = train ? S.A[l] : S.A[l & 1];
        e.AT = train ? S.AT[l] : nullptr;
        CK(launch_gemm(tA, tW, n, 256, 256, 256, 256, e, s), "surrogate forward");
    }
    TMAP(tA, train ? S.A[3] : S.A[1], n, 256, 256, 128);
    TMAP(tW, S.Wp[4], 16, 256, 256, 16);
    GemmEpi o = epi(EPI_OUT, n, S.err);
    o.M_dev = M_dev;
    o.m_off = m_off;
    o.C = S.out;
    o.ldc = 7;
    o.n_store = 7;
    o.bias = S.w + kBOff[4];
    CK(launch_gemm(tA, tW, n, 16, 256, 256, 16, o, s), "surrogate forward");
    return CVX_OK;
}

namespace {

// Loss and gradient (added to S.g) of the batch in S.X / S.Yb after
// sur_forward(train = true).
int sur_backward(cvx_handle *h, int n, cudaStream_t s) {
    Surrogate &S = *h->sur;
    const int ld = S.cap;
    k_loss<<<(n + 255) / 256, 256, 0, s>>>(n, S.out, S.Yb, S.dZo, S.dZoT, ld, S.g + kBOff[4],
                                           S.loss);
    CK(cudaGetLastError(), "surrogate loss");
    const int K = ((n + 15) / 16) * 16;
    const int ks = 1024;
    CUtensorMap ta, tb;
    // last layer: dW4 = dZo^T A4, dZ4 = (dZo W4) * gelu'(Z4)
    TMAP(ta, S.dZoT, 16, n, ld, 128);
    TMAP(tb, S.AT[3], 256, n, ld, 256);
    GemmEpi w = epi(EPI_DW, 16, S.err);
    w.C = S.g + kWOff[4];
    w.ldc = 256;
    w.m_store = 7;
    w.n_store = 256;
    CK(launch_gemm(ta, tb, 16, 256, K, ks, 256, w, s), "surrogate backward");
    TMAP(ta, S.dZo, n, 16, 16, 128);
    TMAP(tb, S.Wt[4], 256, 16, 16, 256);
    GemmEpi d = epi(EPI_DA, n, S.err);
    d.Z = S.Z[3];
    d.ldz = 256;
    d.A = S.dZ[0];
    d.lda = 256;
    d.AT = S.dZT[0];
    d.ldat = ld;
    d.dbias = S.g + kBOff[3];
    CK(launch_gemm(ta, tb, n, 256, 16, 16, 256, d, s), "surrogate backward");
    int cur = 0;
    for (int l = 3; l >= 1; --l) {
        // dW_l = dZ_{l+1}^T A_l (A_l = output of hidden layer l)
        TMAP(ta, S.dZT[cur], 256, n, ld, 128);
        TMAP(tb, S.AT[l - 1], 256, n, ld, 256);
        w.C = S.g + kWOff[l];
        w.m_store = 256;
        w.M_valid = 256;
        CK(launch_gemm(ta, tb, 256, 256, K, ks, 256, w, s), "surrogate backward");
        // dZ_l = (dZ_{l+1} W_l) * gelu'(Z_l)
        TMAP(ta, S.dZ[cur], n, 256, 256, 128);
        TMAP(tb, S.Wt[l], 256, 256, 256, 256);
        d.Z = S.Z[l - 1];
        d.A = S.dZ[cur ^ 1];
        d.AT = S.dZT[cur ^ 1];
        d.dbias = S.g + kBOff[l - 1];
        CK(launch_gemm(ta, tb, n, 256, 256, 256, 256, d, s), "surrogate backward");
        cur ^= 1;
    }
    // dW0 = dZ_1^T X
    TMAP(ta, S.dZT[cur], 256, n, ld, 128);
    TMAP(tb, S.XT, 16, n, ld, 16);
    w.C = S.g + kWOff[0];
    w.ldc = 6;
    w.m_store = 256;
    w.n_store = 6;
    CK(launch_gemm(ta, tb, 256, 16, K, ks, 16, w, s), "surrogate backward");
    return CVX_OK;
}

int check_err(Surrogate &S, cudaStream_t s) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, S.err, sizeof(int), cudaMemcpyDeviceToHost, s), "surrogate");
    CK(cudaStreamSynchronize(s), "surrogate");
    if (e) {
        cudaMemsetAsync(S.err, 0, sizeof(int), s);
        return fail(CVX_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
    }
    return CVX_OK;
}

void init_host(std::vector<float> &p, uint64_t seed) {
    std::mt19937_64 rng(seed);
    p.assign(kSurParams, 0.0f);
    for (int l = 0; l < 5; ++l) {
        const float b = 1.0f / sqrtf((float)kIn[l]);
        std::uniform_real_distribution<float> u(-b, b);
        for (long long i = 0; i < (long long)kOut[l] * kIn[l]; ++i) p[kWOff[l] + i] = u(rng);
        for (int i = 0; i < kOut[l]; ++i) p[kBOff[l] + i] = u(rng);
    }
}

int upload_weights(cvx_handle *h, const float *params, const float *mean, const float *stdv,
                   cudaStream_t s) {
    Surrogate &S = *h->sur;
    for (int k = 0; k < 6; ++k) {
        if (!(stdv[k] > 0.0f) || !isfinite(mean[k]))
            return fail(CVX_ERR_INVALID_ARG, "input scaling: std must be > 0");
        S.scale_h[k] = mean[k];
        S.scale_h[6 + k] = 1.0f / stdv[k];
    }
    CK(cudaMemcpy(S.scale, S.scale_h, sizeof(float) * 12, cudaMemcpyHostToDevice), "surrogate");
    CK(cudaMemcpy(S.w, params, sizeof(float) * kSurParams, cudaMemcpyHostToDevice), "surrogate");
    CK(cudaMemset(S.m, 0, sizeof(float) * kSurParams), "surrogate");
    CK(cudaMemset(S.v, 0, sizeof(float) * kSurParams), "surrogate");
    S.adam_t = 0;
    CK(sur_pack(S, s), "surrogate pack");
    S.has_weights = true;
    return CVX_OK;
}

}  // namespace

}  // namespace cvx

using namespace cvx;

extern "C" {

int cvx_gemm_bf16(cvx_handle *h, int M, int N, int K, const uint16_t *A, const uint16_t *B,
                  float *C, cvx_stream sv) {
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (M < 1 || N < 1 || K < 16 || K % 16) return fail(CVX_ERR_INVALID_ARG, "need M, N >= 1 and K a positive multiple of 16");
    if (!A || !B || !C) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    DeviceGuard g(h->device);
    CUtensorMap ta, tb;
    const int BN = N <= 16 ? 16 : 256;
    TMAP(ta, A, M, K, K, 128);
    TMAP(tb, B, N, K, K, BN);
    int rc = sur_params(h);
    if (rc) return rc;
    GemmEpi e = epi(EPI_F32, M, h->sur->err);
    e.C = C;
    e.ldc = N;
    CK(launch_gemm(ta, tb, M, N, K, ((K + 63) / 64) * 64, BN, e, (cudaStream_t)sv), "cvx_gemm_bf16");
    return check_err(*h->sur, (cudaStream_t)sv);
}

int surrogate_set_weights(cvx_handle *h, const float *params, const float *mean,
                          const float *stdv) {
    if (!h || !params || !mean || !stdv) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(h->device);
    int rc = sur_params(h);
    if (rc) return rc;
    rc = upload_weights(h, params, mean, stdv, 0);
    if (rc) return rc;
    CK(cudaDeviceSynchronize(), "surrogate_set_weights");
    return CVX_OK;
}

int surrogate_get_weights(cvx_handle *h, float *params, float *mean, float *stdv) {
    if (!h || !params || !mean || !stdv) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    if (!h->sur || !h->sur->has_weights) return fail(CVX_ERR_NOT_TRAINED, "no surrogate weights");
    DeviceGuard g(h->device);
    Surrogate &S = *h->sur;
    CK(cudaDeviceSynchronize(), "surrogate_get_weights");
    CK(cudaMemcpy(params, S.w, sizeof(float) * kSurParams, cudaMemcpyDeviceToHost), "surrogate_get_weights");
    for (int k = 0; k < 6; ++k) {
        mean[k] = S.scale_h[k];
        stdv[k] = 1.0f / S.scale_h[6 + k];
    }
    return CVX_OK;
}

int surrogate_forward(cvx_handle *h, int64_t n, const float *X, float *out, cvx_stream sv) {
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 0) return fail(CVX_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!X || !out)) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    if (!h->sur || !h->sur->has_weights) return fail(CVX_ERR_NOT_TRAINED, "no surrogate weights");
    if (n == 0) return CVX_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    Surrogate &S = *h->sur;
    const int chunk = 1 << 16;
    int rc = sur_batch(h, (int)std::min<int64_t>(n, chunk));
    if (rc) return rc;
    for (int64_t o = 0; o < n; o += chunk) {
        const int m = (int)std::min<int64_t>(chunk, n - o);
        k_input<<<(m + 255) / 256, 256, 0, s>>>(m, nullptr, X + 6 * o, S.scale, S.X, nullptr, 0,
                                                nullptr, nullptr);
        CK(cudaGetLastError(), "surrogate_forward");
        rc = sur_forward(h, m, false, s, nullptr, 0);
        if (rc) return rc;
        CK(cudaMemcpyAsync(out + 7 * o, S.out, sizeof(float) * 7 * m, cudaMemcpyDeviceToDevice, s),
           "surrogate_forward");
    }
    return check_err(S, s);
}

int surrogate_loss_grad(cvx_handle *h, int64_t n, const float *X, const float *Y, float *loss,
                        float *grad, cvx_stream sv) {
    if (!h) return fail(CVX_ERR_INVALID_ARG, "handle is NULL");
    if (n < 1 || n > (1 << 20)) return fail(CVX_ERR_INVALID_ARG, "n must be in [1, 2^20]");
    if (!X || !Y || !loss || !grad) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    if (!h->sur || !h->sur->has_weights) return fail(CVX_ERR_NOT_TRAINED, "no surrogate weights");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    Surrogate &S = *h->sur;
    int rc = sur_batch(h, (int)n);
    if (rc) return rc;
    k_input<<<((int)n + 255) / 256, 256, 0, s>>>((int)n, nullptr, X, S.scale, S.X, S.XT, S.cap, Y,
                                                 S.Yb);
    CK(cudaGetLastError(), "surrogate_loss_grad");
    CK(cudaMemsetAsync(S.g, 0, sizeof(float) * kSurParams, s), "surrogate_loss_grad");
    CK(cudaMemsetAsync(S.loss, 0, sizeof(float), s), "surrogate_loss_grad");
    rc = sur_forward(h, (int)n, true, s, nullptr, 0);
    if (rc) return rc;
    rc = sur_backward(h, (int)n, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(grad, S.g, sizeof(float) * kSurParams, cudaMemcpyDeviceToDevice, s), "surrogate_loss_grad");
    CK(cudaMemcpyAsync(loss, S.loss, sizeof(float), cudaMemcpyDeviceToDevice, s), "surrogate_loss_grad");
    return check_err(S, s);
}

int surrogate_train(cvx_handle *h, int64_t n, const float *X, const float *Y,
                    const cvx_train_cfg *cfg, float *loss_log, cvx_stream sv) {
    if (!h || !cfg) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(CVX_ERR_INVALID_ARG, "n out of range");
    if (!X || !Y) return fail(CVX_ERR_INVALID_ARG, "NULL array");
    if (cfg->epochs < 0 || cfg->batch < 16 || cfg->batch > (1 << 16) || !(cfg->lr > 0.0f))
        return fail(CVX_ERR_INVALID_ARG, "train cfg: epochs >= 0, 16 <= batch <= 65536, lr > 0");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)sv;
    int rc = sur_params(h);
    if (rc) return rc;
    Surrogate &S = *h->sur;
    if (cfg->init || !S.has_weights) {
        // input standardisation from the data, fresh weights
        std::vector<float> x((size_t)n * 6);
        CK(cudaMemcpyAsync(x.data(), X, sizeof(float) * x.size(), cudaMemcpyDeviceToHost, s), "surrogate_train");
        CK(cudaStreamSynchronize(s), "surrogate_train");
        float mean[6], stdv[6];
        for (int k = 0; k < 6; ++k) {
            double a = 0.0, b = 0.0;
            for (int64_t i = 0; i < n; ++i) a += x[(size_t)i * 6 + k];
            a /= (double)n;
            for (int64_t i = 0; i < n; ++i) b += (x[(size_t)i * 6 + k] - a) * (x[(size_t)i * 6 + k] - a);
            mean[k] = (float)a;
            stdv[k] = (float)std::max(sqrt(b / (double)n), 1e-6);
        }
        std::vector<float> p;
        init_host(p, cfg->seed);
        rc = upload_weights(h, p.data(), mean, stdv, s);
        if (rc) return rc;
    }
    const int B = cfg->batch;
    rc = sur_batch(h, B);
    if (rc) return rc;
    if (S.idx_cap < n) {
        cudaFree(S.idx);
        S.idx = nullptr;
        S.idx_cap = 0;
        CK(alloc(&S.idx, (size_t)n), "surrogate_train");
        S.idx_cap = n;
    }
    std::vector<int> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
    std::mt19937_64 rng(cfg->seed ^ 0x9E3779B97F4A7C15ull);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < cfg->epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        CK(cudaMemcpyAsync(S.idx, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s), "surrogate_train");
        CK(cudaMemsetAsync(S.loss, 0, sizeof(float), s), "surrogate_train");
        int batches = 0;
        for (int64_t o = 0; o + B <= n || (o == 0 && n < B); o += B) {
            const int m = (int)std::min<int64_t>(B, n - o);
            k_input<<<(m + 255) / 256, 256, 0, s>>>(m, S.idx + o, X, S.scale, S.X, S.XT, S.cap, Y, S.Yb);
            CK(cudaGetLastError(), "surrogate_train");
            CK(cudaMemsetAsync(S.g, 0, sizeof(float) * kSurParams, s), "surrogate_train");
            rc = sur_forward(h, m, true, s, nullptr, 0);
            if (rc) return rc;
            rc = sur_backward(h, m, s);
            if (rc) return rc;
            ++S.adam_t;
            const float c1 = 1.0f - powf(b1, (float)S.adam_t), c2 = 1.0f - powf(b2, (float)S.adam_t);
            k_adam<<<(kSurParams + 255) / 256, 256, 0, s>>>(kSurParams, S.w, S.g, S.m, S.v, cfg->lr, b1, b2, eps, c1, c2);
            CK(sur_pack(S, s), "surrogate_train");
            ++batches;
            if (n < B) break;
        }
        rc = check_err(S, s);
        if (rc) return rc;
        if (loss_log) {
            float l = 0.0f;
            CK(cudaMemcpy(&l, S.loss, sizeof(float), cudaMemcpyDeviceToHost), "surrogate_train");
            loss_log[ep] = l / (float)std::max(batches, 1);
        }
    }
    CK(cudaStreamSynchronize(s), "surrogate_train");
    return CVX_OK;
}

int surrogate_save(cvx_handle *h, const char *path) {
    if (!h || !path) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    if (!h->sur || !h->sur->has_weights) return fail(CVX_ERR_NOT_TRAINED, "no surrogate weights");
    std::vector<float> p(kSurParams);
    float mean[6], stdv[6];
    int rc = surrogate_get_weights(h, p.data(), mean, stdv);
    if (rc) return rc;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(CVX_ERR_INVALID_ARG, "cannot open %s", path);
    const char magic[8] = {'C', 'V', 'X', 'S', 'U', 'R', '0', '1'};
    const int32_t np = (int32_t)kSurParams;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&np, 4, 1, f) == 1 &&
              fwrite(mean, 4, 6, f) == 6 && fwrite(stdv, 4, 6, f) == 6 &&
              fwrite(p.data(), 4, p.size(), f) == p.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? CVX_OK : fail(CVX_ERR_INVALID_ARG, "write to %s failed", path);
}

int surrogate_load(cvx_handle *h, const char *path) {
    if (!h || !path) return fail(CVX_ERR_INVALID_ARG, "NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(CVX_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int32_t np = 0;
    float mean[6], stdv[6];
    std::vector<float> p(kSurParams);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "CVXSUR01", 8) == 0 &&
              fread(&np, 4, 1, f) == 1 && np == (int32_t)kSurParams && fread(mean, 4, 6, f) == 6 &&
              fread(stdv, 4, 6, f) == 6 && fread(p.data(), 4, p.size(), f) == p.size();
    fclose(f);
    if (!ok) return fail(CVX_ERR_INVALID_ARG, "%s is not a surrogate file", path);
    return surrogate_set_weights(h, p.data(), mean, stdv);
}

}  // extern "C"
