// cvx_surrogate.h -- internal interface of the surrogate proposal network
// (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

struct cvx_handle;

namespace cvx {

// Flat FP32 parameters: W0 (256 x 6), b0, W1..W3 (256 x 256), b1..b3,
// W4 (7 x 256), b4 (7); weights row-major as (out, in).
constexpr long long kSurParams = 200967;

// Weights, optimiser state and batch buffers of the network (one per handle).
struct Surrogate {
    bool has_weights = false;
    float scale_h[12];  // mean (6), 1/std (6)
    float *scale = nullptr;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *Wp[5] = {}, *Wt[5] = {};
    long long adam_t = 0;
    int cap = 0;
    __nv_bfloat16 *X = nullptr, *XT = nullptr, *A[4] = {}, *AT[4] = {}, *dZo = nullptr,
                  *dZoT = nullptr, *dZ[2] = {}, *dZT[2] = {};
    float *Z[4] = {}, *out = nullptr, *Yb = nullptr, *loss = nullptr;
    int *err = nullptr;
    int *idx = nullptr;
    long long idx_cap = 0;
};

void destroy_surrogate(cvx_handle *h);
int sur_params(cvx_handle *h);
// Batch buffers for at least n rows.
int sur_batch(cvx_handle *h, int n);
int sur_forward(cvx_handle *h, int n, bool train, cudaStream_t s, const int *M_dev, int m_off);

}  // namespace cvx
