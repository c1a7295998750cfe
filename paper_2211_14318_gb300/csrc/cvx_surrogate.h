// cvx_surrogate.h -- internal interface of the surrogate proposal network
// (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

struct cvx_handle;

namespace cvx {

// Flat FP32 parameters: W0 (256 x 6), b0, W1..W3 (256 x 256), b1..b3,
// W4 (7 x 256), b4 (7); weights row-major as (out, in).
constexpr long long kSurParams = 200967;

struct Surrogate;
void destroy_surrogate(cvx_handle *h);

}  // namespace cvx
