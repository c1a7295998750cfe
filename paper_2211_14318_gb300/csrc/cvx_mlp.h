// cvx_mlp.h -- internal interface of the surrogate network's tensor-core
// kernels (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cvx {

enum GemmEpiMode {
    EPI_F32 = 0,     // C = D (FP32)
    EPI_HIDDEN = 1,  // z = D + bias -> Z (FP32, optional), A = gelu(z) (bf16), AT = A^T (optional)
    EPI_OUT = 2,     // C[:, :n_store] = D + bias (FP32)
    EPI_DA = 3,      // dz = D * gelu'(Z) -> A (bf16), AT = dz^T, dbias += column sums
    EPI_DW = 4       // C[:m_store, :n_store] += D (FP32 atomics; split-K partial sums)
};

struct GemmEpi {
    int mode;
    int M_valid;       // rows holding data (EPI_F32/HIDDEN/OUT/DA)
    const int *M_dev;  // optional device-side row count; rows valid = *M_dev - m_off
    int m_off;
    float *C;
    int ldc;
    int m_store, n_store;
    const float *bias;
    float *Z;
    int ldz;
    __nv_bfloat16 *A;
    int lda;
    __nv_bfloat16 *AT;
    int ldat;
    float *dbias;
    int *err;  // set to 1 if a wait timed out
};

// 2-D tensor map of a row-major bf16 matrix (rows x cols, leading dimension ld
// elements) read in boxes of 8 columns x box_rows rows.  false if the CUDA
// driver's entry point is missing or the layout breaks the TMA rules.
bool make_tmap_bf16(CUtensorMap *map, const void *ptr, long long rows, long long cols,
                    long long ld, int box_rows);

// D = A B^T over M x N (tiles of 128 x BN, BN = 16 or 256), K in slices of
// k_split (multiples of 16).  tA: box rows 128; tB: box rows BN.
cudaError_t launch_gemm(const CUtensorMap &tA, const CUtensorMap &tB, int M, int N, int K,
                        int k_split, int BN, const GemmEpi &ep, cudaStream_t s);

}  // namespace cvx
