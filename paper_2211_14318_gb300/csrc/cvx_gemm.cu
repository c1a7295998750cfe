// cvx_gemm.cu -- the BF16 tensor-core GEMM of the surrogate network
// (tcgen05, FP32 accumulation in TMEM, operands staged by TMA) with the
// epilogues of the network's forward and backward passes fused in.
//
//   D[m][n] = sum_k A[m][k] B[n][k]       (A: M x K, B: N x K, both bf16,
//                                          row-major with K contiguous)
//
// One CTA of 256 threads computes a 128 x BN tile over a K range (split-K for
// the weight gradients).  Thread 0 issues the TMA loads (one box per k-block
// of 8 elements, two stages of 64) and the MMAs (K = 16 each); then warps w
// and w + 4 read the TMEM lanes of rows 32 (w % 4) .. +31 (one accumulator
// row per thread), each half of the columns, and apply the epilogue.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "cvx_mlp.h"
#include "cvx_tc.cuh"

namespace cvx {

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 2;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s per wait, then give up

// Normal CDF Phi(z) and density phi(z) with erf from Abramowitz & Stegun,
// Handbook of Mathematical Functions, formula 7.1.26:
//   erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2),
//   t = 1 / (1 + p x), x >= 0, |error| <= 1.5e-7
// (one exponential shared by Phi and phi).
__device__ __forceinline__ void normal_cdf_pdf(float z, float &Phi, float &phi) {
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f),
                         -0.284496736f),
                 0.254829592f);
    const float ex = __expf(-x * x);
    const float erfx = 1.0f - poly * ex;
    Phi = 0.5f * (1.0f + (z < 0.0f ? -erfx : erfx));
    phi = 0.39894228040143268f * ex;
}
__device__ __forceinline__ float gelu(float z) {
    float Phi, phi;
    normal_cdf_pdf(z, Phi, phi);
    return z * Phi;
}
__device__ __forceinline__ float gelu_grad(float z) {
    float Phi, phi;
    normal_cdf_pdf(z, Phi, phi);
    return Phi + z * phi;
}

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16 *dst, const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// The epilogue of 16 accumulator columns n .. n + 15 of row m (one thread).
__device__ __forceinline__ void gemm_epilogue(const GemmEpi &ep, int m, int n, const float (&v)[16],
                                              int Mv, int N, int lane) {
    switch (ep.mode) {
    case EPI_F32:
        if (m < Mv)
            for (int i = 0; i < 16; ++i)
                if (n + i < N) ep.C[(long long)m * ep.ldc + n + i] = v[i];
        break;
    case EPI_HIDDEN: {
        if (m >= Mv) break;
        float a[16];
        for (int i = 0; i < 16; ++i) {
            const float z = v[i] + ep.bias[n + i];
            if (ep.Z) ep.Z[(long long)m * ep.ldz + n + i] = z;
            a[i] = gelu(z);
        }
        store_bf16x16(ep.A + (long long)m * ep.lda + n, a);
        if (ep.AT)
            for (int i = 0; i < 16; ++i)
                ep.AT[(long long)(n + i) * ep.ldat + m] = __float2bfloat16_rn(a[i]);
        break;
    }
    case EPI_OUT:
        if (m < Mv)
            for (int i = 0; i < 16; ++i)
                if (n + i < ep.n_store)
                    ep.C[(long long)m * ep.ldc + n + i] = v[i] + ep.bias[n + i];
        break;
    case EPI_DA: {
        float dz[16];
        const bool in = m < Mv;
        for (int i = 0; i < 16; ++i)
            dz[i] = in ? v[i] * gelu_grad(ep.Z[(long long)m * ep.ldz + n + i]) : 0.0f;
        if (in) {
            store_bf16x16(ep.A + (long long)m * ep.lda + n, dz);
            if (ep.AT)
                for (int i = 0; i < 16; ++i)
                    ep.AT[(long long)(n + i) * ep.ldat + m] = __float2bfloat16_rn(dz[i]);
        }
        if (ep.dbias) {
            for (int i = 0; i < 16; ++i) {
                float s = dz[i];
                for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) atomicAdd(ep.dbias + n + i, s);
            }
        }
        break;
    }
    case EPI_DW:
        if (m < ep.m_store)
            for (int i = 0; i < 16; ++i)
                if (n + i < ep.n_store) atomicAdd(ep.C + (long long)m * ep.ldc + n + i, v[i]);
        break;
    }
}

template <int BN>
__global__ void __launch_bounds__(256, 1)
    k_gemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int M,
           int N, int K, int k_split, GemmEpi ep) {
    constexpr int A_BYTES = kBM * kBK * 2;
    constexpr int B_BYTES = BN * kBK * 2;
    constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = smem;
    unsigned char *sB = smem + kStages * A_BYTES;
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_mma[kStages], bar_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;

    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kc0 = blockIdx.z * k_split;
    const int kc1 = min(K, kc0 + k_split);
    const int Mv = ep.M_dev ? min(*ep.M_dev - ep.m_off, ep.M_valid) : ep.M_valid;
    if (ep.mode != EPI_DW && m0 >= Mv) return;  // the whole tile is padding
    if (kc0 >= kc1) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_mma[s], 1);
        }
        mbar_init(&bar_done, 1);
        s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    const int nchunks = (kc1 - kc0 + kBK - 1) / kBK;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_bf16(kBM, BN);
        auto issue = [&](int c) {
            const int s = c % kStages;
            const int k0 = kc0 + c * kBK;
            const int kbn = min(kBK, kc1 - k0) / 8;
            mbar_expect_tx(&bar_full[s], (unsigned)(kbn * (kBM + BN) * 16));
            for (int kb = 0; kb < kbn; ++kb) {
                tma_load_2d(sA + s * A_BYTES + kb * kBM * 16, &tA, &bar_full[s], k0 + 8 * kb, m0);
                tma_load_2d(sB + s * B_BYTES + kb * BN * 16, &tB, &bar_full[s], k0 + 8 * kb, n0);
            }
        };
        bool ok = true;
        issue(0);
        for (int c = 0; c < nchunks && ok; ++c) {
            const int s = c % kStages;
            if (c + 1 < nchunks) {
                const int c2 = c + 1, s2 = c2 % kStages;
                if (c2 >= kStages) ok = mbar_wait(&bar_mma[s2], ((c2 - kStages) / kStages) & 1, kWaitNs);
                if (!ok) break;
                issue(c2);
            }
            ok = mbar_wait(&bar_full[s], (c / kStages) & 1, kWaitNs);
            if (!ok) break;
            tc_fence_after();
            const int kbn = min(kBK, kc1 - (kc0 + c * kBK)) / 8;
            const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
            for (int j = 0; j < kbn / 2; ++j) {
                const uint64_t ad = smem_desc(a0 + 2 * j * kBM * 16, kBM * 16, 128);
                const uint64_t bd = smem_desc(b0 + 2 * j * BN * 16, BN * 16, 128);
                umma_bf16(tmem, ad, bd, idesc, (c > 0 || j > 0) ? 1u : 0u);
            }
            umma_commit(&bar_mma[s]);
        }
        if (ok) {
            umma_commit(&bar_done);
        } else {
            s_fail = 1;
            if (ep.err) atomicExch(ep.err, 1);
        }
    }
    __syncwarp();
    bool ok = mbar_wait(&bar_done, 0, kWaitNs);
    if (!ok && ep.err) atomicExch(ep.err, 1);
    tc_fence_after();

    const int quarter = warp & 3;
    const int m = m0 + 32 * quarter + lane;
    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
    // columns of this warp: halves of the tile (BN = 16: warps 0-3 only)
    constexpr int CW = BN >= 32 ? BN / 2 : BN;
    const int cbeg = (warp >> 2) * CW;
    const int cend = BN >= 32 ? cbeg + CW : (warp < 4 ? BN : 0);
    for (int c0 = cbeg; c0 < cend; c0 += 16) {
        float v[16];
        tmem_ld16(trow + c0, v);
        if (ok) gemm_epilogue(ep, m, n0 + c0, v, Mv, N, lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TCOLS);
    }
}

// Persistent, warp-specialised form for K <= 256 (all forward layers and
// the input-gradient products): the B operand (the weights, BN x K) stays in
// shared memory for the whole kernel; A tiles (128 x 64) stream through a
// four-stage ring; two TMEM accumulators let the epilogue of one tile run
// while the MMAs of the next are in flight.  Warp 0 (lane 0) issues the TMA
// loads, warp 1 (lane 0) the MMAs, warps 4..11 run the epilogue (two per
// TMEM lane quarter, each half of the columns); every wait is bounded.
constexpr int kWsStages = 4;
constexpr int kWsThreads = 384;

template <int BN>
constexpr size_t gemm_ws_smem(int K) {
    return (size_t)BN * K * 2 + (size_t)kWsStages * kBM * kBK * 2 + 1024;
}

template <int BN>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_gemm_ws(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
              int M, int N, int K, GemmEpi ep) {
    constexpr int A_STAGE = kBM * kBK * 2;
    constexpr uint32_t TC = BN < 32 ? 32 : BN;  // columns per accumulator
    constexpr uint32_t TCOLS = 2 * TC;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = smem;
    unsigned char *sA = smem + (size_t)BN * K * 2;
    __shared__ __align__(8) uint64_t full[kWsStages], empty[kWsStages], bfull, accf[2], acce[2];
    __shared__ uint32_t s_tmem;

    const int Mv = ep.M_dev ? min(*ep.M_dev - ep.m_off, ep.M_valid) : ep.M_valid;
    const int ntiles = Mv > 0 ? (Mv + kBM - 1) / kBM : 0;
    if ((int)blockIdx.x >= ntiles) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkc = (K + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kWsStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&bfull, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], 8);
        }
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            bool ok = true;
            mbar_expect_tx(&bfull, (unsigned)((K / 8) * BN * 16));
            for (int kb = 0; kb < K / 8; ++kb) tma_load_2d(sB + kb * BN * 16, &tB, &bfull, 8 * kb, 0);
            int u = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int kc = 0; kc < nkc; ++kc, ++u) {
                    const int st = u % kWsStages, use = u / kWsStages;
                    if (use > 0 && !(ok = mbar_wait(&empty[st], (use - 1) & 1, kWaitNs))) break;
                    const int k0 = kc * kBK, kbn = min(kBK, K - k0) / 8;
                    mbar_expect_tx(&full[st], (unsigned)(kbn * kBM * 16));
                    for (int kb = 0; kb < kbn; ++kb)
                        tma_load_2d(sA + st * A_STAGE + kb * kBM * 16, &tA, &full[st], k0 + 8 * kb,
                                    t * kBM);
                }
            }
            if (!ok && ep.err) atomicExch(ep.err, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kBM, BN);
            bool ok = mbar_wait(&bfull, 0, kWaitNs);
            int u = 0, v = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++v) {
                const int acc = v & 1, vu = v >> 1;
                if (vu > 0 && !(ok = mbar_wait(&acce[acc], (vu - 1) & 1, kWaitNs))) break;
                tc_fence_after();
                const uint32_t d = tmem + acc * TC;
                for (int kc = 0; kc < nkc; ++kc, ++u) {
                    const int st = u % kWsStages, use = u / kWsStages;
                    if (!(ok = mbar_wait(&full[st], use & 1, kWaitNs))) break;
                    tc_fence_after();
                    const int kbn = min(kBK, K - kc * kBK) / 8;
                    const uint32_t a0 = smem_u32(sA + st * A_STAGE);
                    const uint32_t b0 = smem_u32(sB + (size_t)kc * 8 * BN * 16);
                    for (int j = 0; j < kbn / 2; ++j) {
                        const uint64_t ad = smem_desc(a0 + 2 * j * kBM * 16, kBM * 16, 128);
                        const uint64_t bd = smem_desc(b0 + 2 * j * BN * 16, BN * 16, 128);
                        umma_bf16(d, ad, bd, idesc, (kc > 0 || j > 0) ? 1u : 0u);
                    }
                    umma_commit(&empty[st]);
                }
                if (!ok) break;
                umma_commit(&accf[acc]);
            }
            if (!ok && ep.err) atomicExch(ep.err, 1);
        }
    } else if (warp >= 4) {
        const int ew = warp - 4, quarter = ew & 3, half = ew >> 2;
        constexpr int CW = BN >= 32 ? BN / 2 : BN;
        const int cbeg = half * CW;
        const int cend = BN >= 32 ? cbeg + CW : (half == 0 ? BN : 0);
        int v = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++v) {
            const int acc = v & 1, vu = v >> 1;
            if (!mbar_wait(&accf[acc], vu & 1, kWaitNs)) {
                if (ep.err) atomicExch(ep.err, 1);
                break;
            }
            tc_fence_after();
            const int m = t * kBM + 32 * quarter + lane;
            const uint32_t trow = tmem + acc * TC + ((uint32_t)(32 * quarter) << 16);
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                float r[16];
                tmem_ld16(trow + c0, r);
                gemm_epilogue(ep, m, c0, r, Mv, N, lane);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, TCOLS);
    }
}

template <int BN>
constexpr size_t gemm_smem() {
    return (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool make_tmap_bf16(CUtensorMap *map, const void *ptr, long long rows, long long cols,
                    long long ld, int box_rows) {
    EncodeTiled enc = encode_fn();
    if (!enc) return false;
    if (((uintptr_t)ptr & 15) || (ld * 2) % 16 || rows < 1 || cols < 1) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

cudaError_t launch_gemm(const CUtensorMap &tA, const CUtensorMap &tB, int M, int N, int K,
                        int k_split, int BN, const GemmEpi &ep, cudaStream_t s) {
    if (K % 16 || k_split % 16 || k_split < 16) return cudaErrorInvalidValue;
    if (ep.mode != EPI_DW && K <= 256 && k_split >= K && N <= BN) {
        // one tile column, the whole K: the persistent warp-specialised form
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned grid = (unsigned)std::max(1, std::min((M + kBM - 1) / kBM, sms));
        cudaError_t e;
        if (BN == 256) {
            const size_t sm = gemm_ws_smem<256>(K);
            if ((e = cudaFuncSetAttribute(k_gemm_ws<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm)) != cudaSuccess)
                return e;
            k_gemm_ws<256><<<grid, kWsThreads, sm, s>>>(tA, tB, M, N, K, ep);
        } else if (BN == 16) {
            const size_t sm = gemm_ws_smem<16>(K);
            if ((e = cudaFuncSetAttribute(k_gemm_ws<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm)) != cudaSuccess)
                return e;
            k_gemm_ws<16><<<grid, kWsThreads, sm, s>>>(tA, tB, M, N, K, ep);
        } else {
            return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, (K + k_split - 1) / k_split);
    if (BN == 256) {
        const size_t sm = gemm_smem<256>();
        cudaError_t e = cudaFuncSetAttribute(k_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gemm<256><<<grid, 256, sm, s>>>(tA, tB, M, N, K, k_split, ep);
    } else if (BN == 16) {
        const size_t sm = gemm_smem<16>();
        cudaError_t e = cudaFuncSetAttribute(k_gemm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gemm<16><<<grid, 256, sm, s>>>(tA, tB, M, N, K, k_split, ep);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cvx
