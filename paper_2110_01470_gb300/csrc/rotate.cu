// rotate.cu -- operand preparation for the tensor-core rotation (split BF16
// planes, row norms, tensor maps) and psso_rotate: z = M (x - o) for N rows
// on the tensor cores.
#include <cmath>
#include <cstdio>
#include <cudaTypedefs.h>
#include <mutex>

#include "psso.h"
#include "psso_internal.h"
#include "sso_common.cuh"
#include "rot_pipeline.h"
#include "tc_gemm.cuh"

namespace psso {
namespace tc {

bool make_tmap_bf16(CUtensorMap* map, const void* base, int Kp, int rows, int box_rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// B planes and row-norm bounds of the FP32 rotation: one block per row j of
// the padded [Jp][Kp] planes (rows >= D and columns >= D are zero).
__global__ void split_matrix(const float* __restrict__ M32, int D, int Jp, int Kp, __nv_bfloat16* B,
                             float* mnorm)
{
    const int j = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        const float v = (j < D && k < D) ? M32[(size_t)j * D + k] : 0.f;
        __nv_bfloat16 h, m, l;
        split3(v, h, m, l);
        const size_t o = (size_t)j * Kp + k, plane = (size_t)Jp * Kp;
        B[o] = h;
        B[plane + o] = m;
        B[2 * plane + o] = l;
        s = fma((double)v, (double)v, s);
    }
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        // FP64 sum of at most 2^20 squares: relative error far below 1e-9.
        mnorm[j] = f64_to_f32_ru(sqrt(t) * (1.0 + 1e-9));
    }
}

// A planes of z = M (x - o) for plain rows (psso_rotate): warp per row.
__global__ void split_rows(const float* __restrict__ X, const float* __restrict__ o, int N, int D, int Np,
                           int Kp, __nv_bfloat16* A)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= Np) return;
    const int lane = threadIdx.x & 31;
    const size_t plane = (size_t)Np * Kp;
    for (int k = lane; k < Kp; k += 32) {
        const float d = (i < N && k < D) ? __fsub_rn(X[(size_t)i * D + k], o[k]) : 0.f;
        __nv_bfloat16 h, m, l;
        split3(d, h, m, l);
        const size_t p = (size_t)i * Kp + k;
        A[p] = h;
        A[plane + p] = m;
        A[2 * plane + p] = l;
    }
}

cudaError_t launch_split_matrix(const float* M32, int D, int Jp, int Kp, __nv_bfloat16* B, float* mnorm,
                                cudaStream_t s)
{
    split_matrix<<<Jp, 256, 0, s>>>(M32, D, Jp, Kp, B, mnorm);
    return cudaGetLastError();
}

cudaError_t launch_split_rows(const float* X, const float* o, int N, int D, int Np, int Kp, __nv_bfloat16* A,
                              cudaStream_t s)
{
    split_rows<<<(Np + 7) / 8, 256, 0, s>>>(X, o, N, D, Np, Kp, A);
    return cudaGetLastError();
}

struct ZEpi {
    float* Z;
    int N, D;
    __device__ void operator()(int c, const float (&z)[32]) const
    {
        const int i = blockIdx.x * BM + threadIdx.x;
        const int j0 = blockIdx.y * BN + 32 * c;
        if (i >= N) return;
#pragma unroll
        for (int t = 0; t < 32; ++t)
            if (j0 + t < D) Z[(size_t)i * D + j0 + t] = z[t];
    }
};

__global__ void __launch_bounds__(128, 1)
    rotate_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs a,
                ZEpi epi)
{
    gemm_tile(&tmA, &tmB, a, epi);
}

}  // namespace tc
}  // namespace psso

extern "C" psso_status psso_rotate(int64_t N, int64_t D, const float* X, const float* shift,
                                   const float* rotation, float* Z, void* stream)
{
    using namespace psso;
    using namespace psso::tc;
    if (!X || !shift || !rotation || !Z || N < 1 || D < 1 || D > 8192 || N > (1 << 24)) {
        set_last_error("psso_rotate: need X, shift, rotation, Z, 1 <= N <= 2^24, 1 <= D <= 8192");
        return PSSO_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int Np = (int)((N + BM - 1) / BM * BM), Jp = (int)((D + BN - 1) / BN * BN),
              Kp = (int)((D + BK - 1) / BK * BK);
    __nv_bfloat16 *A = nullptr, *B = nullptr;
    float* mn = nullptr;
    int* status = nullptr;
    auto cleanup = [&] {
        cudaFree(A);
        cudaFree(B);
        cudaFree(mn);
        cudaFree(status);
    };
    if (cudaMalloc(&A, (size_t)3 * Np * Kp * 2) != cudaSuccess || cudaMalloc(&B, (size_t)3 * Jp * Kp * 2) != cudaSuccess ||
        cudaMalloc(&mn, (size_t)Jp * 4) != cudaSuccess || cudaMalloc(&status, 4) != cudaSuccess) {
        cleanup();
        set_last_error("psso_rotate: device allocation failed");
        return PSSO_ERR_OOM;
    }
    CUtensorMap ta, tb;
    if (!make_tmap_bf16(&ta, A, Kp, 3 * Np) || !make_tmap_bf16(&tb, B, Kp, 3 * Jp)) {
        cleanup();
        set_last_error("psso_rotate: cuTensorMapEncodeTiled failed");
        return PSSO_ERR_CUDA;
    }
    cudaMemsetAsync(status, 0, 4, s);
    split_matrix<<<Jp, 256, 0, s>>>(rotation, (int)D, Jp, Kp, B, mn);
    split_rows<<<(Np + 7) / 8, 256, 0, s>>>(X, shift, (int)N, (int)D, Np, Kp, A);
    cudaFuncSetAttribute(rotate_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    GemmArgs ga{Np, Jp, Kp, status};
    rotate_gemm<<<dim3(Np / BM, Jp / BN), 128, SMEM_BYTES, s>>>(ta, tb, ga, ZEpi{Z, (int)N, (int)D});
    cudaError_t e = cudaGetLastError();
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "psso_rotate: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return PSSO_ERR_CUDA;
    }
    if (st) {
        set_last_error("psso_rotate: a tensor-core pipeline wait ran out");
        return PSSO_ERR_TIMEOUT;
    }
    return PSSO_OK;
}
