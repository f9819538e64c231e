// evaluate.cu -- batched fitness of caller-given rows (psso_evaluate): one warp
// per row, 32-lane chunk layout, FP64 in the fixed oracle order or FP32 with
// its rigorous error bound.
#include <cmath>
#include <string>
#include <vector>

#include "psso.h"
#include "sso_kernel.cuh"

namespace psso {

template <int MAXC>
__device__ Fit32 fit32_row_warp(const Hot& in, const float* row)
{
    const int lane = threadIdx.x & 31;
    float x[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
        if (c < in.nchunks) ld4(row + 4 * c, x[q]);
        else { x[q][0] = x[q][1] = x[q][2] = x[q][3] = 0.f; }
    }
    return fit32<MAXC>(in, x, lane, 0xffffffffu, 32);
}

template <bool F32>
__global__ void evaluate_rows(const InstDev in, const void* X, int64_t N, double* f, double* err)
{
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= N) return;
    if (!PSSO_CHK(in.maxc * 128 >= in.D, CHK_EVAL_ROW, in.D)) return;
    const Hot h = hot_of(in);
    if constexpr (F32) {
        const float* r = static_cast<const float*>(X) + row * in.Dp;
        Fit32 v;
        switch (in.maxc) {
        case 1: v = fit32_row_warp<1>(h, r); break;
        case 2: v = fit32_row_warp<2>(h, r); break;
        case 4: v = fit32_row_warp<4>(h, r); break;
        default: v = fit32_row_warp<8>(h, r); break;
        }
        if ((threadIdx.x & 31) == 0) {
            f[row] = (double)v.f;
            if (err) err[row] = (double)v.E;
        }
    } else {
        const double* r = static_cast<const double*>(X) + row * in.Dp;
        const double v = fit64_row<double>(h, r, false);
        if ((threadIdx.x & 31) == 0) {
            f[row] = v;
            if (err) err[row] = 0.0;
        }
    }
}

}  // namespace psso

extern "C" psso_status psso_evaluate(psso_fn fn, int64_t N, int64_t D, const double* X,
                                     const double* shift, const double* weights,
                                     const double* rotation, int32_t precision, double* f,
                                     double* err, void* stream)
{
    using namespace psso;
    auto bad = [](psso_status st, const char* msg) {
        set_last_error(msg);
        return st;
    };
    if (!X || !f || N < 1 || D < 1 || D > 1024 || fn < PSSO_SPHERE || fn > PSSO_SCHWEFEL)
        return bad(PSSO_ERR_ARG, "psso_evaluate: need X, f, N >= 1, 1 <= D <= 1024, a known function");
    const bool rot = fn >= PSSO_ROT_ELLIPSOID && fn <= PSSO_ROT_ACKLEY;
    if (rot && !rotation)
        return bad(PSSO_ERR_ARG, "psso_evaluate: rotated functions need a rotation matrix");
    if ((fn == PSSO_ELLIPSOID || fn == PSSO_ROT_ELLIPSOID) && !weights)
        return bad(PSSO_ERR_ARG, "psso_evaluate: ellipsoid needs weights");
    if (precision != PSSO_PREC_F64 && precision != PSSO_PREC_F32_RECHECK)
        return bad(PSSO_ERR_ARG, "psso_evaluate: unknown precision");
    const bool f32 = precision == PSSO_PREC_F32_RECHECK;
    if (f32 && fn >= PSSO_SCHWEFEL12)
        return bad(PSSO_ERR_UNSUPPORTED, "psso_evaluate: this function has FP64 fitness only");
    std::vector<double> hyper_w;
    if (fn == PSSO_HYPER_ELLIPSOID) {   // Table 3.2 f2: the ellipsoid with w_j = j + 1
        hyper_w.resize((size_t)D);
        for (int64_t j = 0; j < D; ++j) hyper_w[(size_t)j] = (double)(j + 1);
        weights = hyper_w.data();
        fn = PSSO_ELLIPSOID;
    }
    const int nchunks = (int)((D + 3) / 4), Dp = 4 * nchunks;
    int maxc = 1;
    while (maxc < (nchunks + 31) / 32) maxc <<= 1;
    const size_t pos = f32 ? 4 : 8;
    std::vector<char> hx((size_t)N * Dp * pos, 0);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < D; ++j) {
            const double v = X[i * D + j];
            if (f32) {
                if ((double)(float)v != v) return bad(PSSO_ERR_ARG, "psso_evaluate: FP32 needs float-exact X");
                reinterpret_cast<float*>(hx.data())[i * Dp + j] = (float)v;
            } else {
                reinterpret_cast<double*>(hx.data())[i * Dp + j] = v;
            }
        }
    std::vector<double> o64(Dp, 0.0), w64(Dp, 0.0);
    std::vector<float> o32(Dp, 0.f), w32(Dp, 0.f);
    for (int64_t j = 0; j < D; ++j) {
        o64[j] = shift ? shift[j] : 0.0;
        if (f32 && (double)(float)o64[j] != o64[j])
            return bad(PSSO_ERR_ARG, "psso_evaluate: FP32 needs a float-exact shift");
        o32[j] = (float)o64[j];
        w64[j] = weights ? weights[j] : 0.0;
        w32[j] = (float)w64[j];
    }
    const size_t nM = rot ? (size_t)D * D : 0;
    std::vector<float> M32(2 * nM);   // float(M), then float(M - float(M))
    for (size_t q = 0; q < nM; ++q) {
        M32[q] = (float)rotation[q];
        M32[nM + q] = (float)(rotation[q] - (double)M32[q]);
    }
    char* dev = nullptr;
    const size_t nx = hx.size(), no = (size_t)Dp * 24, nf = (size_t)N * 16;
    const size_t mbytes = ((nM * 16 + 255) / 256) * 256;
    if (cudaMalloc(&dev, nx + 2 * no + nf + 1024 + mbytes) != cudaSuccess)
        return bad(PSSO_ERR_OOM, "psso_evaluate: cudaMalloc failed");
    double* dM64 = reinterpret_cast<double*>(dev + nx + 2 * no + nf + 1024);
    float* dM32 = reinterpret_cast<float*>(dM64 + nM);
    char* dX = dev;
    double* do64 = reinterpret_cast<double*>(dev + ((nx + 255) / 256) * 256);
    double* dw64 = do64 + Dp;
    float* do32 = reinterpret_cast<float*>(dw64 + Dp);
    float* dw32 = do32 + Dp;
    double* df = reinterpret_cast<double*>(reinterpret_cast<char*>(dw32 + Dp) + 256 -
                                           (reinterpret_cast<uintptr_t>(dw32 + Dp) % 256));
    double* derr = df + N;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    psso_status rc = PSSO_OK;
    do {
        if (cudaMemcpyAsync(dX, hx.data(), nx, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(do64, o64.data(), Dp * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dw64, w64.data(), Dp * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(do32, o32.data(), Dp * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dw32, w32.data(), Dp * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = bad(PSSO_ERR_CUDA, "psso_evaluate: upload failed");
            break;
        }
        if (rot && (cudaMemcpyAsync(dM64, rotation, nM * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                    cudaMemcpyAsync(dM32, M32.data(), nM * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)) {
            rc = bad(PSSO_ERR_CUDA, "psso_evaluate: upload failed");
            break;
        }
        InstDev in{};
        in.fn = fn;
        in.D = (int32_t)D;
        in.Dp = Dp;
        in.nchunks = nchunks;
        in.G = 32;
        in.maxc = maxc;
        in.o64 = do64;
        in.o32 = do32;
        in.w64 = weights ? dw64 : nullptr;
        in.w32 = weights ? dw32 : nullptr;
        in.M64 = rot ? dM64 : nullptr;
        in.M32 = rot ? dM32 : nullptr;
        in.M32lo = rot ? dM32 + nM : nullptr;
        const int wpb = 8;
        const unsigned grid = (unsigned)((N + wpb - 1) / wpb);
        if (f32) evaluate_rows<true><<<grid, 32 * wpb, 0, s>>>(in, dX, N, df, derr);
        else evaluate_rows<false><<<grid, 32 * wpb, 0, s>>>(in, dX, N, df, derr);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(f, df, N * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (err && cudaMemcpyAsync(err, derr, N * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = bad(PSSO_ERR_CUDA, "psso_evaluate: kernel or download failed");
            break;
        }
    } while (0);
    cudaFree(dev);
    return rc;
}
