// evaluate_noalloc.cu -- batched fitness for callers that must not allocate
// device memory (psso_evaluate_noalloc).
//
// psso_evaluate stages the caller's rows and the padded shift / weight vectors
// in device buffers it allocates for the call.  This variant takes device
// pointers for the rows and the results and keeps its only scratch -- the
// padded shift and weight vectors in FP64 and FP32 -- in one file-scope device
// array of fixed size, so a call performs no allocation at all.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call rewrites the part it reads (padding included) before the
// evaluation kernel runs.  Calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on the array.
#include <mutex>

#include "psso.h"
#include "sso_kernel.cuh"

namespace psso {
namespace {

constexpr int NOALLOC_MAX_D = 1024;   // largest D this entry point accepts

// Layout of the scratch array: padded shift and weights in FP64, then in FP32.
struct NoAllocScratch {
    double o64[NOALLOC_MAX_D];
    double w64[NOALLOC_MAX_D];
    float o32[NOALLOC_MAX_D];
    float w32[NOALLOC_MAX_D];
};
constexpr size_t SCRATCH_BYTES = sizeof(NoAllocScratch);   // 24 KiB

}  // namespace

// The scratch array (24 KiB, held by every GPU that loads the library until
// the process exits).  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up once per
// device, on the first call made with that device current).
psso_status scratch_on_current_device(NoAllocScratch** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        set_last_error("psso_evaluate_noalloc: no usable current CUDA device");
        return PSSO_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error("psso_evaluate_noalloc: cudaGetSymbolAddress of the scratch array failed");
            return PSSO_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_addr[dev];
    return PSSO_OK;
}

// Fills the padded shift / weight vectors (zeros beyond D); hyper: the
// weights of the hyper-ellipsoid, w_j = j + 1.
__global__ void fill_scratch(NoAllocScratch* s, const double* shift, const double* weights, int D, int Dp,
                             bool hyper)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Dp; j += gridDim.x * blockDim.x) {
        const double o = (j < D && shift) ? shift[j] : 0.0;
        const double w = j >= D ? 0.0 : hyper ? (double)(j + 1) : weights ? weights[j] : 0.0;
        s->o64[j] = o;
        s->o32[j] = (float)o;
        s->w64[j] = w;
        s->w32[j] = (float)w;
    }
}

// One warp per row of X (N x D doubles, unpadded): the same fitness routines
// and the same 32-lane chunk layout as psso_evaluate.
template <bool F32, int MAXC>
__device__ void eval_row(const Hot& in, const double* xr, double* f, double* err)
{
    const int lane = threadIdx.x & 31;
    bool exact = true;
    if constexpr (F32) {
        float x[MAXC][4];
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * (lane + 32 * q) + m;
                const double d = j < in.D ? xr[j] : 0.0;
                x[q][m] = (float)d;
                exact = exact && ((double)x[q][m] == d);
                // the FP32 terms use the shift rounded to float; the bound holds for
                // the FP64 value only when that rounding is exact
                if (j < in.D) exact = exact && ((double)in.o32[j] == in.o64[j]);
            }
        const Fit32 r = fit32<MAXC>(in, x, lane, 0xffffffffu, 32);
        exact = __all_sync(0xffffffffu, exact);
        if (lane == 0) {
            *f = exact ? (double)r.f : __longlong_as_double(0x7ff8000000000000LL);
            if (err) *err = exact ? (double)r.E : __longlong_as_double(0x7ff8000000000000LL);
        }
    } else {
        double x[MAXC][4];
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * (lane + 32 * q) + m;
                x[q][m] = j < in.D ? xr[j] : 0.0;
            }
        const double v = fit64<double, MAXC>(in, x, lane, 0xffffffffu, 32);
        if (lane == 0) {
            *f = v;
            if (err) *err = 0.0;
        }
    }
}

template <bool F32>
__global__ void eval_noalloc(const Hot in, const double* X, int64_t N, double* f, double* err)
{
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= N) return;
    if (!PSSO_CHK(in.maxc * 128 >= in.D, CHK_EVAL_ROW, in.D)) return;
    const double* xr = X + row * in.D;
    double* e = err ? err + row : nullptr;
    switch (in.maxc) {
    case 1: eval_row<F32, 1>(in, xr, f + row, e); break;
    case 2: eval_row<F32, 2>(in, xr, f + row, e); break;
    case 4: eval_row<F32, 4>(in, xr, f + row, e); break;
    default: eval_row<F32, 8>(in, xr, f + row, e); break;
    }
}

}  // namespace
}  // namespace psso

extern "C" psso_status psso_evaluate_noalloc(psso_fn fn, int64_t N, int64_t D, const double* X,
                                             const double* shift, const double* weights,
                                             int32_t precision, double* f, double* err, void* stream)
{
    using namespace psso;
    if (!X || !f || N < 1 || fn < PSSO_SPHERE || fn > PSSO_SCHWEFEL) {
        set_last_error("psso_evaluate_noalloc: need X, f, N >= 1 and a known function");
        return PSSO_ERR_ARG;
    }
    if (D < 1 || D > NOALLOC_MAX_D) {
        set_last_error("psso_evaluate_noalloc: D must be in [1, 1024] (size of the static scratch)");
        return PSSO_ERR_ARG;
    }
    // one warp per row, 8 rows per block: the grid's x extent must stay below 2^31
    if (N > (int64_t)8 * 0x7fffffff) {
        set_last_error("psso_evaluate_noalloc: N above 8 * (2^31 - 1) rows");
        return PSSO_ERR_ARG;
    }
    if (fn >= PSSO_ROT_ELLIPSOID && fn <= PSSO_ROT_ACKLEY) {
        set_last_error("psso_evaluate_noalloc: rotated functions are not available through this entry point");
        return PSSO_ERR_UNSUPPORTED;
    }
    if (precision == PSSO_PREC_F32_RECHECK && fn >= PSSO_SCHWEFEL12) {
        set_last_error("psso_evaluate_noalloc: this function has FP64 fitness only");
        return PSSO_ERR_UNSUPPORTED;
    }
    const bool hyper = fn == PSSO_HYPER_ELLIPSOID;   // the ellipsoid with w_j = j + 1
    if (hyper) fn = PSSO_ELLIPSOID;
    if (fn == PSSO_ELLIPSOID && !weights && !hyper) {
        set_last_error("psso_evaluate_noalloc: the ellipsoid needs weights");
        return PSSO_ERR_ARG;
    }
    if (precision != PSSO_PREC_F64 && precision != PSSO_PREC_F32_RECHECK) {
        set_last_error("psso_evaluate_noalloc: unknown precision");
        return PSSO_ERR_ARG;
    }
    NoAllocScratch* s = nullptr;
    const psso_status st = scratch_on_current_device(&s);
    if (st != PSSO_OK) return st;

    const int nchunks = (int)((D + 3) / 4), Dp = 4 * nchunks;
    int maxc = 1;
    while (maxc < (nchunks + 31) / 32) maxc <<= 1;
    Hot in{};
    in.fn = fn;
    in.D = (int)D;
    in.Dp = Dp;
    in.nchunks = nchunks;
    in.G = 32;
    in.maxc = maxc;
    in.o64 = s->o64;
    in.o32 = s->o32;
    in.w64 = (weights || hyper) ? s->w64 : nullptr;
    in.w32 = (weights || hyper) ? s->w32 : nullptr;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // clear an earlier, unrelated launch error so that only this call's launches are reported
    (void)cudaGetLastError();
    fill_scratch<<<(Dp + 255) / 256, 256, 0, cs>>>(s, shift, weights, (int)D, Dp, hyper);
    const int wpb = 8;
    const unsigned grid = (unsigned)((N + wpb - 1) / wpb);
    if (precision == PSSO_PREC_F32_RECHECK) eval_noalloc<true><<<grid, 32 * wpb, 0, cs>>>(in, X, N, f, err);
    else eval_noalloc<false><<<grid, 32 * wpb, 0, cs>>>(in, X, N, f, err);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error("psso_evaluate_noalloc: kernel launch failed");
        return PSSO_ERR_CUDA;
    }
    return PSSO_OK;
}
