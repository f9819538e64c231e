// microbench.cu -- measured pipe and latency peaks of this GPU
// (psso_microbench), the denominators of the generation kernels' rooflines.
//
// Each throughput kernel runs independent dependency chains of one operation
// on every SM (8 blocks of 256 threads per SM, 8 chains per thread, so that
// the pipe, not the chain latency, sets the rate) and is timed with CUDA
// events on the caller's stream after one warm-up launch.  The latency
// kernels are cooperative launches (every block resident), and every wait in
// them has an iteration limit after which the kernel records a failure and
// returns; the entry point then reports PSSO_ERR_TIMEOUT.
#include <cstdint>
#include <cstring>

#include "psso.h"
#include "psso_internal.h"
#include "devmath.cuh"

namespace psso {
namespace mb {

constexpr int CHAINS = 8;
constexpr int TPB = 256;

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---- throughput ------------------------------------------------------------
__global__ void __launch_bounds__(TPB) fp32_fma(int iters, float* sink, unsigned long long* clk)
{
    float a[CHAINS];
    const float b = 0.999999f, c = 1e-7f * (float)(threadIdx.x & 7);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
    const unsigned long long c0 = clock64(), t0 = globaltimer_ns();
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __fmaf_rn(a[k], b, c);
    const unsigned long long c1 = clock64(), t1 = globaltimer_ns();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 12345.f) sink[0] = s;             // never true: keeps the chains alive
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
}

__global__ void __launch_bounds__(TPB) fp64_fma(int iters, double* sink)
{
    double a[CHAINS];
    const double b = 0.999999, c = 1e-7 * (double)(threadIdx.x & 7);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __fma_rn(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == 12345.0) sink[0] = s;
}

// 32-bit multiply-add (the low half), x <- x * m + c
__global__ void __launch_bounds__(TPB) int_imad(int iters, unsigned* sink)
{
    unsigned a[CHAINS];
    const unsigned m = 0x9E3779B1u, c = threadIdx.x;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = threadIdx.x * 7u + k;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = a[k] * m + c;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s ^= a[k];
    if (s == 0x12345u) sink[0] = s;
}

// the high half of a 32 x 32 product, x <- umulhi(x, m) ^ c (two operations)
__global__ void __launch_bounds__(TPB) int_mulhi(int iters, unsigned* sink)
{
    unsigned a[CHAINS];
    const unsigned m = 0xD2511F53u, c = 0x9E3779B9u + threadIdx.x;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = threadIdx.x * 13u + k + 1u;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = __umulhi(a[k], m) ^ c;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s ^= a[k];
    if (s == 0x12345u) sink[0] = s;
}

// Philox-4x32-10 blocks, the draws of the stepwise update (80 counted
// operations each: per round two 32 x 32 -> 64 products, four xors, two key
// additions)
__global__ void __launch_bounds__(TPB) philox_blocks(int iters, unsigned* sink)
{
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint4 w = philox10(make_uint4((unsigned)(it * 2 + k), tid, 7u, 2u), 0x1234567u, 0x89abcdefu);
            acc ^= w.x ^ w.y ^ w.z ^ w.w;
        }
    }
    if (acc == 0x12345u) sink[0] = acc;
}

// ---- latency -----------------------------------------------------------------
__device__ __forceinline__ unsigned ldv(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void stv(unsigned* p, unsigned v)
{
    asm volatile("st.volatile.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Ping-pong between block 0 and the last block (different SMs): block 0
// stores k to ping, the other polls it and stores k to pong, block 0 polls
// pong.  One round trip = two store -> polled-load hand-offs through L2.
__global__ void l2_pingpong(int rounds, unsigned* words, int64_t limit, int* fail)
{
    if (threadIdx.x != 0) return;
    unsigned* ping = words;
    unsigned* pong = words + 32;   // another 128-byte line
    const bool leader = blockIdx.x == 0;
    if (!leader && blockIdx.x != gridDim.x - 1) return;
    for (int k = 1; k <= rounds; ++k) {
        if (leader) {
            stv(ping, (unsigned)k);
            int64_t it = 0;
            while (ldv(pong) != (unsigned)k)
                if (++it > limit) { atomicExch(fail, 1); return; }
        } else {
            int64_t it = 0;
            while (ldv(ping) != (unsigned)k)
                if (++it > limit || (((it & 63) == 0) && ldv(reinterpret_cast<unsigned*>(fail)))) {
                    atomicExch(fail, 1);
                    return;
                }
            stv(pong, (unsigned)k);
        }
    }
}

// Grid-wide barrier of one block per SM (arrival counter + generation word,
// the barrier the asynchronous flow uses), `rounds` times.
__global__ void grid_barriers(int rounds, unsigned* words, int64_t limit, int* fail)
{
    unsigned* count = words;
    unsigned* gen = words + 32;
    for (int k = 0; k < rounds; ++k) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned g = ldv(gen);
            __threadfence();
            if (atomicAdd(count, 1u) == gridDim.x - 1) {
                *count = 0;
                __threadfence();
                atomicAdd(gen, 1u);
            } else {
                int64_t it = 0;
                while (ldv(gen) == g)
                    if (++it > limit || ldv(reinterpret_cast<unsigned*>(fail))) { atomicExch(fail, 1); break; }
            }
            __threadfence();
        }
        __syncthreads();
        if (ldv(reinterpret_cast<unsigned*>(fail))) return;
    }
}

// Hardware cluster barrier (arrive + wait) of a cluster of CTAs, `rounds` times.
__global__ void cluster_barriers(int rounds, unsigned* sink)
{
    unsigned v = 0;
    for (int k = 0; k < rounds; ++k) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        v += k;
    }
    if (v == 0x12345u && threadIdx.x == 0) sink[0] = v;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st)
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, s); }
    float stop()
    {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
};

cudaError_t coop(const void* fn, int grid, int block, void** args, cudaStream_t s)
{
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3((unsigned)block), args, 0, s);
}

}  // namespace mb
}  // namespace psso

extern "C" psso_status psso_microbench(psso_peaks* out, void* stream)
{
    using namespace psso;
    using namespace psso::mb;
    if (!out) {
        set_last_error("psso_microbench: out is NULL");
        return PSSO_ERR_ARG;
    }
    std::memset(out, 0, sizeof *out);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("psso_microbench: no CUDA device");
        return PSSO_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* mem = nullptr;
    if (cudaMalloc(&mem, 4096) != cudaSuccess) {
        set_last_error("psso_microbench: cudaMalloc failed");
        return PSSO_ERR_OOM;
    }
    char* m = static_cast<char*>(mem);
    auto* sink = reinterpret_cast<unsigned*>(m);
    auto* fsink = reinterpret_cast<float*>(m + 64);
    auto* dsink = reinterpret_cast<double*>(m + 128);
    auto* clk = reinterpret_cast<unsigned long long*>(m + 192);
    auto* words = reinterpret_cast<unsigned*>(m + 1024);
    auto* fail = reinterpret_cast<int*>(m + 3072);
    psso_status rc = PSSO_OK;
    do {
        if (cudaMemsetAsync(mem, 0, 4096, s) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        Timer t(s);
        const int grid = sms * 8;
        const double threads = (double)grid * TPB;
        // FP32 FMA (and the SM clock from clock64 against the global timer)
        const int it32 = 512;
        fp32_fma<<<grid, TPB, 0, s>>>(it32, fsink, clk);
        t.start();
        fp32_fma<<<grid, TPB, 0, s>>>(it32, fsink, clk);
        float ms = t.stop();
        out->fp32_fma_per_s = threads * it32 * CHAINS / (ms * 1e-3);
        unsigned long long hc[2] = {0, 0};
        if (cudaMemcpy(hc, clk, sizeof hc, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        out->sm_clock_mhz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;
        // FP64 FMA
        const int it64 = 32;
        fp64_fma<<<grid, TPB, 0, s>>>(it64, dsink);
        t.start();
        fp64_fma<<<grid, TPB, 0, s>>>(it64, dsink);
        ms = t.stop();
        out->fp64_fma_per_s = threads * it64 * CHAINS / (ms * 1e-3);
        // IMAD, IMAD.HI
        const int iti = 256;
        int_imad<<<grid, TPB, 0, s>>>(iti, sink);
        t.start();
        int_imad<<<grid, TPB, 0, s>>>(iti, sink);
        ms = t.stop();
        out->int_mad_per_s = threads * iti * CHAINS / (ms * 1e-3);
        int_mulhi<<<grid, TPB, 0, s>>>(iti, sink);
        t.start();
        int_mulhi<<<grid, TPB, 0, s>>>(iti, sink);
        ms = t.stop();
        out->int_mulhi_xor_per_s = threads * iti * CHAINS / (ms * 1e-3);
        // Philox-4x32-10 blocks
        const int itp = 2048;
        philox_blocks<<<grid, TPB, 0, s>>>(itp, sink);
        t.start();
        philox_blocks<<<grid, TPB, 0, s>>>(itp, sink);
        ms = t.stop();
        out->philox_blocks_per_s = threads * itp * 2 / (ms * 1e-3);
        if (cudaGetLastError() != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        // store -> polled load through L2 between two SMs (one-way = round trip / 2)
        int rounds = 2000;
        int64_t limit = 20000000;
        void* a1[] = {&rounds, &words, &limit, &fail};
        if (coop((const void*)l2_pingpong, sms, 32, a1, s) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        cudaStreamSynchronize(s);
        t.start();
        coop((const void*)l2_pingpong, sms, 32, a1, s);
        ms = t.stop();
        out->l2_handoff_ns = (double)ms * 1e6 / (2.0 * rounds);
        // grid barrier over one block per SM
        if (cudaMemsetAsync(words, 0, 1024, s) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        int brounds = 2000;
        void* a2[] = {&brounds, &words, &limit, &fail};
        if (coop((const void*)grid_barriers, sms, 128, a2, s) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        cudaStreamSynchronize(s);
        t.start();
        coop((const void*)grid_barriers, sms, 128, a2, s);
        ms = t.stop();
        out->grid_barrier_ns = (double)ms * 1e6 / brounds;
        // hardware cluster barrier, clusters of 8 CTAs (portable size) over the GPU
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(sms / 8 * 8));
        lc.blockDim = dim3(128);
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 8;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int crounds = 20000;
        if (cudaLaunchKernelEx(&lc, cluster_barriers, crounds, sink) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        t.start();
        cudaLaunchKernelEx(&lc, cluster_barriers, crounds, sink);
        ms = t.stop();
        out->cluster_barrier_ns = (double)ms * 1e6 / crounds;
        int hf = 0;
        if (cudaMemcpy(&hf, fail, sizeof hf, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        if (hf) {
            set_last_error("psso_microbench: a latency kernel's wait ran past its limit");
            rc = PSSO_ERR_TIMEOUT;
            break;
        }
        if (cudaGetLastError() != cudaSuccess) { rc = PSSO_ERR_CUDA; break; }
        out->sms = sms;
    } while (0);
    if (rc == PSSO_ERR_CUDA) set_last_error("psso_microbench: a CUDA call failed");
    cudaFree(mem);
    return rc;
}
