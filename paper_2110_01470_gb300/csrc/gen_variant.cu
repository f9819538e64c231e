// gen_variant.cu -- one instantiation of the persistent generation kernel.
// The build compiles this file once per (variant, width) pair, with
//   PSSO_VARIANT  0: positions in double, FP64 fitness
//                 1: positions in float, FP64 fitness
//                 2: positions in float, FP32 fitness with FP64 recheck
//   PSSO_MC       1, 2, 4 or 8 chunks of 4 variables per lane
// so that the twelve kernels compile in parallel.
#include "sso_kernel.cuh"
#if PSSO_MC == 8
#include "bat_stream.cuh"
#endif

#if !defined(PSSO_VARIANT) || !defined(PSSO_MC)
#error "gen_variant.cu is compiled with -DPSSO_VARIANT=v -DPSSO_MC=m"
#endif

#define PSSO_CAT3(a, b, c) a##b##_##c
#define PSSO_NAME(v, m) PSSO_CAT3(gen_variant_, v, m)

namespace psso {

#if PSSO_VARIANT == 0
using VPos = double;
constexpr bool kF32R = false;
#elif PSSO_VARIANT == 1
using VPos = float;
constexpr bool kF32R = false;
#else
using VPos = float;
constexpr bool kF32R = true;
#endif

cudaError_t PSSO_NAME(PSSO_VARIANT, PSSO_MC)(int op, const KParams* p, int grid, int block, size_t smem,
                                              cudaStream_t s, int* out)
{
    return gen_entry_mc<VPos, kF32R, PSSO_MC>(op, p, grid, block, smem, s, out);
}

#define PSSO_BNAME(v, m) PSSO_CAT3(bat_variant_, v, m)
cudaError_t PSSO_BNAME(PSSO_VARIANT, PSSO_MC)(int op, const BatParams* p, int grid, int block, cudaStream_t s,
                                               int* out)
{
#if PSSO_MC == 8
    // ops 2 / 3: the streaming kernel for wide unrotated rows (launch / occupancy)
    if (op >= 2) return bat_stream_entry<VPos, kF32R>(op, p, grid, block, s, out);
#endif
    return bat_entry_mc<VPos, kF32R, PSSO_MC>(op, p, grid, block, s, out);
}

#if defined(PSSO_TRACE) && PSSO_VARIANT == 2 && PSSO_MC == 1
extern "C" int psso_trace_dump(void* host, size_t bytes)
{
    return (int)cudaMemcpyFromSymbol(host, trace_buf, bytes);
}
#endif

}  // namespace psso
