// gen_f32r.cu -- instantiation of the persistent generation kernel: positions
// in float, FP32 fitness with FP64 recheck.
#include "sso_kernel.cuh"

namespace psso {

cudaError_t gen_f32r(int op, int mc_index, const KParams* p, int grid, int block, size_t smem,
                     cudaStream_t s, int* out)
{
    return gen_entry<float, true>(op, mc_index, p, grid, block, smem, s, out);
}

#ifdef PSSO_TRACE
extern "C" int psso_trace_dump(void* host, size_t bytes)
{
    return (int)cudaMemcpyFromSymbol(host, trace_buf, bytes);
}
#endif

}  // namespace psso
