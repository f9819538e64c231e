// gen_f32r.cu -- instantiation of the persistent generation kernel: positions
// in float, FP32 fitness with FP64 recheck.
#include "sso_kernel.cuh"

namespace psso {

cudaError_t launch_gen_f32r(const KParams& p, int grid, int block, size_t smem, cudaStream_t s)
{
    return launch_generations<float, true>(p, grid, block, smem, s);
}

cudaError_t occupancy_gen_f32r(int block, size_t smem, int* n)
{
    return occupancy_generations<float, true>(block, smem, n);
}

cudaError_t smem_gen_f32r(size_t smem) { return smem_generations<float, true>(smem); }

}  // namespace psso
