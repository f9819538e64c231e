// gen_f64_lat32.cu -- instantiation of the persistent generation kernel: positions
// in float, FP64 fitness.
#include "sso_kernel.cuh"

namespace psso {

cudaError_t launch_gen_f64_lat32(const KParams& p, int grid, int block, size_t smem, cudaStream_t s)
{
    return launch_generations<float, false>(p, grid, block, smem, s);
}

cudaError_t occupancy_gen_f64_lat32(int block, size_t smem, int* n)
{
    return occupancy_generations<float, false>(block, smem, n);
}

cudaError_t smem_gen_f64_lat32(size_t smem) { return smem_generations<float, false>(smem); }

}  // namespace psso
