// gen_f64_lat32.cu -- instantiation of the persistent generation kernel: positions
// in float, FP64 fitness.
#include "sso_kernel.cuh"

namespace psso {

cudaError_t gen_f64_lat32(int op, int mc_index, const KParams* p, int grid, int block, size_t smem,
                     cudaStream_t s, int* out)
{
    return gen_entry<float, false>(op, mc_index, p, grid, block, smem, s, out);
}

}  // namespace psso
