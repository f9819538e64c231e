// gen_dispatch.cu -- variant dispatch for occupancy / shared-memory queries and
// the on-demand FP64 evaluation of gBest rows.
#include "sso_kernel.cuh"

namespace psso {

cudaError_t occupancy_gen_f64_lat64(int block, size_t smem, int* n);
cudaError_t occupancy_gen_f64_lat32(int block, size_t smem, int* n);
cudaError_t occupancy_gen_f32r(int block, size_t smem, int* n);
cudaError_t smem_gen_f64_lat64(size_t smem);
cudaError_t smem_gen_f64_lat32(size_t smem);
cudaError_t smem_gen_f32r(size_t smem);

cudaError_t occupancy_gen(int variant, int block, size_t smem, int* blocks_per_sm)
{
    switch (variant) {
    case 0: return occupancy_gen_f64_lat64(block, smem, blocks_per_sm);
    case 1: return occupancy_gen_f64_lat32(block, smem, blocks_per_sm);
    default: return occupancy_gen_f32r(block, smem, blocks_per_sm);
    }
}

cudaError_t set_smem_gen(int variant, size_t smem)
{
    switch (variant) {
    case 0: return smem_gen_f64_lat64(smem);
    case 1: return smem_gen_f64_lat32(smem);
    default: return smem_gen_f32r(smem);
    }
}

cudaError_t launch_best_f64(const InstDev* inst, int n_inst, int lattice, cudaStream_t s)
{
    if (lattice == 1) best_f64_kernel<float><<<n_inst, 32, 0, s>>>(inst, n_inst);
    else best_f64_kernel<double><<<n_inst, 32, 0, s>>>(inst, n_inst);
    return cudaGetLastError();
}

}  // namespace psso
