// gen_dispatch.cu -- variant dispatch for occupancy / shared-memory queries and
// the on-demand FP64 evaluation of gBest rows.
#include "sso_kernel.cuh"

namespace psso {

cudaError_t gen_f64_lat64(int, int, const KParams*, int, int, size_t, cudaStream_t, int*);
cudaError_t gen_f64_lat32(int, int, const KParams*, int, int, size_t, cudaStream_t, int*);
cudaError_t gen_f32r(int, int, const KParams*, int, int, size_t, cudaStream_t, int*);

cudaError_t gen_call(int variant, int op, int mc_index, const KParams* p, int grid, int block,
                     size_t smem, cudaStream_t s, int* out)
{
    switch (variant) {
    case 0: return gen_f64_lat64(op, mc_index, p, grid, block, smem, s, out);
    case 1: return gen_f64_lat32(op, mc_index, p, grid, block, smem, s, out);
    default: return gen_f32r(op, mc_index, p, grid, block, smem, s, out);
    }
}

cudaError_t launch_best_f64(const InstDev* inst, int n_inst, int lattice, cudaStream_t s)
{
    if (lattice == 1) best_f64_kernel<float><<<n_inst, 32, 0, s>>>(inst, n_inst);
    else best_f64_kernel<double><<<n_inst, 32, 0, s>>>(inst, n_inst);
    return cudaGetLastError();
}

}  // namespace psso
