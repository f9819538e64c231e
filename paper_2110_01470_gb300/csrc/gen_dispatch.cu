// gen_dispatch.cu -- variant dispatch for occupancy / shared-memory queries and
// the on-demand FP64 evaluation of gBest rows.
#include "sso_kernel.cuh"

namespace psso {

// One entry per (variant, width), each in its own object built from gen_variant.cu.
using GenFn = cudaError_t (*)(int, const KParams*, int, int, size_t, cudaStream_t, int*);
#define PSSO_DECL(v, m) \
    cudaError_t gen_variant_##v##_##m(int, const KParams*, int, int, size_t, cudaStream_t, int*);
PSSO_DECL(0, 1) PSSO_DECL(0, 2) PSSO_DECL(0, 4) PSSO_DECL(0, 8)
PSSO_DECL(1, 1) PSSO_DECL(1, 2) PSSO_DECL(1, 4) PSSO_DECL(1, 8)
PSSO_DECL(2, 1) PSSO_DECL(2, 2) PSSO_DECL(2, 4) PSSO_DECL(2, 8)
#undef PSSO_DECL

cudaError_t gen_call(int variant, int op, int mc_index, const KParams* p, int grid, int block,
                     size_t smem, cudaStream_t s, int* out)
{
    static const GenFn table[3][4] = {
        {gen_variant_0_1, gen_variant_0_2, gen_variant_0_4, gen_variant_0_8},
        {gen_variant_1_1, gen_variant_1_2, gen_variant_1_4, gen_variant_1_8},
        {gen_variant_2_1, gen_variant_2_2, gen_variant_2_4, gen_variant_2_8}};
    if (variant < 0 || variant > 2 || mc_index < 0 || mc_index > 3) return cudaErrorInvalidValue;
    return table[variant][mc_index](op, p, grid, block, smem, s, out);
}

cudaError_t launch_best_f64(const InstDev* inst, int n_inst, int lattice, cudaStream_t s)
{
    if (lattice == 1) best_f64_kernel<float><<<n_inst, 32, 0, s>>>(inst, n_inst);
    else best_f64_kernel<double><<<n_inst, 32, 0, s>>>(inst, n_inst);
    return cudaGetLastError();
}

}  // namespace psso
