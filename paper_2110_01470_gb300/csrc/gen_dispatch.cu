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

// ---------------------------------------------------------------------------
// Batched throughput pipeline.
using BatFn = cudaError_t (*)(int, const BatParams*, int, int, cudaStream_t, int*);
#define PSSO_BDECL(v, m) \
    cudaError_t bat_variant_##v##_##m(int, const BatParams*, int, int, cudaStream_t, int*);
PSSO_BDECL(0, 1) PSSO_BDECL(0, 2) PSSO_BDECL(0, 4) PSSO_BDECL(0, 8)
PSSO_BDECL(1, 1) PSSO_BDECL(1, 2) PSSO_BDECL(1, 4) PSSO_BDECL(1, 8)
PSSO_BDECL(2, 1) PSSO_BDECL(2, 2) PSSO_BDECL(2, 4) PSSO_BDECL(2, 8)
#undef PSSO_BDECL

cudaError_t bat_call(int variant, int mc_index, int op, const BatParams* p, int grid, int block, cudaStream_t s,
                     int* out)
{
    static const BatFn table[3][4] = {
        {bat_variant_0_1, bat_variant_0_2, bat_variant_0_4, bat_variant_0_8},
        {bat_variant_1_1, bat_variant_1_2, bat_variant_1_4, bat_variant_1_8},
        {bat_variant_2_1, bat_variant_2_2, bat_variant_2_4, bat_variant_2_8}};
    if (variant < 0 || variant > 2 || mc_index < 0 || mc_index > 3) return cudaErrorInvalidValue;
    return table[variant][mc_index](op, p, grid, block, s, out);
}

// gBest of one instance per block: the lowest-index arg-min of the pBests
// (FP32 mode: certain from the bounds, else the pBests that may be the
// minimum made exact in FP64 and the exact arg-min taken), then the record,
// log and gBest row.
template <class Pos, bool F32R>
__global__ void __launch_bounds__(256) bat_argmin(const InstDev* inst, const int32_t* ids, const long long* gen,
                                                  BatCounters* cnt)
{
    __shared__ Cand sh[32];
    __shared__ unsigned long long extra;
    const int k = ids[blockIdx.x];
    const InstDev& d = inst[k];
    const int64_t g = *gen;
    const int64_t N = d.N;
    if (threadIdx.x == 0) extra = 0;
    Cand c = cand_none();
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
        c = cand_merge<F32R>(c, cand_of<F32R>((long long)i, d.pf64[i], F32R ? d.plo[i] : 0.f,
                                              F32R ? d.phi[i] : 0.f, F32R ? (int)(d.pflag[i] & 1u) : 1,
                                              d.pver[i]));
    Cand b = block_reduce_cand<F32R>(c, sh);
    if (F32R && b.l2 <= b.mh) {
        const Hot hin = hot_of(d);
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int64_t i = threadIdx.x >> 5; i < N; i += nw) {
            if (!(d.plo[i] <= b.mh && !(d.pflag[i] & 1u))) continue;   // uniform over the warp
            const double f = fit64_row<Pos>(hin, static_cast<const Pos*>(d.P) + i * d.Dp, false);
            if (lane == 0) {
                d.pf64[i] = f;
                d.pflag[i] = 1u;
                d.plo[i] = f64_to_f32_rd(f);
                d.phi[i] = f64_to_f32_ru(f);
                atomicAdd(&extra, 1ull);
            }
        }
        __syncthreads();
        // every pBest that can be the minimum has its FP64 value now
        Cand e = cand_none();
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
            if (d.pflag[i] & 1u) {
                Cand q = cand_none();
                q.v = d.pf64[i];
                q.i = (long long)i;
                q.ver = d.pver[i];
                e = cand_merge<false>(e, q);
            }
        b = block_reduce_cand<false>(e, sh);
        b.has1 = 1;
        b.l1 = f64_to_f32_rd(b.v);
        b.h1 = f64_to_f32_ru(b.v);
    }
    const Pos* src = static_cast<const Pos*>(d.P) + b.i * d.Dp;
    Pos* dst = static_cast<Pos*>(d.gbrow);
    for (int j = threadIdx.x; j < d.Dp; j += blockDim.x) dst[j] = src[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        Winner w;
        w.idx = b.i;
        w.ver = b.ver;
        w.acc = cnt[k].acc;
        w.rck = cnt[k].rck + extra;
        if (!F32R) {
            w.has64 = 1;
            w.f64 = b.v;
            w.lo = f64_to_f32_rd(b.v);
            w.hi = f64_to_f32_ru(b.v);
        } else {
            w.has64 = b.has1;
            w.f64 = b.has1 ? b.v : 0.0;
            w.lo = b.l1;
            w.hi = b.h1;
        }
        write_gbest(d, w, g);
        cnt[k].acc = 0;
        cnt[k].rck = 0;
    }
}

__global__ void bat_next(long long* gen) { *gen += 1; }
__global__ void bat_set(long long* gen, long long g) { *gen = g; }

cudaError_t launch_bat_argmin(int variant, const InstDev* inst, const int32_t* ids, int n_ids, long long* gen,
                              BatCounters* cnt, cudaStream_t s)
{
    if (variant == 0) bat_argmin<double, false><<<n_ids, 256, 0, s>>>(inst, ids, gen, cnt);
    else if (variant == 1) bat_argmin<float, false><<<n_ids, 256, 0, s>>>(inst, ids, gen, cnt);
    else bat_argmin<float, true><<<n_ids, 256, 0, s>>>(inst, ids, gen, cnt);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bat_next<<<1, 1, 0, s>>>(gen);
    return cudaGetLastError();
}

cudaError_t launch_bat_set_gen(long long* gen, long long g, cudaStream_t s)
{
    bat_set<<<1, 1, 0, s>>>(gen, g);
    return cudaGetLastError();
}

cudaError_t launch_best_f64(const InstDev* inst, int n_inst, int lattice, cudaStream_t s)
{
    if (lattice == 1) best_f64_kernel<float><<<n_inst, 32, 0, s>>>(inst, n_inst);
    else best_f64_kernel<double><<<n_inst, 32, 0, s>>>(inst, n_inst);
    return cudaGetLastError();
}

}  // namespace psso
