// rot_pipeline.h -- descriptors of the tensor-core generation pipeline for
// rotated-function swarms with FP32 fitness and FP64 recheck.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "psso_internal.h"

namespace psso {
namespace rot {

// Per-instance control block in device memory.
struct RotCtl {
    long long gen;                 // generation the next kernels run
    unsigned n1, n2, n3;           // list lengths: undecided after the GEMM, arg-min
                                   // candidates, undecided after the FP32 refinement
    int amb;                       // the arg-min needs the exact pass
    int status;                    // a tensor-core pipeline wait ran out
    unsigned long long acc, rck;   // pBest updates / FP64 evaluations this generation
    unsigned long long refined;    // FP32 refinements (all generations)
    long long win_i;               // gBest of this generation
    double win_v;
    float win_lo, win_hi;
    uint32_t win_ver;
    int win_has;
};

struct RotDev {
    const InstDev* inst;
    const float* inst_w32;
    int fn, D;
    long long N;
    int Np, Jp, Kp, nJt;           // padded extents, tc::SBN-column tiles
    __nv_bfloat16* A;              // [4][Np][Kp] integer slices of d = fl32(x - o) (tc_gemm.cuh)
    float* dscale;                 // [Np] slice scale s_d of particle i (a power of two)
    float* dl1;                    // [Np] sum_k |d_ik|, rounded up
    float* mscale;                 // [Jp] slice scale s_M of output j
    float* ml1;                    // [Jp] sum_k |M32_jk|, rounded up
    uint32_t* same;                // [N] x_i equals pBest_i bit for bit
    float4* part;                  // [N][nJt] tile sums (s1, s2, e1, e2)
    int32_t* list1;                // [N] pBest updates undecided by the GEMM bounds
    int32_t* list2;                // [N] pBests that may be the minimum
    int32_t* list3;                // [N] pBest updates undecided after the refinement
    const float* Mh;               // [D][D] M = Mh + Ml (float pair, |M - Mh - Ml| <= 2^-48 |M|)
    const float* Ml;
    float* z32;                    // [2N][Dp] refined z rows of list1 particles
    float* ez32;                   // [2N][Dp] their error bounds
    double* zbuf;                  // [2N][Dp] FP64 z rows of listed particles
    const double* zero64;          // [Dp] zeros
    RotCtl* ctl;
};

struct RotHost {
    RotDev dev;
    CUtensorMap tmA, tmB;
    __nv_bfloat16* B;              // [4][Jp][Kp] integer slices of M32
    float* Mh;                     // float pair of M (refinement)
    float* Ml;
    const float* M32;
    const double* M64;
    long long N;
    int z64_grid, z32_grid, fix_grid;
    int gemm_grid;                 // persistent GEMM: min(tiles, SMs)
    void* mem;                     // the one allocation holding the buffers above
    size_t mem_bytes;
    cudaGraphExec_t graph1, graphG;  // one generation / GRAPH_GENS generations
};

constexpr int KERNELS_PER_GENERATION = 11;
constexpr int GRAPH_GENS = 16;

cudaError_t enqueue_generation(const RotHost& h, cudaStream_t s);
cudaError_t enqueue_generation_timed(const RotHost& h, cudaStream_t s, cudaEvent_t* ev);
// Captures the generation sequence into graphs of 1 and GRAPH_GENS generations.
cudaError_t make_graphs(RotHost& h);
void destroy_graphs(RotHost& h);
// Enqueues `count` generations (graph replays) on s.
cudaError_t run_generations(const RotHost& h, long long count, cudaStream_t s);
cudaError_t build_constants(const RotHost& h, cudaStream_t s);
// FP64 values of the pBests whose intervals are too wide for 1e-6 relative
// (before the state is read; enqueued on s after the generations).
cudaError_t exact_values_for_read(const RotHost& h, cudaStream_t s);
cudaError_t set_generation(const RotHost& h, long long g, cudaStream_t s);
cudaError_t configure();

}  // namespace rot

namespace tc {
cudaError_t launch_split_matrix(const float* M32, int D, int Jp, int Kp, __nv_bfloat16* B, float* mnorm,
                                cudaStream_t s);
// A planes of d = x - o for N plain rows of D floats (zero padding to Np x Kp).
cudaError_t launch_split_rows(const float* X, const float* o, int N, int D, int Np, int Kp, __nv_bfloat16* A,
                              cudaStream_t s);
}  // namespace tc
}  // namespace psso
