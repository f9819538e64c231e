// rot_pipeline.cu -- one SSO generation of a rotated-function swarm with
// FP32 fitness and FP64 recheck, as a short sequence of kernels around the
// tensor-core rotation (z = M (x - o) for the whole swarm is one N x D x D
// GEMM, which the per-particle persistent kernel cannot share across
// particles).
//
// Generation g (the number g is read from device memory, so the sequence can
// be replayed by a CUDA graph):
//   1. rot_update    Eq. 2.1 for every variable (the same draws as the
//                    persistent kernel), X written in place, d = fl32(x - o)
//                    split into the three BF16 planes, ||d|| bound per row,
//                    "x equals pBest" flag per row.
//   2. rot_gemm_fit  the tcgen05 GEMM; its epilogue turns each z into the
//                    function's FP32 terms and per-term error bounds and
//                    writes per-(particle, 128-column tile) partial sums.
//   3. rot_decide    FP32 fitness and bound per particle; pBest update when
//                    the interval decides it (Alg. 3, <=); else the particle
//                    goes on list 1.
//   4. rot_z32       refinement of list-1 rows: z by a compensated FP32 dot
//                    product (Ogita, Rump, Oishi, "Accurate sum and dot
//                    product", SISC 2005, Algorithm Dot2), error below
//                    u |z| + 2 gamma_n^2 sum |M||d| -- some thousand times
//                    tighter than the tensor-core bound.
//   5. rot_fix32     fitness intervals from the refined z; decides the pBest
//                    update, or the particle goes on list 3.
//   6. rot_z64       FP64 z = M (x - o) of list-3 rows in the oracle's order
//                    (k ascending, fma from +0), one thread per output.
//   7. rot_fix       FP64 fitness of those rows (the oracle's summation) and
//                    the exact pBest decision.
//   8. rot_argmin(0) gBest candidates (Alg. 4, lowest index): unique from the
//                    intervals, or the pBests that can still be the minimum
//                    go on list 2.
//   9-10.            steps 6-7 for list 2 (pBest rows only).
//  11. rot_argmin(1) the exact arg-min if needed, gBest record, log, gBest
//                    row, generation counter + 1.
// Steps 4-7 and 9-10 exit at once when their list is empty.  The refinement
// exists because FP64 on this GPU runs at a small fraction of the FP32 rate:
// one FP64 row costs D^2 FP64 fmas, the refinement about 14 D^2 FP32 ops.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cuda_bf16.h>

#include "psso.h"
#include "psso_internal.h"
#include "rot_pipeline.h"
#include "sso_kernel.cuh"
#include "tc_gemm.cuh"

namespace psso {
namespace rot {

// Appends v to a list of capacity cap (the counter may live in shared memory).
__device__ __forceinline__ void list_push(int32_t* list, unsigned* count, long long cap, int32_t v)
{
    const unsigned slot = atomicAdd(count, 1u);
    if (PSSO_CHK((long long)slot < cap, CHK_LIST, slot)) list[slot] = v;
}

using tc::BM;
using tc::BN;

__global__ void set_gen(RotCtl* ctl, long long g)
{
    ctl->gen = g;
    if (g == 0) ctl->refined = 0;    // counters restart with the swarm, like the gBest record's
    ctl->n1 = 0;
    ctl->n2 = 0;
    ctl->n3 = 0;
    ctl->amb = 0;
    ctl->acc = 0;
    ctl->rck = 0;
}

// ---- 1. update --------------------------------------------------------------
template <int MAXC>
__device__ void update_row(const RotDev& r, const Hot& in, int64_t i, int64_t g)
{
    const int lane = threadIdx.x & 31;
    const InstDev& d = *r.inst;
    float* xr = static_cast<float*>(d.X) + i * in.Dp;
    const float* pr = static_cast<const float*>(d.P) + i * in.Dp;
    const float* gs = static_cast<const float*>(d.gbrow);
    const uint32_t gg = (uint32_t)g;
    const uint32_t ctr3r = TAG_RHO | (in.sid << 8), ctr3f = TAG_FRESH | (in.sid << 8);
    bool eqp = true;
    float dmax = 0.f, l1 = 0.f;
    float dv[MAXC][4], dl[MAXC][4];    // d = x - o exactly, as a float pair
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
#pragma unroll
        for (int m = 0; m < 4; ++m) dv[q][m] = dl[q][m] = 0.f;
        if (c >= in.nchunks) continue;
        const int nvalid = min(4, in.D - 4 * c);
        const uint32_t valid = (1u << nvalid) - 1u;
        float x[4] = {0.f, 0.f, 0.f, 0.f};
        if (g == 0) {
            fresh_chunk(x, valid, (uint32_t)c, (uint32_t)i + in.i_base, 0u, TAG_INIT, in);
        } else {
            const uint4 rb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3r), in.k0, in.k1);
            const uint4 fb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3f), in.k0, in.k1);
            float xo[4], po[4], go[4];
            // xo: the third interval's source, go: the first's (Eq. 2.1 as printed
            // swaps them: keep x first, gBest third)
            ld4((in.order ? gs : xr) + 4 * c, xo);
            ld4(pr + 4 * c, po);
            ld4((in.order ? xr : gs) + 4 * c, go);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t w = word_of(rb, m);
                const bool lg = (w < in.Tg32) || (in.tfull & 1u);
                const bool lp = (w < in.Tp32) || (in.tfull & 2u);
                const bool lw = (w < in.Tw32) || (in.tfull & 4u);
                x[m] = lg ? go[m] : lp ? po[m] : lw ? xo[m] : fresh_f32(word_of(fb, m), in);
                if (m >= nvalid) x[m] = 0.f;
                eqp = eqp && same_bits(x[m], po[m]);
            }
        }
        st4(xr + 4 * c, x);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * c + m;
            if (j < in.D) {
                const float a = x[m], b = -__ldg(in.o32 + j);
                const float sum = __fadd_rn(a, b), bb = __fsub_rn(sum, a);   // TwoSum
                dv[q][m] = sum;
                dl[q][m] = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
            }
            dmax = fmaxf(dmax, fabsf(dv[q][m]));
            l1 = __fadd_ru(l1, fabsf(dv[q][m]));
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
        l1 = __fadd_ru(l1, __shfl_xor_sync(0xffffffffu, l1, off));
    }
    eqp = __all_sync(0xffffffffu, eqp);
    // |d| <= |fl(d)| (1 + 2^-24): the scale and the L1 norm cover the exact d
    l1 = __fmul_ru(l1, 1.f + 0x1p-22f);
    // the 7-bit integer slices of d / s_d (tc_gemm.cuh), four planes
    const float sd = tc::slice_scale(dmax), inv = 1.f / sd;   // powers of two: exact
    const size_t plane = (size_t)r.Np * r.Kp;
    __nv_bfloat16* arow = r.A + (size_t)i * r.Kp;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
        if (c >= in.nchunks) continue;
        __nv_bfloat16 sl[4][tc::SLICES];
#pragma unroll
        for (int m = 0; m < 4; ++m) tc::slice4_pair(__fmul_rn(dv[q][m], inv), __fmul_rn(dl[q][m], inv), sl[m]);
#pragma unroll
        for (int p = 0; p < tc::SLICES; ++p) {
            // 4 consecutive bf16 (8 bytes) per plane
            uint2 u;
            u.x = (uint32_t)__bfloat16_as_ushort(sl[0][p]) | ((uint32_t)__bfloat16_as_ushort(sl[1][p]) << 16);
            u.y = (uint32_t)__bfloat16_as_ushort(sl[2][p]) | ((uint32_t)__bfloat16_as_ushort(sl[3][p]) << 16);
            *reinterpret_cast<uint2*>(arow + p * plane + 4 * c) = u;
        }
    }
    if (lane == 0) {
        r.dscale[i] = sd;
        r.dl1[i] = l1;
        r.same[i] = (g > 0 && eqp) ? 1u : 0u;
    }
}

__global__ void rot_update(const RotDev r)
{
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const InstDev& d = *r.inst;
    if (i >= d.N) return;
    const Hot in = hot_of(d);
    const int64_t g = r.ctl->gen;
    switch (in.maxc) {
    case 1: update_row<1>(r, in, i, g); break;
    case 2: update_row<2>(r, in, i, g); break;
    case 4: update_row<4>(r, in, i, g); break;
    default: update_row<8>(r, in, i, g); break;
    }
}

// ---- 2. GEMM with the fitness epilogue ------------------------------------------
// Per element z~ with error ez (the integer-slice GEMM of tc_gemm.cuh of the
// exact d = x - o and the FP64 M: dropped slice products and remainders, the
// FP32 join, against the FP64 rotation M (x - o)),
// the terms and bounds of the rotated functions (as in the FP32 path of the
// persistent kernel): ellipsoid w z^2; Rastrigin z^2 + 20 sin^2(pi z);
// Ackley z^2 and sin^2(pi z) (two sums).  Sums: 32 terms per column block,
// then 4 blocks per tile, then the tiles (in rot_decide).
__device__ __forceinline__ void term32(int fn, float zt, float ez, const float* w32, int j, float& s,
                                       float& s2, float& e, float& eq)
{
    const float az = fabsf(zt);
    const float xi = az + ez;
    if (fn == FN_ELLIPSOID) {
        const float w = __ldg(w32 + j);
        const float tv = __fmul_rn(w, __fmul_rn(zt, zt));
        s = __fadd_rn(s, tv);
        e = __fadd_rn(e, 4.2f * 0x1p-24f * tv + 1.01f * w * (2.f * az + ez) * ez);
    } else if (fn == FN_RASTRIGIN) {
        const float sn = sinpi_reduced_f32(__fsub_rn(zt, rintf(zt)));
        const float tv = __fmaf_rn(zt, zt, __fmul_rn(20.f, __fmul_rn(sn, sn)));
        s = __fadd_rn(s, tv);
        e = __fadd_rn(e, (2.f * SINPI32_ERR_U + 4.f) * 0x1p-24f * tv +
                             1.01f * (2.f * xi + 62.8318558f * fminf(1.f, 6.28318548f * xi)) * ez);
    } else {   // Ackley
        s = __fadd_rn(s, __fmul_rn(zt, zt));
        const float sn = sinpi_reduced_f32(__fsub_rn(zt, rintf(zt)));
        s2 = __fadd_rn(s2, __fmul_rn(sn, sn));
        e = __fadd_rn(e, 1.01f * (2.f * az + ez) * ez);
        eq = __fadd_rn(eq, 1.01f * 3.14159275f * fminf(1.f, 6.28318548f * xi) * ez);
    }
}

struct FitEpi {
    const RotDev* r;
    int fn, D;
    float drop;                   // SLICE_DROP * D
    // the current tile and row: particle i, column tile nt, s_d, sum |d_k|
    int64_t i;
    int nt;
    float ds, dl1;
    float acc, acc2, accE, rQ;
    __device__ void tile(int tm, int tn, int row)
    {
        i = (int64_t)tm * BM + row;
        nt = tn;
        ds = i < r->N ? r->dscale[i] : 1.f;
        dl1 = i < r->N ? r->dl1[i] : 0.f;
        acc = acc2 = accE = rQ = 0.f;
    }
    __device__ void operator()(int c, const float (&tj)[32], const float (&em)[32])
    {
        const int j0 = nt * tc::SBN + 32 * c;
        float s = 0.f, s2 = 0.f, e = 0.f, eq = 0.f;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int j = j0 + t;
            if (j >= D) break;
            const float sm = __ldg(r->mscale + j), l1m = __ldg(r->ml1 + j);
            const float sc = __fmul_rn(ds, sm);                 // a power of two
            const float zt = __fmul_rn(tj[t], __fmul_rn(sc, 0x1p-14f));
            const float rd = __fmul_rn(sm, dl1), rm = __fmul_rn(ds, l1m);
            // dropped slice products, slice remainders, the FP64 reference's
            // own rounding (D <= 2^13 terms: 2^-40 sum |M||d|), the FP32 join
            const float ez = 1.01f * (drop * sc + tc::SLICE_REM * (rd + rm) + 0x1p-40f * fminf(rd, rm) +
                                      0x1p-38f * em[t] * sc) + 0x1p-126f;
            term32(fn, zt, ez, r->inst_w32, j, s, s2, e, eq);
        }
        acc = __fadd_rn(acc, s);
        acc2 = __fadd_rn(acc2, s2);
        accE = __fadd_rn(accE, e);
        rQ = __fadd_rn(rQ, eq);
        if (c == tc::SBN / 32 - 1) {
            if (i < r->N && PSSO_CHK(nt < r->nJt, CHK_TILE, nt))
                r->part[i * r->nJt + nt] = make_float4(acc, acc2, accE, rQ);
        }
    }
};

// Persistent: one CTA per SM (at most one per tile), tiles in grid-stride order.
__global__ void __launch_bounds__(tc::S_THREADS, 1)
    rot_gemm_fit(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ RotDev r)
{
    FitEpi epi{&r, base_fn(r.fn), r.D, tc::SLICE_DROP * (float)r.D};
    tc::GemmArgs a{r.Np, r.Jp, r.Kp, &r.ctl->status};
    tc::gemm_sliced_persistent(&tmA, &tmB, a, epi);
}

// ---- 3. FP32 decisions ------------------------------------------------------------
// FP32 fitness and its bound from the sums of the terms (the rotated branches
// of the FP32 path); csum = summation depth + 2 (GEMM epilogue: 32 + 4 +
// tiles + 2).
__device__ inline Fit32 rot_final(int fn, int D, float acc, float acc2, float accE, float rQ, float csum)
{
    const float U = 0x1p-24f;
    Fit32 f;
    if (fn != FN_ACKLEY) {
        f.f = acc;
        f.E = 1.1f * (accE + csum * U * acc);
        f.E = __fadd_ru(f.E, 0x1p-40f * (acc + accE));
        return f;
    }
    const float Df = (float)D;
    const float A = __fsqrt_rn(__fdiv_rn(acc, Df));
    const float B = expm1_f32(__fmul_rn(-0.2f, A));
    const float C = expm1_f32(__fmul_rn(-2.f, __fdiv_rn(acc2, Df)));
    const float f1 = __fmul_rn(-20.f, B), f2 = __fmul_rn(-0x1.5bf0a8p+1f, C);
    f.f = __fadd_rn(f1, f2);
    const float ES = accE + (3.1f + csum) * U * acc;
    const float EQ = rQ + (2.f * SINPI32_ERR_U + 1.f + csum) * U * acc2;
    const float d1 = (ES <= 0.5f * acc) ? 1.5f * f1 * ES / acc : 4.f * __fsqrt_ru(ES / Df);
    f.E = 1.1f * (d1 + (EXPM1F_ERR_U + 6.f) * U * f1 + (2.f * 2.7182818f / Df) * EQ +
                  (EXPM1F_ERR_U + 8.f) * U * f2 + U * f.f);
    f.E = __fadd_ru(f.E, 0x1p-40f * (f.f + accE));
    return f;
}

__global__ void rot_decide(const RotDev r)
{
    __shared__ unsigned long long blk_acc;
    if (threadIdx.x == 0) blk_acc = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const InstDev& d = *r.inst;
    const int64_t g = r.ctl->gen;
    if (i < d.N) {
        // tile sums in tile order by lane 0 (a fixed order)
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < r.nJt) p = r.part[i * r.nJt + lane];
        float a = 0.f, a2 = 0.f, ae = 0.f, aq = 0.f;
        for (int t = 0; t < r.nJt; ++t) {
            a = __fadd_rn(a, __shfl_sync(0xffffffffu, p.x, t));
            a2 = __fadd_rn(a2, __shfl_sync(0xffffffffu, p.y, t));
            ae = __fadd_rn(ae, __shfl_sync(0xffffffffu, p.z, t));
            aq = __fadd_rn(aq, __shfl_sync(0xffffffffu, p.w, t));
        }
        const Fit32 f = rot_final(base_fn(r.fn), r.D, a, a2, ae, aq, 38.f + (float)r.nJt);
        const float lo = __fsub_rd(f.f, f.E), hi = __fadd_ru(f.f, f.E);
        int accept = 0, write = 0, undecided = 0;
        if (g == 0) {
            accept = write = 1;
        } else if (r.same[i]) {
            accept = 1;              // identical row: identical fitness, state unchanged
        } else if (hi < d.plo[i]) {
            accept = write = 1;
        } else if (!(lo > d.phi[i])) {
            undecided = 1;
        }
        if (write) {
            const float* xr = static_cast<const float*>(d.X) + i * d.Dp;
            float* prow = static_cast<float*>(d.P) + i * d.Dp;
            for (int c = lane; c < d.nchunks; c += 32) {
                float v[4];
                ld4(xr + 4 * c, v);
                st4(prow + 4 * c, v);
            }
            if (lane == 0) {
                d.plo[i] = lo;
                d.phi[i] = hi;
                d.pflag[i] = 0u;
                d.pf64[i] = 0.0;
                d.pver[i] = (uint32_t)g;
            }
        }
        if (lane == 0) {
            if (undecided) list_push(r.list1, &r.ctl->n1, r.N, (int32_t)i);
            if (accept) atomicAdd(&blk_acc, 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk_acc) atomicAdd(&r.ctl->acc, blk_acc);
}

// ---- 4. refinement: compensated FP32 rotation of list-1 rows ---------------------------
// d = x - o exactly as a float pair (TwoSum), M = Mh + Ml.  Per output j the
// 32 lanes of a warp take k = l, l + 32, ... (coalesced rows of M): the Dot2
// recurrence per lane (TwoProduct of Mh d_h, TwoSum into p, the rounding
// errors and the cross terms Mh d_l + Ml d_h into s), then the 32 lane sums
// merged by a TwoSum butterfly, z = p + s.  With n = ceil(D / 32) + 8 and
// g = gamma_n: |z~ - z| <= 1.01 u |z~| + (2 g^2 + 4 u g + 2^-42) S, where
// S = sum |M||d| <= S~ (1 + 2 gamma_D)(1 + 2^-22) from the FP32 sum S~ of
// |Mh||d_h|; 2^-42 S also covers the oracle's own FP64 rounding of z.
// A block takes Z32_OUT outputs of one listed row; each warp keeps Z32_NJ
// outputs in flight (independent chains sharing the loads of d), so a short
// list still spreads over many blocks and the loads of M overlap.
constexpr int Z32_NJ = 4;                       // outputs per warp in flight
constexpr int Z32_OUT = 32;                     // outputs per block
__global__ void __launch_bounds__(128) rot_z32(const RotDev r)
{
    __shared__ float dh[1024], dl[1024];
    const InstDev& d = *r.inst;
    const unsigned n = r.ctl->n1;
    const int D = r.D;
    if (!PSSO_CHK(n <= r.N && D <= 1024, CHK_LIST, n)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nJb = (D + Z32_OUT - 1) / Z32_OUT;
    const float U = 0x1p-24f;
    const float nl = (float)((D + 31) / 32 + 8);
    const float gam = nl * U / (1.f - nl * U);
    const float gD = (float)D * U / (1.f - (float)D * U);
    const float cS = 1.01f * (2.f * gam * gam + 4.f * U * gam + 0x1p-42f) * (1.f + 2.f * gD) * (1.f + 0x1p-22f);
    const long long items = (long long)n * 2 * nJb;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int jb = (int)(it % nJb);
        const int row = (int)((it / nJb) & 1);
        const long long e = it / nJb / 2;
        const int32_t i = r.list1[e];
        if (!PSSO_CHK(i >= 0 && i < r.N, CHK_ROT_ROW, i)) continue;
        if (row == 1 && (d.pflag[i] & 1u)) continue;     // uniform over the block
        const float* src = static_cast<const float*>(row == 0 ? d.X : d.P) + (int64_t)i * d.Dp;
        __syncthreads();
        for (int k = threadIdx.x; k < D; k += blockDim.x) {
            const float a = src[k], b = -__ldg(d.o32 + k);
            const float sum = __fadd_rn(a, b);
            const float bb = __fsub_rn(sum, a);
            dh[k] = sum;
            dl[k] = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
        }
        __syncthreads();
        const size_t o = (size_t)(2 * e + row) * d.Dp;
#pragma unroll 1
        for (int pass = 0; pass < Z32_OUT / (4 * Z32_NJ); ++pass) {
            const int j0 = jb * Z32_OUT + pass * 4 * Z32_NJ + warp * Z32_NJ;   // warp-uniform
            int nv = D - j0;                     // outputs of this group inside the row
            nv = nv < 0 ? 0 : nv > Z32_NJ ? Z32_NJ : nv;
            if (lane == 0)
                for (int t = nv; t < Z32_NJ; ++t)
                    if (j0 + t < d.Dp) {
                        r.z32[o + j0 + t] = 0.f;
                        r.ez32[o + j0 + t] = 0.f;
                    }
            if (nv == 0) continue;
            const float* mh[Z32_NJ];
            const float* ml[Z32_NJ];
            float p[Z32_NJ], sc[Z32_NJ], S[Z32_NJ];
#pragma unroll
            for (int t = 0; t < Z32_NJ; ++t) {
                const int j = t < nv ? j0 + t : j0;   // rows past the end repeat a valid one, unused
                mh[t] = r.Mh + (size_t)j * D;
                ml[t] = r.Ml + (size_t)j * D;
                p[t] = sc[t] = S[t] = 0.f;
            }
            for (int k = lane; k < D; k += 32) {
                const float b = dh[k], bl = dl[k];
#pragma unroll
                for (int t = 0; t < Z32_NJ; ++t) {
                    const float a = __ldg(mh[t] + k);
                    const float h = __fmul_rn(a, b);
                    const float rr = __fmaf_rn(a, b, -h);                 // a b = h + rr exactly
                    const float tt = __fadd_rn(p[t], h);
                    const float bb = __fsub_rn(tt, p[t]);
                    const float q = __fadd_rn(__fsub_rn(p[t], __fsub_rn(tt, bb)), __fsub_rn(h, bb));   // p + h = tt + q
                    p[t] = tt;
                    const float cross = __fmaf_rn(a, bl, __fmul_rn(__ldg(ml[t] + k), b));
                    sc[t] = __fadd_rn(sc[t], __fadd_rn(__fadd_rn(q, rr), cross));
                    S[t] = __fmaf_rn(fabsf(a), fabsf(b), S[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < Z32_NJ; ++t) {
                for (int off = 16; off > 0; off >>= 1) {       // every lane ends with the same values
                    const float po = __shfl_xor_sync(0xffffffffu, p[t], off);
                    const float so = __shfl_xor_sync(0xffffffffu, sc[t], off);
                    const float Sq = __shfl_xor_sync(0xffffffffu, S[t], off);
                    const float tt = __fadd_rn(p[t], po);
                    const float bb = __fsub_rn(tt, p[t]);
                    const float q = __fadd_rn(__fsub_rn(p[t], __fsub_rn(tt, bb)), __fsub_rn(po, bb));
                    p[t] = tt;
                    sc[t] = __fadd_rn(__fadd_rn(sc[t], so), q);
                    S[t] = __fadd_rn(S[t], Sq);
                }
                if (lane == 0 && t < nv) {
                    const float z = __fadd_rn(p[t], sc[t]);
                    r.z32[o + j0 + t] = z;
                    r.ez32[o + j0 + t] = __fmaf_ru(cS, S[t], 1.01f * U * fabsf(z));
                }
            }
        }
    }
}

// ---- 5. decisions from the refined intervals ---------------------------------------------
template <int MAXC>
__device__ Fit32 fit_refined(const RotDev& r, const InstDev& d, const float* z, const float* ez, int lane)
{
    const int fn = base_fn(r.fn);
    float s = 0.f, s2 = 0.f, e = 0.f, eq = 0.f;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
        if (c >= d.nchunks) continue;
        float zv[4], ev[4];
        ld4(z + 4 * c, zv);
        ld4(ez + 4 * c, ev);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (4 * c + m < d.D) term32(fn, zv[m], ev[m], r.inst_w32, 4 * c + m, s, s2, e, eq);
    }
    for (int off = 16; off > 0; off >>= 1) {
        s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, off));
        s2 = __fadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, off));
        e = __fadd_rn(e, __shfl_xor_sync(0xffffffffu, e, off));
        eq = __fadd_rn(eq, __shfl_xor_sync(0xffffffffu, eq, off));
    }
    return rot_final(fn, d.D, s, s2, e, eq, (float)(4 * MAXC + 5 + 2));
}

template <int MAXC>
__device__ void fix32_one(const RotDev& r, const InstDev& d, long long e, int lane)
{
    const int32_t i = r.list1[e];
    if (!PSSO_CHK(i >= 0 && i < r.N, CHK_ROT_ROW, i)) return;
    const int64_t g = r.ctl->gen;
    const size_t ox = (size_t)(2 * e) * d.Dp, op = ox + d.Dp;
    float plo = d.plo[i], phi = d.phi[i];
    const Fit32 fx = fit_refined<MAXC>(r, d, r.z32 + ox, r.ez32 + ox, lane);
    const float lox = __fsub_rd(fx.f, fx.E), hix = __fadd_ru(fx.f, fx.E);
    const bool have_p = (d.pflag[i] & 1u) != 0;
    if (!have_p) {       // the pBest's interval, tightened the same way (intersection of two bounds)
        const Fit32 fp = fit_refined<MAXC>(r, d, r.z32 + op, r.ez32 + op, lane);
        plo = fmaxf(plo, __fsub_rd(fp.f, fp.E));
        phi = fminf(phi, __fadd_ru(fp.f, fp.E));
    }
    const int accept = hix < plo;
    const int reject = lox > phi;
    if (accept) {
        const float* xr = static_cast<const float*>(d.X) + (int64_t)i * d.Dp;
        float* prow = static_cast<float*>(d.P) + (int64_t)i * d.Dp;
        for (int c = lane; c < d.nchunks; c += 32) {
            float v[4];
            ld4(xr + 4 * c, v);
            st4(prow + 4 * c, v);
        }
    }
    if (lane == 0) {
        if (accept) {
            d.plo[i] = lox;
            d.phi[i] = hix;
            d.pflag[i] = 0u;
            d.pf64[i] = 0.0;
            d.pver[i] = (uint32_t)g;
            atomicAdd(&r.ctl->acc, 1ull);
        } else {
            d.plo[i] = plo;
            d.phi[i] = phi;
            if (!reject) list_push(r.list3, &r.ctl->n3, r.N, i);
        }
        atomicAdd(&r.ctl->refined, have_p ? 1ull : 2ull);
    }
}

__global__ void rot_fix32(const RotDev r)
{
    const int lane = threadIdx.x & 31;
    const InstDev& d = *r.inst;
    const unsigned n = r.ctl->n1;
    if (!PSSO_CHK(n <= r.N, CHK_LIST, n)) return;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < (long long)n;
         e += nwarps) {
        switch (d.maxc) {
        case 1: fix32_one<1>(r, d, e, lane); break;
        case 2: fix32_one<2>(r, d, e, lane); break;
        case 4: fix32_one<4>(r, d, e, lane); break;
        default: fix32_one<8>(r, d, e, lane); break;
        }
    }
}

// The float pair of M for the refinement (setup).
__global__ void split_m64(const double* M64, long long DD, float* Mh, float* Ml)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < DD; q += (long long)gridDim.x * blockDim.x) {
        const double m = M64[q];
        const float h = __double2float_rn(m);
        Mh[q] = h;
        Ml[q] = __double2float_rn(m - (double)h);
    }
}

// ---- 4/7. FP64 rotation of listed rows ------------------------------------------------
// which = 1: entries of list3, row 2e = X_i and row 2e+1 = P_i when its FP64
// value is not known; which = 2: entries of list2, row 2e+1 = P_i.
__global__ void rot_z64(const RotDev r, int which)
{
    __shared__ double dsh[1024];
    const InstDev& d = *r.inst;
    const unsigned n = which == 1 ? r.ctl->n3 : r.ctl->n2;   // which 2 or 4: list 2
    const int D = r.D;
    if (!PSSO_CHK(n <= r.N && D <= 1024, CHK_LIST, n)) return;
    const int nJb = (D + 127) / 128;
    const long long items = (long long)n * 2 * nJb;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int jb = (int)(it % nJb);
        const int row = (int)((it / nJb) & 1);
        const long long e = it / nJb / 2;
        const int32_t i = which == 1 ? r.list3[e] : r.list2[e];
        if (!PSSO_CHK(i >= 0 && i < r.N, CHK_ROT_ROW, i)) continue;
        const bool needed = which == 1 ? (row == 0 || !(d.pflag[i] & 1u)) : row == 1;
        if (!needed) continue;          // uniform over the block
        const float* src = static_cast<const float*>(row == 0 ? d.X : d.P) + (int64_t)i * d.Dp;
        __syncthreads();
        for (int k = threadIdx.x; k < D; k += blockDim.x) dsh[k] = __dsub_rn((double)src[k], d.o64[k]);
        __syncthreads();
        const int j = jb * 128 + threadIdx.x;
        double* out = r.zbuf + (size_t)(2 * e + row) * d.Dp;
        if (j < D) {
            const double* mrow = d.M64 + (size_t)j * D;
            double z = 0.0;
            for (int k = 0; k < D; ++k) z = __fma_rn(__ldg(mrow + k), dsh[k], z);
            out[j] = z;
        } else if (j < d.Dp) {
            out[j] = 0.0;
        }
    }
}

// ---- 5/8. FP64 fitness of the rotated rows and the exact decisions --------------------
__device__ void fix_one(const RotDev& r, const InstDev& d, int which, long long e, int lane)
{
    Hot hz = hot_of(d);
    hz.fn = base_fn(d.fn);   // the rows hold z already: the unrotated function with o = 0
    hz.o64 = r.zero64;
    const int64_t g = r.ctl->gen;
    const double* zx = r.zbuf + (size_t)(2 * e) * d.Dp;
    const double* zp = zx + d.Dp;
    if (which == 1) {
        const int32_t i = r.list3[e];
        if (!PSSO_CHK(i >= 0 && i < r.N, CHK_ROT_ROW, i)) return;
        const bool have_p = (d.pflag[i] & 1u) != 0;
        const double fx = fit64_row<double>(hz, zx, false);
        const double fp = have_p ? d.pf64[i] : fit64_row<double>(hz, zp, false);
        const bool accept = fx <= fp;
        if (accept) {
            const float* xr = static_cast<const float*>(d.X) + (int64_t)i * d.Dp;
            float* prow = static_cast<float*>(d.P) + (int64_t)i * d.Dp;
            for (int c = lane; c < d.nchunks; c += 32) {
                float v[4];
                ld4(xr + 4 * c, v);
                st4(prow + 4 * c, v);
            }
        }
        if (lane == 0) {
            const double v = accept ? fx : fp;
            d.pf64[i] = v;
            d.pflag[i] = 1u;
            d.plo[i] = f64_to_f32_rd(v);
            d.phi[i] = f64_to_f32_ru(v);
            if (accept) d.pver[i] = (uint32_t)g;
            atomicAdd(&r.ctl->rck, have_p ? 1ull : 2ull);
            if (accept) atomicAdd(&r.ctl->acc, 1ull);
        }
    } else {   // list 2 (which 2: in a generation; 4: on demand, outside the counters)
        const int32_t i = r.list2[e];
        if (!PSSO_CHK(i >= 0 && i < r.N, CHK_ROT_ROW, i)) return;
        const double fp = fit64_row<double>(hz, zp, false);
        if (lane == 0) {
            d.pf64[i] = fp;
            d.pflag[i] = 1u;
            d.plo[i] = f64_to_f32_rd(fp);
            d.phi[i] = f64_to_f32_ru(fp);
            if (which == 2) atomicAdd(&r.ctl->rck, 1ull);
        }
    }
}

__global__ void rot_fix(const RotDev r, int which)
{
    const int lane = threadIdx.x & 31;
    const InstDev& d = *r.inst;
    const unsigned n = which == 1 ? r.ctl->n3 : r.ctl->n2;
    if (!PSSO_CHK(n <= r.N, CHK_LIST, n)) return;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < (long long)n;
         e += nwarps)
        fix_one(r, d, which, e, lane);
}


// ---- 6/9. gBest --------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) rot_argmin(const RotDev r, int phase)
{
    __shared__ Cand sh[32];
    __shared__ unsigned n2;
    const InstDev& d = *r.inst;
    RotCtl* ctl = r.ctl;
    const int64_t g = ctl->gen;
    const int64_t N = d.N;
    if (phase == 0) {
        Cand c = cand_none();
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
            c = cand_merge<true>(c, cand_of<true>((long long)i, d.pf64[i], d.plo[i], d.phi[i],
                                                  (int)(d.pflag[i] & 1u), d.pver[i]));
        const Cand b = block_reduce_cand<true>(c, sh);
        if (b.l2 > b.mh) {          // one interval lies below every other: the arg-min
            if (threadIdx.x == 0) {
                // the gBest value the generation reports must lie within 1e-6 of
                // FP64: an interval too wide for that gets the winner's FP64 value
                // (list 2; the exact pass of phase 1 then keeps the same winner)
                const bool wide = !b.has1 && too_wide(r.fn, b.l1, b.h1);
                ctl->amb = wide ? 1 : 0;
                if (wide) {
                    r.list2[0] = (int32_t)b.i;
                    ctl->n2 = 1;
                }
                ctl->win_i = b.i;
                ctl->win_v = b.v;
                ctl->win_lo = b.l1;
                ctl->win_hi = b.h1;
                ctl->win_has = b.has1;
                ctl->win_ver = b.ver;
            }
            return;
        }
        // several pBests may be the minimum: those without an FP64 value go on list2
        if (threadIdx.x == 0) n2 = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
            if (d.plo[i] <= b.mh && !(d.pflag[i] & 1u)) list_push(r.list2, &n2, r.N, (int32_t)i);
        __syncthreads();
        if (threadIdx.x == 0) {
            ctl->amb = 1;
            ctl->n2 = n2;
        }
        return;
    }
    // phase 1
    if (ctl->amb) {
        // every pBest that can be the minimum now has its FP64 value; the others
        // have a lower bound above the smallest upper bound
        Cand c = cand_none();
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
            if (d.pflag[i] & 1u) {
                Cand q = cand_none();
                q.v = d.pf64[i];
                q.i = (long long)i;
                q.ver = d.pver[i];
                c = cand_merge<false>(c, q);
            }
        const Cand b = block_reduce_cand<false>(c, sh);
        if (threadIdx.x == 0) {
            ctl->win_i = b.i;
            ctl->win_v = b.v;
            ctl->win_lo = f64_to_f32_rd(b.v);
            ctl->win_hi = f64_to_f32_ru(b.v);
            ctl->win_has = 1;
            ctl->win_ver = b.ver;
        }
        __syncthreads();
    }
    const long long wi = ctl->win_i;
    const float* src = static_cast<const float*>(d.P) + wi * d.Dp;
    float* dst = static_cast<float*>(d.gbrow);
    for (int j = threadIdx.x; j < d.Dp; j += blockDim.x) dst[j] = src[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        Winner w;
        w.idx = wi;
        w.has64 = ctl->win_has;
        w.f64 = w.has64 ? ctl->win_v : 0.0;
        w.lo = ctl->win_lo;
        w.hi = ctl->win_hi;
        w.ver = ctl->win_ver;
        w.acc = ctl->acc;
        w.rck = ctl->rck;
        write_gbest(d, w, g);
        ctl->gen = g + 1;
        ctl->n1 = 0;
        ctl->n2 = 0;
        ctl->n3 = 0;
        ctl->amb = 0;
        ctl->acc = 0;
        ctl->rck = 0;
    }
}

// ---- values on demand --------------------------------------------------------------------
// Every pBest whose value is known only by an interval too wide for 1e-6
// relative goes on list 2; its FP64 value is then computed (rot_z64 and
// rot_fix with which = 4) -- once, when the state is read.  The trajectory
// does not change: only the stored intervals become exact.
__global__ void list_wide(const RotDev r)
{
    const InstDev& d = *r.inst;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += (int64_t)gridDim.x * blockDim.x)
        if (!(d.pflag[i] & 1u) && too_wide(r.fn, d.plo[i], d.phi[i]))
            list_push(r.list2, &r.ctl->n2, r.N, (int32_t)i);
}

__global__ void clear_n2(RotCtl* ctl) { ctl->n2 = 0; }

// ---- host --------------------------------------------------------------------------------
cudaError_t exact_values_for_read(const RotHost& h, cudaStream_t s)
{
    const RotDev& r = h.dev;
    clear_n2<<<1, 1, 0, s>>>(r.ctl);
    list_wide<<<(unsigned)std::min<long long>((h.N + 255) / 256, 1024), 256, 0, s>>>(r);
    rot_z64<<<h.z64_grid, 128, 0, s>>>(r, 4);
    rot_fix<<<h.fix_grid, 256, 0, s>>>(r, 4);
    clear_n2<<<1, 1, 0, s>>>(r.ctl);
    return cudaGetLastError();
}

cudaError_t enqueue_generation_timed(const RotHost& h, cudaStream_t s, cudaEvent_t* ev);

cudaError_t enqueue_generation(const RotHost& h, cudaStream_t s)
{
    return enqueue_generation_timed(h, s, nullptr);
}

// With ev (KERNELS_PER_GENERATION + 1 events), an event is recorded before
// the first kernel and after each kernel.
cudaError_t enqueue_generation_timed(const RotHost& h, cudaStream_t s, cudaEvent_t* ev)
{
    int q = 0;
    auto mark = [&] {
        if (ev) cudaEventRecord(ev[q++], s);
    };
    mark();
    const RotDev& r = h.dev;
    const int N = (int)h.N;
    const int wpb = 8;
    rot_update<<<(N + wpb - 1) / wpb, 32 * wpb, 0, s>>>(r);
    mark();
    rot_gemm_fit<<<h.gemm_grid, tc::S_THREADS, tc::S_SMEM_BYTES, s>>>(h.tmA, h.tmB, r);
    mark();
    rot_decide<<<(N + wpb - 1) / wpb, 32 * wpb, 0, s>>>(r);
    mark();
    rot_z32<<<h.z32_grid, 128, 0, s>>>(r);
    mark();
    rot_fix32<<<h.fix_grid, 32 * wpb, 0, s>>>(r);
    mark();
    rot_z64<<<h.z64_grid, 128, 0, s>>>(r, 1);
    mark();
    rot_fix<<<h.fix_grid, 32 * wpb, 0, s>>>(r, 1);
    mark();
    rot_argmin<<<1, 1024, 0, s>>>(r, 0);
    mark();
    rot_z64<<<h.z64_grid, 128, 0, s>>>(r, 2);
    mark();
    rot_fix<<<h.fix_grid, 32 * wpb, 0, s>>>(r, 2);
    mark();
    rot_argmin<<<1, 1024, 0, s>>>(r, 1);
    mark();
    return cudaGetLastError();
}

// The generation number lives in device memory, so one captured generation
// replays unchanged; graphs are captured on a private stream and launched on
// the caller's.
cudaError_t make_graphs(RotHost& h)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        const int gens = which == 0 ? 1 : GRAPH_GENS;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int q = 0; q < gens && e == cudaSuccess; ++q) e = enqueue_generation(h, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(which == 0 ? &h.graph1 : &h.graphG, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    return e;
}

void destroy_graphs(RotHost& h)
{
    if (h.graph1) cudaGraphExecDestroy(h.graph1);
    if (h.graphG) cudaGraphExecDestroy(h.graphG);
    h.graph1 = h.graphG = nullptr;
}

cudaError_t run_generations(const RotHost& h, long long count, cudaStream_t s)
{
    for (; count >= GRAPH_GENS; count -= GRAPH_GENS) {
        const cudaError_t e = cudaGraphLaunch(h.graphG, s);
        if (e != cudaSuccess) return e;
    }
    for (; count > 0; --count) {
        const cudaError_t e = cudaGraphLaunch(h.graph1, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// B planes of the integer-slice GEMM from the FP64 rotation: one block per
// row j of the padded [Jp][Kp] planes (rows >= D and columns >= D are zero),
// its scale s_M and sum_k |M_jk| (rounded up).
__global__ void slice_matrix(const double* __restrict__ M64, int D, int Jp, int Kp, __nv_bfloat16* B,
                             float* mscale, float* ml1)
{
    const int j = blockIdx.x;
    double mx = 0.0, l1 = 0.0;
    for (int k = threadIdx.x; k < D; k += blockDim.x) {
        const double v = j < D ? M64[(size_t)j * D + k] : 0.0;
        mx = fmax(mx, fabs(v));
        l1 = __dadd_ru(l1, fabs(v));
    }
    __shared__ double rmx[32], rl1[32];
    __shared__ float sm;
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        l1 = __dadd_ru(l1, __shfl_xor_sync(0xffffffffu, l1, off));
    }
    if ((threadIdx.x & 31) == 0) {
        rmx[threadIdx.x >> 5] = mx;
        rl1[threadIdx.x >> 5] = l1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0, t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            m = fmax(m, rmx[w]);
            t = __dadd_ru(t, rl1[w]);
        }
        sm = tc::slice_scale(__double2float_ru(m));
        mscale[j] = sm;
        ml1[j] = __double2float_ru(t);
    }
    __syncthreads();
    const double inv = 1.0 / (double)sm;
    const size_t plane = (size_t)Jp * Kp;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        const double v = (j < D && k < D) ? M64[(size_t)j * D + k] : 0.0;
        __nv_bfloat16 sl[tc::SLICES];
        tc::slice4_f64(__dmul_rn(v, inv), sl);
        for (int p = 0; p < tc::SLICES; ++p) B[p * plane + (size_t)j * Kp + k] = sl[p];
    }
}

cudaError_t build_constants(const RotHost& h, cudaStream_t s)
{
    const RotDev& r = h.dev;
    const long long DD = (long long)r.D * r.D;
    split_m64<<<(unsigned)std::min<long long>((DD + 255) / 256, 4096), 256, 0, s>>>(h.M64, DD, h.Mh, h.Ml);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    slice_matrix<<<r.Jp, 256, 0, s>>>(h.M64, r.D, r.Jp, r.Kp, h.B, r.mscale, r.ml1);
    return cudaGetLastError();
}

cudaError_t set_generation(const RotHost& h, long long g, cudaStream_t s)
{
    set_gen<<<1, 1, 0, s>>>(h.dev.ctl, g);
    return cudaGetLastError();
}

cudaError_t configure()
{
    return cudaFuncSetAttribute(rot_gemm_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::S_SMEM_BYTES);
}

}  // namespace rot
}  // namespace psso
