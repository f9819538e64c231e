// tc_gemm.cuh -- z = M (x - o) for a tile of 128 particles x 128 outputs on
// the sm_103a tensor cores (tcgen05.mma, operands staged by TMA, FP32
// accumulators in tensor memory).
//
// Precision scheme (split BF16): d = fl32(x - o) and the FP32 copy of M are
// each written exactly as three BF16 parts, v = v_h + v_m + v_l (RN splits:
// |v_m| <= 2^-8 |v| (1.01), |v_l| <= 2^-16 |v| (1.01); the third remainder is
// exactly representable, so the split loses nothing).  Of the nine products
// of the parts, the six above 2^-24 are formed:
//     acc0[kb % 3] += d_h M_h               (main part; three accumulators, K
//                                            blocks dealt round robin, so each
//                                            chain is a third as long)
//     acc1 += d_h M_m + d_m M_h + d_h M_l + d_l M_h + d_m M_m   (corrections)
// and z = fl(fl(fl(acc0[0] + acc0[1]) + acc0[2]) + acc1).  BF16 x BF16
// products are exact in FP32.
//
// Operand layout in global memory (bf16, row-major, K contiguous):
//     A: [3][Np][Kp]   part p of d for particle i at (p, i, k)
//     B: [3][Jp][Kp]   part p of M_jk at (p, j, k)
// Np, Jp multiples of 128, Kp a multiple of 64; padding is zero.  Each
// pipeline stage holds one 64-wide K block of all six planes (6 x 16 KiB,
// TMA boxes of 64 x 128 with the 128-byte swizzle).  One thread issues the
// copies, one thread the MMAs; all four warps run the epilogue, warp w owning
// tensor-memory lanes 32w..32w+31 (one particle each).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace psso {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 2;
constexpr int TILE_BYTES = BM * BK * 2;                    // 16 KiB (BM == BN)
constexpr int STAGE_BYTES = 6 * TILE_BYTES;                // 96 KiB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;    // + alignment slack
constexpr int NCHAIN = 3;                                  // main-part accumulators (K split)
constexpr int TMEM_COLS = 512;                             // acc0[0..2] | acc1
constexpr long long WAIT_CYCLES = 4000000000LL;            // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete; false after
// WAIT_CYCLES (the caller then reports PSSO_ERR_TIMEOUT instead of hanging).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63 && clock64() - t0 > WAIT_CYCLES) return false;
    }
}

// ---- TMA ----------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// ---- tcgen05 ------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrives once on the mbarrier when every MMA issued so far by this thread
// has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle:
// start address >> 4 (bits 0-13), leading offset 16 B (unused with this
// swizzle, bits 16-29), stride between 8-row groups 1024 B (bits 32-45),
// descriptor version 1 (bits 46-47), base offset 0 (the tile is 1024-byte
// aligned), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// 32 consecutive FP32 columns of this warp's 32 lanes (one row per lane).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    // The wait names the registers so that no use of them moves above it.
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
}

// Exact three-part BF16 split of a float (see the header comment).
__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l)
{
    h = __float2bfloat16_rn(v);
    const float r1 = __fsub_rn(v, __bfloat162float(h));
    m = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(m));
    l = __float2bfloat16_rn(r2);
}

// Bound model of the accumulation.  Adversarial probes of kind::f16 MMAs with
// FP32 accumulation on sm_103a (tests/test_gpu_mma_model.py) show an adder
// that aligns its 17 addends (accumulator + 16 exact products) to the largest
// one, truncating each to a multiple of 2^-25 of that addend's leading power
// of two, and truncates the sum to 24 bits: addends below a quarter ulp of
// the largest vanish (an accumulator of 1 absorbs any number of products of
// magnitude 0.99 * 2^-25 unchanged).  One MMA then errs by less than
// 16 * 2^-25 * max|addend| + 2^-23 |sum| <= 0.625 * 2^-20 (|accumulator| +
// sum |products|); MMA_EPS takes 2^-20, a margin of 1.6 over that.
constexpr float MMA_EPS = 0x1p-20f;

// z error per unit of S = sum_k |M32_jk| |d_k| (S <= ||d|| ||M32_j||) for a
// K extent of Kp: the acc0 chains (at most 4 ceil(Kp / 192) MMAs each, over
// products summing to <= 1.03 S in all), the acc1 chain (5 Kp / 16 MMAs
// over products <= 2^-7 1.03 S), the three dropped products (<= 1.03 2^-23
// S), d and M rounded to float (2 x 1.01 2^-24 S), the three additions that
// join the accumulators (3.1 2^-24 S).
__host__ __device__ inline float z_err_per_s(int Kp)
{
    const int nkb = Kp / 64;
    const float n0 = 4.f * (float)((nkb + NCHAIN - 1) / NCHAIN), n1 = 5.f * (float)(Kp / 16);
    return 1.05f * (MMA_EPS * 1.04f * (n0 + n1 * 0x1p-7f) + 1.03f * 0x1p-23f + 2.02f * 0x1p-24f +
                    3.1f * 0x1p-24f);
}

struct GemmArgs {
    int Np, Jp, Kp;   // padded extents (multiples of 128, 128, 64)
    int* status;      // set to 1 when a wait ran out (device memory)
};

// The GEMM main loop for the tile (blockIdx.x, blockIdx.y); the epilogue
// functor gets (row in tile = threadIdx.x, column block c of 32, z[32]).
// Returns false (all threads) if a wait ran out.
template <class Epi>
__device__ __forceinline__ bool gemm_tile(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                          const GemmArgs& a, Epi& epi)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * STAGES + 1];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nkb = a.Kp / BK;
    const uint32_t sbase = smem_u32(smem);
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    const uint32_t done = smem_u32(&bars[2 * STAGES]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        fence_mbar_init();
        failed = 0;
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(empty(s), (uint32_t)((kb / STAGES - 1) & 1))) {
                failed = 1;
                break;
            }
            mbar_expect_tx(full(s), STAGE_BYTES);
            const uint32_t st = sbase + (uint32_t)(s * STAGE_BYTES);
            for (int p = 0; p < 3; ++p) {
                tma_load_2d(st + (uint32_t)(p * TILE_BYTES), tmA, kb * BK, p * a.Np + m0, full(s));
                tma_load_2d(st + (uint32_t)((3 + p) * TILE_BYTES), tmB, kb * BK, p * a.Jp + n0, full(s));
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN);
        const uint32_t acc1 = tmem + NCHAIN * BN;
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(full(s), (uint32_t)((kb / STAGES) & 1))) {
                failed = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = sbase + (uint32_t)(s * STAGE_BYTES);
            const uint32_t acc0 = tmem + (uint32_t)((kb % NCHAIN) * BN);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t off = (uint32_t)(ks * 32);   // 16 bf16 along K
                const uint64_t ah = sdesc_sw128(st + 0 * TILE_BYTES + off);
                const uint64_t am = sdesc_sw128(st + 1 * TILE_BYTES + off);
                const uint64_t al = sdesc_sw128(st + 2 * TILE_BYTES + off);
                const uint64_t bh = sdesc_sw128(st + 3 * TILE_BYTES + off);
                const uint64_t bm = sdesc_sw128(st + 4 * TILE_BYTES + off);
                const uint64_t bl = sdesc_sw128(st + 5 * TILE_BYTES + off);
                const uint32_t first0 = (kb < NCHAIN && ks == 0) ? 0u : 1u;   // chain's first MMA
                const uint32_t first1 = (kb | ks) ? 1u : 0u;
                mma_bf16(acc0, ah, bh, idesc, first0);
                mma_bf16(acc1, ah, bm, idesc, first1);
                mma_bf16(acc1, am, bh, idesc, 1u);
                mma_bf16(acc1, ah, bl, idesc, 1u);
                mma_bf16(acc1, al, bh, idesc, 1u);
                mma_bf16(acc1, am, bm, idesc, 1u);
            }
            mma_commit(empty(s));      // the stage is free once these MMAs are done
        }
        mma_commit(done);              // all MMAs issued (possibly none if a wait failed)
    }
    __syncwarp();

    bool ok = mbar_wait(done, 0u);
    if (!ok) failed = 1;
    tc_fence_after();
    __syncthreads();
    const bool good = !failed;
    if (good) {
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        const int chains = nkb < NCHAIN ? nkb : NCHAIN;   // chains that received products
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
            float z0[32], z1[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(32 * c), z0);
            for (int ch = 1; ch < chains; ++ch) {
                tmem_ld32(tmem + lane_base + (uint32_t)(ch * BN + 32 * c), z1);
#pragma unroll
                for (int t = 0; t < 32; ++t) z0[t] = __fadd_rn(z0[t], z1[t]);
            }
            tmem_ld32(tmem + lane_base + (uint32_t)(NCHAIN * BN + 32 * c), z1);
#pragma unroll
            for (int t = 0; t < 32; ++t) z0[t] = __fadd_rn(z0[t], z1[t]);
            epi(c, z0);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (!good && threadIdx.x == 0 && a.status) atomicExch(a.status, 1);
    return good;
}

// Host: tensor map of a [rows][Kp] bf16 matrix, boxes of 64 x box_rows,
// 128-byte swizzle.
bool make_tmap_bf16(CUtensorMap* map, const void* base, int Kp, int rows, int box_rows = BM);

// ---------------------------------------------------------------------------
// Exact integer-slice GEMM (the tensor pipeline's rotation).
//
// Each operand row is scaled by a power of two s (s_d per particle, s_M per
// output j) such that every entry satisfies |v| < s / 2, and the exact value
// (d = x - o as a float pair, M from its FP64 copy) is written as four 7-bit
// integer slices,
//     v = s (V0 2^-7 + V1 2^-14 + V2 2^-21 + V3 2^-28 + r),
// |V0..V3| <= 64, |r| <= 1.01 2^-29 (successive round-to-nearest with exact
// steps, slicers below).  The slice products of weight w = s + t <= 3 are
// accumulated in four accumulators, one per weight:
//     acc0: D0 M0                        acc1: D0 M1 + D1 M0
//     acc2: D0 M2 + D1 M1 + D2 M0        acc3: D0 M3 + D1 M2 + D2 M1 + D3 M0
// (ten MMAs per K step).  Every product is an integer of magnitude at most
// 64^2 = 4096, so per k an accumulator gains at most 4 * 4096 = 16384; for
// D <= 1023 nonzero k every partial sum stays below 2^24 in magnitude, an FP32
// accumulator represents all of them exactly, and the accumulation is exact
// whatever the MMA datapath's alignment and rounding (24 bits suffice).  The
// products of weight 4 .. 6 and the remainders r are dropped and bounded: per k,
//     s_d s_M SLICE_DROP + SLICE_REM (s_M |d_k| + s_d |M_jk|).
// The epilogue joins the accumulators in FP32 from the smallest weight up,
// t = acc0 + 2^-7 acc1 + 2^-14 acc2 + 2^-21 acc3 (three rounded operations),
// and z = 2^-14 s_d s_M t exactly.
//
// The kernel is persistent and warp-specialised: one CTA per SM walks the
// tiles blockIdx.x, blockIdx.x + gridDim.x, ...; warp 0 issues the TMA copies
// (running ahead into the next tile while the current one computes), warp 1
// issues the MMAs and owns the tensor memory, warps 2..5 run the epilogue.
// Tensor memory holds two accumulator sets of 4 x 64 columns, so the
// epilogue of one tile overlaps the MMAs of the next.
constexpr int SBN = 64;                                     // output columns per tile
constexpr int SLICES = 4;
constexpr int SACC = 4;                                     // accumulators (one per weight)
constexpr int SPAIRS = 10;                                  // MMAs per K step
constexpr int S_A_BYTES = BM * BK * 2;                      // 16 KiB
constexpr int S_B_BYTES = SBN * BK * 2;                     // 8 KiB
constexpr int S_STAGE_BYTES = SLICES * (S_A_BYTES + S_B_BYTES);   // 96 KiB
constexpr int S_SMEM_BYTES = STAGES * S_STAGE_BYTES + 1024;
constexpr int S_ACC_COLS = SACC * SBN;                      // 256 columns per accumulator set
constexpr int S_TMEM_COLS = 2 * S_ACC_COLS;                 // two sets (a power of two)
constexpr int S_THREADS = 192;                              // TMA warp, MMA warp, four epilogue warps
constexpr int S_MAX_K = 1024;                               // padded K extent (D <= 1023 for exactness)
constexpr int S_MAX_D = 1023;
// weight 4..6: 3 * 64^2 * 2^-42 + 2 * 64^2 * 2^-49 + 64^2 * 2^-56, and 3 r^2
constexpr float SLICE_DROP = 3.04f * 0x1p-30f;              // per k, units of s_d s_M
constexpr float SLICE_REM = 1.01f * 0x1p-29f;               // per k, of s_M |d_k| + s_d |M_jk|

// Power-of-two scale s of a row with max |v| <= vmax (1 + 2^-22): every entry
// satisfies |v| < s / 2 (s = 1 if vmax is 0).
__host__ __device__ inline float slice_scale(float vmax)
{
    if (!(vmax > 0.f)) return 1.f;
    int e = 0;
    const float m = vmax * 2.f * (1.f + 0x1p-20f);                 // rounded up
    (void)frexpf(m, &e);                                            // m < 2^e
    return ldexpf(1.f, e);
}

// The four slices of u = u_hi + u_lo (an exact float pair, |u| < 1/2) as
// BF16 integers.  Each step keeps the rest exactly as a float pair: the
// rounded-off part of the high word is exact, a TwoSum renormalises, and the
// scaling by 128 is exact.  The rest after four slices is within 1.01 2^-29.
__device__ __forceinline__ void slice4_pair(float u_hi, float u_lo, __nv_bfloat16 (&o)[SLICES])
{
    float wh = __fmul_rn(u_hi, 128.f), wl = __fmul_rn(u_lo, 128.f);
#pragma unroll
    for (int q = 0; q < SLICES; ++q) {
        const float iq = rintf(wh);
        o[q] = __float2bfloat16_rn(iq);              // an integer of magnitude <= 64
        const float r = __fsub_rn(wh, iq);           // exact
        const float s = __fadd_rn(r, wl);            // TwoSum(r, wl)
        const float bb = __fsub_rn(s, r);
        const float e = __fadd_rn(__fsub_rn(r, __fsub_rn(s, bb)), __fsub_rn(wl, bb));
        wh = __fmul_rn(s, 128.f);
        wl = __fmul_rn(e, 128.f);
    }
}

// The same for an FP64 value u (|u| < 1/2): the steps are exact in FP64.
__device__ __forceinline__ void slice4_f64(double u, __nv_bfloat16 (&o)[SLICES])
{
    double w = __dmul_rn(u, 128.0);
#pragma unroll
    for (int q = 0; q < SLICES; ++q) {
        const double iq = rint(w);
        o[q] = __float2bfloat16_rn((float)iq);
        w = __dmul_rn(__dsub_rn(w, iq), 128.0);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ int vload(const int& v) { return *(volatile const int*)&v; }

// Tiles of the slice GEMM: (Np / BM) * (Jp / SBN) tiles numbered with the
// column tile varying fastest, so that CTAs working at the same time share
// their A slices through L2.  tile_m = t / (Jp / SBN), tile_n = t % (Jp / SBN).

// The slice GEMM over SLICES A planes [SLICES][Np][Kp] and B planes
// [SLICES][Jp][Kp] (Jp a multiple of SBN, Kp of BK, Kp <= S_MAX_K), every tile
// of the grid-stride walk.  Launch with S_THREADS threads and S_SMEM_BYTES of
// dynamic shared memory.  The epilogue functor gets epi.tile(tile_m, tile_n,
// row in tile) at the start of each tile, then (column block c of 32, t[32],
// em[32]) with t the joined accumulators and em the sum of the magnitudes of
// the three rounded partial sums.  Every wait is bounded; returns false (all
// threads) if one ran out.
template <class Epi>
__device__ __forceinline__ bool gemm_sliced_persistent(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                                       const GemmArgs& a, Epi& epi)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // full[STAGES] | empty[STAGES] | tmem full[2] | tmem empty[2] | done
    __shared__ __align__(8) uint64_t bars[2 * STAGES + 5];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nJt = a.Jp / SBN;
    const int ntiles = (a.Np / BM) * nJt;
    const int nkb = a.Kp / BK;
    const uint32_t sbase = smem_u32(smem);
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[STAGES + s]); };
    auto tfull = [&](int b) { return smem_u32(&bars[2 * STAGES + b]); };
    auto tempty = [&](int b) { return smem_u32(&bars[2 * STAGES + 2 + b]); };
    const uint32_t done = smem_u32(&bars[2 * STAGES + 4]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull(b), 1);
            mbar_init(tempty(b), 4);   // one arrival per epilogue warp
        }
        mbar_init(done, 1);
        fence_mbar_init();
        failed = 0;
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&tmem_slot), S_TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: per K block, the four A slices and the four B
            // slices; `it` counts K blocks over all tiles of this CTA
            int it = 0;
            for (int tile = blockIdx.x; tile < ntiles && !vload(failed); tile += gridDim.x) {
                const int m0 = (tile / nJt) * BM, n0 = (tile % nJt) * SBN;
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (it >= STAGES && !mbar_wait(empty(s), (uint32_t)((it / STAGES - 1) & 1))) {
                        failed = 1;
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full(s), S_STAGE_BYTES);
                    const uint32_t st = sbase + (uint32_t)(s * S_STAGE_BYTES);
                    for (int p = 0; p < SLICES; ++p) {
                        tma_load_2d(st + (uint32_t)(p * S_A_BYTES), tmA, kb * BK, p * a.Np + m0, full(s));
                        tma_load_2d(st + (uint32_t)(SLICES * S_A_BYTES + p * S_B_BYTES), tmB, kb * BK,
                                    p * a.Jp + n0, full(s));
                    }
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: the ten slice products into the four accumulators of
            // the tile's accumulator set (tiles alternate between the two)
            constexpr uint32_t idesc = idesc_bf16(BM, SBN);
            // (A slice, B slice, accumulator); the first product of each
            // accumulator starts it at the tile's first K step
            constexpr int PA[SPAIRS] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
            constexpr int PB[SPAIRS] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
            constexpr int PACC[SPAIRS] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
            constexpr int PLEAD[SPAIRS] = {1, 1, 0, 1, 0, 0, 1, 0, 0, 0};
            int it = 0, tl = 0;
            for (int tile = blockIdx.x; tile < ntiles && !vload(failed); tile += gridDim.x, ++tl) {
                const int buf = tl & 1;
                if (tl >= 2 && !mbar_wait(tempty(buf), (uint32_t)(((tl >> 1) - 1) & 1))) {
                    failed = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t accs = tmem + (uint32_t)(buf * S_ACC_COLS);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(full(s), (uint32_t)((it / STAGES) & 1))) {
                        failed = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + (uint32_t)(s * S_STAGE_BYTES);
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint32_t off = (uint32_t)(ks * 32);   // 16 bf16 along K
                        uint64_t ad[SLICES], bd[SLICES];
#pragma unroll
                        for (int p = 0; p < SLICES; ++p) {
                            ad[p] = sdesc_sw128(st + (uint32_t)(p * S_A_BYTES) + off);
                            bd[p] = sdesc_sw128(st + (uint32_t)(SLICES * S_A_BYTES + p * S_B_BYTES) + off);
                        }
                        const uint32_t first = (kb | ks) ? 1u : 0u;
#pragma unroll
                        for (int q = 0; q < SPAIRS; ++q)
                            mma_bf16(accs + (uint32_t)(PACC[q] * SBN), ad[PA[q]], bd[PB[q]], idesc,
                                     PLEAD[q] ? first : 1u);
                    }
                    mma_commit(empty(s));      // the stage is free once these MMAs are done
                }
                if (!ok) break;
                mma_commit(tfull(buf));        // the tile's accumulators are complete
            }
            // every MMA issued by this thread has completed once `done` fires
            mma_commit(done);
            if (!mbar_wait(done, 0u)) failed = 1;
        }
    } else {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31, one
        // particle per lane
        const int qtr = warp & 3;
        const int row = 32 * qtr + lane;
        const uint32_t lane_base = (uint32_t)(32 * qtr) << 16;
        int tl = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
            const int buf = tl & 1;
            const bool ok = mbar_wait(tfull(buf), (uint32_t)((tl >> 1) & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t accs = tmem + lane_base + (uint32_t)(buf * S_ACC_COLS);
            epi.tile(tile / nJt, tile % nJt, row);
#pragma unroll 1
            for (int c = 0; c < SBN / 32; ++c) {
                float t[32], em[32], v[32];
                tmem_ld32(accs + (uint32_t)(3 * SBN + 32 * c), t);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    t[q] = __fmul_rn(t[q], 0x1p-21f);   // exact
                    em[q] = 0.f;
                }
                // (accumulator, weight) from the smallest weight up; each step one
                // rounding (the scaled accumulator is exact)
                constexpr int JA[2] = {2, 1};
                constexpr float JW[2] = {0x1p-14f, 0x1p-7f};
#pragma unroll
                for (int st = 0; st < 2; ++st) {
                    tmem_ld32(accs + (uint32_t)(JA[st] * SBN + 32 * c), v);
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        t[q] = __fmaf_rn(v[q], JW[st], t[q]);
                        em[q] = __fadd_ru(em[q], fabsf(t[q]));
                    }
                }
                tmem_ld32(accs + (uint32_t)(32 * c), v);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    t[q] = __fadd_rn(v[q], t[q]);
                    em[q] = __fadd_ru(em[q], fabsf(t[q]));
                }
                epi(c, t, em);
            }
            // the accumulator set may be overwritten once all four warps have read it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(buf));
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, S_TMEM_COLS);
    }
    const bool good = !vload(failed);
    if (!good && threadIdx.x == 0 && a.status) atomicExch(a.status, 1);
    return good;
}

}  // namespace tc
}  // namespace psso
