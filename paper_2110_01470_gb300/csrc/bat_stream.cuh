// bat_stream.cuh -- streaming step kernel of the batched throughput pipeline
// for wide rows (more than 128 variables, unrotated functions).
//
// One warp per particle; the row is staged in the warp's shared memory and
// processed in three passes:
//   1. Eq. 2.1 slice by slice (32 chunks of 4 variables per slice, the same
//      draws as the persistent kernel): the interval draw of every chunk,
//      the selected source values into the staged row; a chunk with variables
//      in the last interval (about a third of them) queues a request for its
//      fresh-value block, and its staged values there hold the pBest value
//      for the row-equality test;
//   2. the queued fresh-value blocks, 32 per round, one per lane: the Philox
//      work of the last branch is paid only for the chunks that need it;
//   3. slice by slice again: the staged row stored to X and its fitness terms
//      added to the lanes' running sums.
// A lane meets its variables in ascending order, as in the whole-row code, so
// the FP64 value keeps the oracle's summation order bit for bit; the FP32
// value and its bound are those of the whole-row FP32 path (same terms, same
// summation depth).  An accepted row is copied to P from the staged row.
#pragma once
#include <type_traits>

#include "sso_kernel.cuh"

namespace psso {

// Running sums of one lane (FP64: the oracle's forms; FP32: with the terms'
// error bounds where the function needs them).
template <bool F32R>
struct StreamAcc;

template <>
struct StreamAcc<false> {
    double acc = 0.0, acc2 = 0.0;
    __device__ __forceinline__ void term(int fn, const Hot& in, int j, double z, double d1)
    {
        switch (fn) {
        case FN_SPHERE: acc = __fma_rn(z, z, acc); break;
        case FN_ELLIPSOID: acc = __fma_rn(__ldg(in.w64 + j), __dmul_rn(z, z), acc); break;
        case FN_RASTRIGIN: {
            const double s2 = sinpi_sq_f64(z);
            acc = __dadd_rn(acc, __fma_rn(z, z, __dmul_rn(20.0, s2)));
            break;
        }
        case FN_ROSENBROCK:
            if (j < in.D - 1) {
                const double a0 = __dadd_rn(z, 1.0), a1 = __dadd_rn(d1, 1.0);
                const double u = __fma_rn(-a0, a0, a1);
                acc = __dadd_rn(acc, __fma_rn(__dmul_rn(100.0, u), u, __dmul_rn(z, z)));
            }
            break;
        default: {   // Ackley
            acc = __fma_rn(z, z, acc);
            const double s = sinpi_reduced_f64(__dsub_rn(z, rint(z)));
            acc2 = __fma_rn(s, s, acc2);
            break;
        }
        }
    }
    __device__ __forceinline__ double finish(int fn, const Hot& in)
    {
        for (int off = 16; off > 0; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
        if (fn != FN_ACKLEY) return acc;
        for (int off = 16; off > 0; off >>= 1) acc2 = __dadd_rn(acc2, __shfl_xor_sync(0xffffffffu, acc2, off));
        const double Dd = (double)in.D;
        const double A = __dsqrt_rn(__ddiv_rn(acc, Dd));
        const double B = expm1_f64(__dmul_rn(-0.2, A));
        const double C = expm1_f64(__dmul_rn(-2.0, __ddiv_rn(acc2, Dd)));
        return -__dadd_rn(__dmul_rn(20.0, B), __dmul_rn(0x1.5bf0a8b145769p+1, C));   // e
    }
};

template <>
struct StreamAcc<true> {
    float acc = 0.f, acc2 = 0.f, accE = 0.f, accZ = 0.f;
    __device__ __forceinline__ void term(int fn, const Hot& in, int j, float z, float d1)
    {
        switch (fn) {
        case FN_SPHERE: acc = __fadd_rn(acc, __fmul_rn(z, z)); break;
        case FN_ELLIPSOID: acc = __fadd_rn(acc, __fmul_rn(__ldg(in.w32 + j), __fmul_rn(z, z))); break;
        case FN_RASTRIGIN: {
            const float s = sinpi_reduced_f32(__fsub_rn(z, rintf(z)));
            acc = __fadd_rn(acc, __fmaf_rn(z, z, __fmul_rn(20.f, __fmul_rn(s, s))));
            break;
        }
        case FN_ROSENBROCK:
            if (j < in.D - 1) {
                const float s0 = __fadd_rn(z, 2.f);
                const float u = __fmaf_rn(-z, s0, d1);
                const float d2 = __fmul_rn(z, z);
                const float t = __fmaf_rn(__fmul_rn(100.f, u), u, d2);
                acc = __fadd_rn(acc, t);
                const float e0 = 1.01f * U32 * fabsf(z), e1 = 1.01f * U32 * fabsf(d1);
                const float as0 = fabsf(s0);
                const float eu = 1.01f * (U32 * fabsf(u) + e1 + fabsf(z) * (U32 * as0 + e0) + (1.01f * as0 + e0) * e0);
                float et = 100.f * eu * (2.f * fabsf(u) + eu) + 3.f * U32 * 100.f * u * u + 3.1f * U32 * d2 + U32 * t;
                const float a0 = fabsf(z) + 1.f, a1 = fabsf(d1) + 1.f;
                const float eu64 = 0x1p-51f * (a1 + 2.f * a0 * a0 + fabsf(u) + 2.f);
                et += 200.f * fabsf(u) * eu64 + 100.f * eu64 * eu64 + 0x1p-50f * t;
                accE = __fadd_rn(accE, et);
            }
            break;
        default: {   // Ackley
            acc = __fadd_rn(acc, __fmul_rn(z, z));
            const float s = sinpi_reduced_f32(__fsub_rn(z, rintf(z)));
            acc2 = __fadd_rn(acc2, __fmul_rn(s, s));
            accZ = __fadd_rn(accZ, fabsf(z));
            break;
        }
        }
    }
    // FP32 value and bound; nq = chunks per lane (summation depth 4 nq, then
    // 5 butterfly levels).
    __device__ __forceinline__ Fit32 finish(int fn, const Hot& in, int nq)
    {
        for (int off = 16; off > 0; off >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, off));
        const float csum = (float)(4 * nq) + 5.f + 2.f;
        Fit32 r;
        switch (fn) {
        case FN_SPHERE:
            r.f = acc;
            r.E = 1.1f * (3.1f + csum) * U32 * acc;
            break;
        case FN_ELLIPSOID:
            r.f = acc;
            r.E = 1.1f * (5.2f + csum) * U32 * acc;
            break;
        case FN_RASTRIGIN:
            r.f = acc;
            r.E = 1.1f * (2.f * SINPI32_ERR_U + 3.f + 16.1f + 1.f + csum) * U32 * acc;
            break;
        case FN_ROSENBROCK:
            for (int off = 16; off > 0; off >>= 1) accE = __fadd_rn(accE, __shfl_xor_sync(0xffffffffu, accE, off));
            r.f = acc;
            r.E = 1.1f * (accE + csum * U32 * acc);
            break;
        default: {   // Ackley
            for (int off = 16; off > 0; off >>= 1) {
                acc2 = __fadd_rn(acc2, __shfl_xor_sync(0xffffffffu, acc2, off));
                accZ = __fadd_rn(accZ, __shfl_xor_sync(0xffffffffu, accZ, off));
            }
            const float Df = (float)in.D;
            const float A = __fsqrt_rn(__fdiv_rn(acc, Df));
            const float B = expm1_f32(__fmul_rn(-0.2f, A));
            const float C = expm1_f32(__fmul_rn(-2.f, __fdiv_rn(acc2, Df)));
            const float f1 = __fmul_rn(-20.f, B), f2 = __fmul_rn(-0x1.5bf0a8p+1f, C);
            r.f = __fadd_rn(f1, f2);
            const float relS = (3.1f + csum) * U32;
            const float EQ = 1.01f * 3.14159275f * U32 * accZ + (2.f * SINPI32_ERR_U + 1.f + csum) * U32 * acc2;
            r.E = 1.1f * (0.5f * relS * f1 + (EXPM1F_ERR_U + 6.f) * U32 * f1 + (2.f * 2.7182818f / Df) * EQ +
                          (EXPM1F_ERR_U + 8.f) * U32 * f2 + U32 * r.f);
            acc = r.f;
            break;
        }
        }
        r.E = __fadd_ru(r.E, 0x1p-40f * (acc + accE));
        return r;
    }
};

// Shared memory of one warp: the staged row (1024 positions) and the queue of
// fresh-value requests (chunk | mask << 8, at most 256).
constexpr int STREAM_ROW = 1024;
template <class Pos>
__host__ __device__ constexpr size_t stream_smem_per_warp()
{
    return (size_t)STREAM_ROW * sizeof(Pos) + 256 * sizeof(uint32_t);
}

template <class Pos, bool F32R>
__global__ void __launch_bounds__(256, 4) bat_stream(const BatParams p)
{
    using Val = typename std::conditional<F32R, float, double>::type;
    extern __shared__ __align__(16) unsigned char bs_smem[];
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t nwarps = wpb * gridDim.x;
    const int64_t g = *p.gen;
    const uint32_t gg = (uint32_t)g;
    Pos* const row = reinterpret_cast<Pos*>(bs_smem + (threadIdx.x >> 5) * stream_smem_per_warp<Pos>());
    uint32_t* const req = reinterpret_cast<uint32_t*>(row + STREAM_ROW);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t gid = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); gid < p.total; gid += nwarps) {
        int lo = 0, hi = p.n_ids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(p.first + mid) <= gid) lo = mid;
            else hi = mid - 1;
        }
        const int k = __ldg(p.ids + lo);
        const int64_t i = gid - __ldg(p.first + lo);
        const InstDev& d = p.inst[k];
        if (!PSSO_CHK(i >= 0 && i < d.N && d.Dp <= STREAM_ROW, CHK_BAT_ROW, gid)) continue;
        const Hot in = hot_of(d);
        const int fn = in.fn;
        const int nq = (in.nchunks + 31) >> 5;
        const uint32_t ii = (uint32_t)i + in.i_base;
        Pos* xr = static_cast<Pos*>(d.X) + i * in.Dp;
        Pos* prow = static_cast<Pos*>(d.P) + i * in.Dp;
        const Pos* gs = static_cast<const Pos*>(d.gbrow);
        const uint32_t ctr3r = TAG_RHO | (in.sid << 8);
        bool eqp = true;
        __syncwarp();     // the previous row's staged values are consumed

        // ---- pass 1: the interval draws; fresh-value requests --------------------------
        int nreq = 0;     // warp-uniform
        for (int q = 0; q < nq; ++q) {
            const int c = lane + 32 * q;
            uint32_t nf = 0;
            if (c < in.nchunks) {
                const int nvalid = min(4, in.D - 4 * c);
                const uint32_t valid = (1u << nvalid) - 1u;
                Pos x[4] = {Pos(0), Pos(0), Pos(0), Pos(0)};
                if (g == 0) {
                    fresh_chunk(x, valid, (uint32_t)c, ii, 0u, TAG_INIT, in);
                } else {
                    Pos xo[4], po[4], go[4];
                    // xo: the third interval's source, go: the first's (Eq. 2.1 as printed
                    // swaps them: keep x first, gBest third)
                    ld4((in.order ? gs : xr) + 4 * c, xo);
                    ld4(prow + 4 * c, po);
                    ld4((in.order ? xr : gs) + 4 * c, go);
                    const uint4 rb = philox10(make_uint4((uint32_t)c, ii, gg, ctr3r), in.k0, in.k1);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t r = word_of(rb, m);
                        const bool lg = (r < in.Tg32) || (in.tfull & 1u);
                        const bool lp = (r < in.Tp32) || (in.tfull & 2u);
                        const bool lw = (r < in.Tw32) || (in.tfull & 4u);
                        // a variable of the last interval holds its pBest value until
                        // pass 2 compares and replaces it
                        x[m] = lg ? go[m] : (lp || !lw) ? po[m] : xo[m];
                        if (!lw) nf |= 1u << m;
                    }
                    nf &= valid;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (m >= nvalid) x[m] = Pos(0);
                        if (!(nf & (1u << m))) eqp = eqp && same_bits(x[m], po[m]);
                    }
                }
                st4(row + 4 * c, x);
            }
            const unsigned want = __ballot_sync(0xffffffffu, nf != 0u);
            if (nf) req[nreq + __popc(want & lt_mask)] = (uint32_t)c | (nf << 8);
            nreq += __popc(want);
        }
        __syncwarp();

        // ---- pass 2: the queued fresh-value blocks, one per lane and round ------------------
        for (int base = 0; base < nreq; base += 32) {
            const int e = base + lane;
            if (e < nreq) {
                const uint32_t rq = req[e];
                const uint32_t c = rq & 0xffu, nf = rq >> 8;
                Pos fv[4], pv[4];
                ld4(row + 4 * c, pv);     // the pBest values held in pass 1
                fresh_chunk(fv, nf, c, ii, gg, TAG_FRESH, in);
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (nf & (1u << m)) {
                        eqp = eqp && same_bits(fv[m], pv[m]);
                        pv[m] = fv[m];
                    }
                st4(row + 4 * c, pv);
            }
        }
        __syncwarp();

        // ---- pass 3: X and the fitness terms --------------------------------------------------
        StreamAcc<F32R> sa;
        for (int q = 0; q < nq; ++q) {
            const int c = lane + 32 * q;
            if (c >= in.nchunks) continue;
            Pos x[4];
            ld4(row + 4 * c, x);
            st4(xr + 4 * c, x);
            // fitness terms of the chunk (the shift is padded to Dp values)
            Val dv[4], ov[4];
            if constexpr (F32R) ld4(in.o32 + 4 * c, ov);
            else ld4(in.o64 + 4 * c, ov);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                if constexpr (F32R) dv[m] = (j < in.D) ? __fsub_rn((float)x[m], ov[m]) : 0.f;
                else dv[m] = (j < in.D) ? __dsub_rn((double)x[m], ov[m]) : 0.0;
            }
            // Rosenbrock's last term of the chunk needs the next chunk's first variable
            Val next = Val(0);
            if (fn == FN_ROSENBROCK && 4 * c + 4 < in.D) {
                if constexpr (F32R) next = __fsub_rn((float)row[4 * c + 4], __ldg(in.o32 + 4 * c + 4));
                else next = __dsub_rn((double)row[4 * c + 4], __ldg(in.o64 + 4 * c + 4));
            }
            // the four terms of the chunk, one function dispatch per chunk
            // (the switch inside the term is resolved at compile time)
            auto terms = [&](auto fc) {
                constexpr int F = decltype(fc)::value;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int j = 4 * c + m;
                    if (j >= in.D) break;
                    sa.term(F, in, j, dv[m], m < 3 ? dv[m + 1] : next);
                }
            };
            switch (fn) {
            case FN_SPHERE: terms(std::integral_constant<int, FN_SPHERE>()); break;
            case FN_ELLIPSOID: terms(std::integral_constant<int, FN_ELLIPSOID>()); break;
            case FN_RASTRIGIN: terms(std::integral_constant<int, FN_RASTRIGIN>()); break;
            case FN_ROSENBROCK: terms(std::integral_constant<int, FN_ROSENBROCK>()); break;
            default: terms(std::integral_constant<int, FN_ACKLEY>()); break;
            }
        }
        const bool same_row = (g > 0) && __all_sync(0xffffffffu, eqp);
        bool accept, wstate = true, undecided = false;
        double f64v = 0.0;
        float lo32 = 0.f, hi32 = 0.f;
        int has64 = 0;
        if constexpr (!F32R) {
            const double f = sa.finish(fn, in);
            const double pf = (g == 0) ? f : d.pf64[i];
            accept = (g == 0) || (f <= pf);
            f64v = accept ? f : pf;
            has64 = 1;
        } else {
            const Fit32 r = sa.finish(fn, in, nq);
            lo32 = __fsub_rd(r.f, r.E);
            hi32 = __fadd_ru(r.f, r.E);
            if (g == 0) {
                accept = true;
            } else if (same_row) {
                accept = true;
                wstate = false;
            } else if (hi32 < d.plo[i]) {
                accept = true;
            } else if (lo32 > d.phi[i]) {
                accept = false;
            } else {
                accept = false;
                undecided = true;
            }
        }
        unsigned long long n_rck = 0;
        if (F32R && undecided) {
            __syncwarp();
            const Resolved rs = resolve_f64<Pos, 8>(in, xr, prow, (d.pflag[i] & 1u) != 0, d.pf64[i], lane,
                                                    0xffffffffu);
            accept = rs.accept;
            has64 = 1;
            f64v = rs.f64v;
            lo32 = rs.lo;
            hi32 = rs.hi;
            n_rck = rs.rck;
            if (lane == 0 && rs.cachep) {
                d.pf64[i] = rs.cachef;
                d.pflag[i] = 1u;
                d.plo[i] = rs.lo;
                d.phi[i] = rs.hi;
            }
        }
        if (accept && wstate) {
            for (int c = lane; c < in.nchunks; c += 32) {
                Pos v[4];
                ld4(row + 4 * c, v);
                st4(prow + 4 * c, v);
            }
            if (lane == 0) {
                d.pver[i] = gg;
                d.pf64[i] = has64 ? f64v : 0.0;
                if (F32R) {
                    d.pflag[i] = (uint32_t)has64;
                    d.plo[i] = lo32;
                    d.phi[i] = hi32;
                }
            }
        }
        if (lane == 0) {
            if (accept) atomicAdd(&p.cnt[k].acc, 1ull);
            if (n_rck) atomicAdd(&p.cnt[k].rck, n_rck);
        }
    }
}

template <class Pos, bool F32R>
inline cudaError_t bat_stream_entry(int op, const BatParams* p, int grid, int block, cudaStream_t s, int* out)
{
    const size_t smem = (size_t)(block >> 5) * stream_smem_per_warp<Pos>();
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(bat_stream<Pos, F32R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (op == 3) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bat_stream<Pos, F32R>, block, smem);
    bat_stream<Pos, F32R><<<grid, block, smem, s>>>(*p);
    return cudaGetLastError();
}

}  // namespace psso
