// bat_stream.cuh -- streaming step kernel of the batched throughput pipeline
// for wide rows (more than 128 variables, unrotated functions).
//
// One warp per particle walks its row one 32-chunk slice at a time: Eq. 2.1
// for the slice (the same draws as the persistent kernel), the slice stored,
// its fitness terms added to the lanes' running sums.  Registers hold one
// slice instead of the whole row, so many more warps fit on an SM to hide the
// row loads.  A lane meets its variables in ascending order, as in the
// whole-row code, so the FP64 value keeps the oracle's summation order bit for
// bit: the only term that needs the next slice -- Rosenbrock's last term of
// lane 31, which needs the first variable of lane 0's next chunk -- is added
// at the start of the next slice.  The FP32 value and its bound are those of
// the whole-row FP32 path (same terms, same summation depth).  An accepted
// row is copied to P by reading back the stored slices.
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

template <class Pos, bool F32R>
__global__ void __launch_bounds__(256, 4) bat_stream(const BatParams p)
{
    using Val = typename std::conditional<F32R, float, double>::type;
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t nwarps = wpb * gridDim.x;
    const int64_t g = *p.gen;
    const uint32_t gg = (uint32_t)g;
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
        if (!PSSO_CHK(i >= 0 && i < d.N, CHK_BAT_ROW, gid)) continue;
        const Hot in = hot_of(d);
        const int fn = in.fn;
        const int nq = (in.nchunks + 31) >> 5;
        Pos* xr = static_cast<Pos*>(d.X) + i * in.Dp;
        Pos* prow = static_cast<Pos*>(d.P) + i * in.Dp;
        const Pos* gs = static_cast<const Pos*>(d.gbrow);
        const uint32_t ctr3r = TAG_RHO | (in.sid << 8), ctr3f = TAG_FRESH | (in.sid << 8);
        StreamAcc<F32R> sa;
        bool eqp = true;
        Val pend_z = Val(0);
        int pend_j = -1;               // lane 31: Rosenbrock term waiting for the next slice
        for (int q = 0; q < nq; ++q) {
            const int c = lane + 32 * q;
            const bool has = c < in.nchunks;
            Pos x[4] = {Pos(0), Pos(0), Pos(0), Pos(0)};
            if (has) {
                const int nvalid = min(4, in.D - 4 * c);
                const uint32_t valid = (1u << nvalid) - 1u;
                if (g == 0) {
                    fresh_chunk(x, valid, (uint32_t)c, (uint32_t)i + in.i_base, 0u, TAG_INIT, in);
                } else {
                    // the slice's loads first: the draws below do not depend on
                    // them and cover their latency
                    Pos xo[4], po[4], go[4];
                    // xo: the third interval's source, go: the first's (Eq. 2.1 as printed
                    // swaps them: keep x first, gBest third)
                    ld4((in.order ? gs : xr) + 4 * c, xo);
                    ld4(prow + 4 * c, po);
                    ld4((in.order ? xr : gs) + 4 * c, go);
                    const uint4 rb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3r), in.k0, in.k1);
                    uint4 fb = make_uint4(0u, 0u, 0u, 0u);
                    if (sizeof(Pos) == 4)
                        fb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3f), in.k0, in.k1);
                    uint32_t nf = 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t r = word_of(rb, m);
                        const bool lg = (r < in.Tg32) || (in.tfull & 1u);
                        const bool lp = (r < in.Tp32) || (in.tfull & 2u);
                        const bool lw = (r < in.Tw32) || (in.tfull & 4u);
                        x[m] = lg ? go[m] : lp ? po[m] : xo[m];
                        if (!lw) nf |= 1u << m;
                    }
                    nf &= valid;
                    if (nf) {
                        if constexpr (sizeof(Pos) == 4) {
#pragma unroll
                            for (int m = 0; m < 4; ++m)
                                if (nf & (1u << m)) x[m] = (Pos)fresh_f32(word_of(fb, m), in);
                        } else {
                            fresh_chunk(x, nf, (uint32_t)c, (uint32_t)i + in.i_base, gg, TAG_FRESH, in);
                        }
                    }
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (m >= nvalid) x[m] = Pos(0);
                        eqp = eqp && same_bits(x[m], po[m]);
                    }
                }
                st4(xr + 4 * c, x);
            }
            // fitness terms of the slice (the shift is padded to Dp values)
            Val dv[4], ov[4] = {Val(0), Val(0), Val(0), Val(0)};
            if (has) {
                if constexpr (F32R) ld4(in.o32 + 4 * c, ov);
                else ld4(in.o64 + 4 * c, ov);
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                if constexpr (F32R) dv[m] = (has && j < in.D) ? __fsub_rn((float)x[m], ov[m]) : 0.f;
                else dv[m] = (has && j < in.D) ? __dsub_rn((double)x[m], ov[m]) : 0.0;
            }
            Val next = Val(0);
            if (fn == FN_ROSENBROCK) {
                next = __shfl_down_sync(0xffffffffu, dv[0], 1);
                const Val first0 = __shfl_sync(0xffffffffu, dv[0], 0);
                if (lane == 31 && pend_j >= 0) {
                    sa.term(fn, in, pend_j, pend_z, first0);
                    pend_j = -1;
                }
            }
            if (has) {
                // the four terms of the chunk, one function dispatch per chunk
                // (the switch inside the term is resolved at compile time)
                auto terms = [&](auto fc) {
                    constexpr int F = decltype(fc)::value;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int j = 4 * c + m;
                        if (j >= in.D) break;
                        if (F == FN_ROSENBROCK && m == 3 && lane == 31) {
                            pend_j = j;
                            pend_z = dv[3];
                            continue;
                        }
                        sa.term(F, in, j, dv[m], m < 3 ? dv[(m + 1) & 3] : next);
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
        }
        // lane 31's pending term has no next slice: it is the row's last variable (no term)
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
            __syncwarp();
            for (int c = lane; c < in.nchunks; c += 32) {
                Pos v[4];
                ld4(xr + 4 * c, v);
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
    if (op == 3) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bat_stream<Pos, F32R>, block, 0);
    bat_stream<Pos, F32R><<<grid, block, 0, s>>>(*p);
    return cudaGetLastError();
}

}  // namespace psso
