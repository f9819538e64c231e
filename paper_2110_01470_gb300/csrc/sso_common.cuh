// sso_common.cuh -- device building blocks of the SSO generation kernel:
// chunk loads/stores, fresh values, FP64 / FP32 fitness, block reductions.
//
// The generation kernel (sso_kernel.cuh) is summarised here for context.
//
// One cooperative launch runs generations g_begin..g_end of every instance.
// Each block owns one or more "units" (a contiguous particle range of one
// instance) for the whole launch.  Per generation and unit:
//
//   A  gBest of generation g-1 (Alg. 4).  A unit that is the whole swarm keeps
//      it in shared memory.  Otherwise every block of the instance reads the
//      per-block records of g-1 (each 64-bit word tagged with the generation, so
//      no lock or atomic is needed), takes the lowest-index arg-min, and copies
//      the winning row from the winner's double-buffered snapshot only if the
//      winner (index, row version) changed.
//   B  For every owned particle (a group of G lanes; lane l owns variable
//      chunks l, l+32, ... of 4 variables): the stepwise update of Eq. 2.1 with
//      a Philox-4x32-10 block per chunk, the fitness (Kernel Function (E)), and
//      the pBest update of Alg. 3 (f <= pF).  In FP32 mode every comparison the
//      FP32 error bound cannot decide is re-evaluated in FP64 in the oracle's
//      order.
//   C  The unit's lowest-index arg-min of pBest fitness.
//   D  Whole-swarm unit: update the shared gBest row.  Otherwise publish the
//      unit's winner row (double-buffered by generation parity) and record.
//
// The only coupling between blocks is the per-generation record exchange of
// step A/D: the paper's pBest / gBest "resource preemption" (abstract,
// Alg. 3-4) cannot occur because every block writes only its own slots.
#pragma once
#include <algorithm>
#include <cfloat>
#include <cstdint>

#include "devmath.cuh"
#include "psso_internal.h"

namespace psso {

constexpr float U32 = 0x1p-24f;

// ---------------------------------------------------------------------------
// Vector loads / stores of one chunk (4 positions, 16 or 32 bytes).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4])
{
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4_cg(const float* p, float (&v)[4])
{
    const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4_cg(const double* p, double (&v)[4])
{
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4])
{
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v)
{
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
__device__ __forceinline__ bool same_bits(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// The per-particle fields of an instance descriptor, as a small value type
// that the inlined hot path keeps in registers.
struct Hot {
    int fn, D, Dp, nchunks, G, maxc;
    uint32_t Tg32, Tp32, Tw32;    // thresholds, saturated at 2^32 - 1
    uint32_t tfull;               // bit 0/1/2: Tg/Tp/Tw equal 2^32 (always taken)
    uint32_t k0, k1, sid;
    uint32_t order;               // 1: Eq. 2.1 as printed (first interval keeps x, third takes gBest)
    uint32_t i_base;              // draws are keyed by particle index i_base + local index
    float S32, L32, lbf, ubf;
    double lb, ub, span;
    const double* o64;
    const float* o32;
    const double* w64;
    const float* w32;
    const double* M64;   // rotation, row-major D x D (rotated functions only)
    const float* M32;    // the same rounded to float
    const float* M32lo;  // float(M - M32) (the compensated FP32 rotation)
};

__device__ __forceinline__ Hot hot_of(const InstDev& d)
{
    Hot h;
    h.fn = d.fn; h.D = d.D; h.Dp = d.Dp; h.nchunks = d.nchunks; h.G = d.G; h.maxc = d.maxc;
    h.Tg32 = d.Tg >= 0x100000000ULL ? 0xffffffffu : (uint32_t)d.Tg;
    h.Tp32 = d.Tp >= 0x100000000ULL ? 0xffffffffu : (uint32_t)d.Tp;
    h.Tw32 = d.Tw >= 0x100000000ULL ? 0xffffffffu : (uint32_t)d.Tw;
    h.tfull = (d.Tg >= 0x100000000ULL ? 1u : 0u) | (d.Tp >= 0x100000000ULL ? 2u : 0u) |
              (d.Tw >= 0x100000000ULL ? 4u : 0u);
    h.k0 = d.k0; h.k1 = d.k1; h.sid = d.sid; h.order = d.order; h.i_base = d.i_base;
    h.S32 = d.S32; h.L32 = d.L32; h.lbf = d.lbf; h.ubf = d.ubf;
    h.lb = d.lb; h.ub = d.ub; h.span = d.span;
    h.o64 = d.o64; h.o32 = d.o32; h.w64 = d.w64; h.w32 = d.w32;
    h.M64 = d.M64; h.M32 = d.M32; h.M32lo = d.M32lo;
    return h;
}

// ---------------------------------------------------------------------------
// Fresh values (last branch of Eq. 2.1; the initial population).
__device__ __forceinline__ float fresh_f32(uint32_t w, const Hot& in)
{
    const float u = __fmul_rn((float)(w >> 8), 0x1p-24f);
    float x = __fmaf_rn(in.S32, u, in.L32);
    x = (x < in.lbf) ? in.lbf : x;
    x = (x > in.ubf) ? in.ubf : x;
    return x;
}
__device__ __forceinline__ double fresh_f64(uint32_t lo, uint32_t hi, const Hot& in)
{
    const uint64_t m = ((((uint64_t)hi) << 32) | lo) >> 11;
    const double u = __dmul_rn(__ull2double_rn(m), 0x1p-53);
    double x = __fma_rn(in.span, u, in.lb);
    x = (x < in.lb) ? in.lb : x;
    x = (x > in.ub) ? in.ub : x;
    return x;
}

// Fresh values for the chunk's variables selected by `mask` (bit m = variable 4c+m).
__device__ __forceinline__ void fresh_chunk(float (&v)[4], uint32_t mask, uint32_t c, uint32_t i,
                                            uint32_t g, uint32_t tag, const Hot& in)
{
    const uint4 w = philox10(make_uint4(c, i, g, tag | (in.sid << 8)), in.k0, in.k1);
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (mask & (1u << m)) v[m] = fresh_f32(word_of(w, m), in);
}
__device__ __forceinline__ void fresh_chunk(double (&v)[4], uint32_t mask, uint32_t c, uint32_t i,
                                            uint32_t g, uint32_t tag, const Hot& in)
{
    if (mask & 3u) {
        const uint4 w = philox10(make_uint4(2u * c, i, g, tag | (in.sid << 8)), in.k0, in.k1);
        if (mask & 1u) v[0] = fresh_f64(w.x, w.y, in);
        if (mask & 2u) v[1] = fresh_f64(w.z, w.w, in);
    }
    if (mask & 12u) {
        const uint4 w = philox10(make_uint4(2u * c + 1u, i, g, tag | (in.sid << 8)), in.k0, in.k1);
        if (mask & 4u) v[2] = fresh_f64(w.x, w.y, in);
        if (mask & 8u) v[3] = fresh_f64(w.z, w.w, in);
    }
}

// ---------------------------------------------------------------------------
// FP64 fitness of one particle held by a group of G lanes (x: the lane's
// chunks lane_g + 32 q).  Order: per-lane partials in ascending variable index
// from +0.0, then an xor butterfly -- bit-identical to the oracle's 32-lane
// order, since lanes beyond the group hold no variables (their partial is +0.0).
__device__ __forceinline__ bool is_rotated(int fn) { return fn >= FN_ROT_ELLIPSOID && fn <= FN_ROT_ACKLEY; }
// Table 3.2's f3, f7, f8, f9: FP64 fitness only.
__device__ __forceinline__ bool is_fp64_only(int fn) { return fn >= FN_SCHWEFEL12; }
// Function whose terms a rotated function applies to z = M (x - o).
__device__ __forceinline__ int base_fn(int fn)
{
    return fn == FN_ROT_ELLIPSOID ? FN_ELLIPSOID
         : fn == FN_ROT_RASTRIGIN ? FN_RASTRIGIN
         : fn == FN_ROT_ACKLEY ? FN_ACKLEY : fn;
}

// z = M d, d = x - o, for the group's own variables (lane_g owns chunks
// lane_g + 32 q): z_j = sum_k M_jk d_k with k ascending from +0.0 by fma, each
// d_k broadcast from the lane that holds it -- the oracle's order.
template <class T, int MAXC>
struct RowBuf {
    T v[MAXC][4];
};

template <class Pos, int MAXC>
__device__ __noinline__ void rot_matvec64_impl(const Hot& in, const RowBuf<Pos, MAXC>& xb, int lane_g,
                                               unsigned gmask, int G, RowBuf<double, MAXC>& zb)
{
    const auto& x = xb.v;
    auto& z = zb.v;
    const int D = in.D;
    double d[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane_g + 32 * q) + m;
            d[q][m] = (j < D) ? __dsub_rn((double)x[q][m], __ldg(in.o64 + j)) : 0.0;
            z[q][m] = 0.0;
        }
#pragma unroll
    for (int qk = 0; qk < MAXC; ++qk) {
        for (int l = 0; l < G; ++l) {
            if (128 * qk + 4 * l >= D) break;
#pragma unroll
            for (int mk = 0; mk < 4; ++mk) {
                const int k = 128 * qk + 4 * l + mk;
                const double dk = __shfl_sync(gmask, d[qk][mk], l, G);
                if (k < D) {
#pragma unroll
                    for (int q = 0; q < MAXC; ++q)
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int j = 4 * (lane_g + 32 * q) + m;
                            if (j < D) z[q][m] = __fma_rn(__ldg(in.M64 + (size_t)j * D + k), dk, z[q][m]);
                        }
                }
            }
        }
    }
}

// The matvecs are out of line (one copy per width instead of one per call
// site); the rows go through small buffers so that the callers' arrays stay
// in registers.
template <class Pos, int MAXC>
__device__ __forceinline__ void rot_matvec64(const Hot& in, const Pos (&x)[MAXC][4], int lane_g,
                                             unsigned gmask, int G, double (&z)[MAXC][4])
{
    RowBuf<Pos, MAXC> xb;
    RowBuf<double, MAXC> zb;
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) xb.v[q][m] = x[q][m];
    rot_matvec64_impl<Pos, MAXC>(in, xb, lane_g, gmask, G, zb);
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) z[q][m] = zb.v[q][m];
}

template <class Pos, int MAXC, bool ROT>
__device__ __forceinline__ double fit64_impl(const Hot& in, const Pos (&x)[MAXC][4], int lane_g,
                                             unsigned gmask, int G)
{
    const int D = in.D, nch = in.nchunks;
    const bool rot = ROT && is_rotated(in.fn);
    const int fn = base_fn(in.fn);
    double zr[MAXC][4];
    if (rot) rot_matvec64<Pos, MAXC>(in, x, lane_g, gmask, G, zr);
    double acc = 0.0, acc2 = 0.0;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
        double dn = 0.0;   // Rosenbrock: d of variable 4c+4 (first of chunk c+1)
        if (fn == FN_ROSENBROCK) {
            const double first = (c < nch) ? __dsub_rn((double)x[q][0], __ldg(in.o64 + 4 * c)) : 0.0;
            dn = __shfl_down_sync(gmask, first, 1, G);
            if (G == 32 && q + 1 < MAXC) {
                const int cn = c + 32;
                const double nxt = (cn < nch) ? __dsub_rn((double)x[(q + 1) % MAXC][0],
                                                          __ldg(in.o64 + 4 * cn))
                                              : 0.0;
                const double wrap = __shfl_sync(gmask, nxt, 0, 32);
                if (lane_g == 31) dn = wrap;
            }
        }
        if (c < nch) {
            double dv[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                dv[m] = rot ? zr[q][m] : (j < D) ? __dsub_rn((double)x[q][m], __ldg(in.o64 + j)) : 0.0;
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                if (j >= D) break;
                const double z = dv[m];
                switch (fn) {
                case FN_SPHERE:
                    acc = __fma_rn(z, z, acc);
                    break;
                case FN_ELLIPSOID:
                    acc = __fma_rn(__ldg(in.w64 + j), __dmul_rn(z, z), acc);
                    break;
                case FN_RASTRIGIN: {
                    const double s2 = sinpi_sq_f64(z);
                    acc = __dadd_rn(acc, __fma_rn(z, z, __dmul_rn(20.0, s2)));
                    break;
                }
                case FN_ROSENBROCK:
                    if (j < D - 1) {
                        const double d1 = (m < 3) ? dv[(m + 1) & 3] : dn;
                        const double a0 = __dadd_rn(z, 1.0), a1 = __dadd_rn(d1, 1.0);
                        const double u = __fma_rn(-a0, a0, a1);
                        acc = __dadd_rn(acc, __fma_rn(__dmul_rn(100.0, u), u, __dmul_rn(z, z)));
                    }
                    break;
                case FN_ACKLEY: {
                    acc = __fma_rn(z, z, acc);
                    const double s = sinpi_reduced_f64(__dsub_rn(z, rint(z)));
                    acc2 = __fma_rn(s, s, acc2);
                    break;
                }
                default:
                    break;
                }
            }
        }
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(gmask, acc, off, G));
    if (fn != FN_ACKLEY) return acc;
    for (int off = G >> 1; off > 0; off >>= 1) acc2 = __dadd_rn(acc2, __shfl_xor_sync(gmask, acc2, off, G));
    const double Dd = (double)D;
    const double A = __dsqrt_rn(__ddiv_rn(acc, Dd));
    const double B = expm1_f64(__dmul_rn(-0.2, A));
    const double C = expm1_f64(__dmul_rn(-2.0, __ddiv_rn(acc2, Dd)));
    return -__dadd_rn(__dmul_rn(20.0, B), __dmul_rn(0x1.5bf0a8b145769p+1, C));  // e
}

// FP64 fitness of Table 3.2's f3 (Schwefel's problem 1.2), f7 (Griewank), f8
// (Powell) and f9 (Schwefel) on the same lane layout and in the oracle's
// orders:
//   f3  prefix sums c_j of z in the blocked order (4-variable block totals,
//       an inclusive Kogge-Stone scan of the block totals over the lanes of a
//       128-variable slice, a carry across slices, then a running sum inside
//       the block), terms c_j^2 summed like every other function's terms;
//   f7  sum z^2 (lane partials by fma, butterfly) / 4000 and the product of
//       cos(z_j / sqrt(j + 1)) (lane partials in ascending j, butterfly of
//       products), f = (1 - P) + S / 4000;
//   f8  one term per 4-variable block (z = 0 beyond D), lane partials, butterfly;
//   f9  sum z sin(sqrt|z|) by fma, f = 418.9829 D - S.
template <class Pos, int MAXC>
__device__ __noinline__ double fit64_extra(const Hot& in, const RowBuf<Pos, MAXC>& xb, int lane_g,
                                           unsigned gmask, int G)
{
    const auto& x = xb.v;
    const int D = in.D, nch = in.nchunks, fn = in.fn;
    double acc = 0.0, prod = 1.0, carry = 0.0;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
        double dv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * c + m;
            dv[m] = (c < nch && j < D) ? __dsub_rn((double)x[q][m], __ldg(in.o64 + j)) : 0.0;
        }
        if (fn == FN_SCHWEFEL12) {
            if (32 * q >= nch) break;            // uniform over the group
            double v = __dadd_rn(__dadd_rn(__dadd_rn(dv[0], dv[1]), dv[2]), dv[3]);
            for (int off = 1; off < G; off <<= 1) {
                const double o = __shfl_up_sync(gmask, v, off, G);
                if (lane_g >= off) v = __dadd_rn(o, v);
            }
            double e = __shfl_up_sync(gmask, v, 1, G);
            if (lane_g == 0) e = 0.0;
            const double tot = __shfl_sync(gmask, v, G - 1, G);
            double run = __dadd_rn(carry, e);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                if (c < nch && j < D) {
                    run = __dadd_rn(run, dv[m]);
                    acc = __fma_rn(run, run, acc);
                }
            }
            carry = __dadd_rn(carry, tot);
        } else if (c < nch) {
            if (fn == FN_POWELL) {
                const double a = __fma_rn(10.0, dv[1], dv[0]), b = __dsub_rn(dv[2], dv[3]);
                const double cc = __fma_rn(-2.0, dv[2], dv[1]), dd = __dsub_rn(dv[0], dv[3]);
                const double c2 = __dmul_rn(cc, cc), d2 = __dmul_rn(dd, dd);
                const double t = __fma_rn(a, a, __fma_rn(__dmul_rn(5.0, b), b,
                                                         __fma_rn(c2, c2, __dmul_rn(10.0, __dmul_rn(d2, d2)))));
                acc = __dadd_rn(acc, t);
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int j = 4 * c + m;
                    if (j >= D) break;
                    const double z = dv[m];
                    if (fn == FN_GRIEWANK) {
                        acc = __fma_rn(z, z, acc);
                        prod = __dmul_rn(prod, cos_rad_f64(__ddiv_rn(z, __dsqrt_rn((double)(j + 1)))));
                    } else {   // FN_SCHWEFEL
                        acc = __fma_rn(z, sin_rad_f64(__dsqrt_rn(fabs(z))), acc);
                    }
                }
            }
        }
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(gmask, acc, off, G));
    if (fn == FN_GRIEWANK) {
        for (int off = G >> 1; off > 0; off >>= 1) prod = __dmul_rn(prod, __shfl_xor_sync(gmask, prod, off, G));
        return __dadd_rn(__dsub_rn(1.0, prod), __ddiv_rn(acc, 4000.0));
    }
    if (fn == FN_SCHWEFEL) return __dsub_rn(__dmul_rn(418.9829, (double)D), acc);
    return acc;
}

template <class Pos, int MAXC>
__device__ __noinline__ double fit64_rotated(const Hot& in, const RowBuf<Pos, MAXC>& xb, int lane_g,
                                             unsigned gmask, int G)
{
    return fit64_impl<Pos, MAXC, true>(in, xb.v, lane_g, gmask, G);
}

template <class Pos, int MAXC>
__device__ __forceinline__ double fit64(const Hot& in, const Pos (&x)[MAXC][4], int lane_g, unsigned gmask,
                                        int G)
{
    if (is_rotated(in.fn) || is_fp64_only(in.fn)) {
        RowBuf<Pos, MAXC> xb;
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) xb.v[q][m] = x[q][m];
        if (is_fp64_only(in.fn)) return fit64_extra<Pos, MAXC>(in, xb, lane_g, gmask, G);
        return fit64_rotated<Pos, MAXC>(in, xb, lane_g, gmask, G);
    }
    return fit64_impl<Pos, MAXC, false>(in, x, lane_g, gmask, G);
}

// ---------------------------------------------------------------------------
// FP32 fitness with a rigorous bound E on |f - f_oracle| (f_oracle: the FP64
// value of the oracle).  Terms in FP32; per-function bounds:
//   sphere      t = z^2:        3.1u t   (z = fl(x - o), product)
//   ellipsoid   t = w z^2:      5.2u t   (+ w rounded to float)
//   Rastrigin   t = z^2 + 20 s^2: (2 e_sin + 3 + 16.1 + 1) u t, where 16.1u t
//               bounds the effect of rounding z (|t'(z)| |dz| <= 2u z^2 +
//               40 pi u |z||s| and |z||s| <= t / (2 sqrt 20))
//   Rosenbrock  running per-term bound from |d|, |a|, |u| (see below)
//   Ackley      bounds on S1 = sum z^2 and Q = sum s^2 propagated through the
//               tail (|d log f1 / d log S1| <= 1/2; |d f2 / d Q| <= 2e/D)
// plus the summation bound (K + L + 2) u sum|t| (K terms per lane, L butterfly
// levels), a 10% margin for the rounding of E itself, and 2^-40 sum|t| for
// the FP64 oracle's own rounding.
struct Fit32 {
    float f, E;
};

// FP32 z = M d with a running bound: z~_j by fma in FP32 with M rounded to
// float and d~ = fl(x - o), summed in blocks of 32 terms (each block from 0,
// then added to z~_j), and ez_j >= |z~_j - z_j| from S_j = sum |M~_jk||d~_k|:
// |z~ - z| <= (gamma_32 + gamma_nb + 2u) S (1 + O(u)), nb = number of blocks --
// the fma chains, the block sums, M's rounding and d's rounding.
template <int MAXC>
__device__ __noinline__ void rot_matvec32_impl(const Hot& in, const RowBuf<float, MAXC>& xb, int lane_g,
                                               unsigned gmask, int G, RowBuf<float, MAXC>& zb,
                                               RowBuf<float, MAXC>& eb)
{
    const auto& x = xb.v;
    auto& z = zb.v;
    auto& ez = eb.v;
    const int D = in.D;
    float d[MAXC][4], t[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane_g + 32 * q) + m;
            d[q][m] = (j < D) ? __fsub_rn(x[q][m], __ldg(in.o32 + j)) : 0.f;
            z[q][m] = 0.f;
            t[q][m] = 0.f;
            ez[q][m] = 0.f;
        }
#pragma unroll
    for (int qk = 0; qk < MAXC; ++qk) {
        for (int l = 0; l < G; ++l) {
            if (128 * qk + 4 * l >= D) break;
#pragma unroll
            for (int mk = 0; mk < 4; ++mk) {
                const int k = 128 * qk + 4 * l + mk;
                const float dk = __shfl_sync(gmask, d[qk][mk], l, G);
                if (k < D) {
                    const float adk = fabsf(dk);
#pragma unroll
                    for (int q = 0; q < MAXC; ++q)
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int j = 4 * (lane_g + 32 * q) + m;
                            if (j < D) {
                                const float mjk = __ldg(in.M32 + (size_t)j * D + k);
                                t[q][m] = __fmaf_rn(mjk, dk, t[q][m]);
                                ez[q][m] = __fmaf_rn(fabsf(mjk), adk, ez[q][m]);
                            }
                        }
                }
            }
            if ((l & 7) == 7) {   // close a block of 32 terms
#pragma unroll
                for (int q = 0; q < MAXC; ++q)
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        z[q][m] = __fadd_rn(z[q][m], t[q][m]);
                        t[q][m] = 0.f;
                    }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) z[q][m] = __fadd_rn(z[q][m], t[q][m]);
    const int nb = (D + 31) / 32;
    const float c = 1.02f * (float)(32 + nb + 3) * U32;
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) ez[q][m] = c * ez[q][m] * (1.f + (float)D * U32);
}

template <int MAXC>
__device__ __forceinline__ void rot_matvec32(const Hot& in, const float (&x)[MAXC][4], int lane_g,
                                             unsigned gmask, int G, float (&z)[MAXC][4],
                                             float (&ez)[MAXC][4])
{
    RowBuf<float, MAXC> xb, zb, eb;
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) xb.v[q][m] = x[q][m];
    rot_matvec32_impl<MAXC>(in, xb, lane_g, gmask, G, zb, eb);
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            z[q][m] = zb.v[q][m];
            ez[q][m] = eb.v[q][m];
        }
}

// Compensated FP32 z = M d for the FP32 fitness of the rotated functions:
// d = x - o exactly as a float pair (TwoSum; x and o are floats), M as the
// float pair M32 + M32lo, and for every output the Dot2 recurrence of Ogita,
// Rump and Oishi ("Accurate sum and dot product", SISC 2005) over k ascending:
// TwoProduct of M32 d_hi, TwoSum into p, the two rounding errors and the cross
// terms M32 d_lo + M32lo d_hi into s; z = p + s.  With n = D + 8 and
// g = gamma_n, |z~ - z| <= 1.01 u |z~| + (2 g^2 + 4 u g + 2^-42) S, S =
// sum |M||d| <= S~ (1 + 2 gamma_D)(1 + 2^-22) from the FP32 sum S~ of
// |M32||d_hi|; the 2^-42 S also covers the FP64 oracle's own rounding of z.
// About 16 FP32 operations per term against 2 for a plain fma chain, and a
// bound near u |z| instead of D u sum |M||d|: an FP32 rotated fitness within a
// few u of the FP64 value, and far fewer FP64 rechecks.
template <int MAXC>
__device__ __noinline__ void rot_matvec32c_impl(const Hot& in, const RowBuf<float, MAXC>& xb, int lane_g,
                                                unsigned gmask, int G, RowBuf<float, MAXC>& zb,
                                                RowBuf<float, MAXC>& eb)
{
    const auto& x = xb.v;
    auto& z = zb.v;
    auto& ez = eb.v;
    const int D = in.D;
    float dh[MAXC][4], dl[MAXC][4], p[MAXC][4], sc[MAXC][4], S[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane_g + 32 * q) + m;
            const float a = (j < D) ? x[q][m] : 0.f, b = (j < D) ? -__ldg(in.o32 + j) : 0.f;
            const float sum = __fadd_rn(a, b);
            const float bb = __fsub_rn(sum, a);
            dh[q][m] = sum;
            dl[q][m] = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
            p[q][m] = 0.f;
            sc[q][m] = 0.f;
            S[q][m] = 0.f;
        }
#pragma unroll
    for (int qk = 0; qk < MAXC; ++qk) {
        for (int l = 0; l < G; ++l) {
            if (128 * qk + 4 * l >= D) break;
#pragma unroll
            for (int mk = 0; mk < 4; ++mk) {
                const int k = 128 * qk + 4 * l + mk;
                const float bh = __shfl_sync(gmask, dh[qk][mk], l, G);
                const float bl = __shfl_sync(gmask, dl[qk][mk], l, G);
                if (k < D) {
                    const float abh = fabsf(bh);
#pragma unroll
                    for (int q = 0; q < MAXC; ++q)
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int j = 4 * (lane_g + 32 * q) + m;
                            if (j < D) {
                                const size_t o = (size_t)j * D + k;
                                const float a = __ldg(in.M32 + o), al = __ldg(in.M32lo + o);
                                const float h = __fmul_rn(a, bh);
                                const float r = __fmaf_rn(a, bh, -h);        // a bh = h + r exactly
                                const float t = __fadd_rn(p[q][m], h);
                                const float bb = __fsub_rn(t, p[q][m]);
                                const float e = __fadd_rn(__fsub_rn(p[q][m], __fsub_rn(t, bb)), __fsub_rn(h, bb));
                                p[q][m] = t;                                   // p + h = t + e exactly
                                const float cross = __fmaf_rn(a, bl, __fmul_rn(al, bh));
                                sc[q][m] = __fadd_rn(sc[q][m], __fadd_rn(__fadd_rn(e, r), cross));
                                S[q][m] = __fmaf_rn(fabsf(a), abh, S[q][m]);
                            }
                        }
                }
            }
        }
    }
    const float U = 0x1p-24f;
    const float nl = (float)(D + 8);
    const float gam = nl * U / (1.f - nl * U);
    const float gD = (float)D * U / (1.f - (float)D * U);
    const float cS = 1.01f * (2.f * gam * gam + 4.f * U * gam + 0x1p-42f) * (1.f + 2.f * gD) * (1.f + 0x1p-22f);
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            z[q][m] = __fadd_rn(p[q][m], sc[q][m]);
            ez[q][m] = __fmaf_ru(cS, S[q][m], 1.01f * U * fabsf(z[q][m]));
        }
}

template <int MAXC>
__device__ __forceinline__ void rot_matvec32c(const Hot& in, const float (&x)[MAXC][4], int lane_g,
                                              unsigned gmask, int G, float (&z)[MAXC][4],
                                              float (&ez)[MAXC][4])
{
    RowBuf<float, MAXC> xb, zb, eb;
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) xb.v[q][m] = x[q][m];
    rot_matvec32c_impl<MAXC>(in, xb, lane_g, gmask, G, zb, eb);
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            z[q][m] = zb.v[q][m];
            ez[q][m] = eb.v[q][m];
        }
}

template <int MAXC, bool ROT>
__device__ __forceinline__ Fit32 fit32_impl(const Hot& in, const float (&x)[MAXC][4], int lane_g,
                                            unsigned gmask, int G)
{
    const int D = in.D, nch = in.nchunks;
    const bool rot = ROT && is_rotated(in.fn);
    const int fn = base_fn(in.fn);
    float zr[MAXC][4], ezr[MAXC][4];
    if (rot) rot_matvec32c<MAXC>(in, x, lane_g, gmask, G, zr, ezr);
    float acc = 0.f, acc2 = 0.f, accE = 0.f, accZ = 0.f;
    float rS1 = 0.f, rQ = 0.f;   // rotated: absolute error bounds of S1 and Q (Ackley)
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
        float dn = 0.f;
        if (fn == FN_ROSENBROCK) {
            const float first = (c < nch) ? __fsub_rn(x[q][0], __ldg(in.o32 + 4 * c)) : 0.f;
            dn = __shfl_down_sync(gmask, first, 1, G);
            if (G == 32 && q + 1 < MAXC) {
                const int cn = c + 32;
                const float nxt = (cn < nch) ? __fsub_rn(x[(q + 1) % MAXC][0], __ldg(in.o32 + 4 * cn))
                                             : 0.f;
                const float wrap = __shfl_sync(gmask, nxt, 0, 32);
                if (lane_g == 31) dn = wrap;
            }
        }
        if (c < nch) {
            float dv[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                dv[m] = rot ? zr[q][m] : (j < D) ? __fsub_rn(x[q][m], __ldg(in.o32 + j)) : 0.f;
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * c + m;
                if (j >= D) break;
                const float z = dv[m];
                switch (fn) {
                case FN_SPHERE:
                    acc = __fadd_rn(acc, __fmul_rn(z, z));
                    break;
                case FN_ELLIPSOID: {
                    const float wj = __ldg(in.w32 + j);
                    const float t = __fmul_rn(wj, __fmul_rn(z, z));
                    acc = __fadd_rn(acc, t);
                    if (rot) {   // z~ has error ez: w (2|z~| + ez) ez, plus the products' roundings
                        const float ez = ezr[q][m];
                        accE = __fadd_rn(accE, 4.2f * U32 * t + 1.01f * wj * (2.f * fabsf(z) + ez) * ez);
                    }
                    break;
                }
                case FN_RASTRIGIN: {
                    const float s = sinpi_reduced_f32(__fsub_rn(z, rintf(z)));
                    const float t = __fmaf_rn(z, z, __fmul_rn(20.f, __fmul_rn(s, s)));
                    acc = __fadd_rn(acc, t);
                    if (rot) {   // |t'(xi)| <= 2|xi| + 20 pi min(1, 2 pi |xi|), |xi| <= |z~| + ez
                        const float ez = ezr[q][m];
                        const float xi = fabsf(z) + ez;
                        accE = __fadd_rn(accE, (2.f * SINPI32_ERR_U + 4.f) * U32 * t +
                                                   1.01f * (2.f * xi + 62.8318558f * fminf(1.f, 6.28318548f * xi)) * ez);
                    }
                    break;
                }
                case FN_ROSENBROCK:
                    if (j < D - 1) {
                        // a_{j+1} - a_j^2 with a = d + 1 equals d1 - d0 (d0 + 2): evaluated
                        // from d directly, free of the cancellation against 1.
                        const float d1 = (m < 3) ? dv[(m + 1) & 3] : dn;
                        const float s0 = __fadd_rn(z, 2.f);
                        const float u = __fmaf_rn(-z, s0, d1);
                        const float d2 = __fmul_rn(z, z);
                        const float t = __fmaf_rn(__fmul_rn(100.f, u), u, d2);
                        acc = __fadd_rn(acc, t);
                        // d~ = fl(x - o): |d~ - d| <= u|d~|(1 + 2u)
                        const float e0 = 1.01f * U32 * fabsf(z), e1 = 1.01f * U32 * fabsf(d1);
                        // |u~ - u| <= u|u~| + e1 + |d0~| (u|s0~| + e0) + (|s0~| + e0) e0
                        const float as0 = fabsf(s0);
                        const float eu = 1.01f * (U32 * fabsf(u) + e1 + fabsf(z) * (U32 * as0 + e0) +
                                                  (1.01f * as0 + e0) * e0);
                        // 100 u^2 + d^2: propagated part plus the roundings of the tail
                        float et = 100.f * eu * (2.f * fabsf(u) + eu) + 3.f * U32 * 100.f * u * u +
                                   3.1f * U32 * d2 + U32 * t;
                        // the FP64 reference forms a = d + 1 first: its own error on u is
                        // at most 2^-51 (|a1| + 2 a0^2 + |u| + 2), a ~ |d| + 1
                        const float a0 = fabsf(z) + 1.f, a1 = fabsf(d1) + 1.f;
                        const float eu64 = 0x1p-51f * (a1 + 2.f * a0 * a0 + fabsf(u) + 2.f);
                        et += 200.f * fabsf(u) * eu64 + 100.f * eu64 * eu64 + 0x1p-50f * t;
                        accE = __fadd_rn(accE, et);
                    }
                    break;
                case FN_ACKLEY: {
                    acc = __fadd_rn(acc, __fmul_rn(z, z));
                    const float s = sinpi_reduced_f32(__fsub_rn(z, rintf(z)));
                    acc2 = __fadd_rn(acc2, __fmul_rn(s, s));
                    accZ = __fadd_rn(accZ, fabsf(z));
                    if (rot) {   // |d z^2| <= (2|z~| + ez) ez, |d sin^2(pi z)| <= pi min(1, 2 pi |xi|) ez
                        const float ez = ezr[q][m];
                        const float xi = fabsf(z) + ez;
                        rS1 = __fadd_rn(rS1, 1.01f * (2.f * fabsf(z) + ez) * ez);
                        rQ = __fadd_rn(rQ, 1.01f * 3.14159275f * fminf(1.f, 6.28318548f * xi) * ez);
                    }
                    break;
                }
                default:
                    break;
                }
            }
        }
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(gmask, acc, off, G));
    const float L = (float)(__ffs(G) - 1);
    const float csum = (float)(4 * MAXC) + L + 2.f;
    Fit32 r;
    switch (fn) {
    case FN_SPHERE:
        r.f = acc;
        r.E = 1.1f * (3.1f + csum) * U32 * acc;
        break;
    case FN_ELLIPSOID:
        r.f = acc;
        if (rot) {
            for (int off = G >> 1; off > 0; off >>= 1)
                accE = __fadd_rn(accE, __shfl_xor_sync(gmask, accE, off, G));
            r.E = 1.1f * (accE + csum * U32 * acc);
        } else {
            r.E = 1.1f * (5.2f + csum) * U32 * acc;
        }
        break;
    case FN_RASTRIGIN:
        r.f = acc;
        if (rot) {
            for (int off = G >> 1; off > 0; off >>= 1)
                accE = __fadd_rn(accE, __shfl_xor_sync(gmask, accE, off, G));
            r.E = 1.1f * (accE + csum * U32 * acc);
        } else {
            r.E = 1.1f * (2.f * SINPI32_ERR_U + 3.f + 16.1f + 1.f + csum) * U32 * acc;
        }
        break;
    case FN_ROSENBROCK:
        for (int off = G >> 1; off > 0; off >>= 1)
            accE = __fadd_rn(accE, __shfl_xor_sync(gmask, accE, off, G));
        r.f = acc;
        r.E = 1.1f * (accE + csum * U32 * acc);
        break;
    default: {   // Ackley
        for (int off = G >> 1; off > 0; off >>= 1) {
            acc2 = __fadd_rn(acc2, __shfl_xor_sync(gmask, acc2, off, G));
            accZ = __fadd_rn(accZ, __shfl_xor_sync(gmask, accZ, off, G));
        }
        const float Df = (float)D;
        const float A = __fsqrt_rn(__fdiv_rn(acc, Df));
        const float B = expm1_f32(__fmul_rn(-0.2f, A));
        const float C = expm1_f32(__fmul_rn(-2.f, __fdiv_rn(acc2, Df)));
        const float f1 = __fmul_rn(-20.f, B), f2 = __fmul_rn(-0x1.5bf0a8p+1f, C);
        r.f = __fadd_rn(f1, f2);
        if (!rot) {
            const float relS = (3.1f + csum) * U32;
            const float EQ = 1.01f * 3.14159275f * U32 * accZ +
                             (2.f * SINPI32_ERR_U + 1.f + csum) * U32 * acc2;
            r.E = 1.1f * (0.5f * relS * f1 + (EXPM1F_ERR_U + 6.f) * U32 * f1 +
                          (2.f * 2.7182818f / Df) * EQ + (EXPM1F_ERR_U + 8.f) * U32 * f2 + U32 * r.f);
        } else {
            for (int off = G >> 1; off > 0; off >>= 1) {
                rS1 = __fadd_rn(rS1, __shfl_xor_sync(gmask, rS1, off, G));
                rQ = __fadd_rn(rQ, __shfl_xor_sync(gmask, rQ, off, G));
            }
            // absolute bounds on S1 and Q; f1 = -20 expm1(-0.2 sqrt(S1/D)) changes by at most
            // 4 sqrt(dS1 / D) (sqrt is 1/2-Hoelder), or, when dS1 <= S1 / 2, by
            // 1.5 f1 dS1 / S1 (|df1/dS1| <= f1 / (2 S1), f1 concave with f1(0) = 0)
            const float ES = rS1 + (3.1f + csum) * U32 * acc;
            const float EQ = rQ + (2.f * SINPI32_ERR_U + 1.f + csum) * U32 * acc2;
            const float d1 = (ES <= 0.5f * acc) ? 1.5f * f1 * ES / acc : 4.f * __fsqrt_ru(ES / Df);
            r.E = 1.1f * (d1 + (EXPM1F_ERR_U + 6.f) * U32 * f1 + (2.f * 2.7182818f / Df) * EQ +
                          (EXPM1F_ERR_U + 8.f) * U32 * f2 + U32 * r.f);
        }
        acc = r.f;
        break;
    }
    }
    r.E = __fadd_ru(r.E, 0x1p-40f * (acc + accE));
    return r;
}

// The rotated forms run out of line: the plain functions' code carries no
// trace of them, and the row goes through a buffer so the caller's array
// stays in registers.
template <int MAXC>
__device__ __noinline__ Fit32 fit32_rotated(const Hot& in, const RowBuf<float, MAXC>& xb, int lane_g,
                                            unsigned gmask, int G)
{
    return fit32_impl<MAXC, true>(in, xb.v, lane_g, gmask, G);
}

template <int MAXC>
__device__ __forceinline__ Fit32 fit32(const Hot& in, const float (&x)[MAXC][4], int lane_g, unsigned gmask,
                                       int G)
{
    if (is_rotated(in.fn)) {
        RowBuf<float, MAXC> xb;
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) xb.v[q][m] = x[q][m];
        return fit32_rotated<MAXC>(in, xb, lane_g, gmask, G);
    }
    return fit32_impl<MAXC, false>(in, x, lane_g, gmask, G);
}

// True when the interval [lo, hi] of a fitness value is too wide for its
// midpoint to lie within 0.9e-6 relative of the value (relative to
// max(|f|, 1e-6 (20 + e)) for Ackley, whose optimum is 0, else to |f|; every
// test function is >= 0).
__device__ __forceinline__ bool too_wide(int fn, float lo, float hi)
{
    const float floor = (base_fn(fn) == FN_ACKLEY) ? 1e-6f * 22.7182818f : 0.f;
    return __fsub_ru(hi, lo) > 1.8e-6f * fmaxf(lo, floor);
}

// ---------------------------------------------------------------------------
// Block-level reductions (all threads get the result).
struct MinRec {
    double v;
    long long i;
};
__device__ __forceinline__ MinRec min_rec(MinRec a, MinRec b)
{
    return (b.v < a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

struct Scratch {
    double dv[32];
    long long iv[32];
    float fv[32];
    unsigned long long uv[32];
    int flag;
};

__device__ inline MinRec block_min_rec(MinRec r, Scratch& sh)
{
    for (int off = 16; off > 0; off >>= 1) {
        MinRec o;
        o.v = __shfl_xor_sync(0xffffffffu, r.v, off);
        o.i = __shfl_xor_sync(0xffffffffu, r.i, off);
        r = min_rec(r, o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { sh.dv[w] = r.v; sh.iv[w] = r.i; }
    __syncthreads();
    MinRec out = { sh.dv[0], sh.iv[0] };
    for (int k = 1; k < nw; ++k) out = min_rec(out, MinRec{ sh.dv[k], sh.iv[k] });
    return out;
}

__device__ inline float block_min_f32(float v, Scratch& sh)
{
    for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.fv[w] = v;
    __syncthreads();
    float out = sh.fv[0];
    for (int k = 1; k < nw; ++k) out = fminf(out, sh.fv[k]);
    return out;
}

__device__ inline unsigned long long block_sum_u64(unsigned long long v, Scratch& sh)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.uv[w] = v;
    __syncthreads();
    unsigned long long out = 0;
    for (int k = 0; k < nw; ++k) out += sh.uv[k];
    return out;
}

__device__ inline long long block_max_i64(long long v, Scratch& sh)
{
    for (int off = 16; off > 0; off >>= 1) v = max(v, (long long)__shfl_xor_sync(0xffffffffu, v, off));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.iv[w] = v;
    __syncthreads();
    long long out = sh.iv[0];
    for (int k = 1; k < nw; ++k) out = max(out, sh.iv[k]);
    return out;
}

// ---------------------------------------------------------------------------
// FP64 fitness of a row in memory, by one full warp (32-lane layout).
template <class Pos, int MAXC>
__device__ double fit64_row_warp(const Hot& in, const Pos* row, bool l2_only)
{
    const int lane = threadIdx.x & 31;
    Pos x[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
        if (c < in.nchunks) {
            if (l2_only) ld4_cg(row + 4 * c, x[q]); else ld4(row + 4 * c, x[q]);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) x[q][m] = Pos(0);
        }
    }
    return fit64<Pos, MAXC>(in, x, lane, 0xffffffffu, 32);
}

template <class Pos>
__device__ double fit64_row(const Hot& in, const Pos* row, bool l2_only)
{
    switch (in.maxc) {
    case 1: return fit64_row_warp<Pos, 1>(in, row, l2_only);
    case 2: return fit64_row_warp<Pos, 2>(in, row, l2_only);
    case 4: return fit64_row_warp<Pos, 4>(in, row, l2_only);
    default: return fit64_row_warp<Pos, 8>(in, row, l2_only);
    }
}

__device__ __forceinline__ float f64_to_f32_rd(double v) { return __double2float_rd(v); }
__device__ __forceinline__ float f64_to_f32_ru(double v) { return __double2float_ru(v); }

}  // namespace psso
