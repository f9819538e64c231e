// devmath.cuh -- Philox-4x32-10 and the transcendental functions the fitness
// evaluation needs, written for sm_103a.
//
// FP64 routines follow one documented algorithm operation by operation with
// explicit IEEE intrinsics (__fma_rn, __dmul_rn, __dadd_rn, __dsub_rn), so that
// their results are a fixed function of the inputs:
//   sin(pi r), |r| <= 1/2 : r * S(r^2), S the Taylor series of sin(pi r)/r cut
//                           after r^20, Horner with fma; coefficient k is the
//                           nearest double to (-1)^k pi^(2k+1)/(2k+1)!.
//   expm1(x)             : |x| <= ln2/2: x * E(x), E the Taylor series of
//                           (e^x-1)/x cut after x^13/14!; otherwise
//                           x = k ln2 + r (k nearest integer to x/ln2, r by two
//                           fma with the split ln2) and 2^k expm1(r) + (2^k - 1).
// FP32 routines use the same schemes with shorter series; their relative error
// bounds (SINPI32_ERR_U, EXPM1F_ERR_U, in units of 2^-24) are checked
// exhaustively over their input ranges by the GPU tests.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace psso {

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;   // one 32x32->64 multiply each
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                       (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, int m)
{
    return m == 0 ? w.x : m == 1 ? w.y : m == 2 ? w.z : w.w;
}

// ---------------------------------------------------------------------------
// FP64: sin(pi r) for r already reduced to [-1/2, 1/2].
__device__ __forceinline__ double sinpi_reduced_f64(double r)
{
    const double q = __dmul_rn(r, r);
    double p = 0x1.2877020d52cf0p-31;          //  pi^21/21!
    p = __fma_rn(p, q, -0x1.8a404211f9547p-26); // -pi^19/19!
    p = __fma_rn(p, q, 0x1.aaec32af93359p-21);  //  pi^17/17!
    p = __fma_rn(p, q, -0x1.6fadb9f155744p-16); // -pi^15/15!
    p = __fma_rn(p, q, 0x1.e8f434d018d63p-12);  //  pi^13/13!
    p = __fma_rn(p, q, -0x1.e3074fde8871fp-8);  // -pi^11/11!
    p = __fma_rn(p, q, 0x1.50783487ee782p-4);   //  pi^9/9!
    p = __fma_rn(p, q, -0x1.32d2cce62bd86p-1);  // -pi^7/7!
    p = __fma_rn(p, q, 0x1.466bc6775aae2p+1);   //  pi^5/5!
    p = __fma_rn(p, q, -0x1.4abbce625be53p+2);  // -pi^3/3!
    p = __fma_rn(p, q, 0x1.921fb54442d18p+1);   //  pi
    return __dmul_rn(r, p);
}

// sin^2(pi z): the sign (-1)^n of sin(pi (n + r)) cancels in the square.
__device__ __forceinline__ double sinpi_sq_f64(double z)
{
    const double r = __dsub_rn(z, rint(z));
    const double s = sinpi_reduced_f64(r);
    return __dmul_rn(s, s);
}

// sin(pi x) with its sign: x = n + r, n the nearest integer (half even),
// sin(pi x) = (-1)^n sin(pi r); n is odd iff n / 2 is not an integer.
__device__ __forceinline__ double sinpi_f64(double x)
{
    const double n = rint(x);
    const double s = sinpi_reduced_f64(__dsub_rn(x, n));
    const double h = __dmul_rn(n, 0.5);
    return (h != rint(h)) ? -s : s;
}

// sin and cos of an argument in radians through sin(pi q), q = a / pi or
// a / (2 pi) rounded once (the constants are the nearest doubles to 1 / pi and
// 1 / (2 pi)); cos a = 1 - 2 sin^2(a / 2) as one fma.  Error about
// 2^-52 (1 + |a|).
__device__ __forceinline__ double sin_rad_f64(double a)
{
    return sinpi_f64(__dmul_rn(a, 0x1.45f306dc9c883p-2));
}
__device__ __forceinline__ double cos_rad_f64(double a)
{
    const double s = sinpi_f64(__dmul_rn(a, 0x1.45f306dc9c883p-3));
    return __fma_rn(__dmul_rn(-2.0, s), s, 1.0);
}

__device__ __forceinline__ double expm1_series_f64(double x)
{
    double p = 0x1.93974a8c07c9dp-37;          // 1/14!
    p = __fma_rn(p, x, 0x1.6124613a86d09p-33);  // 1/13!
    p = __fma_rn(p, x, 0x1.1eed8eff8d898p-29);  // 1/12!
    p = __fma_rn(p, x, 0x1.ae64567f544e4p-26);  // 1/11!
    p = __fma_rn(p, x, 0x1.27e4fb7789f5cp-22);  // 1/10!
    p = __fma_rn(p, x, 0x1.71de3a556c734p-19);  // 1/9!
    p = __fma_rn(p, x, 0x1.a01a01a01a01ap-16);  // 1/8!
    p = __fma_rn(p, x, 0x1.a01a01a01a01ap-13);  // 1/7!
    p = __fma_rn(p, x, 0x1.6c16c16c16c17p-10);  // 1/6!
    p = __fma_rn(p, x, 0x1.1111111111111p-7);   // 1/5!
    p = __fma_rn(p, x, 0x1.5555555555555p-5);   // 1/4!
    p = __fma_rn(p, x, 0x1.5555555555555p-3);   // 1/3!
    p = __fma_rn(p, x, 0x1.0000000000000p-1);   // 1/2!
    p = __fma_rn(p, x, 1.0);                    // 1/1!
    return __dmul_rn(x, p);
}

__device__ __forceinline__ double expm1_f64(double x)
{
    constexpr double LN2_HI = 0x1.62e42fefa39efp-1;  // nearest double to ln 2
    constexpr double LN2_LO = 0x1.abc9e3b39803fp-56; // nearest double to ln 2 - LN2_HI
    constexpr double INV_LN2 = 0x1.71547652b82fep+0; // nearest double to 1/ln 2
    if (fabs(x) <= 0x1.62e42fefa39efp-2) return expm1_series_f64(x);  // LN2_HI / 2
    const double k = rint(__dmul_rn(x, INV_LN2));
    double r = __fma_rn(-k, LN2_HI, x);
    r = __fma_rn(-k, LN2_LO, r);
    const double e = expm1_series_f64(r);
    const double two_k = __longlong_as_double((long long)((int)k + 1023) << 52);
    return __dadd_rn(__dmul_rn(e, two_k), __dsub_rn(two_k, 1.0));
}

// ---------------------------------------------------------------------------
// FP32: sin(pi r) on [-1/2, 1/2], Taylor series cut after r^14 (truncation
// below 2^-30 relative); coefficient k is the nearest float to
// (-1)^k pi^(2k+1)/(2k+1)!.
constexpr float SINPI32_ERR_U = 4.0f;   // |s - sin(pi r)| <= 4 * 2^-24 * |sin(pi r)|

__device__ __forceinline__ float sinpi_reduced_f32(float r)
{
    const float q = __fmul_rn(r, r);
    float p = -0x1.6fadbap-16f;               // -pi^15/15!
    p = __fmaf_rn(p, q, 0x1.e8f434p-12f);     //  pi^13/13!
    p = __fmaf_rn(p, q, -0x1.e3075p-8f);      // -pi^11/11!
    p = __fmaf_rn(p, q, 0x1.507834p-4f);      //  pi^9/9!
    p = __fmaf_rn(p, q, -0x1.32d2ccp-1f);     // -pi^7/7!
    p = __fmaf_rn(p, q, 0x1.466bc6p+1f);      //  pi^5/5!
    p = __fmaf_rn(p, q, -0x1.4abbcep+2f);     // -pi^3/3!
    p = __fmaf_rn(p, q, 0x1.921fb6p+1f);      //  pi
    return __fmul_rn(r, p);
}

// expm1 in FP32 for x <= 0 (the Ackley arguments): series cut after x^7/8!
// on |x| <= ln2/2, else the same reduction as the FP64 routine.
constexpr float EXPM1F_ERR_U = 6.0f;    // |e - expm1(x)| <= 6 * 2^-24 * |expm1(x)|

__device__ __forceinline__ float expm1_series_f32(float x)
{
    float p = 0x1.a01a02p-16f;                // 1/8!
    p = __fmaf_rn(p, x, 0x1.a01a02p-13f);     // 1/7!
    p = __fmaf_rn(p, x, 0x1.6c16c2p-10f);     // 1/6!
    p = __fmaf_rn(p, x, 0x1.111112p-7f);      // 1/5!
    p = __fmaf_rn(p, x, 0x1.555556p-5f);      // 1/4!
    p = __fmaf_rn(p, x, 0x1.555556p-3f);      // 1/3!
    p = __fmaf_rn(p, x, 0.5f);                // 1/2!
    p = __fmaf_rn(p, x, 1.0f);                // 1/1!
    return __fmul_rn(x, p);
}

__device__ __forceinline__ float expm1_f32(float x)
{
    if (fabsf(x) <= 0x1.62e430p-2f) return expm1_series_f32(x);
    if (x < -30.0f) return -1.0f;             // e^x < 2^-43: expm1 rounds to -1
    const float k = rintf(__fmul_rn(x, 0x1.715476p+0f));   // nearest float to 1/ln 2
    float r = __fmaf_rn(-k, 0x1.62e430p-1f, x);             // nearest float to ln 2
    r = __fmaf_rn(-k, 0x1.05c610p-29f, r);                  // ln 2 - that float
    const float e = expm1_series_f32(r);
    const float two_k = __int_as_float(((int)k + 127) << 23);
    return __fadd_rn(__fmul_rn(e, two_k), __fsub_rn(two_k, 1.0f));
}

}  // namespace psso
