/*
 * psso_oracle.c -- plain, sequential CPU oracle for Parallel Simplified Swarm
 * Optimization (PSSO; Yeh, Liu, Tan, Huang, "Implementation of Parallel
 * Simplified Swarm Optimization in CUDA", arXiv 2110.01470).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness authority the CUDA
 * library is compared against.  Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg load it; the product library never
 * links, loads or calls it, and the two share no code, header or constant
 * table.  The only thing both sides consume is problem *data* (shift vector,
 * rotation matrix, ellipsoid weights) made by the seeded input generators.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * -ffp-contract=off matters: every multiply-add below is either an explicit
 * fma() or two separately rounded operations, exactly as written, so that the
 * FP64 results are a fixed function of the inputs on every host.
 *
 * What one run computes (paper Sec. 2.1, Sec. 3.3, Alg. 2-4):
 *   generation 0 : random population X0 in [lb,ub] (Kernel Function (I),
 *                  Sec. 2.3.1); pBest P = X0; pF = f(X0); gBest = arg-min pF.
 *   generation g : for every particle i and variable j the stepwise update of
 *                  Eq. 2.1 using gBest, pBest and X of generation g-1 (the
 *                  synchronous flow of Alg. 2: all particles search before any
 *                  update); fitness of every particle (Kernel Function (E),
 *                  Sec. 2.3.2); pBest update with "<=" (Alg. 3); gBest = the
 *                  lowest-index arg-min of pF (Alg. 4, with a deterministic
 *                  tie-break).
 *   oracle_run_ex adds the asynchronous flow of Alg. 1 (the sequential CPU-SSO:
 *   particle by particle, gBest replaced as soon as a particle beats it) and
 *   the interval order Eq. 2.1 prints.
 *
 * Readings of the paper taken here (the paper is silent or garbled on each):
 *   * Eq. 2.1's intervals are taken by default in the order gBest, pBest, keep,
 *     fresh with cumulative thresholds Cg <= Cp <= Cw (the same four-way split
 *     as Eq. 2.1, which lists them as keep, pBest, gBest, fresh with
 *     Cw <= Cp <= Cg; order 1 of oracle_run_ex takes that printed order).
 *   * Alg. 1's second test is printed as a repeat of the first ("solF < pF");
 *     it is read as the gBest test solF < gF.
 *   * The uniform draw rho is a 32-bit Philox word r; "rho < C" is the integer
 *     test r < T with T = round-half-even(C * 2^32).
 *   * Random numbers are Philox-4x32-10 blocks (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11) keyed by the seed,
 *     with counter (variable block, particle, generation, tag | stream<<8); the
 *     paper's cuRAND pre-generated stream (Sec. 3.1) is replaced by this
 *     counter-based keying.
 *   * Fitness is summed in a fixed order: variable j feeds lane (j>>2)&31; each
 *     lane accumulates its variables in ascending j from +0.0; the 32 lane
 *     partials are then combined by an xor butterfly over offsets 16,8,4,2,1.
 *   * Rastrigin's 10 - 10 cos(2 pi z) is evaluated as 20 sin^2(pi z) (an exact
 *     identity); Ackley's exp(.)-exp(.)+20+e is evaluated through expm1 of the
 *     same arguments with cos(2 pi z) = 1 - 2 sin^2(pi z) (exact identities);
 *     Rosenbrock is shifted so that f(o) = 0 (z = x - o + 1).
 *   * The rest of Table 3.2 (f2, f3, f7, f8, f9), shifted by o:
 *       f2 hyper-ellipsoid  sum (j+1) z_j^2
 *       f3 Schwefel's       sum_i (sum_{j<=i} z_j)^2 (Schwefel's problem 1.2; the
 *                           printed inner sum of squares would make f3 a
 *                           separable weighted sphere, which the paper's own
 *                           classification of f3 as inseparable rules out)
 *       f7 Griewank         1 + sum z_j^2 / 4000 - prod cos(z_j / sqrt(j+1))
 *       f8 Powell           sum over blocks of 4: (z0 + 10 z1)^2 + 5 (z2 - z3)^2
 *                           + (z1 - 2 z2)^4 + 10 (z0 - z3)^4, z = 0 beyond D
 *                           (the printed form lacks the + between terms)
 *       f9 Schwefel         418.9829 D - sum z_j sin(sqrt|z_j|)
 *     with the fixed evaluation orders written out at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Function ids.  Table 3.2 of the paper lists Sphere, Rosenbrock, Rastrigin,
 * Ackley and the hyper-ellipsoid; the rotated forms apply z = M (x - o). */
enum {
    FN_SPHERE = 0,
    FN_ELLIPSOID = 1,
    FN_RASTRIGIN = 2,
    FN_ROSENBROCK = 3,
    FN_ACKLEY = 4,
    FN_ROT_ELLIPSOID = 5,
    FN_ROT_RASTRIGIN = 6,
    FN_ROT_ACKLEY = 7,
    FN_HYPER_ELLIPSOID = 8,   /* Table 3.2 f2 */
    FN_SCHWEFEL12 = 9,        /* Table 3.2 f3 */
    FN_GRIEWANK = 10,         /* Table 3.2 f7 */
    FN_POWELL = 11,           /* Table 3.2 f8 */
    FN_SCHWEFEL = 12,         /* Table 3.2 f9 */
    FN_COUNT = 13
};

enum { LATTICE_F64 = 0, LATTICE_F32 = 1 };
enum { TAG_INIT = 1, TAG_RHO = 2, TAG_FRESH = 3 };

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11).  Multipliers and Weyl key increments
 * are the published ones.  One round maps (c0,c1,c2,c3) to
 * (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)); the key is bumped
 * by the Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_block(uint64_t seed, uint32_t c0, uint32_t i, uint32_t g,
                         uint32_t tag, uint32_t sid, uint32_t out[4])
{
    uint32_t ctr[4] = { c0, i, g, tag | (sid << 8) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    oracle_philox4x32_10(ctr, key, out);
}

/* The rho word of Eq. 2.1 for variable j of particle i at generation g. */
uint32_t oracle_rho(uint64_t seed, uint32_t sid, uint32_t g, uint32_t i, uint32_t j)
{
    uint32_t w[4];
    philox_block(seed, j >> 2, i, g, TAG_RHO, sid, w);
    return w[j & 3];
}

/* ------------------------------------------------------------------------ */
/* A fresh uniform value in [lb, ub] (the last branch of Eq. 2.1 and the
 * initial population of Kernel Function (I)).
 *   FP64 lattice: 53 random bits from words (2(j&1), 2(j&1)+1) of the block at
 *                 counter j>>1; u = m 2^-53; x = fma(ub-lb, u, lb), clamped.
 *   FP32 lattice: 24 random bits from word j&3 of the block at counter j>>2;
 *                 u = m 2^-24 (a float); x = fmaf(S, u, L) with S, L the
 *                 nearest floats to ub-lb and lb; x is then clamped to
 *                 [lbf, ubf], the smallest / largest floats inside [lb, ub]. */
static float float_at_or_above(double v)
{
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}

static float float_at_or_below(double v)
{
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}

double oracle_fresh(int lattice, uint64_t seed, uint32_t sid, uint32_t tag, uint32_t g,
                    uint32_t i, uint32_t j, double lb, double ub)
{
    uint32_t w[4];
    if (lattice == LATTICE_F64) {
        philox_block(seed, j >> 1, i, g, tag, sid, w);
        uint64_t lo = w[2 * (j & 1)], hi = w[2 * (j & 1) + 1];
        uint64_t m = ((hi << 32) | lo) >> 11;
        double u = ldexp((double)m, -53);
        double x = fma(ub - lb, u, lb);
        if (x < lb) x = lb;
        if (x > ub) x = ub;
        return x;
    } else {
        philox_block(seed, j >> 2, i, g, tag, sid, w);
        float u = ldexpf((float)(w[j & 3] >> 8), -24);
        float S = (float)(ub - lb), L = (float)lb;
        float x = fmaf(S, u, L);
        float lbf = float_at_or_above(lb), ubf = float_at_or_below(ub);
        if (x < lbf) x = lbf;
        if (x > ubf) x = ubf;
        return (double)x;
    }
}

/* ------------------------------------------------------------------------ */
/* sin(pi x), own algorithm: x = n + r with n = nearest integer (half even) and
 * r = x - n exact in [-1/2, 1/2]; sin(pi x) = (-1)^n sin(pi r); sin(pi r) =
 * r * S(r^2) with S the Taylor series of sin(pi r)/r truncated after the r^20
 * term (truncation error < 2e-18 on |r| <= 1/2), evaluated by Horner with fma.
 * Coefficient k is the nearest double to (-1)^k pi^(2k+1) / (2k+1)!.
 * Accuracy: within 3 ulp of sin(pi x) (measured against 300-bit mpmath). */
static const double SINPI_C[11] = {
    0x1.921fb54442d18p+1,  /*  pi          */
    -0x1.4abbce625be53p+2, /* -pi^3/3!     */
    0x1.466bc6775aae2p+1,  /*  pi^5/5!     */
    -0x1.32d2cce62bd86p-1, /* -pi^7/7!     */
    0x1.50783487ee782p-4,  /*  pi^9/9!     */
    -0x1.e3074fde8871fp-8, /* -pi^11/11!   */
    0x1.e8f434d018d63p-12, /*  pi^13/13!   */
    -0x1.6fadb9f155744p-16,/* -pi^15/15!   */
    0x1.aaec32af93359p-21, /*  pi^17/17!   */
    -0x1.8a404211f9547p-26,/* -pi^19/19!   */
    0x1.2877020d52cf0p-31, /*  pi^21/21!   */
};

double oracle_sinpi(double x)
{
    double n = nearbyint(x);
    double r = x - n;
    double q = r * r;
    double p = SINPI_C[10];
    for (int k = 9; k >= 0; --k) p = fma(p, q, SINPI_C[k]);
    double s = r * p;
    if (fmod(n, 2.0) != 0.0) s = -s;
    return s;
}

/* ------------------------------------------------------------------------ */
/* expm1(x) = e^x - 1, own algorithm.  |x| <= ln2/2: x * E(x) with E the Taylor
 * series of (e^x - 1)/x truncated after x^13/14! (truncation < 3e-19).
 * Otherwise Cody-Waite reduction x = k ln2 + r, k = nearest integer to x/ln2,
 * r = x - k*LN2_HI - k*LN2_LO (two fma), and e^x - 1 = 2^k expm1(r) + (2^k - 1),
 * both scalings exact.  Accuracy: within 3 ulp (measured against mpmath). */
static const double LN2_HI = 0x1.62e42fefa39efp-1;  /* nearest double to ln 2      */
static const double LN2_LO = 0x1.abc9e3b39803fp-56; /* nearest double to ln2-LN2_HI */
static const double INV_LN2 = 0x1.71547652b82fep+0; /* nearest double to 1/ln 2    */
static const double EULER_E = 0x1.5bf0a8b145769p+1; /* nearest double to e         */

static double expm1_poly(double x)
{
    /* 1/1! + x/2! + x^2/3! + ... + x^13/14!; n! is exact in FP64 for n <= 18,
     * so each 1.0/n! below is the correctly rounded reciprocal. */
    static const double FACT[15] = { 1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0,
                                     40320.0, 362880.0, 3628800.0, 39916800.0,
                                     479001600.0, 6227020800.0, 87178291200.0 };
    double p = 1.0 / FACT[14];
    for (int k = 13; k >= 1; --k) p = fma(p, x, 1.0 / FACT[k]);
    return x * p;
}

double oracle_expm1(double x)
{
    if (fabs(x) <= 0.5 * LN2_HI) return expm1_poly(x);
    double k = nearbyint(x * INV_LN2);
    double r = fma(-k, LN2_HI, x);
    r = fma(-k, LN2_LO, r);
    double e = expm1_poly(r);
    double two_k = ldexp(1.0, (int)k);
    return (e * two_k) + (two_k - 1.0);
}

/* ------------------------------------------------------------------------ */
/* Fitness of one particle (Kernel Function (E); definitions of Table 3.2, in
 * their shifted / rotated forms).  Summation order: see the file header. */
static double butterfly32(double v[32])
{
    for (int off = 16; off >= 1; off >>= 1) {
        double t[32];
        for (int l = 0; l < 32; ++l) t[l] = v[l] + v[l ^ off];
        memcpy(v, t, sizeof t);
    }
    return v[0];
}

static double butterfly32_mul(double v[32])
{
    for (int off = 16; off >= 1; off >>= 1) {
        double t[32];
        for (int l = 0; l < 32; ++l) t[l] = v[l] * v[l ^ off];
        memcpy(v, t, sizeof t);
    }
    return v[0];
}

/* cos(a) = 1 - 2 sin^2(a / 2) with sin(a / 2) = sin(pi q), q = a * (1 / (2 pi))
 * rounded once (INV_2PI the nearest double to 1 / (2 pi)); 1 - 2 s^2 as one
 * fma.  Error against cos(a): about 2^-52 (1 + |a|). */
static const double INV_2PI = 0x1.45f306dc9c883p-3;
double oracle_sinpi(double x);
static double cos_rad(double a)
{
    double s = oracle_sinpi(a * INV_2PI);
    return fma(-2.0 * s, s, 1.0);
}

/* sin(a) = sin(pi q), q = a * (1 / pi) rounded once (INV_PI the nearest double
 * to 1 / pi).  Error against sin(a): about 2^-52 (1 + |a|). */
static const double INV_PI = 0x1.45f306dc9c883p-2;
static double sin_rad(double a) { return oracle_sinpi(a * INV_PI); }

/* Table 3.2 f3, read as Schwefel's problem 1.2: sum_i (sum_{j<=i} z_j)^2.  The
 * prefix sums c_j follow a fixed blocked order over the 32-lane layout
 * (variable block b = j>>2 of 4 variables on lane b&31, slice s = b>>5 of
 * 128 variables):
 *   block total   T_b = ((z_4b + z_4b+1) + z_4b+2) + z_4b+3   (z = 0 beyond D)
 *   within slice  inclusive Kogge-Stone scan of the 32 block totals: for
 *                 off = 1, 2, 4, 8, 16, v_l <- v_(l-off) + v_l for l >= off
 *   slice carry   C_0 = 0, C_(s+1) = C_s + v_31 of slice s
 *   block start   B_b = C_s + (l > 0 ? v_(l-1) : 0)
 *   variables     c_4b = B_b + z_4b, c_(j+1) = c_j + z_(j+1) within the block
 * and the terms c_j^2 are summed like every other function's terms (lane
 * partials by fma in ascending j, then the butterfly). */
static void schwefel12_prefix(int64_t D, const double* z, double* c)
{
    const int64_t nb = (D + 3) / 4, ns = (nb + 31) / 32;
    double carry = 0.0;
    for (int64_t sl = 0; sl < ns; ++sl) {
        double v[32], nv[32];
        for (int l = 0; l < 32; ++l) {
            const int64_t b = 32 * sl + l;
            double t = 0.0;
            for (int m = 0; m < 4; ++m) {
                const int64_t j = 4 * b + m;
                const double zj = (j < D) ? z[j] : 0.0;
                t = (m == 0) ? zj : t + zj;
            }
            v[l] = (b < nb) ? t : 0.0;
        }
        for (int off = 1; off < 32; off <<= 1) {
            for (int l = 0; l < 32; ++l) nv[l] = (l >= off) ? v[l - off] + v[l] : v[l];
            memcpy(v, nv, sizeof v);
        }
        for (int l = 0; l < 32; ++l) {
            const int64_t b = 32 * sl + l;
            if (b >= nb) break;
            double run = carry + ((l > 0) ? v[l - 1] : 0.0);
            for (int m = 0; m < 4; ++m) {
                const int64_t j = 4 * b + m;
                if (j >= D) break;
                run = run + z[j];
                c[j] = run;
            }
        }
        carry = carry + v[31];
    }
}

double oracle_fitness(int fn, int64_t D, const double* x, const double* o,
                      const double* w, const double* M)
{
    double* z = (double*)malloc((size_t)D * sizeof(double));
    double* d = (double*)malloc((size_t)D * sizeof(double));
    double acc[32], acc2[32];
    for (int l = 0; l < 32; ++l) { acc[l] = 0.0; acc2[l] = 1.0; }
    for (int64_t j = 0; j < D; ++j) d[j] = x[j] - (o ? o[j] : 0.0);
    int rotated = (fn == FN_ROT_ELLIPSOID || fn == FN_ROT_RASTRIGIN || fn == FN_ROT_ACKLEY);
    if (rotated) {
        /* z = M d: row j of M dotted with d, k ascending from +0.0, fma. */
        for (int64_t j = 0; j < D; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < D; ++k) s = fma(M[j * D + k], d[k], s);
            z[j] = s;
        }
    } else {
        for (int64_t j = 0; j < D; ++j) z[j] = d[j];
    }
    int base = fn;
    if (fn == FN_ROT_ELLIPSOID) base = FN_ELLIPSOID;
    if (fn == FN_ROT_RASTRIGIN) base = FN_RASTRIGIN;
    if (fn == FN_ROT_ACKLEY) base = FN_ACKLEY;

    double* c = NULL;
    if (base == FN_SCHWEFEL12) {
        c = (double*)malloc((size_t)D * sizeof(double));
        schwefel12_prefix(D, z, c);
    }
    if (base == FN_ACKLEY)
        for (int l = 0; l < 32; ++l) acc2[l] = 0.0;
    for (int64_t j = 0; j < D; ++j) {
        int l = (int)((j >> 2) & 31);
        double zj = z[j];
        switch (base) {
        case FN_SPHERE:            /* sum z_j^2 */
            acc[l] = fma(zj, zj, acc[l]);
            break;
        case FN_ELLIPSOID:         /* sum w_j z_j^2, w_j = 10^(6 j/(D-1)) given as data */
            acc[l] = fma(w[j], zj * zj, acc[l]);
            break;
        case FN_RASTRIGIN: {       /* 10 D + sum (z^2 - 10 cos 2 pi z) = sum (z^2 + 20 sin^2 pi z) */
            double s = oracle_sinpi(zj);
            acc[l] = acc[l] + fma(zj, zj, 20.0 * (s * s));
            break;
        }
        case FN_ROSENBROCK:        /* sum_{j<D-1} 100 (a_{j+1} - a_j^2)^2 + (a_j - 1)^2, a = x - o + 1 */
            if (j < D - 1) {
                double a0 = d[j] + 1.0, a1 = d[j + 1] + 1.0;
                double u = fma(-a0, a0, a1);
                acc[l] = acc[l] + fma(100.0 * u, u, d[j] * d[j]);
            }
            break;
        case FN_ACKLEY: {          /* S1 = sum z^2, Q = sum sin^2 pi z */
            acc[l] = fma(zj, zj, acc[l]);
            double s = oracle_sinpi(zj);
            acc2[l] = fma(s, s, acc2[l]);
            break;
        }
        case FN_HYPER_ELLIPSOID:   /* f2: sum (j+1) z_j^2 */
            acc[l] = fma((double)(j + 1), zj * zj, acc[l]);
            break;
        case FN_SCHWEFEL12:        /* f3: sum c_j^2, c the prefix sums of z */
            acc[l] = fma(c[j], c[j], acc[l]);
            break;
        case FN_GRIEWANK:          /* f7: S = sum z^2 (divided by 4000 below), P = prod cos(z_j / sqrt(j+1)) */
            acc[l] = fma(zj, zj, acc[l]);
            acc2[l] = acc2[l] * cos_rad(zj / sqrt((double)(j + 1)));
            break;
        case FN_POWELL:            /* f8: one term per block of 4 variables (z = 0 beyond D) */
            if ((j & 3) == 0) {
                const double z0 = zj, z1 = (j + 1 < D) ? z[j + 1] : 0.0;
                const double z2 = (j + 2 < D) ? z[j + 2] : 0.0, z3 = (j + 3 < D) ? z[j + 3] : 0.0;
                const double a = fma(10.0, z1, z0), b = z2 - z3;
                const double cc = fma(-2.0, z2, z1), dd = z0 - z3;
                const double c2 = cc * cc, d2 = dd * dd;
                /* (z0 + 10 z1)^2 + 5 (z2 - z3)^2 + (z1 - 2 z2)^4 + 10 (z0 - z3)^4 */
                const double t = fma(a, a, fma(5.0 * b, b, fma(c2, c2, 10.0 * (d2 * d2))));
                acc[l] = acc[l] + t;
            }
            break;
        case FN_SCHWEFEL:          /* f9: S = sum z_j sin(sqrt|z_j|) */
            acc[l] = fma(zj, sin_rad(sqrt(fabs(zj))), acc[l]);
            break;
        }
    }
    double f = butterfly32(acc);
    if (base == FN_GRIEWANK) {     /* 1 + S / 4000 - P, evaluated as (1 - P) + S / 4000 */
        double P = butterfly32_mul(acc2);
        f = (1.0 - P) + f / 4000.0;
    }
    if (base == FN_SCHWEFEL)       /* 418.9829 D - S */
        f = 418.9829 * (double)D - f;
    free(c);
    if (base == FN_ACKLEY) {
        /* -20 exp(-0.2 sqrt(S1/D)) - exp(sum cos(2 pi z)/D) + 20 + e
         *   = -20 expm1(-0.2 sqrt(S1/D)) - e expm1(-2 Q/D)              */
        double S1 = f, Q = butterfly32(acc2), Dd = (double)D;
        double A = sqrt(S1 / Dd);
        double B = oracle_expm1(-0.2 * A);
        double C = oracle_expm1(-2.0 * (Q / Dd));
        f = -((20.0 * B) + (EULER_E * C));
    }
    free(z);
    free(d);
    return f;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2.1 for one particle: every variable of x_i is replaced by gBest_j,
 * pBest_ij, kept, or drawn fresh, according to the interval its draw falls in.
 *   order 0: intervals [0, Cg) -> gBest, [Cg, Cp) -> pBest, [Cp, Cw) -> keep,
 *            [Cw, 1) -> fresh (cumulative Cg <= Cp <= Cw);
 *   order 1: the order Eq. 2.1 prints: [0, Cw) -> keep, [Cw, Cp) -> pBest,
 *            [Cp, Cg) -> gBest, [Cg, 1) -> fresh (cumulative Cw <= Cp <= Cg).
 * T1 <= T2 <= T3 are the interval ends on the 32-bit draw.  nb counts the
 * branches taken (gBest, pBest, keep, fresh). */
enum { BR_GBEST = 0, BR_PBEST = 1, BR_KEEP = 2, BR_FRESH = 3 };

static void stepwise_update(int order, int lattice, uint64_t seed, uint32_t sid, uint32_t g,
                            uint32_t i, int64_t D, double lb, double ub, uint64_t T1,
                            uint64_t T2, uint64_t T3, const double* G, const double* p,
                            double* x, int64_t nb[4])
{
    const int first = order ? BR_KEEP : BR_GBEST;
    const int third = order ? BR_GBEST : BR_KEEP;
    for (int64_t j = 0; j < D; ++j) {
        uint64_t r = oracle_rho(seed, sid, g, i, (uint32_t)j);
        int br = (r < T1) ? first : (r < T2) ? BR_PBEST : (r < T3) ? third : BR_FRESH;
        if (br == BR_GBEST) x[j] = G[j];
        else if (br == BR_PBEST) x[j] = p[j];
        else if (br == BR_FRESH)
            x[j] = oracle_fresh(lattice, seed, sid, TAG_FRESH, g, i, (uint32_t)j, lb, ub);
        nb[br]++;
    }
}

/* One SSO run.  Returns 0, or a negative code for invalid arguments.
 *   order : 0 or 1, the interval order of Eq. 2.1 (see stepwise_update).
 *   flow  : 0 = synchronous generations (Alg. 2, the PSSO flow): every
 *           particle searches with the gBest of the previous generation, pBest
 *           is replaced when f <= pF (Alg. 3), and gBest is then the
 *           lowest-index arg-min of pF (Alg. 4);
 *           1 = asynchronous generations (Alg. 1, the sequential CPU-SSO):
 *           particles are taken one after the other in index order, each
 *           searches (Eq. 2.1), is evaluated, replaces its pBest when f < pF
 *           and the gBest when f < gF (both strict, as Alg. 1 writes them), so
 *           particle i already sees a gBest found earlier in the same
 *           generation.  Generation 0 is the same in both flows.
 *   X, P : N*D row-major (outputs: final positions and pBests)
 *   pF   : N (output: final pBest fitness)
 *   G    : D (output: final gBest row)
 *   log_b, log_v, log_acc : t+1 entries each or NULL -- per generation g the
 *          gBest index, its fitness and the number of accepted pBest updates.
 *   branch : 4 counters or NULL -- how often each branch of Eq. 2.1 fired
 *          (gBest, pBest, keep, fresh) over generations 1..t.
 *   nthreads : >1 parallelises the per-particle work of a synchronous
 *          generation with OpenMP; every particle's work is independent and
 *          the arg-min is sequential, so the result is bit-identical to
 *          nthreads = 1 (the asynchronous flow is sequential by definition). */
int oracle_run_ex(int fn, int lattice, int order, int flow, int64_t N, int64_t D, double lb,
                  double ub, double Cg, double Cp, double Cw, uint64_t seed, uint32_t sid,
                  const double* o, const double* w, const double* M, int64_t t, int nthreads,
                  double* X, double* P, double* pF, double* G, int64_t* log_b, double* log_v,
                  int64_t* log_acc, int64_t* branch)
{
    if (fn < 0 || fn >= FN_COUNT || N < 1 || D < 1 || t < 0) return -1;
    if (order != 0 && order != 1) return -2;
    if (flow != 0 && flow != 1) return -2;
    if (!(lb < ub)) return -2;
    if (order == 0 && !(0.0 <= Cg && Cg <= Cp && Cp <= Cw && Cw <= 1.0)) return -2;
    if (order == 1 && !(0.0 <= Cw && Cw <= Cp && Cp <= Cg && Cg <= 1.0)) return -2;
    if (lattice != LATTICE_F64 && lattice != LATTICE_F32) return -3;
    if (lattice == LATTICE_F32 && !(float_at_or_above(lb) <= float_at_or_below(ub))) return -2;
    if ((fn == FN_ELLIPSOID || fn == FN_ROT_ELLIPSOID) && !w) return -4;
    if ((fn == FN_ROT_ELLIPSOID || fn == FN_ROT_RASTRIGIN || fn == FN_ROT_ACKLEY) && !M) return -4;
    if (N > 0xffffffffLL || D > 0xffffffffLL || t > 0xffffffffLL || sid >= (1u << 24)) return -5;
    if (nthreads < 1) nthreads = 1;

    /* Eq. 2.1 interval ends on the 32-bit draw, in increasing order. */
    const uint64_t T1 = (uint64_t)nearbyint(ldexp(order ? Cw : Cg, 32));
    const uint64_t T2 = (uint64_t)nearbyint(ldexp(Cp, 32));
    const uint64_t T3 = (uint64_t)nearbyint(ldexp(order ? Cg : Cw, 32));
    int64_t nb[4] = { 0, 0, 0, 0 };

    /* Generation 0: Kernel Function (I) -- random population; pBest = X0. */
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = 0; j < D; ++j)
            X[i * D + j] = oracle_fresh(lattice, seed, sid, TAG_INIT, 0, (uint32_t)i, (uint32_t)j, lb, ub);
        memcpy(P + i * D, X + i * D, (size_t)D * sizeof(double));
        pF[i] = oracle_fitness(fn, D, X + i * D, o, w, M);
    }
    int64_t b = 0;
    for (int64_t i = 1; i < N; ++i) if (pF[i] < pF[b]) b = i;
    memcpy(G, P + b * D, (size_t)D * sizeof(double));
    double gF = pF[b];
    if (log_b) log_b[0] = b;
    if (log_v) log_v[0] = gF;
    if (log_acc) log_acc[0] = N;

    for (int64_t g = 1; g <= t; ++g) {
        int64_t accepted = 0;
        if (flow == 0) {
            int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
            /* Alg. 2: search for all particles (Eq. 2.1) reading gBest of g-1, then
             * evaluate (Kernel Function (E)) and update pBests (Alg. 3, "<="). */
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(+ : accepted, c0, c1, c2, c3)
            for (int64_t i = 0; i < N; ++i) {
                double* xi = X + i * D;
                double* pi = P + i * D;
                int64_t c[4] = { 0, 0, 0, 0 };
                stepwise_update(order, lattice, seed, sid, (uint32_t)g, (uint32_t)i, D, lb, ub, T1,
                                T2, T3, G, pi, xi, c);
                c0 += c[0]; c1 += c[1]; c2 += c[2]; c3 += c[3];
                double fi = oracle_fitness(fn, D, xi, o, w, M);
                if (fi <= pF[i]) {
                    memcpy(pi, xi, (size_t)D * sizeof(double));
                    pF[i] = fi;
                    accepted++;
                }
            }
            nb[0] += c0; nb[1] += c1; nb[2] += c2; nb[3] += c3;
            /* Alg. 4: gBest = lowest-index arg-min over all pBest fitness values. */
            b = 0;
            for (int64_t i = 1; i < N; ++i) if (pF[i] < pF[b]) b = i;
            memcpy(G, P + b * D, (size_t)D * sizeof(double));
            gF = pF[b];
        } else {
            /* Alg. 1: one particle after the other; search, evaluate, then the
             * pBest and gBest replacements ("<" both), in particle order. */
            for (int64_t i = 0; i < N; ++i) {
                double* xi = X + i * D;
                double* pi = P + i * D;
                stepwise_update(order, lattice, seed, sid, (uint32_t)g, (uint32_t)i, D, lb, ub, T1,
                                T2, T3, G, pi, xi, nb);
                double fi = oracle_fitness(fn, D, xi, o, w, M);
                if (fi < pF[i]) {
                    memcpy(pi, xi, (size_t)D * sizeof(double));
                    pF[i] = fi;
                    accepted++;
                    if (fi < gF) {
                        memcpy(G, xi, (size_t)D * sizeof(double));
                        gF = fi;
                        b = i;
                    }
                }
            }
        }
        if (log_b) log_b[g] = b;
        if (log_v) log_v[g] = gF;
        if (log_acc) log_acc[g] = accepted;
    }
    if (branch) for (int k = 0; k < 4; ++k) branch[k] = nb[k];
    return 0;
}

/* The synchronous run in the default interval order (order 0, flow 0). */
int oracle_run(int fn, int lattice, int64_t N, int64_t D, double lb, double ub,
               double Cg, double Cp, double Cw, uint64_t seed, uint32_t sid,
               const double* o, const double* w, const double* M,
               int64_t t, int nthreads,
               double* X, double* P, double* pF, double* G,
               int64_t* log_b, double* log_v, int64_t* log_acc, int64_t* branch)
{
    return oracle_run_ex(fn, lattice, 0, 0, N, D, lb, ub, Cg, Cp, Cw, seed, sid, o, w, M, t,
                         nthreads, X, P, pF, G, log_b, log_v, log_acc, branch);
}

/* Maximum OpenMP threads the compiled oracle can use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
