// gradient.cu -- differentiable batched fitness: FP32 forward and backward
// kernels for every test function (psso_fitness_forward / _backward), and the
// gBest gradient polish of a swarm (the kernel behind psso_polish).
//
// Gradients with z the function's coordinates (z = x - o, or z = M (x - o)):
//   sphere      2 z_j                        ellipsoid   2 w_j z_j
//   Rastrigin   2 z_j + 20 pi sin(2 pi z_j)
//   Rosenbrock  [j<D-1] (2 d_j - 400 a_j u_j) + [j>0] 200 u_{j-1},
//               a = d + 1, u_j = a_{j+1} - a_j^2 = d_{j+1} - d_j (d_j + 2)
//   Ackley      4 e^{-0.2 A} z_j / (A D) + 2 pi e^{C} sin(2 pi z_j) / D,
//               A = sqrt(sum z^2 / D), C = sum cos(2 pi z) / D = 1 - 2 Q / D
// and for rotated functions df/dx = M^T df/dz.
#include "psso.h"
#include "rot_pipeline.h"
#include "sso_kernel.cuh"
#include "tc_gemm.cuh"

namespace psso {

// sin(2 pi z) in FP32: 2z = n + r, sin(pi (n + r)) = (-1)^n sin(pi r).
__device__ __forceinline__ float sin2pi_f32(float z)
{
    const float y = __fmul_rn(2.f, z);
    const float n = rintf(y);
    const float s = sinpi_reduced_f32(__fsub_rn(y, n));
    return (((int)n) & 1) ? -s : s;
}

// Fitness (FP32) and its gradient with respect to x for one row held by a full
// warp in the 32-lane chunk layout (x: lane chunks lane + 32 q).
template <int MAXC, bool WANT_GRAD = true>
__device__ float grad32(const Hot& in, const float (&x)[MAXC][4], float (&gx)[MAXC][4])
{
    const int lane = threadIdx.x & 31;
    const int D = in.D;
    const bool rot = is_rotated(in.fn);
    const int fn = base_fn(in.fn);
    float z[MAXC][4], gz[MAXC][4];
    if (rot) {
        float ez[MAXC][4];
        rot_matvec32<MAXC>(in, x, lane, 0xffffffffu, 32, z, ez);
    } else {
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * (lane + 32 * q) + m;
                z[q][m] = (j < D) ? __fsub_rn(x[q][m], __ldg(in.o32 + j)) : 0.f;
            }
    }
    // Sums each function needs (all lanes end with the totals).
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane + 32 * q) + m;
            if (j >= D) continue;
            const float zj = z[q][m];
            if (fn == FN_ACKLEY) {
                s1 = __fmaf_rn(zj, zj, s1);
                const float s = sinpi_reduced_f32(__fsub_rn(zj, rintf(zj)));
                s2 = __fmaf_rn(s, s, s2);
            }
        }
    float Ae = 0.f, Ce = 0.f, A = 0.f;
    if (fn == FN_ACKLEY) {
        for (int off = 16; off > 0; off >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        }
        A = sqrtf(s1 / (float)D);
        Ae = expf(-0.2f * A);                        // e^{-0.2 A}
        Ce = 2.7182818f * expf(-2.f * s2 / (float)D);  // e^{C}
    }
    // Rosenbrock terms u_j = d_{j+1} - d_j (d_j + 2): d_{j+1} is the same lane's
    // next variable, or the first variable of the next chunk (lane + 1, or lane 0
    // of the next q for lane 31).
    float u[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const float first_next = __shfl_down_sync(0xffffffffu, z[q][0], 1);
        const float wrap = __shfl_sync(0xffffffffu, z[(q + 1) % MAXC][0], 0);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane + 32 * q) + m;
            float nx = (m < 3) ? z[q][m < 3 ? m + 1 : 0] : (lane == 31 ? (q + 1 < MAXC ? wrap : 0.f) : first_next);
            if (j + 1 >= D) nx = 0.f;
            u[q][m] = __fmaf_rn(-z[q][m], __fadd_rn(z[q][m], 2.f), nx);
        }
    }
    float f = 0.f;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        // u_{j-1}: same lane (m > 0), lane - 1's last term, or lane 31's last term of q - 1
        const float last_prev = __shfl_up_sync(0xffffffffu, u[q][3], 1);
        const float wrap = __shfl_sync(0xffffffffu, u[(q + MAXC - 1) % MAXC][3], 31);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane + 32 * q) + m;
            const float up = (m > 0) ? u[q][m > 0 ? m - 1 : 0] : (lane == 0 ? (q > 0 ? wrap : 0.f) : last_prev);
            float g = 0.f;
            const float zj = z[q][m];
            if (j < D) {
                switch (fn) {
                case FN_SPHERE:
                    g = 2.f * zj;
                    f = __fmaf_rn(zj, zj, f);
                    break;
                case FN_ELLIPSOID: {
                    const float w = __ldg(in.w32 + j);
                    g = 2.f * w * zj;
                    f = __fmaf_rn(w * zj, zj, f);
                    break;
                }
                case FN_RASTRIGIN: {
                    const float s = sinpi_reduced_f32(__fsub_rn(zj, rintf(zj)));
                    g = __fmaf_rn(62.8318548f, sin2pi_f32(zj), 2.f * zj);
                    f = __fadd_rn(f, __fmaf_rn(zj, zj, 20.f * s * s));
                    break;
                }
                case FN_ROSENBROCK: {
                    const float a = __fadd_rn(zj, 1.f);
                    if (j < D - 1) {
                        g = __fmaf_rn(-400.f * a, u[q][m], 2.f * zj);
                        f = __fadd_rn(f, __fmaf_rn(100.f * u[q][m], u[q][m], zj * zj));
                    }
                    if (j > 0) g = __fmaf_rn(200.f, up, g);
                    break;
                }
                default: {   // Ackley
                    const float lin = (A > 0.f) ? 4.f * Ae * zj / (A * (float)D) : 0.f;
                    g = __fmaf_rn(6.28318548f * Ce / (float)D, sin2pi_f32(zj), lin);
                    break;
                }
                }
            }
            gz[q][m] = g;
        }
    }
    if (fn == FN_ACKLEY) {
        f = -20.f * expm1f(-0.2f * A) - 2.7182818f * expm1f(-2.f * s2 / (float)D);
    } else {
        for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
    }
    if (!rot || !WANT_GRAD) {
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) gx[q][m] = gz[q][m];
        return f;
    }
    // df/dx_k = sum_j M_jk df/dz_j: each df/dz_j broadcast from its lane.
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) gx[q][m] = 0.f;
#pragma unroll
    for (int qj = 0; qj < MAXC; ++qj) {
        for (int l = 0; l < 32; ++l) {
            if (128 * qj + 4 * l >= D) break;
#pragma unroll
            for (int mj = 0; mj < 4; ++mj) {
                const int j = 128 * qj + 4 * l + mj;
                const float gj = __shfl_sync(0xffffffffu, gz[qj][mj], l);
                if (j < D) {
#pragma unroll
                    for (int q = 0; q < MAXC; ++q)
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int k = 4 * (lane + 32 * q) + m;
                            if (k < D) gx[q][m] = __fmaf_rn(__ldg(in.M32 + (size_t)j * D + k), gj, gx[q][m]);
                        }
                }
            }
        }
    }
    return f;
}

// One warp per row of X (N x D floats, unpadded): f (forward) or grad_X =
// grad_f[row] * df/dx (backward).
template <bool BWD, int MAXC>
__device__ void fb_row(const Hot& in, const float* xr, float gfr, float* f, float* gxr)
{
    const int lane = threadIdx.x & 31;
    float x[MAXC][4], g[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane + 32 * q) + m;
            x[q][m] = j < in.D ? xr[j] : 0.f;
        }
    const float v = grad32<MAXC, BWD>(in, x, g);
    if constexpr (!BWD) {
        if (lane == 0) *f = v;
    } else {
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * (lane + 32 * q) + m;
                if (j < in.D) gxr[j] = gfr * g[q][m];
            }
    }
}

template <bool BWD>
__global__ void fitness_fb(const Hot in, const float* X, int64_t N, const float* gf, float* f, float* gx)
{
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= N) return;
    if (!PSSO_CHK(in.maxc * 128 >= in.D, CHK_EVAL_ROW, in.D)) return;
    const float* xr = X + row * in.D;
    const float gfr = BWD ? gf[row] : 0.f;
    float* fo = BWD ? nullptr : f + row;
    float* gxr = BWD ? gx + row * in.D : nullptr;
    switch (in.maxc) {
    case 1: fb_row<BWD, 1>(in, xr, gfr, fo, gxr); break;
    case 2: fb_row<BWD, 2>(in, xr, gfr, fo, gxr); break;
    case 4: fb_row<BWD, 4>(in, xr, gfr, fo, gxr); break;
    default: fb_row<BWD, 8>(in, xr, gfr, fo, gxr); break;
    }
}

// gBest polish of instance k: `steps` gradient steps x <- clamp(x - lr df/dx)
// from the gBest row, then the polished row's FP64 fitness in the oracle's
// order; it replaces the gBest particle's pBest (and the gBest) only if that
// value is lower.  Multi-block instances also get the owner block's record
// and row of generation g rewritten, so the next launch sees the new gBest.
template <class Pos, int MAXC>
__device__ void polish_row(const InstDev& in, int owner_rank, int64_t g, int steps, float lr)
{
    const int lane = threadIdx.x & 31;
    const Hot hin = hot_of(in);
    const Pos lo_b = sizeof(Pos) == 4 ? (Pos)in.lbf : (Pos)in.lb;
    const Pos hi_b = sizeof(Pos) == 4 ? (Pos)in.ubf : (Pos)in.ub;
    Pos xp[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
        if (c < in.nchunks) ld4(static_cast<const Pos*>(in.gbrow) + 4 * c, xp[q]);
        else xp[q][0] = xp[q][1] = xp[q][2] = xp[q][3] = Pos(0);
    }
    const double fold = in.gb->has64 ? in.gb->f64 : fit64<Pos, MAXC>(hin, xp, lane, 0xffffffffu, 32);
    // The gradient is taken in FP32 at the row rounded to floats; the step is
    // applied to the row in its own precision and clamped to the box.
    for (int s = 0; s < steps; ++s) {
        float x[MAXC][4], gr[MAXC][4];
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) x[q][m] = (float)xp[q][m];
        grad32<MAXC, true>(hin, x, gr);
#pragma unroll
        for (int q = 0; q < MAXC; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int j = 4 * (lane + 32 * q) + m;
                if (j < in.D) {
                    const Pos v = xp[q][m] - (Pos)(lr * gr[q][m]);
                    xp[q][m] = v < lo_b ? lo_b : (v > hi_b ? hi_b : v);
                }
            }
    }
    const double fnew = fit64<Pos, MAXC>(hin, xp, lane, 0xffffffffu, 32);
    if (!(fnew < fold)) return;
    const int64_t b = in.gb->idx;
    if (!PSSO_CHK(b >= 0 && b < in.N && owner_rank < in.R, CHK_GBEST_SRC, b)) return;
    Pos* prow = static_cast<Pos*>(in.P) + b * in.Dp;
    Pos* gw = static_cast<Pos*>(in.gbrow);
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane + 32 * q;
        if (c < in.nchunks) {
            st4(prow + 4 * c, xp[q]);
            st4(gw + 4 * c, xp[q]);
        }
    }
    const float lo = f64_to_f32_rd(fnew), hi = f64_to_f32_ru(fnew);
    if (in.R > 1 && owner_rank >= 0) {
        constexpr int WPE = WordsPer<Pos>::value;
        const uint32_t tag = (uint32_t)g;
        uint64_t* rw = static_cast<uint64_t*>(in.grow) +
                       ((size_t)slot_of(g) * in.R + owner_rank) * (size_t)in.Dp * WPE;
#pragma unroll
        for (int q = 0; q < MAXC; ++q) {
            const int c = lane + 32 * q;
            if (c < in.nchunks) put_chunk(rw + (size_t)4 * c * WPE, tag, xp[q]);
        }
    }
    __syncwarp();
    if (lane == 0) {
        in.pf64[b] = fnew;
        in.pver[b] = (uint32_t)g;
        if (in.plo) {
            in.plo[b] = lo;
            in.phi[b] = hi;
            in.pflag[b] = 1u;
        }
        in.gb->f64 = fnew;
        in.gb->has64 = 1;
        in.gb->lo = lo;
        in.gb->hi = hi;
        in.gb->ver = (uint32_t)g;
        if (in.R > 1 && owner_rank >= 0) {
            uint64_t* rec = in.rec + ((size_t)slot_of(g) * in.R + owner_rank) * REC_WORDS;
            Winner w;
            w.idx = b;
            w.ver = (uint32_t)g;
            w.has64 = 1;
            w.f64 = fnew;
            w.lo = lo;
            w.hi = hi;
            w.acc = rec[RW_ACC] & 0xffffffffffffULL;
            w.rck = rec[RW_RCK] & 0xffffffffffffULL;
            publish_record(rec, (uint32_t)g, w);
        }
    }
}

template <class Pos>
__global__ void polish_kernel(const InstDev* inst, int k, int owner_rank, int64_t g, int steps, float lr)
{
    const InstDev& in = inst[k];
    switch (in.maxc) {
    case 1: polish_row<Pos, 1>(in, owner_rank, g, steps, lr); break;
    case 2: polish_row<Pos, 2>(in, owner_rank, g, steps, lr); break;
    case 4: polish_row<Pos, 4>(in, owner_rank, g, steps, lr); break;
    default: polish_row<Pos, 8>(in, owner_rank, g, steps, lr); break;
    }
}

cudaError_t launch_polish(const InstDev* inst, int k, int lattice, int owner_rank, int64_t g, int steps,
                          float lr, cudaStream_t s)
{
    if (lattice == 1) polish_kernel<float><<<1, 32, 0, s>>>(inst, k, owner_rank, g, steps, lr);
    else polish_kernel<double><<<1, 32, 0, s>>>(inst, k, owner_rank, g, steps, lr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rotated functions on the tensor cores (the *_ws entry points):
//   forward   Z = (X - O) M^T        split-BF16 tcgen05 GEMM (tc_gemm.cuh)
//             f_i from row Z_i       the unrotated function's FP32 kernel, o = 0
//   backward  G_i = grad_f_i df/dz   from Z (same kernel, its z-gradient)
//             grad_X = G M           second GEMM, B operand = the planes of M^T
// Both GEMMs run the six split products of tc_gemm.cuh with FP32
// accumulation: each output carries an error below 2^-20 per MMA of
// sum |A_ik| |B_jk| (tc_gemm.cuh), typically far less.
namespace gtc {

using tc::BM;
using tc::BN;
using tc::BK;

// B planes of M^T: row k of the [Jp][Kp] planes holds column k of M.
__global__ void split_matrix_t(const float* __restrict__ M, int D, int Jp, int Kp, __nv_bfloat16* B)
{
    const int k = blockIdx.x;
    const size_t plane = (size_t)Jp * Kp;
    for (int j = threadIdx.x; j < Kp; j += blockDim.x) {
        const float v = (k < D && j < D) ? M[(size_t)j * D + k] : 0.f;
        __nv_bfloat16 h, m, l;
        tc::split3(v, h, m, l);
        const size_t o = (size_t)k * Kp + j;
        B[o] = h;
        B[plane + o] = m;
        B[2 * plane + o] = l;
    }
}

// C tile -> out[i * D + j] (rows < N, columns < D).
struct StoreEpi {
    float* out;
    int N, D;
    __device__ void operator()(int c, const float (&z)[32]) const
    {
        const int i = blockIdx.x * BM + threadIdx.x;
        const int j0 = blockIdx.y * BN + 32 * c;
        if (i >= N) return;
#pragma unroll
        for (int t = 0; t < 32; ++t)
            if (j0 + t < D) out[(size_t)i * D + j0 + t] = z[t];
    }
};

__global__ void __launch_bounds__(128, 1)
    grad_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, tc::GemmArgs a,
              StoreEpi epi)
{
    tc::gemm_tile(&tmA, &tmB, a, epi);
}

// A planes of G = grad_f_i df/dz for the rows of Z (warp per row of the padded
// Np x Kp planes; padding zero): the unrotated function's gradient at z.
template <int MAXC>
__global__ void gz_split(const Hot hz, const float* Z, int64_t N, const float* gf, int Np, int Kp,
                         __nv_bfloat16* A)
{
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= Np) return;
    const int lane = threadIdx.x & 31;
    const int D = hz.D;
    float z[MAXC][4], g[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane + 32 * q) + m;
            z[q][m] = (i < N && j < D) ? Z[i * D + j] : 0.f;
        }
    if (i < N) grad32<MAXC, true>(hz, z, g);
    const float scale = i < N ? gf[i] : 0.f;
    const size_t plane = (size_t)Np * Kp;
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = 4 * (lane + 32 * q) + m;
            if (j >= Kp) continue;
            const float v = (i < N && j < D) ? __fmul_rn(scale, g[q][m]) : 0.f;
            __nv_bfloat16 h, mm, l;
            tc::split3(v, h, mm, l);
            const size_t o = (size_t)i * Kp + j;
            A[o] = h;
            A[plane + o] = mm;
            A[2 * plane + o] = l;
        }
    // columns beyond this lane layout's reach (Kp may exceed 4 * 32 * MAXC only
    // when D does not fill the last 64-wide block): zero them
    for (int j = 128 * MAXC + lane; j < Kp; j += 32) {
        const size_t o = (size_t)i * Kp + j;
        A[o] = A[plane + o] = A[2 * plane + o] = __float2bfloat16_rn(0.f);
    }
}

// Workspace layout of the tensor-core path (byte offsets, 256-aligned).
struct WsLayout {
    int Np, Jp, Kp;
    size_t a, b, bt, mn, z, zero, status, total;
};
inline size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }
inline WsLayout ws_layout(int64_t N, int64_t D)
{
    WsLayout w{};
    w.Np = (int)((N + BM - 1) / BM * BM);
    w.Jp = (int)((D + BN - 1) / BN * BN);
    w.Kp = (int)((D + BK - 1) / BK * BK);
    size_t off = 0;
    auto take = [&](size_t n) { const size_t at = off; off = al256(off + n); return at; };
    w.a = take((size_t)3 * w.Np * w.Kp * 2);
    w.b = take((size_t)3 * w.Jp * w.Kp * 2);
    w.bt = take((size_t)3 * w.Jp * w.Kp * 2);
    w.mn = take((size_t)w.Jp * 4);
    w.z = take((size_t)N * D * 4);
    w.zero = take((size_t)(D + 4) * 4);
    w.status = take(4);
    w.total = off;
    return w;
}

}  // namespace gtc
}  // namespace psso

namespace {

psso_status fb_check(psso_fn fn, int64_t N, int64_t D, const float* X, const float* shift,
                     const float* weights, const float* rotation)
{
    using namespace psso;
    if (fn > PSSO_ROT_ACKLEY && fn <= PSSO_SCHWEFEL) {
        set_last_error("psso_fitness_forward/backward: no FP32 gradient for this function "
                       "(the hyper-ellipsoid is ELLIPSOID with weights j + 1)");
        return PSSO_ERR_UNSUPPORTED;
    }
    if (!X || !shift || N < 1 || D < 1 || D > 1024 || fn < PSSO_SPHERE || fn > PSSO_ROT_ACKLEY) {
        set_last_error("psso_fitness_forward/backward: need X, shift, N >= 1, 1 <= D <= 1024, a known function");
        return PSSO_ERR_ARG;
    }
    if ((fn == PSSO_ELLIPSOID || fn == PSSO_ROT_ELLIPSOID) && !weights) {
        set_last_error("psso_fitness_forward/backward: the ellipsoid needs weights");
        return PSSO_ERR_ARG;
    }
    if (fn >= PSSO_ROT_ELLIPSOID && !rotation) {
        set_last_error("psso_fitness_forward/backward: rotated functions need a rotation matrix");
        return PSSO_ERR_ARG;
    }
    return PSSO_OK;
}

psso::Hot fb_hot(psso_fn fn, int64_t D, const float* shift, const float* weights, const float* rotation)
{
    psso::Hot in{};
    const int nchunks = (int)((D + 3) / 4);
    int maxc = 1;
    while (maxc < (nchunks + 31) / 32) maxc <<= 1;
    in.fn = fn;
    in.D = (int)D;
    in.Dp = 4 * nchunks;
    in.nchunks = nchunks;
    in.G = 32;
    in.maxc = maxc;
    in.o32 = shift;
    in.w32 = weights;
    in.M32 = rotation;
    return in;
}

}  // namespace

extern "C" psso_status psso_fitness_forward(psso_fn fn, int64_t N, int64_t D, const float* X,
                                            const float* shift, const float* weights,
                                            const float* rotation, float* f, void* stream)
{
    using namespace psso;
    psso_status st = fb_check(fn, N, D, X, shift, weights, rotation);
    if (st != PSSO_OK) return st;
    if (!f) {
        set_last_error("psso_fitness_forward: f is NULL");
        return PSSO_ERR_ARG;
    }
    const Hot in = fb_hot(fn, D, shift, weights, rotation);
    const int wpb = 8;
    fitness_fb<false><<<(unsigned)((N + wpb - 1) / wpb), 32 * wpb, 0, static_cast<cudaStream_t>(stream)>>>(
        in, X, N, nullptr, f, nullptr);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("psso_fitness_forward: launch failed");
        return PSSO_ERR_CUDA;
    }
    return PSSO_OK;
}

extern "C" psso_status psso_fitness_backward(psso_fn fn, int64_t N, int64_t D, const float* X,
                                             const float* shift, const float* weights,
                                             const float* rotation, const float* grad_f,
                                             float* grad_X, void* stream)
{
    using namespace psso;
    psso_status st = fb_check(fn, N, D, X, shift, weights, rotation);
    if (st != PSSO_OK) return st;
    if (!grad_f || !grad_X) {
        set_last_error("psso_fitness_backward: grad_f / grad_X is NULL");
        return PSSO_ERR_ARG;
    }
    const Hot in = fb_hot(fn, D, shift, weights, rotation);
    const int wpb = 8;
    fitness_fb<true><<<(unsigned)((N + wpb - 1) / wpb), 32 * wpb, 0, static_cast<cudaStream_t>(stream)>>>(
        in, X, N, grad_f, nullptr, grad_X);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("psso_fitness_backward: launch failed");
        return PSSO_ERR_CUDA;
    }
    return PSSO_OK;
}

// ---------------------------------------------------------------------------
// Tensor-core entry points (rotated functions; the others run the warp kernels
// above and need no workspace).
namespace {

bool uses_tc(psso_fn fn, int64_t D) { return fn >= PSSO_ROT_ELLIPSOID && fn <= PSSO_ROT_ACKLEY && D >= 16; }

psso::Hot base_hot(psso_fn fn, int64_t D, const float* zero, const float* weights)
{
    psso::Hot h = fb_hot(fn, D, zero, weights, nullptr);
    h.fn = fn == PSSO_ROT_ELLIPSOID ? PSSO_ELLIPSOID : fn == PSSO_ROT_RASTRIGIN ? PSSO_RASTRIGIN : PSSO_ACKLEY;
    return h;
}

// Operand planes of M (and of M^T for the backward pass), d = x - o, and Z.
psso_status tc_forward_z(int64_t N, int64_t D, const float* X, const float* shift, const float* rotation,
                         char* ws, const psso::gtc::WsLayout& L, bool transposed, cudaStream_t s,
                         CUtensorMap* tb_t)
{
    using namespace psso;
    auto* A = reinterpret_cast<__nv_bfloat16*>(ws + L.a);
    auto* B = reinterpret_cast<__nv_bfloat16*>(ws + L.b);
    auto* Bt = reinterpret_cast<__nv_bfloat16*>(ws + L.bt);
    CUtensorMap ta, tb;
    if (!tc::make_tmap_bf16(&ta, A, L.Kp, 3 * L.Np) || !tc::make_tmap_bf16(&tb, B, L.Kp, 3 * L.Jp) ||
        (transposed && !tc::make_tmap_bf16(tb_t, Bt, L.Kp, 3 * L.Jp))) {
        set_last_error("psso_fitness_*_ws: cuTensorMapEncodeTiled failed");
        return PSSO_ERR_CUDA;
    }
    float* Z = reinterpret_cast<float*>(ws + L.z);
    int* status = reinterpret_cast<int*>(ws + L.status);
    if (cudaMemsetAsync(ws + L.zero, 0, (size_t)(D + 4) * 4, s) != cudaSuccess ||
        cudaMemsetAsync(status, 0, 4, s) != cudaSuccess ||
        // a GEMM whose wait runs out writes nothing: its outputs then read NaN
        cudaMemsetAsync(Z, 0xff, (size_t)N * D * 4, s) != cudaSuccess ||
        tc::launch_split_matrix(rotation, (int)D, L.Jp, L.Kp, B, reinterpret_cast<float*>(ws + L.mn), s) !=
            cudaSuccess ||
        tc::launch_split_rows(X, shift, (int)N, (int)D, L.Np, L.Kp, A, s) != cudaSuccess) {
        set_last_error("psso_fitness_*_ws: operand preparation failed");
        return PSSO_ERR_CUDA;
    }
    if (transposed) gtc::split_matrix_t<<<L.Jp, 256, 0, s>>>(rotation, (int)D, L.Jp, L.Kp, Bt);
    static thread_local int smem_set_for = -1;   // the attribute is per device
    int dev = -1;
    cudaGetDevice(&dev);
    if (smem_set_for != dev) {
        cudaFuncSetAttribute(gtc::grad_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
        smem_set_for = dev;
    }
    tc::GemmArgs ga{L.Np, L.Jp, L.Kp, status};
    gtc::grad_gemm<<<dim3(L.Np / psso::tc::BM, L.Jp / psso::tc::BN), 128, tc::SMEM_BYTES, s>>>(ta, tb, ga,
                                                                           gtc::StoreEpi{Z, (int)N, (int)D});
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("psso_fitness_*_ws: GEMM launch failed");
        return PSSO_ERR_CUDA;
    }
    return PSSO_OK;
}

}  // namespace

extern "C" psso_status psso_fitness_workspace_size(psso_fn fn, int64_t N, int64_t D, size_t* bytes)
{
    using namespace psso;
    if (!bytes || N < 1 || D < 1 || D > 1024) {
        set_last_error("psso_fitness_workspace_size: need bytes, N >= 1, 1 <= D <= 1024");
        return PSSO_ERR_ARG;
    }
    *bytes = uses_tc(fn, D) ? gtc::ws_layout(N, D).total : 0;
    return PSSO_OK;
}

extern "C" psso_status psso_fitness_forward_ws(psso_fn fn, int64_t N, int64_t D, const float* X,
                                               const float* shift, const float* weights, const float* rotation,
                                               float* f, void* workspace, size_t ws_bytes, void* stream)
{
    using namespace psso;
    if (!uses_tc(fn, D)) return psso_fitness_forward(fn, N, D, X, shift, weights, rotation, f, stream);
    psso_status st = fb_check(fn, N, D, X, shift, weights, rotation);
    if (st != PSSO_OK) return st;
    const gtc::WsLayout L = gtc::ws_layout(N, D);
    if (!f || !workspace || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_last_error("psso_fitness_forward_ws: need f and a 256-byte aligned workspace of "
                       "psso_fitness_workspace_size bytes");
        return PSSO_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    st = tc_forward_z(N, D, X, shift, rotation, ws, L, false, s, nullptr);
    if (st != PSSO_OK) return st;
    const Hot hz = base_hot(fn, D, reinterpret_cast<const float*>(ws + L.zero), weights);
    const int wpb = 8;
    fitness_fb<false><<<(unsigned)((N + wpb - 1) / wpb), 32 * wpb, 0, s>>>(
        hz, reinterpret_cast<const float*>(ws + L.z), N, nullptr, f, nullptr);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("psso_fitness_forward_ws: launch failed");
        return PSSO_ERR_CUDA;
    }
    return PSSO_OK;
}

extern "C" psso_status psso_fitness_backward_ws(psso_fn fn, int64_t N, int64_t D, const float* X,
                                                const float* shift, const float* weights,
                                                const float* rotation, const float* grad_f, float* grad_X,
                                                void* workspace, size_t ws_bytes, void* stream)
{
    using namespace psso;
    if (!uses_tc(fn, D))
        return psso_fitness_backward(fn, N, D, X, shift, weights, rotation, grad_f, grad_X, stream);
    psso_status st = fb_check(fn, N, D, X, shift, weights, rotation);
    if (st != PSSO_OK) return st;
    const gtc::WsLayout L = gtc::ws_layout(N, D);
    if (!grad_f || !grad_X || !workspace || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_last_error("psso_fitness_backward_ws: need grad_f, grad_X and a 256-byte aligned workspace of "
                       "psso_fitness_workspace_size bytes");
        return PSSO_ERR_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    CUtensorMap tbt;
    st = tc_forward_z(N, D, X, shift, rotation, ws, L, true, s, &tbt);
    if (st != PSSO_OK) return st;
    const Hot hz = base_hot(fn, D, reinterpret_cast<const float*>(ws + L.zero), weights);
    auto* A = reinterpret_cast<__nv_bfloat16*>(ws + L.a);   // reused: the planes of G
    const int wpb = 8;
    const unsigned grid = (unsigned)((L.Np + wpb - 1) / wpb);
    const float* Z = reinterpret_cast<const float*>(ws + L.z);
    switch (hz.maxc) {
    case 1: gtc::gz_split<1><<<grid, 32 * wpb, 0, s>>>(hz, Z, N, grad_f, L.Np, L.Kp, A); break;
    case 2: gtc::gz_split<2><<<grid, 32 * wpb, 0, s>>>(hz, Z, N, grad_f, L.Np, L.Kp, A); break;
    case 4: gtc::gz_split<4><<<grid, 32 * wpb, 0, s>>>(hz, Z, N, grad_f, L.Np, L.Kp, A); break;
    default: gtc::gz_split<8><<<grid, 32 * wpb, 0, s>>>(hz, Z, N, grad_f, L.Np, L.Kp, A); break;
    }
    CUtensorMap ta;
    if (!tc::make_tmap_bf16(&ta, A, L.Kp, 3 * L.Np)) {
        set_last_error("psso_fitness_backward_ws: cuTensorMapEncodeTiled failed");
        return PSSO_ERR_CUDA;
    }
    if (cudaMemsetAsync(grad_X, 0xff, (size_t)N * D * 4, s) != cudaSuccess) {
        set_last_error("psso_fitness_backward_ws: memset failed");
        return PSSO_ERR_CUDA;
    }
    tc::GemmArgs ga{L.Np, L.Jp, L.Kp, reinterpret_cast<int*>(ws + L.status)};
    gtc::grad_gemm<<<dim3(L.Np / psso::tc::BM, L.Jp / psso::tc::BN), 128, tc::SMEM_BYTES, s>>>(ta, tbt, ga,
                                                                           gtc::StoreEpi{grad_X, (int)N, (int)D});
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("psso_fitness_backward_ws: launch failed");
        return PSSO_ERR_CUDA;
    }
    return PSSO_OK;
}
