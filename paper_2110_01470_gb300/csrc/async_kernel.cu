// async_kernel.cu -- the asynchronous SSO flow of Alg. 1 (the sequential
// CPU-SSO) on the GPU, FP64 fitness.
//
// Alg. 1 takes the particles one after the other: particle i searches
// (Eq. 2.1) with the gBest as it stands after particles 0..i-1 of the same
// generation, is evaluated, replaces its pBest when f < pF and the gBest when
// f < gF.  That is a chain through the gBest, but a short one: the gBest
// changes only at the particles that beat it.  A generation therefore runs as
// rounds of speculation and ordered commit:
//
//   round (start s, gBest b):
//     1. every particle i >= s (in parallel over the whole grid) searches with
//        gBest row P_b and is evaluated: x'_i, f'_i into scratch;
//     2. k = the lowest i >= s with f'_i < gF (grid-wide atomic minimum);
//     3. particles s..k commit in index order's result (each its own row: X_i
//        = x'_i, pBest when f'_i < pF_i); if k exists, the gBest becomes
//        particle k (its new pBest row P_k is the gBest row) and the next
//        round starts at k + 1, else the generation ends.
//
// Particles s..k-1 saw the right gBest (none of them changed it) and so did
// k; the particles after k are searched again with the new gBest.  The
// result is the sequential Alg. 1 bit for bit (same draws, same FP64
// summation order as the oracle), at one speculative pass per gBest
// improvement plus one.  Rounds are separated by a grid barrier with a
// bounded wait (a cooperative launch keeps every block resident).
#include <climits>

#include "psso.h"
#include "psso_internal.h"
#include "sso_common.cuh"

namespace psso {
namespace async {

constexpr unsigned NONE = 0xffffffffu;   // "no improving particle"

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier with a bounded wait: the last block to arrive resets the count
// and bumps the generation word; the others poll it.  Returns false (for the
// whole block) once any block gave up, after which every block leaves.
__device__ bool grid_sync(AsyncCtl* c, StatusDev* st, unsigned nblocks, int64_t limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned gen = ld_volatile_u32(&c->bar_gen);
        __threadfence();
        if (atomicAdd(&c->bar_count, 1u) == nblocks - 1) {
            c->bar_count = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            int64_t it = 0;
            while (ld_volatile_u32(&c->bar_gen) == gen) {
                if (((++it) & 31) == 0 && ld_volatile_u32(reinterpret_cast<unsigned*>(&st->abort))) {
                    ok = 0;
                    break;
                }
                if (it > limit) {
                    atomicCAS(&st->err, 0, (int)PSSO_ERR_TIMEOUT);
                    atomicExch(&st->abort, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Eq. 2.1 for the group's chunks of particle i (first-interval source `a`,
// pBest `p`, third-interval source `c`: gBest / keep swapped by the order).
template <class Pos, int MAXC>
__device__ __forceinline__ void search(const Hot& in, const Pos* xr, const Pos* pr, const Pos* gs, int64_t i,
                                       int64_t g, int lane_g, Pos (&x)[MAXC][4])
{
    const uint32_t gg = (uint32_t)g;
    const uint32_t ctr3r = TAG_RHO | (in.sid << 8);
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
#pragma unroll
        for (int m = 0; m < 4; ++m) x[q][m] = Pos(0);
        if (c >= in.nchunks) continue;
        const int nvalid = min(4, in.D - 4 * c);
        const uint32_t valid = (1u << nvalid) - 1u;
        if (g == 0) {
            fresh_chunk(x[q], valid, (uint32_t)c, (uint32_t)i + in.i_base, 0u, TAG_INIT, in);
            continue;
        }
        const uint4 rb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3r), in.k0, in.k1);
        Pos a[4], p[4], t[4];
        ld4_cg((in.order ? xr : gs) + 4 * c, a);
        ld4_cg(pr + 4 * c, p);
        ld4_cg((in.order ? gs : xr) + 4 * c, t);
        uint32_t nf = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t r = word_of(rb, m);
            const bool l1 = (r < in.Tg32) || (in.tfull & 1u);
            const bool l2 = (r < in.Tp32) || (in.tfull & 2u);
            const bool l3 = (r < in.Tw32) || (in.tfull & 4u);
            x[q][m] = l1 ? a[m] : l2 ? p[m] : t[m];
            if (!l3) nf |= 1u << m;
        }
        nf &= valid;
        if (nf) fresh_chunk(x[q], nf, (uint32_t)c, (uint32_t)i + in.i_base, gg, TAG_FRESH, in);
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m >= nvalid) x[q][m] = Pos(0);
    }
}

struct Groups {
    int G, lane_g, gid, ngroups;
    unsigned gmask;
};
__device__ __forceinline__ Groups groups_of(int G)
{
    Groups q;
    const int lane = threadIdx.x & 31, gpw = 32 / G;
    q.G = G;
    q.lane_g = lane & (G - 1);
    q.gid = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * gpw + lane / G;
    q.ngroups = gridDim.x * (blockDim.x >> 5) * gpw;
    q.gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    return q;
}

__device__ inline unsigned block_min_u32(unsigned v)
{
    __shared__ unsigned sh[32];
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned out = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) out = min(out, sh[w]);
    return out;
}

__device__ inline unsigned long long block_sum_u64(unsigned long long v)
{
    __shared__ unsigned long long sh[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long out = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) out += sh[w];
    return out;
}

template <class Pos>
__device__ void write_gbest_async(const InstDev& d, int64_t b, double gF, int64_t g, unsigned long long acc)
{
    GBestDev* gb = d.gb;
    gb->idx = b;
    gb->gen = g;
    gb->accepted = (int64_t)acc;
    gb->rechecks = 0;
    gb->f64 = gF;
    gb->lo = __double2float_rd(gF);
    gb->hi = __double2float_ru(gF);
    gb->ver = d.pver[b];
    gb->has64 = 1;
    if (d.log_stride > 0 && d.log_cap > 0 && (g % d.log_stride) == 0) {
        LogDev* e = d.log + ((g / d.log_stride) % d.log_cap);
        e->gen = g;
        e->idx = b;
        e->value = gF;
        e->lo = gb->lo;
        e->hi = gb->hi;
        e->accepted = (int64_t)acc;
        e->rechecks = 0;
    }
}

template <class Pos, int MAXC>
__global__ void __launch_bounds__(256) sso_async(const AsyncParams p)
{
    const InstDev& d = *p.inst;
    const Hot in = hot_of(d);
    const Groups gr = groups_of(in.G);
    const int64_t N = d.N;
    const int Dp = d.Dp;
    Pos* X = static_cast<Pos*>(d.X);
    Pos* P = static_cast<Pos*>(d.P);
    Pos* Xs = static_cast<Pos*>(p.xs);
    AsyncCtl* c = p.ctl;
    const unsigned nb = gridDim.x;
    __shared__ unsigned s_k;

    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) c->first[q] = NONE;
        c->acc[0] = c->acc[1] = 0;
    }
    if (!grid_sync(c, p.status, nb, p.spin_limit)) return;

    int64_t b = 0;
    double gF = 0.0;
    if (p.g_begin > 0) {
        b = __ldcg(&d.gb->idx);
        gF = __ldcg(&d.gb->f64);
        if (!PSSO_CHK(b >= 0 && b < N, CHK_ASYNC_ROW, b)) return;   // the same in every block
    }
    unsigned rc = 0;   // rounds so far in this launch (selects the `first` slot)
    for (int64_t g = p.g_begin; g <= p.g_end; ++g) {
        if (g == 0) {   // Kernel Function (I): the initial population; pBest = X0
            for (int64_t i = gr.gid; i < N; i += gr.ngroups) {
                Pos x[MAXC][4];
                search<Pos, MAXC>(in, nullptr, nullptr, nullptr, i, 0, gr.lane_g, x);
#pragma unroll
                for (int q = 0; q < MAXC; ++q) {
                    const int cc = gr.lane_g + 32 * q;
                    if (cc < in.nchunks) {
                        st4(X + i * Dp + 4 * cc, x[q]);
                        st4(P + i * Dp + 4 * cc, x[q]);
                    }
                }
                const double f = fit64<Pos, MAXC>(in, x, gr.lane_g, gr.gmask, gr.G);
                if (gr.lane_g == 0) {
                    d.pf64[i] = f;
                    d.pver[i] = 0u;
                }
            }
            if (!grid_sync(c, p.status, nb, p.spin_limit)) return;
            // lowest-index arg-min of pF, every block the same (reads through L2)
            double bv = __longlong_as_double(0x7ff0000000000000LL);
            long long bi = LLONG_MAX;
            for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
                const double v = __ldcg(d.pf64 + i);
                if (v < bv || (v == bv && i < bi)) { bv = v; bi = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            __shared__ double shv[32];
            __shared__ long long shi[32];
            __syncthreads();
            if ((threadIdx.x & 31) == 0) { shv[threadIdx.x >> 5] = bv; shi[threadIdx.x >> 5] = bi; }
            __syncthreads();
            bv = shv[0];
            bi = shi[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (shv[w] < bv || (shv[w] == bv && shi[w] < bi)) { bv = shv[w]; bi = shi[w]; }
            b = bi;
            gF = bv;
            if (blockIdx.x == 0) {
                Pos* gs = static_cast<Pos*>(d.gbrow);
                for (int j = threadIdx.x; j < Dp; j += blockDim.x) gs[j] = __ldcg(P + b * Dp + j);
                if (threadIdx.x == 0) write_gbest_async<Pos>(d, b, gF, 0, (unsigned long long)N);
            }
            continue;
        }
        // Alg. 1, generation g: rounds of speculation and ordered commit
        int64_t s = 0;
        unsigned long long acc = 0;
        while (true) {
            const int slot = (int)(rc % 3);
            if (blockIdx.x == 0 && threadIdx.x == 0) c->first[(rc + 1) % 3] = NONE;
            ++rc;
            const Pos* gs = P + b * Dp;     // the gBest row: particle b's pBest
            unsigned lfirst = NONE;
            for (int64_t i = s + gr.gid; i < N; i += gr.ngroups) {
                Pos x[MAXC][4];
                search<Pos, MAXC>(in, X + i * Dp, P + i * Dp, gs, i, g, gr.lane_g, x);
#pragma unroll
                for (int q = 0; q < MAXC; ++q) {
                    const int cc = gr.lane_g + 32 * q;
                    if (cc < in.nchunks) st4(Xs + i * Dp + 4 * cc, x[q]);
                }
                const double f = fit64<Pos, MAXC>(in, x, gr.lane_g, gr.gmask, gr.G);
                if (gr.lane_g == 0) {
                    p.fs[i] = f;
                    if (f < gF) lfirst = min(lfirst, (unsigned)i);
                }
            }
            const unsigned bmin = block_min_u32(lfirst);
            if (threadIdx.x == 0 && bmin != NONE) atomicMin(&c->first[slot], bmin);
            if (!grid_sync(c, p.status, nb, p.spin_limit)) return;
            if (threadIdx.x == 0) s_k = ld_volatile_u32(&c->first[slot]);
            __syncthreads();
            const unsigned k = s_k;
            if (!PSSO_CHK(k == NONE || (int64_t)k < N, CHK_ASYNC_ROW, k)) return;   // the same in every block
            const int64_t last = (k == NONE) ? N - 1 : (int64_t)k;
            // commit s..last: position, and pBest when strictly better (Alg. 1)
            for (int64_t i = s + gr.gid; i <= last; i += gr.ngroups) {
                const double f = __ldcg(p.fs + i);
                const bool better = f < __ldcg(d.pf64 + i);
#pragma unroll
                for (int q = 0; q < MAXC; ++q) {
                    const int cc = gr.lane_g + 32 * q;
                    if (cc < in.nchunks) {
                        Pos v[4];
                        ld4_cg(Xs + i * Dp + 4 * cc, v);
                        st4(X + i * Dp + 4 * cc, v);
                        if (better) st4(P + i * Dp + 4 * cc, v);
                    }
                }
                if (gr.lane_g == 0 && better) {
                    d.pf64[i] = f;
                    d.pver[i] = (uint32_t)g;
                    ++acc;
                }
            }
            if (k == NONE) break;
            b = (int64_t)k;                  // Alg. 1's gBest replacement
            gF = __ldcg(p.fs + k);
            s = (int64_t)k + 1;
            if (!grid_sync(c, p.status, nb, p.spin_limit)) return;
            if (s >= N) break;
        }
        const unsigned long long bacc = block_sum_u64(acc);
        if (threadIdx.x == 0 && bacc) atomicAdd(&c->acc[g & 1], bacc);
        if (!grid_sync(c, p.status, nb, p.spin_limit)) return;
        if (blockIdx.x == 0) {
            Pos* gsw = static_cast<Pos*>(d.gbrow);
            for (int j = threadIdx.x; j < Dp; j += blockDim.x) gsw[j] = __ldcg(P + b * Dp + j);
            if (threadIdx.x == 0) {
                const unsigned long long tot = *reinterpret_cast<volatile unsigned long long*>(&c->acc[g & 1]);
                c->acc[(g + 1) & 1] = 0;
                write_gbest_async<Pos>(d, b, gF, g, tot);
            }
        }
    }
}

template <class Pos, int MAXC>
cudaError_t launch_mc(int op, const AsyncParams* p, int grid, int block, cudaStream_t s, int* out)
{
    if (op == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, sso_async<Pos, MAXC>, block, 0);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3((unsigned)block);
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident: the barrier waits end
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, sso_async<Pos, MAXC>, *p);
}

}  // namespace async

cudaError_t async_call(int pos_size, int mc_index, int op, const AsyncParams* p, int grid, int block,
                       cudaStream_t s, int* out)
{
    using namespace async;
    if (pos_size == 8) {
        switch (mc_index) {
        case 0: return launch_mc<double, 1>(op, p, grid, block, s, out);
        case 1: return launch_mc<double, 2>(op, p, grid, block, s, out);
        case 2: return launch_mc<double, 4>(op, p, grid, block, s, out);
        default: return launch_mc<double, 8>(op, p, grid, block, s, out);
        }
    }
    switch (mc_index) {
    case 0: return launch_mc<float, 1>(op, p, grid, block, s, out);
    case 1: return launch_mc<float, 2>(op, p, grid, block, s, out);
    case 2: return launch_mc<float, 4>(op, p, grid, block, s, out);
    default: return launch_mc<float, 8>(op, p, grid, block, s, out);
    }
}

}  // namespace psso
