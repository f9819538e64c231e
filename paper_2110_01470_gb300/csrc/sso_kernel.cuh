// sso_kernel.cuh -- the persistent SSO generation kernel (sm_103a).
//
// One cooperative launch runs generations g_begin..g_end of every instance.
// Each block owns one or more "units" (a contiguous particle range of one
// instance) for the whole launch; a unit whose X, P and pBest state fit is
// kept resident in shared memory across all generations of the launch.  Per
// generation and unit:
//
//   A  gBest of generation g-1 (Alg. 4).  A unit that is the whole swarm keeps
//      it in shared memory.  Otherwise every block of the instance reads the
//      per-block records of g-1 (tagged words: no lock, atomic or writer-side
//      fence), takes the lowest-index arg-min, and fetches the winning row --
//      published as tagged words too -- only if the winner (index, row
//      version) changed.
//   B  For every owned particle (a group of G lanes; lane l owns variable
//      chunks l, l+32, ... of 4 variables): the stepwise update of Eq. 2.1 with
//      one Philox-4x32-10 block per chunk, the fitness (Kernel Function (E))
//      and the pBest update of Alg. 3 (f <= pF).  In FP32 mode a comparison
//      the FP32 error bound cannot decide is re-evaluated in FP64 in the
//      oracle's order.  Each warp also folds its particles into an arg-min
//      candidate.
//   C  The unit's lowest-index arg-min from the per-warp candidates.
//   D  Whole-swarm unit: refresh the shared gBest row.  Otherwise publish the
//      unit's winner: its row and its record for generation g.
//
// Every block writes only its own slots, so the pBest / gBest "resource
// preemption" of the paper (abstract; Alg. 3-4) cannot occur.
#pragma once
#include "sso_common.cuh"

namespace psso {

// ---------------------------------------------------------------------------
// Tagged words.
__device__ __forceinline__ uint64_t tw(uint32_t tag, uint64_t payload)
{
    return ((uint64_t)(tag & 0xffffu) << 48) | (payload & 0xffffffffffffULL);
}
__device__ __forceinline__ bool tagged(uint64_t w, uint32_t tag)
{
    return (uint32_t)(w >> 48) == (tag & 0xffffu);
}
__device__ __forceinline__ void ldv2(const uint64_t* p, uint64_t& a, uint64_t& b)
{
    asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void stv2(uint64_t* p, uint64_t a, uint64_t b)
{
    asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Words per position in a published row.
template <class Pos> struct WordsPer;
template <> struct WordsPer<float> { static constexpr int value = 1; };
template <> struct WordsPer<double> { static constexpr int value = 2; };

__device__ __forceinline__ void put_chunk(uint64_t* w, uint32_t tag, const float (&v)[4])
{
    stv2(w, tw(tag, __float_as_uint(v[0])), tw(tag, __float_as_uint(v[1])));
    stv2(w + 2, tw(tag, __float_as_uint(v[2])), tw(tag, __float_as_uint(v[3])));
}
__device__ __forceinline__ void put_chunk(uint64_t* w, uint32_t tag, const double (&v)[4])
{
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint64_t b = (uint64_t)__double_as_longlong(v[m]);
        stv2(w + 2 * m, tw(tag, b & 0xffffffffULL), tw(tag, b >> 32));
    }
}
__device__ __forceinline__ bool get_chunk(const uint64_t* w, uint32_t tag, float (&v)[4])
{
    uint64_t a, b, c, d;
    ldv2(w, a, b);
    ldv2(w + 2, c, d);
    v[0] = __uint_as_float((uint32_t)a);
    v[1] = __uint_as_float((uint32_t)b);
    v[2] = __uint_as_float((uint32_t)c);
    v[3] = __uint_as_float((uint32_t)d);
    return tagged(a, tag) && tagged(b, tag) && tagged(c, tag) && tagged(d, tag);
}
__device__ __forceinline__ bool get_chunk(const uint64_t* w, uint32_t tag, double (&v)[4])
{
    bool ok = true;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        uint64_t lo, hi;
        ldv2(w + 2 * m, lo, hi);
        v[m] = __longlong_as_double((long long)(((hi & 0xffffffffULL) << 32) | (lo & 0xffffffffULL)));
        ok = ok && tagged(lo, tag) && tagged(hi, tag);
    }
    return ok;
}

// Marks the launch as failed (first failure wins) and tells every block to stop.
__device__ inline void give_up(const KParams& p, const UnitDev& un)
{
    if (atomicCAS(&p.status->err, 0, 4 /* PSSO_ERR_TIMEOUT */) == 0)
        p.status->where = un.inst * 65536 + un.rank;
    *(volatile int32_t*)&p.status->abort = 1;
}
__device__ __forceinline__ bool should_stop(const KParams& p, int64_t it)
{
    return it >= p.spin_limit || *(volatile int32_t*)&p.status->abort;
}

// ---------------------------------------------------------------------------
// Where a unit's particle state lives (shared memory or global memory).
template <class Pos>
struct View {
    Pos* X;
    Pos* P;
    double* pf64;
    float* plo;
    float* phi;
    uint32_t* pver;
    uint32_t* pflag;
    int64_t base;       // particle i is entry i - base
};

template <class Pos>
__device__ __forceinline__ View<Pos> make_view(const InstDev& in, const UnitDev& un,
                                               unsigned char* smem)
{
    View<Pos> v;
    if (un.resident) {
        const int64_t n = un.i1 - un.i0;
        unsigned char* s = smem + un.res_off;
        const size_t rows = res_align((size_t)n * in.Dp * sizeof(Pos));
        v.X = reinterpret_cast<Pos*>(s);
        v.P = reinterpret_cast<Pos*>(s + rows);
        s += 2 * rows;
        v.pf64 = reinterpret_cast<double*>(s);
        s += res_align((size_t)n * 8);
        v.plo = reinterpret_cast<float*>(s);
        s += res_align((size_t)n * 4);
        v.phi = reinterpret_cast<float*>(s);
        s += res_align((size_t)n * 4);
        v.pver = reinterpret_cast<uint32_t*>(s);
        s += res_align((size_t)n * 4);
        v.pflag = reinterpret_cast<uint32_t*>(s);
        v.base = un.i0;
    } else {
        v.X = static_cast<Pos*>(in.X);
        v.P = static_cast<Pos*>(in.P);
        v.pf64 = in.pf64;
        v.plo = in.plo;
        v.phi = in.phi;
        v.pver = in.pver;
        v.pflag = in.pflag;
        v.base = 0;
    }
    return v;
}

// Copies a resident unit between global memory and shared memory.
template <class Pos, bool F32R>
__device__ void move_resident(const InstDev& in, const UnitDev& un, unsigned char* smem, bool to_smem)
{
    const View<Pos> v = make_view<Pos>(in, un, smem);
    const int64_t n = un.i1 - un.i0;
    const int64_t nc = n * in.nchunks;
    Pos* gX = static_cast<Pos*>(in.X) + un.i0 * in.Dp;
    Pos* gP = static_cast<Pos*>(in.P) + un.i0 * in.Dp;
    for (int64_t q = threadIdx.x; q < nc; q += blockDim.x) {
        Pos a[4], b[4];
        if (to_smem) {
            ld4(gX + 4 * q, a); st4(v.X + 4 * q, a);
            ld4(gP + 4 * q, b); st4(v.P + 4 * q, b);
        } else {
            ld4(v.X + 4 * q, a); st4(gX + 4 * q, a);
            ld4(v.P + 4 * q, b); st4(gP + 4 * q, b);
        }
    }
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const int64_t i = un.i0 + k;
        if (to_smem) {
            v.pf64[k] = in.pf64[i];
            v.pver[k] = in.pver[i];
            if (F32R) { v.plo[k] = in.plo[i]; v.phi[k] = in.phi[i]; v.pflag[k] = in.pflag[i]; }
        } else {
            in.pf64[i] = v.pf64[k];
            in.pver[i] = v.pver[k];
            if (F32R) { in.plo[i] = v.plo[k]; in.phi[i] = v.phi[k]; in.pflag[i] = v.pflag[k]; }
        }
    }
}

// ---------------------------------------------------------------------------
// Arg-min candidates.  FP64: lexicographic (value, index).  FP32: the smallest
// upper bound mh and the two smallest lower bounds; if the second-smallest
// lower bound exceeds mh, the particle with the smallest lower bound is the
// only one that can be the arg-min.
struct Cand {
    double v;          // FP64: value; FP32: FP64 value of the first (if has1)
    long long i;       // index of the first
    float mh;          // FP32: smallest upper bound
    float l1, h1;      // FP32: bounds of the first
    float l2;          // FP32: second-smallest lower bound
    uint32_t ver;      // row version of the first
    int has1;          // FP64 value of the first known
    int rank;          // publishing rank of the first (records only)
};

__device__ __forceinline__ Cand cand_none()
{
    Cand c;
    c.v = DBL_MAX; c.i = LLONG_MAX; c.mh = FLT_MAX; c.l1 = FLT_MAX; c.h1 = FLT_MAX;
    c.l2 = FLT_MAX; c.ver = 0; c.has1 = 0; c.rank = -1;
    return c;
}

template <bool F32R>
__device__ __forceinline__ Cand cand_merge(const Cand& a, const Cand& b)
{
    if (!F32R) return (b.v < a.v || (b.v == a.v && b.i < a.i)) ? b : a;
    const bool bfirst = (b.l1 < a.l1) || (b.l1 == a.l1 && b.i < a.i);
    Cand r = bfirst ? b : a;
    const Cand& o = bfirst ? a : b;
    r.l2 = fminf(fminf(r.l2, o.l1), o.l2);
    r.mh = fminf(a.mh, b.mh);
    return r;
}

__device__ __forceinline__ Cand cand_shfl(const Cand& c, int off)
{
    Cand o;
    o.v = __shfl_xor_sync(0xffffffffu, c.v, off);
    o.i = __shfl_xor_sync(0xffffffffu, c.i, off);
    o.mh = __shfl_xor_sync(0xffffffffu, c.mh, off);
    o.l1 = __shfl_xor_sync(0xffffffffu, c.l1, off);
    o.h1 = __shfl_xor_sync(0xffffffffu, c.h1, off);
    o.l2 = __shfl_xor_sync(0xffffffffu, c.l2, off);
    o.ver = __shfl_xor_sync(0xffffffffu, c.ver, off);
    o.has1 = __shfl_xor_sync(0xffffffffu, c.has1, off);
    o.rank = __shfl_xor_sync(0xffffffffu, c.rank, off);
    return o;
}

template <bool F32R>
__device__ __forceinline__ Cand cand_warp(Cand c)
{
    for (int off = 16; off > 0; off >>= 1) c = cand_merge<F32R>(c, cand_shfl(c, off));
    return c;
}

// Candidate of one particle from its (post-update) pBest state.
template <bool F32R>
__device__ __forceinline__ Cand cand_of(long long i, double f64, float lo, float hi, int has64,
                                        uint32_t ver)
{
    Cand c = cand_none();
    c.i = i;
    c.ver = ver;
    if (!F32R) {
        c.v = f64;
        return c;
    }
    c.mh = hi; c.l1 = lo; c.h1 = hi; c.has1 = has64; c.v = has64 ? f64 : DBL_MAX;
    return c;
}

struct BlockShared {
    Cand warp_cand[16];
    unsigned long long warp_acc[16], warp_rck[16];
    Cand result;
    unsigned long long acc, rck;
    int flag;
    long long idx[MAX_UNITS_PER_BLOCK];   // identity (index, version) of the row in gs
    uint32_t ver[MAX_UNITS_PER_BLOCK];
};

// Block-wide candidate + counters; the result is in sh.result / sh.acc / sh.rck.
template <bool F32R>
__device__ void block_cand(Cand c, unsigned long long acc, unsigned long long rck, BlockShared& sh)
{
    c = cand_warp<F32R>(c);
    for (int off = 16; off > 0; off >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        rck += __shfl_xor_sync(0xffffffffu, rck, off);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh.warp_cand[w] = c;
        sh.warp_acc[w] = acc;
        sh.warp_rck[w] = rck;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Cand r = sh.warp_cand[0];
        unsigned long long a = sh.warp_acc[0], k = sh.warp_rck[0];
        for (int q = 1; q < nw; ++q) {
            r = cand_merge<F32R>(r, sh.warp_cand[q]);
            a += sh.warp_acc[q];
            k += sh.warp_rck[q];
        }
        sh.result = r;
        sh.acc = a;
        sh.rck = k;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Step B: update, evaluate and pBest-update every particle of the unit; each
// lane returns its group's arg-min candidate.
template <class Pos, bool F32R, int MAXC>
__device__ Cand step_b(const InstDev& in, const UnitDev& un, const View<Pos>& v,
                       const Pos* __restrict__ gs, int64_t g, unsigned long long& n_acc,
                       unsigned long long& n_rck)
{
    const int G = in.G;
    const int lane = threadIdx.x & 31;
    const int lane_g = lane & (G - 1);
    const int gpw = 32 / G;
    const int ngroups = (blockDim.x >> 5) * gpw;
    const int gid = (threadIdx.x >> 5) * gpw + lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t n = un.i1 - un.i0;
    const uint32_t gg = (uint32_t)g;
    Cand best = cand_none();

    for (int64_t k = gid; k < n; k += ngroups) {
        const int64_t i = un.i0 + k;
        const int64_t e = i - v.base;
        Pos* xr = v.X + e * in.Dp;
        Pos* pr = v.P + e * in.Dp;
        Pos x[MAXC][4];
        bool eqp = true;
#pragma unroll
        for (int q = 0; q < MAXC; ++q) {
            const int c = lane_g + 32 * q;
            if (c < in.nchunks) {
                const int nvalid = min(4, in.D - 4 * c);
                const uint32_t valid = (1u << nvalid) - 1u;
                if (g == 0) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) x[q][m] = Pos(0);
                    fresh_chunk(x[q], valid, (uint32_t)c, (uint32_t)i, 0u, TAG_INIT, in);
                } else {
                    const uint4 rb = philox10(make_uint4((uint32_t)c, (uint32_t)i, gg,
                                                         TAG_RHO | (in.sid << 8)), in.k0, in.k1);
                    Pos xo[4], po[4], go[4];
                    ld4(xr + 4 * c, xo);
                    ld4(pr + 4 * c, po);
                    ld4(gs + 4 * c, go);
                    uint32_t nf = 0;
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint64_t r = word_of(rb, m);
                        x[q][m] = (r < in.Tg) ? go[m] : (r < in.Tp) ? po[m] : xo[m];
                        if (r >= in.Tw) nf |= 1u << m;
                    }
                    nf &= valid;
                    if (nf) fresh_chunk(x[q], nf, (uint32_t)c, (uint32_t)i, gg, TAG_FRESH, in);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (m >= nvalid) x[q][m] = Pos(0);
                        eqp = eqp && same_bits(x[q][m], po[m]);
                    }
                }
                st4(xr + 4 * c, x[q]);
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) x[q][m] = Pos(0);
            }
        }

        bool accept;
        Cand mine;
        if constexpr (!F32R) {
            const double f = fit64<Pos, MAXC>(in, x, lane_g, gmask, G);
            const double pf = (g == 0) ? f : v.pf64[e];
            accept = (g == 0) || (f <= pf);
            const uint32_t ver = accept ? gg : v.pver[e];
            if (accept && lane_g == 0) {
                v.pf64[e] = f;
                v.pver[e] = gg;
            }
            mine = cand_of<false>((long long)i, accept ? f : pf, 0.f, 0.f, 1, ver);
        } else {
            const Fit32 r = fit32<MAXC>(in, x, lane_g, gmask, G);
            float lo = __fsub_rd(r.f, r.E), hi = __fadd_ru(r.f, r.E);
            int has64 = 0;
            double f64v = 0.0;
            bool write_state = true;
            if (g == 0) {
                accept = true;
            } else {
                const float plo = v.plo[e], phi = v.phi[e];
                const uint32_t pfl = v.pflag[e];
                const double ppf = v.pf64[e];
                if (__all_sync(gmask, eqp)) {
                    accept = true;           // identical row: identical fitness, keep its state
                    write_state = false;
                    lo = plo; hi = phi; has64 = (int)(pfl & 1u); f64v = ppf;
                } else if (hi < plo) {
                    accept = true;
                } else if (lo > phi) {
                    accept = false;
                    lo = plo; hi = phi; has64 = (int)(pfl & 1u); f64v = ppf;
                } else {
                    // The bound cannot decide: FP64 in the oracle's order.
                    const double fx = fit64<float, MAXC>(in, x, lane_g, gmask, G);
                    double fp = ppf;
                    if (!(pfl & 1u)) {
                        float pv[MAXC][4];
#pragma unroll
                        for (int q = 0; q < MAXC; ++q) {
                            const int c = lane_g + 32 * q;
                            if (c < in.nchunks) ld4(reinterpret_cast<const float*>(pr) + 4 * c, pv[q]);
                            else { pv[q][0] = pv[q][1] = pv[q][2] = pv[q][3] = 0.f; }
                        }
                        fp = fit64<float, MAXC>(in, pv, lane_g, gmask, G);
                        if (lane_g == 0) n_rck++;
                    }
                    if (lane_g == 0) n_rck++;
                    accept = fx <= fp;
                    has64 = 1;
                    f64v = accept ? fx : fp;
                    lo = f64_to_f32_rd(f64v);
                    hi = f64_to_f32_ru(f64v);
                    if (!accept && lane_g == 0) {   // keep the pBest's exact value
                        v.pf64[e] = fp;
                        v.pflag[e] = 1u;
                        v.plo[e] = lo;
                        v.phi[e] = hi;
                    }
                }
            }
            const uint32_t ver = (accept && write_state) ? gg : (g == 0 ? 0u : v.pver[e]);
            if (accept && lane_g == 0 && write_state) {
                v.pver[e] = gg;
                v.pf64[e] = has64 ? f64v : 0.0;
                v.pflag[e] = (uint32_t)has64;
                v.plo[e] = lo;
                v.phi[e] = hi;
            }
            mine = cand_of<true>((long long)i, f64v, lo, hi, has64, ver);
        }
        if (accept) {
#pragma unroll
            for (int q = 0; q < MAXC; ++q) {
                const int c = lane_g + 32 * q;
                if (c < in.nchunks) st4(pr + 4 * c, x[q]);
            }
            if (lane_g == 0) n_acc++;
        }
        best = cand_merge<F32R>(best, mine);
    }
    return best;
}

// ---------------------------------------------------------------------------
struct Winner {
    long long idx;
    double f64;
    float lo, hi;
    uint32_t ver;
    int has64;
    unsigned long long acc, rck;
};

__device__ inline void write_gbest(const InstDev& in, const Winner& w, int64_t g)
{
    GBestDev* gb = in.gb;
    gb->idx = w.idx;
    gb->gen = g;
    gb->accepted = (int64_t)w.acc;
    gb->rechecks = (int64_t)w.rck;
    gb->total_rechecks += (int64_t)w.rck;
    gb->f64 = w.f64;
    gb->lo = w.lo;
    gb->hi = w.hi;
    gb->ver = w.ver;
    gb->has64 = w.has64;
    if (in.log_stride > 0 && in.log_cap > 0 && (g % in.log_stride) == 0) {
        LogDev* e = in.log + ((g / in.log_stride) % in.log_cap);
        e->gen = g;
        e->idx = w.idx;
        e->value = w.has64 ? w.f64 : __longlong_as_double(0x7ff8000000000000LL);
        e->lo = w.lo;
        e->hi = w.hi;
        e->accepted = (int64_t)w.acc;
        e->rechecks = (int64_t)w.rck;
    }
}

// Step C: the unit's winner from the per-lane candidates.  FP32 mode falls
// back to an exact pass (FP64 for every overlapping candidate) when the
// bounds leave more than one candidate.
template <class Pos, bool F32R>
__device__ Winner step_c(const InstDev& in, const UnitDev& un, const View<Pos>& v, Cand c,
                         unsigned long long n_acc, unsigned long long n_rck, BlockShared& sh)
{
    block_cand<F32R>(c, n_acc, n_rck, sh);
    Cand r = sh.result;
    unsigned long long acc = sh.acc, rck = sh.rck;
    if (F32R && r.l2 <= r.mh) {
        // Several particles' bounds reach the smallest upper bound: make every
        // candidate exact, then take the exact lowest-index arg-min.
        const float m = r.mh;
        const int64_t n = un.i1 - un.i0;
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        unsigned long long extra = 0;
        for (int64_t k = warp; k < n; k += nw) {
            const int64_t e = un.i0 + k - v.base;
            if (v.plo[e] <= m && !(v.pflag[e] & 1u)) {
                const double f = fit64_row<Pos>(in, v.P + e * in.Dp, false);
                if ((threadIdx.x & 31) == 0) {
                    v.pf64[e] = f;
                    v.pflag[e] = 1u;
                    v.plo[e] = f64_to_f32_rd(f);
                    v.phi[e] = f64_to_f32_ru(f);
                    extra++;
                }
            }
        }
        __syncthreads();
        Cand ex = cand_none();
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
            const int64_t e = un.i0 + k - v.base;
            if (v.pflag[e] & 1u) {
                Cand q = cand_none();
                q.v = v.pf64[e];
                q.i = (long long)(un.i0 + k);
                q.ver = v.pver[e];
                ex = cand_merge<false>(ex, q);
            }
        }
        block_cand<false>(ex, 0, extra, sh);
        r = sh.result;
        r.has1 = 1;
        r.l1 = f64_to_f32_rd(r.v);
        r.h1 = f64_to_f32_ru(r.v);
        rck += sh.rck;
    }
    Winner w;
    w.idx = r.i;
    w.ver = r.ver;
    w.acc = acc;
    w.rck = rck;
    if (!F32R) {
        w.f64 = r.v;
        w.has64 = 1;
        w.lo = f64_to_f32_rd(r.v);
        w.hi = f64_to_f32_ru(r.v);
    } else {
        w.has64 = r.has1;
        w.f64 = r.has1 ? r.v : 0.0;
        w.lo = r.l1;
        w.hi = r.h1;
    }
    __syncthreads();
    return w;
}

// ---------------------------------------------------------------------------
// Records.
__device__ inline void publish_record(uint64_t* rec, uint32_t tag, const Winner& w)
{
    uint64_t v0, v1;
    if (w.has64) {
        const uint64_t b = (uint64_t)__double_as_longlong(w.f64);
        v0 = b & 0xffffffffULL;
        v1 = b >> 32;
    } else {
        v0 = __float_as_uint(w.lo);
        v1 = __float_as_uint(w.hi);
    }
    stv2(rec + RW_IDX, tw(tag, ((uint64_t)(w.has64 ? 1 : 0) << 32) | (uint32_t)w.idx), tw(tag, w.ver));
    stv2(rec + RW_V0, tw(tag, v0), tw(tag, v1));
    stv2(rec + RW_ACC, tw(tag, w.acc), tw(tag, w.rck));
}

// Reads one record (bounded wait); returns false on timeout / abort.
__device__ inline bool read_record(const uint64_t* rec, uint32_t tag, Winner& w, const KParams& p,
                                   const UnitDev& un)
{
    for (int64_t it = 0;; ++it) {
        uint64_t a, b, c, d, e, f;
        ldv2(rec + RW_IDX, a, b);
        ldv2(rec + RW_V0, c, d);
        ldv2(rec + RW_ACC, e, f);
        if (tagged(a, tag) && tagged(b, tag) && tagged(c, tag) && tagged(d, tag) && tagged(e, tag) &&
            tagged(f, tag)) {
            w.idx = (long long)(uint32_t)a;
            w.has64 = (int)((a >> 32) & 1u);
            w.ver = (uint32_t)b;
            if (w.has64) {
                w.f64 = __longlong_as_double((long long)(((d & 0xffffffffULL) << 32) | (c & 0xffffffffULL)));
                w.lo = f64_to_f32_rd(w.f64);
                w.hi = f64_to_f32_ru(w.f64);
            } else {
                w.f64 = 0.0;
                w.lo = __uint_as_float((uint32_t)c);
                w.hi = __uint_as_float((uint32_t)d);
            }
            w.acc = e & 0xffffffffffffULL;
            w.rck = f & 0xffffffffffffULL;
            return true;
        }
        if (should_stop(p, it)) {
            give_up(p, un);
            return false;
        }
        if (it > 8) __nanosleep(it < 256 ? 32 : 256);
    }
}

// Step A for a unit of a multi-block instance: decide the gBest of generation
// gp from the records and make sure shared memory holds its row.  Returns
// false when the launch is aborting.
template <class Pos, bool F32R>
__device__ bool step_a(const KParams& p, const InstDev& in, const UnitDev& un, const View<Pos>& v,
                       int uslot, Pos* gs, int64_t gp, bool finalize, BlockShared& sh)
{
    const int R = in.R;
    const uint32_t tag = (uint32_t)gp;
    const uint64_t* recs = in.rec + (size_t)(gp & 1) * R * REC_WORDS;
    constexpr int WPE = WordsPer<Pos>::value;
    if (threadIdx.x == 0) sh.flag = 0;
    __syncthreads();

    Cand c = cand_none();
    unsigned long long sacc = 0, srck = 0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        Winner w;
        if (!read_record(recs + (size_t)r * REC_WORDS, tag, w, p, un)) { sh.flag = 1; break; }
        Cand q = cand_of<F32R>(w.idx, w.f64, w.lo, w.hi, w.has64, w.ver);
        q.rank = r;
        c = cand_merge<F32R>(c, q);
        sacc += w.acc;
        srck += w.rck;
    }
    __syncthreads();
    if (sh.flag) return false;
    block_cand<F32R>(c, sacc, srck, sh);
    Cand win = sh.result;
    const unsigned long long tot_acc = sh.acc;
    unsigned long long tot_rck = sh.rck;

    if (F32R && win.l2 <= win.mh) {
        // Several ranks overlap: ranks without an exact value publish it
        // (second round), then the exact lowest-index arg-min is taken.
        const float m = win.mh;
        uint64_t* recs2 = in.rec2 + (size_t)(gp & 1) * R * REC_WORDS;
        if (threadIdx.x < 32) {
            Winner me;
            const bool ok = read_record(recs + (size_t)un.rank * REC_WORDS, tag, me, p, un);
            if (ok && me.lo <= m && !me.has64) {
                const double f = fit64_row<Pos>(in, v.P + (me.idx - v.base) * in.Dp, false);
                if (threadIdx.x == 0) {
                    Winner ww = me;
                    ww.f64 = f;
                    ww.has64 = 1;
                    ww.acc = 0;
                    ww.rck = 1;
                    publish_record(recs2 + (size_t)un.rank * REC_WORDS, tag, ww);
                }
            }
        }
        __syncthreads();
        Cand ex = cand_none();
        unsigned long long r2 = 0;
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            Winner w;
            if (!read_record(recs + (size_t)r * REC_WORDS, tag, w, p, un)) { sh.flag = 1; break; }
            if (w.lo > m) continue;
            if (!w.has64) {
                if (!read_record(recs2 + (size_t)r * REC_WORDS, tag, w, p, un)) { sh.flag = 1; break; }
                r2 += 1;
            }
            Cand q = cand_none();
            q.v = w.f64;
            q.i = w.idx;
            q.ver = w.ver;
            q.rank = r;
            ex = cand_merge<false>(ex, q);
        }
        __syncthreads();
        if (sh.flag) return false;
        block_cand<false>(ex, 0, r2, sh);
        win = sh.result;
        win.has1 = 1;
        win.l1 = f64_to_f32_rd(win.v);
        win.h1 = f64_to_f32_ru(win.v);
        tot_rck += sh.rck;
    }

    // Fetch the winner's row if it is not the one already in shared memory.
    const bool changed = (sh.idx[uslot] != win.i) || (sh.ver[uslot] != win.ver);
    if (changed) {
        const uint64_t* src = static_cast<const uint64_t*>(in.grow) +
                              ((size_t)(gp & 1) * R + win.rank) * (size_t)in.Dp * WPE;
        for (int ch = threadIdx.x; ch < in.nchunks; ch += blockDim.x) {
            Pos vals[4];
            for (int64_t it = 0;; ++it) {
                if (get_chunk(src + (size_t)4 * ch * WPE, tag, vals)) break;
                if (should_stop(p, it)) { give_up(p, un); sh.flag = 1; break; }
                if (it > 8) __nanosleep(64);
            }
            st4(gs + 4 * ch, vals);
        }
    }
    // Everything this block read of generation gp is complete before any of
    // its later publications (the writers reuse these slots at gp + 2).
    fence_acq_rel_gpu();
    __syncthreads();
    if (sh.flag) return false;
    if (threadIdx.x == 0) {
        sh.idx[uslot] = win.i;
        sh.ver[uslot] = win.ver;
    }
    if (un.rank == 0 && finalize) {
        if (changed) {
            Pos* dst = static_cast<Pos*>(in.gbrow);
            for (int ch = threadIdx.x; ch < in.nchunks; ch += blockDim.x) {
                Pos t[4];
                ld4(gs + 4 * ch, t);
                st4(dst + 4 * ch, t);
            }
        }
        if (threadIdx.x == 0) {
            Winner w;
            w.idx = win.i;
            w.ver = win.ver;
            w.acc = tot_acc;
            w.rck = tot_rck;
            w.has64 = F32R ? win.has1 : 1;
            w.f64 = F32R ? (win.has1 ? win.v : 0.0) : win.v;
            w.lo = F32R ? win.l1 : f64_to_f32_rd(win.v);
            w.hi = F32R ? win.h1 : f64_to_f32_ru(win.v);
            write_gbest(in, w, gp);
        }
    }
    __syncthreads();
    return true;
}

// Step D for a multi-block instance: publish the unit's winner row and record.
template <class Pos>
__device__ void step_d_publish(const KParams& p, const InstDev& in, const UnitDev& un,
                               const View<Pos>& v, const Winner& w, int64_t g)
{
    if (p.fault_skip_rank > 0 && un.inst == 0 && un.rank == p.fault_skip_rank - 1) return;
    constexpr int WPE = WordsPer<Pos>::value;
    const int R = in.R;
    const uint32_t tag = (uint32_t)g;
    uint64_t* dst = static_cast<uint64_t*>(in.grow) + ((size_t)(g & 1) * R + un.rank) * (size_t)in.Dp * WPE;
    const Pos* src = v.P + (w.idx - v.base) * in.Dp;
    for (int ch = threadIdx.x; ch < in.nchunks; ch += blockDim.x) {
        Pos t[4];
        ld4(src + 4 * ch, t);
        put_chunk(dst + (size_t)4 * ch * WPE, tag, t);
    }
    if (threadIdx.x == 0)
        publish_record(in.rec + ((size_t)(g & 1) * R + un.rank) * REC_WORDS, tag, w);
}

// Step D for a whole-swarm unit: refresh the shared-memory gBest row.
template <class Pos>
__device__ void step_d_local(const InstDev& in, const View<Pos>& v, const Winner& w, Pos* gs,
                             int uslot, int64_t g, BlockShared& sh)
{
    const bool changed = (sh.idx[uslot] != w.idx) || (sh.ver[uslot] != w.ver);
    if (changed) {
        const Pos* src = v.P + (w.idx - v.base) * in.Dp;
        Pos* dst = static_cast<Pos*>(in.gbrow);
        for (int ch = threadIdx.x; ch < in.nchunks; ch += blockDim.x) {
            Pos t[4];
            ld4(src + 4 * ch, t);
            st4(gs + 4 * ch, t);
            st4(dst + 4 * ch, t);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sh.idx[uslot] = w.idx;
        sh.ver[uslot] = w.ver;
        write_gbest(in, w, g);
    }
}

// ---------------------------------------------------------------------------
template <class Pos, bool F32R>
__device__ Cand unit_b(const InstDev& in, const UnitDev& un, const View<Pos>& v, const Pos* gs,
                       int64_t g, unsigned long long& n_acc, unsigned long long& n_rck)
{
    switch (in.maxc) {
    case 1: return step_b<Pos, F32R, 1>(in, un, v, gs, g, n_acc, n_rck);
    case 2: return step_b<Pos, F32R, 2>(in, un, v, gs, g, n_acc, n_rck);
    case 4: return step_b<Pos, F32R, 4>(in, un, v, gs, g, n_acc, n_rck);
    default: return step_b<Pos, F32R, 8>(in, un, v, gs, g, n_acc, n_rck);
    }
}

template <class Pos, bool F32R>
__global__ void __launch_bounds__(512) sso_generations(const KParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared sh;
    const int u0 = p.block_first[blockIdx.x], u1 = p.block_first[blockIdx.x + 1];

    // Prologue: resident units move into shared memory; whole-swarm units
    // restore their gBest row.
    for (int u = u0; u < u1; ++u) {
        const UnitDev un = p.units[u];
        const InstDev& in = p.inst[un.inst];
        Pos* gs = reinterpret_cast<Pos*>(smem + un.smem_off);
        const int slot = u - u0;
        if (un.resident && p.g_begin > 0) move_resident<Pos, F32R>(in, un, smem, true);
        if (in.R == 1 && p.g_begin > 0) {
            const Pos* src = static_cast<const Pos*>(in.gbrow);
            for (int ch = threadIdx.x; ch < in.nchunks; ch += blockDim.x) {
                Pos t[4];
                ld4_cg(src + 4 * ch, t);
                st4(gs + 4 * ch, t);
            }
            if (threadIdx.x == 0) { sh.idx[slot] = in.gb->idx; sh.ver[slot] = in.gb->ver; }
        } else if (threadIdx.x == 0) {
            sh.idx[slot] = -1;
            sh.ver[slot] = 0xffffffffu;
        }
    }
    __syncthreads();

    for (int64_t g = p.g_begin; g <= p.g_end; ++g) {
        for (int u = u0; u < u1; ++u) {
            const UnitDev un = p.units[u];
            const InstDev& in = p.inst[un.inst];
            Pos* gs = reinterpret_cast<Pos*>(smem + un.smem_off);
            const View<Pos> v = make_view<Pos>(in, un, smem);
            const int slot = u - u0;
            if (in.R > 1 && g > 0) {
                if (!step_a<Pos, F32R>(p, in, un, v, slot, gs, g - 1, g - 1 >= p.g_begin, sh)) return;
            }
            unsigned long long n_acc = 0, n_rck = 0;
            const Cand c = unit_b<Pos, F32R>(in, un, v, gs, g, n_acc, n_rck);
            __syncthreads();
            const Winner w = step_c<Pos, F32R>(in, un, v, c, n_acc, n_rck, sh);
            if (in.R == 1) step_d_local<Pos>(in, v, w, gs, slot, g, sh);
            else step_d_publish<Pos>(p, in, un, v, w, g);
            __syncthreads();
        }
    }
    // Epilogue: finalise the last generation of multi-block instances and
    // write resident units back.
    for (int u = u0; u < u1; ++u) {
        const UnitDev un = p.units[u];
        const InstDev& in = p.inst[un.inst];
        const View<Pos> v = make_view<Pos>(in, un, smem);
        if (in.R > 1) {
            Pos* gs = reinterpret_cast<Pos*>(smem + un.smem_off);
            if (!step_a<Pos, F32R>(p, in, un, v, u - u0, gs, p.g_end, true, sh)) return;
        }
        if (un.resident) {
            move_resident<Pos, F32R>(in, un, smem, false);
            __syncthreads();
        }
    }
}

// FP64 fitness of every instance's gBest row (used when only FP32 bounds are known).
template <class Pos>
__global__ void best_f64_kernel(const InstDev* inst, int n_inst)
{
    const int k = blockIdx.x;
    if (k >= n_inst) return;
    const InstDev& in = inst[k];
    if (in.gb->has64) return;
    const double f = fit64_row<Pos>(in, static_cast<const Pos*>(in.gbrow), true);
    if (threadIdx.x == 0) {
        in.gb->f64 = f;
        in.gb->has64 = 1;
    }
}

template <class Pos, bool F32R>
inline cudaError_t launch_generations(const KParams& p, int grid, int block, size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3((unsigned)block);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident: waits always end
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, sso_generations<Pos, F32R>, p);
}

template <class Pos, bool F32R>
inline cudaError_t occupancy_generations(int block, size_t smem, int* n)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, sso_generations<Pos, F32R>, block, smem);
}

template <class Pos, bool F32R>
inline cudaError_t smem_generations(size_t smem)
{
    return cudaFuncSetAttribute(sso_generations<Pos, F32R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(smem, 1));
}

}  // namespace psso
