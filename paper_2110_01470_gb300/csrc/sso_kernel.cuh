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

// Optional phase timestamps (global timer, ns) for profiling builds compiled
// with -DPSSO_TRACE; the default build compiles them out.
#ifdef PSSO_TRACE
constexpr int TRACE_BLOCKS = 160, TRACE_GENS = 64, TRACE_POINTS = 12;
constexpr int64_t TRACE_G0 = 100;
__device__ unsigned long long trace_buf[TRACE_BLOCKS][TRACE_GENS][TRACE_POINTS];
__device__ __forceinline__ void trace_point(int64_t g, int k)
{
    if (threadIdx.x == 0 && blockIdx.x < TRACE_BLOCKS && g >= TRACE_G0 && g < TRACE_G0 + TRACE_GENS) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        trace_buf[blockIdx.x][g - TRACE_G0][k] = t;
    }
}
#else
__device__ __forceinline__ void trace_point(int64_t, int) {}
#endif

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
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void stv2(uint64_t* p, uint64_t a, uint64_t b)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ int slot_of(int64_t g) { return (int)(g % SLOTS); }

// Named block barriers (0 is __syncthreads): producers arrive, consumers wait.
constexpr int BAR_VERDICT = 1;   // control warp -> compute warps: gBest of g-1 decided
constexpr int BAR_CAND = 2;      // compute warps -> control warp: candidates of g written
constexpr int BAR_PUB = 3;       // control warp -> compute warps: winner of g published
constexpr int BAR_SPEC = 4;      // compute warps -> control warp: speculative candidates of g written
__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

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
// The abort flag is a global load: reading it on every poll would add a second
// round trip to L2 after each poll's own loads, so it is read on every 32nd.
__device__ __forceinline__ bool should_stop(const KParams& p, int64_t it)
{
    return it >= p.spin_limit || ((it & 31) == 31 && *(volatile int32_t*)&p.status->abort);
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
    int64_t n;          // entries (index checks of the checked build)
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
        v.n = n;
    } else {
        v.X = static_cast<Pos*>(in.X);
        v.P = static_cast<Pos*>(in.P);
        v.pf64 = in.pf64;
        v.plo = in.plo;
        v.phi = in.phi;
        v.pver = in.pver;
        v.pflag = in.pflag;
        v.base = 0;
        v.n = in.N;
    }
    return v;
}

// Checked build: a unit's particle range, rank and shared-memory windows.
template <class Pos>
__device__ __forceinline__ bool unit_checked(const InstDev& in, const UnitDev& un)
{
    const size_t dyn = dynamic_smem_bytes();
    bool ok = PSSO_CHK(un.i0 >= 0 && un.i0 <= un.i1 && un.i1 <= in.N && un.rank >= 0 && un.rank < in.R,
                       CHK_UNIT, un.i0);
    ok = ok && PSSO_CHK(un.smem_off >= 0 && (size_t)un.smem_off + (size_t)in.Dp * sizeof(Pos) <= dyn,
                        CHK_UNIT_SMEM, un.smem_off);
    if (un.resident)
        ok = ok && PSSO_CHK(un.res_off >= 0 &&
                                (size_t)un.res_off + resident_bytes(un.i1 - un.i0, in.Dp, sizeof(Pos)) <= dyn,
                            CHK_UNIT_SMEM, un.res_off);
    return ok;
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
    // pipelined blocks: candidates posted before the verdict (speculative)
    Cand spec_cand[16];
    unsigned long long spec_acc[16];
    int spec_bad[16];                     // 1: a decision of the warp needs FP64
    int flag;
    int row_changed;                      // step A replaced the gBest row in gs
    unsigned long long lag_r2;            // pipelined rank 0: second-round FP64 evaluations of
                                          // the generation whose counters are still to be logged
    long long idx[MAX_UNITS_PER_BLOCK];   // identity (index, version) of the row in gs
    uint32_t ver[MAX_UNITS_PER_BLOCK];
};

// Warp reduction of candidates over xor offsets 16 .. first_off: only the keys
// travel (value / bounds and index); the full winner is then read from the lane
// that owns it.  Lanes whose xor partners at those offsets all hold
// candidates (lane 0 in particular) end with the result.
template <bool F32R>
__device__ __forceinline__ Cand cand_warp_reduce(const Cand& c, int first_off, int top_off = 16)
{
    double kv = c.v;
    long long ki = c.i;
    float kmh = c.mh, kl1 = c.l1, kl2 = c.l2;
    for (int off = top_off; off >= first_off; off >>= 1) {
        const long long oi = __shfl_xor_sync(0xffffffffu, ki, off);
        if (!F32R) {
            const double ov = __shfl_xor_sync(0xffffffffu, kv, off);
            if (ov < kv || (ov == kv && oi < ki)) { kv = ov; ki = oi; }
        } else {
            const float omh = __shfl_xor_sync(0xffffffffu, kmh, off);
            const float ol1 = __shfl_xor_sync(0xffffffffu, kl1, off);
            const float ol2 = __shfl_xor_sync(0xffffffffu, kl2, off);
            const bool ofirst = (ol1 < kl1) || (ol1 == kl1 && oi < ki);
            const float l2 = ofirst ? fminf(fminf(ol2, kl1), kl2) : fminf(fminf(kl2, ol1), ol2);
            if (ofirst) { kl1 = ol1; ki = oi; }
            kl2 = l2;
            kmh = fminf(kmh, omh);
        }
    }
    const long long wi = __shfl_sync(0xffffffffu, ki, 0);
    const unsigned own = __ballot_sync(0xffffffffu, c.i == wi);
    const int src = own ? __ffs(own) - 1 : 0;
    Cand r;
    r.i = wi;
    r.v = __shfl_sync(0xffffffffu, c.v, src);
    r.l1 = __shfl_sync(0xffffffffu, c.l1, src);
    r.h1 = __shfl_sync(0xffffffffu, c.h1, src);
    r.ver = __shfl_sync(0xffffffffu, c.ver, src);
    r.has1 = __shfl_sync(0xffffffffu, c.has1, src);
    r.rank = __shfl_sync(0xffffffffu, c.rank, src);
    r.mh = __shfl_sync(0xffffffffu, kmh, 0);
    r.l2 = __shfl_sync(0xffffffffu, kl2, 0);
    return r;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------
// Step B for one particle, split into a pure part (compute: the new position,
// its fitness, the pBest decision and the resulting state, all in registers)
// and the stores (commit).  The split lets a block compute generation g while
// the records of generation g-1 are still travelling, assuming the gBest row it
// holds is still current, and commit only once the records confirm it.
template <class Pos, int MAXC>
struct PartState {
    Pos x[MAXC][4];     // new position chunks of this lane
    double f64v;        // FP64 value of the resulting pBest (when has64)
    double cachef;      // F32: exact pBest value to cache (rejected after a recheck)
    float lo, hi;       // F32: bounds of the resulting pBest
    uint32_t ver;       // row version of the resulting pBest
    uint32_t rck;       // FP64 evaluations done
    int has64;
    bool accept;        // P <- X
    bool wstate;        // write the pBest state (false: identical row accepted)
    bool cachep;        // store cachef as the kept pBest's exact value
    bool undecided;     // F32: the bounds overlap; resolved in FP64 at commit
};

template <class Pos, bool F32R, int MAXC>
__device__ __forceinline__ void particle_compute(const Hot& in, const View<Pos>& v,
                                                 const Pos* __restrict__ gs, int64_t i, int64_t e,
                                                 int64_t g, int lane_g, unsigned gmask,
                                                 PartState<Pos, MAXC>& s)
{
    if (!PSSO_CHK(e >= 0 && e < v.n, CHK_ROW, e)) {
        s.accept = s.wstate = s.cachep = s.undecided = false;
        s.rck = 0;
        s.has64 = 0;
        s.ver = 0;
        s.f64v = s.cachef = DBL_MAX;
        s.lo = s.hi = FLT_MAX;
        return;
    }
    const Pos* xr = v.X + e * in.Dp;
    const Pos* pr = v.P + e * in.Dp;
    const uint32_t gg = (uint32_t)g;
    const uint32_t ctr3r = TAG_RHO | (in.sid << 8), ctr3f = TAG_FRESH | (in.sid << 8);
    bool eqp = true;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
        if (c < in.nchunks) {
            const int nvalid = min(4, in.D - 4 * c);
            const uint32_t valid = (1u << nvalid) - 1u;
            if (g == 0) {
#pragma unroll
                for (int m = 0; m < 4; ++m) s.x[q][m] = Pos(0);
                fresh_chunk(s.x[q], valid, (uint32_t)c, (uint32_t)i + in.i_base, 0u, TAG_INIT, in);
            } else {
                // rho block and (FP32 lattice) fresh block are independent: both
                // are generated together so their latencies overlap.
                const uint4 rb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3r), in.k0, in.k1);
                uint4 fb = make_uint4(0u, 0u, 0u, 0u);
                if (sizeof(Pos) == 4)
                    fb = philox10(make_uint4((uint32_t)c, (uint32_t)i + in.i_base, gg, ctr3f), in.k0, in.k1);
                Pos xo[4], po[4], go[4];
                // xo: the third interval's source, go: the first's (Eq. 2.1 as printed
                // swaps them: keep x first, gBest third)
                ld4((in.order ? gs : xr) + 4 * c, xo);
                ld4(pr + 4 * c, po);
                ld4((in.order ? xr : gs) + 4 * c, go);
                uint32_t nf = 0;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const uint32_t r = word_of(rb, m);
                    const bool lg = (r < in.Tg32) || (in.tfull & 1u);
                    const bool lp = (r < in.Tp32) || (in.tfull & 2u);
                    const bool lw = (r < in.Tw32) || (in.tfull & 4u);
                    s.x[q][m] = lg ? go[m] : lp ? po[m] : xo[m];
                    if (!lw) nf |= 1u << m;
                }
                nf &= valid;
                if (nf) {
                    if constexpr (sizeof(Pos) == 4) {
#pragma unroll
                        for (int m = 0; m < 4; ++m)
                            if (nf & (1u << m)) s.x[q][m] = (Pos)fresh_f32(word_of(fb, m), in);
                    } else {
                        fresh_chunk(s.x[q], nf, (uint32_t)c, (uint32_t)i + in.i_base, gg, TAG_FRESH, in);
                    }
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (m >= nvalid) s.x[q][m] = Pos(0);
                    eqp = eqp && same_bits(s.x[q][m], po[m]);
                }
            }
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) s.x[q][m] = Pos(0);
        }
    }
    s.rck = 0;
    s.cachep = false;
    s.cachef = 0.0;
    s.undecided = false;
    if constexpr (!F32R) {
        const double f = fit64<Pos, MAXC>(in, s.x, lane_g, gmask, in.G);
        const double pf = (g == 0) ? f : v.pf64[e];
        s.accept = (g == 0) || (f <= pf);
        s.wstate = s.accept;
        s.f64v = s.accept ? f : pf;
        s.ver = s.accept ? gg : v.pver[e];
        s.has64 = 1;
        s.lo = 0.f;
        s.hi = 0.f;
    } else {
        const Fit32 r = fit32<MAXC>(in, s.x, lane_g, gmask, in.G);
        s.lo = __fsub_rd(r.f, r.E);
        s.hi = __fadd_ru(r.f, r.E);
        s.has64 = 0;
        s.f64v = 0.0;
        s.wstate = true;
        // A rotated function's accepted value whose bounds are too wide to place
        // it within 1e-6 of the FP64 value is made exact at commit (the decision
        // itself is certain): the pBest fitness of an FP32 run stays within 1e-6
        // relative of the FP64 oracle's.
        const bool tighten = is_rotated(in.fn) && too_wide(in.fn, s.lo, s.hi);
        if (g == 0) {
            s.accept = !tighten;
            s.undecided = tighten;
        } else {
            const float plo = v.plo[e], phi = v.phi[e];
            const uint32_t pfl = v.pflag[e];
            const double ppf = v.pf64[e];
            if (__all_sync(gmask, eqp)) {
                s.accept = true;            // identical row: identical fitness, keep its state
                s.wstate = false;
                s.lo = plo; s.hi = phi; s.has64 = (int)(pfl & 1u); s.f64v = ppf;
            } else if (s.hi < plo) {
                s.accept = !tighten;
                s.undecided = tighten;      // certain accept, value made exact at commit
            } else if (s.lo > phi) {
                s.accept = false;
                s.lo = plo; s.hi = phi; s.has64 = (int)(pfl & 1u); s.f64v = ppf;
            } else {
                s.undecided = true;         // resolved in FP64 at commit
                s.accept = false;
            }
        }
        s.ver = (s.accept && s.wstate) ? gg : (g == 0 ? 0u : v.pver[e]);
    }
}

// FP32 mode, bounds overlapping: the pBest decision in FP64 in the oracle's
// order, from the committed X row and the pBest row (or its cached value).
struct Resolved {
    double f64v, cachef;
    float lo, hi;
    uint32_t rck;
    int accept, cachep;
};

template <class Pos, int MAXC>
__device__ __noinline__ Resolved resolve_f64(const Hot& in, const Pos* xr, const Pos* pr, bool have_p,
                                             double ppf, int lane_g, unsigned gmask)
{
    Pos a[MAXC][4], b[MAXC][4];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
        if (c < in.nchunks) {
            ld4(xr + 4 * c, a[q]);
            ld4(pr + 4 * c, b[q]);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) { a[q][m] = Pos(0); b[q][m] = Pos(0); }
        }
    }
    Resolved r;
    r.rck = 1;
    const double fx = fit64<Pos, MAXC>(in, a, lane_g, gmask, in.G);
    double fp = ppf;
    if (!have_p) {
        fp = fit64<Pos, MAXC>(in, b, lane_g, gmask, in.G);
        r.rck = 2;
    }
    r.accept = fx <= fp;
    r.f64v = r.accept ? fx : fp;
    r.lo = f64_to_f32_rd(r.f64v);
    r.hi = f64_to_f32_ru(r.f64v);
    r.cachep = !r.accept;
    r.cachef = fp;
    return r;
}

template <class Pos, bool F32R, int MAXC>
__device__ __forceinline__ void particle_commit(const Hot& in, const View<Pos>& v, int64_t e,
                                                int64_t g, int lane_g, unsigned gmask,
                                                PartState<Pos, MAXC>& s, unsigned long long& n_acc,
                                                unsigned long long& n_rck)
{
    if (!PSSO_CHK(e >= 0 && e < v.n, CHK_ROW, e)) return;
    Pos* xr = v.X + e * in.Dp;
    Pos* pr = v.P + e * in.Dp;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) {
        const int c = lane_g + 32 * q;
        if (c < in.nchunks) st4(xr + 4 * c, s.x[q]);
    }
    if (F32R && s.undecided) {
        __syncwarp(gmask);
        // generation 0 has no pBest yet: compare against +inf, i.e. accept
        const bool g0 = (g == 0);
        const Resolved r = resolve_f64<Pos, MAXC>(in, xr, pr, g0 || (v.pflag[e] & 1u) != 0,
                                                  g0 ? __longlong_as_double(0x7ff0000000000000LL) : v.pf64[e],
                                                  lane_g, gmask);
        s.accept = r.accept;
        s.has64 = 1;
        s.f64v = r.f64v;
        s.lo = r.lo;
        s.hi = r.hi;
        s.cachep = r.cachep;
        s.cachef = r.cachef;
        s.rck = r.rck;
        s.ver = s.accept ? (uint32_t)g : v.pver[e];
    }
    if (s.accept) {
#pragma unroll
        for (int q = 0; q < MAXC; ++q) {
            const int c = lane_g + 32 * q;
            if (c < in.nchunks) st4(pr + 4 * c, s.x[q]);
        }
    }
    if (lane_g != 0) return;
    n_rck += s.rck;
    if (F32R && s.cachep) {
        v.pf64[e] = s.cachef;
        v.pflag[e] = 1u;
        v.plo[e] = s.lo;
        v.phi[e] = s.hi;
    }
    if (s.accept) {
        n_acc++;
        if (s.wstate) {
            v.pver[e] = (uint32_t)g;
            v.pf64[e] = s.has64 ? s.f64v : 0.0;
            if (F32R) {
                v.pflag[e] = (uint32_t)s.has64;
                v.plo[e] = s.lo;
                v.phi[e] = s.hi;
            }
        }
    }
}

template <class Pos, bool F32R, int MAXC>
__device__ __forceinline__ Cand particle_cand(int64_t i, const PartState<Pos, MAXC>& s)
{
    return cand_of<F32R>((long long)i, s.f64v, s.lo, s.hi, s.has64, s.ver);
}

// Lane geometry of step B: G lanes per particle, groups numbered across the block.
struct Groups {
    int G, lane_g, ngroups, gid;
    unsigned gmask;
};
__device__ __forceinline__ Groups groups_of(int G, int first_warp = 0)
{
    Groups q;
    const int lane = threadIdx.x & 31;
    const int gpw = 32 / G;
    q.G = G;
    q.lane_g = lane & (G - 1);
    q.ngroups = ((blockDim.x >> 5) - first_warp) * gpw;
    q.gid = ((threadIdx.x >> 5) - first_warp) * gpw + lane / G;
    q.gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    return q;
}

// Folds the group leaders' candidates into lane 0 and sums the counters per warp.
template <bool F32R>
__device__ __forceinline__ Cand warp_fold(Cand best, int G, unsigned long long& n_acc,
                                          unsigned long long& n_rck)
{
    if (G < 32) best = cand_warp_reduce<F32R>(best, G);
    // only group leaders (lanes 0, G, 2G, ...) hold counts: lane 0 ends with the sum
    for (int off = 16; off >= G; off >>= 1) {
        n_acc += __shfl_xor_sync(0xffffffffu, n_acc, off);
        n_rck += __shfl_xor_sync(0xffffffffu, n_rck, off);
    }
    return best;
}

// Step B, non-speculative: every particle of the unit, computed and committed.
template <class Pos, bool F32R, int MAXC>
__device__ Cand step_b(const InstDev& desc, const UnitDev& un, const View<Pos>& v,
                       const Pos* __restrict__ gs, int64_t g, unsigned long long& n_acc,
                       unsigned long long& n_rck)
{
    // Loaded once, before any store: the fields stay in registers instead of
    // being reloaded after every store through a generic X / P pointer.
    const Hot in = hot_of(desc);
    const Groups gr = groups_of(in.G);
    const int64_t n = un.i1 - un.i0;
    Cand best = cand_none();
    for (int64_t k = gr.gid; k < n; k += gr.ngroups) {
        const int64_t i = un.i0 + k;
        const int64_t e = i - v.base;
        PartState<Pos, MAXC> st;
        particle_compute<Pos, F32R, MAXC>(in, v, gs, i, e, g, gr.lane_g, gr.gmask, st);
        particle_commit<Pos, F32R, MAXC>(in, v, e, g, gr.lane_g, gr.gmask, st, n_acc, n_rck);
        if (gr.lane_g == 0) best = cand_merge<F32R>(best, particle_cand<Pos, F32R, MAXC>(i, st));
    }
    trace_point(g, 6);
    return warp_fold<F32R>(best, in.G, n_acc, n_rck);
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
    // a reduction without a return value: no load round trip on the path of
    // every generation (and none at all when there was no recheck)
    if (w.rck) atomicAdd(reinterpret_cast<unsigned long long*>(&gb->total_rechecks), (unsigned long long)w.rck);
    gb->f64 = w.f64;
    gb->lo = w.lo;
    gb->hi = w.hi;
    gb->ver = w.ver;
    gb->has64 = w.has64;
    if (in.log_stride > 0 && in.log_cap > 0 && (g % in.log_stride) == 0) {
        const int64_t le = (g / in.log_stride) % in.log_cap;
        if (!PSSO_CHK(le >= 0 && le < in.log_cap, CHK_LOG, le)) return;
        LogDev* e = in.log + le;
        e->gen = g;
        e->idx = w.idx;
        e->value = w.has64 ? w.f64 : __longlong_as_double(0x7ff8000000000000LL);
        e->lo = w.lo;
        e->hi = w.hi;
        e->accepted = (int64_t)w.acc;
        e->rechecks = (int64_t)w.rck;
    }
}

// Step C, exact fallback (FP32 mode, warp 0): several particles' bounds reach
// the smallest upper bound m; make every such candidate exact in FP64 (oracle
// order) and return the exact lowest-index arg-min.  Rare.
template <class Pos>
__device__ __noinline__ Cand step_c_exact(const InstDev& in, const UnitDev un, const View<Pos> v,
                                          float m, unsigned long long* extra)
{
    const int lane = threadIdx.x & 31;
    const int64_t n = un.i1 - un.i0;
    const Hot hin = hot_of(in);
    unsigned long long rck = 0;
    for (int64_t base = 0; base < n; base += 32) {
        const int64_t k = base + lane;
        const int64_t e = un.i0 + k - v.base;
        const bool need = k < n && PSSO_CHK(e >= 0 && e < v.n, CHK_REFINE, e) && v.plo[e] <= m &&
                          !(v.pflag[e] & 1u);
        unsigned bm = __ballot_sync(0xffffffffu, need);
        while (bm) {
            const int l = __ffs(bm) - 1;
            bm &= bm - 1;
            const int64_t e2 = un.i0 + base + l - v.base;
            const double f = fit64_row<Pos>(hin, v.P + e2 * in.Dp, false);
            if (lane == 0) {
                v.pf64[e2] = f;
                v.pflag[e2] = 1u;
                v.plo[e2] = f64_to_f32_rd(f);
                v.phi[e2] = f64_to_f32_ru(f);
                rck++;
            }
            __syncwarp();
        }
    }
    // The true arg-min now has an exact value; every particle without one has
    // a lower bound above m.
    Cand ex = cand_none();
    for (int64_t k = lane; k < n; k += 32) {
        const int64_t e = un.i0 + k - v.base;
        if (PSSO_CHK(e >= 0 && e < v.n, CHK_REFINE, e) && (v.pflag[e] & 1u)) {
            Cand q = cand_none();
            q.v = v.pf64[e];
            q.i = (long long)(un.i0 + k);
            q.ver = v.pver[e];
            ex = cand_merge<false>(ex, q);
        }
    }
    Cand r = cand_warp_reduce<false>(ex, 1);
    r.has1 = 1;
    r.l1 = f64_to_f32_rd(r.v);
    r.h1 = f64_to_f32_ru(r.v);
    *extra = __shfl_sync(0xffffffffu, rck, 0);
    return r;
}

// Step C (warp 0): the unit's winner from the per-warp candidates.
template <class Pos, bool F32R>
__device__ __forceinline__ Winner step_c(const InstDev& in, const UnitDev& un, const View<Pos>& v,
                                         BlockShared& sh, int64_t g)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const Cand c = lane < nw ? sh.warp_cand[lane] : cand_none();   // unused slots hold none
    trace_point(g, 6);
    int top = 1;
    while (2 * top < nw) top <<= 1;                 // lanes >= nw hold nothing
    // The accepted and recheck counts travel as the halves of one word, so the
    // reduction is one shuffle per level: the accepted count (at most one per
    // particle, N < 2^31) never carries into the high half, which holds the
    // recheck count (a statistic).
    unsigned long long packed = lane < nw ? (sh.warp_acc[lane] | (sh.warp_rck[lane] << 32)) : 0ull;
    for (int off = top; off > 0; off >>= 1) packed += __shfl_xor_sync(0xffffffffu, packed, off);
    packed = __shfl_sync(0xffffffffu, packed, 0);
    unsigned long long acc = packed & 0xffffffffull, rck = packed >> 32;
    trace_point(g, 7);
    Cand r = cand_warp_reduce<F32R>(c, 1, top);
    trace_point(g, 10);
    if (F32R && r.l2 <= r.mh) {
        unsigned long long extra = 0;
        r = step_c_exact<Pos>(in, un, v, r.mh, &extra);
        rck += extra;
    }
    trace_point(g, 11);
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
    return w;
}

// Step C of a pipelined block on the candidates its compute warps posted
// before the verdict (valid when the gBest row did not change and no decision
// needed FP64).  Returns false when the candidates' bounds overlap: the exact
// fallback reads pBest state that the compute warps are still committing.
template <bool F32R>
__device__ __forceinline__ bool step_c_spec(const BlockShared& sh, Winner& w)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const Cand c = lane < nw ? sh.spec_cand[lane] : cand_none();
    int top = 1;
    while (2 * top < nw) top <<= 1;
    unsigned long long acc = lane < nw ? sh.spec_acc[lane] : 0ull;
    for (int off = top; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    acc = __shfl_sync(0xffffffffu, acc, 0);
    const Cand r = cand_warp_reduce<F32R>(c, 1, top);
    if (F32R && r.l2 <= r.mh) return false;
    w.idx = r.i;
    w.ver = r.ver;
    w.acc = acc;
    w.rck = 0;
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
    return true;
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

__device__ __forceinline__ bool record_ready(const uint64_t (&w)[REC_WORDS], uint32_t tag)
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < REC_WORDS; ++k) ok = ok && tagged(w[k], tag);
    return ok;
}

__device__ __forceinline__ Winner decode_record(const uint64_t (&w)[REC_WORDS])
{
    Winner r;
    r.idx = (long long)(uint32_t)w[RW_IDX];
    r.has64 = (int)((w[RW_IDX] >> 32) & 1u);
    r.ver = (uint32_t)w[RW_VER];
    if (r.has64) {
        r.f64 = __longlong_as_double((long long)(((w[RW_V1] & 0xffffffffULL) << 32) | (w[RW_V0] & 0xffffffffULL)));
        r.lo = f64_to_f32_rd(r.f64);
        r.hi = f64_to_f32_ru(r.f64);
    } else {
        r.f64 = 0.0;
        r.lo = __uint_as_float((uint32_t)w[RW_V0]);
        r.hi = __uint_as_float((uint32_t)w[RW_V1]);
    }
    r.acc = w[RW_ACC] & 0xffffffffffffULL;
    r.rck = w[RW_RCK] & 0xffffffffffffULL;
    return r;
}

__device__ __forceinline__ void load_record(const uint64_t* rp, uint64_t (&w)[REC_WORDS])
{
    ldv2(rp + RW_IDX, w[0], w[1]);
    ldv2(rp + RW_V0, w[2], w[3]);
    ldv2(rp + RW_ACC, w[4], w[5]);
}

// Reads one record (bounded wait); returns false on timeout / abort.
__device__ inline bool read_record(const uint64_t* rec, uint32_t tag, Winner& w, const KParams& p,
                                   const UnitDev& un)
{
    for (int64_t it = 0;; ++it) {
        uint64_t ww[REC_WORDS];
        load_record(rec, ww);
        if (record_ready(ww, tag)) {
            w = decode_record(ww);
            return true;
        }
        if (should_stop(p, it)) {
            give_up(p, un);
            return false;
        }
        if (it > 16) __nanosleep(it < 512 ? 20 : 200);
    }
}

// Reads the records of ranks lane, lane+32, ... (up to four per pass, all
// loads of a pass in flight together) and folds them into one candidate per
// lane.  Only a reader that sums the counters (COUNTS) loads the counter
// words; the others read the four words that decide the winner, which keeps
// the polled words of a pass in registers.  Returns false on timeout / abort.
template <bool F32R, bool COUNTS>
__device__ inline bool gather_records(const uint64_t* recs, int R, uint32_t tag, Cand& c,
                                      unsigned long long& acc, unsigned long long& rck,
                                      const KParams& p, const UnitDev& un)
{
    constexpr int NW = COUNTS ? REC_WORDS : RW_ACC;   // words read per record
    const int lane = threadIdx.x & 31;
    for (int k0 = 0; k0 * 32 < R; k0 += 4) {
        uint32_t pend = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (lane + 32 * (k0 + q) < R) pend |= 1u << q;
        for (int64_t it = 0; pend; ++it) {
            uint64_t w[4][REC_WORDS];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (pend & (1u << q)) {
                    const uint64_t* rp = recs + (size_t)(lane + 32 * (k0 + q)) * REC_WORDS;
                    ldv2(rp + RW_IDX, w[q][0], w[q][1]);
                    ldv2(rp + RW_V0, w[q][2], w[q][3]);
                    if (COUNTS) ldv2(rp + RW_ACC, w[q][4], w[q][5]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                bool ready = (pend & (1u << q)) != 0;
#pragma unroll
                for (int k = 0; k < NW; ++k) ready = ready && tagged(w[q][k], tag);
                if (ready) {
                    if (!COUNTS) { w[q][RW_ACC] = 0; w[q][RW_RCK] = 0; }
                    const Winner r = decode_record(w[q]);
                    Cand cq = cand_of<F32R>(r.idx, r.f64, r.lo, r.hi, r.has64, r.ver);
                    cq.rank = lane + 32 * (k0 + q);
                    c = cand_merge<F32R>(c, cq);
                    acc += r.acc;
                    rck += r.rck;
                    pend &= ~(1u << q);
                }
            }
            if (!pend) break;
            if (should_stop(p, it)) {
                give_up(p, un);
                return false;
            }
            if (it > 16) __nanosleep(it < 512 ? 20 : 200);
        }
    }
    return true;
}

// Pipelined rank 0 (one warp): the accepted / recheck counters of generation
// gq from every block's record, written into gq's log entry and the running
// recheck total.  Run by a compute warp after its commit of gq+1 (or by the
// control warp in the epilogue), when the counter words are present, so the
// control warp of the block that keeps the gBest state never waits for them.
// Returns false on timeout (after give_up).
static __device__ __noinline__ bool fill_counts(const KParams& p, const InstDev& in, const UnitDev& un, int64_t gq,
                                         unsigned long long extra_rck)
{
    const int lane = threadIdx.x & 31;
    const uint32_t tag = (uint32_t)gq;
    const uint64_t* recs = in.rec + (size_t)slot_of(gq) * in.R * REC_WORDS;
    unsigned long long packed = 0;
    bool ok = true;
    for (int r = lane; r < in.R && ok; r += 32) {
        for (int64_t it = 0;; ++it) {
            uint64_t a, b;
            ldv2(recs + (size_t)r * REC_WORDS + RW_ACC, a, b);
            if (tagged(a, tag) && tagged(b, tag)) {
                packed += (a & 0xffffffffull) | ((b & 0xffffffffull) << 32);
                break;
            }
            if (should_stop(p, it)) { give_up(p, un); ok = false; break; }
            if (it > 16) __nanosleep(20);
        }
    }
    if (__any_sync(0xffffffffu, !ok)) return false;
    packed = warp_sum_u64(packed);
    if (lane == 0) {
        const unsigned long long acc = packed & 0xffffffffull, rck = (packed >> 32) + extra_rck;
        if (in.log_stride > 0 && in.log_cap > 0 && (gq % in.log_stride) == 0) {
            LogDev* e = in.log + ((gq / in.log_stride) % in.log_cap);
            e->accepted = (int64_t)acc;
            e->rechecks = (int64_t)rck;
        }
        if (rck) atomicAdd(reinterpret_cast<unsigned long long*>(&in.gb->total_rechecks), rck);
    }
    __syncwarp();
    return true;
}

// Step A (warp 0) for a unit of a multi-block instance: decide the gBest of
// generation gp from the records and make sure shared memory holds its row.
// With `lag` (pipelined blocks), rank 0 writes gp's gBest state and log entry
// without the counters, which a compute warp of that block fills in during
// the next generation (fill_counts; the last generation's in the epilogue):
// the winner's keys alone are on the critical path of the block that keeps
// the gBest state, which every other block waits for.
// Sets sh.flag when the launch is aborting.
template <class Pos, bool F32R>
__device__ __noinline__ void step_a(const KParams& p, const InstDev& in, const UnitDev& un, const View<Pos>& v,
                       int uslot, Pos* gs, int64_t gp, bool finalize, BlockShared& sh, bool lag = false)
{
    const int lane = threadIdx.x & 31;
    const int R = in.R;
    const uint32_t tag = (uint32_t)gp;
    const uint64_t* recs = in.rec + (size_t)slot_of(gp) * R * REC_WORDS;
    constexpr int WPE = WordsPer<Pos>::value;

    Cand c = cand_none();
    unsigned long long acc = 0, rck = 0;
    // only the block that writes the gBest record and log sums the counters
    // (and, lagging, not yet)
    const bool counts = un.rank == 0 && finalize && !lag;
    bool ok = counts ? gather_records<F32R, true>(recs, R, tag, c, acc, rck, p, un)
                     : gather_records<F32R, false>(recs, R, tag, c, acc, rck, p, un);
    if (__any_sync(0xffffffffu, !ok)) { if (lane == 0) sh.flag = 1; return; }
    trace_point(gp + 1, 5);
    Cand win = cand_warp_reduce<F32R>(c, 1);
    if (counts) {               // halves of one word, as in step C
        const unsigned long long packed = warp_sum_u64(acc | (rck << 32));
        acc = packed & 0xffffffffull;
        rck = packed >> 32;
    }
    trace_point(gp + 1, 8);

    if (F32R && win.l2 <= win.mh) {
        // Several ranks overlap: ranks without an exact value publish it
        // (second round), then the exact lowest-index arg-min is taken.
        const float m = win.mh;
        uint64_t* recs2 = in.rec2 + (size_t)slot_of(gp) * R * REC_WORDS;
        Winner me;
        ok = read_record(recs + (size_t)un.rank * REC_WORDS, tag, me, p, un);
        if (__any_sync(0xffffffffu, !ok)) { if (lane == 0) sh.flag = 1; return; }
        if (me.lo <= m && !me.has64 &&
            PSSO_CHK(me.idx - v.base >= 0 && me.idx - v.base < v.n, CHK_REFINE, me.idx)) {
            const double f = fit64_row<Pos>(hot_of(in), v.P + (me.idx - v.base) * in.Dp, false);
            if (lane == 0) {
                Winner ww = me;
                ww.f64 = f;
                ww.has64 = 1;
                ww.acc = 0;
                ww.rck = 1;
                publish_record(recs2 + (size_t)un.rank * REC_WORDS, tag, ww);
            }
        }
        Cand ex = cand_none();
        unsigned long long r2 = 0;
        for (int r = lane; r < R; r += 32) {
            Winner w;
            if (!read_record(recs + (size_t)r * REC_WORDS, tag, w, p, un)) { ok = false; break; }
            if (w.lo > m) continue;
            if (!w.has64) {
                if (!read_record(recs2 + (size_t)r * REC_WORDS, tag, w, p, un)) { ok = false; break; }
                r2 += 1;
            }
            Cand q = cand_none();
            q.v = w.f64;
            q.i = w.idx;
            q.ver = w.ver;
            q.rank = r;
            ex = cand_merge<false>(ex, q);
        }
        if (__any_sync(0xffffffffu, !ok)) { if (lane == 0) sh.flag = 1; return; }
        win = cand_warp_reduce<false>(ex, 1);
        win.has1 = 1;
        win.l1 = f64_to_f32_rd(win.v);
        win.h1 = f64_to_f32_ru(win.v);
        r2 = warp_sum_u64(r2);
        rck += r2;
        if (lag && lane == 0) sh.lag_r2 = r2;
    } else if (lag && lane == 0) {
        sh.lag_r2 = 0;
    }

    // Fetch the winner's row if it is not the one already in shared memory.
    const bool changed = (sh.idx[uslot] != win.i) || (sh.ver[uslot] != win.ver);
    if (changed && !PSSO_CHK(win.rank >= 0 && win.rank < R, CHK_SLOT, win.rank)) {
        if (lane == 0) give_up(p, un);
        ok = false;
    } else if (changed) {
        const uint64_t* src = static_cast<const uint64_t*>(in.grow) +
                              ((size_t)slot_of(gp) * R + win.rank) * (size_t)in.Dp * WPE;
        for (int ch = lane; ch < in.nchunks; ch += 32) {
            Pos vals[4];
            for (int64_t it = 0;; ++it) {
                if (get_chunk(src + (size_t)4 * ch * WPE, tag, vals)) break;
                if (should_stop(p, it)) { give_up(p, un); ok = false; break; }
                if (it > 16) __nanosleep(32);
            }
            st4(gs + 4 * ch, vals);
        }
    }
    trace_point(gp + 1, 9);
    if (__any_sync(0xffffffffu, !ok)) { if (lane == 0) sh.flag = 1; return; }
    __syncwarp();
    if (un.rank == 0 && finalize) {
        if (changed) {
            Pos* dst = static_cast<Pos*>(in.gbrow);
            for (int ch = lane; ch < in.nchunks; ch += 32) {
                Pos t[4];
                ld4(gs + 4 * ch, t);
                st4(dst + 4 * ch, t);
            }
        }
        if (lane == 0) {
            Winner w;
            w.idx = win.i;
            w.ver = win.ver;
            w.acc = lag ? 0 : acc;       // lagging: fill_counts writes them
            w.rck = lag ? 0 : rck;
            w.has64 = F32R ? win.has1 : 1;
            w.f64 = F32R ? (win.has1 ? win.v : 0.0) : win.v;
            w.lo = F32R ? win.l1 : f64_to_f32_rd(win.v);
            w.hi = F32R ? win.h1 : f64_to_f32_ru(win.v);
            write_gbest(in, w, gp);
        }
    }
    if (lane == 0) {
        sh.idx[uslot] = win.i;
        sh.ver[uslot] = win.ver;
        sh.row_changed = changed ? 1 : 0;
    }
}

// Step D (warp 0) for a multi-block instance: publish the unit's winner row and record.
template <class Pos>
__device__ __forceinline__ void step_d_publish(const KParams& p, const InstDev& in, const UnitDev& un,
                               const View<Pos>& v, const Winner& w, int64_t g, bool with_record = true)
{
    if (p.fault_skip_rank > 0 && un.inst == 0 && un.rank == p.fault_skip_rank - 1) return;
    constexpr int WPE = WordsPer<Pos>::value;
    const int lane = threadIdx.x & 31;
    const int R = in.R;
    const uint32_t tag = (uint32_t)g;
    uint64_t* dst = static_cast<uint64_t*>(in.grow) + ((size_t)slot_of(g) * R + un.rank) * (size_t)in.Dp * WPE;
    if (!PSSO_CHK(w.idx - v.base >= 0 && w.idx - v.base < v.n, CHK_GBEST_SRC, w.idx)) return;
    const Pos* src = v.P + (w.idx - v.base) * in.Dp;
    for (int ch = lane; ch < in.nchunks; ch += 32) {
        Pos t[4];
        ld4(src + 4 * ch, t);
        put_chunk(dst + (size_t)4 * ch * WPE, tag, t);
    }
    if (lane == 0 && with_record) publish_record(in.rec + ((size_t)slot_of(g) * R + un.rank) * REC_WORDS, tag, w);
}

// The record alone (lane 0 of warp 0); its row follows with step_d_publish(..., false).
// Readers poll the row words' tags, so a row published after its record is
// only waited for, never read stale.
__device__ __forceinline__ void publish_record_of(const KParams& p, const InstDev& in, const UnitDev& un,
                                                  const Winner& w, int64_t g)
{
    if (p.fault_skip_rank > 0 && un.inst == 0 && un.rank == p.fault_skip_rank - 1) return;
    publish_record(in.rec + ((size_t)slot_of(g) * in.R + un.rank) * REC_WORDS, (uint32_t)g, w);
}

// Step D (warp 0) for a whole-swarm unit: refresh the shared-memory gBest row.
template <class Pos>
__device__ __noinline__ void step_d_local(const InstDev& in, const View<Pos>& v, const Winner& w, Pos* gs,
                             int uslot, int64_t g, BlockShared& sh)
{
    const int lane = threadIdx.x & 31;
    const bool changed = (sh.idx[uslot] != w.idx) || (sh.ver[uslot] != w.ver);
    if (changed && PSSO_CHK(w.idx - v.base >= 0 && w.idx - v.base < v.n, CHK_GBEST_SRC, w.idx)) {
        const Pos* src = v.P + (w.idx - v.base) * in.Dp;
        Pos* dst = static_cast<Pos*>(in.gbrow);
        for (int ch = lane; ch < in.nchunks; ch += 32) {
            Pos t[4];
            ld4(src + 4 * ch, t);
            st4(gs + 4 * ch, t);
            st4(dst + 4 * ch, t);
        }
    }
    __syncwarp();
    if (lane == 0) {
        sh.idx[uslot] = w.idx;
        sh.ver[uslot] = w.ver;
        write_gbest(in, w, g);
    }
}

// ---------------------------------------------------------------------------
template <class Pos, bool F32R, int MC>
__device__ Cand unit_b(const InstDev& in, const UnitDev& un, const View<Pos>& v, const Pos* gs,
                       int64_t g, unsigned long long& n_acc, unsigned long long& n_rck)
{
    if (MC == 1 || in.maxc == 1) return step_b<Pos, F32R, 1>(in, un, v, gs, g, n_acc, n_rck);
    if (MC == 2 || in.maxc == 2) return step_b<Pos, F32R, (MC < 2 ? MC : 2)>(in, un, v, gs, g, n_acc, n_rck);
    if (MC == 4 || in.maxc == 4) return step_b<Pos, F32R, (MC < 4 ? MC : 4)>(in, un, v, gs, g, n_acc, n_rck);
    return step_b<Pos, F32R, MC>(in, un, v, gs, g, n_acc, n_rck);
}

// Step B overlapped with step A: each group (at most one particle per group)
// computes generation g with the gBest row it holds, while warp 0 reads the
// records of g-1.  If the winner's row is the one used, the results are
// committed as computed; otherwise (the gBest moved) they are recomputed.
template <class Pos, bool F32R, int MAXC>
__device__ Cand spec_b(const KParams& p, const InstDev& desc, const UnitDev& un, const View<Pos>& v,
                       Pos* gs, int slot, int64_t g, BlockShared& sh, unsigned long long& n_acc,
                       unsigned long long& n_rck)
{
    const Hot in = hot_of(desc);
    const Groups gr = groups_of(in.G);
    const int64_t n = un.i1 - un.i0;
    const bool have = gr.gid < n;
    const int64_t i = un.i0 + gr.gid, e = i - v.base;
    PartState<Pos, MAXC> st;
    bool need = have;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        if (need) particle_compute<Pos, F32R, MAXC>(in, v, gs, i, e, g, gr.lane_g, gr.gmask, st);
        if (pass == 1) break;
        trace_point(g, 7);
        if ((threadIdx.x >> 5) == 0)
            step_a<Pos, F32R>(p, desc, un, v, slot, gs, g - 1, g - 1 >= p.g_begin, sh);
        __syncthreads();
        if (sh.flag) return cand_none();
        trace_point(g, 1);
        need = have && sh.row_changed;     // the gBest moved: recompute with the new row
        if (!need) break;
    }
    Cand best = cand_none();
    if (have) {
        particle_commit<Pos, F32R, MAXC>(in, v, e, g, gr.lane_g, gr.gmask, st, n_acc, n_rck);
        if (gr.lane_g == 0) best = particle_cand<Pos, F32R, MAXC>(i, st);
    }
    trace_point(g, 6);
    return warp_fold<F32R>(best, in.G, n_acc, n_rck);
}

template <class Pos, bool F32R, int MC>
__device__ Cand unit_spec(const KParams& p, const InstDev& in, const UnitDev& un, const View<Pos>& v,
                          Pos* gs, int slot, int64_t g, BlockShared& sh, unsigned long long& n_acc,
                          unsigned long long& n_rck)
{
    if (MC == 1 || in.maxc == 1) return spec_b<Pos, F32R, 1>(p, in, un, v, gs, slot, g, sh, n_acc, n_rck);
    if (MC == 2 || in.maxc == 2)
        return spec_b<Pos, F32R, (MC < 2 ? MC : 2)>(p, in, un, v, gs, slot, g, sh, n_acc, n_rck);
    if (MC == 4 || in.maxc == 4)
        return spec_b<Pos, F32R, (MC < 4 ? MC : 4)>(p, in, un, v, gs, slot, g, sh, n_acc, n_rck);
    return spec_b<Pos, F32R, MC>(p, in, un, v, gs, slot, g, sh, n_acc, n_rck);
}

// Warp-specialised pipeline for a block that owns one unit of a multi-block
// instance with at most one particle per compute group.  Warp 0 (control)
// runs steps C and D of generation g and step A of g (reading every block's
// record); once it has published, warps 1.. (compute) already evaluate
// generation g+1 with the gBest row they hold while the records travel.  When
// the verdict of step A says the row was current, their results are committed
// as computed; otherwise they are recomputed.  The compute warps start only
// after the publication so that steps C and D, on the critical path of every
// block, do not share issue slots with them.  Before the verdict they post
// the arg-min candidates their evaluation implies: when the row did not change
// and no decision needs FP64, the control warp sends the record on those while
// the compute warps commit, and the row after the commit.  In rank 0 (FP32
// fitness) a compute warp also fills in the previous generation's counters of
// the gBest log.  Four named barriers carry the hand-offs: speculative
// candidates and committed candidates (compute -> control), verdict and
// publication (control -> compute).
template <class Pos, bool F32R, int MAXC>
__device__ void pipelined_unit(const KParams& p, const InstDev& desc, const UnitDev& un,
                               const View<Pos>& v, Pos* gs, int slot, BlockShared& sh)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nth = blockDim.x;
    if (warp == 0) {
        if (lane == 0) {      // the control warp's own slots hold no candidate
            sh.warp_cand[0] = cand_none(); sh.warp_acc[0] = 0; sh.warp_rck[0] = 0;
            sh.spec_cand[0] = cand_none(); sh.spec_acc[0] = 0; sh.spec_bad[0] = 0;
        }
        __syncwarp();
        const int nw = nth >> 5;
        for (int64_t g = p.g_begin; g <= p.g_end; ++g) {
            trace_point(g, 0);
            if (g > 0) {
                step_a<Pos, F32R>(p, desc, un, v, slot, gs, g - 1, g - 1 >= p.g_begin, sh, F32R);
            } else if (lane == 0) {
                sh.row_changed = 0;
            }
            __syncwarp();
            trace_point(g, 1);
            bar_arrive(BAR_VERDICT, nth);
            if (sh.flag) return;
            // When the speculation held, the winner's record goes out on the
            // candidates posted before the verdict, while the compute warps
            // commit; the row follows once they have.
            bar_sync(BAR_SPEC, nth);
            trace_point(g, 2);
            const bool bad = __any_sync(0xffffffffu, lane < nw && sh.spec_bad[lane] != 0);
            Winner w;
            bool sent = false;
            if (!sh.row_changed && !bad) {
                sent = step_c_spec<F32R>(sh, w);
                if (sent && lane == 0) publish_record_of(p, desc, un, w, g);
            }
            trace_point(g, 3);
            bar_sync(BAR_CAND, nth);
            if (sent) {
                step_d_publish<Pos>(p, desc, un, v, w, g, false);
            } else {
                w = step_c<Pos, F32R>(desc, un, v, sh, g);
                step_d_publish<Pos>(p, desc, un, v, w, g);
            }
            trace_point(g, 4);
            if (g < p.g_end) bar_arrive(BAR_PUB, nth);
        }
        return;
    }
    const Hot in = hot_of(desc);
    const Groups gr = groups_of(in.G, 1);
    const int64_t n = un.i1 - un.i0;
    const bool have = gr.gid < n;
    const int64_t i = un.i0 + gr.gid, e = i - v.base;
    for (int64_t g = p.g_begin; g <= p.g_end; ++g) {
        if (g > p.g_begin) bar_sync(BAR_PUB, nth);
        PartState<Pos, MAXC> st;
        if (have) particle_compute<Pos, F32R, MAXC>(in, v, gs, i, e, g, gr.lane_g, gr.gmask, st);
        {   // speculative candidate: exact unless the row changes or a decision needs FP64
            unsigned long long s_acc = 0, s_rck = 0;
            Cand sb = cand_none();
            int bad = 0;
            if (have && gr.lane_g == 0) {
                if (F32R && st.undecided) bad = 1;
                else {
                    sb = particle_cand<Pos, F32R, MAXC>(i, st);
                    s_acc = st.accept ? 1ull : 0ull;
                }
            }
            bad = __any_sync(0xffffffffu, bad);
            sb = warp_fold<F32R>(sb, in.G, s_acc, s_rck);
            if (lane == 0) {
                sh.spec_cand[warp] = sb;
                sh.spec_acc[warp] = s_acc;
                sh.spec_bad[warp] = bad;
            }
        }
        bar_arrive(BAR_SPEC, nth);
        if (threadIdx.x == 32) trace_point(g, 7);
        bar_sync(BAR_VERDICT, nth);
        if (sh.flag) return;
        const unsigned long long r2_prev = sh.lag_r2;   // stashed by step A of g-1
        if (have && sh.row_changed)       // the gBest moved: recompute with the new row
            particle_compute<Pos, F32R, MAXC>(in, v, gs, i, e, g, gr.lane_g, gr.gmask, st);
        unsigned long long n_acc = 0, n_rck = 0;
        Cand best = cand_none();
        if (have) {
            particle_commit<Pos, F32R, MAXC>(in, v, e, g, gr.lane_g, gr.gmask, st, n_acc, n_rck);
            if (gr.lane_g == 0) best = particle_cand<Pos, F32R, MAXC>(i, st);
        }
        best = warp_fold<F32R>(best, in.G, n_acc, n_rck);
        if (lane == 0) {
            sh.warp_cand[warp] = best;
            sh.warp_acc[warp] = n_acc;
            sh.warp_rck[warp] = n_rck;
        }
        if (threadIdx.x == 32) trace_point(g, 6);
        bar_arrive(BAR_CAND, nth);
        // rank 0: the counters of g-1 go into its log entry while this warp
        // would otherwise wait for the publication
        // (FP32 fitness only: with FP64 fitness the compute warps have no slack
        // before the next speculative candidates, and the counters stay in step A)
        if (F32R && un.rank == 0 && warp == 1 && g - 1 >= p.g_begin) fill_counts(p, desc, un, g - 1, r2_prev);
    }
}

template <class Pos, bool F32R, int MC>
__device__ void pipelined(const KParams& p, const InstDev& in, const UnitDev& un, const View<Pos>& v,
                          Pos* gs, int slot, BlockShared& sh)
{
    if (MC == 1 || in.maxc == 1) return pipelined_unit<Pos, F32R, 1>(p, in, un, v, gs, slot, sh);
    if (MC == 2 || in.maxc == 2) return pipelined_unit<Pos, F32R, (MC < 2 ? MC : 2)>(p, in, un, v, gs, slot, sh);
    if (MC == 4 || in.maxc == 4) return pipelined_unit<Pos, F32R, (MC < 4 ? MC : 4)>(p, in, un, v, gs, slot, sh);
    return pipelined_unit<Pos, F32R, MC>(p, in, un, v, gs, slot, sh);
}

// Launch bound: kernels for wide rows (4 or 8 chunks of 4 variables per lane)
// are limited to 256 threads so that each thread may use up to 255 registers.
template <int MC> struct GenBound { static constexpr int threads = MC >= 4 ? 256 : 512; };

// Per generation and unit, warp 0 runs steps A, C and D; all warps run step B.
// Two block barriers per generation: after step A (the gBest row is in shared
// memory) and after step B (every particle's candidate is in shared memory).
template <class Pos, bool F32R, int MC>
__global__ void __launch_bounds__(GenBound<MC>::threads) sso_generations(const KParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockShared sh;
    const int u0 = p.block_first[blockIdx.x], u1 = p.block_first[blockIdx.x + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Prologue: resident units move into shared memory; whole-swarm units
    // restore their gBest row.
    if (threadIdx.x == 0) sh.flag = 0;
    for (int u = u0; u < u1; ++u) {
        const UnitDev un = p.units[u];
        const InstDev& in = p.inst[un.inst];
        if (!unit_checked<Pos>(in, un)) {
            if (threadIdx.x == 0) { sh.flag = 1; give_up(p, un); }
            break;
        }
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
#ifdef PSSO_CHECKED
    if (sh.flag) return;
#endif

    if (u1 - u0 == 1 && p.units[u0].pipelined) {
        const UnitDev un = p.units[u0];
        const InstDev& in = p.inst[un.inst];
        Pos* gs = reinterpret_cast<Pos*>(smem + un.smem_off);
        const View<Pos> v = make_view<Pos>(in, un, smem);
        pipelined<Pos, F32R, MC>(p, in, un, v, gs, 0, sh);
    } else {
    for (int64_t g = p.g_begin; g <= p.g_end; ++g) {
        for (int u = u0; u < u1; ++u) {
            const UnitDev un = p.units[u];
            const InstDev& in = p.inst[un.inst];
            Pos* gs = reinterpret_cast<Pos*>(smem + un.smem_off);
            const View<Pos> v = make_view<Pos>(in, un, smem);
            const int slot = u - u0;
            trace_point(g, 0);
            const bool exchange = in.R > 1 && g > 0;
            const int ngroups = (blockDim.x >> 5) * (32 / in.G);
            unsigned long long n_acc = 0, n_rck = 0;
            Cand c;
            if (exchange && un.i1 - un.i0 <= ngroups) {
                c = unit_spec<Pos, F32R, MC>(p, in, un, v, gs, slot, g, sh, n_acc, n_rck);
                if (sh.flag) return;
            } else {
                if (warp == 0 && exchange)
                    step_a<Pos, F32R>(p, in, un, v, slot, gs, g - 1, g - 1 >= p.g_begin, sh);
                __syncthreads();
                if (sh.flag) return;
                trace_point(g, 1);
                c = unit_b<Pos, F32R, MC>(in, un, v, gs, g, n_acc, n_rck);
            }
            if (lane == 0) {
                sh.warp_cand[warp] = c;
                sh.warp_acc[warp] = n_acc;
                sh.warp_rck[warp] = n_rck;
            }
            __syncthreads();
            trace_point(g, 2);
            if (warp == 0) {
                const Winner w = step_c<Pos, F32R>(in, un, v, sh, g);
                trace_point(g, 3);
                if (in.R == 1) step_d_local<Pos>(in, v, w, gs, slot, g, sh);
                else step_d_publish<Pos>(p, in, un, v, w, g);
            }
            trace_point(g, 4);
        }
    }
    }
    __syncthreads();
    // Epilogue: finalise the last generation of multi-block instances and
    // write resident units back.
    for (int u = u0; u < u1; ++u) {
        const UnitDev un = p.units[u];
        const InstDev& in = p.inst[un.inst];
        const View<Pos> v = make_view<Pos>(in, un, smem);
        if (in.R > 1 && warp == 0) {
            Pos* gs = reinterpret_cast<Pos*>(smem + un.smem_off);
            // pipelined blocks lag their counters by one generation: the last
            // one is logged here, after step A of the last generation
            const bool lag = F32R && un.pipelined != 0;
            step_a<Pos, F32R>(p, in, un, v, u - u0, gs, p.g_end, true, sh, lag);
            __syncwarp();
            if (lag && un.rank == 0 && !sh.flag && !fill_counts(p, in, un, p.g_end, sh.lag_r2) && lane == 0)
                sh.flag = 1;
        }
        __syncthreads();
        if (sh.flag) return;
        if (un.resident) move_resident<Pos, F32R>(in, un, smem, false);
        __syncthreads();
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
    const double f = fit64_row<Pos>(hot_of(in), static_cast<const Pos*>(in.gbrow), true);
    if (threadIdx.x == 0) {
        in.gb->f64 = f;
        in.gb->has64 = 1;
    }
}

template <class Pos, bool F32R, int MC>
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
    return cudaLaunchKernelEx(&lc, sso_generations<Pos, F32R, MC>, p);
}

template <class Pos, bool F32R, int MC>
inline cudaError_t occupancy_generations(int block, size_t smem, int* n)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, sso_generations<Pos, F32R, MC>, block, smem);
}

template <class Pos, bool F32R, int MC>
inline cudaError_t smem_generations(size_t smem)
{
    return cudaFuncSetAttribute(sso_generations<Pos, F32R, MC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1));
}

// One kernel variant: launch / occupancy / shared-memory entry points for the
// four chunk widths (index 0..3 = 1, 2, 4, 8 chunks per lane).
// Block-wide candidate reduction (every thread gets the result); sh holds one
// Cand per warp.
template <bool F32R>
__device__ inline Cand block_reduce_cand(Cand c, Cand* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1) c = cand_merge<F32R>(c, cand_shfl(c, off));
    if (lane == 0) sh[w] = c;
    __syncthreads();
    if (w == 0) {
        c = lane < nw ? sh[lane] : cand_none();
        for (int off = 16; off > 0; off >>= 1) c = cand_merge<F32R>(c, cand_shfl(c, off));
        if (lane == 0) sh[0] = c;
    }
    __syncthreads();
    const Cand out = sh[0];
    __syncthreads();
    return out;
}

// ---------------------------------------------------------------------------
// Batched throughput pipeline, step kernel: every particle of the class range
// by a group of G lanes -- the persistent kernel's Eq. 2.1 update, fitness
// and pBest commit, reading the instance's gBest row from global memory.
// Blocks per SM the step kernel is compiled for: narrow rows trade registers
// (some spilled to L1) for the warps that hide the row loads' latency.
template <int MC> struct BatBound { static constexpr int min_blocks = MC == 1 ? 4 : MC == 2 ? 3 : MC == 4 ? 2 : 1; };

template <class Pos, bool F32R, int MC>
__global__ void __launch_bounds__(256, BatBound<MC>::min_blocks) bat_step(const BatParams p)
{
    const int lane = threadIdx.x & 31;
    const int G = p.G;
    const int lane_g = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int64_t gpb = (int64_t)(blockDim.x / G);
    const int64_t g = *p.gen;
    // Each block walks one contiguous range of the class's particles, so a
    // group's consecutive particles are mostly of one instance: the class
    // entry is found by one binary search and then advanced linearly.
    const int64_t per_block = (p.total + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per_block;
    const int64_t b1 = min(p.total, b0 + per_block);
    int lo = -1;
    int64_t ent_end = 0;
    for (int64_t gid = b0 + threadIdx.x / G; gid < b1; gid += gpb) {
        // the class entry holding particle gid (first[] ascending)
        if (lo < 0 || gid >= ent_end) {
            if (lo >= 0 && lo + 1 < p.n_ids && gid < __ldg(p.first + lo + 2)) {
                ++lo;
            } else {
                int a = 0, z = p.n_ids - 1;
                while (a < z) {
                    const int mid = (a + z + 1) >> 1;
                    if (__ldg(p.first + mid) <= gid) a = mid;
                    else z = mid - 1;
                }
                lo = a;
            }
            ent_end = __ldg(p.first + lo + 1);
        }
        if (!PSSO_CHK(lo >= 0 && lo < p.n_ids, CHK_BAT_INST, gid)) break;
        const int k = __ldg(p.ids + lo);
        const int64_t i = gid - __ldg(p.first + lo);
        const InstDev& d = p.inst[k];
        const Hot in = hot_of(d);
        View<Pos> v;
        v.X = static_cast<Pos*>(d.X);
        v.P = static_cast<Pos*>(d.P);
        v.pf64 = d.pf64;
        v.plo = d.plo;
        v.phi = d.phi;
        v.pver = d.pver;
        v.pflag = d.pflag;
        v.base = 0;
        v.n = d.N;
        unsigned long long n_acc = 0, n_rck = 0;
        PartState<Pos, MC> st;
        particle_compute<Pos, F32R, MC>(in, v, static_cast<const Pos*>(d.gbrow), i, i, g, lane_g, gmask, st);
        particle_commit<Pos, F32R, MC>(in, v, i, g, lane_g, gmask, st, n_acc, n_rck);
        if (lane_g == 0 && (n_acc | n_rck)) {
            if (n_acc) atomicAdd(&p.cnt[k].acc, n_acc);
            if (n_rck) atomicAdd(&p.cnt[k].rck, n_rck);
        }
    }
}

template <class Pos, bool F32R, int MC>
inline cudaError_t bat_entry_mc(int op, const BatParams* p, int grid, int block, cudaStream_t s, int* out)
{
    if (op == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bat_step<Pos, F32R, MC>, block, 0);
    bat_step<Pos, F32R, MC><<<grid, block, 0, s>>>(*p);
    return cudaGetLastError();
}

template <class Pos, bool F32R, int MCV>
inline cudaError_t gen_entry_mc(int op, const KParams* p, int grid, int block, size_t smem, cudaStream_t s,
                                int* out)
{
    if (op == 0) return launch_generations<Pos, F32R, MCV>(*p, grid, block, smem, s);
    if (op == 1) return occupancy_generations<Pos, F32R, MCV>(block, smem, out);
    if (op == 2) return smem_generations<Pos, F32R, MCV>(smem);
    *out = GenBound<MCV>::threads;
    return cudaSuccess;
}

}  // namespace psso
