// psso_api.cu -- the C ABI declared in include/psso.h: argument checks, the
// launch planner, the device arena, and the host side of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "psso.h"
#include "psso_internal.h"
#include "rot_pipeline.h"
#include "tc_gemm.cuh"

using namespace psso;

namespace {

// NVTX range around an entry point, so that a profiler's timeline shows the
// host side of create / run / reset / sync / best (no effect without one).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

thread_local std::string g_last_error;

psso_status fail(psso_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

#define CUDA_TRY(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? PSSO_ERR_OOM : PSSO_ERR_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int pow2_ceil(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

float float_at_or_above(double v)
{
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

float float_at_or_below(double v)
{
    float f = (float)v;
    if ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

enum Variant { V_F64_LAT64 = 0, V_F64_LAT32 = 1, V_F32R = 2 };

struct HostInst {
    psso_problem pr;
    std::vector<double> o, w, M;
    int G = 0, maxc = 0, nchunks = 0, Dp = 0, R = 1;
    size_t off_X = 0, off_P = 0, off_pf64 = 0, off_plo = 0, off_phi = 0, off_pver = 0,
           off_pflag = 0, off_grow = 0, off_rec = 0, off_rec2 = 0, off_gb = 0, off_gbrow = 0,
           off_log = 0, off_o64 = 0, off_o32 = 0, off_w64 = 0, off_w32 = 0, off_M64 = 0, off_M32 = 0;
    int64_t i_base = 0;           // shard of a larger swarm: index of its first particle
    bool tc = false;              // generations run by the tensor-core pipeline
    bool bp = false;              // generations run by the batched throughput pipeline
    rot::RotHost rh{};
};

// The batched throughput pipeline of a handle.
struct BatHost {
    struct Class {
        int mc_index = 0, G = 32, grid = 0;
        bool stream = false;       // wide unrotated rows: the streaming kernel
        int32_t* ids = nullptr;
        int64_t* first = nullptr;
        int32_t n = 0;
        int64_t total = 0;
    };
    std::vector<Class> classes;
    int32_t* all_ids = nullptr;   // every batched instance (arg-min blocks)
    int32_t n_all = 0;
    BatCounters* cnt = nullptr;
    long long* gen = nullptr;
    void* mem = nullptr;
    cudaGraphExec_t graph1 = nullptr, graphG = nullptr;
    static constexpr int GRAPH_GENS = 16;
    // classes after the first run on side streams (parallel branches of the
    // captured graphs): they touch disjoint swarms
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};

}  // namespace

void psso::set_last_error(const char* msg) { g_last_error = msg; }

struct psso_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    psso_config cfg{};
    int precision = PSSO_PREC_F64;
    int lattice = PSSO_LATTICE_F64;
    int variant = V_F64_LAT64;
    int mc_index = 0;           // kernel width: up to 1, 2, 4, 8 chunks per lane
    size_t pos_size = 8;
    std::vector<HostInst> inst;
    BatHost bat;
    std::vector<UnitDev> units;
    std::vector<int32_t> block_first;
    int grid = 0, block = 256;
    size_t smem = 0;
    char* arena = nullptr;
    size_t arena_size = 0, state_off = 0;
    size_t off_instdev = 0, off_units = 0, off_block_first = 0, off_status = 0;
    int64_t gen = 0;
    int64_t evals = 0, updates = 0;
    int64_t h2d = 0, d2h = 0;
    int64_t launches = 0;       // kernels this handle enqueued (graph nodes included)
    bool failed = false;
    // asynchronous flow (Alg. 1): one cooperative kernel; its scratch and control words
    bool async = false;
    bool shard = false;           // created by psso_create_shard
    // tensor-pipeline swarms run on their own streams after the persistent
    // kernel in stream order (never beside it: its blocks wait on one another),
    // concurrently with one another and with the batched graphs
    std::vector<cudaStream_t> tc_side;
    std::vector<cudaEvent_t> tc_join;
    cudaEvent_t tc_fork = nullptr;
    void* amem = nullptr;
    AsyncCtl* actl = nullptr;
    void* axs = nullptr;
    double* afs = nullptr;
    int agrid = 0, ablock = 256;
};

namespace {

cudaError_t launch_variant(int v, int mc, const KParams& p, int grid, int block, size_t smem,
                           cudaStream_t s)
{
    return gen_call(v, 0, mc, &p, grid, block, smem, s, nullptr);
}

cudaError_t occupancy_of(int v, int mc, int block, size_t smem, int* n)
{
    return gen_call(v, 1, mc, nullptr, 0, block, smem, nullptr, n);
}

cudaError_t set_smem_of(int v, int mc, size_t smem)
{
    return gen_call(v, 2, mc, nullptr, 0, 0, smem, nullptr, nullptr);
}

psso_status check_problem(const psso_problem& pr, int precision, int idx)
{
    const std::string at = "problem " + std::to_string(idx) + ": ";
    if (pr.fn < PSSO_SPHERE || pr.fn > PSSO_SCHWEFEL) return fail(PSSO_ERR_ARG, at + "unknown function id");
    const bool rotated = pr.fn >= PSSO_ROT_ELLIPSOID && pr.fn <= PSSO_ROT_ACKLEY;
    if (rotated && !pr.rotation)
        return fail(PSSO_ERR_ARG, at + "rotated functions need a rotation matrix");
    if (pr.N < 1 || pr.N > 0x7fffffffLL) return fail(PSSO_ERR_ARG, at + "N must be in [1, 2^31-1]");
    if (pr.D < 1 || pr.D > 32 * MAX_CHUNKS_PER_LANE * 4) return fail(PSSO_ERR_ARG, at + "D must be in [1, 1024]");
    if (!std::isfinite(pr.lb) || !std::isfinite(pr.ub) || !(pr.lb < pr.ub))
        return fail(PSSO_ERR_ARG, at + "bounds must be finite with lb < ub");
    if (pr.order != PSSO_ORDER_GPX && pr.order != PSSO_ORDER_PAPER)
        return fail(PSSO_ERR_ARG, at + "unknown interval order");
    if (pr.order == PSSO_ORDER_GPX && !(0.0 <= pr.Cg && pr.Cg <= pr.Cp && pr.Cp <= pr.Cw && pr.Cw <= 1.0))
        return fail(PSSO_ERR_ARG, at + "need 0 <= Cg <= Cp <= Cw <= 1");
    if (pr.order == PSSO_ORDER_PAPER && !(0.0 <= pr.Cw && pr.Cw <= pr.Cp && pr.Cp <= pr.Cg && pr.Cg <= 1.0))
        return fail(PSSO_ERR_ARG, at + "the paper's interval order needs 0 <= Cw <= Cp <= Cg <= 1");
    if (pr.lattice != PSSO_LATTICE_F64 && pr.lattice != PSSO_LATTICE_F32)
        return fail(PSSO_ERR_ARG, at + "unknown lattice");
    if (pr.stream_id >= (1u << 24)) return fail(PSSO_ERR_ARG, at + "stream_id must be < 2^24");
    if ((pr.fn == PSSO_ELLIPSOID || pr.fn == PSSO_ROT_ELLIPSOID) && !pr.weights)
        return fail(PSSO_ERR_ARG, at + "ellipsoid functions need weights");
    if (pr.lattice == PSSO_LATTICE_F32 && !(float_at_or_above(pr.lb) <= float_at_or_below(pr.ub)))
        return fail(PSSO_ERR_ARG, at + "no float lies inside [lb, ub]");
    if (pr.shift)
        for (int64_t j = 0; j < pr.D; ++j)
            if (!std::isfinite(pr.shift[j])) return fail(PSSO_ERR_ARG, at + "shift must be finite");
    if (rotated)
        for (int64_t q = 0; q < pr.D * pr.D; ++q)
            if (!std::isfinite(pr.rotation[q])) return fail(PSSO_ERR_ARG, at + "rotation must be finite");
    if (precision == PSSO_PREC_F32_RECHECK) {
        if (pr.fn >= PSSO_SCHWEFEL12)
            return fail(PSSO_ERR_UNSUPPORTED, at + "Schwefel 1.2, Griewank, Powell and Schwefel run with FP64 fitness only");
        if (pr.lattice != PSSO_LATTICE_F32)
            return fail(PSSO_ERR_ARG, at + "F32_RECHECK precision needs the F32 lattice");
        if (pr.shift)
            for (int64_t j = 0; j < pr.D; ++j)
                if ((double)(float)pr.shift[j] != pr.shift[j])
                    return fail(PSSO_ERR_ARG, at + "F32_RECHECK precision needs a float-exact shift");
    }
    return PSSO_OK;
}

// Picks blocks per instance and assigns units to blocks.
psso_status plan(psso_ctx* h)
{
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, h->device));
    int TB = h->block;
    int nw = TB / 32;
    const int sbm = h->cfg.single_block_max == 0 ? 4 : (h->cfg.single_block_max < 0 ? 0 : h->cfg.single_block_max);
    size_t unit_smem_max = 0;
    double total_cost = 0.0;
    int n_kernel = 0, only = -1;           // instances the persistent kernel runs
    for (size_t k = 0; k < h->inst.size(); ++k) {
        HostInst& I = h->inst[k];
        I.nchunks = (int)((I.pr.D + 3) / 4);
        I.Dp = 4 * I.nchunks;
        I.G = std::min(32, pow2_ceil(I.nchunks));
        I.maxc = pow2_ceil((I.nchunks + 31) / 32);
        I.R = 1;
        if (I.tc || I.bp) continue;
        ++n_kernel;
        only = (int)k;
        unit_smem_max = std::max(unit_smem_max, align_up((size_t)I.Dp * h->pos_size, 16));
        total_cost += (double)I.pr.N * I.Dp;
        h->mc_index = std::max(h->mc_index, I.maxc >= 8 ? 3 : I.maxc >= 4 ? 2 : I.maxc >= 2 ? 1 : 0);
    }
    if (n_kernel == 0 || h->async) {        // every instance runs on the tensor-core pipeline,
                                            // or the handle runs the asynchronous flow
        h->grid = 0;
        h->units.clear();
        h->block_first.assign(1, 0);
        h->smem = 0;
        return PSSO_OK;
    }
    int max_threads = 0;
    CUDA_TRY(gen_call(h->variant, 3, h->mc_index, nullptr, 0, 0, 0, nullptr, &max_threads));
    if (h->block > max_threads) {
        if (h->cfg.threads_per_block != 0)
            return fail(PSSO_ERR_ARG, "threads_per_block above " + std::to_string(max_threads) +
                                          " for rows of this width");
        h->block = max_threads;
    }
    // One multi-block swarm: a control warp plus enough compute warps for one
    // particle per compute group and about one block per SM (pipelined blocks).
    bool pipe = false;
    if (n_kernel == 1 && h->cfg.pipeline != 2) {
        const HostInst& I = h->inst[only];
        const int gpw = 32 / I.G;
        const int64_t groups = (I.pr.N + gpw - 1) / gpw;
        const int64_t single_passes = (I.pr.N + (int64_t)nw * gpw - 1) / ((int64_t)nw * gpw);
        if (single_passes > sbm) {
            // at most 128 blocks: each lane of the control warp then polls <= 4
            // records, all in flight at once
            const int64_t blocks_cap = std::min<int64_t>(prop.multiProcessorCount, 128);
            int cw = (int)std::min<int64_t>((groups + blocks_cap - 1) / blocks_cap, max_threads / 32 - 1);
            if (h->cfg.threads_per_block != 0) cw = h->block / 32 - 1;
            if (cw >= 1) {
                pipe = true;
                h->block = 32 * (cw + 1);
            }
        }
    }
    TB = h->block;
    nw = TB / 32;
    // Occupancy with the largest single-unit footprint.
    int bps = 0;
    CUDA_TRY(occupancy_of(h->variant, h->mc_index, TB, unit_smem_max, &bps));
    if (bps < 1) return fail(PSSO_ERR_UNSUPPORTED, "kernel does not fit on one SM with this block size");
    int grid_max = bps * prop.multiProcessorCount;
    if (h->cfg.max_blocks > 0) grid_max = std::min(grid_max, h->cfg.max_blocks);

    for (int attempt = 0; attempt < 32; ++attempt) {
        // Blocks per instance, proportional to its work.
        std::vector<int> R(h->inst.size());
        int64_t sumR = 0;
        for (size_t k = 0; k < h->inst.size(); ++k) {
            const HostInst& I = h->inst[k];
            if (I.tc || I.bp) {
                R[k] = 1;               // no blocks of the persistent kernel
                continue;
            }
            const int ppp = (pipe ? nw - 1 : nw) * (32 / I.G);
            const int64_t passes = (I.pr.N + ppp - 1) / ppp;
            int64_t r = 1;
            if (pipe && passes > grid_max) {     // pipelined blocks must all be co-resident
                pipe = false;
                h->block = h->cfg.threads_per_block ? h->cfg.threads_per_block : std::min(256, max_threads);
                TB = h->block;
                nw = TB / 32;
                R.assign(h->inst.size(), 1);
                sumR = 0;
                k = (size_t)-1;                  // restart the loop with plain blocks
                continue;
            }
            if (pipe) {
                r = passes;
            } else if (passes > sbm) {
                r = (int64_t)std::floor((double)grid_max * ((double)I.pr.N * I.Dp) / total_cost);
                r = std::max<int64_t>(1, std::min<int64_t>(r, passes));
                r = std::min<int64_t>(r, grid_max);
            }
            R[k] = (int)r;
            sumR += r;
        }
        // Units: whole passes per block.
        std::vector<UnitDev> units;
        std::vector<double> cost;
        for (size_t k = 0; k < h->inst.size(); ++k) {
            HostInst& I = h->inst[k];
            I.R = R[k];
            if (I.tc || I.bp) continue;
            const int ppp = (pipe ? nw - 1 : nw) * (32 / I.G);
            const int64_t passes = (I.pr.N + ppp - 1) / ppp;
            for (int r = 0; r < R[k]; ++r) {
                UnitDev u{};
                u.inst = (int32_t)k;
                u.rank = r;
                u.i0 = std::min<int64_t>(I.pr.N, (passes * r / R[k]) * ppp);
                u.i1 = std::min<int64_t>(I.pr.N, (passes * (r + 1) / R[k]) * ppp);
                u.pipelined = (pipe && R[k] > 1) ? 1 : 0;
                units.push_back(u);
                cost.push_back((double)(u.i1 - u.i0) * I.Dp + 64.0 * I.Dp);
            }
        }
        // Pack units onto blocks (longest first onto the least loaded block).
        const int nblocks = (int)std::min<int64_t>(sumR, grid_max);
        std::vector<std::vector<int>> members(nblocks);
        std::vector<double> load(nblocks, 0.0);
        std::vector<int> order(units.size());
        for (size_t q = 0; q < units.size(); ++q) order[q] = (int)q;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        bool ok = true;
        for (int q : order) {
            int best = -1;
            for (int b = 0; b < nblocks; ++b)
                if ((int)members[b].size() < MAX_UNITS_PER_BLOCK && (best < 0 || load[b] < load[best])) best = b;
            if (best < 0) { ok = false; break; }
            members[best].push_back(q);
            load[best] += cost[q];
        }
        if (!ok) return fail(PSSO_ERR_UNSUPPORTED, "too many instances for one launch");
        // Shared memory: every unit keeps its gBest row there; units whose X, P
        // and pBest state also fit the per-block budget stay resident.
        const int per_sm = std::max(1, (nblocks + prop.multiProcessorCount - 1) / prop.multiProcessorCount);
        const size_t sm_total = (size_t)prop.sharedMemPerMultiprocessor;
        const size_t budget = std::min<size_t>((size_t)prop.sharedMemPerBlockOptin - 8192,
                                               sm_total / per_sm > 12288 ? sm_total / per_sm - 12288 : 0);
        h->units.clear();
        h->block_first.assign(1, 0);
        size_t smem = 0;
        for (int b = 0; b < nblocks; ++b) {
            std::sort(members[b].begin(), members[b].end(), [&](int a, int c) {
                return units[a].inst != units[c].inst ? units[a].inst < units[c].inst
                                                      : units[a].rank < units[c].rank;
            });
            size_t off = 0;
            for (int q : members[b]) off += align_up((size_t)h->inst[units[q].inst].Dp * h->pos_size, 16);
            for (int q : members[b]) {
                UnitDev u = units[q];
                const HostInst& I = h->inst[u.inst];
                const size_t rb = resident_bytes(u.i1 - u.i0, I.Dp, (int)h->pos_size);
                u.resident = (h->cfg.residency != 2 && off + rb <= budget) ? 1 : 0;
                u.res_off = u.resident ? (int32_t)off : 0;
                if (u.resident) off += rb;
                units[q] = u;
            }
            size_t goff = 0;
            for (int q : members[b]) {
                UnitDev u = units[q];
                u.smem_off = (int32_t)goff;
                goff += align_up((size_t)h->inst[u.inst].Dp * h->pos_size, 16);
                h->units.push_back(u);
            }
            smem = std::max(smem, off);
            h->block_first.push_back((int32_t)h->units.size());
        }
        if (smem > (size_t)prop.sharedMemPerBlockOptin - 8192)
            return fail(PSSO_ERR_UNSUPPORTED, "per-block gBest rows exceed shared memory");
        CUDA_TRY(set_smem_of(h->variant, h->mc_index, smem));
        int bps2 = 0;
        CUDA_TRY(occupancy_of(h->variant, h->mc_index, TB, smem, &bps2));
        if ((int64_t)bps2 * prop.multiProcessorCount >= nblocks) {
            h->grid = nblocks;
            h->smem = smem;
            return PSSO_OK;
        }
        if (pipe) {           // too many blocks to be co-resident: plain blocks instead
            pipe = false;
            h->block = h->cfg.threads_per_block ? h->cfg.threads_per_block : std::min(256, max_threads);
            TB = h->block;
            nw = TB / 32;
            continue;
        }
        grid_max = std::max(1, bps2 * prop.multiProcessorCount);
    }
    return fail(PSSO_ERR_UNSUPPORTED, "could not find a co-resident launch shape");
}

void fill_instdev(psso_ctx* h, std::vector<InstDev>& out)
{
    char* A = h->arena;
    out.resize(h->inst.size());
    for (size_t k = 0; k < h->inst.size(); ++k) {
        const HostInst& I = h->inst[k];
        InstDev d{};
        d.fn = I.pr.fn;
        d.D = (int32_t)I.pr.D;
        d.Dp = I.Dp;
        d.nchunks = I.nchunks;
        d.G = I.G;
        d.maxc = I.maxc;
        d.R = I.R;
        d.lattice = I.pr.lattice;
        d.N = I.pr.N;
        // thresholds of the first, second and third interval (Eq. 2.1)
        const bool paper_order = I.pr.order == PSSO_ORDER_PAPER;
        d.Tg = (uint64_t)std::nearbyint(std::ldexp(paper_order ? I.pr.Cw : I.pr.Cg, 32));
        d.Tp = (uint64_t)std::nearbyint(std::ldexp(I.pr.Cp, 32));
        d.Tw = (uint64_t)std::nearbyint(std::ldexp(paper_order ? I.pr.Cg : I.pr.Cw, 32));
        d.order = paper_order ? 1u : 0u;
        d.k0 = (uint32_t)I.pr.seed;
        d.k1 = (uint32_t)(I.pr.seed >> 32);
        d.sid = I.pr.stream_id;
        d.lb = I.pr.lb;
        d.ub = I.pr.ub;
        d.span = I.pr.ub - I.pr.lb;
        d.S32 = (float)(I.pr.ub - I.pr.lb);
        d.L32 = (float)I.pr.lb;
        d.lbf = float_at_or_above(I.pr.lb);
        d.ubf = float_at_or_below(I.pr.ub);
        d.o64 = reinterpret_cast<const double*>(A + I.off_o64);
        d.o32 = reinterpret_cast<const float*>(A + I.off_o32);
        d.w64 = I.w.empty() ? nullptr : reinterpret_cast<const double*>(A + I.off_w64);
        d.w32 = I.w.empty() ? nullptr : reinterpret_cast<const float*>(A + I.off_w32);
        d.M64 = I.M.empty() ? nullptr : reinterpret_cast<const double*>(A + I.off_M64);
        d.M32 = I.M.empty() ? nullptr : reinterpret_cast<const float*>(A + I.off_M32);
        d.M32lo = I.M.empty() ? nullptr : reinterpret_cast<const float*>(A + I.off_M32) + I.M.size();
        d.X = A + I.off_X;
        d.P = A + I.off_P;
        d.pf64 = reinterpret_cast<double*>(A + I.off_pf64);
        d.plo = reinterpret_cast<float*>(A + I.off_plo);
        d.phi = reinterpret_cast<float*>(A + I.off_phi);
        d.pver = reinterpret_cast<uint32_t*>(A + I.off_pver);
        d.pflag = reinterpret_cast<uint32_t*>(A + I.off_pflag);
        d.grow = A + I.off_grow;
        d.rec = reinterpret_cast<uint64_t*>(A + I.off_rec);
        d.rec2 = reinterpret_cast<uint64_t*>(A + I.off_rec2);
        d.gb = reinterpret_cast<GBestDev*>(A + I.off_gb);
        d.gbrow = A + I.off_gbrow;
        d.log = reinterpret_cast<LogDev*>(A + I.off_log);
        d.log_cap = h->cfg.log_stride > 0 ? h->cfg.log_capacity : 0;
        d.log_stride = h->cfg.log_stride;
        d.i_base = (uint32_t)I.i_base;
        out[k] = d;
    }
}

psso_status launch(psso_ctx* h, int64_t g_begin, int64_t g_end)
{
    if (h->async) {
        const HostInst& I = h->inst[0];
        AsyncParams a{};
        a.inst = reinterpret_cast<const InstDev*>(h->arena + h->off_instdev);
        a.status = reinterpret_cast<StatusDev*>(h->arena + h->off_status);
        a.ctl = h->actl;
        a.xs = h->axs;
        a.fs = h->afs;
        a.g_begin = g_begin;
        a.g_end = g_end;
        a.spin_limit = h->cfg.spin_limit > 0 ? h->cfg.spin_limit : (int64_t)50000000;
        const int mc = I.maxc >= 8 ? 3 : I.maxc >= 4 ? 2 : I.maxc >= 2 ? 1 : 0;
        CUDA_TRY(async_call((int)h->pos_size, mc, 0, &a, h->agrid, h->ablock, h->stream, nullptr));
        ++h->launches;
        return PSSO_OK;
    }
    KParams p{};
    p.inst = reinterpret_cast<const InstDev*>(h->arena + h->off_instdev);
    p.units = reinterpret_cast<const UnitDev*>(h->arena + h->off_units);
    p.block_first = reinterpret_cast<const int32_t*>(h->arena + h->off_block_first);
    p.status = reinterpret_cast<StatusDev*>(h->arena + h->off_status);
    p.g_begin = g_begin;
    p.g_end = g_end;
    p.spin_limit = h->cfg.spin_limit > 0 ? h->cfg.spin_limit : (int64_t)50000000;
    p.fault_skip_rank = h->cfg.fault_skip_rank;
    if (h->grid > 0) {
        CUDA_TRY(launch_variant(h->variant, h->mc_index, p, h->grid, h->block, h->smem, h->stream));
        ++h->launches;
    }
    if (h->bat.n_all > 0) {
        CUDA_TRY(launch_bat_set_gen(h->bat.gen, g_begin, h->stream));
        int64_t count = g_end - g_begin + 1;
        for (; count >= BatHost::GRAPH_GENS; count -= BatHost::GRAPH_GENS)
            CUDA_TRY(cudaGraphLaunch(h->bat.graphG, h->stream));
        for (; count > 0; --count) CUDA_TRY(cudaGraphLaunch(h->bat.graph1, h->stream));
        h->launches += 1 + (int64_t)(h->bat.classes.size() + 2) * (g_end - g_begin + 1);
    }
    // tensor-pipeline swarms: forked after everything above in stream order,
    // one side stream each (the handle's stream when there is no side stream)
    const bool fork = !h->tc_side.empty();
    if (fork) CUDA_TRY(cudaEventRecord(h->tc_fork, h->stream));
    size_t j = 0;
    for (auto& I : h->inst) {
        if (!I.tc) continue;
        cudaStream_t st = fork ? h->tc_side[j] : h->stream;
        if (fork) CUDA_TRY(cudaStreamWaitEvent(st, h->tc_fork, 0));
        CUDA_TRY(rot::set_generation(I.rh, g_begin, st));
        CUDA_TRY(rot::run_generations(I.rh, g_end - g_begin + 1, st));
        if (fork) CUDA_TRY(cudaEventRecord(h->tc_join[j], st));
        h->launches += 1 + rot::KERNELS_PER_GENERATION * (g_end - g_begin + 1);
        ++j;
    }
    for (size_t q = 0; fork && q < h->tc_join.size(); ++q) CUDA_TRY(cudaStreamWaitEvent(h->stream, h->tc_join[q], 0));
    return PSSO_OK;
}

// Side streams of the tensor-pipeline swarms: one per swarm when there are
// two or more of them (released by psso_destroy).
psso_status setup_tc_streams(psso_ctx* h)
{
    size_t n = 0;
    for (const auto& I : h->inst) n += I.tc ? 1 : 0;
    if (n < 2) return PSSO_OK;
    CUDA_TRY(cudaEventCreateWithFlags(&h->tc_fork, cudaEventDisableTiming));
    for (size_t q = 0; q < n; ++q) {
        cudaStream_t st = nullptr;
        cudaEvent_t je = nullptr;
        CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        h->tc_side.push_back(st);
        CUDA_TRY(cudaEventCreateWithFlags(&je, cudaEventDisableTiming));
        h->tc_join.push_back(je);
    }
    return PSSO_OK;
}

// Buffers, tensor maps and constant operand planes of a tensor-pipeline instance.
psso_status setup_tc(psso_ctx* h, size_t k)
{
    HostInst& I = h->inst[k];
    rot::RotHost& R = I.rh;
    rot::RotDev& r = R.dev;
    const int64_t N = I.pr.N;
    const int D = (int)I.pr.D;
    r.fn = I.pr.fn;
    r.D = D;
    r.N = N;
    r.Np = (int)((N + tc::BM - 1) / tc::BM * tc::BM);
    r.Jp = (D + tc::SBN - 1) / tc::SBN * tc::SBN;
    r.Kp = (D + tc::BK - 1) / tc::BK * tc::BK;
    r.nJt = r.Jp / tc::SBN;
    if (r.Kp > tc::S_MAX_K || D > tc::S_MAX_D)
        return fail(PSSO_ERR_UNSUPPORTED, "tensor pipeline: D above the slice GEMM's exact range");
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t oA = take((size_t)tc::SLICES * r.Np * r.Kp * 2), oB = take((size_t)tc::SLICES * r.Jp * r.Kp * 2),
                 oms = take((size_t)r.Jp * 4), oml1 = take((size_t)r.Jp * 4), ods = take((size_t)r.Np * 4),
                 odl1 = take((size_t)r.Np * 4), osame = take((size_t)N * 4),
                 opart = take((size_t)N * r.nJt * 16), ol1 = take((size_t)N * 4), ol2 = take((size_t)N * 4),
                 oz = take((size_t)2 * N * I.Dp * 8), oz0 = take((size_t)I.Dp * 8),
                 octl = take(sizeof(rot::RotCtl)), ol3 = take((size_t)N * 4),
                 omh = take((size_t)D * D * 4), oml = take((size_t)D * D * 4),
                 oz32 = take((size_t)2 * N * I.Dp * 4), oez = take((size_t)2 * N * I.Dp * 4);
    R.mem_bytes = align_up(off, 256);
    CUDA_TRY(cudaMalloc(&R.mem, R.mem_bytes));
    CUDA_TRY(cudaMemsetAsync(R.mem, 0, R.mem_bytes, h->stream));
    char* b = static_cast<char*>(R.mem);
    r.A = reinterpret_cast<__nv_bfloat16*>(b + oA);
    R.B = reinterpret_cast<__nv_bfloat16*>(b + oB);
    r.mscale = reinterpret_cast<float*>(b + oms);
    r.ml1 = reinterpret_cast<float*>(b + oml1);
    r.dscale = reinterpret_cast<float*>(b + ods);
    r.dl1 = reinterpret_cast<float*>(b + odl1);
    r.same = reinterpret_cast<uint32_t*>(b + osame);
    r.part = reinterpret_cast<float4*>(b + opart);
    r.list1 = reinterpret_cast<int32_t*>(b + ol1);
    r.list2 = reinterpret_cast<int32_t*>(b + ol2);
    r.zbuf = reinterpret_cast<double*>(b + oz);
    r.zero64 = reinterpret_cast<const double*>(b + oz0);
    r.ctl = reinterpret_cast<rot::RotCtl*>(b + octl);
    r.list3 = reinterpret_cast<int32_t*>(b + ol3);
    R.Mh = reinterpret_cast<float*>(b + omh);
    R.Ml = reinterpret_cast<float*>(b + oml);
    r.Mh = R.Mh;
    r.Ml = R.Ml;
    r.z32 = reinterpret_cast<float*>(b + oz32);
    r.ez32 = reinterpret_cast<float*>(b + oez);
    R.M64 = reinterpret_cast<const double*>(h->arena + I.off_M64);
    r.inst = reinterpret_cast<const InstDev*>(h->arena + h->off_instdev) + k;
    r.inst_w32 = I.w.empty() ? nullptr : reinterpret_cast<const float*>(h->arena + I.off_w32);
    R.M32 = reinterpret_cast<const float*>(h->arena + I.off_M32);
    R.N = N;
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, h->device));
    R.z64_grid = 2 * prop.multiProcessorCount;
    R.z32_grid = 8 * prop.multiProcessorCount;
    R.fix_grid = prop.multiProcessorCount;
    R.gemm_grid = (int)std::min<long long>((long long)(r.Np / tc::BM) * r.nJt, prop.multiProcessorCount);
    if (!tc::make_tmap_bf16(&R.tmA, r.A, r.Kp, tc::SLICES * r.Np) ||
        !tc::make_tmap_bf16(&R.tmB, R.B, r.Kp, tc::SLICES * r.Jp, tc::SBN))
        return fail(PSSO_ERR_CUDA, "cuTensorMapEncodeTiled failed for the tensor-core operands");
    CUDA_TRY(rot::configure());
    CUDA_TRY(rot::build_constants(R, h->stream));
    CUDA_TRY(rot::make_graphs(R));
    return PSSO_OK;
}

// With ev (classes + 2 events), an event is recorded before the first kernel
// and after each kernel (one step kernel per class, then the arg-min).
cudaError_t enqueue_bat_generation(psso_ctx* h, cudaStream_t s, cudaEvent_t* ev = nullptr)
{
    const InstDev* inst = reinterpret_cast<const InstDev*>(h->arena + h->off_instdev);
    BatHost& B = h->bat;
    auto step = [&](const BatHost::Class& c, cudaStream_t st) {
        BatParams p{inst, c.ids, c.first, c.n, c.G, c.total, B.gen, B.cnt};
        return c.stream ? bat_call(h->variant, 3, 2, &p, c.grid, 256, st, nullptr)
                        : bat_call(h->variant, c.mc_index, 0, &p, c.grid, 256, st, nullptr);
    };
    int q = 0;
    if (ev) cudaEventRecord(ev[q++], s);
    // With per-kernel events (psso_time_kernels) the classes run one after another.
    const bool branch = !ev && B.side.size() + 1 == B.classes.size() && B.classes.size() > 1;
    cudaError_t e = cudaSuccess;
    if (branch) e = cudaEventRecord(B.fork, s);
    for (size_t k = 0; k < B.classes.size() && e == cudaSuccess; ++k) {
        cudaStream_t st = s;
        if (branch && k > 0) {
            st = B.side[k - 1];
            e = cudaStreamWaitEvent(st, B.fork, 0);
            if (e != cudaSuccess) break;
        }
        e = step(B.classes[k], st);
        if (e == cudaSuccess && branch && k > 0) e = cudaEventRecord(B.join[k - 1], st);
        if (ev) cudaEventRecord(ev[q++], s);
    }
    for (size_t k = 0; branch && k + 1 < B.classes.size() && e == cudaSuccess; ++k)
        e = cudaStreamWaitEvent(s, B.join[k], 0);
    if (e != cudaSuccess) return e;
    e = launch_bat_argmin(h->variant, inst, B.all_ids, B.n_all, B.gen, B.cnt, s);
    if (ev) cudaEventRecord(ev[q++], s);
    return e;
}

// Classes of equal (lane-group width, chunks per lane), their device tables,
// grid sizes from the occupancy of each step kernel, and the captured graphs.
psso_status setup_bat(psso_ctx* h)
{
    BatHost& B = h->bat;
    std::vector<std::vector<int32_t>> members;
    std::vector<std::pair<int, int>> keys;   // (mc_index, G); mc_index 4 = streaming kernel
    std::vector<int32_t> all;
    for (size_t k = 0; k < h->inst.size(); ++k) {
        const HostInst& I = h->inst[k];
        if (!I.bp) continue;
        int mci = I.maxc >= 8 ? 3 : I.maxc >= 4 ? 2 : I.maxc >= 2 ? 1 : 0;
        // Unrotated rows over 128 variables (one particle per warp) run on the
        // streaming kernel: it holds one 32-chunk slice in registers instead
        // of the whole row, so more warps fit on an SM.
        if (mci >= 1 && I.pr.fn < PSSO_ROT_ELLIPSOID) mci = 4;
        const std::pair<int, int> key(mci, I.G);
        size_t c = 0;
        while (c < keys.size() && keys[c] != key) ++c;
        if (c == keys.size()) {
            keys.push_back(key);
            members.emplace_back();
        }
        members[c].push_back((int32_t)k);
        all.push_back((int32_t)k);
    }
    B.n_all = (int32_t)all.size();
    if (B.n_all == 0) return PSSO_OK;
    size_t bytes = 0;
    auto take = [&](size_t n) {
        bytes = align_up(bytes, 256);
        const size_t at = bytes;
        bytes += n;
        return at;
    };
    std::vector<size_t> oid(keys.size()), ofirst(keys.size());
    for (size_t c = 0; c < keys.size(); ++c) {
        oid[c] = take(members[c].size() * 4);
        ofirst[c] = take((members[c].size() + 1) * 8);
    }
    const size_t oall = take(all.size() * 4), ocnt = take(h->inst.size() * sizeof(BatCounters)),
                 ogen = take(sizeof(long long));
    CUDA_TRY(cudaMalloc(&B.mem, bytes));
    std::vector<char> host(bytes, 0);
    char* base = static_cast<char*>(B.mem);
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, h->device));
    for (size_t c = 0; c < keys.size(); ++c) {
        BatHost::Class cl;
        cl.stream = keys[c].first == 4;
        cl.mc_index = cl.stream ? 3 : keys[c].first;
        cl.G = keys[c].second;
        cl.n = (int32_t)members[c].size();
        std::vector<int64_t> first(members[c].size() + 1, 0);
        for (size_t q = 0; q < members[c].size(); ++q) first[q + 1] = first[q] + h->inst[members[c][q]].pr.N;
        cl.total = first.back();
        std::memcpy(host.data() + oid[c], members[c].data(), members[c].size() * 4);
        std::memcpy(host.data() + ofirst[c], first.data(), first.size() * 8);
        cl.ids = reinterpret_cast<int32_t*>(base + oid[c]);
        cl.first = reinterpret_cast<int64_t*>(base + ofirst[c]);
        int bps = 0;
        CUDA_TRY(bat_call(h->variant, cl.mc_index, cl.stream ? 3 : 1, nullptr, 0, 256, nullptr, &bps));
        if (h->cfg.batch_blocks_per_sm > 0) bps = std::min(bps, (int)h->cfg.batch_blocks_per_sm);
        const int64_t groups_per_block = cl.stream ? 8 : 256 / cl.G;
        const int64_t need = (cl.total + groups_per_block - 1) / groups_per_block;
        cl.grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(1, bps) * prop.multiProcessorCount));
        B.classes.push_back(cl);
    }
    std::memcpy(host.data() + oall, all.data(), all.size() * 4);
    B.all_ids = reinterpret_cast<int32_t*>(base + oall);
    B.cnt = reinterpret_cast<BatCounters*>(base + ocnt);
    B.gen = reinterpret_cast<long long*>(base + ogen);
    CUDA_TRY(cudaMemcpy(B.mem, host.data(), bytes, cudaMemcpyHostToDevice));
    h->h2d += (int64_t)bytes;
    // side streams of the classes after the first (released by psso_destroy)
    if (B.classes.size() > 1) {
        CUDA_TRY(cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming));
        for (size_t k = 1; k < B.classes.size(); ++k) {
            cudaStream_t st = nullptr;
            cudaEvent_t je = nullptr;
            CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            B.side.push_back(st);
            CUDA_TRY(cudaEventCreateWithFlags(&je, cudaEventDisableTiming));
            B.join.push_back(je);
        }
    }
    // graphs of 1 and GRAPH_GENS generations, captured on a private stream
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaSuccess;
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        const int gens = which == 0 ? 1 : BatHost::GRAPH_GENS;
        cudaGraph_t gr = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int q = 0; q < gens && e == cudaSuccess; ++q) e = enqueue_bat_generation(h, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(which == 0 ? &B.graph1 : &B.graphG, gr, 0);
        if (gr) cudaGraphDestroy(gr);
    }
    cudaStreamDestroy(cs);
    CUDA_TRY(e);
    return PSSO_OK;
}

// The asynchronous flow's scratch (searched rows and their fitness) and
// control words, and its grid: co-resident blocks, no more than the
// particles need.
psso_status setup_async(psso_ctx* h)
{
    if (!h->async) return PSSO_OK;
    const HostInst& I = h->inst[0];
    const size_t N = (size_t)I.pr.N, row = (size_t)I.Dp * h->pos_size;
    const size_t ctl = align_up(sizeof(AsyncCtl), 256), xs = align_up(N * row, 256);
    cudaError_t e = cudaMalloc(&h->amem, ctl + xs + N * 8);
    if (e != cudaSuccess) {
        h->amem = nullptr;
        return fail(PSSO_ERR_OOM, std::string("cudaMalloc of the asynchronous flow's scratch: ") +
                                      cudaGetErrorString(e));
    }
    h->actl = static_cast<AsyncCtl*>(h->amem);
    h->axs = static_cast<char*>(h->amem) + ctl;
    h->afs = reinterpret_cast<double*>(static_cast<char*>(h->amem) + ctl + xs);
    CUDA_TRY(cudaMemsetAsync(h->amem, 0, ctl, h->stream));
    const int mc = I.maxc >= 8 ? 3 : I.maxc >= 4 ? 2 : I.maxc >= 2 ? 1 : 0;
    int per_sm = 0, sms = 0;
    CUDA_TRY(async_call((int)h->pos_size, mc, 1, nullptr, 0, h->ablock, nullptr, &per_sm));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    if (per_sm < 1) return fail(PSSO_ERR_UNSUPPORTED, "the asynchronous kernel does not fit an SM");
    const int64_t groups_per_block = (int64_t)(h->ablock / 32) * (32 / I.G);
    const int64_t need = ((int64_t)I.pr.N + groups_per_block - 1) / groups_per_block;
    h->agrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, need));
    return PSSO_OK;
}

psso_status read_status(psso_ctx* h)
{
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    StatusDev st;
    CUDA_TRY(cudaMemcpy(&st, h->arena + h->off_status, sizeof st, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < h->inst.size(); ++k) {
        if (!h->inst[k].tc) continue;
        int tst = 0;
        CUDA_TRY(cudaMemcpy(&tst, &h->inst[k].rh.dev.ctl->status, sizeof tst, cudaMemcpyDeviceToHost));
        if (tst) {
            h->failed = true;
            return fail(PSSO_ERR_TIMEOUT, "a tensor-core pipeline wait ran out (instance " + std::to_string(k) + ")");
        }
    }
    if (st.err != 0) {
        h->failed = true;
        return fail((psso_status)st.err, "a cross-block wait ran out (instance " +
                                             std::to_string(st.where >> 16) + ", block rank " +
                                             std::to_string(st.where & 0xffff) + ")");
    }
    return PSSO_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
#ifdef PSSO_CHECKED
namespace {
std::vector<chk::Reader>& checked_readers()
{
    static std::vector<chk::Reader> v;   // filled while the library loads (static initialisers)
    return v;
}
// A failed check with no memory access: proves the record and report path.
__global__ void check_selftest_kernel(long long index) { (void)PSSO_CHK(false, CHK_SELFTEST, index); }
}  // namespace
void psso::chk::add_reader(Reader r) { checked_readers().push_back(r); }
#endif

extern "C" {

const char* psso_last_error(void) { return g_last_error.c_str(); }

psso_status create_impl(const psso_problem* problems, int32_t count, const psso_config* cfg, int64_t i_base,
                        psso_handle* out);

psso_status psso_create_ex(const psso_problem* problems, int32_t count, const psso_config* cfg,
                           psso_handle* out)
{
    return create_impl(problems, count, cfg, 0, out);
}

psso_status psso_create_shard(const psso_problem* problem, int64_t first, int64_t count, const psso_config* cfg,
                              psso_handle* out)
{
    if (!out) return fail(PSSO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!problem) return fail(PSSO_ERR_ARG, "problem is NULL");
    if (first < 0 || count < 1 || first + count > problem->N || first + count > 0xffffffffLL)
        return fail(PSSO_ERR_ARG, "psso_create_shard: need 0 <= first, 1 <= count, first + count <= N");
    psso_config c{};
    if (cfg) c = *cfg;
    if (c.flow != PSSO_FLOW_SYNC)
        return fail(PSSO_ERR_UNSUPPORTED, "psso_create_shard: the asynchronous flow cannot be split");
    // the whole shard in one block: its gBest row is restored from the handle's
    // gBest state at every launch, where psso_set_gbest puts the swarm's
    c.single_block_max = 0x3fffffff;
    psso_problem pr = *problem;
    pr.N = count;
    const psso_status st = create_impl(&pr, 1, &c, first, out);
    if (st == PSSO_OK) (*out)->shard = true;
    return st;
}

psso_status create_impl(const psso_problem* problems, int32_t count, const psso_config* cfg, int64_t i_base,
                        psso_handle* out)
{
    const Range range("psso_create_ex");
    if (!out) return fail(PSSO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!problems || count < 1 || count > 65536) return fail(PSSO_ERR_ARG, "need 1..65536 problems");
    psso_config c{};
    if (cfg) c = *cfg;
    if (c.precision != PSSO_PREC_F64 && c.precision != PSSO_PREC_F32_RECHECK)
        return fail(PSSO_ERR_ARG, "unknown precision");
    if (c.threads_per_block != 0 &&
        (c.threads_per_block < 64 || c.threads_per_block > 512 || c.threads_per_block % 32))
        return fail(PSSO_ERR_ARG, "threads_per_block must be a multiple of 32 in [64, 512]");
    if (c.log_stride < 0 || c.log_capacity < 0) return fail(PSSO_ERR_ARG, "negative log settings");
    if (c.log_stride > 0 && c.log_capacity == 0) return fail(PSSO_ERR_ARG, "log_capacity must be > 0");
    if (c.fault_skip_rank < 0) return fail(PSSO_ERR_ARG, "fault_skip_rank must be >= 0");
    if (c.residency != 0 && c.residency != 2) return fail(PSSO_ERR_ARG, "residency must be 0 or 2");
    if (c.pipeline != 0 && c.pipeline != 2) return fail(PSSO_ERR_ARG, "pipeline must be 0 or 2");
    if (c.tensor_rotation < -1 || c.tensor_rotation > 1) return fail(PSSO_ERR_ARG, "tensor_rotation must be -1, 0 or 1");
    if (c.batch_stream < -1 || c.batch_stream > 1) return fail(PSSO_ERR_ARG, "batch_stream must be -1, 0 or 1");
    if (c.batch_blocks_per_sm < 0 || c.batch_blocks_per_sm > 64)
        return fail(PSSO_ERR_ARG, "batch_blocks_per_sm must be in [0, 64]");
    if (c.flow != PSSO_FLOW_SYNC && c.flow != PSSO_FLOW_ASYNC) return fail(PSSO_ERR_ARG, "unknown flow");
    if (c.flow == PSSO_FLOW_ASYNC && (count != 1 || c.precision != PSSO_PREC_F64))
        return fail(PSSO_ERR_UNSUPPORTED, "the asynchronous flow runs one instance with PSSO_PREC_F64");
    for (int32_t k = 0; k < count; ++k) {
        psso_status st = check_problem(problems[k], c.precision, k);
        if (st != PSSO_OK) return st;
        if (problems[k].lattice != problems[0].lattice)
            return fail(PSSO_ERR_ARG, "all problems must share one lattice");
    }

    psso_ctx* h = new psso_ctx();
    h->cfg = c;
    h->precision = c.precision;
    h->lattice = problems[0].lattice;
    h->variant = c.precision == PSSO_PREC_F32_RECHECK ? V_F32R
                 : (h->lattice == PSSO_LATTICE_F32 ? V_F64_LAT32 : V_F64_LAT64);
    h->pos_size = h->lattice == PSSO_LATTICE_F32 ? 4 : 8;
    h->block = c.threads_per_block ? c.threads_per_block : 256;
    h->stream = static_cast<cudaStream_t>(c.stream);
    h->async = c.flow == PSSO_FLOW_ASYNC;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return fail(PSSO_ERR_CUDA, "no CUDA device");
    }
    h->inst.resize(count);
    for (int32_t k = 0; k < count; ++k) {
        HostInst& I = h->inst[k];
        I.pr = problems[k];
        I.i_base = i_base;
        I.o.assign((size_t)I.pr.D, 0.0);
        if (I.pr.shift) std::copy(I.pr.shift, I.pr.shift + I.pr.D, I.o.begin());
        if (I.pr.weights) I.w.assign(I.pr.weights, I.pr.weights + I.pr.D);
        if (I.pr.fn == PSSO_HYPER_ELLIPSOID) {   // Table 3.2 f2: the ellipsoid with w_j = j + 1
            I.pr.fn = PSSO_ELLIPSOID;
            I.w.resize((size_t)I.pr.D);
            for (int64_t j = 0; j < I.pr.D; ++j) I.w[(size_t)j] = (double)(j + 1);
        }
        const bool rot = I.pr.fn >= PSSO_ROT_ELLIPSOID && I.pr.fn <= PSSO_ROT_ACKLEY;
        if (rot) I.M.assign(I.pr.rotation, I.pr.rotation + I.pr.D * I.pr.D);
        I.pr.shift = I.pr.weights = I.pr.rotation = nullptr;
        I.tc = h->precision == PSSO_PREC_F32_RECHECK && rot &&
               (c.tensor_rotation == 1 ||
                (c.tensor_rotation == 0 && I.pr.N >= 128 && I.pr.D >= 32 && I.pr.D <= tc::S_MAX_D));
    }
    {
        int n_plain = 0;
        for (const auto& I : h->inst) n_plain += I.tc ? 0 : 1;
        const bool bat = !h->async && (c.batch_stream == 1 || (c.batch_stream == 0 && n_plain >= 16));
        for (auto& I : h->inst) I.bp = bat && !I.tc;
    }
    psso_status st = plan(h);
    if (st != PSSO_OK) {
        delete h;
        return st;
    }

    // Arena: descriptors first, then per-instance state (saved by psso_save).
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    h->off_instdev = take(sizeof(InstDev) * h->inst.size());
    h->off_units = take(sizeof(UnitDev) * h->units.size());
    h->off_block_first = take(sizeof(int32_t) * h->block_first.size());
    h->off_status = take(sizeof(StatusDev));
    h->state_off = align_up(off, 256);
    const bool f32r = h->precision == PSSO_PREC_F32_RECHECK;
    const size_t logcap = c.log_stride > 0 ? (size_t)c.log_capacity : 0;
    for (auto& I : h->inst) {
        const size_t N = (size_t)I.pr.N, row = (size_t)I.Dp * h->pos_size;
        I.off_X = take(N * row);
        I.off_P = take(N * row);
        I.off_pf64 = take(N * 8);
        I.off_plo = take(f32r ? N * 4 : 0);
        I.off_phi = take(f32r ? N * 4 : 0);
        I.off_pver = take(N * 4);
        I.off_pflag = take(f32r ? N * 4 : 0);
        I.off_grow = take(SLOTS * (size_t)I.R * I.Dp * (h->pos_size / 4) * 8);   // tagged words
        I.off_rec = take(SLOTS * (size_t)I.R * REC_WORDS * 8);
        I.off_rec2 = take(SLOTS * (size_t)I.R * REC_WORDS * 8);
        I.off_gb = take(sizeof(GBestDev));
        I.off_gbrow = take(row);
        I.off_log = take(logcap * sizeof(LogDev));
        I.off_o64 = take((size_t)I.Dp * 8);
        I.off_o32 = take((size_t)I.Dp * 4);
        I.off_w64 = take(I.w.empty() ? 0 : (size_t)I.Dp * 8);
        I.off_w32 = take(I.w.empty() ? 0 : (size_t)I.Dp * 4);
        I.off_M64 = take(I.M.size() * 8);
        I.off_M32 = take(I.M.size() * 8);   // float(M), then float(M - float(M))
    }
    h->arena_size = align_up(off, 256);
    cudaError_t e = cudaMalloc(&h->arena, h->arena_size);
    if (e != cudaSuccess) {
        delete h;
        return fail(PSSO_ERR_OOM, std::string("cudaMalloc of the state arena: ") + cudaGetErrorString(e));
    }
    auto cleanup_fail = [&](psso_status s2) {
        psso_destroy(h);
        return s2;
    };
    // Zero the arena, mark records / log as empty, then upload descriptors and data.
    std::vector<InstDev> instdev;
    fill_instdev(h, instdev);
    const size_t desc = h->state_off;
    std::vector<char> host(desc, 0);
    std::memcpy(host.data() + h->off_instdev, instdev.data(), sizeof(InstDev) * instdev.size());
    std::memcpy(host.data() + h->off_units, h->units.data(), sizeof(UnitDev) * h->units.size());
    std::memcpy(host.data() + h->off_block_first, h->block_first.data(),
                sizeof(int32_t) * h->block_first.size());
    e = cudaMemsetAsync(h->arena, 0, h->arena_size, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->arena, host.data(), desc, cudaMemcpyHostToDevice, h->stream);
    h->h2d += (int64_t)desc;
    std::vector<std::vector<char>> staging;   // kept alive until the stream sync below
    for (auto& I : h->inst) {
        if (e != cudaSuccess) break;
        const size_t rb = SLOTS * (size_t)I.R * REC_WORDS * 8;
        e = cudaMemsetAsync(h->arena + I.off_rec, 0xff, rb, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->arena + I.off_rec2, 0xff, rb, h->stream);
        if (e == cudaSuccess && logcap)
            e = cudaMemsetAsync(h->arena + I.off_log, 0xff, logcap * sizeof(LogDev), h->stream);
        const size_t nd = (size_t)I.pr.D;
        const bool hw = !I.w.empty();
        staging.emplace_back(nd * (hw ? 24 : 12));
        char* b = staging.back().data();
        double* o64 = reinterpret_cast<double*>(b);
        float* o32 = reinterpret_cast<float*>(b + nd * 8);
        for (size_t j = 0; j < nd; ++j) {
            o64[j] = I.o[j];
            o32[j] = (float)I.o[j];
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->arena + I.off_o64, o64, nd * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->arena + I.off_o32, o32, nd * 4, cudaMemcpyHostToDevice, h->stream);
        h->h2d += (int64_t)(nd * 12);
        if (hw) {
            double* w64 = reinterpret_cast<double*>(b + nd * 12);
            float* w32 = reinterpret_cast<float*>(b + nd * 20);
            for (size_t j = 0; j < nd; ++j) {
                w64[j] = I.w[j];
                w32[j] = (float)I.w[j];
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->arena + I.off_w64, w64, nd * 8, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->arena + I.off_w32, w32, nd * 4, cudaMemcpyHostToDevice, h->stream);
            h->h2d += (int64_t)(nd * 12);
        }
        if (!I.M.empty()) {
            staging.emplace_back(I.M.size() * 8);
            float* m32 = reinterpret_cast<float*>(staging.back().data());
            for (size_t q = 0; q < I.M.size(); ++q) {
                m32[q] = (float)I.M[q];
                m32[I.M.size() + q] = (float)(I.M[q] - (double)m32[q]);
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->arena + I.off_M64, I.M.data(), I.M.size() * 8, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->arena + I.off_M32, m32, I.M.size() * 8, cudaMemcpyHostToDevice, h->stream);
            h->h2d += (int64_t)(I.M.size() * 16);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        fail(PSSO_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
        return cleanup_fail(PSSO_ERR_CUDA);
    }
    for (size_t k = 0; k < h->inst.size(); ++k) {
        if (!h->inst[k].tc) continue;
        st = setup_tc(h, k);
        if (st != PSSO_OK) return cleanup_fail(st);
    }
    st = setup_bat(h);
    if (st != PSSO_OK) return cleanup_fail(st);
    st = setup_async(h);
    if (st != PSSO_OK) return cleanup_fail(st);
    st = setup_tc_streams(h);
    if (st != PSSO_OK) return cleanup_fail(st);
    st = launch(h, 0, 0);
    if (st != PSSO_OK) return cleanup_fail(st);
    for (auto& I : h->inst) h->evals += I.pr.N;
    *out = h;
    return PSSO_OK;
}

psso_status psso_create(psso_fn fn, int64_t N, int64_t D, double lb, double ub, double Cg,
                        double Cp, double Cw, uint64_t seed, psso_handle* out)
{
    psso_problem pr{};
    pr.fn = fn;
    pr.lattice = PSSO_LATTICE_F64;
    pr.N = N;
    pr.D = D;
    pr.lb = lb;
    pr.ub = ub;
    pr.Cg = Cg;
    pr.Cp = Cp;
    pr.Cw = Cw;
    pr.seed = seed;
    std::vector<double> w;
    if ((fn == PSSO_ELLIPSOID || fn == PSSO_ROT_ELLIPSOID) && D >= 1 && D <= 1024) {
        w.resize((size_t)D);
        for (int64_t j = 0; j < D; ++j) w[j] = D == 1 ? 1.0 : std::pow(10.0, 6.0 * (double)j / (double)(D - 1));
        pr.weights = w.data();
    }
    return psso_create_ex(&pr, 1, nullptr, out);
}

psso_status psso_run(psso_handle h, int64_t generations)
{
    const Range range("psso_run");
    if (!h) return fail(PSSO_ERR_ARG, "handle is NULL");
    if (generations < 0) return fail(PSSO_ERR_ARG, "generations must be >= 0");
    if (h->failed) return fail(PSSO_ERR_STATE, "the handle failed earlier; destroy it or psso_load a state");
    if (generations == 0) return PSSO_OK;
    if (h->gen + generations > 0xfffffff0LL) return fail(PSSO_ERR_ARG, "generation counter would exceed 2^32");
    CUDA_TRY(cudaSetDevice(h->device));
    psso_status st = launch(h, h->gen + 1, h->gen + generations);
    if (st != PSSO_OK) return st;
    h->gen += generations;
    for (auto& I : h->inst) {
        h->evals += I.pr.N * generations;
        h->updates += I.pr.N * I.pr.D * generations;
    }
    return PSSO_OK;
}

psso_status psso_reset(psso_handle h)
{
    const Range range("psso_reset");
    if (!h) return fail(PSSO_ERR_ARG, "handle is NULL");
    CUDA_TRY(cudaSetDevice(h->device));
    const size_t logcap = h->cfg.log_stride > 0 ? (size_t)h->cfg.log_capacity : 0;
    for (const auto& I : h->inst) {
        const size_t rb = SLOTS * (size_t)I.R * REC_WORDS * 8;
        CUDA_TRY(cudaMemsetAsync(h->arena + I.off_rec, 0xff, rb, h->stream));
        CUDA_TRY(cudaMemsetAsync(h->arena + I.off_rec2, 0xff, rb, h->stream));
        if (logcap) CUDA_TRY(cudaMemsetAsync(h->arena + I.off_log, 0xff, logcap * sizeof(LogDev), h->stream));
        CUDA_TRY(cudaMemsetAsync(h->arena + I.off_gb, 0, sizeof(GBestDev), h->stream));
    }
    CUDA_TRY(cudaMemsetAsync(h->arena + h->off_status, 0, sizeof(StatusDev), h->stream));
    for (auto& I : h->inst)
        if (I.tc) CUDA_TRY(cudaMemsetAsync(&I.rh.dev.ctl->status, 0, sizeof(int), h->stream));
    if (h->actl) CUDA_TRY(cudaMemsetAsync(h->actl, 0, sizeof(AsyncCtl), h->stream));
    psso_status st = launch(h, 0, 0);
    if (st != PSSO_OK) return st;
    h->gen = 0;
    h->failed = false;
    h->evals = 0;
    h->updates = 0;
    for (const auto& I : h->inst) h->evals += I.pr.N;
    return PSSO_OK;
}

psso_status psso_sync(psso_handle h)
{
    const Range range("psso_sync");
    if (!h) return fail(PSSO_ERR_ARG, "handle is NULL");
    return read_status(h);
}

int64_t psso_generation(psso_handle h) { return h ? h->gen : -1; }

static psso_status copy_row(psso_ctx* h, const HostInst& I, size_t off, int64_t nrows, double* dst)
{
    const size_t row = (size_t)I.Dp * h->pos_size;
    std::vector<char> buf((size_t)nrows * row);
    CUDA_TRY(cudaMemcpy(buf.data(), h->arena + off, buf.size(), cudaMemcpyDeviceToHost));
    h->d2h += (int64_t)buf.size();
    for (int64_t i = 0; i < nrows; ++i)
        for (int64_t j = 0; j < I.pr.D; ++j)
            dst[i * I.pr.D + j] = h->pos_size == 8
                                      ? reinterpret_cast<const double*>(buf.data() + i * row)[j]
                                      : (double)reinterpret_cast<const float*>(buf.data() + i * row)[j];
    return PSSO_OK;
}

psso_status psso_best(psso_handle h, int32_t instance, double* value, int64_t* index, double* row)
{
    const Range range("psso_best");
    if (!h) return fail(PSSO_ERR_ARG, "handle is NULL");
    if (instance < 0 || instance >= (int32_t)h->inst.size()) return fail(PSSO_ERR_ARG, "instance out of range");
    psso_status st = read_status(h);
    if (st != PSSO_OK) return st;
    if (h->precision == PSSO_PREC_F32_RECHECK) {
        CUDA_TRY(launch_best_f64(reinterpret_cast<const InstDev*>(h->arena + h->off_instdev),
                                 (int)h->inst.size(), h->lattice, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    const HostInst& I = h->inst[instance];
    GBestDev gb;
    CUDA_TRY(cudaMemcpy(&gb, h->arena + I.off_gb, sizeof gb, cudaMemcpyDeviceToHost));
    h->d2h += (int64_t)sizeof gb;
    if (value) *value = gb.f64;
    if (index) *index = gb.idx;
    if (row) return copy_row(h, I, I.off_gbrow, 1, row);
    return PSSO_OK;
}

psso_status psso_set_gbest(psso_handle h, int32_t instance, double value, int64_t index, const double* row)
{
    if (!h || !row) return fail(PSSO_ERR_ARG, "handle or row is NULL");
    if (instance < 0 || instance >= (int32_t)h->inst.size()) return fail(PSSO_ERR_ARG, "instance out of range");
    if (!std::isfinite(value)) return fail(PSSO_ERR_ARG, "psso_set_gbest: value must be finite");
    if (h->failed) return fail(PSSO_ERR_STATE, "the handle failed earlier");
    const HostInst& I = h->inst[instance];
    if (h->async || (!I.tc && !I.bp && I.R != 1))
        return fail(PSSO_ERR_UNSUPPORTED,
                    "psso_set_gbest: the instance's gBest comes from a cross-block exchange or the "
                    "asynchronous flow (create it with psso_create_shard)");
    const size_t D = (size_t)I.pr.D;
    std::vector<char> buf((size_t)I.Dp * h->pos_size + sizeof(GBestDev), 0);
    for (size_t j = 0; j < D; ++j) {
        if (!(row[j] >= I.pr.lb && row[j] <= I.pr.ub))
            return fail(PSSO_ERR_ARG, "psso_set_gbest: the row must lie inside [lb, ub]");
        if (h->pos_size == 4) {
            const float f = (float)row[j];
            if ((double)f != row[j]) return fail(PSSO_ERR_ARG, "psso_set_gbest: F32 lattice rows hold floats");
            reinterpret_cast<float*>(buf.data())[j] = f;
        } else {
            reinterpret_cast<double*>(buf.data())[j] = row[j];
        }
    }
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    GBestDev gb;
    CUDA_TRY(cudaMemcpy(&gb, h->arena + I.off_gb, sizeof gb, cudaMemcpyDeviceToHost));
    gb.idx = index;
    gb.f64 = value;
    gb.has64 = 1;
    gb.lo = float_at_or_below(value);   // the largest float <= value
    gb.hi = float_at_or_above(value);
    gb.ver = 0xffffffffu;   // no local pBest row has this version: the row cache is refreshed
    CUDA_TRY(cudaMemcpy(h->arena + I.off_gbrow, buf.data(), (size_t)I.Dp * h->pos_size, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h->arena + I.off_gb, &gb, sizeof gb, cudaMemcpyHostToDevice));
    h->h2d += (int64_t)((size_t)I.Dp * h->pos_size + sizeof gb);
    return PSSO_OK;
}

psso_status psso_get_state(psso_handle h, int32_t instance, double* X, double* P, double* pF)
{
    if (!h) return fail(PSSO_ERR_ARG, "handle is NULL");
    if (instance < 0 || instance >= (int32_t)h->inst.size()) return fail(PSSO_ERR_ARG, "instance out of range");
    psso_status st = read_status(h);
    if (st != PSSO_OK) return st;
    const HostInst& I = h->inst[instance];
    if (X && (st = copy_row(h, I, I.off_X, I.pr.N, X)) != PSSO_OK) return st;
    if (P && (st = copy_row(h, I, I.off_P, I.pr.N, P)) != PSSO_OK) return st;
    if (pF && I.tc) {
        // the tensor-core pipeline keeps most pBest values as certified intervals;
        // those too wide for 1e-6 relative get their FP64 value before the read
        CUDA_TRY(rot::exact_values_for_read(I.rh, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    if (pF) {
        const size_t N = (size_t)I.pr.N;
        CUDA_TRY(cudaMemcpy(pF, h->arena + I.off_pf64, N * 8, cudaMemcpyDeviceToHost));
        if (h->precision == PSSO_PREC_F32_RECHECK) {
            std::vector<float> lo(N), hi(N);
            std::vector<uint32_t> flag(N);
            CUDA_TRY(cudaMemcpy(lo.data(), h->arena + I.off_plo, N * 4, cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(hi.data(), h->arena + I.off_phi, N * 4, cudaMemcpyDeviceToHost));
            CUDA_TRY(cudaMemcpy(flag.data(), h->arena + I.off_pflag, N * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < N; ++i)
                if (!(flag[i] & 1u)) pF[i] = 0.5 * ((double)lo[i] + (double)hi[i]);
        }
    }
    return PSSO_OK;
}

psso_status psso_get_log(psso_handle h, int32_t instance, psso_log_entry* buf, int64_t cap, int64_t* n)
{
    if (!h || !n) return fail(PSSO_ERR_ARG, "handle or n is NULL");
    if (instance < 0 || instance >= (int32_t)h->inst.size()) return fail(PSSO_ERR_ARG, "instance out of range");
    *n = 0;
    psso_status st = read_status(h);
    if (st != PSSO_OK) return st;
    const int64_t lc = h->cfg.log_stride > 0 ? h->cfg.log_capacity : 0;
    if (lc == 0) return PSSO_OK;
    const HostInst& I = h->inst[instance];
    std::vector<LogDev> all((size_t)lc);
    CUDA_TRY(cudaMemcpy(all.data(), h->arena + I.off_log, all.size() * sizeof(LogDev), cudaMemcpyDeviceToHost));
    std::vector<LogDev> valid;
    for (const auto& e : all)
        if (e.gen >= 0) valid.push_back(e);
    std::sort(valid.begin(), valid.end(), [](const LogDev& a, const LogDev& b) { return a.gen < b.gen; });
    const int64_t m = std::min<int64_t>(cap, (int64_t)valid.size());
    static_assert(sizeof(LogDev) == sizeof(psso_log_entry), "log layout");
    if (buf && m > 0) std::memcpy(buf, valid.data(), (size_t)m * sizeof(LogDev));
    *n = buf ? m : (int64_t)valid.size();
    return PSSO_OK;
}

psso_status psso_stats(psso_handle h, psso_stats_t* out)
{
    if (!h || !out) return fail(PSSO_ERR_ARG, "handle or out is NULL");
    std::memset(out, 0, sizeof *out);
    out->generations = h->gen;
    out->evaluations = h->evals;
    out->updates = h->updates;
    out->blocks = h->async ? h->agrid : h->grid;
    out->threads_per_block = h->async ? h->ablock : h->block;
    out->instances = (int32_t)h->inst.size();
    out->batch_classes = (int32_t)h->bat.classes.size();
    int64_t r = 0;
    for (const auto& I : h->inst) {
        GBestDev gb;
        if (cudaMemcpy(&gb, h->arena + I.off_gb, sizeof gb, cudaMemcpyDeviceToHost) == cudaSuccess)
            r += gb.total_rechecks;
    }
    out->rechecks = r;
    int64_t refined = 0;
    for (const auto& I : h->inst) {
        if (!I.tc) continue;
        unsigned long long v = 0;
        if (cudaMemcpy(&v, &I.rh.dev.ctl->refined, sizeof v, cudaMemcpyDeviceToHost) == cudaSuccess)
            refined += (int64_t)v;
    }
    out->refinements = refined;
    out->launches = h->launches;
    out->h2d_bytes = h->h2d;
    out->d2h_bytes = h->d2h;
    return PSSO_OK;
}

psso_status psso_polish(psso_handle h, int32_t instance, int32_t steps, double lr, int32_t* improved)
{
    if (!h) return fail(PSSO_ERR_ARG, "handle is NULL");
    if (instance < 0 || instance >= (int32_t)h->inst.size()) return fail(PSSO_ERR_ARG, "instance out of range");
    if (steps < 0 || !(lr >= 0.0) || !std::isfinite(lr)) return fail(PSSO_ERR_ARG, "need steps >= 0 and a finite lr >= 0");
    if (h->failed) return fail(PSSO_ERR_STATE, "the handle failed earlier");
    if (h->shard)
        return fail(PSSO_ERR_UNSUPPORTED,
                    "psso_polish: a shard's gBest may be another shard's particle (polish the swarm's "
                    "gBest on its owner and pass the result with psso_set_gbest)");
    psso_status st = read_status(h);
    if (st != PSSO_OK) return st;
    const HostInst& I = h->inst[instance];
    GBestDev before;
    CUDA_TRY(cudaMemcpy(&before, h->arena + I.off_gb, sizeof before, cudaMemcpyDeviceToHost));
    if (before.idx < 0 || before.idx >= I.pr.N)
        return fail(PSSO_ERR_STATE, "psso_polish: the gBest index (set by psso_set_gbest) names no particle "
                                    "of this instance; run a generation first");
    int owner = -1;
    if (I.R > 1)
        for (const auto& u : h->units)
            if (u.inst == instance && before.idx >= u.i0 && before.idx < u.i1) owner = u.rank;
    CUDA_TRY(launch_polish(reinterpret_cast<const InstDev*>(h->arena + h->off_instdev), instance, h->lattice,
                           owner, h->gen, steps, (float)lr, h->stream));
    GBestDev after;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    CUDA_TRY(cudaMemcpy(&after, h->arena + I.off_gb, sizeof after, cudaMemcpyDeviceToHost));
    // The kernel only ever replaces the gBest by a row with a strictly lower FP64
    // value (and then always records that value).
    if (improved) *improved = (after.has64 && (!before.has64 || after.f64 < before.f64)) ? 1 : 0;
    return PSSO_OK;
}

// Batched pipeline: per generation, the streaming step kernels (rows over 128
// variables), the narrow-row step kernels, and the arg-min kernel.
static psso_status time_bat_kernels(psso_ctx* h, int32_t generations, float* ms, int32_t n)
{
    if (n < 3) return fail(PSSO_ERR_ARG, "psso_time_kernels needs room for 3 values on a batched handle");
    if (h->failed) return fail(PSSO_ERR_STATE, "the handle failed earlier");
    if (h->gen + generations > 0xfffffff0LL) return fail(PSSO_ERR_ARG, "generation counter would exceed 2^32");
    CUDA_TRY(cudaSetDevice(h->device));
    const int K = (int)h->bat.classes.size() + 1;
    std::vector<cudaEvent_t> ev(K + 1);
    for (auto& x : ev) CUDA_TRY(cudaEventCreate(&x));
    double acc[3] = {0.0, 0.0, 0.0};
    cudaError_t e = launch_bat_set_gen(h->bat.gen, h->gen + 1, h->stream);
    for (int32_t g = 0; g < generations && e == cudaSuccess; ++g) {
        e = enqueue_bat_generation(h, h->stream, ev.data());
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[K]);
        for (int q = 0; q < K && e == cudaSuccess; ++q) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
            const int slot = q + 1 == K ? 2 : (h->bat.classes[q].stream ? 0 : 1);
            acc[slot] += t;
        }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(PSSO_ERR_CUDA, std::string("psso_time_kernels: ") + cudaGetErrorString(e));
    h->gen += generations;
    for (const auto& I : h->inst) {
        h->evals += I.pr.N * generations;
        h->updates += I.pr.N * I.pr.D * generations;
    }
    h->launches += 1 + (int64_t)K * generations;
    for (int q = 0; q < n; ++q) ms[q] = q < 3 ? (float)(acc[q] / generations) : 0.f;
    return PSSO_OK;
}

psso_status psso_time_kernels(psso_handle h, int32_t instance, int32_t generations, float* ms, int32_t n)
{
    if (!h || !ms) return fail(PSSO_ERR_ARG, "handle or ms is NULL");
    if (instance < 0 || instance >= (int32_t)h->inst.size()) return fail(PSSO_ERR_ARG, "instance out of range");
    if (generations < 1 || n < rot::KERNELS_PER_GENERATION)
        return fail(PSSO_ERR_ARG, "need generations >= 1 and room for every kernel of a generation");
    if (h->bat.n_all > 0 && h->bat.n_all == (int32_t)h->inst.size())
        return time_bat_kernels(h, generations, ms, n);
    if (h->inst.size() != 1) return fail(PSSO_ERR_ARG, "psso_time_kernels needs a single-instance handle");
    HostInst& I = h->inst[instance];
    if (!I.tc) return fail(PSSO_ERR_UNSUPPORTED, "the instance runs on the persistent kernel (one launch per run)");
    if (h->failed) return fail(PSSO_ERR_STATE, "the handle failed earlier");
    if (h->gen + generations > 0xfffffff0LL) return fail(PSSO_ERR_ARG, "generation counter would exceed 2^32");
    CUDA_TRY(cudaSetDevice(h->device));
    constexpr int K = rot::KERNELS_PER_GENERATION;
    cudaEvent_t ev[K + 1];
    for (int q = 0; q <= K; ++q) CUDA_TRY(cudaEventCreate(&ev[q]));
    std::vector<double> acc(K, 0.0);
    psso_status st = PSSO_OK;
    cudaError_t e = rot::set_generation(I.rh, h->gen + 1, h->stream);
    for (int32_t g = 0; g < generations && e == cudaSuccess; ++g) {
        e = rot::enqueue_generation_timed(I.rh, h->stream, ev);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[K]);
        for (int q = 0; q < K && e == cudaSuccess; ++q) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
            acc[q] += t;
        }
    }
    for (int q = 0; q <= K; ++q) cudaEventDestroy(ev[q]);
    if (e != cudaSuccess) return fail(PSSO_ERR_CUDA, std::string("psso_time_kernels: ") + cudaGetErrorString(e));
    h->gen += generations;
    h->evals += I.pr.N * generations;
    h->updates += I.pr.N * I.pr.D * generations;
    h->launches += 1 + (int64_t)K * generations;
    for (int q = 0; q < n; ++q) ms[q] = q < K ? (float)(acc[q] / generations) : 0.f;
    return st;
}

struct SaveHeader {
    char magic[8];
    int64_t gen, evals, updates, state_bytes;
    int32_t grid, block, n_inst, variant;
};

psso_status psso_save(psso_handle h, void* buf, size_t cap, size_t* n)
{
    if (!h || !n) return fail(PSSO_ERR_ARG, "handle or n is NULL");
    const size_t state = h->arena_size - h->state_off;
    *n = sizeof(SaveHeader) + state;
    if (!buf) return PSSO_OK;
    if (cap < *n) return fail(PSSO_ERR_ARG, "buffer too small");
    psso_status st = read_status(h);
    if (st != PSSO_OK) return st;
    SaveHeader hd{};
    std::memcpy(hd.magic, "PSSOST01", 8);
    hd.gen = h->gen;
    hd.evals = h->evals;
    hd.updates = h->updates;
    hd.state_bytes = (int64_t)state;
    hd.grid = h->grid;
    hd.block = h->block;
    hd.n_inst = (int32_t)h->inst.size();
    hd.variant = h->variant;
    std::memcpy(buf, &hd, sizeof hd);
    CUDA_TRY(cudaMemcpy(static_cast<char*>(buf) + sizeof hd, h->arena + h->state_off, state,
                        cudaMemcpyDeviceToHost));
    return PSSO_OK;
}

psso_status psso_load(psso_handle h, const void* buf, size_t n)
{
    if (!h || !buf) return fail(PSSO_ERR_ARG, "handle or buf is NULL");
    if (n < sizeof(SaveHeader)) return fail(PSSO_ERR_ARG, "buffer too small");
    SaveHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    const size_t state = h->arena_size - h->state_off;
    if (std::memcmp(hd.magic, "PSSOST01", 8) != 0 || hd.state_bytes != (int64_t)state ||
        n != sizeof hd + state || hd.grid != h->grid || hd.block != h->block ||
        hd.n_inst != (int32_t)h->inst.size() || hd.variant != h->variant)
        return fail(PSSO_ERR_ARG, "state was saved from a handle with other problems or launch shape");
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    CUDA_TRY(cudaMemcpy(h->arena + h->state_off, static_cast<const char*>(buf) + sizeof hd, state,
                        cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(h->arena + h->off_status, 0, sizeof(StatusDev)));
    for (auto& I : h->inst)
        if (I.tc) CUDA_TRY(cudaMemset(&I.rh.dev.ctl->status, 0, sizeof(int)));
    if (h->actl) CUDA_TRY(cudaMemset(h->actl, 0, sizeof(AsyncCtl)));
    h->gen = hd.gen;
    h->evals = hd.evals;
    h->updates = hd.updates;
    h->failed = false;
    return PSSO_OK;
}

void psso_destroy(psso_handle h)
{
    if (!h) return;
    if (h->arena) {
        cudaSetDevice(h->device);
        cudaStreamSynchronize(h->stream);
        cudaFree(h->arena);
    }
    for (auto& I : h->inst) {
        rot::destroy_graphs(I.rh);
        if (I.rh.mem) cudaFree(I.rh.mem);
    }
    if (h->bat.graph1) cudaGraphExecDestroy(h->bat.graph1);
    if (h->bat.graphG) cudaGraphExecDestroy(h->bat.graphG);
    if (h->bat.mem) cudaFree(h->bat.mem);
    for (auto st : h->bat.side) cudaStreamDestroy(st);
    for (auto st : h->tc_side) cudaStreamDestroy(st);
    for (auto je : h->tc_join) cudaEventDestroy(je);
    if (h->tc_fork) cudaEventDestroy(h->tc_fork);
    for (auto je : h->bat.join) cudaEventDestroy(je);
    if (h->bat.fork) cudaEventDestroy(h->bat.fork);
    if (h->amem) cudaFree(h->amem);
    delete h;
}


// Index checks of the checked build: the first failure any kernel recorded.
psso_status psso_check_report(int32_t* site, int64_t* index, int32_t clear)
{
    if (!site || !index) return fail(PSSO_ERR_ARG, "psso_check_report: site and index must not be NULL");
    *site = 0;
    *index = 0;
#ifndef PSSO_CHECKED
    (void)clear;
    return fail(PSSO_ERR_UNSUPPORTED, "psso_check_report: not a checked build (compile with -DPSSO_CHECKED)");
#else
    CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long first = 0;
    for (chk::Reader r : checked_readers()) {
        unsigned long long v = 0;
        CUDA_TRY(r(&v, clear != 0));
        if (!first) first = v;
    }
    if (first) {
        *site = (int32_t)(first >> 48);
        *index = (int64_t)(first << 16) >> 16;   // the 48-bit index, sign-extended
    }
    return PSSO_OK;
#endif
}

psso_status psso_check_selftest(int64_t index, void* stream)
{
#ifndef PSSO_CHECKED
    (void)index;
    (void)stream;
    return fail(PSSO_ERR_UNSUPPORTED, "psso_check_selftest: not a checked build (compile with -DPSSO_CHECKED)");
#else
    check_selftest_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>((long long)index);
    CUDA_TRY(cudaGetLastError());
    return PSSO_OK;
#endif
}

}  // extern "C"
