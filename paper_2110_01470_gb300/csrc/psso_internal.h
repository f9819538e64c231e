// psso_internal.h -- structures shared by the host planner (psso_api.cu) and
// the persistent generation kernel (sso_kernel.cuh).  Not part of the ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "checked.cuh"

namespace psso {

enum FnId {
    FN_SPHERE = 0,
    FN_ELLIPSOID = 1,
    FN_RASTRIGIN = 2,
    FN_ROSENBROCK = 3,
    FN_ACKLEY = 4,
    FN_ROT_ELLIPSOID = 5,
    FN_ROT_RASTRIGIN = 6,
    FN_ROT_ACKLEY = 7,
    FN_HYPER_ELLIPSOID = 8,   // run as FN_ELLIPSOID with w_j = j + 1
    FN_SCHWEFEL12 = 9,        // the FP64-only functions: 9 .. 12
    FN_GRIEWANK = 10,
    FN_POWELL = 11,
    FN_SCHWEFEL = 12
};

constexpr uint32_t TAG_INIT = 1, TAG_RHO = 2, TAG_FRESH = 3;

// Cross-block exchange.  A published record is REC_WORDS 64-bit words and a
// published row is one word per float position (two per double).  Every word
// carries the low 16 bits of its generation in bits 48..63 and 48 payload
// bits; each aligned 64-bit access is single-copy atomic, so a reader that
// sees the expected tag in every word has read a consistent record / row
// without any lock, atomic or fence.  Slots rotate over SLOTS generations: a
// block rewrites the slot of generation g only at g + SLOTS, after it has seen
// every block's records of g + SLOTS - 1, which those blocks published after
// consuming generation g + SLOTS - 2's data, which they published after
// consuming generation g's data -- two full rounds of dependent publications
// separate a read from the overwrite of its slot.  A reader that saw a newer
// tag would wait (and report a timeout); it can never use wrong data.
constexpr int REC_WORDS = 6;
constexpr int SLOTS = 3;
enum RecWord {
    RW_IDX = 0,   // bits 0..31 particle index, bit 32 = FP64 value present
    RW_VER,       // generation the row was last written
    RW_V0,        // FP64 value low 32 bits, or the FP32 lower bound
    RW_V1,        // FP64 value high 32 bits, or the FP32 upper bound
    RW_ACC,       // accepted pBest updates of the block in this generation
    RW_RCK        // FP64 re-evaluations of the block in this generation
};

constexpr int MAX_UNITS_PER_BLOCK = 32;
constexpr int MAX_CHUNKS_PER_LANE = 8;   // D <= 32 lanes * 8 chunks * 4 = 1024

// Device-side status words.
struct StatusDev {
    int32_t err;      // psso_status of the first device-side failure
    int32_t abort;    // set once any block gives up; every block then exits
    int32_t where;    // instance * 65536 + rank of the block that timed out
    int32_t pad;
};

// gBest of one instance after its last finalised generation.
struct GBestDev {
    int64_t idx;
    int64_t gen;
    int64_t accepted;     // pBest updates in that generation
    int64_t rechecks;     // FP64 re-evaluations in that generation
    int64_t total_rechecks;
    double f64;           // valid iff has64
    float lo, hi;         // rigorous FP32 bounds of the fitness
    uint32_t ver;         // generation the winning pBest row was last written
    int32_t has64;
};

// One log entry; same layout as psso_log_entry.
struct LogDev {
    int64_t gen, idx;
    double value;
    float lo, hi;
    int64_t accepted, rechecks;
};

// Everything the kernel needs about one instance (one independent swarm).
struct InstDev {
    int32_t fn, D, Dp, nchunks;   // Dp = D rounded up to 4; nchunks = Dp / 4
    int32_t G, maxc, R, lattice;  // lanes per particle, chunks per lane, blocks, lattice
    int64_t N;
    uint64_t Tg, Tp, Tw;          // Eq. 2.1 thresholds on a 32-bit draw (0 .. 2^32), in
                                  // increasing order: the first, second and third interval
    uint32_t k0, k1, sid;         // Philox key and stream id
    uint32_t order;               // 0: intervals gBest, pBest, keep; 1: keep, pBest, gBest
    double lb, ub, span;          // FP64 lattice: span = ub - lb
    float S32, L32, lbf, ubf;     // FP32 lattice
    const double* o64;            // shift (never null; zeros for "no shift")
    const float* o32;
    const double* w64;            // ellipsoid weights or null
    const float* w32;
    const double* M64;            // rotation [D][D] (rotated functions) or null
    const float* M32;             // M rounded to float
    const float* M32lo;           // float(M - M32): M = M32 + M32lo to about 2^-48 |M|
    void* X;                      // positions  [N][Dp] (float or double)
    void* P;                      // pBests     [N][Dp]
    double* pf64;                 // pBest fitness in FP64 (F32 mode: valid iff pflag)
    float* plo;                   // F32 mode: rigorous bounds of the pBest fitness
    float* phi;
    uint32_t* pver;               // generation each pBest row was last written
    uint32_t* pflag;              // F32 mode: bit 0 = pf64 valid
    void* grow;                   // exchange rows [SLOTS][R][Dp] (tagged words)
    uint64_t* rec;                // exchange records [SLOTS][R][REC_WORDS]
    uint64_t* rec2;               // second-round records [SLOTS][R][REC_WORDS]
    GBestDev* gb;
    void* gbrow;                  // gBest row [Dp]
    LogDev* log;
    int64_t log_cap;
    int32_t log_stride;
    uint32_t i_base;              // particle index of the first particle in the whole swarm
                                  // (a shard of a swarm split over several GPUs; 0 otherwise):
                                  // every draw is keyed by i_base + the local index
};

// A contiguous range of one instance's particles owned by one block.
struct UnitDev {
    int32_t inst, rank;
    int64_t i0, i1;
    int32_t smem_off;             // byte offset of this unit's gBest row in shared memory
    int32_t resident;             // 1: X, P and pBest state live in shared memory
    int32_t res_off;              // byte offset of the resident state
    int32_t pipelined;            // 1: warp 0 exchanges while warps 1.. compute ahead
};

// Shared-memory layout of a resident unit of n particles (X, P, pf64, plo,
// phi, pver, pflag), identical on host and device.
__host__ __device__ inline size_t res_align(size_t v) { return (v + 15) & ~(size_t)15; }
__host__ __device__ inline size_t resident_bytes(int64_t n, int Dp, int pos_size)
{
    const size_t rows = res_align((size_t)n * Dp * pos_size);
    return 2 * rows + res_align((size_t)n * 8) + 4 * res_align((size_t)n * 4);
}

struct KParams {
    const InstDev* inst;
    const UnitDev* units;
    const int32_t* block_first;   // [grid + 1]: units of block b are [first[b], first[b+1])
    StatusDev* status;
    int64_t g_begin, g_end;       // generations to run (g_begin = 0: the initial population)
    int64_t spin_limit;
    int32_t fault_skip_rank;      // see psso_config.fault_skip_rank
    int32_t pad;
};

// Generation-kernel entry points.  variant: 0 = FP64 fitness with double
// positions, 1 = FP64 fitness with float positions, 2 = FP32 fitness with FP64
// recheck.  mc_index: 0..3 = up to 1, 2, 4, 8 chunks per lane.  op: 0 = launch,
// 1 = occupancy (blocks per SM into *out), 2 = set the dynamic shared-memory
// limit, 3 = maximum threads per block into *out.
cudaError_t gen_call(int variant, int op, int mc_index, const KParams* p, int grid, int block,
                     size_t smem, cudaStream_t s, int* out);
cudaError_t launch_best_f64(const InstDev* inst, int n_inst, int lattice, cudaStream_t s);

// Batched throughput pipeline: one generation of many independent swarms as
// one kernel per class of equal lane-group width G and chunks per lane (each
// group of G lanes updates, evaluates and commits one particle, the particles
// of every instance of the class in one flat range), then one block per
// instance for the gBest.  Positions of instance ids[q] are particles
// first[q] .. first[q+1]-1 of the class range.
struct BatCounters {
    unsigned long long acc, rck;   // pBest updates / FP64 evaluations this generation
};
struct BatParams {
    const InstDev* inst;
    const int32_t* ids;            // [n_ids] instance of each class entry
    const int64_t* first;          // [n_ids + 1] prefix sums of N
    int32_t n_ids, G;
    int64_t total;                 // first[n_ids]
    const long long* gen;          // generation being run (device)
    BatCounters* cnt;              // [instances]
};
// op 0: launch bat_step over p (grid x block); op 1: occupancy (blocks per SM
// into *out) for `block` threads; ops 2 / 3: the same for the streaming kernel
// of wide unrotated rows (one warp per particle; mc_index 3 only).
cudaError_t bat_call(int variant, int mc_index, int op, const BatParams* p, int grid, int block, cudaStream_t s,
                     int* out);
// One block per listed instance: gBest arg-min (exact lowest index), record,
// log, gBest row; then the generation counter + 1 (last kernel of a generation).
cudaError_t launch_bat_argmin(int variant, const InstDev* inst, const int32_t* ids, int n_ids, long long* gen,
                              BatCounters* cnt, cudaStream_t s);
cudaError_t launch_bat_set_gen(long long* gen, long long g, cudaStream_t s);

// Asynchronous flow (Alg. 1): control words of the grid barrier and of the
// rounds of speculation and ordered commit (async_kernel.cu).
struct AsyncCtl {
    unsigned bar_count, bar_gen;   // grid barrier: arrivals, generation word
    unsigned first[3];             // lowest improving particle of a round (3 rotating slots)
    unsigned pad;
    unsigned long long acc[2];     // pBest updates of a generation (by parity)
};
struct AsyncParams {
    const InstDev* inst;
    StatusDev* status;
    AsyncCtl* ctl;
    void* xs;                      // [N][Dp] searched positions of the current round
    double* fs;                    // [N] their FP64 fitness
    int64_t g_begin, g_end, spin_limit;
};
// op 0: launch (cooperative) over grid x block; op 1: occupancy (blocks per SM).
cudaError_t async_call(int pos_size, int mc_index, int op, const AsyncParams* p, int grid, int block,
                       cudaStream_t s, int* out);

cudaError_t launch_polish(const InstDev* inst, int k, int lattice, int owner_rank, int64_t g, int steps,
                          float lr, cudaStream_t s);

// Records the calling thread's last error message (psso_last_error).
void set_last_error(const char* msg);

}  // namespace psso
