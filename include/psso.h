/*
 * psso.h -- C ABI of the GB300 (sm_103a) implementation of the hot path of
 * Parallel Simplified Swarm Optimization (PSSO; Yeh, Liu, Tan, Huang,
 * arXiv 2110.01470): one SSO generation over a whole swarm, i.e.
 *   (a) the per-variable stepwise update of Eq. 2.1,
 *   (b) the fitness of every particle (Kernel Function (E), Sec. 2.3.2;
 *       test functions of Table 3.2 in shifted / rotated form),
 *   (c) the pBest update (Alg. 3) and the gBest arg-min (Alg. 4),
 * repeated for t synchronous generations (Alg. 2), for one swarm or for many
 * independent swarms in one persistent launch.
 *
 * Conventions
 *   * Every call returns a psso_status; nothing aborts or throws across the ABI.
 *     psso_last_error() returns a message for the calling thread's last failure.
 *   * The library owns all device memory it allocates.  Caller buffers are host
 *     pointers unless stated otherwise; they are copied in (create) or out
 *     (best, get_state, get_log) and never retained.
 *   * Work is enqueued on the handle's CUDA stream (psso_config.stream, NULL =
 *     the legacy default stream).  psso_run returns once the work is enqueued;
 *     device-side failures (e.g. PSSO_ERR_TIMEOUT) surface at the next call that
 *     synchronises (psso_sync, psso_best, psso_get_state, psso_get_log,
 *     psso_save) or at the next psso_run.
 *   * A handle may be used from one host thread at a time.
 *
 * Semantics (the readings of the paper this library implements; identical to
 * the CPU oracle shipped with the tests):
 *   * Eq. 2.1 with cumulative thresholds Cg <= Cp <= Cw in [0,1]: a 32-bit
 *     Philox-4x32-10 word r per variable picks gBest_j if r < T(Cg), pBest_ij if
 *     r < T(Cp), keeps x_ij if r < T(Cw), else a fresh uniform value in [lb,ub],
 *     with T(C) = round-half-even(C * 2^32).  psso_problem.order selects the
 *     interval order of Eq. 2.1 as printed instead (x, pBest, gBest, fresh with
 *     Cw <= Cp <= Cg).
 *   * Draws are keyed by (seed, stream_id) with counter (variable block,
 *     particle, generation, tag); the result of a run depends on nothing else
 *     (not on the launch shape, the GPU, or how generations are split between
 *     psso_run calls).
 *   * Generation 0 (the initial population, Kernel Function (I), Sec. 2.3.1)
 *     is enqueued by psso_create / psso_create_ex; psso_run(h, t) then runs
 *     generations g+1 .. g+t.
 *   * pBest_i <- x_i when f(x_i) <= f(pBest_i) (Alg. 3); gBest is the
 *     lowest-index arg-min of the pBest fitness (Alg. 4).
 */
#ifndef PSSO_H
#define PSSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psso_ctx* psso_handle;

typedef enum {
    PSSO_OK = 0,
    PSSO_ERR_ARG = 1,         /* invalid argument; nothing was changed            */
    PSSO_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has details)  */
    PSSO_ERR_OOM = 3,         /* device memory allocation failed                   */
    PSSO_ERR_TIMEOUT = 4,     /* a cross-block wait ran past its limit; the handle
                                 is left in an undefined state and must be destroyed
                                 or reloaded with psso_load                          */
    PSSO_ERR_STATE = 5,       /* call not valid in the handle's current state       */
    PSSO_ERR_UNSUPPORTED = 6  /* valid request the library does not implement       */
} psso_status;

/* Test functions (Table 3.2 of the paper; shifted by o, rotated by M).
 * z = x - o (or z = M (x - o) for the rotated forms), j = 0 .. D-1:
 *   SPHERE           sum z_j^2                                         (f1)
 *   ELLIPSOID        sum w_j z_j^2            (w given, e.g. 10^(6j/(D-1)))
 *   RASTRIGIN        10 D + sum (z_j^2 - 10 cos(2 pi z_j))              (f5)
 *   ROSENBROCK       sum_{j<D-1} 100 (a_{j+1} - a_j^2)^2 + (a_j - 1)^2,
 *                    a = z + 1                                         (f4)
 *   ACKLEY           -20 exp(-0.2 sqrt(sum z^2 / D)) - exp(sum cos(2 pi z) / D)
 *                    + 20 + e                                          (f6)
 *   HYPER_ELLIPSOID  sum (j + 1) z_j^2 (ELLIPSOID with w_j = j + 1)    (f2)
 *   SCHWEFEL12       sum_i (sum_{j<=i} z_j)^2                          (f3)
 *   GRIEWANK         1 + sum z_j^2 / 4000 - prod cos(z_j / sqrt(j + 1)) (f7)
 *   POWELL           sum over blocks of 4 variables of (z0 + 10 z1)^2 +
 *                    5 (z2 - z3)^2 + (z1 - 2 z2)^4 + 10 (z0 - z3)^4, with
 *                    z = 0 beyond D                                    (f8)
 *   SCHWEFEL         418.9829 D - sum z_j sin(sqrt|z_j|)                (f9)
 * Every function but SCHWEFEL is 0 at x = o (SCHWEFEL is near its minimum,
 * about 1.3e-5 D, at z_j = 420.9687).  SCHWEFEL12, GRIEWANK, POWELL and
 * SCHWEFEL have FP64 fitness only: PSSO_PREC_F32_RECHECK and the FP32
 * gradient calls return PSSO_ERR_UNSUPPORTED for them. */
typedef enum {
    PSSO_SPHERE = 0,
    PSSO_ELLIPSOID = 1,
    PSSO_RASTRIGIN = 2,
    PSSO_ROSENBROCK = 3,
    PSSO_ACKLEY = 4,
    PSSO_ROT_ELLIPSOID = 5,
    PSSO_ROT_RASTRIGIN = 6,
    PSSO_ROT_ACKLEY = 7,
    PSSO_HYPER_ELLIPSOID = 8,
    PSSO_SCHWEFEL12 = 9,
    PSSO_GRIEWANK = 10,
    PSSO_POWELL = 11,
    PSSO_SCHWEFEL = 12
} psso_fn;

/* Position lattice: which grid fresh values (Eq. 2.1's last branch and the
 * initial population) are drawn on.
 *   F64: x = fma(ub - lb, m 2^-53, lb), m = 53 random bits.
 *   F32: x = fmaf(S, m 2^-24, L) clamped to the floats inside [lb, ub], with
 *        S, L the nearest floats to ub - lb and lb, m = 24 random bits.  Every
 *        position is then a float, so FP32 and FP64 fitness see the same x. */
typedef enum { PSSO_LATTICE_F64 = 0, PSSO_LATTICE_F32 = 1 } psso_lattice;

/* Fitness precision.
 *   F64          fitness in FP64 in a fixed summation order; results are
 *                bit-identical to the CPU oracle.
 *   F32_RECHECK  fitness in FP32 with a rigorous per-evaluation error bound;
 *                every pBest / gBest comparison the bound cannot decide is
 *                re-evaluated in FP64 (oracle order), so all decisions -- and
 *                therefore all positions -- equal the F64 run's.  Needs the F32
 *                lattice and a float-exact shift. */
typedef enum { PSSO_PREC_F64 = 0, PSSO_PREC_F32_RECHECK = 1 } psso_precision;

/* Interval order of Eq. 2.1 (psso_problem.order).
 *   GPX    r < T(Cg) -> gBest_j, r < T(Cp) -> pBest_ij, r < T(Cw) -> x_ij, else a
 *          fresh value; needs 0 <= Cg <= Cp <= Cw <= 1 (the default).
 *   PAPER  the order Eq. 2.1 prints: r < T(Cw) -> x_ij, r < T(Cp) -> pBest_ij,
 *          r < T(Cg) -> gBest_j, else a fresh value; needs 0 <= Cw <= Cp <= Cg
 *          <= 1 (e.g. the paper's Cw, Cp, Cg = 0.3, 0.6, 0.8, Sec. 3.4).
 * Both draw the same words r; for the same branch probabilities they give
 * different, equally distributed trajectories. */
typedef enum { PSSO_ORDER_GPX = 0, PSSO_ORDER_PAPER = 1 } psso_order;

/* One problem instance (one independent swarm). */
typedef struct {
    int32_t fn;          /* psso_fn                                                */
    int32_t lattice;     /* psso_lattice                                           */
    int64_t N;           /* particles, 1 .. 2^31-1                                  */
    int64_t D;           /* variables, 1 .. 1024                                    */
    double lb, ub;       /* search bounds, lb < ub, finite                          */
    double Cg, Cp, Cw;   /* cumulative Eq. 2.1 thresholds, ordered as `order` says  */
    uint64_t seed;       /* Philox key                                              */
    uint32_t stream_id;  /* Philox counter stream, < 2^24 (independent instances)   */
    uint32_t order;      /* psso_order (0 = GPX)                                    */
    const double* shift;    /* host, D values, or NULL for o = 0                    */
    const double* weights;  /* host, D values; required by ELLIPSOID, ROT_ELLIPSOID  */
    const double* rotation; /* host, D*D row-major M; required by rotated functions */
} psso_problem;

/* Launch and bookkeeping options; zero-initialise for the defaults. */
typedef struct {
    int32_t precision;          /* psso_precision                                   */
    int32_t threads_per_block;  /* 0 = 256; a multiple of 32 in [64, 512]           */
    int32_t single_block_max;   /* 0 = auto: swarms of at most this many particle
                                   passes run in one block with no cross-block
                                   exchange; -1 = never                            */
    int32_t log_stride;         /* log every log_stride-th generation (0 = off)     */
    int64_t log_capacity;       /* log entries kept per instance (ring)             */
    int64_t spin_limit;         /* polls of a cross-block wait before the run fails
                                   with PSSO_ERR_TIMEOUT (0 = default, ~seconds)     */
    void* stream;               /* cudaStream_t to enqueue on (NULL = default)      */
    int32_t max_blocks;         /* 0 = all co-resident blocks; else an upper bound  */
    int32_t fault_skip_rank;    /* testing only: 0 = off; k > 0 makes block rank k-1
                                   of instance 0 never publish, so its peers' waits
                                   run out and psso_run reports PSSO_ERR_TIMEOUT     */
    int32_t residency;          /* 0 = auto (particle state in shared memory when it
                                   fits), 2 = always stream it from global memory   */
    int32_t pipeline;           /* 0 = auto: a single swarm spread over many blocks
                                   uses a control warp that exchanges gBest while
                                   the other warps compute the next generation;
                                   2 = never                                        */
    int32_t tensor_rotation;    /* rotated functions with F32_RECHECK precision:
                                   0 = auto (swarms with N >= 128 and D >= 32 run
                                   each generation as a kernel sequence around a
                                   tcgen05 tensor-core GEMM for z = M (x - o));
                                   1 = always; -1 = never (per-particle kernel).
                                   The GEMM is exact for D <= 1023: a swarm with
                                   D = 1024 runs the per-particle kernel (auto) or
                                   fails with PSSO_ERR_UNSUPPORTED (always)        */
    int32_t batch_stream;       /* handles of many swarms: 0 = auto (16 or more
                                   swarms that are not on the tensor-core pipeline
                                   run each generation as one kernel per row-width
                                   class over every particle of every swarm, then
                                   one block per swarm for the gBest, replayed as
                                   CUDA graphs); 1 = always; -1 = never (the
                                   persistent kernel)                              */
    int32_t batch_blocks_per_sm;/* batched pipeline: resident blocks per SM of each
                                   step kernel's grid (0 = the occupancy maximum;
                                   larger values are clamped to it)                 */
    int32_t flow;               /* psso_flow: 0 = synchronous generations (Alg. 2),
                                   1 = asynchronous generations (Alg. 1)           */
} psso_config;

/* Generation flow (psso_config.flow).
 *   SYNC   Alg. 2, the PSSO flow: every particle searches with the gBest of the
 *          previous generation; pBest_i <- x_i when f <= pF (Alg. 3); gBest is
 *          then the lowest-index arg-min of the pBest fitness (Alg. 4).
 *   ASYNC  Alg. 1, the sequential CPU-SSO: particles are taken in index order;
 *          particle i searches with the gBest left by particles 0..i-1 of the
 *          same generation, replaces its pBest when f < pF and the gBest when
 *          f < gF (both strict, as Alg. 1 writes them).  Runs as rounds of
 *          speculative search of all remaining particles and ordered commit up
 *          to the first one that beats the gBest.  One instance per handle,
 *          PSSO_PREC_F64 only (else PSSO_ERR_UNSUPPORTED); results are
 *          bit-identical to the CPU oracle's Alg. 1. */
typedef enum { PSSO_FLOW_SYNC = 0, PSSO_FLOW_ASYNC = 1 } psso_flow;

/* One log entry (psso_get_log). */
typedef struct {
    int64_t generation;
    int64_t index;       /* gBest particle index                                    */
    double value;        /* gBest fitness in FP64 (NaN if only the FP32 bounds are
                            known at that generation)                              */
    float value_lo;      /* rigorous lower / upper bound of the gBest fitness       */
    float value_hi;
    int64_t accepted;    /* pBest updates in this generation (all particles)        */
    int64_t rechecks;    /* FP64 re-evaluations in this generation                  */
} psso_log_entry;

/* Counters since creation (psso_stats). */
typedef struct {
    int64_t generations;     /* generations completed (excluding generation 0)     */
    int64_t evaluations;     /* fitness evaluations, all instances                  */
    int64_t updates;         /* particle-variable updates, all instances            */
    int64_t rechecks;        /* FP64 re-evaluations (F32_RECHECK)                   */
    int64_t h2d_bytes;       /* bytes this handle copied host -> device             */
    int64_t d2h_bytes;       /* bytes this handle copied device -> host             */
    int32_t blocks;          /* blocks of the persistent launch                     */
    int32_t threads_per_block;
    int32_t instances;
    int32_t batch_classes;   /* step kernels per generation of the batched pipeline
                                (0 when the handle does not use it)               */
    int64_t refinements;     /* rotated functions on the tensor-core pipeline: rows
                                re-evaluated by the compensated FP32 rotation
                                before any FP64 recheck                           */
    int64_t launches;        /* kernels this handle enqueued for psso_create,
                                psso_run and psso_reset (graph nodes included)     */
} psso_stats_t;

/* Creates one swarm with the zero shift, FP64 lattice and FP64 precision,
 * and enqueues generation 0 on the default stream.  Ellipsoid weights are
 * 10^(6 j/(D-1)).  Rotated functions need psso_create_ex (they need M).
 * Paper: Sec. 3.3 (problem f on [L,U] with Nvar variables and Nsol particles),
 * Table 3.1 (Sol, PBests, GBest, Cw/Cp/Cg, [varMin, varMax]). */
psso_status psso_create(psso_fn fn, int64_t N, int64_t D, double lb, double ub,
                        double Cg, double Cp, double Cw, uint64_t seed, psso_handle* out);

/* Creates `count` independent swarms (1 .. 65536) that always advance
 * together, copies their data (shift, weights, rotation) to the device, and
 * enqueues generation 0 for all of them.  cfg may be NULL (defaults).  All
 * instances must share one lattice. */
psso_status psso_create_ex(const psso_problem* problems, int32_t count,
                           const psso_config* cfg, psso_handle* out);

/* Enqueues `generations` (>= 0) further SSO generations (Alg. 2) for every
 * instance as one persistent cooperative launch. */
psso_status psso_run(psso_handle h, int64_t generations);

/* Restarts every instance at generation 0 with the same seeds and data:
 * clears the exchange records, gBest state and log, and enqueues the initial
 * population again (Kernel Function (I), Sec. 2.3.1).  No allocation; also
 * clears a failed state.  The run that follows is identical to one on a new
 * handle. */
psso_status psso_reset(psso_handle h);

/* Waits for the handle's stream and reports any device-side failure. */
psso_status psso_sync(psso_handle h);

/* gBest of instance `instance` after the last completed generation: FP64
 * fitness (`value`), particle index, and the D-value row (`row`, may be NULL).
 * In F32_RECHECK mode the FP64 value is computed on demand.  Synchronises.
 * Paper: Alg. 2's final step, which sends the data back to the CPU to
 * calculate fOpt (the best fitness found; Table 3.1's GBest and fOpt). */
psso_status psso_best(psso_handle h, int32_t instance, double* value, int64_t* index,
                      double* row);

/* One swarm split over several GPUs: every GPU runs the update, fitness and
 * pBest step of its own particles, and the gBest is the lowest-index arg-min
 * over all of them (one exchange per generation).
 *
 * psso_create_shard creates a handle for particles first .. first+count-1 of
 * `problem` (problem->N particles in all): its draws are those of these
 * particles in the whole swarm, so the union of the shards' runs is the run of
 * the whole swarm, provided that before every generation each shard is given
 * the swarm's gBest of the previous generation with psso_set_gbest (value,
 * global index, row: the minimum over the shards' psso_best by (value, index)).
 * The shard runs in one block (its gBest row is restored from the handle's
 * gBest state at every psso_run).  The asynchronous flow cannot be split
 * (PSSO_ERR_UNSUPPORTED).  Indices the shard reports (psso_best, the log)
 * are local: add `first`.
 *
 * psso_set_gbest replaces the gBest the next generation searches with: FP64
 * value, an index (stored as given; any label), and the row (host, D values
 * inside [lb, ub]; floats for the F32 lattice).  Synchronises.  Valid for
 * shard handles and single-block, tensor-pipeline or batched-pipeline
 * instances; PSSO_ERR_UNSUPPORTED for an instance spread over several blocks
 * or the asynchronous flow. */
psso_status psso_create_shard(const psso_problem* problem, int64_t first, int64_t count,
                              const psso_config* cfg, psso_handle* out);
psso_status psso_set_gbest(psso_handle h, int32_t instance, double value, int64_t index, const double* row);

/* Copies positions X (N*D), pBests P (N*D) and pBest fitness pF (N) of one
 * instance to the host (FP64 values; any pointer may be NULL).  In
 * F32_RECHECK mode pF holds the FP64 value where known, else the midpoint of
 * the FP32 bounds.  Synchronises. */
psso_status psso_get_state(psso_handle h, int32_t instance, double* X, double* P, double* pF);

/* Copies up to `cap` of instance `instance`'s log entries (oldest first) and
 * sets *n to the number copied.  Synchronises. */
psso_status psso_get_log(psso_handle h, int32_t instance, psso_log_entry* buf, int64_t cap,
                         int64_t* n);

/* Counters since creation.  Does not synchronise. */
psso_status psso_stats(psso_handle h, psso_stats_t* out);

/* Generation number of the last enqueued generation (0 after create). */
int64_t psso_generation(psso_handle h);

/* Serialises the full state (positions, pBests, fitness, gBest, generation,
 * counters) into `buf` (host, `cap` bytes); *n receives the size needed.  With
 * buf == NULL only *n is set.  Runs resumed from a saved state are
 * bit-identical to uninterrupted runs.  Synchronises. */
psso_status psso_save(psso_handle h, void* buf, size_t cap, size_t* n);

/* Restores a state written by psso_save for a handle created with the same
 * problems and configuration. */
psso_status psso_load(psso_handle h, const void* buf, size_t n);

/* Batched fitness (Kernel Function (E), Sec. 2.3.2): f_i = f(X_i) for N rows of
 * D values.  X (N*D, row-major), shift/weights/rotation as in psso_problem and
 * the outputs are host pointers.  precision = PSSO_PREC_F64 gives the FP64
 * value in the library's fixed summation order (bit-identical to the oracle);
 * PSSO_PREC_F32_RECHECK gives the FP32 value and, in err (may be NULL), its
 * rigorous bound |f32 - f64| <= err; it needs every X and shift value to be a
 * float.  stream: cudaStream_t or NULL.  Synchronises. */
psso_status psso_evaluate(psso_fn fn, int64_t N, int64_t D, const double* X, const double* shift,
                          const double* weights, const double* rotation, int32_t precision,
                          double* f, double* err, void* stream);

/* Batched fitness for callers that cannot allocate device memory: code that
 * runs while another allocator owns the device memory, code that must not let
 * cudaMalloc / cudaFree synchronise the device in its steady state (a
 * real-time or latency-critical loop), or code that has a fixed device-memory
 * budget set aside up front.  The paper has no counterpart; this is a
 * convenience of this library.
 *
 * Computes what psso_evaluate computes (same routines, same summation order,
 * bit-identical results) but takes DEVICE pointers: X (N*D doubles,
 * row-major), shift and weights (D doubles each, or NULL as in psso_problem),
 * and the outputs f (N doubles) and err (N doubles, or NULL).  It allocates
 * nothing: its only scratch, the padded shift / weight vectors, lives in one
 * static device array of 24 KiB (D at most 1024; larger D is rejected with
 * PSSO_ERR_ARG; N at most 8 * (2^31 - 1)).  With PSSO_PREC_F32_RECHECK the
 * FP32 terms and the bound err are only valid for float inputs: every row
 * holding an X value that is not a float gets NaN in f and err, and so does
 * every row when a shift value is not a float.  Rotated functions are not
 * available here (they need a D x D matrix, which does not fit the static
 * scratch): they return PSSO_ERR_UNSUPPORTED.
 *
 * Work is enqueued on `stream` (cudaStream_t, NULL = default) and the call
 * returns without waiting.  The first call on a device looks up the scratch
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  The address is cached for the
 * life of the process, so the library must not be used on a device across a
 * cudaDeviceReset.  Every call shares the array and rewrites what it reads
 * (calls queued one after another on one stream are safe); calls that overlap
 * on the GPU (unordered streams) race on it. */
psso_status psso_evaluate_noalloc(psso_fn fn, int64_t N, int64_t D, const double* X,
                                  const double* shift, const double* weights, int32_t precision,
                                  double* f, double* err, void* stream);

/* Differentiable batched fitness in FP32 (the fitness of Kernel Function (E),
 * Sec. 2.3.2, and its gradient; the paper names gradient descent in the title
 * of Sec. 2 only, so these calls have no counterpart in its method).
 *
 * DEVICE pointers, all float32, row-major and unpadded: X (N*D), shift (D),
 * weights (D; ELLIPSOID / ROT_ELLIPSOID only, else may be NULL), rotation
 * (D*D, M[j*D + k] for z_j = sum_k M_jk (x_k - o_k); rotated functions only).
 *   psso_fitness_forward:  f (N) = f(X_i) in FP32 (relative error a few 2^-24
 *                          for well-conditioned sums; not the bit pattern of
 *                          psso_evaluate).
 *   psso_fitness_backward: grad_X (N*D) = grad_f[i] * df/dx (X_i); for rotated
 *                          functions df/dx = M^T df/dz.
 * Gradients (z the function's coordinates):
 *   sphere 2 z_j;  ellipsoid 2 w_j z_j;  Rastrigin 2 z_j + 20 pi sin(2 pi z_j);
 *   Rosenbrock [j<D-1](2 z_j - 400 a_j u_j) + [j>0] 200 u_{j-1},
 *     a = z + 1, u_j = a_{j+1} - a_j^2;
 *   Ackley 4 e^{-0.2 A} z_j / (A D) + 2 pi e^{C} sin(2 pi z_j) / D,
 *     A = sqrt(sum z^2 / D), C = sum cos(2 pi z) / D  (the first term is 0 at A = 0).
 * 1 <= D <= 1024; otherwise, or for a NULL pointer the function needs,
 * PSSO_ERR_ARG.  Work is enqueued on `stream` (cudaStream_t, NULL = default);
 * the calls allocate nothing and return without waiting. */
psso_status psso_fitness_forward(psso_fn fn, int64_t N, int64_t D, const float* X, const float* shift,
                                 const float* weights, const float* rotation, float* f, void* stream);
psso_status psso_fitness_backward(psso_fn fn, int64_t N, int64_t D, const float* X, const float* shift,
                                  const float* weights, const float* rotation, const float* grad_f,
                                  float* grad_X, void* stream);

/* The same two calls with the rotated functions' products on the tensor
 * cores: z = M (x - o) for all N rows as one split-BF16 tcgen05 GEMM
 * (Z = (X - O) M^T), the function and its z-gradient per row from Z, and
 * the backward product M^T df/dz as a second GEMM (grad_X = G M, G the rows
 * grad_f[i] df/dz).  Each GEMM output carries an error of at most about
 * 2^-20 per MMA of sum |A_ik| |B_jk| (typically far less).  `workspace` is caller-owned DEVICE memory,
 * 256-byte aligned, of at least psso_fitness_workspace_size bytes; the calls
 * allocate nothing, enqueue on `stream` and return without waiting.  Unrotated
 * functions (and D < 16) need no workspace and run psso_fitness_forward /
 * _backward.  Should a tensor-core wait run out (it does not in normal
 * operation), the outputs are left NaN.  Calls sharing one workspace must be
 * ordered on one stream. */
psso_status psso_fitness_workspace_size(psso_fn fn, int64_t N, int64_t D, size_t* bytes);
psso_status psso_fitness_forward_ws(psso_fn fn, int64_t N, int64_t D, const float* X, const float* shift,
                                    const float* weights, const float* rotation, float* f, void* workspace,
                                    size_t ws_bytes, void* stream);
psso_status psso_fitness_backward_ws(psso_fn fn, int64_t N, int64_t D, const float* X, const float* shift,
                                     const float* weights, const float* rotation, const float* grad_f,
                                     float* grad_X, void* workspace, size_t ws_bytes, void* stream);

/* gBest polish (an optional local search; the paper has no counterpart and
 * psso_run never calls it): from instance k's gBest row, `steps` FP32 steps
 * x <- clamp(x - lr df/dx, [lb, ub]) with the gradient of
 * psso_fitness_backward.  The polished row replaces the gBest particle's pBest
 * (and the gBest) only if its FP64 fitness is strictly lower; the particle's
 * position x is untouched.  A run that never calls psso_polish is unaffected;
 * one that does leaves the oracle's trajectory.  *improved (may be NULL) is
 * set to 1 when the row was replaced, else 0.  Synchronises the handle's
 * stream.  PSSO_ERR_ARG for a bad instance, steps < 0 or lr not a finite
 * value >= 0; PSSO_ERR_UNSUPPORTED on a shard handle (its gBest may be
 * another shard's particle); PSSO_ERR_STATE while the gBest is one that
 * psso_set_gbest put there with an index outside the instance. */
psso_status psso_polish(psso_handle h, int32_t instance, int32_t steps, double lr, int32_t* improved);

/* Rotation z = M (x - o) of N rows on the tensor cores (the transform of the
 * rotated test functions; the paper's functions are unrotated, the rotated
 * forms follow the usual z = M (x - o) convention).  DEVICE pointers, float32,
 * row-major: X (N*D), shift (D), rotation (D*D, M[j*D + k]), Z (N*D, out).
 * d = fl32(x - o) and M are split exactly into three BF16 parts each; the six
 * products above 2^-24 are accumulated in FP32 by tcgen05 MMAs (the main part
 * in three accumulators over K blocks dealt round robin, the corrections in a
 * fourth) and added.  Error model:
 * |z~_j - sum_k M_jk d_k| <= c(Kp) * sum_k |M_jk| |d_k| + 2^-24 |z~_j|,
 * Kp = D rounded up to 64, c(Kp) = 1.05 (2^-20 1.04 (4 ceil(Kp/192)
 * + 5 (Kp/16) 2^-7) + 1.03 2^-23 + 5.12 2^-24) when every MMA instruction
 * errs by at most 2^-20 of its operand magnitudes (the probed accumulation
 * of sm_103a errs by at most 0.625 2^-20).  1 <= N <= 2^24, 1 <= D <= 8192.  Allocates its
 * operand planes for the call and synchronises `stream`.  PSSO_ERR_TIMEOUT if
 * a pipeline wait ran out (the device is left usable). */
psso_status psso_rotate(int64_t N, int64_t D, const float* X, const float* shift, const float* rotation,
                        float* Z, void* stream);

/* Measurement aid for single-instance handles whose swarm runs on the
 * tensor-core pipeline (rotated function, F32_RECHECK): runs `generations`
 * generations exactly as psso_run would (same results), with a CUDA event
 * between consecutive kernels on the handle's stream, and writes each
 * kernel's mean duration in ms to ms[0..10] (update, GEMM + fitness epilogue,
 * decisions, FP32 refinement rotation and decisions, FP64 rotation and
 * decisions, arg-min, FP64 rotation and decisions of arg-min candidates,
 * gBest); n >= 11.  On a handle whose swarms all run on the batched
 * pipeline it times that pipeline instead, writing the mean per-generation
 * duration of its streaming step kernels (rows over 128 variables), of its
 * other step kernels and of its arg-min kernel to ms[0..2] (n >= 3; instance
 * is ignored).  The paper has no counterpart.  Synchronises.
 * PSSO_ERR_UNSUPPORTED for a swarm on the persistent kernel. */
psso_status psso_time_kernels(psso_handle h, int32_t instance, int32_t generations, float* ms, int32_t n);

/* Result of psso_autotune. */
typedef struct {
    int32_t candidates;          /* configurations timed (0: answered from the cache) */
    int32_t threads_per_block;   /* chosen psso_config.threads_per_block              */
    int32_t batch_blocks_per_sm; /* chosen psso_config.batch_blocks_per_sm            */
    int32_t reserved;
    double best_ms;              /* mean ms per generation, chosen configuration      */
    double default_ms;           /* mean ms per generation, configuration as given    */
} psso_tune_report;

/* Launch-shape autotuner (the paper has no counterpart; its kernels use one
 * fixed shape).  Creates a scratch handle for each candidate configuration of
 * `problems`, runs 3 warm-up generations and then times `generations` (1 ..
 * 100000) generations with CUDA events on a private stream, and writes into
 * `tuned` a copy of `cfg` (NULL = defaults) with the fastest candidate's
 * shape:
 *   - threads_per_block (particles per block of the persistent kernel), when
 *     some swarm runs on it;
 *   - batch_blocks_per_sm (grid of the batched pipeline's step kernels), when
 *     the handle uses that pipeline.
 * The given configuration is always a candidate, so the chosen one is never
 * slower in the sweep.  Swarms on the tensor-core pipeline have fixed tile
 * shapes and add no candidates.  The launch shape never changes results, so
 * a handle made with `tuned` computes exactly what one made with `cfg` does.
 * Results are cached per process by (problem shapes, functions, lattice,
 * configuration): a repeated call times nothing.  `report` may be NULL.
 * Allocates and frees device memory for each candidate; synchronises. */
psso_status psso_autotune(const psso_problem* problems, int32_t count, const psso_config* cfg,
                          int32_t generations, psso_config* tuned, psso_tune_report* report);

/* Measured peaks of this GPU (psso_microbench); the paper has no counterpart.
 * Rates are operations per second over the whole GPU; latencies in ns. */
typedef struct {
    double fp32_fma_per_s;       /* FP32 fused multiply-adds                           */
    double fp64_fma_per_s;       /* FP64 fused multiply-adds                           */
    double int_mad_per_s;        /* 32-bit integer multiply-adds (low half)            */
    double int_mulhi_xor_per_s;  /* pairs (high half of a 32 x 32 product, xor)        */
    double philox_blocks_per_s;  /* Philox-4x32-10 blocks (the update's draws)          */
    double l2_handoff_ns;        /* a store on one SM seen by a polling load on another */
    double grid_barrier_ns;      /* a grid barrier of one block per SM (counter + flag) */
    double cluster_barrier_ns;   /* a hardware barrier of an 8-CTA cluster              */
    double sm_clock_mhz;         /* SM clock during the FP32 kernel (clock64 / timer)   */
    int32_t sms;                 /* streaming multiprocessors                           */
    int32_t reserved;
} psso_peaks;

/* Runs the microbenchmarks behind psso_peaks on the current device and
 * `stream` (cudaStream_t, NULL = default): independent dependency chains of
 * each operation on every SM, timed with CUDA events after a warm-up launch,
 * and cooperative latency kernels whose waits are bounded (PSSO_ERR_TIMEOUT
 * if one ran out).  Takes well under a second; allocates 4 KiB for the call;
 * synchronises.  Changes no device setting. */
psso_status psso_microbench(psso_peaks* out, void* stream);

/* Index checks (a debugging build; the paper has no counterpart).  A library
 * compiled with -DPSSO_CHECKED verifies, in every kernel, each index it
 * computes into a buffer -- a particle's row, a unit's range and shared-memory
 * window, an exchange slot, a log entry, a list slot -- before the access; a
 * failed check records (site, index) of the first failure and skips the
 * access (nothing traps).  psso_check_report waits for the device, then sets
 * *site (0 = no failure; otherwise a site number, 2..15, naming the kind of
 * index) and *index (the offending index); with clear != 0 the record is reset.
 * psso_check_selftest enqueues, on `stream`, one failed check of site 1 with
 * the given index and no memory access (it proves the record and report path).
 * Both return PSSO_ERR_UNSUPPORTED in the default build, PSSO_ERR_ARG for a
 * NULL pointer. */
psso_status psso_check_report(int32_t* site, int64_t* index, int32_t clear);
psso_status psso_check_selftest(int64_t index, void* stream);

/* Message for the calling thread's last failed call ("" if none). */
const char* psso_last_error(void);

/* Frees the handle and its device memory.  NULL is ignored. */
void psso_destroy(psso_handle h);

#ifdef __cplusplus
}
#endif

#endif /* PSSO_H */
