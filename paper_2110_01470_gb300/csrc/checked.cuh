// checked.cuh -- index checks of the checked build.
//
// Compiled with -DPSSO_CHECKED, every kernel verifies the indices it computes
// into its buffers -- a particle's row inside its unit or instance, a unit's
// range and shared-memory window, an exchange slot and rank, a log entry, the
// row a gBest is copied from, a batched particle's instance, a list slot of
// the tensor pipeline -- against the extent of the buffer before the access.
// A failed check records (site, index) of the first failure in a device word
// and the access is skipped; nothing traps, so the context stays usable and
// the host reads the record through psso_check_report.  Loops whose bound is
// the row length of a checked row are covered by that row's check.
//
// The default build compiles every check to `true`.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace psso {

enum ChkSite : uint32_t {
    CHK_NONE = 0,
    CHK_SELFTEST = 1,      // psso_check_selftest
    CHK_UNIT = 2,          // a unit's particle range inside its instance
    CHK_UNIT_SMEM = 3,     // a unit's gBest row / resident state inside dynamic shared memory
    CHK_ROW = 4,           // a particle's entry inside its unit's view
    CHK_SLOT = 5,          // exchange slot and rank of a record or row
    CHK_LOG = 6,           // log ring entry
    CHK_GBEST_SRC = 7,     // entry the gBest row is copied from
    CHK_REFINE = 8,        // entry re-evaluated in FP64 for the arg-min
    CHK_BAT_INST = 9,      // batched: class entry of a flat particle index
    CHK_BAT_ROW = 10,      // batched: particle inside its instance
    CHK_LIST = 11,         // tensor pipeline: list slot below the list's capacity
    CHK_ROT_ROW = 12,      // tensor pipeline: row inside its instance
    CHK_EVAL_ROW = 13,     // psso_evaluate / gradient: row below N
    CHK_ASYNC_ROW = 14,    // asynchronous flow: particle inside its instance
    CHK_TILE = 15          // tensor-core GEMM: tile inside the padded operands
};

#ifdef PSSO_CHECKED
namespace chk {

// First failure of this translation unit: site in bits 48..63, the low 48
// bits of the offending index below.
static __device__ unsigned long long first_fail;

static __device__ __noinline__ void record(uint32_t site, long long index)
{
    const unsigned long long code = ((unsigned long long)site << 48) |
                                    ((unsigned long long)index & 0xffffffffffffull);
    atomicCAS(&first_fail, 0ull, code);
}

__device__ __forceinline__ bool ok(bool cond, uint32_t site, long long index)
{
    if (!cond) record(site, index);
    return cond;
}

// Host side: every translation unit registers a reader of its own word.
using Reader = cudaError_t (*)(unsigned long long* code, bool clear);
void add_reader(Reader r);   // psso_api.cu

namespace {
cudaError_t read_this_unit(unsigned long long* code, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(code, first_fail, sizeof(unsigned long long));
    if (e == cudaSuccess && clear) {
        const unsigned long long z = 0;
        e = cudaMemcpyToSymbol(first_fail, &z, sizeof z);
    }
    return e;
}
struct Registrar {
    Registrar() { add_reader(read_this_unit); }
};
Registrar registrar;
}  // namespace

}  // namespace chk
#define PSSO_CHK(cond, site, index) (::psso::chk::ok((cond), (site), (long long)(index)))
#else
#define PSSO_CHK(cond, site, index) (true)
#endif

// Bytes of dynamic shared memory of the running block.
__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

}  // namespace psso
