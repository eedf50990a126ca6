// Device helpers shared by the step kernels: bounded mbarrier waits, TMA
// (cp.async.bulk.tensor) copies, programmatic dependent launch, per-slot
// counters.  Included by the kernel translation units only.
#pragma once
#include "pedsim_internal.h"

namespace pedsim {

constexpr int kErrTimeout = -110;
// A bounded wait gives up after this many SM clock cycles (about 2 s at the
// 2.07 GHz maximum clock).
constexpr long long kWaitCycles = 4000000000ll;

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and TMA (cp.async.bulk.tensor)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity; false after `limit` SM clock
// cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long limit = kWaitCycles)
{
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Programmatic dependent launch: wait until the preceding kernel in the
// stream has completed and its memory is visible (no-op when the launch did
// not overlap), and let the next kernel start its prologue.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Starts fetching a tensor map (kept in global memory) into the TMA unit's
// descriptor cache, so that the copy issued later does not wait for it.
__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// Shared -> global tiled bulk copy (elements outside the tensor are skipped).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
        "r"(x), "r"(y), "r"(smem_u32(src))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Waits until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copies a scenario's descriptor header into shared memory (16 bytes per
// thread of the first kDescHeaderBytes / 16 threads); the caller
// synchronises.  The copy goes through the read-only path, so only fields
// that no kernel writes may be read from it (not the step index).
__device__ __forceinline__ void load_header(ScenarioDesc *dst, const ScenarioDesc *src)
{
    if (threadIdx.x < kDescHeaderBytes / 16)
        reinterpret_cast<uint4 *>(dst)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint4 *>(src) + threadIdx.x);
}

// Per-thread step counters (moved, conflicts, crossings per group).
struct Counts {
    unsigned moved = 0, conflicts = 0, crossed_a = 0, crossed_b = 0;
};

// Adds the warp's counts to counter slot `slot` of the scenario (warp-shuffle
// reduction; each tile or CTA owns its slot, so the adds never contend).
__device__ __forceinline__ void flush_counts(const ScenarioDesc &d, Counts &c, uint32_t slot)
{
    const unsigned m = __reduce_add_sync(0xffffffffu, c.moved);
    const unsigned k = __reduce_add_sync(0xffffffffu, c.conflicts);
    const unsigned a = __reduce_add_sync(0xffffffffu, c.crossed_a);
    const unsigned b = __reduce_add_sync(0xffffffffu, c.crossed_b);
    if ((threadIdx.x & 31) == 0 && (m | k | a | b)) {
        unsigned long long *ps = d.part + (size_t)slot * kNumCounters;
        if (m) atomicAdd(&ps[kMoved], (unsigned long long)m);
        if (k) atomicAdd(&ps[kConflicts], (unsigned long long)k);
        if (a) atomicAdd(&ps[kCrossedA], (unsigned long long)a);
        if (b) atomicAdd(&ps[kCrossedB], (unsigned long long)b);
    }
    c = Counts{};
}

// Launch that may overlap the previous kernel in the stream (programmatic
// dependent launch); the kernel orders itself with pdl_wait.
template <class... KArgs, class... Args>
static cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                                   unsigned smem, cudaStream_t stream, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <class... KArgs, class... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                              cudaStream_t stream, Args... args)
{
    return launch_pdl_smem(kernel, grid, block, 0u, stream, args...);
}

}  // namespace pedsim
