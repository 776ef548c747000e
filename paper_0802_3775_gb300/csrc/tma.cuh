// Shared-memory staging helpers of the TMA step kernels: mbarriers with a
// bounded wait, TMA bulk-tensor loads, per-thread cp.async copies,
// proxy fences, and the copy of a grid record into shared memory.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "fdtd_internal.cuh"

namespace fdtd {

__host__ __device__ constexpr size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// Copy a grid record into shared memory (all threads of the block).
template <typename T>
__device__ __forceinline__ void load_record(const StepGrid<T>* g, unsigned char* dst_raw, int tid, int nthreads) {
  const int* src = reinterpret_cast<const int*>(g);
  int* dst = reinterpret_cast<int*>(dst_raw);
  for (int w = tid; w < (int)(sizeof(StepGrid<T>) / 4); w += nthreads) dst[w] = src[w];
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Order this thread's later TMA uses of the 128-byte tensor map at `map`
// after the generic-proxy writes that filled it (a host copy before the
// launch): the map's memory may have held another grid's map before.
__device__ __forceinline__ void tensormap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// try_wait that lets the hardware suspend the thread for up to `ns`
// nanoseconds while the phase is incomplete (instead of spinning).
__device__ __forceinline__ bool mbar_try_wait_for(uint64_t* bar, unsigned parity, unsigned ns) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Limit of a drain wait (the copies a block issued before giving up).
constexpr long long kDrainWaitNs = 2000000000LL;

// Wait for phase `parity` of an mbarrier, giving up after `limit_ns`
// nanoseconds (a grid's bounded-wait limit, 2 s unless set otherwise); a
// limit <= 0 gives up at once, without looking at the barrier (the error
// path's test).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit_ns) {
  if (limit_ns <= 0) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_for(bar, parity, 100000u)) return true;  // suspended up to 0.1 ms per try
    if (global_ns() - t0 > (unsigned long long)limit_ns) return false;
  }
}

// Issued TMA loads of one block, per stage: the producer records every load
// it issues, and a block that gives up waits (bounded) for the loads still in
// flight before it exits, so no copy lands in shared memory after the block
// has left the SM.  Each stage holds at most one load in flight (a stage is
// refilled only after its plane was consumed), and the k-th load into a stage
// completes its barrier's phase k, of parity k & 1.
struct IssuedLoads {
  unsigned used = 0;  // bit s: stage s received a load
  unsigned par = 0;   // bit s: parity of the phase the latest load into stage s completes
  __device__ __forceinline__ void note(int s) {
    par = (used >> s) & 1u ? par ^ (1u << s) : par & ~(1u << s);
    used |= 1u << s;
  }
  // wait for the latest load of every used stage (returns false if one never landed)
  __device__ __forceinline__ bool drain(uint64_t* full, int stages) const {
    bool all = true;
    for (int s = 0; s < stages; ++s)
      if ((used >> s) & 1u) all = mbar_wait(&full[s], (par >> s) & 1u, kDrainWaitNs) && all;
    return all;
  }
};

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}


template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc) {
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
// 8-byte copy of two consecutive binary32 words (both addresses 8-byte aligned).
__device__ __forceinline__ void cp_async_pair(float* smem_dst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor in the
// stream still runs; grid_dependency_wait() returns once the predecessor has
// completed and its writes are visible (at once without the attribute), and
// allow_dependents() lets the successor start early (when every block of this
// grid has called it or exited).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with the programmatic stream-serialization attribute: the kernel
// may become resident while its predecessor finishes and waits for it with
// grid_dependency_wait() before touching memory.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_programmatic(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace fdtd
