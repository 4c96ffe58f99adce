// Device helpers shared by the kernels of the 3DPIFCM library (sm_103a).
//
// PTX wrappers for mbarrier and the tensor-memory accelerator (TMA), the
// bounded wait every kernel uses, the device status word, and the kernel
// argument blocks.  Nothing here is specific to one kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/pifcm.h"

namespace pifcm {

// Programmatic dependent launch.  A kernel launched by launch_dependent() may
// be scheduled while the kernel before it on the stream is still running; it
// calls grid_dep_wait() before its first access to memory, which returns once
// that kernel has completed and its writes are visible.  grid_dep_trigger()
// lets the next such kernel be scheduled; it takes effect once every CTA of
// the grid has called it or exited, so the grids before it are all resident.
// A stream being captured into a CUDA graph gets ordinary launches: the graph
// already hides the launch latency, and programmatic edges there measured
// slower (whole 165^2 and 285^2 runs 4-6 %), where direct launches gain
// 6-23 %.  Without a programmatic dependency grid_dep_wait() returns at once.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... K, typename... A>
cudaError_t launch_dependent(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  cfg.attrs = at;
  cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

constexpr int kMaxC = 8;            // clusters supported by the kernels
constexpr int kMaxP = 1024;         // particles per swarm / batch

// Device status word layout inside every workspace (first 256 bytes).
struct DevStatus {
  int32_t status;       // first error recorded (an ifcm_status), 0 = OK
  int32_t where;        // diagnostic: which wait / check fired
  int64_t pad;
};

__device__ __forceinline__ void set_status(DevStatus* s, int code, int where) {
  if (atomicCAS(&s->status, 0, code) == 0) s->where = where;
}

// The checked build (-DIFCM_CHECKED): every computed global index of the
// kernels is tested against the extent of its buffer before the access; a
// violation records IFCM_ERR_BOUNDS with the site in the status word and the
// access is skipped (no trap).  In the normal build the test is `true`.
#ifdef IFCM_CHECKED
__device__ __forceinline__ bool check_index(bool ok, DevStatus* s, int where) {
  if (!ok) set_status(s, IFCM_ERR_BOUNDS, where);
  return ok;
}
#define IFCM_CHECK(cond, st, where) ::pifcm::check_index((cond), (st), (where))
#else
#define IFCM_CHECK(cond, st, where) true
#endif

// ---------------------------------------------------------------- PTX glue
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of one phase of an mbarrier (acquire): true once the
// phase has completed.  Unlike try_wait it never suspends the thread, so it
// can be issued well before its result is needed.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Default bound of a wait: about one second.
constexpr uint64_t kWaitLimitNs = 1ull << 30;
// Bounds below this give up at the first unsuccessful non-blocking test
// (the global timer ticks more coarsely than that).
constexpr uint64_t kWaitImmediateNs = 1000;

// Bounded wait on one phase of an mbarrier: a non-blocking test, then
// try_waits (each may suspend the thread for a while) until limit_ns
// nanoseconds of %globaltimer have passed without the phase completing.  It
// then gives up and returns false, so that the caller can record
// IFCM_ERR_TIMEOUT and leave instead of spinning forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_test_wait(bar, parity)) return true;
  if (limit_ns < kWaitImmediateNs) return false;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 >= limit_ns) return false;
  }
}

// 3D / 4D tiled TMA loads into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2),
      "r"(c3)
      : "memory");
}

// ------------------------------------------------------------ warp sums
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// -------------------------------------------------- iteration bookkeeping
// Per-particle state of a batch of IFCM runs (device memory in the workspace).
struct RunState {
  double* centres;      // [P][c]   C^t
  double* J;            // [P]      J of the last finished iteration
  int32_t* active;      // [P]      1 while the run has not stopped
  int32_t* iters;       // [P]      iterations finished
  unsigned long long* updates;  // voxel x iteration updates finished (all P)
};

}  // namespace pifcm
