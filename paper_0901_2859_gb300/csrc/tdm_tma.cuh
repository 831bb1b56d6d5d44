// tdm_tma.cuh -- Tensor Memory Accelerator staging for the solve kernels:
// 2D tensor maps over the right-hand-side matrix, mbarrier completion, and a
// bounded wait that records a device error instead of spinning forever.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

// device error codes written to the plan's error word
enum { kDevErrTmaTimeout = 1, kDevErrNotConverged = 2, kDevErrGroupTimeout = 3 };

// Encode a row-major [rows][cols] tensor with row pitch `ld_bytes` and a box
// of [box_rows][box_cols].  Returns false when the layout cannot be described
// (alignment rules of the copy engine) or the driver entry point is missing.
bool tdm_encode_tma_2d(CUtensorMap* out, const void* base, bool fp64, uint64_t cols, uint64_t rows,
                       uint64_t ld_bytes, uint32_t box_cols, uint32_t box_rows);

__device__ __forceinline__ uint32_t tdm_smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tdm_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tdm_smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tdm_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tdm_smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tdm_tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(tdm_smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(tdm_smem_addr(bar))
      : "memory");
}

// order earlier generic-proxy accesses of shared memory before later async-proxy (TMA) writes
__device__ __forceinline__ void tdm_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Wait for phase `parity` of the barrier.  Each try_wait may suspend the
// thread for up to ~100 us until the phase completes; after `limit` clock
// cycles in total (by default 2^31, about a second) the wait gives up,
// records kDevErrTmaTimeout and returns false.
__device__ __forceinline__ bool tdm_mbar_wait(uint64_t* bar, uint32_t parity, int* err, long long limit = 1ll << 31) {
  const uint32_t addr = tdm_smem_addr(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity), "r"(100000u)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) {
      if (err) atomicExch(err, kDevErrTmaTimeout);
      return false;
    }
  }
}

// Warp 0 waits on the barrier while the other warps sleep in __syncthreads;
// returns false (in every thread) when the wait timed out.
__device__ __forceinline__ bool tdm_mbar_wait_cta(uint64_t* bar, uint32_t parity, int* err, int* flag) {
  if (threadIdx.x < 32) {
    const bool ok = tdm_mbar_wait(bar, parity, err);
    if (threadIdx.x == 0) *flag = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag != 0;
}
