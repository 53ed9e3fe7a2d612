// Tensor-memory-accelerator (TMA) loads and mbarrier waits for the column
// kernels, in inline PTX (sm_90 and later; built here for sm_103a).
//
// A tile is brought from global memory into shared memory by one thread with
// cp.async.bulk.tensor; the copy signals an mbarrier with its byte count, and
// the consumers wait on that barrier's phase.  Every wait is bounded: after
// about a second (SM clock cycles) it gives up, records UR_DEVERR_TMA_TIMEOUT in
// the error word it is given (the library's device error word) and reports
// failure, so that a kernel can leave without hanging the GPU (ur_sync_status
// turns the word into UR_ERR_TIMEOUT).
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; the encoder is fetched at run time)
#include <stdint.h>

#include "ur_common.cuh"

enum { UR_DEVERR_TMA_TIMEOUT = 1 };

__device__ __forceinline__ uint32_t ur_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ur_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ur_smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async (TMA) proxy
__device__ __forceinline__ void ur_fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void ur_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void ur_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ur_smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool ur_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(ur_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false (and the error word errw
// set) after `limit` SM cycles (default 2^31, about a second).
__device__ __forceinline__ bool ur_mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* errw,
                                                     long long limit = (1ll << 31)) {
  if (ur_mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!ur_mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicOr(errw, UR_DEVERR_TMA_TIMEOUT);
      return false;
    }
  }
  return true;
}

// 2D tiled load of the box at (x, y) (elements; x * element size must be a multiple of 16 bytes)
// into shared memory at dst, completing on bar.
__device__ __forceinline__ void ur_tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(ur_smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(ur_smem_u32(bar))
      : "memory");
}

// Host: encode a 2D tiled tensor map of 8-byte elements: dim0 (contiguous) of d0 elements,
// dim1 of d1 rows at stride1 bytes; box b0 x b1; 128-byte swizzle when swz128.
ur_status ur_tmap_2d_u64(CUtensorMap* out, const void* base, uint64_t d0, uint64_t d1, uint64_t stride1, uint32_t b0,
                         uint32_t b1, bool swz128);
