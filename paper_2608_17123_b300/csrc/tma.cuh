// Tensor-memory-accelerator (TMA) tile loads and their mbarrier, as inline
// PTX for sm_103a (cp.async.bulk.tensor, mbarrier.*). Used for the halo
// window of the level-0 blur: one 2-D box copy per tile, issued by one
// thread, with the zero boundary of the fine blur supplied by the copy's
// out-of-bounds fill.
//
// Rules every caller keeps (checked on the host before a tensor map is made,
// see make_window_map in deblur.cu):
//  * the innermost box coordinate x, times the element size, is a multiple
//    of 16 bytes (x is a multiple of 8 for every element type used here);
//  * the global base is 16-byte aligned and the row pitch a multiple of 16
//    bytes; the box's inner extent is a multiple of 16 bytes;
//  * the shared-memory destination is 128-byte aligned;
//  * only loads are issued (no tensor store or reduce), so a negative start
//    coordinate is allowed.
// Every wait on the mbarrier has a time limit; on expiry the caller records
// an error and waits once more (also bounded) for the copy still in flight
// before it leaves.
#pragma once
#include <cuda.h>
#include "common.cuh"

namespace db {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // the initialised barrier becomes visible to the async proxy (the copy
  // engine completes transactions on it)
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One arrival that also announces `bytes` of transactions to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
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

// Waits until the phase with the given parity has completed, at most
// limit_ns; false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Orders this thread's earlier generic-proxy accesses (and, after an
// acquire, those it has observed from other threads) before its following
// async-proxy accesses of global and shared memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled box load: box {x .. x+box0-1} x {y .. y+box1-1} of the tensor
// described by `map` (in global memory) into shared memory at `dst`
// (row-major in the box: x fastest), completing `bar`'s transactions.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Contiguous bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completing `bar`'s transactions.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

}  // namespace db
