// gb_tma.cuh -- TMA bulk copies and mbarrier waits shared by the TMA kernels.
// Every wait is bounded by %globaltimer (kWaitLimitNs); a kernel whose wait
// gives up records kStatusTimeout in its status word and returns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gb_status.cuh"

namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kStatusTimeout = 8;                              // FFT_ERR_DEVICE_TIMEOUT

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for phase `parity` of the mbarrier at `bar`, giving up after limit_ns
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}

// bounded wait for phase `parity` of the mbarrier at `bar`
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, kWaitLimitNs);
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// tiled tensor copy of one box through a tensor map (a __grid_constant__
// kernel parameter); coordinates innermost first, x * element size a
// multiple of 16 bytes, the shared-memory destination on a 128-byte boundary
__device__ __forceinline__ void tensor_copy_4d(uint32_t dst, const void* tmap, int x, int y, int z, int w,
                                               uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

// coordinate of tensor-map dim i (1..3) of a column tile whose rows, first and
// second vector loop sit at the map dims packed in pos (rows | nb1 << 2 | nb2 << 4)
__device__ __forceinline__ int map_coord(int pos, int i, int r0, int b1, int b2) {
  return (pos & 3) == i ? r0 : (((pos >> 2) & 3) == i ? b1 : b2);
}

__device__ __forceinline__ void tensor_copy_3d(uint32_t dst, const void* tmap, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

}  // namespace
