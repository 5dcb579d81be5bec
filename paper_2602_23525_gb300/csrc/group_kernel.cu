// group_kernel.cu -- the persistent executor of several plans in one launch
// (sm_103a): a device queue of (segment, tile) items over the generic pass
// tiles of gb_generic_stages.cuh and the element-wise Bluestein and copy
// steps.  Compiled apart from the pass kernel so the two build in parallel;
// gb_group_grid and gb_launch_group (stockham.cu) call in here.
#include <cuda_runtime.h>

#include "gb_generic_stages.cuh"

namespace {

// bounded wait until *p >= need (device scope), by %globaltimer
__device__ __forceinline__ bool wait_count(const unsigned long long* p, unsigned long long need,
                                           unsigned long long limit_ns) {
  if (*(volatile const unsigned long long*)p >= need) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (*(volatile const unsigned long long*)p >= need) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
    __nanosleep(200);
  }
}

// Persistent executor: each CTA takes the next item of a device queue ordered
// by step level (every dependency comes earlier in the queue, so a waiting
// CTA only waits for items already taken by running CTAs), waits until the
// segment it depends on has completed, runs the item and counts it done.
// Data written earlier in the same launch is read through L2 (coherent).
template <int MAXT>
__global__ void __launch_bounds__(MAXT) gb_group_kernel(const __grid_constant__ GbGroupArgs a) {
  extern __shared__ float2 sm[];
  __shared__ long long s_item;
  __shared__ int s_fail;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.head, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= a.total) return;
    int s = 0;
    while (s + 1 < a.nseg && a.segs[s + 1].first <= item) ++s;
    const GbGroupSeg& g = a.segs[s];
    if (threadIdx.x == 0) {
      int fail = 0;
      if (g.dep >= 0 && !wait_count(a.done + g.dep, (unsigned long long)a.segs[g.dep].ntiles, a.wait_ns)) fail = 1;
      __threadfence();
      s_fail = fail;
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0 && a.status) atomicExch(a.status, 8);  // FFT_ERR_DEVICE_TIMEOUT
      return;
    }
    const int64_t tile = item - g.first;
    float2* src = a.bufs[g.src];
    float2* dst = a.bufs[g.dst];
    const int64_t i0 = tile * GB_SEG_CHUNK;
    switch (g.kind) {
      case GB_SEG_PASS:
        gb_pass_tile(*g.pass, src, dst, sm, tile, 1);
        break;
      case GB_SEG_COPY:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.copy.total; i += blockDim.x)
          gb_copy_elem(g.copy, src, dst, i, 1);
        break;
      case GB_SEG_BLUE_PRE:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.blue.count * g.blue.m; i += blockDim.x)
          gb_blue_pre_elem(g.blue, src, dst, i, 1);
        break;
      case GB_SEG_BLUE_MUL:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.blue.count * g.blue.m; i += blockDim.x)
          gb_blue_mul_elem(g.blue, dst, i);
        break;
      case GB_SEG_BLUE_POST:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.blue.count * g.blue.n; i += blockDim.x)
          gb_blue_post_elem(g.blue, src, dst, i);
        break;
      default:
        break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(a.done + s, 1ull);
  }
}

}  // namespace

template <int MAXT>
static int group_grid_for(size_t smem) {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaFuncSetAttribute(gb_group_kernel<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gb_group_kernel<MAXT>, MAXT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * (per_sm > 0 ? per_sm : 1);
}

int gb_group_kernel_grid(int threads, size_t smem) {
  if (threads <= 256) return group_grid_for<256>(smem);
  if (threads <= 512) return group_grid_for<512>(smem);
  return group_grid_for<1024>(smem);
}

cudaError_t gb_group_kernel_launch(const GbGroupArgs& a, int threads, size_t smem, int64_t grid,
                                   cudaStream_t st) {
  if (a.total <= 0) return cudaSuccess;
  if (grid > a.total) grid = a.total;
  if (grid < 1) grid = 1;
  cudaError_t e;
  if (threads <= 256) {
    e = cudaFuncSetAttribute(gb_group_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_group_kernel<256><<<(unsigned)grid, 256, smem, st>>>(a);
  } else if (threads <= 512) {
    e = cudaFuncSetAttribute(gb_group_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_group_kernel<512><<<(unsigned)grid, 512, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(gb_group_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_group_kernel<1024><<<(unsigned)grid, 1024, smem, st>>>(a);
  }
  return cudaGetLastError();
}
