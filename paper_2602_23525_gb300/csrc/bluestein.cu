// bluestein.cu -- pointwise steps of Bluestein's chirp-z algorithm for
// convolution lengths m too large for one CTA (sec. 4.2, "Plans for prime
// sizes").  With w_l = exp(-pi i l^2 / n) and w^{l k} = w_l w_k conj(w_{k-l}):
//   Y[k] = w_k sum_l (x_l w_l) conj(w_{k-l}),
// a length-m circular convolution (m >= 2n - 1) evaluated by FFTs:
//   pre:  a = pad_m(x w)
//   (forward DFT_m of a, planned separately)
//   mul:  Z = conj(A * Bhat),  Bhat = DFT_m(b) / m
//   (forward DFT_m of Z)
//   post: Y[k] = w_k conj(D[k]),  k < n
#include <cuda_runtime.h>

#include "gb_kernels.h"
#include "gb_pointwise.cuh"

namespace {

__global__ void gb_blue_pre_kernel(const GbBlueIO b) {
  const int64_t total = b.count * b.m;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    gb_blue_pre_elem(b, b.in, b.work, i, 0);
}

__global__ void gb_blue_mul_kernel(const GbBlueIO b, float2* data) {
  const int64_t total = b.count * b.m;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    gb_blue_mul_elem(b, data, i);
}

__global__ void gb_blue_post_kernel(const GbBlueIO b, const float2* data) {
  const int64_t total = b.count * b.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    gb_blue_post_elem(b, data, b.out, i);
}

unsigned grid_for(int64_t count) {
  int64_t g = (count + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t gb_launch_blue_pre(const GbBlueIO& b, cudaStream_t st) {
  gb_blue_pre_kernel<<<grid_for(b.count * b.m), 256, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t gb_launch_blue_mul(const GbBlueIO& b, float2* data, cudaStream_t st) {
  gb_blue_mul_kernel<<<grid_for(b.count * b.m), 256, 0, st>>>(b, data);
  return cudaGetLastError();
}

cudaError_t gb_launch_blue_post(const GbBlueIO& b, const float2* data, cudaStream_t st) {
  gb_blue_post_kernel<<<grid_for(b.count * b.n), 256, 0, st>>>(b, data);
  return cudaGetLastError();
}
