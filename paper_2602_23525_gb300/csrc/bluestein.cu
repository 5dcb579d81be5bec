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

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void vec_offsets(const GbBlueIO& b, int64_t v, int64_t* io, int64_t* oo) {
  int64_t a = 0, c = 0;
  for (int d = b.nv - 1; d >= 0; --d) {
    const int64_t q = v / b.vn[d];
    const int64_t i = v - q * b.vn[d];
    v = q;
    a += i * b.vis[d];
    c += i * b.vos[d];
  }
  *io = a;
  *oo = c;
}

__global__ void gb_blue_pre_kernel(const GbBlueIO b) {
  const int64_t total = b.count * b.m;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t v = i / b.m, l = i - (i / b.m) * b.m;
    float2 val = make_float2(0.f, 0.f);
    if (l < b.n) {
      int64_t io, oo;
      vec_offsets(b, v, &io, &oo);
      float2 x = __ldg(b.in + io + l * b.is);
      if (b.conj) x.y = -x.y;
      val = cmul(x, __ldg(b.w + l));
    }
    b.work[i] = val;
  }
}

__global__ void gb_blue_mul_kernel(const GbBlueIO b, float2* data) {
  const int64_t total = b.count * b.m;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const float2 z = cmul(data[i], __ldg(b.B + i % b.m));
    data[i] = make_float2(z.x, -z.y);
  }
}

__global__ void gb_blue_post_kernel(const GbBlueIO b, const float2* data) {
  const int64_t total = b.count * b.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t v = i / b.n, k = i - (i / b.n) * b.n;
    int64_t io, oo;
    vec_offsets(b, v, &io, &oo);
    float2 d = data[v * b.m + k];
    d.y = -d.y;
    float2 y = cmul(d, __ldg(b.w + k));
    if (b.conj) y.y = -y.y;
    b.out[oo + k * b.os] = y;
  }
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
