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

// The standalone kernels walk transforms along blockIdx.y and the entries of
// one transform along x, so that the offsets of a transform are computed once
// per thread and the entry index needs no 64-bit division (the group
// executor uses the per-element forms of gb_pointwise.cuh instead).
// The pointwise steps take U entries a thread, all loads before the stores,
// so that a thread's round trips to memory overlap (the compiler cannot tell
// that a store does not alias the next entry's loads).
constexpr int kU = 4;

__global__ void gb_blue_pre_kernel(const GbBlueIO b) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x * kU;
  for (int64_t v = blockIdx.y; v < b.count; v += gridDim.y) {
    int64_t io, oo;
    gb_pw_offsets(b, v, &io, &oo);
    const float2* x = b.in + io;
    float2* a = b.work + v * b.m;
    for (int64_t l0 = (int64_t)blockIdx.x * blockDim.x * kU + threadIdx.x; l0 < b.m; l0 += step) {
      float2 xv[kU], wv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t l = l0 + (int64_t)u * blockDim.x;
        xv[u] = wv[u] = make_float2(0.f, 0.f);
        if (l < b.n) {
          xv[u] = __ldg(x + l * b.is);
          wv[u] = __ldg(b.w + l);
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t l = l0 + (int64_t)u * blockDim.x;
        if (l < b.m) {
          if (b.conj) xv[u].y = -xv[u].y;
          a[l] = gb_pw_cmul(xv[u], wv[u]);  // zero beyond n
        }
      }
    }
  }
}

__global__ void gb_blue_mul_kernel(const GbBlueIO b, float2* data) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x * kU;
  for (int64_t v = blockIdx.y; v < b.count; v += gridDim.y) {
    float2* z = data + v * b.m;
    for (int64_t l0 = (int64_t)blockIdx.x * blockDim.x * kU + threadIdx.x; l0 < b.m; l0 += step) {
      float2 zv[kU], bv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t l = l0 + (int64_t)u * blockDim.x;
        if (l < b.m) {
          zv[u] = __ldcg(z + l);
          bv[u] = __ldg(b.B + l);
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t l = l0 + (int64_t)u * blockDim.x;
        if (l < b.m) {
          const float2 p = gb_pw_cmul(zv[u], bv[u]);
          z[l] = make_float2(p.x, -p.y);
        }
      }
    }
  }
}

__global__ void gb_blue_post_kernel(const GbBlueIO b, const float2* data) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.y; v < b.count; v += gridDim.y) {
    int64_t io, oo;
    gb_pw_offsets(b, v, &io, &oo);
    const float2* d = data + v * b.m;
    float2* y = b.out + oo;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b.n; k += step) {
      float2 dv = __ldcg(d + k);
      dv.y = -dv.y;
      float2 r = gb_pw_cmul(dv, __ldg(b.w + k));
      if (b.conj) r.y = -r.y;
      y[k * b.os] = r;
    }
  }
}

// blocks along the transforms (y, one row each while they last) and along
// the entries of a transform (x): about 32 x 152 blocks of 256 threads in
// all, each thread taking several entries of one transform
dim3 grid_for(int64_t count, int64_t len) {
  const int64_t want = 152 * 32;
  int64_t gy = count < 65535 ? count : 65535;
  if (gy < 1) gy = 1;
  int64_t gx = (want + gy - 1) / gy;
  const int64_t most = (len + 255) / 256;
  if (gx > most) gx = most;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)gy);
}

}  // namespace

cudaError_t gb_launch_blue_pre(const GbBlueIO& b, cudaStream_t st) {
  gb_blue_pre_kernel<<<grid_for(b.count, b.m), 256, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t gb_launch_blue_mul(const GbBlueIO& b, float2* data, cudaStream_t st) {
  gb_blue_mul_kernel<<<grid_for(b.count, b.m), 256, 0, st>>>(b, data);
  return cudaGetLastError();
}

cudaError_t gb_launch_blue_post(const GbBlueIO& b, const float2* data, cudaStream_t st) {
  gb_blue_post_kernel<<<grid_for(b.count, b.n), 256, 0, st>>>(b, data);
  return cudaGetLastError();
}
