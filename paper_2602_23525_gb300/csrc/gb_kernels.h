// gb_kernels.h -- host-side launchers of the library's CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gb_pass.h"

// Stockham pass (stockham.cu).  p is the host copy of the descriptor, dev its
// device copy (what the kernel reads).  grid <= 0 launches one CTA per tile.
cudaError_t gb_launch_pass(const GbPass& p, const GbPass* dev, const float2* in, float2* out, int threads,
                           size_t smem, int64_t grid, cudaStream_t st);
cudaError_t gb_launch_copy(const GbCopy& c, cudaStream_t st);
int gb_pass_max_smem_optin(void);

// Bluestein helper kernels for convolution lengths beyond one CTA (bluestein.cu).
struct GbBlueIO {
  const float2* in;     // user input, element 0
  float2* out;          // user output, element 0
  float2* work;         // m * count contiguous scratch
  int64_t n, m;         // true length, convolution length
  int64_t is, os;       // transform strides
  int nv;
  int64_t vn[GB_MAX_VDIMS], vis[GB_MAX_VDIMS], vos[GB_MAX_VDIMS];
  int64_t count;        // product of vn
  const float2* w;      // chirp, n entries
  const float2* B;      // Bhat, m entries
  int conj;
};
cudaError_t gb_launch_blue_pre(const GbBlueIO& b, cudaStream_t st);     // work = pad(x w)
cudaError_t gb_launch_blue_mul(const GbBlueIO& b, float2* data, cudaStream_t st);  // data = conj(data Bhat)
cudaError_t gb_launch_blue_post(const GbBlueIO& b, const float2* data, cudaStream_t st);  // y = w conj(data)

// FP64 table generation (tables.cu).
cudaError_t gb_make_roots(float2* out, int64_t count, int64_t N, int64_t mult, cudaStream_t st);
cudaError_t gb_make_chirp(float2* out, int64_t n, cudaStream_t st);
cudaError_t gb_make_bluestein_kernel(float2* out, int64_t n, int64_t m, const int* radices, int nrad,
                                     double2* work, cudaStream_t st);
