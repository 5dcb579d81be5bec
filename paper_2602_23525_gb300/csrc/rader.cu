// rader.cu -- pointwise steps of Rader's algorithm for prime lengths p
// (sec. 4.2.5, "Plans for prime sizes": a prime-size DFT in O(p log p) time).
//
// With g a generator of the multiplicative group modulo p, every nonzero
// input index is l = g^r and every nonzero output index k = g^{-q}, so
//   Y[0]        = x[0] + sum_{r} x[g^r]
//   Y[g^{-q}]   = x[0] + sum_{r < p-1} x[g^r] w_p^{g^{r-q}},   q < p - 1,
// a cyclic convolution of length p - 1 of a[r] = x[g^r] with
// b[m] = w_p^{g^{-m}}.  It is evaluated by FFTs of a length L: L = p - 1, or
// (zero padding) any L >= 2p - 3, with b extended cyclically at both ends:
//   pre:  a = pad_L(x[perm[r]]),  side[v].x0 = x[0]
//   (forward DFT_L of a, planned separately)
//   mul:  side[v].dc = A[0] (= sum of a);  Z = conj(A Bhat),  Bhat = DFT_L(b) / L
//   (forward DFT_L of Z: conj of the cyclic convolution)
//   post: Y[0] = x0 + dc,  Y[k] = x0 + conj(D[qidx[k]]) for k >= 1
// Backward transforms conjugate the input in pre and the output in post.
#include <cuda_runtime.h>

#include "gb_kernels.h"
#include "gb_pointwise.cuh"

namespace {

__device__ __forceinline__ void rader_offsets(const GbRaderIO& b, int64_t v, int64_t* io, int64_t* oo) {
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

// transforms along blockIdx.y, entries of one transform along x
__global__ void gb_rader_pre_kernel(const GbRaderIO b, float2* work, float2* side) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.y; v < b.count; v += gridDim.y) {
    int64_t io, oo;
    rader_offsets(b, v, &io, &oo);
    const float2* x = b.in + io;
    float2* a = work + v * b.L;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < b.L; r += step) {
      float2 val = make_float2(0.f, 0.f);
      if (r < b.p - 1) {
        val = __ldg(x + (int64_t)__ldg(b.perm + r) * b.is);
        if (b.conj) val.y = -val.y;
      }
      a[r] = val;
      if (r == 0) {
        float2 x0 = __ldg(x);
        if (b.conj) x0.y = -x0.y;
        side[2 * v] = x0;
      }
    }
  }
}

__global__ void gb_rader_mul_kernel(const GbRaderIO b, float2* data, float2* side) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.y; v < b.count; v += gridDim.y) {
    float2* z = data + v * b.L;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < b.L; l += step) {
      const float2 A = __ldcg(z + l);
      if (l == 0) side[2 * v + 1] = A;
      const float2 p = gb_pw_cmul(A, __ldg(b.B + l));
      z[l] = make_float2(p.x, -p.y);
    }
  }
}

__global__ void gb_rader_post_kernel(const GbRaderIO b, const float2* data, const float2* side) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.y; v < b.count; v += gridDim.y) {
    int64_t io, oo;
    rader_offsets(b, v, &io, &oo);
    const float2* d = data + v * b.L;
    const float2 x0 = __ldcg(side + 2 * v);
    float2* y = b.out + oo;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b.p; k += step) {
      float2 r;
      if (k == 0) {
        const float2 dc = __ldcg(side + 2 * v + 1);
        r = make_float2(x0.x + dc.x, x0.y + dc.y);
      } else {
        const float2 c = __ldcg(d + __ldg(b.qidx + k));
        r = make_float2(x0.x + c.x, x0.y - c.y);  // x0 + conj(D[q])
      }
      if (b.conj) r.y = -r.y;
      y[k * b.os] = r;
    }
  }
}

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

cudaError_t gb_launch_rader_pre(const GbRaderIO& b, float2* work, float2* side, cudaStream_t st) {
  gb_rader_pre_kernel<<<grid_for(b.count, b.L), 256, 0, st>>>(b, work, side);
  return cudaGetLastError();
}

cudaError_t gb_launch_rader_mul(const GbRaderIO& b, float2* data, float2* side, cudaStream_t st) {
  gb_rader_mul_kernel<<<grid_for(b.count, b.L), 256, 0, st>>>(b, data, side);
  return cudaGetLastError();
}

cudaError_t gb_launch_rader_post(const GbRaderIO& b, const float2* data, const float2* side, cudaStream_t st) {
  gb_rader_post_kernel<<<grid_for(b.count, b.p), 256, 0, st>>>(b, data, side);
  return cudaGetLastError();
}
