// gb_pointwise.cuh -- element operations of Bluestein's algorithm and of the
// rank-0 copy, shared by their standalone kernels and the persistent group
// kernel (sec. 4.2, "Plans for prime sizes" and "Rank-0 plans").
//   pre:  a[v m + l] = x_v[l] w_l for l < n, 0 for n <= l < m
//   mul:  z = conj(z Bhat[i mod m])
//   post: y_v[k] = w_k conj(d[v m + k]) for k < n
#pragma once
#include <cuda_runtime.h>

#include "gb_kernels.h"

__device__ __forceinline__ float2 gb_pw_cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Bluestein's pointwise steps applied to an FFT output y as it is stored
// (the store epilogue of the last pass, table entry t = tab[k]):
//   mode 1 (mul):  conj(y t)          with t = Bhat[k]
//   mode 2 (post): t conj(y)          with t = w_k (forward)
//   mode 3 (post): conj(t conj(y))    (backward: the output conjugated)
__device__ __forceinline__ float2 gb_epi_apply(int mode, float2 y, float2 t) {
  if (mode == 1) {
    const float2 z = gb_pw_cmul(y, t);
    return make_float2(z.x, -z.y);
  }
  const float2 z = gb_pw_cmul(t, make_float2(y.x, -y.y));
  return mode == 3 ? make_float2(z.x, -z.y) : z;
}

__device__ __forceinline__ void gb_pw_offsets(const GbBlueIO& b, int64_t v, int64_t* io, int64_t* oo) {
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

// element i of the padded product a (i < count m); coherent: read through L2
__device__ __forceinline__ void gb_blue_pre_elem(const GbBlueIO& b, const float2* in, float2* work, int64_t i,
                                                 int coherent) {
  const int64_t v = i / b.m, l = i - (i / b.m) * b.m;
  float2 val = make_float2(0.f, 0.f);
  if (l < b.n) {
    int64_t io, oo;
    gb_pw_offsets(b, v, &io, &oo);
    float2 x = coherent ? __ldcg(in + io + l * b.is) : __ldg(in + io + l * b.is);
    if (b.conj) x.y = -x.y;
    val = gb_pw_cmul(x, __ldg(b.w + l));
  }
  work[i] = val;
}

__device__ __forceinline__ void gb_blue_mul_elem(const GbBlueIO& b, float2* data, int64_t i) {
  const float2 z = gb_pw_cmul(__ldcg(data + i), __ldg(b.B + i % b.m));
  data[i] = make_float2(z.x, -z.y);
}

// element i of the outputs (i < count n)
__device__ __forceinline__ void gb_blue_post_elem(const GbBlueIO& b, const float2* data, float2* out, int64_t i) {
  const int64_t v = i / b.n, k = i - (i / b.n) * b.n;
  int64_t io, oo;
  gb_pw_offsets(b, v, &io, &oo);
  float2 d = __ldcg(data + v * b.m + k);
  d.y = -d.y;
  float2 y = gb_pw_cmul(d, __ldg(b.w + k));
  if (b.conj) y.y = -y.y;
  out[oo + k * b.os] = y;
}

__device__ __forceinline__ void gb_copy_elem(const GbCopy& c, const float2* in, float2* out, int64_t i,
                                             int coherent) {
  int64_t r = i, a = 0, b = 0;
  for (int d = c.nv - 1; d >= 0; --d) {
    const int64_t q = r / c.vn[d];
    const int64_t k = r - q * c.vn[d];
    r = q;
    a += k * c.vis[d];
    b += k * c.vos[d];
  }
  out[b] = coherent ? __ldcg(in + a) : __ldg(in + a);
}
