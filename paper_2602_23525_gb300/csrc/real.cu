// real.cu -- pointwise steps of the DFTs of real data (sec. 5: a real input's
// spectrum is conjugate-symmetric, so about half of the work and of the
// output is redundant; sec. 7: real-data transforms).
//
// Even n = 2m, unit real stride.  The real input read as m complex pairs
// z[j] = x[2j] + i x[2j+1] has the DFT Z = Ze + i Zo, with Ze, Zo the
// (conjugate-symmetric) DFTs of the even and odd samples; eq. (2) with
// n1 = 2 gives X[k] = Ze[k] + w_n^k Zo[k], where
//   Ze[k] = (Z[k] + conj Z[m-k]) / 2,   Zo[k] = (Z[k] - conj Z[m-k]) / (2i),
// and X[m-k] = conj(Ze[k] - w_n^k Zo[k]) for the partner index (Z[m] = Z[0]).
// The backward direction inverts this step: from the half spectrum,
//   W[k] = (X[k] + conj X[m-k]) + i w_n^{-k} (X[k] - conj X[m-k]),  k < m,
// whose unnormalised backward DFT of length m is y[2j] + i y[2j+1] scaled by
// n (the self-conjugate bins X[0], X[m] enter through their real parts).
// Other lengths and layouts widen the real data to complex (promote), or
// extend the half spectrum to the full conjugate-symmetric one (expand) and
// keep the real parts of a full-length backward DFT.
#include <cuda_runtime.h>

#include "gb_kernels.h"
#include "gb_pointwise.cuh"

namespace {

__device__ __forceinline__ void real_offsets(const GbRealIO& r, int64_t v, int64_t* io, int64_t* oo) {
  int64_t a = 0, c = 0;
  for (int d = r.nv - 1; d >= 0; --d) {
    const int64_t q = v / r.vn[d];
    const int64_t i = v - q * r.vn[d];
    v = q;
    a += i * r.vis[d];
    c += i * r.vos[d];
  }
  *io = a;
  *oo = c;
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// pairs (k, m - k), k = 0 .. m/2, of transform v, in place.  A thread takes
// U pairs at once (k, k + blockDim, ...): all their loads before any store,
// so that U round trips to memory overlap instead of following each other
// (the pairs are distinct, but the compiler cannot know that the stores of
// one pair do not alias the loads of the next).
__global__ void gb_r2c_post_kernel(const GbRealIO r, float2* z) {
  constexpr int U = 4;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * U;
  const int64_t pairs = r.m / 2 + 1;
  for (int64_t v = blockIdx.y; v < r.count; v += gridDim.y) {
    int64_t io, oo;
    real_offsets(r, v, &io, &oo);
    float2* y = z + oo;
    for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x; k0 < pairs; k0 += step) {
      float2 a[U], b[U], w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * blockDim.x, kk = r.m - k;
        if (k < pairs) {
          a[u] = y[k * r.os];
          b[u] = kk == r.m ? a[u] : y[kk * r.os];  // Z[m] = Z[0]
          w[u] = __ldg(r.tw + k);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * blockDim.x, kk = r.m - k;
        if (k < pairs) {
          const float2 bc = conjf2(b[u]);
          const float2 ze = make_float2(0.5f * (a[u].x + bc.x), 0.5f * (a[u].y + bc.y));
          // (a - conj b) / (2i) = -i (a - conj b) / 2
          const float2 d = make_float2(a[u].x - bc.x, a[u].y - bc.y);
          const float2 zo = make_float2(0.5f * d.y, -0.5f * d.x);
          const float2 t = gb_pw_cmul(w[u], zo);
          y[k * r.os] = make_float2(ze.x + t.x, ze.y + t.y);
          if (kk != k) y[kk * r.os] = make_float2(ze.x - t.x, -(ze.y - t.y));
        }
      }
    }
  }
}

__global__ void gb_r2c_promote_kernel(const GbRealIO r, const float* x, float2* w) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.y; v < r.count; v += gridDim.y) {
    int64_t io, oo;
    real_offsets(r, v, &io, &oo);
    const float* xi = x + io;
    float2* wo = w + v * r.n;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < r.n; l += step)
      wo[l] = make_float2(__ldg(xi + l * r.is), 0.f);
  }
}

// U entries a thread, all loads before the stores (as in the r2c step)
__global__ void gb_c2r_pre_kernel(const GbRealIO r, const float2* X, float2* w) {
  constexpr int U = 4;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * U;
  for (int64_t v = blockIdx.y; v < r.count; v += gridDim.y) {
    int64_t io, oo;
    real_offsets(r, v, &io, &oo);
    const float2* xi = X + io;
    float2* wo = w + v * r.m;
    for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x * U + threadIdx.x; k0 < r.m; k0 += step) {
      float2 a[U], b[U], tw[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * blockDim.x;
        if (k < r.m) {
          a[u] = __ldg(xi + k * r.is);
          b[u] = conjf2(__ldg(xi + (r.m - k) * r.is));
          tw[u] = __ldg(r.tw + k);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * blockDim.x;
        if (k < r.m) {
          if (k == 0) {  // X[0] and X[m] are self-conjugate: their real parts
            a[u].y = 0.f;
            b[u].y = 0.f;
          }
          const float2 s = make_float2(a[u].x + b[u].x, a[u].y + b[u].y);
          const float2 d = make_float2(a[u].x - b[u].x, a[u].y - b[u].y);
          const float2 t = gb_pw_cmul(conjf2(tw[u]), d);  // w_n^{-k} (a - b)
          wo[k] = make_float2(s.x - t.y, s.y + t.x);      // s + i t
        }
      }
    }
  }
}

__global__ void gb_c2r_expand_kernel(const GbRealIO r, const float2* X, float2* w) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  const int64_t half = r.n / 2;
  for (int64_t v = blockIdx.y; v < r.count; v += gridDim.y) {
    int64_t io, oo;
    real_offsets(r, v, &io, &oo);
    const float2* xi = X + io;
    float2* wo = w + v * r.n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < r.n; k += step) {
      float2 val;
      if (k <= half) {
        val = __ldg(xi + k * r.is);
        if (k == 0 || 2 * k == r.n) val.y = 0.f;  // self-conjugate bins
      } else {
        val = conjf2(__ldg(xi + (r.n - k) * r.is));
      }
      wo[k] = val;
    }
  }
}

__global__ void gb_c2r_real_kernel(const GbRealIO r, const float2* w, float* y) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.y; v < r.count; v += gridDim.y) {
    int64_t io, oo;
    real_offsets(r, v, &io, &oo);
    const float2* wi = w + v * r.n;
    float* yo = y + oo;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < r.n; l += step)
      yo[l * r.os] = __ldcg(wi + l).x;
  }
}

// blocks along the transforms (y) and along one transform's entries (x)
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

cudaError_t gb_launch_r2c_post(const GbRealIO& r, float2* z, cudaStream_t st) {
  gb_r2c_post_kernel<<<grid_for(r.count, r.m / 2 + 1), 256, 0, st>>>(r, z);
  return cudaGetLastError();
}

cudaError_t gb_launch_r2c_promote(const GbRealIO& r, const float* x, float2* w, cudaStream_t st) {
  gb_r2c_promote_kernel<<<grid_for(r.count, r.n), 256, 0, st>>>(r, x, w);
  return cudaGetLastError();
}

cudaError_t gb_launch_c2r_pre(const GbRealIO& r, const float2* X, float2* w, cudaStream_t st) {
  gb_c2r_pre_kernel<<<grid_for(r.count, r.m), 256, 0, st>>>(r, X, w);
  return cudaGetLastError();
}

cudaError_t gb_launch_c2r_expand(const GbRealIO& r, const float2* X, float2* w, cudaStream_t st) {
  gb_c2r_expand_kernel<<<grid_for(r.count, r.n), 256, 0, st>>>(r, X, w);
  return cudaGetLastError();
}

cudaError_t gb_launch_c2r_real(const GbRealIO& r, const float2* w, float* y, cudaStream_t st) {
  gb_c2r_real_kernel<<<grid_for(r.count, r.n), 256, 0, st>>>(r, w, y);
  return cudaGetLastError();
}
