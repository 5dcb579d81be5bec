// tables.cu -- FP64 generation of twiddle and chirp tables on the device.
//
// Sec. 6 of the paper: the O(log n) error growth of Cooley-Tukey holds only
// if the twiddle factors are accurate to about machine precision, so they
// come from precomputed tables, never from trigonometric recurrences.  Here
// every root w_N^m is evaluated in FP64 with the exponent reduced exactly in
// 64-bit integers (m = (i * mult) mod N, chirp exponent k^2 mod 2n) and then
// rounded once to FP32.  FP64 is used for nothing else on the device.
#include <cuda_runtime.h>

#include "gb_kernels.h"

namespace {

// out[i] = w_N^{(i*mult) mod N} = exp(-2 pi i m / N), i < count
__global__ void gb_roots_kernel(float2* out, int64_t count, int64_t N, int64_t mult) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const int64_t m = (int64_t)(((unsigned long long)i * (unsigned long long)mult) % (unsigned long long)N);
    double s, c;
    sincospi(2.0 * (double)m / (double)N, &s, &c);
    out[i] = make_float2((float)c, (float)(-s));
  }
}

// per-stage table [k][4]: w_N^{(p k step) mod N} for p = 1, 2, 4, 8, step = N/(L R)
__global__ void gb_stage_tw_kernel(float2* out, int64_t N, int64_t L, int R) {
  const int64_t total = L * 4;
  const int64_t step = N / (L * R);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t k = i >> 2;
    const int64_t r = (int64_t)1 << (i & 3);
    float2 w = make_float2(1.f, 0.f);
    if (r < R) {
      const int64_t m = (int64_t)(((unsigned long long)(r * k) * (unsigned long long)step) % (unsigned long long)N);
      double s, c;
      sincospi(2.0 * (double)m / (double)N, &s, &c);
      w = make_float2((float)c, (float)(-s));
    }
    out[i] = w;
  }
}

__device__ __forceinline__ float2 root64(int64_t m, int64_t N) {
  double s, c;
  sincospi(2.0 * (double)m / (double)N, &s, &c);
  return make_float2((float)c, (float)(-s));
}

__global__ void gb_posttw_kernel(float2* A, float2* B, int64_t N, int64_t ncols, int64_t L) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t na = ncols * L;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < na + ncols * 4; i += stride) {
    if (i < na) {
      const int64_t c = i / L, j = i - (i / L) * L;
      A[i] = root64((int64_t)(((unsigned long long)c * (unsigned long long)j) % (unsigned long long)N), N);
    } else {
      const int64_t q = i - na, c = q >> 2, p = (int64_t)1 << (q & 3);
      const unsigned long long e = ((unsigned long long)c * (unsigned long long)(L * p)) % (unsigned long long)N;
      B[q] = root64((int64_t)e, N);
    }
  }
}

// full per-stage table [k][W]: w_{L R}^{r k} at [k][r-1] for k < L, r = 1 .. R-1,
// rows of W = R-1 rounded up to even entries (the padding entry is 1)
__global__ void gb_full_stage_tw_kernel(float2* out, int64_t L, int R) {
  const int64_t W = R & ~1;  // (R - 1) rounded up to even
  const int64_t total = L * W;
  const int64_t N = L * R;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t k = i / W, r = i - k * W + 1;
    out[i] = r < R ? root64((int64_t)(((unsigned long long)(r * k)) % (unsigned long long)N), N) : make_float2(1.f, 0.f);
  }
}

// chirp w_k = exp(-pi i (k^2 mod 2n) / n), k < n   (Bluestein)
__global__ void gb_chirp_kernel(float2* out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int64_t q = (int64_t)(((unsigned long long)k * (unsigned long long)k) % (unsigned long long)(2 * n));
    double s, c;
    sincospi((double)q / (double)n, &s, &c);
    out[k] = make_float2((float)c, (float)(-s));
  }
}

// b[j] = conj(w_j) for j < n, b[m - j] = conj(w_j) for 0 < j < n, else 0 (FP64)
__global__ void gb_blue_b_kernel(double2* b, int64_t n, int64_t m) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    int64_t j = -1;
    if (i < n) j = i;
    else if (i > m - n) j = m - i;
    double2 v = make_double2(0.0, 0.0);
    if (j >= 0) {
      const int64_t q = (int64_t)(((unsigned long long)j * (unsigned long long)j) % (unsigned long long)(2 * n));
      double s, c;
      sincospi((double)q / (double)n, &s, &c);
      v = make_double2(c, s);  // conj(exp(-pi i q / n))
    }
    b[i] = v;
  }
}

// One FP64 Stockham stage of radix R on m points (one output per thread):
//   y[(j div L) L R + (j mod L) + t L] = sum_r w_{LR}^{r ((j mod L) + t L)} x[j + r m/R]
__global__ void gb_fft64_stage_kernel(const double2* x, double2* y, int64_t m, int R, int64_t L) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t LR = L * R;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < m; o += stride) {
    const int64_t k = o % L;
    const int64_t rest = o / L;
    const int64_t t = rest % R;
    const int64_t jd = rest / R;
    const int64_t j = jd * L + k;
    const int64_t f = k + t * L;
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < R; ++r) {
      const int64_t e = ((int64_t)r * f) % LR;
      double s, c;
      sincospi(2.0 * (double)e / (double)LR, &s, &c);
      const double2 v = x[j + (int64_t)r * (m / R)];
      // v * (c - i s)
      acc.x += v.x * c + v.y * s;
      acc.y += v.y * c - v.x * s;
    }
    y[o] = acc;
  }
}

__global__ void gb_scale_to_f32_kernel(const double2* x, float2* y, int64_t m, double scale) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    y[i] = make_float2((float)(x[i].x * scale), (float)(x[i].y * scale));
}

unsigned grid_for(int64_t count) {
  int64_t b = (count + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

cudaError_t gb_make_roots(float2* out, int64_t count, int64_t N, int64_t mult, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  gb_roots_kernel<<<grid_for(count), 256, 0, st>>>(out, count, N, mult);
  return cudaGetLastError();
}

cudaError_t gb_make_stage_twiddles(float2* out, int64_t N, int64_t L, int R, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  gb_stage_tw_kernel<<<grid_for(L * 4), 256, 0, st>>>(out, N, L, R);
  return cudaGetLastError();
}

cudaError_t gb_make_full_stage_twiddles(float2* out, int64_t L, int R, cudaStream_t st) {
  if (L <= 0 || R < 2) return cudaSuccess;
  gb_full_stage_tw_kernel<<<grid_for(L * (R & ~1)), 256, 0, st>>>(out, L, R);
  return cudaGetLastError();
}

cudaError_t gb_make_posttw(float2* A, float2* B, int64_t N, int64_t ncols, int64_t L, cudaStream_t st) {
  gb_posttw_kernel<<<grid_for(ncols * (L + 4)), 256, 0, st>>>(A, B, N, ncols, L);
  return cudaGetLastError();
}

cudaError_t gb_make_chirp(float2* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  gb_chirp_kernel<<<grid_for(n), 256, 0, st>>>(out, n);
  return cudaGetLastError();
}

// Bhat = DFT_m(b) / m in FP64, rounded to FP32.  work: 2*m double2.
cudaError_t gb_make_bluestein_kernel(float2* out, int64_t n, int64_t m, const int* radices, int nrad,
                                     double2* work, cudaStream_t st) {
  double2* x = work;
  double2* y = work + m;
  gb_blue_b_kernel<<<grid_for(m), 256, 0, st>>>(x, n, m);
  int64_t L = 1;
  for (int s = 0; s < nrad; ++s) {
    gb_fft64_stage_kernel<<<grid_for(m), 256, 0, st>>>(x, y, m, radices[s], L);
    L *= radices[s];
    double2* t = x;
    x = y;
    y = t;
  }
  gb_scale_to_f32_kernel<<<grid_for(m), 256, 0, st>>>(x, out, m, 1.0 / (double)m);
  return cudaGetLastError();
}
