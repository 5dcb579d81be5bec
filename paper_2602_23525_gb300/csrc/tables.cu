// tables.cu -- FP64 generation of twiddle and chirp tables on the device.
//
// Sec. 6 of the paper: the O(log n) error growth of Cooley-Tukey holds only
// if the twiddle factors are accurate to about machine precision, so they
// come from precomputed tables, never from trigonometric recurrences.  Here
// every root w_N^m is evaluated in FP64 with the exponent reduced exactly in
// 64-bit integers (m = (i * mult) mod N, chirp exponent k^2 mod 2n) and then
// rounded once to FP32.  FP64 is used for nothing else on the device.
#include <cuda_runtime.h>

#include "gb_index.h"
#include "gb_kernels.h"

namespace {

// out[i] = w_N^{(i*mult) mod N} = exp(-2 pi i m / N), i < count
__global__ void gb_roots_kernel(float2* out, int64_t count, int64_t N, int64_t mult) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const int64_t m = gb_exp_root(i, N, mult);
    double s, c;
    sincospi(2.0 * (double)m / (double)N, &s, &c);
    out[i] = make_float2((float)c, (float)(-s));
  }
}

// per-stage table [k][4]: w_N^{(p k step) mod N} for p = 1, 2, 4, 8, step = N/(L R)
__global__ void gb_stage_tw_kernel(float2* out, int64_t N, int64_t L, int R) {
  const int64_t total = L * 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t m = gb_exp_stage(i, N, L, R);
    float2 w = make_float2(1.f, 0.f);
    if (m >= 0) {
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
      A[i] = root64(gb_exp_posttw_a(i, N, L), N);
    } else {
      const int64_t q = i - na;
      B[q] = root64(gb_exp_posttw_b(q, N, L), N);
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
    const int64_t m = gb_exp_full_stage(i, L, R);
    out[i] = m >= 0 ? root64(m, N) : make_float2(1.f, 0.f);
  }
}

// chirp w_k = exp(-pi i (k^2 mod 2n) / n), k < n   (Bluestein)
__global__ void gb_chirp_kernel(float2* out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int64_t q = gb_exp_chirp(k, n);
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
      const int64_t q = gb_exp_chirp(j, n);
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
      const int64_t e = gb_mulmod(r, f, LR);
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

// Rader's b, extended to the convolution length L (FP64): for m < p - 1,
// b[m] = w_p^{ginv^m mod p}; where L > p - 1 the cyclic extension
// b[L - j] = b[p - 1 - j] for 0 < j < p - 1, zeros between
__global__ void gb_rader_b_kernel(double2* b, int64_t p, int64_t ginv, int64_t L) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += stride) {
    int64_t j = -1;
    if (i < p - 1) j = i;
    else if (i > L - (p - 1)) j = i - L + (p - 1);
    double2 v = make_double2(0.0, 0.0);
    if (j >= 0) {
      const int64_t e = gb_powmod(ginv, j, p);
      double s, c;
      sincospi(2.0 * (double)e / (double)p, &s, &c);
      v = make_double2(c, -s);
    }
    b[i] = v;
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

cudaError_t gb_make_rader_kernel(float2* out, int64_t p, int64_t ginv, int64_t L, const int* radices, int nrad,
                                 double2* work, cudaStream_t st) {
  double2* x = work;
  double2* y = work + L;
  gb_rader_b_kernel<<<grid_for(L), 256, 0, st>>>(x, p, ginv, L);
  int64_t Lc = 1;
  for (int s = 0; s < nrad; ++s) {
    gb_fft64_stage_kernel<<<grid_for(L), 256, 0, st>>>(x, y, L, radices[s], Lc);
    Lc *= radices[s];
    double2* t = x;
    x = y;
    y = t;
  }
  gb_scale_to_f32_kernel<<<grid_for(L), 256, 0, st>>>(x, out, L, 1.0 / (double)L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- diagnostics
// The exponent and value of every entry of one table, computed by the same
// code the planner runs, for checking against exact integer arithmetic and
// an FP64 evaluation on the host.

#include "gb_plan.hpp"

namespace {

// exponent of entry i of a table of the given kind (-1: the entry is 1)
int64_t table_exponent(int kind, int64_t N, int64_t a, int64_t b, int64_t i) {
  switch (kind) {
    case FFT_TABLE_ROOTS: return gb_exp_root(i, N, a);
    case FFT_TABLE_STAGE: return gb_exp_stage(i, N, a, (int)b);
    case FFT_TABLE_FULL_STAGE: return gb_exp_full_stage(i, a, (int)b);
    case FFT_TABLE_POSTTW: return i < a * b ? gb_exp_posttw_a(i, N, a) : gb_exp_posttw_b(i - a * b, N, a);
    case FFT_TABLE_CHIRP: return gb_exp_chirp(i, N);
    case FFT_TABLE_RADER: return gb_powmod(a, i, N);
    default: return -2;
  }
}

// arguments of a table: its size, or -1 when they do not describe one
int64_t table_size(int kind, int64_t N, int64_t a, int64_t b) {
  const int64_t lim = (int64_t)1 << 31;
  if (N < 1 || N > lim) return -1;
  switch (kind) {
    case FFT_TABLE_ROOTS: return a >= 0 ? -2 : -1;  // any count
    case FFT_TABLE_STAGE:
      return (a >= 1 && b >= 2 && b <= 16 && N % (a * b) == 0) ? 4 * a : -1;
    case FFT_TABLE_FULL_STAGE:
      return (a >= 1 && b >= 2 && b <= 64 && N == a * b) ? a * (b & ~1) : -1;
    case FFT_TABLE_POSTTW: return (a >= 1 && b >= 1 && a * b <= lim) ? b * (a + 4) : -1;
    case FFT_TABLE_CHIRP: return N;  // 2N <= 2^32 keeps k^2 mod 2N exact
    case FFT_TABLE_RADER: return (a >= 1 && a < N) ? -2 : -1;
    default: return -1;
  }
}

}  // namespace

extern "C" int fft_twiddle_exponents(int kind, int64_t N, int64_t a, int64_t b, int64_t count, int64_t* out) {
  // the first `count` entries of the table (count <= its size)
  const int64_t sz = table_size(kind, N, a, b);
  if (sz == -1 || count < 0 || (sz >= 0 && count > sz) || (count > 0 && !out))
    return gb::set_err(FFT_ERR_INVALID_ARG);
  for (int64_t i = 0; i < count; ++i) out[i] = table_exponent(kind, N, a, b, i);
  return gb::set_err(FFT_OK);
}

extern "C" int fft_twiddle_table(int kind, int64_t N, int64_t a, int64_t b, int64_t count, void* dev_out,
                                 void* stream) {
  const int64_t sz = table_size(kind, N, a, b);
  if (kind == FFT_TABLE_RADER || sz == -1 || count < 0 || (sz >= 0 && count != sz) || (count > 0 && !dev_out))
    return gb::set_err(FFT_ERR_INVALID_ARG);
  if (count == 0) return gb::set_err(FFT_OK);
  float2* o = (float2*)dev_out;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case FFT_TABLE_ROOTS: e = gb_make_roots(o, count, N, a, st); break;
    case FFT_TABLE_STAGE: e = gb_make_stage_twiddles(o, N, a, (int)b, st); break;
    case FFT_TABLE_FULL_STAGE: e = gb_make_full_stage_twiddles(o, a, (int)b, st); break;
    case FFT_TABLE_POSTTW: e = gb_make_posttw(o, o + a * b, N, b, a, st); break;
    case FFT_TABLE_CHIRP: e = gb_make_chirp(o, N, st); break;
    default: return gb::set_err(FFT_ERR_INVALID_ARG);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return gb::set_err(FFT_ERR_CUDA);
  }
  return gb::set_err(FFT_OK);
}
