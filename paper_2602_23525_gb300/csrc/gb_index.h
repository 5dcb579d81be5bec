// gb_index.h -- the exact integer exponent arithmetic behind every twiddle and
// chirp table (sec. 6: accurate twiddles need the exponent of w_N^m reduced
// exactly before the angle is formed; sec. 4.2.5: the Bluestein chirp).
//
// Each function returns the exponent m of the root w_N^m = exp(-2 pi i m / N)
// (or, for the chirp, the q of exp(-pi i q / n)) that one table entry holds.
// Products are formed in unsigned 64-bit integers from operands already
// reduced modulo N, so they are exact for N <= 2^32 (every length this library
// plans fits an int).  The same inline code runs on the device (tables.cu) and
// on the host (fft_twiddle_exponents), which lets the host pin it bit for bit.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define GB_HD __host__ __device__ __forceinline__
#else
#define GB_HD inline
#endif

// (a * b) mod N for 0 <= a, b and N <= 2^32
GB_HD int64_t gb_mulmod(int64_t a, int64_t b, int64_t N) {
  const unsigned long long n = (unsigned long long)N;
  const unsigned long long x = (unsigned long long)a % n, y = (unsigned long long)b % n;
  return (int64_t)((x * y) % n);
}

// root table entry i: w_N^{(i * mult) mod N}  (eq. (1); the two sqrt(N) tables
// of the four-step twiddles use mult = 1 and mult = S)
GB_HD int64_t gb_exp_root(int64_t i, int64_t N, int64_t mult) { return gb_mulmod(i, mult, N); }

// power-of-two stage table [k][4]: entry i = 4k + log2(p), p = 1, 2, 4, 8:
// w_N^{(p k step) mod N} with step = N / (L R); -1 where p >= R (entry is 1)
GB_HD int64_t gb_exp_stage(int64_t i, int64_t N, int64_t L, int R) {
  const int64_t k = i >> 2, p = (int64_t)1 << (i & 3);
  if (p >= R) return -1;
  return gb_mulmod(p * k, N / (L * (int64_t)R), N);
}

// mixed-radix stage table [k][W], W = (R - 1) rounded up to even: entry
// i = k W + r - 1 is w_{L R}^{(r k) mod (L R)}; -1 for the padding entry r = R
GB_HD int64_t gb_exp_full_stage(int64_t i, int64_t L, int R) {
  const int64_t W = R & ~1;
  const int64_t k = i / W, r = i - k * W + 1;
  if (r >= R) return -1;
  return gb_mulmod(r, k, L * (int64_t)R);
}

// four-step post twiddle w_N^{l2 k1} (eq. (2)), k1 = j + q L: table A entry
// i = c L + j is w_N^{(c j) mod N}; table B entry c*4 + t is w_N^{(c L 2^t) mod N}
GB_HD int64_t gb_exp_posttw_a(int64_t i, int64_t N, int64_t L) { return gb_mulmod(i / L, i % L, N); }
GB_HD int64_t gb_exp_posttw_b(int64_t i, int64_t N, int64_t L) {
  return gb_mulmod(i >> 2, L << (i & 3), N);
}

// Bluestein chirp w_k = exp(-pi i (k^2 mod 2n) / n): the exponent k^2 mod 2n
GB_HD int64_t gb_exp_chirp(int64_t k, int64_t n) { return gb_mulmod(k, k, 2 * n); }

// Rader's permutation (sec. 4.2.5): g^e mod p by square-and-multiply
GB_HD int64_t gb_powmod(int64_t g, int64_t e, int64_t p) {
  int64_t r = 1 % p, b = g % p;
  while (e > 0) {
    if (e & 1) r = gb_mulmod(r, b, p);
    b = gb_mulmod(b, b, p);
    e >>= 1;
  }
  return r;
}
