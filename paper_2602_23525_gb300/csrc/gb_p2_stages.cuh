// gb_p2_stages.cuh -- the compile-time power-of-two Stockham stages shared by
// the TMA pass kernels (stockham_pow2.cu) and the cluster kernel (cluster.cu).
//
// n = 2^LOGN, radix schedule 2^(LOGN mod 4) first (when not 1) and 16 after
// (eq. (2) with n1 = L, n2 = R at every stage, auto-sorted output, sec. 2);
// every thread holds 16 values (n/16 threads per transform).  Stage twiddles
// w_{16L}^{r k} come from per-stage tables [k][4] = (w, w^2, w^4, w^8); every
// other power is a product of at most three entries (the small-table scheme
// of sec. 6, never a running recurrence).  Exchange rows are padded,
// phys(i) = i + i/32, with an odd pitch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "codelets.cuh"
#include "gb_pointwise.cuh"

namespace {

template <int LOGN>
struct P2 {
  static constexpr int N = 1 << LOGN;
  static constexpr int REM = LOGN % 4;
  static constexpr int R0 = REM ? (1 << REM) : 16;
  static constexpr int NST = LOGN / 4 + (REM ? 1 : 0);
  static constexpr int TPT = N / 16;
  static constexpr int PITCH = ((N + (N - 1) / 32 + 1) | 1);
  __host__ __device__ static constexpr int radix(int s) { return s == 0 ? R0 : 16; }
  __host__ __device__ static constexpr int L(int s) { return s == 0 ? 1 : R0 << (4 * (s - 1)); }
  // stage s >= 1 table: [k][4] = (w, w^2, w^4, w^8), w = w_{16 L}^k
  __host__ __device__ static constexpr int twoff(int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += L(i) * 4;
    return o;
  }
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int phys(int i) { return i + (i >> 5); }

// barrier of the threads that compute: the whole CTA (NBT = 0), or the first
// NBT threads on named barrier 1 (kernels with a separate control warp)
template <int NBT>
__device__ __forceinline__ void gb_bar() {
  if constexpr (NBT == 0) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"n"(NBT) : "memory");
}

template <int R>
__device__ __forceinline__ void codelet(float2* v);
template <> __device__ __forceinline__ void codelet<2>(float2* v) { gb_dft2(v); }
template <> __device__ __forceinline__ void codelet<4>(float2* v) { gb_dft4(v); }
template <> __device__ __forceinline__ void codelet<8>(float2* v) { gb_dft8(v); }
template <> __device__ __forceinline__ void codelet<16>(float2* v) { gb_dft16(v); }

// the powers w^1..w^15 from (w, w^2) = a and (w^4, w^8) = b, at most three
// products each
__device__ __forceinline__ void powers16v(float2* p, const float4 a, const float4 b) {
  p[1] = make_float2(a.x, a.y);
  p[2] = make_float2(a.z, a.w);
  p[4] = make_float2(b.x, b.y);
  p[8] = make_float2(b.z, b.w);
  p[3] = cmul(p[2], p[1]);
  p[5] = cmul(p[4], p[1]);
  p[6] = cmul(p[4], p[2]);
  p[7] = cmul(p[4], p[3]);
#pragma unroll
  for (int r = 9; r < 16; ++r) p[r] = cmul(p[8], p[r - 8]);
}

__device__ __forceinline__ void powers16(float2* p, const float4* tw) { powers16v(p, __ldg(tw), __ldg(tw + 1)); }

__device__ __forceinline__ void twiddle16(float2* v, const float4* tw) {
  float2 p[16];
  powers16(p, tw);
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], p[r]);
}

// Stage S reads (+ twiddles + butterfly) for butterflies j = u + b*TPT of one
// transform: from its padded exchange row, or (stage 0) from the landed tile
// where element e sits at src[e * ESTRIDE].  TWS: the stage table twt is a
// copy in shared memory (plain loads) instead of the global one (__ldg).
template <int LOGN, int S, bool FROM_TILE, int ESTRIDE, bool TWS = false>
__device__ __forceinline__ void stage_in(float2* v, const float2* src, const float2* __restrict__ twt, int u,
                                         int conj) {
  using C = P2<LOGN>;
  constexpr int R = C::radix(S), B = 16 / R, NB = C::N / R, L = C::L(S);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = u + b * C::TPT;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = j + r * NB;
      float2 x = FROM_TILE ? src[idx * ESTRIDE] : src[phys(idx)];
      if (FROM_TILE && conj) x.y = -x.y;
      v[b * R + r] = x;
    }
    if constexpr (L > 1) {
      static_assert(R == 16, "twiddled stages are radix 16");
      const int k = j & (L - 1);
      const float4* t4 = reinterpret_cast<const float4*>(twt + C::twoff(S) + k * 4);
      if constexpr (TWS) {
        float2 p[16];
        powers16v(p, t4[0], t4[1]);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[b * R + r] = cmul(v[b * R + r], p[r]);
      } else {
        twiddle16(v + b * R, t4);
      }
    }
    codelet<R>(v + b * R);
  }
}

// Stage S writes to the padded exchange row
template <int LOGN, int S>
__device__ __forceinline__ void stage_out_x(const float2* v, float2* dst, int u) {
  using C = P2<LOGN>;
  constexpr int R = C::radix(S), B = 16 / R, L = C::L(S);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = u + b * C::TPT;
    const int k = j & (L - 1);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) dst[phys(base + q * L)] = v[b * R + q];
  }
}

// Last stage writes global memory: output k = j + q*L of the transform goes
// to dst[k * ostride].  POSTTW multiplies output k of column l2 by
// w_N^{l2 k} = A[l2 L + j] * s^q with s = w_N^{l2 L} from B[l2] = (s, s^2, s^4, s^8).
// PW applies the store epilogue e (outputs col + k * e->kstride >= e->K skipped).
// The table entries of the epilogue, for the last stage's outputs of thread u
// (loaded at the start of a tile, so that their latency hides behind the stages).
template <int LOGN>
__device__ __forceinline__ void epi_prefetch(float2* t, const GbP2Epi* e, int u, int64_t col) {
  using C = P2<LOGN>;
  constexpr int S = C::NST - 1;
  constexpr int R = C::radix(S), L = C::L(S);
  static_assert(R == 16, "the epilogue needs a radix-16 last stage");
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int64_t kk = col + (int64_t)(u + q * L) * e->kstride;
    t[q] = kk < e->K ? __ldg(e->tab + kk) : make_float2(0.f, 0.f);
  }
}

template <int LOGN, bool POSTTW, bool PW = false>
__device__ __forceinline__ void stage_out_g(const float2* v, float2* dst, int64_t ostride, int u, int conj,
                                            const float2* __restrict__ A, const float2* __restrict__ Bt,
                                            int64_t col, const GbP2Epi* e = nullptr, const float2* t = nullptr) {
  using C = P2<LOGN>;
  constexpr int S = C::NST - 1;
  constexpr int R = C::radix(S), B = 16 / R, L = C::L(S);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = u + b * C::TPT;  // j < L in the last stage
    float2 p[16];
    float2 a = make_float2(1.f, 0.f);
    if constexpr (POSTTW) {
      static_assert(R == 16, "post twiddles need a radix-16 last stage");
      powers16(p, reinterpret_cast<const float4*>(Bt + col * 4));
      a = __ldg(A + col * L + j);
    }
    if constexpr (PW) static_assert(B == 1, "the epilogue needs a radix-16 last stage");
#pragma unroll
    for (int q = 0; q < R; ++q) {
      float2 x = v[b * R + q];
      if constexpr (POSTTW) x = cmul(x, q == 0 ? a : cmul(a, p[q]));
      if constexpr (PW) {
        if (col + (int64_t)(j + q * L) * e->kstride >= e->K) continue;
        x = gb_epi_apply(e->mode, x, t[q]);  // t: epi_prefetch
      }
      if (conj) x.y = -x.y;
      dst[(int64_t)(j + q * L) * ostride] = x;
    }
  }
}

template <int LOGN, int S, bool POSTTW, bool PW = false, int NBT = 0>
__device__ __forceinline__ void later_stages(float2* v, float2* xrow_j, float2* xrow_s, float2* gout,
                                             int64_t ostride, const float2* __restrict__ twt, int uj, int us,
                                             int conj, bool valid, const float2* A, const float2* Bt, int64_t col,
                                             const GbP2Epi* e = nullptr, const float2* t = nullptr) {
  using C = P2<LOGN>;
  if constexpr (S < C::NST) {
    if constexpr (S == C::NST - 1) {
      // the last stage runs in the store mapping
      stage_in<LOGN, S, false, 1>(v, xrow_s, twt, us, conj);
      if (valid) stage_out_g<LOGN, POSTTW, PW>(v, gout, ostride, us, conj, A, Bt, col, e, t);
    } else {
      stage_in<LOGN, S, false, 1>(v, xrow_j, twt, uj, conj);
      gb_bar<NBT>();
      stage_out_x<LOGN, S>(v, xrow_j, uj);
      gb_bar<NBT>();
      later_stages<LOGN, S + 1, POSTTW, PW, NBT>(v, xrow_j, xrow_s, gout, ostride, twt, uj, us, conj, valid, A, Bt,
                                                 col, e, t);
    }
  }
}

}  // namespace
