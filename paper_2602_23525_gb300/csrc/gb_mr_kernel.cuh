// gb_mr_kernel.cuh -- mixed-radix Stockham pass kernel with TMA tiles (sm_103a).
//
// The Stockham stages of eq. (2) (n1 = L, n2 = R at every stage, output
// auto-sorted, sec. 2) for any length n = R_0 R_1 ... with radices 2, 3, 4,
// 5, 7, 8, 9, 11, 13, 16 (and a first stage of one prime 17..61 by the
// generic O(R^2) DFT): the schedule is a run-time parameter, every stage
// switches once (uniformly across the CTA) to the generated straight-line
// codelet of its radix (sec. 5), and each thread keeps at most 16 values per
// stage in registers.  Stage s > 0 multiplies by w_{L R}^{r k} from a full
// per-stage table [k][W], W = R-1 rounded up to even for 128-bit loads
// (sec. 6: accurate precomputed roots, no recurrence); k = j mod L comes from a multiply-high by a precomputed
// reciprocal with one correction step.
//
// Tiles and copies follow the power-of-two kernels (stockham_pow2.cu): a
// persistent CTA computes tiles of T transforms adjacent along the tile
// dimension while one thread keeps the copy engine busy with the next tiles
// (cp.async.bulk for contiguous transforms, a tensor-map box of T columns for
// strided ones, double-buffered on mbarriers whose waits are bounded by
// %globaltimer).  Layouts the copy engine cannot describe (odd lengths with
// odd tile counts, 8-byte-aligned pointers) load the tile with plain
// coalesced loads instead.  The last stage writes global memory directly:
// lanes along the transform (STORE_CONTIG) or across the T transforms
// (STORE_COLS), optionally multiplied by the four-step twiddle w_N^{c k}
// (c = column along the tile dimension) from two sqrt(N) tables.
//
// The kernel templates are instantiated in two translation units by CTA size
// (stockham_mr.cu: 256 threads, stockham_mr512.cu: 512) so they compile in
// parallel; the host logic lives in stockham_mr.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <cstring>
#include <type_traits>

#include "codelets.cuh"
#include "gb_kernels.h"
#include "gb_tma.cuh"

namespace {

__device__ __forceinline__ float2 cmulm(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int physm(int i) { return i + (i >> 5); }

// q = x div d, r = x mod d for x < 2^31 from magic = floor(2^32 / d) (d > 1)
__device__ __forceinline__ void divmod_magic(unsigned x, unsigned d, unsigned magic, unsigned* q, unsigned* r) {
  unsigned qq = __umulhi(x, magic);
  unsigned rr = x - qq * d;
  if (rr >= d) {
    ++qq;
    rr -= d;
  }
  *q = qq;
  *r = rr;
}

template <int R>
__device__ __forceinline__ void mr_codelet(float2* v);
template <> __device__ __forceinline__ void mr_codelet<2>(float2* v) { gb_dft2(v); }
template <> __device__ __forceinline__ void mr_codelet<3>(float2* v) { gb_dft3(v); }
template <> __device__ __forceinline__ void mr_codelet<4>(float2* v) { gb_dft4(v); }
template <> __device__ __forceinline__ void mr_codelet<5>(float2* v) { gb_dft5(v); }
template <> __device__ __forceinline__ void mr_codelet<7>(float2* v) { gb_dft7(v); }
template <> __device__ __forceinline__ void mr_codelet<8>(float2* v) { gb_dft8(v); }
template <> __device__ __forceinline__ void mr_codelet<9>(float2* v) { gb_dft9(v); }
template <> __device__ __forceinline__ void mr_codelet<11>(float2* v) { gb_dft11(v); }
template <> __device__ __forceinline__ void mr_codelet<13>(float2* v) { gb_dft13(v); }
template <> __device__ __forceinline__ void mr_codelet<16>(float2* v) { gb_dft16(v); }

// Where a stage reads its inputs: element e of the thread's transform is at
// src[e * stride] (landing tile) or src[phys(e)] (padded exchange row).
struct Src {
  const float2* p;
  int stride;
  bool padded;
  bool conj;  // conjugate on the way in (backward transforms, stage 0 only)
};

// Stage inputs of butterflies j = u + b*tpt (< nb): R values each, twiddled
// (stage s > 0), through the codelet; kept in v[b*R + r].
template <int R>
__device__ __forceinline__ void stage_in(float2* v, const Src& src, int u, int tpt, int nb, int L, unsigned Lmagic,
                                         const float2* __restrict__ tw) {
  constexpr int BMAX = 16 / R;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int j = u + b * tpt;
    if (j < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = j + r * nb;
        float2 x = src.padded ? src.p[physm(e)] : src.p[e * src.stride];
        if (src.conj) x.y = -x.y;
        v[b * R + r] = x;
      }
      if (L > 1) {
        unsigned q, k;
        divmod_magic((unsigned)j, (unsigned)L, Lmagic, &q, &k);
        constexpr int W = ((R - 1) + 1) & ~1;  // row length, even: 128-bit loads
        const float4* t = reinterpret_cast<const float4*>(tw + k * W);
#pragma unroll
        for (int h = 0; h < W / 2; ++h) {
          const float4 w = __ldg(t + h);
          if (2 * h + 1 < R) v[b * R + 2 * h + 1] = cmulm(v[b * R + 2 * h + 1], make_float2(w.x, w.y));
          if (2 * h + 2 < R) v[b * R + 2 * h + 2] = cmulm(v[b * R + 2 * h + 2], make_float2(w.z, w.w));
        }
      }
      mr_codelet<R>(v + b * R);
    }
  }
}

// output index of value q of butterfly j: (j div L) L R + (j mod L) + q L
__device__ __forceinline__ int out_base(int j, int L, int R, unsigned Lmagic) {
  if (L == 1) return j * R;
  unsigned q, k;
  divmod_magic((unsigned)j, (unsigned)L, Lmagic, &q, &k);
  return (int)(q * (unsigned)(L * R) + k);
}

template <int R>
__device__ __forceinline__ void stage_out_x(const float2* v, float2* row, int u, int tpt, int nb, int L,
                                           unsigned Lmagic) {
  constexpr int BMAX = 16 / R;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int j = u + b * tpt;
    if (j < nb) {
      const int base = out_base(j, L, R, Lmagic);
#pragma unroll
      for (int q = 0; q < R; ++q) row[physm(base + q * L)] = v[b * R + q];
    }
  }
}

// Global destination of one transform's outputs (last stage)
struct Dst {
  float2* p;         // output element 0 of the transform
  int64_t stride;    // between outputs k
  bool conj;
  bool posttw;       // multiply output k by w_N^{col k}
  unsigned col;      // column index along the tile dimension
  const float2* lo;
  const float2* hi;
  unsigned N, S, Smagic;
};

// one output of the last stage to global memory
__device__ __forceinline__ void store_g(const Dst& d, int idx, float2 x) {
  if (d.posttw) {
    const unsigned m = d.col * (unsigned)idx;
    unsigned hi, lo;
    divmod_magic(m, d.S, d.Smagic, &hi, &lo);
    x = cmulm(x, cmulm(__ldg(d.hi + hi), __ldg(d.lo + lo)));
  }
  if (d.conj) x.y = -x.y;
  d.p[(int64_t)idx * d.stride] = x;
}

// Stage 0 of a prime radix R in 17..61 by the generic O(R^2) DFT (sec. 4.2.5,
// eq. (1) in its conjugate-pair form): output q of butterfly j is
//   y_q = x_0 + sum_{r=1}^{(R-1)/2} [c (x_r + x_{R-r}) + i s (x_r - x_{R-r})],
// w_R^{rq} = c + i s.  Each thread computes outputs idx = u + i*tpt (j = idx
// div R, q = idx mod R) from the R inputs of its butterfly; L = 1 at stage 0,
// so no twiddles and output idx lands at position j R + q = idx.
__device__ __noinline__ void generic_stage(const Src& src, float2* xrow, const Dst* dst, int u, int tpt, int n,
                                              int R, const float2* __restrict__ wp, bool valid) {
  const int nb = n / R, h = (R - 1) / 2;
  float2 y[16];
  if (valid) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int idx = u + i * tpt;
      if (idx < n) {
        const int j = idx / R, q = idx - (idx / R) * R;
        auto ld = [&](int e) {
          float2 x = src.padded ? src.p[physm(e)] : src.p[e * src.stride];
          if (src.conj) x.y = -x.y;
          return x;
        };
        float2 acc = ld(j);
        int m = 0;
        for (int r = 1; r <= h; ++r) {
          m += q;
          if (m >= R) m -= R;
          const float2 a = ld(j + r * nb), b = ld(j + (R - r) * nb);
          const float2 w = __ldg(wp + m);
          const float sx = a.x + b.x, sy = a.y + b.y, dx = a.x - b.x, dy = a.y - b.y;
          acc.x = fmaf(w.x, sx, fmaf(-w.y, dy, acc.x));
          acc.y = fmaf(w.x, sy, fmaf(w.y, dx, acc.y));
        }
        y[i] = acc;
      }
    }
  }
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int idx = u + i * tpt;
      if (idx < n) {
        if (dst) store_g(*dst, idx, y[i]);
        else xrow[physm(idx)] = y[i];
      }
    }
  }
}

template <int R, bool UNIT>
__device__ __forceinline__ void stage_out_g(const float2* v, const Dst& d, int u, int tpt, int nb, int L,
                                            unsigned Lmagic) {
  constexpr int BMAX = 16 / R;
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int j = u + b * tpt;
    if (j < nb) {
      const int base = out_base(j, L, R, Lmagic);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int idx = base + q * L;
        float2 x = v[b * R + q];
        if (d.posttw) {
          // m = (col * idx) mod N, col * idx < N for a four-step first pass
          const unsigned m = d.col * (unsigned)idx;
          unsigned hi, lo;
          divmod_magic(m, d.S, d.Smagic, &hi, &lo);
          x = cmulm(x, cmulm(__ldg(d.hi + hi), __ldg(d.lo + lo)));
        }
        if (d.conj) x.y = -x.y;
        if (UNIT) d.p[idx] = x;
        else d.p[(int64_t)idx * d.stride] = x;
      }
    }
  }
}

// one stage of radix R: inputs, (barrier), outputs to the exchange row or to global memory
template <int R>
__device__ __forceinline__ void run_stage(float2* v, const Src& src, float2* xrow, const Dst* dst, int u, int tpt,
                                          int n, int L, unsigned Lmagic, const float2* tw, bool valid, bool sync_mid) {
  const int nb = n / R;
  if (valid) stage_in<R>(v, src, u, tpt, nb, L, Lmagic, tw);
  if (sync_mid) __syncthreads();
  if (valid) {
    if (dst) {
      if (dst->stride == 1) stage_out_g<R, true>(v, *dst, u, tpt, nb, L, Lmagic);
      else stage_out_g<R, false>(v, *dst, u, tpt, nb, L, Lmagic);
    }
    else stage_out_x<R>(v, xrow, u, tpt, nb, L, Lmagic);
  }
}

__device__ __forceinline__ void any_stage(int R, float2* v, const Src& src, float2* xrow, const Dst* dst, int u,
                                          int tpt, int n, int L, unsigned Lmagic, const float2* tw, bool valid,
                                          bool sync_mid) {
  switch (R) {
    case 16: run_stage<16>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 8: run_stage<8>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 4: run_stage<4>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 2: run_stage<2>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 3: run_stage<3>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 9: run_stage<9>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 5: run_stage<5>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 7: run_stage<7>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 11: run_stage<11>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    case 13: run_stage<13>(v, src, xrow, dst, u, tpt, n, L, Lmagic, tw, valid, sync_mid); break;
    default:
      if (sync_mid) __syncthreads();
      break;
  }
}

// A radix schedule fixed at compile time (radices 2..16 of the codelets):
// every stage's radix, L, butterfly count and divisor are constants, so each
// stage is straight-line code for its radix -- no switch over radices, no
// run-time division by L.  Threads per transform as gb_mr_threads.
template <int... RS>
struct MRS {
  static constexpr int NST = sizeof...(RS);
  static constexpr int N = (RS * ...);
  __host__ __device__ static constexpr int radix(int s) {
    constexpr int r[] = {RS...};
    return r[s];
  }
  __host__ __device__ static constexpr int L(int s) {
    int l = 1;
    for (int i = 0; i < s; ++i) l *= radix(i);
    return l;
  }
  __host__ __device__ static constexpr int tpt() {
    int t = 1;
    for (int s = 0; s < NST; ++s) {
      const int R = radix(s), need = (N / R + 16 / R - 1) / (16 / R);
      if (need > t) t = need;
    }
    return t;
  }
  static bool matches(const GbMR& k) {
    if (k.n != N || k.nst != NST || k.tpt != tpt()) return false;
    for (int s = 0; s < NST; ++s)
      if (k.radix[s] != radix(s)) return false;
    return true;
  }
};

// stages S.. of a compile-time schedule from the exchange rows, the last one
// to global memory
template <class SCH, int S>
__device__ __forceinline__ void static_stages(float2* v, float2* xbuf, const Dst& dst, const GbMR& k, int tj, int uj,
                                              bool vj, int ts, int us, bool vs, int64_t cnt) {
  if constexpr (S < SCH::NST) {
    constexpr bool last = S == SCH::NST - 1;
    constexpr int R = SCH::radix(S), L = SCH::L(S);
    constexpr unsigned LM = (unsigned)((1ull << 32) / (unsigned long long)L);
    const int t = last ? ts : tj, u = last ? us : uj;
    const bool ok = (last ? vs : vj) && t < cnt;
    Src sx;
    sx.p = xbuf + t * k.pitch;
    sx.stride = 1;
    sx.padded = true;
    sx.conj = false;
    run_stage<R>(v, sx, xbuf + t * k.pitch, last ? &dst : nullptr, u, SCH::tpt(), SCH::N, L, LM, k.tw[S], ok, true);
    __syncthreads();
    static_stages<SCH, S + 1>(v, xbuf, dst, k, tj, uj, vj, ts, us, vs, cnt);
  }
}

// NT threads per CTA; TMA: 0 plain loads, 1 copy engine; SCH: a compile-time
// radix schedule (MRS) or void (the schedule in k, read at run time)
template <int NT, int LOAD, int STORE, bool POSTTW, class SCH = void>
__global__ void __launch_bounds__(NT, NT <= 256 ? (std::is_void_v<SCH> ? 2 : 3) : 1)
    gb_mr_kernel(const __grid_constant__ GbMR k, const __grid_constant__ CUtensorMap tm, int tma) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float2* land = reinterpret_cast<float2*>(smem_raw + 128);
  // elements per landing buffer, rounded up so that each buffer starts on a
  // 128-byte boundary (tensor-map copies require it)
  const int TL = (k.T * k.land + 15) & ~15;
  float2* xbuf = land + 2 * TL;

  constexpr bool kStatic = !std::is_void_v<SCH>;
  const int tid = threadIdx.x;
  const int T = k.T;
  int tpt = k.tpt, n = k.n;
  if constexpr (kStatic) {
    tpt = SCH::tpt();
    n = SCH::N;
  }
  const int tj = tid / tpt, uj = tid - tj * tpt;  // lanes along a transform
  const int tt = tid % T, ut = tid / T;           // lanes across the transforms
  const bool vj = tj < T, vt = ut < tpt;
  const int t0 = LOAD == GB_P2_LOAD_ROWS ? tt : tj, u0 = LOAD == GB_P2_LOAD_ROWS ? ut : uj;
  const bool v0 = LOAD == GB_P2_LOAD_ROWS ? vt : vj;
  const int ts = STORE == GB_P2_STORE_COLS ? tt : tj, us = STORE == GB_P2_STORE_COLS ? ut : uj;
  const bool vs = STORE == GB_P2_STORE_COLS ? vt : vj;

  const int64_t cblocks = (k.V0 + T - 1) / T;
  const int64_t ntiles = cblocks * k.nb1;
  const int boxr = n < 256 ? n : 256;

  if (tma && tid == 0) {
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto origin = [&](int64_t tile, int64_t* ib, int64_t* ob, int64_t* c0, int64_t* b1) {
    const int64_t cb = tile % cblocks;
    *b1 = tile / cblocks;
    *c0 = cb * T;
    *ib = *b1 * k.vis1 + *c0 * k.vis0;
    *ob = *b1 * k.vos1 + *c0 * k.vos0;
  };

  // thread 0 issues the copies of one tile into landing buffer b
  auto issue = [&](int b, int64_t tile) {
    int64_t ib, ob, c0, b1;
    origin(tile, &ib, &ob, &c0, &b1);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const uint32_t bar = smem_addr(bars + b);
    float2* dst = land + b * TL;
    if (LOAD == GB_P2_LOAD_CONTIG) {
      expect_tx(bar, (uint32_t)(cnt * n * 8));
      if (cnt == 1 || k.vis0 == n) {
        bulk_copy(smem_addr(dst), k.in + ib, (uint32_t)(cnt * n * 8), bar);
      } else {
        for (int64_t i = 0; i < cnt; ++i) bulk_copy(smem_addr(dst + i * n), k.in + ib + i * k.vis0, (uint32_t)(n * 8), bar);
      }
    } else {
      expect_tx(bar, (uint32_t)(T * k.land * 8));
      for (int r0 = 0; r0 < k.land; r0 += boxr)
        tensor_copy_3d(smem_addr(dst + r0 * T), &tm, (int)c0, r0, (int)b1, bar);
    }
  };

  if (tma && tid == 0)
    for (int b = 0; b < 2; ++b) {
      const int64_t tile = blockIdx.x + (int64_t)b * gridDim.x;
      if (tile < ntiles) issue(b, tile);
    }

  float2 v[16];
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = tma ? (it & 1) : 0;
    int64_t ib, ob, c0, b1;
    origin(tile, &ib, &ob, &c0, &b1);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    float2* lb = land + b * TL;
    if (tma) {
      const bool ok = mbar_wait(smem_addr(bars + b), (uint32_t)((it >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        if (tid == 0 && k.status) gb_set_status(k.status, kStatusTimeout);
        return;
      }
    } else {
      // plain coalesced loads (lanes along the unit-stride direction)
      const int total = T * n;
      for (int i = tid; i < total; i += NT) {
        int t, e;
        if (LOAD == GB_P2_LOAD_ROWS) {
          t = i % T;
          e = i / T;
        } else {
          t = i / n;
          e = i - t * n;
        }
        if (t < cnt) {
          const float2 x = k.in[ib + t * k.vis0 + (int64_t)e * k.is];
          if (LOAD == GB_P2_LOAD_ROWS) lb[e * T + t] = x;
          else lb[t * n + e] = x;
        }
      }
      __syncthreads();
    }

    Dst dst;
    dst.p = k.out + ob + (int64_t)ts * k.vos0;
    dst.stride = k.os;
    dst.conj = k.conj != 0;
    dst.posttw = POSTTW;
    dst.col = (unsigned)(c0 + ts);
    dst.lo = k.ptw_lo;
    dst.hi = k.ptw_hi;
    dst.N = k.ptwN;
    dst.S = k.ptwS;
    dst.Smagic = k.ptwSmagic;

    // stage 0 from the landing tile
    Src s0;
    s0.p = LOAD == GB_P2_LOAD_ROWS ? lb + t0 : lb + t0 * n;
    s0.stride = LOAD == GB_P2_LOAD_ROWS ? T : 1;
    s0.padded = false;
    s0.conj = k.conj != 0;
    const bool last0 = k.nst == 1;
    const bool ok0 = v0 && t0 < cnt;
    // one stage: the host builds this only when the load and store mappings agree
    if constexpr (kStatic)
      run_stage<SCH::radix(0)>(v, s0, xbuf + t0 * k.pitch, SCH::NST == 1 ? &dst : nullptr, u0, tpt, n, 1, 0, nullptr,
                               ok0, true);
    else if (k.radix[0] > 16)
      generic_stage(s0, xbuf + t0 * k.pitch, last0 ? &dst : nullptr, u0, tpt, n, k.radix[0], k.wp, ok0);
    else
      any_stage(k.radix[0], v, s0, xbuf + t0 * k.pitch, last0 ? &dst : nullptr, u0, tpt, n, k.L[0], k.Lmagic[0],
                nullptr, ok0, true);
    // the landing buffer is free: refill it with the tile two ahead
    if (tma && tid == 0) {
      const int64_t next = tile + 2 * (int64_t)gridDim.x;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(b, next);
      }
    }
    __syncthreads();
    if constexpr (kStatic) {
      static_stages<SCH, 1>(v, xbuf, dst, k, tj, uj, vj, ts, us, vs, cnt);
    } else {
      for (int s = 1; s < k.nst; ++s) {
        const bool last = s == k.nst - 1;
        const int t = last ? ts : tj, u = last ? us : uj;
        const bool ok = (last ? vs : vj) && t < cnt;
        Src sx;
        sx.p = xbuf + t * k.pitch;
        sx.stride = 1;
        sx.padded = true;
        sx.conj = false;
        any_stage(k.radix[s], v, sx, xbuf + t * k.pitch, last ? &dst : nullptr, u, tpt, n, k.L[s], k.Lmagic[s],
                  k.tw[s], ok, true);
        __syncthreads();
      }
    }
  }
}

template <int NT, int LOAD, int STORE, bool POSTTW, class SCH = void>
cudaError_t launch(const GbMR& k, cudaStream_t st) {
  auto fn = gb_mr_kernel<NT, LOAD, STORE, POSTTW, SCH>;
  const size_t smem = gb_mr_smem(k);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = ((k.V0 + k.T - 1) / k.T) * k.nb1;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (k.grid > 0) grid = k.grid;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;

  // copy-engine eligibility of this launch's pointers and strides
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  int tma = 0;
  const bool aligned = (reinterpret_cast<uintptr_t>(k.in) & 15) == 0;
  if (LOAD == GB_P2_LOAD_CONTIG) {
    const bool adj = k.vis0 == k.n;
    const bool even_rows = (k.n % 2) == 0;
    // every copy starts on a 16-byte boundary and moves a multiple of 16 bytes
    tma = aligned && (k.vis1 % 2) == 0 && (adj ? (even_rows || (k.T % 2 == 0 && k.V0 % 2 == 0)) : (even_rows && k.vis0 % 2 == 0));
  } else {
    PFN_cuTensorMapEncodeTiled_v12000 enc = (PFN_cuTensorMapEncodeTiled_v12000)gb_tensor_map_encoder();
    if (enc && aligned && k.T % 2 == 0 && k.V0 % k.T == 0 && k.vis0 == 1 && k.is > 0 && (k.is % 2) == 0 &&
        (k.nb1 == 1 || (k.vis1 > 0 && (k.vis1 % 2) == 0)) && (k.is * 8) >= k.V0 * 8) {
      const int boxr = k.n < 256 ? k.n : 256;
      cuuint64_t dim[3] = {(cuuint64_t)k.V0, (cuuint64_t)k.n, (cuuint64_t)k.nb1};
      cuuint64_t str[2] = {(cuuint64_t)k.is * 8, (cuuint64_t)(k.nb1 > 1 ? k.vis1 : k.is * k.n) * 8};
      cuuint32_t box[3] = {(cuuint32_t)k.T, (cuuint32_t)boxr, 1};
      cuuint32_t es[3] = {1, 1, 1};
      if (str[1] >= str[0] && str[1] < (cuuint64_t(1) << 40) &&
          enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(k.in), dim, str, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        tma = 1;
    }
  }
  fn<<<(unsigned)grid, NT, smem, st>>>(k, tm, tma);
  return cudaGetLastError();
}

template <int NT, class SCH = void>
cudaError_t dispatch(const GbMR& k, cudaStream_t st) {
  if (k.load == GB_P2_LOAD_CONTIG && k.store == GB_P2_STORE_CONTIG && !k.posttw)
    return launch<NT, GB_P2_LOAD_CONTIG, GB_P2_STORE_CONTIG, false, SCH>(k, st);
  if (k.load == GB_P2_LOAD_CONTIG && k.store == GB_P2_STORE_COLS && !k.posttw)
    return launch<NT, GB_P2_LOAD_CONTIG, GB_P2_STORE_COLS, false, SCH>(k, st);
  if (k.load == GB_P2_LOAD_ROWS && k.store == GB_P2_STORE_CONTIG && !k.posttw)
    return launch<NT, GB_P2_LOAD_ROWS, GB_P2_STORE_CONTIG, false, SCH>(k, st);
  if (k.load == GB_P2_LOAD_ROWS && k.store == GB_P2_STORE_COLS)
    return k.posttw ? launch<NT, GB_P2_LOAD_ROWS, GB_P2_STORE_COLS, true, SCH>(k, st)
                    : launch<NT, GB_P2_LOAD_ROWS, GB_P2_STORE_COLS, false, SCH>(k, st);
  return cudaErrorInvalidValue;
}

}  // namespace

// the kernel launch for CTAs of 256 / 512 threads (one translation unit each)
cudaError_t gb_mr_dispatch_256(const GbMR& k, cudaStream_t st);
cudaError_t gb_mr_dispatch_512(const GbMR& k, cudaStream_t st);
// the compile-time schedules (stockham_mrc.cu): returns 1 and sets *e when
// k's length and schedule are one of them, else 0
int gb_mr_dispatch_static(const GbMR& k, cudaStream_t st, cudaError_t* e);
