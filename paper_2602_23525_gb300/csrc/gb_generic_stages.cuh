// gb_generic_stages.cuh -- the stage code of the generic Stockham pass: one
// CTA computes T transforms of one GbPass tile.  Each stage loads R values per
// butterfly into registers, multiplies by the stage twiddles w_{LR}^{rk}
// (table lookups, sec. 6: precomputed accurate roots), runs the generated
// straight-line radix-R codelet (sec. 5) and writes the R outputs to their
// auto-sorted positions.  The first stage may read global memory directly and
// the last stage may write it directly (coalesced when lanes run along the
// unit-stride index); otherwise the tile moves through shared memory with a
// copy order chosen for coalescing (the buffered copies of sec. 3.3).  See
// gb_pass.h for the index algebra.  Shared by the pass kernel (stockham.cu)
// and the persistent group kernel (group_kernel.cu).
#pragma once
#include <cuda_runtime.h>

#include "codelets.cuh"
#include "gb_status.cuh"
#include "gb_kernels.h"
#include "gb_pass.h"
#include "gb_pointwise.cuh"

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// padded shared-memory index: one pad element per 32, breaks power-of-two bank strides
__device__ __forceinline__ int phys(int i) { return i + (i >> 5); }

__device__ __forceinline__ float2 load_c(const float2* p, int conj, int coherent = 0) {
  float2 v = coherent ? __ldcg(p) : __ldg(p);
  if (conj) v.y = -v.y;
  return v;
}

__device__ __forceinline__ void store_c(float2* p, float2 v, int conj) {
  if (conj) v.y = -v.y;
  *p = v;
}

// w_N^m for 0 <= m < N from two sqrt(N)-sized tables (sec. 6)
__device__ __forceinline__ float2 split_twiddle(const GbPass& p, int64_t m) {
  const int64_t hi = m / p.twS;
  const int64_t lo = m - hi * p.twS;
  return cmul(__ldg(p.tw_hi + hi), __ldg(p.tw_lo + lo));
}

template <int R>
__device__ __forceinline__ void codelet(float2* v);
template <> __device__ __forceinline__ void codelet<2>(float2* v) { gb_dft2(v); }
template <> __device__ __forceinline__ void codelet<3>(float2* v) { gb_dft3(v); }
template <> __device__ __forceinline__ void codelet<4>(float2* v) { gb_dft4(v); }
template <> __device__ __forceinline__ void codelet<5>(float2* v) { gb_dft5(v); }
template <> __device__ __forceinline__ void codelet<7>(float2* v) { gb_dft7(v); }
template <> __device__ __forceinline__ void codelet<8>(float2* v) { gb_dft8(v); }
template <> __device__ __forceinline__ void codelet<9>(float2* v) { gb_dft9(v); }
template <> __device__ __forceinline__ void codelet<11>(float2* v) { gb_dft11(v); }
template <> __device__ __forceinline__ void codelet<13>(float2* v) { gb_dft13(v); }
template <> __device__ __forceinline__ void codelet<16>(float2* v) { gb_dft16(v); }

struct TileCtx {
  const float2* in;  // pass input, element 0
  float2* out;       // pass output, element 0
  int coherent;      // 1: data may have been written earlier in this launch (load through L2)
  int t, u;          // transform within the tile, thread within the transform
  bool tvalid;       // this thread's transform exists
  int64_t bin, bout; // element offsets of this thread's transform
  int64_t v0;        // its index along vector dim 0
  int64_t col;       // post-twiddle column: its index along vector dim tw_dim
};

// One Stockham stage (see gb_pass.h).  from_g: stage 0 reads global memory;
// to_g: the last stage writes global memory (applying the post twiddle).
template <int R>
__device__ __forceinline__ void stage(const GbPass& p, int s, float2* sm, const TileCtx& c,
                                      bool from_g, bool to_g) {
  constexpr int BMAX = GB_VALS / R;
  const int nb = p.n / R;
  const int L = p.Ls[s];
  const int step = p.twstep[s];
  float2* smt = sm + c.t * p.pitch;
  float2 v[BMAX][R];
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int j = c.u + b * p.tpt;
    if (c.tvalid && j < nb) {
      if (from_g) {
        const float2* src = c.in + c.bin;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = load_c(src + (int64_t)(j + r * nb) * p.is, p.conj, c.coherent);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = smt[phys(j + r * nb)];
      }
      if (L > 1) {
        const int k = j % L;
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], __ldg(p.tw + r * k * step));
      }
      codelet<R>(v[b]);
    }
  }
  if (!from_g && !to_g) __syncthreads();
#pragma unroll
  for (int b = 0; b < BMAX; ++b) {
    const int j = c.u + b * p.tpt;
    if (c.tvalid && j < nb) {
      const int k = j % L;
      const int base = (j - k) * R + k;  // (j div L) L R + (j mod L)
      if (to_g) {
        float2* dst = c.out + c.bout;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int idx = base + q * L;
          float2 val = v[b][q];
          if (p.post_tw) val = cmul(val, split_twiddle(p, c.col * (int64_t)idx));
          if (p.epi_mode) {
            const int64_t kk = c.v0 + (int64_t)idx * p.epi_kstride;
            if (kk >= p.epi_K) continue;
            val = gb_epi_apply(p.epi_mode, val, __ldg(p.epi_tab + kk));
          }
          store_c(dst + (int64_t)idx * p.os, val, p.conj);
        }
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) smt[phys(base + q * L)] = v[b][q];
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void run_stage(const GbPass& p, int s, float2* sm, const TileCtx& c,
                                          bool from_g, bool to_g) {
  switch (p.radix[s]) {
    case 16: stage<16>(p, s, sm, c, from_g, to_g); break;
    case 8: stage<8>(p, s, sm, c, from_g, to_g); break;
    case 4: stage<4>(p, s, sm, c, from_g, to_g); break;
    case 2: stage<2>(p, s, sm, c, from_g, to_g); break;
    case 3: stage<3>(p, s, sm, c, from_g, to_g); break;
    case 5: stage<5>(p, s, sm, c, from_g, to_g); break;
    case 7: stage<7>(p, s, sm, c, from_g, to_g); break;
    case 9: stage<9>(p, s, sm, c, from_g, to_g); break;
    case 11: stage<11>(p, s, sm, c, from_g, to_g); break;
    case 13: stage<13>(p, s, sm, c, from_g, to_g); break;
    default:
      if (threadIdx.x == 0 && p.status) gb_set_status(p.status, 2);
      break;
  }
}

// tile index -> base offsets of transform 0 of the tile, its dim-0 index and
// its index along vector dim tw_dim (when that is not dim 0)
__device__ __forceinline__ void tile_origin(const GbPass& p, int64_t tile, int64_t* bin,
                                            int64_t* bout, int64_t* v0, int64_t* vtw) {
  int64_t rest = tile / p.tiles0;
  const int64_t i0 = (tile - rest * p.tiles0) * p.T;
  int64_t a = i0 * p.vis[0], b = i0 * p.vos[0];
  *vtw = 0;
  for (int d = p.nv - 1; d >= 1; --d) {
    const int64_t q = rest / p.vn[d];
    const int64_t i = rest - q * p.vn[d];
    rest = q;
    a += i * p.vis[d];
    b += i * p.vos[d];
    if (d == p.tw_dim) *vtw = i;
  }
  *bin = a;
  *bout = b;
  *v0 = i0;
}

__device__ __forceinline__ void tile_index(const GbPass& p, int idx, int order, int* t, int* e) {
  if (order == GB_COPY_ELEM_FAST) {
    *t = idx / p.n;
    *e = idx - *t * p.n;
  } else {
    *t = idx % p.T;
    *e = idx / p.T;
  }
}

__device__ void tile_load(const GbPass& p, const float2* in, float2* sm, int64_t bin, int ntv, int coherent) {
  const int total = p.T * p.n;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int t, e;
    tile_index(p, idx, p.load_copy, &t, &e);
    if (t < ntv)
      sm[t * p.pitch + phys(e)] = load_c(in + bin + t * p.vis[0] + (int64_t)e * p.is, p.conj, coherent);
  }
}

__device__ void tile_store(const GbPass& p, float2* out, const float2* sm, int64_t bout, int64_t v0,
                           int64_t vtw, int ntv) {
  const int total = p.T * p.n;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int t, e;
    tile_index(p, idx, p.store_copy, &t, &e);
    if (t < ntv) {
      float2 val = sm[t * p.pitch + phys(e)];
      if (p.post_tw) val = cmul(val, split_twiddle(p, (p.tw_dim ? vtw : v0 + t) * (int64_t)e));
      if (p.epi_mode) {
        const int64_t kk = v0 + t + (int64_t)e * p.epi_kstride;
        if (kk >= p.epi_K) continue;
        val = gb_epi_apply(p.epi_mode, val, __ldg(p.epi_tab + kk));
      }
      store_c(out + bout + t * p.vos[0] + (int64_t)e * p.os, val, p.conj);
    }
  }
}

// Bluestein (chirp-z) for the whole tile, data kept in shared memory:
// a = x w (zero-padded to m), A = DFT_m(a), Z = conj(A Bhat),
// D = DFT_m(Z), Y[k] = w_k conj(D[k]) for k < bn.
__device__ void bluestein_tile(const GbPass& p, float2* sm, const TileCtx& c, int64_t bin,
                               int64_t bout, int ntv) {
  const int m = p.n;
  const int total = p.T * m;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int t = idx / m, e = idx - (idx / m) * m;
    if (t < ntv) {
      float2 val = make_float2(0.f, 0.f);
      if (e < p.bn)
        val = cmul(load_c(c.in + bin + t * p.vis[0] + (int64_t)e * p.is, p.conj, c.coherent), __ldg(p.bw + e));
      sm[t * p.pitch + phys(e)] = val;
    }
  }
  __syncthreads();
  for (int s = 0; s < p.nst; ++s) run_stage(p, s, sm, c, false, false);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int t = idx / m, e = idx - (idx / m) * m;
    if (t < ntv) {
      float2* q = sm + t * p.pitch + phys(e);
      *q = conjf2(cmul(*q, __ldg(p.bB + e)));
    }
  }
  __syncthreads();
  for (int s = 0; s < p.nst; ++s) run_stage(p, s, sm, c, false, false);
  const int tot_out = p.T * p.bn;
  for (int idx = threadIdx.x; idx < tot_out; idx += blockDim.x) {
    const int t = idx / p.bn, k = idx - (idx / p.bn) * p.bn;
    if (t < ntv) {
      const float2 val = cmul(conjf2(sm[t * p.pitch + phys(k)]), __ldg(p.bw + k));
      store_c(c.out + bout + t * p.vos[0] + (int64_t)k * p.os, val, p.conj);
    }
  }
  __syncthreads();
}

// One tile of a generic pass, computed by the whole CTA (any block size of at
// least T * tpt threads; extra threads idle through the barriers).
__device__ __forceinline__ void gb_pass_tile(const GbPass& p, const float2* in, float2* out, float2* sm, int64_t tile,
                             int coherent) {
  const int tid = threadIdx.x;
  TileCtx c;
  c.in = in;
  c.out = out;
  c.coherent = coherent;
  if (p.t_fast) {
    c.t = tid % p.T;
    c.u = tid / p.T;
  } else {
    c.t = tid / p.tpt;
    c.u = tid - c.t * p.tpt;
  }
  int64_t bin, bout, v0, vtw;
  tile_origin(p, tile, &bin, &bout, &v0, &vtw);
  const int64_t left = p.vn[0] - v0;
  const int ntv = left < p.T ? (int)left : p.T;
  c.tvalid = c.t < ntv && c.u < p.tpt;
  c.bin = bin + c.t * p.vis[0];
  c.bout = bout + c.t * p.vos[0];
  c.v0 = v0 + c.t;
  c.col = p.tw_dim ? vtw : c.v0;
  if (p.blue) {
    bluestein_tile(p, sm, c, bin, bout, ntv);
    return;
  }
  if (p.load_mode == GB_MOVE_SMEM) {
    tile_load(p, in, sm, bin, ntv, coherent);
    __syncthreads();
  }
  for (int s = 0; s < p.nst; ++s) {
    const bool from_g = (s == 0) && p.load_mode == GB_MOVE_DIRECT;
    const bool to_g = (s == p.nst - 1) && p.store_mode == GB_MOVE_DIRECT;
    run_stage(p, s, sm, c, from_g, to_g);
  }
  if (p.store_mode == GB_MOVE_SMEM) {
    tile_store(p, out, sm, bout, v0, vtw, ntv);
    __syncthreads();
  }
}

}  // namespace

// the persistent group kernel (group_kernel.cu): grid size and launch behind
// gb_group_grid and gb_launch_group
int gb_group_kernel_grid(int threads, size_t smem);
cudaError_t gb_group_kernel_launch(const GbGroupArgs& a, int threads, size_t smem, int64_t grid,
                                   cudaStream_t st);
