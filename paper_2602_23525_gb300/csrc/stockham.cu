// stockham.cu -- the batched Stockham pass kernel (sm_103a).
//
// One CTA computes T transforms of one GbPass tile.  Each stage loads R
// values per butterfly into registers, multiplies by the stage twiddles
// w_{LR}^{rk} (table lookups, sec. 6: precomputed accurate roots), runs the
// generated straight-line radix-R codelet (sec. 5) and writes the R outputs
// to their auto-sorted positions.  The first stage may read global memory
// directly and the last stage may write it directly (coalesced when lanes
// run along the unit-stride index); otherwise the tile moves through shared
// memory with a copy order chosen for coalescing (the buffered copies of
// sec. 3.3).  See gb_pass.h for the index algebra.
#include <cuda_runtime.h>

#include "codelets.cuh"
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
      if (threadIdx.x == 0 && p.status) atomicExch(p.status, 2);
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

template <int MAXT>
__global__ void __launch_bounds__(MAXT)
    gb_stockham_kernel(const GbPass* __restrict__ P, const float2* in, float2* out) {
  extern __shared__ float2 sm[];
  for (int64_t tile = blockIdx.x; tile < P->ntiles; tile += gridDim.x) gb_pass_tile(*P, in, out, sm, tile, 0);
}

// bounded wait until *p >= need (device scope), by %globaltimer
__device__ __forceinline__ bool wait_count(const unsigned long long* p, unsigned long long need,
                                           unsigned long long limit_ns) {
  if (*(volatile const unsigned long long*)p >= need) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (*(volatile const unsigned long long*)p >= need) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
    __nanosleep(200);
  }
}

// Persistent executor: each CTA takes the next item of a device queue ordered
// by step level (every dependency comes earlier in the queue, so a waiting
// CTA only waits for items already taken by running CTAs), waits until the
// segment it depends on has completed, runs the item and counts it done.
// Data written earlier in the same launch is read through L2 (coherent).
template <int MAXT>
__global__ void __launch_bounds__(MAXT) gb_group_kernel(const __grid_constant__ GbGroupArgs a) {
  extern __shared__ float2 sm[];
  __shared__ long long s_item;
  __shared__ int s_fail;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(a.head, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= a.total) return;
    int s = 0;
    while (s + 1 < a.nseg && a.segs[s + 1].first <= item) ++s;
    const GbGroupSeg& g = a.segs[s];
    if (threadIdx.x == 0) {
      int fail = 0;
      if (g.dep >= 0 && !wait_count(a.done + g.dep, (unsigned long long)a.segs[g.dep].ntiles, a.wait_ns)) fail = 1;
      __threadfence();
      s_fail = fail;
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0 && a.status) atomicExch(a.status, 8);  // FFT_ERR_DEVICE_TIMEOUT
      return;
    }
    const int64_t tile = item - g.first;
    float2* src = a.bufs[g.src];
    float2* dst = a.bufs[g.dst];
    const int64_t i0 = tile * GB_SEG_CHUNK;
    switch (g.kind) {
      case GB_SEG_PASS:
        gb_pass_tile(*g.pass, src, dst, sm, tile, 1);
        break;
      case GB_SEG_COPY:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.copy.total; i += blockDim.x)
          gb_copy_elem(g.copy, src, dst, i, 1);
        break;
      case GB_SEG_BLUE_PRE:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.blue.count * g.blue.m; i += blockDim.x)
          gb_blue_pre_elem(g.blue, src, dst, i, 1);
        break;
      case GB_SEG_BLUE_MUL:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.blue.count * g.blue.m; i += blockDim.x)
          gb_blue_mul_elem(g.blue, dst, i);
        break;
      case GB_SEG_BLUE_POST:
        for (int64_t i = i0 + threadIdx.x; i < i0 + GB_SEG_CHUNK && i < g.blue.count * g.blue.n; i += blockDim.x)
          gb_blue_post_elem(g.blue, src, dst, i);
        break;
      default:
        break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(a.done + s, 1ull);
  }
}

__global__ void gb_copy_kernel(const GbCopy c) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.total; i += stride)
    gb_copy_elem(c, c.in, c.out, i, 0);
}

// Rank-0 copy that transposes: dims da (unit input stride) and db (unit
// output stride) are moved through a 32 x 32 shared-memory tile so that both
// the loads (lanes along da) and the stores (lanes along db) coalesce; every
// other dimension is a batch loop.  Tiles are taken grid-stride.
__global__ void __launch_bounds__(256) gb_transpose_kernel(const GbCopy c, int da, int db) {
  __shared__ float2 tile[32][33];
  const int64_t na = c.vn[da], nb = c.vn[db];
  const int64_t ta_n = (na + 31) / 32, tb_n = (nb + 31) / 32;
  const int64_t nrest = c.total / (na * nb);
  const int64_t ntiles = ta_n * tb_n * nrest;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ta = t % ta_n, r1 = t / ta_n, tb = r1 % tb_n;
    int64_t rest = r1 / tb_n, rin = 0, rout = 0;
    for (int d = c.nv - 1; d >= 0; --d) {
      if (d == da || d == db) continue;
      const int64_t q = rest / c.vn[d], k = rest - q * c.vn[d];
      rest = q;
      rin += k * c.vis[d];
      rout += k * c.vos[d];
    }
    const int64_t ia = ta * 32 + tx;
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
      const int64_t ib = tb * 32 + k;
      if (ia < na && ib < nb) tile[k][tx] = __ldg(c.in + rin + ia * c.vis[da] + ib * c.vis[db]);
    }
    __syncthreads();
    const int64_t ib = tb * 32 + tx;
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
      const int64_t ja = ta * 32 + k;
      if (ja < na && ib < nb) c.out[rout + ja * c.vos[da] + ib * c.vos[db]] = tile[tx][k];
    }
    __syncthreads();
  }
}

}  // namespace

int gb_pass_max_smem_optin(void) {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

cudaError_t gb_launch_pass(const GbPass& p, const GbPass* dev, const float2* in, float2* out, int threads,
                           size_t smem, int64_t grid, cudaStream_t st) {
  if (p.ntiles <= 0) return cudaSuccess;
  if (grid <= 0 || grid > p.ntiles) grid = p.ntiles;
  if (grid > 0x7fffffffLL) grid = 0x7fffffffLL;
  cudaError_t e;
  if (threads <= 256) {
    e = cudaFuncSetAttribute(gb_stockham_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_stockham_kernel<256><<<(unsigned)grid, threads, smem, st>>>(dev, in, out);
  } else if (threads <= 512) {
    e = cudaFuncSetAttribute(gb_stockham_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_stockham_kernel<512><<<(unsigned)grid, threads, smem, st>>>(dev, in, out);
  } else {
    e = cudaFuncSetAttribute(gb_stockham_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_stockham_kernel<1024><<<(unsigned)grid, threads, smem, st>>>(dev, in, out);
  }
  return cudaGetLastError();
}

template <int MAXT>
static int group_grid_for(size_t smem) {
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaFuncSetAttribute(gb_group_kernel<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gb_group_kernel<MAXT>, MAXT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * (per_sm > 0 ? per_sm : 1);
}

int gb_group_grid(int threads, size_t smem) {
  if (threads <= 256) return group_grid_for<256>(smem);
  if (threads <= 512) return group_grid_for<512>(smem);
  return group_grid_for<1024>(smem);
}

cudaError_t gb_launch_group(const GbGroupArgs& a, int threads, size_t smem, int64_t grid, cudaStream_t st) {
  if (a.total <= 0) return cudaSuccess;
  if (grid > a.total) grid = a.total;
  if (grid < 1) grid = 1;
  cudaError_t e;
  if (threads <= 256) {
    e = cudaFuncSetAttribute(gb_group_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_group_kernel<256><<<(unsigned)grid, 256, smem, st>>>(a);
  } else if (threads <= 512) {
    e = cudaFuncSetAttribute(gb_group_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_group_kernel<512><<<(unsigned)grid, 512, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(gb_group_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gb_group_kernel<1024><<<(unsigned)grid, 1024, smem, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t gb_launch_copy(const GbCopy& c, cudaStream_t st) {
  if (c.total <= 0) return cudaSuccess;
  // a transposing copy: one dimension is unit-stride on the input side, another
  // on the output side
  int da = -1, db = -1;
  for (int d = 0; d < c.nv; ++d) {
    if (c.vis[d] == 1 && c.vn[d] > 1) da = d;
    if (c.vos[d] == 1 && c.vn[d] > 1) db = d;
  }
  if (da >= 0 && db >= 0 && da != db && c.vn[da] >= 8 && c.vn[db] >= 8) {
    const int64_t tiles = ((c.vn[da] + 31) / 32) * ((c.vn[db] + 31) / 32) * (c.total / (c.vn[da] * c.vn[db]));
    int64_t blocks = tiles < 152 * 8 ? tiles : 152 * 8;
    gb_transpose_kernel<<<(unsigned)blocks, 256, 0, st>>>(c, da, db);
    return cudaGetLastError();
  }
  int64_t blocks = (c.total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  gb_copy_kernel<<<(unsigned)blocks, 256, 0, st>>>(c);
  return cudaGetLastError();
}
