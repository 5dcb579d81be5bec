// tc.cu -- radix-16 Stockham stages on the tensor cores (sm_103a).
//
// A radix-16 stage applies the 16-point DFT matrix F (F[s][r] = w_16^{r s},
// eq. (1)) to every butterfly after the stage twiddles.  Here a warp takes 16
// butterflies at a time as the rows of X (16 x 16, butterfly x point) and
// computes Y = X F^T with mma.sync.m16n8k16 (two output halves of 8), complex
// arithmetic as four real products:
//   Y_re = X_re F_re^T + X_im (-F_im)^T,   Y_im = X_re F_im^T + X_im F_re^T,
// operands rounded to FP16 or BF16, accumulation in FP32.  Twiddles are
// applied in FP32 before the rounding (table of (w, w^2, w^4, w^8), as in
// the FP32 kernels).  The split variants write every operand as hi + lo
// (hi = round(v), lo = round(v - hi)) and accumulate
// hi*hi + hi*lo + lo*hi, recovering about twice the operand precision.
// With F as the B operand, the output columns a thread holds are the same
// point indices as the input columns it loaded, so each butterfly's data
// stays with the same four lanes from load to store.
//
// Tiles move as in stockham_pow2.cu: TMA bulk copies double-buffered on
// mbarriers (bounded waits) into a persistent CTA, contiguous transforms
// (LOAD_CONTIG) or T adjacent columns (LOAD_ROWS), stores contiguous or
// column-wise.  Sizes: 2^8 and 2^12 points (all stages radix 16).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gb_kernels.h"
#include "gb_tma.cuh"

namespace {

// w_16^m = C16[m] + i S16[m]
__constant__ float C16[16] = {1.0f, 0.9238795325112867f, 0.7071067811865476f, 0.38268343236508984f, 0.0f, -0.3826834323650897f, -0.7071067811865475f, -0.9238795325112867f, -1.0f, -0.9238795325112868f, -0.7071067811865477f, -0.38268343236509034f, 0.0f, 0.38268343236509f, 0.7071067811865474f, 0.9238795325112865f};
__constant__ float S16[16] = {0.0f, -0.3826834323650898f, -0.7071067811865475f, -0.9238795325112867f, -1.0f, -0.9238795325112867f, -0.7071067811865476f, -0.3826834323650899f, 0.0f, 0.38268343236508967f, 0.7071067811865475f, 0.9238795325112865f, 1.0f, 0.9238795325112866f, 0.7071067811865477f, 0.3826834323650904f};

template <int LOGN>
struct TC {
  static constexpr int N = 1 << LOGN;
  static constexpr int NST = LOGN / 4;
  static constexpr int NBF = N / 16;  // butterflies per transform and stage
  static constexpr int PITCH = ((N + (N - 1) / 32 + 1) | 1);
  __host__ __device__ static constexpr int L(int s) { return 1 << (4 * s); }
  __host__ __device__ static constexpr int twoff(int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += L(i) * 4;
    return o;
  }
};

__device__ __forceinline__ int phys(int i) { return i + (i >> 5); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// operand rounding: PREC 1/3 = FP16, 2/4 = BF16; 3/4 split into hi + lo
template <int PREC>
__device__ __forceinline__ uint32_t pack(float a, float b) {
  if constexpr (PREC == 1 || PREC == 3) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

template <int PREC>
__device__ __forceinline__ float2 unpack(uint32_t u) {
  if constexpr (PREC == 1 || PREC == 3) {
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
  } else {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(h);
  }
}

// hi and lo words of the pair (a, b)
template <int PREC>
__device__ __forceinline__ void pack_split(float a, float b, uint32_t* hi, uint32_t* lo) {
  *hi = pack<PREC>(a, b);
  const float2 h = unpack<PREC>(*hi);
  *lo = pack<PREC>(a - h.x, b - h.y);
}

template <int PREC>
__device__ __forceinline__ void mma(float* d, const uint32_t* a, const uint32_t* b) {
  if constexpr (PREC == 1 || PREC == 3) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
}

// The DFT matrix as B operands (F^T, 16 x 8 per output half h): lane (g, t4)
// holds rows 2t4, 2t4+1 (word 0) and 2t4+8, 2t4+9 (word 1) of column 8h+g.
template <int PREC>
struct FragF {
  uint32_t re[2][2], im[2][2], nim[2][2];           // hi (or only) words
  uint32_t re_l[2][2], im_l[2][2], nim_l[2][2];     // lo words (split)
  __device__ void init(int g, int t4) {
    constexpr bool split = PREC >= 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = 8 * h + g;
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int r0 = 2 * t4 + 8 * w, r1 = r0 + 1;
        const int m0 = (r0 * s) & 15, m1 = (r1 * s) & 15;
        if (split) {
          pack_split<PREC>(C16[m0], C16[m1], &re[h][w], &re_l[h][w]);
          pack_split<PREC>(S16[m0], S16[m1], &im[h][w], &im_l[h][w]);
          pack_split<PREC>(-S16[m0], -S16[m1], &nim[h][w], &nim_l[h][w]);
        } else {
          re[h][w] = pack<PREC>(C16[m0], C16[m1]);
          im[h][w] = pack<PREC>(S16[m0], S16[m1]);
          nim[h][w] = pack<PREC>(-S16[m0], -S16[m1]);
        }
      }
    }
  }
};

// w^e for e in {2t4, 2t4+1, 2t4+8, 2t4+9} from the (w, w^2, w^4, w^8) table entry
__device__ __forceinline__ void lane_powers(const float4* tw, int t4, float2* p) {
  const float4 a = __ldg(tw), b = __ldg(tw + 1);
  const float2 w1 = make_float2(a.x, a.y), w2 = make_float2(a.z, a.w);
  const float2 w4 = make_float2(b.x, b.y), w8 = make_float2(b.z, b.w);
  float2 e = make_float2(1.f, 0.f);
  if (t4 & 1) e = w2;
  if (t4 & 2) e = cmul(e, w4);
  p[0] = e;
  p[1] = cmul(e, w1);
  p[2] = cmul(e, w8);
  p[3] = cmul(p[1], w8);
}

// One tensor-core radix-16 stage for the 256 butterflies of a tile (8 warps x
// 32).  Loads + twiddles + MMAs happen before the caller's barrier (via
// stage_mma), the stores after it (stage_store).
template <int LOGN, int PREC>
struct Stage {
  float yre[2][2][4], yim[2][2][4];  // [group][output half][fragment]

  // src(t, e) gives the address of element e of tile transform t
  template <int S, typename Src>
  __device__ __forceinline__ void load_mma(const Src& src, const float2* __restrict__ twt, const FragF<PREC>& F,
                                           int w, int g, int t4, int conj) {
    using C = TC<LOGN>;
    constexpr int L = C::L(S);
    constexpr bool split = PREC >= 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float2 x[2][4];  // [row: g, g+8][point: 2t4, 2t4+1, 2t4+8, 2t4+9]
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int G = 32 * w + 16 * q + g + 8 * hr;
        const int t = G / C::NBF, j = G % C::NBF;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = 2 * t4 + (i & 1) + 8 * (i >> 1);
          float2 v = src(t, j + r * C::NBF);
          if (S == 0 && conj) v.y = -v.y;
          x[hr][i] = v;
        }
        if constexpr (L > 1) {
          float2 p[4];
          lane_powers(reinterpret_cast<const float4*>(twt + C::twoff(S) + (j & (L - 1)) * 4), t4, p);
#pragma unroll
          for (int i = 0; i < 4; ++i) x[hr][i] = cmul(x[hr][i], p[i]);
        }
      }
      // A fragments: word 0 = row g points (2t4, 2t4+1), word 1 = row g+8, words 2/3 = points +8
      uint32_t ar[4], ai[4], arl[4], ail[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int hr = k & 1, i0 = (k >> 1) * 2;
        if (split) {
          pack_split<PREC>(x[hr][i0].x, x[hr][i0 + 1].x, &ar[k], &arl[k]);
          pack_split<PREC>(x[hr][i0].y, x[hr][i0 + 1].y, &ai[k], &ail[k]);
        } else {
          ar[k] = pack<PREC>(x[hr][i0].x, x[hr][i0 + 1].x);
          ai[k] = pack<PREC>(x[hr][i0].y, x[hr][i0 + 1].y);
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float* dr = yre[q][h];
        float* di = yim[q][h];
#pragma unroll
        for (int i = 0; i < 4; ++i) dr[i] = di[i] = 0.f;
        mma<PREC>(dr, ar, F.re[h]);
        mma<PREC>(dr, ai, F.nim[h]);
        mma<PREC>(di, ar, F.im[h]);
        mma<PREC>(di, ai, F.re[h]);
        if (split) {
          mma<PREC>(dr, arl, F.re[h]);
          mma<PREC>(dr, ar, F.re_l[h]);
          mma<PREC>(dr, ail, F.nim[h]);
          mma<PREC>(dr, ai, F.nim_l[h]);
          mma<PREC>(di, arl, F.im[h]);
          mma<PREC>(di, ar, F.im_l[h]);
          mma<PREC>(di, ail, F.re[h]);
          mma<PREC>(di, ai, F.re_l[h]);
        }
      }
    }
  }

  // dst(t, idx) gives the address of output idx of tile transform t
  template <int S, typename Dst>
  __device__ __forceinline__ void store(const Dst& dst, int w, int g, int t4, int conj, bool last,
                                        int64_t valid_T) {
    using C = TC<LOGN>;
    constexpr int L = C::L(S);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int row = g + 8 * (f >> 1);
          const int s = 8 * h + 2 * t4 + (f & 1);
          const int G = 32 * w + 16 * q + row;
          const int t = G / C::NBF, j = G % C::NBF;
          const int k = j & (L - 1);
          const int idx = (j - k) * 16 + k + s * L;
          float2 v = make_float2(yre[q][h][f], yim[q][h][f]);
          if (last) {
            if (t >= valid_T) continue;
            if (conj) v.y = -v.y;
          }
          *dst(t, idx) = v;
        }
  }
};

template <int LOGN, int PREC, int LOAD, int STORE>
__global__ void __launch_bounds__(256, 1) gb_tc_kernel(const __grid_constant__ GbP2 k) {
  using C = TC<LOGN>;
  constexpr int T = (LOAD == GB_P2_LOAD_CONTIG && STORE == GB_P2_STORE_CONTIG) ? 4096 / C::N : 16;
  static_assert(T * C::NBF == 256, "a tile is 256 butterflies");
  constexpr int TILE = T * C::N;
  constexpr int NBUF = 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float2* ibuf = reinterpret_cast<float2*>(smem_raw + 128);
  float2* xbuf = ibuf + NBUF * TILE;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  FragF<PREC> F;
  F.init(g, t4);
  const int64_t cblocks = (k.V0 + T - 1) / T;
  const int64_t ntiles = cblocks * k.nb1 * k.nb2;
  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto origin = [&](int64_t tile, int64_t* ib, int64_t* ob, int64_t* c0) {
    const int64_t cb = tile % cblocks, r = tile / cblocks;
    const int64_t b1 = r % k.nb1, b2 = r / k.nb1;
    *c0 = cb * T;
    *ib = b1 * k.vis1 + b2 * k.vis2 + *c0 * k.vis0;
    *ob = b1 * k.vos1 + b2 * k.vos2 + *c0 * k.vos0;
  };
  auto issue = [&](int b, int64_t tile) {
    int64_t ib, ob, c0;
    origin(tile, &ib, &ob, &c0);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const uint32_t bar = smem_addr(bars + b);
    float2* dst = ibuf + b * TILE;
    if (LOAD == GB_P2_LOAD_CONTIG) {
      if (lane == 0) expect_tx(bar, (uint32_t)(cnt * C::N * 8));
      __syncwarp();
      if (k.vis0 == C::N) {
        if (lane == 0) bulk_copy(smem_addr(dst), k.in + ib, (uint32_t)(cnt * C::N * 8), bar);
      } else {
        for (int64_t i = lane; i < cnt; i += 32)
          bulk_copy(smem_addr(dst + i * C::N), k.in + ib + i * k.vis0, (uint32_t)(C::N * 8), bar);
      }
    } else {
      if (lane == 0) expect_tx(bar, (uint32_t)(C::N * T * 8));
      __syncwarp();
      for (int e = lane; e < C::N; e += 32)
        bulk_copy(smem_addr(dst + e * T), k.in + ib + (int64_t)e * k.is, (uint32_t)(T * 8), bar);
    }
  };
  if (tid < 32)
    for (int b = 0; b < NBUF; ++b) {
      const int64_t tile = blockIdx.x + (int64_t)b * gridDim.x;
      if (tile < ntiles) issue(b, tile);
    }
  Stage<LOGN, PREC> st;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it % NBUF;
    const bool ok = mbar_wait(smem_addr(bars + b), (uint32_t)((it / NBUF) & 1));
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && k.status) atomicExch(k.status, kStatusTimeout);
      return;
    }
    int64_t ib, ob, c0;
    origin(tile, &ib, &ob, &c0);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const float2* tb = ibuf + b * TILE;
    auto tile_src = [&](int t, int e) -> float2 {
      return LOAD == GB_P2_LOAD_CONTIG ? tb[t * C::N + e] : tb[e * T + t];
    };
    auto x_src = [&](int t, int e) -> float2 { return xbuf[t * C::PITCH + phys(e)]; };
    auto x_dst = [&](int t, int e) -> float2* { return xbuf + t * C::PITCH + phys(e); };
    auto g_dst = [&](int t, int e) -> float2* {
      return k.out + ob + (int64_t)t * k.vos0 + (STORE == GB_P2_STORE_COLS ? (int64_t)e * k.os : (int64_t)e);
    };
    st.template load_mma<0>(tile_src, k.twt, F, w, g, t4, k.conj);
    __syncthreads();  // tile buffer read; previous tile's exchange reads done
    if (tid < 32) {
      const int64_t next = tile + (int64_t)NBUF * gridDim.x;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(b, next);
      }
    }
    st.template store<0>(x_dst, w, g, t4, k.conj, false, T);
    __syncthreads();
    st.template load_mma<1>(x_src, k.twt, F, w, g, t4, k.conj);
    if constexpr (C::NST == 2) {
      st.template store<1>(g_dst, w, g, t4, k.conj, true, cnt);
    } else {
      __syncthreads();
      st.template store<1>(x_dst, w, g, t4, k.conj, false, T);
      __syncthreads();
      st.template load_mma<2>(x_src, k.twt, F, w, g, t4, k.conj);
      st.template store<2>(g_dst, w, g, t4, k.conj, true, cnt);
    }
  }
}

template <int LOGN, int PREC, int LOAD, int STORE>
cudaError_t launch(const GbP2& k, cudaStream_t st) {
  using C = TC<LOGN>;
  constexpr int T = (LOAD == GB_P2_LOAD_CONTIG && STORE == GB_P2_STORE_CONTIG) ? 4096 / C::N : 16;
  const size_t smem = 128 + sizeof(float2) * (2 * (size_t)T * C::N + (size_t)T * C::PITCH);
  auto fn = gb_tc_kernel<LOGN, PREC, LOAD, STORE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
  if (e != cudaSuccess) return e;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = ((k.V0 + T - 1) / T) * k.nb1 * k.nb2;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (k.grid > 0) grid = k.grid;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  fn<<<(unsigned)grid, 256, smem, st>>>(k);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t dispatch_prec(const GbP2& k, cudaStream_t st) {
  const bool cc = k.load == GB_P2_LOAD_CONTIG && k.store == GB_P2_STORE_CONTIG;
  const bool rc = k.load == GB_P2_LOAD_ROWS && k.store == GB_P2_STORE_COLS;
  if (k.logn == 12 && cc) return launch<12, PREC, GB_P2_LOAD_CONTIG, GB_P2_STORE_CONTIG>(k, st);
  if (k.logn == 8 && cc) return launch<8, PREC, GB_P2_LOAD_CONTIG, GB_P2_STORE_CONTIG>(k, st);
  if (k.logn == 8 && rc) return launch<8, PREC, GB_P2_LOAD_ROWS, GB_P2_STORE_COLS>(k, st);
  return cudaErrorInvalidValue;
}

}  // namespace

int gb_tc_supported(int logn, int load, int store, int posttw) {
  if (posttw) return 0;
  const bool cc = load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_CONTIG;
  const bool rc = load == GB_P2_LOAD_ROWS && store == GB_P2_STORE_COLS;
  return (logn == 12 && cc) || (logn == 8 && (cc || rc));
}

int gb_tc_tile(int logn, int load, int store) {
  return (load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_CONTIG) ? (4096 >> logn) : 16;
}

cudaError_t gb_launch_tc(const GbP2& k, cudaStream_t st) {
  switch (k.prec) {
    case 1: return dispatch_prec<1>(k, st);
    case 2: return dispatch_prec<2>(k, st);
    case 3: return dispatch_prec<3>(k, st);
    case 4: return dispatch_prec<4>(k, st);
    default: return cudaErrorInvalidValue;
  }
}
