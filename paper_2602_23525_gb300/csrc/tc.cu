// tc.cu -- radix-16 Stockham stages on the 5th-generation tensor cores
// (tcgen05, sm_103a).
//
// A radix-16 stage applies the 16-point DFT matrix F (F[q][r] = w_16^{r q},
// eq. (1)) to every butterfly after the stage twiddles.  A tile holds 256
// butterflies (4096 points), one per thread; the stage is the real product
//   [Y_re | Y_im] = [X_re | X_im] . [[F_re, F_im], [-F_im, F_re]]
// of a 256 x 32 operand A (butterflies x points, re then im, rounded to FP16
// or BF16) with the constant 32 x 32 operand B, accumulated in FP32 in tensor
// memory: two tcgen05.mma of M = 128, N = 32 (K = 32 in two steps of 16),
// issued by one thread, completion signalled on an mbarrier through
// tcgen05.commit.  Each thread writes its butterfly as row `tid` of A in
// shared memory (the canonical K-major layout of 8 x 16-byte core matrices,
// no swizzle) and reads row `tid` of the result -- TMEM lane tid mod 128 in
// the column block of M-tile tid / 128 -- with tcgen05.ld.  Twiddles are
// applied in FP32 before the rounding (table of (w, w^2, w^4, w^8), as in the
// FP32 kernels).  The split forms write every operand as a sum of rounded
// components (hi = round(v), lo = round(v - hi), ...): FP16 as hi + lo with
// the products hi*hi + lo*hi + hi*lo, BF16 as hi + mid + lo with the six
// products of order down to 2^-16 (struct Prec).
//
// Tiles move as in stockham_pow2.cu: copy-engine loads (bulk copies of
// contiguous transforms, tensor-map boxes of T columns) on an mbarrier into
// one landing buffer per persistent CTA, refilled as soon as stage 0 has read
// it; two CTAs per SM hide each other's copy and MMA waits.  Stores are
// contiguous or column-wise.  Sizes:
// 2^8 and 2^12 points (all stages radix 16).  Every wait is bounded by
// %globaltimer; a CTA whose wait gives up records FFT_ERR_DEVICE_TIMEOUT,
// leaves the tile loop, waits (bounded) for the MMA and the tile copy it had
// in flight, and always frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

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

// operand precision: PREC 1/3 = FP16, 2/4 = BF16.  PREC 3 splits every
// operand into hi + lo (FP16 keeps 11 bits each, ~22 together) and sums the
// products hi.hi + lo.hi + hi.lo; PREC 4 splits into hi + mid + lo (BF16 keeps
// 8 bits each, ~24 together: the FP32 mantissa) and sums the six products
// whose order is at most 2^-16: hi.hi, mid.hi, lo.hi, hi.mid, mid.mid, hi.lo.
// Each product is a K = 32 block; A holds NC components side by side, B one
// block per product (its B component), and K step s of the MMA pairs A
// component acomp(s/2) with B block s/2.
template <int PREC>
struct Prec {
  static constexpr bool split = PREC >= 3;
  static constexpr int NC = PREC == 4 ? 3 : (PREC == 3 ? 2 : 1);  // components per operand
  static constexpr int NP = PREC == 4 ? 6 : (PREC == 3 ? 3 : 1);  // products summed
  static constexpr int KA = 4 * NC;  // 8-element K chunks per row of A: [hi | mid | lo]
  static constexpr int KB = 4 * NP;  // per row of B: one K = 32 block per product
  static constexpr uint32_t fmt = (PREC == 1 || PREC == 3) ? 0u : 1u;  // F16 0, BF16 1
  // (A component, B component) of product p
  __host__ __device__ static constexpr int acomp(int p) {
    return NP == 6 ? (p < 3 ? p : (p == 4 ? 1 : 0)) : (NP == 3 ? (p == 1 ? 1 : 0) : 0);
  }
  __host__ __device__ static constexpr int bcomp(int p) {
    return NP == 6 ? (p < 3 ? 0 : (p < 5 ? 1 : 2)) : (NP == 3 ? (p == 2 ? 1 : 0) : 0);
  }
};

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

// (a, b) as NC packed components: c[0] = round(a, b), c[i] = round(residual
// after c[0..i-1]); the residuals are exact in FP32
template <int PREC>
__device__ __forceinline__ void pack_split(float a, float b, uint32_t* c) {
#pragma unroll
  for (int i = 0; i < Prec<PREC>::NC; ++i) {
    c[i] = pack<PREC>(a, b);
    const float2 h = unpack<PREC>(c[i]);
    a -= h.x;
    b -= h.y;
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int phys(int i) { return i + (i >> 5); }

// byte offset of the 16-byte row piece (row, K chunk c) in the canonical
// K-major layout without swizzle: core matrices of 8 rows x 16 bytes, K
// chunks adjacent (leading byte offset 128), 8-row groups KC*128 apart
__device__ __forceinline__ uint32_t core_off(int row, int c, int KC) {
  return (uint32_t)(((row >> 3) * KC + c) * 128 + (row & 7) * 16);
}

// shared-memory matrix descriptor (start >> 4, LBO >> 4, SBO >> 4, version 1,
// no swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// the powers w^1..w^15 from (w, w^2, w^4, w^8), at most three products each
__device__ __forceinline__ void twiddle16(float2* v, const float4* tw) {
  const float4 a = __ldg(tw), b = __ldg(tw + 1);
  float2 p[16];
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
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], p[r]);
}

// row `row` of A: points 0..15 re (chunks 0, 1), im (chunks 2, 3) of each
// component (component i at chunks 4i .. 4i+3)
template <int PREC>
__device__ __forceinline__ void write_row(uint32_t abase, int row, const float2* x) {
  using P = Prec<PREC>;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int r0 = (c & 1) * 8;
    uint32_t h[4][P::NC];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float a = (c < 2) ? x[r0 + 2 * i].x : x[r0 + 2 * i].y;
      const float b = (c < 2) ? x[r0 + 2 * i + 1].x : x[r0 + 2 * i + 1].y;
      pack_split<PREC>(a, b, h[i]);
    }
#pragma unroll
    for (int q = 0; q < P::NC; ++q)
      st_shared_v4(abase + core_off(row, 4 * q + c, P::KA), h[0][q], h[1][q], h[2][q], h[3][q]);
  }
}

// B^T (rows n = output re 0..15 then im 0..15, K = points re then im):
// n < 16:  [C(nr) | -S(nr)],  n >= 16: [S(qr) | C(qr)] with q = n - 16;
// block p (chunks 4p .. 4p+3) holds component bcomp(p)
template <int PREC>
__device__ void build_b(uint32_t bbase, int tid) {
  using P = Prec<PREC>;
  if (tid >= 32) return;
  const int n = tid, q = n & 15;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t h[4][P::NC];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float v2[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int k = c * 8 + 2 * i + e;  // 0..31
        const int r = k & 15, m = (q * r) & 15;
        const bool kim = k >= 16;
        v2[e] = n < 16 ? (kim ? -S16[m] : C16[m]) : (kim ? C16[m] : S16[m]);
      }
      pack_split<PREC>(v2[0], v2[1], h[i]);
    }
#pragma unroll
    for (int p = 0; p < P::NP; ++p) {
      const int q2 = P::bcomp(p);
      st_shared_v4(bbase + core_off(n, 4 * p + c, P::KB), h[0][q2], h[1][q2], h[2][q2], h[3][q2]);
    }
  }
}

// D (TMEM, 2 M-tiles x 32 columns) = A . B for the 256 rows of A; the split
// forms accumulate one K = 32 block per product (A component acomp(p) times
// B block p)
template <int PREC>
__device__ __forceinline__ void issue_mma(uint32_t tmem, uint32_t abase, uint32_t bbase, uint32_t bar) {
  using P = Prec<PREC>;
  constexpr uint32_t idesc = (1u << 4) | (P::fmt << 7) | (P::fmt << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
  constexpr int KSTEPS = P::KB / 2;  // 16 elements = 2 chunks per step
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
    for (int s = 0; s < KSTEPS; ++s) {
      const int sa = 2 * P::acomp(s / 2) + (s & 1);  // A's K step within its component
      const uint64_t ad = smem_desc(abase + (uint32_t)(mt * 16 * P::KA * 128 + sa * 256), 128, P::KA * 128);
      const uint64_t bd = smem_desc(bbase + (uint32_t)(s * 256), 128, P::KB * 128);
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)(32 * mt)),
          "l"(ad), "l"(bd), "r"(idesc), "r"(s) : "memory");
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// row `tid` of D: 32 FP32 columns = Y_re[0..15], Y_im[0..15]
__device__ __forceinline__ void read_row(uint32_t tmem, int tid, float2* y) {
  const int w = tid >> 5;
  const uint32_t ta = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(32 * (w >> 2));
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) y[q] = make_float2(__uint_as_float(r[q]), __uint_as_float(r[16 + q]));
}

template <int LOGN, int PREC, int LOAD, int STORE>
__global__ void __launch_bounds__(256, 2) gb_tc_kernel(const __grid_constant__ GbP2 k,
                                                       const __grid_constant__ CUtensorMap tm, int tmap, int pos) {
  using C = TC<LOGN>;
  using P = Prec<PREC>;
  constexpr int T = (LOAD == GB_P2_LOAD_CONTIG && STORE == GB_P2_STORE_CONTIG) ? 4096 / C::N : 16;
  static_assert(T * C::NBF == 256, "a tile is 256 butterflies");
  constexpr int TILE = T * C::N;
  constexpr int NBUF = 1;  // one landing buffer: two CTAs per SM overlap each other's waits
  constexpr uint32_t ABYTES = 256 * P::KA * 16, BBYTES = 32 * P::KB * 16;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);  // [0, NBUF) tiles, [NBUF] mma
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + 64);
  const uint32_t abase = smem_addr(smem_raw + 1024);
  const uint32_t bbase = abase + ABYTES;
  float2* ibuf = reinterpret_cast<float2*>(smem_raw + 1024 + ABYTES + BBYTES);
  float2* xbuf = ibuf + NBUF * TILE;
  const int tid = threadIdx.x, lane = tid & 31;
  // butterfly of this thread: lanes across the transforms for column tiles
  constexpr bool TFAST = LOAD == GB_P2_LOAD_ROWS;
  const int bt = TFAST ? tid % T : tid / C::NBF, bj = TFAST ? tid / T : tid % C::NBF;

  if (tid == 0) {
    for (int b = 0; b < NBUF + 1; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_addr(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  build_b<PREC>(bbase, tid);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t mbar = smem_addr(bars + NBUF);

  const int64_t cblocks = (k.V0 + T - 1) / T;
  const int64_t ntiles = cblocks * k.nb1 * k.nb2;
  auto origin = [&](int64_t tile, int64_t* ib, int64_t* ob, int64_t* c0, int64_t* b1, int64_t* b2) {
    const int64_t cb = tile % cblocks, r = tile / cblocks;
    *b1 = r % k.nb1;
    *b2 = r / k.nb1;
    *c0 = cb * T;
    *ib = *b1 * k.vis1 + *b2 * k.vis2 + *c0 * k.vis0;
    *ob = *b1 * k.vos1 + *b2 * k.vos2 + *c0 * k.vos0;
  };
  auto issue = [&](int b, int64_t tile) {
    int64_t ib, ob, c0, b1, b2;
    origin(tile, &ib, &ob, &c0, &b1, &b2);
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
      if (tmap) {
        if (lane == 0) {
          constexpr int BOXR = C::N < 256 ? C::N : 256;
#pragma unroll
          for (int r0 = 0; r0 < C::N; r0 += BOXR)
            tensor_copy_4d(smem_addr(dst + r0 * T), &tm, (int)c0, map_coord(pos, 1, r0, (int)b1, (int)b2),
                           map_coord(pos, 2, r0, (int)b1, (int)b2), map_coord(pos, 3, r0, (int)b1, (int)b2), bar);
        }
      } else {
        for (int e = lane; e < C::N; e += 32)
          bulk_copy(smem_addr(dst + e * T), k.in + ib + (int64_t)e * k.is, (uint32_t)(T * 8), bar);
      }
    }
  };
  if (tid < 32)
    for (int b = 0; b < NBUF; ++b) {
      const int64_t tile = blockIdx.x + (int64_t)b * gridDim.x;
      if (tile < ntiles) issue(b, tile);
    }

  uint32_t mphase = 0;
  bool bad = false;
  int it = 0;
  // what is in flight, for the exit after a wait gave up: the iteration whose
  // tile copy was issued and not yet waited for, and an MMA not yet complete
  int64_t load_it = (int64_t)blockIdx.x < ntiles ? 0 : -1;
  bool mma_pending = false;
  for (int64_t tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x, ++it) {
    const int b = it % NBUF;
    const bool ok = mbar_wait(smem_addr(bars + b), (uint32_t)((it / NBUF) & 1));
    if (__syncthreads_or(!ok)) {
      bad = true;
      break;
    }
    load_it = -1;
    int64_t ib, ob, c0, b1, b2;
    origin(tile, &ib, &ob, &c0, &b1, &b2);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const float2* tb = ibuf + b * TILE;
#pragma unroll 1
    for (int s = 0; s < C::NST; ++s) {
      const int L = C::L(s);
      float2 x[16];
      // inputs of butterfly (bt, bj): elements bj + r*NBF
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int e = bj + r * C::NBF;
        float2 v;
        if (s == 0) {
          v = LOAD == GB_P2_LOAD_CONTIG ? tb[bt * C::N + e] : tb[e * T + bt];
          if (k.conj) v.y = -v.y;
        } else {
          v = xbuf[bt * C::PITCH + phys(e)];
        }
        x[r] = v;
      }
      if (s > 0) twiddle16(x, reinterpret_cast<const float4*>(k.twt + C::twoff(s) + (bj & (L - 1)) * 4));
      write_row<PREC>(abase, tid, x);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // A written, stage inputs read (tile or exchange rows), previous D read
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (s == 0) {
        // the landing buffer is free: refill it with the next tile of this CTA
        const int64_t next = tile + (int64_t)NBUF * gridDim.x;
        if (next < ntiles) {
          load_it = it + NBUF;
          if (tid < 32) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(b, next);
          }
        }
      }
      if (tid == 0) issue_mma<PREC>(tmem, abase, bbase, mbar);
      mma_pending = true;
      const bool done = mbar_wait(mbar, mphase);
      if (__syncthreads_or(!done)) {
        bad = true;
        break;
      }
      mphase ^= 1;
      mma_pending = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float2 y[16];
      read_row(tmem, tid, y);
      // outputs q of butterfly bj land at (bj - kk)*16 + kk + q*L
      const int kk = bj & (L - 1);
      const int base = (bj - kk) * 16 + kk;
      if (s == C::NST - 1) {
        if (bt < cnt) {
          float2* g = k.out + ob + (int64_t)bt * k.vos0;
          const int64_t os = STORE == GB_P2_STORE_COLS ? k.os : 1;
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            float2 v = y[q];
            if (k.conj) v.y = -v.y;
            g[(int64_t)(base + q * L) * os] = v;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) xbuf[bt * C::PITCH + phys(base + q * L)] = y[q];
      }
      __syncthreads();  // exchange rows written before the next stage reads them
    }
  }
  if (bad) {
    // a wait gave up: let the MMA and the tile copy already issued land
    // (each wait bounded again) before tensor and shared memory are released
    if (mma_pending) mbar_wait(mbar, mphase);
    if (load_it >= 0) mbar_wait(smem_addr(bars + (int)(load_it % NBUF)), (uint32_t)((load_it / NBUF) & 1));
    if (tid == 0 && k.status) gb_set_status(k.status, kStatusTimeout);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

template <int LOGN, int PREC, int LOAD, int STORE>
cudaError_t launch(const GbP2& k, cudaStream_t st) {
  using C = TC<LOGN>;
  using P = Prec<PREC>;
  constexpr int T = (LOAD == GB_P2_LOAD_CONTIG && STORE == GB_P2_STORE_CONTIG) ? 4096 / C::N : 16;
  const size_t smem = 1024 + (size_t)256 * P::KA * 16 + (size_t)32 * P::KB * 16 +
                      sizeof(float2) * ((size_t)T * C::N + (size_t)T * C::PITCH);
  auto fn = gb_tc_kernel<LOGN, PREC, LOAD, STORE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = ((k.V0 + T - 1) / T) * k.nb1 * k.nb2;
  // CTAs per SM from the shared memory they need (1 KB reserved each); the
  // occupancy query reports one for this kernel although two are resident.
  // Registers (launch bound 2) and tensor memory (64 columns each) allow two.
  int sm_bytes = 0;
  cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int per_sm = (sm_bytes >= 2 * (int)(smem + 1024)) ? 2 : 1;
  int64_t grid = (int64_t)sms * per_sm;
  if (k.grid > 0) grid = k.grid;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  alignas(128) CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  int pos = 0, tmap = 0;
  if (LOAD == GB_P2_LOAD_ROWS) tmap = gb_p2_rows_map(k, T, &tm, &pos);
  fn<<<(unsigned)grid, 256, smem, st>>>(k, tm, tmap, pos);
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
