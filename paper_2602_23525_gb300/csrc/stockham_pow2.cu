// stockham_pow2.cu -- batched power-of-two Stockham pass kernels with TMA tile
// loads (sm_103a), n = 2^4 .. 2^13.
//
// The Stockham stages of stockham.cu (eq. (2) applied with n1 = L, n2 = R at
// every stage, output auto-sorted, sec. 2), specialised at compile time: the
// radix schedule is 2^(log2 n mod 4) first (when not 1) and 16 after, every
// thread holds exactly 16 values (n/16 threads per transform), index
// arithmetic is shifts and masks, and the stage twiddles w_{16L}^{r k} come
// from per-stage tables [k][4] = (w, w^2, w^4, w^8) (two 128-bit loads; every
// other power is a product of at most three entries -- the small-table
// scheme of sec. 6, never a running recurrence).
//
// A CTA computes a tile of T transforms that are adjacent along the tile
// dimension of the vector loops, and is persistent over tiles.  One warp
// issues TMA bulk copies (cp.async.bulk, completion counted on an mbarrier)
// of the next NBUF tiles while all threads compute the current one, so HBM
// reads stay in flight through the compute phases (the buffered copies of
// sec. 3.3, done by the copy engine).  Two tile shapes:
//   LOAD_CONTIG: each transform is contiguous (unit element stride); one copy
//                per tile when the tile's transforms are adjacent, else one per
//                transform.
//   LOAD_ROWS:   the tile is T adjacent columns of a row-major matrix whose
//                columns are the transforms (unit stride along the tile
//                dimension) -- the strided first pass of a four-step plan
//                (sec. 3.3, radix-sqrt(n)).  The tile arrives as tensor-map
//                boxes of T columns x up to 256 rows (cp.async.bulk.tensor,
//                one instruction per box); where no tensor map can describe
//                the layout, as one bulk copy of T elements per row.
// and two store shapes: STORE_CONTIG (unit element stride, lanes along the
// transform) and STORE_COLS (unit stride along the tile dimension, lanes
// across the T transforms, so T adjacent outputs form one segment).
// With POSTTW the outputs are multiplied by the four-step twiddle
// w_N^{l2 k1} of eq. (2) (l2 = column, k1 = output index).
// Every mbarrier wait is bounded by %globaltimer; on timeout the CTA waits
// (bounded) for the copies it has in flight, records FFT_ERR_DEVICE_TIMEOUT
// in the status word and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <cstring>
#include <mutex>
#include <utility>

#include "gb_kernels.h"
#include "gb_p2_stages.cuh"
#include "gb_tma.cuh"

namespace {


// Tensor map of a LOAD_ROWS input: dims (column, then the rows and the two
// vector loops ordered by stride); pos = the map dims of the rows, nb1 and nb2
// (packed as for map_coord).
struct GbRowsMap {
  CUtensorMap map;
  int use;
  int pos;
};

// After a wait gave up at iteration `it` (tile `tile`): the copies of
// iterations it .. it + NBUF - 1 were issued into this CTA's shared memory;
// wait for each (bounded again) before the CTA exits.
template <int NBUF>
__device__ __forceinline__ void drain_copies(uint64_t* bars, int it, int64_t tile, int64_t ntiles) {
  for (int j = 0; j < NBUF; ++j)
    if (tile + (int64_t)j * gridDim.x < ntiles)
      mbar_wait(smem_addr(bars + (it + j) % NBUF), (uint32_t)(((it + j) / NBUF) & 1));
}

// Thread -> (transform t, thread u within the transform):
//   "j-fast": t = tid / TPT, u = tid % TPT (lanes along a transform)
//   "t-fast": t = tid % T,   u = tid / T   (lanes across the T transforms)
// Stage 0 uses the mapping that reads the landed tile without bank conflicts,
// the last stage the one that makes the global stores coalesce.
template <int LOGN, int T, int NBUF, int MINB, int LOAD, int STORE, bool POSTTW, bool PW>
__global__ void __launch_bounds__(T*(1 << LOGN) / 16, MINB)
    gb_p2_kernel(const __grid_constant__ GbP2 k, const __grid_constant__ GbRowsMap rm) {
  using C = P2<LOGN>;
  constexpr int TILE = T * C::N;  // elements per tile buffer
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float2* ibuf = reinterpret_cast<float2*>(smem_raw + 128);
  float2* xbuf = ibuf + NBUF * TILE;

  const int tid = threadIdx.x;
  const int tj = tid / C::TPT, uj = tid - tj * C::TPT;  // j-fast
  const int tt = tid % T, ut = tid / T;                 // t-fast
  const int t0 = (LOAD == GB_P2_LOAD_ROWS) ? tt : tj;
  const int u0 = (LOAD == GB_P2_LOAD_ROWS) ? ut : uj;
  const int ts = (STORE == GB_P2_STORE_COLS) ? tt : tj;
  const int us = (STORE == GB_P2_STORE_COLS) ? ut : uj;

  const int64_t cblocks = (k.V0 + T - 1) / T;
  const int64_t ntiles = cblocks * k.nb1 * k.nb2;

  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // tile -> element offsets of its transform 0 and its first index along the tile dim
  auto origin = [&](int64_t tile, int64_t* ib, int64_t* ob, int64_t* c0) {
    const int64_t cb = tile % cblocks;
    const int64_t r = tile / cblocks;
    const int64_t b1 = r % k.nb1, b2 = r / k.nb1;
    *c0 = cb * T;
    *ib = b1 * k.vis1 + b2 * k.vis2 + *c0 * k.vis0;
    *ob = b1 * k.vos1 + b2 * k.vos2 + *c0 * k.vos0;
  };

  // warp 0 issues the copies of one tile into buffer b
  auto issue = [&](int b, int64_t tile) {
    int64_t ib, ob, c0;
    origin(tile, &ib, &ob, &c0);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const uint32_t bar = smem_addr(bars + b);
    float2* dst = ibuf + b * TILE;
    const int lane = tid & 31;
    if (LOAD == GB_P2_LOAD_CONTIG) {
      if (lane == 0) expect_tx(bar, (uint32_t)(cnt * C::N * 8));
      __syncwarp();
      if (T == 1 || k.vis0 == C::N) {
        if (lane == 0) bulk_copy(smem_addr(dst), k.in + ib, (uint32_t)(cnt * C::N * 8), bar);
      } else {
        for (int64_t i = lane; i < cnt; i += 32)
          bulk_copy(smem_addr(dst + i * C::N), k.in + ib + i * k.vis0, (uint32_t)(C::N * 8), bar);
      }
    } else {
      // rows of T adjacent columns (the host makes V0 a multiple of T):
      // element e of column t lands at dst[e * T + t]
      if (lane == 0) expect_tx(bar, (uint32_t)(C::N * T * 8));
      __syncwarp();
      if (rm.use) {
        if (lane == 0) {
          const int64_t r = tile / cblocks;
          const int b1 = (int)(r % k.nb1), b2 = (int)(r / k.nb1);
          constexpr int BOXR = C::N < 256 ? C::N : 256;
#pragma unroll
          for (int r0 = 0; r0 < C::N; r0 += BOXR)
            tensor_copy_4d(smem_addr(dst + r0 * T), &rm.map, (int)c0, map_coord(rm.pos, 1, r0, b1, b2),
                           map_coord(rm.pos, 2, r0, b1, b2), map_coord(rm.pos, 3, r0, b1, b2), bar);
        }
      } else {
        for (int e = lane; e < C::N; e += 32)
          bulk_copy(smem_addr(dst + e * T), k.in + ib + (int64_t)e * k.is, (uint32_t)(T * 8), bar);
      }
    }
  };

  if (tid < 32) {
    for (int b = 0; b < NBUF; ++b) {
      const int64_t tile = blockIdx.x + (int64_t)b * gridDim.x;
      if (tile < ntiles) issue(b, tile);
    }
  }

  float2 v[16];
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it % NBUF;
    const uint32_t parity = (uint32_t)((it / NBUF) & 1);
    const bool ok = mbar_wait(smem_addr(bars + b), parity);
    if (__syncthreads_or(!ok)) {
      drain_copies<NBUF>(bars, it, tile, ntiles);
      if (tid == 0 && k.status) gb_set_status(k.status, kStatusTimeout);
      return;
    }
    int64_t ib, ob, c0;
    origin(tile, &ib, &ob, &c0);
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const bool valid = ts < cnt;
    float2* gout = k.out + ob + (int64_t)ts * k.vos0;
    const int64_t ostride = (STORE == GB_P2_STORE_COLS) ? k.os : 1;
    int64_t col = c0 + ts;  // post-twiddle column index: the tile dimension's,
    if (POSTTW && k.ptw_dim) {  // or that of a vector loop
      const int64_t r = tile / cblocks;
      col = k.ptw_dim == 1 ? r % k.nb1 : r / k.nb1;
    }
    const float2* tile_buf = ibuf + b * TILE;
    float2 et[PW ? 16 : 1];
    if constexpr (PW) epi_prefetch<LOGN>(et, &k.epi, us, col);
    if constexpr (LOAD == GB_P2_LOAD_ROWS)
      stage_in<LOGN, 0, true, T>(v, tile_buf + t0, k.twt, u0, k.conj);
    else
      stage_in<LOGN, 0, true, 1>(v, tile_buf + t0 * C::N, k.twt, u0, k.conj);
    __syncthreads();  // tile buffer b fully read; previous tile's exchange reads done
    if (tid < 32) {
      const int64_t next = tile + (int64_t)NBUF * gridDim.x;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(b, next);
      }
    }
    if constexpr (C::NST == 1) {
      // one stage: the host only builds this when both mappings agree
      if (valid) stage_out_g<LOGN, POSTTW, PW>(v, gout, ostride, u0, k.conj, k.ptwA, k.ptwB, col, &k.epi, et);
    } else {
      stage_out_x<LOGN, 0>(v, xbuf + t0 * C::PITCH, u0);
      __syncthreads();
      later_stages<LOGN, 1, POSTTW, PW>(v, xbuf + tj * C::PITCH, xbuf + ts * C::PITCH, gout, ostride, k.twt, uj, us,
                                    k.conj, valid, k.ptwA, k.ptwB, col, &k.epi, et);
    }
  }
}


// Tensor map for the LOAD_ROWS tiles of k: 8-byte elements, dims (V0 columns,
// then the n rows and the two vector loops by increasing stride, extent-1
// loops last), box T columns x min(n, 256) rows.  Leaves rm->use = 0 (per-row
// bulk copies) when the layout has no such map: an unaligned base, a stride
// that is not a multiple of 16 bytes or that decreases along the dims, or an
// encoder error.
void make_rows_map(const GbP2& k, int T, GbRowsMap* rm) {
  memset(rm, 0, sizeof(*rm));
  if (k.load != GB_P2_LOAD_ROWS || k.vis0 != 1) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = (PFN_cuTensorMapEncodeTiled_v12000)gb_tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(k.in) & 15)) return;
  const int64_t n = int64_t(1) << k.logn;
  struct D {
    int64_t n, s;
    int who;  // 0 rows, 1 nb1, 2 nb2
  } d[3] = {{n, k.is * 8, 0}, {k.nb1, k.vis1 * 8, 1}, {k.nb2, k.vis2 * 8, 2}};
  for (int i = 0; i < 3; ++i)
    if (d[i].n > 1 && d[i].s <= 0) return;
  auto before = [](const D& x, const D& y) { return (x.n > 1) != (y.n > 1) ? x.n > 1 : x.s < y.s; };
  for (int i = 1; i < 3; ++i)  // stable insertion sort of three
    for (int j = i; j > 0 && before(d[j], d[j - 1]); --j) std::swap(d[j], d[j - 1]);
  cuuint64_t dim[4] = {(cuuint64_t)k.V0, (cuuint64_t)d[0].n, (cuuint64_t)d[1].n, (cuuint64_t)d[2].n};
  cuuint64_t str[3] = {(cuuint64_t)d[0].s, (cuuint64_t)d[1].s, (cuuint64_t)d[2].s};
  for (int i = 1; i < 3; ++i)
    if (d[i].n == 1) str[i] = str[i - 1] * d[i - 1].n;  // extent-1 dims: any valid stride
  for (int i = 0; i < 3; ++i)
    if ((str[i] & 15) || str[i] >= (cuuint64_t(1) << 40)) return;
  if (str[0] < (cuuint64_t)(k.V0 * 8) || str[1] < str[0] || str[2] < str[1]) return;
  for (int i = 0; i < 4; ++i)
    if (dim[i] < 1 || dim[i] > (cuuint64_t(1) << 32)) return;
  cuuint32_t box[4] = {(cuuint32_t)T, 1, 1, 1};
  int pos = 0;
  for (int i = 0; i < 3; ++i) {
    if (d[i].who == 0) box[1 + i] = (cuuint32_t)(n < 256 ? n : 256);
    pos |= (i + 1) << (2 * d[i].who);
  }
  cuuint32_t es[4] = {1, 1, 1, 1};
  if (enc(&rm->map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<float2*>(k.in), dim, str, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return;
  rm->use = 1;
  rm->pos = pos;
}

template <int LOGN, int T, int NBUF, int MINB, int LOAD, int STORE, bool POSTTW, bool PW>
cudaError_t launch(const GbP2& k, cudaStream_t st) {
  using C = P2<LOGN>;
  static_assert(LOAD != GB_P2_LOAD_ROWS || (T % 2 == 0), "tensor-map boxes need 16-byte rows");
  const size_t smem = 128 + sizeof(float2) * ((size_t)NBUF * T * C::N + (C::NST > 1 ? (size_t)T * C::PITCH : 0));
  auto fn = gb_p2_kernel<LOGN, T, NBUF, MINB, LOAD, STORE, POSTTW, PW>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T * C::TPT, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = ((k.V0 + T - 1) / T) * k.nb1 * k.nb2;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (k.grid > 0) grid = k.grid;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  GbRowsMap rm;
  make_rows_map(k, T, &rm);
  fn<<<(unsigned)grid, T * C::TPT, smem, st>>>(k, rm);
  return cudaGetLastError();
}

// Small transforms, n = 16 .. 128, contiguous tiles of 4096 points (T = 4096/n
// transforms) in and out.  Landing a tile of many short transforms unpadded
// would make every stage-0 read a bank conflict (the transforms sit a multiple
// of 32 banks apart), so after the bulk copy lands the CTA re-lays it into
// odd-pitch rows with 128-bit reads; every stage then runs with lanes across
// the transforms, and the outputs leave from the rows with 128-bit stores.
template <int LOGN>
__global__ void __launch_bounds__(256, 2) gb_p2small_kernel(const __grid_constant__ GbP2 k) {
  using C = P2<LOGN>;
  constexpr int T = 4096 / C::N;
  constexpr int TILE = 4096;
  constexpr int NBUF = 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float2* ibuf = reinterpret_cast<float2*>(smem_raw + 128);
  float2* xbuf = ibuf + NBUF * TILE;
  const int tid = threadIdx.x;
  const int t = tid % T, u = tid / T;  // lanes across transforms
  const int64_t ntiles = (k.V0 + T - 1) / T;
  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int b, int64_t tile) {
    const int64_t c0 = tile * T;
    const int64_t cnt = (k.V0 - c0) < T ? (k.V0 - c0) : T;
    const uint32_t bar = smem_addr(bars + b);
    expect_tx(bar, (uint32_t)(cnt * C::N * 8));
    bulk_copy(smem_addr(ibuf + b * TILE), k.in + c0 * C::N, (uint32_t)(cnt * C::N * 8), bar);
  };
  if (tid == 0)
    for (int b = 0; b < NBUF; ++b) {
      const int64_t tile = blockIdx.x + (int64_t)b * gridDim.x;
      if (tile < ntiles) issue(b, tile);
    }
  float2 v[16];
  float2* xrow = xbuf + t * C::PITCH;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it % NBUF;
    const bool ok = mbar_wait(smem_addr(bars + b), (uint32_t)((it / NBUF) & 1));
    if (__syncthreads_or(!ok)) {
      drain_copies<NBUF>(bars, it, tile, ntiles);
      if (tid == 0 && k.status) gb_set_status(k.status, kStatusTimeout);
      return;
    }
    const int64_t c0 = tile * T;
    const int cnt = (int)((k.V0 - c0) < T ? (k.V0 - c0) : T);
    // re-layout: 128-bit reads of the landed tile into odd-pitch rows
    const float4* src4 = reinterpret_cast<const float4*>(ibuf + b * TILE);
    for (int i = tid; i < TILE / 2; i += 256) {
      float4 w = src4[i];
      if (k.conj) {
        w.y = -w.y;
        w.w = -w.w;
      }
      const int e = 2 * i, tt = e >> LOGN, p = e & (C::N - 1);
      xbuf[tt * C::PITCH + phys(p)] = make_float2(w.x, w.y);
      xbuf[tt * C::PITCH + phys(p + 1)] = make_float2(w.z, w.w);
    }
    __syncthreads();
    if (tid == 0) {
      const int64_t next = tile + (int64_t)NBUF * gridDim.x;
      if (next < ntiles) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(b, next);
      }
    }
    stage_in<LOGN, 0, false, 1>(v, xrow, k.twt, u, 0);
    __syncthreads();
    stage_out_x<LOGN, 0>(v, xrow, u);
    __syncthreads();
    if constexpr (C::NST > 1) {
      static_assert(C::NST == 2, "small kernel covers two stages at most");
      stage_in<LOGN, 1, false, 1>(v, xrow, k.twt, u, 0);
      __syncthreads();
      stage_out_x<LOGN, 1>(v, xrow, u);
      __syncthreads();
    }
    // 128-bit stores of the rows, transforms adjacent in the output
    float4* dst4 = reinterpret_cast<float4*>(k.out + c0 * C::N);
    for (int i = tid; i < cnt * C::N / 2; i += 256) {
      const int e = 2 * i, tt = e >> LOGN, p = e & (C::N - 1);
      const float2 a = xbuf[tt * C::PITCH + phys(p)], c = xbuf[tt * C::PITCH + phys(p + 1)];
      dst4[i] = k.conj ? make_float4(a.x, -a.y, c.x, -c.y) : make_float4(a.x, a.y, c.x, c.y);
    }
    __syncthreads();  // rows read out before the next tile's re-layout
  }
}

template <int LOGN>
cudaError_t launch_small(const GbP2& k, cudaStream_t st) {
  using C = P2<LOGN>;
  constexpr int T = 4096 / C::N;
  const size_t smem = 128 + sizeof(float2) * (2 * 4096 + (size_t)T * C::PITCH);
  auto fn = gb_p2small_kernel<LOGN>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (k.V0 + T - 1) / T;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (k.grid > 0) grid = k.grid;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) return cudaSuccess;
  fn<<<(unsigned)grid, 256, smem, st>>>(k);
  return cudaGetLastError();
}

// transforms per CTA tile, by size and tile shape (tiles of 32-64 KB); column
// tiles are at least 16 columns (128-byte row segments) and 4096 points below
// n = 256, so that n = 64 / 128 move 512 / 256-byte row segments
constexpr int tile_T(int logn, int load, int store) {
  return (load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_CONTIG)
             ? (logn <= 12 ? (1 << (12 - logn)) : 1)
             : (logn <= 7 ? (1 << (12 - logn)) : logn <= 9 ? 16 : (logn == 10 ? 8 : (logn == 11 ? 4 : 2)));
}

constexpr int min_blocks(int logn, int load, int store) {
  return (load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_CONTIG)
             ? (logn >= 9 && logn <= 12 ? 3 : (logn <= 12 ? 2 : 1))
             : (logn <= 8 ? 2 : 1);
}

// landing buffers per CTA: contiguous passes of 2^9..2^12 points keep one, so
// that three CTAs fit an SM (their exchange rows and one 32 KB tile each)
constexpr int land_bufs(int logn, int load, int store) {
  return (load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_CONTIG && logn >= 9 && logn <= 12) ? 1 : 2;
}

template <int LOGN, int LOAD, int STORE, bool POSTTW, bool PW = false>
cudaError_t launch_n(const GbP2& k, cudaStream_t st) {
  return launch<LOGN, tile_T(LOGN, LOAD, STORE), land_bufs(LOGN, LOAD, STORE), min_blocks(LOGN, LOAD, STORE), LOAD,
                STORE, POSTTW, PW>(k, st);
}

// the store epilogue: contiguous transforms in, column tiles out (the last
// pass of a four-step), n = 2^6 .. 2^12
cudaError_t dispatch_epi(const GbP2& k, cudaStream_t st) {
  constexpr int LD = GB_P2_LOAD_CONTIG, SC = GB_P2_STORE_COLS;
  switch (k.logn) {
    case 6: return launch_n<6, LD, SC, false, true>(k, st);
    case 7: return launch_n<7, LD, SC, false, true>(k, st);
    case 8: return launch_n<8, LD, SC, false, true>(k, st);
    case 9: return launch_n<9, LD, SC, false, true>(k, st);
    case 10: return launch_n<10, LD, SC, false, true>(k, st);
    case 11: return launch_n<11, LD, SC, false, true>(k, st);
    case 12: return launch_n<12, LD, SC, false, true>(k, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOAD, int STORE, bool POSTTW>
cudaError_t dispatch(const GbP2& k, cudaStream_t st) {
  constexpr bool cc = LOAD == GB_P2_LOAD_CONTIG && STORE == GB_P2_STORE_CONTIG;
  switch (k.logn) {
    case 4: if constexpr (cc && !POSTTW) return launch_small<4>(k, st); break;
    case 5: if constexpr (cc && !POSTTW) return launch_small<5>(k, st); break;
    case 6:
      if constexpr (cc && !POSTTW) return launch_small<6>(k, st);
      else if constexpr (!cc) return launch_n<6, LOAD, STORE, POSTTW>(k, st);
      break;
    case 7:
      if constexpr (cc && !POSTTW) return launch_small<7>(k, st);
      else if constexpr (!cc) return launch_n<7, LOAD, STORE, POSTTW>(k, st);
      break;
    case 8: return launch_n<8, LOAD, STORE, POSTTW>(k, st);
    case 9: return launch_n<9, LOAD, STORE, POSTTW>(k, st);
    case 10: return launch_n<10, LOAD, STORE, POSTTW>(k, st);
    case 11: return launch_n<11, LOAD, STORE, POSTTW>(k, st);
    case 12: return launch_n<12, LOAD, STORE, POSTTW>(k, st);
    case 13: if constexpr (cc && !POSTTW) return launch_n<13, LOAD, STORE, POSTTW>(k, st); break;
    default: break;
  }
  return cudaErrorInvalidValue;
}

// The debug stall of a plan (FFT_DEBUG_STALL): one wait, bounded at
// limit_ns, on an mbarrier that nothing arrives on.  The wait runs out, the
// kernel records FFT_ERR_DEVICE_TIMEOUT in the plan's status word exactly
// as a pass kernel whose tile copy never landed would, and returns; nothing
// faults and the context stays usable.
__global__ void gb_stall_kernel(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait_for(smem_addr(&bar), 0, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) gb_set_status(status, kStatusTimeout);
}

}  // namespace

cudaError_t gb_launch_stall(int* status, unsigned long long limit_ns, cudaStream_t st) {
  gb_stall_kernel<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

void* gb_tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return reinterpret_cast<void*>(fn);
}

int gb_p2_rows_map(const GbP2& k, int T, void* map, int* pos) {
  GbRowsMap rm;
  make_rows_map(k, T, &rm);
  memcpy(map, &rm.map, sizeof(CUtensorMap));
  *pos = rm.pos;
  return rm.use;
}

int gb_p2_epi_supported(int logn, int load, int store, int posttw) {
  return load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_COLS && !posttw && logn >= 6 && logn <= 12;
}

int gb_p2_supported(int logn, int load, int store, int posttw) {
  const bool cc = load == GB_P2_LOAD_CONTIG && store == GB_P2_STORE_CONTIG;
  if (cc) return !posttw && logn >= 4 && logn <= 13;
  if (logn < 6 || logn > 12) return 0;
  if (posttw && load != GB_P2_LOAD_ROWS) return 0;
  if (posttw && logn % 4 != 0 && logn / 4 + 1 < 2) return 0;
  return 1;
}

int gb_p2_tile(int logn, int load, int store) { return tile_T(logn, load, store); }

// the small-transform kernel needs adjacent transforms on both sides
int gb_p2_small(int logn) { return logn >= 4 && logn <= 7; }

int gb_p2_twiddle_elems(int logn) {
  const int rem = logn % 4, r0 = rem ? (1 << rem) : 16, nst = logn / 4 + (rem ? 1 : 0);
  int o = 0;
  for (int i = 1; i < nst; ++i) o += (r0 << (4 * (i - 1))) * 4;
  return o;
}

// stage s >= 1 of the schedule: (L, R) and the table offset, for the generator
int gb_p2_stage(int logn, int s, int* L, int* R, int* offset) {
  const int rem = logn % 4, r0 = rem ? (1 << rem) : 16, nst = logn / 4 + (rem ? 1 : 0);
  if (s < 1 || s >= nst) return 0;
  *R = 16;
  *L = r0 << (4 * (s - 1));
  int o = 0;
  for (int i = 1; i < s; ++i) o += (r0 << (4 * (i - 1))) * 4;
  *offset = o;
  return 1;
}

// L of the last stage (the post-twiddle table has N_cols x L base entries)
int gb_p2_last_L(int logn) {
  const int rem = logn % 4, r0 = rem ? (1 << rem) : 16, nst = logn / 4 + (rem ? 1 : 0);
  return nst <= 1 ? 1 : (r0 << (4 * (nst - 2)));
}

cudaError_t gb_launch_p2(const GbP2& k, cudaStream_t st) {
  if (k.epi.mode)
    return gb_p2_epi_supported(k.logn, k.load, k.store, k.posttw) ? dispatch_epi(k, st) : cudaErrorInvalidValue;
  if (k.load == GB_P2_LOAD_CONTIG && k.store == GB_P2_STORE_CONTIG)
    return dispatch<GB_P2_LOAD_CONTIG, GB_P2_STORE_CONTIG, false>(k, st);
  if (k.load == GB_P2_LOAD_CONTIG && k.store == GB_P2_STORE_COLS)
    return dispatch<GB_P2_LOAD_CONTIG, GB_P2_STORE_COLS, false>(k, st);
  if (k.load == GB_P2_LOAD_ROWS && k.store == GB_P2_STORE_CONTIG)
    return k.posttw ? dispatch<GB_P2_LOAD_ROWS, GB_P2_STORE_CONTIG, true>(k, st)
                    : dispatch<GB_P2_LOAD_ROWS, GB_P2_STORE_CONTIG, false>(k, st);
  if (k.load == GB_P2_LOAD_ROWS && k.store == GB_P2_STORE_COLS)
    return k.posttw ? dispatch<GB_P2_LOAD_ROWS, GB_P2_STORE_COLS, true>(k, st)
                    : dispatch<GB_P2_LOAD_ROWS, GB_P2_STORE_COLS, false>(k, st);
  return cudaErrorInvalidValue;
}
