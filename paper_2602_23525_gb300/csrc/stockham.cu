// stockham.cu -- the batched generic Stockham pass kernel, the rank-0 copy
// kernels and the launchers of these and of the persistent group kernel
// (group_kernel.cu) (sm_103a).  The stage code is in gb_generic_stages.cuh.
#include <cuda_runtime.h>

#include "gb_generic_stages.cuh"

namespace {

template <int MAXT>
__global__ void __launch_bounds__(MAXT)
    gb_stockham_kernel(const GbPass* __restrict__ P, const float2* in, float2* out) {
  extern __shared__ float2 sm[];
  for (int64_t tile = blockIdx.x; tile < P->ntiles; tile += gridDim.x) gb_pass_tile(*P, in, out, sm, tile, 0);
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

// In-place square transpose (the rank-0 problem of sec. 4.1.1 with I = O:
// dims da, db of equal length s whose input and output strides are swapped;
// every other dimension a batch loop with equal strides).  Element (i, j) at
// i sa + j sb moves to j sa + i sb.  A block takes one pair of 32 x 32 tiles
// (ti, tj), ti <= tj, of one batch index: both tiles are read into shared
// memory before either is written back into the other's place (a diagonal
// tile is transposed onto itself), so no element is overwritten before it
// is read, and pairs are disjoint.
__global__ void __launch_bounds__(256) gb_transpose_inplace_kernel(const GbCopy c, int da, int db) {
  __shared__ float2 A[32][33], B[32][33];
  float2* x = c.out;
  const int64_t s = c.vn[da], sa = c.vis[da], sb = c.vis[db];
  const int64_t T = (s + 31) / 32, npairs = T * (T + 1) / 2;
  const int64_t nrest = c.total / (s * s);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int64_t t = blockIdx.x; t < npairs * nrest; t += gridDim.x) {
    int64_t pair = t % npairs, rest = t / npairs, off = 0;
    for (int d = c.nv - 1; d >= 0; --d) {
      if (d == da || d == db) continue;
      const int64_t q = rest / c.vn[d], k = rest - q * c.vn[d];
      rest = q;
      off += k * c.vis[d];
    }
    int64_t ti = 0;
    while (pair >= T - ti) {  // upper triangle, row by row
      pair -= T - ti;
      ++ti;
    }
    const int64_t tj = ti + pair;
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
      const int64_t i = ti * 32 + k, j = tj * 32 + tx;
      if (i < s && j < s) A[k][tx] = x[off + i * sa + j * sb];
      const int64_t i2 = tj * 32 + k, j2 = ti * 32 + tx;
      if (ti != tj && i2 < s && j2 < s) B[k][tx] = x[off + i2 * sa + j2 * sb];
    }
    __syncthreads();
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
      // row tj*32 + k, column ti*32 + tx receives element (ti*32 + tx, tj*32 + k) of tile A
      const int64_t i = tj * 32 + k, j = ti * 32 + tx;
      if (i < s && j < s) x[off + i * sa + j * sb] = A[tx][k];
      const int64_t i2 = ti * 32 + k, j2 = tj * 32 + tx;
      if (ti != tj && i2 < s && j2 < s) x[off + i2 * sa + j2 * sb] = B[tx][k];
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t gb_launch_transpose_inplace(const GbCopy& c, cudaStream_t st) {
  if (c.total <= 0) return cudaSuccess;
  int da = -1, db = -1;
  for (int a = 0; a < c.nv && da < 0; ++a)
    for (int b = 0; b < c.nv; ++b)
      if (a != b && c.vn[a] == c.vn[b] && c.vn[a] > 1 && c.vis[a] == c.vos[b] && c.vos[a] == c.vis[b] &&
          c.vis[a] != c.vos[a]) {
        da = a;
        db = b;
        break;
      }
  if (da < 0 || c.in != c.out) return cudaErrorInvalidValue;
  const int64_t T = (c.vn[da] + 31) / 32;
  const int64_t tiles = T * (T + 1) / 2 * (c.total / (c.vn[da] * c.vn[da]));
  const int64_t blocks = tiles < 152 * 8 ? tiles : 152 * 8;
  gb_transpose_inplace_kernel<<<(unsigned)blocks, 256, 0, st>>>(c, da, db);
  return cudaGetLastError();
}

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

int gb_group_grid(int threads, size_t smem) { return gb_group_kernel_grid(threads, smem); }

cudaError_t gb_launch_group(const GbGroupArgs& a, int threads, size_t smem, int64_t grid, cudaStream_t st) {
  return gb_group_kernel_launch(a, threads, smem, grid, st);
}
