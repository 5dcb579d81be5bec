// cluster.cu -- one-pass transforms of n = 2^13 .. 2^17 over a thread-block
// cluster, exchanging through distributed shared memory (sm_103a).
//
// Blocking for the memory hierarchy (sec. 3.3): a transform whose working set
// exceeds one CTA's shared memory still makes a single round trip to HBM when
// the C CTAs of a cluster hold it together.  The transform is one Cooley-Tukey
// step with n = n1 n2 (eq. (2)), input index l1 n2 + l2, output index
// k1 + n1 k2:
//   phase 1  CTA s loads the n1 x T tile of columns l2 in [s T, (s+1) T),
//            T = n2 / C (one tensor-map copy, rows of T contiguous elements),
//            computes the n1-point DFTs down the columns and multiplies by the
//            twiddles w_n^{l2 k1}; the results stay in its shared memory as
//            [k1][t];
//   exchange after a cluster barrier, CTA r reads rows k1 in [r R, (r+1) R),
//            R = n1 / C, from every CTA of the cluster (ld.shared::cluster,
//            128-bit) into padded rows of n2 points;
//   phase 2  CTA r computes the n2-point DFTs of its R rows and stores output
//            k1 + n1 k2 (R adjacent outputs per segment).
// Both phases use the compile-time Stockham stages of gb_p2_stages.cuh.
// Clusters are persistent over the batch; each CTA prefetches the tile of the
// transform two iterations ahead into the buffer whose exchange just ended.
// The landing buffer of a transform doubles as its phase-1 result, so a
// buffer is refilled only after the second cluster barrier of the iteration
// (no CTA reads it any more).  mbarrier waits are bounded by %globaltimer; a
// CTA whose wait gives up records FFT_ERR_DEVICE_TIMEOUT and skips the
// arithmetic of the remaining iterations but keeps taking part in every
// cluster barrier, so that the cluster never waits on an exited CTA.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <cstring>

#include "gb_kernels.h"
#include "gb_p2_stages.cuh"
#include "gb_tma.cuh"

namespace {

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// the shared::cluster address of local shared address a in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank) {
  uint32_t o;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(a), "r"(rank));
  return o;
}

__device__ __forceinline__ float4 ld_cluster_v4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}

template <int LOGN1, int LOGN2, int C, int NB>
struct CL {
  using A1 = P2<LOGN1>;
  using A2 = P2<LOGN2>;
  static constexpr int N1 = A1::N, N2 = A2::N;
  static constexpr int T = N2 / C;             // columns per CTA in phase 1
  static constexpr int R = N1 / C;             // rows per CTA in phase 2
  static constexpr int CP = N1 * N2 / C;       // points per CTA
  static constexpr int THREADS = CP / 16;
  static constexpr int XSZ = (T * A1::PITCH > R * A2::PITCH) ? T * A1::PITCH : R * A2::PITCH;
  static constexpr size_t SMEM = 128 + sizeof(float2) * (NB * (size_t)CP + XSZ);
  static constexpr int MINB = CP <= 4096 ? (NB == 1 ? 3 : 2) : 1;
  static_assert(T >= 2 && T % 2 == 0 && R >= 1, "tile shape");
  static_assert(THREADS % T == 0 && THREADS % R == 0, "thread mappings");
  static_assert(A1::NST >= 2 && A2::NST >= 2, "two stages at least on each side");
};

template <int LOGN1, int LOGN2, int C, int NB>
__global__ void __launch_bounds__(CL<LOGN1, LOGN2, C, NB>::THREADS, CL<LOGN1, LOGN2, C, NB>::MINB)
    gb_cluster_kernel(const __grid_constant__ GbCluster k, const __grid_constant__ CUtensorMap tm, int use_tm) {
  using G = CL<LOGN1, LOGN2, C, NB>;
  using A1 = typename G::A1;
  using A2 = typename G::A2;
  constexpr int T = G::T, R = G::R, CP = G::CP, THREADS = G::THREADS, N1 = G::N1, N2 = G::N2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  float2* lbuf = reinterpret_cast<float2*>(smem_raw + 128);
  float2* xbuf = lbuf + NB * CP;

  const int tid = threadIdx.x;
  const int rank = (int)cluster_rank();
  const int64_t cid = blockIdx.x / C, ncl = gridDim.x / C;
  const int tt = tid % T, ut = tid / T;                  // phase 1, lanes across columns
  const int tj = tid / A1::TPT, uj = tid % A1::TPT;      // phase 1, lanes along a column
  const int rs = tid % R, vs = tid / R;                  // phase 2, lanes across rows
  const int rj = tid / A2::TPT, vj = tid % A2::TPT;      // phase 2, lanes along a row

  auto issue = [&](int p, int64_t b) {
    const uint32_t bar = smem_addr(bars + p);
    expect_tx(bar, (uint32_t)(CP * 8));
    constexpr int BOXR = N1 < 256 ? N1 : 256;
#pragma unroll
    for (int r0 = 0; r0 < N1; r0 += BOXR)
      tensor_copy_3d(smem_addr(lbuf + p * CP + r0 * T), &tm, rank * T, r0, (int)b, bar);
  };

  if (use_tm && tid == 0) {
    for (int p = 0; p < NB; ++p)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + p)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (use_tm && tid == 0)
    for (int p = 0; p < NB; ++p)
      if (cid + p * ncl < k.count) issue(p, cid + p * ncl);

  bool bad = false;
  float2 v[16];
  for (int64_t it = 0;; ++it) {
    const int64_t b = cid + it * ncl;
    if (b >= k.count) break;
    const int p = NB == 1 ? 0 : (int)(it & 1);
    float2* L = lbuf + p * CP;
    if (use_tm) {
      const uint32_t parity = (uint32_t)((NB == 1 ? it : (it >> 1)) & 1);
      const bool ok = bad ? false : mbar_wait(smem_addr(bars + p), parity);
      if (__syncthreads_or(!ok)) {
        if (!bad && tid == 0 && k.status) gb_set_status(k.status, kStatusTimeout);
        bad = true;
      }
    } else {
      const float2* src = k.in + b * k.vis + rank * T;
      for (int i = tid; i < CP; i += THREADS) L[i] = src[(int64_t)(i / T) * N2 + (i % T)];
      __syncthreads();
    }
    if (!bad) {
      // phase 1: n1-point DFTs down the T columns, twiddled, into L as [k1][t]
      stage_in<LOGN1, 0, true, T>(v, L + tt, k.tw1, ut, k.conj);
      __syncthreads();
      stage_out_x<LOGN1, 0>(v, xbuf + tt * A1::PITCH, ut);
      __syncthreads();
      later_stages<LOGN1, 1, true>(v, xbuf + tj * A1::PITCH, xbuf + tt * A1::PITCH, L + tt, T, k.tw1, uj, ut, 0,
                                   true, k.ptwA, k.ptwB, (int64_t)rank * T + tt);
    }
    cluster_arrive();
    cluster_wait();  // every CTA's [k1][t] block is complete
    if (!bad) {
      // exchange: rows k1 in [rank R, (rank+1) R) from every CTA, sources staggered by rank
      constexpr int PER = R * T;
      const uint32_t base = smem_addr(L) + (uint32_t)(rank * PER * 8);
      float4 w[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = 2 * (tid + q * THREADS);
        const int si = e / PER, rem = e - si * PER;
        w[q] = ld_cluster_v4(map_rank(base + (uint32_t)rem * 8, (uint32_t)((si + rank) & (C - 1))));
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = 2 * (tid + q * THREADS);
        const int si = e / PER, rem = e - si * PER;
        const int s = (si + rank) & (C - 1);
        const int k1l = rem / T, c = s * T + rem % T;
        float2* row = xbuf + k1l * A2::PITCH;
        row[phys(c)] = make_float2(w[q].x, w[q].y);
        row[phys(c + 1)] = make_float2(w[q].z, w[q].w);
      }
    }
    __syncthreads();
    // this CTA no longer reads the cluster's blocks (the values are in its own
    // shared memory already, so the arrive needs no release)
    cluster_arrive_relaxed();
    if constexpr (NB == 1) {
      cluster_wait();  // no CTA reads L any more: refill it with the next transform
      if (use_tm && !bad && tid == 0 && b + ncl < k.count) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(0, b + ncl);
      }
    }
    if (!bad) {
      // phase 2: n2-point DFTs of the R rows; output k1 + n1 k2
      stage_in<LOGN2, 0, false, 1>(v, xbuf + rj * A2::PITCH, k.tw2, vj, 0);
      __syncthreads();
      stage_out_x<LOGN2, 0>(v, xbuf + rj * A2::PITCH, vj);
      __syncthreads();
      float2* gout = k.out + b * k.vos + rank * R + rs;
      later_stages<LOGN2, 1, false>(v, xbuf + rj * A2::PITCH, xbuf + rs * A2::PITCH, gout, N1, k.tw2, vj, vs,
                                    k.conj, true, nullptr, nullptr, 0);
    }
    if constexpr (NB == 2) {
      cluster_wait();  // no CTA reads L any more: refill it with the transform two ahead
      if (use_tm && !bad && tid == 0 && b + 2 * ncl < k.count) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(p, b + 2 * ncl);
      }
    } else {
      __syncthreads();  // xbuf reads of phase 2 done before the next phase 1
    }
  }
}

// input tensor map: dims (n2 columns, n1 rows, count), box (T, min(n1, 256), 1)
template <int LOGN1, int LOGN2, int C, int NB>
int make_map(const GbCluster& k, CUtensorMap* tm) {
  using G = CL<LOGN1, LOGN2, C, NB>;
  memset(tm, 0, sizeof(*tm));
  PFN_cuTensorMapEncodeTiled_v12000 enc = (PFN_cuTensorMapEncodeTiled_v12000)gb_tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(k.in) & 15) || (k.vis & 1) || k.vis <= 0 || k.count > (int64_t(1) << 31))
    return 0;
  cuuint64_t dim[3] = {(cuuint64_t)G::N2, (cuuint64_t)G::N1, (cuuint64_t)k.count};
  cuuint64_t str[2] = {(cuuint64_t)G::N2 * 8, (cuuint64_t)k.vis * 8};
  if (str[1] >= (cuuint64_t(1) << 40)) return 0;
  cuuint32_t box[3] = {(cuuint32_t)G::T, (cuuint32_t)(G::N1 < 256 ? G::N1 : 256), 1};
  cuuint32_t es[3] = {1, 1, 1};
  if (enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(k.in), dim, str, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 0;
  return 1;
}

template <int LOGN1, int LOGN2, int C, int NB>
cudaError_t prepare(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at, int* max_clusters) {
  using G = CL<LOGN1, LOGN2, C, NB>;
  auto fn = gb_cluster_kernel<LOGN1, LOGN2, C, NB>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  memset(cfg, 0, sizeof(*cfg));
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->blockDim = dim3(G::THREADS);
  cfg->gridDim = dim3(C);
  cfg->dynamicSmemBytes = G::SMEM;
  cfg->attrs = at;
  cfg->numAttrs = 1;
  *max_clusters = 0;
  return cudaOccupancyMaxActiveClusters(max_clusters, fn, cfg);
}

template <int LOGN1, int LOGN2, int C, int NB>
int max_active() {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  int n = 0;
  if (prepare<LOGN1, LOGN2, C, NB>(&cfg, at, &n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int LOGN1, int LOGN2, int C, int NB>
cudaError_t launch(const GbCluster& k, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  int maxc = 0;
  cudaError_t e = prepare<LOGN1, LOGN2, C, NB>(&cfg, at, &maxc);
  if (e != cudaSuccess) return e;
  if (maxc < 1) return cudaErrorInvalidConfiguration;
  int64_t ncl = k.clusters > 0 ? k.clusters : maxc;
  if (ncl > k.count) ncl = k.count;
  if (ncl < 1) return cudaSuccess;
  CUtensorMap tm;
  const int use = make_map<LOGN1, LOGN2, C, NB>(k, &tm);
  cfg.gridDim = dim3((unsigned)(ncl * C));
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, gb_cluster_kernel<LOGN1, LOGN2, C, NB>, k, tm, use);
}

// (logn1, logn2, C, landing buffers) of the instantiated kernels; for each n
// the preferred first.  One landing buffer leaves room for three CTAs per SM
// (the other CTAs cover the load of the next transform); two keep one load in
// flight per CTA.
#define GB_CLUSTER_CONFIGS(X) \
  X(6, 7, 2, 1)               \
  X(6, 7, 2, 2)               \
  X(7, 7, 4, 1)               \
  X(7, 7, 4, 2)               \
  X(7, 7, 2, 2)               \
  X(7, 8, 8, 1)               \
  X(7, 8, 8, 2)               \
  X(7, 8, 4, 2)               \
  X(7, 9, 16, 1)              \
  X(8, 8, 8, 2)               \
  X(8, 8, 16, 1)              \
  X(8, 9, 16, 2)

#define GB_ROW(A, B, Cs, Nb) {A + B, A, B, Cs, Nb},
constexpr int kConfigs[][5] = {GB_CLUSTER_CONFIGS(GB_ROW)};
#undef GB_ROW

}  // namespace

int gb_cluster_configs(int logn, int (*cfg)[4], int max_cfg) {
  int n = 0;
  for (const auto& c : kConfigs)
    if (c[0] == logn && n < max_cfg) {
      for (int i = 0; i < 4; ++i) cfg[n][i] = c[i + 1];
      ++n;
    }
  return n;
}

int gb_cluster_max_active(int logn1, int logn2, int csize, int nbuf) {
#define GB_CASE(A, B, Cs, Nb) \
  if (logn1 == A && logn2 == B && csize == Cs && nbuf == Nb) return max_active<A, B, Cs, Nb>();
  GB_CLUSTER_CONFIGS(GB_CASE)
#undef GB_CASE
  return 0;
}

cudaError_t gb_launch_cluster(const GbCluster& k, cudaStream_t st) {
#define GB_CASE(A, B, Cs, Nb) \
  if (k.logn1 == A && k.logn2 == B && k.csize == Cs && k.nbuf == Nb) return launch<A, B, Cs, Nb>(k, st);
  GB_CLUSTER_CONFIGS(GB_CASE)
#undef GB_CASE
  return cudaErrorInvalidValue;
}
