// l2fourstep.cu -- the radix-sqrt(n) step of eq. (2) for batches of
// contiguous power-of-two transforms, n = n1 n2 = 2^14 .. 2^22, with its
// intermediate kept in L2 (one HBM round trip per transform).
//
// The two passes of the four-step plan (sec. 3.3; eq. (2) with the twiddles
// w_n^{l2 k1} fused) become two kinds of work item of one persistent kernel:
//   A(t, j): columns l2 in [j T1, (j+1) T1) of transform t -- a tensor-map
//            box from HBM, the n1-point DFTs over l1, the twiddle, stored as
//            rows k1 of the transform's slot of a scratch ring (k1 n2 + l2);
//   B(t, j): rows k1 in [j T2, (j+1) T2) of that slot -- read back from L2,
//            the n2-point DFTs over l2, stored to Y[k1 + k2 n1] in HBM.
// The ring holds S transforms (slot t mod S), a few tens of MiB, so the
// intermediate stays in the 129 MB L2 instead of making a round trip
// through HBM; only the input reads and output writes reach DRAM.
//
// Order and dependencies.  CTAs take items one at a time from a device
// counter, in a fixed order: step k holds the A items of transform k and the
// B items of transform k - D (lag D), so a B item is taken about D steps
// after the A items it needs.  B(t, .) waits until all A items of t are done;
// A(t, .) waits, before writing its slot, until all B items of t - S are done
// (S > D).  An item only ever waits on items taken before it, by CTAs that
// are running, so the kernel cannot deadlock, with or without other kernels
// on the GPU.  Every wait is bounded by %globaltimer (2 s); a CTA whose wait
// gives up waits (bounded) for its copies in flight, records
// FFT_ERR_DEVICE_TIMEOUT and exits, and the CTAs that depend on it time out
// in turn.  Completion counters and the item counter are cleared by the host
// (cudaMemsetAsync) before each launch.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <cstring>

#include "gb_kernels.h"
#include "gb_p2_stages.cuh"
#include "gb_tma.cuh"

namespace {

struct ItemRef {
  int kind;     // 0 A, 1 B, -1 none
  int64_t t;    // transform
  int64_t j;    // tile within the transform
};

// item i of the fixed order (steps of D-lagged A and B items)
__device__ __forceinline__ ItemRef decode(int64_t i, int64_t count, int64_t D, int64_t nA, int64_t nB) {
  ItemRef r{-1, 0, 0};
  const int64_t head = D * nA, mid = (count - D) * (nA + nB), tail = D * nB;
  if (i < 0) return r;
  if (i < head) {
    r.kind = 0;
    r.t = i / nA;
    r.j = i - r.t * nA;
    return r;
  }
  i -= head;
  if (i < mid) {
    const int64_t k = D + i / (nA + nB), q = i - (i / (nA + nB)) * (nA + nB);
    if (q < nA) {
      r.kind = 0;
      r.t = k;
      r.j = q;
    } else {
      r.kind = 1;
      r.t = k - D;
      r.j = q - nA;
    }
    return r;
  }
  i -= mid;
  if (i < tail) {
    r.kind = 1;
    r.t = count - D + i / nB;
    r.j = i - (i / nB) * nB;
  }
  return r;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// bounded wait until *p >= target
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned target) {
  if (ld_acquire(p) >= target) return true;
  const unsigned long long t0 = globaltimer();
  while (ld_acquire(p) < target) {
    if (globaltimer() - t0 > kWaitLimitNs) return false;
    __nanosleep(64);
  }
  return true;
}

}  // namespace

namespace {

// an L2 policy that evicts the lines it touches first (the input and output
// streams), so that the ring keeps its place in L2
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tensor_copy_4d_ef(uint32_t dst, const void* tmap, int x, int y, int z, int w,
                                                  uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3, %4, %5}], [%6], %7;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The stages after stage 0 of one n-point DFT of an item, with the stage
// tables read from their copy in shared memory (tws); the last stage runs in
// the store mapping.  POSTTW multiplies output k = us + q L of column col by
// w_N^{col k} = pa s^q, where pa and s, s^2, s^4, s^8 (pb0, pb1) were loaded
// from the post-twiddle tables at the start of the item, so that their
// latency hides behind the stages.
template <int LOGN, int S, bool POSTTW, int NT>
__device__ __forceinline__ void item_stages(float2* v, float2* xrow_j, float2* xrow_s, float2* gout,
                                            int64_t ostride, const float2* tws, int uj, int us, int conj,
                                            float2 pa, float4 pb0, float4 pb1) {
  using C = P2<LOGN>;
  if constexpr (S == C::NST - 1) {
    static_assert(C::radix(S) == 16, "the last stage is radix 16");
    constexpr int L = C::L(S);
    stage_in<LOGN, S, false, 1, true>(v, xrow_s, tws, us, conj);
    float2 p[16];
    if constexpr (POSTTW) powers16v(p, pb0, pb1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      float2 x = v[q];
      if constexpr (POSTTW) x = cmul(x, q == 0 ? pa : cmul(pa, p[q]));
      if (conj) x.y = -x.y;
      if constexpr (POSTTW) gout[(int64_t)(us + q * L) * ostride] = x;  // the ring: stays in L2
      else __stcs(gout + (int64_t)(us + q * L) * ostride, x);            // the output stream
    }
  } else {
    stage_in<LOGN, S, false, 1, true>(v, xrow_j, tws, uj, conj);
    gb_bar<NT>();
    stage_out_x<LOGN, S>(v, xrow_j, uj);
    gb_bar<NT>();
    item_stages<LOGN, S + 1, POSTTW, NT>(v, xrow_j, xrow_s, gout, ostride, tws, uj, us, conj, pa, pb0, pb1);
  }
}

struct ItemSlot {
  long long t, j;
  int kind;  // 0 A, 1 B, -1 no more items, -2 abort
  int slot;  // t mod S, formed once by the producer (a 64-bit remainder)
};

template <int L1, int L2>
struct L2FSCfg {
  // items of 4096 points (two CTAs per SM) while a column tile is at least 16
  // columns wide; 8192 points (one CTA per SM, 8 columns and more) above,
  // where 4096-point items measured slower (2^18..2^21)
  static constexpr int TP = (L1 <= 8) ? 4096 : 8192;
  static constexpr int MINB = TP == 4096 ? 2 : 1;
  static constexpr int T1 = TP >> L1, T2 = TP >> L2;
  static constexpr int XB = (T1 * P2<L1>::PITCH > T2 * P2<L2>::PITCH) ? T1 * P2<L1>::PITCH : T2 * P2<L2>::PITCH;
  // NB item buffers, each first the landing tile of its item, then its
  // exchange rows (a multiple of 128 bytes, the bulk copies' alignment)
  static constexpr int NB = 3;
  static constexpr int BUFE = (((TP > XB) ? TP : XB) + 15) / 16 * 16;
  static constexpr int TW = P2<L1>::twoff(P2<L1>::NST) + P2<L2>::twoff(P2<L2>::NST);
  static constexpr size_t smem = 256 + sizeof(float2) * ((size_t)NB * BUFE + (size_t)TW);
};

// TP points per item (T1 = TP / n1 columns, T2 = TP / n2 rows), 16 values a
// compute thread, NT = TP / 16 compute threads plus two control warps, so
// that no compute warp ever stalls on a global round trip:
//   producer warp: takes the next item from the device counter (indices
//     fetched one ahead), waits (bounded) until its inputs are complete,
//     fills item buffer b (A: tensor-map boxes of the input, evict-first in
//     L2; B: one bulk copy of the ring rows, from L2) and arrives on full[b];
//   compute warps: wait on full[b], compute the item's stages (named barrier
//     1 among themselves) with buffer b as the exchange rows once the tile is
//     read, store, arrive on done[b] (one arrival per warp);
//   publisher warp: after done[b], hands buffer b back (pub[b]) and publishes
//     the item to the other CTAs (a gpu-scope fence, then the count).
// CONJ: the backward transform (inputs and outputs conjugated), a template
// argument so that the forward kernel carries no conjugation code.
// GB > 1: a B item takes T2 / GB consecutive rows k1 of GB consecutive
// transforms (a group) and stores outputs k = k1 + k2 n1 of transform t at
// out + off(t) + k os, off(t) = (t / nt1) vos2 + (t % nt1) vos: with vos = 1
// the GB transforms' outputs are adjacent, so strided outputs (the inner
// transforms of a larger four-step, whose outputs interleave) still store
// runs of GB x 8 bytes.  The schedule then runs in groups of GB transforms.
template <int L1, int L2, int TP, int MINB, int CONJ, int GB = 1>
__global__ void __launch_bounds__(TP / 16 + 64, MINB)
    gb_l2fs_kernel(const __grid_constant__ GbL2FS k, const __grid_constant__ CUtensorMap tm, int tmap_ok, int pos) {
  using CA = P2<L1>;
  using CB = P2<L2>;
  constexpr int N1 = CA::N, N2 = CB::N, T1 = TP / N1, T2 = TP / N2, NT = TP / 16;
  constexpr int64_t N = (int64_t)N1 * N2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int NB = L2FSCfg<L1, L2>::NB, BUFE = L2FSCfg<L1, L2>::BUFE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);                  // full[NB], done[NB], pub[NB]
  ItemSlot* info = reinterpret_cast<ItemSlot*>(smem_raw + 128);            // NB x 24 bytes
  float2* ibuf = reinterpret_cast<float2*>(smem_raw + 256);                // NB item buffers
  float2* twa = ibuf + NB * BUFE;        // stage tables of the n1-point DFTs
  float2* twb = twa + CA::twoff(CA::NST);  // and of the n2-point DFTs
  const int tid = threadIdx.x;
  // group mode: a B item holds RB consecutive rows k1 of the group's GB
  // transforms (RB GB = T2 rows of the tile)
  static_assert(GB == 1 || T2 % GB == 0, "a group's rows fill the tile");
  constexpr int RB = GB > 1 ? T2 / GB : T2;
  const int64_t NG = k.count / GB;  // groups (transforms when GB = 1)
  const int64_t nA = N2 / T1, nB = N1 / RB;  // A items per transform, B items per group
  const int64_t total = NG * (GB * nA + nB);

  if (tid == 0) {
    for (int b = 0; b < NB; ++b) {
      // full: one arrival per producer lane (lane 0's with the expected bytes
      // of the bulk copies) plus lane 0's release of info[b]
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + b)), "r"(33));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + NB + b)), "r"(NT / 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bars + 2 * NB + b)), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < CA::twoff(CA::NST); i += blockDim.x) twa[i] = k.tw1[i];
  for (int i = tid; i < CB::twoff(CB::NST); i += blockDim.x) twb[i] = k.tw2[i];
  __syncthreads();
  unsigned* ctr = k.sync;
  unsigned* doneA = k.sync + 1;
  unsigned* doneB = k.sync + 1 + NG;

  if (tid >= NT + 32) {
    // ---------------------------------------------------------------- publisher warp
    // after the compute warps finish item `it` (done[b]) it hands buffer b
    // back to the producer (pub[b]), then publishes the item to the other
    // CTAs: a gpu-scope fence (the compute warps' stores, ordered before
    // their arrival on done[b], become visible first), then the count.
    const int lane = tid - NT - 32;
    for (int b = 0, par = 0;; b = (b + 1 == NB) ? 0 : b + 1, par ^= (b == 0)) {
      if (!mbar_wait(smem_addr(bars + b), par)) {
        if (lane == 0) gb_set_status(k.status, kStatusTimeout);
        break;
      }
      const ItemSlot r = info[b];
      if (r.kind < 0) break;
      if (!mbar_wait(smem_addr(bars + NB + b), par)) {
        if (lane == 0) gb_set_status(k.status, kStatusTimeout);
        break;
      }
      if (lane == 0) {
        mbar_arrive(smem_addr(bars + 2 * NB + b));
        __threadfence();
        atomicAdd(r.kind == 0 ? doneA + r.t / GB : doneB + r.t, 1u);
      }
      __syncwarp();
    }
    return;
  }

  if (tid >= NT) {
    // ---------------------------------------------------------------- producer warp
    // takes the next item (indices fetched one ahead), waits (bounded) until
    // its inputs are complete -- B: the A items of its transform; A: the B
    // items of the transform whose slot it rewrites -- and fills landing
    // buffer b once the publisher has handed it back.
    const int lane = tid - NT;
    long long f_a = 0;
    if (lane == 0) f_a = (long long)atomicAdd(ctr, 1u);
    const uint64_t pol = evict_first_policy();
    unsigned tma = 0, tpar = 0;  // bit b: bulk copies in flight into buffer b, and their phase
    bool fail = false;
    int it = 0, b = 0;
    uint32_t ph = 0;  // phase of the buffers in this round of NB items
    for (;; ++it, b = (b + 1 == NB) ? 0 : b + 1, ph ^= (b == 0)) {
      const uint32_t full = smem_addr(bars + b);
      if (it >= NB) {
        if (!mbar_wait(smem_addr(bars + 2 * NB + b), ph ^ 1)) {
          fail = true;
          break;
        }
        tma &= ~(1u << b);
      }
      long long idx = 0;
      if (lane == 0) {
        // one claim ahead hides the atomic's round trip; two held items
        // longer before they started and measured slower
        idx = f_a;
        f_a = (long long)atomicAdd(ctr, 1u);
      }
      idx = __shfl_sync(0xffffffffu, idx, 0);
      ItemSlot r{0, 0, -1, 0};
      if (idx < total) {
        const ItemRef d = decode(idx, NG, k.D, GB * nA, nB);
        if (d.kind == 0) {
          const int64_t t = d.t * GB + d.j / nA;  // d.t: the group
          r = ItemSlot{t, d.j % nA, 0, (int)(GB == 1 ? t % k.S : d.t % (k.S / GB))};
        } else {
          r = ItemSlot{d.t, d.j, d.kind, (int)(d.t % (k.S / GB))};  // GB > 1: t is the group
        }
      }
      int ok = 1;
      if (lane == 0) {
        if (r.kind == 1) ok = wait_count(doneA + r.t, (unsigned)(GB * nA));
        else if (r.kind == 0 && r.t >= k.S) ok = wait_count(doneB + (r.t - k.S) / GB, (unsigned)nB);
        info[b] = r;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        fail = true;
        break;
      }
      __syncwarp();
      float2* dst = ibuf + b * BUFE;
      if ((r.kind == 0 && tmap_ok) || r.kind == 1) {
        if (lane == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          expect_tx(full, (uint32_t)(TP * 8));
          if (r.kind == 0) {
            constexpr int BOXR = N1 < 256 ? N1 : 256;
#pragma unroll
            for (int r0 = 0; r0 < N1; r0 += BOXR)
              tensor_copy_4d_ef(smem_addr(dst + r0 * T1), &tm, (int)(r.j * T1), map_coord(pos, 1, r0, (int)r.t, 0),
                                map_coord(pos, 2, r0, (int)r.t, 0), map_coord(pos, 3, r0, (int)r.t, 0), full, pol);
          } else {
            // B: the T2 ring rows are one contiguous run of TP points; the
            // other CTAs wrote them with ordinary stores, which the acquire
            // above made visible to this thread, and the proxy fence to its
            // bulk copy
            asm volatile("fence.proxy.async.global;" ::: "memory");
            if constexpr (GB == 1) {
              bulk_copy(smem_addr(dst), k.ring + (int64_t)r.slot * N + r.j * T2 * N2, (uint32_t)(TP * 8), full);
            } else {
              // row k1 = j of the group's transforms: adjacent in the group's
              // slot ([k1][transform][l2], as the A items store it)
              bulk_copy(smem_addr(dst), k.ring + (int64_t)r.slot * GB * N + r.j * RB * GB * N2, (uint32_t)(TP * 8),
                        full);
            }
          }
        } else {
          mbar_arrive(full);
        }
        tma |= 1u << b;
        tpar = (tpar & ~(1u << b)) | (ph << b);
      } else {
        mbar_arrive(full);  // an A item without tensor map (loaded by the compute warps), or the end
      }
      if (lane == 0) mbar_arrive(full);  // releases info[b] to the compute and publisher warps
      if (r.kind < 0) break;
    }
    if (fail) {
      // a wait gave up: stop the compute and publisher warps at the item they
      // wait for next (buffer b, not armed), then let copies in flight land
      if (lane == 0) {
        gb_set_status(k.status, kStatusTimeout);
        info[b] = ItemSlot{0, 0, -2, 0};
      }
      __syncwarp();
      mbar_arrive(smem_addr(bars + b));
      if (lane == 0) mbar_arrive(smem_addr(bars + b));
      for (int q = 0; q < NB; ++q)
        if ((tma >> q) & 1) mbar_wait(smem_addr(bars + q), (tpar >> q) & 1);
    }
    return;
  }

  // ---------------------------------------------------------------- compute warps
  // pass A mapping: lanes across the T1 columns (tile loads and column stores)
  const int at = tid % T1, au = tid / T1;
  const int aj = tid / CA::TPT, auj = tid % CA::TPT;
  // pass B mapping: lanes along a row for the loads, across the T2 rows for the stores
  const int bj = tid / CB::TPT, buj = tid % CB::TPT;
  const int bt = tid % T2, bu = tid / T2;
  float2 v[16];
  for (int b = 0, ph = 0;; b = (b + 1 == NB) ? 0 : b + 1, ph ^= (b == 0)) {
    if (!mbar_wait(smem_addr(bars + b), ph)) {
      if (tid == 0) gb_set_status(k.status, kStatusTimeout);
      break;
    }
    const ItemSlot r = info[b];
    if (r.kind < 0) break;
    float2* xbuf = ibuf + b * BUFE;  // the item's tile, then its exchange rows
    const float2* tile = xbuf;
    // the item's transform in the ring: slot [k1][l2] (GB = 1), or its rows
    // interleaved with the group's other transforms, [k1][t mod GB][l2]
    float2* slot = GB == 1 ? k.ring + (int64_t)r.slot * N : k.ring + (int64_t)r.slot * GB * N + (r.t % GB) * N2;
    if (r.kind == 0) {
      // ---- A(t, j): columns [j T1, (j+1) T1) of transform t into the slot
      const int64_t col = r.j * T1 + at;  // l2
      const float4* pb = reinterpret_cast<const float4*>(k.ptwB + col * 4);
      const float4 pb0 = __ldg(pb), pb1 = __ldg(pb + 1);
      const float2 pa = __ldg(k.ptwA + col * CA::L(CA::NST - 1) + au);
      if (tmap_ok) stage_in<L1, 0, true, T1>(v, tile + at, k.tw1, au, CONJ);
      else stage_in<L1, 0, true, N2>(v, k.in + r.t * k.vis + r.j * T1 + at, k.tw1, au, CONJ);
      gb_bar<NT>();  // the tile is read: its buffer takes the exchange rows
      stage_out_x<L1, 0>(v, xbuf + at * CA::PITCH, au);
      gb_bar<NT>();
      item_stages<L1, 1, true, NT>(v, xbuf + aj * CA::PITCH, xbuf + at * CA::PITCH, slot + col, GB * N2, twa, auj, au,
                                   CONJ, pa, pb0, pb1);
    } else {
      // ---- B(t, j): rows [j T2, (j+1) T2) of the slot into Y[k1 + k2 n1]
      const int64_t row0 = r.j * T2;
      stage_in<L2, 0, true, 1>(v, tile + bj * N2, k.tw2, buj, CONJ);
      gb_bar<NT>();  // the tile is read: its buffer takes the exchange rows
      stage_out_x<L2, 0>(v, xbuf + bj * CB::PITCH, buj);
      gb_bar<NT>();
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float2* gout;
      int64_t ostr;
      if constexpr (GB == 1) {
        gout = k.out + r.t * k.vos + row0 + bt;
        ostr = N1;
      } else {
        // tile row bt: row k1 = j RB + bt / GB of transform g GB + bt % GB
        const int t = (int)(r.t * GB) + bt % GB, nt1 = (int)k.nt1;
        gout = k.out + (int64_t)(t / nt1) * k.vos2 + (int64_t)(t % nt1) * k.vos + (r.j * RB + bt / GB) * k.os;
        ostr = (int64_t)N1 * k.os;
      }
      item_stages<L2, 1, false, NT>(v, xbuf + bj * CB::PITCH, xbuf + bt * CB::PITCH, gout, ostr, twb, buj, bu,
                                    CONJ, make_float2(0.f, 0.f), z4, z4);
    }
    // the warp's stores are done: one arrival per warp, after a warp barrier
    // that orders the other lanes' stores before lane 0's (release) arrival
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(smem_addr(bars + NB + b));
  }
}


template <int L1, int L2>
int grid_of() {
  using G = L2FSCfg<L1, L2>;
  auto fn = gb_l2fs_kernel<L1, L2, G::TP, G::MINB, 0>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, G::TP / 16 + 64, G::smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <int L1, int L2>
cudaError_t launch(const GbL2FS& k, cudaStream_t st) {
  using G = L2FSCfg<L1, L2>;
  const int64_t items = k.count * ((int64_t)(1 << L2) / G::T1 + (int64_t)(1 << L1) / G::T2);
  int64_t grid = k.grid > 0 ? k.grid : grid_of<L1, L2>();
  if (grid < 1) return cudaErrorInvalidConfiguration;
  if (grid > items) grid = items;
  cudaError_t e = cudaMemsetAsync(k.sync, 0, sizeof(unsigned) * gb_l2fs_sync_words(k.count, k.gb), st);
  if (e != cudaSuccess) return e;
  // the input's tensor map: dims (n2 columns, n1 rows, count transforms)
  GbP2 g{};
  g.logn = L1;
  g.load = GB_P2_LOAD_ROWS;
  g.in = k.in;
  g.V0 = 1 << L2;
  g.vis0 = 1;
  g.is = 1 << L2;
  g.nb1 = k.count;
  g.vis1 = k.vis;
  g.nb2 = 1;
  alignas(128) CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  int pos = 0;
  const int tmap_ok = gb_p2_rows_map(g, G::T1, &tm, &pos);
  auto go = [&](auto fn) -> cudaError_t {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem) != cudaSuccess)
      return cudaGetLastError();
    fn<<<(unsigned)grid, G::TP / 16 + 64, G::smem, st>>>(k, tm, tmap_ok, pos);
    return cudaGetLastError();
  };
  if (k.gb > 1) {
    // groups of 8 transforms: built for n = 256 x 256 (the inner transforms
    // of 2^22..2^24-point four-steps)
    if constexpr (L1 == 8 && L2 == 8) {
      if (k.gb != 8 || k.count % k.gb || k.S % k.gb || k.nt1 % k.gb) return cudaErrorInvalidValue;
      return k.conj ? go(gb_l2fs_kernel<L1, L2, G::TP, G::MINB, 1, 8>) : go(gb_l2fs_kernel<L1, L2, G::TP, G::MINB, 0, 8>);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  return k.conj ? go(gb_l2fs_kernel<L1, L2, G::TP, G::MINB, 1>) : go(gb_l2fs_kernel<L1, L2, G::TP, G::MINB, 0>);
}

#define GB_L2FS_CASES(X) X(7, 7) X(7, 8) X(8, 8) X(8, 9) X(9, 9) X(9, 10) X(10, 10) X(10, 11) X(11, 11)

}  // namespace

int gb_l2fs_supported(int logn1, int logn2) {
#define GB_L2FS_SUP(a, b) if (logn1 == a && logn2 == b) return 1;
  GB_L2FS_CASES(GB_L2FS_SUP)
#undef GB_L2FS_SUP
  return 0;
}

int gb_l2fs_tiles(int logn1, int logn2, int* T1, int* T2) {
#define GB_L2FS_T(a, b)                 \
  if (logn1 == a && logn2 == b) {       \
    *T1 = L2FSCfg<a, b>::T1;            \
    *T2 = L2FSCfg<a, b>::T2;            \
    return 1;                           \
  }
  GB_L2FS_CASES(GB_L2FS_T)
#undef GB_L2FS_T
  return 0;
}

int gb_l2fs_grid(int logn1, int logn2) {
#define GB_L2FS_G(a, b) if (logn1 == a && logn2 == b) return grid_of<a, b>();
  GB_L2FS_CASES(GB_L2FS_G)
#undef GB_L2FS_G
  return 0;
}

size_t gb_l2fs_sync_words(int64_t count, int gb) { return (size_t)(1 + 2 * (count / (gb > 1 ? gb : 1))); }

// groups of 8 transforms, B items over two rows of each: 3 % faster than 16
// transforms and one row (a B item then waits on 128 A items instead of 256)
int gb_l2fs_group(int logn1, int logn2) { return logn1 == 8 && logn2 == 8 ? 8 : 0; }

cudaError_t gb_launch_l2fs(const GbL2FS& k, cudaStream_t st) {
#define GB_L2FS_L(a, b) if (k.logn1 == a && k.logn2 == b) return launch<a, b>(k, st);
  GB_L2FS_CASES(GB_L2FS_L)
#undef GB_L2FS_L
  return cudaErrorInvalidValue;
}
