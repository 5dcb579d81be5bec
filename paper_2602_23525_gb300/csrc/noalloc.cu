// noalloc.cu -- a batched 1-D transform that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a
// transform: a host thread that must not block on the device-wide
// synchronisation cudaMalloc/cudaFree may imply, a process whose device
// memory is owned entirely by another allocator (a framework's caching
// allocator or a fixed memory pool), or code running inside a callback that
// is not allowed to allocate.  fft_plan_dft allocates twiddle tables, pass
// descriptors and scratch, so it is not usable there.  This entry point
// runs the same two-pass Cooley-Tukey computation (the radix-sqrt(n) step:
// a pass of n2 DFTs of size n1 with the twiddles fused, into scratch, then
// a pass of n1 DFTs of size n2 into the output), but takes every piece of
// device memory it needs -- scratch, twiddle tables and the two pass
// descriptors -- from one file-scope static device array.  The paper has no
// counterpart: it is a deployment convenience of this library.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "gb_plan.hpp"

namespace {

// Static scratch: GBFFT_NOALLOC_MAX_POINTS complex values of data scratch plus
// a fixed area for twiddle tables and pass descriptors.  Every GPU that loads
// the library holds it until the process exits.
constexpr int64_t kMaxPoints = GBFFT_NOALLOC_MAX_POINTS;
constexpr int64_t kTableElems = 3 * 4096 + 2 * 2048 + 64;      // two root tables + split tables (+slack)
constexpr int64_t kDescElems = (2 * sizeof(GbPass) + 15) / 8 + 2;  // two descriptors, in float2 units
constexpr int64_t kTotalElems = kMaxPoints + kTableElems + kDescElems;

static __device__ __align__(256) float2 g_noalloc_scratch[kTotalElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device, looked up once
// per device (the symbol's host-side name is not a device address).
int scratch_address(float2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FFT_ERR_NO_DEVICE;
  }
  if (dev < 0 || dev >= kMaxDevices) return FFT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FFT_ERR_CUDA;
    }
    g_dev_ptr[dev] = (float2*)p;
  }
  *out = g_dev_ptr[dev];
  return FFT_OK;
}

// Writes the two pass descriptors into the static array.  They travel as
// kernel parameters, so no host buffer has to stay alive and nothing is
// copied from pageable memory (which would block the calling thread).
__global__ void gb_noalloc_desc_kernel(GbPass* d1, const __grid_constant__ GbPass p1, GbPass* d2,
                                       const __grid_constant__ GbPass p2) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *d1 = p1;
    *d2 = p2;
  }
}

bool smooth(int64_t n) { return gb::smooth_codelet(n); }

// n = n1 n2 with both factors codelet-smooth and at most 4096; n1 the largest
// such factor not above sqrt(n).
int64_t pick_n1(int64_t n) {
  int64_t best = 0;
  for (int64_t a = 2; a * a <= n; ++a)
    if (n % a == 0 && a <= 4096 && n / a <= 4096 && smooth(a) && smooth(n / a)) best = a;
  return best;
}

void fill_stages(GbPass& p, int64_t n) {
  const std::vector<int> rad = gb::default_radices(n);
  p.n = (int)n;
  p.nst = (int)rad.size();
  int64_t L = 1;
  for (int s = 0; s < p.nst; ++s) {
    p.radix[s] = rad[s];
    p.Ls[s] = (int)L;
    p.twstep[s] = (int)(n / (L * rad[s]));
    L *= rad[s];
  }
  p.tpt = gb::threads_per_transform(n, rad);
  p.pitch = gb::smem_pitch(n);
}

int pick_T(const GbPass& p, int want) {
  int T = want;
  const int64_t pitch_bytes = (int64_t)p.pitch * 8;
  while (T > 1 && (T * p.tpt > 1024 || T * pitch_bytes > gb::smem_limit())) T /= 2;
  return std::max(1, T);
}

}  // namespace

extern "C" int fft_execute_1d_noalloc(int64_t n, int64_t batch, int sign, const void* in, void* out,
                                      void* stream) {
  using namespace gb;
  if (!in || !out || n < 0 || batch < 0 || (sign != -1 && sign != 1)) return set_err(FFT_ERR_INVALID_ARG);
  if (n == 0 || batch == 0) return set_err(FFT_OK);
  if (batch > kMaxPoints / n || n * batch > kMaxPoints) return set_err(FFT_ERR_UNSUPPORTED);
  const int64_t n1 = pick_n1(n);
  if (n1 < 2) return set_err(FFT_ERR_UNSUPPORTED);
  const int64_t n2 = n / n1;
  const char* a0 = (const char*)in;
  const char* b0 = (const char*)out;
  const int64_t bytes = 8 * n * batch;
  if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes) return set_err(FFT_ERR_ALIAS);
  float2* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FFT_OK) return set_err(rc);
  cudaStream_t st = (cudaStream_t)stream;

  // carve the static array: data scratch | tables | descriptors
  float2* scratch = base;
  float2* tw1 = base + kMaxPoints;
  float2* tw2 = tw1 + 4096;
  int64_t S = (int64_t)std::ceil(std::sqrt((double)n));
  while (S * S < n) ++S;
  float2* lo = tw2 + 4096;
  float2* hi = lo + S;
  GbPass* d1 = (GbPass*)(base + kMaxPoints + kTableElems);
  GbPass* d2 = d1 + 1;

  // every table is rewritten by every call (the array keeps the last call's contents)
  if (gb_make_roots(tw1, n1, n1, 1, st) != cudaSuccess || gb_make_roots(tw2, n2, n2, 1, st) != cudaSuccess ||
      gb_make_roots(lo, S, n, 1, st) != cudaSuccess || gb_make_roots(hi, n / S + 1, n, S, st) != cudaSuccess)
    return set_err(FFT_ERR_CUDA);

  // pass 1: for each l2, the length-n1 DFT over l1 of x[l1 n2 + l2], times w_n^{l2 k1}
  GbPass p1;
  memset(&p1, 0, sizeof(p1));
  fill_stages(p1, n1);
  p1.tw = tw1;
  p1.is = n2;
  p1.os = n2;
  p1.nv = 2;
  p1.vn[0] = n2;    p1.vis[0] = 1; p1.vos[0] = 1;
  p1.vn[1] = batch; p1.vis[1] = n; p1.vos[1] = n;
  p1.t_fast = 1;
  p1.load_mode = p1.store_mode = GB_MOVE_DIRECT;
  p1.T = (int)std::min<int64_t>(pick_T(p1, 32), n2);
  p1.tiles0 = (n2 + p1.T - 1) / p1.T;
  p1.ntiles = p1.tiles0 * batch;
  p1.conj = sign > 0 ? 1 : 0;
  p1.post_tw = 1;
  p1.twN = n;
  p1.twS = S;
  p1.tw_lo = lo;
  p1.tw_hi = hi;

  // pass 2: for each k1, the length-n2 DFT over l2, written to Y[k1 + k2 n1]
  GbPass p2;
  memset(&p2, 0, sizeof(p2));
  fill_stages(p2, n2);
  p2.tw = tw2;
  p2.is = 1;
  p2.os = n1;
  p2.nv = 2;
  p2.vn[0] = n1;    p2.vis[0] = n2; p2.vos[0] = 1;
  p2.vn[1] = batch; p2.vis[1] = n;  p2.vos[1] = n;
  p2.t_fast = 0;
  p2.load_mode = p2.tpt >= 16 ? GB_MOVE_DIRECT : GB_MOVE_SMEM;
  p2.load_copy = GB_COPY_ELEM_FAST;
  p2.store_mode = GB_MOVE_SMEM;
  p2.store_copy = GB_COPY_T_FAST;
  p2.T = (int)std::min<int64_t>(pick_T(p2, 16), n1);
  p2.tiles0 = (n1 + p2.T - 1) / p2.T;
  p2.ntiles = p2.tiles0 * batch;
  p2.conj = p1.conj;

  gb_noalloc_desc_kernel<<<1, 32, 0, st>>>(d1, p1, d2, p2);
  if (cudaGetLastError() != cudaSuccess) return set_err(FFT_ERR_CUDA);
  const size_t sm1 = (size_t)p1.T * p1.pitch * sizeof(float2);
  const size_t sm2 = (size_t)p2.T * p2.pitch * sizeof(float2);
  if (gb_launch_pass(p1, d1, (const float2*)in, scratch, p1.T * p1.tpt, sm1, 0, st) != cudaSuccess ||
      gb_launch_pass(p2, d2, scratch, (float2*)out, p2.T * p2.tpt, sm2, 0, st) != cudaSuccess)
    return set_err(FFT_ERR_CUDA);
  return set_err(FFT_OK);
}
