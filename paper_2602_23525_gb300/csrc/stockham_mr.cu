// stockham_mr.cu -- the mixed-radix Stockham pass kernel with TMA tiles
// (gb_mr_kernel.cuh): its host logic (threads per transform, tile choice,
// shared memory, launch) and the 256-thread instantiations.
#include "gb_mr_kernel.cuh"

int gb_mr_threads(int n, const int* radix, int nst) {
  int tpt = 1;
  for (int s = 0; s < nst; ++s) {
    const int R = radix[s];
    // at most 16 values per thread; the generic prime stage: 16 outputs
    const int need = R > 16 ? (n + 15) / 16 : (n / R + 16 / R - 1) / (16 / R);
    if (need > tpt) tpt = need;
  }
  return tpt;
}

// transforms per tile: the most that fit 512 threads and 4096 points (32 KB
// per landing buffer, two CTAs per SM), the fewest allowed when one alone is
// larger; column tiles need T to divide V0 and (strided loads) be even;
// contiguous tiles of odd lengths prefer an even T (whole 16-byte copies)
int gb_mr_tile(int n, int tpt, int load, int store, int64_t V0) {
  const bool cols = load == GB_P2_LOAD_ROWS || store == GB_P2_STORE_COLS;
  const int tmin = load == GB_P2_LOAD_ROWS ? 2 : 1;  // strided tiles: 16-byte box rows
  const bool odd_contig = !cols && (n % 2) != 0;
  // 256-thread CTAs (two per SM) unless a transform needs more threads or
  // the tile shape needs a wider CTA (an even tile for odd lengths or
  // strided loads)
  const int tmax = (tpt * tmin <= 256 && !(odd_contig && 2 * tpt > 256)) ? 256 / tpt : 512 / tpt;
  for (int pass = 0; pass < 2; ++pass) {
    for (int T = tmax; T >= 1; --T) {
      const int64_t cap = (pass == 0 && odd_contig && T == 2) ? 8192 : 4096;
      if ((int64_t)T * n > cap && T > tmin) continue;
      if (cols && (V0 % T != 0 || (load == GB_P2_LOAD_ROWS && T % 2 != 0))) continue;
      if (!cols && V0 < T) continue;
      if (pass == 0 && !cols && (n % 2) != 0 && (T % 2) != 0) continue;
      return T;
    }
  }
  return 0;
}

size_t gb_mr_smem(const GbMR& k) {
  const size_t tl = ((size_t)k.T * k.land + 15) & ~(size_t)15;  // as in the kernel
  return 128 + sizeof(float2) * (2 * tl + (size_t)k.T * k.pitch);
}

cudaError_t gb_mr_dispatch_256(const GbMR& k, cudaStream_t st) { return dispatch<256>(k, st); }

cudaError_t gb_launch_mr(const GbMR& k, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (gb_mr_dispatch_static(k, st, &e)) return e;
  if (k.T * k.tpt <= 256) return gb_mr_dispatch_256(k, st);
  if (k.T * k.tpt <= 512) return gb_mr_dispatch_512(k, st);
  return cudaErrorInvalidValue;
}
