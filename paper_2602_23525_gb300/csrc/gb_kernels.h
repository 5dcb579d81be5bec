// gb_kernels.h -- host-side launchers of the library's CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gb_pass.h"

// Stockham pass (stockham.cu).  p is the host copy of the descriptor, dev its
// device copy (what the kernel reads).  grid <= 0 launches one CTA per tile.
cudaError_t gb_launch_pass(const GbPass& p, const GbPass* dev, const float2* in, float2* out, int threads,
                           size_t smem, int64_t grid, cudaStream_t st);
cudaError_t gb_launch_copy(const GbCopy& c, cudaStream_t st);
// in place (c.in == c.out): a square transpose of two dims whose input and
// output strides are swapped, batched over dims with equal strides
cudaError_t gb_launch_transpose_inplace(const GbCopy& c, cudaStream_t st);
int gb_pass_max_smem_optin(void);

// Power-of-two pass kernels with TMA tile loads (stockham_pow2.cu),
// n = 2^4 .. 2^13.  Transforms of length n along (is, os); the tile dimension
// (V0, vis0, vos0) holds T adjacent transforms per CTA; up to two more
// vector loops (nb1, vis1, vos1), (nb2, vis2, vos2).
enum { GB_P2_LOAD_CONTIG = 0, GB_P2_LOAD_ROWS = 1 };     // is == 1  |  vis0 == 1
enum { GB_P2_STORE_CONTIG = 0, GB_P2_STORE_COLS = 1 };   // os == 1  |  vos0 == 1
// Store epilogue of a last pass (Bluestein's pointwise steps, gb_epi_apply):
// output k = col + (index along the transform) * kstride, col the tile
// dimension's index; outputs with k >= K are not stored.  mode 0: none.
struct GbP2Epi {
  const float2* tab;
  int64_t K, kstride;
  int mode;
};
struct GbP2 {
  int logn, load, store, posttw;
  int prec;           // 0 FP32; tensor-core radix-16 stages: 1 FP16, 2 BF16, 3 FP16 split, 4 BF16 split
  const float2* in;   // set at execute time
  float2* out;
  int64_t V0, is, os, vis0, vos0;
  int64_t nb1, nb2, vis1, vos1, vis2, vos2;
  int conj;
  const float2* twt;   // per-stage [k][4] twiddle tables (gb_make_stage_twiddles)
  const float2* ptwA;  // post twiddle: A[c*L + j] = w_N^{c j}
  const float2* ptwB;  //               B[c] = (s, s^2, s^4, s^8), s = w_N^{c L}
  int ptw_dim;         // the column c: 0 the index along the tile dimension, 1 along nb1, 2 along nb2
  GbP2Epi epi;         // store epilogue (LOAD_CONTIG / STORE_COLS without post twiddle only)
  int* status;
  int64_t grid;        // <= 0: persistent grid sized by occupancy
};
int gb_p2_supported(int logn, int load, int store, int posttw);
int gb_p2_epi_supported(int logn, int load, int store, int posttw);  // a store epilogue is built
// tensor map (128 bytes at map, 64-byte aligned) of the LOAD_ROWS tiles of k
// with T columns: dims (V0, then the rows and the two vector loops ordered by
// stride), box T x min(n, 256) rows; returns 0 when the layout has none;
// *pos = the map dims (1..3) of the rows, nb1 and nb2, packed as
// rows | nb1 << 2 | nb2 << 4
int gb_p2_rows_map(const GbP2& k, int T, void* map, int* pos);
// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query, so the library needs no link-time libcuda); nullptr if unavailable
void* gb_tensor_map_encoder(void);
int gb_p2_tile(int logn, int load, int store);   // transforms per CTA tile
int gb_p2_small(int logn);                       // 1: n = 2^logn uses the small-transform kernel
int gb_p2_twiddle_elems(int logn);               // float2 entries of the stage tables
int gb_p2_stage(int logn, int s, int* L, int* R, int* offset);
int gb_p2_last_L(int logn);
cudaError_t gb_launch_p2(const GbP2& k, cudaStream_t st);
// one bounded wait on an mbarrier nothing arrives on; records the timeout code
cudaError_t gb_launch_stall(int* status, unsigned long long limit_ns, cudaStream_t st);
// tensor-core variants (tc.cu): 2^12 contiguous tiles, 2^8 contiguous or column tiles
int gb_tc_supported(int logn, int load, int store, int posttw);
int gb_tc_tile(int logn, int load, int store);
cudaError_t gb_launch_tc(const GbP2& k, cudaStream_t st);

// The four-step of eq. (2) with its intermediate kept in L2 (l2fourstep.cu):
// contiguous transforms of n = 2^logn1 x 2^logn2 points in a batch (count,
// vis, vos), one persistent kernel whose A items compute the n1-point column
// DFTs (+ w_n^{l2 k1}) into a ring of S transform slots and whose B items
// compute the n2-point row DFTs from the ring into the output (lag D < S).
struct GbL2FS {
  int logn1, logn2;        // column DFT length (pass A), row DFT length (pass B)
  const float2* in;        // set at execute time
  float2* out;
  float2* ring;            // S * n elements (scratch)
  unsigned* sync;          // [0] item counter, [1 + g] A items done, [1 + count / gb + g] B items done,
                           // g the transform (gb = 1) or group of gb transforms
  int64_t count, vis, vos;
  int64_t S, D;
  int conj;
  const float2* tw1;       // stage tables of n1 and n2 (gb_make_stage_twiddles)
  const float2* tw2;
  const float2* ptwA;      // w_n^{l2 k1}: gb_make_posttw(ncols = n2, L = last L of n1)
  const float2* ptwB;
  int* status;
  int64_t grid;            // <= 0: one CTA per SM times occupancy
  int gb;                  // 1, or gb_l2fs_group(): B items over row k1 of gb transforms
  int64_t os, nt1, vos2;   // gb > 1: output of transform t, element k at
                           // (t / nt1) vos2 + (t % nt1) vos + k os
};
// supported (logn1, logn2) and the tile shape: transforms' columns / rows per item
int gb_l2fs_supported(int logn1, int logn2);
int gb_l2fs_tiles(int logn1, int logn2, int* T1, int* T2);
// persistent CTAs the launch uses on the current device (for the lag D)
int gb_l2fs_grid(int logn1, int logn2);
size_t gb_l2fs_sync_words(int64_t count, int gb);  // unsigned words of k.sync
int gb_l2fs_group(int logn1, int logn2);  // transforms per B item in group mode (0: not built)
cudaError_t gb_launch_l2fs(const GbL2FS& k, cudaStream_t st);

// Single-pass transforms of n = 2^13 .. 2^17 spread over a thread-block
// cluster (cluster.cu): n = n1 x n2 (eq. (2)); CTA s of the cluster computes
// the n1-point DFTs of columns [s n2/C, (s+1) n2/C) with the twiddles
// w_n^{l2 k1}, the CTAs exchange through distributed shared memory, and CTA r
// computes the n2-point DFTs of rows [r n1/C, (r+1) n1/C).  Contiguous
// transforms (unit stride) in a batch (count, vis, vos).
struct GbCluster {
  int logn1, logn2, csize;  // n1 = 2^logn1, n2 = 2^logn2, CTAs per cluster
  int nbuf;                 // landing buffers per CTA (1 or 2)
  const float2* in;         // set at execute time
  float2* out;
  int64_t count, vis, vos;
  int conj;
  const float2* tw1;   // stage tables of n1 (gb_make_stage_twiddles)
  const float2* tw2;   // stage tables of n2
  const float2* ptwA;  // w_n^{l2 k1}: A[l2*L + j], B[l2*4 + i] (gb_make_posttw, ncols = n2, L = last L of n1)
  const float2* ptwB;
  int* status;
  int64_t clusters;    // <= 0: as many as are co-resident
};
// the (logn1, logn2, csize, nbuf) configurations of n = 2^logn, preferred
// first; returns the count
int gb_cluster_configs(int logn, int (*cfg)[4], int max_cfg);
// co-resident clusters of a configuration on the current device (0: cannot launch)
int gb_cluster_max_active(int logn1, int logn2, int csize, int nbuf);
cudaError_t gb_launch_cluster(const GbCluster& k, cudaStream_t st);

// Mixed-radix pass kernel with TMA tiles (stockham_mr.cu): one Stockham pass
// over transforms of length n <= GB_MR_MAX_N whose radix schedule (2, 3, 4,
// 5, 7, 8, 9, 11, 13, 16, and as the first stage one prime 17..61 computed by
// the generic O(R^2) DFT) comes at run time.  Tile shapes as for
// GbP2: LOAD_CONTIG / LOAD_ROWS, STORE_CONTIG / STORE_COLS; one extra vector
// loop; optional four-step post twiddle w_N^{col * k} from two sqrt(N) tables.
#define GB_MR_MAX_ST 8
#define GB_MR_MAX_N 8192
struct GbMR {
  int n, nst, T, tpt;
  int load, store, posttw, conj;
  int radix[GB_MR_MAX_ST], L[GB_MR_MAX_ST];
  unsigned Lmagic[GB_MR_MAX_ST];     // floor(2^32 / L) (quotients corrected once)
  const float2* tw[GB_MR_MAX_ST];    // stage s >= 1: [k][W] = w_{L R}^{r k}, W = even(R-1)
  const float2* in;                  // set at execute time
  float2* out;
  int64_t V0, is, os, vis0, vos0;    // tile dimension: V0 transforms
  int64_t nb1, vis1, vos1;           // one more vector loop
  const float2* ptw_lo;              // post twiddle w_N^m = hi[m / S] * lo[m % S]
  const float2* ptw_hi;
  unsigned ptwN, ptwS, ptwSmagic;
  const float2* wp;                  // stage 0 of radix > 16 (a prime 17..61): w_R^m, m < R
  int pitch;                         // padded exchange row (odd, in elements)
  int land;                          // landing elements per transform (n, or rows rounded to boxes)
  int* status;
  int64_t grid;                      // <= 0: persistent grid sized by occupancy
};
int gb_mr_threads(int n, const int* radix, int nst);   // threads per transform (<= 16 values each)
int gb_mr_tile(int n, int tpt, int load, int store, int64_t V0);  // transforms per tile (0: none fits)
size_t gb_mr_smem(const GbMR& k);
cudaError_t gb_launch_mr(const GbMR& k, cudaStream_t st);

// Bluestein helper kernels for convolution lengths beyond one CTA (bluestein.cu).
struct GbBlueIO {
  const float2* in;     // user input, element 0
  float2* out;          // user output, element 0
  float2* work;         // m * count contiguous scratch
  int64_t n, m;         // true length, convolution length
  int64_t is, os;       // transform strides
  int nv;
  int64_t vn[GB_MAX_VDIMS], vis[GB_MAX_VDIMS], vos[GB_MAX_VDIMS];
  int64_t count;        // product of vn
  const float2* w;      // chirp, n entries
  const float2* B;      // Bhat, m entries
  int conj;
};
cudaError_t gb_launch_blue_pre(const GbBlueIO& b, cudaStream_t st);     // work = pad(x w)
cudaError_t gb_launch_blue_mul(const GbBlueIO& b, float2* data, cudaStream_t st);  // data = conj(data Bhat)
cudaError_t gb_launch_blue_post(const GbBlueIO& b, const float2* data, cudaStream_t st);  // y = w conj(data)

// Rader's algorithm for a prime length p (rader.cu): a cyclic convolution of
// length p - 1 evaluated by FFTs of length L (p - 1, or >= 2p - 3 padded).
struct GbRaderIO {
  const float2* in;     // user input, element 0 (set at execute time)
  float2* out;          // user output, element 0
  int64_t p, L;         // prime length, convolution FFT length
  int64_t is, os;       // transform strides
  int nv;
  int64_t vn[GB_MAX_VDIMS], vis[GB_MAX_VDIMS], vos[GB_MAX_VDIMS];
  int64_t count;        // product of vn
  const int* perm;      // perm[r] = g^r mod p, r < p - 1
  const int* qidx;      // qidx[k] = q with g^{-q} = k mod p, 0 < k < p
  const float2* B;      // Bhat = DFT_L(b) / L, L entries
  int conj;
};
cudaError_t gb_launch_rader_pre(const GbRaderIO& b, float2* work, float2* side, cudaStream_t st);
cudaError_t gb_launch_rader_mul(const GbRaderIO& b, float2* data, float2* side, cudaStream_t st);
cudaError_t gb_launch_rader_post(const GbRaderIO& b, const float2* data, const float2* side, cudaStream_t st);

// Real-data steps (real.cu).  One transform of real length n per vector
// index; strides along the transform and of the vector loops in the units of
// the array each step reads or writes (FP32 values on a real side, complex64
// values on a complex side).
struct GbRealIO {
  int64_t n, m;        // real length, m = n / 2
  int64_t is, os;      // strides along the transform (input side, output side)
  int nv;
  int64_t vn[GB_MAX_VDIMS], vis[GB_MAX_VDIMS], vos[GB_MAX_VDIMS];
  int64_t count;       // product of vn
  const float2* tw;    // w_n^k = exp(-2 pi i k / n), k < n
};
// in place on the complex array z (element 0 of transform v at the vector
// offset, stride os): Z[k], k < m, the DFT of the real input read as m pairs
// -> X[k], k <= m (writes entry m)
cudaError_t gb_launch_r2c_post(const GbRealIO& r, float2* z, cudaStream_t st);
// real x (strides is, vis) -> dense complex w[v n + l] = (x, 0)
cudaError_t gb_launch_r2c_promote(const GbRealIO& r, const float* x, float2* w, cudaStream_t st);
// half spectrum X (strides is, vis) -> dense w[v m + k] = (X[k] + conj X[m-k]) + i w_n^{-k} (X[k] - conj X[m-k])
cudaError_t gb_launch_c2r_pre(const GbRealIO& r, const float2* X, float2* w, cudaStream_t st);
// half spectrum X -> dense w[v n + k], the conjugate-symmetric extension
cudaError_t gb_launch_c2r_expand(const GbRealIO& r, const float2* X, float2* w, cudaStream_t st);
// dense complex w[v n + l] -> real y (strides os, vos): y = Re w
cudaError_t gb_launch_c2r_real(const GbRealIO& r, const float2* w, float* y, cudaStream_t st);

// Persistent executor of several plans in one launch (stockham.cu).  Work
// items are (segment, tile); a segment is one step of one plan and may wait
// for the segment holding the previous step of the same plan.
enum { GB_SEG_PASS = 0, GB_SEG_COPY = 1, GB_SEG_BLUE_PRE = 2, GB_SEG_BLUE_MUL = 3, GB_SEG_BLUE_POST = 4 };
#define GB_SEG_CHUNK 4096  // elements per item of an element-wise segment
struct GbGroupSeg {
  int kind;
  int src, dst;          // slots of the per-execution pointer table
  int dep;               // segment that must complete first, or -1
  const GbPass* pass;    // GB_SEG_PASS: device descriptor
  GbBlueIO blue;         // Bluestein element-wise segments (pointers come from slots)
  GbCopy copy;           // GB_SEG_COPY
  int64_t ntiles;        // work items of the segment
  int64_t first;         // global index of its first item
};
struct GbGroupArgs {
  const GbGroupSeg* segs;
  int nseg;
  float2* const* bufs;          // pointer table
  unsigned long long* head;     // next item to hand out
  unsigned long long* done;     // completed items per segment
  int64_t total;                // items in the queue
  int* status;                  // FFT_ERR_DEVICE_TIMEOUT when a wait gives up
  unsigned long long wait_ns;   // bound of every dependency wait
};
cudaError_t gb_launch_group(const GbGroupArgs& a, int threads, size_t smem, int64_t grid, cudaStream_t st);
int gb_group_grid(int threads, size_t smem);

// FP64 table generation (tables.cu).
cudaError_t gb_make_roots(float2* out, int64_t count, int64_t N, int64_t mult, cudaStream_t st);
cudaError_t gb_make_chirp(float2* out, int64_t n, cudaStream_t st);
// out[k*4 + i] = w_N^{p k N/(L R)} for k < L and p = 1, 2, 4, 8 (i = log2 p)
cudaError_t gb_make_stage_twiddles(float2* out, int64_t N, int64_t L, int R, cudaStream_t st);
// out[k*W + r-1] = w_{L R}^{r k} for k < L, 0 < r < R, W = R-1 rounded up to
// even (mixed-radix stage tables; L*W entries, 16-byte rows)
cudaError_t gb_make_full_stage_twiddles(float2* out, int64_t L, int R, cudaStream_t st);
// four-step post twiddles w_N^{c k}, k = j + q L: A[c*L + j] = w_N^{c j},
// B[c*4 + i] = w_N^{c L 2^i}, for c < ncols, j < L
cudaError_t gb_make_posttw(float2* A, float2* B, int64_t N, int64_t ncols, int64_t L, cudaStream_t st);
cudaError_t gb_make_bluestein_kernel(float2* out, int64_t n, int64_t m, const int* radices, int nrad,
                                     double2* work, cudaStream_t st);
// Rader: Bhat = DFT_L(b) / L in FP64, b[m] = w_p^{ginv^m mod p} extended to L
// (work: 2 L double2; radices: a factorisation of L)
cudaError_t gb_make_rader_kernel(float2* out, int64_t p, int64_t ginv, int64_t L, const int* radices, int nrad,
                                 double2* work, cudaStream_t st);
