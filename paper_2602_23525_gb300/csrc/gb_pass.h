// gb_pass.h -- the descriptor of one pass of a plan, shared by the host
// planner (C++) and the CUDA kernels.
//
// A pass solves  dft({(n, is, os)}, V, I, O)  (sec. 4.1): a loop over up to
// GB_MAX_VDIMS vector dimensions of 1-D DFTs of length n, each computed
// inside one CTA by breadth-first Stockham stages (sec. 2, "auto-sort";
// each stage is one step of eq. (2) with a small radix R_s, so the output
// comes out in order without a digit-reversal pass).
//
// Stage s (radix R = radix[s], L = Ls[s] points already combined) maps the
// array A_s to A_{s+1}, where A_s[q L + k] (q < n/L, k < L) holds the
// length-L DFT, at frequency k, of the decimated subsequence x[q + i n/L].
// With j < n/R, k = j mod L, q = j div L:
//   A_{s+1}[q L R + k + L t] = sum_{r<R} w_R^{r t} ( w_{L R}^{r k} A_s[j + r n/R] )
// which is eq. (2) with n1 = L and n2 = R applied to every subsequence at
// once; A_0 = x and A_nst = DFT(x) in natural order.
//
// Optional twiddles make the pass one step of a multi-pass Cooley-Tukey
// plan (sec. 4.2, "Cooley-Tukey plans"; radix-sqrt(n), sec. 3.3):
//   post_tw: output k of the transform whose vector-dim-0 index is v is
//            multiplied by w_N^{v k}, from two sqrt(N) tables (sec. 6).
// The Bluestein mode fuses the whole chirp-z convolution (sec. 4.2, "Plans
// for prime sizes") of one transform into the CTA.
#pragma once
#include <stdint.h>

#define GB_MAX_STAGES 16
#define GB_MAX_VDIMS 6
#define GB_VALS 16            // complex values a thread holds in one stage

enum GbMove { GB_MOVE_DIRECT = 0, GB_MOVE_SMEM = 1 };
enum GbTileCopy { GB_COPY_ELEM_FAST = 0, GB_COPY_T_FAST = 1 };

// The descriptor lives in device memory owned by the plan; the data pointers
// are kernel arguments (plans do not depend on them).
struct GbPass {
  // ---- transform -----------------------------------------------------------
  int n;                // transform length (the convolution length m in Bluestein mode)
  int nst;              // number of Stockham stages
  int radix[GB_MAX_STAGES];
  int Ls[GB_MAX_STAGES];      // points combined before stage s
  int twstep[GB_MAX_STAGES];  // n / (Ls[s] * radix[s])
  const float2* tw;     // tw[m] = w_n^m (forward sign), m < n
  int64_t is, os;       // strides along the transform, in complex elements
  // ---- vector loops --------------------------------------------------------
  int nv;               // >= 1 (a length-1 dim is added when there are none)
  int64_t vn[GB_MAX_VDIMS], vis[GB_MAX_VDIMS], vos[GB_MAX_VDIMS];
  // ---- CTA tiling ----------------------------------------------------------
  int T;                // transforms per CTA, consecutive along vector dim 0
  int tpt;              // threads per transform
  int t_fast;           // 1: tid -> (t = tid % T, u = tid / T); 0: (t = tid / tpt, u = tid % tpt)
  int load_mode;        // GbMove
  int store_mode;       // GbMove
  int load_copy;        // GbTileCopy ordering of the smem tile copy
  int store_copy;
  int pitch;            // smem elements per transform (padded, odd)
  int64_t tiles0;       // ceil(vn[0] / T)
  int64_t ntiles;       // tiles0 * prod(vn[1..])
  // ---- sign ------------------------------------------------------------------
  int conj;             // 1: backward transform as conj(DFT_fwd(conj(x)))
  // ---- fused four-step twiddle ------------------------------------------------
  int post_tw;          // multiply out[k] of transform v by w_N^{c k}, c = its index along vector dim tw_dim
  int tw_dim;           // 0: c = the tile dimension's index; 1, 2: another vector dim
  int64_t twN;          // N
  int64_t twS;          // w_N^m = hi[m / S] * lo[m % S]
  const float2* tw_lo;  // lo[i] = w_N^i,      i < S
  const float2* tw_hi;  // hi[i] = w_N^{i S},  i <= N / S
  // ---- store epilogue (Bluestein's pointwise steps, gb_epi_apply) --------------
  const float2* epi_tab;  // table by output k = v0 + (index along the transform) * epi_kstride
  int64_t epi_K;          // outputs with k >= epi_K are not stored
  int64_t epi_kstride;
  int epi_mode;           // 0: none
  // ---- fused Bluestein (n = m, the convolution length) ------------------------
  int blue;             // 1: Y[k] = w_k * IDFT_m( DFT_m(x w) * Bhat )[k], k < bn
  int bn;               // true transform length (prime)
  const float2* bw;     // chirp w_l = exp(-pi i l^2 / bn), l < bn
  const float2* bB;     // Bhat[k] = DFT_m(b)[k] / m,  k < m
  // ---- device status -------------------------------------------------------------
  int* status;          // device status word (0 = ok)
};

// Strided rank-0 copy (the copy plan of sec. 4.2, "Rank-0 plans").
struct GbCopy {
  const float2* in;
  float2* out;
  int nv;
  int64_t vn[GB_MAX_VDIMS], vis[GB_MAX_VDIMS], vos[GB_MAX_VDIMS];
  int64_t total;
  int conj;             // unused by copies; kept 0
};
