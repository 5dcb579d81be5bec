// builder.cpp -- composition of algorithmic steps into a plan, and the
// measuring planner (sec. 4.2 and 4.3 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "gb_index.h"
#include "gb_plan.hpp"

namespace gb {

static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

static int64_t prod_n(const std::vector<Dim>& V) {
  int64_t c = 1;
  for (const Dim& d : V) c *= d.n;
  return c;
}

// Vector loops in canonical order: outermost first; adjacent stride runs merged.
static std::vector<Dim> canon_vec(std::vector<Dim> V) {
  std::vector<Dim> W;
  for (const Dim& d : V)
    if (d.n != 1) W.push_back(d);
  std::stable_sort(W.begin(), W.end(), [](const Dim& a, const Dim& b) {
    if (iabs64(a.os) != iabs64(b.os)) return iabs64(a.os) > iabs64(b.os);
    return iabs64(a.is) > iabs64(b.is);
  });
  std::vector<Dim> M;
  for (const Dim& d : W) {
    if (!M.empty()) {
      Dim& a = M.back();
      if (a.is == d.n * d.is && a.os == d.n * d.os) {
        a = {a.n * d.n, d.is, d.os};
        continue;
      }
    }
    M.push_back(d);
  }
  return M;
}

struct PostTw {
  int64_t N;
  int dim = 0;  // the column is the index along this vector dim (0: the tile dimension)
};

struct Builder {
  PlanData* P;
  bool device;
  bool measure;
  bool wisdom_only;
  std::ostringstream info;
  std::map<int64_t, const float2*> roots_cache;
  std::map<int64_t, std::pair<const float2*, const float2*>> split_cache;
  std::map<std::string, std::string> forced;  // choices imposed while timing a candidate
  int prec = 0;  // 0 FP32; tensor-core radix-16 stages: 1 FP16, 2 BF16, 3 FP16 split, 4 BF16 split
  int err = FFT_OK;

  Builder(PlanData* p, bool dev, bool meas, bool wonly) : P(p), device(dev), measure(meas), wisdom_only(wonly) {}

  void line(int depth, const std::string& s) { info << std::string(2 * depth, ' ') << s << "\n"; }

  void* dalloc(size_t bytes) {
    if (!device || err) return nullptr;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      err = FFT_ERR_OOM;
      return nullptr;
    }
    P->tables.push_back(ptr);
    return ptr;
  }

  // tw[m] = w_n^m, m < n (sec. 6: accurate precomputed table)
  const float2* roots(int64_t n) {
    auto it = roots_cache.find(n);
    if (it != roots_cache.end()) return it->second;
    float2* t = (float2*)dalloc(sizeof(float2) * n);
    if (t && gb_make_roots(t, n, n, 1, 0) != cudaSuccess) err = FFT_ERR_CUDA;
    roots_cache[n] = t;
    return t;
  }

  // two sqrt(N) tables: lo[i] = w_N^i (i < S), hi[i] = w_N^{i S} (i <= N/S)
  void split_roots(int64_t N, const float2** lo, const float2** hi, int64_t* S) {
    int64_t s = (int64_t)std::ceil(std::sqrt((double)N));
    while (s * s < N) ++s;
    *S = s;
    auto it = split_cache.find(N);
    if (it != split_cache.end()) {
      *lo = it->second.first;
      *hi = it->second.second;
      return;
    }
    const int64_t nhi = N / s + 1;
    float2* a = (float2*)dalloc(sizeof(float2) * s);
    float2* b = (float2*)dalloc(sizeof(float2) * nhi);
    if (a && b) {
      if (gb_make_roots(a, s, N, 1, 0) != cudaSuccess || gb_make_roots(b, nhi, N, s, 0) != cudaSuccess)
        err = FFT_ERR_CUDA;
    }
    split_cache[N] = {a, b};
    *lo = a;
    *hi = b;
  }

  // device copy of a pass descriptor, owned by the plan
  const GbPass* upload(const GbPass& p) {
    GbPass* d = (GbPass*)dalloc(sizeof(GbPass));
    if (d && cudaMemcpy(d, &p, sizeof(GbPass), cudaMemcpyHostToDevice) != cudaSuccess) err = FFT_ERR_CUDA;
    return d;
  }

  int new_scratch(size_t bytes) {
    const int id = BUF_SCRATCH0 + (int)P->scratch.size();
    void* ptr = nullptr;
    if (P->external_scratch) {
      // carved from the caller's work area at execute time, 256-byte aligned
      size_t off = 0;
      for (size_t b : P->scratch_bytes) off += (b + 255) & ~(size_t)255;
      P->scratch_offset.push_back(off);
    } else if (device && !err) {
      if (cudaMalloc(&ptr, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        err = FFT_ERR_OOM;
        ptr = nullptr;
      }
    }
    P->scratch.push_back(ptr);
    P->scratch_bytes.push_back(bytes);
    return id;
  }

  // ---------------------------------------------------------------- heuristics

  // Estimate-mode pass configuration: coalescing first, then ~256 threads per CTA.
  PassCfg estimate_cfg(const Dim& d, const Dim& v0, bool has_v, const std::vector<int>& rad) const {
    PassCfg c;
    c.radices = rad;
    const int tpt = threads_per_transform(d.n, rad);
    const bool in_e = iabs64(d.is) == 1, out_e = iabs64(d.os) == 1;
    const bool in_t = has_v && iabs64(v0.is) == 1, out_t = has_v && iabs64(v0.os) == 1;
    if (in_e && tpt >= 16) c.t_fast = 0;
    else if (in_t) c.t_fast = 1;
    else c.t_fast = 0;
    c.load_mode = (c.t_fast ? in_t : (in_e && tpt >= 16)) ? GB_MOVE_DIRECT : GB_MOVE_SMEM;
    c.store_mode = (c.t_fast ? out_t : (out_e && tpt >= 16)) ? GB_MOVE_DIRECT : GB_MOVE_SMEM;
    c.load_copy = (!has_v || iabs64(d.is) <= iabs64(v0.is)) ? GB_COPY_ELEM_FAST : GB_COPY_T_FAST;
    c.store_copy = (!has_v || iabs64(d.os) <= iabs64(v0.os)) ? GB_COPY_ELEM_FAST : GB_COPY_T_FAST;
    const bool want_wide = c.t_fast || (c.load_mode == GB_MOVE_SMEM && c.load_copy == GB_COPY_T_FAST) ||
                           (c.store_mode == GB_MOVE_SMEM && c.store_copy == GB_COPY_T_FAST);
    int T = want_wide ? 32 : std::max(1, 256 / tpt);
    const int64_t pitch_bytes = (int64_t)smem_pitch(d.n) * 8;
    const int64_t soft = 96 * 1024, hard = std::min<int64_t>(smem_limit(), 200 * 1024);
    while (T > 1 && T * tpt > 1024) T /= 2;
    while (T > 1 && T * pitch_bytes > soft && !(want_wide && T <= 8 && T * pitch_bytes <= hard)) T /= 2;
    while (T > 1 && T * pitch_bytes > hard) T /= 2;
    const int64_t vn0 = has_v ? v0.n : 1;
    while (T > 1 && T / 2 >= vn0) T /= 2;
    c.T = std::max(1, T);
    return c;
  }

  // n = n1 n2 for the radix-sqrt(n) step: n1 the largest codelet-smooth divisor
  // <= sqrt(n) whose cofactor is also smooth.
  int64_t estimate_split(int64_t n) const {
    const int lg = log2_exact(n);
    if (lg >= 12) {
      // powers of two: a near-square split, so that both passes are one-CTA
      // TMA passes up to 2^20; 2^22..2^24 as n1 x 65536, whose 65536-point
      // transforms the L2-resident four-step takes in groups; three passes
      // otherwise
      const int e1 = lg <= 20 ? lg / 2 : (lg >= 22 && lg <= 24) ? lg - 16 : (lg + 2) / 3;
      return (int64_t)1 << e1;
    }
    int64_t best = 0;
    for (int64_t a = 2; a * a <= n; ++a)
      if (n % a == 0 && smooth_codelet(a) && smooth_codelet(n / a) &&
          single_pass_ok(a, default_radices(a)))
        best = a;
    return best;
  }

  static int64_t bluestein_length(int64_t n) {
    int64_t m = 2 * n - 1;
    for (;; ++m) {
      int64_t r = m;
      for (int p : {2, 3, 5, 7})
        while (r % p == 0) r /= p;
      if (r == 1) return m;
    }
  }

  // ---------------------------------------------------------------- steps

  // the in-place rank-0 problems this library solves (sec. 4.2, rank-0 plans):
  // the identity, and a square transpose -- two dims of equal length with
  // their input and output strides swapped -- batched over dims with equal
  // strides.  Returns 0 none (identity), 1 transpose, -1 unsupported.
  static int inplace_permutation(const std::vector<Dim>& V, int* a, int* b) {
    int pa = -1, pb = -1;
    for (int i = 0; i < (int)V.size(); ++i) {
      if (V[i].is == V[i].os || V[i].n == 1) continue;
      if (pa < 0) pa = i;
      else if (pb < 0) pb = i;
      else return -1;
    }
    if (pa < 0) return 0;
    if (pb < 0) return -1;
    const Dim& x = V[pa];
    const Dim& y = V[pb];
    if (x.n != y.n || x.is != y.os || x.os != y.is) return -1;  // non-square in place: not built
    *a = pa;
    *b = pb;
    return 1;
  }

  void emit_copy(const std::vector<Dim>& V, int src, int dst, int depth) {
    if (src == dst) {
      int a = -1, b = -1;
      const int kind = inplace_permutation(V, &a, &b);
      if (kind < 0 || (int)V.size() > GB_MAX_VDIMS) {
        err = FFT_ERR_UNSUPPORTED;  // a non-square in-place transpose
        return;
      }
      if (kind == 0) {
        line(depth, "copy in place: nothing to do");
        return;
      }
      Step s;
      s.kind = STEP_TRANSPOSE_IP;
      s.src = src;
      s.dst = dst;
      s.copy.nv = (int)V.size();
      s.copy.total = 1;
      for (int i = 0; i < (int)V.size(); ++i) {
        s.copy.vn[i] = V[i].n;
        s.copy.vis[i] = V[i].is;
        s.copy.vos[i] = V[i].os;
        s.copy.total *= V[i].n;
      }
      P->steps.push_back(s);
      line(depth, "transpose in place " + std::to_string(V[a].n) + " x " + std::to_string(V[b].n) +
                      " (32 x 32 tile pairs swapped through shared memory) vdims=" + dims_str(V));
      return;
    }
    if ((int)V.size() > GB_MAX_VDIMS) {
      err = FFT_ERR_UNSUPPORTED;
      return;
    }
    Step s;
    s.kind = STEP_COPY;
    s.src = src;
    s.dst = dst;
    std::vector<Dim> W = V;
    std::stable_sort(W.begin(), W.end(), [](const Dim& a, const Dim& b) { return iabs64(a.is) > iabs64(b.is); });
    s.copy.nv = (int)W.size();
    s.copy.total = 1;
    for (int i = 0; i < (int)W.size(); ++i) {
      s.copy.vn[i] = W[i].n;
      s.copy.vis[i] = W[i].is;
      s.copy.vos[i] = W[i].os;
      s.copy.total *= W[i].n;
    }
    P->steps.push_back(s);
    line(depth, "copy (rank-0) vdims=" + dims_str(W));
  }

  void emit_single(const Dim& d, const std::vector<Dim>& Vin, int src, int dst, int conj, const PassCfg& cfg,
                   const PostTw* tw, int depth) {
    Step s;
    std::string desc;
    if (!make_single(d, Vin, src, dst, conj, cfg, tw, &s, &desc)) return;
    P->steps.push_back(s);
    line(depth, desc);
  }

  static std::string epi_str(const GbP2Epi& e) {
    static const char* what[] = {"", "Z = conj(y Bhat)", "y = w conj(D)", "y = conj(w conj(D))"};
    return std::string(" epilogue ") + what[e.mode & 3] + " for k < " + std::to_string(e.K);
  }

  bool make_single(const Dim& d, const std::vector<Dim>& Vin, int src, int dst, int conj, const PassCfg& cfg,
                   const PostTw* tw, Step* out, std::string* desc, const GbP2Epi* epi = nullptr) {
    std::vector<Dim> V = Vin;
    if (V.empty()) V.push_back({1, 0, 0});
    if ((int)V.size() > GB_MAX_VDIMS || (int)cfg.radices.size() > GB_MAX_STAGES) {
      err = FFT_ERR_UNSUPPORTED;
      return false;
    }
    GbPass p;
    memset(&p, 0, sizeof(p));
    p.n = (int)d.n;
    p.nst = (int)cfg.radices.size();
    int64_t L = 1;
    for (int s = 0; s < p.nst; ++s) {
      const int R = cfg.radices[s];
      p.radix[s] = R;
      p.Ls[s] = (int)L;
      p.twstep[s] = (int)(d.n / (L * R));
      L *= R;
    }
    if (L != d.n) {
      err = FFT_ERR_INVALID_ARG;
      return false;
    }
    p.tw = roots(d.n);
    p.is = d.is;
    p.os = d.os;
    p.nv = (int)V.size();
    for (int i = 0; i < p.nv; ++i) {
      p.vn[i] = V[i].n;
      p.vis[i] = V[i].is;
      p.vos[i] = V[i].os;
    }
    p.tpt = threads_per_transform(d.n, cfg.radices);
    p.T = (int)std::max<int64_t>(1, std::min<int64_t>(cfg.T, V[0].n));
    p.t_fast = cfg.t_fast;
    p.load_mode = cfg.load_mode;
    p.store_mode = cfg.store_mode;
    p.load_copy = cfg.load_copy;
    p.store_copy = cfg.store_copy;
    p.pitch = smem_pitch(d.n);
    p.tiles0 = (V[0].n + p.T - 1) / p.T;
    p.ntiles = p.tiles0;
    for (int i = 1; i < p.nv; ++i) p.ntiles *= V[i].n;
    p.conj = conj;
    if (epi) {
      p.epi_tab = epi->tab;
      p.epi_K = epi->K;
      p.epi_kstride = epi->kstride;
      p.epi_mode = epi->mode;
    }
    if (tw) {
      p.post_tw = 1;
      p.tw_dim = tw->dim;
      p.twN = tw->N;
      split_roots(tw->N, &p.tw_lo, &p.tw_hi, &p.twS);
    }
    p.status = P->d_status;
    Step s;
    s.kind = STEP_PASS;
    s.pass = p;
    s.dpass = upload(p);
    s.src = src;
    s.dst = dst;
    s.threads = p.T * p.tpt;
    const bool no_smem = p.nst == 1 && p.load_mode == GB_MOVE_DIRECT && p.store_mode == GB_MOVE_DIRECT;
    s.smem = no_smem ? 0 : (size_t)p.T * p.pitch * sizeof(float2);
    if (s.threads > 1024 || (int64_t)s.smem > smem_limit()) {
      err = FFT_ERR_UNSUPPORTED;
      return false;
    }
    std::ostringstream o;
    o << "pass stockham n=" << d.n << " is=" << d.is << " os=" << d.os << " cfg=" << cfg.str()
      << " tpt=" << p.tpt << " threads=" << s.threads << " smem=" << s.smem << " tiles=" << p.ntiles
      << " vdims=" << dims_str(V);
    if (tw) o << " post-twiddle w_" << tw->N << "^(v" << tw->dim << "*k)";
    if (epi) o << epi_str(*epi);
    if (conj) o << " conj";
    *out = s;
    *desc = o.str();
    return true;
  }

  static int log2_exact(int64_t n) {
    int e = 0;
    while ((int64_t(1) << e) < n) ++e;
    return (int64_t(1) << e) == n ? e : -1;
  }

  // The power-of-two TMA pass kernels (stockham_pow2.cu) apply to 2^6..2^13
  // points when one side is unit-stride along the transform (CONTIG) or along
  // the tile dimension (ROWS / COLS), and every offset a bulk copy starts at
  // is even (16 bytes).
  struct P2Choice {
    int logn = -1, load = -1, store = -1, T = 1, prec = 0;
    Dim v0{1, 0, 0};
    std::vector<Dim> rest;
  };

  static bool p2_choose(const Dim& d, const std::vector<Dim>& Vin, bool posttw, P2Choice* c, int prec = 0) {
    const int e = log2_exact(d.n);
    if (e < 0 || Vin.size() > 3) return false;
    const std::vector<Dim> V = order_for_pass(Vin);
    P2Choice ch;
    ch.logn = e;
    if (!V.empty()) ch.v0 = V[0];
    for (size_t i = 1; i < V.size(); ++i) ch.rest.push_back(V[i]);
    const Dim& v0 = ch.v0;
    const bool rows_ok = v0.is == 1 && (d.is % 2) == 0 && v0.n > 1;
    const bool cols_ok = v0.os == 1 && v0.n > 1;
    if (posttw) {
      ch.load = rows_ok ? GB_P2_LOAD_ROWS : -1;
      ch.store = cols_ok ? GB_P2_STORE_COLS : (d.os == 1 ? GB_P2_STORE_CONTIG : -1);
    } else {
      ch.load = d.is == 1 ? GB_P2_LOAD_CONTIG : (rows_ok ? GB_P2_LOAD_ROWS : -1);
      ch.store = d.os == 1 ? GB_P2_STORE_CONTIG : (cols_ok ? GB_P2_STORE_COLS : -1);
    }
    if (ch.load < 0 || ch.store < 0 || !gb_p2_supported(e, ch.load, ch.store, posttw ? 1 : 0)) return false;
    ch.T = gb_p2_tile(e, ch.load, ch.store);
    ch.prec = 0;
    if (prec && gb_tc_supported(e, ch.load, ch.store, posttw ? 1 : 0)) {
      ch.prec = prec;
      ch.T = gb_tc_tile(e, ch.load, ch.store);
      if ((ch.load == GB_P2_LOAD_ROWS || ch.store == GB_P2_STORE_COLS) && v0.n % ch.T != 0) ch.prec = 0;
      if (ch.prec == 0) ch.T = gb_p2_tile(e, ch.load, ch.store);
    }
    if (ch.load == GB_P2_LOAD_CONTIG && ch.store == GB_P2_STORE_CONTIG && gb_p2_small(e)) {
      // small transforms: adjacent on both sides, one vector loop
      if (!ch.rest.empty() || (v0.n > 1 && (v0.is != d.n || v0.os != d.n))) return false;
      ch.T = 4096 >> e;
    }
    if ((ch.load == GB_P2_LOAD_ROWS || ch.store == GB_P2_STORE_COLS) && v0.n % ch.T != 0) return false;
    if (ch.load == GB_P2_LOAD_CONTIG && v0.n > 1 && (v0.is % 2) != 0) return false;
    for (const Dim& r : ch.rest)
      if ((r.is % 2) != 0) return false;
    *c = ch;
    return true;
  }

  // ptw_dim: the post-twiddle column is the index along the tile dimension (0)
  // or along the pass's first / second other vector loop (1, 2; order_for_pass)
  void emit_p2(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t posttwN, int depth,
               int ptw_dim = 0, const GbP2Epi* epi = nullptr) {
    P2Choice c;
    if (!p2_choose(d, V, posttwN > 0, &c, prec) || (ptw_dim && (c.prec || ptw_dim > (int)c.rest.size())) ||
        (epi && (c.prec || !gb_p2_epi_supported(c.logn, c.load, c.store, posttwN > 0 ? 1 : 0)))) {
      err = FFT_ERR_WISDOM;
      return;
    }
    GbP2 k{};
    k.prec = c.prec;
    k.logn = c.logn;
    k.load = c.load;
    k.store = c.store;
    k.posttw = posttwN > 0 ? 1 : 0;
    k.V0 = c.v0.n;
    k.vis0 = c.v0.is;
    k.vos0 = c.v0.os;
    k.is = d.is;
    k.os = d.os;
    k.nb1 = k.nb2 = 1;
    if (c.rest.size() > 0) {
      k.nb1 = c.rest[0].n;
      k.vis1 = c.rest[0].is;
      k.vos1 = c.rest[0].os;
    }
    if (c.rest.size() > 1) {
      k.nb2 = c.rest[1].n;
      k.vis2 = c.rest[1].is;
      k.vos2 = c.rest[1].os;
    }
    k.conj = conj;
    k.ptw_dim = k.posttw ? ptw_dim : 0;
    if (epi) k.epi = *epi;
    k.status = P->d_status;
    float2* tw = (float2*)dalloc(sizeof(float2) * (size_t)std::max(16, gb_p2_twiddle_elems(c.logn)));
    for (int st = 1; tw && !err; ++st) {
      int L, R, off;
      if (!gb_p2_stage(c.logn, st, &L, &R, &off)) break;
      if (gb_make_stage_twiddles(tw + off, d.n, L, R, 0) != cudaSuccess) err = FFT_ERR_CUDA;
    }
    k.twt = tw;
    if (k.posttw) {
      const int64_t L = gb_p2_last_L(c.logn);
      const int64_t ncols = ptw_dim ? c.rest[ptw_dim - 1].n : k.V0;
      float2* A = (float2*)dalloc(sizeof(float2) * (size_t)(ncols * L));
      float2* B = (float2*)dalloc(sizeof(float2) * (size_t)(ncols * 4));
      if (A && B && gb_make_posttw(A, B, posttwN, ncols, L, 0) != cudaSuccess) err = FFT_ERR_CUDA;
      k.ptwA = A;
      k.ptwB = B;
    }
    // the generic pass over the same sub-problem runs when the input pointer
    // is not 16-byte aligned
    const std::vector<Dim> VV = order_for_pass(V);
    Dim v0{1, 0, 0};
    if (!VV.empty()) v0 = VV[0];
    PostTw tw2{posttwN, ptw_dim};
    Step s;
    std::string desc;
    if (!make_single(d, VV, src, dst, conj, estimate_cfg(d, v0, !VV.empty(), default_radices(d.n)),
                     k.posttw ? &tw2 : nullptr, &s, &desc, epi))
      return;
    s.kind = STEP_POW2;
    s.p2 = k;
    P->steps.push_back(s);
    static const char* ln[] = {"contig", "rows"};
    static const char* sn[] = {"contig", "cols"};
    std::ostringstream o;
    static const char* pn[] = {"p2-tma", "tc-fp16", "tc-bf16", "tc-fp16-split", "tc-bf16-split"};
    o << "pass " << pn[c.prec] << " n=" << d.n << " load=" << ln[c.load] << " store=" << sn[c.store] << " T=" << c.T
      << " is=" << d.is << " os=" << d.os << " tile=" << dims_str({c.v0}) << " rest=" << dims_str(c.rest)
      << (k.posttw ? " post-twiddle w_" + std::to_string(posttwN) + "^(v" + std::to_string(ptw_dim) + "*k)"
                   : std::string())
      << (epi ? epi_str(*epi) : std::string()) << (conj ? " conj" : "")
      << " (fallback: " << desc << ")";
    line(depth, o.str());
  }

  // Mixed-radix TMA pass kernel (stockham_mr.cu): smooth lengths that are not
  // powers of two, up to GB_MR_MAX_N points, at most two vector loops, tile
  // shapes as for the power-of-two kernels.
  struct MRChoice {
    int load = -1, store = -1, T = 0, tpt = 0;
    std::vector<int> rad;
    Dim v0{1, 0, 0};
    Dim rest{1, 0, 0};
  };

  // the prime factor of n beyond the codelet radices, if it is the only one
  // and lies in 17..61 (the generic O(p^2) stage); 0 for smooth n, -1 else
  static int generic_prime(int64_t n) {
    for (int p : {2, 3, 5, 7, 11, 13})
      while (n % p == 0) n /= p;
    if (n == 1) return 0;
    if (n < 17 || n > 61) return -1;
    for (int64_t f = 2; f * f <= n; ++f)
      if (n % f == 0) return -1;
    return (int)n;
  }

  static bool mr_choose(const Dim& d, const std::vector<Dim>& Vin, bool posttw, MRChoice* c) {
    if (d.n < 2 || d.n > GB_MR_MAX_N || log2_exact(d.n) >= 0 || Vin.size() > 2) return false;
    const int gp = generic_prime(d.n);
    if (gp < 0) return false;
    const std::vector<Dim> V = order_for_pass(Vin);
    MRChoice ch;
    if (gp) {
      ch.rad.push_back(gp);
      if (d.n > gp)
        for (int R : default_radices(d.n / gp)) ch.rad.push_back(R);
    } else {
      ch.rad = default_radices(d.n);
    }
    if (ch.rad.empty() || ch.rad.size() > GB_MR_MAX_ST || (ch.rad.size() < 2 && !gp)) return false;
    if (!V.empty()) ch.v0 = V[0];
    if (V.size() > 1) ch.rest = V[1];
    const Dim& v0 = ch.v0;
    const bool rows_ok = v0.is == 1 && v0.n > 1;
    const bool cols_ok = v0.os == 1 && v0.n > 1;
    if (posttw) {
      ch.load = rows_ok ? GB_P2_LOAD_ROWS : -1;
      ch.store = cols_ok ? GB_P2_STORE_COLS : -1;
    } else {
      ch.load = d.is == 1 ? GB_P2_LOAD_CONTIG : (rows_ok ? GB_P2_LOAD_ROWS : -1);
      ch.store = d.os == 1 ? GB_P2_STORE_CONTIG : (cols_ok ? GB_P2_STORE_COLS : -1);
    }
    if (ch.load < 0 || ch.store < 0) return false;
    // a single stage loads and stores with one thread mapping
    if (ch.rad.size() == 1 && (ch.load == GB_P2_LOAD_ROWS) != (ch.store == GB_P2_STORE_COLS)) return false;
    ch.tpt = gb_mr_threads((int)d.n, ch.rad.data(), (int)ch.rad.size());
    if (ch.tpt > 512) return false;
    ch.T = gb_mr_tile((int)d.n, ch.tpt, ch.load, ch.store, v0.n);
    if (ch.T < 1) return false;
    *c = ch;
    return true;
  }

  void emit_mr(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t posttwN, int depth) {
    MRChoice c;
    if (!mr_choose(d, V, posttwN > 0, &c)) {
      err = FFT_ERR_WISDOM;
      return;
    }
    GbMR k{};
    k.n = (int)d.n;
    k.nst = (int)c.rad.size();
    k.T = c.T;
    k.tpt = c.tpt;
    k.load = c.load;
    k.store = c.store;
    k.posttw = posttwN > 0 ? 1 : 0;
    k.conj = conj;
    int64_t L = 1;
    for (int s = 0; s < k.nst; ++s) {
      const int R = c.rad[s];
      k.radix[s] = R;
      k.L[s] = (int)L;
      k.Lmagic[s] = L > 1 ? (unsigned)((uint64_t(1) << 32) / (uint64_t)L) : 0u;
      if (s > 0) {
        float2* t = (float2*)dalloc(sizeof(float2) * (size_t)(L * (R & ~1)));
        if (t && gb_make_full_stage_twiddles(t, L, R, 0) != cudaSuccess) err = FFT_ERR_CUDA;
        k.tw[s] = t;
      }
      L *= R;
    }
    k.V0 = c.v0.n;
    k.vis0 = c.v0.is;
    k.vos0 = c.v0.os;
    k.is = d.is;
    k.os = d.os;
    k.nb1 = c.rest.n;
    k.vis1 = c.rest.is;
    k.vos1 = c.rest.os;
    if (k.posttw) {
      const float2 *lo = nullptr, *hi = nullptr;
      int64_t S = 0;
      split_roots(posttwN, &lo, &hi, &S);
      k.ptw_lo = lo;
      k.ptw_hi = hi;
      k.ptwN = (unsigned)posttwN;
      k.ptwS = (unsigned)S;
      k.ptwSmagic = (unsigned)((uint64_t(1) << 32) / (uint64_t)S);
    }
    if (c.rad[0] > 16) {
      float2* w = (float2*)dalloc(sizeof(float2) * (size_t)c.rad[0]);
      if (w && gb_make_roots(w, c.rad[0], c.rad[0], 1, 0) != cudaSuccess) err = FFT_ERR_CUDA;
      k.wp = w;
    }
    k.pitch = smem_pitch(d.n);
    const int boxr = d.n < 256 ? (int)d.n : 256;
    k.land = c.load == GB_P2_LOAD_ROWS ? (int)((d.n + boxr - 1) / boxr * boxr) : (int)d.n;
    k.status = P->d_status;
    if ((int64_t)gb_mr_smem(k) > smem_limit()) {
      err = FFT_ERR_WISDOM;
      return;
    }
    // the generic pass over the same sub-problem: what the persistent group
    // queue runs (none for a prime radix beyond the codelets)
    const std::vector<Dim> VV = order_for_pass(V);
    Dim v0{1, 0, 0};
    if (!VV.empty()) v0 = VV[0];
    PostTw tw2{posttwN};
    Step s;
    std::string desc = "none";
    if (c.rad[0] <= 16 &&
        !make_single(d, VV, src, dst, conj, estimate_cfg(d, v0, !VV.empty(), default_radices(d.n)),
                     k.posttw ? &tw2 : nullptr, &s, &desc))
      return;
    s.src = src;
    s.dst = dst;
    s.kind = STEP_MR;
    s.mr = k;
    P->steps.push_back(s);
    static const char* ln[] = {"contig", "rows"};
    static const char* sn[] = {"contig", "cols"};
    std::ostringstream o;
    o << "pass mr-tma n=" << d.n << " R=";
    for (size_t i = 0; i < c.rad.size(); ++i) o << (i ? "." : "") << c.rad[i];
    o << " load=" << ln[c.load] << " store=" << sn[c.store] << " T=" << c.T << " tpt=" << c.tpt << " is=" << d.is
      << " os=" << d.os << " tile=" << dims_str({c.v0}) << " rest=" << dims_str({c.rest})
      << (k.posttw ? " post-twiddle w_" + std::to_string(posttwN) + "^(v0*k)" : std::string()) << (conj ? " conj" : "")
      << " (group fallback: " << desc << ")";
    line(depth, o.str());
  }

  // "transpose first" applies to an out-of-place transform whose output is
  // contiguous per transform while its input is strided with a unit-stride
  // vector loop; all output strides non-negative (the scratch copy of the
  // output layout starts at element 0)
  static bool xpose_ok(const Dim& d, const std::vector<Dim>& V) {
    if (d.os != 1 || d.is == 1 || d.is == 0 || V.empty() || V.size() > 3) return false;
    bool unit_in = false;
    for (const Dim& v : V) {
      if (v.os <= 0) return false;
      if (v.is == 1) unit_in = true;
    }
    return unit_in;
  }

  void emit_xpose(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int depth) {
    if (!xpose_ok(d, V) || src == dst) {
      err = FFT_ERR_WISDOM;
      return;
    }
    int64_t lo = 0, hi = 0;
    footprint({d}, V, false, &lo, &hi);
    line(depth, "transpose first: the input into the output's layout, then the transform (sec. 4.2.4 copy + sec. 4.2)");
    const int S = new_scratch((size_t)(hi + 1) * sizeof(float2));
    std::vector<Dim> W;
    W.push_back({d.n, d.is, d.os});
    for (const Dim& v : V) W.push_back(v);
    emit_copy(canon_vec(W), src, S, depth + 1);
    std::vector<Dim> V2;
    for (const Dim& v : V) V2.push_back({v.n, v.os, v.os});
    solve_rank1({d.n, d.os, d.os}, V2, S, dst, conj, depth + 1);
  }

  // One-pass cluster kernel (cluster.cu) for contiguous transforms of
  // 2^13..2^17 points, at most one vector loop.
  static bool cluster_ok(const Dim& d, const std::vector<Dim>& V) {
    const int e = log2_exact(d.n);
    if (e < 13 || e > 17 || d.is != 1 || d.os != 1 || V.size() > 1) return false;
    if (!V.empty() && (V[0].is <= 0 || V[0].os <= 0)) return false;
    return true;
  }

  bool cluster_parse(const std::string& c, int* l1, int* l2, int* cs, int* nb) {
    return sscanf(c.c_str(), "cluster:%d.%d.%d.%d", l1, l2, cs, nb) == 4;
  }

  void emit_cluster(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int l1, int l2, int cs,
                    int nb, int depth) {
    const int e = log2_exact(d.n);
    int cfg[16][4];
    const int nc = gb_cluster_configs(e, cfg, 16);
    bool known = false;
    for (int i = 0; i < nc; ++i) known |= cfg[i][0] == l1 && cfg[i][1] == l2 && cfg[i][2] == cs && cfg[i][3] == nb;
    if (!known || !cluster_ok(d, V)) {
      err = FFT_ERR_WISDOM;
      return;
    }
    GbCluster k{};
    k.logn1 = l1;
    k.logn2 = l2;
    k.csize = cs;
    k.nbuf = nb;
    k.count = V.empty() ? 1 : V[0].n;
    k.vis = V.empty() ? d.n : V[0].is;
    k.vos = V.empty() ? d.n : V[0].os;
    k.conj = conj;
    k.status = P->d_status;
    const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
    float2* t1 = (float2*)dalloc(sizeof(float2) * (size_t)std::max(16, gb_p2_twiddle_elems(l1)));
    float2* t2 = (float2*)dalloc(sizeof(float2) * (size_t)std::max(16, gb_p2_twiddle_elems(l2)));
    for (int st = 1; t1 && t2 && !err; ++st) {
      int L, R, off, any = 0;
      if (gb_p2_stage(l1, st, &L, &R, &off)) {
        any = 1;
        if (gb_make_stage_twiddles(t1 + off, n1, L, R, 0) != cudaSuccess) err = FFT_ERR_CUDA;
      }
      if (gb_p2_stage(l2, st, &L, &R, &off)) {
        any = 1;
        if (gb_make_stage_twiddles(t2 + off, n2, L, R, 0) != cudaSuccess) err = FFT_ERR_CUDA;
      }
      if (!any) break;
    }
    const int64_t Ll = gb_p2_last_L(l1);
    float2* A = (float2*)dalloc(sizeof(float2) * (size_t)(n2 * Ll));
    float2* B = (float2*)dalloc(sizeof(float2) * (size_t)(n2 * 4));
    if (A && B && gb_make_posttw(A, B, d.n, n2, Ll, 0) != cudaSuccess) err = FFT_ERR_CUDA;
    k.tw1 = t1;
    k.tw2 = t2;
    k.ptwA = A;
    k.ptwB = B;
    Step s;
    std::string desc = "none";
    std::vector<int> rad = default_radices(d.n);
    if (single_pass_ok(d.n, rad)) {
      // a one-CTA pass over the same sub-problem (the persistent group executor runs that)
      Dim v0 = V.empty() ? Dim{1, 0, 0} : V[0];
      const int saved = err;
      if (!make_single(d, V, src, dst, conj, estimate_cfg(d, v0, !V.empty(), rad), nullptr, &s, &desc)) {
        err = saved;  // no fallback: the plan still runs, only not inside a group
        s = Step();
        desc = "none";
      }
    }
    s.src = src;
    s.dst = dst;
    s.kind = STEP_CLUSTER;
    s.cl = k;
    P->steps.push_back(s);
    std::ostringstream o;
    o << "pass cluster n=" << d.n << " = " << n1 << " x " << n2 << " C=" << cs << " buffers=" << nb << " (eq. 2 over " << cs
      << " CTAs, distributed shared memory exchange) T=" << n2 / cs << " R=" << n1 / cs << " count=" << k.count
      << " vis=" << k.vis << " vos=" << k.vos << (conj ? " conj" : "") << " (one-CTA fallback: " << desc << ")";
    line(depth, o.str());
  }

  static bool same_dim(const Dim& a, const Dim& b) { return a.n == b.n && a.is == b.is && a.os == b.os; }

  // Four-step with the scratch layout [l2][k1][vector index] and one vector
  // loop of unit input and output stride innermost (the transform runs down
  // the columns of a row-major array: a rank-2/3 dimension other than the
  // last, or a batch-fastest layout).  Both passes then tile along that loop
  // (rows of adjacent columns in, rows out), and the pass-1 twiddle w_n^{l2 k1}
  // takes its column l2 from a vector loop.  Returns false, emitting nothing,
  // where the layout does not apply.
  bool emit_fourstep_cols(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t n1,
                          int depth) {
    if (prec || d.is == 1 || V.empty() || V.size() > 2) return false;
    int vs = -1;
    for (int i = 0; i < (int)V.size(); ++i)
      if (V[i].n > 1 && V[i].is == 1 && V[i].os == 1) vs = i;
    if (vs < 0) return false;
    const int64_t n = d.n, n2 = n / n1, count = prod_n(V);
    // scratch strides: loop vs 1, the other loop next, k1 count, l2 n1 count
    std::vector<Dim> Vs(V.size());
    int64_t st = 1;
    for (int i : {vs, 1 - vs}) {
      if (i < 0 || i >= (int)V.size()) continue;
      Vs[i] = {V[i].n, V[i].is, st};
      st *= V[i].n;
    }
    const Dim l2{n2, d.is, n1 * count};
    std::vector<Dim> V1{Vs[vs], l2};
    if (V.size() == 2) V1.push_back(Vs[1 - vs]);
    const Dim d1{n1, n2 * d.is, count};
    const std::vector<Dim> O = order_for_pass(V1);
    P2Choice pc;
    if (!same_dim(O[0], Vs[vs]) || !p2_choose(d1, V1, true, &pc) || pc.load != GB_P2_LOAD_ROWS ||
        pc.store != GB_P2_STORE_COLS)
      return false;
    int pos = -1;
    for (int i = 1; i < (int)O.size(); ++i)
      if (same_dim(O[i], l2)) pos = pos < 0 ? i : 99;  // unique match only
    if (pos < 1 || pos > 2) return false;
    std::ostringstream o;
    o << "cooley-tukey n=" << n << " = " << n1 << " x " << n2 << " (radix-" << n1
      << " step, eq. 2; columns innermost in the scratch)";
    line(depth, o.str());
    const int S = new_scratch((size_t)count * n * sizeof(float2));
    // pass 1: n2 x count DFTs of size n1 over l1, twiddle w_n^{l2 k1}
    emit_p2(d1, V1, src, S, conj, n, depth + 1, pos);
    if (err) return true;
    // pass 2: n1 x count DFTs of size n2 over l2, output Y[k1 + k2 n1]
    std::vector<Dim> V2{{n1, count, d.os}, {V[vs].n, 1, V[vs].os}};
    if (V.size() == 2) V2.push_back({V[1 - vs].n, Vs[1 - vs].os, V[1 - vs].os});
    solve_rank1({n2, n1 * count, n1 * d.os}, V2, S, dst, conj, depth + 1);
    return true;
  }

  // Four-step for a batch-fastest input and transform-contiguous output (a
  // vector loop b of unit input stride, d.os == 1): the scratch [l2][b][k1]
  // keeps each pass-1 transform's outputs contiguous, so that pass 1 loads
  // tiles of adjacent b (rows over l1) and stores whole transforms (twiddle
  // column l2 from a vector loop), and pass 2 loads tiles of adjacent k1
  // (rows over l2) and stores them as adjacent outputs k1 + n1 k2: two passes
  // where transposing first takes three.  Returns false, emitting nothing,
  // where the layout does not apply.
  bool emit_fourstep_bfin(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t n1,
                          int depth, bool dry = false) {
    if (n1 < 2 || d.n % n1 != 0) return false;
    if (prec || d.is == 1 || d.os != 1 || V.empty() || V.size() > 2) return false;
    int vb = -1;
    for (int i = 0; i < (int)V.size(); ++i)
      if (V[i].n > 1 && V[i].is == 1 && V[i].os != 1) vb = i;
    if (vb < 0) return false;
    const int64_t n = d.n, n2 = n / n1, count = prod_n(V);
    const int vo = V.size() == 2 ? 1 - vb : -1;
    // scratch strides: k1 1, loop vb n1, the other loop n1 * V[vb].n, l2 n1 * count
    const Dim b1{V[vb].n, 1, n1};
    const Dim l2{n2, d.is, n1 * count};
    std::vector<Dim> V1{b1, l2};
    if (vo >= 0) V1.push_back({V[vo].n, V[vo].is, n1 * V[vb].n});
    const Dim d1{n1, n2 * d.is, 1};
    const std::vector<Dim> O = order_for_pass(V1);
    P2Choice pc;
    if (!same_dim(O[0], b1) || !p2_choose(d1, V1, true, &pc) || pc.load != GB_P2_LOAD_ROWS ||
        pc.store != GB_P2_STORE_CONTIG)
      return false;
    int pos = -1;
    for (int i = 1; i < (int)O.size(); ++i)
      if (same_dim(O[i], l2)) pos = pos < 0 ? i : 99;  // unique match only
    if (pos < 1 || pos > 2) return false;
    // pass 2 must tile along k1 (rows over l2, adjacent outputs)
    std::vector<Dim> V2{{n1, 1, 1}, {V[vb].n, n1, V[vb].os}};
    if (vo >= 0) V2.push_back({V[vo].n, n1 * V[vb].n, V[vo].os});
    const Dim d2{n2, n1 * count, n1};
    P2Choice pc2;
    if (!p2_choose(d2, V2, false, &pc2) || !same_dim(pc2.v0, V2[0]) || pc2.load != GB_P2_LOAD_ROWS ||
        pc2.store != GB_P2_STORE_COLS)
      return false;
    if (dry) return true;
    std::ostringstream o;
    o << "cooley-tukey n=" << n << " = " << n1 << " x " << n2 << " (radix-" << n1
      << " step, eq. 2; batch-fastest input, scratch [l2][b][k1])";
    line(depth, o.str());
    const int S = new_scratch((size_t)count * n * sizeof(float2));
    emit_p2(d1, V1, src, S, conj, n, depth + 1, pos);
    if (err) return true;
    emit_p2(d2, V2, S, dst, conj, 0, depth + 1);
    return true;
  }

  void emit_fourstep(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t n1,
                     int depth) {
    if (emit_fourstep_cols(d, V, src, dst, conj, n1, depth)) return;
    if (emit_fourstep_bfin(d, V, src, dst, conj, n1, depth)) return;
    const int64_t n = d.n, n2 = n / n1;
    std::ostringstream o;
    o << "cooley-tukey n=" << n << " = " << n1 << " x " << n2 << " (radix-" << n1 << " step, eq. 2)";
    line(depth, o.str());
    const int64_t count = prod_n(V);
    const int S = new_scratch((size_t)count * n * sizeof(float2));
    // scratch layout: [vector index][k1][l2]
    std::vector<Dim> Vs(V.size());
    int64_t st = n;
    for (int i = (int)V.size() - 1; i >= 0; --i) {
      Vs[i] = {V[i].n, V[i].is, st};
      st *= V[i].n;
    }
    // pass 1: n2 DFTs of size n1 over l1 (input stride n2 is), twiddle w_n^{l2 k1}
    std::vector<Dim> V1;
    V1.push_back({n2, d.is, 1});
    for (const Dim& v : Vs) V1.push_back(v);
    const Dim d1{n1, n2 * d.is, n2};
    P2Choice pc;
    MRChoice mc;
    if (p2_choose(d1, V1, true, &pc) && order_for_pass(V1)[0].n == n2 && order_for_pass(V1)[0].os == 1) {
      emit_p2(d1, V1, src, S, conj, n, depth + 1);
    } else if (!prec && n <= 0xffffffffLL && mr_choose(d1, V1, true, &mc) && order_for_pass(V1)[0].n == n2 &&
               order_for_pass(V1)[0].os == 1) {
      emit_mr(d1, V1, src, S, conj, n, depth + 1);
    } else {
      PassCfg c1 = estimate_cfg(d1, V1[0], true, default_radices(n1));
      PostTw tw{n};
      emit_single(d1, V1, src, S, conj, c1, &tw, depth + 1);
    }
    // sub-problem: n1 DFTs of size n2 over l2, output Y[k1 + k2 n1]
    std::vector<Dim> V2;
    V2.push_back({n1, n2, d.os});
    int64_t st2 = n;
    for (int i = (int)V.size() - 1; i >= 0; --i) {
      V2.push_back({V[i].n, st2, V[i].os});
      st2 *= V[i].n;
    }
    solve_rank1({n2, 1, n1 * d.os}, V2, S, dst, conj, depth + 1);
  }

  // Bluestein's convolution FFTs (m = n1 n2 a power of two, 2^14 .. 2^24) as
  // two four-step passes each (eq. (2)) whose last pass applies the pointwise
  // step as it stores: Z = conj(A Bhat) after the first FFT, y = w conj(D)
  // straight into the output after the second (only k < n), so neither step
  // makes a round trip through HBM of its own.  The work buffers hold the
  // transforms contiguously, the caller's loops in order, the last fastest (as
  // the pre step writes them); the output needs unit stride along k.
  struct BlueFused {
    int64_t n1, n2;
    Dim d1, d2;
    std::vector<Dim> V1, V2w, V2y;
  };

  bool blue_fused_plan(const Dim& d, const std::vector<Dim>& V, int64_t m, BlueFused* f) {
    const int lg = log2_exact(m);
    if (prec || lg < 14 || lg > 24 || d.os != 1 || V.size() > 2) return false;
    f->n1 = (int64_t)1 << (lg / 2);
    f->n2 = m / f->n1;
    const int64_t n1 = f->n1, n2 = f->n2, count = prod_n(V);
    f->d1 = {n1, n2, n2};  // [v][l1 n2 + l2] -> [v][k1 n2 + l2], twiddle w_m^{l2 k1}
    f->V1 = {{n2, 1, 1}, {count, m, m}};
    f->d2 = {n2, 1, n1};   // [v][k1 n2 + l2] -> Y[v][k1 + k2 n1]
    f->V2w = {{n1, n2, 1}, {count, m, m}};
    f->V2y = {{n1, n2, 1}};
    int64_t st = m;
    std::vector<Dim> Vy(V.size());
    for (int i = (int)V.size() - 1; i >= 0; --i) {
      Vy[i] = {V[i].n, st, V[i].os};
      st *= V[i].n;
    }
    for (const Dim& v : Vy)
      if (v.n > 1) f->V2y.push_back(v);
    P2Choice c1, cw, cy;
    if (!p2_choose(f->d1, f->V1, true, &c1) || !p2_choose(f->d2, f->V2w, false, &cw) ||
        !p2_choose(f->d2, f->V2y, false, &cy))
      return false;
    if (!same_dim(c1.v0, f->V1[0]) || c1.load != GB_P2_LOAD_ROWS || c1.store != GB_P2_STORE_COLS) return false;
    for (const P2Choice* c : {&cw, &cy})
      if (!same_dim(c->v0, f->V2w[0]) || !gb_p2_epi_supported(c->logn, c->load, c->store, 0)) return false;
    return true;
  }

  bool blue_fused_ok(const Dim& d, const std::vector<Dim>& V, int64_t m) {
    BlueFused f;
    return blue_fused_plan(d, V, m, &f);
  }

  void emit_blue_fused(const Dim& d, const std::vector<Dim>& V, int dst, int conj, int64_t m, const float2* w,
                       const float2* B, int S0, int S1, int depth) {
    BlueFused f;
    if (!blue_fused_plan(d, V, m, &f)) {
      err = FFT_ERR_UNSUPPORTED;
      return;
    }
    std::ostringstream o;
    o << "cooley-tukey m=" << m << " = " << f.n1 << " x " << f.n2 << " (eq. 2), the multiply fused into its store";
    line(depth, o.str());
    const GbP2Epi mul{B, m, f.n1, 1};
    emit_p2(f.d1, f.V1, S0, S1, 0, m, depth + 1);
    emit_p2(f.d2, f.V2w, S1, S0, 0, 0, depth + 1, 0, &mul);
    std::ostringstream q;
    q << "cooley-tukey m=" << m << " = " << f.n1 << " x " << f.n2 << " (eq. 2), y = w conj(D) fused into its store";
    line(depth, q.str());
    const GbP2Epi post{w, d.n, f.n1, conj ? 3 : 2};
    emit_p2(f.d1, f.V1, S0, S1, 0, m, depth + 1);
    emit_p2(f.d2, f.V2y, S1, dst, 0, 0, depth + 1, 0, &post);
  }

  void emit_bluestein(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t m,
                      int depth) {
    const int64_t n = d.n;
    std::vector<int> rad = default_radices(m);
    std::ostringstream o;
    o << "bluestein n=" << n << " m=" << m << " (chirp-z, prime-size plan)";
    line(depth, o.str());
    float2* w = (float2*)dalloc(sizeof(float2) * n);
    float2* B = (float2*)dalloc(sizeof(float2) * m);
    if (device && !err) {
      // FP64 work of the chirp's transform: stream-ordered allocation, since
      // a plain cudaFree would wait for every stream of the device (a plan
      // made while other transforms run would stall them)
      double2* work = nullptr;
      if (cudaMallocAsync((void**)&work, sizeof(double2) * 2 * m, 0) != cudaSuccess) {
        cudaGetLastError();
        err = FFT_ERR_OOM;
        return;
      }
      if (gb_make_chirp(w, n, 0) != cudaSuccess ||
          gb_make_bluestein_kernel(B, n, m, rad.data(), (int)rad.size(), work, 0) != cudaSuccess)
        err = FFT_ERR_CUDA;
      if (cudaFreeAsync(work, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) err = FFT_ERR_CUDA;
    }
    std::vector<Dim> VV = V;
    if (VV.empty()) VV.push_back({1, 0, 0});
    const bool fused = single_pass_ok(m, rad) && (int)VV.size() <= GB_MAX_VDIMS;
    if (fused) {
      GbPass p;
      memset(&p, 0, sizeof(p));
      p.n = (int)m;
      p.nst = (int)rad.size();
      int64_t L = 1;
      for (int s = 0; s < p.nst; ++s) {
        p.radix[s] = rad[s];
        p.Ls[s] = (int)L;
        p.twstep[s] = (int)(m / (L * rad[s]));
        L *= rad[s];
      }
      p.tw = roots(m);
      p.is = d.is;
      p.os = d.os;
      p.nv = (int)VV.size();
      for (int i = 0; i < p.nv; ++i) {
        p.vn[i] = VV[i].n;
        p.vis[i] = VV[i].is;
        p.vos[i] = VV[i].os;
      }
      p.tpt = threads_per_transform(m, rad);
      p.T = 1;
      p.pitch = smem_pitch(m);
      p.load_mode = p.store_mode = GB_MOVE_SMEM;
      p.tiles0 = VV[0].n;
      p.ntiles = prod_n(VV);
      p.conj = conj;
      p.blue = 1;
      p.bn = (int)n;
      p.bw = w;
      p.bB = B;
      p.status = P->d_status;
      Step s;
      s.kind = STEP_PASS;
      s.pass = p;
      s.dpass = upload(p);
      s.src = src;
      s.dst = dst;
      s.threads = p.tpt;
      s.smem = (size_t)p.pitch * sizeof(float2);
      P->steps.push_back(s);
      std::ostringstream q;
      q << "pass bluestein-fused m=" << m << " radices=" << PassCfg{rad}.str() << " threads=" << s.threads
        << " smem=" << s.smem << " vdims=" << dims_str(VV);
      line(depth + 1, q.str());
      return;
    }
    if ((int)V.size() > GB_MAX_VDIMS) {
      err = FFT_ERR_UNSUPPORTED;
      return;
    }
    const int64_t count = prod_n(V);
    const bool fuse = blue_fused_ok(d, V, m);
    const int S0 = new_scratch((size_t)count * m * sizeof(float2));
    const int S1 = new_scratch((size_t)count * m * sizeof(float2));
    GbBlueIO b;
    memset(&b, 0, sizeof(b));
    b.n = n;
    b.m = m;
    b.is = d.is;
    b.os = d.os;
    b.nv = (int)V.size();
    for (int i = 0; i < b.nv; ++i) {
      b.vn[i] = V[i].n;
      b.vis[i] = V[i].is;
      b.vos[i] = V[i].os;
    }
    b.count = count;
    b.w = w;
    b.B = B;
    b.conj = conj;
    Step pre;
    pre.kind = STEP_BLUE_PRE;
    pre.blue = b;
    pre.src = src;
    pre.dst = S0;
    P->steps.push_back(pre);
    line(depth + 1, "pointwise a = pad(x w)");
    if (fuse) {
      emit_blue_fused(d, V, dst, conj, m, w, B, S0, S1, depth + 1);
      return;
    }
    solve_rank1({m, 1, 1}, {{count, m, m}}, S0, S1, 0, depth + 1);
    Step mul;
    mul.kind = STEP_BLUE_MUL;
    mul.blue = b;
    mul.src = S1;
    mul.dst = S1;
    P->steps.push_back(mul);
    line(depth + 1, "pointwise Z = conj(A Bhat)");
    solve_rank1({m, 1, 1}, {{count, m, m}}, S1, S0, 0, depth + 1);
    Step post;
    post.kind = STEP_BLUE_POST;
    post.blue = b;
    post.src = S0;
    post.dst = dst;
    P->steps.push_back(post);
    line(depth + 1, "pointwise Y = w conj(D)");
  }

  // per-stage tables [k][4] of the power-of-two pass kernels for n = 2^logn
  const float2* p2_stage_tables(int logn) {
    float2* tw = (float2*)dalloc(sizeof(float2) * (size_t)std::max(16, gb_p2_twiddle_elems(logn)));
    for (int st = 1; tw && !err; ++st) {
      int L, R, off;
      if (!gb_p2_stage(logn, st, &L, &R, &off)) break;
      if (gb_make_stage_twiddles(tw + off, (int64_t)1 << logn, L, R, 0) != cudaSuccess) err = FFT_ERR_CUDA;
    }
    return tw;
  }

  // The four-step of eq. (2) as one persistent kernel whose intermediate stays
  // in an L2-resident ring (l2fourstep.cu): contiguous power-of-two transforms
  // of 2^14 .. 2^22 points, at most one vector loop, and (group mode) the
  // 65536-point inner transforms of 2^22..2^24-point four-steps.  The lag D between the A
  // and B items of a transform is kL2Lag items per CTA of the persistent grid
  // (a CTA holds up to four items at once: one claimed, three in its buffers;
  // with a lag of two the B items waited on their A items for a fifth of the
  // time, and lags of eight, with rings up to 96 MiB, were slower again than
  // five: measured); the ring holds S = 2D transforms within kL2RingBytes
  // (S > D is required).
  static constexpr int64_t kL2RingBytes = (int64_t)64 << 20;
  static constexpr int64_t kL2Lag = 5;

  // The shapes the kernel takes: contiguous transforms (unit element strides,
  // at most one vector loop), or -- group mode, n = 256 x 256 -- the inner
  // transforms of a larger four-step: inputs one contiguous run of
  // transforms, outputs of consecutive transforms adjacent (vos 1) with
  // elements os apart, and at most one more output loop (vos2) over groups of
  // nt1 transforms.
  struct L2Shape {
    int l1, l2, gb;
    int64_t count, vis, vos, os, nt1, vos2;
  };

  bool l2fs_shape(const Dim& d, const std::vector<Dim>& V, int64_t n1, L2Shape* sh) const {
    const int lg = log2_exact(d.n), e1 = log2_exact(n1);
    if (prec || lg < 14 || lg > 22 || e1 < 0 || d.is != 1 || V.size() > 2) return false;
    if (!gb_l2fs_supported(e1, lg - e1)) return false;
    *sh = L2Shape{e1, lg - e1, 1, 1, d.n, d.n, 1, 0, 0};
    if (d.os == 1 && V.size() <= 1) {
      if (!V.empty()) {
        sh->count = V[0].n;
        sh->vis = V[0].is;
        sh->vos = V[0].os;
      }
      return sh->vis > 0 && sh->vos > 0;
    }
    const int g = gb_l2fs_group(e1, lg - e1);
    if (g <= 1 || d.os < 1) return false;
    int ia = -1;
    for (int i = 0; i < (int)V.size(); ++i)
      if (V[i].os == 1 && V[i].is == d.n && V[i].n % g == 0) ia = i;
    if (ia < 0) return false;
    sh->gb = g;
    sh->count = V[ia].n;
    sh->nt1 = V[ia].n;
    sh->vos = V[ia].os;  // 1: a group's outputs adjacent
    sh->os = d.os;
    if (V.size() == 2) {
      const Dim& b = V[1 - ia];
      if (b.is != V[ia].n * d.n || b.os <= 0) return false;
      sh->count *= b.n;
      sh->vos2 = b.os;
    }
    return true;
  }

  bool l2fs_ring(const L2Shape& sh, int64_t* S, int64_t* D) const {
    int T1 = 0, T2 = 0;
    if (!gb_l2fs_tiles(sh.l1, sh.l2, &T1, &T2)) return false;
    const int64_t n = (int64_t)1 << (sh.l1 + sh.l2);
    // items per step of the schedule: the A items of a transform (a group of
    // gb transforms) and the B items of an earlier one
    const int64_t nA = ((int64_t)1 << sh.l2) / T1;
    const int64_t nB = ((int64_t)1 << sh.l1) * sh.gb / T2;  // B items per transform or group
    const int64_t per = sh.gb * nA + nB, units = sh.count / sh.gb;
    int64_t grid = device ? gb_l2fs_grid(sh.l1, sh.l2) : 0;
    if (grid <= 0) grid = (T1 << sh.l1) <= 4096 ? 304 : 152;
    int64_t d = std::max<int64_t>(1, (kL2Lag * grid + per - 1) / per);
    int64_t s = 2 * d;
    const int64_t cap = std::max<int64_t>(1, kL2RingBytes / (sh.gb * n * 8));
    if (s > cap) s = cap;
    if (d >= s) d = s - 1;
    if (d < 1) return false;
    if (d > units) d = units;
    if (s > units) s = units;
    *S = s * sh.gb;  // transforms
    *D = d;          // steps
    return true;
  }

  void emit_l2fs(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t n1, int depth) {
    L2Shape sh;
    int64_t S, D;
    if (!l2fs_shape(d, V, n1, &sh) || !l2fs_ring(sh, &S, &D)) {
      err = FFT_ERR_WISDOM;
      return;
    }
    if (sh.gb > 1 && src == dst) {  // a group's outputs interleave with other transforms' inputs
      err = FFT_ERR_WISDOM;
      return;
    }
    const int l1 = sh.l1, l2 = sh.l2;
    const int64_t count = sh.count, vis = sh.vis, vos = sh.vos;
    const int64_t n = d.n, n2 = n / n1;
    GbL2FS k{};
    k.logn1 = l1;
    k.logn2 = l2;
    k.count = count;
    k.vis = vis;
    k.vos = vos;
    k.S = S;
    k.D = D;
    k.conj = conj;
    k.tw1 = p2_stage_tables(l1);
    k.tw2 = p2_stage_tables(l2);
    const int64_t L = gb_p2_last_L(l1);
    float2* A = (float2*)dalloc(sizeof(float2) * (size_t)(n2 * L));
    float2* B = (float2*)dalloc(sizeof(float2) * (size_t)(n2 * 4));
    if (A && B && gb_make_posttw(A, B, n, n2, L, 0) != cudaSuccess) err = FFT_ERR_CUDA;
    k.ptwA = A;
    k.ptwB = B;
    k.status = P->d_status;
    k.gb = sh.gb;
    k.os = sh.os;
    k.nt1 = sh.nt1;
    k.vos2 = sh.vos2;
    const size_t ring = (size_t)S * n * sizeof(float2);
    Step s;
    s.kind = STEP_L2FS;
    s.l2 = k;
    s.src = src;
    s.dst = dst;
    s.aux = new_scratch(ring + sizeof(unsigned) * gb_l2fs_sync_words(count, sh.gb));
    P->steps.push_back(s);
    int T1 = 0, T2 = 0;
    gb_l2fs_tiles(l1, l2, &T1, &T2);
    std::ostringstream o;
    o << "pass l2-fourstep n=" << n << " = " << n1 << " x " << n2 << " (eq. 2 in one persistent kernel, "
      << "intermediate in an L2-resident ring of " << S << " transforms, lag " << D << ") T1=" << T1 << " T2=" << T2
      << " count=" << count << " vis=" << vis << " vos=" << vos;
    if (sh.gb > 1)
      o << " (B items over " << T2 / sh.gb << " rows of " << sh.gb << " transforms; output element stride " << sh.os
        << ", loops " << sh.nt1 << " x vos " << sh.vos2 << ")";
    o << (conj ? " conj" : "");
    line(depth, o.str());
  }

  // Rader's algorithm (sec. 4.2.5) for a prime length p: the nonzero indices
  // permuted by powers of a generator g turn the DFT into a cyclic
  // convolution of length p - 1, evaluated by two forward FFTs of length L
  // (L = p - 1, or a length >= 2p - 3 with zero padding) around a pointwise
  // multiply by Bhat = DFT_L(b) / L (rader.cu).
  static bool is_prime(int64_t n) {
    if (n < 2) return false;
    for (int64_t q = 2; q * q <= n; ++q)
      if (n % q == 0) return false;
    return true;
  }

  // the smallest generator of the multiplicative group modulo the prime p
  static int64_t primitive_root(int64_t p) {
    std::vector<int64_t> f;
    int64_t m = p - 1;
    for (int64_t q = 2; q * q <= m; ++q)
      if (m % q == 0) {
        f.push_back(q);
        while (m % q == 0) m /= q;
      }
    if (m > 1) f.push_back(m);
    for (int64_t g = 2; g < p; ++g) {
      bool gen = true;
      for (int64_t q : f) gen = gen && gb_powmod(g, (p - 1) / q, p) != 1;
      if (gen) return g;
    }
    return 1;  // p = 2
  }

  static bool rader_length_ok(int64_t p, int64_t L) {
    return is_prime(p) && p > 2 && p < ((int64_t)1 << 30) && (L == p - 1 || L >= 2 * p - 3) &&
           smooth_codelet(L);
  }

  void emit_rader(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int64_t L, int depth) {
    const int64_t p = d.n;
    if (!rader_length_ok(p, L) || (int)V.size() > GB_MAX_VDIMS) {
      err = FFT_ERR_WISDOM;
      return;
    }
    const int64_t g = primitive_root(p), ginv = gb_powmod(g, p - 2, p);
    std::ostringstream o;
    o << "rader p=" << p << " g=" << g << " L=" << L << (L == p - 1 ? " (cyclic convolution of length p-1)"
                                                                    : " (zero-padded convolution)");
    line(depth, o.str());
    // permutations, exact in integers: perm[r] = g^r, qidx[g^{-q}] = q
    std::vector<int> perm(p - 1), qidx(p, 0);
    int64_t a = 1, c = 1;
    for (int64_t r = 0; r < p - 1; ++r) {
      perm[r] = (int)a;
      qidx[c] = (int)r;
      a = gb_mulmod(a, g, p);
      c = gb_mulmod(c, ginv, p);
    }
    int* dperm = (int*)dalloc(sizeof(int) * (p - 1));
    int* dq = (int*)dalloc(sizeof(int) * p);
    float2* B = (float2*)dalloc(sizeof(float2) * L);
    if (device && !err) {
      if (cudaMemcpy(dperm, perm.data(), sizeof(int) * (p - 1), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(dq, qidx.data(), sizeof(int) * p, cudaMemcpyHostToDevice) != cudaSuccess) {
        err = FFT_ERR_CUDA;
        return;
      }
      double2* work = nullptr;  // stream-ordered, as for Bluestein's table
      if (cudaMallocAsync((void**)&work, sizeof(double2) * 2 * L, 0) != cudaSuccess) {
        cudaGetLastError();
        err = FFT_ERR_OOM;
        return;
      }
      const std::vector<int> rad = default_radices(L);
      if (gb_make_rader_kernel(B, p, ginv, L, rad.data(), (int)rad.size(), work, 0) != cudaSuccess)
        err = FFT_ERR_CUDA;
      if (cudaFreeAsync(work, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) err = FFT_ERR_CUDA;
    }
    const int64_t count = prod_n(V);
    GbRaderIO r;
    memset(&r, 0, sizeof(r));
    r.p = p;
    r.L = L;
    r.is = d.is;
    r.os = d.os;
    r.nv = (int)V.size();
    for (int i = 0; i < r.nv; ++i) {
      r.vn[i] = V[i].n;
      r.vis[i] = V[i].is;
      r.vos[i] = V[i].os;
    }
    r.count = count;
    r.perm = dperm;
    r.qidx = dq;
    r.B = B;
    r.conj = conj;
    const int S0 = new_scratch((size_t)count * L * sizeof(float2));
    const int S1 = new_scratch((size_t)count * L * sizeof(float2));
    const int SD = new_scratch((size_t)count * 2 * sizeof(float2));
    Step pre;
    pre.kind = STEP_RADER_PRE;
    pre.rader = r;
    pre.src = src;
    pre.dst = S0;
    pre.aux = SD;
    P->steps.push_back(pre);
    line(depth + 1, "pointwise a = pad(x[g^r]), x0 kept");
    solve_rank1({L, 1, 1}, {{count, L, L}}, S0, S1, 0, depth + 1);
    Step mul;
    mul.kind = STEP_RADER_MUL;
    mul.rader = r;
    mul.src = S1;
    mul.dst = S1;
    mul.aux = SD;
    P->steps.push_back(mul);
    line(depth + 1, "pointwise dc = A[0], Z = conj(A Bhat)");
    solve_rank1({L, 1, 1}, {{count, L, L}}, S1, S0, 0, depth + 1);
    Step post;
    post.kind = STEP_RADER_POST;
    post.rader = r;
    post.src = S0;
    post.dst = dst;
    post.aux = SD;
    P->steps.push_back(post);
    line(depth + 1, "pointwise Y[0] = x0 + dc, Y[g^-q] = x0 + conj(D[q])");
  }

  // ---------------------------------------------------------------- in place
  // An in-place transform of n = s^2 contiguous points without scratch (sec.
  // 4.2, in-place plans from DIT/DIF steps and in-place transposes): the
  // column DFTs of the s x s matrix in place, each CTA loading its whole
  // column tile before writing it back (twiddle w_n^{l2 k1} fused), the row
  // DFTs in place, then an in-place square transpose puts Y[k1 + s k2] in
  // natural order.
  bool ip4_ok(const Dim& d, const std::vector<Dim>& V, int64_t s) const {
    const int e = log2_exact(s);
    if (prec || e < 6 || e > 12 || s * s != d.n || d.is != 1 || d.os != 1 || V.size() > 1) return false;
    return V.empty() || V[0].is == V[0].os;
  }

  void emit_ip4(const Dim& d, const std::vector<Dim>& V, int buf, int conj, int64_t s, int depth) {
    if (!ip4_ok(d, V, s)) {
      err = FFT_ERR_WISDOM;
      return;
    }
    const int64_t n = d.n, count = V.empty() ? 1 : V[0].n, vs = V.empty() ? n : V[0].is;
    line(depth, "cooley-tukey n=" + std::to_string(n) + " = " + std::to_string(s) + " x " + std::to_string(s) +
                    " in place without scratch (columns, rows, square transpose)");
    std::vector<Dim> V1{{s, 1, 1}}, V2{{s, s, s}};
    if (count > 1) {
      V1.push_back({count, vs, vs});
      V2.push_back({count, vs, vs});
    }
    emit_p2({s, s, s}, canon_vec(V1), buf, buf, conj, n, depth + 1);
    if (err) return;
    emit_p2({s, 1, 1}, canon_vec(V2), buf, buf, conj, 0, depth + 1);  // rows and batch merge into one loop
    if (err) return;
    std::vector<Dim> T{{s, s, 1}, {s, 1, s}};
    if (count > 1) T.push_back({count, vs, vs});
    emit_copy(T, buf, buf, depth + 1);
  }

  // The indirect plan of sec. 4.2: the data first rearranged into the output's
  // layout (a rank-0 copy), then the transform solved in place there.
  void emit_indirect(const Dim& d, const std::vector<Dim>& V, int src, int dst, int conj, int depth) {
    line(depth, "indirect: copy into the output's layout, then the transform in place");
    std::vector<Dim> all = V;
    all.push_back(d);
    emit_copy(canon_vec(all), src, dst, depth + 1);
    if (err) return;
    std::vector<Dim> Vo;
    for (const Dim& v : V) Vo.push_back({v.n, v.os, v.os});
    solve_rank1({d.n, d.os, d.os}, Vo, dst, dst, conj, depth + 1);
  }

  // ---------------------------------------------------------------- real data
  // DFTs of real data (sec. 5, sec. 7), built from the complex plans above and
  // the pointwise steps of real.cu.  `loops` are the vector loops of the 1-D
  // real transform, strides in the units of each side.

  // dense row-major strides (last loop fastest) of loops of the given lengths, times unit
  static std::vector<int64_t> dense_strides(const std::vector<Dim>& loops, int64_t unit) {
    std::vector<int64_t> st(loops.size());
    int64_t s = unit;
    for (int i = (int)loops.size() - 1; i >= 0; --i) {
      st[i] = s;
      s *= loops[i].n;
    }
    return st;
  }

  bool real_io(GbRealIO* r, int64_t n, int64_t is, int64_t os, const std::vector<Dim>& loops, bool in_side,
               bool out_side, int64_t in_div = 1, int64_t out_div = 1) {
    if ((int)loops.size() > GB_MAX_VDIMS) {
      err = FFT_ERR_UNSUPPORTED;
      return false;
    }
    memset(r, 0, sizeof(*r));
    r->n = n;
    r->m = n / 2;
    r->is = is;
    r->os = os;
    r->nv = (int)loops.size();
    r->count = 1;
    for (int i = 0; i < r->nv; ++i) {
      r->vn[i] = loops[i].n;
      r->vis[i] = in_side ? loops[i].is / in_div : 0;
      r->vos[i] = out_side ? loops[i].os / out_div : 0;
      r->count *= loops[i].n;
    }
    if (r->nv == 0) {
      r->nv = 1;
      r->vn[0] = 1;
    }
    r->tw = roots(n);
    return true;
  }

  void emit_r2c_1d(const Dim& d, const std::vector<Dim>& loops, int src, int dst, int depth) {
    const int64_t n = d.n, half = n / 2 + 1;
    bool pairs = n % 2 == 0 && d.is == 1;
    for (const Dim& L : loops) pairs = pairs && (L.is % 2 == 0);
    int64_t count = 1;
    for (const Dim& L : loops) count *= L.n;
    std::ostringstream o;
    Step s;
    if (pairs) {
      const int64_t m = n / 2;
      o << "real-input dft n=" << n << ": the input read as " << m << " complex pairs, a complex dft of " << m
        << ", then the half spectrum (eq. 2 with n1 = 2)";
      line(depth, o.str());
      std::vector<Dim> Vc;
      for (const Dim& L : loops) Vc.push_back({L.n, L.is / 2, L.os});
      solve_rank1({m, 1, d.os}, Vc, src, dst, 0, depth + 1);
      if (err || !real_io(&s.real, n, 0, d.os, loops, false, true)) return;
      for (int i = 0; i < s.real.nv && !loops.empty(); ++i) s.real.vis[i] = s.real.vos[i];
      s.kind = STEP_R2C_POST;
      s.src = dst;
      s.dst = dst;
      P->steps.push_back(s);
      line(depth + 1, "pointwise X[k] = Ze[k] + w_n^k Zo[k], X[m-k] = conj(Ze[k] - w_n^k Zo[k]), in place");
      P->align8_in = true;
      return;
    }
    o << "real-input dft n=" << n << ": widened to complex, a complex dft of " << n << ", the half spectrum kept";
    line(depth, o.str());
    const int S1 = new_scratch((size_t)count * n * sizeof(float2));
    const int S2 = new_scratch((size_t)count * n * sizeof(float2));
    if (!real_io(&s.real, n, d.is, 0, loops, true, false)) return;
    s.kind = STEP_R2C_PROMOTE;
    s.src = src;
    s.dst = S1;
    P->steps.push_back(s);
    line(depth + 1, "pointwise promote x -> (x, 0)");
    solve_rank1({n, 1, 1}, {{count, n, n}}, S1, S2, 0, depth + 1);
    if (err) return;
    const std::vector<int64_t> ds = dense_strides(loops, n);
    std::vector<Dim> cp{{half, 1, d.os}};
    for (size_t i = 0; i < loops.size(); ++i) cp.push_back({loops[i].n, ds[i], loops[i].os});
    emit_copy(cp, S2, dst, depth + 1);
  }

  void emit_c2r_1d(const Dim& d, const std::vector<Dim>& loops, int src, int dst, int depth) {
    const int64_t n = d.n;
    bool pairs = n % 2 == 0 && d.os == 1;
    for (const Dim& L : loops) pairs = pairs && (L.os % 2 == 0);
    int64_t count = 1;
    for (const Dim& L : loops) count *= L.n;
    std::ostringstream o;
    Step s;
    if (pairs) {
      const int64_t m = n / 2;
      o << "real-output dft n=" << n << ": the half spectrum folded to " << m << " complex values, a backward "
        << "complex dft of " << m << " written as real pairs";
      line(depth, o.str());
      const int S = new_scratch((size_t)count * m * sizeof(float2));
      if (!real_io(&s.real, n, d.is, 0, loops, true, false)) return;
      s.kind = STEP_C2R_PRE;
      s.src = src;
      s.dst = S;
      P->steps.push_back(s);
      line(depth + 1, "pointwise W[k] = (X[k] + conj X[m-k]) + i w_n^-k (X[k] - conj X[m-k])");
      const std::vector<int64_t> ds = dense_strides(loops, m);
      std::vector<Dim> Vc;
      for (size_t i = 0; i < loops.size(); ++i) Vc.push_back({loops[i].n, ds[i], loops[i].os / 2});
      solve_rank1({m, 1, 1}, Vc, S, dst, 1, depth + 1);
      P->align8_out = true;
      return;
    }
    o << "real-output dft n=" << n << ": the conjugate-symmetric extension, a backward complex dft of " << n
      << ", the real parts kept";
    line(depth, o.str());
    const int S1 = new_scratch((size_t)count * n * sizeof(float2));
    const int S2 = new_scratch((size_t)count * n * sizeof(float2));
    if (!real_io(&s.real, n, d.is, 0, loops, true, false)) return;
    s.kind = STEP_C2R_EXPAND;
    s.src = src;
    s.dst = S1;
    P->steps.push_back(s);
    line(depth + 1, "pointwise conjugate-symmetric extension (self-conjugate bins real)");
    solve_rank1({n, 1, 1}, {{count, n, n}}, S1, S2, 1, depth + 1);
    if (err) return;
    Step r;
    if (!real_io(&r.real, n, 0, d.os, loops, false, true)) return;
    r.kind = STEP_C2R_REAL;
    r.src = S2;
    r.dst = dst;
    P->steps.push_back(r);
    line(depth + 1, "pointwise y = Re(w)");
  }

  // a real-data problem: the 1-D real transform along the last dimension and
  // complex DFTs along the others (separable, sec. 4.1)
  void solve_real(const Problem& Q, int depth) {
    const Dim d = Q.N.back();
    const std::vector<Dim> O(Q.N.begin(), Q.N.end() - 1);
    const int64_t half = d.n / 2 + 1;
    if (Q.kind == 1) {
      std::vector<Dim> loops = O;
      loops.insert(loops.end(), Q.V.begin(), Q.V.end());
      emit_r2c_1d(d, loops, BUF_IN, BUF_OUT, depth);
      std::vector<int> order(O.size());
      for (size_t i = 0; i < O.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return iabs64(O[a].os) < iabs64(O[b].os); });
      for (int a : order) {
        if (err) return;
        std::vector<Dim> others;
        for (size_t b = 0; b < O.size(); ++b)
          if ((int)b != a) others.push_back({O[b].n, O[b].os, O[b].os});
        others.push_back({half, d.os, d.os});
        for (const Dim& v : Q.V) others.push_back({v.n, v.os, v.os});
        solve_rank1({O[a].n, O[a].os, O[a].os}, others, BUF_OUT, BUF_OUT, 0, depth);
      }
      return;
    }
    if (O.empty()) {
      emit_c2r_1d(d, Q.V, BUF_IN, BUF_OUT, depth);
      return;
    }
    // backward complex DFTs over the other dimensions, from the input into a
    // dense scratch [V][O][half], then the real transform from there
    std::vector<Dim> shape = Q.V;
    shape.insert(shape.end(), O.begin(), O.end());
    shape.push_back({half, 0, 0});
    const std::vector<int64_t> ds = dense_strides(shape, 1);
    int64_t total = 1;
    for (const Dim& x : shape) total *= x.n;
    const int S = new_scratch((size_t)total * sizeof(float2));
    const size_t nv = Q.V.size();
    std::vector<Dim> Od, vec;
    for (size_t i = 0; i < O.size(); ++i) Od.push_back({O[i].n, O[i].is, ds[nv + i]});
    vec.push_back({half, d.is, 1});
    for (size_t j = 0; j < nv; ++j) vec.push_back({Q.V[j].n, Q.V[j].is, ds[j]});
    line(depth, "complex dfts over the other dimensions into a dense work array");
    solve(Od, vec, BUF_IN, S, 1, depth + 1);
    if (err) return;
    std::vector<Dim> loops;
    for (size_t i = 0; i < O.size(); ++i) loops.push_back({O[i].n, ds[nv + i], O[i].os});
    for (size_t j = 0; j < nv; ++j) loops.push_back({Q.V[j].n, ds[j], Q.V[j].os});
    emit_c2r_1d({d.n, 1, d.os}, loops, S, BUF_OUT, depth);
  }

  // ---------------------------------------------------------------- planner

  std::string key_rank1(const Dim& d, const std::vector<Dim>& V, bool inplace) const {
    std::ostringstream o;
    o << "r1 n=" << d.n << " is=" << d.is << " os=" << d.os << " v=" << dims_str(V) << " ip=" << (inplace ? 1 : 0);
    if (prec) o << " tc=" << prec;
    return o.str();
  }

  std::vector<std::string> candidates(const Dim& d, const std::vector<Dim>& V, bool inplace = false) {
    std::vector<std::string> c;
    const int64_t n = d.n;
    // a caller's in-place problem (not the in-place sub-problems of other
    // plans): in estimate mode the scratch-free forms come first, since memory
    // is why a caller asks for in place; measure mode times them with the rest
    const bool caller_inplace = inplace && P->inplace;
    const bool no_scratch_first = caller_inplace && !measure;
    int64_t ip4_s = 1;
    while (ip4_s * ip4_s < n) ip4_s <<= 1;
    const bool ip4 = inplace && log2_exact(n) >= 14 && ip4_ok(d, V, ip4_s);
    if (ip4 && caller_inplace) c.push_back("ip4:" + std::to_string(ip4_s));
    Dim v0{1, 0, 0};
    bool has_v = false;
    if (!V.empty()) {
      v0 = V[tile_dim(V)];
      has_v = true;
    }
    // transpose first: a batch-fastest input into the output's layout, then
    // the same-layout transform (estimate mode: long lengths, where the
    // strided tiles get thin)
    const bool xpose = !prec && xpose_ok(d, V);
    if (!measure && log2_exact(n) >= 14) {
      // a batch-fastest input into transform-contiguous output, too long for
      // one pass: the two-pass four-step with the scratch [l2][b][k1] before
      // transposing first (measured faster: 65536 x 512 in 0.18 ms against
      // 0.27 ms for the transpose and two passes)
      const int64_t a = estimate_split(n);
      if (a > 1 && emit_fourstep_bfin(d, V, 0, 0, 0, a, 0, true)) c.push_back("split:" + std::to_string(a));
    }
    if (xpose && !measure && n >= 4096) c.push_back("xpose");
    // estimate mode: transforms of 2^12 and more down the columns of a
    // row-major array take the four-step with the columns innermost (two
    // passes of 64-column tiles beat one pass of two-column tiles when measured)
    if (!prec && !measure && !no_scratch_first && d.is != 1 && log2_exact(n) >= 12) {
      const int64_t a = estimate_split(n);
      bool unit = false;
      for (const Dim& v : V) unit = unit || (v.is == 1 && v.os == 1 && v.n % 64 == 0);
      if (unit && a >= 64 && n / a >= 64) c.push_back("split:" + std::to_string(a));
    }
    P2Choice pc;
    if (p2_choose(d, V, false, &pc, prec)) {
      c.push_back("p2");
      if (pc.prec) return c;  // the requested tensor-core precision decides the pass
    }
    const int lg = log2_exact(n);
    // the four-step with its intermediate in L2 (one HBM round trip)
    bool l2fs_ok = false, l2fs_busy = false;
    const int64_t l2fs_n1 = lg >= 0 ? ((int64_t)1 << (lg / 2)) : 0;
    {
      L2Shape sh;
      int T1, T2;
      int64_t S, D;
      // in place: transform t is written only after all its A items have read
      // it, so equal input and output strides suffice (contiguous mode only:
      // a group's outputs interleave with other transforms' inputs)
      l2fs_ok = lg >= 14 && l2fs_shape(d, V, l2fs_n1, &sh) &&
                (!inplace || (sh.gb == 1 && sh.vis == sh.vos)) && l2fs_ring(sh, &S, &D);
      // enough work items to fill the GPU several times over
      if (l2fs_ok && gb_l2fs_tiles(sh.l1, sh.l2, &T1, &T2))
        l2fs_busy = sh.count * (((int64_t)1 << sh.l2) / T1 + ((int64_t)1 << sh.l1) / T2) >= 8 * 304;
    }
    // estimate mode takes the first candidate: the L2-resident four-step where
    // it beat the two and three TMA passes when measured (2^14..2^21, batches
    // that fill the GPU), then the cluster pass where it beat two TMA passes
    // (2^14), the two passes above
    if (!measure && l2fs_ok && l2fs_busy && lg <= 21) c.push_back("l2fs:" + std::to_string(l2fs_n1));
    if (!measure && lg >= 15 && lg <= 17 && smooth_codelet(n)) {
      const int64_t a = estimate_split(n);
      if (a > 1) c.push_back("split:" + std::to_string(a));
    }
    if (!prec && cluster_ok(d, V)) {
      int cfg[16][4];
      const int nc = gb_cluster_configs(lg, cfg, 16);
      for (int i = 0; i < nc; ++i) {
        if (device && gb_cluster_max_active(cfg[i][0], cfg[i][1], cfg[i][2], cfg[i][3]) < 1) {
          cudaGetLastError();
          continue;
        }
        c.push_back("cluster:" + std::to_string(cfg[i][0]) + "." + std::to_string(cfg[i][1]) + "." +
                    std::to_string(cfg[i][2]) + "." + std::to_string(cfg[i][3]));
        if (!measure) break;
      }
    }
    if (lg >= 14 && smooth_codelet(n)) {
      // power of two beyond the one-CTA kernels: TMA passes of a split first
      const int64_t a = estimate_split(n);
      if (a > 1) c.push_back("split:" + std::to_string(a));
    }
    if (measure && l2fs_ok) c.push_back("l2fs:" + std::to_string(l2fs_n1));
    MRChoice mc;
    if (!prec && mr_choose(d, V, false, &mc)) c.push_back("mr");
    if (smooth_codelet(n)) {
      std::vector<int> rad = default_radices(n);
      if (single_pass_ok(n, rad)) {
        PassCfg base = estimate_cfg(d, v0, has_v, rad);
        c.push_back("single:" + base.str());
        if (measure) {
          // radix order reversed
          std::vector<int> rr(rad.rbegin(), rad.rend());
          if (rr != rad) {
            PassCfg x = base;
            x.radices = rr;
            c.push_back("single:" + x.str());
          }
          // 16 -> 4 x 4 where it keeps the thread count legal
          std::vector<int> r4;
          for (int R : rad) {
            if (R == 16) {
              r4.push_back(4);
              r4.push_back(4);
            } else r4.push_back(R);
          }
          if (r4 != rad && (int)r4.size() <= GB_MAX_STAGES && threads_per_transform(n, r4) <= 1024) {
            PassCfg x = estimate_cfg(d, v0, has_v, r4);
            c.push_back("single:" + x.str());
          }
          for (int f : {2, -2}) {
            PassCfg x = base;
            x.T = f > 0 ? base.T * 2 : std::max(1, base.T / 2);
            const int tpt = threads_per_transform(n, rad);
            if (x.T != base.T && x.T * tpt <= 1024 && x.T * (int64_t)smem_pitch(n) * 8 <= smem_limit())
              c.push_back("single:" + x.str());
          }
          if (base.load_mode == GB_MOVE_DIRECT || base.store_mode == GB_MOVE_DIRECT) {
            PassCfg x = base;
            x.load_mode = x.store_mode = GB_MOVE_SMEM;
            c.push_back("single:" + x.str());
          }
        }
      }
      if (n > 64) {
        const int64_t a = estimate_split(n);
        if (a > 1) {
          c.push_back("split:" + std::to_string(a));
          if (measure) {
            // every power-of-two column length 16..4096 whose row length is at
            // least 16 (non-square splits often win: wider column tiles on one
            // side, a one-pass row length on the other)
            for (int64_t b = 16; b <= 4096; b *= 2) {
              if (b != a && n % b == 0 && n / b >= 16 && smooth_codelet(n / b))
                c.push_back("split:" + std::to_string(b));
            }
          }
        }
      }
    }
    if (xpose && measure) c.push_back("xpose");
    if (ip4 && measure) c.push_back("ip4:" + std::to_string(ip4_s));
    // the indirect plan (sec. 4.2): copy into the output's layout, transform in place
    if (measure && !inplace && !prec) {
      bool differs = d.is != d.os;
      for (const Dim& v : V) differs = differs || v.is != v.os;
      if (differs) c.push_back("indirect");
    }
    // Rader for a prime length: estimate mode takes it first where p - 1 is
    // smooth (one FFT of length p - 1 each way, against Bluestein's two of
    // length >= 2p - 1) unless p is small enough for the one-CTA fused
    // Bluestein pass (one launch); measure mode times it always, and also the
    // zero-padded power of two
    const bool rader = !prec && n > 13 && is_prime(n) && n < ((int64_t)1 << 30);
    int64_t r2 = 1;
    while (r2 < 2 * n - 3) r2 <<= 1;
    const int64_t mb = bluestein_length(n);
    const bool blue_one_cta = n <= 1024 && single_pass_ok(mb, default_radices(mb));
    if (rader && smooth_codelet(n - 1) && (measure || (generic_prime(n) < 0 && !blue_one_cta)))
      c.push_back("rader:" + std::to_string(n - 1));
    if (!smooth_codelet(n) || c.empty()) {
      // the convolution length: the smallest 2^a 3^b 5^c 7^d >= 2n - 1, and
      // (measure mode) the next power of two, whose passes run on the
      // power-of-two kernels.  Estimate mode takes the power of two first
      // where the smooth length needs several passes and the power of two
      // runs as the fused four-step (the multiply and output step in the FFT
      // stores): measured faster than the smooth length's mixed-radix passes
      // (n = 10007 x 512: m = 32768 fused in 0.26 ms, m = 20160 in 0.48 ms)
      const int64_t m = bluestein_length(n);
      int64_t m2 = 1;
      while (m2 < 2 * n - 1) m2 <<= 1;
      if (!measure && m2 != m && !single_pass_ok(m, default_radices(m)) && blue_fused_ok(d, V, m2))
        c.push_back("blue:" + std::to_string(m2));
      c.push_back("blue:" + std::to_string(m));
      if (measure && m2 != m) c.push_back("blue:" + std::to_string(m2));
      if (rader && measure) c.push_back("rader:" + std::to_string(r2));
    }
    std::vector<std::string> u;
    for (const std::string& x : c)
      if (std::find(u.begin(), u.end(), x) == u.end()) u.push_back(x);
    return u;
  }

  static int tile_dim(const std::vector<Dim>& V) {
    int best = 0;
    for (int i = 1; i < (int)V.size(); ++i) {
      const int64_t a = std::min(iabs64(V[i].is), iabs64(V[i].os)), b = std::min(iabs64(V[best].is), iabs64(V[best].os));
      const int64_t sa = iabs64(V[i].is) + iabs64(V[i].os), sb = iabs64(V[best].is) + iabs64(V[best].os);
      if (a < b || (a == b && sa < sb)) best = i;
    }
    return best;
  }

  // vector loops for a pass: tile dim first, then outermost .. innermost
  static std::vector<Dim> order_for_pass(const std::vector<Dim>& V) {
    if (V.empty()) return V;
    const int t = tile_dim(V);
    std::vector<Dim> rest;
    for (int i = 0; i < (int)V.size(); ++i)
      if (i != t) rest.push_back(V[i]);
    std::stable_sort(rest.begin(), rest.end(), [](const Dim& a, const Dim& b) { return iabs64(a.is) > iabs64(b.is); });
    std::vector<Dim> out;
    out.push_back(V[t]);
    out.insert(out.end(), rest.begin(), rest.end());
    return out;
  }

  double time_choice(const Dim& d, const std::vector<Dim>& V, bool inplace, const std::string& key,
                     const std::string& choice);

  std::string choose(const Dim& d, const std::vector<Dim>& V, bool inplace) {
    const std::string key = key_rank1(d, V, inplace);
    auto f = forced.find(key);
    if (f != forced.end()) return f->second;
    std::string val;
    if (wisdom_get(key, &val)) return val;
    if (wisdom_only) {
      err = FFT_ERR_WISDOM;
      return "";
    }
    std::vector<std::string> cands = candidates(d, V, inplace);
    if (!measure || !device || cands.size() == 1) {
      if (measure && device) wisdom_put(key, cands[0]);
      return cands[0];
    }
    double best = 1e30;
    std::string pick = cands[0];
    for (const std::string& c : cands) {
      const double t = time_choice(d, V, inplace, key, c);
      if (t > 0 && t < best) {
        best = t;
        pick = c;
      }
    }
    wisdom_put(key, pick);
    return pick;
  }

  void solve_rank1(const Dim& d, const std::vector<Dim>& Vraw, int src, int dst, int conj, int depth) {
    if (err) return;
    std::vector<Dim> V = canon_vec(Vraw);
    if (d.n == 1) {
      std::vector<Dim> W = V;
      W.push_back({1, d.is, d.os});
      emit_copy(canon_vec(W), src, dst, depth);
      return;
    }
    const std::string choice = choose(d, V, src == dst);
    if (err) return;
    if (choice == "p2") {
      emit_p2(d, V, src, dst, conj, 0, depth);
    } else if (choice == "mr") {
      emit_mr(d, V, src, dst, conj, 0, depth);
    } else if (choice == "xpose") {
      emit_xpose(d, V, src, dst, conj, depth);
    } else if (choice.rfind("single:", 0) == 0) {
      PassCfg cfg;
      if (!cfg.parse(choice.substr(7))) {
        err = FFT_ERR_WISDOM;
        return;
      }
      emit_single(d, order_for_pass(V), src, dst, conj, cfg, nullptr, depth);
    } else if (choice.rfind("cluster:", 0) == 0) {
      int l1, l2, cs, nb;
      if (!cluster_parse(choice, &l1, &l2, &cs, &nb)) {
        err = FFT_ERR_WISDOM;
        return;
      }
      emit_cluster(d, V, src, dst, conj, l1, l2, cs, nb, depth);
    } else if (choice.rfind("split:", 0) == 0) {
      const int64_t n1 = atoll(choice.c_str() + 6);
      if (n1 < 2 || d.n % n1 != 0) {
        err = FFT_ERR_WISDOM;
        return;
      }
      emit_fourstep(d, V, src, dst, conj, n1, depth);
    } else if (choice.rfind("ip4:", 0) == 0) {
      if (src != dst) {
        err = FFT_ERR_WISDOM;
        return;
      }
      emit_ip4(d, V, dst, conj, atoll(choice.c_str() + 4), depth);
    } else if (choice == "indirect") {
      if (src == dst) {
        err = FFT_ERR_WISDOM;
        return;
      }
      emit_indirect(d, V, src, dst, conj, depth);
    } else if (choice.rfind("l2fs:", 0) == 0) {
      emit_l2fs(d, V, src, dst, conj, atoll(choice.c_str() + 5), depth);
    } else if (choice.rfind("rader:", 0) == 0) {
      emit_rader(d, V, src, dst, conj, atoll(choice.c_str() + 6), depth);
    } else if (choice.rfind("blue:", 0) == 0) {
      const int64_t m = atoll(choice.c_str() + 5);
      if (m < 2 * d.n - 1) {
        err = FFT_ERR_WISDOM;
        return;
      }
      emit_bluestein(d, V, src, dst, conj, m, depth);
    } else {
      err = FFT_ERR_WISDOM;
    }
  }

  // separable multi-dimensional DFT: one rank-1 sub-problem per dimension
  void solve(const std::vector<Dim>& N, const std::vector<Dim>& V, int src, int dst, int conj, int depth) {
    if (N.empty()) {
      emit_copy(V, src, dst, depth);
      return;
    }
    if (N.size() == 1) {
      solve_rank1(N[0], V, src, dst, conj, depth);
      return;
    }
    std::vector<int> order(N.size());
    for (size_t i = 0; i < N.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return iabs64(N[a].is) < iabs64(N[b].is); });
    line(depth, "separable rank-" + std::to_string(N.size()) + " DFT, one pass group per dimension");
    for (size_t k = 0; k < order.size(); ++k) {
      const int a = order[k];
      std::vector<Dim> others;
      if (k == 0) {
        for (size_t b = 0; b < N.size(); ++b)
          if ((int)b != a) others.push_back(N[b]);
        others.insert(others.end(), V.begin(), V.end());
        solve_rank1(N[a], others, src, dst, conj, depth + 1);
      } else {
        for (size_t b = 0; b < N.size(); ++b)
          if ((int)b != a) others.push_back({N[b].n, N[b].os, N[b].os});
        for (const Dim& v : V) others.push_back({v.n, v.os, v.os});
        solve_rank1({N[a].n, N[a].os, N[a].os}, others, dst, dst, conj, depth + 1);
      }
      if (err) return;
    }
  }
};

static void release(PlanData* p) {
  for (void* t : p->tables)
    if (t) cudaFree(t);
  for (void* s : p->scratch)
    if (s) cudaFree(s);
  if (p->h_status) cudaFreeHost(p->h_status);
  else if (p->d_status) cudaFree(p->d_status);
  if (p->done) cudaEventDestroy(p->done);
  p->tables.clear();
  p->scratch.clear();
  p->scratch_bytes.clear();
  p->d_status = nullptr;
  p->h_status = nullptr;
  p->done = nullptr;
  p->done_valid = false;
}

int take_status(PlanData* p, bool wait) {
  if (!p->d_status) return FFT_OK;
  if (wait && p->done_valid && cudaEventSynchronize(p->done) != cudaSuccess) return FFT_ERR_CUDA;
  int v = 0;
  if (p->h_status) {
    v = *reinterpret_cast<volatile int*>(p->h_status);
    if (v) *reinterpret_cast<volatile int*>(p->h_status) = 0;
  } else {
    if (!wait) return FFT_OK;  // a device-memory word is read only after a wait
    if (cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FFT_ERR_CUDA;
    if (v && cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return FFT_ERR_CUDA;
  }
  return v;
}

void free_plan(PlanData* p) { release(p); }

int launch_step(const Step& s, float2* const* bufs, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  switch (s.kind) {
    case STEP_PASS: {
      e = gb_launch_pass(s.pass, s.dpass, bufs[s.src], bufs[s.dst], s.threads, s.smem, s.grid, st);
      break;
    }
    case STEP_POW2: {
      const bool small = s.p2.load == GB_P2_LOAD_CONTIG && s.p2.store == GB_P2_STORE_CONTIG && gb_p2_small(s.p2.logn);
      if (((uintptr_t)bufs[s.src] & 15) == 0 && (!small || ((uintptr_t)bufs[s.dst] & 15) == 0))
      {
        GbP2 k = s.p2;
        k.in = bufs[s.src];
        k.out = bufs[s.dst];
        e = k.prec ? gb_launch_tc(k, st) : gb_launch_p2(k, st);
      }
      else
        e = gb_launch_pass(s.pass, s.dpass, bufs[s.src], bufs[s.dst], s.threads, s.smem, s.grid, st);
      break;
    }
    case STEP_MR: {
      GbMR k = s.mr;
      k.in = bufs[s.src];
      k.out = bufs[s.dst];
      e = gb_launch_mr(k, st);
      break;
    }
    case STEP_CLUSTER: {
      GbCluster k = s.cl;
      k.in = bufs[s.src];
      k.out = bufs[s.dst];
      e = gb_launch_cluster(k, st);
      break;
    }
    case STEP_COPY: {
      GbCopy c = s.copy;
      c.in = bufs[s.src];
      c.out = bufs[s.dst];
      e = gb_launch_copy(c, st);
      break;
    }
    case STEP_BLUE_PRE: {
      GbBlueIO b = s.blue;
      b.in = bufs[s.src];
      b.work = bufs[s.dst];
      e = gb_launch_blue_pre(b, st);
      break;
    }
    case STEP_BLUE_MUL: {
      e = gb_launch_blue_mul(s.blue, bufs[s.dst], st);
      break;
    }
    case STEP_L2FS: {
      GbL2FS k = s.l2;
      k.in = bufs[s.src];
      k.out = bufs[s.dst];
      k.ring = bufs[s.aux];
      k.sync = reinterpret_cast<unsigned*>(k.ring + k.S * ((int64_t)1 << (k.logn1 + k.logn2)));
      e = gb_launch_l2fs(k, st);
      break;
    }
    case STEP_TRANSPOSE_IP: {
      GbCopy c = s.copy;
      c.in = bufs[s.dst];
      c.out = bufs[s.dst];
      e = gb_launch_transpose_inplace(c, st);
      break;
    }
    case STEP_R2C_POST: e = gb_launch_r2c_post(s.real, bufs[s.dst], st); break;
    case STEP_R2C_PROMOTE:
      e = gb_launch_r2c_promote(s.real, reinterpret_cast<const float*>(bufs[s.src]), bufs[s.dst], st);
      break;
    case STEP_C2R_PRE: e = gb_launch_c2r_pre(s.real, bufs[s.src], bufs[s.dst], st); break;
    case STEP_C2R_EXPAND: e = gb_launch_c2r_expand(s.real, bufs[s.src], bufs[s.dst], st); break;
    case STEP_C2R_REAL:
      e = gb_launch_c2r_real(s.real, bufs[s.src], reinterpret_cast<float*>(bufs[s.dst]), st);
      break;
    case STEP_RADER_PRE: {
      GbRaderIO r = s.rader;
      r.in = bufs[s.src];
      e = gb_launch_rader_pre(r, bufs[s.dst], bufs[s.aux], st);
      break;
    }
    case STEP_RADER_MUL: {
      e = gb_launch_rader_mul(s.rader, bufs[s.dst], bufs[s.aux], st);
      break;
    }
    case STEP_RADER_POST: {
      GbRaderIO r = s.rader;
      r.out = bufs[s.dst];
      e = gb_launch_rader_post(r, bufs[s.src], bufs[s.aux], st);
      break;
    }
    case STEP_STALL: {
      e = gb_launch_stall(s.pass.status, 50000000ull, st);  // 50 ms
      break;
    }
    case STEP_BLUE_POST: {
      GbBlueIO b = s.blue;
      b.out = bufs[s.dst];
      e = gb_launch_blue_post(b, bufs[s.src], st);
      break;
    }
    default:
      return FFT_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

static int run_steps(PlanData* p, const void* in, void* out, cudaStream_t st, void* work = nullptr) {
  std::vector<float2*> bufs(BUF_SCRATCH0 + p->scratch.size());
  bufs[BUF_IN] = (float2*)in;
  bufs[BUF_OUT] = (float2*)out;
  for (size_t k = 0; k < p->scratch.size(); ++k)
    bufs[BUF_SCRATCH0 + k] =
        p->external_scratch ? (float2*)((char*)work + p->scratch_offset[k]) : (float2*)p->scratch[k];
  for (const Step& s : p->steps) {
    const int rc = launch_step(s, bufs.data(), st);
    if (rc != FFT_OK) return rc;
  }
  return FFT_OK;
}

// Time one candidate for a rank-1 sub-problem: best of 3 after a warm-up,
// on planner-owned buffers sized like the sub-problem (the outermost loop is
// shortened when the footprint exceeds 1 GiB).
double Builder::time_choice(const Dim& d, const std::vector<Dim>& Vin, bool inplace, const std::string& key,
                            const std::string& choice) {
  std::vector<Dim> V = Vin;
  std::vector<Dim> N1{d};
  const int64_t cap = (int64_t)1 << 27;  // elements per buffer
  for (int guard = 0; guard < 64; ++guard) {
    int64_t a, b, c, e;
    footprint(N1, V, true, &a, &b);
    footprint(N1, V, false, &c, &e);
    if (b - a + 1 <= cap && e - c + 1 <= cap) break;
    int big = -1;
    for (int i = 0; i < (int)V.size(); ++i)
      if (V[i].n > 1 && (big < 0 || iabs64(V[i].is) > iabs64(V[big].is))) big = i;
    if (big < 0) return -1;
    V[big].n = (V[big].n + 1) / 2;
  }
  PlanData tmp;
  if (cudaMalloc(&tmp.d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaMemset(tmp.d_status, 0, sizeof(int));
  Builder b(&tmp, true, true, false);
  b.prec = prec;
  b.forced = forced;
  b.forced[key] = choice;
  b.forced[key_rank1(d, canon_vec(V), inplace)] = choice;
  b.solve_rank1(d, V, 0, inplace ? 0 : 1, 0, 0);
  double best = -1;
  int64_t ilo, ihi, olo, ohi;
  footprint(N1, V, true, &ilo, &ihi);
  footprint(N1, V, false, &olo, &ohi);
  float2 *ib = nullptr, *ob = nullptr;
  if (!b.err && cudaMalloc(&ib, sizeof(float2) * (ihi - ilo + 1)) == cudaSuccess &&
      (inplace || cudaMalloc(&ob, sizeof(float2) * (ohi - olo + 1)) == cudaSuccess)) {
    cudaMemset(ib, 0, sizeof(float2) * (ihi - ilo + 1));
    if (ob) cudaMemset(ob, 0, sizeof(float2) * (ohi - olo + 1));
    float2* in0 = ib - ilo;
    float2* out0 = inplace ? in0 : ob - olo;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bool ok = run_steps(&tmp, in0, out0, 0) == FFT_OK && cudaDeviceSynchronize() == cudaSuccess;
    for (int rep = 0; ok && rep < 3; ++rep) {
      cudaEventRecord(e0, 0);
      ok = run_steps(&tmp, in0, out0, 0) == FFT_OK;
      cudaEventRecord(e1, 0);
      if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0 || ms < best) best = ms;
      } else ok = false;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaGetLastError();
  if (ib) cudaFree(ib);
  if (ob) cudaFree(ob);
  release(&tmp);
  // decisions for nested sub-problems made while timing stay in the memo
  return best;
}

int build_plan(const Problem& P, bool device, PlanData* out) {
  out->prob = P;
  out->inplace = (P.flags & FFT_INPLACE) != 0;
  out->external_scratch = (P.flags & FFT_EXTERNAL_SCRATCH) != 0;
  std::ostringstream head;
  static const char* kinds[] = {"dft", "rdft r2c", "rdft c2r"};
  head << kinds[P.kind] << " rank=" << P.N.size() << " n=" << dims_str(P.N) << " howmany=" << dims_str(P.V)
       << " sign=" << P.sign << (out->inplace ? " in-place" : "") << ((P.flags & FFT_ESTIMATE) ? " estimate" : "")
       << "\n";
  if (P.empty) {
    out->info = head.str() + "  empty problem: no-op\n";
    return FFT_OK;
  }
  int64_t pts = 1, count = 1;
  for (const Dim& d : P.N) pts *= d.n;
  for (const Dim& d : P.V) count *= d.n;
  if (P.kind == 0) {
    footprint(P.N, P.V, true, &out->in_lo, &out->in_hi);
    footprint(P.N, P.V, false, &out->out_lo, &out->out_hi);
    out->bytes = 16.0 * (double)pts * (double)count;
    out->flops = pts > 1 ? 5.0 * (double)pts * std::log2((double)pts) * (double)count : 0.0;
  } else {
    // the complex side's last dimension has n / 2 + 1 entries; real sides are FP32
    std::vector<Dim> H = P.N;
    H.back().n = H.back().n / 2 + 1;
    const int64_t hpts = pts / P.N.back().n * H.back().n;
    footprint(P.kind == 1 ? P.N : H, P.V, true, &out->in_lo, &out->in_hi);
    footprint(P.kind == 1 ? H : P.N, P.V, false, &out->out_lo, &out->out_hi);
    out->in_elem = P.kind == 1 ? 4 : 8;
    out->out_elem = P.kind == 1 ? 8 : 4;
    out->bytes = (4.0 * (double)pts + 8.0 * (double)hpts) * (double)count;
    out->flops = pts > 1 ? 2.5 * (double)pts * std::log2((double)pts) * (double)count : 0.0;
  }
  if (device) {
    if (cudaGetDevice(&out->device) != cudaSuccess) {
      cudaGetLastError();
      return FFT_ERR_NO_DEVICE;
    }
    // the status word in mapped page-locked memory, so that fft_execute can
    // see an earlier execution's error without synchronising the device
    void* hp = nullptr;
    if (cudaHostAlloc(&hp, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess &&
        cudaHostGetDevicePointer((void**)&out->d_status, hp, 0) == cudaSuccess) {
      out->h_status = (int*)hp;
      *out->h_status = 0;
    } else {
      cudaGetLastError();
      if (hp) cudaFreeHost(hp);
      out->d_status = nullptr;
      if (cudaMalloc(&out->d_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return FFT_ERR_OOM;
      }
      cudaMemset(out->d_status, 0, sizeof(int));
    }
    if (cudaEventCreateWithFlags(&out->done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release(out);
      return FFT_ERR_CUDA;
    }
  }
  const bool measure = device && !(P.flags & FFT_ESTIMATE);
  Builder b(out, device, measure, (P.flags & FFT_WISDOM_ONLY) != 0);
  if (P.flags & (FFT_PREC_TC_FP16 | FFT_PREC_TC_BF16))
    b.prec = ((P.flags & FFT_PREC_TC_FP16) ? 1 : 2) + ((P.flags & FFT_PREC_SPLIT) ? 2 : 0);
  const int conj = P.sign > 0 ? 1 : 0;
  if (P.flags & FFT_DEBUG_STALL) {
    Step st;
    st.kind = STEP_STALL;
    st.pass.status = out->d_status;
    out->steps.push_back(st);
    b.line(1, "debug stall: one wait on an mbarrier nothing arrives on, bounded at 50 ms (reports "
              "FFT_ERR_DEVICE_TIMEOUT)");
  }
  if (P.kind) b.solve_real(P, 1);
  else b.solve(P.N, P.V, BUF_IN, out->inplace ? BUF_IN : BUF_OUT, conj, 1);
  if (!b.err && device && cudaStreamSynchronize(0) != cudaSuccess) b.err = FFT_ERR_CUDA;
  out->info = head.str() + b.info.str();
  if (b.err) {
    release(out);
    return b.err;
  }
  return FFT_OK;
}

int check_execute_args(const PlanData* p, const void* in, const void* out) {
  if (p->prob.empty) return FFT_OK;
  if (!in || !out) return FFT_ERR_INVALID_ARG;
  if (p->inplace) {
    if (in != out) return FFT_ERR_INPLACE_MISMATCH;
  } else {
    const char* a0 = (const char*)in + p->in_elem * p->in_lo;
    const char* a1 = (const char*)in + p->in_elem * (p->in_hi + 1);
    const char* b0 = (const char*)out + p->out_elem * p->out_lo;
    const char* b1 = (const char*)out + p->out_elem * (p->out_hi + 1);
    if (a0 < b1 && b0 < a1) return FFT_ERR_ALIAS;
  }
  if ((p->align8_in && ((uintptr_t)in & 7)) || (p->align8_out && ((uintptr_t)out & 7))) return FFT_ERR_INVALID_ARG;
  return FFT_OK;
}

int execute_plan(PlanData* p, const void* in, void* out, cudaStream_t st, void* work, bool api) {
  if (p->prob.empty) return FFT_OK;
  const int rc = check_execute_args(p, in, out);
  if (rc != FFT_OK) return rc;
  if (p->external_scratch && !p->scratch.empty() && (!work || ((uintptr_t)work & 255)))
    return FFT_ERR_INVALID_ARG;
  if (api) {
    // an error an earlier execution left in the status word (seen without a
    // device synchronisation) is reported now, and nothing is enqueued
    const int prev = take_status(p, false);
    if (prev != FFT_OK) return prev;
  }
  const int r = run_steps(p, in, p->inplace ? (void*)in : out, st, work);
  if (api && r == FFT_OK && p->done) {
    // the completion event of the last execution (not inside a stream capture,
    // where a recorded event cannot be waited on from the host)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FFT_ERR_CUDA;
    if (cs == cudaStreamCaptureStatusNone) {
      if (cudaEventRecord(p->done, st) != cudaSuccess) return FFT_ERR_CUDA;
      p->done_valid = true;
    }
  }
  return r;
}

}  // namespace gb
