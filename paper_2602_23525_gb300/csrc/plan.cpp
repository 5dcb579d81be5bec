// plan.cpp -- problems, plans and the planner (sec. 4 of the paper), and the
// C ABI declared in include/gbfft.h.
//
//  * canonicalize(): the problem dft(N, V, I, O) of sec. 4.1 -- validation,
//    dropping length-1 dimensions, merging vector dimensions that form one
//    stride run, and the injectivity check of the output map.
//  * Builder::solve(): the algorithmic steps of sec. 4.2 composed into a plan:
//      rank 0          -> copy (rank-0 plans)
//      rank >= 2       -> one rank-1 sub-problem per dimension, the other
//                         dimensions joining the vector loops (separable DFT)
//      rank 1, small   -> one Stockham pass (direct/codelet plans + the
//                         Cooley-Tukey twiddle codelets, fused in one CTA)
//      rank 1, large   -> Cooley-Tukey with an arbitrary radix n1 (the
//                         radix-sqrt(n) / four-step step, eq. (2)): a pass of
//                         n2 DFTs of size n1 with the twiddles w_n^{l2 k1}
//                         fused, then the n1 DFTs of size n2 as a sub-problem
//      large prime     -> Bluestein (prime-size plans)
//  * the planner (sec. 4.3): every rank-1 sub-problem is solved by timing the
//    applicable candidates on the device (measure mode) or by a heuristic
//    (estimate mode), and the decision is memoised per canonical sub-problem
//    (dynamic programming); the memo is the exportable wisdom.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/gbfft.h"
#include "gb_kernels.h"
#include "gb_pass.h"
#include "gb_plan.hpp"

namespace gb {

thread_local int g_last_error = FFT_OK;

int set_err(int e) {
  g_last_error = e;
  return e;
}

static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

// --------------------------------------------------------------------------
// Canonical problems (sec. 4.1)

std::string dims_str(const std::vector<Dim>& v) {
  std::ostringstream o;
  o << "[";
  for (size_t i = 0; i < v.size(); ++i) {
    if (i) o << ",";
    o << "(" << v[i].n << "," << v[i].is << "," << v[i].os << ")";
  }
  o << "]";
  return o.str();
}

static const unsigned kKnownFlags = FFT_ESTIMATE | FFT_WISDOM_ONLY | FFT_INPLACE | FFT_EXTERNAL_SCRATCH | FFT_PREC_TC_FP16 |
                                    FFT_PREC_TC_BF16 | FFT_PREC_SPLIT | FFT_DEBUG_STALL;

int canonicalize(int rank, const fft_iodim* dims, int hr, const fft_iodim* hd, int sign,
                 unsigned flags, Problem& P) {
  if (rank < 0 || hr < 0) return FFT_ERR_INVALID_ARG;
  if ((rank > 0 && !dims) || (hr > 0 && !hd)) return FFT_ERR_INVALID_ARG;
  if (sign != -1 && sign != 1) return FFT_ERR_INVALID_ARG;
  if (flags & ~kKnownFlags) return FFT_ERR_INVALID_ARG;
  if ((flags & FFT_PREC_TC_FP16) && (flags & FFT_PREC_TC_BF16)) return FFT_ERR_INVALID_ARG;
  if ((flags & FFT_PREC_SPLIT) && !(flags & (FFT_PREC_TC_FP16 | FFT_PREC_TC_BF16))) return FFT_ERR_INVALID_ARG;
  if (rank > 3 || hr > 3) return FFT_ERR_UNSUPPORTED;
  P = Problem();
  P.sign = sign;
  P.flags = flags;
  for (int i = 0; i < rank; ++i) {
    if (dims[i].n < 0) return FFT_ERR_INVALID_ARG;
    if (dims[i].n == 0) P.empty = true;
  }
  for (int i = 0; i < hr; ++i) {
    if (hd[i].n < 0) return FFT_ERR_INVALID_ARG;
    if (hd[i].n == 0) P.empty = true;
  }
  if (flags & FFT_INPLACE) {
    // a transform in place needs equal strides; a rank-0 problem in place is
    // a permutation (sec. 4.1.1), which the planner accepts or refuses
    for (int i = 0; i < rank; ++i)
      if (dims[i].is != dims[i].os) return FFT_ERR_INPLACE_MISMATCH;
    for (int i = 0; i < hr && rank > 0; ++i)
      if (hd[i].is != hd[i].os) return FFT_ERR_INPLACE_MISMATCH;
  }
  if (P.empty) return FFT_OK;
  for (int i = 0; i < rank; ++i)
    if (dims[i].n > 1) P.N.push_back({dims[i].n, dims[i].is, dims[i].os});
  std::vector<Dim> V;
  for (int i = 0; i < hr; ++i)
    if (hd[i].n > 1) V.push_back({hd[i].n, hd[i].is, hd[i].os});
  // vector loops: outermost (largest strides) first, then merge stride runs
  std::stable_sort(V.begin(), V.end(), [](const Dim& a, const Dim& b) {
    if (iabs64(a.os) != iabs64(b.os)) return iabs64(a.os) > iabs64(b.os);
    return iabs64(a.is) > iabs64(b.is);
  });
  std::vector<Dim> M;
  for (const Dim& d : V) {
    if (!M.empty()) {
      Dim& a = M.back();
      if (a.is == d.n * d.is && a.os == d.n * d.os) {
        a = {a.n * d.n, d.is, d.os};
        continue;
      }
    }
    M.push_back(d);
  }
  P.V = M;
  // the output map must be injective: sorted by |os|, each stride must exceed
  // the span of the smaller ones (a mixed-radix numbering of the outputs)
  std::vector<Dim> all = P.N;
  all.insert(all.end(), P.V.begin(), P.V.end());
  std::sort(all.begin(), all.end(), [](const Dim& a, const Dim& b) { return iabs64(a.os) < iabs64(b.os); });
  int64_t span = 0;
  for (const Dim& d : all) {
    if (iabs64(d.os) <= span) return FFT_ERR_OUTPUT_OVERLAP;
    span += (d.n - 1) * iabs64(d.os);
  }
  return FFT_OK;
}

// A real-data problem (sec. 5, sec. 7): N's last dimension is the real one;
// on the complex side it has n / 2 + 1 entries.  Strides stay in the units of
// each side.  Length-1 dimensions other than the last are dropped (the last
// one is kept: a length-1 real transform is still a real-to-complex copy).
int canonicalize_real(int rank, const fft_iodim* dims, int hr, const fft_iodim* hd, int kind, unsigned flags,
                      Problem& P) {
  if (rank < 1 || hr < 0 || !dims || (hr > 0 && !hd) || (kind != 1 && kind != 2)) return FFT_ERR_INVALID_ARG;
  if (flags & ~kKnownFlags) return FFT_ERR_INVALID_ARG;
  if (rank > 3 || hr > 3) return FFT_ERR_UNSUPPORTED;
  if (flags & (FFT_INPLACE | FFT_EXTERNAL_SCRATCH | FFT_PREC_TC_FP16 | FFT_PREC_TC_BF16 | FFT_PREC_SPLIT))
    return FFT_ERR_UNSUPPORTED;
  P = Problem();
  P.kind = kind;
  P.sign = kind == 1 ? -1 : 1;
  P.flags = flags;
  for (int i = 0; i < rank; ++i) {
    if (dims[i].n < 0) return FFT_ERR_INVALID_ARG;
    if (dims[i].n == 0) P.empty = true;
  }
  for (int i = 0; i < hr; ++i) {
    if (hd[i].n < 0) return FFT_ERR_INVALID_ARG;
    if (hd[i].n == 0) P.empty = true;
  }
  if (P.empty) return FFT_OK;
  for (int i = 0; i + 1 < rank; ++i)
    if (dims[i].n > 1) P.N.push_back({dims[i].n, dims[i].is, dims[i].os});
  P.N.push_back({dims[rank - 1].n, dims[rank - 1].is, dims[rank - 1].os});
  for (int i = 0; i < hr; ++i)
    if (hd[i].n > 1) P.V.push_back({hd[i].n, hd[i].is, hd[i].os});
  // the output map must be injective (the complex side with n / 2 + 1 entries)
  std::vector<Dim> all = P.N;
  if (kind == 1) all.back().n = all.back().n / 2 + 1;
  all.insert(all.end(), P.V.begin(), P.V.end());
  std::sort(all.begin(), all.end(), [](const Dim& a, const Dim& b) { return iabs64(a.os) < iabs64(b.os); });
  int64_t span = 0;
  for (const Dim& d : all) {
    if (d.n > 1 && iabs64(d.os) <= span) return FFT_ERR_OUTPUT_OVERLAP;
    span += (d.n - 1) * iabs64(d.os);
  }
  return FFT_OK;
}

void footprint(const std::vector<Dim>& N, const std::vector<Dim>& V, bool input, int64_t* lo, int64_t* hi) {
  int64_t a = 0, b = 0;
  auto acc = [&](const Dim& d) {
    const int64_t s = input ? d.is : d.os;
    const int64_t e = (d.n - 1) * s;
    if (e < 0) a += e;
    else b += e;
  };
  for (const Dim& d : N) acc(d);
  for (const Dim& d : V) acc(d);
  *lo = a;
  *hi = b;
}

// --------------------------------------------------------------------------
// Radix schedules

bool smooth_codelet(int64_t n) {
  for (int p : {2, 3, 5, 7, 11, 13})
    while (n % p == 0) n /= p;
  return n == 1;
}

int64_t largest_prime_factor(int64_t n) {
  int64_t best = 1;
  for (int64_t p = 2; p * p <= n; ++p)
    while (n % p == 0) {
      best = p;
      n /= p;
    }
  return n > 1 ? std::max(best, n) : best;
}

std::vector<int> default_radices(int64_t n) {
  std::vector<int> r;
  int e2 = 0, e3 = 0;
  while (n % 2 == 0) { n /= 2; ++e2; }
  while (n % 3 == 0) { n /= 3; ++e3; }
  while (e2 >= 4) { r.push_back(16); e2 -= 4; }
  if (e2 == 3) r.push_back(8);
  if (e2 == 2) r.push_back(4);
  if (e2 == 1) r.push_back(2);
  while (e3 >= 2) { r.push_back(9); e3 -= 2; }
  if (e3 == 1) r.push_back(3);
  for (int p : {5, 7, 11, 13})
    while (n % p == 0) { r.push_back(p); n /= p; }
  return r;
}

int threads_per_transform(int64_t n, const std::vector<int>& rad) {
  int tpt = 1;
  for (int R : rad) {
    const int bmax = GB_VALS / R;
    const int64_t nb = n / R;
    const int need = (int)((nb + bmax - 1) / bmax);
    tpt = std::max(tpt, need);
  }
  return tpt;
}

int smem_pitch(int64_t n) {
  int p = (int)(n + ((n - 1) >> 5) + 1);
  if ((p & 1) == 0) ++p;
  return p;
}

std::string PassCfg::str() const {
  std::ostringstream o;
  o << "R=";
  for (size_t i = 0; i < radices.size(); ++i) o << (i ? "." : "") << radices[i];
  o << ":T=" << T << ":f=" << t_fast << ":l=" << load_mode << ":s=" << store_mode << ":lc=" << load_copy
    << ":sc=" << store_copy;
  return o.str();
}

bool PassCfg::parse(const std::string& s) {
  PassCfg c;
  std::string body = s;
  std::vector<std::string> parts;
  size_t st = 0;
  while (true) {
    size_t q = body.find(':', st);
    parts.push_back(body.substr(st, q == std::string::npos ? std::string::npos : q - st));
    if (q == std::string::npos) break;
    st = q + 1;
  }
  for (const std::string& kv : parts) {
    const size_t e = kv.find('=');
    if (e == std::string::npos) return false;
    const std::string k = kv.substr(0, e), v = kv.substr(e + 1);
    if (k == "R") {
      size_t a = 0;
      while (a <= v.size()) {
        size_t b = v.find('.', a);
        std::string tok = v.substr(a, b == std::string::npos ? std::string::npos : b - a);
        if (tok.empty()) return false;
        c.radices.push_back(atoi(tok.c_str()));
        if (b == std::string::npos) break;
        a = b + 1;
      }
    } else if (k == "T") c.T = atoi(v.c_str());
    else if (k == "f") c.t_fast = atoi(v.c_str());
    else if (k == "l") c.load_mode = atoi(v.c_str());
    else if (k == "s") c.store_mode = atoi(v.c_str());
    else if (k == "lc") c.load_copy = atoi(v.c_str());
    else if (k == "sc") c.store_copy = atoi(v.c_str());
    else return false;
  }
  if (c.radices.empty() || c.T < 1) return false;
  for (int R : c.radices)
    if (R != 2 && R != 3 && R != 4 && R != 5 && R != 7 && R != 8 && R != 9 && R != 11 && R != 13 && R != 16)
      return false;
  *this = c;
  return true;
}

// --------------------------------------------------------------------------
// Wisdom: the planner's memo (sec. 4.3, dynamic programming), keyed by the
// canonical rank-1 sub-problem, exportable as text.

std::mutex g_wisdom_mu;
std::map<std::string, std::string> g_wisdom;

bool wisdom_get(const std::string& key, std::string* val) {
  std::lock_guard<std::mutex> g(g_wisdom_mu);
  auto it = g_wisdom.find(key);
  if (it == g_wisdom.end()) return false;
  *val = it->second;
  return true;
}

void wisdom_put(const std::string& key, const std::string& val) {
  std::lock_guard<std::mutex> g(g_wisdom_mu);
  g_wisdom[key] = val;
}

// --------------------------------------------------------------------------
// Device context of the planner

int g_smem_optin = 0;

int smem_limit() {
  if (g_smem_optin <= 0) {
    g_smem_optin = gb_pass_max_smem_optin();
    if (g_smem_optin <= 0) g_smem_optin = 227 * 1024;  // explain mode without a device
  }
  return g_smem_optin;
}

bool single_pass_ok(int64_t n, const std::vector<int>& rad) {
  if (n > 65536) return false;
  const int tpt = threads_per_transform(n, rad);
  if (tpt > 1024) return false;
  return (int64_t)smem_pitch(n) * 8 <= smem_limit();
}

}  // namespace gb
