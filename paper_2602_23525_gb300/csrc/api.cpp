// api.cpp -- the extern "C" entry points declared in include/gbfft.h.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <sstream>
#include <string>

#include "gb_plan.hpp"

using namespace gb;

static int copy_out(const std::string& s, char* buf, size_t len) {
  if (buf && len > 0) {
    const size_t k = std::min(len - 1, s.size());
    memcpy(buf, s.data(), k);
    buf[k] = '\0';
  }
  return (int)s.size();
}

extern "C" {

int fft_last_error(void) { return g_last_error; }

const char* fft_error_string(int code) {
  switch (code) {
    case FFT_OK: return "ok";
    case FFT_ERR_INVALID_ARG: return "invalid argument";
    case FFT_ERR_UNSUPPORTED: return "unsupported problem";
    case FFT_ERR_ALIAS: return "input and output overlap";
    case FFT_ERR_INPLACE_MISMATCH: return "in-place plan needs in == out and equal strides";
    case FFT_ERR_OOM: return "device allocation failed";
    case FFT_ERR_BUDGET: return "byte budget exceeded";
    case FFT_ERR_CUDA: return "CUDA runtime error";
    case FFT_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case FFT_ERR_WISDOM: return "wisdom missing or malformed";
    case FFT_ERR_NO_DEVICE: return "no usable CUDA device";
    case FFT_ERR_OUTPUT_OVERLAP: return "output map is not injective";
    default: return "unknown error";
  }
}

fft_plan fft_plan_dft(int rank, const fft_iodim* dims, int howmany_rank, const fft_iodim* howmany_dims, int sign,
                      unsigned flags) {
  Problem P;
  int rc = canonicalize(rank, dims, howmany_rank, howmany_dims, sign, flags, P);
  if (rc != FFT_OK) {
    set_err(rc);
    return nullptr;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    set_err(FFT_ERR_NO_DEVICE);
    return nullptr;
  }
  fft_plan p = new (std::nothrow) fft_plan_s;
  if (!p) {
    set_err(FFT_ERR_OOM);
    return nullptr;
  }
  rc = build_plan(P, true, &p->d);
  if (rc != FFT_OK) {
    delete p;
    set_err(rc);
    return nullptr;
  }
  set_err(FFT_OK);
  return p;
}

static fft_plan plan_real(int rank, const fft_iodim* dims, int howmany_rank, const fft_iodim* howmany_dims,
                          int kind, unsigned flags) {
  Problem P;
  int rc = canonicalize_real(rank, dims, howmany_rank, howmany_dims, kind, flags, P);
  if (rc != FFT_OK) {
    set_err(rc);
    return nullptr;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    set_err(FFT_ERR_NO_DEVICE);
    return nullptr;
  }
  fft_plan p = new (std::nothrow) fft_plan_s;
  if (!p) {
    set_err(FFT_ERR_OOM);
    return nullptr;
  }
  rc = build_plan(P, true, &p->d);
  if (rc != FFT_OK) {
    delete p;
    set_err(rc);
    return nullptr;
  }
  set_err(FFT_OK);
  return p;
}

fft_plan fft_plan_dft_r2c(int rank, const fft_iodim* dims, int howmany_rank, const fft_iodim* howmany_dims,
                          unsigned flags) {
  return plan_real(rank, dims, howmany_rank, howmany_dims, 1, flags);
}

fft_plan fft_plan_dft_c2r(int rank, const fft_iodim* dims, int howmany_rank, const fft_iodim* howmany_dims,
                          unsigned flags) {
  return plan_real(rank, dims, howmany_rank, howmany_dims, 2, flags);
}

int fft_plan_explain(int rank, const fft_iodim* dims, int howmany_rank, const fft_iodim* howmany_dims, int sign,
                     unsigned flags, char* buf, size_t len) {
  Problem P;
  int rc = canonicalize(rank, dims, howmany_rank, howmany_dims, sign, flags, P);
  if (rc != FFT_OK) {
    set_err(rc);
    return -1;
  }
  P.flags |= FFT_ESTIMATE;
  PlanData d;
  rc = build_plan(P, false, &d);
  if (rc != FFT_OK) {
    set_err(rc);
    return -1;
  }
  set_err(FFT_OK);
  return copy_out(d.info, buf, len);
}

int fft_execute(fft_plan p, const void* in, void* out, void* stream) {
  if (!p) return set_err(FFT_ERR_INVALID_ARG);
  if (p->d.external_scratch && !p->d.scratch.empty()) return set_err(FFT_ERR_INVALID_ARG);
  const int rc = execute_plan(&p->d, in, out, (cudaStream_t)stream, nullptr, true);
  return set_err(rc);
}

int fft_execute_scratch(fft_plan p, const void* in, void* out, void* scratch, void* stream) {
  if (!p) return set_err(FFT_ERR_INVALID_ARG);
  if (!p->d.external_scratch) return set_err(FFT_ERR_INVALID_ARG);
  return set_err(execute_plan(&p->d, in, out, (cudaStream_t)stream, scratch, true));
}

int fft_sync_status(fft_plan p) {
  if (!p) return set_err(FFT_ERR_INVALID_ARG);
  return set_err(take_status(&p->d, true));
}

void fft_destroy(fft_plan p) {
  if (!p) return;
  free_plan(&p->d);
  delete p;
}

int fft_plan_info(fft_plan p, char* buf, size_t len) {
  if (!p) {
    set_err(FFT_ERR_INVALID_ARG);
    return -1;
  }
  return copy_out(p->d.info, buf, len);
}

double fft_plan_bytes(fft_plan p) { return p ? p->d.bytes : 0.0; }
double fft_plan_flops(fft_plan p) { return p ? p->d.flops : 0.0; }
int fft_plan_launches(fft_plan p) { return p ? (int)p->d.steps.size() : 0; }

size_t fft_plan_scratch_bytes(fft_plan p) {
  if (!p) return 0;
  size_t s = 0;
  for (size_t b : p->d.scratch_bytes) s += (b + 255) & ~(size_t)255;
  return s;
}

}  // extern "C"

// ---------------------------------------------------------------- wisdom
// Text format: a header line "gbfft-wisdom 1", then one decision per line,
// "<canonical sub-problem key>\t<choice>".

extern "C" int fft_export_wisdom(char* buf, size_t len) {
  std::ostringstream o;
  o << "gbfft-wisdom 1\n";
  {
    std::lock_guard<std::mutex> g(g_wisdom_mu);
    for (const auto& kv : g_wisdom) o << kv.first << "\t" << kv.second << "\n";
  }
  set_err(FFT_OK);
  return copy_out(o.str(), buf, len);
}

extern "C" int fft_import_wisdom(const char* text) {
  if (!text) return set_err(FFT_ERR_INVALID_ARG);
  std::istringstream in(text);
  std::string line;
  if (!std::getline(in, line) || line != "gbfft-wisdom 1") return set_err(FFT_ERR_WISDOM);
  std::map<std::string, std::string> add;
  while (std::getline(in, line)) {
    if (line.empty()) continue;
    const size_t tab = line.find('\t');
    if (tab == std::string::npos || tab == 0 || tab + 1 >= line.size()) return set_err(FFT_ERR_WISDOM);
    const std::string key = line.substr(0, tab), val = line.substr(tab + 1);
    if (key.rfind("r1 ", 0) != 0) return set_err(FFT_ERR_WISDOM);
    if (val == "p2" || val == "mr" || val == "xpose" || val == "indirect") {
    } else if (val.rfind("ip4:", 0) == 0) {
      if (atoll(val.c_str() + 4) < 2) return set_err(FFT_ERR_WISDOM);
    } else if (val.rfind("single:", 0) == 0) {
      PassCfg c;
      if (!c.parse(val.substr(7))) return set_err(FFT_ERR_WISDOM);
    } else if (val.rfind("split:", 0) == 0) {
      if (atoll(val.c_str() + 6) < 2) return set_err(FFT_ERR_WISDOM);
    } else if (val.rfind("blue:", 0) == 0) {
      if (atoll(val.c_str() + 5) < 3) return set_err(FFT_ERR_WISDOM);
    } else if (val.rfind("l2fs:", 0) == 0) {
      if (atoll(val.c_str() + 5) < 2) return set_err(FFT_ERR_WISDOM);
    } else if (val.rfind("rader:", 0) == 0) {
      if (atoll(val.c_str() + 6) < 2) return set_err(FFT_ERR_WISDOM);
    } else if (val.rfind("cluster:", 0) == 0) {
      int l1 = 0, l2 = 0, cs = 0, nb = 0, cfg[16][4];
      if (sscanf(val.c_str(), "cluster:%d.%d.%d.%d", &l1, &l2, &cs, &nb) != 4) return set_err(FFT_ERR_WISDOM);
      const int nc = gb_cluster_configs(l1 + l2, cfg, 16);
      bool known = false;
      for (int i = 0; i < nc; ++i)
        known |= cfg[i][0] == l1 && cfg[i][1] == l2 && cfg[i][2] == cs && cfg[i][3] == nb;
      if (!known) return set_err(FFT_ERR_WISDOM);
    } else {
      return set_err(FFT_ERR_WISDOM);
    }
    add[key] = val;
  }
  for (const auto& kv : add) wisdom_put(kv.first, kv.second);
  return set_err(FFT_OK);
}

extern "C" void fft_forget_wisdom(void) {
  std::lock_guard<std::mutex> g(g_wisdom_mu);
  g_wisdom.clear();
}
