// gb_plan.hpp -- internal host-side structures of problems and plans.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gbfft.h"
#include "gb_kernels.h"
#include "gb_pass.h"

namespace gb {

// An I/O dimension (n, is, os) of sec. 4.1, strides in complex elements.
struct Dim {
  int64_t n, is, os;
};

// A canonical problem dft(N, V, I, O) without its pointers.
struct Problem {
  std::vector<Dim> N, V;
  int kind = 0;  // 0 complex, 1 real input (r2c), 2 real output (c2r)
  int sign = -1;
  unsigned flags = 0;
  bool empty = false;
};

// Configuration of one Stockham pass (the choices the planner makes).
struct PassCfg {
  std::vector<int> radices;
  int T = 1, t_fast = 0, load_mode = 0, store_mode = 0, load_copy = 0, store_copy = 0;
  std::string str() const;
  bool parse(const std::string& s);
};

enum StepKind {
  STEP_PASS = 0,
  STEP_COPY = 1,
  STEP_BLUE_PRE = 2,
  STEP_BLUE_MUL = 3,
  STEP_BLUE_POST = 4,
  STEP_POW2 = 5,
  STEP_CLUSTER = 6,
  STEP_MR = 7,
  STEP_STALL = 8,  // FFT_DEBUG_STALL: a bounded wait that runs out
  STEP_RADER_PRE = 9,
  STEP_RADER_MUL = 10,
  STEP_RADER_POST = 11,
  STEP_L2FS = 12,  // four-step with the intermediate in an L2-resident ring
  STEP_R2C_POST = 13,    // real input: half spectrum from the half-length complex DFT, in place
  STEP_R2C_PROMOTE = 14, // real input widened to complex
  STEP_C2R_PRE = 15,     // real output: the half-length complex input of the backward DFT
  STEP_C2R_EXPAND = 16,  // half spectrum extended to the full conjugate-symmetric spectrum
  STEP_C2R_REAL = 17,    // real parts to the real output
  STEP_TRANSPOSE_IP = 18 // in-place square transpose (rank 0, I = O)
};

// Buffer ids used by steps: 0 = user input, 1 = user output, 2+k = scratch k.
enum { BUF_IN = 0, BUF_OUT = 1, BUF_SCRATCH0 = 2 };

struct Step {
  int kind = STEP_PASS;
  GbPass pass{};
  const GbPass* dpass = nullptr;  // device copy of pass (what the kernel reads)
  GbP2 p2{};                      // STEP_POW2; pass/dpass hold the generic fallback
                                  // used when the input pointer is not 16-byte aligned
  GbCluster cl{};                 // STEP_CLUSTER; pass/dpass hold a one-CTA fallback where one exists
  GbMR mr{};                      // STEP_MR; pass/dpass hold the generic pass (run by the group executor)
  GbCopy copy{};
  GbBlueIO blue{};
  GbRaderIO rader{};
  GbL2FS l2{};                    // STEP_L2FS: ring and counters come from scratch buffer `aux`
  GbRealIO real{};                // real-data steps
  int src = BUF_IN, dst = BUF_OUT;
  int aux = -1;                   // a further buffer id (Rader's per-transform side values)
  int threads = 0;
  size_t smem = 0;
  int64_t grid = 0;
};

struct PlanData {
  Problem prob;
  std::vector<Step> steps;
  std::vector<void*> tables;   // device memory owned by the plan
  std::vector<void*> scratch;  // scratch buffers (ids BUF_SCRATCH0 + k)
  std::vector<size_t> scratch_bytes;
  std::vector<size_t> scratch_offset;  // external scratch: offsets in the caller's work area
  bool external_scratch = false;
  // status word: page-locked host memory mapped into the device (h_status,
  // its device alias d_status), or device memory alone (h_status null)
  int* d_status = nullptr;
  int* h_status = nullptr;
  cudaEvent_t done = nullptr;  // recorded after each fft_execute outside stream capture
  bool done_valid = false;
  std::string info;
  double bytes = 0.0, flops = 0.0;
  int64_t in_lo = 0, in_hi = 0, out_lo = 0, out_hi = 0;  // footprints in elements
  int in_elem = 8, out_elem = 8;                          // element bytes (4 on a real side)
  bool align8_in = false, align8_out = false;             // a real side read or written as complex pairs
  bool inplace = false;
  int device = -1;
};

// plan.cpp
extern thread_local int g_last_error;
int set_err(int e);
int canonicalize(int rank, const fft_iodim* dims, int hr, const fft_iodim* hd, int sign, unsigned flags,
                 Problem& P);
// a real-data problem (kind 1 r2c, 2 c2r); strides as given (real or complex units per side)
int canonicalize_real(int rank, const fft_iodim* dims, int hr, const fft_iodim* hd, int kind, unsigned flags,
                      Problem& P);
void footprint(const std::vector<Dim>& N, const std::vector<Dim>& V, bool input, int64_t* lo, int64_t* hi);
std::string dims_str(const std::vector<Dim>& v);
bool smooth_codelet(int64_t n);
int64_t largest_prime_factor(int64_t n);
std::vector<int> default_radices(int64_t n);
int threads_per_transform(int64_t n, const std::vector<int>& rad);
int smem_pitch(int64_t n);
int smem_limit();
bool single_pass_ok(int64_t n, const std::vector<int>& rad);
extern std::mutex g_wisdom_mu;
extern std::map<std::string, std::string> g_wisdom;
bool wisdom_get(const std::string& key, std::string* val);
void wisdom_put(const std::string& key, const std::string& val);

// builder.cpp
// Build the steps of a plan.  device = false builds the estimate-mode plan
// text only (no allocation, no timing).  Returns an FFT_* code.
int build_plan(const Problem& P, bool device, PlanData* out);
void free_plan(PlanData* p);
// api: a call of the public entry points (reports an error an earlier
// execution left, records the completion event); internal callers (groups,
// the serving loop) pass false
int execute_plan(PlanData* p, const void* in, void* out, cudaStream_t st, void* work = nullptr, bool api = false);
int check_execute_args(const PlanData* p, const void* in, const void* out);
int launch_step(const Step& s, float2* const* bufs, cudaStream_t st);
// the plan's device-side error code (0 = none), cleared; `wait` first waits
// for the plan's last execution
int take_status(PlanData* p, bool wait);

}  // namespace gb

struct fft_plan_s {
  gb::PlanData d;
};
