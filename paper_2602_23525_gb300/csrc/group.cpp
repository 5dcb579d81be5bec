// group.cpp -- uneven batches of plans executed by one persistent launch.
//
// Every step of every plan becomes a segment of (step, tile) work items; the
// queue is ordered by step level so the dependency of a segment (the previous
// step of its own plan) always precedes it.  Passes run through the generic
// Stockham tile code (a plan's TMA pass kernels contribute their generic
// fallback descriptor), Bluestein and copy steps as element-wise chunks.
// The launch itself -- clearing the counters, then the kernel -- is captured
// once into a CUDA graph and replayed; the pointer table the kernel reads is
// rewritten only when the caller's pointers change.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gb_plan.hpp"

using namespace gb;

struct fft_group_s {
  std::vector<fft_plan> plans;
  std::vector<int> slot_base;          // first pointer-table slot of each plan
  int nslots = 0;
  std::vector<GbGroupSeg> segs;
  GbGroupSeg* dsegs = nullptr;
  unsigned long long* dcount = nullptr;  // [0] = queue head, [1 + s] = done of segment s
  float2** dbufs = nullptr;
  int* dstatus = nullptr;
  std::vector<GbPass*> own_desc;       // narrowed copies of pass descriptors
  int64_t total = 0;
  int threads = 256;
  size_t smem = 0;
  int64_t grid = 0;
  unsigned long long wait_ns = 1000000000ull;
  std::vector<float2*> last_ptrs;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  bool have_graph = false;
};

namespace {

int64_t chunks(int64_t elems) { return (elems + GB_SEG_CHUNK - 1) / GB_SEG_CHUNK; }

// block size the group prefers (128 registers per thread); passes that need
// more threads per transform raise it to 1024
constexpr int kGroupThreads = 512;

void release(fft_group_s* g) {
  for (GbPass* d : g->own_desc) cudaFree(d);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->dsegs) cudaFree(g->dsegs);
  if (g->dcount) cudaFree(g->dcount);
  if (g->dbufs) cudaFree(g->dbufs);
  if (g->dstatus) cudaFree(g->dstatus);
}

GbGroupArgs args_of(const fft_group_s* g) {
  GbGroupArgs a;
  a.segs = g->dsegs;
  a.nseg = (int)g->segs.size();
  a.bufs = g->dbufs;
  a.head = g->dcount;
  a.done = g->dcount + 1;
  a.total = g->total;
  a.status = g->dstatus;
  a.wait_ns = g->wait_ns;
  return a;
}

cudaError_t enqueue(fft_group_s* g, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(g->dcount, 0, sizeof(unsigned long long) * (1 + g->segs.size()), st);
  if (e != cudaSuccess) return e;
  return gb_launch_group(args_of(g), g->threads, g->smem, g->grid, st);
}

}  // namespace

extern "C" fft_group fft_group_create(int nplans, const fft_plan* plans, unsigned flags) {
  if (nplans < 1 || !plans || (flags & ~FFT_GROUP_DEBUG_STALL)) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  fft_group_s* g = new (std::nothrow) fft_group_s;
  if (!g) {
    set_err(FFT_ERR_OOM);
    return nullptr;
  }
  struct Pending {
    GbGroupSeg seg;
    int plan, level, prev;  // prev: index (in pending order) of the previous step of the plan
  };
  std::vector<Pending> pend;
  int err = FFT_OK;
  for (int i = 0; i < nplans && !err; ++i) {
    if (!plans[i]) {
      err = FFT_ERR_INVALID_ARG;
      break;
    }
    const PlanData& P = plans[i]->d;
    if (P.external_scratch && !P.scratch.empty()) {
      err = FFT_ERR_UNSUPPORTED;
      break;
    }
    g->plans.push_back(plans[i]);
    g->slot_base.push_back(g->nslots);
    g->nslots += BUF_SCRATCH0 + (int)P.scratch.size();
    int prev = -1;
    for (size_t k = 0; k < P.steps.size(); ++k) {
      const Step& st = P.steps[k];
      Pending q;
      memset(&q.seg, 0, sizeof(q.seg));
      q.seg.src = g->slot_base.back() + st.src;
      q.seg.dst = g->slot_base.back() + st.dst;
      switch (st.kind) {
        case STEP_PASS:
        case STEP_CLUSTER:  // a cluster pass contributes its one-CTA fallback, where it has one
        case STEP_MR:       // a mixed-radix TMA pass contributes its generic pass
        case STEP_POW2: {  // a power-of-two pass contributes its generic fallback descriptor
          q.seg.kind = GB_SEG_PASS;
          q.seg.pass = st.dpass;
          q.seg.ntiles = st.pass.ntiles;
          int threads = st.threads;
          size_t smem = st.smem;
          if (threads > kGroupThreads && st.pass.tpt <= kGroupThreads && !st.pass.blue) {
            // fewer transforms per tile so that every item fits the group's block size
            GbPass n = st.pass;
            n.T = std::max(1, kGroupThreads / n.tpt);
            n.tiles0 = (n.vn[0] + n.T - 1) / n.T;
            n.ntiles = n.tiles0;
            for (int d = 1; d < n.nv; ++d) n.ntiles *= n.vn[d];
            GbPass* dn = nullptr;
            if (cudaMalloc(&dn, sizeof(GbPass)) != cudaSuccess ||
                cudaMemcpy(dn, &n, sizeof(GbPass), cudaMemcpyHostToDevice) != cudaSuccess) {
              cudaGetLastError();
              if (dn) cudaFree(dn);
              err = FFT_ERR_OOM;
              break;
            }
            g->own_desc.push_back(dn);
            q.seg.pass = dn;
            q.seg.ntiles = n.ntiles;
            threads = n.T * n.tpt;
            smem = st.smem ? (size_t)n.T * n.pitch * sizeof(float2) : 0;
          }
          g->threads = std::max(g->threads, threads);
          g->smem = std::max(g->smem, smem);
          break;
        }
        case STEP_COPY:
          q.seg.kind = GB_SEG_COPY;
          q.seg.copy = st.copy;
          q.seg.ntiles = chunks(st.copy.total);
          break;
        case STEP_BLUE_PRE:
          q.seg.kind = GB_SEG_BLUE_PRE;
          q.seg.blue = st.blue;
          q.seg.ntiles = chunks(st.blue.count * st.blue.m);
          break;
        case STEP_BLUE_MUL:
          q.seg.kind = GB_SEG_BLUE_MUL;
          q.seg.blue = st.blue;
          q.seg.ntiles = chunks(st.blue.count * st.blue.m);
          break;
        case STEP_BLUE_POST:
          q.seg.kind = GB_SEG_BLUE_POST;
          q.seg.blue = st.blue;
          q.seg.ntiles = chunks(st.blue.count * st.blue.n);
          break;
        default:
          err = FFT_ERR_UNSUPPORTED;
      }
      if (!q.seg.pass && q.seg.kind == GB_SEG_PASS) err = FFT_ERR_UNSUPPORTED;
      q.plan = i;
      q.level = (int)k;
      q.prev = prev;
      prev = (int)pend.size();
      pend.push_back(q);
    }
  }
  if (!err && g->threads > 1024) err = FFT_ERR_UNSUPPORTED;
  if (err) {
    release(g);
    delete g;
    set_err(err);
    return nullptr;
  }
  // queue order: by step level, then plan; remap dependencies
  std::vector<int> order(pend.size());
  for (size_t i = 0; i < pend.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pend[a].level < pend[b].level; });
  std::vector<int> pos(pend.size());
  for (size_t r = 0; r < order.size(); ++r) pos[order[r]] = (int)r;
  int64_t first = 0;
  for (size_t r = 0; r < order.size(); ++r) {
    GbGroupSeg s = pend[order[r]].seg;
    s.dep = pend[order[r]].prev >= 0 ? pos[pend[order[r]].prev] : -1;
    s.first = first;
    first += s.ntiles;
    g->segs.push_back(s);
  }
  g->total = first;
  if (flags & FFT_GROUP_DEBUG_STALL) {
    // one item that waits on a segment no item belongs to: the wait must give up
    GbGroupSeg never;
    memset(&never, 0, sizeof(never));
    never.kind = GB_SEG_COPY;
    never.dep = -1;
    never.ntiles = 1;
    never.first = (int64_t)1 << 62;
    GbGroupSeg stall = never;
    stall.first = g->total;
    stall.dep = (int)g->segs.size() + 1;
    stall.copy.total = 0;
    g->segs.push_back(stall);
    g->segs.push_back(never);
    g->total += 1;
    g->wait_ns = 50000000ull;  // 50 ms
  }
  const size_t nseg = g->segs.size();
  if (cudaMalloc(&g->dsegs, sizeof(GbGroupSeg) * std::max<size_t>(1, nseg)) != cudaSuccess ||
      cudaMalloc(&g->dcount, sizeof(unsigned long long) * (1 + nseg)) != cudaSuccess ||
      cudaMalloc(&g->dbufs, sizeof(float2*) * std::max(1, g->nslots)) != cudaSuccess ||
      cudaMalloc(&g->dstatus, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    release(g);
    delete g;
    set_err(FFT_ERR_OOM);
    return nullptr;
  }
  if (cudaMemcpy(g->dsegs, g->segs.data(), sizeof(GbGroupSeg) * nseg, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(g->dstatus, 0, sizeof(int)) != cudaSuccess) {
    release(g);
    delete g;
    set_err(FFT_ERR_CUDA);
    return nullptr;
  }
  g->grid = gb_group_grid(g->threads, g->smem);
  if (g->grid <= 0) {
    release(g);
    delete g;
    set_err(FFT_ERR_CUDA);
    return nullptr;
  }
  set_err(FFT_OK);
  return g;
}

extern "C" int fft_group_execute(fft_group g, const void* const* ins, void* const* outs, void* stream) {
  if (!g || !ins || !outs) return set_err(FFT_ERR_INVALID_ARG);
  std::vector<float2*> ptrs(g->nslots, nullptr);
  for (size_t i = 0; i < g->plans.size(); ++i) {
    const PlanData& P = g->plans[i]->d;
    const int rc = check_execute_args(&g->plans[i]->d, ins[i], outs[i]);
    if (rc != FFT_OK) return set_err(rc);
    const int b = g->slot_base[i];
    ptrs[b + BUF_IN] = (float2*)ins[i];
    ptrs[b + BUF_OUT] = P.inplace ? (float2*)ins[i] : (float2*)outs[i];
    for (size_t k = 0; k < P.scratch.size(); ++k) ptrs[b + BUF_SCRATCH0 + k] = (float2*)P.scratch[k];
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (ptrs != g->last_ptrs) {
    if (cudaMemcpyAsync(g->dbufs, ptrs.data(), sizeof(float2*) * ptrs.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return set_err(FFT_ERR_CUDA);
    g->last_ptrs = ptrs;
  }
  if (st == nullptr) {  // the legacy stream cannot be captured: launch directly
    return set_err(enqueue(g, st) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA);
  }
  if (!g->have_graph) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return set_err(enqueue(g, st) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA);
    }
    const cudaError_t e1 = enqueue(g, st);
    const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess || !graph ||
        cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return set_err(FFT_ERR_CUDA);
    }
    cudaGraphDestroy(graph);
    g->have_graph = true;
  }
  return set_err(cudaGraphLaunch(g->exec, st) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA);
}

extern "C" int fft_group_status(fft_group g) {
  if (!g) return set_err(FFT_ERR_INVALID_ARG);
  int v = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&v, g->dstatus, sizeof(int), cudaMemcpyDeviceToHost) !=
                                                    cudaSuccess)
    return set_err(FFT_ERR_CUDA);
  if (v != 0) cudaMemset(g->dstatus, 0, sizeof(int));
  return set_err(v == 0 ? FFT_OK : FFT_ERR_DEVICE_TIMEOUT);
}

extern "C" int fft_group_launches(fft_group g) { return g ? 1 : 0; }

extern "C" void fft_group_destroy(fft_group g) {
  if (!g) return;
  release(g);
  delete g;
}
