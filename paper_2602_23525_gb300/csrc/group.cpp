// group.cpp -- uneven batches of plans executed together.
//
// Two executors, chosen per group by timing both once at creation (the
// measuring idea of sec. 4.3 applied to the whole batch):
//  * persistent queue: every step of every plan becomes a segment of (step,
//    tile) work items; the queue is ordered by step level so the dependency
//    of a segment (the previous step of its own plan) always precedes it.
//    Passes run through the generic Stockham tile code (a plan's specialised
//    pass kernels contribute their generic descriptor), Bluestein and copy
//    steps as element-wise chunks.  The launch -- clearing the counters, then
//    the kernel -- is captured once into a CUDA graph and replayed; the pointer
//    table the kernel reads is rewritten only when the caller's pointers change.
//  * graph of plan launches: each plan's own kernels on one of several forked
//    streams (independent plans run concurrently), joined back into the
//    caller's stream; captured into a CUDA graph that is updated in place when
//    the caller's pointers change.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
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
  // executor choice
  bool persistent_ok = true;
  int mode = 0;  // 1 persistent queue, 2 graph of plan launches
  // graph of plan launches
  std::vector<cudaStream_t> streams;
  std::vector<int> plan_stream;  // stream of each plan (a plan listed twice stays on one stream)
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraphExec_t pexec = nullptr;
  std::vector<const void*> pexec_ptrs;  // pointers the plan graph was captured with
  int plan_launches = 0;
};

namespace {

int64_t chunks(int64_t elems) { return (elems + GB_SEG_CHUNK - 1) / GB_SEG_CHUNK; }

// block size the group prefers (128 registers per thread); passes that need
// more threads per transform raise it to 1024
constexpr int kGroupThreads = 512;

void release(fft_group_s* g) {
  for (GbPass* d : g->own_desc) cudaFree(d);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->pexec) cudaGraphExecDestroy(g->pexec);
  for (cudaStream_t s : g->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->joins) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
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

// every plan's own launches on the forked streams, joined back into st
cudaError_t enqueue_plans(fft_group_s* g, const void* const* ins, void* const* outs, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(g->fork, st);
  for (size_t i = 0; e == cudaSuccess && i < g->streams.size(); ++i) e = cudaStreamWaitEvent(g->streams[i], g->fork, 0);
  for (size_t i = 0; e == cudaSuccess && i < g->plans.size(); ++i) {
    PlanData* P = &g->plans[i]->d;
    if (execute_plan(P, ins[i], P->inplace ? const_cast<void*>(ins[i]) : outs[i], g->streams[g->plan_stream[i]]) !=
        FFT_OK)
      e = cudaErrorLaunchFailure;
  }
  for (size_t i = 0; e == cudaSuccess && i < g->streams.size(); ++i) {
    e = cudaEventRecord(g->joins[i], g->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g->joins[i], 0);
  }
  return e;
}

// the plan graph for these pointers: captured on st, instantiated once and
// updated in place afterwards
cudaError_t plan_graph(fft_group_s* g, const void* const* ins, void* const* outs, cudaStream_t st) {
  std::vector<const void*> ptrs;
  for (size_t i = 0; i < g->plans.size(); ++i) {
    ptrs.push_back(ins[i]);
    ptrs.push_back(outs[i]);
  }
  if (g->pexec && ptrs == g->pexec_ptrs) return cudaSuccess;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t e1 = enqueue_plans(g, ins, outs, st);
  e = cudaStreamEndCapture(st, &graph);
  if (e1 != cudaSuccess || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return e1 != cudaSuccess ? e1 : (e != cudaSuccess ? e : cudaErrorUnknown);
  }
  bool done = false;
  if (g->pexec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(g->pexec, graph, &info) == cudaSuccess) done = true;
    else {
      cudaGetLastError();
      cudaGraphExecDestroy(g->pexec);
      g->pexec = nullptr;
    }
  }
  if (!done) e = cudaGraphInstantiate(&g->pexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->pexec = nullptr;
    return e;
  }
  g->pexec_ptrs = ptrs;
  return cudaSuccess;
}

// pointer table of the persistent queue for these pointers
std::vector<float2*> queue_ptrs(fft_group_s* g, const void* const* ins, void* const* outs) {
  std::vector<float2*> ptrs(g->nslots, nullptr);
  for (size_t i = 0; i < g->plans.size(); ++i) {
    const PlanData& P = g->plans[i]->d;
    const int b = g->slot_base[i];
    ptrs[b + BUF_IN] = (float2*)ins[i];
    ptrs[b + BUF_OUT] = P.inplace ? (float2*)ins[i] : (float2*)outs[i];
    for (size_t k = 0; k < P.scratch.size(); ++k) ptrs[b + BUF_SCRATCH0 + k] = (float2*)P.scratch[k];
  }
  return ptrs;
}

// Time both executors on buffers shaped like the plans' arrays (best of three
// after a warm-up each) and keep the faster; the graph of plan launches when
// buffers cannot be had.
int choose_mode(fft_group_s* g) {
  if (!g->persistent_ok) return 2;
  std::vector<void*> bufs;
  std::vector<const void*> ins;
  std::vector<void*> outs;
  bool ok = true;
  for (fft_plan p : g->plans) {
    const PlanData& P = p->d;
    const size_t in_n = (size_t)(P.in_hi - P.in_lo + 1), out_n = (size_t)(P.out_hi - P.out_lo + 1);
    void *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, sizeof(float2) * in_n) != cudaSuccess ||
        (!P.inplace && cudaMalloc(&b, sizeof(float2) * out_n) != cudaSuccess)) {
      cudaGetLastError();
      if (a) cudaFree(a);
      ok = false;
      break;
    }
    cudaMemset(a, 0, sizeof(float2) * in_n);
    bufs.push_back(a);
    if (b) bufs.push_back(b);
    ins.push_back((float2*)a - P.in_lo);
    outs.push_back(P.inplace ? (void*)((float2*)a - P.in_lo) : (void*)((float2*)b - P.out_lo));
  }
  int mode = 2;
  cudaStream_t st = nullptr;
  if (ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto best = [&](bool persistent) {
      float t = -1.f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        cudaError_t e;
        if (persistent) {
          const std::vector<float2*> ptrs = queue_ptrs(g, ins.data(), outs.data());
          e = cudaMemcpyAsync(g->dbufs, ptrs.data(), sizeof(float2*) * ptrs.size(), cudaMemcpyHostToDevice, st);
          if (e == cudaSuccess) e = enqueue(g, st);
        } else {
          e = enqueue_plans(g, ins.data(), outs.data(), st);
        }
        cudaEventRecord(e1, st);
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (t < 0 || ms < t)) t = ms;
      }
      return t;
    };
    const float tq = best(true);
    const float tg = best(false);
    if (tq > 0 && (tg < 0 || tq < tg)) mode = 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
  }
  cudaGetLastError();
  for (void* b : bufs) cudaFree(b);
  g->last_ptrs.clear();  // the pointer table holds the timing buffers
  return mode;
}

}  // namespace

extern "C" fft_group fft_group_create(int nplans, const fft_plan* plans, unsigned flags) {
  const unsigned known = FFT_GROUP_DEBUG_STALL | FFT_GROUP_PERSISTENT | FFT_GROUP_GRAPH;
  if (nplans < 1 || !plans || (flags & ~known) ||
      ((flags & FFT_GROUP_GRAPH) && (flags & (FFT_GROUP_PERSISTENT | FFT_GROUP_DEBUG_STALL)))) {
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
          g->persistent_ok = false;
      }
      if (!q.seg.pass && q.seg.kind == GB_SEG_PASS) g->persistent_ok = false;
      q.plan = i;
      q.level = (int)k;
      q.prev = prev;
      prev = (int)pend.size();
      pend.push_back(q);
    }
  }
  if (g->threads > 1024) g->persistent_ok = false;
  const bool want_queue = (flags & (FFT_GROUP_PERSISTENT | FFT_GROUP_DEBUG_STALL)) != 0;
  if (!err && want_queue && !g->persistent_ok) err = FFT_ERR_UNSUPPORTED;
  // graph of plan launches: up to eight forked streams, a plan listed twice
  // stays on one stream (its scratch is used by one execution at a time)
  if (!err) {
    const int ns = std::min<int>(nplans, 8);
    std::map<fft_plan, int> seen;
    for (int i = 0; i < nplans; ++i) {
      auto it = seen.find(plans[i]);
      const int sidx = it != seen.end() ? it->second : (int)(seen.size() % ns);
      seen[plans[i]] = sidx;
      g->plan_stream.push_back(sidx);
      g->plan_launches += plans[i]->d.steps.size();
    }
    g->streams.assign(ns, nullptr);
    g->joins.assign(ns, nullptr);
    for (int i = 0; i < ns && !err; ++i)
      if (cudaStreamCreateWithFlags(&g->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&g->joins[i], cudaEventDisableTiming) != cudaSuccess)
        err = FFT_ERR_CUDA;
    if (!err && cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) err = FFT_ERR_CUDA;
  }
  if (err) {
    cudaGetLastError();
    release(g);
    delete g;
    set_err(err);
    return nullptr;
  }
  if (!g->persistent_ok) {  // only the graph of plan launches applies
    g->mode = 2;
    set_err(FFT_OK);
    return g;
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
  g->mode = want_queue ? 1 : (flags & FFT_GROUP_GRAPH) ? 2 : choose_mode(g);
  set_err(FFT_OK);
  return g;
}

extern "C" int fft_group_execute(fft_group g, const void* const* ins, void* const* outs, void* stream) {
  if (!g || !ins || !outs) return set_err(FFT_ERR_INVALID_ARG);
  for (size_t i = 0; i < g->plans.size(); ++i) {
    const int rc = check_execute_args(&g->plans[i]->d, ins[i], outs[i]);
    if (rc != FFT_OK) return set_err(rc);
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (g->mode == 2) {
    // graph of plan launches; launched directly on the legacy stream or when
    // the caller's stream is itself being captured
    if (st == nullptr || plan_graph(g, ins, outs, st) != cudaSuccess) {
      cudaGetLastError();
      return set_err(enqueue_plans(g, ins, outs, st) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA);
    }
    return set_err(cudaGraphLaunch(g->pexec, st) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA);
  }
  const std::vector<float2*> ptrs = queue_ptrs(g, ins, outs);
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
  if (cudaDeviceSynchronize() != cudaSuccess) return set_err(FFT_ERR_CUDA);
  int bad = 0;
  if (g->dstatus) {
    int v = 0;
    if (cudaMemcpy(&v, g->dstatus, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return set_err(FFT_ERR_CUDA);
    if (v != 0) {
      bad = 1;
      cudaMemset(g->dstatus, 0, sizeof(int));
    }
  }
  for (fft_plan p : g->plans) {
    const int v = take_status(&p->d, true);
    if (v == FFT_ERR_CUDA) return set_err(FFT_ERR_CUDA);
    if (v != FFT_OK) bad = 1;
  }
  return set_err(bad ? FFT_ERR_DEVICE_TIMEOUT : FFT_OK);
}

extern "C" int fft_group_launches(fft_group g) { return g ? (g->mode == 2 ? g->plan_launches : 1) : 0; }

extern "C" int fft_group_mode(fft_group g) { return g ? g->mode : 0; }

extern "C" void fft_group_destroy(fft_group g) {
  if (!g) return;
  release(g);
  delete g;
}
