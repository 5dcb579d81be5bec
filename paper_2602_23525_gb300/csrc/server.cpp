// server.cpp -- a continuous-batching request loop over the plan library.
//
// Requests are dense row-major transforms (rank 1..3, a batch, a sign) with
// host input and output buffers.  One worker thread runs the loop:
//   * retire: launches whose completion event has fired release their device
//     work buffers and complete their requests (latency = completion - arrival);
//   * admit: waiting requests are taken in arrival order; the ones still
//     waiting with the same shape and sign join the same launch (merged into
//     one batch); a launch is admitted when its work buffers (input, output,
//     plan scratch) fit in the unused part of the byte budget and a stream has
//     a free slot, so requests that arrive while others run are admitted as
//     memory and slots free up, and their copies and transforms overlap on the
//     device across the streams;
//   * launch: a three-stage pipeline over streams joined by events: the
//     host->device copies of each request's input on the copy-in stream (one
//     queue in admission order), the plan execution of the merged batch on the
//     least busy compute stream, the device->host copies of each output on the
//     copy-out stream (one queue); so both directions of the host link stay
//     busy while transforms run, and a launch's copies never wait behind
//     another launch's transform on the same stream.
// Plans stay resident in a cache keyed by (shape, sign, batch bucket); they
// use external scratch, so one plan serves launches on several streams.
// A merged batch is padded up to its bucket (power of two); the padding
// transforms compute on whatever the work buffer held and are never copied out.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "gb_plan.hpp"

using namespace gb;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device allocation (offsets 256-byte aligned).
struct Pool {
  char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length

  bool init(size_t bytes) {
    size = bytes;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      return false;
    }
    free_[0] = bytes;
    return true;
  }
  void destroy() {
    if (base) cudaFree(base);
    base = nullptr;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Request {
  uint64_t ticket = 0;
  int rank = 1;
  int64_t n[3] = {1, 1, 1};
  int64_t batch = 1;
  int sign = -1;
  const void* hin = nullptr;
  void* hout = nullptr;
  int64_t points = 0;  // per transform
  std::string key;     // rank, extents and sign (requests that may merge)
  double arrival = 0, done = 0;
  int state = 0;       // 0 waiting, 1 running, 2 done, 3 failed
  int status = FFT_OK;
};

struct Launch {
  std::vector<Request*> reqs;
  int stream = 0;
  cudaEvent_t ev_in = nullptr, ev_fft = nullptr;  // inputs copied; transform done
  cudaEvent_t ev = nullptr;                        // outputs copied (completion)
  size_t off = 0, bytes = 0;
};

std::string shape_key(const Request& r) {
  std::ostringstream o;
  o << r.rank << ":" << r.n[0] << "x" << r.n[1] << "x" << r.n[2] << ":" << r.sign;
  return o.str();
}

int64_t bucket_of(int64_t b) {
  int64_t p = 1;
  while (p < b) p <<= 1;
  return p;
}

}  // namespace

struct fft_server_s {
  size_t budget = 0;
  int nstreams = 1;
  int depth = 4;  // launches in flight per compute stream
  std::vector<cudaStream_t> streams;  // compute streams
  cudaStream_t cin = nullptr, cout = nullptr;  // copy-in and copy-out queues
  std::vector<int> busy;
  Pool pool;
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<Request*> waiting;
  std::map<uint64_t, Request*> reqs;
  std::vector<Launch*> inflight;
  std::map<std::string, fft_plan> plans;
  uint64_t next_ticket = 1;
  double t0 = 0;
  bool stop = false;
  std::thread worker;
  int64_t max_merge_points = (int64_t)1 << 27;
  // statistics
  std::vector<double> lat;
  uint64_t n_done = 0, n_failed = 0, n_launches = 0, n_merged = 0, n_rejected = 0;
  double flops = 0, bytes_alg = 0;
  size_t hwm = 0, in_use = 0;
  double first_arrival = -1, last_done = 0;
  int device = 0;
  // why the head of the queue last waited: 0 not waiting, 1 stream slots, 2 memory
  int blocked = 0;
  double stall_slots = 0, stall_memory = 0;  // seconds the queue head waited, by reason

  fft_plan get_plan(const Request& r, int64_t bucket, int* err) {
    std::ostringstream k;
    k << r.key << ":" << bucket;
    auto it = plans.find(k.str());
    if (it != plans.end()) return it->second;
    fft_iodim d[3], h;
    int64_t st = 1;
    for (int i = r.rank - 1; i >= 0; --i) {
      d[i].n = r.n[i];
      d[i].is = d[i].os = st;
      st *= r.n[i];
    }
    h.n = bucket;
    h.is = h.os = st;
    fft_plan p = fft_plan_dft(r.rank, d, 1, &h, r.sign, FFT_ESTIMATE | FFT_EXTERNAL_SCRATCH);
    if (!p) {
      *err = fft_last_error();
      return nullptr;
    }
    plans[k.str()] = p;
    return p;
  }

  void retire_locked() {
    for (size_t i = 0; i < inflight.size();) {
      Launch* L = inflight[i];
      const cudaError_t q = cudaEventQuery(L->ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const double t = now_s() - t0;
      for (Request* r : L->reqs) {
        // a launch step that failed at submission keeps its code
        const bool ok = q == cudaSuccess && r->status == FFT_OK;
        r->state = ok ? 2 : 3;
        if (q != cudaSuccess && r->status == FFT_OK) r->status = FFT_ERR_CUDA;
        r->done = t;
        if (ok) {
          ++n_done;
          lat.push_back(r->done - r->arrival);
          flops += 5.0 * r->points * std::log2((double)std::max<int64_t>(2, r->points)) * r->batch;
          bytes_alg += 16.0 * r->points * r->batch;
          last_done = std::max(last_done, t);
        } else {
          ++n_failed;
        }
      }
      if (q != cudaSuccess) cudaGetLastError();
      pool.release(L->off, L->bytes);
      in_use -= (L->bytes + 255) & ~(size_t)255;
      busy[L->stream]--;
      for (cudaEvent_t e : {L->ev_in, L->ev_fft, L->ev})
        if (e) cudaEventDestroy(e);
      delete L;
      inflight.erase(inflight.begin() + i);
      cv_done.notify_all();
    }
  }

  // admit as many launches as budget and stream slots allow; returns the count
  int admit_locked() {
    int admitted = 0;
    blocked = 0;
    while (!waiting.empty()) {
      int s = -1;
      for (int i = 0; i < nstreams; ++i)
        if (busy[i] < depth && (s < 0 || busy[i] < busy[s])) s = i;
      if (s < 0) {
        blocked = 1;
        break;
      }
      Request* r = waiting.front();
      const std::string& key = r->key;
      // merge the waiting requests of the same shape and sign (arrival order kept)
      std::vector<Request*> group{r};
      int64_t total = r->batch;
      for (size_t i = 1; i < waiting.size() && i < 256; ++i) {
        Request* q = waiting[i];
        if (q->key == key && (total + q->batch) * r->points <= max_merge_points) {
          group.push_back(q);
          total += q->batch;
        }
      }
      // a merged launch takes at most its input, output and (bounded by twice
      // the data) scratch; drop merged requests until that fits what is free
      auto bound = [&](int64_t b) { return (size_t)bucket_of(b) * r->points * 8 * 4; };
      while (group.size() > 1 && in_use + bound(total) > budget) {
        total -= group.back()->batch;
        group.pop_back();
      }
      fft_plan p = nullptr;
      size_t data = 0, scratch = 0, need = 0;
      int err = FFT_OK;
      for (;;) {
        p = get_plan(*r, bucket_of(total), &err);
        if (!p) break;
        data = (size_t)bucket_of(total) * r->points * 8;
        scratch = fft_plan_scratch_bytes(p);
        need = ((data + 255) & ~(size_t)255) * 2 + scratch;
        if (need <= budget || group.size() == 1) break;
        group.resize(1);  // merged launch too large: the head request alone
        total = r->batch;
      }
      if (!p) {
        r->state = 3;
        r->status = err;
        ++n_failed;
        waiting.pop_front();
        cv_done.notify_all();
        continue;
      }
      if (need > budget) {
        r->state = 3;
        r->status = FFT_ERR_BUDGET;
        ++n_rejected;
        waiting.pop_front();
        cv_done.notify_all();
        continue;
      }
      size_t off = 0;
      if (in_use + need > budget || !pool.alloc(need, &off)) {  // wait for memory
        blocked = 2;
        break;
      }
      in_use += (need + 255) & ~(size_t)255;
      hwm = std::max(hwm, in_use);
      Launch* L = new Launch;
      L->reqs = group;
      L->stream = s;
      L->off = off;
      L->bytes = need;
      char* din = pool.base + off;
      char* dout = din + ((data + 255) & ~(size_t)255);
      char* dscr = dout + ((data + 255) & ~(size_t)255);
      cudaStream_t st = streams[s];
      int rc = FFT_OK;
      if (cudaEventCreateWithFlags(&L->ev_in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&L->ev_fft, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&L->ev, cudaEventDisableTiming) != cudaSuccess)
        rc = FFT_ERR_CUDA;
      size_t pos = 0;
      for (Request* q : group) {
        const size_t b = (size_t)q->batch * q->points * 8;
        if (rc == FFT_OK && cudaMemcpyAsync(din + pos, q->hin, b, cudaMemcpyHostToDevice, cin) != cudaSuccess)
          rc = FFT_ERR_CUDA;
        pos += b;
      }
      if (rc == FFT_OK && (cudaEventRecord(L->ev_in, cin) != cudaSuccess ||
                           cudaStreamWaitEvent(st, L->ev_in, 0) != cudaSuccess))
        rc = FFT_ERR_CUDA;
      if (rc == FFT_OK) rc = fft_execute_scratch(p, din, dout, scratch ? dscr : nullptr, st);
      if (rc == FFT_OK && (cudaEventRecord(L->ev_fft, st) != cudaSuccess ||
                           cudaStreamWaitEvent(cout, L->ev_fft, 0) != cudaSuccess))
        rc = FFT_ERR_CUDA;
      pos = 0;
      for (Request* q : group) {
        const size_t b = (size_t)q->batch * q->points * 8;
        if (rc == FFT_OK && cudaMemcpyAsync(q->hout, dout + pos, b, cudaMemcpyDeviceToHost, cout) != cudaSuccess)
          rc = FFT_ERR_CUDA;
        pos += b;
      }
      // completion: after the copy-out queue, and after every stream that may
      // still touch the buffers when an earlier step failed
      if (L->ev) {
        if (rc != FFT_OK) {
          cudaGetLastError();
          if (L->ev_in && cudaEventRecord(L->ev_in, cin) == cudaSuccess) cudaStreamWaitEvent(cout, L->ev_in, 0);
          if (L->ev_fft && cudaEventRecord(L->ev_fft, st) == cudaSuccess) cudaStreamWaitEvent(cout, L->ev_fft, 0);
        }
        cudaEventRecord(L->ev, cout);
      }
      for (Request* q : group) {
        q->state = 1;
        if (rc != FFT_OK) q->status = rc;
      }
      // remove the group from the waiting queue
      std::set<Request*> in(group.begin(), group.end());
      std::deque<Request*> rest;
      for (Request* q : waiting)
        if (!in.count(q)) rest.push_back(q);
      waiting.swap(rest);
      busy[s]++;
      inflight.push_back(L);
      ++n_launches;
      if (group.size() > 1) n_merged += group.size() - 1;
      ++admitted;
    }
    return admitted;
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    double last = now_s();
    while (true) {
      retire_locked();
      admit_locked();
      if (stop && waiting.empty() && inflight.empty()) break;
      const int why = waiting.empty() ? 0 : blocked;
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(inflight.empty() && waiting.empty() ? 200 : 20));
      lk.lock();
      const double t = now_s();
      if (why == 1) stall_slots += t - last;
      if (why == 2) stall_memory += t - last;
      last = t;
    }
  }
};

extern "C" fft_server fft_server_create(size_t budget_bytes, int nstreams, unsigned flags) {
  if (budget_bytes < 4096 || nstreams < 1 || nstreams > 64 || flags != 0) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  fft_server s = new (std::nothrow) fft_server_s;
  if (!s) {
    set_err(FFT_ERR_OOM);
    return nullptr;
  }
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    set_err(FFT_ERR_NO_DEVICE);
    return nullptr;
  }
  s->budget = budget_bytes;
  s->nstreams = nstreams;
  s->busy.assign(nstreams, 0);
  if (!s->pool.init(budget_bytes)) {
    delete s;
    set_err(FFT_ERR_OOM);
    return nullptr;
  }
  for (int i = 0; i < nstreams + 2; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      if (s->cin) cudaStreamDestroy(s->cin);
      s->pool.destroy();
      delete s;
      set_err(FFT_ERR_CUDA);
      return nullptr;
    }
    if (i < nstreams)
      s->streams.push_back(st);
    else if (!s->cin)
      s->cin = st;
    else
      s->cout = st;
  }
  s->t0 = now_s();
  s->worker = std::thread([s] { s->loop(); });
  set_err(FFT_OK);
  return s;
}

extern "C" double fft_server_now(fft_server s) { return s ? now_s() - s->t0 : 0.0; }

extern "C" int fft_server_submit(fft_server s, int rank, const int64_t* n, int64_t batch, int sign,
                                 const void* host_in, void* host_out, double arrival, uint64_t* ticket) {
  if (!s || rank < 1 || rank > 3 || !n || batch < 1 || (sign != -1 && sign != 1) || !host_in || !host_out ||
      !ticket)
    return set_err(FFT_ERR_INVALID_ARG);
  Request* r = new (std::nothrow) Request;
  if (!r) return set_err(FFT_ERR_OOM);
  r->rank = rank;
  r->points = 1;
  for (int i = 0; i < rank; ++i) {
    if (n[i] < 1) {
      delete r;
      return set_err(FFT_ERR_INVALID_ARG);
    }
    r->n[i] = n[i];
    r->points *= n[i];
  }
  r->batch = batch;
  r->sign = sign;
  r->key = shape_key(*r);
  r->hin = host_in;
  r->hout = host_out;
  std::lock_guard<std::mutex> g(s->mu);
  r->arrival = arrival >= 0 ? arrival : now_s() - s->t0;
  if (s->first_arrival < 0 || r->arrival < s->first_arrival) s->first_arrival = r->arrival;
  r->ticket = s->next_ticket++;
  s->reqs[r->ticket] = r;
  s->waiting.push_back(r);
  *ticket = r->ticket;
  return set_err(FFT_OK);
}

// FFT_OK: done; 1: still queued or running; an error code: failed or unknown ticket
extern "C" int fft_server_poll(fft_server s, uint64_t ticket) {
  if (!s) return FFT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FFT_ERR_INVALID_ARG;
  const Request* r = it->second;
  if (r->state == 2) return r->status;
  if (r->state == 3) return r->status != FFT_OK ? r->status : FFT_ERR_CUDA;
  return 1;
}

extern "C" int fft_server_wait(fft_server s, uint64_t ticket, double timeout_s) {
  if (!s) return FFT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FFT_ERR_INVALID_ARG;
  Request* r = it->second;
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state < 2) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && r->state < 2) return 1;
  }
  return r->state == 2 ? r->status : (r->status != FFT_OK ? r->status : FFT_ERR_CUDA);
}

extern "C" int fft_server_drain(fft_server s, double timeout_s) {
  if (!s) return FFT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (!s->waiting.empty() || !s->inflight.empty()) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
        (!s->waiting.empty() || !s->inflight.empty()))
      return 1;
  }
  return FFT_OK;
}

static double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p * (double)(v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

extern "C" int fft_server_stats(fft_server s, char* buf, size_t len) {
  if (!s) return -1;
  std::ostringstream o;
  {
    std::lock_guard<std::mutex> g(s->mu);
    const double span = s->last_done - std::max(0.0, s->first_arrival);
    o.setf(std::ios::fixed);
    o.precision(6);
    o << "{\"completed\": " << s->n_done << ", \"failed\": " << s->n_failed << ", \"rejected\": " << s->n_rejected
      << ", \"waiting\": " << s->waiting.size() << ", \"in_flight_launches\": " << s->inflight.size()
      << ", \"launches\": " << s->n_launches << ", \"merged_requests\": " << s->n_merged
      << ", \"p50_latency_s\": " << percentile(s->lat, 0.50) << ", \"p99_latency_s\": " << percentile(s->lat, 0.99)
      << ", \"mean_latency_s\": "
      << (s->lat.empty() ? 0.0 : [&] { double a = 0; for (double x : s->lat) a += x; return a / s->lat.size(); }())
      << ", \"span_s\": " << span << ", \"gflops\": " << (span > 0 ? s->flops / span / 1e9 : 0.0)
      << ", \"gbs_algorithmic\": " << (span > 0 ? s->bytes_alg / span / 1e9 : 0.0)
      << ", \"requests_per_s\": " << (span > 0 ? s->n_done / span : 0.0) << ", \"budget_bytes\": " << s->budget
      << ", \"budget_high_water_bytes\": " << s->hwm << ", \"cached_plans\": " << s->plans.size()
      << ", \"streams\": " << s->nstreams << ", \"stall_slots_s\": " << s->stall_slots
      << ", \"stall_memory_s\": " << s->stall_memory << "}";
  }
  const std::string str = o.str();
  if (buf && len > 0) {
    const size_t k = std::min(len - 1, str.size());
    memcpy(buf, str.data(), k);
    buf[k] = '\0';
  }
  return (int)str.size();
}

extern "C" void fft_server_destroy(fft_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  cudaStreamSynchronize(s->cin);
  cudaStreamSynchronize(s->cout);
  for (auto& kv : s->plans) fft_destroy(kv.second);
  for (auto& kv : s->reqs) delete kv.second;
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  cudaStreamDestroy(s->cin);
  cudaStreamDestroy(s->cout);
  s->pool.destroy();
  delete s;
}
