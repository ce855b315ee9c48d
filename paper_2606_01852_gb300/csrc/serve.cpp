// Serving loop: continuous admission of contraction requests.
//
// A request names a plan and carries host inputs. The scheduler thread admits queued
// requests in arrival order whenever an in-flight slot is free and the device
// workspace the request needs fits the HBM budget; admitted requests run
// concurrently on a ring of CUDA streams, so requests that arrive while others are
// on the GPU start as soon as resources free up. Each plan keeps a pool of resident
// device instances (its workspace plus pinned staging), reused across requests.
#include <atomic>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "tn_internal.h"

namespace tn {
namespace {

struct Instance {
  Plan P;                 // copy of the template plan with its own workspace
  char* pinned_in = nullptr;
  char* pinned_out = nullptr;
  int64_t in_bytes = 0, out_bytes = 0;
  std::vector<int64_t> in_off;  // per leaf offset in pinned_in
  bool busy = false;
  uint64_t last_used = 0;       // admission tick of the last request it ran
};

struct PlanPool {
  std::vector<std::unique_ptr<Instance>> inst;
};

enum class RState { Queued, Running, Done };

struct Request {
  uint64_t id = 0;
  tn_plan_s* plan = nullptr;
  std::vector<char> inputs;       // concatenated host copies of the leaves
  std::vector<int64_t> in_off;
  RState state = RState::Queued;
  Instance* inst = nullptr;
  int stream = 0;
  cudaEvent_t done = nullptr;
  std::vector<char> result;
  double log_scale = 0.0;
  tn_status status = TN_OK;
  std::string err;
};

int64_t leaf_bytes(const Plan& P, int32_t t) {
  int64_t full = 1;
  for (int32_t x : P.tensors[t].decl) full *= P.extent[x];
  return full * elem_bytes(P);
}

}  // namespace
}  // namespace tn

using namespace tn;

struct tn_server_s {
  tn_serve_config cfg{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::map<uint64_t, PlanPool> pools;  // by plan uid
  std::vector<Request*> running;
  int64_t hbm_in_use = 0;        // device bytes held by resident instances (busy or idle)
  uint64_t tick = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread thr;

  static void release(Instance& in) {
    if (in.P.dev) cudaFree(in.P.dev);
    if (in.pinned_in) cudaFreeHost(in.pinned_in);
    if (in.pinned_out) cudaFreeHost(in.pinned_out);
    in.P.dev = nullptr;
    in.pinned_in = in.pinned_out = nullptr;
  }

  // Free idle instances (of any plan), least recently used first, until `need` more bytes
  // fit the budget or no idle instance is left.
  void evict_idle(int64_t need) {
    while (hbm_in_use + need > cfg.hbm_budget_bytes) {
      PlanPool* best_pool = nullptr;
      size_t best_i = 0;
      uint64_t best_tick = UINT64_MAX;
      for (auto& kv : pools)
        for (size_t i = 0; i < kv.second.inst.size(); ++i) {
          const Instance& in = *kv.second.inst[i];
          if (!in.busy && in.last_used < best_tick) {
            best_tick = in.last_used;
            best_pool = &kv.second;
            best_i = i;
          }
        }
      if (!best_pool) return;
      Instance& victim = *best_pool->inst[best_i];
      hbm_in_use -= victim.P.total_bytes;
      release(victim);
      best_pool->inst.erase(best_pool->inst.begin() + (std::ptrdiff_t)best_i);
    }
  }

  // Find or create an idle instance of `plan`; nullptr if the budget forbids it for now.
  // The budget bounds the device memory held by resident instances: idle instances of
  // other plans are freed (least recently used first) to make room before a request waits.
  Instance* acquire(tn_plan_s* plan, std::string& err, bool& fatal) {
    fatal = false;
    PlanPool& pool = pools[plan->P.uid];
    for (auto& in : pool.inst)
      if (!in->busy) return in.get();
    const int64_t need = plan->P.total_bytes;
    if (cfg.hbm_budget_bytes > 0 && hbm_in_use + need > cfg.hbm_budget_bytes) evict_idle(need);
    if (cfg.hbm_budget_bytes > 0 && hbm_in_use + need > cfg.hbm_budget_bytes) {
      if (running.empty()) {
        err = "request workspace exceeds the serve HBM budget";
        fatal = true;
      }
      return nullptr;
    }
    auto in = std::make_unique<Instance>();
    in->P = plan->P;
    in->P.dev = nullptr;
    void* mem = nullptr;
    if (cudaMalloc(&mem, (size_t)need) != cudaSuccess) {
      cudaGetLastError();
      if (running.empty()) {
        err = "cudaMalloc of a request workspace failed";
        fatal = true;
      }
      return nullptr;
    }
    in->P.dev = static_cast<char*>(mem);
    in->in_off.resize(in->P.n_leaves);
    for (int32_t t = 0; t < in->P.n_leaves; ++t) {
      in->in_off[t] = in->in_bytes;
      in->in_bytes += (leaf_bytes(in->P, t) + 255) / 256 * 256;
    }
    in->out_bytes = in->P.out_elems * (in->P.is_complex ? 16 : 8) + 16;
    void* pi = nullptr;
    void* po = nullptr;
    if (cudaMallocHost(&pi, (size_t)in->in_bytes) != cudaSuccess ||
        cudaMallocHost(&po, (size_t)in->out_bytes) != cudaSuccess) {
      cudaGetLastError();
      if (pi) cudaFreeHost(pi);
      cudaFree(mem);
      err = "pinned staging allocation failed";
      fatal = true;
      return nullptr;
    }
    in->pinned_in = static_cast<char*>(pi);
    in->pinned_out = static_cast<char*>(po);
    hbm_in_use += need;
    pool.inst.push_back(std::move(in));
    return pool.inst.back().get();
  }

  // Launch an admitted request (called with the lock held; launches are async).
  void launch(Request* r) {
    Instance* in = r->inst;
    Plan& P = in->P;
    cudaStream_t st = streams[r->stream];
    std::vector<const void*> dptr(P.n_leaves);
    for (int32_t t = 0; t < P.n_leaves; ++t) {
      const int64_t nb = leaf_bytes(P, t);
      std::memcpy(in->pinned_in + in->in_off[t], r->inputs.data() + r->in_off[t], (size_t)nb);
      char* d = P.dev + P.stage_in_off[t];
      cudaMemcpyAsync(d, in->pinned_in + in->in_off[t], nb, cudaMemcpyHostToDevice, st);
      dptr[t] = d;
    }
    char* dout = P.dev + P.total_bytes - ((P.out_elems * 16 + 16 + 255) / 256 * 256);
    double* dls = reinterpret_cast<double*>(dout + P.out_elems * 16);
    std::string err;
    tn_status s = run_slices(P, dptr.data(), 0, P.n_slices, dout, dls, st, err);
    if (s == TN_OK) {
      const int64_t ob = P.out_elems * (P.is_complex ? 16 : 8);
      cudaMemcpyAsync(in->pinned_out, dout, ob, cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(in->pinned_out + ob, dls, sizeof(double), cudaMemcpyDeviceToHost, st);
      cudaEventRecord(r->done, st);
    }
    r->status = s;
    r->err = err;
    r->state = RState::Running;
  }

  void finish(Request* r) {
    Instance* in = r->inst;
    if (r->status == TN_OK) {
      cudaError_t e = cudaEventSynchronize(r->done);
      if (e != cudaSuccess) {
        r->status = TN_ERR_CUDA;
        r->err = cudaGetErrorString(e);
      } else {
        const int64_t ob = in->P.out_elems * (in->P.is_complex ? 16 : 8);
        r->result.assign(in->pinned_out, in->pinned_out + ob);
        std::memcpy(&r->log_scale, in->pinned_out + ob, sizeof(double));
      }
    }
    in->busy = false;
    r->inst = nullptr;
    r->state = RState::Done;
    r->inputs.clear();
    r->inputs.shrink_to_fit();
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progressed = false;
      // retire finished requests
      for (size_t i = 0; i < running.size();) {
        Request* r = running[i];
        if (r->status != TN_OK || cudaEventQuery(r->done) != cudaErrorNotReady) {
          finish(r);
          running[i] = running.back();
          running.pop_back();
          progressed = true;
        } else {
          ++i;
        }
      }
      if (progressed) cv_done.notify_all();
      // admit in arrival order while slots and memory allow
      while (!queue.empty() && (int)running.size() < cfg.max_inflight) {
        Request* r = reqs[queue.front()].get();
        std::string err;
        bool fatal = false;
        Instance* in = acquire(r->plan, err, fatal);
        if (!in) {
          if (fatal) {
            queue.pop_front();
            r->status = TN_ERR_OOM;
            r->err = err;
            r->state = RState::Done;
            cv_done.notify_all();
            continue;
          }
          break;  // wait for a running request to release memory
        }
        queue.pop_front();
        in->busy = true;
        in->last_used = ++tick;
        r->inst = in;
        r->stream = next_stream;
        next_stream = (next_stream + 1) % (int)streams.size();
        launch(r);
        running.push_back(r);
        progressed = true;
      }
      if (stop && queue.empty() && running.empty()) break;
      if (running.empty() && queue.empty()) {
        cv_work.wait(lk);
      } else if (!progressed) {
        // in-flight work: poll completions without holding the lock
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
};

extern "C" {

tn_status tn_serve_create(const tn_serve_config* cfg, tn_server_t* out) {
  if (!cfg || !out || cfg->max_inflight <= 0 || cfg->n_streams <= 0 || cfg->queue_capacity <= 0) {
    set_error("bad serve config");
    return TN_ERR_INVALID;
  }
  auto* s = new tn_server_s();
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    set_error("no CUDA device");
    return TN_ERR_CUDA;
  }
  for (int i = 0; i < cfg->n_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      set_error("stream creation failed");
      return TN_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  s->thr = std::thread([s] { s->loop(); });
  *out = s;
  return TN_OK;
}

tn_status tn_serve_submit(tn_server_t srv, tn_plan_t plan, const void* const* host_inputs,
                          uint64_t* ticket) {
  if (!srv || !plan || !host_inputs || !ticket) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  if (!plan->P.dev) {
    set_error("plan was built with TN_PLAN_HOST_ONLY");
    return TN_ERR_INVALID;
  }
  auto r = std::make_unique<Request>();
  r->plan = plan;
  int64_t tot = 0;
  r->in_off.resize(plan->P.n_leaves);
  for (int32_t t = 0; t < plan->P.n_leaves; ++t) {
    if (!host_inputs[t]) {
      set_error("null input pointer");
      return TN_ERR_INVALID;
    }
    r->in_off[t] = tot;
    tot += leaf_bytes(plan->P, t);
  }
  r->inputs.resize((size_t)tot);
  for (int32_t t = 0; t < plan->P.n_leaves; ++t)
    std::memcpy(r->inputs.data() + r->in_off[t], host_inputs[t], (size_t)leaf_bytes(plan->P, t));
  if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
    set_error("event creation failed");
    return TN_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(srv->mu);
  if ((int)srv->queue.size() >= srv->cfg.queue_capacity) {
    cudaEventDestroy(r->done);
    set_error("serve queue full");
    return TN_ERR_BUSY;
  }
  r->id = srv->next_id++;
  *ticket = r->id;
  srv->queue.push_back(r->id);
  srv->reqs[r->id] = std::move(r);
  srv->cv_work.notify_one();
  return TN_OK;
}

tn_status tn_serve_poll(tn_server_t srv, uint64_t ticket, void* result, double* log_scale,
                        int32_t timeout_us) {
  if (!srv) {
    set_error("null server");
    return TN_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) {
    set_error("unknown ticket");
    return TN_ERR_INVALID;
  }
  Request* r = it->second.get();
  auto ready = [&] { return r->state == RState::Done; };
  if (!ready()) {
    if (timeout_us == 0) return TN_ERR_NOT_READY;
    if (timeout_us < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
      return TN_ERR_NOT_READY;
  }
  tn_status s = r->status;
  if (s == TN_OK) {
    if (result) std::memcpy(result, r->result.data(), r->result.size());
    if (log_scale) *log_scale = r->log_scale;
  } else {
    set_error(r->err);
  }
  cudaEventDestroy(r->done);
  srv->reqs.erase(it);
  return s;
}

tn_status tn_serve_destroy(tn_server_t srv) {
  if (!srv) return TN_OK;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
    srv->cv_work.notify_all();
  }
  srv->thr.join();
  for (auto& kv : srv->pools)
    for (auto& in : kv.second.inst) tn_server_s::release(*in);
  for (auto& kv : srv->reqs)
    if (kv.second->done) cudaEventDestroy(kv.second->done);
  for (auto st : srv->streams) cudaStreamDestroy(st);
  delete srv;
  return TN_OK;
}

}  // extern "C"
