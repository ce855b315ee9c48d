// Serving loop: continuous admission of contraction requests.
//
// A request names a plan and carries host inputs. The scheduler thread admits queued
// requests in arrival order whenever an in-flight slot is free and the device
// workspace the request needs fits the HBM budget; admitted requests run
// concurrently on a ring of CUDA streams, so requests that arrive while others are
// on the GPU start as soon as resources free up. Each plan keeps a pool of resident
// device instances (its workspace plus pinned staging), reused across requests.
//
// Packing (tn_serve_config.pack_max > 0): requests on small closed unsliced plans whose
// steps all run on the CUDA cores share one launch of the batched small-network kernel
// (batch.cu; one CTA per request). The admission step takes the queue's first request and
// every later queued request of the same arithmetic kind, up to pack_max, concatenates the
// plans' per-network tables (computed once per plan) and the requests' inputs into one
// pinned buffer, copies it to a resident device buffer, launches the kernel, and copies the
// values and log scales back; the pack holds one in-flight slot.
#include <algorithm>
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

#include "batch.h"
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

// Device and pinned buffers of one packed launch, reused by later packs.
struct PackBuf {
  char* dev = nullptr;
  char* pin = nullptr;
  size_t dev_bytes = 0, pin_bytes = 0;
  bool busy = false;
};

// The batched kernel's tables of a plan (computed once), or why it cannot be packed.
struct PackTemplate {
  bool ok = false;
  BatchTemplate T;
  int kind = 0;  // 1 complex, 2 real, 3 real with scaling, 4 max-plus
};

struct Request;

struct Pack {
  std::vector<Request*> reqs;
  PackBuf* buf = nullptr;
  cudaEvent_t done = nullptr;
  size_t out_off = 0;   // values then logs, in the pinned buffer
  bool cplx = false;
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
  Pack* pack = nullptr;           // set while it runs in a packed launch
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
  std::vector<Pack*> running_packs;
  std::map<uint64_t, PackTemplate> templates;  // by plan uid
  std::vector<std::unique_ptr<PackBuf>> packbufs;
  int num_sms = 148;
  int64_t hbm_in_use = 0;        // device bytes held by resident instances and pack buffers
  tn_serve_stats stats{};
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
      if (!best_pool) {
        // then idle pack buffers
        for (size_t i = 0; i < packbufs.size(); ++i)
          if (!packbufs[i]->busy) {
            hbm_in_use -= (int64_t)packbufs[i]->dev_bytes;
            release_packbuf(*packbufs[i]);
            packbufs.erase(packbufs.begin() + (std::ptrdiff_t)i);
            break;
          }
        bool any_idle = false;
        for (auto& pb : packbufs) any_idle = any_idle || !pb->busy;
        if (hbm_in_use + need > cfg.hbm_budget_bytes && !any_idle) return;
        continue;
      }
      Instance& victim = *best_pool->inst[best_i];
      hbm_in_use -= victim.P.total_bytes;
      release(victim);
      best_pool->inst.erase(best_pool->inst.begin() + (std::ptrdiff_t)best_i);
    }
  }

  static void release_packbuf(PackBuf& b) {
    if (b.dev) cudaFree(b.dev);
    if (b.pin) cudaFreeHost(b.pin);
    b.dev = b.pin = nullptr;
  }

  // The batched-kernel tables of `plan` (built on first use).
  const PackTemplate& pack_template(tn_plan_s* plan) {
    auto it = templates.find(plan->P.uid);
    if (it != templates.end()) return it->second;
    PackTemplate pt;
    const Plan& P = plan->P;
    const bool simt_only = std::all_of(P.steps.begin(), P.steps.end(),
                                       [](const StepRec& st) { return st.cls != TN_CLASS_TC; });
    std::string why;
    if (simt_only && P.batch == 1 && batch_template(P, pt.T, why)) {
      pt.ok = true;
      const bool maxplus = P.policy.semiring == TN_SEMIRING_MAXPLUS;
      pt.kind = P.is_complex ? 1 : (maxplus ? 4 : (P.policy.exp_scaling ? 3 : 2));
      if (P.is_complex && P.policy.exp_scaling) pt.ok = false;  // the complex batched kernel is unscaled
    }
    return templates.emplace(P.uid, std::move(pt)).first->second;
  }

  // A free pack buffer of at least the given sizes (freeing a smaller idle one, under the
  // budget); nullptr if the budget forbids it for now, with `fatal` if it never will.
  PackBuf* acquire_packbuf(size_t dev_bytes, size_t pin_bytes, std::string& err, bool& fatal) {
    fatal = false;
    for (auto& b : packbufs)
      if (!b->busy && b->dev_bytes >= dev_bytes && b->pin_bytes >= pin_bytes) return b.get();
    for (size_t i = 0; i < packbufs.size(); ++i)
      if (!packbufs[i]->busy) {  // too small: give its memory back
        hbm_in_use -= (int64_t)packbufs[i]->dev_bytes;
        release_packbuf(*packbufs[i]);
        packbufs.erase(packbufs.begin() + (std::ptrdiff_t)i);
        --i;
      }
    if (cfg.hbm_budget_bytes > 0 && hbm_in_use + (int64_t)dev_bytes > cfg.hbm_budget_bytes) evict_idle((int64_t)dev_bytes);
    if (cfg.hbm_budget_bytes > 0 && hbm_in_use + (int64_t)dev_bytes > cfg.hbm_budget_bytes) {
      if (running.empty() && running_packs.empty()) {
        err = "a packed launch exceeds the serve HBM budget";
        fatal = true;
      }
      return nullptr;
    }
    auto b = std::make_unique<PackBuf>();
    if (cudaMalloc(&b->dev, dev_bytes) != cudaSuccess || cudaMallocHost(&b->pin, pin_bytes) != cudaSuccess) {
      cudaGetLastError();
      release_packbuf(*b);
      if (running.empty() && running_packs.empty()) {
        err = "allocation of a pack buffer failed";
        fatal = true;
      }
      return nullptr;
    }
    b->dev_bytes = dev_bytes;
    b->pin_bytes = pin_bytes;
    hbm_in_use += (int64_t)dev_bytes;
    packbufs.push_back(std::move(b));
    return packbufs.back().get();
  }

  // Launch `group` (requests of one kind) as one batched-kernel launch; false if the
  // buffers are not available yet (the requests stay queued), fatal errors retire them.
  bool launch_pack(const std::vector<Request*>& group, bool& fatal, std::string& err) {
    const PackTemplate& first = pack_template(group[0]->plan);
    const bool cplx = first.kind == 1;
    const size_t eb = cplx ? 8 : 4;
    std::vector<BNet> nets;
    std::vector<BLeaf> leaves;
    std::vector<BStep> steps;
    int64_t arena = 0, in_elems = 0;
    int32_t tab_ints = 0;
    for (Request* r : group) {
      const PackTemplate& pt = pack_template(r->plan);
      tab_ints = std::max(tab_ints, std::min(pt.T.max_tab, kMaxTabInts));
      BNet bn{};
      bn.arena = arena;
      bn.leaf0 = (int32_t)leaves.size();
      bn.n_leaves = (int32_t)pt.T.leaves.size();
      bn.step0 = (int32_t)steps.size();
      bn.n_steps = (int32_t)pt.T.steps.size();
      bn.root = pt.T.root;
      bn.root_size = pt.T.root_size;
      bn.arena_floats = static_cast<int32_t>(pt.T.arena_floats);
      for (BLeaf L : pt.T.leaves) {
        L.src += in_elems;
        leaves.push_back(L);
      }
      steps.insert(steps.end(), pt.T.steps.begin(), pt.T.steps.end());
      in_elems += pt.T.input_elems;
      arena += pt.T.arena_floats;
      nets.push_back(bn);
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t n = group.size();
    const size_t b_nets = al(sizeof(BNet) * n), b_leaves = al(sizeof(BLeaf) * leaves.size());
    const size_t b_steps = al(sizeof(BStep) * std::max<size_t>(1, steps.size()));
    const size_t b_in = al(eb * (size_t)in_elems), b_out = al(sizeof(double) * 3 * n);
    const size_t up = b_nets + b_leaves + b_steps + b_in;            // copied to the device
    const size_t dev_bytes = up + al(sizeof(float) * (size_t)arena) + b_out + 256;
    const size_t pin_bytes = up + b_out;
    PackBuf* buf = acquire_packbuf(dev_bytes, pin_bytes, err, fatal);
    if (!buf) return false;
    char* h = buf->pin;
    std::memcpy(h, nets.data(), sizeof(BNet) * n);
    std::memcpy(h + b_nets, leaves.data(), sizeof(BLeaf) * leaves.size());
    if (!steps.empty()) std::memcpy(h + b_nets + b_leaves, steps.data(), sizeof(BStep) * steps.size());
    size_t pos = b_nets + b_leaves + b_steps;
    for (Request* r : group) {
      std::memcpy(h + pos, r->inputs.data(), r->inputs.size());
      pos += r->inputs.size();
    }
    char* d = buf->dev;
    const size_t off_arena = up, off_out = up + al(sizeof(float) * (size_t)arena), off_q = off_out + b_out;
    cudaStream_t st = streams[next_stream];
    next_stream = (next_stream + 1) % (int)streams.size();
    auto* pk = new Pack();
    pk->reqs = group;
    pk->buf = buf;
    pk->cplx = cplx;
    pk->out_off = up;
    cudaError_t e = cudaEventCreateWithFlags(&pk->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h, up, cudaMemcpyHostToDevice, st);
    const int threads = 128;
    const int grid = (int)std::min<size_t>(n, (size_t)num_sms * 4);
    double* vals = reinterpret_cast<double*>(d + off_out);
    double* logs = vals + 2 * n;
    if (e == cudaSuccess)
      e = launch_batch_kernel(reinterpret_cast<BNet*>(d), reinterpret_cast<BLeaf*>(d + b_nets),
                              reinterpret_cast<BStep*>(d + b_nets + b_leaves), (int32_t)n,
                              d + b_nets + b_leaves + b_steps, reinterpret_cast<float*>(d + off_arena),
                              reinterpret_cast<int32_t*>(d + off_q), cplx, first.kind == 3, first.kind == 4,
                              threads, grid, vals, logs, st, false, 0, tab_ints);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + up, d + off_out, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(pk->done, st);
    buf->busy = true;
    for (Request* r : group) {
      r->pack = pk;
      r->state = RState::Running;
      r->status = e == cudaSuccess ? TN_OK : TN_ERR_CUDA;
      if (e != cudaSuccess) r->err = std::string("packed launch: ") + cudaGetErrorString(e);
    }
    running_packs.push_back(pk);
    stats.packs += 1;
    stats.packed_requests += (int64_t)n;
    stats.max_pack = std::max<int64_t>(stats.max_pack, (int64_t)n);
    return true;
  }

  void finish_pack(Pack* pk) {
    cudaError_t e = pk->reqs.front()->status == TN_OK ? cudaEventSynchronize(pk->done) : cudaSuccess;
    const double* vals = reinterpret_cast<const double*>(pk->buf->pin + pk->out_off);
    const size_t n = pk->reqs.size();
    for (size_t i = 0; i < n; ++i) {
      Request* r = pk->reqs[i];
      if (r->status == TN_OK && e != cudaSuccess) {
        r->status = TN_ERR_CUDA;
        r->err = cudaGetErrorString(e);
      }
      if (r->status == TN_OK) {
        const size_t ob = pk->cplx ? 16 : 8;
        r->result.assign(reinterpret_cast<const char*>(vals + 2 * i), reinterpret_cast<const char*>(vals + 2 * i) + ob);
        r->log_scale = vals[2 * n + i];
      }
      r->pack = nullptr;
      r->state = RState::Done;
      stats.completed += 1;
      r->inputs.clear();
      r->inputs.shrink_to_fit();
    }
    pk->buf->busy = false;
    if (pk->done) cudaEventDestroy(pk->done);
    delete pk;
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
    if (upload_chain_table(in->P) != TN_OK) {
      cudaFree(mem);
      err = "writing a request workspace's step-chain table failed";
      fatal = true;
      return nullptr;
    }
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
    stats.completed += 1;
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
      for (size_t i = 0; i < running_packs.size();) {
        Pack* pk = running_packs[i];
        if (pk->reqs.front()->status != TN_OK || cudaEventQuery(pk->done) != cudaErrorNotReady) {
          finish_pack(pk);
          running_packs[i] = running_packs.back();
          running_packs.pop_back();
          progressed = true;
        } else {
          ++i;
        }
      }
      if (progressed) cv_done.notify_all();
      // admit in arrival order while slots and memory allow
      while (!queue.empty() && (int)(running.size() + running_packs.size()) < cfg.max_inflight) {
        Request* r = reqs[queue.front()].get();
        if (cfg.pack_max > 0 && pack_template(r->plan).ok) {
          // the first request and every later queued one of the same kind, up to pack_max
          const int kind = pack_template(r->plan).kind;
          std::vector<Request*> group;
          std::vector<size_t> idx;
          for (size_t i = 0; i < queue.size() && (int)group.size() < cfg.pack_max; ++i) {
            Request* q2 = reqs[queue[i]].get();
            const PackTemplate& pt = pack_template(q2->plan);
            if (pt.ok && pt.kind == kind) {
              group.push_back(q2);
              idx.push_back(i);
            }
          }
          bool fatal = false;
          std::string err;
          const bool launched = launch_pack(group, fatal, err);
          if (launched || fatal) {
            for (size_t k = idx.size(); k-- > 0;) queue.erase(queue.begin() + (std::ptrdiff_t)idx[k]);
          }
          if (fatal) {
            for (Request* q2 : group) {
              q2->status = TN_ERR_OOM;
              q2->err = err;
              q2->state = RState::Done;
            }
            cv_done.notify_all();
            continue;
          }
          if (!launched) break;  // wait for running work to release memory
          progressed = true;
          continue;
        }
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
        stats.plan_launches += 1;
        running.push_back(r);
        progressed = true;
      }
      if (stop && queue.empty() && running.empty() && running_packs.empty()) break;
      if (running.empty() && running_packs.empty() && queue.empty()) {
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
  if (cfg->pack_max < 0) {
    delete s;
    set_error("bad serve config: pack_max < 0");
    return TN_ERR_INVALID;
  }
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
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
  return tn_serve_submit_batch(srv, 1, &plan, &host_inputs, ticket);
}

tn_status tn_serve_submit_batch(tn_server_t srv, int32_t n, const tn_plan_t* plans,
                                const void* const* const* host_inputs, uint64_t* tickets) {
  if (!srv || n < 0 || (n > 0 && (!plans || !host_inputs || !tickets))) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  // copy every request's inputs before taking the lock; nothing is queued on an error
  std::vector<std::unique_ptr<Request>> made;
  made.reserve((size_t)n);
  auto drop = [&made]() {
    for (auto& r : made) cudaEventDestroy(r->done);
  };
  for (int32_t j = 0; j < n; ++j) {
    tn_plan_t plan = plans[j];
    const void* const* in = host_inputs[j];
    if (!plan || !in) {
      drop();
      set_error("null argument");
      return TN_ERR_INVALID;
    }
    if (!plan->P.dev) {
      drop();
      set_error("plan was built with TN_PLAN_HOST_ONLY");
      return TN_ERR_INVALID;
    }
    auto r = std::make_unique<Request>();
    r->plan = plan;
    int64_t tot = 0;
    r->in_off.resize(plan->P.n_leaves);
    for (int32_t t = 0; t < plan->P.n_leaves; ++t) {
      if (!in[t]) {
        drop();
        set_error("null input pointer");
        return TN_ERR_INVALID;
      }
      r->in_off[t] = tot;
      tot += leaf_bytes(plan->P, t);
    }
    r->inputs.resize((size_t)tot);
    for (int32_t t = 0; t < plan->P.n_leaves; ++t)
      std::memcpy(r->inputs.data() + r->in_off[t], in[t], (size_t)leaf_bytes(plan->P, t));
    if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
      drop();
      set_error("event creation failed");
      return TN_ERR_CUDA;
    }
    made.push_back(std::move(r));
  }
  std::lock_guard<std::mutex> g(srv->mu);
  if ((int64_t)srv->queue.size() + n > srv->cfg.queue_capacity) {
    drop();
    set_error("serve queue full");
    return TN_ERR_BUSY;
  }
  for (int32_t j = 0; j < n; ++j) {
    std::unique_ptr<Request>& r = made[(size_t)j];
    r->id = srv->next_id++;
    tickets[j] = r->id;
    srv->queue.push_back(r->id);
    srv->reqs[r->id] = std::move(r);
  }
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

tn_status tn_serve_stats_get(tn_server_t srv, tn_serve_stats* out) {
  if (!srv || !out) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(srv->mu);
  *out = srv->stats;
  out->hbm_in_use = srv->hbm_in_use;
  return TN_OK;
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
  for (auto& b : srv->packbufs) tn_server_s::release_packbuf(*b);
  for (auto& kv : srv->reqs)
    if (kv.second->done) cudaEventDestroy(kv.second->done);
  for (auto st : srv->streams) cudaStreamDestroy(st);
  delete srv;
  return TN_OK;
}

}  // extern "C"
