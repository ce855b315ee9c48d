// C ABI entry points and the executor that replays a plan on a CUDA stream.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "kernels.h"
#include "staging.cuh"
#include "tn_internal.h"

namespace tn {

namespace {
thread_local std::string g_last_error;

#define TN_CUDA_TRY(expr)                                                         \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      err = std::string(#expr) + ": " + cudaGetErrorString(e_);                   \
      return TN_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)

int64_t batch_footprint(Plan& P, int64_t b) {
  assign_workspace(P, b);
  return P.total_bytes;
}

StepArgs step_args(const Plan& P, const StepRec& st) {
  const TensorRec& A = P.tensors[st.a];
  const TensorRec& B = P.tensors[st.b];
  const TensorRec& C = P.tensors[st.out];
  const int64_t np = P.is_complex ? 2 : 1;
  StepArgs a{};
  a.A = reinterpret_cast<const float*>(P.dev + A.offset);
  a.B = reinterpret_cast<const float*>(P.dev + B.offset);
  a.C = reinterpret_cast<float*>(P.dev + C.offset);
  a.m = st.m;
  a.n = st.n;
  a.k = st.k;
  a.a_plane = A.size;
  a.b_plane = B.size;
  a.c_plane = C.size;
  // floats per element of each stored copy: 1 real, 2 complex, 3 in the 3M split form
  const auto fl = [&](const TensorRec& R) { return np == 1 ? int64_t(1) : (R.split == 2 ? int64_t(3) : int64_t(2)); };
  a.a_bstride = A.batched ? fl(A) * A.size : 0;
  a.b_bstride = B.batched ? fl(B) * B.size : 0;
  a.c_bstride = C.batched ? fl(C) * C.size : 0;
  a.rows = st.rows;
  a.cols = st.cols;
  a.recs = P.policy.exp_scaling ? reinterpret_cast<ScaleRec*>(P.dev + P.off_scale) : nullptr;
  a.rec_a = P.rec_index[st.a];
  a.rec_b = P.rec_index[st.b];
  a.rec_c = P.rec_index[st.out];
  a.c_split = C.split;
  a.maxplus = P.policy.semiring == TN_SEMIRING_MAXPLUS ? 1 : 0;
  a.ksplit = st.ksplit;
  a.part = st.ksplit > 1 ? reinterpret_cast<float*>(P.dev + P.off_scratch) : nullptr;
  return a;
}
void* take_event(Plan& P) {
  if (!P.prof_pool.empty()) {
    void* e = P.prof_pool.back();
    P.prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

// After the stream has been synchronized: a kernel whose bounded wait expired left a
// nonzero code in the plan's error word.
tn_status check_device_error(Plan& P) {
  int code = 0;
  cudaError_t e = cudaMemcpy(&code, P.dev + P.off_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string("reading the device error word: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  if (code != 0) {
    set_error("a tensor-core kernel gave up a bounded wait (code " + std::to_string(code) + ")");
    return TN_ERR_TIMEOUT;
  }
  return TN_OK;
}

tn_status upload_chain_table(Plan& P) {
  if (P.chains.empty() || !P.dev) return TN_OK;
  std::vector<ChainStep> table;
  for (const ChainRec& c : P.chains)
    for (int32_t q = c.first; q < c.first + c.n; ++q) {
      ChainStep cs{};
      cs.a = step_args(P, P.steps[q]);
      cs.batched = P.steps[q].batched ? 1 : 0;
      table.push_back(cs);
    }
  cudaError_t e = cudaMemcpy(P.dev + P.off_chain, table.data(), sizeof(ChainStep) * table.size(),
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("writing the step-chain table: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  return TN_OK;
}

tn_status run_slices(Plan& P, const void* const* inputs, int64_t begin, int64_t count, void* output,
                     double* log_scale, void* stream, std::string& err, void* pinned) {
  if (!P.dev) {
    err = "plan was built with TN_PLAN_HOST_ONLY (no device workspace)";
    return TN_ERR_INVALID;
  }
  if (!inputs || !output) {
    err = "null inputs or output";
    return TN_ERR_INVALID;
  }
  if (begin < 0 || count <= 0 || begin + count > P.n_slices) {
    err = "slice range out of bounds";
    return TN_ERR_INVALID;
  }
  for (int32_t t = 0; t < P.n_leaves; ++t)
    if (!inputs[t]) {
      err = "null input pointer";
      return TN_ERR_INVALID;
    }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool cplx = P.is_complex;
  const bool scaling = P.policy.exp_scaling != 0;
  const int32_t T = P.n_leaves, S = (int32_t)P.steps.size();
  const int32_t root = T + S - 1;
  for (int32_t t = 0; t < T; ++t) {
    P.leafdesc[t].src = inputs[t];
    P.leafdesc[t].dst = P.tensors[t].offset;
  }
  // descriptors from pageable memory (the copy is staged before the call returns), or from
  // the caller's pinned buffer
  const void* desc_src = P.leafdesc.data();
  const void* rec_src = P.rec_index.data();
  if (pinned) {
    char* pb = static_cast<char*>(pinned);
    std::memcpy(pb, P.leafdesc.data(), sizeof(LeafDesc) * P.leafdesc.size());
    std::memcpy(pb + sizeof(LeafDesc) * T, P.rec_index.data(), sizeof(int32_t) * T);
    desc_src = pb;
    rec_src = pb + sizeof(LeafDesc) * T;
  }
  TN_CUDA_TRY(cudaMemcpyAsync(P.dev + P.off_leafdesc, desc_src, sizeof(LeafDesc) * P.leafdesc.size(),
                              cudaMemcpyHostToDevice, st));
  ScaleRec* recs = scaling ? reinterpret_cast<ScaleRec*>(P.dev + P.off_scale) : nullptr;
  int32_t* recidx = reinterpret_cast<int32_t*>(P.dev + P.off_recidx);
  if (scaling) TN_CUDA_TRY(cudaMemcpyAsync(recidx, rec_src, sizeof(int32_t) * T, cudaMemcpyHostToDevice, st));
  const LeafDesc* descs = reinterpret_cast<const LeafDesc*>(P.dev + P.off_leafdesc);
  double* acc = reinterpret_cast<double*>(P.dev + P.off_acc);
  int64_t* ref = reinterpret_cast<int64_t*>(P.dev + P.off_ref);
  int* errw = reinterpret_cast<int*>(P.dev + P.off_err);
  TN_CUDA_TRY(cudaMemsetAsync(errw, 0, sizeof(int), st));
  const int64_t npass = (count + P.batch - 1) / P.batch;
  for (int64_t p = 0; p < npass; ++p) {
    const int32_t nb = (int32_t)std::min<int64_t>(P.batch, count - p * P.batch);
    const int64_t sb = begin + p * P.batch;
    if (scaling) {
      // 0x80 bytes make every emax very negative (the atomicMax identity)
      if (p == 0)
        TN_CUDA_TRY(cudaMemsetAsync(recs, 0x80, sizeof(ScaleRec) * P.n_rec_total, st));
      else
        TN_CUDA_TRY(cudaMemsetAsync(recs + P.n_rec_unbatched, 0x80,
                                    sizeof(ScaleRec) * (P.n_rec_total - P.n_rec_unbatched), st));
    }
    Plan::ProfRec sp{};
    if (P.prof_on) {
      sp.e0 = take_event(P);
      sp.e1 = take_event(P);
      sp.cls = TN_CLASS_PERM;
      sp.step = -1;
      double staged = 0.0;
      for (int32_t t = 0; t < T; ++t) {
        const TensorRec& R = P.tensors[t];
        if (p > 0 && !R.batched) continue;
        staged += double(R.size) * (R.batched ? nb : 1);
      }
      sp.bytes = 2.0 * (cplx ? 8.0 : 4.0) * staged;
      TN_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(sp.e0), st));
    }
    launch_stage_leaves(descs, P.leafdesc.data(), T, P.dev, sb, nb, p > 0, cplx, recs, recidx, st);
    if (P.prof_on) {
      TN_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(sp.e1), st));
      P.prof_pending.push_back(sp);
    }
    for (int32_t s = 0; s < S; ++s) {
      const StepRec& sr = P.steps[s];
      if (sr.chain >= 0) {
        // a step chain: one launch for the run at its first step
        const ChainRec& c = P.chains[sr.chain];
        if (s != c.first || (p > 0 && !c.any_batched)) continue;
        Plan::ProfRec pr{};
        if (P.prof_on) {
          pr.e0 = take_event(P);
          pr.e1 = take_event(P);
          pr.cls = TN_CLASS_SIMT;
          pr.step = s;
          for (int32_t q = c.first; q < c.first + c.n; ++q) {
            const StepRec& qr = P.steps[q];
            if (!qr.batched && p > 0) continue;
            const double nq = qr.batched ? nb : 1, m = double(qr.m), n = double(qr.n), k = double(qr.k);
            const TensorRec &QA = P.tensors[qr.a], &QB = P.tensors[qr.b];
            pr.flops += (cplx ? 8.0 : 2.0) * m * n * k * nq;
            pr.bytes += (cplx ? 8.0 : 4.0) * (m * k * (QA.batched ? nq : 1) + n * k * (QB.batched ? nq : 1) + m * n * nq);
          }
          TN_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(pr.e0), st));
        }
        launch_contract_chain(reinterpret_cast<const ChainStep*>(P.dev + P.off_chain) + c.table, c.n, nb, p > 0,
                              cplx, P.policy.semiring == TN_SEMIRING_MAXPLUS, st);
        if (P.prof_on) {
          TN_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(pr.e1), st));
          P.prof_pending.push_back(pr);
        }
        continue;
      }
      if (!sr.batched && p > 0) continue;  // slice-invariant: computed once, kept
      StepArgs a = step_args(P, sr);
      const int32_t nbs = sr.batched ? nb : 1;
      Plan::ProfRec pr{};
      if (P.prof_on) {
        pr.e0 = take_event(P);
        pr.e1 = take_event(P);
        pr.cls = sr.cls;
        pr.step = s;
        const double eb = cplx ? 8.0 : 4.0;
        const double m = double(sr.m), n = double(sr.n), k = double(sr.k);
        pr.flops = (cplx ? 8.0 : 2.0) * m * n * k * nbs;
        pr.bytes = eb * (m * k * (a.a_bstride ? nbs : 1) + n * k * (a.b_bstride ? nbs : 1) + m * n * nbs);
        TN_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(pr.e0), st));
      }
      if (sr.cls == TN_CLASS_TC) {
        const int32_t form = (P.policy.prec == TN_C64_BF16X3 && P.policy.complex_mult == 3) ? kPrecBF16x3M
                                                                                              : P.policy.prec;
        TN_CUDA_TRY(launch_contract_tc(a, nbs, form, cplx, errw, st,
                                       (P.policy.flags & TN_PLAN_SINGLE_SM_TILES) == 0 && !sr.single_sm));
      } else if (sr.cls == TN_CLASS_STREAM) {
        launch_contract_stream(a, nbs, cplx, P.num_sms, errw, st);
      } else if (sr.cls == TN_CLASS_SPLITK) {
        launch_contract_splitk(a, nbs, cplx, reinterpret_cast<double*>(P.dev + P.off_scratch), st);
      } else {
        launch_contract_simt(a, nbs, cplx, st);
      }
      if (P.prof_on) {
        TN_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(pr.e1), st));
        P.prof_pending.push_back(pr);
      }
    }
    const TensorRec& R = P.tensors[root];
    const int64_t np = cplx ? 2 : 1;
    launch_accumulate_root(reinterpret_cast<const float*>(P.dev + R.offset), R.size,
                           R.batched ? nb : 1, R.batched ? np * R.size : 0, R.size, cplx, acc, recs,
                           P.rec_index[root], R.batched, ref, p == 0, p == npass - 1,
                           P.policy.semiring == TN_SEMIRING_MAXPLUS, output, log_scale, P.num_sms, st);
  }
  TN_CUDA_TRY(cudaGetLastError());
  return TN_OK;
}

// FP32 FMA peak probe: 8 independent chains x <- x * m + c per thread (the fixed point
// c / (1 - m) keeps every value normal); the sum is stored only if it hits an impossible
// value, so the chains stay live without memory traffic.
__global__ void __launch_bounds__(256) ffma_probe_kernel(int64_t iters, float m, float c, float* out) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0.05f + 1e-3f * j + 1e-6f * threadIdx.x;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == -1.0f) out[blockIdx.x] = s;
}

// FP64 FMA rate probe: the same form as ffma_probe_kernel in double precision.
__global__ void __launch_bounds__(256) dfma_probe_kernel(int64_t iters, double m, double c, double* out) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0.05 + 1e-3 * j + 1e-6 * threadIdx.x;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == -1.0) out[blockIdx.x] = s;
}

}  // namespace tn

using namespace tn;


extern "C" {

const char* tn_last_error(void) { return g_last_error.c_str(); }

tn_status tn_plan(const tn_network* net, const tn_path* path, const int32_t* sliced_modes,
                  int32_t n_sliced, tn_dtype_policy policy, tn_plan_t* out) {
  if (!out) {
    set_error("null output handle");
    return TN_ERR_INVALID;
  }
  tn_plan_s* h = new (std::nothrow) tn_plan_s();
  if (!h) {
    set_error("host allocation failed");
    return TN_ERR_OOM;
  }
  std::string err;
  tn_status s;
  try {
    s = build_plan(net, path, sliced_modes, n_sliced, policy, h->P, err);
  } catch (const std::exception& e) {
    err = std::string("planner exception: ") + e.what();
    s = TN_ERR_INVALID;
  }
  if (s != TN_OK) {
    set_error(err);
    delete h;
    return s;
  }
  Plan& P = h->P;
  static std::atomic<uint64_t> next_uid{1};
  P.uid = next_uid++;
  const bool host_only = (policy.flags & TN_PLAN_HOST_ONLY) != 0;
  int64_t want = policy.max_slice_batch > 0 ? std::min<int64_t>(P.n_slices, policy.max_slice_batch)
                                            : P.n_slices;
  want = std::min<int64_t>(want, 65535);  // the batch is a grid dimension
  if (host_only) {
    if (policy.max_slice_batch <= 0) want = 1;
    assign_workspace(P, want);
    if (!P.workspace_ok) {
      set_error("internal error: workspace assignment failed its self-check");
      delete h;
      return TN_ERR_INVALID;
    }
    *out = h;
    return TN_OK;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev);
  size_t free_b = 0, total_b = 0;
  if (ce == cudaSuccess) ce = cudaMemGetInfo(&free_b, &total_b);
  if (ce != cudaSuccess) {
    set_error(std::string("CUDA unavailable: ") + cudaGetErrorString(ce));
    delete h;
    return TN_ERR_CUDA;
  }
  const int64_t budget = int64_t(double(free_b) * 0.9);
  int64_t b = want;
  while (b > 1 && batch_footprint(P, b) > budget) b = (b + 1) / 2;
  if (batch_footprint(P, b) > budget || !P.workspace_ok) {
    if (!P.workspace_ok) {
      set_error("internal error: workspace assignment failed its self-check");
      delete h;
      return TN_ERR_INVALID;
    }
    set_error("workspace of " + std::to_string(P.total_bytes) + " bytes exceeds free device memory");
    delete h;
    return TN_ERR_OOM;
  }
  void* mem = nullptr;
  ce = cudaMalloc(&mem, (size_t)P.total_bytes);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc of workspace failed: ") + cudaGetErrorString(ce));
    delete h;
    return TN_ERR_OOM;
  }
  P.dev = static_cast<char*>(mem);
  const tn_status cs = upload_chain_table(P);
  if (cs != TN_OK) {
    cudaFree(mem);
    delete h;
    return cs;
  }
  *out = h;
  return TN_OK;
}

tn_status tn_plan_info(tn_plan_t plan, tn_plan_stats* out) {
  if (!plan || !out) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  *out = plan->P.stats;
  return TN_OK;
}

tn_status tn_plan_layout(tn_plan_t plan, int32_t id, int32_t* modes_out, int32_t* rank_out) {
  if (!plan || !rank_out || id < 0 || id >= (int32_t)plan->P.tensors.size()) {
    set_error("bad plan or tensor id");
    return TN_ERR_INVALID;
  }
  const auto& m = plan->P.tensors[id].modes;
  *rank_out = (int32_t)m.size();
  if (modes_out) std::copy(m.begin(), m.end(), modes_out);
  return TN_OK;
}

tn_status tn_plan_launches(tn_plan_t plan, int64_t slice_count, int64_t* out) {
  if (!plan || !out || slice_count <= 0 || slice_count > plan->P.n_slices) {
    set_error("bad plan, slice count or output");
    return TN_ERR_INVALID;
  }
  const Plan& P = plan->P;
  const int32_t T = P.n_leaves;
  const int64_t npass = (slice_count + P.batch - 1) / P.batch;
  const bool pairs = (P.policy.flags & TN_PLAN_SINGLE_SM_TILES) == 0;
  const int32_t form =
      (P.policy.prec == TN_C64_BF16X3 && P.policy.complex_mult == 3) ? kPrecBF16x3M : P.policy.prec;
  int64_t n = 0;
  for (int64_t p = 0; p < npass; ++p) {
    const int32_t nb = (int32_t)std::min<int64_t>(P.batch, slice_count - p * P.batch);
    if (T > 0) n += 1;  // stage_leaves_kernel
    for (int32_t t = 0; t < T; ++t)
      if (P.leafdesc[t].tiled && !(p > 0 && !P.tensors[t].batched)) n += 1;
    for (int32_t q = 0; q < (int32_t)P.steps.size(); ++q) {
      const StepRec& st = P.steps[q];
      if (st.chain >= 0) {  // one launch per step chain, at its first step
        const ChainRec& c = P.chains[st.chain];
        if (q == c.first && (p == 0 || c.any_batched)) n += 1;
        continue;
      }
      if (!st.batched && p > 0) continue;
      const int32_t nbs = st.batched ? nb : 1;
      if (st.cls == TN_CLASS_TC)
        n += tc_launches(st.m, st.n, st.k, nbs, form, pairs && !st.single_sm, P.policy.exp_scaling != 0);
      else if (st.cls == TN_CLASS_SPLITK) n += 2;
      else if (st.cls == TN_CLASS_SIMT) n += st.ksplit > 1 ? 2 : 1;
      else n += 1;
    }
    n += 1;  // the slice sum (or the output widening)
  }
  *out = n;
  return TN_OK;
}

tn_status tn_plan_step(tn_plan_t plan, int32_t s, tn_step_info* out) {
  if (!plan || !out || s < 0 || s >= (int32_t)plan->P.steps.size()) {
    set_error("bad plan or step");
    return TN_ERR_INVALID;
  }
  const StepRec& st = plan->P.steps[s];
  out->m = st.m;
  out->n = st.n;
  out->k = st.k;
  out->a_id = st.a;
  out->b_id = st.b;
  out->cls = st.cls;
  out->batched = st.batched ? 1 : 0;
  out->n_row_dims = st.rows.n;
  out->n_col_dims = st.cols.n;
  for (int d = 0; d < 12; ++d) {
    out->row_ext[d] = d < st.rows.n ? st.rows.ext[d] : 0;
    out->row_stride[d] = d < st.rows.n ? st.rows.stride[d] : 0;
    out->col_ext[d] = d < st.cols.n ? st.cols.ext[d] : 0;
    out->col_stride[d] = d < st.cols.n ? st.cols.stride[d] : 0;
  }
  out->ksplit = st.ksplit;
  out->single_sm = st.single_sm ? 1 : 0;
  out->chain = st.chain;
  out->reserved = 0;
  return TN_OK;
}

tn_status tn_plan_tensor(tn_plan_t plan, int32_t id, tn_tensor_info* out) {
  if (!plan || !out || id < 0 || id >= (int32_t)plan->P.tensors.size()) {
    set_error("bad plan or tensor id");
    return TN_ERR_INVALID;
  }
  const TensorRec& R = plan->P.tensors[id];
  out->size = R.size;
  out->offset = R.offset;
  out->bytes = R.bytes;
  out->batched = R.batched ? 1 : 0;
  out->pinned = R.pinned ? 1 : 0;
  out->producer = R.producer;
  out->consumer = R.consumer;
  out->format = R.split;
  out->tiled = id < plan->P.n_leaves ? (plan->P.leafdesc[id].tiled ? (plan->P.leafdesc[id].fast ? 2 : 1) : 0) : 0;
  return TN_OK;
}

tn_status tn_contract_slices(tn_plan_t plan, const void* const* inputs, int64_t slice_begin,
                             int64_t slice_count, void* output, double* out_log_scale, void* stream) {
  if (!plan) {
    set_error("null plan");
    return TN_ERR_INVALID;
  }
  std::string err;
  tn_status s = run_slices(plan->P, inputs, slice_begin, slice_count, output, out_log_scale, stream, err);
  if (s != TN_OK) set_error(err);
  return s;
}

tn_status tn_contract(tn_plan_t plan, const void* const* inputs, void* output, double* out_log_scale,
                      void* stream) {
  if (!plan) {
    set_error("null plan");
    return TN_ERR_INVALID;
  }
  return tn_contract_slices(plan, inputs, 0, plan->P.n_slices, output, out_log_scale, stream);
}

tn_status tn_plan_autotune(tn_plan_t plan, const void* const* inputs, void* output, void* stream) {
  if (!plan || !inputs || !output) {
    set_error("null plan, inputs or output");
    return TN_ERR_INVALID;
  }
  Plan& P = plan->P;
  if (!P.dev) {
    set_error("plan was built with TN_PLAN_HOST_ONLY (no device workspace)");
    return TN_ERR_INVALID;
  }
  // the steps with a choice: BF16x3 4M tensor-core steps that the paired-SM kernels take
  std::vector<int32_t> cand;
  // (scaled plans run every BF16x3 step on one SM per tile: no choice)
  const bool bf16x3_4m = P.policy.prec == TN_C64_BF16X3 && P.policy.complex_mult != 3 && !P.policy.exp_scaling;
  if (bf16x3_4m && (P.policy.flags & TN_PLAN_SINGLE_SM_TILES) == 0)
    for (int32_t s = 0; s < (int32_t)P.steps.size(); ++s) {
      const StepRec& st = P.steps[s];
      if (st.cls == TN_CLASS_TC && tc_launches(st.m, st.n, st.k, 1, TN_C64_BF16X3, true, false) >= 1 &&
          st.m >= 256 && st.k > 256)
        cand.push_back(s);
    }
  if (cand.empty()) return TN_OK;
  // the caller's profile is set aside and restored
  const bool prof_was = P.prof_on;
  tn_profile acc_keep{};
  tn_status s = tn_plan_profile_read(plan, &acc_keep, 1);
  if (s != TN_OK) return s;
  const std::vector<double> steps_keep = P.prof_last_step_ms;
  const int64_t count = std::min<int64_t>(P.batch, P.n_slices);
  std::vector<double> t[2];
  std::string err;
  for (int v = 0; v < 2 && s == TN_OK; ++v) {
    for (int32_t c : cand) P.steps[c].single_sm = v == 1;
    P.prof_on = false;
    s = run_slices(P, inputs, 0, count, output, nullptr, stream, err);  // warm
    if (s != TN_OK) break;
    P.prof_on = true;
    s = run_slices(P, inputs, 0, count, output, nullptr, stream, err);
    if (s != TN_OK) break;
    tn_profile tmp{};
    s = tn_plan_profile_read(plan, &tmp, 1);
    t[v] = P.prof_last_step_ms;
  }
  P.prof_on = prof_was;
  P.prof_acc = acc_keep;
  P.prof_last_step_ms = steps_keep;
  if (s != TN_OK) {
    for (int32_t c : cand) P.steps[c].single_sm = false;
    if (!err.empty()) set_error(err);
    return s;
  }
  for (int32_t c : cand) P.steps[c].single_sm = t[1][c] < t[0][c];
  return TN_OK;
}

tn_status tn_contract_graph(tn_plan_t plan, const void* const* inputs, void* output, double* out_log_scale,
                            void* stream) {
  if (!plan || !inputs || !output) {
    set_error("null plan, inputs or output");
    return TN_ERR_INVALID;
  }
  Plan& P = plan->P;
  if (!P.dev) {
    set_error("plan was built with TN_PLAN_HOST_ONLY (no device workspace)");
    return TN_ERR_INVALID;
  }
  if (P.prof_on) {
    set_error("tn_contract_graph: per-step profiling is on (tn_plan_profile)");
    return TN_ERR_INVALID;
  }
  const int32_t T = P.n_leaves;
  bool same = P.g_exec && P.g_out == output && P.g_ls == out_log_scale && P.g_stream == stream &&
              (int32_t)P.g_inputs.size() == T;
  for (int32_t t = 0; same && t < T; ++t) same = P.g_inputs[t] == inputs[t];
  if (same) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGraphLaunch(static_cast<cudaGraphExec_t>(P.g_exec), st);
    if (e == cudaSuccess) e = cudaEventRecord(static_cast<cudaEvent_t>(P.g_done), st);
    if (e != cudaSuccess) {
      set_error(std::string("graph launch: ") + cudaGetErrorString(e));
      return TN_ERR_CUDA;
    }
    return TN_OK;
  }
  // new pointers or stream: run the call as usual (which also performs any one-time
  // kernel configuration), then capture the same call on a private stream
  tn_status s = tn_contract(plan, inputs, output, out_log_scale, stream);
  if (s != TN_OK) return s;
  if (P.g_done) {
    // the previous graph's copy nodes read the pinned buffer: let its last launch finish
    cudaEventSynchronize(static_cast<cudaEvent_t>(P.g_done));
  } else if (cudaEventCreateWithFlags(reinterpret_cast<cudaEvent_t*>(&P.g_done), cudaEventDisableTiming) !=
             cudaSuccess) {
    set_error("event creation failed");
    return TN_ERR_CUDA;
  }
  if (P.g_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(P.g_exec));
  P.g_exec = nullptr;
  if (!P.g_pinned && cudaMallocHost(&P.g_pinned, (sizeof(LeafDesc) + sizeof(int32_t)) * T + 16) != cudaSuccess) {
    P.g_pinned = nullptr;
    set_error("pinned descriptor buffer");
    return TN_ERR_OOM;
  }
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("graph capture stream");
    return TN_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  std::string err;
  s = TN_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = TN_ERR_CUDA;
  if (s == TN_OK) s = run_slices(P, inputs, 0, P.n_slices, output, out_log_scale, cap, err, P.g_pinned);
  cudaError_t e = cudaStreamEndCapture(cap, &g);
  cudaGraphExec_t ge = nullptr;
  if (s == TN_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (s != TN_OK || e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("graph capture failed: ") + (err.empty() ? cudaGetErrorString(e) : err));
    return TN_ERR_CUDA;
  }
  P.g_exec = ge;
  P.g_inputs.assign(inputs, inputs + T);
  P.g_out = output;
  P.g_ls = out_log_scale;
  P.g_stream = stream;
  return TN_OK;
}

tn_status tn_contract_slices_host(tn_plan_t plan, const void* const* host_inputs, int64_t slice_begin,
                                  int64_t slice_count, void* host_output, double* out_log_scale, void* stream) {
  if (!plan || !host_inputs || !host_output) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  Plan& P = plan->P;
  if (!P.dev) {
    set_error("plan was built with TN_PLAN_HOST_ONLY (no device workspace)");
    return TN_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t eb = elem_bytes(P);
  std::vector<const void*> dptr(P.n_leaves);
  std::string err;
  auto fail = [&](cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  };
  for (int32_t t = 0; t < P.n_leaves; ++t) {
    if (!host_inputs[t]) {
      set_error("null input pointer");
      return TN_ERR_INVALID;
    }
    int64_t full = 1;
    for (int32_t x : P.tensors[t].decl) full *= P.extent[x];
    char* d = P.dev + P.stage_in_off[t];
    cudaError_t e = cudaMemcpyAsync(d, host_inputs[t], full * eb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(e, "host-to-device copy of an input");
    dptr[t] = d;
  }
  char* dout = P.dev + P.total_bytes - ((P.out_elems * 16 + 16 + 255) / 256 * 256);
  double* dls = reinterpret_cast<double*>(dout + P.out_elems * 16);
  tn_status s = run_slices(P, dptr.data(), slice_begin, slice_count, dout, dls, stream, err);
  if (s != TN_OK) {
    set_error(err);
    return s;
  }
  const int64_t ob = P.out_elems * (P.is_complex ? 16 : 8);
  cudaError_t e = cudaMemcpyAsync(host_output, dout, ob, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return fail(e, "device-to-host copy of the result");
  if (out_log_scale) {
    e = cudaMemcpyAsync(out_log_scale, dls, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(e, "device-to-host copy of the log scale");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e, "stream synchronize");
  return check_device_error(P);
}

tn_status tn_contract_host(tn_plan_t plan, const void* const* host_inputs, void* host_output,
                           double* out_log_scale, void* stream) {
  if (!plan) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  return tn_contract_slices_host(plan, host_inputs, 0, plan->P.n_slices, host_output, out_log_scale, stream);
}

tn_status tn_plan_destroy(tn_plan_t plan) {
  if (!plan) return TN_OK;
  if (plan->P.g_done) {
    cudaEventSynchronize(static_cast<cudaEvent_t>(plan->P.g_done));
    cudaEventDestroy(static_cast<cudaEvent_t>(plan->P.g_done));
  }
  if (plan->P.g_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(plan->P.g_exec));
  if (plan->P.g_pinned) cudaFreeHost(plan->P.g_pinned);
  if (plan->P.dev) cudaFree(plan->P.dev);
  for (auto& r : plan->P.prof_pending) {
    cudaEventDestroy(static_cast<cudaEvent_t>(r.e0));
    cudaEventDestroy(static_cast<cudaEvent_t>(r.e1));
  }
  for (void* e : plan->P.prof_pool) cudaEventDestroy(static_cast<cudaEvent_t>(e));
  delete plan;
  return TN_OK;
}

tn_status tn_plan_profile_steps(tn_plan_t plan, double* ms_out, int32_t n_steps) {
  if (!plan || !ms_out || n_steps != (int32_t)plan->P.steps.size()) {
    set_error("bad plan, buffer or step count");
    return TN_ERR_INVALID;
  }
  // totals of the last read with reset, else those accumulated since
  const std::vector<double>& v =
      plan->P.prof_step_ms.empty() || std::all_of(plan->P.prof_step_ms.begin(), plan->P.prof_step_ms.end(),
                                                   [](double x) { return x == 0.0; })
          ? plan->P.prof_last_step_ms
          : plan->P.prof_step_ms;
  for (int32_t s = 0; s < n_steps; ++s) ms_out[s] = s < (int32_t)v.size() ? v[s] : 0.0;
  return TN_OK;
}

tn_status tn_selftest_bounded_wait(tn_plan_t plan, int32_t arrive, int64_t limit_us, void* stream) {
  if (!plan || !plan->P.dev || limit_us <= 0 || limit_us > 10000000) {
    set_error("tn_selftest_bounded_wait: needs a device plan and 0 < limit_us <= 1e7");
    return TN_ERR_INVALID;
  }
  Plan& P = plan->P;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* errw = reinterpret_cast<int*>(P.dev + P.off_err);
  cudaError_t e = cudaMemsetAsync(errw, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_bounded_wait_selftest(arrive ? 1 : 0, uint64_t(limit_us) * 1000ull, errw, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("tn_selftest_bounded_wait: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  return check_device_error(P);
}

tn_status tn_plan_check_staging(tn_plan_t plan, int64_t max_slices) {
  if (!plan || max_slices < 1) {
    set_error("tn_plan_check_staging: bad arguments");
    return TN_ERR_INVALID;
  }
  const Plan& P = plan->P;
  for (int32_t t = 0; t < P.n_leaves; ++t) {
    const LeafDesc& d = P.leafdesc[t];
    if (!d.tiled) continue;
    const TensorRec& R = P.tensors[t];
    int64_t src_elems = 1;
    for (int32_t x : R.decl) src_elems *= P.extent[x];
    const int64_t tiles = d.Pr * ((d.Po + 31) / 32) * ((d.Pi + 31) / 32);
    if (tiles > 0x7fffffffll || d.Po * d.Pi * d.Pr != d.size) {
      set_error("tiled staging of leaf " + std::to_string(t) + ": bad grid or group sizes");
      return TN_ERR_INVALID;
    }
    const int64_t n_sid = d.batched ? std::min<int64_t>(P.n_slices, max_slices) : 1;
    for (int64_t q = 0; q < n_sid; ++q) {
      // slices 0, n-1, and evenly spread ones between
      const int64_t sid = n_sid == 1 ? 0 : q * (P.n_slices - 1) / (n_sid - 1);
      if (d.fast) {
        // the pipelined form's offsets: every tile's rest offset as its CTA's high part plus
        // the tile's low part, the tables of chunk (0, 0) -- equal to the cursor form's
        if (d.Po != 32 || d.Pi != 32 || tiles % kTilesPerCta != 0 || !d.vec_load) {
          set_error("tiled staging of leaf " + std::to_string(t) + ": pipelined form on an unfit leaf");
          return TN_ERR_INVALID;
        }
        for (int64_t blk = 0; blk < tiles; ++blk) {
          int64_t hs, hd, ls, ld;
          rest_hi_offsets(d, blk / kTilesPerCta, sid, hs, hd);
          rest_lo_offsets(d, blk % kTilesPerCta, ls, ld);
          const TileBase tb = tile_base(d, blk, sid);
          if (tb.go0 != 0 || tb.gi0 != 0 || hs + ls != tb.src0 || hd + ld != tb.dst0) {
            set_error("tiled staging of leaf " + std::to_string(t) + ": pipelined offsets disagree with tile " +
                      std::to_string(blk));
            return TN_ERR_INVALID;
          }
        }
      }
      std::vector<char> seen(d.size, 0);
      // each CTA as the kernel runs it: iterations of kTilesInFlight tiles, slot tables
      // rebuilt only when iteration_tiles says so, element offsets read from the tables
      constexpr int TT = kTilesInFlight;
      for (int64_t blk0 = 0; blk0 < tiles; blk0 += kTilesPerCta) {
        const int64_t blk1 = std::min<int64_t>(blk0 + kTilesPerCta, tiles);
        TileCursor cur[TT];
        int64_t built[TT][2];
        int rebuild[TT] = {};
        for (int u = 0; u < TT; ++u) built[u][0] = built[u][1] = -1;
        int64_t isrc[TT][32] = {}, osrc[TT][32] = {}, irow[TT][32] = {};
        for (int64_t blk = blk0; blk < blk1; blk += TT) {
          const int nt = iteration_tiles(d, blk, blk0, blk1, sid, cur, built, rebuild);
          for (int u = 0; u < nt; ++u) {
            const TileBase tb = tile_base(d, blk + u, sid);
            if (cur[u].co * 32 != tb.go0 || cur[u].ci * 32 != tb.gi0 || cur[u].src0 != tb.src0 ||
                cur[u].dst0 != tb.dst0) {
              set_error("tiled staging of leaf " + std::to_string(t) + ": the tile cursor disagrees with tile " +
                        std::to_string(blk + u));
              return TN_ERR_INVALID;
            }
            if (rebuild[u])
              for (int r = 0; r < 32; ++r) table_entry(d, tb.go0, tb.gi0, r, isrc[u][r], osrc[u][r], irow[u][r]);
          }
          for (int u = 0; u < nt; ++u) {
            const TileBase tb = tile_base(d, blk + u, sid);
            for (int ti = 0; ti < 32; ++ti) {
              const int64_t gi = tb.gi0 + ti;
              if (gi >= d.Pi) continue;
              for (int to = 0; to < 32; ++to) {
                const int64_t go = tb.go0 + to;
                if (go >= d.Po) continue;
                const int64_t so = cur[u].src0 + isrc[u][ti] + osrc[u][to], el = cur[u].dst0 + irow[u][ti] + to;
                // what the per-leaf kernel reads for staged element el
                int64_t want = 0, e = el;
                for (int r = d.rank - 1; r >= 0; --r) {
                  want += (e % d.ext[r]) * d.sstride[r];
                  e /= d.ext[r];
                }
                for (int k = 0; k < d.n_sl; ++k) want += ((sid / d.sl_div[k]) % d.sl_ext[k]) * d.sl_stride[k];
                bool ok = el >= 0 && el < d.size && so == want && so >= 0 && so < src_elems && !seen[el] &&
                          so == tile_src(d, tb, gi, go) && el == tile_dst_row(d, tb, gi) + to;
                if (ok && d.vec_load && (ti % 2) == 0)
                  ok = so % 2 == 0 && cur[u].src0 + isrc[u][ti + 1] + osrc[u][to] == so + 1;
                if (!ok) {
                  set_error("tiled staging of leaf " + std::to_string(t) + ": tile " + std::to_string(blk + u) +
                            " entry (" + std::to_string(ti) + ", " + std::to_string(to) + ") maps source " +
                            std::to_string(so) + " to element " + std::to_string(el) + " (expected source " +
                            std::to_string(want) + ")");
                  return TN_ERR_INVALID;
                }
                seen[el] = 1;
              }
            }
          }
        }
      }
      for (int64_t el = 0; el < d.size; ++el)
        if (!seen[el]) {
          set_error("tiled staging of leaf " + std::to_string(t) + ": element " + std::to_string(el) +
                    " is never written");
          return TN_ERR_INVALID;
        }
    }
  }
  return TN_OK;
}

tn_status tn_cost_model_set(const tn_cost_model* m) {
  if (!m || !(m->hbm_bytes_per_s > 0) || !(m->simt_flops > 0) || !(m->tc_flops[0] > 0) ||
      !(m->tc_flops[1] > 0) || !(m->tc_flops[2] > 0)) {
    set_error("tn_cost_model_set: every rate must be positive");
    return TN_ERR_INVALID;
  }
  g_cost = *m;
  return TN_OK;
}

tn_status tn_cost_model_get(tn_cost_model* out) {
  if (!out) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  *out = g_cost;
  return TN_OK;
}

// Time one FMA-chain probe launch (4 CTAs of 256 threads per SM, 8 chains per thread).
static tn_status measure_fma(bool fp64, int64_t iters, double* flops_per_s, double* ms, void* stream) {
  const char* name = fp64 ? "tn_measure_dfma" : "tn_measure_ffma";
  if (iters <= 0 || iters > (int64_t(1) << 24) || !flops_per_s) {
    set_error(std::string(name) + ": needs 0 < iters <= 2^24 and an output pointer");
    return TN_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = 4 * sms;
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    if (fp64) dfma_probe_kernel<<<grid, 256, 0, st>>>(iters, 0.999999999, 1e-10, nullptr);
    else ffma_probe_kernel<<<grid, 256, 0, st>>>(iters, 0.999999f, 1e-7f, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_error(std::string(name) + ": " + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  *flops_per_s = 2.0 * 8.0 * double(iters) * double(grid) * 256.0 / (double(t) * 1e-3);
  if (ms) *ms = t;
  return TN_OK;
}

tn_status tn_measure_ffma(int64_t iters, double* flops_per_s, double* ms, void* stream) {
  return measure_fma(false, iters, flops_per_s, ms, stream);
}

tn_status tn_measure_dfma(int64_t iters, double* flops_per_s, double* ms, void* stream) {
  return measure_fma(true, iters, flops_per_s, ms, stream);
}

tn_status tn_plan_profile(tn_plan_t plan, int32_t enable) {
  if (!plan) {
    set_error("null plan");
    return TN_ERR_INVALID;
  }
  plan->P.prof_on = enable != 0;
  return TN_OK;
}

tn_status tn_plan_profile_read(tn_plan_t plan, tn_profile* out, int32_t reset) {
  if (!plan || !out) {
    set_error("null argument");
    return TN_ERR_INVALID;
  }
  Plan& P = plan->P;
  for (auto& r : P.prof_pending) {
    cudaEvent_t e0 = static_cast<cudaEvent_t>(r.e0), e1 = static_cast<cudaEvent_t>(r.e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      set_error(std::string("profile event: ") + cudaGetErrorString(e));
      return TN_ERR_CUDA;
    }
    P.prof_acc.launches[r.cls] += 1;
    if (P.prof_step_ms.size() != P.steps.size()) P.prof_step_ms.assign(P.steps.size(), 0.0);
    if (r.step >= 0) P.prof_step_ms[r.step] += ms;
    P.prof_acc.ms[r.cls] += ms;
    P.prof_acc.flops[r.cls] += r.flops;
    P.prof_acc.bytes[r.cls] += r.bytes;
    P.prof_pool.push_back(r.e0);
    P.prof_pool.push_back(r.e1);
  }
  P.prof_pending.clear();
  tn_status ds = check_device_error(P);
  if (ds != TN_OK) return ds;
  *out = P.prof_acc;
  if (reset) {
    P.prof_last_step_ms = P.prof_step_ms;
    P.prof_acc = tn_profile{};
    P.prof_step_ms.assign(P.steps.size(), 0.0);
  }
  return TN_OK;
}

}  // extern "C"
