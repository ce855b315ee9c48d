// Batched independent small networks in one persistent launch.
//
// Each network has its own path and its own plan (the same planner as tn_plan: step
// analysis, GEMM-oriented reordering of Sec. IV-A, liveness offsets), flattened into
// compact device tables. One CTA takes the next network from an atomic queue and runs
// its whole path: stage the leaves into the network's arena (planned orders), then for
// each step C = A (m x k) . B (n x k)^T written through the output offset maps, with
// every thread of the CTA working on the step. With exponent scaling each tensor is
// renormalised in place after it is made (an exact power of two chosen from its largest
// entry) and the exponents are summed per network in an int64; the network's result is
// (value, log2 scale) and ln|Z| = ln|value| + log2 * ln 2 in FP64 on the host side. In the
// max-plus semiring (real, unscaled) a step is C = max_k (A + B) instead. (Taking the
// costliest networks first was measured: 1.4-1.5x slower on both ensembles -- the big
// arenas then run at the same time and contend for L2 -- so the queue stays in order.)
// The CTA width (threads per network) and CTAs per SM are chosen by an autotuner that
// times the real batch; the launch (queue reset + kernel) can be replayed as a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "batch.h"
#include "kernels.h"
#include "tn_internal.h"

namespace tn {
namespace {

__device__ __forceinline__ int bexp_of(float v) { return ((__float_as_int(v) >> 23) & 0xff) - 127; }
__device__ __forceinline__ float bpow2_neg(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((127 - e) << 23);
}

template <bool CPLX>
__device__ void renormalise(float* t, int size, int* smax, long long* slog) {
  int lmax = -127;
  for (int i = threadIdx.x; i < size; i += blockDim.x) {
    float v = fabsf(t[i]);
    if (CPLX) v = fmaxf(v, fabsf(t[size + i]));
    lmax = max(lmax, bexp_of(v));
  }
  for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(smax, lmax);
  __syncthreads();
  const int e = *smax < -126 ? 0 : *smax;  // an all-zero tensor is left as is
  if (e != 0) {
    const float s = bpow2_neg(e);
    for (int i = threadIdx.x; i < size; i += blockDim.x) {
      t[i] *= s;
      if (CPLX) t[size + i] *= s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *slog += e;
    *smax = -127;
  }
  __syncthreads();
}

// leaves whose exponents one pass takes together (networks with more renormalise leaf by leaf)
constexpr int kLeafExpCap = 256;

// Output offset of row x (x < m) or of column x - m (x >= m) of step S: the mixed-radix
// digits over the merged dims, each times its stride.
__device__ __forceinline__ int step_offset(const BStep& S, int x) {
  int off = 0;
  if (x < S.m) {
    for (int d = S.nr - 1; d >= 0; --d) {
      off += (x % S.rext[d]) * S.rstr[d];
      x /= S.rext[d];
    }
  } else {
    x -= S.m;
    for (int d = S.nc - 1; d >= 0; --d) {
      off += (x % S.cext[d]) * S.cstr[d];
      x /= S.cext[d];
    }
  }
  return off;
}

template <bool CPLX, bool MAXPLUS = false>
__global__ void batch_kernel(const BNet* __restrict__ nets, const BLeaf* __restrict__ leaves,
                             const BStep* __restrict__ steps, int32_t n_nets, const float* __restrict__ in,
                             float* arena, int32_t* queue, int32_t scaling, double* values, double* logs,
                             int32_t smem_arena, int32_t tab_ints) {
  // dynamic shared memory: [arena: smem_arena floats | offset table: tab_ints ints]
  extern __shared__ float s_arena[];
  int* s_tab = reinterpret_cast<int*>(s_arena + smem_arena);
  __shared__ int s_lexp[kLeafExpCap];  // per-leaf maximum exponents
  __shared__ int s_net;
  __shared__ int s_max;
  __shared__ long long s_log;
  constexpr int NP = CPLX ? 2 : 1;
  if (threadIdx.x == 0) s_max = -127;
  while (true) {
    if (threadIdx.x == 0) {
      s_net = atomicAdd(queue, 1);
      s_log = 0;
    }
    __syncthreads();
    const int w = s_net;
    if (w >= n_nets) break;
    const BNet net = nets[w];
    // the network's arena: in shared memory when it fits the launch's shared-memory arena
    // (smem_arena floats per CTA), else its own slice of the global batch arena
    float* ar = net.arena_floats <= smem_arena ? s_arena : arena + net.arena;
    // stage the leaves (declared order -> planned order; complex64 -> planar)
    for (int l = 0; l < net.n_leaves; ++l) {
      const BLeaf& L = leaves[net.leaf0 + l];
      for (int e = threadIdx.x; e < L.size; e += blockDim.x) {
        int r = e, src = 0;
        for (int d = L.rank - 1; d >= 0; --d) {
          src += (r % L.ext[d]) * L.sstride[d];
          r /= L.ext[d];
        }
        if (CPLX) {
          const float2 v = reinterpret_cast<const float2*>(in)[L.src + src];
          ar[L.dst + e] = v.x;
          ar[L.dst + L.size + e] = v.y;
        } else {
          ar[L.dst + e] = in[L.src + src];
        }
      }
    }
    __syncthreads();
    if (scaling && net.n_leaves <= kLeafExpCap) {
      // every leaf renormalised in one pass: per-leaf maxima by shared-memory atomics, then
      // each leaf scaled by its own exact power of two (the same exponents as one leaf at a
      // time, with three barriers instead of three per leaf)
      for (int l = threadIdx.x; l < net.n_leaves; l += blockDim.x) s_lexp[l] = -127;
      __syncthreads();
      for (int l = 0; l < net.n_leaves; ++l) {
        const BLeaf& L = leaves[net.leaf0 + l];
        int lmax = -127;
        for (int i = threadIdx.x; i < L.size; i += blockDim.x) {
          float v = fabsf(ar[L.dst + i]);
          if (CPLX) v = fmaxf(v, fabsf(ar[L.dst + L.size + i]));
          lmax = max(lmax, bexp_of(v));
        }
        if (lmax > -127) atomicMax(&s_lexp[l], lmax);
      }
      __syncthreads();
      long long sum = 0;
      for (int l = 0; l < net.n_leaves; ++l) {
        const BLeaf& L = leaves[net.leaf0 + l];
        const int e = s_lexp[l] < -126 ? 0 : s_lexp[l];  // an all-zero leaf is left as is
        sum += e;
        if (e == 0) continue;
        const float sc = bpow2_neg(e);
        for (int i = threadIdx.x; i < L.size; i += blockDim.x) {
          ar[L.dst + i] *= sc;
          if (CPLX) ar[L.dst + L.size + i] *= sc;
        }
      }
      if (threadIdx.x == 0) s_log += sum;
      __syncthreads();
    } else if (scaling) {
      for (int l = 0; l < net.n_leaves; ++l) {
        const BLeaf& L = leaves[net.leaf0 + l];
        renormalise<CPLX>(ar + L.dst, L.size, &s_max, &s_log);
      }
    }
    for (int s = 0; s < net.n_steps; ++s) {
      const BStep& S = steps[net.step0 + s];
      const int mn = S.m * S.n;
      // the output offset of every row and column, once per step (not once per element)
      const bool tab = S.m + S.n <= tab_ints;
      if (tab) {
        for (int x = threadIdx.x; x < S.m + S.n; x += blockDim.x) s_tab[x] = step_offset(S, x);
        __syncthreads();
      }
      for (int o = threadIdx.x; o < mn; o += blockDim.x) {
        const int i = o / S.n, j = o - i * S.n;
        const float* A = ar + S.a + i * S.k;
        const float* B = ar + S.b + j * S.k;
        // max-plus (real, unscaled): the semiring's zero is -inf, its product +
        float cr = MAXPLUS ? __int_as_float(0xff800000) : 0.f, ci = 0.f;
        for (int t = 0; t < S.k; ++t) {
          if (CPLX) {
            const float xr = A[t], xi = A[S.a_size + t], yr = B[t], yi = B[S.b_size + t];
            cr = fmaf(xr, yr, fmaf(-xi, yi, cr));
            ci = fmaf(xr, yi, fmaf(xi, yr, ci));
          } else if (MAXPLUS) {
            cr = fmaxf(cr, A[t] + B[t]);
          } else {
            cr = fmaf(A[t], B[t], cr);
          }
        }
        const int off = tab ? s_tab[i] + s_tab[S.m + j] : step_offset(S, i) + step_offset(S, S.m + j);
        ar[S.c + off] = cr;
        if (CPLX) ar[S.c + S.c_size + off] = ci;
      }
      __syncthreads();
      if (scaling) renormalise<CPLX>(ar + S.c, S.c_size, &s_max, &s_log);
    }
    if (threadIdx.x == 0) {
      // scalar results (closed networks): value and log2 scale
      values[2 * (int64_t)w] = ar[net.root];
      values[2 * (int64_t)w + 1] = CPLX ? ar[net.root + net.root_size] : 0.0;
      logs[w] = double(s_log) * 0.69314718055994530942;
    }
    __syncthreads();
  }
}

// The warp-per-network form of batch_kernel (K-FUSE): each warp takes networks from the
// queue and runs a whole path with warp-synchronous steps -- no block barriers between
// steps, and as many networks in flight per SM as resident warps. The same tables, the
// same arithmetic per output element (one lane, k in order) and the same exact power-of-two
// renormalisation, so a network's value does not depend on the form that computed it.
template <bool CPLX>
__device__ int warp_renormalise(float* t, int size, int lane) {
  int lmax = -127;
  for (int i = lane; i < size; i += 32) {
    float v = fabsf(t[i]);
    if (CPLX) v = fmaxf(v, fabsf(t[size + i]));
    lmax = max(lmax, bexp_of(v));
  }
  for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  const int e = lmax < -126 ? 0 : lmax;  // an all-zero tensor is left as is
  if (e != 0) {
    const float sc = bpow2_neg(e);
    for (int i = lane; i < size; i += 32) {
      t[i] *= sc;
      if (CPLX) t[size + i] *= sc;
    }
  }
  __syncwarp();
  return e;
}

template <bool CPLX, bool MAXPLUS = false>
__global__ void batch_warp_kernel(const BNet* __restrict__ nets, const BLeaf* __restrict__ leaves,
                                  const BStep* __restrict__ steps, int32_t n_nets, const float* __restrict__ in,
                                  float* arena, int32_t* queue, int32_t scaling, double* values, double* logs,
                                  int32_t smem_arena, int32_t tab_ints) {
  // dynamic shared memory: [arenas: smem_arena floats per warp | tables: tab_ints ints per warp]
  extern __shared__ float s_arena[];
  const int lane = threadIdx.x & 31;
  int* s_tab = reinterpret_cast<int*>(s_arena + smem_arena * (blockDim.x >> 5)) + (threadIdx.x >> 5) * tab_ints;
  while (true) {
    int w = 0;
    if (lane == 0) w = atomicAdd(queue, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= n_nets) break;
    const BNet net = nets[w];
    float* ar = net.arena_floats <= smem_arena ? s_arena + (threadIdx.x >> 5) * smem_arena : arena + net.arena;
    long long slog = 0;
    for (int l = 0; l < net.n_leaves; ++l) {
      const BLeaf& L = leaves[net.leaf0 + l];
      for (int e = lane; e < L.size; e += 32) {
        int r = e, src = 0;
        for (int d = L.rank - 1; d >= 0; --d) {
          src += (r % L.ext[d]) * L.sstride[d];
          r /= L.ext[d];
        }
        if (CPLX) {
          const float2 v = reinterpret_cast<const float2*>(in)[L.src + src];
          ar[L.dst + e] = v.x;
          ar[L.dst + L.size + e] = v.y;
        } else {
          ar[L.dst + e] = in[L.src + src];
        }
      }
    }
    __syncwarp();
    if (scaling)
      for (int l = 0; l < net.n_leaves; ++l) {
        const BLeaf& L = leaves[net.leaf0 + l];
        slog += warp_renormalise<CPLX>(ar + L.dst, L.size, lane);
      }
    for (int s = 0; s < net.n_steps; ++s) {
      const BStep& S = steps[net.step0 + s];
      const int mn = S.m * S.n;
      const bool tab = S.m + S.n <= tab_ints;
      if (tab) {
        for (int x = lane; x < S.m + S.n; x += 32) s_tab[x] = step_offset(S, x);
        __syncwarp();
      }
      for (int o = lane; o < mn; o += 32) {
        const int i = o / S.n, j = o - i * S.n;
        const float* A = ar + S.a + i * S.k;
        const float* B = ar + S.b + j * S.k;
        float cr = MAXPLUS ? __int_as_float(0xff800000) : 0.f, ci = 0.f;
        for (int t = 0; t < S.k; ++t) {
          if (CPLX) {
            const float xr = A[t], xi = A[S.a_size + t], yr = B[t], yi = B[S.b_size + t];
            cr = fmaf(xr, yr, fmaf(-xi, yi, cr));
            ci = fmaf(xr, yi, fmaf(xi, yr, ci));
          } else if (MAXPLUS) {
            cr = fmaxf(cr, A[t] + B[t]);
          } else {
            cr = fmaf(A[t], B[t], cr);
          }
        }
        const int off = tab ? s_tab[i] + s_tab[S.m + j] : step_offset(S, i) + step_offset(S, S.m + j);
        ar[S.c + off] = cr;
        if (CPLX) ar[S.c + S.c_size + off] = ci;
      }
      __syncwarp();
      if (scaling) slog += warp_renormalise<CPLX>(ar + S.c, S.c_size, lane);
    }
    if (lane == 0) {
      values[2 * (int64_t)w] = ar[net.root];
      values[2 * (int64_t)w + 1] = CPLX ? ar[net.root + net.root_size] : 0.0;
      logs[w] = double(slog) * 0.69314718055994530942;
    }
    __syncwarp();
  }
}

}  // namespace
}  // namespace tn

using namespace tn;

struct tn_batch_s {
  int32_t n_nets = 0;
  bool cplx = false, scaling = false, maxplus = false;
  std::vector<BNet> nets;
  std::vector<BLeaf> leaves;
  std::vector<BStep> steps;
  std::vector<int64_t> leaf_offset;  // packed input offset of every leaf (+ total)
  int64_t arena_floats = 0;
  char* dev = nullptr;               // tables + arena + queue
  BNet* d_nets = nullptr;
  BLeaf* d_leaves = nullptr;
  BStep* d_steps = nullptr;
  float* d_arena = nullptr;
  int32_t* d_queue = nullptr;
  int threads = 128, ctas_per_sm = 4, num_sms = 148;
  int nets_per_cta = 1;              // > 1: one warp per network, this many warps per CTA
  int32_t smem_arena = 0;            // shared-memory arena per network slot (floats; 0: none)
  int64_t max_arena_floats = 0;      // largest network arena
  int32_t tab_ints = 0;              // offset-table ints per network slot
  double flops = 0;
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  const void* g_in = nullptr;
  void* g_vals = nullptr;
  void* g_logs = nullptr;
  cudaStream_t g_stream = nullptr;
};

namespace tn {

template <typename K>
cudaError_t set_smem(K kernel, int bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_batch_kernel(const BNet* nets, const BLeaf* leaves, const BStep* steps, int32_t n_nets,
                                const void* packed, float* arena, int32_t* queue, bool cplx, bool scaling,
                                bool maxplus, int threads, int grid, double* values, double* logs,
                                cudaStream_t st, bool warp, int32_t smem_arena, int32_t tab_ints) {
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  const float* in = static_cast<const float*>(packed);
  const int sc = scaling ? 1 : 0;
  // dynamic shared memory: an arena and an offset table per CTA, or per warp in the warp form
  const int smem = (smem_arena + tab_ints) * 4 * (warp ? threads / 32 : 1);
  if (warp) {
    if (cplx) {
      if (smem && (e = set_smem(batch_warp_kernel<true>, smem)) != cudaSuccess) return e;
      batch_warp_kernel<true><<<grid, threads, smem, st>>>(nets, leaves, steps, n_nets, in, arena, queue, sc, values,
                                                           logs, smem_arena, tab_ints);
    } else if (maxplus) {
      if (smem && (e = set_smem(batch_warp_kernel<false, true>, smem)) != cudaSuccess) return e;
      batch_warp_kernel<false, true><<<grid, threads, smem, st>>>(nets, leaves, steps, n_nets, in, arena, queue, 0,
                                                                  values, logs, smem_arena, tab_ints);
    } else {
      if (smem && (e = set_smem(batch_warp_kernel<false>, smem)) != cudaSuccess) return e;
      batch_warp_kernel<false><<<grid, threads, smem, st>>>(nets, leaves, steps, n_nets, in, arena, queue, sc,
                                                            values, logs, smem_arena, tab_ints);
    }
    return cudaGetLastError();
  }
  if (cplx) {
    if (smem && (e = set_smem(batch_kernel<true>, smem)) != cudaSuccess) return e;
    batch_kernel<true><<<grid, threads, smem, st>>>(nets, leaves, steps, n_nets, in, arena, queue, sc, values, logs,
                                                    smem_arena, tab_ints);
  } else if (maxplus) {
    if (smem && (e = set_smem(batch_kernel<false, true>, smem)) != cudaSuccess) return e;
    batch_kernel<false, true><<<grid, threads, smem, st>>>(nets, leaves, steps, n_nets, in, arena, queue, 0, values,
                                                           logs, smem_arena, tab_ints);
  } else {
    if (smem && (e = set_smem(batch_kernel<false>, smem)) != cudaSuccess) return e;
    batch_kernel<false><<<grid, threads, smem, st>>>(nets, leaves, steps, n_nets, in, arena, queue, sc, values,
                                                     logs, smem_arena, tab_ints);
  }
  return cudaGetLastError();
}

bool batch_template(const Plan& P, BatchTemplate& T, std::string& err) {
  if (P.n_slices != 1) {
    err = "sliced networks are not batched";
    return false;
  }
  if (!P.open_modes.empty()) {
    err = "open labels (closed networks only)";
    return false;
  }
  if (P.arena_bytes / 4 > (int64_t(1) << 30)) {
    err = "network too large for the batched kernel";
    return false;
  }
  auto foff = [&](int32_t t) { return static_cast<int32_t>(P.tensors[t].offset / 4); };
  T = BatchTemplate{};
  const int32_t root = P.n_leaves + (int32_t)P.steps.size() - 1;
  T.root = foff(root);
  T.root_size = (int32_t)P.tensors[root].size;
  for (int32_t t = 0; t < P.n_leaves; ++t) {
    const TensorRec& R = P.tensors[t];
    const LeafDesc& d = P.leafdesc[t];
    if (d.rank > kBMaxRank || R.split) {
      err = d.rank > kBMaxRank ? "leaf rank too large" : "split-BF16 operands (tensor-core steps)";
      return false;
    }
    BLeaf L{};
    L.src = T.input_elems;
    L.dst = foff(t);
    L.size = (int32_t)R.size;
    L.rank = d.rank;
    for (int r = 0; r < d.rank; ++r) {
      L.ext[r] = (int32_t)d.ext[r];
      L.sstride[r] = (int32_t)d.sstride[r];
    }
    int64_t full = 1;
    for (int32_t x : R.decl) full *= P.extent[x];
    T.input_elems += full;
    T.leaves.push_back(L);
  }
  for (const StepRec& st : P.steps) {
    if (st.rows.n > kBMaxDims || st.cols.n > kBMaxDims || st.cls == TN_CLASS_TC) {
      err = st.cls == TN_CLASS_TC ? "tensor-core steps" : "output interleaving too fine";
      return false;
    }
    BStep S{};
    S.a = foff(st.a);
    S.b = foff(st.b);
    S.c = foff(st.out);
    S.a_size = (int32_t)P.tensors[st.a].size;
    S.b_size = (int32_t)P.tensors[st.b].size;
    S.c_size = (int32_t)P.tensors[st.out].size;
    S.m = (int32_t)st.m;
    S.n = (int32_t)st.n;
    S.k = (int32_t)st.k;
    S.nr = (int8_t)st.rows.n;
    S.nc = (int8_t)st.cols.n;
    for (int d = 0; d < st.rows.n; ++d) {
      S.rext[d] = (int32_t)st.rows.ext[d];
      S.rstr[d] = (int32_t)st.rows.stride[d];
    }
    for (int d = 0; d < st.cols.n; ++d) {
      S.cext[d] = (int32_t)st.cols.ext[d];
      S.cstr[d] = (int32_t)st.cols.stride[d];
    }
    T.steps.push_back(S);
    T.max_tab = std::max<int32_t>(T.max_tab, static_cast<int32_t>(st.m + st.n));
    T.flops += (P.is_complex ? 8.0 : 2.0) * double(st.m) * double(st.n) * double(st.k);
  }
  T.arena_floats = (P.arena_bytes + 255) / 256 * 64;  // keep every arena 256-byte aligned
  return true;
}

}  // namespace tn

namespace {
constexpr int64_t kMaxSmemPerCta = 227 * 1024;  // dynamic shared memory one CTA may take
constexpr int64_t kSmemPerSm = 224 * 1024;      // what the SM's resident CTAs share (with headroom)

tn_status launch_batch(tn_batch_s* B, const void* packed, double* values, double* logs, cudaStream_t st) {
  const bool warp = B->nets_per_cta > 1;
  const int64_t ctas_needed = warp ? (B->n_nets + B->nets_per_cta - 1) / B->nets_per_cta : B->n_nets;
  const int grid = std::min<int64_t>(ctas_needed, (int64_t)B->num_sms * B->ctas_per_sm);
  const int threads = warp ? 32 * B->nets_per_cta : B->threads;
  cudaError_t e = launch_batch_kernel(B->d_nets, B->d_leaves, B->d_steps, B->n_nets, packed, B->d_arena, B->d_queue,
                                      B->cplx, B->scaling, B->maxplus, threads, grid, values, logs, st, warp,
                                      B->smem_arena, B->tab_ints);
  if (e != cudaSuccess) {
    set_error(std::string("batch kernel launch: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  return TN_OK;
}
}  // namespace

extern "C" {

tn_status tn_batch_plan(int32_t n_nets, const tn_network* nets, const tn_path* paths, tn_dtype_policy policy,
                        tn_batch_t* out) {
  if (n_nets <= 0 || !nets || !paths || !out) {
    set_error("tn_batch_plan: bad arguments");
    return TN_ERR_INVALID;
  }
  if (policy.prec != TN_C64_FP32_SIMT && policy.prec != TN_R32_FP32_SIMT) {
    set_error("tn_batch_plan: batched small networks run the FP32 form (C64_FP32_SIMT or R32_FP32_SIMT)");
    return TN_ERR_UNSUPPORTED;
  }
  auto B = std::make_unique<tn_batch_s>();
  B->n_nets = n_nets;
  B->cplx = policy.prec == TN_C64_FP32_SIMT;
  B->scaling = policy.exp_scaling != 0;
  B->maxplus = policy.semiring == TN_SEMIRING_MAXPLUS;
  if (B->maxplus && (B->cplx || B->scaling)) {
    set_error("tn_batch_plan: the max-plus semiring runs R32 without exponent scaling");
    return TN_ERR_UNSUPPORTED;
  }
  int64_t in_off = 0;
  tn_dtype_policy hp = policy;
  hp.flags |= TN_PLAN_HOST_ONLY;
  hp.max_slice_batch = 1;
  for (int32_t w = 0; w < n_nets; ++w) {
    Plan P;
    std::string err;
    tn_status s = build_plan(&nets[w], &paths[w], nullptr, 0, hp, P, err);
    if (s != TN_OK) {
      set_error("network " + std::to_string(w) + ": " + err);
      return s;
    }
    if (!P.open_modes.empty()) {
      set_error("tn_batch_plan: network " + std::to_string(w) + " has open labels (closed networks only)");
      return TN_ERR_UNSUPPORTED;
    }
    assign_workspace(P, 1);
    if (!P.workspace_ok) {
      set_error("tn_batch_plan: workspace self-check failed");
      return TN_ERR_INVALID;
    }
    BatchTemplate T;
    std::string why;
    if (!batch_template(P, T, why)) {
      set_error("tn_batch_plan: network " + std::to_string(w) + ": " + why);
      return TN_ERR_UNSUPPORTED;
    }
    BNet bn{};
    bn.arena = B->arena_floats;
    bn.leaf0 = (int32_t)B->leaves.size();
    bn.n_leaves = (int32_t)T.leaves.size();
    bn.step0 = (int32_t)B->steps.size();
    bn.n_steps = (int32_t)T.steps.size();
    bn.root = T.root;
    bn.root_size = T.root_size;
    bn.arena_floats = static_cast<int32_t>(T.arena_floats);
    for (BLeaf L : T.leaves) {
      B->leaf_offset.push_back(in_off + L.src);
      L.src += in_off;
      B->leaves.push_back(L);
    }
    in_off += T.input_elems;
    B->steps.insert(B->steps.end(), T.steps.begin(), T.steps.end());
    B->flops += T.flops;
    B->arena_floats += T.arena_floats;
    B->max_arena_floats = std::max(B->max_arena_floats, T.arena_floats);
    B->tab_ints = std::max(B->tab_ints, std::min(T.max_tab, kMaxTabInts));
    B->nets.push_back(bn);
  }
  B->leaf_offset.push_back(in_off);
  if ((policy.flags & TN_PLAN_HOST_ONLY) == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&B->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      set_error("tn_batch_plan: no CUDA device");
      return TN_ERR_CUDA;
    }
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t b_nets = al(sizeof(BNet) * B->nets.size()), b_leaves = al(sizeof(BLeaf) * B->leaves.size());
    const size_t b_steps = al(sizeof(BStep) * std::max<size_t>(1, B->steps.size()));
    const size_t b_arena = al(sizeof(float) * B->arena_floats);
    const size_t total = b_nets + b_leaves + b_steps + b_arena + 256;
    void* mem = nullptr;
    if (cudaMalloc(&mem, total) != cudaSuccess) {
      cudaGetLastError();
      set_error("tn_batch_plan: cudaMalloc failed");
      return TN_ERR_OOM;
    }
    B->dev = static_cast<char*>(mem);
    B->d_nets = reinterpret_cast<BNet*>(B->dev);
    B->d_leaves = reinterpret_cast<BLeaf*>(B->dev + b_nets);
    B->d_steps = reinterpret_cast<BStep*>(B->dev + b_nets + b_leaves);
    B->d_arena = reinterpret_cast<float*>(B->dev + b_nets + b_leaves + b_steps);
    B->d_queue = reinterpret_cast<int32_t*>(B->dev + b_nets + b_leaves + b_steps + b_arena);
    if (cudaMemcpy(B->d_nets, B->nets.data(), sizeof(BNet) * B->nets.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_leaves, B->leaves.data(), sizeof(BLeaf) * B->leaves.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        (!B->steps.empty() && cudaMemcpy(B->d_steps, B->steps.data(), sizeof(BStep) * B->steps.size(),
                                         cudaMemcpyHostToDevice) != cudaSuccess)) {
      cudaFree(mem);
      set_error("tn_batch_plan: table upload failed");
      return TN_ERR_CUDA;
    }
  }
  *out = B.release();
  return TN_OK;
}

tn_status tn_batch_info(tn_batch_t b, int64_t* leaf_offsets, double* flops, int32_t* threads,
                        int32_t* ctas_per_sm, int32_t* nets_per_cta, int32_t* smem_arena) {
  if (!b) {
    set_error("null batch");
    return TN_ERR_INVALID;
  }
  if (leaf_offsets) std::copy(b->leaf_offset.begin(), b->leaf_offset.end(), leaf_offsets);
  if (flops) *flops = b->flops;
  if (threads) *threads = b->threads;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (nets_per_cta) *nets_per_cta = b->nets_per_cta;
  if (smem_arena) *smem_arena = b->smem_arena;
  return TN_OK;
}

tn_status tn_batch_contract(tn_batch_t b, const void* packed_inputs, double* values, double* log_scales,
                            void* stream) {
  if (!b || !b->dev || !packed_inputs || !values || !log_scales) {
    set_error("tn_batch_contract: bad arguments (or a host-only batch)");
    return TN_ERR_INVALID;
  }
  return launch_batch(b, packed_inputs, values, log_scales, reinterpret_cast<cudaStream_t>(stream));
}

tn_status tn_batch_contract_graph(tn_batch_t b, const void* packed_inputs, double* values, double* log_scales,
                                  void* stream) {
  if (!b || !b->dev || !packed_inputs || !values || !log_scales) {
    set_error("tn_batch_contract_graph: bad arguments (or a host-only batch)");
    return TN_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!b->gexec || b->g_in != packed_inputs || b->g_vals != values || b->g_logs != log_scales ||
      b->g_stream != st) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("graph capture stream");
      return TN_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    tn_status s = TN_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = TN_ERR_CUDA;
    if (s == TN_OK) s = launch_batch(b, packed_inputs, values, log_scales, cap);
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (s == TN_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (s != TN_OK || e != cudaSuccess) {
      cudaGetLastError();
      set_error(std::string("batch graph capture failed: ") + cudaGetErrorString(e));
      return TN_ERR_CUDA;
    }
    b->g_in = packed_inputs;
    b->g_vals = values;
    b->g_logs = log_scales;
    b->g_stream = st;
  }
  cudaError_t e = cudaGraphLaunch(b->gexec, st);
  if (e != cudaSuccess) {
    set_error(std::string("graph launch: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  return TN_OK;
}

tn_status tn_batch_autotune(tn_batch_t b, const void* packed_inputs, double* values, double* log_scales,
                            void* stream) {
  if (!b || !b->dev) {
    set_error("tn_batch_autotune: bad batch");
    return TN_ERR_INVALID;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int cand_threads[] = {32, 64, 128, 256};
  const int cand_ctas[] = {2, 4, 8, 16};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bt = b->threads, bc = b->ctas_per_sm, bg = b->nets_per_cta;
  int32_t bs = b->smem_arena;
  // (threads per network, networks per CTA): a CTA per network at 32-256 threads, or a warp
  // per network with 4 or 8 warps per CTA
  struct Shape { int t, g; };
  std::vector<Shape> shapes;
  for (int t : cand_threads) shapes.push_back({t, 1});
  shapes.push_back({32, 4});
  shapes.push_back({32, 8});
  // shared-memory arena per network slot: none, or the largest that c CTAs of g slots fit
  // (networks above it keep their global arenas), no larger than the largest arena
  for (const Shape& sh : shapes)
    for (int c : cand_ctas)
      for (int sm = 0; sm < 2; ++sm) {
      const int cta_threads = sh.g > 1 ? 32 * sh.g : sh.t;
      if (cta_threads * c > 2048) continue;
      int64_t cap = 0;
      const int64_t per_slot = std::min<int64_t>(kSmemPerSm / (4 * sh.g * c), kMaxSmemPerCta / (4 * sh.g));
      if (per_slot < b->tab_ints) continue;  // the offset tables alone do not fit this shape
      if (sm) {
        cap = std::min<int64_t>(per_slot - b->tab_ints, b->max_arena_floats) / 64 * 64;
        if (cap < 64) continue;
      }
      b->threads = sh.t;
      b->nets_per_cta = sh.g;
      b->ctas_per_sm = c;
      b->smem_arena = static_cast<int32_t>(cap);
      float ms_best = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        tn_status s = launch_batch(b, packed_inputs, values, log_scales, st);
        cudaEventRecord(e1, st);
        if (s != TN_OK || cudaEventSynchronize(e1) != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          set_error("tn_batch_autotune: a candidate failed");
          return TN_ERR_CUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_best = std::min(ms_best, ms);
      }
      if (ms_best < best) {
        best = ms_best;
        bt = sh.t;
        bg = sh.g;
        bc = c;
        bs = b->smem_arena;
      }
    }
  b->threads = bt;
  b->nets_per_cta = bg;
  b->ctas_per_sm = bc;
  b->smem_arena = bs;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return TN_OK;
}

tn_status tn_batch_set_shape(tn_batch_t b, int32_t threads, int32_t ctas_per_sm, int32_t nets_per_cta,
                             int32_t smem_arena) {
  const bool warp = nets_per_cta > 1;
  const int cta_threads = warp ? 32 * nets_per_cta : threads;
  if (!b || ctas_per_sm < 1 || nets_per_cta < 1 || (warp && threads != 32) || cta_threads < 32 ||
      cta_threads > 1024 || cta_threads % 32 != 0 || cta_threads * ctas_per_sm > 2048 ||
      smem_arena < 0 || int64_t(smem_arena + b->tab_ints) * 4 * nets_per_cta > kMaxSmemPerCta ||
      int64_t(smem_arena + b->tab_ints) * 4 * nets_per_cta * ctas_per_sm > kSmemPerSm) {
    set_error("tn_batch_set_shape: bad launch shape");
    return TN_ERR_INVALID;
  }
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  b->nets_per_cta = nets_per_cta;
  b->smem_arena = smem_arena;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  return TN_OK;
}

tn_status tn_batch_destroy(tn_batch_t b) {
  if (!b) return TN_OK;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->dev) cudaFree(b->dev);
  delete b;
  return TN_OK;
}

}  // extern "C"
