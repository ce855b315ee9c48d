// Allocation-free batched dot products: tn_dot_noalloc.
//
// Some callers cannot allocate device memory on the path that calls this library: a
// host process whose device memory is already handed out by another allocator, or a
// latency-critical loop where cudaMalloc (which may synchronize the device) is not
// acceptable. For them this entry point computes a reduction of the same shape as the
// engine's split-K step for few-output steps (k cut in chunks, FP64 partials, chunks
// added in order) with its own pair of kernels and without the plan workspace: its FP64
// partial sums live in one file-scope device array of fixed size.
//
// The array is shared by every call in the process. Each call overwrites every
// partial it later reads (nothing has to start at zero), so calls that run one after
// another need no clearing; calls that overlap on the GPU (different streams, or
// host threads without ordering) race on it.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "kernels.h"
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int64_t kNoAllocSlots = int64_t(1) << 18;  // complex-double partials: 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocSlots];

std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id;  // context the address belongs to (0: not looked up)
  double2* ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

// Driver calls reached through the runtime's entry-point table (no -lcuda link): the id
// of the current context tells whether a cached address still belongs to it.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  }
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's context. It is looked up
// (cudaGetSymbolAddress) on the first call with that context current, and again when the
// context has changed since (the device was reset and its primary context re-created),
// since an address cached for a destroyed context no longer points at the array.
cudaError_t scratch_address(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  ScratchAddr& c = g_scratch_addr[dev];
  unsigned long long ctx = 0;
  // no context bound to this thread yet, or a different one: look the address up (which
  // also makes the device's primary context current) and record the context it is for
  if (!current_context_id(&ctx) || !c.ptr || c.ctx_id != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    c.ptr = static_cast<double2*>(p);
    c.ctx_id = current_context_id(&ctx) ? ctx : 0;  // 0: looked up again on every call
  }
  *out = c.ptr;
  return cudaSuccess;
}

// partial[b][chunk][i*n+j] = sum over the chunk's k of a[b][i][t] * b[b][j][t]
__global__ void __launch_bounds__(256) dot_partial_kernel(const float2* __restrict__ A, const float2* __restrict__ B,
                                                          int64_t m, int64_t n, int64_t k, int32_t chunks,
                                                          double2* scratch) {
  const int chunk = blockIdx.x, b = blockIdx.y;
  const int mn = (int)(m * n);
  const float2* a = A + (int64_t)b * m * k;
  const float2* bb = B + (int64_t)b * n * k;
  float accr[kSplitMaxOut], acci[kSplitMaxOut];
#pragma unroll
  for (int o = 0; o < kSplitMaxOut; ++o) accr[o] = acci[o] = 0.f;
  const int64_t k0 = (int64_t)chunk * kSplitChunk;
  const int64_t k1 = min(k, k0 + kSplitChunk);
  for (int64_t t = k0 + threadIdx.x; t < k1; t += blockDim.x) {
#pragma unroll
    for (int o = 0; o < kSplitMaxOut; ++o) {
      if (o >= mn) break;
      const float2 x = a[(o / n) * k + t];
      const float2 y = bb[(o % n) * k + t];
      accr[o] = fmaf(x.x, y.x, fmaf(-x.y, y.y, accr[o]));
      acci[o] = fmaf(x.x, y.y, fmaf(x.y, y.x, acci[o]));
    }
  }
  __shared__ double red[2][kSplitMaxOut][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < kSplitMaxOut; ++o) {
    if (o >= mn) break;
    double vr = accr[o], vi = acci[o];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      vr += __shfl_xor_sync(0xffffffffu, vr, s);
      vi += __shfl_xor_sync(0xffffffffu, vi, s);
    }
    if (lane == 0) {
      red[0][o][warp] = vr;
      red[1][o][warp] = vi;
    }
  }
  __syncthreads();
  if (threadIdx.x < mn) {
    double vr = 0.0, vi = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      vr += red[0][threadIdx.x][w];
      vi += red[1][threadIdx.x][w];
    }
    scratch[((int64_t)b * chunks + chunk) * mn + threadIdx.x] = make_double2(vr, vi);
  }
}

// out[b][o] = sum over chunks, in chunk order, of the partials
__global__ void dot_final_kernel(const double2* scratch, int32_t mn, int32_t chunks, double2* out) {
  const int b = blockIdx.x;
  for (int o = threadIdx.x; o < mn; o += blockDim.x) {
    double vr = 0.0, vi = 0.0;
    for (int c = 0; c < chunks; ++c) {
      const double2 p = scratch[((int64_t)b * chunks + c) * mn + o];
      vr += p.x;
      vi += p.y;
    }
    out[(int64_t)b * mn + o] = make_double2(vr, vi);
  }
}

}  // namespace
}  // namespace tn

extern "C" tn_status tn_dot_noalloc(const void* a, const void* b, int64_t batch, int64_t m, int64_t n, int64_t k,
                                    void* out, void* stream) {
  using namespace tn;
  if (!a || !b || !out || batch < 1 || m < 1 || n < 1 || k < 1) {
    set_error("tn_dot_noalloc: null pointer or non-positive size");
    return TN_ERR_INVALID;
  }
  // m and n are bounded one at a time first, so that m * n cannot overflow
  if (m > kSplitMaxOut || n > kSplitMaxOut || m * n > kSplitMaxOut) {
    set_error("tn_dot_noalloc: m = " + std::to_string(m) + ", n = " + std::to_string(n) +
              ": m*n exceeds the maximum of " + std::to_string(kSplitMaxOut) + " outputs per batch entry");
    return TN_ERR_INVALID;
  }
  if (batch > 65535) {
    set_error("tn_dot_noalloc: batch exceeds 65535");
    return TN_ERR_INVALID;
  }
  // chunks <= kNoAllocSlots before the product, so batch * chunks * m*n stays below 2^43
  const int64_t chunks = k / kSplitChunk + (k % kSplitChunk != 0);
  if (chunks > kNoAllocSlots || batch * chunks * m * n > kNoAllocSlots) {
    set_error("tn_dot_noalloc: batch * ceil(k/4096) * m*n partial sums (batch " + std::to_string(batch) +
              ", " + std::to_string(chunks) + " chunks, " + std::to_string(m * n) +
              " outputs) exceed the fixed scratch of " + std::to_string(kNoAllocSlots));
    return TN_ERR_INVALID;
  }
  double2* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    set_error(std::string("tn_dot_noalloc: scratch set-up failed: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid(static_cast<unsigned>(chunks), static_cast<unsigned>(batch));
  dot_partial_kernel<<<grid, 256, 0, st>>>(static_cast<const float2*>(a), static_cast<const float2*>(b), m, n, k,
                                           static_cast<int32_t>(chunks), scratch);
  dot_final_kernel<<<static_cast<unsigned>(batch), 32, 0, st>>>(scratch, static_cast<int32_t>(m * n),
                                                                static_cast<int32_t>(chunks),
                                                                static_cast<double2*>(out));
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("tn_dot_noalloc: launch failed: ") + cudaGetErrorString(e));
    return TN_ERR_CUDA;
  }
  return TN_OK;
}
