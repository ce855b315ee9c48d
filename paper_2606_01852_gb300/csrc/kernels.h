// Launch interface of the device kernels (internal).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "tn_internal.h"

namespace tn {

// Output offset of GEMM row (or column) idx under a separable offset map: the mixed-radix
// digits of idx over the map's extents (last fastest), each times its stride. Indices
// below 2^32 take 32-bit digits, and a power-of-two extent a shift and a mask, instead of
// 64-bit division (the same values, a fraction of the instructions).
__host__ __device__ inline int64_t map_offset(const OffsetMap& om, int64_t idx) {
  int64_t off = 0;
  if (idx >= 0 && idx <= int64_t(0xffffffff)) {
    uint32_t i = static_cast<uint32_t>(idx);
    for (int d = om.n - 1; d >= 0; --d) {
      const uint32_t e = om.ext[d];
      uint32_t q, r;
      if ((e & (e - 1u)) == 0u) {
#ifdef __CUDA_ARCH__
        const int sh = __ffs(static_cast<int>(e)) - 1;
#else
        const int sh = __builtin_ctz(e);
#endif
        q = i >> sh;
        r = i & (e - 1u);
      } else {
        q = i / e;
        r = i - q * e;
      }
      off += int64_t(r) * om.stride[d];
      i = q;
    }
    return off;
  }
  for (int d = om.n - 1; d >= 0; --d) {
    const uint32_t e = om.ext[d];
    off += (idx % e) * om.stride[d];
    idx /= e;
  }
  return off;
}

// Per tensor (and per batch entry of a batched tensor): the largest binary exponent
// of the stored values, and the power of two the stored values must be multiplied by
// to give the true tensor (exponent scaling).
struct ScaleRec {
  int32_t emax;
  int32_t pad;
  int64_t log2;
};

// One pairwise step C[b] = A[b] (m x k, row-major) . B[b] (n x k, row-major)^T.
// Planar complex: the imaginary plane of each tensor copy follows its real plane at
// +*_plane floats. C is written at rows(m) + cols(n). Batch strides are 0 for tensors
// that do not depend on a sliced label. c_split is C's storage mode (split_bf16.cuh):
// planar FP32, the four BF16 planes of the split form (the operand layout of a 4M BF16x3
// step) or the six planes of the 3M split form; batch strides count floats (2 or 3 per
// complex element).
struct StepArgs {
  const float* A;
  const float* B;
  float* C;
  int64_t m, n, k;
  int64_t a_bstride, b_bstride, c_bstride;  // floats
  int64_t a_plane, b_plane, c_plane;        // floats
  OffsetMap rows, cols;
  ScaleRec* recs;                           // null: no exponent scaling
  int32_t rec_a, rec_b, rec_c;
  int32_t c_split;                          // C's storage mode: 0 planar, 1 split, 2 split 3M
  int32_t maxplus;                          // 1: (max, +) semiring (real, unscaled)
  int32_t ksplit;                           // SIMT: k cut in ksplit parts (partials in `part`)
  float* part;                              // ksplit * nb * planes * m * n floats, or null
};

// A run of consecutive tiny CUDA-core steps executed by one CTA in one launch (the step
// chain): each step's StepArgs as for launch_contract_simt, and whether it is batched.
struct ChainStep {
  StepArgs a;
  int32_t batched;
  int32_t pad;
};
// A chain step's work bound: m n k (x the slice batch when batched) at most this many
// multiply-adds (complex ones count four).
constexpr int64_t kChainMaxWork = int64_t(1) << 16;
// steps[0 .. n): the run, in path order; nb: slices of this pass; skip_unbatched: a pass
// after the first (the slice-invariant steps were computed by the first and are kept).
// Every step's outputs are the same bits as launch_contract_simt's (k summed in order by FMA).
void launch_contract_chain(const ChainStep* steps, int32_t n, int32_t nb, bool skip_unbatched, bool cplx,
                           bool maxplus, cudaStream_t st);

// Small leaves: one CTA per leaf. Large leaves (LeafDesc::tiled): the tiled permutation
// kernel, one launch per leaf; host_descs is the host copy of the table (grid sizes).
void launch_stage_leaves(const LeafDesc* descs, const LeafDesc* host_descs, int32_t n_leaves, char* ws,
                         int64_t slice_begin, int32_t nb, bool only_batched, bool is_complex, ScaleRec* recs,
                         const int32_t* rec_index, cudaStream_t st);
// With a.ksplit > 1 each part of k goes to its own CTAs and a second kernel combines the
// partial tiles (in part order) and writes C.
void launch_contract_simt(const StepArgs& a, int32_t nb, bool cplx, cudaStream_t st);
// k parts for a SIMT step of m x n outputs per batch entry, `copies` entries, depth k on
// num_sms SMs (1 = no split: at least 2 x num_sms tiles, k < 2048, or a scaled step)
int32_t simt_ksplit(int64_t m, int64_t n, int64_t k, int64_t copies, int num_sms, bool scaled);
// err: the plan's error word (the bulk-copy form records an expired wait there)
void launch_contract_stream(const StepArgs& a, int32_t nb, bool cplx, int num_sms, int* err, cudaStream_t st);

// split-K steps: at most kSplitMaxOut outputs, k cut in chunks of kSplitChunk; scratch
// holds nb * splitk_chunks(k) * m*n complex doubles
constexpr int kSplitMaxOut = 16;
constexpr int64_t kSplitChunk = 4096;
int32_t splitk_chunks(int64_t k);
void launch_contract_splitk(const StepArgs& a, int32_t nb, bool cplx, double* scratch, cudaStream_t st);
// maxplus: the slices combine by maximum instead of the compensated sum; last: this pass
// writes the result (FP64, complex interleaved) to out and the log scale, not to acc
void launch_accumulate_root(const float* root, int64_t size, int32_t nb, int64_t bstride,
                            int64_t plane, bool cplx, double* acc, const ScaleRec* recs,
                            int32_t rec_root, bool root_batched, int64_t* ref_exp, bool first, bool last,
                            bool maxplus, void* out, double* log_scale, int num_sms, cudaStream_t st);

// tensor-core path (tcgen05); returns false if the step cannot take it
bool tc_supported();
cudaError_t launch_bounded_wait_selftest(int arrive, uint64_t limit_ns, int* err, cudaStream_t st);
// A and B of a BF16X3 step are in the split-BF16 form; prec = kPrecBF16x3M selects the 3M
// kernel (operands in the 3M split form).
constexpr int32_t kPrecBF16x3M = 103;
// pairs: BF16x3 4M steps with m >= 256 and k above the persistent kernel's range run on
// pairs of SMs (contract_tcb2_kernel). cplx false: a real step (TF32 and 3xTF32 forms).
// a.recs (exponent scaling): every form but the 3M product (a scaled BF16x3 4M step runs
// contract_tcb_kernel, one SM per tile, for every k).
cudaError_t launch_contract_tc(const StepArgs& a, int32_t nb, int32_t prec, bool cplx, int* err,
                               cudaStream_t st, bool pairs = true);
// kernel launches launch_contract_tc makes for such a step (more than one for the deep
// steps, launched in bands of tiles)
int64_t tc_launches(int64_t m, int64_t n, int64_t k, int32_t nb, int32_t prec, bool pairs, bool scaled);
// The TF32 and 3xTF32 forms (gemm_tf32.cu), complex (prec TN_C64_TF32 / TN_C64_3XTF32) or
// real (TN_R32_TF32 / TN_R32_3XTF32, cplx false), with exponent scaling when a.recs is set;
// and the launches such a step makes.
cudaError_t launch_contract_tf32(const StepArgs& a, int32_t nb, int32_t prec, bool cplx, int* err,
                                 cudaStream_t st);
int64_t tf32_launches(int64_t m, int64_t n, int32_t nb, bool real);

}  // namespace tn
