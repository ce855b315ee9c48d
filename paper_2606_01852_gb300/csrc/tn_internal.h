// Internal declarations shared by the planner, the executor and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tn.h"

namespace tn {

constexpr int kMaxDims = 12;     // merged output-offset dims per GEMM side
constexpr int kMaxLeafRank = 32; // planned rank of a leaf the staging kernels handle
constexpr int kMaxSliced = 24;   // sliced labels carried by one leaf

// Maps a GEMM row (or column) index to an output offset: the index is read as
// mixed radix over `n` merged dims (last dim fastest) and each digit is scaled by
// that dim's output stride. Sec. IV-A lets an output interleave the modes of its two
// operands; this is how the kernels write such an output without a transpose.
struct OffsetMap {
  int32_t n;
  uint32_t ext[kMaxDims];
  int64_t stride[kMaxDims];
};

// Per-leaf staging descriptor (a4): copy leaf t from its declared order into its
// planned order, fixing sliced labels from the slice id, and split complex64 into
// planar float32 (re plane, im plane).
struct LeafDesc {
  const void* src;          // caller's leaf, declared order
  int64_t dst;              // byte offset of the staged tensor in the workspace
  int64_t size;             // elements of one staged copy (sliced labels removed)
  int32_t rank;             // planned rank
  int32_t batched;          // carries a sliced label
  int32_t n_sl;             // sliced labels on this leaf
  int32_t split;            // storage mode of the staged copy (0 planar, 1 split, 2 split 3M)
  uint32_t ext[kMaxLeafRank];      // planned extents
  int64_t sstride[kMaxLeafRank];   // source stride (elements) of each planned position
  int64_t sl_div[kMaxSliced];      // slice id -> label value: (sid / div) % ext
  uint32_t sl_ext[kMaxSliced];
  int64_t sl_stride[kMaxSliced];   // source stride of that sliced label
  // Tiled permutation (large leaves): the planned positions split into three groups --
  // the output group (the trailing `no` planned positions, contiguous in the staged
  // copy), the input group (ipos[0..ni-1], the fastest-varying positions of the declared
  // order outside the output group, slowest first) and the rest (rpos[0..nr-1]). A CTA
  // moves one 32 x 32 tile (output-group index x input-group index) through shared
  // memory, reading along the input group and writing along the output group.
  int32_t tiled;                   // staged by the tiled kernel (else by the per-leaf kernel)
  int32_t no, ni, nr;
  int32_t load_o;                  // the declared order's innermost position is in the
                                   // output group: load along it instead
  int32_t vec_load;                // input group's fastest position has source stride 1
                                   // and an even extent: two elements per 16-byte load
  int64_t Po, Pi, Pr;              // extents of the three groups
  int32_t fast;                    // the pipelined form applies: Po = Pi = 32, 16-byte loads, and
                                   // the last `nlo` rest positions span exactly the tiles of a CTA
  int32_t nlo;
  int8_t ipos[kMaxLeafRank], rpos[kMaxLeafRank];
  int64_t dstride[kMaxLeafRank];   // stride of each planned position in the staged copy
};
// leaves of at least this many elements (per copy) are staged by the tiled kernel
constexpr int64_t kTiledLeafElems = 2048;

struct TensorRec {
  std::vector<int32_t> decl;   // declared modes (leaves only; incl. sliced)
  std::vector<int32_t> modes;  // planned order, sliced labels removed
  int64_t size = 1;            // elements per slice
  bool batched = false;
  int32_t producer = -1;       // step, or -1 for a leaf
  int32_t consumer = -1;       // step, or -1 for the root
  bool pinned = false;         // unbatched, consumed by a batched step: kept for all passes
  int32_t split = 0;           // storage mode (split_bf16.cuh): 0 planar FP32, 1 split BF16
                               // (its consumer is a 4M BF16x3 step), 2 split BF16 with the
                               // 3M sum planes (its consumer is a 3M BF16x3 step)
  int64_t offset = 0;          // byte offset in the workspace
  int64_t bytes = 0;           // bytes including the batch copies
};

struct StepRec {
  int32_t a = -1, b = -1, out = -1;  // SSA ids; a is the row operand
  std::vector<int32_t> M, N, K;
  int64_t m = 1, n = 1, k = 1;
  int32_t cls = TN_CLASS_SIMT;
  bool batched = false;
  OffsetMap rows{}, cols{};
  int32_t ksplit = 1;  // SIMT steps too few tiles to fill the GPU: k cut in this many parts
  bool single_sm = false;  // tensor-core step kept on one SM per tile (tn_plan_autotune's choice)
  int32_t chain = -1;      // index of the step chain (a run of tiny CUDA-core steps) it is in
};

// A step chain: steps first .. first + n - 1 run in one launch (entries table .. table + n - 1
// of the device table at off_chain)
struct ChainRec {
  int32_t first = 0, n = 0, table = 0;
  bool any_batched = false;
};

struct Plan {
  // network
  int32_t n_leaves = 0, n_labels = 0;
  std::vector<int64_t> extent;
  std::vector<int32_t> open_modes;
  std::vector<int32_t> sliced;
  std::vector<int64_t> slice_div;   // per sliced label position
  int64_t n_slices = 1;
  bool is_complex = true;
  tn_dtype_policy policy{};
  // plan
  std::vector<TensorRec> tensors;   // SSA ids
  std::vector<StepRec> steps;
  int64_t batch = 1;                // slices per pass
  int64_t arena_bytes = 0;
  int64_t out_elems = 1;
  // workspace regions (byte offsets from the workspace base)
  int64_t off_acc = 0;              // FP64 Neumaier accumulator: [sum, comp] x re/im x out
  int64_t off_scale = 0;            // per tensor x batch: int32 emax, int32 pad, int64 log2
  int64_t off_recidx = 0;           // int32 record index of each leaf (device copy)
  int64_t off_ref = 0;              // int64 reference exponent of the accumulator
  int64_t off_err = 0;              // int error word set by kernels whose bounded waits expire
  int64_t off_scratch = 0;          // split-K partial sums (complex double)
  int64_t scratch_bytes = 0;
  std::vector<int32_t> rec_index;   // per tensor: first scale record
  int64_t n_rec_unbatched = 0, n_rec_total = 0;
  int64_t off_leafdesc = 0;         // LeafDesc table
  int64_t off_chain = 0;            // ChainStep table of the step chains
  std::vector<ChainRec> chains;
  int64_t off_stage_in = 0;         // device copies of host inputs (tn_contract_host)
  std::vector<int64_t> stage_in_off;
  int64_t total_bytes = 0;
  bool workspace_ok = false;        // liveness assignment passed its self-check
  // device state
  char* dev = nullptr;
  std::vector<LeafDesc> leafdesc;   // host copy; src filled per call
  int num_sms = 148;
  // per-class timing (tn_plan_profile): event pairs around step launches
  struct ProfRec {
    void* e0;
    void* e1;
    int32_t cls;
    int32_t step;
    double flops, bytes;
  };
  bool prof_on = false;
  std::vector<ProfRec> prof_pending;
  std::vector<void*> prof_pool;
  tn_profile prof_acc{};
  std::vector<double> prof_step_ms, prof_last_step_ms;
  uint64_t uid = 0;                 // unique per plan (serve pools key on it)
  // tn_contract_graph: the captured call (graph exec), the pointers and stream it was
  // captured for, a pinned copy of the leaf descriptors and scale-record indices its copy
  // nodes read, and an event after its last launch (the pinned copy is rewritten only
  // after that event)
  void* g_exec = nullptr;
  std::vector<const void*> g_inputs;
  void* g_out = nullptr;
  double* g_ls = nullptr;
  void* g_stream = nullptr;
  void* g_pinned = nullptr;
  void* g_done = nullptr;
  // stats
  tn_plan_stats stats{};
};

// rates of the planner's kernel choice (process-wide; tn_cost_model_set)
extern tn_cost_model g_cost;

// planner (host only)
tn_status build_plan(const tn_network* net, const tn_path* path, const int32_t* sliced,
                     int32_t n_sliced, const tn_dtype_policy& pol, Plan& P, std::string& err);
// liveness assignment of workspace offsets for a given slice batch
void assign_workspace(Plan& P, int64_t batch);

// executor
// pinned: null (descriptors copied from pageable host memory, staged before the call
// returns), or a pinned buffer of sizeof(LeafDesc) x n_leaves + 4 x n_leaves bytes that the
// descriptor and record-index copies read from (capturable in a CUDA graph)
tn_status run_slices(Plan& P, const void* const* inputs, int64_t begin, int64_t count,
                     void* output, double* log_scale, void* stream, std::string& err,
                     void* pinned = nullptr);

void set_error(const std::string& msg);
tn_status check_device_error(Plan& P);
// writes the step chains' ChainStep table into the workspace (once P.dev is set)
tn_status upload_chain_table(Plan& P);

// true when the tcgen05 kernels are compiled in
bool tc_supported();
// the tensor-core kernel's shape limits for a step (rows m, columns n, depth k) in form prec
bool tc_step_ok(int64_t m, int64_t n, int64_t k, int32_t prec);

inline int64_t elem_bytes(const Plan& P) { return P.is_complex ? 8 : 4; }
// bytes per element of a tensor's stored copies (the 3M split form holds 12)
inline int64_t stored_bytes(const Plan& P, const TensorRec& R) {
  return P.is_complex ? (R.split == 2 ? 12 : 8) : 4;
}

}  // namespace tn

// opaque handle of the C ABI
struct tn_plan_s {
  tn::Plan P;
};
