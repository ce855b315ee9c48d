// Tables of the batched small-network engine (batch.cu), shared with the serve loop,
// which packs compatible small requests into one launch of the same kernel.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "tn_internal.h"

namespace tn {

constexpr int kBMaxDims = 8;    // merged offset dims per side in the batch tables
constexpr int kBMaxRank = 8;    // planned leaf rank in the batch tables

struct BLeaf {
  int64_t src;                  // element offset in the packed input buffer
  int32_t dst;                  // float offset in the network's arena (real plane)
  int32_t size;
  int32_t rank;
  int32_t pad;
  int32_t ext[kBMaxRank];
  int32_t sstride[kBMaxRank];   // declared stride of each planned position
};

struct BStep {
  int32_t a, b, c;              // float offsets in the arena (real planes)
  int32_t a_size, b_size, c_size;
  int32_t m, n, k;
  int8_t nr, nc;
  int16_t pad;
  int32_t rext[kBMaxDims], rstr[kBMaxDims];
  int32_t cext[kBMaxDims], cstr[kBMaxDims];
};

struct BNet {
  int64_t arena;                // float offset of the network's arena in the batch arena
  int32_t leaf0, n_leaves;      // index range in the leaf table
  int32_t step0, n_steps;       // index range in the step table
  int32_t root, root_size;      // float offset and size of the result tensor
  int32_t arena_floats;         // size of the network's arena
  int32_t pad;
};

// One network's tables, offsets relative to the network itself (arena floats from 0,
// leaf sources from 0 in the network's own packed inputs, leaf and step indices from 0).
struct BatchTemplate {
  std::vector<BLeaf> leaves;
  std::vector<BStep> steps;
  int64_t arena_floats = 0;     // 256-byte aligned
  int64_t input_elems = 0;      // elements of the network's packed inputs
  int32_t root = 0, root_size = 0;
  int32_t max_tab = 0;          // largest m + n of its steps (the offset table it needs)
  double flops = 0;
};

// offset-table entries per network slot at most (steps with larger m + n compute offsets
// element by element)
constexpr int32_t kMaxTabInts = 4096;

// Tables of a closed, unsliced network from its plan (workspace assigned for one copy, no
// tensor-core steps); false with a reason when the batched kernel cannot run it.
bool batch_template(const Plan& P, BatchTemplate& T, std::string& err);

// Launch the persistent kernel over n_nets networks (queue reset included): a CTA of
// `threads` per network, or with `warp` a warp per network (threads = 32 x warps per CTA).
// smem_arena > 0: a network whose arena holds at most smem_arena floats runs in a
// shared-memory arena of that size (one per CTA, or per warp), the others in `arena`.
// tab_ints > 0: each slot also gets a shared-memory table of that many ints for the output
// offsets of a step's rows and columns (steps with m + n above it compute them per element).
cudaError_t launch_batch_kernel(const BNet* nets, const BLeaf* leaves, const BStep* steps, int32_t n_nets,
                                const void* packed, float* arena, int32_t* queue, bool cplx, bool scaling,
                                bool maxplus, int threads, int grid, double* values, double* logs,
                                cudaStream_t st, bool warp = false, int32_t smem_arena = 0, int32_t tab_ints = 0);

}  // namespace tn
