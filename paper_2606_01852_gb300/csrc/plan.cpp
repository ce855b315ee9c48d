// Host planner: step analysis (Sec. II-B), GEMM-oriented mode reordering (Sec. IV-A),
// kernel choice by the roofline cost model of Sec. IV-C, and workspace assignment by
// liveness. No CUDA calls here.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <set>
#include <sstream>

#include "kernels.h"
#include "staging.cuh"
#include "tn_internal.h"

namespace tn {

namespace {

constexpr int64_t kAlign = 256;
inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

bool tc_prec_built(int32_t p) {
  return p == TN_C64_TF32 || p == TN_C64_3XTF32 || p == TN_C64_BF16X3 || p == TN_R32_TF32 || p == TN_R32_3XTF32;
}

bool is_tc_prec(int32_t p) {
  return p == TN_C64_TF32 || p == TN_C64_3XTF32 || p == TN_C64_BF16X3 || p == TN_R32_TF32 ||
         p == TN_R32_3XTF32 || p == TN_R32_BF16X3;
}

}  // namespace

// Rates of the kernel choice (t = max(bytes/B, flops/F), Sec. IV-C Eq. 6): B the HBM copy
// rate, F per kernel family its peak in algorithmic flops (8 per complex MAC). Defaults:
// this part's measured copy rate and sustained dense BF16 rate (the BF16x3 form does three
// BF16 products per algorithmic one; TF32 is 1.1/2.25 of BF16, 3xTF32 a third of that) and
// the FP32 FMA rate of 152 SMs x 128 lanes at 1.9 GHz. tn_cost_model_set replaces them.
tn_cost_model g_cost = {6.8e12, 152.0 * 128.0 * 2.0 * 1.9e9, {1.7e15 * 1.1 / 2.25, 1.7e15 * 1.1 / 2.25 / 3.0,
                                                             1.7e15 / 3.0}};

namespace {

double tc_flops(int32_t p) {
  switch (p) {
    case TN_C64_TF32: case TN_R32_TF32: return g_cost.tc_flops[0];
    case TN_C64_3XTF32: case TN_R32_3XTF32: return g_cost.tc_flops[1];
    case TN_C64_BF16X3: case TN_R32_BF16X3: return g_cost.tc_flops[2];
    case -3: return g_cost.tc_flops[2] * 4.0 / 3.0;  // BF16x3, 3M: 9 BF16 products per complex MAC, not 12
    default: return 0;
  }
}

// Offsets of the output for the GEMM rows over labels `side` (in the operand's order,
// which is the output order restricted to those labels): merge maximal runs of labels
// that are consecutive in the output.
bool build_offset_map(const std::vector<int32_t>& side, const std::vector<int32_t>& out,
                      const std::vector<int64_t>& extent, OffsetMap& om) {
  std::vector<int64_t> ostride(out.size());
  int64_t s = 1;
  for (int i = (int)out.size() - 1; i >= 0; --i) {
    ostride[i] = s;
    s *= extent[out[i]];
  }
  std::map<int32_t, int> pos;
  for (size_t i = 0; i < out.size(); ++i) pos[out[i]] = (int)i;
  om.n = 0;
  size_t i = 0;
  while (i < side.size()) {
    size_t j = i;
    int64_t e = extent[side[i]];
    while (j + 1 < side.size() && pos[side[j + 1]] == pos[side[j]] + 1) {
      ++j;
      e *= extent[side[j]];
    }
    if (om.n >= kMaxDims) return false;
    if (e > 0xffffffffll) return false;
    om.ext[om.n] = (uint32_t)e;
    om.stride[om.n] = ostride[pos[side[j]]];
    ++om.n;
    i = j + 1;
  }
  return true;
}

}  // namespace

tn_status build_plan(const tn_network* net, const tn_path* path, const int32_t* sliced,
                     int32_t n_sliced, const tn_dtype_policy& pol, Plan& P, std::string& err) {
  std::ostringstream es;
  if (!net || !path || net->n_tensors <= 0 || net->n_labels <= 0 || !net->rank ||
      !net->modes || !net->extent) {
    err = "null or empty network";
    return TN_ERR_INVALID;
  }
  if (pol.prec < 0 || pol.prec > TN_R32_BF16X3) {
    err = "unknown precision";
    return TN_ERR_INVALID;
  }
  if (pol.semiring != TN_SEMIRING_STANDARD && pol.semiring != TN_SEMIRING_MAXPLUS) {
    err = "unknown semiring";
    return TN_ERR_INVALID;
  }
  if (pol.semiring == TN_SEMIRING_MAXPLUS && (pol.prec != TN_R32_FP32_SIMT || pol.exp_scaling)) {
    err = "the max-plus semiring runs in the R32 FP32 form without exponent scaling";
    return TN_ERR_UNSUPPORTED;
  }
  if (pol.prec == TN_R32_BF16X3) {
    err = "the real BF16x3 form is not built: real networks take TN_R32_TF32, TN_R32_3XTF32 or TN_R32_FP32_SIMT";
    return TN_ERR_UNSUPPORTED;
  }
  if (pol.prec == TN_C64_BF16X3 && pol.complex_mult == 3 && pol.exp_scaling) {
    err = "exponent scaling is not built for the 3M product: the 4M BF16x3 form (complex_mult 4) takes it";
    return TN_ERR_UNSUPPORTED;
  }
  if (pol.complex_mult != 0 && pol.complex_mult != 4 && pol.complex_mult != 3) {
    err = "complex_mult must be 4 (4M), 3 (3M) or 0 (4M)";
    return TN_ERR_INVALID;
  }
  if (pol.complex_mult == 3 && pol.prec != TN_C64_BF16X3) {
    err = "the 3M complex product is built for the BF16X3 form only";
    return TN_ERR_UNSUPPORTED;
  }
  const int32_t T = net->n_tensors, L = net->n_labels;
  P.n_leaves = T;
  P.n_labels = L;
  P.policy = pol;
  P.is_complex = pol.prec <= TN_C64_BF16X3;
  P.extent.assign(net->extent, net->extent + L);
  for (int32_t x = 0; x < L; ++x)
    if (P.extent[x] < 1) {
      err = "extent < 1";
      return TN_ERR_INVALID;
    }
  // ---- network validation: every closed label in exactly two tensors, open in one
  std::vector<int32_t> count(L, 0);
  std::vector<char> is_open(L, 0);
  if (net->n_open < 0 || (net->n_open > 0 && !net->open_modes)) {
    err = "bad open_modes";
    return TN_ERR_INVALID;
  }
  for (int32_t i = 0; i < net->n_open; ++i) {
    int32_t x = net->open_modes[i];
    if (x < 0 || x >= L || is_open[x]) {
      err = "bad or repeated open label";
      return TN_ERR_INVALID;
    }
    is_open[x] = 1;
  }
  P.open_modes.assign(net->open_modes, net->open_modes + net->n_open);
  P.tensors.assign(T + std::max(0, path->n_steps), TensorRec{});
  for (int32_t t = 0; t < T; ++t) {
    if (net->rank[t] < 0 || (net->rank[t] > 0 && !net->modes[t])) {
      err = "bad rank";
      return TN_ERR_INVALID;
    }
    std::set<int32_t> seen;
    for (int32_t r = 0; r < net->rank[t]; ++r) {
      int32_t x = net->modes[t][r];
      if (x < 0 || x >= L || !seen.insert(x).second) {
        es << "tensor " << t << ": bad or repeated label " << x;
        err = es.str();
        return TN_ERR_INVALID;
      }
      ++count[x];
      P.tensors[t].decl.push_back(x);
    }
  }
  for (int32_t x = 0; x < L; ++x) {
    if (count[x] == 0) continue;
    if (is_open[x] && count[x] != 1) {
      es << "open label " << x << " appears in " << count[x] << " tensors (hyper-edge)";
      err = es.str();
      return TN_ERR_UNSUPPORTED;
    }
    if (!is_open[x] && count[x] != 2) {
      es << "closed label " << x << " appears in " << count[x]
         << " tensors (hyper-edge or single-tensor trace)";
      err = es.str();
      return TN_ERR_UNSUPPORTED;
    }
  }
  for (int32_t x : P.open_modes)
    if (count[x] != 1) {
      err = "open label not on any tensor";
      return TN_ERR_INVALID;
    }
  // ---- slicing (Sec. II-C): mixed radix, first sliced label most significant
  std::vector<char> is_sliced(L, 0);
  P.sliced.clear();
  if (n_sliced < 0 || (n_sliced > 0 && !sliced)) {
    err = "bad sliced list";
    return TN_ERR_INVALID;
  }
  for (int32_t i = 0; i < n_sliced; ++i) {
    int32_t x = sliced[i];
    if (x < 0 || x >= L || is_sliced[x] || count[x] == 0) {
      err = "bad sliced label";
      return TN_ERR_INVALID;
    }
    if (is_open[x]) {
      err = "an open label cannot be sliced";
      return TN_ERR_UNSUPPORTED;
    }
    is_sliced[x] = 1;
    P.sliced.push_back(x);
  }
  P.slice_div.assign(P.sliced.size(), 1);
  P.n_slices = 1;
  for (int i = (int)P.sliced.size() - 1; i >= 0; --i) {
    P.slice_div[i] = P.n_slices;
    P.n_slices *= P.extent[P.sliced[i]];
    if (P.n_slices > (int64_t(1) << 40)) {
      err = "too many slices";
      return TN_ERR_UNSUPPORTED;
    }
  }
  // ---- path validation: a single binary tree in SSA form
  const int32_t S = path->n_steps;
  if (S != T - 1 || (S > 0 && !path->pair)) {
    es << "path must have n_tensors-1 = " << T - 1 << " steps, got " << S;
    err = es.str();
    return TN_ERR_INVALID;
  }
  std::vector<char> used(T + S, 0);
  P.steps.assign(S, StepRec{});
  std::vector<std::set<int32_t>> labset(T + S);
  for (int32_t t = 0; t < T; ++t) {
    TensorRec& R = P.tensors[t];
    for (int32_t x : R.decl) {
      if (is_sliced[x]) R.batched = true;
      else labset[t].insert(x);
    }
  }
  for (int32_t s = 0; s < S; ++s) {
    int32_t i = path->pair[2 * s], j = path->pair[2 * s + 1];
    if (i < 0 || j < 0 || i >= T + s || j >= T + s || i == j || used[i] || used[j]) {
      es << "step " << s << ": bad or reused operand (" << i << "," << j << ")";
      err = es.str();
      return TN_ERR_INVALID;
    }
    used[i] = used[j] = 1;
    StepRec& st = P.steps[s];
    st.out = T + s;
    st.a = i;
    st.b = j;
    std::set<int32_t>& A = labset[i];
    std::set<int32_t>& B = labset[j];
    std::set<int32_t> out;
    for (int32_t x : A) {
      if (B.count(x)) {
        if (is_open[x]) {
          err = "open label shared by two operands";
          return TN_ERR_UNSUPPORTED;
        }
      } else {
        out.insert(x);
      }
    }
    for (int32_t x : B)
      if (!A.count(x)) out.insert(x);
    labset[T + s] = out;
    P.tensors[i].consumer = s;
    P.tensors[j].consumer = s;
    P.tensors[T + s].producer = s;
    P.tensors[T + s].batched = P.tensors[i].batched || P.tensors[j].batched;
    st.batched = P.tensors[T + s].batched;
  }
  const int32_t root = T + S - 1;
  for (int32_t t = 0; t < T + S - 1; ++t)
    if (!used[t]) {
      es << "tensor " << t << " is never consumed (path is not one tree)";
      err = es.str();
      return TN_ERR_INVALID;
    }
  {
    std::set<int32_t> want(P.open_modes.begin(), P.open_modes.end());
    if (labset[root] != want) {
      err = "root labels differ from open_modes";
      return TN_ERR_INVALID;
    }
  }
  // ---- GEMM-oriented mode reordering: one backward pass (Sec. IV-A).
  // The root order is fixed by open_modes. Visiting steps from last to first, each
  // operand's order becomes [its retained labels in the output's order | the labels
  // reduced here]; that order is also the producer's output order. Each tensor has
  // one consumer, so its order is set exactly once. Reduced labels are appended in
  // ascending label id so that both operands agree.
  P.tensors[root].modes = P.open_modes;
  for (int32_t s = S - 1; s >= 0; --s) {
    StepRec& st = P.steps[s];
    const std::vector<int32_t>& O = P.tensors[st.out].modes;
    std::set<int32_t>& A = labset[st.a];
    std::set<int32_t>& B = labset[st.b];
    std::vector<int32_t> K;
    for (int32_t x : A)
      if (B.count(x)) K.push_back(x);  // std::set iterates in ascending id
    std::vector<int32_t> ra, rb;
    for (int32_t x : O) {
      if (A.count(x)) ra.push_back(x);
      else if (B.count(x)) rb.push_back(x);
    }
    st.K = K;
    std::vector<int32_t> la = ra, lb = rb;
    la.insert(la.end(), K.begin(), K.end());
    lb.insert(lb.end(), K.begin(), K.end());
    P.tensors[st.a].modes = la;
    P.tensors[st.b].modes = lb;
    st.M = ra;
    st.N = rb;
  }
  if (S == 0) P.tensors[0].modes = P.open_modes;
  // ---- sizes
  for (auto& R : P.tensors) {
    R.size = 1;
    for (int32_t x : R.modes) R.size *= P.extent[x];
  }
  // ---- roles (the GEMM A/B assignment) and kernel class per step
  const bool tc_form = is_tc_prec(pol.prec);
  const double eb = P.is_complex ? 8.0 : 4.0, fm = P.is_complex ? 8.0 : 2.0;
  for (int32_t s = 0; s < S; ++s) {
    StepRec& st = P.steps[s];
    const std::vector<int32_t>& O = P.tensors[st.out].modes;
    auto prod = [&](const std::vector<int32_t>& v) {
      int64_t p = 1;
      for (int32_t x : v) p *= P.extent[x];
      return p;
    };
    // Z3 reading: B (columns) owns the output's innermost label, so consecutive
    // columns land in consecutive addresses; for a scalar output the larger operand
    // takes the row role.
    bool swap = false;
    if (!O.empty()) {
      int32_t last = O.back();
      swap = std::find(st.M.begin(), st.M.end(), last) != st.M.end();
    } else {
      swap = P.tensors[st.b].size > P.tensors[st.a].size;
    }
    if (swap) {
      std::swap(st.a, st.b);
      std::swap(st.M, st.N);
    }
    st.m = prod(st.M);
    st.n = prod(st.N);
    st.k = prod(st.K);
    // A big x small step streams the big operand in the row role whatever Z3 says.
    auto stream_ok = [](int64_t m, int64_t n, int64_t k) {
      return n * k <= 256 && n <= 16 && m >= 1024;
    };
    if (!stream_ok(st.m, st.n, st.k) && stream_ok(st.n, st.m, st.k)) {
      std::swap(st.a, st.b);
      std::swap(st.M, st.N);
      std::swap(st.m, st.n);
    }
    // The tensor-core kernel tiles 128 rows: give the row role to the operand that
    // fills them when only one orientation qualifies.
    const bool tc_form_here = tc_form && tc_prec_built(pol.prec) && tc_supported();
    if (tc_form_here && !tc_step_ok(st.m, st.n, st.k, pol.prec) && tc_step_ok(st.n, st.m, st.k, pol.prec)) {
      std::swap(st.a, st.b);
      std::swap(st.M, st.N);
      std::swap(st.m, st.n);
    }
    if (!build_offset_map(st.M, O, P.extent, st.rows) ||
        !build_offset_map(st.N, O, P.extent, st.cols)) {
      err = "output interleaving too fine for the offset maps";
      return TN_ERR_UNSUPPORTED;
    }
    const double flops = fm * double(st.m) * double(st.n) * double(st.k);
    const double bytes = eb * (double(st.m) * st.k + double(st.n) * st.k + double(st.m) * st.n);
    const double t_simt = std::max(bytes / g_cost.hbm_bytes_per_s, flops / g_cost.simt_flops);
    st.cls = TN_CLASS_SIMT;
    if (tc_form_here && tc_step_ok(st.m, st.n, st.k, pol.prec)) {
      // a step narrower than the tile (128 columns, 256 for a real step) uses that fraction
      // of the tensor core
      const double fill = std::min(1.0, double(st.n) / (P.is_complex ? 128.0 : 256.0));
      const double rate = tc_flops(pol.complex_mult == 3 ? -3 : pol.prec);
      const double t_tc = std::max(bytes / g_cost.hbm_bytes_per_s, flops / (rate * fill));
      // ties (both bound by the same HBM bytes) go to the tensor-core kernel, whose
      // epilogue stores are the better coalesced
      if (t_tc <= t_simt) st.cls = TN_CLASS_TC;
    }
    // (the streaming kernel computes in (+, x) only)
    if (st.cls == TN_CLASS_SIMT && stream_ok(st.m, st.n, st.k) && pol.semiring == TN_SEMIRING_STANDARD)
      st.cls = TN_CLASS_STREAM;
    // few outputs over a long reduction: the tiled kernel would leave all but a few
    // threads idle and sum k terms serially in FP32
    if (st.cls == TN_CLASS_SIMT && st.m * st.n <= kSplitMaxOut && st.k >= kSplitChunk)
      st.cls = TN_CLASS_SPLITK;
  }
  // ---- pinned tensors: unbatched but consumed by a batched step (kept for all passes)
  for (int32_t s = 0; s < S; ++s) {
    const StepRec& st = P.steps[s];
    if (!st.batched) continue;
    if (!P.tensors[st.a].batched) P.tensors[st.a].pinned = true;
    if (!P.tensors[st.b].batched) P.tensors[st.b].pinned = true;
  }
  // ---- split-BF16 operands: a BF16x3 tensor-core step reads both operands in the split
  // form, so their producers (leaf staging or the producing step) write that form
  if (pol.prec == TN_C64_BF16X3) {
    const int32_t mode = pol.complex_mult == 3 ? 2 : 1;
    for (int32_t s = 0; s < S; ++s) {
      const StepRec& st = P.steps[s];
      if (st.cls != TN_CLASS_TC) continue;
      P.tensors[st.a].split = mode;
      P.tensors[st.b].split = mode;
    }
  }
  // ---- leaf descriptors (sources filled per call)
  P.leafdesc.assign(T, LeafDesc{});
  int64_t leaf_permutes = 0;
  for (int32_t t = 0; t < T; ++t) {
    const TensorRec& R = P.tensors[t];
    LeafDesc& d = P.leafdesc[t];
    if ((int)R.modes.size() > kMaxLeafRank) {
      err = "leaf rank too large for staging";
      return TN_ERR_UNSUPPORTED;
    }
    std::vector<int64_t> dstride(R.decl.size());
    int64_t sstr = 1;
    for (int i = (int)R.decl.size() - 1; i >= 0; --i) {
      dstride[i] = sstr;
      sstr *= P.extent[R.decl[i]];
    }
    d.rank = (int32_t)R.modes.size();
    d.size = R.size;
    d.batched = R.batched ? 1 : 0;
    d.split = R.split;
    for (int i = 0; i < d.rank; ++i) {
      int32_t x = R.modes[i];
      int pos = int(std::find(R.decl.begin(), R.decl.end(), x) - R.decl.begin());
      d.ext[i] = (uint32_t)P.extent[x];
      d.sstride[i] = dstride[pos];
    }
    d.n_sl = 0;
    for (size_t i = 0; i < R.decl.size(); ++i) {
      int32_t x = R.decl[i];
      if (!is_sliced[x]) continue;
      if (d.n_sl >= kMaxSliced) {
        err = "too many sliced labels on one leaf";
        return TN_ERR_UNSUPPORTED;
      }
      int q = int(std::find(P.sliced.begin(), P.sliced.end(), x) - P.sliced.begin());
      d.sl_div[d.n_sl] = P.slice_div[q];
      d.sl_ext[d.n_sl] = (uint32_t)P.extent[x];
      d.sl_stride[d.n_sl] = dstride[i];
      ++d.n_sl;
    }
    std::vector<int32_t> undecl;
    for (int32_t x : R.decl)
      if (!is_sliced[x]) undecl.push_back(x);
    if (undecl != R.modes) ++leaf_permutes;
    // tiled permutation groups (large leaves): output group = shortest suffix of the planned
    // order holding >= 32 elements; input group = the declared order's fastest remaining
    // positions up to >= 32 elements; the rest in planned order
    {
      int64_t ds = 1;
      for (int i = d.rank - 1; i >= 0; --i) {
        d.dstride[i] = ds;
        ds *= d.ext[i];
      }
      d.tiled = (d.size >= kTiledLeafElems && d.rank >= 1) ? 1 : 0;
      std::vector<char> in_o(d.rank, 0), in_i(d.rank, 0);
      d.no = 0;
      d.Po = 1;
      for (int i = d.rank - 1; i >= 0 && d.Po < 32; --i) {
        in_o[i] = 1;
        d.Po *= d.ext[i];
        ++d.no;
      }
      d.ni = 0;
      d.Pi = 1;
      std::vector<int> ip;  // fastest first
      for (int j = (int)undecl.size() - 1; j >= 0 && d.Pi < 32; --j) {
        const int pos = int(std::find(R.modes.begin(), R.modes.end(), undecl[j]) - R.modes.begin());
        if (in_o[pos]) continue;
        in_i[pos] = 1;
        ip.push_back(pos);
        d.Pi *= d.ext[pos];
      }
      d.ni = (int32_t)ip.size();
      for (int q = 0; q < d.ni; ++q) d.ipos[q] = (int8_t)ip[d.ni - 1 - q];  // slowest first
      d.nr = 0;
      d.Pr = 1;
      for (int i = 0; i < d.rank; ++i)
        if (!in_o[i] && !in_i[i]) {
          d.rpos[d.nr++] = (int8_t)i;
          d.Pr *= d.ext[i];
        }
      const int inner = undecl.empty() ? -1
                                       : int(std::find(R.modes.begin(), R.modes.end(), undecl.back()) -
                                             R.modes.begin());
      d.load_o = (inner >= 0 && in_o[inner]) ? 1 : 0;
      d.vec_load = (!d.load_o && d.ni > 0 && d.sstride[d.ipos[d.ni - 1]] == 1 && d.ext[d.ipos[d.ni - 1]] % 2 == 0)
                       ? 1 : 0;
      // pipelined form: each group one 32-wide chunk, 16-byte loads, and the rest index's
      // fastest positions multiplying to exactly the tiles one CTA walks
      d.fast = 0;
      d.nlo = 0;
      if (d.tiled && d.Po == 32 && d.Pi == 32 && d.vec_load && P.is_complex) {
        int64_t lo = 1;
        int nlo = 0;
        while (nlo < d.nr && lo < kTilesPerCta) lo *= d.ext[d.rpos[d.nr - 1 - nlo++]];
        if (lo == kTilesPerCta) {
          d.fast = 1;
          d.nlo = nlo;
        }
      }
    }
  }
  // ---- statistics (Sec. II-B Eqs. 1-3, per slice; algorithmic flops and bytes)
  tn_plan_stats& S0 = P.stats;
  S0 = tn_plan_stats{};
  S0.n_steps = S;
  S0.n_leaves = T;
  S0.n_slices = P.n_slices;
  S0.leaf_permutes = leaf_permutes;
  double Ct = 0, Cm = 0, Cs = 0, fl_batched = 0, fl_fixed = 0, by_batched = 0, by_fixed = 0;
  int64_t peak = 0;
  for (auto& R : P.tensors) peak = std::max(peak, R.size);
  for (int32_t s = 0; s < S; ++s) {
    const StepRec& st = P.steps[s];
    double m = double(st.m), n = double(st.n), k = double(st.k);
    Ct += m * n * k;
    Cm += m * k + k * n + m * n;
    Cs = std::max(Cs, std::max(m * k, std::max(k * n, m * n)));
    double f = fm * m * n * k, b = eb * (m * k + k * n + m * n);
    (st.batched ? fl_batched : fl_fixed) += f;
    (st.batched ? by_batched : by_fixed) += b;
    S0.steps_per_class[st.cls] += 1;
    S0.flops_per_class[st.cls] += f * (st.batched ? double(P.n_slices) : 1.0);
  }
  for (int32_t t = 0; t < T; ++t) {
    const TensorRec& R = P.tensors[t];
    double b = 2.0 * eb * double(R.size);
    (R.batched ? by_batched : by_fixed) += b;
  }
  S0.Ct = Ct;
  S0.Cm = Cm;
  S0.Cs = Cs;
  S0.peak_elems = peak;
  S0.flops = fl_fixed + fl_batched * double(P.n_slices);
  S0.bytes = by_fixed + by_batched * double(P.n_slices);
  P.out_elems = P.tensors[root].size;
  return TN_OK;
}

// Liveness: a leaf is born when the pass stages it (event -1) and a step output at its
// step; each dies at its consuming step (the root after the final accumulation). Two
// tensors share memory only if their lifetimes are disjoint. Offsets are static, so
// every pass replays the same layout -- which is why a pinned tensor (made once in the
// first pass, read by every pass) is reserved over the whole timeline [-1, inf]: a
// tensor that dies before the pinned one is made in the first pass is made again in
// later passes, and must not land on it.
void assign_workspace(Plan& P, int64_t batch) {
  P.batch = batch;
  const int32_t T = P.n_leaves, S = (int32_t)P.steps.size();
  const int64_t eb = elem_bytes(P);
  const int32_t N = T + S;
  const int32_t kInf = S + 1;
  std::vector<int32_t> birth(N), death(N);
  for (int32_t t = 0; t < N; ++t) {
    TensorRec& R = P.tensors[t];
    birth[t] = t < T ? -1 : R.producer;
    death[t] = R.consumer < 0 ? S : R.consumer;
    if (R.pinned) {
      birth[t] = -1;
      death[t] = kInf;
    }
    R.bytes = align_up(std::max<int64_t>(1, R.size) * stored_bytes(P, R) * (R.batched ? batch : 1), kAlign);
  }
  std::vector<int32_t> order(N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return birth[x] < birth[y]; });
  struct Blk { int64_t off, bytes; int32_t death; };
  std::vector<Blk> live;
  std::map<int64_t, int64_t> freel;  // offset -> bytes
  int64_t top = 0, max_top = 0;
  auto release = [&](int32_t now) {
    for (size_t i = 0; i < live.size();) {
      if (live[i].death < now) {
        freel[live[i].off] = live[i].bytes;
        live[i] = live.back();
        live.pop_back();
      } else {
        ++i;
      }
    }
    // coalesce neighbours
    for (auto it = freel.begin(); it != freel.end();) {
      auto nx = std::next(it);
      if (nx != freel.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        freel.erase(nx);
      } else {
        it = nx;
      }
    }
    // give a free block at the top back to the bump pointer
    if (!freel.empty()) {
      auto last = std::prev(freel.end());
      if (last->first + last->second == top) {
        top = last->first;
        freel.erase(last);
      }
    }
  };
  for (int32_t t : order) {
    release(birth[t]);
    int64_t need = P.tensors[t].bytes;
    auto best = freel.end();
    for (auto it = freel.begin(); it != freel.end(); ++it)
      if (it->second >= need && (best == freel.end() || it->second < best->second)) best = it;
    int64_t off;
    if (best != freel.end()) {
      off = best->first;
      int64_t rem = best->second - need;
      freel.erase(best);
      if (rem > 0) freel[off + need] = rem;
    } else {
      off = top;
      top += need;
      max_top = std::max(max_top, top);
    }
    P.tensors[t].offset = off;
    live.push_back({off, need, death[t]});
  }
  P.arena_bytes = align_up(max_top, kAlign);
  // Self-check of the assignment: every tensor inside the arena, and no two tensors
  // that are alive at the same time share a byte.
  P.workspace_ok = true;
  for (int32_t t = 0; t < N && P.workspace_ok; ++t) {
    const TensorRec& A = P.tensors[t];
    if (A.offset < 0 || A.offset + A.bytes > P.arena_bytes) P.workspace_ok = false;
    for (int32_t u = t + 1; u < N && P.workspace_ok; ++u) {
      const TensorRec& B = P.tensors[u];
      const bool time = birth[t] <= death[u] && birth[u] <= death[t];
      const bool mem = A.offset < B.offset + B.bytes && B.offset < A.offset + A.bytes;
      if (time && mem) P.workspace_ok = false;
    }
  }
  int64_t cur = P.arena_bytes;
  // cross-slice accumulator [sum re, sum im, comp re, comp im] per output element: only
  // calls of more than one pass keep it between passes (the last pass writes the output)
  P.off_acc = cur;
  if (P.n_slices > batch) cur += align_up(P.out_elems * 4 * (int64_t)sizeof(double), kAlign);
  // scale records: unbatched tensors first (reset once per call), then batched ones
  // (reset every pass)
  P.rec_index.assign(N, 0);
  int64_t r = 0;
  for (int32_t t = 0; t < N; ++t)
    if (!P.tensors[t].batched) P.rec_index[t] = (int32_t)r++;
  P.n_rec_unbatched = r;
  for (int32_t t = 0; t < N; ++t)
    if (P.tensors[t].batched) {
      P.rec_index[t] = (int32_t)r;
      r += batch;
    }
  P.n_rec_total = r;
  P.off_scale = cur;
  cur += align_up(r * 16, kAlign);
  P.off_recidx = cur;
  cur += align_up(int64_t(T) * 4, kAlign);
  P.off_ref = cur;
  cur += kAlign;
  P.off_err = cur;
  cur += kAlign;
  // split-K partials: the largest need of any split-K step (one pass)
  int64_t scratch = 0;
  for (StepRec& st : P.steps) {
    st.ksplit = st.cls == TN_CLASS_SIMT ? simt_ksplit(st.m, st.n, st.k, st.batched ? batch : 1, P.num_sms,
                                                      P.policy.exp_scaling != 0)
                                        : 1;
    if (st.ksplit > 1)
      scratch = std::max(scratch, int64_t(st.ksplit) * (st.batched ? batch : 1) * st.m * st.n *
                                      (P.is_complex ? 2 : 1) * 4);
  }
  for (const StepRec& st : P.steps)
    if (st.cls == TN_CLASS_SPLITK)
      scratch = std::max(scratch, (st.batched ? batch : 1) * ((st.k + kSplitChunk - 1) / kSplitChunk) *
                                      st.m * st.n * 16);
  P.off_scratch = cur;
  P.scratch_bytes = scratch;
  cur += align_up(scratch, kAlign);
  // step chains: maximal runs (two or more) of consecutive tiny CUDA-core steps, each run
  // one launch of a single CTA instead of a launch per step (launch-bound paths)
  P.chains.clear();
  int32_t n_table = 0;
  const int64_t cw = P.is_complex ? 4 : 1;
  auto tiny = [&](const StepRec& st) {
    return st.cls == TN_CLASS_SIMT && st.ksplit == 1 &&
           double(st.m) * double(st.n) * double(st.k) * double(cw * (st.batched ? batch : 1)) <=
               double(kChainMaxWork);
  };
  for (StepRec& st : P.steps) st.chain = -1;
  for (int32_t s = 0; s < (int32_t)P.steps.size();) {
    int32_t e = s;
    while (e < (int32_t)P.steps.size() && tiny(P.steps[e])) ++e;
    if (e - s >= 2) {
      ChainRec c;
      c.first = s;
      c.n = e - s;
      c.table = n_table;
      for (int32_t q = s; q < e; ++q) {
        P.steps[q].chain = (int32_t)P.chains.size();
        c.any_batched = c.any_batched || P.steps[q].batched;
      }
      n_table += c.n;
      P.chains.push_back(c);
    }
    s = e > s ? e : s + 1;
  }
  P.off_chain = cur;
  cur += align_up(int64_t(n_table) * (int64_t)sizeof(ChainStep), kAlign);
  P.off_leafdesc = cur;
  cur += align_up(int64_t(T) * (int64_t)sizeof(LeafDesc), kAlign);
  P.off_stage_in = cur;
  P.stage_in_off.assign(T, 0);
  for (int32_t t = 0; t < T; ++t) {
    int64_t full = 1;
    for (int32_t x : P.tensors[t].decl) full *= P.extent[x];
    P.stage_in_off[t] = cur;
    cur += align_up(full * eb, kAlign);
  }
  cur += align_up(P.out_elems * 16 + 16, kAlign);  // host-form output staging
  P.total_bytes = cur;
  P.stats.slice_batch = batch;
  P.stats.n_passes = (P.n_slices + batch - 1) / batch;
  P.stats.workspace_bytes = P.total_bytes;
}

}  // namespace tn
