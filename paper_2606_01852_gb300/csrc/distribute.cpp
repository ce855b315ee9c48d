// Offline distribution planning of Sec. IV-B (host only): large-step identification,
// prefix selection of the split modes (Eq. 4), mode tracking along use-chains,
// Activate / Keep / Redistribute / Gather, the cost model of Eqs. 6-7 and the dynamic
// programme over split-mode sets that places the redistributions.
#include <algorithm>
#include <cmath>
#include <limits>
#include <string>
#include <vector>

#include "tn.h"
#include "tn_internal.h"

namespace tn {
namespace {

struct Model {
  const Plan& P;
  const tn_dist_config& cfg;
  double eb, fm;  // bytes per element, flops per MAC
  double gather_bytes;

  double bytes(int32_t t) const { return double(P.tensors[t].size) * eb; }
  double flops(int32_t s) const {
    const StepRec& st = P.steps[s];
    return fm * double(st.m) * double(st.n) * double(st.k);
  }
  // Eq. 6 for a step run whole on one device
  double t_whole(int32_t s) const {
    const StepRec& st = P.steps[s];
    const double rw = bytes(st.a) + bytes(st.b) + bytes(st.out);
    return std::max(rw / cfg.dev_bw, flops(s) / cfg.dev_flops);
  }
  // Eq. 6 per device for a chain step: `split` operand (or none, -1, at activation),
  // the output and the flops divided P ways, the other operand whole
  double t_split(int32_t s, int32_t split) const {
    const StepRec& st = P.steps[s];
    const double p = cfg.n_gpus;
    double rw = bytes(st.out) / p;
    for (int32_t t : {st.a, st.b}) rw += (t == split) ? bytes(t) / p : bytes(t);
    return std::max(rw / cfg.dev_bw, flops(s) / (p * cfg.dev_flops));
  }
  // Eq. 7 for tensor t whose split modes change from `from` to `to` (to empty: a gather)
  double t_comm(int32_t t, const std::vector<int32_t>& from, const std::vector<int32_t>& to,
                int64_t* n_blk_out) const {
    const TensorRec& R = P.tensors[t];
    const double p = cfg.n_gpus;
    int inner = -1;
    for (int i = 0; i < (int)R.modes.size(); ++i) {
      const int32_t x = R.modes[i];
      if (std::find(from.begin(), from.end(), x) != from.end() || std::find(to.begin(), to.end(), x) != to.end())
        inner = i;
    }
    double run = 1;
    for (int i = inner + 1; i < (int)R.modes.size(); ++i) run *= double(P.extent[R.modes[i]]);
    const double n_blk = std::max(1.0, double(R.size) / (p * run));
    if (n_blk_out) *n_blk_out = static_cast<int64_t>(n_blk);
    const double bw = bytes(t) * (p - 1) / (p * cfg.net_bw);
    return bw + n_blk * std::max(cfg.latency, cfg.block_bytes / cfg.net_bw);
  }
  // Eq. 4: the shortest leading prefix of t's planned order, skipping labels in `avoid`,
  // whose extents multiply to >= P; empty if none exists
  std::vector<int32_t> prefix(int32_t t, const std::vector<int32_t>& avoid) const {
    std::vector<int32_t> D;
    double prod = 1;
    for (int32_t x : P.tensors[t].modes) {
      if (prod >= cfg.n_gpus) break;
      if (std::find(avoid.begin(), avoid.end(), x) != avoid.end()) continue;
      D.push_back(x);
      prod *= double(P.extent[x]);
    }
    if (prod < cfg.n_gpus) D.clear();
    return D;
  }
};

bool meets(const std::vector<int32_t>& D, const std::vector<int32_t>& K) {
  for (int32_t x : D)
    if (std::find(K.begin(), K.end(), x) != K.end()) return true;
  return false;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" tn_status tn_plan_distribute(tn_plan_t plan, const tn_dist_config* cfg, tn_dist_report* report,
                                        tn_dist_step* steps_out) {
  if (!plan || !cfg || !report) {
    set_error("tn_plan_distribute: null argument");
    return TN_ERR_INVALID;
  }
  if (cfg->n_gpus < 1 || !(cfg->large_bytes > 0) || !(cfg->dev_bw > 0) || !(cfg->dev_flops > 0) ||
      !(cfg->net_bw > 0) || cfg->latency < 0 || cfg->block_bytes < 0 || cfg->gather_bytes < 0) {
    set_error("tn_plan_distribute: P >= 1 and positive sizes and rates are required");
    return TN_ERR_INVALID;
  }
  const Plan& P = plan->P;
  Model M{P, *cfg, double(elem_bytes(P)), P.is_complex ? 8.0 : 2.0,
          cfg->gather_bytes > 0 ? cfg->gather_bytes : cfg->large_bytes};
  const int32_t S = (int32_t)P.steps.size();
  const int32_t T = (int32_t)P.tensors.size();

  std::vector<tn_dist_step> rec(S);
  for (auto& r : rec) {
    r = tn_dist_step{};
    r.chain = -1;
  }
  tn_dist_report rep{};
  for (int32_t s = 0; s < S; ++s) {
    rec[s].out_bytes = M.bytes(P.steps[s].out);
    rec[s].t_gemm = M.t_whole(s);
    rep.t_single += rec[s].t_gemm;
    const StepRec& st = P.steps[s];
    if (std::max({M.bytes(st.a), M.bytes(st.b), M.bytes(st.out)}) >= cfg->large_bytes) ++rep.n_large_steps;
  }

  // ---- use-chains: path order is topological, so a step sees its operands' status
  std::vector<int32_t> chain_of(S, -1);     // chain index of a step
  std::vector<int32_t> carried(S, -1);      // the split operand a chain step inherits
  std::vector<char> dist(T, 0);             // tensor produced split and still split
  std::vector<std::vector<int32_t>> chains;
  if (cfg->n_gpus > 1) {
    for (int32_t s = 0; s < S; ++s) {
      const StepRec& st = P.steps[s];
      const bool da = dist[st.a], db = dist[st.b];
      int32_t ch = -1;
      if (da || db) {
        int32_t c = da ? st.a : st.b;
        if (da && db && M.bytes(st.b) > M.bytes(st.a)) c = st.b;  // the larger carries on
        // it carries on only if enough of its modes survive this step to split it P ways
        if (!M.prefix(c, st.K).empty()) {
          carried[s] = c;
          ch = chain_of[P.tensors[c].producer];
        }
        for (int32_t o : {st.a, st.b})
          if (o != carried[s] && dist[o]) dist[o] = 0;  // its chain ends in a gather
      }
      if (ch < 0 && std::max({M.bytes(st.a), M.bytes(st.b), M.bytes(st.out)}) >= cfg->large_bytes &&
          !M.prefix(st.out, {}).empty()) {
        ch = (int32_t)chains.size();  // Activate
        chains.emplace_back();
      }
      if (ch < 0) continue;
      chain_of[s] = ch;
      chains[ch].push_back(s);
      const TensorRec& out = P.tensors[st.out];
      dist[st.out] = (out.consumer >= 0 && M.bytes(st.out) >= M.gather_bytes) ? 1 : 0;
    }
  }
  // Each tensor has one consumer and only a chain's newest output can still be split, so
  // every chain is a linear sequence: step i + 1 carries the output of step i.

  // ---- DP per chain over the split-mode set of each output
  for (size_t ci = 0; ci < chains.size(); ++ci) {
    const std::vector<int32_t>& c = chains[ci];
    const int L = (int)c.size();
    struct State {
      std::vector<int32_t> D;
      double cost;
      int prev;      // index into the previous position's states
      bool redist;
      bool forced;
      double comm;
      int64_t n_blk;
    };
    std::vector<std::vector<State>> dp(L);
    auto next_K = [&](int i) -> std::vector<int32_t> {
      return i + 1 < L ? P.steps[c[i + 1]].K : std::vector<int32_t>{};
    };
    {
      const int32_t s0 = c[0];
      std::vector<int32_t> D0 = M.prefix(P.steps[s0].out, next_K(0));
      if (D0.empty() || D0.size() > TN_DIST_MAX_MODES) {
        set_error("tn_plan_distribute: a chain output cannot be split P ways");
        return TN_ERR_UNSUPPORTED;
      }
      dp[0].push_back(State{D0, M.t_split(s0, -1), -1, false, false, 0.0, 0});
      ++rep.dp_states;
    }
    for (int i = 1; i < L; ++i) {
      const int32_t s = c[i], out = P.steps[s].out;
      const double tg = M.t_split(s, carried[s]);
      const std::vector<int32_t> Kn = next_K(i);
      const std::vector<int32_t> fresh = M.prefix(out, Kn);
      for (int j = 0; j < (int)dp[i - 1].size(); ++j) {
        const State& pr = dp[i - 1][j];
        ++rep.dp_states;
        const bool keep_ok = !meets(pr.D, Kn);
        if (keep_ok) {
          const double cost = pr.cost + tg;
          auto it = std::find_if(dp[i].begin(), dp[i].end(), [&](const State& x) { return x.D == pr.D; });
          if (it == dp[i].end()) dp[i].push_back(State{pr.D, cost, j, false, false, 0.0, 0});
          else if (cost < it->cost) *it = State{pr.D, cost, j, false, false, 0.0, 0};
        }
        if (!fresh.empty() && fresh != pr.D) {
          int64_t nb = 0;
          const double cm = M.t_comm(out, pr.D, fresh, &nb);
          const double cost = pr.cost + tg + cm;
          const State st{fresh, cost, j, true, !keep_ok, cm, nb};
          auto it = std::find_if(dp[i].begin(), dp[i].end(), [&](const State& x) { return x.D == fresh; });
          if (it == dp[i].end()) dp[i].push_back(st);
          else if (cost < it->cost) *it = st;
        }
      }
      if (dp[i].empty()) {
        set_error("tn_plan_distribute: no feasible split for a chain step");
        return TN_ERR_UNSUPPORTED;
      }
    }
    // gather at the end; pick the best final state and backtrack
    int best = -1;
    double best_cost = std::numeric_limits<double>::infinity(), best_g = 0;
    int64_t best_nb = 0;
    for (int j = 0; j < (int)dp[L - 1].size(); ++j) {
      int64_t nb = 0;
      const double g = M.t_comm(P.steps[c[L - 1]].out, dp[L - 1][j].D, {}, &nb);
      if (dp[L - 1][j].cost + g < best_cost) {
        best_cost = dp[L - 1][j].cost + g;
        best = j;
        best_g = g;
        best_nb = nb;
      }
    }
    for (int i = L - 1, j = best; i >= 0; j = dp[i].at(j).prev, --i) {
      const State& st = dp[i][j];
      tn_dist_step& r = rec[c[i]];
      r.chain = (int32_t)ci;
      r.n_dist = (int32_t)st.D.size();
      // split modes in the output's planned order
      int q = 0;
      for (int32_t x : P.tensors[P.steps[c[i]].out].modes)
        if (std::find(st.D.begin(), st.D.end(), x) != st.D.end() && q < TN_DIST_MAX_MODES) r.dist_modes[q++] = x;
      r.t_gemm = i == 0 ? M.t_split(c[0], -1) : M.t_split(c[i], carried[c[i]]);
      r.state = i == 0 ? TN_DIST_ACTIVATE : (st.redist ? TN_DIST_REDISTRIBUTE : TN_DIST_KEEP);
      r.forced = st.forced ? 1 : 0;
      r.t_comm = st.comm;
      r.n_blk = st.n_blk;
      if (st.redist) {
        ++rep.n_redistributions;
        rep.n_forced += st.forced ? 1 : 0;
        rep.bytes_redistributed += r.out_bytes;
      }
      if (i == L - 1) {
        // the chain's last output is gathered; a single-step chain is both
        if (i > 0) r.state = st.redist ? TN_DIST_REDISTRIBUTE : TN_DIST_GATHER;
        if (st.redist) {
          r.t_comm += best_g;
        } else {
          r.t_comm = best_g;
          r.n_blk = best_nb;
        }
        ++rep.n_gathers;
        rep.bytes_redistributed += r.out_bytes;
      }
    }
  }
  rep.n_chains = (int32_t)chains.size();
  for (int32_t s = 0; s < S; ++s) {
    rep.t_total += rec[s].t_gemm + rec[s].t_comm;
    rep.t_comm_total += rec[s].t_comm;
  }
  rep.speedup = rep.t_total > 0 ? rep.t_single / rep.t_total : 1.0;
  rep.extra_speedup = rep.speedup / cfg->n_gpus;
  rep.projected_total = rep.t_total * double(P.n_slices);
  *report = rep;
  if (steps_out)
    for (int32_t s = 0; s < S; ++s) steps_out[s] = rec[s];
  return TN_OK;
}
