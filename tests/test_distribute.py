"""The offline distribution planner of Sec. IV-B (tn_plan_distribute), host only.

The planner's dynamic programme is checked against exhaustive search: for every
use-chain it reports, all keep/redistribute sequences are enumerated here with the cost
model written out from Eqs. 4, 6 and 7 (and the readings the header states: the other
operand of a chain step is held whole, a chain ends with a gather, base block size
`block_bytes`), and the planner's schedule must cost exactly the minimum."""
import itertools

import numpy as np
import pytest

from tests._lib import ensure_built
from tn_inputs import workloads
from tn_inputs.network import Network, Path

CFG = dict(large_bytes=8 * 2**8, dev_bw=1e12, dev_flops=1e13, net_bw=1e11, latency=1e-6, block_bytes=256.0)


def caterpillar(seed, n_tensors=9, n_labels=26, n_open=6):
    """A connected random network contracted left to right: ((T0 T1) T2) T3 ..., so every
    intermediate feeds the next step (long use-chains)."""
    rng = np.random.default_rng(seed)
    modes = [[] for _ in range(n_tensors)]
    lab = 0
    for t in range(1, n_tensors):
        u = int(rng.integers(0, t))
        modes[u].append(lab)
        modes[t].append(lab)
        lab += 1
    while lab < n_labels - n_open:
        u, v = rng.choice(n_tensors, size=2, replace=False)
        modes[int(u)].append(lab)
        modes[int(v)].append(lab)
        lab += 1
    opens = []
    while lab < n_labels:
        modes[int(rng.integers(0, n_tensors))].append(lab)
        opens.append(lab)
        lab += 1
    ext = {x: 2 for x in range(n_labels)}
    tensors = [np.zeros(tuple(ext[x] for x in m), dtype=np.complex128) for m in modes]
    pairs = [(0, 1)] + [(n_tensors + i, i + 2) for i in range(n_tensors - 2)]
    return Network(tensors, [tuple(m) for m in modes], ext, tuple(opens)), Path(pairs)


class CostModel:
    """Eqs. 4, 6, 7 over a plan's planned layouts (complex64: 8 bytes per element)."""

    def __init__(self, plan, net, P, cfg):
        self.plan, self.P, self.cfg = plan, P, cfg
        self.ext = dict(net.extent)
        self.n_steps = plan.info()["n_steps"]
        self.steps = [plan.step(s) for s in range(self.n_steps)]
        self.layout = {}
        n_t = len(net.tensors) + self.n_steps
        for t in range(n_t):
            self.layout[t] = plan.layout(t)
        self.out = {s: len(net.tensors) + s for s in range(self.n_steps)}

    def size(self, t):
        return int(np.prod([self.ext[x] for x in self.layout[t]])) if self.layout[t] else 1

    def bytes(self, t):
        return 8.0 * self.size(t)

    def K(self, s):
        st = self.steps[s]
        return set(self.layout[st["a_id"]]) & set(self.layout[st["b_id"]])

    def flops(self, s):
        st = self.steps[s]
        return 8.0 * st["m"] * st["n"] * st["k"]

    def t_split(self, s, split):
        st, c = self.steps[s], self.cfg
        rw = self.bytes(self.out[s]) / self.P
        for t in (st["a_id"], st["b_id"]):
            rw += self.bytes(t) / self.P if t == split else self.bytes(t)
        return max(rw / c["dev_bw"], self.flops(s) / (self.P * c["dev_flops"]))

    def t_comm(self, t, old, new):
        c, modes = self.cfg, self.layout[t]
        pos = [i for i, x in enumerate(modes) if x in set(old) | set(new)]
        run = int(np.prod([self.ext[x] for x in modes[max(pos) + 1:]])) if pos else self.size(t)
        n_blk = max(1.0, self.size(t) / (self.P * run))
        return self.bytes(t) * (self.P - 1) / (self.P * c["net_bw"]) + n_blk * max(c["latency"],
                                                                              c["block_bytes"] / c["net_bw"])

    def prefix(self, t, avoid):
        D, prod = [], 1
        for x in self.layout[t]:
            if prod >= self.P:
                break
            if x in avoid:
                continue
            D.append(x)
            prod *= self.ext[x]
        return D if prod >= self.P else []


def chains_of(steps):
    chains = {}
    for s, st in enumerate(steps):
        if st["chain"] >= 0:
            chains.setdefault(st["chain"], []).append(s)
    return [chains[k] for k in sorted(chains)]


def exhaustive_chain_cost(cm, chain):
    """Minimum over every keep/redistribute sequence of one chain (gather at the end)."""
    L = len(chain)
    nextK = [cm.K(chain[i + 1]) if i + 1 < L else set() for i in range(L)]
    D0 = cm.prefix(cm.out[chain[0]], nextK[0])
    best = float("inf")
    for choice in itertools.product((False, True), repeat=L - 1):
        D, cost, ok = D0, cm.t_split(chain[0], None), True
        for i in range(1, L):
            s = chain[i]
            cost += cm.t_split(s, cm.out[chain[i - 1]])
            if choice[i - 1]:
                F = cm.prefix(cm.out[s], nextK[i])
                if not F or F == D:
                    ok = False
                    break
                cost += cm.t_comm(cm.out[s], D, F)
                D = F
            elif set(D) & nextK[i]:
                ok = False
                break
        if ok:
            best = min(best, cost + cm.t_comm(cm.out[chain[-1]], D, []))
    return best


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("P", [4, 16, 64])
def test_dp_matches_exhaustive_search(seed, P):
    tn = ensure_built()
    net, path = caterpillar(seed)
    plan = tn.Plan(net, path, host_only=True)
    rep, steps = plan.distribute(P, **CFG)
    cm = CostModel(plan, net, P, CFG)
    chains = chains_of(steps)
    assert rep["n_chains"] == len(chains) >= 1
    for chain in chains:
        got = sum(steps[s]["t_gemm"] + steps[s]["t_comm"] for s in chain)
        want = exhaustive_chain_cost(cm, chain)
        assert got == pytest.approx(want, rel=1e-12), (seed, P, chain)
        # the schedule itself is feasible and follows Eq. 4 where it (re)splits
        for i, s in enumerate(chain):
            st = steps[s]
            nxt = cm.K(chain[i + 1]) if i + 1 < len(chain) else set()
            assert not set(st["dist_modes"]) & nxt
            assert np.prod([cm.ext[x] for x in st["dist_modes"]]) >= P
            if st["state"] in ("activate", "redistribute"):
                assert st["dist_modes"] == cm.prefix(cm.out[s], nxt)
            if st["state"] == "keep":
                assert st["dist_modes"] == steps[chain[i - 1]]["dist_modes"] and st["t_comm"] == 0.0
            if st["forced"]:
                assert set(steps[chain[i - 1]]["dist_modes"]) & nxt
    # every step off the chains runs whole: Eq. 6 with undivided sizes
    for s, st in enumerate(steps):
        if st["chain"] < 0:
            a, b, o = cm.steps[s]["a_id"], cm.steps[s]["b_id"], cm.out[s]
            whole = max((cm.bytes(a) + cm.bytes(b) + cm.bytes(o)) / CFG["dev_bw"], cm.flops(s) / CFG["dev_flops"])
            assert st["state"] == "none" and st["t_gemm"] == pytest.approx(whole, rel=1e-12)
    assert rep["t_total"] == pytest.approx(sum(st["t_gemm"] + st["t_comm"] for st in steps), rel=1e-12)
    assert rep["extra_speedup"] == pytest.approx(rep["speedup"] / P, rel=1e-12)


def test_all_schedule_kinds_occur():
    """Across the seeds the planner keeps, redistributes electively and under force, and
    gathers (so the exhaustive comparison above covers each transition)."""
    tn = ensure_built()
    seen = set()
    for seed in range(12):
        net, path = caterpillar(seed)
        plan = tn.Plan(net, path, host_only=True)
        for P in (4, 16, 64):
            _, steps = plan.distribute(P, **CFG)
            for st in steps:
                seen.add(st["state"] + ("/forced" if st["forced"] else ""))
    assert {"activate", "keep", "redistribute", "redistribute/forced", "gather"} <= seen


def test_single_device_and_bad_config():
    tn = ensure_built()
    net, path = caterpillar(0)
    plan = tn.Plan(net, path, host_only=True)
    rep, steps = plan.distribute(1, **CFG)
    assert rep["n_chains"] == 0 and rep["t_total"] == rep["t_single"] and rep["speedup"] == 1.0
    assert all(st["state"] == "none" for st in steps)
    for bad in (dict(CFG, large_bytes=0.0), dict(CFG, net_bw=-1.0)):
        with pytest.raises(tn.TnError):
            plan.distribute(4, **bad)
    with pytest.raises(tn.TnError):
        plan.distribute(0, **CFG)


def test_unsliced_40_qubit_amplitude_report():
    """The 40-qubit circuit without slicing (intermediates up to 2^32 complex64 = 32 GiB):
    on 8 devices with the paper's 8 GiB threshold the large steps form use-chains and the
    simulated time drops below the one-device time of the same path."""
    tn = ensure_built()
    w = workloads.random_circuit(5, 8, 13, 40)
    plan = tn.Plan(w.net, w.path, prec="bf16x3", host_only=True)
    rep, steps = plan.distribute(8)
    assert rep["n_large_steps"] > 0 and rep["n_chains"] > 0
    assert 1.0 < rep["speedup"] <= 8.0
    assert rep["projected_total"] == pytest.approx(rep["t_total"])  # one slice
    big = [st for st in steps if st["out_bytes"] >= 8 * 2**30]
    assert big and all(st["chain"] >= 0 for st in big)


def test_report_cli(capsys):
    """The report module prints one JSON line per device count with the Eq. 8-10 figures."""
    import json
    from paper_2606_01852_gb300 import distplan
    distplan.main(["--workload", "rc12", "--gpus", "1", "4", "--large-gib", "1e-6"])
    lines = [json.loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    assert [x["n_gpus"] for x in lines] == [1, 4]
    assert lines[0]["n_chains"] == 0 and lines[0]["speedup"] == 1.0
    assert lines[1]["n_chains"] >= 1 and lines[1]["schedule"]
    assert lines[1]["extra_speedup"] == pytest.approx(lines[1]["speedup"] / 4)


def _einsum_pair(a, ma, b, mb, keep):
    """Contract two labelled arrays over their shared labels (unless kept open)."""
    letters = {x: chr(ord("a") + i) if i < 26 else chr(ord("A") + i - 26)
               for i, x in enumerate(sorted(set(ma) | set(mb)))}
    shared = [x for x in ma if x in mb and x not in keep]
    mc = tuple(x for x in ma if x not in shared) + tuple(x for x in mb if x not in shared)
    spec = "".join(letters[x] for x in ma) + "," + "".join(letters[x] for x in mb) + "->" + \
        "".join(letters[x] for x in mc)
    return np.einsum(spec, a, b), mc


def _shard(arr, modes, split, dev, ext):
    """Device `dev`'s part of a tensor split on the labels `split` (mixed radix, first label
    most significant): those labels fixed, removed from the shard."""
    vals, r = {}, dev
    for x in reversed(split):
        vals[x] = r % ext[x]
        r //= ext[x]
    idx = tuple(vals[x] if x in vals else slice(None) for x in modes)
    return arr[idx], tuple(x for x in modes if x not in vals)


def _assemble(shards, modes_shard, split, ext, full_modes):
    """Inverse of _shard: the whole tensor (in full_modes order) from every device's part."""
    shape = tuple(ext[x] for x in full_modes)
    out = np.zeros(shape, dtype=shards[0].dtype)
    for dev, s in enumerate(shards):
        vals, r = {}, dev
        for x in reversed(split):
            vals[x] = r % ext[x]
            r //= ext[x]
        idx = tuple(vals[x] if x in vals else slice(None) for x in full_modes)
        perm = [modes_shard.index(x) for x in full_modes if x not in vals]
        out[idx] = np.transpose(s, perm)
    return out


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("P", [4, 16])
def test_schedule_executes_on_emulated_devices(seed, P):
    """Run the planned schedule on P emulated devices with real data. A tensor made by a
    chain step stays split -- P shards, one per assignment of its split labels -- while
    its consumer is on the same chain; a chain step contracts each shard locally with the
    other operand held whole; a redistribution reassembles and re-splits; a chain's last
    output is gathered. The result must equal the oracle's: it would not if a split label
    were ever contracted locally (each device would sum over its part only)."""
    import oracle
    tn = ensure_built()
    net, path = caterpillar(seed)
    rng = np.random.default_rng(1000 + seed)
    net.tensors = [rng.standard_normal(t.shape) + 1j * rng.standard_normal(t.shape) for t in net.tensors]
    plan = tn.Plan(net, path, host_only=True)
    _, steps = plan.distribute(P, **CFG)
    ext, keep = dict(net.extent), set(net.open_modes)
    T, S = len(net.tensors), len(path.pairs)
    consumer = {}
    for s_, (i, j) in enumerate(path.pairs):
        consumer[i] = consumer[j] = s_
    whole = {t: (np.asarray(net.tensors[t]), tuple(net.modes[t])) for t in range(T)}
    split = {}  # tensor -> (shards, shard modes, split labels, full modes)
    n_split_steps = 0
    for s_, (i, j) in enumerate(path.pairs):
        st, out = steps[s_], T + s_
        carried = [t for t in (i, j) if t in split and steps[t - T]["chain"] == st["chain"] >= 0]
        for t in (i, j):  # a split tensor whose chain ended before this step was gathered
            if t in split and t not in carried:
                sh, ms, sp, fm = split.pop(t)
                whole[t] = (_assemble(sh, ms, sp, ext, fm), fm)
        if carried:
            assert len(carried) == 1 and st["state"] in ("keep", "redistribute", "gather")
            tc = carried[0]
            sh, ms, sp, fm = split.pop(tc)
            b, mb = whole.pop(j if tc == i else i)
            assert not set(sp) & set(mb), "a split label reached the other operand"
            res = [_einsum_pair(x, ms, b, mb, keep) for x in sh]
            cm = res[0][1]
            full = _assemble([r[0] for r in res], cm, sp, ext, tuple(sp) + cm)
            cfull = tuple(sp) + cm
            if st["state"] == "keep":
                assert sorted(st["dist_modes"]) == sorted(sp)
            n_split_steps += 1
        else:
            assert st["state"] in ("none", "activate")
            a, ma = whole.pop(i)
            b, mb = whole.pop(j)
            full, cfull = _einsum_pair(a, ma, b, mb, keep)
        stays_split = st["chain"] >= 0 and out in consumer and steps[consumer[out]]["chain"] == st["chain"]
        if stays_split:
            D = list(st["dist_modes"])
            split[out] = ([_shard(full, cfull, D, d, ext)[0] for d in range(P)], _shard(full, cfull, D, 0, ext)[1],
                          D, cfull)
        else:
            whole[out] = (full, cfull)
    assert n_split_steps > 0
    got, gm = whole[T + S - 1]
    got = np.transpose(got, [gm.index(x) for x in net.open_modes])
    want = oracle.contract(net, path)
    assert np.allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(want).max())
