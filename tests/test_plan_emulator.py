"""CPU replay of a plan exactly as the executor runs it: the same workspace offsets,
the same slice batches and passes (slice-invariant steps only in the first pass,
pinned tensors kept), the same operand roles and output offset maps -- with numpy
matrix products in place of the kernels. It checks the planner's memory plan and
layouts end to end against the oracle without a GPU: an aliasing error between
tensors that are live in different passes, or a wrong offset map, changes the result.
"""
import math

import numpy as np
import pytest

import oracle
from tests._lib import ensure_built
from tests.test_gpu_parity import gate_chain_network, rel_err
from tests.test_oracle_pins import random_network
from tn_inputs import greedy, workloads


def offsets(dims, count):
    idx = np.arange(count, dtype=np.int64)
    off = np.zeros(count, dtype=np.int64)
    for ext, stride in reversed(dims):
        off += (idx % ext) * stride
        idx //= ext
    return off


def replay(plan, net, sliced, begin=0, count=None, cplx=True):
    info = plan.info()
    T, S = net.n_tensors, info["n_steps"]
    B = info["slice_batch"]
    count = info["n_slices"] if count is None else count
    ws = np.full(info["workspace_bytes"] // 4 + 1, np.nan)  # poisoned: unwritten reads show
    tens = [plan.tensor(t) for t in range(T + S)]
    steps = [plan.step(s) for s in range(S)]
    layout = [plan.layout(t) for t in range(T)]

    # floats per element of a stored copy: 1 real, 2 complex, 3 in the 3M split form (whose
    # planes this float replay does not reproduce, only their footprint)
    fpe = [1 if not cplx else (3 if x["format"] == 2 else 2) for x in tens]

    def base(t, b, p):
        return tens[t]["offset"] // 4 + (b * fpe[t] + p) * tens[t]["size"]

    def read(t, b, shape):
        sz = tens[t]["size"]
        bb = b if tens[t]["batched"] else 0
        x = ws[base(t, bb, 0): base(t, bb, 0) + sz]
        if cplx:
            x = x + 1j * ws[base(t, bb, 1): base(t, bb, 1) + sz]
        return x.reshape(shape)

    total = 0.0
    for p in range(math.ceil(count / B)):
        nb = min(B, count - p * B)
        for t in range(T):
            if p > 0 and not tens[t]["batched"]:
                continue
            for b in range(nb if tens[t]["batched"] else 1):
                sid, vals = begin + p * B + b, {}
                for x in reversed(sliced):
                    vals[x] = sid % net.extent[x]
                    sid //= net.extent[x]
                a = np.asarray(net.tensors[t])[tuple(vals.get(x, slice(None)) for x in net.modes[t])]
                kept = [x for x in net.modes[t] if x not in vals]
                a = np.transpose(a, [kept.index(x) for x in layout[t]]).ravel()
                ws[base(t, b, 0): base(t, b, 0) + a.size] = a.real
                if cplx:
                    ws[base(t, b, 1): base(t, b, 1) + a.size] = a.imag
        for s, st in enumerate(steps):
            if p > 0 and not st["batched"]:
                continue
            m, n, k = st["m"], st["n"], st["k"]
            idx = offsets(st["rows"], m)[:, None] + offsets(st["cols"], n)[None, :]
            for b in range(nb if st["batched"] else 1):
                c = read(st["a_id"], b, (m, k)) @ read(st["b_id"], b, (n, k)).T
                ws[base(T + s, b, 0) + idx] = c.real
                if cplx:
                    ws[base(T + s, b, 1) + idx] = c.imag
        root = T + S - 1
        for b in range(nb if tens[root]["batched"] else 1):
            total = total + read(root, b, (tens[root]["size"],))
    shape = tuple(net.extent[x] for x in net.open_modes)
    return np.asarray(total).reshape(shape)


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


@pytest.mark.parametrize("batch", [1, 3, 5, 16])
def test_replay_sliced_circuit(tn, batch):
    w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=batch, host_only=True)
    got = replay(plan, w.net, w.sliced)
    assert not np.isnan(got).any()
    assert rel_err(got, oracle.contract(w.net, w.path, w.sliced)) < 1e-12


@pytest.mark.parametrize("batch", [1, 2, 3])
def test_replay_many_pinned(tn, batch):
    """A deeper circuit with 3 sliced labels: many slice-invariant tensors are made late
    in the first pass and read by every later pass."""
    w = workloads.random_circuit(4, 5, 12, 40, n_sliced=3)
    plan = tn.Plan(w.net, w.path, w.sliced, prec="3xtf32", max_slice_batch=batch, host_only=True)
    pinned = sum(plan.tensor(t)["pinned"] for t in range(w.net.n_tensors + len(w.path.pairs)))
    assert pinned > 0
    got = replay(plan, w.net, w.sliced)
    assert rel_err(got, oracle.contract(w.net, w.path, w.sliced)) < 1e-12


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x3m"])
@pytest.mark.parametrize("batch", [1, 3])
def test_replay_split_forms(tn, prec, batch):
    """Plans whose tensor-core operands are stored split (4 BF16 planes in 8 bytes, or the
    3M form's 6 planes in 12 bytes per element): every copy inside its reserved bytes and no
    live overlap, replayed against the oracle."""
    w = workloads.random_circuit(4, 5, 12, 40, n_sliced=3)
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=batch, host_only=True)
    fmts = {plan.tensor(t)["format"] for t in range(w.net.n_tensors + len(w.path.pairs))}
    assert fmts == {0, 2 if prec == "bf16x3m" else 1}
    for t in range(w.net.n_tensors + len(w.path.pairs)):
        x = plan.tensor(t)
        per = 12 if x["format"] == 2 else 8
        assert x["bytes"] >= x["size"] * per * (batch if x["batched"] else 1)
    got = replay(plan, w.net, w.sliced)
    assert rel_err(got, oracle.contract(w.net, w.path, w.sliced)) < 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_replay_random_open_networks(tn, seed):
    net = random_network(200 + seed, n_tensors=8, n_labels=15, n_open=3)
    path = greedy.greedy_path(net, seed=seed, temperature=0.5)
    plan = tn.Plan(net, path, host_only=True)
    assert rel_err(replay(plan, net, []), oracle.contract(net, path)) < 1e-12


def test_replay_stream_chain(tn):
    net, path = gate_chain_network()
    plan = tn.Plan(net, path, host_only=True)
    assert rel_err(replay(plan, net, []), oracle.contract(net, path)) < 1e-12


def test_replay_rc40_sampled_slices(tn):
    """The headline plan's layout and memory plan, at its real slice batch, on two
    passes of one-slice batches is too costly here; check instead that every tensor of
    the plan at its benchmark batch sits inside the workspace with no two simultaneously
    live tensors overlapping (the planner's own self-check passed when the plan built)."""
    w = workloads.rc40()
    plan = tn.Plan(w.net, w.path, w.sliced, prec="3xtf32", max_slice_batch=128, host_only=True)
    info = plan.info()
    ts = [plan.tensor(t) for t in range(w.net.n_tensors + len(w.path.pairs))]
    assert all(t["offset"] + t["bytes"] <= info["workspace_bytes"] for t in ts)
    pinned = [t for t in ts if t["pinned"]]
    for p in pinned:
        for t in ts:
            if t is p:
                continue
            overlap = t["offset"] < p["offset"] + p["bytes"] and p["offset"] < t["offset"] + t["bytes"]
            assert not overlap, (p, t)
