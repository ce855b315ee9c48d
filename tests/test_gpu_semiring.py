"""GPU parity of the max-plus (tropical) semiring path against the CPU oracle (Sec. III-C:
independent sets on King's subgraphs). Max and add of integers below 2^24 are exact in
FP32, so maximum-independent-set sizes must match exactly; the counting networks run in
the ordinary semiring with exponent scaling and are held to FP32 accuracy (1e-5)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import pins
from tests._lib import ROOT, ensure_built
from tn_inputs import greedy, kings, workloads
from tn_inputs.network import Network, Path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def run_real(tn, plan, net, exp_scaling=False):
    ins = [torch.tensor(np.asarray(t), dtype=torch.float32, device="cuda") for t in net.tensors]
    out = torch.zeros(plan.out_shape, dtype=torch.float64, device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.contract(ins, out, ls)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(ls.cpu()[0])


@pytest.mark.parametrize("L,rho,seed,n_sliced", [(6, 0.8, 1, 0), (8, 0.8, 2, 0), (10, 0.8, 3, 0),
                                                 (12, 0.8, 4, 0), (10, 0.8, 5, 3), (8, 0.9, 6, 4)])
def test_kings_mis_exact(tn, L, rho, seed, n_sliced):
    w = workloads.kings_mis(L, rho, seed, n_sliced)
    plan = tn.Plan(w.net, w.path, w.sliced, prec=tn.TN_R32_FP32_SIMT, semiring="maxplus", max_slice_batch=4)
    got, _ = run_real(tn, plan, w.net)
    want = oracle.contract(w.net, w.path, w.sliced, semiring="maxplus")
    assert float(got) == float(want)
    plan.destroy()


@pytest.mark.parametrize("seed", range(4))
def test_random_graph_mis_and_count_vs_enumeration(tn, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(10, 17))
    edges = sorted({(int(min(u, v)), int(max(u, v))) for u, v in rng.integers(0, n, size=(2 * n, 2)) if u != v})
    want_count, want_mis = pins.independent_sets_enumerate(n, edges)
    t = kings.independent_set_network(n, edges, "tropical")
    c = kings.independent_set_network(n, edges, "counting")
    path = greedy.greedy_path(t, seed=seed, alpha=1.0)
    pt = tn.Plan(t, path, prec=tn.TN_R32_FP32_SIMT, semiring="maxplus")
    pc = tn.Plan(c, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    mis, _ = run_real(tn, pt, t)
    cnt, log_scale = run_real(tn, pc, c)
    assert float(mis) == want_mis
    assert abs(float(cnt) * np.exp(log_scale) / want_count - 1.0) < 1e-5
    pt.destroy()
    pc.destroy()


def test_kings_count_scaled(tn):
    """Number of independent sets of a 10 x 10 King's subgraph (~1e13): the counting
    semiring with per-intermediate exponent scaling, against the oracle."""
    net = kings.kings_network(10, 0.8, 3, "counting")
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    val, log_scale = run_real(tn, plan, net)
    want = float(oracle.contract(net, path))
    assert abs(np.log(float(val)) + log_scale - np.log(want)) < 1e-5
    plan.destroy()


def test_maxplus_splitk_long_reduction(tn):
    """max_k (A[i, k] + B[j, k]) over k = 2^16 with 2 x 2 outputs: the split-K class in the
    max-plus semiring (chunk maxima, then the maximum over chunks)."""
    rng = np.random.default_rng(5)
    kd = (2,) * 16
    A = np.floor(rng.standard_normal((2,) + kd) * 100)
    B = np.floor(rng.standard_normal((2,) + kd) * 100)
    K = tuple(range(16))
    net = Network([A, B], [(16,) + K, (17,) + K], {x: 2 for x in range(18)}, (16, 17))
    path = Path([(0, 1)])
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, semiring="maxplus")
    assert plan.step(0)["cls"] == tn.TN_CLASS_SPLITK
    got, _ = run_real(tn, plan, net)
    a2, b2 = A.reshape(2, -1), B.reshape(2, -1)
    want = np.max(a2[:, None, :] + b2[None, :, :], axis=2)
    assert np.array_equal(got, want)
    plan.destroy()


def test_kings16_full(tn):
    w = workloads.kings16()
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_values.json")))["kings16"]["value"]
    plan = tn.Plan(w.net, w.path, prec=tn.TN_R32_FP32_SIMT, semiring="maxplus")
    got, _ = run_real(tn, plan, w.net)
    assert float(got) == gold[0] == 64.0
    plan.destroy()


def test_batch_maxplus_vs_oracle(tn):
    """48 King's subgraphs (L 4-7) in one persistent launch of the batch engine in the
    max-plus semiring, each MIS size exact, graph replay included."""
    ws = workloads.kings_batch(48, seed=11)
    nets, paths = [w.net for w in ws], [w.path for w in ws]
    b = tn.Batch(nets, paths, complex_=False, exp_scaling=False, semiring="maxplus")
    packed = torch.tensor(b.pack(nets), device="cuda")
    vals = torch.zeros((len(ws), 2), dtype=torch.float64, device="cuda")
    logs = torch.zeros(len(ws), dtype=torch.float64, device="cuda")
    want = np.array([float(oracle.contract(n, p, semiring="maxplus")) for n, p in zip(nets, paths)])
    for graph in (False, True):
        vals.zero_()
        b.contract(packed, vals, logs, graph=graph)
        torch.cuda.synchronize()
        assert np.array_equal(vals[:, 0].cpu().numpy(), want)
        assert np.all(logs.cpu().numpy() == 0.0)
    b.destroy()


def test_maxplus_simt_ksplit(tn):
    """max over k = 2^13 for a 64 x 96 output: the split CUDA-core path in max-plus (part
    maxima, then the maximum over parts) is exact."""
    rng = np.random.default_rng(9)
    kd = (2,) * 13
    A = np.floor(rng.standard_normal((64,) + kd) * 50)
    B = np.floor(rng.standard_normal((96,) + kd) * 50)
    K = tuple(range(2, 15))
    net = Network([A, B], [(0,) + K, (1,) + K], {0: 64, 1: 96, **{x: 2 for x in K}}, (0, 1))
    plan = tn.Plan(net, Path([(0, 1)]), prec=tn.TN_R32_FP32_SIMT, semiring="maxplus")
    assert plan.step(0)["cls"] == tn.TN_CLASS_SIMT
    got, _ = run_real(tn, plan, net)
    want = np.max(A.reshape(64, -1)[:, None, :] + B.reshape(96, -1)[None, :, :], axis=2)
    assert np.array_equal(got, want)
    plan.destroy()
