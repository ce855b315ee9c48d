"""tn_contract_graph: a plan's whole call (all passes and steps) replayed from a CUDA graph
gives the same bits as tn_contract, re-reads its input buffers at every launch, and
re-captures when a pointer changes."""
import numpy as np
import pytest
import torch

import oracle
from tests._lib import ensure_built
from tests.test_gpu_parity import dev_inputs, rel_err
from tn_inputs import greedy, ising_pf, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


@pytest.mark.parametrize("name,prec,batch", [("kising44", "bf16x3", 0), ("rc12", "fp32", 0),
                                             ("rc12s", "fp32", 3)])
def test_graph_replay_same_bits(tn, name, prec, batch):
    if name == "rc12s":  # the 12-qubit circuit sliced 16 ways, 3 slices per pass: 6 passes
        w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    else:
        w = workloads.BY_NAME[name]()
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=batch)
    ins = dev_inputs(w.net, True)
    ref = torch.zeros(plan.out_shape, dtype=torch.complex128, device="cuda")
    plan.contract(ins, ref)
    out = torch.zeros(plan.out_shape, dtype=torch.complex128, device="cuda")
    plan.contract_graph(ins, out)            # runs, then captures
    torch.cuda.synchronize()
    assert np.array_equal(bits(out.cpu().numpy()), bits(ref.cpu().numpy()))
    for _ in range(3):                       # replays
        out.zero_()
        plan.contract_graph(ins, out)
        torch.cuda.synchronize()
        assert np.array_equal(bits(out.cpu().numpy()), bits(ref.cpu().numpy()))
    if name != "kising44":  # (its oracle value is checked in the full-size tests)
        want = oracle.contract(w.net, w.path, w.sliced)
        assert rel_err(out.cpu().numpy(), want) < 1e-5
    plan.destroy()


def test_graph_reads_buffers_and_recaptures(tn):
    """New values in the captured input buffers are contracted by a replay; another output
    buffer re-captures; per-step profiling refuses graph mode."""
    net = ising_pf.random_3regular_network(40, 5, beta=0.4)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True)
    ins = dev_inputs(net, False)
    out = torch.zeros((), dtype=torch.float64, device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan.contract_graph(ins, out, ls)
    plan.contract_graph(ins, out, ls)
    torch.cuda.synchronize()
    lnz = float(np.log(float(out.cpu()))) + float(ls.cpu()[0])
    assert abs(lnz - np.log(oracle.contract(net, path))) < 1e-5
    # double every vertex tensor in place: ln Z grows by n ln 2
    for t in ins:
        t.mul_(2.0)
    plan.contract_graph(ins, out, ls)
    torch.cuda.synchronize()
    lnz2 = float(np.log(float(out.cpu()))) + float(ls.cpu()[0])
    assert abs(lnz2 - lnz - 40 * np.log(2.0)) < 1e-5
    # another output buffer: a new capture, the same value
    out2 = torch.zeros((), dtype=torch.float64, device="cuda")
    plan.contract_graph(ins, out2, ls)
    plan.contract_graph(ins, out2, ls)
    torch.cuda.synchronize()
    assert float(out2.cpu()) == float(out.cpu())
    plan.profile(True)
    with pytest.raises(tn.binding.TnError):
        plan.contract_graph(ins, out2, ls)
    plan.profile(False)
    plan.destroy()
