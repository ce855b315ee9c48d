"""Many small networks in one persistent launch (tn_batch_*) against the CPU oracle.

Partition functions are compared on ln Z (absolute 1e-5: FP32 arithmetic along paths
of ~60 steps, every intermediate renormalised by an exact power of two), amplitudes at
the relative 1e-5 bar of the other GPU tests.
"""
import numpy as np
import pytest
import torch

import oracle
from tests._lib import ensure_built
from tn_inputs import circuits, greedy, ising_pf, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def run_batch(tn, nets, paths, complex_=False, scaling=True, graph=False, autotune=False, semiring="standard"):
    b = tn.Batch(nets, paths, complex_=complex_, exp_scaling=scaling, semiring=semiring)
    packed = torch.tensor(b.pack(nets), device="cuda")
    b._packed = packed
    vals = torch.zeros((len(nets), 2), dtype=torch.float64, device="cuda")
    logs = torch.zeros(len(nets), dtype=torch.float64, device="cuda")
    if autotune:
        b.autotune(packed, vals, logs)
    b.contract(packed, vals, logs, graph=graph)
    torch.cuda.synchronize()
    v, l = vals.cpu().numpy(), logs.cpu().numpy()
    return b, v, l


def test_ising_ensemble_lnz(tn):
    ws = workloads.ising3r(128, seed=11)
    b, v, l = run_batch(tn, [w.net for w in ws], [w.path for w in ws])
    for i, w in enumerate(ws):
        want = oracle.contract(w.net, w.path)
        assert v[i, 0] > 0
        assert abs(np.log(v[i, 0]) + l[i] - np.log(want)) < 1e-5, i


def test_overflowing_rings_need_scaling(tn):
    """Rings of 200-400 spins at beta = 1: Z ~ 1e100-1e200 (beyond FP32 and, for some,
    FP64 without the log scale); checked against the transfer-matrix closed form."""
    nets, paths, want = [], [], []
    for n in (200, 300, 400):
        net = ising_pf.ring_network(n, 1.0, 1.0)
        nets.append(net)
        paths.append(greedy.greedy_path(net, seed=0))
        want.append(n * np.log(2 * np.cosh(1.0)) + np.log1p(np.tanh(1.0) ** n))
    b, v, l = run_batch(tn, nets, paths)
    for i in range(3):
        assert abs(np.log(v[i, 0]) + l[i] - want[i]) < 1e-5 * want[i]


@pytest.mark.parametrize("scaling", [False, True])
def test_complex_amplitudes(tn, scaling):
    nets, paths = [], []
    for s in range(24):
        net = circuits.amplitude_network(3, 3, 8, 100 + s)
        nets.append(net)
        paths.append(greedy.greedy_path(net, seed=s, alpha=1.0))
    b, v, l = run_batch(tn, nets, paths, complex_=True, scaling=scaling)
    # Amplitudes of a normalised 9-qubit state are ~2^-4.5 in size; one that happens to
    # be much smaller comes out of cancellation between terms of that size, so FP32
    # rounding bounds its error relative to the typical size, not to itself.
    typical = 2.0 ** (-9 / 2)
    for i in range(len(nets)):
        got = complex(v[i, 0], v[i, 1]) * np.exp(l[i])
        want = oracle.contract(nets[i], paths[i])
        assert abs(got - want) / max(abs(want), typical) < 1e-5, i


def test_graph_replay_and_autotune_match(tn):
    ws = workloads.ising3r(64, seed=12)
    nets, paths = [w.net for w in ws], [w.path for w in ws]
    _, v0, l0 = run_batch(tn, nets, paths)
    _, v1, l1 = run_batch(tn, nets, paths, graph=True)
    b2, v2, l2 = run_batch(tn, nets, paths, autotune=True, graph=True)
    t, c, g, sm = b2.launch_shape()
    assert t in (32, 64, 128, 256) and c in (2, 4, 8, 16) and g in (1, 4, 8)
    # same per-network arithmetic whatever the launch shape: bitwise equal
    assert np.array_equal(v0, v1) and np.array_equal(l0, l1)
    assert np.array_equal(v0, v2) and np.array_equal(l0, l2)


@pytest.mark.parametrize("kind", ["ising", "complex", "maxplus"])
def test_warp_per_network_form_bitwise_equal(tn, kind):
    """The warp-per-network form (warp-synchronous steps, several networks per CTA) and the
    arenas in shared memory give the same bits as the CTA-per-network form with global
    arenas: one lane computes each output element with k in order, and the renormalisation
    is an exact power of two chosen from the same maximum. Checked on partition functions (scaled), complex amplitudes and max-plus
    independent sets, with a ragged last CTA (networks not a multiple of the warps per CTA)."""
    from tn_inputs import kings
    if kind == "ising":
        ws = workloads.ising3r(45, seed=21)
        nets, paths = [w.net for w in ws], [w.path for w in ws]
        kw = dict(complex_=False, scaling=True)
    elif kind == "complex":
        nets = [circuits.amplitude_network(3, 3, 8, 300 + s) for s in range(13)]
        paths = [greedy.greedy_path(n, seed=0, alpha=1.0) for n in nets]
        kw = dict(complex_=True, scaling=False)
    else:
        ws = workloads.kings_batch(19, seed=4)
        nets, paths = [w.net for w in ws], [w.path for w in ws]
        kw = dict(complex_=False, scaling=False, semiring="maxplus")
    b, v0, l0 = run_batch(tn, nets, paths, **kw)
    # shared-memory arenas of 1 Ki, 4 Ki and 12 Ki floats: the networks above the size keep
    # their global arenas, so one launch mixes both
    for shape in ((32, 4, 4), (32, 8, 8), (32, 16, 1), (256, 2, 1), (256, 2, 1, 12288), (32, 2, 4, 4096),
                  (128, 4, 1, 1024)):
        b.set_launch_shape(*shape)
        v = torch.zeros_like(torch.tensor(v0)).cuda()
        l = torch.zeros_like(torch.tensor(l0)).cuda()
        b.contract(b._packed, v, l)
        torch.cuda.synchronize()
        assert np.array_equal(v.cpu().numpy(), v0) and np.array_equal(l.cpu().numpy(), l0), shape
    with pytest.raises(tn.TnError):
        b.set_launch_shape(64, 4, 4)  # a warp per network takes 32 threads
    with pytest.raises(tn.TnError):
        b.set_launch_shape(32, 8, 8, 8192)  # 8 x 8 slots of 32 KiB exceed an SM's shared memory
