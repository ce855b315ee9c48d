"""Tiled leaf staging (the permutation kernel for large leaves): its index arithmetic,
replayed on the host by tn_plan_check_staging, maps every staged element to the source
element the declared order places there, writes each once, and pairs 16-byte loads only
on adjacent elements -- for shuffled orders, identity orders, extents other than 2,
sliced labels and the split-BF16 layout."""
import numpy as np
import pytest

from tests._lib import ensure_built
from tn_inputs import circuits


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def plan_of(tn, net, sliced=(), prec="fp32", batch=0):
    return tn.Plan(net, circuits.state_path(net), sliced, prec=prec, host_only=True, max_slice_batch=batch)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("shuffle", [True, False])
def test_state_leaf_power_of_two(tn, seed, shuffle):
    net = circuits.state_network(16, 3, seed, shuffle=shuffle)
    for prec in ("fp32", "bf16x3"):
        plan = plan_of(tn, net, prec=prec)
        # the pipelined form where each index group is one 32-wide chunk and the declared
        # innermost qubit is outside the staged copy's innermost ones (16-byte loads), else
        # the general form (seeds 1 and 2 put it among them)
        want = 2 if (not shuffle or seed in (0, 3)) else 1
        if not shuffle:
            want = plan.tensor(0)["tiled"]  # identity order: either form, checked below
        assert plan.tensor(0)["tiled"] == want and plan.tensor(1)["tiled"] == 0
        plan.check_staging()
        plan.destroy()


def test_state_leaf_other_extents(tn):
    ext = [3, 5, 2, 7, 4, 3, 2, 6]
    net = circuits.state_network(8, 0, 5, extents=ext, gate_pairs=[(0, 1), (2, 3), (4, 5), (6, 7)])
    plan = plan_of(tn, net)
    assert plan.tensor(0)["tiled"] == 1  # extents that do not make 32-wide chunks: the general form
    plan.check_staging()


def test_state_leaf_vector_loads_chosen(tn):
    """A shuffled 2^14 state whose declared innermost qubit is not among the staged copy's
    innermost ones: loads go along the input group (16-byte pairs)."""
    net = circuits.state_network(14, 0, 2, gate_pairs=[(q, (q + 1) % 14) for q in range(0, 14, 2)])
    plan = plan_of(tn, net)
    plan.check_staging()


@pytest.mark.parametrize("n_sliced", [1, 3])
def test_state_leaf_sliced(tn, n_sliced):
    """Sliced labels of the large leaf are fixed per batch entry (every slice id checked up
    to the limit)."""
    net = circuits.state_network(16, 0, 7, gate_pairs=[(q, q + 1) for q in range(0, 16, 2)])
    sliced = list(net.modes[0][:n_sliced])  # the first declared labels (all consumed by gates)
    plan = plan_of(tn, net, sliced, batch=2)
    assert plan.tensor(0)["tiled"] in (1, 2) and plan.tensor(0)["batched"] == 1
    plan.check_staging(max_slices=8)
    sliced = list(net.modes[0][-n_sliced:])  # the last declared labels: no 16-byte pairs
    plan = plan_of(tn, net, sliced, batch=2)
    plan.check_staging(max_slices=8)


def test_large_leaf_2_to_20(tn):
    net = circuits.state_network(20, 2, 11)
    plan = plan_of(tn, net, prec="bf16x3")
    plan.check_staging()


def test_large_leaf_2_to_26(tn):
    """The size of the GPU staging test and of the sv26 benchmark leaf (rank 26)."""
    net = circuits.state_network(26, 3, 26)
    plan = plan_of(tn, net)
    assert plan.tensor(0)["tiled"] == 2
    plan.check_staging()
