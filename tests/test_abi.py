"""The C-ABI library loads and exports every symbol include/tn.h declares, and the
host-only planner follows Sec. IV-A (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from tests._lib import ROOT, ensure_built
from tn_inputs import greedy, workloads, circuits, kings
from tn_inputs.network import Network, Path


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "tn.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    tn = ensure_built()
    lib = ctypes.CDLL(tn.LIB_PATH)
    names = declared_functions()
    assert "tn_plan" in names and "tn_serve_poll" in names and "tn_last_error" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _fig2_network():
    a, b, c, d, e, f, g, h = range(8)
    ext = {x: 2 for x in range(8)}
    rng = np.random.default_rng(0)
    I1 = (c, a, d, b)   # arbitrary local orders (panel A)
    I2 = (f, d, e, c)
    I3 = (b, h, f, g)
    mk = lambda ms: rng.standard_normal((2,) * len(ms)) + 0j
    net = Network([mk(I1), mk(I2), mk(I3)], [I1, I2, I3], ext, (g, a, h, e))
    net.check()
    return net, Path([(0, 1), (3, 2)])


def test_fig2_worked_example_golden():
    tn = ensure_built()
    net, path = _fig2_network()
    plan = tn.Plan(net, path, host_only=True)
    want = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "fig2_mode_reorder.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            want[k] = v
    name = lambda ms: "".join("abcdefgh"[x] for x in ms)
    ids = {"I1": 0, "I2": 1, "I3": 2, "I4": 3, "I5": 4}
    for k, v in want.items():
        assert name(plan.layout(ids[k])) == v, (k, name(plan.layout(ids[k])), v)
    # step 1's output interleaves the two operands' modes (e outlives b)
    assert plan.info()["leaf_permutes"] == 3


def _lifetimes(net, path):
    """Step index at which each label is summed; open labels never are."""
    T = net.n_tensors
    sets = [set(m) for m in net.modes]
    when = {}
    for s, (i, j) in enumerate(path.pairs):
        for x in sets[i] & sets[j]:
            when[x] = s
        sets.append((sets[i] | sets[j]) - (sets[i] & sets[j]))
    return when


@pytest.mark.parametrize("seed", range(5))
def test_reorder_invariants_random_trees(seed):
    """Every operand is [retained in output order | reduced]; every tensor's modes are
    sorted by remaining lifetime, longest-lived leftmost (Sec. IV-A); no label is
    created or dropped."""
    tn = ensure_built()
    net = circuits.amplitude_network(3, 3, 6, seed)
    path = greedy.greedy_path(net, seed=seed, temperature=0.3)
    plan = tn.Plan(net, path, host_only=True)
    T = net.n_tensors
    when = _lifetimes(net, path)
    inf = 10**9
    sets = [set(m) for m in net.modes]
    for s, (i, j) in enumerate(path.pairs):
        sets.append((sets[i] | sets[j]) - (sets[i] & sets[j]))
    for tid in range(T + len(path.pairs)):
        lay = plan.layout(tid)
        assert set(lay) == sets[tid]
        life = [when.get(x, inf) for x in lay]
        assert life == sorted(life, reverse=True), (tid, lay, life)
    for s, (i, j) in enumerate(path.pairs):
        out = plan.layout(T + s)
        K = sorted(sets[i] & sets[j])
        for op in (i, j):
            lay = plan.layout(op)
            kept = [x for x in out if x in sets[op]]
            assert list(lay) == kept + K


def test_plan_step_costs_match_oracle_counts():
    """tn_plan_info's C_t, C_m, C_s (Sec. II-B Eqs. 1-3) equal the oracle's counts."""
    import oracle
    tn = ensure_built()
    w = workloads.rc12()
    plan = tn.Plan(w.net, w.path, host_only=True)
    info = plan.info()
    want = oracle.path_costs(w.net, w.path)
    assert info["Ct"] == want["Ct"] and info["Cm"] == want["Cm"] and info["Cs"] == want["Cs"]
    assert info["flops"] == 8 * want["Ct"]
    for s, c in enumerate(oracle.step_costs(w.net, w.path)):
        st = plan.step(s)
        assert st["m"] * st["n"] * st["k"] == c["Ct"]
        assert sorted([st["m"], st["n"]]) == sorted([c["m"], c["n"]]) and st["k"] == c["k"]


def test_plan_rejects_bad_input():
    tn = ensure_built()
    net, path = _fig2_network()
    with pytest.raises(tn.TnError) as e:
        tn.Plan(net, Path([(0, 1)]), host_only=True)       # not a full tree
    assert e.value.status == tn.TN_ERR_INVALID
    with pytest.raises(tn.TnError):
        tn.Plan(net, Path([(0, 1), (3, 3)]), host_only=True)  # reused operand
    bad = Network(net.tensors, [net.modes[0], net.modes[1], net.modes[0]], net.extent, net.open_modes)
    with pytest.raises(tn.TnError) as e:
        tn.Plan(bad, path, host_only=True)                  # label in three tensors
    assert e.value.status in (tn.TN_ERR_UNSUPPORTED, tn.TN_ERR_INVALID)
    with pytest.raises(tn.TnError) as e:
        tn.Plan(net, path, sliced=[6], host_only=True)       # slicing an open label
    assert e.value.status == tn.TN_ERR_UNSUPPORTED


def test_sliced_plan_batches():
    tn = ensure_built()
    w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=4, host_only=True)
    info = plan.info()
    assert info["n_slices"] == 16 and info["slice_batch"] == 4 and info["n_passes"] == 4


@pytest.mark.parametrize("prec", ["bf16x3", "3xtf32", "fp32"])
def test_split_bf16_operands_exactly_the_tc_operands(prec):
    """In a BF16x3 plan every operand of a tensor-core step (and nothing else) is stored
    in the split-BF16 form, so its producer writes hi/lo planes and the GEMM reads them
    as they are; the other forms store everything planar."""
    tn = ensure_built()
    w = workloads.random_circuit(4, 5, 12, 40, n_sliced=3)
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, max_slice_batch=4, host_only=True)
    n_t = len(w.net.tensors) + len(w.path.pairs)
    tc_operands = set()
    for s in range(len(w.path.pairs)):
        st = plan.step(s)
        if st["cls"] == tn.TN_CLASS_TC:
            tc_operands |= {st["a_id"], st["b_id"]}
    if prec != "fp32":
        assert tc_operands, "the circuit should have tensor-core steps"
    split = {t for t in range(n_t) if plan.tensor(t)["format"] == 1}
    assert split == (tc_operands if prec == "bf16x3" else set())
    plan.destroy()


def test_maxplus_policy_checks():
    tn = ensure_built()
    net = kings.kings_network(5, 0.8, 1)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    plan = tn.Plan(net, path, prec=tn.TN_R32_FP32_SIMT, semiring="maxplus", host_only=True)
    classes = {plan.step(s)["cls"] for s in range(len(path.pairs))}
    assert classes <= {tn.TN_CLASS_SIMT, tn.TN_CLASS_SPLITK}
    plan.destroy()
    for kw in (dict(prec="3xtf32"), dict(prec=tn.TN_R32_FP32_SIMT, exp_scaling=True), dict(prec="fp32")):
        with pytest.raises(tn.TnError) as e:
            tn.Plan(net, path, semiring="maxplus", host_only=True, **kw)
        assert "TN_ERR_UNSUPPORTED" in str(e.value)


def test_batch_maxplus_policy_checks():
    tn = ensure_built()
    ws = workloads.kings_batch(4, seed=2)
    nets, paths = [w.net for w in ws], [w.path for w in ws]
    b = tn.Batch(nets, paths, complex_=False, exp_scaling=False, semiring="maxplus", host_only=True)
    assert b.flops > 0
    b.destroy()
    with pytest.raises(tn.TnError) as e:
        tn.Batch(nets, paths, complex_=False, exp_scaling=True, semiring="maxplus", host_only=True)
    assert "TN_ERR_UNSUPPORTED" in str(e.value)


def test_unbuilt_forms_are_refused_not_substituted():
    """A request the engine cannot run as asked is a status, not a silent change of form:
    the real BF16x3 form is not built, and the 3M product does not rescale."""
    tn = ensure_built()
    from tn_inputs import ising_pf
    net = ising_pf.random_3regular_network(20, 1, beta=0.5)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    for scaling in (False, True):
        with pytest.raises(tn.TnError) as e:
            tn.Plan(net, path, prec=tn.TN_R32_BF16X3, exp_scaling=scaling, host_only=True)
        assert e.value.status == tn.TN_ERR_UNSUPPORTED and "not built" in str(e.value)
    w = workloads.rc12()
    with pytest.raises(tn.TnError) as e:
        tn.Plan(w.net, w.path, prec="bf16x3m", exp_scaling=True, host_only=True)
    assert e.value.status == tn.TN_ERR_UNSUPPORTED and "scaling" in str(e.value)
    # every other form takes scaling, real networks the TF32 and 3xTF32 forms
    for prec in (tn.TN_R32_FP32_SIMT, tn.TN_R32_TF32, tn.TN_R32_3XTF32):
        tn.Plan(net, path, prec=prec, exp_scaling=True, host_only=True).destroy()
    for prec in ("fp32", "tf32", "3xtf32", "bf16x3"):
        tn.Plan(w.net, w.path, prec=prec, exp_scaling=True, host_only=True).destroy()


def test_real_tensor_core_forms_take_the_large_steps():
    """Eq. 6 on a real network: an Ising spin glass on a 16 x 16 lattice planned in the
    real TF32 and 3xTF32 forms puts its large steps (the flops) on the tensor cores, in the
    plain FP32 form on the CUDA cores; the step analysis is the same in every form."""
    tn = ensure_built()
    from tn_inputs import ising_pf
    net = ising_pf.lattice_network(16, 16, 0.44, seed=1)
    path = greedy.greedy_path(net, seed=0, alpha=1.0)
    shapes = None
    for prec in (tn.TN_R32_FP32_SIMT, tn.TN_R32_TF32, tn.TN_R32_3XTF32):
        plan = tn.Plan(net, path, prec=prec, exp_scaling=True, host_only=True)
        try:
            steps = [plan.step(s) for s in range(len(path.pairs))]
            info = plan.info()
        finally:
            plan.destroy()
        sh = sorted((s["m"] * s["n"] * s["k"]) for s in steps)
        shapes = shapes or sh
        assert sh == shapes
        tc_flops = info["flops_per_class"][tn.TN_CLASS_TC]
        if prec == tn.TN_R32_FP32_SIMT:
            assert tc_flops == 0
        else:
            assert tc_flops > 0.95 * info["flops"]
            big = max(steps, key=lambda s: s["m"] * s["n"] * s["k"])
            assert big["cls"] == tn.TN_CLASS_TC


def test_cost_model_rates_drive_the_kernel_choice():
    """Eq. 6 with the configured rates: a 4096^2 x 4096 complex step goes to the tensor
    cores at the default rates and to the CUDA cores when the tensor-core rate is set far
    below the FMA rate; bad rates are refused."""
    tn = ensure_built()
    from tn_inputs.network import Network as N2
    ext = {0: 4096, 1: 4096, 2: 4096}
    z = np.zeros((1, 1), np.complex128)
    net = N2([z, z], [(0, 2), (1, 2)], ext, (0, 1))
    old = tn.binding.cost_model()
    try:
        assert tn.Plan(net, Path([(0, 1)]), prec="bf16x3", host_only=True).step(0)["cls"] == tn.TN_CLASS_TC
        tn.binding.set_cost_model(old["hbm_bytes_per_s"], old["simt_flops"], [1e9, 1e9, 1e9])
        assert tn.binding.cost_model()["tc_flops"] == [1e9, 1e9, 1e9]
        assert tn.Plan(net, Path([(0, 1)]), prec="bf16x3", host_only=True).step(0)["cls"] == tn.TN_CLASS_SIMT
        with pytest.raises(tn.TnError) as e:
            tn.binding.set_cost_model(0.0, 1.0, [1.0, 1.0, 1.0])
        assert e.value.status == tn.TN_ERR_INVALID
    finally:
        tn.binding.set_cost_model(old["hbm_bytes_per_s"], old["simt_flops"], old["tc_flops"])
    assert tn.binding.cost_model() == old


def test_plan_launches_counts_the_call():
    """tn_plan_launches on host-only plans (no paired-SM bands without a device): per pass one
    staging launch, one per tiled leaf, one per step outside step chains (two for split-k and
    k-split steps; the slice-invariant steps only in the first pass), one per step chain (in
    later passes only if it holds a batched step) and one for the slice sum."""
    tn = ensure_built()
    w = workloads.random_circuit(3, 4, 8, 3, n_sliced=4)
    for batch in (16, 3, 1):
        plan = tn.Plan(w.net, w.path, w.sliced, max_slice_batch=batch, host_only=True)
        info = plan.info()
        steps = [plan.step(s) for s in range(info["n_steps"])]
        per = [0 if st["chain"] >= 0 else (2 if (st["cls"] == tn.TN_CLASS_SPLITK or st["ksplit"] > 1) else 1)
               for st in steps]
        chains = sorted({st["chain"] for st in steps if st["chain"] >= 0})
        chain_b = sum(1 for c in chains if any(st["batched"] for st in steps if st["chain"] == c))
        leaves = [plan.tensor(t) for t in range(plan.n_leaves)]
        tiled = sum(1 for x in leaves if x["tiled"])
        tiled_b = sum(1 for x in leaves if x["tiled"] and x["batched"])
        for count in (1, 5, 16):
            passes = -(-count // info["slice_batch"])
            batched = sum(p for p, st in zip(per, steps) if st["batched"])
            want = (passes * 2 + sum(per) + (passes - 1) * batched + tiled + (passes - 1) * tiled_b +
                    len(chains) + (passes - 1) * chain_b)
            assert plan.launches_per_call(count) == want, (batch, count)
        plan.destroy()


def test_step_chains_are_runs_of_tiny_cuda_core_steps():
    """The step chains: maximal runs (at least two) of consecutive CUDA-core steps, without a
    k split, whose work (m n k, times the slice batch for batched steps, complex counted four
    times) is at most 2^16 multiply-adds; every step outside a chain that is such a step
    stands alone between steps that are not. A larger slice batch takes batched steps out."""
    tn = ensure_built()
    for w, kw in ((workloads.kising44(), {}), (workloads.rc12(), {}),
                  (workloads.random_circuit(3, 4, 8, 3, n_sliced=4), {"max_slice_batch": 16})):
        plan = tn.Plan(w.net, w.path, w.sliced, host_only=True, **kw)
        info = plan.info()
        steps = [plan.step(s) for s in range(info["n_steps"])]
        nb = info["slice_batch"]
        cw = 4 if plan.is_complex else 1
        tiny = [st["cls"] == tn.TN_CLASS_SIMT and st["ksplit"] == 1 and
                st["m"] * st["n"] * st["k"] * cw * (nb if st["batched"] else 1) <= 1 << 16 for st in steps]
        chain = [st["chain"] for st in steps]
        assert any(c >= 0 for c in chain)
        for s, st in enumerate(steps):
            if chain[s] >= 0:
                assert tiny[s]
                if s > 0 and chain[s - 1] >= 0:
                    assert chain[s - 1] in (chain[s], chain[s] - 1)
                if s > 0 and chain[s - 1] == chain[s] - 1 and chain[s - 1] >= 0:
                    raise AssertionError("two chains back to back would be one run")
            elif tiny[s]:
                assert not (s > 0 and tiny[s - 1]) and not (s + 1 < len(steps) and tiny[s + 1])
        ids = [c for c in chain if c >= 0]
        assert ids == sorted(ids) and all(ids.count(c) >= 2 for c in set(ids))
        plan.destroy()
