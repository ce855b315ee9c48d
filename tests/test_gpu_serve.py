"""The serve loop (tn_serve_*): continuous admission, results independent of the mix,
refusals returned as statuses."""
import time

import numpy as np
import pytest

import oracle
import paper_2606_01852_gb300  # noqa: F401  (built by the fixture)
from tests._lib import ensure_built
from tn_inputs import circuits, greedy, ising_pf, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    return ensure_built()


def amp_requests(n, seed=0):
    """n amplitude requests of one 3x4 circuit with different bitstrings (one plan)."""
    rng = np.random.default_rng(seed)
    nets = []
    for _ in range(n):
        bits = tuple(int(b) for b in rng.integers(0, 2, size=12))
        nets.append(circuits.amplitude_network(3, 4, 8, 12, bitstring=bits))
    return nets


def host_inputs(net, cplx=True):
    dt = np.complex64 if cplx else np.float32
    return [np.ascontiguousarray(np.asarray(t, dtype=dt)) for t in net.tensors]


def test_mixed_results_equal_alone(tn):
    amps = amp_requests(24)
    path = greedy.greedy_path(amps[0], seed=0, alpha=1.0)
    p_amp = tn.Plan(amps[0], path)
    ising = [ising_pf.random_3regular_network(n, s) for n, s in ((20, 1), (40, 2), (60, 3))]
    i_paths = [greedy.greedy_path(n, seed=0, alpha=1.0) for n in ising]
    p_ising = [tn.Plan(n, p, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True) for n, p in zip(ising, i_paths)]
    big = workloads.random_circuit(4, 5, 12, 40)
    p_big = tn.Plan(big.net, big.path, prec="3xtf32")

    jobs = [(p_amp, n, True) for n in amps] + [(p, n, False) for p, n in zip(p_ising, ising)]
    jobs += [(p_big, big.net, True)] * 2
    rng = np.random.default_rng(3)
    order = rng.permutation(len(jobs))
    # alone: the synchronous host entry point, one at a time
    alone = {}
    for j in order:
        plan, net, cplx = jobs[j]
        out = np.zeros((), dtype=np.complex128 if cplx else np.float64)
        ls = np.zeros(1)
        plan.contract_host(host_inputs(net, cplx), out, ls)
        alone[j] = (out.copy(), ls[0])
    srv = tn.Server(max_inflight=6, n_streams=3)
    tickets = {}
    for j in order:
        plan, net, cplx = jobs[j]
        tickets[j] = srv.submit(plan, host_inputs(net, cplx))
    for j, t in tickets.items():
        plan, net, cplx = jobs[j]
        out = np.zeros((), dtype=np.complex128 if cplx else np.float64)
        ls = np.zeros(1)
        assert srv.poll(t, out, ls, timeout_us=-1) == tn.TN_OK
        # same launch sequence on the same data: bit-for-bit the same result
        assert out == alone[j][0] and ls[0] == alone[j][1], j
    srv.destroy()
    # and the values are right
    for j in (0, 7, 23):
        want = oracle.contract(amps[j], path)
        assert abs(complex(alone[j][0]) - want) / abs(want) < 1e-5
    for j in range(3):
        v, ls = alone[len(amps) + j]
        assert abs(np.log(v) + ls - np.log(oracle.contract(ising[j], i_paths[j]))) < 1e-5


def test_busy_and_unknown_ticket(tn):
    big = workloads.random_circuit(4, 5, 12, 40)
    p_big = tn.Plan(big.net, big.path, prec="fp32")
    srv = tn.Server(max_inflight=1, n_streams=1, queue_capacity=1)
    ins = host_inputs(big.net)
    saw_busy = False
    tickets = []
    for _ in range(200):
        s, t = srv.try_submit(p_big, ins)
        if s == tn.TN_ERR_BUSY:
            saw_busy = True
            break
        assert s == tn.TN_OK
        tickets.append(t)
    assert saw_busy
    out = np.zeros((), dtype=np.complex128)
    assert srv.poll(10**12, out) == tn.TN_ERR_INVALID
    for t in tickets:
        assert srv.poll(t, out, timeout_us=-1) == tn.TN_OK
    srv.destroy()


def test_hbm_budget_refusal(tn):
    big = workloads.random_circuit(4, 5, 12, 40)
    p_big = tn.Plan(big.net, big.path, prec="fp32")
    srv = tn.Server(max_inflight=2, n_streams=1, hbm_budget_bytes=1024)
    t = srv.submit(p_big, host_inputs(big.net))
    out = np.zeros((), dtype=np.complex128)
    assert srv.poll(t, out, timeout_us=-1) == tn.TN_ERR_OOM
    srv.destroy()


def test_poll_not_ready_then_done(tn):
    big = workloads.random_circuit(4, 5, 12, 40)
    p_big = tn.Plan(big.net, big.path, prec="fp32")
    srv = tn.Server(max_inflight=1, n_streams=1)
    t = srv.submit(p_big, host_inputs(big.net))
    out = np.zeros((), dtype=np.complex128)
    s = srv.poll(t, out, timeout_us=0)
    assert s in (tn.TN_ERR_NOT_READY, tn.TN_OK)
    if s == tn.TN_ERR_NOT_READY:
        assert srv.poll(t, out, timeout_us=-1) == tn.TN_OK
    want = oracle.contract(big.net, big.path)
    assert abs(complex(out) - want) / abs(want) < 1e-5
    srv.destroy()


def test_device_wait_timeout_is_a_status(tn):
    """A device wait that nothing completes runs out (100 ms limit), is reported as
    TN_ERR_TIMEOUT, and the context stays usable: a contraction right after is correct."""
    w = workloads.rc12()
    plan = tn.Plan(w.net, w.path)
    assert plan.selftest_bounded_wait(True, 100000) == tn.TN_OK
    t0 = time.time()
    assert plan.selftest_bounded_wait(False, 100000) == tn.TN_ERR_TIMEOUT
    assert time.time() - t0 < 5.0
    assert "bounded wait" in tn.last_error()
    out = np.zeros((), dtype=np.complex128)
    plan.contract_host(host_inputs(w.net), out)
    want = oracle.contract(w.net, w.path)
    assert abs(complex(out) - want) / abs(want) < 1e-5


def test_hbm_budget_two_plans_one_at_a_time(tn):
    """A budget that holds one workspace of either plan: A, A, B, B submitted together.
    B's first request frees A's idle instance instead of being refused; every result is
    OK and matches the oracle."""
    a = workloads.random_circuit(4, 5, 12, 40)
    b = workloads.random_circuit(3, 4, 8, 12)
    p_a = tn.Plan(a.net, a.path, prec="fp32")
    p_b = tn.Plan(b.net, b.path, prec="fp32")
    wa, wb = p_a.info()["workspace_bytes"], p_b.info()["workspace_bytes"]
    budget = max(wa, wb) + min(wa, wb) // 2  # one instance at a time, never both
    srv = tn.Server(max_inflight=2, n_streams=2, hbm_budget_bytes=budget)
    jobs = [(p_a, a), (p_a, a), (p_b, b), (p_b, b)]
    tickets = [srv.submit(p, host_inputs(w.net)) for p, w in jobs]
    want = {id(a): oracle.contract(a.net, a.path), id(b): oracle.contract(b.net, b.path)}
    for t, (p, w) in zip(tickets, jobs):
        out = np.zeros((), dtype=np.complex128)
        assert srv.poll(t, out, timeout_us=-1) == tn.TN_OK, tn.last_error()
        assert abs(complex(out) - want[id(w)]) / abs(want[id(w)]) < 1e-5
    # and back to A after B: A's instance was freed, a new one fits again
    out = np.zeros((), dtype=np.complex128)
    assert srv.poll(srv.submit(p_a, host_inputs(a.net)), out, timeout_us=-1) == tn.TN_OK
    assert abs(complex(out) - want[id(a)]) / abs(want[id(a)]) < 1e-5
    srv.destroy()


def _pack_jobs(tn):
    amps = amp_requests(40, seed=4)
    path = greedy.greedy_path(amps[0], seed=0, alpha=1.0)
    p_amp = tn.Plan(amps[0], path, prec="3xtf32")  # no step is large enough for the tensor cores
    assert all(p_amp.step(s)["cls"] != tn.TN_CLASS_TC for s in range(len(path.pairs)))
    ising = [ising_pf.random_3regular_network(n, s) for n, s in ((20, 5), (32, 6), (48, 7))]
    i_paths = [greedy.greedy_path(n, seed=0, alpha=1.0) for n in ising]
    p_ising = [tn.Plan(n, p, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True) for n, p in zip(ising, i_paths)]
    big = workloads.random_circuit(4, 5, 12, 40)
    p_big = tn.Plan(big.net, big.path, prec="3xtf32")  # tensor-core steps: never packed
    jobs = [(p_amp, n, True) for n in amps] + [(p, n, False) for p, n in zip(p_ising, ising)] * 3
    jobs += [(p_big, big.net, True)] * 2
    order = np.random.default_rng(8).permutation(len(jobs))
    return [jobs[j] for j in order], (amps, path, ising, i_paths, big)


def test_packed_results_identical_alone_and_in_mix(tn):
    """With packing on, a request gives the same bits served alone (a pack of one) and in a
    mix where it shares a launch with others (one CTA per request, fixed order within it),
    and the values match the oracle. The mix is queued by one tn_serve_submit_batch, so the
    packs form whatever the timing."""
    jobs, (amps, path, ising, i_paths, big) = _pack_jobs(tn)

    def serve_all(one_at_a_time):
        srv = tn.Server(max_inflight=4, n_streams=2, pack_max=64)
        res = []
        if one_at_a_time:
            for plan, net, cplx in jobs:
                out = np.zeros((), dtype=np.complex128 if cplx else np.float64)
                ls = np.zeros(1)
                assert srv.poll(srv.submit(plan, host_inputs(net, cplx)), out, ls, timeout_us=-1) == tn.TN_OK
                res.append((out.copy(), ls[0]))
        else:  # queued together (one submit_batch): the scheduler sees the whole mix
            ts = srv.submit_batch([(plan, host_inputs(net, cplx)) for plan, net, cplx in jobs])
            for t, (plan, net, cplx) in zip(ts, jobs):
                out = np.zeros((), dtype=np.complex128 if cplx else np.float64)
                ls = np.zeros(1)
                assert srv.poll(t, out, ls, timeout_us=-1) == tn.TN_OK, tn.last_error()
                res.append((out.copy(), ls[0]))
        st = srv.stats()
        srv.destroy()
        return res, st

    alone, st_alone = serve_all(True)
    mixed, st_mixed = serve_all(False)
    n_small = len(jobs) - 2
    assert st_alone["packed_requests"] == n_small and st_alone["max_pack"] == 1
    assert st_mixed["packed_requests"] == n_small and st_mixed["max_pack"] > 1
    assert st_mixed["plan_launches"] == 2 and st_mixed["completed"] == len(jobs)
    for (a, la), (m, lm) in zip(alone, mixed):
        assert a == m and la == lm
    # the values: amplitudes, partition functions (ln Z), and the unpacked circuit
    want_amp = {id(n): oracle.contract(n, path) for n in amps}
    want_z = {id(n): np.log(oracle.contract(n, p)) for n, p in zip(ising, i_paths)}
    want_big = oracle.contract(big.net, big.path)
    for (plan, net, cplx), (v, ls) in zip(jobs, mixed):
        if id(net) in want_amp:
            w = want_amp[id(net)]
            assert abs(complex(v) - w) / abs(w) < 1e-5
        elif id(net) in want_z:
            assert abs(np.log(float(v)) + ls - want_z[id(net)]) < 1e-5
        else:
            assert abs(complex(v) - want_big) / abs(want_big) < 1e-5


def test_packed_under_budget(tn):
    """Packing with an HBM budget that also holds the plans' instances: every result OK."""
    jobs, _ = _pack_jobs(tn)
    srv = tn.Server(max_inflight=2, n_streams=2, pack_max=16, hbm_budget_bytes=64 << 20)
    ts = [srv.submit(plan, host_inputs(net, cplx)) for plan, net, cplx in jobs]
    for t, (plan, net, cplx) in zip(ts, jobs):
        out = np.zeros((), dtype=np.complex128 if cplx else np.float64)
        assert srv.poll(t, out, None, timeout_us=-1) == tn.TN_OK, tn.last_error()
    assert srv.stats()["hbm_in_use"] <= 64 << 20
    srv.destroy()


def test_submit_batch_all_or_nothing(tn):
    """tn_serve_submit_batch queues all n requests or none: a batch larger than the free
    queue space is refused with TN_ERR_BUSY and leaves nothing queued; a batch that fits
    returns n tickets in order, each completing with its own result."""
    amps = amp_requests(6, seed=11)
    path = greedy.greedy_path(amps[0], seed=0, alpha=1.0)
    plan = tn.Plan(amps[0], path, prec="3xtf32")
    srv = tn.Server(max_inflight=1, n_streams=1, queue_capacity=4, pack_max=8)
    reqs = [(plan, host_inputs(n)) for n in amps]
    with pytest.raises(tn.binding.TnError):
        srv.submit_batch(reqs[:5])
    assert srv.stats()["completed"] == 0
    ts = srv.submit_batch(reqs[:4])
    assert len(ts) == 4 and ts == sorted(ts)
    for t, n in zip(ts, amps):
        out = np.zeros((), dtype=np.complex128)
        assert srv.poll(t, out, timeout_us=-1) == tn.TN_OK
        want = oracle.contract(n, path)
        assert abs(complex(out) - want) / abs(want) < 1e-5
    assert srv.stats()["completed"] == 4
    srv.destroy()
