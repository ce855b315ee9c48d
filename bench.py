#!/usr/bin/env python
"""Benchmark: exact contraction of a sliced 40-qubit random-circuit amplitude on one GB300.

Default workload rc40c14: 40 qubits on a 5x8 grid, 14 cycles, one amplitude, 7 sliced
labels (128 slices), each slice's largest intermediate 2^30 complex64 elements. One step
= one tn_contract_slices over a fixed batch of slices (leaf staging and slicing, every
pairwise step, the FP64 cross-slice sum), inputs resident in HBM; successive steps take
successive slice ranges, so the warm-up and timed steps together cover every slice. The
full contraction time is projected as T_proj = t_slice * n_slices (Sec. V-A, Eq. 8).
Workloads whose whole contraction fits a step (rc40, ...) contract all slices per step.
Prints one JSON line (see the keys below). `--impl reference` times the CPU
complex128 oracle instead, on a bounded sample of the same workload per step.
Under torchrun every rank contracts its own full copy of the workload (independent
units, no data-path collective: weak scaling); rank 0 prints.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from tn_inputs import workloads  # noqa: E402

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
NOMINAL_TF32_PER_BF16 = 1.1 / 2.25     # nominal dense tf32 / bf16 rate of the part
SM_COUNT, FP32_LANES = 152, 128
WORKLOAD_DESC = {
    "rc40c14": "40-qubit 5x8 grid random circuit, 14 brick-wall cycles of Haar 2-qubit gates, one "
               "amplitude, greedy path (least flops of a seeded search), 7 sliced labels (128 slices) "
               "so that each slice's largest intermediate is 2^30 elements, complex64",
    "rc40": "40-qubit 5x8 grid random circuit, 13 brick-wall cycles of Haar 2-qubit gates, "
            "one amplitude, greedy path, 8 sliced labels (256 slices), complex64",
    "kising44": "4x4 kicked Ising, 10 Trotter steps (J=1, dt=0.25, h=0.9), <Z_centre>, complex64",
    "khex45": "kicked Ising on a 4x5 honeycomb (brick-wall) lattice, 6 Trotter steps (J=1, dt=0.25, "
              "h=0.9), <Z_centre>, complex64",
    "ktri44": "kicked Ising on a 4x4 triangular lattice, 8 Trotter steps (J=1, dt=0.25, h=0.9), "
              "<Z_centre>, complex64",
    "rc12": "12-qubit 3x4 random circuit, 8 cycles, one amplitude, complex64",
    "tcgemm": "one dense complex step A[2^14 x 2^13] . B[2^14 x 2^13]^T closed by two vectors (the 14-cycle "
              "circuit's dominant step shape at k = 2^13), complex64",
    "sv26": "a 26-qubit state (2^26-element leaf, complex64) declared in a shuffled qubit order, "
            "absorbing 4 Haar 2-qubit gates; open output (the state), complex64",
    "rc40c14sub": "the rc40c14 network and path with two more sliced labels (512 slices, largest "
                  "intermediate 2^29), complex64",
    "rc40u": "the rc40 network and path without slicing: every intermediate whole (largest 2^32 "
             "complex64 elements), one contraction per step, complex64",
    "rc40open": "the 40-qubit rc40 circuit with the 2x2 corner qubits (30, 31, 38, 39) left open: "
                "16 correlated amplitudes per contraction, greedy path, 8 sliced labels (256 slices), "
                "complex64",
    "isingsq20": "partition function of a +-J Ising spin glass on an open 20x20 square lattice (400 spins, "
                 "beta 0.44), greedy path (largest intermediate 2^29), real FP32 storage with "
                 "per-intermediate exponent scaling",
}
PREC = {"fp32": 0, "tf32": 1, "3xtf32": 2, "bf16x3": 3, "bf16x3m": 3}
# the real forms (tn_precision R32_*) of a real network's --prec
REAL_PREC = {"fp32": 4, "tf32": 5, "3xtf32": 6}
# forms run with the 3M complex product (three real products per complex MAC, not four)
THREE_M = {"bf16x3m"}
# arithmetic of each form (complex64 storage; products as named, FP32 accumulation)
DTYPE_NAME = {"fp32": "f32", "tf32": "tf32", "3xtf32": "3xtf32", "bf16x3": "bf16x3", "bf16x3m": "bf16x3 (3M)"}
# DRAM bytes (read + write) of the dominant tensor-core step (below) over the slices of a
# pass, captured on that step itself: its 108 launches (bands of the paired-SM kernel's
# tiles), one metric group, one pass each: 787.7 GB read, 15.9 GB written; see
# profiles/contract_tcb2_bf16x3_rc40c14_step310_dram.md. Valid for the kernel build it was
# taken on: drop an entry when that kernel changes.
NCU_TRAFFIC_DOMINANT_LAUNCH = {("rc40c14", "bf16x3"): {"step": 310, "bytes": 787.698e9 + 15.940e9}}
# Full values of the CPU oracle stored by the scripts in tests/golden/ (they call only the
# oracle): the 40-qubit sum over all slices, and the full values of the smaller workloads.
GOLDEN = os.path.join(ROOT, "tests", "golden")
# Slices per step where one contraction of every slice is far longer than a benchmark step:
# rc40c14 takes ~0.2 s per slice, so 8 slices make a step of under two seconds; successive
# steps take successive slice ranges, and once 16 steps have run every slice has been
# contracted once (their sum is the whole amplitude).
SLICES_PER_STEP = {"rc40c14": 8, "rc40c14sub": 32}


def stored_oracle_value(workload):
    if workload in ("rc40", "rc40u"):
        path, key = os.path.join(GOLDEN, "rc40_total.json"), None
    else:
        path, key = os.path.join(GOLDEN, "oracle_values.json"), workload
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if key is not None:
        d = d.get(key, {})
        v = d.get("value")
    else:
        v = d.get("total")
    return complex(*v) if v is not None else None


def stored_slice_partial(workload):
    """(slice id, complex partial) the oracle stored for one slice of a workload whose full
    value is beyond the host (tests/golden/make_rc40c14_values.py), or None."""
    if workload != "rc40c14":
        return None
    path = os.path.join(GOLDEN, "rc40c14_values.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    return int(d["slice"]), complex(*d["slice_partial"])


def measure_local_peaks(tn, seconds=2.0):
    """Peaks MEASURED_PEAKS.json does not hold, measured here the same way on this GPU: the
    dense TF32 rate (torch.matmul of 8192^2 FP32 matrices with TF32 allowed, 2 * 8192^3
    flops) and the FP32 FMA rate (tn_measure_ffma: 8 independent FMA chains per thread,
    4 x 256 threads per SM), each as a burst (best of 10 CUDA-event timings) and sustained
    (back to back for `seconds`, the mean), and the FP64 FMA rate (tn_measure_dfma, the same
    probe in double precision, burst), with the SM clock sampled meanwhile."""
    import torch
    out = {}
    clocks = ClockSampler(torch.cuda.current_device())
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    c = a @ b
    best = 0.0
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3))
    reps = max(1, int(seconds * best / (2.0 * n ** 3)))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch.matmul(a, b, out=c)
    e1.record()
    torch.cuda.synchronize()
    out["tf32_tflops"] = best / 1e12
    out["tf32_tflops_sustained"] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b, c
    rates = [tn.binding.measure_ffma(1 << 18)[0] for _ in range(10)]
    f1, ms1 = tn.binding.measure_ffma(1 << 18)
    iters = max(1 << 18, min(1 << 24, int((1 << 18) * seconds * 1e3 / max(ms1, 1e-3))))
    out["ffma_tflops"] = max(rates) / 1e12
    out["ffma_tflops_sustained"] = tn.binding.measure_ffma(iters)[0] / 1e12
    # FP64 (the cross-slice sum's arithmetic), best of 5 short launches
    out["dfma_tflops"] = max(tn.binding.measure_dfma(1 << 12)[0] for _ in range(5)) / 1e12
    ck = clocks.stop()
    out["sm_mhz_median"] = ck.get("sm_mhz")
    out["reasons"] = ck.get("reasons")
    out["how"] = ("tf32: torch.matmul 8192^3 FP32 with TF32 allowed, best of 10 (burst) and back to back "
                  f"for {seconds:g} s (sustained); ffma: tn_measure_ffma, best of 10 (burst) and one "
                  f"{seconds:g} s launch (sustained); dfma: tn_measure_dfma, best of 5; CUDA events")
    return out


def form_peaks(peaks):
    """Peaks (flop/s) the roofline fractions divide by: each tensor-core form's algorithmic
    peak (three BF16 or TF32 products per algorithmic product for the split forms) from the
    sustained dense rates, and the FP32 ALU peak (FFMA, 2 flops per lane-cycle; max-plus: an
    FADD and an FMNMX per term, half the flop rate) -- measured on this GPU where
    measure_local_peaks ran, else derived (nominal TF32/BF16 ratio, 128 lanes x 152 SMs at
    the maximum clock), each labelled with its source."""
    bf = peaks["bf16_tflops_sustained"] * 1e12
    tf = peaks.get("tf32_tflops_sustained")
    tf32 = tf * 1e12 if tf else bf * NOMINAL_TF32_PER_BF16
    ff = peaks.get("ffma_tflops_sustained")
    alu = ff * 1e12 if ff else SM_COUNT * FP32_LANES * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    # per form: algorithmic flops (8 per complex MAC) per hardware flop -- 4M: 4 real products
    # (8 flops) per complex MAC, 3xTF32 / BF16x3 three per real product; 3M: 3 real products
    tc = {"tf32": tf32, "3xtf32": tf32 / 3.0, "bf16x3": bf / 3.0, "bf16x3m": bf * 8.0 / 18.0}
    tc.update({1: tc["tf32"], 2: tc["3xtf32"], 3: tc["bf16x3"]})
    return {"tc": tc, "alu": alu, "maxplus": alu / 2.0,
            "source": {"tc_bf16": peaks["_source"], "tf32": "measured here" if tf else "derived (nominal ratio)",
                       "alu": "measured here" if ff else "derived (max clock)"}}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(FALLBACK_PEAKS)
    d["_source"] = "fallback"
    return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(w, budget_s, slice_id=0):
    """The CPU oracle, as it stands, on one slice of the workload, step by step in path
    order until `budget_s` of CPU time: returns (flops done, seconds, steps done). A step
    predicted to overrun the budget is not started (one step of an unsliced large network
    can take minutes): the prediction takes the longer of the step's flops at the host's
    matrix-product rate (timed here; for the max-plus loop the rate of the steps done so far)
    and its bytes (operands permuted and copied, result written, complex128) at the host's
    copy rate (timed here)."""
    import oracle
    from oracle import core
    vals = core.slice_assignment(w.net, w.sliced, slice_id)
    arrays, modes = core.restrict_leaves(w.net, vals)
    semiring = w.info.get("semiring", "standard")
    ts = [np.asarray(t, dtype=np.complex128 if w.net.is_complex else np.float64) for t in arrays]
    ms = [tuple(m) for m in modes]
    keep = set(w.net.open_modes)
    costs = oracle.step_costs(w.net, w.path, w.sliced)
    flops, done = 0.0, 0
    t0 = time.perf_counter()
    fm = 8.0 if w.net.is_complex else 2.0
    probe = np.ones((512, 512), dtype=ts[0].dtype)
    tp = time.perf_counter()
    for _ in range(4):
        probe = probe @ probe * 1e-3
    host_rate = 4 * fm * 512.0 ** 3 / (time.perf_counter() - tp)
    big = np.ones(1 << 24, dtype=ts[0].dtype)
    tp = time.perf_counter()
    big2 = big.reshape(4096, -1).T.copy()
    host_bw = 2.0 * big.nbytes / (time.perf_counter() - tp)  # a transposed copy: read + write
    del big, big2
    eb = 16.0 if w.net.is_complex else 8.0
    t0 = time.perf_counter()
    for s, (i, j) in enumerate(w.path.pairs):
        el = time.perf_counter() - t0
        rate = host_rate if semiring == "standard" else (flops / el if flops > 0 and el > 0 else None)
        # permuted copies of both operands, the product's read of them, its result
        moved = eb * (3.0 * costs[s]["m"] * costs[s]["k"] + 3.0 * costs[s]["n"] * costs[s]["k"] +
                      2.0 * costs[s]["m"] * costs[s]["n"])
        if done > 0 and rate and el + max(fm * costs[s]["Ct"] / rate, moved / host_bw) > budget_s:
            break
        c, mc = core.pairwise(ts[i], ms[i], ts[j], ms[j], keep, semiring)
        ts.append(c)
        ms.append(mc)
        ts[i] = ts[j] = None
        flops += fm * costs[s]["Ct"]
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return flops, time.perf_counter() - t0, done


def path_roofline(plan, prec, semiring, peaks, ms_per_step, cplx=True, count=None, form=None):
    """The path's roofline time: over the steps of one contraction (all slices, or the
    `count` slices a step contracts), the sum of
    t_roof = max(bytes / B, flops / F) -- Eq. 6 of Sec. IV-C with this GPU's measured
    rates: B the HBM copy rate, F the peak of the step's kernel class (the form's tensor
    peak for tensor-core steps, the FP32 or max-plus ALU peak otherwise) -- against the
    measured time of the contraction. Bytes count each operand once per launch that reads
    it (slice-invariant operands of sliced steps once per pass)."""
    from paper_2606_01852_gb300 import TN_CLASS_TC
    info = plan.info()
    n_sl = info["n_slices"] if count is None else count
    n_pass = -(-n_sl // info["slice_batch"])
    e, fm = (8.0, 8.0) if cplx else (4.0, 2.0)
    hbm = peaks["hbm_gbs"] * 1e9
    fp = form_peaks(peaks)
    tc_peak = fp["tc"].get(form if form is not None else prec)
    alu = fp["maxplus"] if semiring == "maxplus" else fp["alu"]
    total = 0.0
    for s in range(info["n_steps"]):
        st = plan.step(s)
        copies = n_sl if st["batched"] else 1
        reads = lambda t: n_sl if plan.tensor(t)["batched"] else (n_pass if st["batched"] else 1)
        m, n, k = st["m"], st["n"], st["k"]
        flops = fm * m * n * k * copies
        nbytes = e * (m * k * reads(st["a_id"]) + n * k * reads(st["b_id"]) + m * n * copies)
        peak = tc_peak if st["cls"] == TN_CLASS_TC else alu
        total += max(nbytes / hbm, flops / peak)
    return {"sum_t_roof_ms": total * 1e3, "ms_per_step": ms_per_step, "frac": total * 1e3 / ms_per_step}


def replica_throughput(ms_local, units_local, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas (one per rank, no data-path
    collective): the units all ranks processed over the slowest rank's time. Returns
    (units per second, max milliseconds over ranks)."""
    import torch
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        mx = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
        tot = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        return float(tot.item()) / (float(mx.item()) / 1e3), float(mx.item())
    return units_local / (ms_local / 1e3), ms_local


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workloads.BY_NAME[args.workload]()
    # each step a bounded sample: the whole run (warm-up of 1 s per step) stays near 2.5 min
    budget = args.ref_budget if args.ref_budget else max(3.0, 150.0 / max(1, args.steps))
    for _ in range(args.warmup):
        oracle_sample(w, min(1.0, budget))
    vals, secs, samples = [], [], []
    for k in range(args.steps):
        f, s, done = oracle_sample(w, budget, slice_id=k % max(1, w.n_slices))
        vals.append(f / s / 1e12)
        secs.append(s)
        samples.append(done)
    v = statistics.mean(vals)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "contraction TFLOP/s", "value": v, "unit": "TFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if w.net.is_complex else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload, ""),
                   "prec": "complex128 oracle" if w.net.is_complex else "float64 oracle",
                   "semiring": w.info.get("semiring", "standard"),
                   "slices": w.n_slices},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {min(samples)}-{max(samples)} of {len(w.path.pairs)} path steps of "
                                   f"one slice per step, {budget:.0f} s budget per step"},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_2606_01852_gb300 as tn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    peaks = load_peaks()
    peaks.update(measure_local_peaks(tn))
    fpk = form_peaks(peaks)
    # the planner's Eq. 6 rates: this GPU's measured peaks
    tn.binding.set_cost_model(peaks["hbm_gbs"] * 1e9, fpk["alu"], [fpk["tc"][1], fpk["tc"][2], fpk["tc"][3]])
    w = workloads.BY_NAME[args.workload]()
    semiring = w.info.get("semiring", "standard")
    scaled = bool(w.info.get("exp_scaling", False))
    cplx = w.net.is_complex
    # real networks: the max-plus workloads run the R32 FP32 form; the others the real form
    # of --prec (fp32, tf32, 3xtf32; the complex-only BF16x3 forms, the default, read as
    # 3xtf32)
    if cplx:
        prec, form = PREC[args.prec], args.prec
    elif semiring == "maxplus":
        prec, form = tn.TN_R32_FP32_SIMT, "fp32"
    else:
        form = args.prec if args.prec in REAL_PREC else "3xtf32"
        prec = REAL_PREC[form]
    cmult = 3 if (cplx and args.prec in THREE_M) else 4
    n_sl = w.n_slices
    per_step = args.slices_per_step or SLICES_PER_STEP.get(args.workload, n_sl)
    per_step = max(1, min(per_step, n_sl))
    # a slice-batched step runs its slices in one pass unless told otherwise
    batch = args.max_slice_batch or (per_step if per_step < n_sl else 0)
    plan = tn.Plan(w.net, w.path, w.sliced, prec=prec, exp_scaling=scaled, max_slice_batch=batch,
                   semiring=semiring, complex_mult=cmult, single_sm_tiles=args.single_sm_tiles)
    info = plan.info()
    stream = torch.cuda.current_stream()
    # step j contracts slices [j * per_step, (j + 1) * per_step) modulo n_slices
    ranges = [((j * per_step) % n_sl, min(per_step, n_sl - (j * per_step) % n_sl))
              for j in range(args.warmup + args.steps)]
    in_dt, out_dt = (torch.complex64, torch.complex128) if cplx else (torch.float32, torch.float64)
    ins = [torch.tensor(np.asarray(t), dtype=in_dt, device="cuda") for t in w.net.tensors]
    outs = torch.zeros((len(ranges),) + tuple(plan.out_shape), dtype=out_dt, device="cuda")
    ls = torch.zeros(len(ranges), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    # --graph (whole-contraction workloads): every step replays one CUDA graph of the call
    # (tn_contract_graph), into one output buffer so that the captured pointers stay the same
    use_graph = args.graph and all(c == n_sl for _, c in ranges)

    def step(j, graph=use_graph):
        b, c = ranges[j]
        if graph:
            plan.contract_graph(ins, outs[0], ls[0:1], stream)
        elif c == n_sl:
            plan.contract(ins, outs[j], ls[j:j + 1], stream)
        else:
            plan.contract_slices(ins, b, c, outs[j], ls[j:j + 1], stream)

    if args.autotune:
        # per paired-SM step, the faster of paired SMs and one SM per tile (the same bits)
        plan.autotune(ins, outs[0], stream)
        torch.cuda.synchronize()
    for j in range(args.warmup):
        step(j)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    if not use_graph:
        plan.profile(True)
        plan.profile_read(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps, outside the events
        ev[k][0].record(stream)
        step(args.warmup + k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if use_graph:
        # the per-class times come from the same steps run without the graph (the kernels are
        # the same; per-step events cannot be recorded inside a replayed graph)
        outs[1:] = outs[0]
        ls[1:] = ls[0]
        plan.profile(True)
        plan.profile_read(reset=True)
        for k in range(args.steps):
            flush.zero_()
            step(args.warmup + k, graph=False)
        torch.cuda.synchronize()
    plan.profile(False)
    prof = plan.profile_read(reset=True)
    if dist:
        dist.barrier()
    ck = clocks.stop()
    times = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(times)
    timed = ranges[args.warmup:]
    flops = statistics.mean(plan.flops_per_call(c) for _, c in timed)
    slices_per_step = statistics.mean(c for _, c in timed)
    tflop_per_s, ms_max = replica_throughput(ms, flops / 1e12, dist, device="cuda")
    value = tflop_per_s
    all_out = outs.cpu().numpy()
    # the whole result once the steps have covered every slice: the first n_sl / per_step
    # ranges tile the slices exactly (else the last step's partial)
    tiles = n_sl // per_step
    whole = per_step < n_sl and n_sl % per_step == 0 and len(ranges) >= tiles
    result = all_out[:tiles].sum(axis=0) if whole else all_out[-1]
    result_ls = float(ls[-1].item())  # log scale of the last step's result (exponent scaling)

    # dominant kernel class by device time, and its roofline
    cls = max(range(len(prof["ms"])), key=lambda c: prof["ms"][c])
    names = dict(enumerate(tn.binding.CLASS_NAMES))
    launches = prof["launches"][cls]
    per_launch_ms = prof["ms"][cls] / max(1, launches)
    step_ms = plan.profile_steps()
    top = sorted(range(len(step_ms)), key=lambda s: -step_ms[s])[:8]
    top_steps = []
    for s in top:
        st = plan.step(s)
        top_steps.append({"step": s, "kernel": names[st["cls"]], "m": st["m"], "n": st["n"], "k": st["k"],
                          "ms_per_step": step_ms[s] / args.steps})
    if cls in (1, 3, 4):
        achieved = prof["bytes"][cls] / (prof["ms"][cls] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    elif cls == 2:
        achieved = prof["flops"][cls] / (prof["ms"][cls] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": fpk["tc"][form] / 1e12, "unit": "TFLOP/s"}
        if form == "bf16x3m":
            # the 4M form's peak for comparison (the 3M form does 3/4 of its tensor work)
            roof["peak_4m"] = fpk["tc"]["bf16x3"] / 1e12
            roof["frac_of_4m_peak"] = achieved / roof["peak_4m"]
    else:
        alu = (fpk["maxplus"] if semiring == "maxplus" else fpk["alu"]) / 1e12
        achieved = prof["flops"][cls] / (prof["ms"][cls] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["algorithmic_bytes_per_launch"] = prof["bytes"][cls] / max(1, launches)
    # the class's longest launch (one step over the slices of a pass) with its own rate and
    # its DRAM traffic where a capture of that kernel build covers it
    s_top = max(range(len(step_ms)), key=lambda s: step_ms[s])
    st_top = plan.step(s_top)
    nb_top = info["slice_batch"] if st_top["batched"] else 1
    f_top = (8.0 if cplx else 2.0) * st_top["m"] * st_top["n"] * st_top["k"] * nb_top
    e_top = 8.0 if cplx else 4.0
    b_top = e_top * nb_top * (st_top["m"] * st_top["k"] + st_top["n"] * st_top["k"] + st_top["m"] * st_top["n"])
    ms_top = step_ms[s_top] / max(1, args.steps) / max(1, -(-per_step // info["slice_batch"]))
    cap = NCU_TRAFFIC_DOMINANT_LAUNCH.get((args.workload, args.prec))
    roof["dominant_launch"] = {"step": s_top, "m": st_top["m"], "n": st_top["n"], "k": st_top["k"],
                               "copies": nb_top, "ms": ms_top, "flops": f_top,
                               "achieved": f_top / (ms_top / 1e3) / 1e12 if cls == 2 else None,
                               "algorithmic_bytes": b_top,
                               "traffic": cap["bytes"] if cap and cap["step"] == s_top else None}
    if cap and cap["step"] == s_top:
        roof["traffic"] = cap["bytes"]
        roof["traffic_scope"] = ("DRAM bytes of the dominant step (%d) over the slices of a pass, from a "
                                 "one-pass capture of its launches" % s_top)
    roof["kernel"] = names[cls]
    roof["launches_per_step"] = launches / args.steps
    roof["ms_per_launch"] = per_launch_ms
    roof["share_of_step"] = prof["ms"][cls] / sum(prof["ms"])
    roof["peak_source"] = {1: fpk["source"]["tf32"], 2: fpk["source"]["tf32"], 3: fpk["source"]["tc_bf16"],
                           5: fpk["source"]["tf32"], 6: fpk["source"]["tf32"]}.get(
        prec, fpk["source"]["alu"]) if cls == 2 else (peaks["_source"] if cls in (1, 3, 4) else fpk["source"]["alu"])
    path_roof = path_roofline(plan, prec, semiring, peaks, ms_max, cplx, count=round(slices_per_step), form=form)
    perm = None
    if prof["launches"][4] > 0 and prof["ms"][4] > 0:
        # leaf staging (the permutation kernels): staged bytes read + written over its event time
        gbs = prof["bytes"][4] / (prof["ms"][4] / 1e3) / 1e9
        perm = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "bytes_per_step": prof["bytes"][4] / args.steps,
                "ms_per_step": prof["ms"][4] / args.steps, "tiled_leaves": sum(
                    1 for t in range(len(w.net.modes)) if plan.tensor(t)["tiled"])}

    # end to end through the public C ABI with host buffers
    host_in = [np.ascontiguousarray(np.asarray(t, dtype=np.complex64 if cplx else np.float32))
               for t in w.net.tensors]
    host_out = np.zeros(plan.out_shape, dtype=np.complex128 if cplx else np.float64)
    host_ls = np.zeros(1)
    h2d = int(sum(a.nbytes for a in host_in))
    e2e_b, e2e_c = ranges[-1]
    plan.contract_slices_host(host_in, e2e_b, e2e_c, host_out, host_ls)
    e2e_steps = max(1, min(args.steps, 3 if per_step == n_sl else 2))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.contract_slices_host(host_in, e2e_b, e2e_c, host_out, host_ls)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_val = ws * plan.flops_per_call(e2e_c) / e2e_s / 1e12

    line = {
        "metric": "contraction TFLOP/s", "value": value, "unit": "TFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "data": "synthetic",
        "dtype": DTYPE_NAME[args.prec] if cplx else ("f32 (max,+)" if semiring == "maxplus" else
                                                     {"fp32": "f32", "tf32": "tf32", "3xtf32": "3xtf32"}[form]),
        "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload, ""),
                   "prec": args.prec if cplx else "r32_" + form, "semiring": semiring,
                   "exp_scaling": scaled,
                   "slices": n_sl, "sliced_labels": len(w.sliced),
                   "largest_intermediate_per_slice": info["peak_elems"],
                   "slices_per_step": slices_per_step, "slice_batch": info["slice_batch"],
                   "passes_per_step": -(-per_step // info["slice_batch"]), "flops_per_step": flops,
                   "flops_full_contraction": info["flops"],
                   "algorithmic_bytes_full_contraction": info["bytes"],
                   "l2": "256 MiB buffer written between timed steps (L2 is 129 MB); "
                         "intermediates are GBs", "parallelism": f"replicas{ws}",
                   **({"graph": "each step one replay of a CUDA graph of the call (tn_contract_graph)"}
                      if use_graph else {}),
                   **({"tiles": "one SM per tensor-core tile"} if args.single_sm_tiles else {}),
                   **({"autotune": [plan.step(s)["single_sm"] for s in range(info["n_steps"])
                                    if plan.step(s)["cls"] == tn.TN_CLASS_TC]} if args.autotune else {})},
        "slices_per_s": ws * slices_per_step / (ms_max / 1e3),
        "projected_full_contraction_s": (n_sl / (slices_per_step / (ms_max / 1e3)) if per_step < n_sl
                                         else ms_max / 1e3),
        "projection": ("T_proj = t_slice * n_slices (Sec. V-A, Eq. 8): a step contracts a batch of slices"
                       if per_step < n_sl else "measured: every slice in each step"),
        "result": ([float(result.real), float(result.imag)] if result.ndim == 0 else
                   {"shape": list(result.shape), "sum_abs2": float(np.sum(np.abs(result) ** 2)),
                    "first": [float(result.flat[0].real), float(result.flat[0].imag)]}),
        "roofline": roof,
        "path_roofline": path_roof,
        "staging_roofline": perm,
        "per_class": {names[c]: {"launches": prof["launches"][c], "ms": prof["ms"][c],
                                 "flops": prof["flops"][c], "bytes": prof["bytes"][c]}
                      for c in range(len(prof["ms"]))},
        "top_steps": top_steps,
        "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": host_out.nbytes + host_ls.nbytes},
        "gpu_launches": sum(plan.launches_per_call(c) for _, c in timed),
        "clocks": ck,
        "peaks": {k: v for k, v in peaks.items() if not k.startswith("_") and k not in ("when", "image", "torch")},
    }
    if per_step < n_sl:
        line["result_scope"] = (f"all {n_sl} slices (the sum of the first {tiles} steps' slice ranges)"
                                if whole else f"slices {ranges[-1][0]}..{ranges[-1][0] + ranges[-1][1] - 1}")
    sp = stored_slice_partial(args.workload)
    if sp is not None:
        # one slice again, untimed, against the oracle's value of it (its four finer pieces)
        sid, want_sl = sp
        one = torch.zeros(plan.out_shape, dtype=out_dt, device="cuda")
        plan.contract_slices(ins, sid, 1, one, None, stream)
        torch.cuda.synchronize()
        got_sl = complex(one.cpu().numpy())
        line["oracle_slice"] = {"slice": sid, "oracle": [want_sl.real, want_sl.imag],
                                "got": [got_sl.real, got_sl.imag]}
        line["rel_err_vs_oracle"] = abs(got_sl - want_sl) / abs(want_sl)
        line["rel_err_scope"] = f"slice {sid} of {n_sl} (the oracle's sum of its 4 pieces)"
    want = stored_oracle_value(args.workload)
    covers_all = per_step >= n_sl or whole  # the result is the sum over every slice
    if want is not None and result.ndim == 0 and covers_all:
        line["oracle_total"] = [want.real, want.imag]
        line["rel_err_vs_oracle"] = abs(complex(result) - want) / abs(want)
    if args.check and covers_all:
        import oracle
        want = np.asarray(oracle.contract(w.net, w.path, w.sliced, semiring=semiring))
        line["oracle"] = [float(want.flat[0].real), float(want.flat[0].imag)]
        line["rel_err_vs_oracle"] = float(np.max(np.abs(result - want)) / np.max(np.abs(want)))
    if scaled and result.ndim == 0:
        # the value is result * e^(log scale): report ln of it (|ln got - ln want| is the
        # relative error of the value)
        line["log_scale"] = result_ls
        line["ln_result"] = float(np.log(abs(float(result.real)))) + result_ls
        if args.check and covers_all:
            line["ln_oracle"] = float(np.log(abs(float(np.asarray(want).flat[0].real))))
            line["rel_err_vs_oracle"] = abs(line["ln_result"] - line["ln_oracle"])
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        f, s, done = oracle_sample(w, args.ref_budget or 20.0)
        line["cpu_baseline"] = {"value": f / s / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"first {done} of {len(w.path.pairs)} path steps of slice 0 "
                                          f"({f:.3g} of {plan.flops_per_call(1):.3g} flops of one "
                                          f"slice, {s:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.destroy()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch_bench(args):
    """Many small networks in one persistent graph-replayed launch (launch shape from the
    autotuner), against one tn_contract launch sequence per network. Metric: networks/s.
      ising3r    : 4096 Ising partition functions on random 3-regular graphs (20-60 spins,
                   J = +-1, beta = 0.5), FP32 with exponent scaling;
      kingsbatch : 4096 maximum independent sets of King's subgraphs (L 4-7, density
                   0.8), the max-plus semiring."""
    import torch
    import paper_2606_01852_gb300 as tn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    count = args.networks
    peaks = load_peaks()
    peaks.update(measure_local_peaks(tn))
    maxplus = args.workload == "kingsbatch"
    semiring = "maxplus" if maxplus else "standard"
    wl = workloads.kings_batch(count) if maxplus else workloads.ising3r(count, seed=3)
    nets, paths = [w.net for w in wl], [w.path for w in wl]
    b = tn.Batch(nets, paths, complex_=False, exp_scaling=not maxplus, semiring=semiring)
    packed = torch.tensor(b.pack(nets), device="cuda")
    vals = torch.zeros((count, 2), dtype=torch.float64, device="cuda")
    logs = torch.zeros(count, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    b.autotune(packed, vals, logs, stream)
    for _ in range(args.warmup):
        b.contract(packed, vals, logs, stream, graph=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(stream)
        b.contract(packed, vals, logs, stream, graph=True)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = statistics.mean(a.elapsed_time(c) for a, c in ev)
    # one launch sequence per network (the per-contraction baseline)
    plans = [tn.Plan(n, p, prec=tn.TN_R32_FP32_SIMT, exp_scaling=not maxplus, semiring=semiring)
             for n, p in zip(nets, paths)]
    dins = [[torch.tensor(np.asarray(t, dtype=np.float32), device="cuda") for t in n.tensors] for n in nets]
    outs = torch.zeros(count, dtype=torch.float64, device="cuda")
    lss = torch.zeros(count, dtype=torch.float64, device="cuda")
    for i in range(count):
        plans[i].contract(dins[i], outs[i:i + 1], lss[i:i + 1], stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(count):
        plans[i].contract(dins[i], outs[i:i + 1], lss[i:i + 1], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    if maxplus:  # both are exact integers
        diff = float(np.max(np.abs(vals[:, 0].cpu().numpy() - outs.cpu().numpy())))
    else:
        lnz_b = np.log(vals[:, 0].cpu().numpy()) + logs.cpu().numpy()
        lnz_s = np.log(outs.cpu().numpy()) + lss.cpu().numpy()
        diff = float(np.max(np.abs(lnz_b - lnz_s)))
    t, c, g, sm = b.launch_shape()
    fpk = form_peaks(peaks)
    alu = (fpk["maxplus"] if maxplus else fpk["alu"]) / 1e12
    line = {
        "metric": "networks/s", "value": ws * count / (ms / 1e3), "unit": "networks/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (max,+)" if maxplus else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "networks": count,
                   "desc": ("maximum independent sets of King's subgraphs, L 4-7, density 0.8, max-plus FP32"
                            if maxplus else "Ising partition functions, random 3-regular graphs, 20-60 spins, "
                            "J=+-1, beta=0.5, FP32 + exponent scaling"),
                   "launch_shape": {"threads_per_network": t, "ctas_per_sm": c, "networks_per_cta": g,
                                    "form": "warp per network" if g > 1 else "CTA per network",
                                    "smem_arena_bytes_per_network": 4 * sm},
                   "graph": True},
        "one_launch_per_contraction": {"ms": ms_seq, "networks_per_s": count / (ms_seq / 1e3),
                                       "speedup_of_persistent": ms_seq / ms},
        ("max_abs_diff_vs_per_contraction" if maxplus else "max_abs_lnz_diff_vs_per_contraction"): diff,
        "roofline": {"bound": "alu", "achieved": b.flops / (ms / 1e3) / 1e12, "peak": alu, "unit": "TFLOP/s",
                     "frac": b.flops / (ms / 1e3) / 1e12 / alu, "traffic": None, "kernel": "batch_kernel"},
        "gpu_launches": args.steps, "clocks": ck,
        "peaks": {k: v for k, v in peaks.items() if k.startswith(("ffma", "tf32", "sm_mhz"))},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve_bench(args):
    """Serving mix: open-loop Poisson arrivals (mean args.rate req/s for args.serve_seconds):
    70 % 12-qubit circuit amplitudes (random bitstrings, one plan), 25 % Ising partition
    functions (a pool of 64 graphs, FP32 + exponent scaling), 5 % 5x5 kicked-Ising
    expectations (2 Trotter steps; largest intermediate 2^26). Served by the continuous-
    batching loop with the 3xTF32 form, against the plain FP32 form served one request at
    a time. Latency = completion (observed by polling) - submission."""
    import threading
    import torch
    import paper_2606_01852_gb300 as tn
    from tn_inputs import circuits

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    rng = np.random.default_rng(2026)
    amp_w = workloads.rc12()
    pf_pool = workloads.ising3r(64, seed=5)
    kis = workloads.kising55()
    n_req = int(args.rate * args.serve_seconds)
    gaps = rng.exponential(1.0 / args.rate, size=n_req)
    arrive = np.cumsum(gaps)
    cls = rng.choice(3, size=n_req, p=[0.70, 0.25, 0.05])
    pf_idx = rng.integers(0, len(pf_pool), size=n_req)
    bits = rng.integers(0, 2, size=(n_req, 12))
    base = [np.ascontiguousarray(np.asarray(t, dtype=np.complex64)) for t in amp_w.net.tensors]
    n_leaf = len(base)
    e0 = np.array([1.0, 0.0], dtype=np.complex64)
    e1 = np.array([0.0, 1.0], dtype=np.complex64)
    pf_in = [[np.ascontiguousarray(np.asarray(t, dtype=np.float32)) for t in w.net.tensors] for w in pf_pool]
    kis_in = [np.ascontiguousarray(np.asarray(t, dtype=np.complex64)) for t in kis.net.tensors]

    def inputs(i):
        if cls[i] == 0:
            ins = list(base)
            for q in range(12):  # the last 12 leaves are the <x| projections
                ins[n_leaf - 12 + q] = e1 if bits[i, q] else e0
            return ins
        if cls[i] == 1:
            return pf_in[pf_idx[i]]
        return kis_in

    def serve(prec, max_inflight, n_streams, pack_max=0, budget=0):
        p_amp = tn.Plan(amp_w.net, amp_w.path, prec=prec)
        p_pf = [tn.Plan(w.net, w.path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True) for w in pf_pool]
        p_kis = tn.Plan(kis.net, kis.path, prec=prec)
        plan_of = lambda i: p_amp if cls[i] == 0 else (p_pf[pf_idx[i]] if cls[i] == 1 else p_kis)
        srv = tn.Server(max_inflight=max_inflight, n_streams=n_streams, queue_capacity=1 << 20, pack_max=pack_max,
                        hbm_budget_bytes=budget)
        for i in range(min(n_req, 64)):  # warm every plan's first instance
            t = srv.submit(plan_of(i), inputs(i))
            srv.poll(t, np.zeros(2), None, -1)
        for p in [p_kis] + p_pf:
            srv.poll(srv.submit(p, kis_in if p is p_kis else pf_in[p_pf.index(p)]), np.zeros(2), None, -1)
        sub_t = np.zeros(n_req)
        done_t = np.zeros(n_req)
        results = np.zeros((n_req, 2))
        tickets = [None] * n_req
        lock = threading.Lock()
        outstanding = []
        finished = threading.Event()
        t0 = time.perf_counter() + 0.05

        def submitter():
            for i in range(n_req):
                delay = t0 + arrive[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                sub_t[i] = time.perf_counter()
                tk = srv.submit(plan_of(i), inputs(i))
                with lock:
                    tickets[i] = tk
                    outstanding.append(i)
            finished.set()

        th = threading.Thread(target=submitter)
        th.start()
        buf = np.zeros(2)
        ls = np.zeros(1)
        n_done = 0
        while n_done < n_req:
            with lock:
                cur = list(outstanding)
            for i in cur:
                s = srv.poll(tickets[i], buf, ls, 0)
                if s == tn.TN_ERR_NOT_READY:
                    continue
                done_t[i] = time.perf_counter()
                results[i] = buf
                with lock:
                    outstanding.remove(i)
                n_done += 1
            time.sleep(0.0001)
        th.join()
        stats = srv.stats()
        srv.destroy()
        lat = (done_t - sub_t) * 1e3
        span = done_t.max() - sub_t.min()
        out = {"throughput_req_s": n_req / span, "p50_ms": float(np.percentile(lat, 50)),
               "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
               "pack_max": pack_max, "hbm_budget_bytes": budget,
               "launches": stats["plan_launches"] + stats["packs"], "packs": stats["packs"],
               "packed_requests": stats["packed_requests"], "max_pack": stats["max_pack"],
               "hbm_held_bytes": stats["hbm_in_use"]}
        for c, name in enumerate(["amplitude", "partition_function", "kicked_ising_5x5"]):
            sel = lat[cls == c]
            out[name] = {"n": int(sel.size), "p50_ms": float(np.percentile(sel, 50)),
                         "p99_ms": float(np.percentile(sel, 99))}
        for p in [p_amp, p_kis] + p_pf:
            p.destroy()
        return out, results

    def burst(pack_max, n_burst=2048, prec=None, inflight=None, streams=None, large=False):
        """n_burst requests submitted at once (one tn_serve_submit_batch): requests/s from the
        submission to the last completion. large=False: the small ones (amplitudes and
        partition functions); large=True: the mix as it arrives (the 5x5 kicked-Ising
        expectations included)."""
        prec = PREC[args.serve_prec] if prec is None else prec
        p_amp = tn.Plan(amp_w.net, amp_w.path, prec=prec)
        p_pf = [tn.Plan(w.net, w.path, prec=tn.TN_R32_FP32_SIMT, exp_scaling=True) for w in pf_pool]
        p_kis = tn.Plan(kis.net, kis.path, prec=prec) if large else None
        sel = [i for i in range(n_req) if large or cls[i] != 2][:n_burst]
        plan_of = lambda i: p_amp if cls[i] == 0 else (p_pf[pf_idx[i]] if cls[i] == 1 else p_kis)
        srv = tn.Server(max_inflight=inflight or args.serve_inflight, n_streams=streams or args.serve_streams,
                        queue_capacity=1 << 20, pack_max=pack_max)
        warm = sel[:64] + ([next(i for i in range(n_req) if cls[i] == 2)] if large else [])
        for i in warm:
            srv.poll(srv.submit(plan_of(i), inputs(i)), np.zeros(2), None, -1)
        ins = [inputs(i) for i in sel]
        t0 = time.perf_counter()
        ts = srv.submit_batch([(plan_of(i), x) for i, x in zip(sel, ins)])
        for t in ts:
            srv.poll(t, np.zeros(2), None, -1)
        dt = time.perf_counter() - t0
        st = srv.stats()
        srv.destroy()
        for p in [p_amp] + p_pf + ([p_kis] if large else []):
            p.destroy()
        return {"requests": len(sel), "large_requests": int(sum(cls[i] == 2 for i in sel)), "seconds": dt,
                "requests_per_s": len(sel) / dt, "launches": st["plan_launches"] + st["packs"] - len(warm),
                "max_pack": st["max_pack"]}

    budget = int(args.serve_budget_gib * 2 ** 30)
    burst_packed, burst_unpacked = burst(args.serve_pack), burst(0)
    # saturated throughput on the mix itself: the served mixed-precision form (continuous
    # batching, packing) against the plain FP32 form served one request at a time
    sat_mixed = burst(args.serve_pack, n_burst=1000, large=True)
    sat_plain = burst(0, n_burst=1000, prec=tn.TN_C64_FP32_SIMT, inflight=1, streams=1, large=True)
    mixed, r_mixed = serve(PREC[args.serve_prec], args.serve_inflight, args.serve_streams, args.serve_pack, budget)
    unpacked, r_unpacked = serve(PREC[args.serve_prec], args.serve_inflight, args.serve_streams, 0, budget)
    plain, r_plain = serve(tn.TN_C64_FP32_SIMT, 1, 1)
    # the two forms must agree: amplitudes (CUDA-core steps in both forms) and the kicked-
    # Ising expectations (tensor-core steps in the mixed form), relative differences
    c0, c2 = cls == 0, cls == 2
    amp_err = float(np.max(np.abs(r_mixed[c0] - r_plain[c0]).sum(1) / (np.abs(r_plain[c0]).sum(1) + 2 ** -6)))
    kis_err = float(np.max(np.abs(r_mixed[c2] - r_plain[c2]).sum(1) / np.abs(r_plain[c2]).sum(1))) if c2.any() else 0.0
    kis_want = stored_oracle_value("kising55")
    kis_vs_oracle = None
    if kis_want is not None and c2.any():
        kis_vs_oracle = {f: float(np.max(np.abs(r[c2, 0] + 1j * r[c2, 1] - kis_want)) / abs(kis_want))
                         for f, r in (("mixed", r_mixed), ("plain_fp32", r_plain))}
    line = {
        "metric": "serve throughput (requests/s) and p50/p99 latency", "value": mixed["throughput_req_s"],
        "unit": "requests/s", "n_gpus": ws, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64/f32", "data": "synthetic",
        "config": {"workload": "serve-mix", "rate_req_s": args.rate, "seconds": args.serve_seconds,
                   "requests": n_req, "mix": {"amplitude_3x4_m8": 0.70, "ising_pf_3reg_20_60": 0.25,
                                              "kicked_ising_5x5_T2": 0.05},
                   "form": args.serve_prec, "max_inflight": args.serve_inflight,
                   "streams": args.serve_streams, "pack_max": args.serve_pack, "hbm_budget_bytes": budget},
        "mixed": mixed, "mixed_without_packing": unpacked, "plain_fp32_one_at_a_time": plain,
        "p99_speedup": plain["p99_ms"] / mixed["p99_ms"],
        "p99_speedup_of_packing": unpacked["p99_ms"] / mixed["p99_ms"],
        "burst_of_small_requests": {"packed": burst_packed, "unpacked": burst_unpacked,
                                    "speedup_of_packing": burst_packed["requests_per_s"] /
                                    burst_unpacked["requests_per_s"]},
        "saturated_mix": {"mixed": sat_mixed, "plain_fp32_one_at_a_time": sat_plain,
                          "speedup_vs_plain": sat_mixed["requests_per_s"] / sat_plain["requests_per_s"]},
        "max_rel_diff_amplitudes_packed_vs_unpacked": float(np.max(
            np.abs(r_mixed[cls == 0] - r_unpacked[cls == 0]).sum(1) / (np.abs(r_unpacked[cls == 0]).sum(1) + 2 ** -6))),
        "max_rel_diff_amplitudes_mixed_vs_plain": amp_err,
        "max_rel_diff_kicked_ising_mixed_vs_plain": kis_err,
        "kicked_ising_rel_err_vs_oracle": kis_vs_oracle,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rc40c14",
                    choices=sorted(workloads.BY_NAME) + ["ising3r", "kingsbatch", "serve"])
    ap.add_argument("--networks", type=int, default=4096, help="ising3r: networks per launch")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-inflight", type=int, default=16)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-pack", type=int, default=256,
                    help="serve: requests per packed launch of the batched kernel (0: no packing)")
    ap.add_argument("--serve-budget-gib", type=float, default=8.0,
                    help="serve: HBM budget of the request workspaces and pack buffers")
    ap.add_argument("--serve-prec", default="3xtf32", choices=sorted(PREC),
                    help="serve: form of the mixed run (3xtf32: FP32-accurate on every request type)")
    ap.add_argument("--prec", default="bf16x3", choices=sorted(PREC),
                    help="GEMM form: bf16x3 (default), 3xtf32, tf32, fp32 (the plain CUDA-core form)")
    ap.add_argument("--max-slice-batch", type=int, default=0)
    ap.add_argument("--autotune", action="store_true",
                    help="time paired SMs against one SM per tile for each such step first (tn_plan_autotune)")
    ap.add_argument("--graph", action="store_true",
                    help="whole-contraction workloads: replay each step from a CUDA graph (tn_contract_graph)")
    ap.add_argument("--single-sm-tiles", action="store_true",
                    help="BF16x3 4M steps on one SM per output tile (no paired-SM kernel)")
    ap.add_argument("--slices-per-step", type=int, default=0,
                    help="slices contracted per step (0: the workload's default, else all slices)")
    ap.add_argument("--ref-budget", type=float, default=0.0,
                    help="oracle seconds per sample (0: 20 s for the cpu_baseline; for --impl reference, "
                         "150 s spread over the timed steps, at least 3 s each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--check", action="store_true", help="also contract with the CPU oracle and report the error")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload in ("ising3r", "kingsbatch") and args.impl == "ours":
        return run_batch_bench(args)
    if args.workload == "serve" and args.impl == "ours":
        return run_serve_bench(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
