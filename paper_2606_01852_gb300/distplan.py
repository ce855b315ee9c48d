"""Simulated-time report of the offline distribution planner (Sec. IV-B).

    python -m paper_2606_01852_gb300.distplan --workload rc40 --unsliced --gpus 8

Builds a host-only plan of a named workload (optionally with its slicing removed, so
the intermediates reach the sizes the paper distributes), runs tn_plan_distribute for
each device count and prints one JSON line per count: the report (Eqs. 8-10 for the
fixed path) and the schedule of the steps on use-chains.
"""
from __future__ import annotations

import argparse
import json

from tn_inputs import workloads

from .binding import Plan


def report(w, gpus, sliced=True, **cfg):
    plan = Plan(w.net, w.path, w.sliced if sliced else (), prec="bf16x3", host_only=True)
    out = []
    for P in gpus:
        rep, steps = plan.distribute(P, **cfg)
        sched = [dict(step=s, **{k: st[k] for k in ("state", "forced", "chain", "dist_modes", "t_gemm", "t_comm",
                                                     "out_bytes", "n_blk")})
                 for s, st in enumerate(steps) if st["state"] != "none"]
        out.append({"workload": w.name + ("" if sliced else "_unsliced"), "n_gpus": P, **rep, "schedule": sched})
    plan.destroy()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="rc40", choices=sorted(workloads.BY_NAME))
    ap.add_argument("--unsliced", action="store_true", help="drop the workload's sliced labels")
    ap.add_argument("--gpus", type=int, nargs="+", default=[1, 2, 4, 8])
    ap.add_argument("--large-gib", type=float, default=8.0, help="large-step threshold s (GiB)")
    ap.add_argument("--dev-bw", type=float, default=6.6e12)
    ap.add_argument("--dev-flops", type=float, default=5.5e14)
    ap.add_argument("--net-bw", type=float, default=9.0e11)
    ap.add_argument("--latency", type=float, default=5e-6)
    ap.add_argument("--block-bytes", type=float, default=4096.0)
    a = ap.parse_args(argv)
    w = workloads.BY_NAME[a.workload]()
    for line in report(w, a.gpus, sliced=not a.unsliced, large_bytes=a.large_gib * 2**30, dev_bw=a.dev_bw,
                       dev_flops=a.dev_flops, net_bw=a.net_bw, latency=a.latency, block_bytes=a.block_bytes):
        print(json.dumps(line))


if __name__ == "__main__":
    main()
