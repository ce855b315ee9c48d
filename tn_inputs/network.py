"""Plain containers for a tensor network, a contraction path and slicing metadata.

This module holds data only: no contraction arithmetic. Both the CPU oracle and the
GPU library consume the same `Network`/`Path` objects, which is the only thing the two
sides share.

Conventions (Sec. II-A/B of the paper):
  * a network is a list of tensors, each a row-major array whose axes are named by
    integer mode labels; every label has one extent (all 2 in the generated workloads);
  * a label shared by two tensors is closed (summed), a label listed in `open_modes`
    survives in the result, in that order;
  * a contraction path is the ordered list of pairwise steps in SSA form: leaves are
    0..T-1 and step s produces tensor T+s (a binary contraction tree, Sec. II-B);
  * sliced labels are fixed to each of their values in turn and the partial results
    summed (Sec. II-C); slice ids enumerate the mixed-radix assignment with the first
    sliced label most significant.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    tensors: list            # numpy arrays, one axis per mode, row-major
    modes: list              # list of tuples of int labels, one per tensor
    extent: dict             # label -> extent
    open_modes: tuple = ()   # labels of the result, in result order
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_tensors(self) -> int:
        return len(self.tensors)

    @property
    def is_complex(self) -> bool:
        return any(np.iscomplexobj(t) for t in self.tensors)

    def labels(self) -> list:
        seen = []
        s = set()
        for ms in self.modes:
            for x in ms:
                if x not in s:
                    s.add(x)
                    seen.append(x)
        return seen

    def n_labels(self) -> int:
        return max(self.extent) + 1 if self.extent else 0

    def check(self) -> None:
        count = {}
        for t, ms in zip(self.tensors, self.modes):
            assert t.ndim == len(ms), (t.shape, ms)
            assert len(set(ms)) == len(ms), f"repeated label in {ms}"
            for ax, x in enumerate(ms):
                assert t.shape[ax] == self.extent[x]
                count[x] = count.get(x, 0) + 1
        for x, c in count.items():
            want = 1 if x in self.open_modes else 2
            assert c == want, f"label {x} appears {c} times (open={x in self.open_modes})"
        for x in self.open_modes:
            assert x in count


@dataclass
class Path:
    pairs: list              # list of (i, j) SSA ids

    @property
    def n_steps(self) -> int:
        return len(self.pairs)


def relabel_compact(net: Network) -> Network:
    """Renumber labels to 0..L-1 in order of first appearance (keeps results identical)."""
    order = net.labels()
    remap = {x: i for i, x in enumerate(order)}
    return Network(
        tensors=list(net.tensors),
        modes=[tuple(remap[x] for x in ms) for ms in net.modes],
        extent={remap[x]: net.extent[x] for x in order},
        open_modes=tuple(remap[x] for x in net.open_modes),
        name=net.name,
        meta=dict(net.meta),
    )
