"""CPU oracle for exact tensor-network contraction along a fixed path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its
binding) may import or call this module; it is used by tests/, by the package's
smoke check and by the timed CPU baseline in bench.py.

What it computes (Sec. II-A): result[open] = sum over all closed labels of the product
of all tensors. It evaluates that sum pairwise along the given path (Sec. II-B: the
result does not depend on the order), in complex128 (float64 for real networks):
  1. for each slice assignment (Sec. II-C; mixed radix, first sliced label most
     significant), restrict every leaf that carries a sliced label;
  2. for each step A x B -> C: the labels both operands carry are reduced (K), the
     rest are retained (M from A, N from B) -- the A_MK x B_KN -> C_MN view of
     Sec. II-B; permute A to [M, K] and B to [K, N] with numpy transposes, multiply
     with one matrix product, and give C the natural order M then N (the oracle does
     not reorder modes, so it is independent of the GEMM-oriented reordering);
  3. permute the root into the requested open-mode order;
  4. sum the slice results with Neumaier's compensated summation in slice-id order.

Semirings (Sec. III-C: counting and optimisation problems as contractions over other
semirings): semiring="maxplus" replaces the sum over labels by a maximum and the product
of tensors by a sum, so step 2 computes C[i, j] = max_k (A[i, k] + B[k, j]) (a plain loop
over k) and step 4 takes the maximum over slices. The default is the ordinary (+, x).

Also: the per-step cost counts of Sec. II-B (Eqs. 1-3), restated here on the oracle
side from the same definitions, for checking plan statistics.
"""
from __future__ import annotations

import math

import numpy as np


def slice_assignment(net, sliced, slice_id):
    """Values of the sliced labels for `slice_id` (first sliced label most significant)."""
    vals = {}
    r = int(slice_id)
    for x in reversed(list(sliced)):
        d = net.extent[x]
        vals[x] = r % d
        r //= d
    return vals


def restrict_leaves(net, vals):
    """Fix every sliced label of every leaf to its value; returns (arrays, modes)."""
    arrays, modes = [], []
    for t, ms in zip(net.tensors, net.modes):
        index = tuple(vals[x] if x in vals else slice(None) for x in ms)
        arrays.append(np.asarray(t)[index])
        modes.append(tuple(x for x in ms if x not in vals))
    return arrays, modes


def pairwise(a, ma, b, mb, keep, semiring="standard"):
    """One step: reduce the labels both operands carry (unless kept open)."""
    K = [x for x in ma if x in mb and x not in keep]
    M = [x for x in ma if x not in K]
    N = [x for x in mb if x not in K]
    # a label shared but kept open would be a hyper-edge; the workloads have none
    assert not any(x in mb for x in M), "shared open label (hyper-edge) not supported"
    pa = [ma.index(x) for x in M] + [ma.index(x) for x in K]
    pb = [mb.index(x) for x in K] + [mb.index(x) for x in N]
    m = int(np.prod([a.shape[ma.index(x)] for x in M], dtype=np.int64))
    n = int(np.prod([b.shape[mb.index(x)] for x in N], dtype=np.int64))
    k = int(np.prod([a.shape[ma.index(x)] for x in K], dtype=np.int64))
    A = np.transpose(a, pa).reshape(m, k)
    B = np.transpose(b, pb).reshape(k, n)
    if semiring == "maxplus":
        C = np.full((m, n), -np.inf)
        for kk in range(k):
            C = np.maximum(C, A[:, kk, None] + B[None, kk, :])
    else:
        C = A @ B
    shape = [a.shape[ma.index(x)] for x in M] + [b.shape[mb.index(x)] for x in N]
    return C.reshape(shape), tuple(M + N)


def contract_one(net, path, arrays, modes, semiring="standard"):
    dtype = np.complex128 if any(np.iscomplexobj(t) for t in arrays) else np.float64
    ts = [np.asarray(t, dtype=dtype) for t in arrays]
    ms = [tuple(m) for m in modes]
    keep = set(net.open_modes)
    for (i, j) in path.pairs:
        c, mc = pairwise(ts[i], ms[i], ts[j], ms[j], keep, semiring)
        ts.append(c)
        ms.append(mc)
        ts[i] = ts[j] = None  # each tensor is consumed once
    root, mroot = ts[-1], ms[-1]
    if len(path.pairs) == 0:
        root, mroot = ts[0], ms[0]
    perm = [mroot.index(x) for x in net.open_modes]
    return np.transpose(root, perm) if perm else root.reshape(())


class Neumaier:
    """Compensated running sum (Neumaier's variant of Kahan summation)."""

    def __init__(self, like):
        self.s = np.zeros_like(like, dtype=np.float64)
        self.c = np.zeros_like(self.s)

    def add(self, x):
        x = np.asarray(x, dtype=np.float64)
        t = self.s + x
        big = np.abs(self.s) >= np.abs(x)
        self.c = self.c + np.where(big, (self.s - t) + x, (x - t) + self.s)
        self.s = t

    def value(self):
        return self.s + self.c


def contract_slices(net, path, sliced=(), slice_ids=None, return_partials=False, semiring="standard"):
    """Sum (max-plus: maximum) of the slice results over `slice_ids` (default: all)."""
    sliced = list(sliced)
    n_slices = 1
    for x in sliced:
        n_slices *= net.extent[x]
    ids = range(n_slices) if slice_ids is None else list(slice_ids)
    partials = []
    acc_re = acc_im = None
    best = None
    for sid in ids:
        vals = slice_assignment(net, sliced, sid)
        arrays, modes = restrict_leaves(net, vals)
        r = contract_one(net, path, arrays, modes, semiring)
        if return_partials:
            partials.append(r)
        if semiring == "maxplus":
            best = r if best is None else np.maximum(best, r)
            continue
        if acc_re is None:
            acc_re, acc_im = Neumaier(np.real(r)), Neumaier(np.real(r))
        acc_re.add(np.real(r))
        acc_im.add(np.imag(r))
    if semiring == "maxplus":
        total = best
    else:
        total = acc_re.value() + 1j * acc_im.value() if net.is_complex else acc_re.value()
    if return_partials:
        return total, partials
    return total


def contract(net, path, sliced=(), semiring="standard"):
    """Exact result of the network along `path`, summing every slice."""
    return contract_slices(net, path, sliced, semiring=semiring)


# ---- cost counts (Sec. II-B, Eqs. 1-3), for plan-statistics checks -------------------

def step_costs(net, path, sliced=()):
    """Per step (m, n, k, Ct=mnk, Cs=max(mk,kn,mn), Cm=mk+kn+mn) after slicing."""
    sl = set(sliced)
    keep = set(net.open_modes)
    ms = [tuple(x for x in m if x not in sl) for m in net.modes]
    out = []
    for (i, j) in path.pairs:
        a, b = ms[i], ms[j]
        K = [x for x in a if x in b and x not in keep]
        M = [x for x in a if x not in K]
        N = [x for x in b if x not in K]
        m = math.prod(net.extent[x] for x in M)
        n = math.prod(net.extent[x] for x in N)
        k = math.prod(net.extent[x] for x in K)
        out.append(dict(m=m, n=n, k=k, Ct=m * n * k, Cs=max(m * k, k * n, m * n),
                        Cm=m * k + k * n + m * n))
        ms.append(tuple(M + N))
    return out


def path_costs(net, path, sliced=()):
    st = step_costs(net, path, sliced)
    return dict(Ct=sum(s["Ct"] for s in st), Cm=sum(s["Cm"] for s in st),
                Cs=max((s["Cs"] for s in st), default=0))
