"""ctypes binding of the C ABI in include/tn.h (argument marshalling only).

Every step of the contraction runs in the CUDA library; this module only converts
Python network descriptions and tensor handles into the plain arrays and pointers
the C functions take. Importing it fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtn_gb300.so")

# tn_status
TN_OK, TN_ERR_INVALID, TN_ERR_UNSUPPORTED, TN_ERR_OOM, TN_ERR_CUDA, TN_ERR_BUSY, \
    TN_ERR_TIMEOUT, TN_ERR_NOT_READY = range(8)
STATUS_NAMES = ["TN_OK", "TN_ERR_INVALID", "TN_ERR_UNSUPPORTED", "TN_ERR_OOM", "TN_ERR_CUDA",
                "TN_ERR_BUSY", "TN_ERR_TIMEOUT", "TN_ERR_NOT_READY"]
# tn_precision
TN_C64_FP32_SIMT, TN_C64_TF32, TN_C64_3XTF32, TN_C64_BF16X3, TN_R32_FP32_SIMT, TN_R32_TF32, \
    TN_R32_3XTF32, TN_R32_BF16X3 = range(8)
PREC_NAMES = {"fp32": 0, "tf32": 1, "3xtf32": 2, "bf16x3": 3, "bf16x3m": 3,
              "r32_fp32": 4, "r32_tf32": 5, "r32_3xtf32": 6, "r32_bf16x3": 7}
# forms named with the 3M complex product (three real products per complex MAC)
THREE_M = {"bf16x3m"}
TN_PLAN_HOST_ONLY = 1
TN_PLAN_SINGLE_SM_TILES = 2
TN_CLASS_SIMT, TN_CLASS_STREAM, TN_CLASS_TC, TN_CLASS_SPLITK, TN_CLASS_PERM = range(5)
N_CLASSES = 5
CLASS_NAMES = ["contract_simt", "contract_stream", "contract_tc", "contract_splitk", "stage_leaves"]


class TnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class tn_network(C.Structure):
    _fields_ = [("n_tensors", C.c_int32), ("rank", C.POINTER(C.c_int32)),
                ("modes", C.POINTER(C.POINTER(C.c_int32))), ("n_labels", C.c_int32),
                ("extent", C.POINTER(C.c_int64)), ("n_open", C.c_int32),
                ("open_modes", C.POINTER(C.c_int32))]


class tn_path(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("pair", C.POINTER(C.c_int32))]


class tn_dtype_policy(C.Structure):
    _fields_ = [("prec", C.c_int32), ("complex_mult", C.c_int32), ("exp_scaling", C.c_int32),
                ("max_slice_batch", C.c_int32), ("flags", C.c_uint32), ("semiring", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class tn_plan_stats(C.Structure):
    _fields_ = [("n_steps", C.c_int64), ("n_leaves", C.c_int64), ("n_slices", C.c_int64),
                ("slice_batch", C.c_int64), ("n_passes", C.c_int64), ("flops", C.c_double),
                ("bytes", C.c_double), ("Ct", C.c_double), ("Cm", C.c_double), ("Cs", C.c_double),
                ("peak_elems", C.c_int64), ("workspace_bytes", C.c_int64),
                ("steps_per_class", C.c_int64 * 5), ("flops_per_class", C.c_double * 5),
                ("leaf_permutes", C.c_int64)]


class tn_step_info(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("k", C.c_int64), ("a_id", C.c_int32),
                ("b_id", C.c_int32), ("cls", C.c_int32), ("batched", C.c_int32),
                ("n_row_dims", C.c_int32), ("n_col_dims", C.c_int32),
                ("row_ext", C.c_int64 * 12), ("row_stride", C.c_int64 * 12),
                ("col_ext", C.c_int64 * 12), ("col_stride", C.c_int64 * 12),
                ("ksplit", C.c_int32), ("single_sm", C.c_int32), ("chain", C.c_int32), ("reserved", C.c_int32)]


class tn_tensor_info(C.Structure):
    _fields_ = [("size", C.c_int64), ("offset", C.c_int64), ("bytes", C.c_int64),
                ("batched", C.c_int32), ("pinned", C.c_int32), ("producer", C.c_int32),
                ("consumer", C.c_int32),
                ("format", C.c_int32),
                ("tiled", C.c_int32)]


class tn_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 5), ("ms", C.c_double * 5), ("flops", C.c_double * 5),
                ("bytes", C.c_double * 5)]


class tn_serve_config(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("n_streams", C.c_int32),
                ("hbm_budget_bytes", C.c_int64), ("queue_capacity", C.c_int32),
                ("pack_max", C.c_int32), ("reserved", C.c_int32 * 2)]


class tn_serve_stats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("plan_launches", C.c_int64), ("packs", C.c_int64),
                ("packed_requests", C.c_int64), ("max_pack", C.c_int64), ("hbm_in_use", C.c_int64)]


class tn_cost_model(C.Structure):
    _fields_ = [("hbm_bytes_per_s", C.c_double), ("simt_flops", C.c_double), ("tc_flops", C.c_double * 3)]


class tn_dist_config(C.Structure):
    _fields_ = [("n_gpus", C.c_int32), ("reserved0", C.c_int32), ("large_bytes", C.c_double),
                ("gather_bytes", C.c_double), ("dev_bw", C.c_double), ("dev_flops", C.c_double),
                ("net_bw", C.c_double), ("latency", C.c_double), ("block_bytes", C.c_double)]


class tn_dist_step(C.Structure):
    _fields_ = [("state", C.c_int32), ("forced", C.c_int32), ("chain", C.c_int32), ("n_dist", C.c_int32),
                ("dist_modes", C.c_int32 * 16), ("t_gemm", C.c_double), ("t_comm", C.c_double),
                ("out_bytes", C.c_double), ("n_blk", C.c_int64)]


class tn_dist_report(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("n_redistributions", C.c_int32), ("n_forced", C.c_int32),
                ("n_gathers", C.c_int32), ("n_large_steps", C.c_int64), ("dp_states", C.c_int64),
                ("t_total", C.c_double), ("t_single", C.c_double), ("t_comm_total", C.c_double),
                ("bytes_redistributed", C.c_double), ("speedup", C.c_double), ("extra_speedup", C.c_double),
                ("projected_total", C.c_double)]


DIST_STATES = ("none", "activate", "keep", "redistribute", "gather")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2606_01852_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "tn_plan": [C.POINTER(tn_network), C.POINTER(tn_path), C.POINTER(i32), i32, tn_dtype_policy,
                    C.POINTER(vp)],
        "tn_plan_info": [vp, C.POINTER(tn_plan_stats)],
        "tn_plan_layout": [vp, i32, C.POINTER(i32), C.POINTER(i32)],
        "tn_plan_step": [vp, i32, C.POINTER(tn_step_info)],
        "tn_plan_launches": [vp, i64, C.POINTER(i64)],
        "tn_plan_tensor": [vp, i32, C.POINTER(tn_tensor_info)],
        "tn_contract": [vp, C.POINTER(vp), vp, vp, vp],
        "tn_contract_graph": [vp, C.POINTER(vp), vp, vp, vp],
        "tn_plan_autotune": [vp, C.POINTER(vp), vp, vp],
        "tn_contract_slices": [vp, C.POINTER(vp), i64, i64, vp, vp, vp],
        "tn_contract_host": [vp, C.POINTER(vp), vp, vp, vp],
        "tn_contract_slices_host": [vp, C.POINTER(vp), i64, i64, vp, vp, vp],
        "tn_plan_destroy": [vp],
        "tn_plan_profile": [vp, i32],
        "tn_plan_profile_read": [vp, C.POINTER(tn_profile), i32],
        "tn_plan_profile_steps": [vp, C.POINTER(C.c_double), i32],
        "tn_selftest_bounded_wait": [vp, i32, i64, vp],
        "tn_serve_create": [C.POINTER(tn_serve_config), C.POINTER(vp)],
        "tn_serve_submit": [vp, vp, C.POINTER(vp), C.POINTER(u64)],
        "tn_serve_submit_batch": [vp, i32, C.POINTER(vp), C.POINTER(C.POINTER(vp)), C.POINTER(u64)],
        "tn_serve_poll": [vp, u64, vp, vp, i32],
        "tn_serve_destroy": [vp],
        "tn_serve_stats_get": [vp, C.POINTER(tn_serve_stats)],
        "tn_dot_noalloc": [vp, vp, i64, i64, i64, i64, vp, vp],
        "tn_batch_plan": [i32, C.POINTER(tn_network), C.POINTER(tn_path), tn_dtype_policy, C.POINTER(vp)],
        "tn_batch_info": [vp, C.POINTER(i64), C.POINTER(C.c_double), C.POINTER(i32), C.POINTER(i32),
                          C.POINTER(i32), C.POINTER(i32)],
        "tn_batch_contract": [vp, vp, vp, vp, vp],
        "tn_batch_contract_graph": [vp, vp, vp, vp, vp],
        "tn_batch_autotune": [vp, vp, vp, vp, vp],
        "tn_batch_set_shape": [vp, i32, i32, i32, i32],
        "tn_batch_destroy": [vp],
        "tn_plan_distribute": [vp, C.POINTER(tn_dist_config), C.POINTER(tn_dist_report), C.POINTER(tn_dist_step)],
        "tn_cost_model_set": [C.POINTER(tn_cost_model)],
        "tn_plan_check_staging": [vp, i64],
        "tn_cost_model_get": [C.POINTER(tn_cost_model)],
        "tn_measure_ffma": [i64, C.POINTER(C.c_double), C.POINTER(C.c_double), vp],
        "tn_measure_dfma": [i64, C.POINTER(C.c_double), C.POINTER(C.c_double), vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.tn_last_error.argtypes = []
    lib.tn_last_error.restype = C.c_char_p
    return lib


lib = _load()


def check(status):
    if status != TN_OK:
        raise TnError(status, lib.tn_last_error().decode())


def last_error() -> str:
    return lib.tn_last_error().decode()


def _ptr(x):
    """Raw address of a tensor/array/int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


SEMIRINGS = {"standard": 0, "maxplus": 1}


def make_policy(prec=TN_C64_FP32_SIMT, exp_scaling=False, max_slice_batch=0, host_only=False, semiring="standard",
                complex_mult=4, single_sm_tiles=False):
    """prec: a tn_precision or a form name ("bf16x3m" = BF16X3 with the 3M product; the
    real forms "r32_fp32", "r32_tf32", "r32_3xtf32")."""
    if isinstance(prec, str):
        if prec in THREE_M:
            complex_mult = 3
        prec = PREC_NAMES[prec]
    p = tn_dtype_policy()
    p.semiring = SEMIRINGS[semiring]
    p.prec = int(prec)
    p.complex_mult = int(complex_mult)
    p.exp_scaling = 1 if exp_scaling else 0
    p.max_slice_batch = int(max_slice_batch)
    p.flags = (TN_PLAN_HOST_ONLY if host_only else 0) | (TN_PLAN_SINGLE_SM_TILES if single_sm_tiles else 0)
    return p


class _NetArrays:
    """Keeps the ctypes arrays of a network description alive."""

    def __init__(self, modes, extent, open_modes, pairs):
        n_labels = (max(extent) + 1) if extent else 0
        self.rank = (C.c_int32 * len(modes))(*[len(m) for m in modes])
        self.mode_arrays = [(C.c_int32 * max(1, len(m)))(*m) for m in modes]
        self.modes = (C.POINTER(C.c_int32) * len(modes))(
            *[C.cast(a, C.POINTER(C.c_int32)) for a in self.mode_arrays])
        ext = [1] * n_labels
        for x, e in extent.items():
            ext[x] = int(e)
        self.extent = (C.c_int64 * max(1, n_labels))(*ext)
        self.open = (C.c_int32 * max(1, len(open_modes)))(*open_modes)
        flat = [int(v) for p in pairs for v in p]
        self.pair = (C.c_int32 * max(1, len(flat)))(*flat)
        self.net = tn_network(len(modes), self.rank, self.modes, n_labels, self.extent,
                              len(open_modes), self.open)
        self.path = tn_path(len(pairs), self.pair)


class Plan:
    """A contraction plan (tn_plan). `net` needs .modes, .extent, .open_modes;
    `path` is a list of SSA pairs or an object with .pairs."""

    def __init__(self, net, path, sliced=(), prec=TN_C64_FP32_SIMT, exp_scaling=False,
                 max_slice_batch=0, host_only=False, semiring="standard", complex_mult=4, single_sm_tiles=False):
        pairs = path.pairs if hasattr(path, "pairs") else path
        self._arr = _NetArrays([tuple(m) for m in net.modes], dict(net.extent), tuple(net.open_modes),
                               pairs)
        sl = list(sliced)
        self._sl = (C.c_int32 * max(1, len(sl)))(*sl)
        self.policy = make_policy(prec, exp_scaling, max_slice_batch, host_only, semiring, complex_mult,
                                  single_sm_tiles)
        self.is_complex = self.policy.prec <= TN_C64_BF16X3
        self.n_leaves = len(net.modes)
        self.n_open = len(net.open_modes)
        self.out_shape = tuple(net.extent[x] for x in net.open_modes)
        h = C.c_void_p()
        check(lib.tn_plan(C.byref(self._arr.net), C.byref(self._arr.path), self._sl, len(sl),
                          self.policy, C.byref(h)))
        self.handle = h

    # -- queries
    def info(self) -> dict:
        s = tn_plan_stats()
        check(lib.tn_plan_info(self.handle, C.byref(s)))
        d = {f: getattr(s, f) for f, _ in tn_plan_stats._fields_}
        d["steps_per_class"] = list(s.steps_per_class)
        d["flops_per_class"] = list(s.flops_per_class)
        return d

    def layout(self, tid: int):
        r = C.c_int32()
        check(lib.tn_plan_layout(self.handle, tid, None, C.byref(r)))
        buf = (C.c_int32 * max(1, r.value))()
        check(lib.tn_plan_layout(self.handle, tid, buf, C.byref(r)))
        return tuple(buf[: r.value])

    def step(self, s: int) -> dict:
        i = tn_step_info()
        check(lib.tn_plan_step(self.handle, s, C.byref(i)))
        d = {f: getattr(i, f) for f, _ in tn_step_info._fields_[:7]}
        d["ksplit"] = i.ksplit
        d["single_sm"] = i.single_sm
        d["chain"] = i.chain
        d["rows"] = [(i.row_ext[x], i.row_stride[x]) for x in range(i.n_row_dims)]
        d["cols"] = [(i.col_ext[x], i.col_stride[x]) for x in range(i.n_col_dims)]
        return d

    def tensor(self, tid: int) -> dict:
        i = tn_tensor_info()
        check(lib.tn_plan_tensor(self.handle, tid, C.byref(i)))
        return {f: getattr(i, f) for f, _ in tn_tensor_info._fields_}

    # -- execution
    def _inputs(self, inputs):
        if len(inputs) != self.n_leaves:
            raise ValueError(f"expected {self.n_leaves} inputs, got {len(inputs)}")
        arr = (C.c_void_p * self.n_leaves)(*[_ptr(t) for t in inputs])
        return arr

    def contract(self, inputs, output, log_scale=None, stream=None):
        check(lib.tn_contract(self.handle, self._inputs(inputs), _ptr(output), _ptr(log_scale),
                              _ptr_stream(stream)))

    def autotune(self, inputs, output, stream=None):
        """tn_plan_autotune: per paired-SM step, keep the faster of paired SMs and one SM."""
        check(lib.tn_plan_autotune(self.handle, self._inputs(inputs), _ptr(output), _ptr_stream(stream)))

    def contract_graph(self, inputs, output, log_scale=None, stream=None):
        """tn_contract_graph: as contract, replayed from a CUDA graph captured on the first call
        with these pointers and stream."""
        check(lib.tn_contract_graph(self.handle, self._inputs(inputs), _ptr(output), _ptr(log_scale),
                                    _ptr_stream(stream)))

    def contract_slices(self, inputs, begin, count, output, log_scale=None, stream=None):
        check(lib.tn_contract_slices(self.handle, self._inputs(inputs), int(begin), int(count),
                                     _ptr(output), _ptr(log_scale), _ptr_stream(stream)))

    def contract_host(self, host_inputs, host_output, log_scale=None, stream=None):
        check(lib.tn_contract_host(self.handle, self._inputs(host_inputs), _ptr(host_output),
                                   _ptr(log_scale), _ptr_stream(stream)))

    def contract_slices_host(self, host_inputs, begin, count, host_output, log_scale=None, stream=None):
        check(lib.tn_contract_slices_host(self.handle, self._inputs(host_inputs), int(begin), int(count),
                                          _ptr(host_output), _ptr(log_scale), _ptr_stream(stream)))

    def flops_per_call(self, count=None) -> float:
        """Algorithmic flops of one contract over `count` slices (default all): the
        slice-invariant steps once, the sliced steps once per slice."""
        info = self.info()
        count = info["n_slices"] if count is None else count
        fm = 8.0 if self.is_complex else 2.0
        tot = 0.0
        for s in range(info["n_steps"]):
            st = self.step(s)
            tot += fm * st["m"] * st["n"] * st["k"] * (count if st["batched"] else 1)
        return tot

    def check_staging(self, max_slices=4):
        """Host replay of the tiled staging kernel's index arithmetic (tn_plan_check_staging)."""
        check(lib.tn_plan_check_staging(self.handle, int(max_slices)))

    def profile(self, enable: bool):
        check(lib.tn_plan_profile(self.handle, 1 if enable else 0))

    def profile_read(self, reset=True) -> dict:
        p = tn_profile()
        check(lib.tn_plan_profile_read(self.handle, C.byref(p), 1 if reset else 0))
        return {f: list(getattr(p, f)) for f, _ in tn_profile._fields_}

    def selftest_bounded_wait(self, arrive: bool, limit_us: int, stream=None) -> int:
        """Run the kernels' bounded mbarrier wait on a barrier completed only if `arrive`;
        returns the status (TN_OK, or TN_ERR_TIMEOUT when the wait ran out)."""
        return lib.tn_selftest_bounded_wait(self.handle, 1 if arrive else 0, int(limit_us), _ptr_stream(stream))

    def profile_steps(self):
        """Per-step device milliseconds of the last profile_read(reset=True)."""
        n = self.info()["n_steps"]
        buf = (C.c_double * max(1, n))()
        check(lib.tn_plan_profile_steps(self.handle, buf, n))
        return list(buf[:n])

    def distribute(self, n_gpus, large_bytes=8 * 2**30, gather_bytes=0.0, dev_bw=6.6e12, dev_flops=5.5e14,
                   net_bw=9.0e11, latency=5e-6, block_bytes=4096.0):
        """Offline distribution plan of Sec. IV-B (tn_plan_distribute): returns (report,
        steps), the per-step schedule as dicts (state name, split modes, Eq. 6/7 times).
        Defaults: one GB300 (measured HBM copy rate, the BF16x3 form's rate) on an NVLink
        domain (900 GB/s per direction), 5 us per message, 4 KiB base blocks."""
        cfg = tn_dist_config(n_gpus=n_gpus, large_bytes=large_bytes, gather_bytes=gather_bytes, dev_bw=dev_bw,
                             dev_flops=dev_flops, net_bw=net_bw, latency=latency, block_bytes=block_bytes)
        n = self.info()["n_steps"]
        rep = tn_dist_report()
        buf = (tn_dist_step * max(1, n))()
        check(lib.tn_plan_distribute(self.handle, C.byref(cfg), C.byref(rep), buf))
        report = {f: getattr(rep, f) for f, _ in tn_dist_report._fields_}
        steps = []
        for s in range(n):
            r = buf[s]
            steps.append({"state": DIST_STATES[r.state], "forced": bool(r.forced), "chain": r.chain,
                          "dist_modes": list(r.dist_modes[:r.n_dist]), "t_gemm": r.t_gemm, "t_comm": r.t_comm,
                          "out_bytes": r.out_bytes, "n_blk": r.n_blk})
        return report, steps

    def launches_per_call(self, count=None) -> int:
        """Kernel launches of one contract over `count` slices (default all): tn_plan_launches."""
        count = self.info()["n_slices"] if count is None else count
        n = C.c_int64()
        check(lib.tn_plan_launches(self.handle, int(count), C.byref(n)))
        return n.value

    def destroy(self):
        if getattr(self, "handle", None):
            lib.tn_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Batch:
    """Many small closed networks, one persistent launch (tn_batch_*)."""

    def __init__(self, nets, paths, complex_=False, exp_scaling=True, host_only=False, semiring="standard"):
        self._arrs = [_NetArrays([tuple(m) for m in n.modes], dict(n.extent), tuple(n.open_modes),
                                 p.pairs if hasattr(p, "pairs") else p) for n, p in zip(nets, paths)]
        self.n_nets = len(nets)
        self.complex = complex_
        netv = (tn_network * self.n_nets)(*[a.net for a in self._arrs])
        pathv = (tn_path * self.n_nets)(*[a.path for a in self._arrs])
        pol = make_policy(TN_C64_FP32_SIMT if complex_ else TN_R32_FP32_SIMT, exp_scaling, 1, host_only, semiring)
        h = C.c_void_p()
        check(lib.tn_batch_plan(self.n_nets, netv, pathv, pol, C.byref(h)))
        self.handle = h
        self.n_leaves = sum(len(n.modes) for n in nets)
        off = (C.c_int64 * (self.n_leaves + 1))()
        fl = C.c_double()
        check(lib.tn_batch_info(h, off, C.byref(fl), None, None, None, None))
        self.leaf_offsets = list(off)
        self.flops = fl.value

    def pack(self, nets):
        """Concatenate every leaf (declared order) into one host array."""
        dt = np.complex64 if self.complex else np.float32
        out = np.empty(self.leaf_offsets[-1], dtype=dt)
        i = 0
        for n in nets:
            for t in n.tensors:
                a = np.asarray(t, dtype=dt).ravel()
                out[self.leaf_offsets[i]: self.leaf_offsets[i] + a.size] = a
                i += 1
        return out

    def launch_shape(self):
        """(threads per network, CTAs per SM, networks per CTA, shared-memory arena floats)."""
        t, c, g, m = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        check(lib.tn_batch_info(self.handle, None, None, C.byref(t), C.byref(c), C.byref(g), C.byref(m)))
        return t.value, c.value, g.value, m.value

    def set_launch_shape(self, threads, ctas_per_sm, nets_per_cta=1, smem_arena=0):
        """Choose a launch shape by hand (tn_batch_set_shape); smem_arena: floats of shared
        memory per network slot (0: global arenas only)."""
        check(lib.tn_batch_set_shape(self.handle, int(threads), int(ctas_per_sm), int(nets_per_cta),
                                     int(smem_arena)))

    def contract(self, packed, values, logs, stream=None, graph=False):
        f = lib.tn_batch_contract_graph if graph else lib.tn_batch_contract
        check(f(self.handle, _ptr(packed), _ptr(values), _ptr(logs), _ptr_stream(stream)))

    def autotune(self, packed, values, logs, stream=None):
        check(lib.tn_batch_autotune(self.handle, _ptr(packed), _ptr(values), _ptr(logs), _ptr_stream(stream)))

    def destroy(self):
        if getattr(self, "handle", None):
            lib.tn_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def cost_model() -> dict:
    """The planner's Eq. 6 rates (tn_cost_model_get)."""
    m = tn_cost_model()
    check(lib.tn_cost_model_get(C.byref(m)))
    return {"hbm_bytes_per_s": m.hbm_bytes_per_s, "simt_flops": m.simt_flops, "tc_flops": list(m.tc_flops)}


def set_cost_model(hbm_bytes_per_s, simt_flops, tc_flops):
    """Replace the planner's Eq. 6 rates (tn_cost_model_set); tc_flops = [TF32, 3xTF32, BF16x3]."""
    m = tn_cost_model(hbm_bytes_per_s, simt_flops, (C.c_double * 3)(*tc_flops))
    check(lib.tn_cost_model_set(C.byref(m)))


def measure_dfma(iters=1 << 14, stream=None):
    """FP64 FMA rate of the current device (tn_measure_dfma): (flop/s, ms)."""
    f, ms = C.c_double(), C.c_double()
    check(lib.tn_measure_dfma(int(iters), C.byref(f), C.byref(ms), _ptr_stream(stream)))
    return f.value, ms.value


def measure_ffma(iters=1 << 18, stream=None):
    """FP32 FMA rate of the current device (tn_measure_ffma): (flop/s, ms)."""
    f, ms = C.c_double(), C.c_double()
    check(lib.tn_measure_ffma(int(iters), C.byref(f), C.byref(ms), _ptr_stream(stream)))
    return f.value, ms.value


def dot_noalloc(a, b, batch, m, n, k, out, stream=None):
    """tn_dot_noalloc: out[b][i][j] = sum_t a[b][i][t] b[b][j][t] with no device allocation
    (device complex64 inputs, device complex128 output, caller-owned)."""
    check(lib.tn_dot_noalloc(_ptr(a), _ptr(b), int(batch), int(m), int(n), int(k), _ptr(out),
                             _ptr_stream(stream)))


def _ptr_stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Server:
    """Continuous-batching request loop (tn_serve_*)."""

    def __init__(self, max_inflight=8, n_streams=4, hbm_budget_bytes=0, queue_capacity=4096, pack_max=0):
        cfg = tn_serve_config()
        cfg.max_inflight = max_inflight
        cfg.n_streams = n_streams
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.queue_capacity = queue_capacity
        cfg.pack_max = pack_max
        h = C.c_void_p()
        check(lib.tn_serve_create(C.byref(cfg), C.byref(h)))
        self.handle = h

    def submit(self, plan: Plan, host_inputs) -> int:
        t = C.c_uint64()
        check(lib.tn_serve_submit(self.handle, plan.handle, plan._inputs(host_inputs), C.byref(t)))
        return t.value

    def submit_batch(self, requests) -> list:
        """Queue [(plan, host_inputs), ...] together (tn_serve_submit_batch); the tickets."""
        n = len(requests)
        plans = (C.c_void_p * max(1, n))(*[p.handle.value if hasattr(p.handle, "value") else p.handle
                                          for p, _ in requests])
        arrs = [p._inputs(x) for p, x in requests]
        ins = (C.POINTER(C.c_void_p) * max(1, n))(*[C.cast(a, C.POINTER(C.c_void_p)) for a in arrs])
        tickets = (C.c_uint64 * max(1, n))()
        check(lib.tn_serve_submit_batch(self.handle, n, plans, ins, tickets))
        return list(tickets)[:n]

    def try_submit(self, plan: Plan, host_inputs):
        t = C.c_uint64()
        s = lib.tn_serve_submit(self.handle, plan.handle, plan._inputs(host_inputs), C.byref(t))
        return s, t.value

    def poll(self, ticket, result, log_scale=None, timeout_us=-1):
        return lib.tn_serve_poll(self.handle, C.c_uint64(ticket), _ptr(result), _ptr(log_scale),
                                 int(timeout_us))

    def stats(self) -> dict:
        s = tn_serve_stats()
        check(lib.tn_serve_stats_get(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in tn_serve_stats._fields_}

    def destroy(self):
        if getattr(self, "handle", None):
            check(lib.tn_serve_destroy(self.handle))
            self.handle = None
