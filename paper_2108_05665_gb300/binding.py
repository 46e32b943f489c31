"""ctypes binding of the C ABI in include/xeb.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  The library
must have been built (``paper_2108_05665_gb300.build.build()``); loading fails
loudly otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

XEB_OK = 0
STATUS_NAMES = {0: "XEB_OK", 1: "XEB_EINVAL", 2: "XEB_ENOMEM", 3: "XEB_ECUDA", 4: "XEB_ETIMEOUT",
                5: "XEB_EUNSUPPORTED", 6: "XEB_ECANCELLED", 7: "XEB_EDEVICE"}

XEB_PREC_FP32 = 0
XEB_PREC_TF32X3 = 1
XEB_PREC_FP64 = 2

XEB_PLANNER_AUTO = 0
XEB_PLANNER_GREEDY = 1
XEB_PLANNER_SWEEP = 2
XEB_PLANNER_ANNEAL = 3

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_dblp = ctypes.POINTER(ctypes.c_double)


class XebError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class xeb_circuit(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("n_gates", ctypes.c_int), ("kinds", _i32p),
                ("q0", _i32p), ("q1", _i32p), ("mats", _dblp)]


class xeb_tree(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("children", _i32p)]


class xeb_slices(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("legs", _i32p)]


class xeb_plan_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("planner", ctypes.c_int), ("block_qubits", ctypes.c_int),
                ("group_leaves", ctypes.c_int), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("mem_budget", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("greedy_trials", ctypes.c_int),
                ("reserved", ctypes.c_int * 8), ("split_bits", ctypes.c_int), ("split_terms", ctypes.c_int),
                ("timeout_ms", ctypes.c_uint32), ("fold_legs", ctypes.c_int)]


class xeb_stats(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("n_leaves", ctypes.c_int), ("n_legs", ctypes.c_int),
                ("n_nodes", ctypes.c_int), ("n_sliced", ctypes.c_int), ("k", ctypes.c_uint64),
                ("k_distinct", ctypes.c_uint64), ("flops_per_slice", ctypes.c_double),
                ("single_amp_flops", ctypes.c_double), ("rw_elems_per_slice", ctypes.c_double),
                ("permute_elems_per_slice", ctypes.c_double), ("objective", ctypes.c_double),
                ("arena_bytes", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("n_slices", ctypes.c_uint64), ("n_gemm_ops", ctypes.c_int), ("n_permute_ops", ctypes.c_int),
                ("planner_used", ctypes.c_int), ("n_tc_launches", ctypes.c_int), ("n_tc_tma", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]

    def as_dict(self):
        d = {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "reserved"}
        d["n_reused"] = self.reserved[0]   # nodes kept across slices (cross-slice reuse)
        d["n_folded"] = self.reserved[1]   # nodes evaluated on the host (constant folding)
        d["n_fold_roots"] = self.reserved[2]
        return d


_PROTOS = {
    "xeb_default_opts": (None, [ctypes.POINTER(xeb_plan_opts)]),
    "xeb_plan_test_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "xeb_round_keep_norm": (None, [_dblp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_float)]),
    "xeb_network_info": (ctypes.c_int, [ctypes.POINTER(xeb_circuit), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "xeb_network_leaves": (ctypes.c_int, [ctypes.POINTER(xeb_circuit), _i32p, _i32p]),
    "xeb_plan_create": (ctypes.c_int, [ctypes.POINTER(xeb_circuit), _u64p, ctypes.c_size_t,
                                       ctypes.POINTER(xeb_tree), ctypes.POINTER(xeb_slices),
                                       ctypes.POINTER(xeb_plan_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "xeb_plan_destroy": (None, [ctypes.c_void_p]),
    "xeb_plan_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(xeb_stats)]),
    "xeb_plan_tree": (ctypes.c_int, [ctypes.c_void_p, _i32p, _i32p]),
    "xeb_plan_node": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _i64p, _i32p, _i32p, _i32p, _i32p]),
    "xeb_plan_device_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "xeb_plan_bind": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "xeb_set_bitstrings": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "xeb_amplitudes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "xeb_fidelity": (ctypes.c_int, [ctypes.c_void_p, _dblp, _dblp, _dblp, ctypes.c_void_p]),
    "xeb_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, _dblp,
                               ctypes.c_void_p]),
    "xeb_plan_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _i32p, _i32p, _i32p, ctypes.c_void_p]),
    "xeb_plan_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "xeb_plan_candidates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "xeb_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "xeb_mlp_destroy": (None, [ctypes.c_void_p]),
    "xeb_mlp_n_params": (ctypes.c_size_t, [ctypes.c_void_p]),
    "xeb_mlp_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "xeb_mlp_set_norm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "xeb_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64]),
    "xeb_mlp_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "xeb_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_uint64]),
    "xeb_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.POINTER(ctypes.c_int32)]),
    "xeb_plan_profile_read": (ctypes.c_int, [ctypes.c_void_p, _dblp, _dblp, _dblp, _dblp]),
    "xeb_linear_xeb_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "xeb_set_slice_subset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64,
                                            ctypes.POINTER(ctypes.c_int64)]),
    "xeb_set_slice_block": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "xeb_plan_slice_ids": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "xeb_plan_create_batched": (ctypes.c_int, [ctypes.POINTER(xeb_circuit), _u64p, ctypes.c_size_t, ctypes.c_uint64,
                                               ctypes.POINTER(xeb_tree), ctypes.POINTER(xeb_slices),
                                               ctypes.POINTER(xeb_plan_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "xeb_run_chunked": (ctypes.c_int, [ctypes.POINTER(xeb_circuit), _u64p, ctypes.c_size_t, ctypes.POINTER(xeb_tree),
                                       ctypes.POINTER(xeb_slices), ctypes.POINTER(xeb_plan_opts), ctypes.c_size_t,
                                       _dblp, _dblp, _dblp, _dblp, ctypes.c_void_p]),
    "xeb_plan_buffers": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _i32p]),
    "xeb_plan_step_flops": (ctypes.c_int, [ctypes.c_void_p, _dblp, _dblp]),
    "xeb_plan_op_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _i32p, ctypes.c_int, _i32p]),
    "xeb_plan_profile_ops": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dblp, _dblp, _i32p, _dblp,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "xeb_plan_op_form": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _i32p]),
    "xeb_plan_create_learned": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, _dblp,
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "xeb_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libxeb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = path or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("native library %s is missing: run paper_2108_05665_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status):
    if status != XEB_OK:
        raise XebError(status, load().xeb_last_error().decode())


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class CircuitArrays:
    """Keeps the numpy arrays behind an xeb_circuit alive."""

    def __init__(self, circuit):
        kinds, q0, q1, mats = circuit.as_arrays()
        self.kinds = np.ascontiguousarray(kinds, dtype=np.int32)
        self.q0 = np.ascontiguousarray(q0, dtype=np.int32)
        self.q1 = np.ascontiguousarray(q1, dtype=np.int32)
        self.mats = np.ascontiguousarray(mats, dtype=np.complex128).view(np.float64)
        self.c = xeb_circuit(circuit.n_qubits, len(self.kinds), _ptr(self.kinds, ctypes.c_int32),
                             _ptr(self.q0, ctypes.c_int32), _ptr(self.q1, ctypes.c_int32),
                             _ptr(self.mats, ctypes.c_double))


def xeb_default_opts() -> xeb_plan_opts:
    o = xeb_plan_opts()
    load().xeb_default_opts(ctypes.byref(o))
    return o


def xeb_round_keep_norm(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(x.shape, dtype=np.float32)
    load().xeb_round_keep_norm(x.ctypes.data_as(_dblp), x.size, y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return y


def xeb_network_info(circuit):
    ca = CircuitArrays(circuit)
    nl, ng = ctypes.c_int(), ctypes.c_int()
    _check(load().xeb_network_info(ctypes.byref(ca.c), ctypes.byref(nl), ctypes.byref(ng)))
    return nl.value, ng.value


def xeb_network_leaves(circuit):
    nl, _ = xeb_network_info(circuit)
    ca = CircuitArrays(circuit)
    out = np.empty(2 * nl, dtype=np.int32)
    legs = np.empty(4 * nl, dtype=np.int32)
    _check(load().xeb_network_leaves(ctypes.byref(ca.c), _ptr(out, ctypes.c_int32), _ptr(legs, ctypes.c_int32)))
    return ([list(x[x >= 0]) for x in out.reshape(-1, 2)], [list(x[x >= 0]) for x in legs.reshape(-1, 4)])


def xeb_plan_create(circuit, bitstrings, tree: Optional[Sequence] = None, slices: Optional[Sequence[int]] = None,
                    opts: Optional[xeb_plan_opts] = None, open_qubits: Optional[Sequence[int]] = None) -> ctypes.c_void_p:
    """xeb_plan_create, or xeb_plan_create_batched when open_qubits is given."""
    ca = CircuitArrays(circuit)
    bs = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    tp = None
    if tree is not None:
        ch = np.ascontiguousarray(np.asarray(tree, dtype=np.int32).reshape(-1))
        t = xeb_tree(len(ch) // 2, _ptr(ch, ctypes.c_int32))
        tp = ctypes.byref(t)
    sp = None
    if slices is not None:
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.int32))
        s = xeb_slices(len(sl), _ptr(sl, ctypes.c_int32))
        sp = ctypes.byref(s)
    out = ctypes.c_void_p()
    op = ctypes.byref(opts) if opts is not None else None
    if open_qubits is not None:
        mask = 0
        for q in open_qubits:
            mask |= 1 << int(q)
        _check(load().xeb_plan_create_batched(ctypes.byref(ca.c), _ptr(bs, ctypes.c_uint64), len(bs), mask, tp, sp,
                                              op, ctypes.byref(out)))
    else:
        _check(load().xeb_plan_create(ctypes.byref(ca.c), _ptr(bs, ctypes.c_uint64), len(bs), tp, sp, op,
                                      ctypes.byref(out)))
    return out


def xeb_plan_create_learned(circuit, bitstrings, mlp, opts=None, max_cands: int = 256, stream: int = 0):
    """xeb_plan_create_learned: the plan of the candidate `mlp` (a Mlp) predicts
    fastest; returns (plan handle, predicted log2 ms)."""
    ca = CircuitArrays(circuit)
    bs = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    out = ctypes.c_void_p()
    pred = ctypes.c_double()
    op = ctypes.byref(opts) if opts is not None else None
    _check(load().xeb_plan_create_learned(ctypes.byref(ca.c), _ptr(bs, ctypes.c_uint64), len(bs), op, mlp.handle,
                                          max_cands, ctypes.c_void_p(stream or None), ctypes.byref(pred),
                                          ctypes.byref(out)))
    return out, pred.value


def xeb_plan_destroy(plan):
    load().xeb_plan_destroy(plan)


def xeb_plan_stats(plan) -> dict:
    s = xeb_stats()
    _check(load().xeb_plan_stats(plan, ctypes.byref(s)))
    return s.as_dict()


def xeb_plan_tree(plan):
    st = xeb_plan_stats(plan)
    ch = np.empty(2 * st["n_nodes"], dtype=np.int32)
    sl = np.empty(max(st["n_sliced"], 1), dtype=np.int32)
    _check(load().xeb_plan_tree(plan, _ptr(ch, ctypes.c_int32), _ptr(sl, ctypes.c_int32)))
    return [tuple(int(x) for x in p) for p in ch.reshape(-1, 2)], [int(x) for x in sl[: st["n_sliced"]]]


def xeb_plan_node(plan, node: int):
    kv = ctypes.c_int64()
    a, b, nl, ns = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().xeb_plan_node(plan, node, ctypes.byref(kv), ctypes.byref(a), ctypes.byref(b),
                                ctypes.byref(nl), ctypes.byref(ns)))
    return {"kv": kv.value, "a": a.value, "b": b.value, "n_legs": nl.value, "n_shared": ns.value}


def xeb_plan_device_bytes(plan) -> int:
    return int(load().xeb_plan_device_bytes(plan))


def xeb_plan_bind(plan, workspace_ptr: int, nbytes: int, stream: int):
    _check(load().xeb_plan_bind(plan, ctypes.c_void_p(workspace_ptr or None), nbytes, ctypes.c_void_p(stream or None)))


def xeb_set_bitstrings(plan, bits_dev_ptr: int, k: int, stream: int):
    _check(load().xeb_set_bitstrings(plan, ctypes.c_void_p(bits_dev_ptr), k, ctypes.c_void_p(stream or None)))


def xeb_amplitudes(plan, out_dev_ptr: int, stream: int):
    _check(load().xeb_amplitudes(plan, ctypes.c_void_p(out_dev_ptr or None), ctypes.c_void_p(stream or None)))


def xeb_plan_profile_ops(plan):
    """Per contraction: ms, launches, kernel class name, (M, N, K, kv)."""
    n = ctypes.c_int32()
    _check(load().xeb_plan_profile_ops(plan, 0, None, None, None, None, ctypes.byref(n)))
    cnt = n.value
    ms = np.zeros(cnt)
    la = np.zeros(cnt)
    cls = np.zeros(cnt, dtype=np.int32)
    shp = np.zeros((cnt, 4))
    _check(load().xeb_plan_profile_ops(plan, cnt, ms.ctypes.data_as(_dblp), la.ctypes.data_as(_dblp),
                                       cls.ctypes.data_as(_i32p), shp.ctypes.data_as(_dblp), ctypes.byref(n)))
    return [{"ms": float(ms[i]), "launches": int(la[i]),
             "kernel": KERNEL_CLASSES[cls[i]] if 0 <= cls[i] < len(KERNEL_CLASSES) else None,
             "M": int(shp[i, 0]), "N": int(shp[i, 1]), "K": int(shp[i, 2]), "kv": int(shp[i, 3])}
            for i in range(cnt)]


def xeb_plan_op_layout(plan, op_index: int):
    """Addressing of one program step: kind, node, A/B nodes and the address
    bit lists a_pos_m, a_pos_k, b_pos_k, b_pos_n, c_pos_m, c_pos_n."""
    n = ctypes.c_int32()
    _check(load().xeb_plan_op_layout(plan, op_index, None, 0, ctypes.byref(n)))
    v = np.zeros(n.value, dtype=np.int32)
    _check(load().xeb_plan_op_layout(plan, op_index, _ptr(v, ctypes.c_int32), n.value, ctypes.byref(n)))
    v = [int(x) for x in v]
    lens = v[4:10]
    out = {"kind": v[0], "node": v[1], "a_node": v[2], "b_node": v[3]}
    pos = 10
    for name, ln in zip(("a_pos_m", "a_pos_k", "b_pos_k", "b_pos_n", "c_pos_m", "c_pos_n"), lens):
        out[name] = v[pos:pos + ln]
        pos += ln
    return out


def xeb_plan_op_form(plan, op_index: int) -> dict:
    """Kernel form of one contraction step: class name, keyed rows per lane,
    streaming columns per thread and rows per tile, TMA loads."""
    v = np.zeros(5, dtype=np.int32)
    _check(load().xeb_plan_op_form(plan, op_index, _ptr(v, ctypes.c_int32)))
    return {"kernel": KERNEL_CLASSES[v[0]] if 0 <= v[0] < len(KERNEL_CLASSES) else None, "rows_per_lane": int(v[1]),
            "cols_per_thread": int(v[2]), "rows_per_tile": int(v[3]), "tma": int(v[4])}


def xeb_plan_buffers(plan):
    """Per node: arena element offset, size, cross-slice mask (numpy arrays)."""
    n = ctypes.c_int32()
    _check(load().xeb_plan_buffers(plan, None, None, None, ctypes.byref(n)))
    off = np.zeros(n.value, dtype=np.int64)
    el = np.zeros(n.value, dtype=np.int64)
    mk = np.zeros(n.value, dtype=np.uint32)
    _check(load().xeb_plan_buffers(plan, off.ctypes.data_as(ctypes.c_void_p), el.ctypes.data_as(ctypes.c_void_p),
                                   mk.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
    return off, el, mk


def xeb_plan_step_flops(plan):
    """(flops, contractions) one xeb_amplitudes step launches, with cross-slice reuse."""
    fl, nc = ctypes.c_double(), ctypes.c_double()
    _check(load().xeb_plan_step_flops(plan, ctypes.byref(fl), ctypes.byref(nc)))
    return fl.value, nc.value


def xeb_run_chunked(circuit, bitstrings, chunk: int, tree=None, slices=None, opts=None, stream: int = 0):
    """Streamed evaluation in Alg. 4's order, `chunk` bitstrings at a time;
    returns (amplitudes complex128 [k] in input order, F, mean 2^n p,
    mean (2^n p)^2)."""
    ca = CircuitArrays(circuit)
    bs = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    tp = sp = None
    if tree is not None:
        chl = np.ascontiguousarray(np.asarray(tree, dtype=np.int32).reshape(-1))
        t = xeb_tree(len(chl) // 2, _ptr(chl, ctypes.c_int32))
        tp = ctypes.byref(t)
    if slices is not None:
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.int32))
        s = xeb_slices(len(sl), _ptr(sl, ctypes.c_int32))
        sp = ctypes.byref(s)
    amps = np.zeros(2 * len(bs), dtype=np.float64)
    F, m1, m2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().xeb_run_chunked(ctypes.byref(ca.c), _ptr(bs, ctypes.c_uint64), len(bs), tp, sp,
                                  ctypes.byref(opts) if opts is not None else None, chunk,
                                  amps.ctypes.data_as(_dblp), ctypes.byref(F), ctypes.byref(m1), ctypes.byref(m2),
                                  ctypes.c_void_p(stream or None)))
    return amps.view(np.complex128), F.value, m1.value, m2.value


def xeb_set_slice_subset(plan, frac: float, seed: int) -> int:
    """Run only a seeded subset of the slice values (partial sums); returns its size."""
    n = ctypes.c_int64()
    _check(load().xeb_set_slice_subset(plan, float(frac), int(seed), ctypes.byref(n)))
    return n.value


def xeb_set_slice_block(plan, lo: int, hi: int, frac: float = 1.0, seed: int = 0) -> int:
    """Run positions lo .. hi-1 of the slice list (all values, or a seeded
    subset when frac < 1): partial sums for one rank's block; returns hi - lo."""
    n = ctypes.c_int64()
    _check(load().xeb_set_slice_block(plan, float(frac), int(seed), int(lo), int(hi), ctypes.byref(n)))
    return n.value


def xeb_plan_slice_ids(plan, n: int) -> np.ndarray:
    ids = np.zeros(n, dtype=np.int64)
    _check(load().xeb_plan_slice_ids(plan, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return ids


def xeb_fidelity(plan, stream: int):
    F, m1, m2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().xeb_fidelity(plan, ctypes.byref(F), ctypes.byref(m1), ctypes.byref(m2),
                               ctypes.c_void_p(stream or None)))
    return F.value, m1.value, m2.value


def xeb_run(plan, bits_host_ptr: int, k: int, amps_host_ptr: int, stream: int) -> float:
    F = ctypes.c_double()
    _check(load().xeb_run(plan, ctypes.c_void_p(bits_host_ptr), k, ctypes.c_void_p(amps_host_ptr or None),
                          ctypes.byref(F), ctypes.c_void_p(stream or None)))
    return F.value


def xeb_plan_keys(plan, node: int, k: int, kv: int, stream: int):
    key = np.empty(k, dtype=np.int32)
    uL = np.empty(max(kv, 1), dtype=np.int32)
    uR = np.empty(max(kv, 1), dtype=np.int32)
    _check(load().xeb_plan_keys(plan, node, _ptr(key, ctypes.c_int32), _ptr(uL, ctypes.c_int32),
                                _ptr(uR, ctypes.c_int32), ctypes.c_void_p(stream or None)))
    return key, uL[:kv], uR[:kv]


def xeb_plan_test_wait(plan, enable: bool):
    _check(load().xeb_plan_test_wait(plan, 1 if enable else 0))


def xeb_linear_xeb_noalloc(amps_dev_ptr: int, k: int, n_qubits: int, out_dev_ptr: int, stream: int):
    _check(load().xeb_linear_xeb_noalloc(ctypes.c_void_p(amps_dev_ptr), k, n_qubits,
                                         ctypes.c_void_p(out_dev_ptr), ctypes.c_void_p(stream or None)))


KERNEL_CLASSES = ["trie", "leaves", "permute", "gemm_tiled", "gemm_gemv", "gemm_tail", "gemm_generic",
                  "accum", "xeb", "gemm_tc", "gemm_stream", "gemm_memo", "gemm_kdeep", "gemm_tc_kdeep",
                  "gemm_keyed"]
XEB_N_KC = 16


XEB_N_FEATURES = 32


def xeb_plan_candidates(circuit, bitstrings, opts=None, max_cands: int = 256):
    """Planner candidates: list of dicts with tree [(l, r)...], slices, features, planner."""
    c = CircuitArrays(circuit)
    bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    o = opts or xeb_default_opts()
    n_leaves, _ = xeb_network_info(circuit)
    nn = n_leaves - 1
    trees = np.zeros((max_cands, nn, 2), dtype=np.int32)
    slices = np.full((max_cands, 30), -1, dtype=np.int32)
    nsl = np.zeros(max_cands, dtype=np.int32)
    feats = np.zeros((max_cands, XEB_N_FEATURES), dtype=np.float64)
    fam = np.zeros(max_cands, dtype=np.int32)
    n = ctypes.c_int32()
    _check(load().xeb_plan_candidates(ctypes.byref(c.c), bits.ctypes.data_as(ctypes.c_void_p), len(bits),
                                      ctypes.byref(o), max_cands, trees.ctypes.data_as(ctypes.c_void_p),
                                      slices.ctypes.data_as(ctypes.c_void_p), nsl.ctypes.data_as(ctypes.c_void_p),
                                      feats.ctypes.data_as(ctypes.c_void_p), fam.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(n)))
    out = []
    for i in range(n.value):
        out.append({"tree": [tuple(int(x) for x in pr) for pr in trees[i]],
                    "slices": [int(x) for x in slices[i, :nsl[i]]],
                    "features": feats[i].copy(), "planner": int(fam[i])})
    return out


class Mlp:
    """The learned cost model's network on the device (hand-written kernels)."""

    def __init__(self, n_in=XEB_N_FEATURES, n_hidden=128, n_layers=3, seed=0):
        h = ctypes.c_void_p()
        _check(load().xeb_mlp_create(n_in, n_hidden, n_layers, seed, ctypes.byref(h)))
        self.handle, self.n_in, self.n_hidden, self.n_layers = h.value, n_in, n_hidden, n_layers

    def close(self):
        if self.handle:
            load().xeb_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_params(self):
        return int(load().xeb_mlp_n_params(self.handle))

    def get_weights(self):
        w = np.zeros(self.n_params, dtype=np.float32)
        _check(load().xeb_mlp_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p), 0))
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.n_params
        _check(load().xeb_mlp_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p), 1))

    def set_norm(self, mean, scale):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        _check(load().xeb_mlp_set_norm(self.handle, m.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p)))

    def forward(self, x_dev_ptr, n, y_dev_ptr, stream):
        _check(load().xeb_mlp_forward(self.handle, x_dev_ptr, n, y_dev_ptr, stream))

    def gradients(self, x_dev_ptr, t_dev_ptr, n, stream):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(load().xeb_mlp_gradients(self.handle, x_dev_ptr, t_dev_ptr, n, g.ctypes.data_as(ctypes.c_void_p),
                                        loss.ctypes.data_as(ctypes.c_void_p), stream))
        return g, float(loss[0])

    def train_step(self, x_dev_ptr, t_dev_ptr, n, lr, loss_dev_ptr, stream):
        _check(load().xeb_mlp_train_step(self.handle, x_dev_ptr, t_dev_ptr, n, ctypes.c_float(lr), loss_dev_ptr, stream))


def xeb_plan_autotune(plan, reps: int, stream: int) -> int:
    n = ctypes.c_int32()
    _check(load().xeb_plan_autotune(plan, reps, stream, ctypes.byref(n)))
    return n.value


def xeb_plan_profile(plan, enable: bool):
    _check(load().xeb_plan_profile(plan, 1 if enable else 0))


def xeb_plan_profile_read(plan) -> dict:
    arrs = [np.zeros(XEB_N_KC) for _ in range(4)]
    _check(load().xeb_plan_profile_read(plan, *[_ptr(a, ctypes.c_double) for a in arrs]))
    out = {}
    for c, name in enumerate(KERNEL_CLASSES):
        if arrs[1][c] > 0:
            out[name] = {"ms": arrs[0][c], "launches": int(arrs[1][c]), "flops": arrs[2][c], "bytes": arrs[3][c]}
    return out


class Plan:
    """Owner of one xeb_plan handle plus the torch buffers it is bound to."""

    def __init__(self, circuit, bitstrings, tree=None, slices=None, opts=None, open_qubits=None):
        self.handle = xeb_plan_create(circuit, bitstrings, tree, slices, opts, open_qubits)
        self.k = len(bitstrings)
        self.n = circuit.n_qubits
        self.w = len(set(open_qubits)) if open_qubits is not None else 0   # 2^w amplitudes per bitstring
        self.workspace = None

    @classmethod
    def learned(cls, circuit, bitstrings, mlp, opts=None, max_cands: int = 256, stream: int = 0):
        """The plan of the candidate the cost model `mlp` predicts fastest
        (xeb_plan_create_learned); .predicted_log2_ms holds the prediction."""
        self = cls.__new__(cls)
        self.handle, self.predicted_log2_ms = xeb_plan_create_learned(circuit, bitstrings, mlp, opts, max_cands, stream)
        self.k = len(bitstrings)
        self.n = circuit.n_qubits
        self.w = 0
        self.workspace = None
        return self

    def stats(self):
        return xeb_plan_stats(self.handle)

    def tree(self):
        return xeb_plan_tree(self.handle)

    def bind(self, device="cuda"):
        import torch
        nbytes = xeb_plan_device_bytes(self.handle)
        dev = torch.device(device)
        total = torch.cuda.get_device_properties(dev.index if dev.index is not None else torch.cuda.current_device()).total_memory
        if nbytes + 256 > total:
            raise XebError(2, "plan needs %.3g GB of device memory, the device has %.3g GB"
                           % (nbytes / 1e9, total / 1e9))
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        ptr = self.workspace.data_ptr()
        ptr = (ptr + 255) // 256 * 256
        xeb_plan_bind(self.handle, ptr, nbytes, torch.cuda.current_stream().cuda_stream)
        return self

    def close(self):
        if self.handle is not None:
            xeb_plan_destroy(self.handle)
            self.handle = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
