"""Python front-end of the FP64 state-vector oracle (``statevec.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The amplitude of bitstring s is <s|C|0^n> (Sec. "Multi-batch simulator"),
computed here by applying the gates of C one by one to |0^n> in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_statevec.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile statevec.c with gcc -O2 -fopenmp into oracle/_build/."""
    src = os.path.join(_HERE, "statevec.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                           "-std=c99", src, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            up = ctypes.POINTER(ctypes.c_uint64)
            lib.sv_run_circuit.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, dp]
            lib.sv_run_circuit.restype = None
            lib.sv_gather.argtypes = [dp, ctypes.c_size_t, up, dp]
            lib.sv_moments.argtypes = [dp, ctypes.c_int, dp, dp]
            lib.sv_sample_sorted.argtypes = [dp, ctypes.c_int, ctypes.c_size_t, dp, up]
            lib.sv_apply_1q.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.sv_apply_2q.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def state(circuit) -> np.ndarray:
    """Full FP64 state C|0^n> as complex128[2^n] (index bit q = qubit q)."""
    lib = _load()
    kinds, q0, q1, mats = circuit.as_arrays()
    n = circuit.n_qubits
    psi = np.empty(1 << n, dtype=np.complex128)
    mats = np.ascontiguousarray(mats)
    lib.sv_run_circuit(_ptr(psi.view(np.float64), ctypes.c_double), n, len(kinds),
                       _ptr(kinds, ctypes.c_int32), _ptr(q0, ctypes.c_int32),
                       _ptr(q1, ctypes.c_int32),
                       _ptr(mats.view(np.float64), ctypes.c_double))
    return psi


def gather(psi: np.ndarray, bitstrings: np.ndarray) -> np.ndarray:
    """Amplitudes psi[s_i] for uint64 bitstrings, in input order."""
    lib = _load()
    x = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    out = np.empty(len(x), dtype=np.complex128)
    lib.sv_gather(_ptr(psi.view(np.float64), ctypes.c_double), len(x),
                  _ptr(x, ctypes.c_uint64), _ptr(out.view(np.float64), ctypes.c_double))
    return out


def amplitudes(circuit, bitstrings: np.ndarray) -> np.ndarray:
    """<s_i|C|0^n> in FP64 for every bitstring (input order, duplicates kept)."""
    return gather(state(circuit), bitstrings)


def moments(psi: np.ndarray):
    """(sum |psi|^2, sum |psi|^4)."""
    lib = _load()
    n = int(np.log2(len(psi)))
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib.sv_moments(_ptr(psi.view(np.float64), ctypes.c_double), n,
                   ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def sample_ideal(psi: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Bitstrings x ~ |psi_x|^2 by inverse CDF, one per uniform draw u_j in
    [0, 1) (draws supplied by the caller; output in the order of u)."""
    lib = _load()
    n = int(np.log2(len(psi)))
    order = np.argsort(u, kind="stable")
    us = np.ascontiguousarray(u[order], dtype=np.float64)
    out_sorted = np.empty(len(u), dtype=np.uint64)
    lib.sv_sample_sorted(_ptr(psi.view(np.float64), ctypes.c_double), n, len(u),
                         _ptr(us, ctypes.c_double), _ptr(out_sorted, ctypes.c_uint64))
    out = np.empty_like(out_sorted)
    out[order] = out_sorted
    return out
