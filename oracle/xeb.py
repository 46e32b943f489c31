"""Linear cross-entropy benchmark, Eq. (1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

F_XEB = 2^n / k * sum_{i=1..k} p_C(s_i) - 1 with p_C(s) = |<s|C|0^n>|^2, summed
over the sequence of bitstrings (duplicates count every time they occur).
"""
from __future__ import annotations

import numpy as np


def fidelity(amplitudes: np.ndarray, n_qubits: int) -> float:
    p = np.abs(np.asarray(amplitudes, dtype=np.complex128)) ** 2
    return float(2.0 ** n_qubits * p.sum() / len(p) - 1.0)


def moments(amplitudes: np.ndarray, n_qubits: int):
    """(mean of 2^n p, mean of (2^n p)^2) over the sequence."""
    p = np.abs(np.asarray(amplitudes, dtype=np.complex128)) ** 2 * 2.0 ** n_qubits
    return float(p.mean()), float((p * p).mean())
