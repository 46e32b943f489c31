"""Brute-force circuit unitary for n <= 6 qubits.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Builds the full 2^n x 2^n operator of every gate independently of the
state-vector code (Kronecker products for 1-qubit gates, element-wise
definition for 2-qubit gates), multiplies them in time order and applies the
result to e_0, giving <x|C|0^n> for every x (Sec. "Multi-batch simulator").
"""
from __future__ import annotations

import numpy as np


def one_qubit_operator(n: int, q: int, m: np.ndarray) -> np.ndarray:
    # basis index x has bit q = qubit q, so qubit n-1 is the leftmost Kronecker
    # factor and qubit 0 the rightmost
    op = np.ones((1, 1), dtype=np.complex128)
    for j in range(n - 1, -1, -1):
        op = np.kron(op, m if j == q else np.eye(2))
    return op


def two_qubit_operator(n: int, qa: int, qb: int, m: np.ndarray) -> np.ndarray:
    dim = 1 << n
    op = np.zeros((dim, dim), dtype=np.complex128)
    others = ~((1 << qa) | (1 << qb))
    for xo in range(dim):
        for xi in range(dim):
            if (xo & others) != (xi & others):
                continue
            r = 2 * ((xo >> qa) & 1) + ((xo >> qb) & 1)
            c = 2 * ((xi >> qa) & 1) + ((xi >> qb) & 1)
            op[xo, xi] = m[r, c]
    return op


def circuit_unitary(circuit) -> np.ndarray:
    n = circuit.n_qubits
    u = np.eye(1 << n, dtype=np.complex128)
    for g in circuit.gates:
        if len(g.qubits) == 1:
            op = one_qubit_operator(n, g.qubits[0], g.matrix)
        else:
            op = two_qubit_operator(n, g.qubits[0], g.qubits[1], g.matrix)
        u = op @ u
    return u


def state(circuit) -> np.ndarray:
    """C|0^n> as the first column of the brute-force unitary."""
    return circuit_unitary(circuit)[:, 0].copy()
