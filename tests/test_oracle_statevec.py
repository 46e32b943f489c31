"""Pins of the FP64 state-vector oracle: brute force, norm, unitarity and
Porter-Thomas statistics."""
import math

import numpy as np
import pytest

from paper_2108_05665_gb300 import inputs
from oracle import brute, statevec


@pytest.mark.parametrize("rows,cols,cycles,seed", [(2, 2, 5, 11), (2, 3, 8, 12),
                                                   (1, 5, 6, 13), (3, 2, 7, 14)])
def test_statevec_matches_brute_force(rows, cols, cycles, seed):
    c = inputs.random_grid_circuit(rows, cols, cycles, seed)
    a = statevec.state(c)
    b = brute.state(c)
    assert np.abs(a - b).max() < 1e-12


def test_two_qubit_gate_orientation_and_distance():
    # a non-symmetric 2q gate on far-apart qubits in both orders pins the
    # |b_a b_b> basis convention and the bit-insertion arithmetic
    rng = np.random.default_rng(5)
    z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    q, _ = np.linalg.qr(z)
    gates = [inputs.Gate(1, (i,), inputs.SQRT_W) for i in range(5)]
    gates += [inputs.Gate(2, (4, 1), q), inputs.Gate(2, (0, 3), q.T.copy()),
              inputs.Gate(1, (2,), inputs.SQRT_X), inputs.Gate(2, (2, 0), q)]
    c = inputs.Circuit(5, gates)
    assert np.abs(statevec.state(c) - brute.state(c)).max() < 1e-12


def test_gates_are_unitary():
    for m in (inputs.SQRT_X, inputs.SQRT_Y, inputs.SQRT_W):
        assert np.abs(m.conj().T @ m - np.eye(2)).max() < 1e-14
    assert np.abs(inputs.FSIM.conj().T @ inputs.FSIM - np.eye(4)).max() < 1e-14
    # sqrt gates square to the Pauli rotations by pi: X, Y, W up to phase -i
    x = np.array([[0, 1], [1, 0]])
    y = np.array([[0, -1j], [1j, 0]])
    w = (x + y) / math.sqrt(2)
    for s, p in ((inputs.SQRT_X, x), (inputs.SQRT_Y, y), (inputs.SQRT_W, w)):
        assert np.abs(s @ s - (-1j) * p).max() < 1e-14


def test_norm_is_one():
    c = inputs.random_grid_circuit(3, 4, 8, 1001)
    psi = statevec.state(c)
    s2, _ = statevec.moments(psi)
    assert abs(s2 - 1.0) < 1e-12


def test_porter_thomas_collision_probability():
    # deep random circuits: 2^n sum p^2 -> 2 (Porter-Thomas)
    c = inputs.random_grid_circuit(4, 5, 14, 77)
    psi = statevec.state(c)
    s2, s4 = statevec.moments(psi)
    assert abs(s2 - 1) < 1e-12
    assert abs((2 ** 20) * s4 - 2.0) < 0.06


def test_circuit_structure():
    c = inputs.random_grid_circuit(5, 6, 14, 1002)
    two = [g for g in c.gates if g.kind == 2]
    # A,B,C,D coupler counts on 5x6: 15, 12, 10, 12; cycles ABCDABCDABCDAB
    assert len(two) == 4 * 15 + 4 * 12 + 3 * 10 + 3 * 12
    one = [g for g in c.gates if g.kind == 1]
    assert len(one) == 30 * 15
    # no single-qubit gate repeats on a qubit in consecutive layers
    last = {}
    for g in one:
        q = g.qubits[0]
        assert last.get(q) != g.name
        last[q] = g.name
    missing = inputs.random_grid_circuit(6, 9, 2, 5, missing=((0, 0),))
    assert missing.n_qubits == 53
