"""Seeded synthetic inputs: random 2D-grid circuits and bitstring sets.

This module only *creates inputs*.  It holds none of the arithmetic of the
multi-amplitude contraction (no contraction, no amplitudes, no XEB); both the
CUDA path and the FP64 oracle consume what it produces.

Circuit family (a synthetic stand-in for the random grid circuits whose linear
XEB the paper verifies, Sec. "Verification of Google's experiment"; the paper
does not print the gate set, so the textbook forms below are used):

* qubits on an R x C grid, numbered row-major (qubit ``r*C + c``), optionally
  with some grid sites missing (then renumbered row-major over what is left);
* ``cycles`` cycles, each = one layer of single-qubit gates on every qubit
  (uniform over {sqrt(X), sqrt(Y), sqrt(W)} in cycle 0, afterwards uniform over
  the two gates that differ from the previous one on that qubit), then one
  layer of fSim(pi/2, pi/6) on the couplers of pattern A, B, C, D (cyclic):
  A = horizontal pairs with even left column, B = vertical pairs with even top
  row, C = horizontal pairs with odd left column, D = vertical pairs with odd
  top row;
* a final single-qubit layer (same no-repeat rule) before measurement.

Gate matrix conventions: a 1-qubit gate is a 2x2 matrix acting as
``out = M @ in``; a 2-qubit gate on (qa, qb) is a 4x4 matrix in the basis
``|b_a b_b>`` with qa's bit as the high bit (index ``2*b_a + b_b``).

Bitstring convention: bit ``q`` of a uint64 word is qubit ``q``'s measured
value (so ``n <= 64``).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

S2 = 1.0 / math.sqrt(2.0)

#: sqrt(X) = R_X(pi/2)
SQRT_X = np.array([[S2, -1j * S2], [-1j * S2, S2]], dtype=np.complex128)
#: sqrt(Y) = R_Y(pi/2)
SQRT_Y = np.array([[S2, -S2], [S2, S2]], dtype=np.complex128)
#: sqrt(W) = R_W(pi/2) with W = (X + Y)/sqrt(2)
SQRT_W = np.array([[S2, S2 * np.exp(-0.75j * np.pi)],
                   [S2 * np.exp(-0.25j * np.pi), S2]], dtype=np.complex128)

ONE_QUBIT_GATES = (("sqrtX", SQRT_X), ("sqrtY", SQRT_Y), ("sqrtW", SQRT_W))

GATE_1Q = 1
GATE_2Q = 2


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) in the |b_a b_b> basis (qa high bit)."""
    c, s = math.cos(theta), math.sin(theta)
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = 1.0
    m[1, 1] = c
    m[1, 2] = -1j * s
    m[2, 1] = -1j * s
    m[2, 2] = c
    m[3, 3] = np.exp(-1j * phi)
    return m


FSIM = fsim(math.pi / 2, math.pi / 6)


@dataclasses.dataclass
class Gate:
    kind: int                 # GATE_1Q or GATE_2Q
    qubits: Tuple[int, ...]   # (q,) or (qa, qb)
    matrix: np.ndarray        # (2,2) or (4,4) complex128
    name: str = ""


@dataclasses.dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    rows: int = 0
    cols: int = 0

    def as_arrays(self):
        """Flat arrays for the C ABI: kinds[int32], q0[int32], q1[int32],
        mats[complex128, (n_gates, 4, 4)] (a 1q gate uses the top-left 2x2)."""
        g = len(self.gates)
        kinds = np.zeros(g, dtype=np.int32)
        q0 = np.zeros(g, dtype=np.int32)
        q1 = np.full(g, -1, dtype=np.int32)
        mats = np.zeros((g, 4, 4), dtype=np.complex128)
        for i, gate in enumerate(self.gates):
            kinds[i] = gate.kind
            q0[i] = gate.qubits[0]
            if gate.kind == GATE_2Q:
                q1[i] = gate.qubits[1]
                mats[i] = gate.matrix
            else:
                mats[i, :2, :2] = gate.matrix
        return kinds, q0, q1, mats


def grid_sites(rows: int, cols: int, missing: Sequence[Tuple[int, int]] = ()):
    """Row-major numbering of the present grid sites -> dict (r, c) -> qubit."""
    miss = set(missing)
    index = {}
    for r in range(rows):
        for c in range(cols):
            if (r, c) not in miss:
                index[(r, c)] = len(index)
    return index


def coupler_pattern(rows: int, cols: int, index, pattern: str):
    """Couplers of pattern A/B/C/D as (qa, qb) pairs with qa < qb."""
    pairs = []
    for r in range(rows):
        for c in range(cols):
            if pattern in "AC":
                if (c % 2 == 0) != (pattern == "A"):
                    continue
                other = (r, c + 1)
            else:
                if (r % 2 == 0) != (pattern == "B"):
                    continue
                other = (r + 1, c)
            if (r, c) in index and other in index:
                pairs.append((index[(r, c)], index[other]))
    return pairs


def random_grid_circuit(rows: int, cols: int, cycles: int, seed: int,
                        missing: Sequence[Tuple[int, int]] = (),
                        final_layer: bool = True) -> Circuit:
    """Seeded random grid circuit of the family described in the module doc."""
    rng = np.random.Generator(np.random.PCG64(seed))
    index = grid_sites(rows, cols, missing)
    n = len(index)
    gates: List[Gate] = []
    prev = [-1] * n

    def one_qubit_layer():
        for q in range(n):
            if prev[q] < 0:
                choice = int(rng.integers(0, 3))
            else:
                others = [g for g in range(3) if g != prev[q]]
                choice = others[int(rng.integers(0, 2))]
            prev[q] = choice
            name, mat = ONE_QUBIT_GATES[choice]
            gates.append(Gate(GATE_1Q, (q,), mat.copy(), name))

    for cyc in range(cycles):
        one_qubit_layer()
        for qa, qb in coupler_pattern(rows, cols, index, "ABCD"[cyc % 4]):
            gates.append(Gate(GATE_2Q, (qa, qb), FSIM.copy(), "fSim"))
    if final_layer:
        one_qubit_layer()
    return Circuit(n, gates, rows, cols)


def uniform_bitstrings(n: int, k: int, seed: int) -> np.ndarray:
    """k bitstrings uniform over {0,1}^n as uint64 words (bit q = qubit q)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    words = rng.integers(0, np.iinfo(np.uint64).max, size=k, dtype=np.uint64,
                         endpoint=True)
    if n < 64:
        words &= np.uint64((1 << n) - 1)
    return words


def uniform_unit_draws(k: int, seed: int) -> np.ndarray:
    """k doubles uniform in [0, 1): the random numbers an inverse-CDF sampler
    of the ideal output distribution consumes (the sampler itself lives with
    whoever owns the distribution)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random(k)


# --- named workloads -------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    rows: int
    cols: int
    cycles: int
    k: int
    circuit_seed: int
    bitstring_seed: int
    ideal_fraction: float = 0.0   # share of bitstrings drawn from |psi|^2
    ideal_seed: int = 0
    missing: Tuple[Tuple[int, int], ...] = ()
    trie_depth: int = 0

    def circuit(self) -> Circuit:
        return random_grid_circuit(self.rows, self.cols, self.cycles,
                                   self.circuit_seed, self.missing)

    @property
    def n_qubits(self) -> int:
        return self.rows * self.cols - len(self.missing)


WORKLOADS = {
    # 3x4 grid, 8 cycles, 1,000 uniform bitstrings, no slicing.
    "grid3x4_m8_k1000": Workload("grid3x4_m8_k1000", 3, 4, 8, 1000, 1001, 2001),
    # 5x6 grid, 14 cycles, 10,000 bitstrings: half ideal samples, half uniform;
    # memo trie over the first 10 output bits.
    "grid5x6_m14_k10000": Workload("grid5x6_m14_k10000", 5, 6, 14, 10000, 1002,
                                   2002, ideal_fraction=0.5, ideal_seed=3002,
                                   trie_depth=10),
    # 5x5 grid, 12 cycles, 2,000 uniform bitstrings: small profiling case
    # (256 MB state, larger than L2).
    "grid5x5_m12_k2000": Workload("grid5x5_m12_k2000", 5, 5, 12, 2000, 1004, 2004),
    # 3x9 grid, 12 cycles, 2,000 uniform bitstrings: profiling case whose body
    # contractions have K = N = 64 like the benchmark's (1 GB state).
    "grid3x9_m12_k2000": Workload("grid3x9_m12_k2000", 3, 9, 12, 2000, 1005, 2005),
    # 5x8 grid, 12 cycles, 100,000 uniform bitstrings (sliced).
    "grid5x8_m12_k100000": Workload("grid5x8_m12_k100000", 5, 8, 12, 100000,
                                    1003, 2003),
    # 6x9 grid without its (0, 0) corner (53 qubits), 12 cycles, 300,000
    # uniform bitstrings (sliced; timed on a seeded subset of the slices).
    "grid6x9m1_m12_k300000": Workload("grid6x9m1_m12_k300000", 6, 9, 12, 300000,
                                      1004, 2004, missing=((0, 0),)),
    # the same grid, 14 cycles, 1,000,000 uniform bitstrings.
    "grid6x9m1_m14_k1000000": Workload("grid6x9m1_m14_k1000000", 6, 9, 14, 1000000,
                                       1005, 2005, missing=((0, 0),)),
}
