"""Tensor networks of quantum circuits, written plainly in FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A circuit C becomes a tensor network N_C with n open legs, one per output
qubit (Sec. "Multi-batch simulator"); fixing the open legs to the bits of s
gives a network whose full contraction is <s|C|0^n>.  Gate fusion is assumed
to have been applied (same passage).  The fusion rule, the leaf numbering and
the leg numbering below form the interface convention shared with the
library's C ABI (the library implements it separately):

* one leaf per 2-qubit gate, numbered in time order;
* a 1-qubit gate on qubit q is fused into the output side (q's leg) of the
  latest 2-qubit gate on q before it; 1-qubit gates before the first 2-qubit
  gate on q act on |0> and that vector is contracted into the first 2-qubit
  gate's input for q (the input leg disappears);
* a qubit with no 2-qubit gate gets a rank-1 leaf (its 1-qubit gates applied
  to |0>), appended after the gate leaves in qubit order;
* bond legs are numbered in the order they are closed: when a 2-qubit gate on
  (qa, qb) is reached, first qa's incoming wire (if qa had an earlier 2-qubit
  gate), then qb's;
* the output leg of qubit q sits on the last leaf touching q; a leaf that
  carries two output legs lists them in the gate's qubit order (qa, qb).

Leaf tensors here have axes ``out_qubits + legs`` (output-bit axes first, in
listed order, then bond legs in ``legs`` order).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Leaf:
    out_qubits: List[int]
    legs: List[int]
    tensor: np.ndarray


@dataclasses.dataclass
class Network:
    n_qubits: int
    leaves: List[Leaf]
    n_legs: int

    def leg_dims(self):
        return {l: 2 for leaf in self.leaves for l in leaf.legs}


def _apply_on_axis(t: np.ndarray, m: np.ndarray, ax: int) -> np.ndarray:
    """t'[.., i, ..] = sum_j m[i, j] t[.., j, ..] on axis ax."""
    r = np.tensordot(m, t, axes=([1], [ax]))
    return np.moveaxis(r, 0, ax)


def fused_network(circuit) -> Network:
    n = circuit.n_qubits
    init = [np.array([1.0, 0.0], dtype=np.complex128) for _ in range(n)]
    last: List[Optional[int]] = [None] * n      # raw index of last 2q leaf on q
    raw = []                                    # {"T": ndarray, "labels": [...]}
    next_leg = 0
    for g in circuit.gates:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            if last[q] is None:
                init[q] = g.matrix @ init[q]
            else:
                rec = raw[last[q]]
                ax = rec["labels"].index(("out", q))
                rec["T"] = _apply_on_axis(rec["T"], g.matrix, ax)
            continue
        a, b = g.qubits
        t = g.matrix.reshape(2, 2, 2, 2)           # [out_a, out_b, in_a, in_b]
        labels = [("out", a), ("out", b), ("in", a), ("in", b)]
        for s in (a, b):
            if last[s] is None:
                ax = labels.index(("in", s))
                t = np.tensordot(t, init[s], axes=([ax], [0]))
                labels.pop(ax)
            else:
                prev = raw[last[s]]
                pa = prev["labels"].index(("out", s))
                prev["labels"][pa] = ("leg", next_leg)
                labels[labels.index(("in", s))] = ("leg", next_leg)
                next_leg += 1
        raw.append({"T": t, "labels": labels})
        last[a] = last[b] = len(raw) - 1
    for q in range(n):
        if last[q] is None:
            raw.append({"T": init[q].copy(), "labels": [("out", q)]})
        else:
            rec = raw[last[q]]
            rec["labels"][rec["labels"].index(("out", q))] = ("bit", q)
    leaves = []
    for rec in raw:
        labels = [("bit", l[1]) if l[0] == "out" else l for l in rec["labels"]]
        bit_axes = [i for i, l in enumerate(labels) if l[0] == "bit"]
        leg_axes = [i for i, l in enumerate(labels) if l[0] == "leg"]
        t = np.transpose(rec["T"], bit_axes + leg_axes).copy()
        leaves.append(Leaf([labels[i][1] for i in bit_axes],
                           [labels[i][1] for i in leg_axes], t))
    return Network(n, leaves, next_leg)


# --- the worked example of App. B --------------------------------------------

H_GATE = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2)
T_GATE = np.diag([1.0, np.exp(0.25j * np.pi)]).astype(np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]],
                dtype=np.complex128)


def worked_example_network() -> Network:
    """The 3-qubit network of App. B (Fig. "Example of multi-amplitude
    contraction"): leaves X0..X8 with the paper's numbering, bond legs 0..7,
    open legs 8, 9, 10 = output qubits 0, 1, 2.

    X0, X1, X2 = |0> on q0, q1, q2; X3 = H on q0 (in 0, out 3);
    X4 = T on q2 (in 2, out 6); X5 = CNOT q0->q1 (in 3, 1; out 4, 5);
    X6 = CNOT q1->q2 (in 5, 6; out 7 and open leg 10);
    X7 = H on q0 (in 4, open leg 8); X8 = H on q1 (in 7, open leg 9).
    """
    ket0 = np.array([1.0, 0.0], dtype=np.complex128)
    cx = CNOT.reshape(2, 2, 2, 2)             # [o_ctrl, o_tgt, i_ctrl, i_tgt]
    leaves = [
        Leaf([], [0], ket0.copy()),                       # X0
        Leaf([], [1], ket0.copy()),                       # X1
        Leaf([], [2], ket0.copy()),                       # X2
        Leaf([], [3, 0], H_GATE.copy()),                  # X3 [out, in]
        Leaf([], [6, 2], T_GATE.copy()),                  # X4
        Leaf([], [4, 5, 3, 1], cx.copy()),                # X5
        Leaf([2], [7, 5, 6], np.transpose(cx, (1, 0, 2, 3)).copy()),  # X6
        Leaf([0], [4], H_GATE.copy()),                    # X7 [bit, in]
        Leaf([1], [7], H_GATE.copy()),                    # X8
    ]
    return Network(3, leaves, 8)


#: The contraction tree of App. B, (((X0*X3)*(X1*X5))*((X2*X4)*(X6*X8)))*X7,
#: in the children format used throughout (post-order; leaf j = -1-j).
WORKED_EXAMPLE_TREE = [(-1, -4), (-2, -6), (0, 1), (-3, -5), (-7, -9), (3, 4),
                       (2, 5), (6, -8)]


def project_leaf(leaf: Leaf, word: int, sliced: Optional[Dict[int, int]] = None):
    """Fix the leaf's output legs to the bits of ``word`` (bit q = qubit q) and
    its sliced legs to the given values; returns (tensor, remaining legs)."""
    t = leaf.tensor
    for q in leaf.out_qubits:
        t = t[(word >> q) & 1]
    legs = list(leaf.legs)
    if sliced:
        for leg, val in sliced.items():
            if leg in legs:
                ax = legs.index(leg)
                t = np.take(t, val, axis=ax)
                legs.pop(ax)
    return np.asarray(t), legs


def pair_contract(a: np.ndarray, la: Sequence[int], b: np.ndarray,
                  lb: Sequence[int]):
    """T*S of Eq. (elem-cont): sum over the legs the two tensors share.
    Result legs: a's unshared legs, then b's unshared legs."""
    shared = [l for l in la if l in set(lb)]
    out = [l for l in la if l not in shared] + [l for l in lb if l not in shared]
    # the sum over the shared legs as one matrix product (library tensordot)
    r = np.tensordot(a, b, axes=([list(la).index(l) for l in shared],
                                 [list(lb).index(l) for l in shared]))
    return r, out
