"""The worked example of App. B pins the memoization semantics: evaluation
counts per subtree and the amplitudes (closed form of the circuit)."""
import math
import os

import numpy as np

from paper_2108_05665_gb300 import inputs
from oracle import contract, memo, network, statevec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split("=", 1)
            vals[key.strip()] = val.strip()
    return vals


def _tree(g):
    return [tuple(int(x) for x in p.strip("()").split(",")) for p in g["tree"].split()]


def test_golden_tree_is_the_papers():
    g = _golden()
    assert _tree(g) == network.WORKED_EXAMPLE_TREE


def test_worked_example_counts():
    g = _golden()
    net = network.worked_example_network()
    tree = _tree(g)
    bs = np.array([int(x) for x in g["bitstrings"].split()], dtype=np.uint64)
    _, c12 = memo.alg12(net, tree, bs)
    _, c34 = memo.alg34(net, tree, bs)
    kt = memo.key_tables(net, tree, bs)
    for counts in (c12, c34, kt["k"]):
        assert counts[2] == int(g["count (X0*X3)*(X1*X5)"])
        assert counts[5] == int(g["count (X2*X4)*(X6*X8)"])
        assert counts[7] == int(g["count root"])
    assert kt["k"][-8] == int(g["values X7"])
    # a single-amplitude simulator would contract every subtree 3 times
    assert sum(c12.values()) < 3 * len(tree)


def test_worked_example_amplitudes():
    g = _golden()
    net = network.worked_example_network()
    tree = _tree(g)
    bs = np.array([int(x) for x in g["bitstrings"].split()], dtype=np.uint64)
    want = np.array([float(g["amplitude %d" % int(b)]) for b in bs])
    a12, _ = memo.alg12(net, tree, bs)
    r34, _ = memo.alg34(net, tree, bs)
    a34 = np.array([r34[int(b)] for b in bs])
    aN = contract.amplitudes(net, bs)
    for a in (a12, a34, aN):
        assert np.abs(a - want).max() < 1e-15
    # all 8 amplitudes against the closed form, and the same circuit run
    # through the state vector
    allb = np.arange(8, dtype=np.uint64)
    a_all, _ = memo.alg12(net, tree, allb)
    closed = np.array([(1 if (b >> 2) & 1 == 0 else (-1) ** (((b >> 0) & 1) + ((b >> 1) & 1)))
                       / (2 * math.sqrt(2)) for b in range(8)])
    assert np.abs(a_all - closed).max() < 1e-15
    gates = [inputs.Gate(1, (0,), network.H_GATE), inputs.Gate(1, (2,), network.T_GATE),
             inputs.Gate(2, (0, 1), network.CNOT), inputs.Gate(2, (1, 2), network.CNOT),
             inputs.Gate(1, (0,), network.H_GATE), inputs.Gate(1, (1,), network.H_GATE)]
    psi = statevec.state(inputs.Circuit(3, gates))
    assert np.abs(psi - closed).max() < 1e-15
