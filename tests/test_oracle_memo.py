"""Pins of the memoization oracle: key tables against brute-force distinct
counts, Alg. 1/2 and Alg. 3/4 evaluation counts, amplitudes against the state
vector, the cost counters against counted multiplications, slicing
invariance."""
import itertools

import numpy as np
import pytest

from paper_2108_05665_gb300 import inputs
from oracle import contract, memo, network, statevec
from _trees import random_tree


@pytest.fixture(scope="module")
def small():
    c = inputs.random_grid_circuit(2, 3, 6, 21)
    net = network.fused_network(c)
    psi = statevec.state(c)
    return c, net, psi


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_key_tables_brute_force(small, seed):
    c, net, _ = small
    tree = random_tree([l.legs for l in net.leaves], seed)
    memo.check_tree(tree, len(net.leaves))
    bs = inputs.uniform_bitstrings(c.n_qubits, 40, 100 + seed)
    kt = memo.key_tables(net, tree, bs)
    # pi is a permutation of the qubits
    assert sorted(kt["pi"]) == list(range(c.n_qubits))
    for i in range(len(tree)):
        leaves = memo.inorder_leaves(tree, i)
        qs = [q for j in leaves for q in net.leaves[j].out_qubits]
        proj = [tuple((int(w) >> q) & 1 for q in qs) for w in bs]
        distinct = sorted(set(proj))
        assert kt["k"][i] == len(distinct)
        # key ids are ranks in lexicographic order of the pi-ordered bits
        ids = [distinct.index(p) for p in proj]
        assert list(kt["key"][i]) == ids
        # children ids reproduce each key's bits
        l, r = tree[i]
        for u in range(kt["k"][i]):
            lv = kt["unique"][l][kt["uL"][i][u]]
            rv = kt["unique"][r][kt["uR"][i][u]]
            wr = kt["range"][r][1] - kt["range"][r][0]
            assert (int(lv) << wr) | int(rv) == int(kt["unique"][i][u])


@pytest.mark.parametrize("seed", [3, 4])
def test_alg12_alg34_counts_and_amplitudes(small, seed):
    c, net, psi = small
    tree = random_tree([l.legs for l in net.leaves], seed)
    bs = inputs.uniform_bitstrings(c.n_qubits, 30, 200 + seed)
    bs = np.concatenate([bs, bs[:5]])          # duplicates are kept in order
    want = statevec.gather(psi, bs)
    a12, c12 = memo.alg12(net, tree, bs)
    assert np.abs(a12 - want).max() < 1e-13
    r34, c34 = memo.alg34(net, tree, bs)
    assert np.abs(np.array([r34[int(b)] for b in bs]) - want).max() < 1e-13
    kt = memo.key_tables(net, tree, bs)
    for i in range(len(tree)):
        assert c12.get(i, 0) == kt["k"][i]
        assert c34.get(i, 0) == kt["k"][i]


def test_bound_counts_dominate_exact(small):
    c, net, _ = small
    tree = random_tree([l.legs for l in net.leaves], 9)
    bs = inputs.uniform_bitstrings(c.n_qubits, 25, 300)
    kt = memo.key_tables(net, tree, bs)
    kb = memo.bound_counts(net, tree, len(bs), {j: kt["k"][j] for j in kt["k"] if j < 0})
    for i in range(len(tree)):
        assert kt["k"][i] <= kb[i] <= len(bs)
        # 2^min(r, m) rule: at most 2^(bits the subtree depends on)
        a, b = kt["range"][i]
        assert kt["k"][i] <= 2 ** (b - a)


def test_cost_counters_match_counted_work(small, monkeypatch):
    c, net, _ = small
    tree = random_tree([l.legs for l in net.leaves], 5)
    bs = inputs.uniform_bitstrings(c.n_qubits, 30, 400)
    counted = {"mul": 0, "rw": 0}
    orig = memo.pair_contract

    def counting(a, la, b, lb):
        r, out = orig(a, la, b, lb)
        shared = set(la) & set(lb)
        counted["mul"] += r.size * (2 ** len(shared))
        counted["rw"] += a.size + b.size + r.size
        return r, out

    monkeypatch.setattr(memo, "pair_contract", counting)
    memo.alg12(net, tree, bs)
    kt = memo.key_tables(net, tree, bs)
    cc, rw = memo.costs(net, tree, kt["k"])
    assert cc == counted["mul"]
    assert rw == counted["rw"]


def test_slicing_invariance(small):
    c, net, psi = small
    bs = inputs.uniform_bitstrings(c.n_qubits, 12, 500)
    want = statevec.gather(psi, bs)
    sliced = [0, 3, 5]
    assert np.abs(contract.amplitudes(net, bs, sliced=sliced) - want).max() < 1e-13
    tree = random_tree([l.legs for l in net.leaves], 6, sliced=sliced)
    acc = np.zeros(len(bs), dtype=np.complex128)
    for vals in itertools.product([0, 1], repeat=len(sliced)):
        a, _ = memo.alg12(net, tree, bs, sliced=dict(zip(sliced, vals)))
        acc += a
    assert np.abs(acc - want).max() < 1e-13
