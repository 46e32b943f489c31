"""Host-side checks of the C ABI (no GPU): the library loads and exports
every declared entry point, the tensor-network convention matches the
oracle's, the planner's exact evaluation counts and cost counters agree with
the oracle, and invalid input is rejected."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2108_05665_gb300 import build, binding as B, inputs
from oracle import memo, network
from _trees import random_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return B.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(xeb_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert "xeb_plan_create" in names and len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_network_convention_matches_oracle():
    for seed, (r, c, m) in enumerate([(3, 4, 8), (2, 3, 5), (5, 6, 3)]):
        circ = inputs.random_grid_circuit(r, c, m, 70 + seed)
        outs, legs = B.xeb_network_leaves(circ)
        net = network.fused_network(circ)
        assert outs == [l.out_qubits for l in net.leaves]
        assert [sorted(x) for x in legs] == [sorted(l.legs) for l in net.leaves]
        assert B.xeb_network_info(circ) == (len(net.leaves), net.n_legs)


@pytest.mark.parametrize("planner", [B.XEB_PLANNER_GREEDY, B.XEB_PLANNER_SWEEP, None])
def test_plan_counts_and_costs_match_oracle(planner):
    w = inputs.WORKLOADS["grid3x4_m8_k1000"]
    circ = w.circuit()
    bs = inputs.uniform_bitstrings(circ.n_qubits, w.k, w.bitstring_seed)
    net = network.fused_network(circ)
    if planner is None:
        tree = random_tree([l.legs for l in net.leaves], 3)
        p = B.xeb_plan_create(circ, bs, tree=tree)
    else:
        o = B.xeb_default_opts()
        o.planner = planner
        p = B.xeb_plan_create(circ, bs, opts=o)
    try:
        tree, sliced = B.xeb_plan_tree(p)
        memo.check_tree(tree, len(net.leaves))
        kt = memo.key_tables(net, tree, bs)
        for i in range(len(tree)):
            info = B.xeb_plan_node(p, i)
            assert info["kv"] == kt["k"][i]
            assert (info["a"], info["b"]) == kt["range"][i]
        st = B.xeb_plan_stats(p)
        c, rw = memo.costs(net, tree, kt["k"], sliced)
        assert st["flops_per_slice"] == 8 * c
        assert st["rw_elems_per_slice"] == rw
        assert st["k_distinct"] == len(np.unique(bs))
        assert st["single_amp_flops"] >= st["flops_per_slice"]
    finally:
        B.xeb_plan_destroy(p)


def test_slicing_planner_respects_budget():
    w = inputs.WORKLOADS["grid3x4_m8_k1000"]
    circ = w.circuit()
    bs = inputs.uniform_bitstrings(circ.n_qubits, 4, 5)
    p0 = B.xeb_plan_create(circ, bs)
    full = B.xeb_plan_stats(p0)
    B.xeb_plan_destroy(p0)
    o = B.xeb_default_opts()
    o.mem_budget = full["arena_bytes"] * 3 // 4
    p = B.xeb_plan_create(circ, bs, opts=o)
    try:
        st = B.xeb_plan_stats(p)
        # slicing trades memory for work (App. A, "Slicing")
        assert st["n_sliced"] >= 1
        assert st["n_slices"] == 2 ** st["n_sliced"]
        assert st["arena_bytes"] < full["arena_bytes"]
        assert st["flops_per_slice"] * st["n_slices"] >= full["flops_per_slice"]
    finally:
        B.xeb_plan_destroy(p)


def test_invalid_inputs_rejected():
    circ = inputs.random_grid_circuit(2, 3, 4, 9)
    bs = inputs.uniform_bitstrings(6, 10, 1)
    net = network.fused_network(circ)
    L = len(net.leaves)
    bad = [(-1, -2)] * (L - 1)          # leaf used twice
    with pytest.raises(B.XebError) as e:
        B.xeb_plan_create(circ, bs, tree=bad)
    assert e.value.status == 1
    with pytest.raises(B.XebError):
        B.xeb_plan_create(circ, bs, tree=[(-1, -2)])   # wrong node count
    with pytest.raises(B.XebError):
        B.xeb_plan_create(circ, np.array([1 << 7], dtype=np.uint64))  # bit above n
    with pytest.raises(B.XebError):
        B.xeb_plan_create(circ, bs, slices=[10 ** 6])
    bad_c = inputs.Circuit(6, [inputs.Gate(2, (0, 0), inputs.FSIM)])
    with pytest.raises(B.XebError):
        B.xeb_network_info(bad_c)
