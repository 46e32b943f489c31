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


@pytest.mark.parametrize("planner", [B.XEB_PLANNER_GREEDY, B.XEB_PLANNER_SWEEP, B.XEB_PLANNER_ANNEAL, None])
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


def test_anneal_fits_budget_and_keeps_exact_counts():
    """The local search of App. A under a budget 1/16 of the unsliced arena:
    the plan fits, slices some legs, its counts and costs still agree with
    the oracle's memo semantics, and AUTO (which runs the search when slicing
    is needed and keeps it only if better) is never worse than either
    constructed family alone."""
    circ = inputs.random_grid_circuit(4, 5, 12, 4242)
    bs = inputs.uniform_bitstrings(20, 700, 4343)
    net = network.fused_network(circ)
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    p0 = B.xeb_plan_create(circ, bs, opts=o)
    full = B.xeb_plan_stats(p0)
    B.xeb_plan_destroy(p0)
    o.mem_budget = full["arena_bytes"] // 16
    objs = {}
    for planner in (B.XEB_PLANNER_ANNEAL, B.XEB_PLANNER_AUTO, B.XEB_PLANNER_GREEDY, B.XEB_PLANNER_SWEEP):
        o.planner = planner
        p = B.xeb_plan_create(circ, bs, opts=o)
        try:
            st = B.xeb_plan_stats(p)
            objs[planner] = st["objective"]
            if planner == B.XEB_PLANNER_ANNEAL:
                assert st["planner_used"] == B.XEB_PLANNER_ANNEAL
                assert st["arena_bytes"] <= o.mem_budget
                assert st["n_sliced"] >= 1
                tree, sliced = B.xeb_plan_tree(p)
                memo.check_tree(tree, len(net.leaves))
                kt = memo.key_tables(net, tree, bs)
                c, rw = memo.costs(net, tree, kt["k"], sliced)
                assert st["flops_per_slice"] == 8 * c
                assert st["rw_elems_per_slice"] == rw
        finally:
            B.xeb_plan_destroy(p)
    assert objs[B.XEB_PLANNER_AUTO] <= min(objs[B.XEB_PLANNER_GREEDY], objs[B.XEB_PLANNER_SWEEP]) + 1e-12


def test_slice_subset_is_seeded_and_distinct():
    circ = inputs.random_grid_circuit(3, 4, 8, 11)
    bs = inputs.uniform_bitstrings(12, 50, 12)
    net = network.fused_network(circ)
    bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
    p = B.xeb_plan_create(circ, bs, slices=bonds[:6])
    try:
        assert B.xeb_set_slice_subset(p, 1.0, 0) == 64
        assert list(B.xeb_plan_slice_ids(p, 64)) == list(range(64))
        n = B.xeb_set_slice_subset(p, 0.25, 99)
        assert n == 16
        ids = B.xeb_plan_slice_ids(p, n)
        assert len(set(ids.tolist())) == 16 and ids.min() >= 0 and ids.max() < 64
        B.xeb_set_slice_subset(p, 0.25, 99)
        assert np.array_equal(B.xeb_plan_slice_ids(p, n), ids)       # same seed, same subset
        B.xeb_set_slice_subset(p, 0.25, 100)
        assert not np.array_equal(B.xeb_plan_slice_ids(p, n), ids)
        assert B.xeb_set_slice_subset(p, 1e-9, 1) == 1                # at least one value
        with pytest.raises(B.XebError):
            B.xeb_set_slice_subset(p, 0.0, 1)
    finally:
        B.xeb_plan_destroy(p)


def test_wide_plan_saturates_and_is_refused_at_bind(lib):
    """A tree that first joins every output leaf of a 40-qubit circuit (300
    distinct keys) and then absorbs the other leaves from the last gate
    backwards carries ~300 keys x 2^40 elements: no device holds it.  Its
    sizes saturate at 2^48 elements per tensor (a finite byte count below
    2^62, no integer overflow) and binding refuses it with XEB_ENOMEM before
    any device call."""
    w = inputs.WORKLOADS["grid5x8_m12_k100000"]
    circ = w.circuit()
    bits = inputs.uniform_bitstrings(circ.n_qubits, 300, 11)
    outq, _ = B.xeb_network_leaves(circ)
    order = [j for j in range(len(outq)) if outq[j]] + [j for j in range(len(outq)) if not outq[j]][::-1]
    tree = [(-1 - order[0], -1 - order[1])] + [(i - 1, -1 - order[i + 1]) for i in range(1, len(order) - 1)]
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_FP32
    plan = B.xeb_plan_create(circ, bits, tree=tree, slices=[], opts=o)
    try:
        nbytes = B.xeb_plan_device_bytes(plan)
        assert 8 * 2 ** 48 <= nbytes < 2 ** 62
        assert B.xeb_plan_stats(plan)["arena_bytes"] >= 8 * 2 ** 48
        with pytest.raises(B.XebError) as e:
            B.xeb_plan_bind(plan, 0, 0, 0)
        assert e.value.status == 2
    finally:
        B.xeb_plan_destroy(plan)


def test_batched_plan_root_holds_the_open_legs(lib):
    """Multi-batch plans (Sec. "Multi-batch simulator"): the w open output
    legs are never summed, so the root tensor carries exactly them, its pi
    range covers the n - w projected qubits, and its evaluation count is the
    number of distinct values of the projected bits (the open bits of the
    input bitstrings are ignored)."""
    circ = inputs.random_grid_circuit(3, 4, 8, 808)
    bits = inputs.uniform_bitstrings(12, 400, 909)
    open_q = [1, 6, 10]
    mask = sum(1 << q for q in open_q)
    o = B.xeb_default_opts()
    plan = B.xeb_plan_create(circ, bits, opts=o, open_qubits=open_q)
    try:
        st = B.xeb_plan_stats(plan)
        root = B.xeb_plan_node(plan, st["n_nodes"] - 1)
        assert root["n_legs"] == 3
        assert root["b"] - root["a"] == 12 - 3
        fixed = {int(b) & ~mask for b in bits}
        assert root["kv"] == len(fixed)
    finally:
        B.xeb_plan_destroy(plan)
    # bond legs keep their ids, the open legs follow them; an open leg cannot be sliced
    _, n_legs = B.xeb_network_info(circ)
    with pytest.raises(B.XebError) as e:
        B.xeb_plan_create(circ, bits, slices=[n_legs + 1], opts=o, open_qubits=open_q)
    assert e.value.status == 1
    p2 = B.xeb_plan_create(circ, bits, slices=[3], opts=o, open_qubits=open_q)   # a bond leg: fine
    B.xeb_plan_destroy(p2)
    with pytest.raises(B.XebError) as e:
        B.xeb_plan_create(circ, bits, opts=o, open_qubits=list(range(12)))
    assert e.value.status == 5
    big = inputs.random_grid_circuit(4, 5, 2, 7)
    with pytest.raises(B.XebError) as e:
        B.xeb_plan_create(big, inputs.uniform_bitstrings(20, 10, 1), opts=o, open_qubits=list(range(17)))
    assert e.value.status == 5


def test_op_layout_lists_are_permutations(lib):
    """xeb_plan_op_layout: for every contraction of a plan, the row and
    summed bits of A, the summed and column bits of B, and the row and
    column bits of C are each a permutation of that tensor's address bits,
    and the bit counts match the node ranks (App. A: 2^(q+r) products of a
    pairwise contraction, legs of dimension 2)."""
    circ = inputs.random_grid_circuit(4, 5, 10, 515)
    bits = inputs.uniform_bitstrings(20, 500, 616)
    for prec in (B.XEB_PREC_FP32, B.XEB_PREC_TF32X3):
        o = B.xeb_default_opts()
        o.precision = prec
        plan = B.xeb_plan_create(circ, bits, opts=o)
        try:
            n_leaves = len(B.xeb_network_leaves(circ)[0])
            n_gemm = 0
            i = 0
            while True:
                try:
                    L = B.xeb_plan_op_layout(plan, i)
                except B.XebError as e:
                    assert e.status == 1
                    break
                i += 1
                if L["kind"] != 2:
                    continue
                n_gemm += 1
                ra = len(L["a_pos_m"]) + len(L["a_pos_k"])
                rb = len(L["b_pos_k"]) + len(L["b_pos_n"])
                rc = len(L["c_pos_m"]) + len(L["c_pos_n"])
                assert sorted(L["a_pos_m"] + L["a_pos_k"]) == list(range(ra))
                assert sorted(L["b_pos_k"] + L["b_pos_n"]) == list(range(rb))
                assert sorted(L["c_pos_m"] + L["c_pos_n"]) == list(range(rc))
                assert len(L["a_pos_k"]) == len(L["b_pos_k"])
                assert len(L["c_pos_m"]) == len(L["a_pos_m"]) and len(L["c_pos_n"]) == len(L["b_pos_n"])
                nd = B.xeb_plan_node(plan, L["node"] - n_leaves)
                assert nd["n_legs"] == rc and nd["n_shared"] == len(L["a_pos_k"])
            assert n_gemm == n_leaves - 1
        finally:
            B.xeb_plan_destroy(plan)


def test_chunked_run_rejects_bad_arguments(lib):
    circ = inputs.random_grid_circuit(3, 4, 8, 1)
    bits = inputs.uniform_bitstrings(12, 50, 2)
    with pytest.raises(B.XebError) as e:
        B.xeb_run_chunked(circ, bits, 0)
    assert e.value.status == 1
    with pytest.raises(B.XebError) as e:
        B.xeb_run_chunked(circ, bits[:0], 10)
    assert e.value.status == 1


def _reuse_launches(plan, circ, ids):
    """Contractions one step launches under the cross-slice rule, walked in
    plain Python: masks of slice bits per subtree, effective masks top-down,
    a node runs in slice t iff t = 0 or (s_t ^ s_{t-1}) & e_v != 0."""
    tree, sliced = B.xeb_plan_tree(plan)
    _, legs = B.xeb_network_leaves(circ)
    L = len(legs)
    m = [sum(1 << sliced.index(l) for l in legs[j] if l in sliced) for j in range(L)]
    kids = []
    for a, b in tree:
        ca = -1 - a if a < 0 else L + a
        cb = -1 - b if b < 0 else L + b
        kids.append((ca, cb))
        m.append(m[ca] | m[cb])
    e = [0] * len(m)
    e[-1] = (1 << len(sliced)) - 1
    for v in range(len(m) - 1, L - 1, -1):
        for c in kids[v - L]:
            e[c] = m[c] if (m[c] != e[v] and c >= L) else e[v]
    n = 0
    for v in range(L, len(m)):
        prev = None
        for s in ids:
            if prev is None or ((s ^ prev) & e[v]):
                n += 1
            prev = s
    return n


def test_cross_slice_reuse_counts(lib):
    """Slice-invariant and partly invariant subtrees run once per value of
    the sliced legs they hold: the step's work with reuse is below the plain
    sum over slices, equal to it with reuse off (opts.reserved[7] = 1), and
    the count of launched contractions matches a plain walk of the rule, both
    for all slices (closed form) and for a seeded subset (enumerated)."""
    circ = inputs.random_grid_circuit(3, 4, 8, 4545)
    bits = inputs.uniform_bitstrings(12, 60, 4646)
    net = network.fused_network(circ)
    bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
    sliced = [bonds[3], bonds[17], bonds[40], bonds[55]]
    res = {}
    for off in (0, 1):
        o = B.xeb_default_opts()
        o.reserved[7] = off
        o.fold_legs = -1   # every contraction on the device (folding has its own test)
        plan = B.xeb_plan_create(circ, bits, slices=sliced, opts=o)
        try:
            st = B.xeb_plan_stats(plan)
            fl, nc = B.xeb_plan_step_flops(plan)
            ids = list(range(st["n_slices"]))
            assert nc == _reuse_launches(plan, circ, ids) if off == 0 else nc == st["n_gemm_ops"] * st["n_slices"]
            res[off] = (fl, nc, st["n_reused"], st["flops_per_slice"] * st["n_slices"])
            if off == 0:
                n_sub = B.xeb_set_slice_subset(plan, 0.5, 99)
                sub = [int(x) for x in B.xeb_plan_slice_ids(plan, n_sub)]
                fl2, nc2 = B.xeb_plan_step_flops(plan)
                assert nc2 == _reuse_launches(plan, circ, sub)
        finally:
            B.xeb_plan_destroy(plan)
    assert res[1][0] == res[1][3] and res[1][2] == 0
    assert res[0][2] >= 1 and res[0][0] < res[0][3] and res[0][1] < res[1][1]


def _replay_step(plan, circ, elem, ids):
    """Replay one step's data flow over the plan's arena placement, slices in
    the order ids: every slice rewrites the leaves and runs each contraction
    whose cross-slice mask saw a change (all of them in the first slice); an
    operand must still hold its node's value for the current slice (the
    node's own sliced-leg bits).  Returns the number of stale operand reads
    and the number of nodes kept across slices."""
    off, el, mk = B.xeb_plan_buffers(plan)
    st = B.xeb_plan_stats(plan)
    tree, sliced = B.xeb_plan_tree(plan)
    _, legs = B.xeb_network_leaves(circ)
    L = len(legs)
    m = [sum(1 << sliced.index(l) for l in legs[j] if l in sliced) for j in range(L)]
    for a, b in tree:
        m.append(m[-1 - a if a < 0 else L + a] | m[-1 - b if b < 0 else L + b])
    ops, i = [], 0
    while True:
        try:
            lay = B.xeb_plan_op_layout(plan, i)
        except B.XebError:
            break
        i += 1
        if lay["kind"] == 2:
            ops.append((lay["node"], lay["a_node"], lay["b_node"]))
    n_arena = st["arena_bytes"] // elem
    owner = np.full(n_arena, -1, dtype=np.int32)
    ver = np.zeros(n_arena, dtype=np.int64)

    def holds(v, s):
        sl = slice(off[v], off[v] + el[v])
        return bool(np.all(owner[sl] == v) and np.all(ver[sl] == (s & m[v])))

    def put(v, s):
        sl = slice(off[v], off[v] + el[v])
        owner[sl] = v
        ver[sl] = s & m[v]

    bad, prev = 0, None
    for s in ids:
        for j in range(L):
            put(j, s)
        for v, a, b in ops:
            if prev is not None and not ((s ^ prev) & int(mk[v])):
                continue
            bad += (not holds(a, s)) + (not holds(b, s))
            put(v, s)
        bad += not holds(len(m) - 1, s)
        prev = s
    return bad, st["n_reused"]


@pytest.mark.parametrize("case", ["given", "annealed", "batched", "subset"])
def test_cross_slice_reuse_replay_reads_fresh_operands(lib, case):
    """The arena placement with buffers kept across slices is consistent with
    the skip rule: replaying a step's data flow (every slice in counting
    order, or a shuffled seeded subset) finds no operand overwritten before
    it is read."""
    o = B.xeb_default_opts()
    if case == "given":
        circ = inputs.random_grid_circuit(3, 4, 8, 4545)
        bits = inputs.uniform_bitstrings(12, 60, 4646)
        net = network.fused_network(circ)
        bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
        plan = B.xeb_plan_create(circ, bits, slices=[bonds[3], bonds[17], bonds[40], bonds[55]], opts=o)
    else:
        circ = inputs.random_grid_circuit(4, 5, 10, 5353)
        bits = inputs.uniform_bitstrings(20, 400, 5454)
        o.planner = B.XEB_PLANNER_ANNEAL
        o.mem_budget = 4 << 20
        plan = B.xeb_plan_create(circ, bits, opts=o, open_qubits=[2, 11, 17] if case == "batched" else None)
    try:
        frac, seed = (0.75, 2024) if case == "subset" else (1.0, 0)
        n = B.xeb_set_slice_subset(plan, frac, seed)
        ids = [int(x) for x in B.xeb_plan_slice_ids(plan, n)]
        if case == "subset":
            assert ids != sorted(ids)
        bad, kept = _replay_step(plan, circ, 8, ids)
        assert kept >= 1 and len(ids) >= 4
        assert bad == 0
    finally:
        B.xeb_plan_destroy(plan)


def test_new_entry_points_reject_bad_arguments(lib):
    import ctypes as C
    circ = inputs.random_grid_circuit(3, 4, 8, 77)
    bits = inputs.uniform_bitstrings(12, 20, 78)
    with pytest.raises(B.XebError) as e:        # open qubit outside the circuit
        B.xeb_plan_create(circ, bits, open_qubits=[12])
    assert e.value.status == 1
    n = C.c_int32()
    assert B.load().xeb_plan_buffers(None, None, None, None, C.byref(n)) == 1
    assert B.load().xeb_plan_step_flops(None, None, None) == 1
    assert B.load().xeb_plan_op_layout(None, 0, None, 0, C.byref(n)) == 1
    form = np.zeros(5, dtype=np.int32)
    assert B.load().xeb_plan_op_form(None, 0, form.ctypes.data_as(C.POINTER(C.c_int32))) == 1
    out = C.c_void_p()
    assert B.load().xeb_plan_create_learned(None, None, 0, None, None, 1, None, None, C.byref(out)) == 1
    plan = B.xeb_plan_create(circ, bits)
    try:
        assert B.load().xeb_plan_buffers(plan, None, None, None, None) == 1
        with pytest.raises(B.XebError):
            B.xeb_plan_op_layout(plan, -1)
        with pytest.raises(B.XebError):      # not bound: no kernel forms yet
            B.xeb_plan_op_form(plan, 0)
        assert B.load().xeb_plan_op_form(plan, 0, None) == 1
        off, el, mk = B.xeb_plan_buffers(plan)
        assert len(off) == 2 * len(B.xeb_network_leaves(circ)[0]) - 1
        assert np.all(el > 0) and np.all(off >= 0) and np.all(mk == 0xFFFFFFFF)   # unsliced: no reuse
    finally:
        B.xeb_plan_destroy(plan)


def _foldable(plan, circ, sliced, max_legs=16):
    """Nodes that constant folding takes, walked in plain Python: a subtree
    qualifies when no leaf in it carries an output bit or a sliced leg and no
    tensor in it has more than max_legs legs; the qualifying internal nodes
    whose parent does not qualify are folded with their whole subtree."""
    tree, _ = B.xeb_plan_tree(plan)
    out_bits, legs = B.xeb_network_leaves(circ)
    L = len(legs)
    ok = [len(out_bits[j]) == 0 and not any(l in sliced for l in legs[j]) and len(legs[j]) <= max_legs
          for j in range(L)]
    kids, parent = [], {}
    for i, (a, b) in enumerate(tree):
        ca = -1 - a if a < 0 else L + a
        cb = -1 - b if b < 0 else L + b
        kids.append((ca, cb))
        parent[ca] = parent[cb] = L + i
        nd = B.xeb_plan_node(plan, i)
        ok.append(ok[ca] and ok[cb] and nd["a"] == nd["b"] and nd["n_legs"] <= max_legs)
    roots = [v for v in range(L, L + len(tree) - 1) if ok[v] and not ok[parent[v]]]
    inside = 0
    for r in roots:
        stack = [r]
        while stack:
            u = stack.pop()
            inside += 1
            if u >= L:
                stack.extend(kids[u - L])
    return roots, inside


@pytest.mark.parametrize("sliced_idx", [(), (3, 17, 40, 55)])
def test_constant_folding_counts(lib, sliced_idx):
    """Subtrees that depend on no output bit and no sliced leg are folded on
    the host: the plan folds exactly the subtrees a plain walk of the rule
    finds, and a step launches every other contraction (all slices: with
    cross-slice reuse off, n_gemm_ops minus the folded internal nodes per
    slice)."""
    circ = inputs.random_grid_circuit(3, 4, 8, 4545)
    bits = inputs.uniform_bitstrings(12, 60, 4646)
    net = network.fused_network(circ)
    bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
    sliced = [bonds[i] for i in sliced_idx]
    o = B.xeb_default_opts()
    o.reserved[7] = 1
    plan = B.xeb_plan_create(circ, bits, slices=sliced or None, opts=o)
    try:
        st = B.xeb_plan_stats(plan)
        roots, inside = _foldable(plan, circ, sliced)
        assert st["n_fold_roots"] == len(roots) and len(roots) > 0
        assert st["n_folded"] == inside
        # a folded subtree of r internal nodes holds r + 1 leaves
        folded_internal = (inside - len(roots)) // 2
        _, nc = B.xeb_plan_step_flops(plan)
        assert nc == (st["n_gemm_ops"] - folded_internal) * st["n_slices"]
    finally:
        B.xeb_plan_destroy(plan)
    o.fold_legs = -1
    plan = B.xeb_plan_create(circ, bits, slices=sliced or None, opts=o)
    try:
        st = B.xeb_plan_stats(plan)
        assert st["n_folded"] == 0 and st["n_fold_roots"] == 0
        assert B.xeb_plan_step_flops(plan)[1] == st["n_gemm_ops"] * st["n_slices"]
    finally:
        B.xeb_plan_destroy(plan)


def test_round_keep_norm_stays_between_neighbours_and_keeps_the_norm(lib):
    """xeb_round_keep_norm: every value is one of the two floats nearest its
    input (so each error is below one float spacing), the sum of squares lands
    within one flip of the exact one and never farther than nearest rounding
    leaves it, exactly representable inputs stay as they are, and for a
    tensor of many values the norm error falls far below nearest rounding's.
    The leaves of the fused network (unitary gate tensors) are the inputs the
    library feeds it."""
    rng = np.random.default_rng(7)
    net = network.fused_network(inputs.random_grid_circuit(3, 4, 8, 11))
    cases = [np.stack([lf.tensor.real.ravel(), lf.tensor.imag.ravel()], 1).ravel() for lf in net.leaves]
    cases += [rng.standard_normal(n) * s for n, s in ((7, 0.3), (64, 1.0), (4096, 1e-3))]
    cases.append(np.array([0.5, -0.25, 1.0, 0.0, 3.0]))   # exactly representable
    big_gain = []
    for x in cases:
        y = B.xeb_round_keep_norm(x).astype(np.float64)
        rn = x.astype(np.float32).astype(np.float64)
        lo = np.nextafter(rn.astype(np.float32), np.float32(-np.inf)).astype(np.float64)
        hi = np.nextafter(rn.astype(np.float32), np.float32(np.inf)).astype(np.float64)
        # y is the nearest float or the other float on the far side of x
        assert np.all((y == rn) | ((y == lo) & (rn > x)) | ((y == hi) & (rn < x)))
        assert np.all(y[rn == x] == x[rn == x])
        e_keep = abs(np.sum(y * y) - np.sum(x * x))
        e_rn = abs(np.sum(rn * rn) - np.sum(x * x))
        assert e_keep <= e_rn + 1e-30
        step = 2 * np.max(np.abs(x)) * np.max(np.abs(hi - lo)) + 1e-300
        assert e_keep <= step
        if x.size >= 64:
            big_gain.append(e_keep / max(e_rn, 1e-300))
    assert max(big_gain) < 0.1


def test_noalloc_xeb_refuses_bad_arguments_before_any_launch(lib):
    """The allocation-free XEB checks its arguments on the host before it
    touches the device: NULL pointers, an amplitude pointer that is not
    16-byte aligned (amplitudes are read as 16-byte values), k = 0, k beyond
    the fixed scratch array and n_qubits outside [1, 64] return XEB_EINVAL
    (these calls run here, where there is no GPU)."""
    aligned, misaligned = 0x10000, 0x10008
    bad = [(0, 10, 12, aligned), (aligned, 10, 12, 0), (misaligned, 10, 12, aligned), (aligned, 0, 12, aligned),
           (aligned, 16777217, 12, aligned), (aligned, 10, 0, aligned), (aligned, 10, 65, aligned)]
    for a, k, n, o in bad:
        with pytest.raises(B.XebError) as e:
            B.xeb_linear_xeb_noalloc(a, k, n, o, 0)
        assert e.value.status == 1
    with pytest.raises(B.XebError) as e:
        B.xeb_linear_xeb_noalloc(misaligned, 10, 12, aligned, 0)
    assert "16-byte" in str(e.value)


def test_deep_k_cases_hold_their_contraction_form():
    """The plans of the deep-K tensor-core parity cases still contain the
    keyed contraction each case is there to exercise."""
    from kdeep_cases import CASES, plan_opts, deep_k_shapes
    for case in CASES:
        r, c = case["grid"]
        circ = inputs.random_grid_circuit(r, c, case["cycles"], 4242)
        bits = inputs.uniform_bitstrings(r * c, case["k"], 4343)
        plan = B.Plan(circ, bits, opts=plan_opts(case))
        assert case["shape"] in deep_k_shapes(plan), (case["id"], deep_k_shapes(plan))
        plan.close()
