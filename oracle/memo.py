"""Memoization semantics of the multi-tensor contraction, written plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Trees use the children format shared with the library's C ABI: a list of
(left, right) pairs in post-order; a child ``c >= 0`` is an earlier internal
node, ``c < 0`` is leaf ``-1-c``; the last pair is the root.

Contents
* ``key_tables``: for every node v, the distinct values of the output bits it
  depends on, as plain sort/dedup.  A subexpression is evaluated once per
  distinct value of its variables (Sec. "Multi-tensor contraction algorithm",
  Fig. "main idea"); variables are numbered by their position in the tree and
  tuples are ordered lexicographically (App. C, eval_all).  Reading used here:
  the output bits, taken in in-order leaf order pi (each leaf contributing its
  open legs in its listed order), form a contiguous range [a_v, b_v) for every
  node; the node's key value is that bit range read as a binary number with
  pi's first bit most significant, so lexicographic order = numeric order; key
  ids are ranks in ascending order; the children's ids of key u are
  (uL(u), uR(u)).
* ``alg12``: what Alg. 1 driving Alg. 2 (eval with a global cache keyed by
  (subexpression; values of its variables)) computes, tabulated bottom-up
  over the tree's post-order: each node contracted once per distinct value
  of its variables among the bitstrings; returns the results and the number
  of contractions performed per node.
* ``alg34``: what Alg. 3 (eval_all) and Alg. 4 (eval') compute: over the
  sorted distinct tuples of leaf value indices, each node evaluated once per
  distinct sub-tuple, its right child for all distinct right parts at once
  and its left child over the consecutive groups of equal prefixes (the
  text's loop bound "i=1,...,m" is read as i = 1..|t|).
* ``costs``: the contraction cost C = sum_v k_v 2^(q_v + r_v) and read/write
  count RW = sum_v k_v (m(L) + m(R) + m(v)) of App. A/C, with exact or bound
  evaluation counts k_v (App. C, "Complexity estimation").
"""
from __future__ import annotations

from collections import defaultdict
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .network import Network, pair_contract, project_leaf


# --- tree helpers -------------------------------------------------------------

def check_tree(tree: Sequence[Tuple[int, int]], n_leaves: int):
    seen_leaf = [0] * n_leaves
    used_node = [0] * len(tree)
    for i, (l, r) in enumerate(tree):
        for c in (l, r):
            if c < 0:
                seen_leaf[-1 - c] += 1
            else:
                assert c < i, "children must precede their parent"
                used_node[c] += 1
    assert all(s == 1 for s in seen_leaf), "every leaf exactly once"
    assert all(u == 1 for u in used_node[:-1]) and used_node[-1] == 0


def inorder_leaves(tree, ref: int) -> List[int]:
    if ref < 0:
        return [-1 - ref]
    l, r = tree[ref]
    return inorder_leaves(tree, l) + inorder_leaves(tree, r)


def root_ref(tree) -> int:
    return len(tree) - 1


def pi_order(net: Network, tree) -> List[int]:
    """Output qubits in in-order leaf order."""
    order = []
    for j in inorder_leaves(tree, root_ref(tree)):
        order += list(net.leaves[j].out_qubits)
    return order


def bit_ranges(net: Network, tree) -> Dict[int, Tuple[int, int]]:
    """ref -> [a, b) range in pi of the output bits the subtree depends on."""
    ranges: Dict[int, Tuple[int, int]] = {}

    def walk(ref, start):
        if ref < 0:
            w = len(net.leaves[-1 - ref].out_qubits)
            ranges[ref] = (start, start + w)
            return start + w
        l, r = tree[ref]
        mid = walk(l, start)
        end = walk(r, mid)
        ranges[ref] = (start, end)
        return end

    walk(root_ref(tree), 0)
    return ranges


def range_values(bitstrings: np.ndarray, pi: Sequence[int], a: int, b: int):
    """Bits pi[a..b) of every word as a number, pi[a] most significant."""
    v = np.zeros(len(bitstrings), dtype=np.uint64)
    for t in range(a, b):
        bit = (bitstrings >> np.uint64(pi[t])) & np.uint64(1)
        v = (v << np.uint64(1)) | bit
    return v


# --- key tables (plain sort/dedup) --------------------------------------------

def key_tables(net: Network, tree, bitstrings) -> dict:
    bitstrings = np.asarray(bitstrings, dtype=np.uint64)
    pi = pi_order(net, tree)
    ranges = bit_ranges(net, tree)
    out = {"pi": pi, "range": ranges, "unique": {}, "key": {}, "k": {},
           "uL": {}, "uR": {}}
    for ref, (a, b) in ranges.items():
        vals = range_values(bitstrings, pi, a, b)
        uniq, inv = np.unique(vals, return_inverse=True)
        out["unique"][ref] = uniq
        out["key"][ref] = inv.astype(np.int64).reshape(-1)
        out["k"][ref] = len(uniq)
    for i, (l, r) in enumerate(tree):
        a_r, b_r = ranges[r]
        wr = np.uint64(b_r - a_r)
        uv = out["unique"][i]
        left_part = uv >> wr
        right_part = uv & ((np.uint64(1) << wr) - np.uint64(1))
        out["uL"][i] = np.searchsorted(out["unique"][l], left_part).astype(np.int64)
        out["uR"][i] = np.searchsorted(out["unique"][r], right_part).astype(np.int64)
        assert np.array_equal(out["unique"][l][out["uL"][i]], left_part)
        assert np.array_equal(out["unique"][r][out["uR"][i]], right_part)
    return out


# --- Alg. 1 / Alg. 2 ------------------------------------------------------------

def _leaf_value_id(net: Network, j: int, word: int) -> Tuple[int, ...]:
    return tuple((word >> q) & 1 for q in net.leaves[j].out_qubits)


def alg12(net: Network, tree, bitstrings, sliced: Optional[Dict[int, int]] = None):
    """What Alg. 1 (the loop over bitstrings) with Alg. 2 (eval with one
    global cache) computes, tabulated bottom-up instead of recursively: the
    cache ends up holding one entry per node and per distinct value of the
    variables below it (the value indices of the node's leaves) that some
    bitstring reaches, each computed once from its children's entries.  So
    walk the nodes in post-order (the tree's own order), and for each node
    contract once per distinct tuple of its leaves' value indices among the
    bitstrings.  Returns (results in input order, contractions per node)."""
    words = [int(w) for w in np.asarray(bitstrings, dtype=np.uint64)]
    leaves_of = {i: inorder_leaves(tree, i) for i in range(len(tree))}
    counts: Dict[int, int] = defaultdict(int)

    def sub(ref, word):
        """the tuple of leaf value indices of subtree ref for this bitstring"""
        js = [-1 - ref] if ref < 0 else leaves_of[ref]
        return tuple(_leaf_value_id(net, j, word) for j in js)

    table: Dict[int, Dict[tuple, tuple]] = {}

    def lookup(ref, word):
        if ref < 0:
            return project_leaf(net.leaves[-1 - ref], word, sliced)
        return table[ref][sub(ref, word)]

    for i, (l, r) in enumerate(tree):
        table[i] = {}
        for w in words:
            t = sub(i, w)
            if t in table[i]:
                continue
            a, b = lookup(l, w), lookup(r, w)
            table[i][t] = pair_contract(a[0], a[1], b[0], b[1])
            counts[i] += 1
    root = root_ref(tree)
    res = []
    for w in words:
        t, legs = table[root][sub(root, w)]
        assert not legs
        res.append(complex(t))
    return np.array(res, dtype=np.complex128), dict(counts)


# --- Alg. 3 / Alg. 4 ------------------------------------------------------------

def alg34(net: Network, tree, bitstrings, sliced: Optional[Dict[int, int]] = None):
    """Alg. 3 (eval_all) with Alg. 4 (eval'), restated by what they compute.

    Each bitstring becomes the tuple of its leaves' value indices, leaves in
    in-order position, where leaf j's values V_j are its distinct projected
    tensors in ascending order of its output-bit value; the tuples are sorted
    and made distinct.  A node's sub-tuple is the slice of a tuple over the
    leaves below it.  Evaluating a node for a sorted list of distinct
    sub-tuples means: evaluate its right child once for the distinct right
    parts of the list (the right cache), its left child once for the distinct
    left parts (prefixes, so equal ones are consecutive: the left cache holds
    one value at a time), then contract once per entry of the list.  Returns
    ({word: result}, contractions per node)."""
    bitstrings = np.asarray(bitstrings, dtype=np.uint64)
    order = inorder_leaves(tree, root_ref(tree))
    pos = {j: p for p, j in enumerate(order)}
    vid, V = [], []
    for j in order:
        ids = [_leaf_value_id(net, j, int(w)) for w in bitstrings]
        distinct = sorted(set(ids))
        V.append([project_leaf(net.leaves[j],
                               sum(b << q for b, q in zip(d, net.leaves[j].out_qubits)),
                               sliced) for d in distinct])
        vid.append({x: n for n, x in enumerate(distinct)})
        vid[-1] = [vid[-1][x] for x in ids]
    tuples = [tuple(vid[p][i] for p in range(len(order))) for i in range(len(bitstrings))]
    width = {}     # leaves below each node

    def count_leaves(ref):
        if ref < 0:
            width[ref] = 1
        else:
            l, r = tree[ref]
            count_leaves(l)
            count_leaves(r)
            width[ref] = width[l] + width[r]
        return width[ref]

    count_leaves(root_ref(tree))
    counts: Dict[int, int] = defaultdict(int)

    def evaluate(ref, subs):
        """{sub-tuple: value} of node ref for the sorted distinct sub-tuples subs."""
        if ref < 0:
            p = pos[-1 - ref]
            return {s: V[p][s[0]] for s in subs}
        l, r = tree[ref]
        nl = width[l]
        right = evaluate(r, sorted({s[nl:] for s in subs}))
        left = evaluate(l, sorted({s[:nl] for s in subs}))
        out = {}
        for s in subs:
            a, b = left[s[:nl]], right[s[nl:]]
            out[s] = pair_contract(a[0], a[1], b[0], b[1])
            counts[ref] += 1
        return out

    R = evaluate(root_ref(tree), sorted(set(tuples)))
    results = {}
    for i, w in enumerate(bitstrings):
        tval, legs = R[tuples[i]]
        assert not legs
        results[int(w)] = complex(tval)
    return results, dict(counts)


# --- cost counters (App. A, App. C) ---------------------------------------------

def node_legs(net: Network, tree, sliced: Sequence[int] = ()):
    """ref -> list of legs of the node's tensor, plus per internal node the
    number of summed legs q_v."""
    sl = set(sliced)
    legs = {}
    shared = {}
    for j, leaf in enumerate(net.leaves):
        legs[-1 - j] = [l for l in leaf.legs if l not in sl]
    for i, (l, r) in enumerate(tree):
        s = set(legs[l]) & set(legs[r])
        shared[i] = len(s)
        legs[i] = [x for x in legs[l] if x not in s] + [x for x in legs[r] if x not in s]
    return legs, shared


def bound_counts(net: Network, tree, k: int, value_counts: Dict[int, int]):
    """k_T bound of App. C: leaves min(|V_j|, k); internal min(k_L k_R, k)."""
    kb = {}
    for j in range(len(net.leaves)):
        kb[-1 - j] = min(value_counts[-1 - j], k)
    for i, (l, r) in enumerate(tree):
        kb[i] = min(kb[l] * kb[r], k)
    return kb


def costs(net: Network, tree, kv: Dict[int, int], sliced: Sequence[int] = ()):
    """(C, RW) per slice: C = sum_v k_v 2^(q_v + r_v) complex multiply-adds,
    RW = sum_v k_v (m(L) + m(R) + m(v)) elements, m = 2^(number of legs)."""
    legs, shared = node_legs(net, tree, sliced)
    c = 0
    rw = 0
    for i, (l, r) in enumerate(tree):
        c += kv[i] * (1 << (shared[i] + len(legs[i])))
        rw += kv[i] * ((1 << len(legs[l])) + (1 << len(legs[r])) + (1 << len(legs[i])))
    return c, rw
