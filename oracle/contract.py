"""Naive FP64 pairwise tensor-network contractor (no memoization).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For one bitstring s the amplitude <s|C|0^n> is the full contraction of the
circuit network with its open legs fixed to s (Sec. "Multi-batch simulator");
pairwise contractions T*S follow Eq. (elem-cont).  The order is this module's
own: repeatedly contract the connected pair whose result is smallest (ties by
lowest indices).  The order depends only on shapes, so it is chosen once and
replayed for every bitstring.
"""
from __future__ import annotations

from typing import Dict, List, Optional

import numpy as np

from .network import Network, pair_contract, project_leaf


def greedy_order(leg_sets: List[List[int]]):
    """Sequence of (i, j) merges over a working list (the merged tensor is
    appended at the end, i and j removed)."""
    work = [list(s) for s in leg_sets]
    seq = []
    while len(work) > 1:
        best = None
        for i in range(len(work)):
            si = set(work[i])
            for j in range(i + 1, len(work)):
                sj = set(work[j])
                if not (si & sj):
                    continue
                size = len(si ^ sj)
                if best is None or size < best[0]:
                    best = (size, i, j)
        if best is None:              # disconnected: outer product of the two smallest
            order = sorted(range(len(work)), key=lambda t: (len(work[t]), t))
            i, j = sorted(order[:2])
        else:
            _, i, j = best
        merged = [l for l in work[i] if l not in work[j]] + \
                 [l for l in work[j] if l not in work[i]]
        seq.append((i, j))
        work = [w for t, w in enumerate(work) if t not in (i, j)] + [merged]
    return seq


def sequence_cost(leg_sets: List[List[int]], seq):
    """Multiplications of a merge sequence: a pairwise contraction costs
    2^(q + r) (App. A), i.e. 2 to the number of distinct legs of its two
    operands."""
    work = [set(s) for s in leg_sets]
    cost = 0
    for i, j in seq:
        cost += 2 ** len(work[i] | work[j])
        merged = work[i] ^ work[j]
        work = [w for t, w in enumerate(work) if t not in (i, j)] + [merged]
    return cost


def search_order(leg_sets: List[List[int]], trials: int = 64, temperature: float = 0.5, seed: int = 0):
    """A cheaper order for large networks: randomised greedy merging -- among
    the connected pairs, the one whose merged rank grows least over its larger
    operand, with Gumbel noise of the given temperature on that score -- run
    `trials` times; the sequence with the fewest multiplications wins (the
    noiseless min-size greedy_order is always one of the candidates).  The
    order changes only the cost, never the result."""
    rng = np.random.default_rng(seed)
    best = greedy_order(leg_sets)
    best_cost = sequence_cost(leg_sets, best)
    for _ in range(trials):
        work = [set(s) for s in leg_sets]
        ids = list(range(len(work)))          # working list of tensor ids
        sets = {i: work[i] for i in ids}
        owners = {}
        for i, st in sets.items():
            for l in st:
                owners.setdefault(l, set()).add(i)
        nxt = len(work)
        seq = []
        while len(ids) > 1:
            pairs = {tuple(sorted(o)) for o in owners.values() if len(o) == 2}
            pick = None
            for a, b in sorted(pairs):
                sa, sb = sets[a], sets[b]
                score = len(sa ^ sb) - max(len(sa), len(sb)) - temperature * np.log(-np.log(rng.random()))
                if pick is None or score < pick[0]:
                    pick = (score, a, b)
            if pick is None:                  # disconnected: the two smallest
                a, b = sorted(sorted(ids, key=lambda t: (len(sets[t]), t))[:2])
            else:
                _, a, b = pick
            i, j = sorted((ids.index(a), ids.index(b)))
            seq.append((i, j))
            merged = sets[a] ^ sets[b]
            for l in sets[a] | sets[b]:
                owners[l].discard(a)
                owners[l].discard(b)
                if not owners[l]:
                    del owners[l]
            for l in merged:
                owners.setdefault(l, set()).add(nxt)
            del sets[a], sets[b]
            sets[nxt] = merged
            ids = [t for t in ids if t not in (a, b)] + [nxt]
            nxt += 1
        c = sequence_cost(leg_sets, seq)
        if c < best_cost:
            best, best_cost = seq, c
    return best


def amplitudes(net: Network, bitstrings, sliced: Optional[List[int]] = None,
               values: Optional[List[int]] = None, seq=None):
    """<s|C|0^n> for each bitstring.  If ``sliced`` legs are given, the sum over
    all their values is taken explicitly (Sec. "Slicing": contract per value,
    then add); ``values`` restricts that sum to the listed slice values (bit b
    of a value is the value of sliced[b]) and then gives a partial sum, not an
    amplitude.  ``seq`` is a merge sequence (default: greedy_order)."""
    bitstrings = np.asarray(bitstrings, dtype=np.uint64)
    sliced = list(sliced or [])
    if values is None:
        values = range(1 << len(sliced))
    assignments = [dict(zip(sliced, [(v >> t) & 1 for t in range(len(sliced))]))
                   for v in values] if sliced else [None]
    out = np.zeros(len(bitstrings), dtype=np.complex128)
    for assign in assignments:
        for idx, word in enumerate(bitstrings):
            items = [project_leaf(l, int(word), assign) for l in net.leaves]
            if seq is None:
                seq = greedy_order([legs for _, legs in items])
            work = list(items)
            for i, j in seq:
                r = pair_contract(work[i][0], work[i][1], work[j][0], work[j][1])
                work = [w for t, w in enumerate(work) if t not in (i, j)] + [r]
            t, legs = work[0]
            assert not legs
            out[idx] += complex(t)
    return out
