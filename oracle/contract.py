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


def amplitudes(net: Network, bitstrings, sliced: Optional[List[int]] = None):
    """<s|C|0^n> for each bitstring.  If ``sliced`` legs are given, the sum over
    all their values is taken explicitly (Sec. "Slicing": contract per value,
    then add)."""
    bitstrings = np.asarray(bitstrings, dtype=np.uint64)
    sliced = list(sliced or [])
    assignments = [dict(zip(sliced, [(v >> t) & 1 for t in range(len(sliced))]))
                   for v in range(1 << len(sliced))] if sliced else [None]
    out = np.zeros(len(bitstrings), dtype=np.complex128)
    seq = None
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
