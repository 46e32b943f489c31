"""Seeded random contraction trees for tests (children format: post-order,
leaf j = -1-j).  Merges a random pair among the few connected pairs with the
smallest result, so trees vary but stay small enough to evaluate."""
import numpy as np


def random_tree(leaf_legs, seed, choices=3, sliced=()):
    rng = np.random.default_rng(seed)
    sl = set(sliced)
    work = [(-1 - j, set(l) - sl) for j, l in enumerate(leaf_legs)]
    tree = []
    while len(work) > 1:
        cands = []
        for i in range(len(work)):
            for j in range(i + 1, len(work)):
                if work[i][1] & work[j][1]:
                    cands.append((len(work[i][1] ^ work[j][1]), i, j))
        if not cands:
            cands = [(0, 0, 1)]
        cands.sort()
        _, i, j = cands[int(rng.integers(0, min(choices, len(cands))))]
        if rng.integers(0, 2):
            i, j = j, i
        tree.append((work[i][0], work[j][0]))
        merged = (len(tree) - 1, work[i][1] ^ work[j][1])
        work = [w for t, w in enumerate(work) if t not in (i, j)] + [merged]
    return tree
