"""World-size-2 gloo tests (CPU) of the multi-process host logic.

* Contiguous sharding covers every unit exactly once.
* Max-over-ranks timing.
* Slice partition through the library (App. A, "Slicing": the values of the
  sliced legs are independent terms added at the end): each rank restricts
  its plan's slice loop to its block with the library's host-side call
  (xeb_set_slice_block), reads back the slice values the plan will run
  (xeb_plan_slice_ids), and the ranks' lists, gathered over gloo, cover every
  value exactly once -- for all values and for a seeded subset.
* The one exchange step: each rank sums its slice values' partial amplitudes
  (computed on CPU by the oracle's contractor for exactly the values the
  library gave that rank, since the library's own contractions need a GPU)
  and the FP64 all-reduce of the partials equals the unsliced amplitudes.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2108_05665_gb300 import dist as D


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 1025):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = D.shard_range(n, r, world)
                seen += list(range(lo, hi))
                assert hi - lo in (n // world, n // world + 1)
            assert seen == list(range(n))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


CIRC = (2, 3, 5, 31)
SLICED = [1, 4, 6]


def _partial(net, bits, sliced, values):
    from oracle import contract
    from oracle.network import pair_contract, project_leaf
    part = np.zeros(len(bits), dtype=np.complex128)
    for s in values:
        assign = {leg: (int(s) >> t) & 1 for t, leg in enumerate(sliced)}
        for i, w in enumerate(bits):
            items = [project_leaf(l, int(w), assign) for l in net.leaves]
            seq = contract.greedy_order([lg for _, lg in items])
            work = list(items)
            for a, b in seq:
                r_ = pair_contract(work[a][0], work[a][1], work[b][0], work[b][1])
                work = [x for t, x in enumerate(work) if t not in (a, b)] + [r_]
            part[i] += complex(work[0][0])
    return part


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2108_05665_gb300 import binding as B, inputs
        from oracle import network
        D.barrier(world)
        m = D.max_over_ranks(float(rank * 3 + 1), world)
        circ = inputs.random_grid_circuit(*CIRC)
        bits = inputs.uniform_bitstrings(6, 9, 32)
        big = inputs.random_grid_circuit(3, 4, 8, 4545)
        big_bits = inputs.uniform_bitstrings(12, 60, 4646)
        bnet = network.fused_network(big)
        bonds = sorted({l for leaf in bnet.leaves for l in leaf.legs})
        covers = {}
        for frac, seed in ((1.0, 0), (0.5, 99)):
            plan = B.xeb_plan_create(big, big_bits, slices=[bonds[i] for i in (3, 17, 40, 55)])
            try:
                n_all = B.xeb_set_slice_subset(plan, frac, seed)
                lo, hi = D.shard_range(n_all, rank, world)
                n = B.xeb_set_slice_block(plan, lo, hi, frac, seed)
                mine = B.xeb_plan_slice_ids(plan, n)
                B.xeb_set_slice_subset(plan, frac, seed)
                want = B.xeb_plan_slice_ids(plan, n_all)
            finally:
                B.xeb_plan_destroy(plan)
            got = [None] * world
            dist.all_gather_object(got, [int(x) for x in mine])
            covers[frac] = (sorted(sum(got, [])), sorted(int(x) for x in want), sum(got, []) == [int(x) for x in want])
        # the partial amplitudes of this rank's block of the small plan's slices
        plan = B.xeb_plan_create(circ, bits, slices=SLICED)
        try:
            n_sl = B.xeb_set_slice_subset(plan, 1.0, 0)
            lo, hi = D.shard_range(n_sl, rank, world)
            n = B.xeb_set_slice_block(plan, lo, hi)
            values = B.xeb_plan_slice_ids(plan, n)
            _, sliced = B.xeb_plan_tree(plan)
        finally:
            B.xeb_plan_destroy(plan)
        part = _partial(network.fused_network(circ), bits, sliced, values)
        total = D.sum_partial_amplitudes(part, world)
        q.put((rank, m, total, covers))
    finally:
        dist.destroy_process_group()


def test_gloo_world2_slice_blocks_cover_and_sum():
    from paper_2108_05665_gb300 import inputs
    from oracle import statevec
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circ = inputs.random_grid_circuit(*CIRC)
    bits = inputs.uniform_bitstrings(6, 9, 32)
    want = statevec.amplitudes(circ, bits)
    for rank, m, total, covers in res:
        assert m == 4.0
        assert np.abs(total - want).max() < 1e-13
        for frac, (union, every, in_order) in covers.items():
            assert union == every and len(set(union)) == len(union), frac
            assert in_order   # blocks concatenate to the plan's own loop order
