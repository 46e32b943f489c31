"""World-size-2 gloo tests (CPU) of the multi-process host logic: contiguous
sharding covers every unit exactly once, max-over-ranks timing, and the FP64
sum of slice-partitioned partial amplitudes equals the unsliced amplitudes
(slicing invariance, App. A "Slicing"), with the partials computed by the
oracle on CPU."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2108_05665_gb300 import inputs
        from oracle import network, contract
        D.barrier(world)
        m = D.max_over_ranks(float(rank * 3 + 1), world)
        circ = inputs.random_grid_circuit(2, 3, 5, 31)
        net = network.fused_network(circ)
        bits = inputs.uniform_bitstrings(6, 9, 32)
        sliced = [1, 4, 6]
        n_sl = 1 << len(sliced)
        lo, hi = D.shard_range(n_sl, rank, world)
        part = np.zeros(len(bits), dtype=np.complex128)
        for s in range(lo, hi):
            assign = {leg: (s >> t) & 1 for t, leg in enumerate(sliced)}
            # contract with the sliced legs fixed to this slice's values
            for i, w in enumerate(bits):
                from oracle.network import project_leaf, pair_contract
                items = [project_leaf(l, int(w), assign) for l in net.leaves]
                seq = contract.greedy_order([lg for _, lg in items])
                work = list(items)
                for a, b in seq:
                    r_ = pair_contract(work[a][0], work[a][1], work[b][0], work[b][1])
                    work = [x for t, x in enumerate(work) if t not in (a, b)] + [r_]
                part[i] += complex(work[0][0])
        total = D.sum_partial_amplitudes(part, world)
        q.put((rank, m, total))
    finally:
        dist.destroy_process_group()


def test_gloo_world2_max_and_slice_sum():
    from paper_2108_05665_gb300 import inputs
    from oracle import statevec
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circ = inputs.random_grid_circuit(2, 3, 5, 31)
    bits = inputs.uniform_bitstrings(6, 9, 32)
    want = statevec.amplitudes(circ, bits)
    for rank, m, total in res:
        assert m == 4.0
        assert np.abs(total - want).max() < 1e-13
