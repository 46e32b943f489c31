"""Write tests/golden/grid5x8_m12_k200.npz with the ORACLE only.

Workload: 5x8 grid (40 qubits), 12 cycles (circuit seed 1003); the first 200
of its 100,000 uniform bitstrings (seed 2003).  Stored: the bitstrings, their
FP64 amplitudes from the oracle's naive pairwise contractor (one full
contraction per bitstring, no memoization; a randomised-greedy merge order
found by the oracle's own search), and the linear XEB F (Eq. 1) over them.

Usage: python tests/golden/make_grid5x8_fixture.py [workers]
(about 30 s of one core per amplitude; workers default to the core count)
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "grid5x8_m12_k200.npz")
K = 200


def _setup():
    from paper_2108_05665_gb300 import inputs
    from oracle import network
    w = inputs.WORKLOADS["grid5x8_m12_k100000"]
    circ = w.circuit()
    net = network.fused_network(circ)
    bits = inputs.uniform_bitstrings(circ.n_qubits, w.k, w.bitstring_seed)[:K]
    return circ, net, bits


def _work(args):
    idx, seq = args
    _, net, bits = _setup()
    from oracle import contract
    return idx, contract.amplitudes(net, bits[idx:idx + 1], seq=seq)[0]


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    circ, net, bits = _setup()
    from oracle import contract, network, xeb
    t0 = time.time()
    legsets = [legs for _, legs in (network.project_leaf(l, 0) for l in net.leaves)]
    seq = contract.search_order(legsets, trials=128, seed=0)
    cost = contract.sequence_cost(legsets, seq)
    amps = np.zeros(K, dtype=np.complex128)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for idx, a in pool.imap_unordered(_work, [(i, seq) for i in range(K)]):
            amps[idx] = a
    F = xeb.fidelity(amps, circ.n_qubits)
    np.savez(OUT, bitstrings=bits, amplitudes=amps, F=F, order_multiplications=cost,
             oracle_seconds=time.time() - t0)
    print("wrote", OUT, "F=%.6f order cost %.3g, %.0f s" % (F, cost, time.time() - t0))


if __name__ == "__main__":
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    main()
