"""Write tests/golden/grid5x6_m14_k10000.npz with the ORACLE only.

Workload: 5x6 grid, 14 cycles (circuit seed 1002); 10,000 bitstrings = 5,000
drawn from the ideal output distribution |<x|C|0^n>|^2 by inverse CDF
(uniform draws seed 3002) followed by 5,000 uniform ones (seed 2002).
Stored: the bitstrings, their FP64 amplitudes from the state-vector oracle,
the oracle's linear XEB F (Eq. 1) over the sequence and 2^n sum p^2.

Usage: python tests/golden/make_grid5x6_fixture.py   (needs ~17 GB RAM)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_2108_05665_gb300 import inputs  # noqa: E402
from oracle import statevec, xeb  # noqa: E402

OUT = os.path.join(HERE, "grid5x6_m14_k10000.npz")


def main():
    w = inputs.WORKLOADS["grid5x6_m14_k10000"]
    circ = w.circuit()
    n = circ.n_qubits
    t0 = time.time()
    psi = statevec.state(circ)
    t_sv = time.time() - t0
    s2, s4 = statevec.moments(psi)
    n_ideal = int(round(w.k * w.ideal_fraction))
    ideal = statevec.sample_ideal(psi, inputs.uniform_unit_draws(n_ideal, w.ideal_seed))
    uni = inputs.uniform_bitstrings(n, w.k - n_ideal, w.bitstring_seed)
    bits = np.concatenate([ideal, uni]).astype(np.uint64)
    amps = statevec.gather(psi, bits)
    F = xeb.fidelity(amps, n)
    np.savez(OUT, bitstrings=bits, amplitudes=amps, F=F, collision=2.0 ** n * s4, norm=s2,
             statevec_seconds=t_sv)
    print("wrote", OUT, "F=%.6f 2^n sum p^2=%.4f norm-1=%.2e sv %.0fs" % (F, 2.0 ** n * s4, s2 - 1, t_sv))


if __name__ == "__main__":
    main()
