"""Pins of the naive einsum contractor (against the state vector) and of the
linear XEB (Eq. 1) statistics: F ~ 0 for uniform bitstrings, F ~ 2^n sum p^2 - 1
(~1 under Porter-Thomas) for ideal samples, within 5 sigma (Fig. XEB's error
bars are +-5 sigma with sigma = 1/sqrt(k))."""
import math

import numpy as np

from paper_2108_05665_gb300 import inputs
from oracle import contract, network, statevec, xeb


def test_fused_network_contraction_matches_statevec():
    c = inputs.random_grid_circuit(3, 4, 8, 1001)
    net = network.fused_network(c)
    # structure of the fusion convention
    assert len(net.leaves) == sum(1 for g in c.gates if g.kind == 2)
    outs = sorted(q for l in net.leaves for q in l.out_qubits)
    assert outs == list(range(12))
    legs = [l for leaf in net.leaves for l in leaf.legs]
    assert sorted(legs) == sorted(list(range(net.n_legs)) * 2)
    bs = inputs.uniform_bitstrings(12, 24, 2001)
    want = statevec.amplitudes(c, bs)
    assert np.abs(contract.amplitudes(net, bs) - want).max() < 1e-13


def test_xeb_uniform_and_ideal():
    c = inputs.random_grid_circuit(4, 4, 12, 31)
    n = 16
    psi = statevec.state(c)
    s2, s4 = statevec.moments(psi)
    k = 20000
    uni = inputs.uniform_bitstrings(n, k, 41)
    f_u = xeb.fidelity(statevec.gather(psi, uni), n)
    assert abs(f_u) < 5 / math.sqrt(k)
    ideal = statevec.sample_ideal(psi, inputs.uniform_unit_draws(k, 51))
    f_i = xeb.fidelity(statevec.gather(psi, ideal), n)
    expect = 2 ** n * s4 - 1
    assert abs(expect - 1) < 0.1
    assert abs(f_i - expect) < 5 * math.sqrt(2 / k)
    mix = np.concatenate([ideal[: k // 2], uni[: k // 2]])
    f_m = xeb.fidelity(statevec.gather(psi, mix), n)
    assert abs(f_m - expect / 2) < 5 * math.sqrt(2 / k)


def test_xeb_closed_forms():
    # p = 2^-n for every bitstring -> F = 0; a single bitstring of p = 1 -> 2^n - 1
    n = 5
    a = np.full(7, 2 ** (-n / 2), dtype=np.complex128)
    assert abs(xeb.fidelity(a, n)) < 1e-15
    assert xeb.fidelity(np.array([1.0 + 0j]), n) == 2 ** n - 1
    # duplicates count every time (sum over the sequence)
    b = np.array([1.0, 0.0, 0.0, 0.0], dtype=np.complex128)
    assert xeb.fidelity(b, 2) == 0.0


def test_grid5x6_fixture_consistent():
    """The stored oracle values of the benchmark workload obey Eq. (1) and
    the statistics: half ideal samples, half uniform -> F ~ (2^n sum p^2 - 1)/2."""
    import os
    z = np.load(os.path.join(os.path.dirname(__file__), "golden", "grid5x6_m14_k10000.npz"))
    n, k = 30, len(z["bitstrings"])
    assert k == 10000
    assert abs(xeb.fidelity(z["amplitudes"], n) - float(z["F"])) < 1e-12
    assert abs(float(z["norm"]) - 1) < 1e-10
    assert abs(float(z["collision"]) - 2) < 0.01
    assert abs(float(z["F"]) - (float(z["collision"]) - 1) / 2) < 5 * math.sqrt(2 / k)
    uni = z["bitstrings"][5000:]
    w = inputs.WORKLOADS["grid5x6_m14_k10000"]
    assert np.array_equal(uni, inputs.uniform_bitstrings(n, 5000, w.bitstring_seed))
