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


def test_sequence_cost_by_hand():
    # A(l0,l1) * B(l1,l2): 2^3 multiplications, result (l0,l2); then * C(l2): 2^2
    assert contract.sequence_cost([[0, 1], [1, 2], [2]], [(0, 1), (0, 1)]) == 8 + 4
    # a worse order: B * C first (2^2), then A * (B C): legs l0, l1 -> 2^2
    assert contract.sequence_cost([[0, 1], [1, 2], [2]], [(1, 2), (0, 1)]) == 4 + 4


def test_search_order_same_amplitudes_fewer_multiplications():
    circ = inputs.random_grid_circuit(3, 4, 10, 808)
    net = network.fused_network(circ)
    bits = inputs.uniform_bitstrings(12, 6, 809)
    legsets = [legs for _, legs in (network.project_leaf(l, 0) for l in net.leaves)]
    seq = contract.search_order(legsets, trials=24, seed=3)
    assert contract.sequence_cost(legsets, seq) <= contract.sequence_cost(legsets, contract.greedy_order(legsets))
    ref = statevec.amplitudes(circ, bits)
    assert np.abs(contract.amplitudes(net, bits, seq=seq) - ref).max() < 1e-12


def test_slice_value_subsets_partition_the_sum():
    circ = inputs.random_grid_circuit(3, 3, 6, 606)
    net = network.fused_network(circ)
    bits = inputs.uniform_bitstrings(9, 5, 607)
    bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
    sliced = [bonds[2], bonds[9], bonds[20]]
    part = contract.amplitudes(net, bits, sliced, values=[0, 3, 5])
    rest = contract.amplitudes(net, bits, sliced, values=[1, 2, 4, 6, 7])
    ref = statevec.amplitudes(circ, bits)
    assert np.abs(part + rest - ref).max() < 1e-12
    assert np.abs(part - ref).max() > 1e-6          # a subset alone is not the amplitude
