"""Parity of the CUDA path against the FP64 oracle (element by element on the
same seeded inputs), bit-exact memo key tables, slicing, duplicates and the
end-to-end host entry point."""
import math

import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import memo, network, statevec, xeb
from _trees import random_tree
from gpu_util import rel_err, run

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5      # |a - a_ref| <= 1e-5 max(|a_ref|, 2^(-n/2))
F_TOL = 1e-6        # absolute, on the same bitstrings
FP64_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


@pytest.fixture(scope="module")
def cfg1():
    w = inputs.WORKLOADS["grid3x4_m8_k1000"]
    circ = w.circuit()
    bits = inputs.uniform_bitstrings(circ.n_qubits, w.k, w.bitstring_seed)
    ref = statevec.amplitudes(circ, bits)
    return circ, bits, ref


@pytest.mark.parametrize("planner", [B.XEB_PLANNER_GREEDY, B.XEB_PLANNER_SWEEP, B.XEB_PLANNER_AUTO])
def test_grid3x4_fp32_amplitudes_and_fidelity(cfg1, planner):
    circ, bits, ref = cfg1
    amps, F, plan = run(circ, bits, planner=planner)
    n = circ.n_qubits
    assert rel_err(amps, ref, n).max() < AMP_TOL
    assert abs(F - xeb.fidelity(ref, n)) < F_TOL
    plan.close()


def test_grid3x4_fp64_amplitudes(cfg1):
    circ, bits, ref = cfg1
    amps, F, plan = run(circ, bits, precision=B.XEB_PREC_FP64)
    assert np.abs(amps - ref).max() < FP64_TOL
    assert abs(F - xeb.fidelity(ref, circ.n_qubits)) < 1e-10
    plan.close()


@pytest.mark.parametrize("planner", [B.XEB_PLANNER_GREEDY, B.XEB_PLANNER_SWEEP])
def test_key_tables_bit_exact(cfg1, planner):
    circ, bits, _ = cfg1
    _, _, plan = run(circ, bits, planner=planner)
    tree, _ = plan.tree()
    kt = memo.key_tables(network.fused_network(circ), tree, bits)
    import torch
    st = torch.cuda.current_stream().cuda_stream
    for i in range(len(tree)):
        kv = kt["k"][i]
        key, uL, uR = B.xeb_plan_keys(plan.handle, i, len(bits), kv, st)
        assert np.array_equal(key, kt["key"][i]), i
        if kt["range"][i][1] > kt["range"][i][0]:
            assert np.array_equal(uL, kt["uL"][i]), i
            assert np.array_equal(uR, kt["uR"][i]), i
    plan.close()


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_trees_fp64(seed):
    circ = inputs.random_grid_circuit(3, 3, 6, 600 + seed)
    bits = inputs.uniform_bitstrings(9, 150, 700 + seed)
    net = network.fused_network(circ)
    tree = random_tree([l.legs for l in net.leaves], seed)
    ref = statevec.amplitudes(circ, bits)
    amps, _, plan = run(circ, bits, tree=tree, precision=B.XEB_PREC_FP64)
    assert np.abs(amps - ref).max() < FP64_TOL
    amps32, _, plan32 = run(circ, bits, tree=tree)
    assert rel_err(amps32, ref, 9).max() < AMP_TOL
    plan.close()
    plan32.close()


def test_slicing_invariance(cfg1):
    circ, bits, ref = cfg1
    net = network.fused_network(circ)
    sliced = [3, 17, 29, 40]
    tree = random_tree([l.legs for l in net.leaves], 11, sliced=sliced)
    amps, F, plan = run(circ, bits, tree=tree, slices=sliced, precision=B.XEB_PREC_FP64)
    assert plan.stats()["n_slices"] == 16
    assert np.abs(amps - ref).max() < FP64_TOL
    amps32, F32, plan32 = run(circ, bits, tree=tree, slices=sliced)
    assert rel_err(amps32, ref, circ.n_qubits).max() < AMP_TOL
    plan.close()
    plan32.close()


def test_duplicates_ragged_and_single(cfg1):
    circ, bits, ref = cfg1
    n = circ.n_qubits
    rng = np.random.default_rng(3)
    idx = rng.integers(0, 37, size=53)
    b2 = bits[:37][idx]                     # duplicates, ragged k
    amps, F, plan = run(circ, b2)
    assert rel_err(amps, ref[:37][idx], n).max() < AMP_TOL
    assert abs(F - xeb.fidelity(ref[:37][idx], n)) < F_TOL
    assert plan.stats()["k_distinct"] == len(np.unique(b2))
    plan.close()
    amps1, _, plan1 = run(circ, bits[:1])
    assert rel_err(amps1, ref[:1], n).max() < AMP_TOL
    plan1.close()


def test_worked_example_circuit():
    # App. B circuit: H q0, T q2, CNOT q0->q1, CNOT q1->q2, H q0, H q1;
    # <s|C|000> = 2^(-3/2) (s2 = 0) and 2^(-3/2) (-1)^(s0+s1) (s2 = 1)
    gates = [inputs.Gate(1, (0,), network.H_GATE), inputs.Gate(1, (2,), network.T_GATE),
             inputs.Gate(2, (0, 1), network.CNOT), inputs.Gate(2, (1, 2), network.CNOT),
             inputs.Gate(1, (0,), network.H_GATE), inputs.Gate(1, (1,), network.H_GATE)]
    circ = inputs.Circuit(3, gates)
    bits = np.array([0, 1, 7, 4, 5, 2], dtype=np.uint64)
    closed = np.array([(1 if (b >> 2) & 1 == 0 else (-1) ** ((b & 1) + ((b >> 1) & 1))) / (2 * math.sqrt(2))
                       for b in (int(x) for x in bits)])
    amps, F, plan = run(circ, bits, precision=B.XEB_PREC_FP64)
    assert np.abs(amps - closed).max() < 1e-15
    plan.close()


def test_end_to_end_host_entry(cfg1):
    import torch
    circ, bits, ref = cfg1
    o = B.xeb_default_opts()
    plan = B.Plan(circ, bits, opts=o).bind()
    hb = torch.from_numpy(bits.view(np.int64).copy()).pin_memory()
    ha = torch.empty(2 * len(bits), dtype=torch.float64).pin_memory()
    F = B.xeb_run(plan.handle, hb.data_ptr(), len(bits), ha.data_ptr(), torch.cuda.current_stream().cuda_stream)
    amps = ha.numpy().view(np.complex128)
    assert rel_err(amps, ref, circ.n_qubits).max() < AMP_TOL
    assert abs(F - xeb.fidelity(ref, circ.n_qubits)) < F_TOL
    # a second run reuses the plan and gives identical results
    F2 = B.xeb_run(plan.handle, hb.data_ptr(), len(bits), ha.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert F2 == F
    plan.close()


def test_mismatched_bitstrings_flagged(cfg1):
    import torch
    circ, bits, _ = cfg1
    plan = B.Plan(circ, bits).bind()
    other = inputs.uniform_bitstrings(circ.n_qubits, len(bits), 99)
    dev = torch.from_numpy(other.view(np.int64).copy()).cuda()
    st = torch.cuda.current_stream().cuda_stream
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
    B.xeb_amplitudes(plan.handle, 0, st)
    with pytest.raises(B.XebError) as e:
        B.xeb_fidelity(plan.handle, st)
    assert e.value.status == 7
    plan.close()


@pytest.fixture(scope="module")
def grid4x5():
    circ = inputs.random_grid_circuit(4, 5, 12, 4242)
    bits = inputs.uniform_bitstrings(20, 700, 4343)
    return circ, bits, statevec.amplitudes(circ, bits)


@pytest.mark.parametrize("planner,block", [(B.XEB_PLANNER_SWEEP, 6), (B.XEB_PLANNER_SWEEP, 5),
                                           (B.XEB_PLANNER_SWEEP, 4), (B.XEB_PLANNER_AUTO, 0)])
def test_tf32x3_tensor_core_parity(grid4x5, planner, block):
    """3xTF32 tcgen05 contractions against the FP64 oracle: the tensor-core
    kernel must actually run (M = 2^13..2^16 rows, K, N = 16..64), amplitudes
    within 1e-5 and F within 1e-6 on the same bitstrings."""
    circ, bits, ref = grid4x5
    o = B.xeb_default_opts()
    o.block_qubits = block
    amps, F, plan = run(circ, bits, precision=B.XEB_PREC_TF32X3, planner=planner, opts=o)
    err = rel_err(amps, ref, 20)
    shrink = -np.mean(np.real(np.conj(ref) * (amps - ref))) / np.mean(np.abs(ref) ** 2)
    print("tf32x3 block %d: max rel err %.2e, mean shrink %.2e, |dF| %.2e, tc launches %s"
          % (block, err.max(), shrink, abs(F - xeb.fidelity(ref, 20)), plan.profile.get("gemm_tc")))
    if planner == B.XEB_PLANNER_SWEEP:
        assert plan.profile.get("gemm_tc", {}).get("launches", 0) > 0
    assert err.max() < AMP_TOL
    assert abs(F - xeb.fidelity(ref, 20)) < F_TOL
    plan.close()


@pytest.mark.parametrize("bits,terms", [(11, 4), (11, 3)])
def test_tf32x3_split_options(grid4x5, bits, terms):
    """The split options reach the kernel: with 11-bit big parts the split
    carries at least as many bits as the default one, so the amplitudes meet
    1e-5.  (F is not asserted here: an 11-bit grid lets big*big sums pass
    2^24 grid units, where the tensor cores truncate; that bias is what the
    default 10-bit grid avoids.)"""
    circ, bits_, ref = grid4x5
    o = B.xeb_default_opts()
    o.block_qubits = 6
    o.split_bits, o.split_terms = bits, terms
    amps, F, plan = run(circ, bits_, precision=B.XEB_PREC_TF32X3, planner=B.XEB_PLANNER_SWEEP, opts=o)
    err = rel_err(amps, ref, 20)
    print("split bits %d terms %d: max rel err %.2e, |dF| %.2e" % (bits, terms, err.max(),
                                                                  abs(F - xeb.fidelity(ref, 20))))
    assert plan.profile.get("gemm_tc", {}).get("launches", 0) > 0
    assert err.max() < AMP_TOL
    plan.close()


@pytest.mark.parametrize("block", [6, 5])
def test_tf32x3_tma_matches_gather(grid4x5, block):
    """Tensor-core contractions whose A operand is a row-major matrix load it
    with TMA boxes; the plain-load gather path builds the same shared-memory
    operands, so both give identical bits (and both meet the oracle bound)."""
    import torch
    circ, bits, ref = grid4x5
    res = {}
    for gather in (0, 1):
        o = B.xeb_default_opts()
        o.block_qubits = block
        o.reserved[3] = gather
        amps, F, plan = run(circ, bits, precision=B.XEB_PREC_TF32X3, planner=B.XEB_PLANNER_SWEEP, opts=o)
        st = plan.stats()
        print("block %d gather %d: tc launches %d, tma %d" % (block, gather, st["n_tc_launches"], st["n_tc_tma"]))
        if gather:
            assert st["n_tc_tma"] == 0
        else:
            assert st["n_tc_tma"] > 0
        assert rel_err(amps, ref, 20).max() < AMP_TOL
        res[gather] = (amps, F)
        plan.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
