"""Sliced plans from the local-search planner (App. A), the deep-K keyed
contraction kernel they use near the root, and seeded slice subsets.

* Slice subsets against the oracle: the partial sum over a seeded subset of
  slice values equals the oracle's sum over the same values (App. A,
  "Slicing": an amplitude is the sum over all values of the sliced legs).
* 40 qubits (5x8 grid, 12 cycles): all 200 bitstrings of
  tests/golden/make_grid5x8_fixture.py (FP64 oracle, one full contraction per
  bitstring) against a plan the annealer sliced to fit a small budget.
* The full 100,000-bitstring 40-qubit plan on a seeded subset of its slices:
  the partial sums of the 200 fixture bitstrings equal those of a plan over
  just those 200 with the same tree, slices and subset (a bitstring's partial
  sum does not depend on the other bitstrings sharing the memo tables).
"""
import os

import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import contract, network, xeb
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

FIX = os.path.join(os.path.dirname(__file__), "golden", "grid5x8_m12_k200.npz")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


def _amps(plan, bits, frac=None, seed=0):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    n_run = B.xeb_set_slice_subset(plan.handle, frac, seed) if frac is not None else None
    dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
    out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
    B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
    F = B.xeb_fidelity(plan.handle, st)[0]
    return out.cpu().numpy().view(np.complex128).copy(), F, n_run


@pytest.mark.parametrize("precision", [B.XEB_PREC_FP32, B.XEB_PREC_TF32X3])
def test_slice_subset_partial_sums_match_oracle(precision):
    circ = inputs.random_grid_circuit(3, 4, 8, 4545)
    bits = inputs.uniform_bitstrings(12, 60, 4646)
    net = network.fused_network(circ)
    bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
    sliced = [bonds[3], bonds[17], bonds[40], bonds[55]]
    o = B.xeb_default_opts()
    o.precision = precision
    plan = B.Plan(circ, bits, slices=sliced, opts=o).bind()
    full, _, _ = _amps(plan, bits)
    part, _, n_run = _amps(plan, bits, 0.25, 31)
    assert n_run == 4
    ids = B.xeb_plan_slice_ids(plan.handle, n_run)
    _, sl = plan.tree()
    assert list(sl) == sliced
    ref_part = contract.amplitudes(net, bits, sliced, values=[int(v) for v in ids])
    ref_full = contract.amplitudes(net, bits, sliced)
    scale = np.maximum(np.abs(ref_part), 2.0 ** (-12 / 2))
    assert (np.abs(part - ref_part) / scale).max() < 1e-5
    assert rel_err(full, ref_full, 12).max() < 1e-5
    again, _, _ = _amps(plan, bits, 1.0, 0)          # back to the full sum
    assert np.array_equal(again, full)
    plan.close()


def _fixture():
    z = np.load(FIX)
    w = inputs.WORKLOADS["grid5x8_m12_k100000"]
    return w, w.circuit(), np.asarray(z["bitstrings"], dtype=np.uint64), z["amplitudes"], float(z["F"])


@pytest.mark.parametrize("precision", [B.XEB_PREC_FP32, B.XEB_PREC_TF32X3])
def test_grid5x8_sliced_plan_matches_oracle(precision):
    w, circ, bits, ref, F_ref = _fixture()
    o = B.xeb_default_opts()
    o.precision = precision
    o.planner = B.XEB_PLANNER_ANNEAL
    o.mem_budget = 256 << 20                       # forces slicing
    plan = B.Plan(circ, bits, opts=o).bind()
    st = plan.stats()
    assert st["n_sliced"] >= 4 and st["arena_bytes"] <= o.mem_budget
    B.xeb_plan_profile(plan.handle, True)
    amps, F, _ = _amps(plan, bits)
    prof = B.xeb_plan_profile_read(plan.handle)
    B.xeb_plan_profile(plan.handle, False)
    print({k: (round(v["ms"], 2), v["launches"]) for k, v in prof.items()})
    # the near-root contractions of sliced plans (narrow results, deep sums)
    assert "gemm_kdeep" in prof, prof
    err = rel_err(amps, ref, 40)
    print("40q k=200: %d sliced legs, max rel err %.3e, |dF| %.3e" % (st["n_sliced"], err.max(), abs(F - F_ref)))
    assert err.max() < 1e-5
    assert abs(F - xeb.fidelity(ref, 40)) < 1e-6
    plan.close()


def test_grid5x8_full_plan_subset_is_memo_invariant():
    import torch
    w, circ, bits200, _, _ = _fixture()
    bits = inputs.uniform_bitstrings(40, w.k, w.bitstring_seed)
    assert np.array_equal(bits[:200], bits200)
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    o.planner = B.XEB_PLANNER_ANNEAL
    big = B.Plan(circ, bits, opts=o).bind()
    st = big.stats()
    assert 1 <= st["n_sliced"] <= 16, st["n_sliced"]
    frac = 4.0 / st["n_slices"]
    a_big, _, n_run = _amps(big, bits, frac, 77)
    ids = B.xeb_plan_slice_ids(big.handle, n_run)
    tree, sliced = big.tree()
    big.close()
    torch.cuda.empty_cache()
    small = B.Plan(circ, bits200, tree=tree, slices=list(sliced), opts=o).bind()
    a_small, _, n2 = _amps(small, bits200, frac, 77)
    assert n2 == n_run and np.array_equal(B.xeb_plan_slice_ids(small.handle, n2), ids)
    small.close()
    ref = a_small
    scale = np.maximum(np.abs(ref), np.sqrt(np.mean(np.abs(ref) ** 2)))
    d = np.abs(a_big[:200] - ref) / scale
    print("40q k=100000, %d of %d slices: max rel diff %.3e" % (n_run, st["n_slices"], d.max()))
    assert d.max() < 1e-5


@pytest.mark.parametrize("precision", [B.XEB_PREC_FP32, B.XEB_PREC_FP64])
def test_deep_sum_contractions_match_statevec(precision):
    """Trees whose contractions have narrow results over deep sums (the
    left/right halves of a 4x5 grid joined through their middle cut, the
    output leaves attached last) run the deep-K kernel; amplitudes against
    the FP64 state vector."""
    from oracle import statevec
    circ = inputs.random_grid_circuit(4, 5, 10, 5151)
    bits = inputs.uniform_bitstrings(20, 300, 5252)
    net = network.fused_network(circ)
    o = B.xeb_default_opts()
    o.precision = precision
    o.planner = B.XEB_PLANNER_ANNEAL
    o.mem_budget = 24 << 20
    from gpu_util import run
    amps, F, plan = run(circ, bits, precision=precision, opts=o)
    print({k: (round(v["ms"], 3), v["launches"]) for k, v in plan.profile.items()})
    ref = statevec.amplitudes(circ, bits)
    tol = 1e-5 if precision == B.XEB_PREC_FP32 else 1e-11
    assert rel_err(amps, ref, 20).max() < tol
    plan.close()


def test_grid6x9m1_split_precision_matches_fp64_on_gpu():
    """53 qubits (6x9 grid without its (0, 0) corner, 14 cycles): no CPU
    oracle reaches this size, so the TF32x3 result on a seeded slice of a
    sliced plan is checked against an FP64 recomputation on the GPU with the
    same tree, slices and slice (App. A, "Slicing": the partial sum over a
    fixed set of slice values is a well-defined quantity).  The first 1,000
    bitstrings of the 1,000,000-bitstring workload's generator."""
    import torch
    w = inputs.WORKLOADS["grid6x9m1_m14_k1000000"]
    circ = w.circuit()
    bits = inputs.uniform_bitstrings(53, w.k, w.bitstring_seed)[:1000]
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    o.mem_budget = 16 << 30
    plan = B.Plan(circ, bits, opts=o).bind()
    st = plan.stats()
    assert st["n_sliced"] >= 8 and st["arena_bytes"] <= o.mem_budget
    frac = 1.0 / st["n_slices"]
    a, _, n_run = _amps(plan, bits, frac, 2005)
    assert n_run == 1
    ids = B.xeb_plan_slice_ids(plan.handle, n_run)
    tree, sliced = plan.tree()
    plan.close()
    torch.cuda.empty_cache()
    o64 = B.xeb_default_opts()
    o64.precision = B.XEB_PREC_FP64
    o64.mem_budget = 64 << 30
    ref_plan = B.Plan(circ, bits, tree=tree, slices=list(sliced), opts=o64).bind()
    r, _, n2 = _amps(ref_plan, bits, frac, 2005)
    assert n2 == 1 and np.array_equal(B.xeb_plan_slice_ids(ref_plan.handle, n2), ids)
    ref_plan.close()
    scale = np.maximum(np.abs(r), np.sqrt(np.mean(np.abs(r) ** 2)))
    d = np.abs(a - r) / scale
    # mean relative shrink (a bias of the split arithmetic would show here)
    shrink = -np.mean(np.real(np.conj(r) * (a - r))) / np.mean(np.abs(r) ** 2)
    print("53q m=14, slice %d of %d: max rel diff %.3e, mean shrink %.2e" % (int(ids[0]), st["n_slices"], d.max(), shrink))
    assert np.all(np.isfinite(a)) and np.abs(r).max() > 0
    assert d.max() < 1e-5


@pytest.mark.parametrize("precision", [B.XEB_PREC_FP32, B.XEB_PREC_TF32X3])
def test_cross_slice_reuse_leaves_results_unchanged(precision):
    """Subtrees whose sliced legs did not change value since the previous
    slice keep their tensors instead of being contracted again; the full sum
    and a seeded partial sum are the same as with every contraction run in
    every slice (opts.reserved[7] = 1), and the full sum matches the FP64
    state vector."""
    from oracle import statevec
    circ = inputs.random_grid_circuit(4, 5, 10, 5353)
    bits = inputs.uniform_bitstrings(20, 400, 5454)
    out = {}
    for off in (0, 1):
        o = B.xeb_default_opts()
        o.precision = precision
        o.planner = B.XEB_PLANNER_ANNEAL
        o.mem_budget = 4 << 20                       # forces several sliced legs
        o.reserved[7] = off
        tree = slices = None
        if off == 1:
            tree, slices = out[0][3]
        plan = B.Plan(circ, bits, tree=tree, slices=list(slices) if slices is not None else None, opts=o).bind()
        st = plan.stats()
        full, F, _ = _amps(plan, bits)
        part, _, n_run = _amps(plan, bits, 0.5, 808)
        out[off] = (full, part, st, plan.tree())
        plan.close()
    st0 = out[0][2]
    print("reuse: %d sliced legs, %d nodes kept across slices" % (st0["n_sliced"], st0["n_reused"]))
    assert st0["n_sliced"] >= 2 and out[1][2]["n_reused"] == 0
    for a, b in ((out[0][0], out[1][0]), (out[0][1], out[1][1])):
        scale = np.sqrt(np.mean(np.abs(b) ** 2))
        assert np.abs(a - b).max() <= 1e-6 * scale
    ref = statevec.amplitudes(circ, bits)
    assert rel_err(out[0][0], ref, 20).max() < 1e-5


def test_deep_sum_few_rows_contraction_matches_statevec():
    """An annealed, sliced 3x6-grid plan whose tree holds an N = 1
    contraction with a deep sum over few rows (M = 4, K = 128): it runs one
    warp per output; the amplitudes match the FP64 state vector."""
    from oracle import statevec
    circ = inputs.random_grid_circuit(3, 6, 12, 12)
    bits = inputs.uniform_bitstrings(18, 300, 13)
    o = B.xeb_default_opts()
    o.planner = B.XEB_PLANNER_ANNEAL
    o.mem_budget = 4 << 20
    from gpu_util import run
    amps, F, plan = run(circ, bits, precision=B.XEB_PREC_FP32, opts=o)
    print({k: (round(v["ms"], 3), v["launches"]) for k, v in plan.profile.items()})
    assert "gemm_tail" in plan.profile
    ref = statevec.amplitudes(circ, bits)
    assert rel_err(amps, ref, 18).max() < 1e-5
    assert abs(F - xeb.fidelity(ref, 18)) < 1e-6
    plan.close()
