"""Multi-batch plans (Sec. "Multi-batch simulator"): the output legs of w
chosen qubits stay uncontracted, so each input bitstring stands for the batch
of 2^w bitstrings that share its other bits, and the CUDA path returns all
2^w amplitudes of every batch.  Reference: the FP64 state vector read at the
expanded bitstrings (an independent construction: no tensor network), and
Eq. (1) over the k 2^w bitstrings."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import statevec, xeb
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

AMP_TOL = {B.XEB_PREC_FP32: 1e-5, B.XEB_PREC_TF32X3: 1e-5, B.XEB_PREC_FP64: 1e-11}
# 3xTF32: the tensor cores' truncating FP32 accumulation biases F (see the
# TF32 parity tests); FP32 meets the 1e-6 target
F_TOL = {B.XEB_PREC_FP32: 1e-6, B.XEB_PREC_TF32X3: 1e-6, B.XEB_PREC_FP64: 1e-11}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


def expand(bits, open_q):
    """[k][2^w] bitstrings: bitstring i with open qubit j (ascending) set to bit j of x."""
    qs = sorted(open_q)
    mask = np.uint64(sum(1 << q for q in qs))
    out = np.empty((len(bits), 1 << len(qs)), dtype=np.uint64)
    for x in range(1 << len(qs)):
        v = sum(1 << q for j, q in enumerate(qs) if (x >> j) & 1)
        out[:, x] = (np.asarray(bits, dtype=np.uint64) & ~mask) | np.uint64(v)
    return out


def run_batched(circ, bits, open_q, precision, opts=None):
    import torch
    o = opts or B.xeb_default_opts()
    o.precision = precision
    plan = B.Plan(circ, bits, opts=o, open_qubits=open_q).bind()
    k, w = len(bits), len(open_q)
    st = torch.cuda.current_stream().cuda_stream
    dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
    out = torch.empty(2 * (k << w), dtype=torch.float64, device="cuda")
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), k, st)
    B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
    F = B.xeb_fidelity(plan.handle, st)[0]
    return out.cpu().numpy().view(np.complex128).reshape(k, 1 << w).copy(), F, plan


@pytest.mark.parametrize("precision", [B.XEB_PREC_FP32, B.XEB_PREC_TF32X3, B.XEB_PREC_FP64])
def test_batches_match_statevec(precision):
    circ = inputs.random_grid_circuit(4, 5, 10, 6161)
    bits = inputs.uniform_bitstrings(20, 300, 6262)
    open_q = [13, 0, 19, 7]                      # any order: bit j of x is the j-th smallest
    bits[7] = bits[3] ^ np.uint64(1 << 13)       # differs from bitstring 3 only in an open bit
    amps, F, plan = run_batched(circ, bits, open_q, precision)
    exp = expand(bits, open_q)
    ref = statevec.amplitudes(circ, exp.reshape(-1)).reshape(exp.shape)
    err = rel_err(amps, ref, 20)
    print("batched w=4 precision %d: max rel err %.2e, |dF| %.2e" % (precision, err.max(),
                                                                     abs(F - xeb.fidelity(ref.reshape(-1), 20))))
    assert err.max() < AMP_TOL[precision]
    assert np.array_equal(amps[7], amps[3])       # the same batch
    assert abs(F - xeb.fidelity(ref.reshape(-1), 20)) < F_TOL[precision]
    plan.close()


def test_sliced_batched_plan_matches_statevec():
    """A batched plan the annealer slices to fit a small budget: the sum over
    slice values still gives every batch amplitude."""
    circ = inputs.random_grid_circuit(4, 5, 10, 7171)
    bits = inputs.uniform_bitstrings(20, 200, 7272)
    open_q = [2, 11, 17]
    o = B.xeb_default_opts()
    o.planner = B.XEB_PLANNER_ANNEAL
    o.mem_budget = 4 << 20                        # the unsliced plan needs ~20 MB
    amps, F, plan = run_batched(circ, bits, open_q, B.XEB_PREC_FP32, o)
    st = plan.stats()
    assert st["n_sliced"] >= 2 and st["arena_bytes"] <= o.mem_budget
    exp = expand(bits, open_q)
    ref = statevec.amplitudes(circ, exp.reshape(-1)).reshape(exp.shape)
    assert rel_err(amps, ref, 20).max() < 1e-5
    assert abs(F - xeb.fidelity(ref.reshape(-1), 20)) < 1e-6
    plan.close()


def test_xeb_run_returns_every_batch_to_host():
    import torch
    circ = inputs.random_grid_circuit(3, 4, 8, 8181)
    bits = inputs.uniform_bitstrings(12, 100, 8282)
    open_q = [4, 9]
    plan = B.Plan(circ, bits, opts=B.xeb_default_opts(), open_qubits=open_q).bind()
    k = len(bits)
    hb = torch.from_numpy(bits.view(np.int64).copy()).pin_memory()
    ha = torch.zeros(2 * (k << 2), dtype=torch.float64).pin_memory()
    F = B.xeb_run(plan.handle, hb.data_ptr(), k, ha.data_ptr(), torch.cuda.current_stream().cuda_stream)
    amps = ha.numpy().view(np.complex128).reshape(k, 4)
    exp = expand(bits, open_q)
    ref = statevec.amplitudes(circ, exp.reshape(-1)).reshape(exp.shape)
    assert rel_err(amps, ref, 12).max() < 1e-5
    assert abs(F - xeb.fidelity(ref.reshape(-1), 12)) < 1e-6
    plan.close()
