"""Memo-trie levels as grouped tensor-core GEMMs (one GEMM per left-key group,
its keys as the columns) against the FP64 oracle and against the SIMT
memo-level kernel on the same plan."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import statevec, xeb
from gpu_util import rel_err, run

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
TF32_F_TOL = 1e-6   # absolute, on the same bitstrings


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


@pytest.fixture(scope="module")
def grid4x6():
    # the planner's tree for this circuit has a memo level of 16 groups x
    # 16 keys with 65,536 rows each
    circ = inputs.random_grid_circuit(4, 6, 12, 77)
    bits = inputs.uniform_bitstrings(24, 2000, 78)
    return circ, bits, statevec.amplitudes(circ, bits)


def test_grouped_memo_levels(grid4x6):
    circ, bits, ref = grid4x6
    res = {}
    for simt in (1, 0):
        o = B.xeb_default_opts()
        o.reserved[4] = 1 - simt   # 1: grouped tensor-core form
        amps, F, plan = run(circ, bits, precision=B.XEB_PREC_TF32X3, opts=o)
        st = plan.stats()
        res[simt] = (amps, F, st["n_tc_launches"])
        print("simt memo %d: tc launches %d, max rel err %.2e, F %.6f" %
              (simt, st["n_tc_launches"], rel_err(amps, ref, 24).max(), F))
        assert rel_err(amps, ref, 24).max() < AMP_TOL
        assert abs(F - xeb.fidelity(ref, 24)) < TF32_F_TOL
        plan.close()
    assert res[0][2] == res[1][2] + 1   # the memo level ran as one grouped tensor-core launch


def test_autotuned_plan_keeps_parity(grid4x6):
    """The autotuner times every kernel form of every contraction and keeps
    the fastest; the tuned plan must still meet the oracle bound."""
    import torch
    circ, bits, ref = grid4x6
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    plan = B.Plan(circ, bits, opts=o).bind()
    st = torch.cuda.current_stream().cuda_stream
    dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
    changed = B.xeb_plan_autotune(plan.handle, 2, st)
    print("autotune changed %d contractions" % changed)
    out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
    B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
    F = B.xeb_fidelity(plan.handle, st)[0]
    amps = out.cpu().numpy().view(np.complex128)
    assert rel_err(amps, ref, 24).max() < AMP_TOL
    assert abs(F - xeb.fidelity(ref, 24)) < TF32_F_TOL
    plan.close()
