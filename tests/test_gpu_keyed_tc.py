"""Keyed contractions (k_v > 1 keys, C_u = A_uL(u) B_uR(u), Eq. (elem-cont)
evaluated once per key of the memo tables) on the tcgen05 3xTF32 kernel:
with the keyed tensor-core form on (opts.reserved[6] = 1) and off the amplitudes
match the FP64 state vector, and the form moves those contractions onto the
tensor cores."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import statevec, xeb
from gpu_util import rel_err, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


@pytest.mark.parametrize("rows,cols,budget", [(4, 5, None), (4, 6, None), (4, 5, 16 << 20)])
def test_keyed_tensor_core_form_matches_statevec(rows, cols, budget):
    n = rows * cols
    circ = inputs.random_grid_circuit(rows, cols, 10, 4242)
    bits = inputs.uniform_bitstrings(n, 2000, 4343)
    ref = statevec.amplitudes(circ, bits)
    F_ref = xeb.fidelity(ref, n)
    res = {}
    for off in (0, 1):
        o = B.xeb_default_opts()
        o.planner = B.XEB_PLANNER_GREEDY     # its trees hold keyed 128+-row contractions
        if budget:
            o.mem_budget = budget
        o.reserved[6] = 1 - off
        amps, F, plan = run(circ, bits, precision=B.XEB_PREC_TF32X3, opts=o)
        tc = plan.profile.get("gemm_tc", {"launches": 0, "ms": 0.0})
        res[off] = (amps, F, tc["launches"])
        print("%dx%d keyed form %s: tc launches %d (%.3f ms), max rel err %.2e, |dF| %.2e" % (
            rows, cols, "off" if off else "on", tc["launches"], tc["ms"], rel_err(amps, ref, n).max(), abs(F - F_ref)))
        plan.close()
    assert res[0][2] > res[1][2]
    for amps, F, _ in res.values():
        assert rel_err(amps, ref, n).max() < 1e-5
        assert abs(F - F_ref) < 1e-6
