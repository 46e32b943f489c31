"""Deep-K keyed contractions on the tcgen05 split-precision kernel
(tc_kdeep.cu): C_u = A_uL(u) B_uR(u) per key u with small results and a deep
summed index (App. A, keyed contraction of the memo tables).  Each case is a
plan whose near-root contraction has that form: (32, 16) results (run as the
transposed product on the (16, 32) kernel), (32, 32) with a key count that is
not a multiple of the keys stacked per MMA.  Plans come from the greedy
planner, which gives the same tree on every host.  Amplitudes are compared with the FP64
state vector, F with the oracle's F."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import statevec, xeb
from gpu_util import rel_err, run
from kdeep_cases import CASES, plan_opts, deep_k_shapes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


@pytest.mark.parametrize("case", CASES, ids=[c["id"] for c in CASES])
def test_deep_k_tensor_core_matches_statevec(case):
    r, c = case["grid"]
    n = r * c
    circ = inputs.random_grid_circuit(r, c, case["cycles"], 4242)
    bits = inputs.uniform_bitstrings(n, case["k"], 4343)
    ref = statevec.amplitudes(circ, bits)
    F_ref = xeb.fidelity(ref, n)
    amps, F, plan = run(circ, bits, precision=B.XEB_PREC_TF32X3, opts=plan_opts(case))
    assert case["shape"] in deep_k_shapes(plan)
    kd = plan.profile.get("gemm_tc_kdeep", {"launches": 0, "ms": 0.0})
    err = rel_err(amps, ref, n)
    print("%s: deep-K tensor-core launches %d (%.3f ms), max rel err %.2e, |dF| %.2e"
          % (case["id"], kd["launches"], kd["ms"], err.max(), abs(F - F_ref)))
    assert kd["launches"] >= 1, plan.profile
    assert err.max() < 1e-5
    assert abs(F - F_ref) < 1e-6
    plan.close()
