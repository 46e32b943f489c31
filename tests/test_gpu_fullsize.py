"""Full-size parity on the 5x6-grid, 14-cycle, 10,000-bitstring workload (the
benchmark's), in the launch configuration bench.py times: every amplitude
against the FP64 state-vector oracle values stored by
tests/golden/make_grid5x6_fixture.py, and F against the oracle's F."""
import os

import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from gpu_util import rel_err, run

pytestmark = pytest.mark.gpu

FIX = os.path.join(os.path.dirname(__file__), "golden", "grid5x6_m14_k10000.npz")


@pytest.fixture(scope="module")
def fixture():
    build.build()
    z = np.load(FIX)
    w = inputs.WORKLOADS["grid5x6_m14_k10000"]
    return w.circuit(), np.asarray(z["bitstrings"], dtype=np.uint64), z["amplitudes"], float(z["F"])


@pytest.mark.parametrize("precision", [B.XEB_PREC_FP32, B.XEB_PREC_TF32X3])
def test_grid5x6_all_amplitudes(fixture, precision):
    circ, bits, ref, F_ref = fixture
    amps, F, plan = run(circ, bits, precision=precision)
    if precision == B.XEB_PREC_TF32X3:
        assert "gemm_tc" in plan.profile, plan.profile
    # the memo-trie levels (keyed, N = 1, K = 16) run on the keyed SIMT kernel
    assert plan.profile.get("gemm_keyed", {}).get("launches", 0) > 0, plan.profile
    # the default forms the measurements chose are the ones checked here: the
    # keyed SIMT kernel for single-key contractions, and (split-TF32 plan) two
    # result columns per thread for the K = 1, N = 64 streaming contraction
    forms = B.xeb_plan_profile_ops(plan.handle)
    single_keyed = [i for i, op in enumerate(forms)
                    if op["kernel"] == "gemm_keyed" and op["kv"] == 1]
    assert single_keyed, "no single-key contraction on the keyed kernel"
    if precision == B.XEB_PREC_TF32X3:
        wide = [i for i, op in enumerate(forms) if op["kernel"] == "gemm_stream" and op["K"] <= 4 and op["N"] >= 32]
        assert wide and all(B.xeb_plan_op_form(plan.handle, i)["cols_per_thread"] == 2 for i in wide)
    err = rel_err(amps, ref, circ.n_qubits)
    shrink = -np.mean(np.real(np.conj(ref) * (amps - ref))) / np.mean(np.abs(ref) ** 2)
    print("max rel err %.3e  median %.3e  mean shrink %.2e  |dF| %.3e"
          % (err.max(), np.median(err), shrink, abs(F - F_ref)))
    assert err.max() < 1e-5
    assert abs(F - F_ref) < 1e-6
    plan.close()
