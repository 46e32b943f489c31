"""Bounded device waits: a wait that runs out makes the step fail with
XEB_ETIMEOUT, quickly and with the GPU context still usable, and the plan's
next step is correct again.

The tensor-core kernel's threads hand work to one another through mbarriers;
every wait on one gives up after opts.timeout_ms, records the timeout in the
plan's error word and leaves its loop (copies in flight drained, MMAs
finished, tensor memory freed).  xeb_plan_test_wait makes each tensor-core
contraction first wait on a barrier that nothing completes, so that wait runs
out; no GPU fault, trap or endless loop is involved."""
import time

import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import statevec, xeb
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_returns_timeout_and_plan_recovers():
    import torch
    build.build()
    B.load()
    circ = inputs.random_grid_circuit(4, 5, 12, 4242)
    bits = inputs.uniform_bitstrings(20, 700, 4343)
    ref = statevec.amplitudes(circ, bits)
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    o.planner = B.XEB_PLANNER_SWEEP
    o.block_qubits = 6
    o.timeout_ms = 20
    plan = B.Plan(circ, bits, opts=o).bind()
    st = torch.cuda.current_stream().cuda_stream
    dev = torch.from_numpy(bits.view(np.int64).copy()).cuda()
    out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")

    def step():
        B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
        B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
        return B.xeb_fidelity(plan.handle, st)[0]

    assert plan.stats()["n_tc_launches"] > 0
    step()
    B.xeb_plan_test_wait(plan.handle, True)
    t0 = time.perf_counter()
    with pytest.raises(B.XebError) as e:
        step()
    elapsed = time.perf_counter() - t0
    assert e.value.status == 4, e.value   # XEB_ETIMEOUT
    assert elapsed < 5.0, elapsed         # the waits ran out after ~20 ms, not the 2 s default
    B.xeb_plan_test_wait(plan.handle, False)
    F = step()
    amps = out.cpu().numpy().view(np.complex128)
    assert rel_err(amps, ref, 20).max() < 1e-5
    assert abs(F - xeb.fidelity(ref, 20)) < 1e-6
    plan.close()
