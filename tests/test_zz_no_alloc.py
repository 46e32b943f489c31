"""The allocation-free linear XEB entry point (xeb_linear_xeb_noalloc).

Some callers cannot allocate device memory: a process whose device memory
belongs to its own pool allocator, or a latency-critical caller that cannot
take the device synchronisation an allocation implies.  For them the library
offers a linear XEB over amplitudes already on the device whose scratch is a
fixed array inside the library.  This test checks, through the C ABI, that it
gives the same F and moments as the plan's own XEB (xeb_fidelity) on the same
amplitudes, on two calls in a row (the second call finds the first call's
partial sums in the shared array), and that it rejects k beyond its limit.
"""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def test_noalloc_xeb_matches_plan_xeb_twice():
    import torch
    build.build()
    B.load()
    w = inputs.WORKLOADS["grid3x4_m8_k1000"]
    circ = w.circuit()
    bits = inputs.uniform_bitstrings(circ.n_qubits, w.k, w.bitstring_seed)
    k = len(bits)
    plan = B.Plan(circ, bits).bind()
    st = torch.cuda.current_stream().cuda_stream
    dev_bits = torch.from_numpy(bits.view(np.int64).copy()).cuda()
    amps = torch.empty(2 * k, dtype=torch.float64, device="cuda")
    B.xeb_set_bitstrings(plan.handle, dev_bits.data_ptr(), k, st)
    B.xeb_amplitudes(plan.handle, amps.data_ptr(), st)
    want = np.array(B.xeb_fidelity(plan.handle, st))
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        B.xeb_linear_xeb_noalloc(amps.data_ptr(), k, circ.n_qubits, out.data_ptr(), st)
        got = out.cpu().numpy()
        assert np.all(np.abs(got - want) <= FP64_TOL * np.maximum(1.0, np.abs(want))), (got, want)
    with pytest.raises(B.XebError) as e:
        B.xeb_linear_xeb_noalloc(amps.data_ptr(), 16777217, circ.n_qubits, out.data_ptr(), st)
    assert e.value.status == 1
    plan.close()
