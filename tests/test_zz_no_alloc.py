"""The allocation-free linear XEB entry point (xeb_linear_xeb_noalloc).

Some callers cannot allocate device memory: a process whose device memory
belongs to its own pool allocator, or a latency-critical caller that cannot
take the device synchronisation an allocation implies.  For them the library
offers a linear XEB over amplitudes already on the device whose scratch is a
fixed array inside the library.  This test checks, through the C ABI:

* on the amplitudes of a plan (k = 1,000, one block of partial sums) it gives
  the plan's own XEB (xeb_fidelity) and the oracle's Eq. (1) and moments
  computed on the host from the same amplitudes, on two calls in a row (the
  second call finds the first call's partial sums in the shared array);
* on 123,457 seeded amplitudes (31 blocks, a ragged last block) the block
  partials and their cross-block sum give the oracle's values;
* a call allocates nothing: after a first call (which may load the library's
  kernels), further calls leave the device's free memory and torch's
  allocations unchanged;
* k beyond the fixed array's limit is refused.

The file sorts last, so a run that stops at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import xeb

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def _close(got, want):
    return np.all(np.abs(np.asarray(got) - np.asarray(want)) <= FP64_TOL * np.maximum(1.0, np.abs(want)))


def _oracle(amps, n):
    m1, m2 = xeb.moments(amps, n)
    return np.array([xeb.fidelity(amps, n), m1, m2])


def test_noalloc_xeb_matches_plan_and_oracle_twice():
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
    host = amps.cpu().numpy().view(np.complex128)
    ref = _oracle(host, circ.n_qubits)
    assert _close(want, ref)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        B.xeb_linear_xeb_noalloc(amps.data_ptr(), k, circ.n_qubits, out.data_ptr(), st)
        got = out.cpu().numpy()
        assert _close(got, want), (got, want)
        assert _close(got, ref), (got, ref)
    with pytest.raises(B.XebError) as e:
        B.xeb_linear_xeb_noalloc(amps.data_ptr(), 16777217, circ.n_qubits, out.data_ptr(), st)
    assert e.value.status == 1
    plan.close()


def test_noalloc_xeb_many_blocks_and_allocates_nothing():
    import torch
    build.build()
    B.load()
    n, k = 24, 123457
    rng = np.random.default_rng(2024)
    host = (rng.standard_normal(k) + 1j * rng.standard_normal(k)) * 2.0 ** (-(n + 1) / 2)
    ref = _oracle(host, n)
    st = torch.cuda.current_stream().cuda_stream
    amps = torch.from_numpy(host.view(np.float64).copy()).cuda()
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    # first call: may load the library's kernels and look up the array's address
    B.xeb_linear_xeb_noalloc(amps.data_ptr(), k, n, out.data_ptr(), st)
    torch.cuda.synchronize()
    assert _close(out.cpu().numpy(), ref)
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        out.fill_(float("nan"))
        B.xeb_linear_xeb_noalloc(amps.data_ptr(), k, n, out.data_ptr(), st)
        got = out.cpu().numpy()
        assert _close(got, ref), (got, ref)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
