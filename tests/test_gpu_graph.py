"""The captured-graph step against the kernel-by-kernel step: same kernels,
same inputs, so identical bits; a replay after new bitstrings were copied in
must read them (a permutation of the plan's bitstrings keeps its counts)."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import statevec, xeb
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


def _step(plan, bits, out, st):
    import torch
    dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
    B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
    F = B.xeb_fidelity(plan.handle, st)[0]
    return out.cpu().numpy().view(np.complex128).copy(), F


@pytest.mark.parametrize("precision,slices", [(B.XEB_PREC_FP32, None), (B.XEB_PREC_TF32X3, None),
                                              (B.XEB_PREC_FP64, [2, 3])])
def test_graph_replay_matches_eager(precision, slices):
    import torch
    circ = inputs.random_grid_circuit(4, 5, 12, 4242)
    bits = inputs.uniform_bitstrings(20, 700, 4343)
    ref = statevec.amplitudes(circ, bits)
    st = torch.cuda.current_stream().cuda_stream
    res = {}
    for eager in (1, 0):
        o = B.xeb_default_opts()
        o.precision = precision
        o.reserved[2] = eager
        plan = B.Plan(circ, bits, slices=slices, opts=o).bind()
        out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")
        a1, F1 = _step(plan, bits, out, st)
        a2, F2 = _step(plan, bits, out, st)          # graph: replay
        assert np.array_equal(a1, a2) and F1 == F2
        perm = np.random.default_rng(7).permutation(len(bits))
        a3, F3 = _step(plan, bits[perm], out, st)   # new bitstrings, same counts
        assert rel_err(a3, ref[perm], 20).max() < 1e-5
        assert abs(F3 - F1) < 1e-9
        out2 = torch.empty_like(out)                 # another output buffer
        a4, _ = _step(plan, bits, out2, st)
        assert np.array_equal(a4, a1)
        res[eager] = (a1, F1)
        plan.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
    assert rel_err(res[0][0], ref, 20).max() < 1e-5
    assert abs(res[0][1] - xeb.fidelity(ref, 20)) < 1e-6
