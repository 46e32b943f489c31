"""Streamed evaluation in the lexicographic order of Alg. 4
(xeb_run_chunked): the bitstrings are sorted by their bits in the tree's
order and contracted a chunk at a time with one tree and slice set.  The
amplitudes (input order, duplicates included) and Eq. (1) must not depend on
the chunking: checked against the FP64 state vector and against one plan
over all bitstrings."""
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


@pytest.mark.parametrize("precision,chunk", [(B.XEB_PREC_FP32, 700), (B.XEB_PREC_FP32, 1), (B.XEB_PREC_TF32X3, 1024)])
def test_chunked_matches_statevec_and_one_plan(precision, chunk):
    circ = inputs.random_grid_circuit(4, 5, 10, 9191)
    bits = inputs.uniform_bitstrings(20, 3000 if chunk > 1 else 60, 9292)
    bits[5] = bits[11]                                   # a duplicate
    ref = statevec.amplitudes(circ, bits)
    o = B.xeb_default_opts()
    o.precision = precision
    amps, F, m1, m2 = B.xeb_run_chunked(circ, bits, chunk, opts=o)
    err = rel_err(amps, ref, 20)
    F_ref = xeb.fidelity(ref, 20)
    print("chunk %d precision %d: max rel err %.2e, |dF| %.2e" % (chunk, precision, err.max(), abs(F - F_ref)))
    assert err.max() < 1e-5
    assert amps[5] == amps[11]
    assert abs(F - F_ref) < 1e-6
    assert abs(m1 - (F + 1)) < 1e-12
    p = np.abs(ref) ** 2 * 2.0 ** 20
    assert abs(m2 - np.mean(p ** 2)) < 1e-4 * np.mean(p ** 2)
    _, F1, plan = run(circ, bits, precision=precision, opts=o)
    plan.close()
    assert abs(F - F1) < 1e-6
