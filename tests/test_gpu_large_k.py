"""Key tables and amplitudes beyond one CTA's key-table sort (k > 16,384):
the multi-CTA radix-sort path must give the oracle's key ids, child ids and
amplitudes exactly as the single-CTA path does."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, inputs
from oracle import memo, network, statevec, xeb
from gpu_util import rel_err, run

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
F_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


@pytest.fixture(scope="module")
def grid4x5_40k():
    circ = inputs.random_grid_circuit(4, 5, 10, 5151)
    # 40,000 draws over 2^20 values: ~760 duplicates; 9.8 tiles of 4,096
    bits = inputs.uniform_bitstrings(20, 40000, 5252)
    return circ, bits, statevec.amplitudes(circ, bits)


@pytest.mark.parametrize("planner", [B.XEB_PLANNER_GREEDY, B.XEB_PLANNER_SWEEP])
def test_large_k_key_tables_bit_exact(grid4x5_40k, planner):
    import torch
    circ, bits, ref = grid4x5_40k
    amps, F, plan = run(circ, bits, planner=planner)
    tree, _ = plan.tree()
    kt = memo.key_tables(network.fused_network(circ), tree, bits)
    st = torch.cuda.current_stream().cuda_stream
    for i in range(len(tree)):
        key, uL, uR = B.xeb_plan_keys(plan.handle, i, len(bits), kt["k"][i], st)
        assert np.array_equal(key, kt["key"][i]), i
        if kt["range"][i][1] > kt["range"][i][0]:
            assert np.array_equal(uL, kt["uL"][i]), i
            assert np.array_equal(uR, kt["uR"][i]), i
    assert rel_err(amps, ref, 20).max() < AMP_TOL
    assert abs(F - xeb.fidelity(ref, 20)) < F_TOL
    plan.close()


def test_large_k_graph_replay_and_permutation(grid4x5_40k):
    """The captured step (key tables included) replays on new bitstrings."""
    import torch
    circ, bits, ref = grid4x5_40k
    plan = B.Plan(circ, bits).bind()
    st = torch.cuda.current_stream().cuda_stream
    out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")
    perm = np.random.default_rng(11).permutation(len(bits))
    for b, r in ((bits, ref), (bits[perm], ref[perm])):
        dev = torch.from_numpy(np.asarray(b, dtype=np.uint64).view(np.int64).copy()).cuda()
        B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(b), st)
        B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
        B.xeb_fidelity(plan.handle, st)
        amps = out.cpu().numpy().view(np.complex128)
        assert rel_err(amps, r, 20).max() < AMP_TOL
    plan.close()
