"""Slice blocks (App. A, "Slicing": the values of the sliced legs are
independent terms added at the end), the unit ranks share when they split one
sum over slices: the FP64 partial sums of blocks that tile the slice list add
up to the full sum, for all slice values and for a seeded subset, with the
blocks run one after the other on one GPU (the multi-rank path of bench.py
runs each block on its own rank and all-reduces the partials)."""
import numpy as np
import pytest

from paper_2108_05665_gb300 import binding as B, build, dist, inputs
from oracle import network, statevec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    build.build()
    B.load()


def _run(plan, bits):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
    out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")
    B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), st)
    B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
    return out.cpu().numpy().view(np.complex128).copy()


@pytest.mark.parametrize("precision,tol", [(B.XEB_PREC_FP64, 1e-11), (B.XEB_PREC_FP32, 1e-11)])
@pytest.mark.parametrize("world", [2, 3, 40])
def test_slice_blocks_sum_to_the_full_sum(precision, tol, world):
    circ = inputs.random_grid_circuit(3, 4, 8, 4545)
    bits = inputs.uniform_bitstrings(12, 60, 4646)
    net = network.fused_network(circ)
    bonds = sorted({l for leaf in net.leaves for l in leaf.legs})
    sliced = [bonds[i] for i in (3, 17, 29, 40, 55)]
    o = B.xeb_default_opts()
    o.precision = precision
    plan = B.Plan(circ, bits, slices=sliced, opts=o).bind()
    try:
        full = _run(plan, bits)
        n = B.xeb_set_slice_subset(plan.handle, 1.0, 0)
        total = np.zeros_like(full)
        for r in range(world):
            lo, hi = dist.shard_range(n, r, world)
            assert B.xeb_set_slice_block(plan.handle, lo, hi) == hi - lo
            part = _run(plan, bits)
            if hi == lo:
                assert np.all(part == 0)
            total += part
        scale = np.abs(full).max()
        assert np.abs(total - full).max() <= tol * scale
        if precision == B.XEB_PREC_FP64:
            ref = statevec.amplitudes(circ, bits)
            assert np.abs(total - ref).max() <= 1e-11 * np.abs(ref).max()
        # a seeded subset split into blocks sums to the subset's partial sum
        m = B.xeb_set_slice_subset(plan.handle, 0.5, 77)
        sub = _run(plan, bits)
        total = np.zeros_like(sub)
        for r in range(world):
            lo, hi = dist.shard_range(m, r, world)
            B.xeb_set_slice_block(plan.handle, lo, hi, 0.5, 77)
            total += _run(plan, bits)
        assert np.abs(total - sub).max() <= tol * np.abs(sub).max()
    finally:
        plan.close()
