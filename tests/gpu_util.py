"""Helpers for GPU tests: run a plan through the C ABI on torch memory."""
import numpy as np

from paper_2108_05665_gb300 import binding as B


def rel_err(a, ref, n):
    """|a - ref| / max(|ref|, 2^(-n/2)) per amplitude (the 1e-5 criterion)."""
    return np.abs(a - ref) / np.maximum(np.abs(ref), 2.0 ** (-n / 2))


def run(circ, bits, tree=None, slices=None, precision=B.XEB_PREC_FP32, planner=None, opts=None):
    import torch
    o = opts or B.xeb_default_opts()
    o.precision = precision
    if planner is not None:
        o.planner = planner
    plan = B.Plan(circ, bits, tree=tree, slices=slices, opts=o).bind()
    st = torch.cuda.current_stream().cuda_stream
    k = len(bits)
    bits_dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
    out = torch.empty(2 * k, dtype=torch.float64, device="cuda")
    B.xeb_plan_profile(plan.handle, True)
    B.xeb_set_bitstrings(plan.handle, bits_dev.data_ptr(), k, st)
    B.xeb_amplitudes(plan.handle, out.data_ptr(), st)
    F, m1, m2 = B.xeb_fidelity(plan.handle, st)
    plan.profile = B.xeb_plan_profile_read(plan.handle)
    B.xeb_plan_profile(plan.handle, False)
    amps = out.cpu().numpy().view(np.complex128).copy()
    return amps, F, plan
