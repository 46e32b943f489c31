"""Circuits and planner settings whose plans hold keyed contractions with
small results and a deep summed index (the form of tc_kdeep.cu), shared by
the host test that checks the plans still have that form and the GPU parity
test.  shape = (M, N, K, k_v) of the contraction, in complex elements."""
from paper_2108_05665_gb300 import binding as B

CASES = [
    dict(id="m32n16_k128", grid=(4, 6), cycles=12, k=5000, planner=B.XEB_PLANNER_GREEDY, budget=8 << 20,
         shape=(32, 16, 128, 256)),
    dict(id="m32n32_k512_tail", grid=(4, 6), cycles=14, k=5000, planner=B.XEB_PLANNER_GREEDY, budget=128 << 20,
         shape=(32, 32, 512, 4803)),
]


def plan_opts(case):
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    o.planner = case["planner"]
    o.mem_budget = case["budget"]
    return o


def deep_k_shapes(plan):
    """(M, N, K, k_v) of every keyed contraction of the plan with M, N in
    {16, 32}, 64 <= K <= 8192 a multiple of 64, both operands keyed."""
    st = plan.stats()
    L = st["n_leaves"]
    out = []
    for i in range(st["n_gemm_ops"] + st["n_permute_ops"]):
        lo = B.xeb_plan_op_layout(plan.handle, i)
        if lo["kind"] != 2 or lo["node"] < L or lo["a_node"] < L or lo["b_node"] < L:
            continue
        kv = B.xeb_plan_node(plan.handle, lo["node"] - L)["kv"]
        M, K, N = 2 ** len(lo["a_pos_m"]), 2 ** len(lo["a_pos_k"]), 2 ** len(lo["b_pos_n"])
        if kv >= 2 and M in (16, 32) and N in (16, 32) and 64 <= K <= 8192 and K % 64 == 0:
            out.append((M, N, K, kv))
    return out
