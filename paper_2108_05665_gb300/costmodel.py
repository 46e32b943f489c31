"""Learned cost model of plans: the planner's candidates (tree, slice set)
described by XEB_N_FEATURES features, a small MLP (hand-written CUDA kernels
behind the C ABI) trained on measured GB300 step times, and the choice of the
candidate with the lowest predicted time.  Without a model the plain planner
(xeb_plan_create's own objective) decides.

Training data come from the planner itself: `xeb_plan_candidates` lists every
tree it would weigh with the slices its slicing step adds; `time_plan` binds
each candidate and times its captured step with CUDA events.
"""
from __future__ import annotations

import numpy as np

from . import binding as B

N_FEATURES = B.XEB_N_FEATURES


def time_plan(circ, bits, tree, slices, opts, reps=3, warmup=1, slice_count=None, slice_seed=12345):
    """Measured milliseconds of one step (key tables + contraction + XEB) of
    the plan with this tree and slice set, bitstrings already on the device.
    slice_count: run only that many slices (a seeded subset,
    xeb_set_slice_subset) and scale the time to the full sum over slices."""
    import torch
    plan = B.Plan(circ, bits, tree=tree, slices=slices or None, opts=opts).bind()
    try:
        scale = 1.0
        if slice_count:
            n_slices = plan.stats()["n_slices"]
            n_run = B.xeb_set_slice_subset(plan.handle, min(1.0, slice_count / n_slices), slice_seed)
            scale = n_slices / n_run
        stream = torch.cuda.current_stream()
        sp = stream.cuda_stream
        dev = torch.from_numpy(np.asarray(bits, dtype=np.uint64).view(np.int64).copy()).cuda()
        out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")

        def step():
            B.xeb_set_bitstrings(plan.handle, dev.data_ptr(), len(bits), sp)
            B.xeb_amplitudes(plan.handle, out.data_ptr(), sp)

        for _ in range(warmup):
            step()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * scale
    finally:
        plan.close()


class CostModel:
    """MLP from plan features to log2(step milliseconds), on the device."""

    def __init__(self, n_hidden=128, n_layers=3, seed=0):
        self.n_hidden, self.n_layers = n_hidden, n_layers
        self.mlp = B.Mlp(N_FEATURES, n_hidden, n_layers, seed)
        self.mean = np.zeros(N_FEATURES, np.float32)
        self.scale = np.ones(N_FEATURES, np.float32)

    def set_norm_from(self, X):
        X = np.asarray(X, np.float64)
        self.mean = X.mean(0).astype(np.float32)
        sd = X.std(0)
        self.scale = (1.0 / np.where(sd > 1e-6, sd, 1.0)).astype(np.float32)
        self.mlp.set_norm(self.mean, self.scale)

    def fit(self, X, y, epochs=300, batch=256, lr=1e-3, seed=0):
        """Adam on mean squared error of log2 time; returns the loss per epoch."""
        import torch
        X = np.asarray(X, np.float32)
        y = np.asarray(y, np.float32)
        self.set_norm_from(X)
        sp = torch.cuda.current_stream().cuda_stream
        Xd = torch.from_numpy(X).cuda()
        yd = torch.from_numpy(y).cuda()
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        rng = np.random.default_rng(seed)
        hist = []
        n = len(X)
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).cuda()
            loss.zero_()
            nb = 0
            for b0 in range(0, n, batch):
                idx = perm[b0:b0 + batch]
                xb = Xd[idx].contiguous()
                yb = yd[idx].contiguous()
                self.mlp.train_step(xb.data_ptr(), yb.data_ptr(), len(idx), lr, loss.data_ptr(), sp)
                nb += 1
            hist.append(float(loss.item()) / nb)
        return hist

    def predict(self, X):
        import torch
        X = np.ascontiguousarray(X, np.float32)
        sp = torch.cuda.current_stream().cuda_stream
        Xd = torch.from_numpy(X).cuda()
        yd = torch.empty(len(X), dtype=torch.float32, device="cuda")
        self.mlp.forward(Xd.data_ptr(), len(X), yd.data_ptr(), sp)
        return yd.cpu().numpy().astype(np.float64)

    def save(self, path, n_train=0):
        np.savez(path, weights=self.mlp.get_weights(), mean=self.mean, scale=self.scale,
                 n_hidden=self.n_hidden, n_layers=self.n_layers, n_train=n_train)

    @classmethod
    def load(cls, path, seed=0):
        d = np.load(path)
        m = cls(int(d["n_hidden"]), int(d["n_layers"]), seed)
        m.mlp.set_weights(d["weights"])
        m.mean, m.scale = d["mean"].astype(np.float32), d["scale"].astype(np.float32)
        m.mlp.set_norm(m.mean, m.scale)
        return m


def choose(circ, bits, opts=None, model=None, max_cands=256):
    """The candidate (dict with tree, slices, features) the model predicts
    fastest, or None (then the plain planner of xeb_plan_create decides)."""
    if model is None:
        return None
    cands = B.xeb_plan_candidates(circ, bits, opts, max_cands)
    if not cands:
        return None
    pred = model.predict(np.array([c["features"] for c in cands]))
    best = int(np.argmin(pred))
    c = dict(cands[best])
    c["predicted_log2_ms"] = float(pred[best])
    return c


def choose_verified(circ, bits, opts=None, model=None, top=3, max_cands=256, reps=3, slice_count=None):
    """The model proposes its `top` fastest-predicted candidates; they and the
    plain planner's plan are timed on the GPU and the fastest measured one is
    kept (so the result is never a plan the plain planner beats by more than
    timing noise).  Returns a dict with tree, slices, measured_ms and source
    ("model" or "plain")."""
    o = opts or B.xeb_default_opts()
    plain = B.Plan(circ, bits, opts=o)
    tree, slices = plain.tree()
    plain.close()
    best = {"tree": tree, "slices": slices, "source": "plain",
            "measured_ms": time_plan(circ, bits, tree, slices, o, reps=reps, slice_count=slice_count)}
    if model is None:
        return best
    cands = B.xeb_plan_candidates(circ, bits, o, max_cands)
    if not cands:
        return best
    pred = model.predict(np.array([c["features"] for c in cands]))
    for i in np.argsort(pred)[:top]:
        c = cands[int(i)]
        try:
            ms = time_plan(circ, bits, c["tree"], c["slices"], o, reps=reps, slice_count=slice_count)
        except B.XebError:
            continue
        if ms < best["measured_ms"]:
            best = {"tree": c["tree"], "slices": c["slices"], "source": "model", "measured_ms": ms,
                    "predicted_log2_ms": float(pred[int(i)])}
    return best
