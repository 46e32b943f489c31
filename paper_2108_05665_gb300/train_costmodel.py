"""Train the learned cost model on GB300 timings of the planner's own
candidates, then compare its choices with the plain planner's on held-out
circuits.

    python -m paper_2108_05665_gb300.train_costmodel --out costmodel_weights.npz \
        --summary summary.json [--train-circuits 60] [--eval-circuits 8] [--max-seconds 420]

Circuits are seeded random grid circuits (the family of the benchmark,
16-25 qubits so a step takes milliseconds); bitstrings are uniform.  Every
candidate of `xeb_plan_candidates` is bound and its captured step timed with
CUDA events; the target is log2 of the milliseconds.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding as B, build, inputs
from .costmodel import CostModel, choose, choose_verified, time_plan

SHAPES = [(4, 4), (4, 5), (5, 4), (3, 6), (4, 6), (5, 5), (3, 7)]


def circuit_spec(i, base_seed):
    rng = np.random.default_rng(base_seed + i)
    r, c = SHAPES[int(rng.integers(len(SHAPES)))]
    m = int(rng.choice([8, 10, 12, 14]))
    k = int(rng.choice([300, 1000, 3000]))
    prec = B.XEB_PREC_TF32X3 if rng.random() < 0.75 else B.XEB_PREC_FP32
    return r, c, m, k, prec, base_seed + 1000 + i


def make(spec):
    r, c, m, k, prec, seed = spec
    circ = inputs.random_grid_circuit(r, c, m, seed)
    bits = inputs.uniform_bitstrings(circ.n_qubits, k, seed + 7)
    o = B.xeb_default_opts()
    o.precision = prec
    return circ, bits, o


def measure_circuit(spec, max_cands, reps):
    circ, bits, o = make(spec)
    cands = B.xeb_plan_candidates(circ, bits, o, max_cands)
    feats, ms = [], []
    for c in cands:
        try:
            t = time_plan(circ, bits, c["tree"], c["slices"], o, reps=reps)
        except B.XebError:
            continue   # e.g. a candidate whose arena does not fit
        feats.append(c["features"])
        ms.append(t)
    return cands, np.array(feats), np.array(ms)


def evaluate(model, args):
    """Held-out circuits: measured time of the plain planner's plan, of the
    model's choice, of the verified choice (model's top 3 and the plain plan
    timed, fastest kept) and of the best measured candidate."""
    evals = []
    for j in range(args.eval_circuits):
        spec = circuit_spec(10000 + j, args.seed)
        circ, bits, o = make(spec)
        cands, f, ms = measure_circuit(spec, args.max_cands, args.reps)
        if not len(ms):
            continue
        plain = B.Plan(circ, bits, opts=o)
        plain_tree, plain_slices = plain.tree()
        plain.close()
        t_plain = time_plan(circ, bits, plain_tree, plain_slices, o, reps=args.reps)
        ch = choose(circ, bits, o, model, args.max_cands)
        t_model = time_plan(circ, bits, ch["tree"], ch["slices"], o, reps=args.reps)
        ver = choose_verified(circ, bits, o, model, top=3, max_cands=args.max_cands, reps=args.reps)
        t_ver = time_plan(circ, bits, ver["tree"], ver["slices"], o, reps=args.reps)
        p = model.predict(f)
        evals.append({"spec": list(spec), "n_cands": int(len(ms)), "plain_ms": t_plain, "model_ms": t_model,
                      "verified_ms": t_ver, "verified_source": ver["source"],
                      "best_ms": float(ms.min()), "median_ms": float(np.median(ms)),
                      "rank_corr": float(np.corrcoef(np.argsort(np.argsort(p)), np.argsort(np.argsort(ms)))[0, 1]),
                      "rmse_log2": float(np.sqrt(np.mean((p - np.log2(ms)) ** 2)))})
    return evals


def evaluate_workload(model, name, slice_count, reps, max_cands):
    """A benchmark workload (e.g. the 53-qubit sliced one): every candidate,
    the plain planner's plan, the model's choice and the verified choice,
    each timed on the same seeded subset of slice_count slices and scaled to
    the full sum over slices."""
    w = inputs.WORKLOADS[name]
    circ = w.circuit()
    bits = inputs.uniform_bitstrings(w.n_qubits, w.k, w.bitstring_seed)
    o = B.xeb_default_opts()
    o.precision = B.XEB_PREC_TF32X3
    t0 = time.time()
    plain = B.Plan(circ, bits, opts=o)
    plain_tree, plain_slices = plain.tree()
    plain.close()
    t_plan = time.time() - t0
    cands = B.xeb_plan_candidates(circ, bits, o, max_cands)
    ms = []
    for c in cands:
        try:
            ms.append(time_plan(circ, bits, c["tree"], c["slices"], o, reps=reps, slice_count=slice_count))
        except B.XebError:
            ms.append(float("nan"))
    ms = np.array(ms)
    pred = model.predict(np.array([c["features"] for c in cands])) if cands else np.array([])
    t_plain = time_plan(circ, bits, plain_tree, plain_slices, o, reps=reps, slice_count=slice_count)
    pick = int(np.argmin(pred)) if len(pred) else -1
    ver = choose_verified(circ, bits, o, model, top=3, max_cands=max_cands, reps=reps, slice_count=slice_count)
    return {"workload": name, "slice_count": slice_count, "plain_plan_seconds": t_plan, "n_cands": len(cands),
            "cand_ms": [float(x) for x in ms], "pred_log2_ms": [float(x) for x in pred], "plain_ms": t_plain,
            "model_ms": float(ms[pick]) if pick >= 0 else None, "verified_ms": ver["measured_ms"],
            "verified_source": ver["source"], "best_ms": float(np.nanmin(ms)) if len(ms) else None}


def geo_means(evals):
    def gm(a, b):
        return float(np.exp(np.mean([np.log(e[a] / e[b]) for e in evals]))) if evals else None
    return {"geo_mean_model_over_plain": gm("model_ms", "plain_ms"),
            "geo_mean_verified_over_plain": gm("verified_ms", "plain_ms"),
            "geo_mean_plain_over_best": gm("plain_ms", "best_ms"),
            "geo_mean_model_over_best": gm("model_ms", "best_ms"),
            "geo_mean_verified_over_best": gm("verified_ms", "best_ms")}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--summary", required=True)
    ap.add_argument("--train-circuits", type=int, default=60)
    ap.add_argument("--eval-circuits", type=int, default=8)
    ap.add_argument("--max-seconds", type=float, default=420.0)
    ap.add_argument("--max-cands", type=int, default=96)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--seed", type=int, default=5000)
    ap.add_argument("--eval-only", default=None, help="saved weights: skip data generation and training")
    ap.add_argument("--eval-workload", action="append", default=[],
                    help="also compare on this benchmark workload (inputs.WORKLOADS), sliced plans timed on a subset")
    ap.add_argument("--eval-slice-count", type=int, default=4)
    ap.add_argument("--max-samples", type=int, default=0, help="stop generating data after this many timed plans")
    ap.add_argument("--data-out", default=None, help="save the generated (features, log2 ms) pairs here")
    ap.add_argument("--data-in", default=None, help="train on saved pairs instead of generating them")
    args = ap.parse_args(argv)
    build.build()
    B.load()
    if args.eval_only:
        model = CostModel.load(args.eval_only)
        summary = {"weights": args.eval_only, "eval": evaluate(model, args)}
        summary.update(geo_means(summary["eval"]))
        summary["workloads"] = [evaluate_workload(model, n, args.eval_slice_count, args.reps, args.max_cands)
                                for n in args.eval_workload]
        with open(args.summary, "w") as fh:
            json.dump(summary, fh, indent=1)
        print(json.dumps({k: v for k, v in summary.items() if k != "eval"}))
        return
    t0 = time.time()
    if args.data_in:
        d = np.load(args.data_in)
        X, y, n_circ, t_data = d["X"], d["y"], int(d["n_circuits"]), float(d["seconds"])
    else:
        X, y, n_circ = [], [], 0
        for i in range(args.train_circuits):
            if time.time() - t0 > args.max_seconds or (args.max_samples and sum(len(v) for v in y) >= args.max_samples):
                break
            _, f, ms = measure_circuit(circuit_spec(i, args.seed), args.max_cands, args.reps)
            if len(ms):
                X.append(f)
                y.append(np.log2(ms))
                n_circ += 1
        X = np.concatenate(X)
        y = np.concatenate(y)
        t_data = time.time() - t0
        if args.data_out:
            np.savez(args.data_out, X=X, y=y, n_circuits=n_circ, seconds=t_data)
    model = CostModel(seed=1)
    hist = model.fit(X, y, epochs=args.epochs, batch=256, lr=1e-3)
    model.save(args.out, n_train=int(len(y)))
    pred = model.predict(X)
    train_rmse = float(np.sqrt(np.mean((pred - y) ** 2)))
    summary = {"train_circuits": n_circ, "train_samples": int(len(y)), "data_seconds": t_data,
               "epochs": args.epochs, "final_loss": hist[-1], "train_rmse_log2": train_rmse}
    with open(args.summary, "w") as fh:   # written before the (long) evaluation
        json.dump(summary, fh, indent=1)
    evals = evaluate(model, args)
    summary["eval"] = evals
    summary.update(geo_means(evals))
    summary["workloads"] = [evaluate_workload(model, n, args.eval_slice_count, args.reps, args.max_cands)
                            for n in args.eval_workload]
    with open(args.summary, "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k != "eval"}))


if __name__ == "__main__":
    main()
