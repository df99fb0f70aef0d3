"""Learned warm start for the lid-driven cavity (orchestration over the C ABI).

1. Steady states: the solver (FP32 storage) runs each cavity until the mean
   per-step velocity change over the check interval k,
   ||u^n - u^(n-k)|| / (k ||u^n||), is <= tol (lbm_run_to_steady).
   With ``continuation`` the Reynolds numbers are visited in increasing order
   and each run starts from the previous steady state (faster data generation;
   the targets are still the converged states).
2. Training: the network (lbm_cnn_*) learns Re -> (rho, u); one Adam step per
   steady state, cosine learning-rate schedule.
3. Evaluation: for held-out Reynolds numbers, wall time and steps to the
   residual from rest (cold) and from the network's prediction (warm;
   inference time included).  The solver judges the network: the report
   gives, per case, the prediction's relative L2 error against the cold run's
   converged fields and the relative L2 difference between the warm and cold
   runs' final fields (u, and rho - 1 against its own norm).
4. Weights: ``save_weights``/``load_weights`` keep a trained network in an
   ``.npz`` file (FP32 master weights plus the training recipe).

Every numerical step runs in the CUDA library; this module only sequences the
calls.  ``python -m paper_2010_01628_gb300.surrogate --n 128 ...`` runs the
whole study and writes a JSON report.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time

import numpy as np

from . import binding as L
from . import inputs

LID = 0.1


def cavity_omega(n, reynolds):
    nu = LID * n / reynolds
    return 1.0 / (3.0 * nu + 0.5)


def _cavity(n, reynolds, precision="fp32"):
    return L.lbm_create((n, n, n), cavity_omega(n, reynolds), periodic=(False, False, False), lid_u=(LID, 0.0, 0.0),
                        precision=precision)


def steady_states(n, re_list, tol=1e-6, check_every=100, max_steps=400_000, continuation=True, precision="fp32",
                  log=None):
    """Converged steady states (dicts with re, rho, u on the GPU, steps,
    residual, seconds), in increasing Re.  Runs that do not reach `tol` within
    `max_steps` are reported with ``converged`` False; the caller decides."""
    import torch
    out = []
    prev = None
    for k in np.argsort(re_list):
        re = float(re_list[k])
        ctx = _cavity(n, re, precision)
        try:
            if continuation and prev is not None:
                L.lbm_init_fields(ctx, prev[0], prev[1])
            t = time.perf_counter()
            steps, res = L.lbm_run_to_steady(ctx, max_steps, check_every, tol)
            dt = time.perf_counter() - t
            rho = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
            u = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
            L.lbm_fields(ctx, (n, n, n), rho=rho, u=u)
        finally:
            L.lbm_destroy(ctx)
        ok = 0 <= res <= tol
        if ok:
            prev = (rho, u)
        out.append({"re": re, "rho": rho, "u": u, "steps": steps, "residual": res, "seconds": dt, "converged": ok})
        if log:
            log(f"steady Re={re:7.1f} steps={steps} residual={res:.2e} {dt:.2f}s")
    return out


def train(n, data, epochs, lr, seed=0, net=None, log=None):
    if net is None:
        net = L.lbm_cnn_create((n, n, n))
    rng = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs)))
        tot = 0.0
        for i in rng.permutation(len(data)):
            d = data[i]
            L.lbm_cnn_set_input(net, d["re"])
            tot += L.lbm_cnn_train_step(net, d["rho"], d["u"], lr_ep)
        history.append(tot / len(data))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4e} lr {lr_ep:.2e}")
    train.history = history
    return net


def _fields(ctx, n):
    import torch
    rho = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    u = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    L.lbm_fields(ctx, (n, n, n), rho=rho, u=u)
    return rho, u


def _run(n, re, tol, check_every, max_steps, net=None, keep_fields=False):
    """Steps, residual and wall seconds to the steady residual from rest
    (net None) or from the network's prediction (inference inside the timed
    region); with keep_fields, also the final (rho, u) on the GPU."""
    import torch
    ctx = _cavity(n, re)
    fields = None
    try:
        torch.cuda.synchronize()
        t = time.perf_counter()
        if net is not None:
            L.lbm_cnn_warm_start(net, ctx, re)
        steps, res = L.lbm_run_to_steady(ctx, max_steps, check_every, tol)
        dt = time.perf_counter() - t
        if keep_fields:
            fields = _fields(ctx, n)
    finally:
        L.lbm_destroy(ctx)
    return steps, res, dt, fields


def prediction(net, n, re):
    """The network's (rho, u) for `re` as the solver sees it: a context
    initialised by lbm_cnn_warm_start, read back before any step."""
    ctx = _cavity(n, re)
    try:
        L.lbm_cnn_warm_start(net, ctx, re)
        return _fields(ctx, n)
    finally:
        L.lbm_destroy(ctx)


def _rel(a, b, ref):
    import torch
    d = float(torch.linalg.vector_norm(a - b))
    r = float(torch.linalg.vector_norm(ref))
    return d / r if r > 0 else d


def judge(pred, cold, warm):
    """Relative L2 errors: the prediction against the cold run's converged
    fields, and the warm run's final fields against the cold run's (u against
    ||u_cold||, rho against ||rho_cold - 1||)."""
    (rp, up), (rc, uc), (rw, uw) = pred, cold, warm
    drc = rc - 1.0
    return {"net_err_u": _rel(up, uc, uc), "net_err_rho": _rel(rp, rc, drc),
            "warm_vs_cold_u": _rel(uw, uc, uc), "warm_vs_cold_rho": _rel(rw, rc, drc)}


def evaluate(net, n, re_list, tol=1e-6, check_every=100, max_steps=400_000, log=None, judged=True):
    cases = []
    for re in re_list:
        re = float(re)
        cs, cr, ct, cf = _run(n, re, tol, check_every, max_steps, keep_fields=judged)
        ws, wr, wt, wf = _run(n, re, tol, check_every, max_steps, net, keep_fields=judged)
        case = {"re": re, "cold_steps": cs, "cold_seconds": ct, "cold_residual": cr, "warm_steps": ws,
                "warm_seconds": wt, "warm_residual": wr}
        if judged:
            case.update(judge(prediction(net, n, re), cf, wf))
            del cf, wf
        cases.append(case)
        if log:
            extra = (f" | net err u {case['net_err_u']:.2e} warm-cold u {case['warm_vs_cold_u']:.2e}"
                     if judged else "")
            log(f"Re={re:7.1f} cold {cs} steps {ct:.2f}s | warm {ws} steps {wt:.2f}s{extra}")
    cold = [c["cold_seconds"] for c in cases]
    warm = [c["warm_seconds"] for c in cases]
    rep = {"cases": cases, "cold_mean_s": statistics.mean(cold), "warm_mean_s": statistics.mean(warm),
           "cold_median_s": statistics.median(cold), "warm_median_s": statistics.median(warm),
           "mean_time_reduction": 1.0 - statistics.mean(warm) / statistics.mean(cold),
           "median_time_reduction": 1.0 - statistics.median(warm) / statistics.median(cold),
           "cold_mean_steps": statistics.mean(c["cold_steps"] for c in cases),
           "warm_mean_steps": statistics.mean(c["warm_steps"] for c in cases)}
    if judged:
        for k in ("net_err_u", "net_err_rho", "warm_vs_cold_u", "warm_vs_cold_rho"):
            rep[k + "_max"] = max(c[k] for c in cases)
            rep[k + "_median"] = statistics.median(c[k] for c in cases)
    return rep


def save_weights(net, path, **meta):
    """Write the network's FP32 master weights and `meta` (the training
    recipe) to an .npz file."""
    w = L.lbm_cnn_get_weights(net)
    np.savez_compressed(path, weights=w, meta=json.dumps(meta))


def load_weights(path):
    """(FP32 weights, meta dict) from an .npz file written by save_weights;
    the parameter count must match the library's network."""
    with np.load(path) as z:
        w = np.ascontiguousarray(z["weights"], dtype=np.float32)
        meta = json.loads(str(z["meta"]))
    if w.size != L.lbm_cnn_param_count():
        raise ValueError(f"{path}: {w.size} parameters, the network has {L.lbm_cnn_param_count()}")
    return w, meta


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--heldout", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--max-steps", type=int, default=400_000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-weights", default=None, help="write the trained network to this .npz file")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)

    def log(msg):
        print(msg, flush=True)

    res = inputs.cavity_reynolds(args.train + args.heldout, seed=4)
    train_re, held_re = res[:args.train], res[args.train:]
    t0 = time.perf_counter()
    all_states = steady_states(args.n, train_re, args.tol, args.check_every, max_steps=args.max_steps, log=log)
    data = [d for d in all_states if d["converged"]]
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    net = train(args.n, data, args.epochs, args.lr, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if args.save_weights:
        save_weights(net, args.save_weights, grid=args.n, train_states=len(data), epochs=args.epochs, lr=args.lr,
                     tol=args.tol, check_every=args.check_every, reynolds_seed=4, train_count=args.train,
                     heldout_count=args.heldout)
    rep = evaluate(net, args.n, held_re, args.tol, args.check_every, max_steps=args.max_steps, log=log)
    L.lbm_cnn_destroy(net)
    rep.update({"grid": args.n, "train_states": len(data), "heldout": len(held_re), "epochs": args.epochs,
                "lr": args.lr, "tol": args.tol, "check_every": args.check_every,
                "data_generation_s": t_data, "training_s": t_train, "loss_history": train.history,
                "data_steps_total": int(sum(d["steps"] for d in all_states)),
                "unconverged_training_states": [d["re"] for d in all_states if not d["converged"]]})
    txt = json.dumps(rep, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(txt)
    print(json.dumps({k: v for k, v in rep.items() if k not in ("cases", "loss_history")}), flush=True)


if __name__ == "__main__":
    main()
