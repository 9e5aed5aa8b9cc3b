"""Training of the warm-start network on systems the solver generates and solves itself.

For every training seed a synthetic system of the c4 shape (50,000 stars x
200 observations, 2,000 attitude knots per axis, 500 instrumental unknowns,
sinusoid attitude) is generated on the device and solved by plain LSQR to a
tight tolerance; the pair (features of the system, attitude part of its
solution) is one training example. The network predicts the correction of
the Jacobi estimate in feature units:
    target = x_att / scale - features[:, 0:3].
Training uses the library's own kernels (gsr_net_train_step: BF16 tensor-core
forward and backward, Adam on fp32 master weights). Evaluation counts, on
held-out seeds, the LSQR iterations needed to bring every block within 1e-9
of a tightly converged reference, from x0 = 0, from the Jacobi start and from
the learned start.

    python -m paper_2308_00778_gb300.train --out paper_2308_00778_gb300/weights/warmstart.bin

The shipped network can also be evaluated, without training, on held-out systems of another
shape, e.g. the combined-at-scale configuration's (60,000 knots per axis, 20,000 instrumental
unknowns, 250 observations per star) with fewer stars:

    python -m paper_2308_00778_gb300.train --evaluate-only --shape 80000,250,60000,20000 \
        --eval-seeds 500:505 --eval-out paper_2308_00778_gb300/weights/eval_60000_knots.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

import gsrgen

from . import gsr as g
from .data import device_system, new_context

TOL = 1e-9
SHAPE = dict(n_stars=50_000, obs=200, n_dfa=2000, n_instr=500)


def cfg_for(seed: int, shape=None):
    sh = dict(SHAPE if shape is None else shape)
    return gsrgen.make_cfg(seed, sh["n_stars"], sh["obs"], sh["n_dfa"], sh["n_instr"], att_kind=1)


def block_ranges(cfg):
    a = 5 * cfg.n_stars
    t = a + 3 * cfg.n_dfa
    i = t + cfg.n_instr
    return {"astro": (0, a), "att": (a, t), "instr": (t, i), "glob": (i, i + cfg.n_glob)}


def max_block_err(x, ref, cfg) -> float:
    worst = 0.0
    for a, z in block_ranges(cfg).values():
        if z > a:
            num = torch.linalg.vector_norm(x[a:z] - ref[a:z]).item()
            worst = max(worst, num / max(torch.linalg.vector_norm(ref[a:z]).item(), 1e-3))
    return worst


def example(ctx, cfg, device, damp=1e-6):
    """(features [n_dfa, 6], target [n_dfa, 3], x_ref) of the system loaded in ctx."""
    L = cfg.n_dfa
    f = torch.zeros((L, 6), dtype=torch.float32, device=device)
    scale = ctx.warm_features(f)
    x = torch.zeros(cfg.ncols(), dtype=torch.float64, device=device)
    ctx.solve(x, itnlim=5000, atol=1e-14, btol=1e-14, conlim=0.0, damp=damp)
    a0 = 5 * cfg.n_stars
    att = x[a0:a0 + 3 * L].view(3, L).t().float()
    target = att / scale - f[:, :3]
    return f, target, x


def make_dataset(seeds, fp32=True, shape=None, device=None, log=None):
    device = device or torch.device("cuda", 0)
    X, Y = [], []
    ctx = None
    t0 = time.time()
    for i, seed in enumerate(seeds):
        cfg = cfg_for(seed, shape)
        ctx, _, _ = device_system(cfg, fp32, True, device, ctx=ctx)
        f, t, _ = example(ctx, cfg, device)
        X.append(f)
        Y.append(t)
        if log and (i % 20 == 0 or i == len(seeds) - 1):
            log(f"  example {i + 1}/{len(seeds)} (seed {seed}) {time.time() - t0:.1f}s")
    if ctx is not None:
        ctx.close()
    return torch.stack(X), torch.stack(Y)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases; the last layer scaled by 0.1 (start near the Jacobi estimate)."""
    rng = np.random.default_rng(seed)
    chans = [6, 64, 64, 64, 64, 64, 3]
    parts = []
    for i, (ci, co) in enumerate(zip(chans[:-1], chans[1:])):
        W = rng.standard_normal((co, ci, 5)) * np.sqrt(2.0 / (5 * ci))
        if i == len(chans) - 2:
            W *= 0.1
        parts += [W.ravel(), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def train(X, Y, steps=1500, batch=16, lr=2e-3, lr_min=5e-5, seed=0, log=None, Xv=None, Yv=None):
    net = g.Net()
    net.set_params(init_params(seed))
    rng = np.random.default_rng(seed + 1)
    n = X.shape[0]
    hist = []
    for step in range(steps):
        idx = torch.tensor(rng.choice(n, size=min(batch, n), replace=False), device=X.device)
        cur = lr_min + 0.5 * (lr - lr_min) * (1 + np.cos(np.pi * step / steps))
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), float(cur))
        if step % 100 == 0 or step == steps - 1:
            entry = {"step": step, "lr": cur, "train_loss": loss}
            if Xv is not None:
                entry["val_loss"] = validation_loss(net, Xv, Yv)
            hist.append(entry)
            if log:
                log(f"  step {step} " + " ".join(f"{k} {v:.4g}" for k, v in entry.items() if k != "step"))
    return net, hist


def validation_loss(net, Xv, Yv) -> float:
    out = torch.empty(Yv.shape, dtype=torch.float32, device=Xv.device)
    net.forward(Xv.contiguous(), out)
    torch.cuda.synchronize()
    return float(((out - Yv) ** 2).mean())


def iterations_to_tol(ctx, cfg, x_ref, device, damp=1e-6, **warm):
    """Smallest LSQR iteration count reaching TOL per block from the given start."""
    x = torch.zeros(cfg.ncols(), dtype=torch.float64, device=device)

    def err(k):
        ctx.solve(x, itnlim=k, atol=0.0, btol=0.0, conlim=0.0, damp=damp, **warm)
        torch.cuda.synchronize()
        return max_block_err(x, x_ref, cfg)

    hi = 4
    while err(hi) > TOL and hi < 400:
        hi *= 2
    lo = hi // 2 if hi > 4 else 0
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if err(mid) <= TOL:
            hi = mid
        else:
            lo = mid
    return hi


def evaluate(weights_path, seeds, fp32=True, shape=None, device=None, log=None):
    """Per held-out seed: iterations to TOL from cold / Jacobi / learned starts."""
    device = device or torch.device("cuda", 0)
    rows = []
    ctx = None
    for seed in seeds:
        cfg = cfg_for(seed, shape)
        ctx, _, _ = device_system(cfg, fp32, True, device, ctx=ctx)
        xr = torch.zeros(cfg.ncols(), dtype=torch.float64, device=device)
        ctx.solve(xr, itnlim=5000, atol=1e-15, btol=1e-15, conlim=0.0, damp=1e-6)
        r = {"seed": seed,
             "cold": iterations_to_tol(ctx, cfg, xr, device),
             "jacobi": iterations_to_tol(ctx, cfg, xr, device, warm=g.GSR_WARM_JACOBI),
             "learned": iterations_to_tol(ctx, cfg, xr, device, warm=g.GSR_WARM_LEARNED,
                                          weights_path=str(weights_path))}
        # how close each start is to the solution
        for name, kw in (("jacobi", dict(warm=g.GSR_WARM_JACOBI)),
                         ("learned", dict(warm=g.GSR_WARM_LEARNED, weights_path=str(weights_path)))):
            x0 = torch.zeros(cfg.ncols(), dtype=torch.float64, device=device)
            net = None
            if name == "learned":
                net = g.Net()
                net.load(weights_path)
            ctx.warm_start(x0, net)
            if net is not None:
                net.close()
            r[f"x0_err_{name}"] = max_block_err(x0, xr, cfg)
            for blk, (a, z) in block_ranges(cfg).items():
                num = torch.linalg.vector_norm(x0[a:z] - xr[a:z]).item()
                r[f"x0_err_{name}_{blk}"] = num / max(torch.linalg.vector_norm(xr[a:z]).item(), 1e-3)
        rows.append(r)
        if log:
            log(f"  held-out seed {seed}: {r}")
    if ctx is not None:
        ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "weights", "warmstart.bin"))
    ap.add_argument("--train-seeds", default="100:300")
    ap.add_argument("--eval-seeds", default="300:320")
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--evaluate-only", action="store_true",
                    help="evaluate the weights at --out on the held-out seeds, without training")
    ap.add_argument("--shape", default=None,
                    help="n_stars,obs,n_dfa,n_instr of the evaluation systems (default: the training shape)")
    ap.add_argument("--eval-out", default=None, help="--evaluate-only: where to write the record (JSON)")
    args = ap.parse_args()
    a, b = map(int, args.train_seeds.split(":"))
    ea, eb = map(int, args.eval_seeds.split(":"))
    log = lambda m: print(m, flush=True)  # noqa: E731
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.evaluate_only:
        shape = SHAPE
        if args.shape:
            ns, ob, nd, ni = map(int, args.shape.split(","))
            shape = dict(n_stars=ns, obs=ob, n_dfa=nd, n_instr=ni)
        rows = evaluate(args.out, range(ea, eb), shape=shape, device=dev, log=log)
        rec = {"weights": os.path.relpath(args.out, os.path.dirname(os.path.dirname(os.path.abspath(__file__)))),
               "shape": shape, "fp32_storage": True, "eval_seeds": [ea, eb], "tolerance": TOL, "evaluation": rows,
               "mean_iterations": {k: float(np.mean([r[k] for r in rows])) for k in ("cold", "jacobi", "learned")}}
        if args.eval_out:
            with open(args.eval_out, "w") as f:
                json.dump(rec, f, indent=1)
        log(json.dumps(rec["mean_iterations"]))
        return
    t0 = time.time()
    log(f"training examples: seeds {a}..{b - 1}")
    X, Y = make_dataset(range(a, b), device=dev, log=log)
    log(f"validation examples: seeds {ea}..{eb - 1}")
    Xv, Yv = make_dataset(range(ea, eb), device=dev, log=log)
    t_data = time.time() - t0
    net, hist = train(X, Y, steps=args.steps, batch=args.batch, lr=args.lr, log=log, Xv=Xv, Yv=Yv)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    net.save(args.out)
    net.close()
    t_train = time.time() - t0 - t_data
    log("evaluation on held-out seeds")
    rows = evaluate(args.out, range(ea, eb), device=dev, log=log)
    meta = {"shape": SHAPE, "fp32_storage": True, "train_seeds": [a, b], "eval_seeds": [ea, eb],
            "steps": args.steps, "batch": args.batch, "lr": args.lr, "history": hist,
            "data_s": t_data, "train_s": t_train, "evaluation": rows,
            "mean_iterations": {k: float(np.mean([r[k] for r in rows])) for k in ("cold", "jacobi", "learned")}}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    log(json.dumps(meta["mean_iterations"]))


if __name__ == "__main__":
    main()
