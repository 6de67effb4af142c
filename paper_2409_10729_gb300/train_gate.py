"""Train the troubled-cell gate network on the GPU with the library's kernels.

Data: seeded 2-D shock / water-column runs (512 x 256 cells) advanced with the
mixed form; every `every` steps the library emits, for every cell and
direction, the normalised density and pressure stencils labelled by plain
WENO5-JS itself (troubled when a nonlinear weight departs from its linear
weight by more than tau on a stencil whose variation is above the round-off
floor).  Flat sensor stencils (below the floor) are left out: the gate calls
them smooth without the network.  Each snapshot contributes its troubled
samples and as many smooth ones (capped), so the classes are balanced.

Training: mean weighted binary cross-entropy, Adam, minibatches, with the
loss/gradient and Adam kernels of libmfc5 (mfc_mlp_loss_grad, mfc_mlp_adam).
The decision threshold is then shifted (into the output bias) so that on
held-out runs a sample is called smooth only below the logit that keeps
`recall` of the troubled samples above it.

  python -m paper_2409_10729_gb300.train_gate [--runs 64] [--steps 500] [--out DIR]

Writes gate_weights.npy (float32, 1281) and gate_training.json next to this
file (or into --out).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "gate_weights.npy")


def collect(seeds, nx, ny, steps, every, cap, tau, rng):
    """Balanced labelled samples from runs with the given seeds (torch CUDA tensors)."""
    import torch

    from . import inputs as I
    from . import mfc
    xs, ys = [], []
    stats = {"snapshots": 0, "troubled_fraction": [], "flat_fraction": []}
    for seed in seeds:
        p, w = I.shock_water_column(nx, ny, seed=seed)
        s = mfc.Solver(p, "mixed")
        s.set_state_prim(w)
        for k in range(0, steps + 1, every):
            if k > 0:
                s.step_rk3(0.4, every)
            X, Y = s.gate_samples(tau)
            pos = torch.nonzero(Y > 0.5).flatten()
            neg = torch.nonzero((Y >= 0) & (Y <= 0.5)).flatten()
            stats["snapshots"] += 1
            stats["troubled_fraction"].append(float(len(pos)) / float(len(Y)))
            stats["flat_fraction"].append(1.0 - float(len(pos) + len(neg)) / float(len(Y)))
            npos = min(len(pos), cap)
            nneg = min(len(neg), max(npos, cap // 8))
            g = torch.Generator(device="cuda")
            g.manual_seed(int(rng.integers(1 << 31)))
            pi = pos[torch.randperm(len(pos), device="cuda", generator=g)[:npos]]
            ni = neg[torch.randperm(len(neg), device="cuda", generator=g)[:nneg]]
            idx = torch.cat([pi, ni])
            xs.append(X[idx].clone())
            ys.append(Y[idx].clone())
        s.close()
    stats["troubled_fraction"] = float(np.mean(stats["troubled_fraction"]))
    stats["flat_fraction"] = float(np.mean(stats["flat_fraction"]))
    return torch.cat(xs), torch.cat(ys), stats


def train(X, Y, epochs, batch, lr, pos_weight, seed):
    import torch

    from . import mfc
    torch.manual_seed(seed)
    n = X.shape[0]
    theta = torch.empty(1281, dtype=torch.float32, device="cuda")
    # He-style initialisation of the three layers, zero biases
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    theta.zero_()
    theta[0:160] = torch.randn(160, device="cuda", generator=g) * (2.0 / 5) ** 0.5
    theta[192:1216] = torch.randn(1024, device="cuda", generator=g) * (2.0 / 32) ** 0.5
    theta[1248:1280] = torch.randn(32, device="cuda", generator=g) * (1.0 / 32) ** 0.5
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    grad = torch.empty_like(theta)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    history = []
    t = 0
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda")
        ep_loss = torch.zeros(1, device="cuda")
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            mfc.mlp_loss_grad(xb, yb, theta, grad, loss, pos_weight)
            t += 1
            # cosine decay of the learning rate over the run
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * t / total))
            mfc.mlp_adam(theta, grad, m, v, t, lr=lr_t)
            ep_loss += loss
        history.append(float(ep_loss.item()) / steps_per_epoch)
    return theta, history


def evaluate(theta, X, Y):
    import torch

    from . import mfc
    z = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    mfc.mlp_forward(X.contiguous(), theta, z)
    return z, Y


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=64)
    ap.add_argument("--val-runs", type=int, default=4)
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--every", type=int, default=25)
    ap.add_argument("--cap", type=int, default=4096, help="max troubled samples per snapshot")
    ap.add_argument("--tau", type=float, default=0.1)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--pos-weight", type=float, default=2.0)
    ap.add_argument("--recall", type=float, default=0.995)
    ap.add_argument("--out", default=HERE)
    args = ap.parse_args(argv)

    import torch

    from . import build as B
    B.build()
    t0 = time.time()
    rng = np.random.default_rng(2409)
    X, Y, st = collect(range(args.runs), args.nx, args.ny, args.steps, args.every, args.cap, args.tau, rng)
    Xv, Yv, stv = collect(range(args.runs, args.runs + args.val_runs), args.nx, args.ny, args.steps, args.every,
                          args.cap, args.tau, rng)
    t_data = time.time() - t0
    theta, hist = train(X, Y, args.epochs, args.batch, args.lr, args.pos_weight, seed=0)
    torch.cuda.synchronize()
    t_train = time.time() - t0 - t_data
    zv, yv = evaluate(theta, Xv, Yv)
    # decision shift: smooth only below the logit that keeps `recall` of the
    # held-out troubled samples at or above it
    zt = zv[yv > 0.5]
    shift = float(torch.quantile(zt, 1.0 - args.recall).item()) if len(zt) else 0.0
    shift = min(shift, 0.0)
    theta[1280] -= shift
    zv = zv - shift
    pred_smooth = zv < 0
    tp = float(((yv > 0.5) & ~pred_smooth).sum())
    fn = float(((yv > 0.5) & pred_smooth).sum())
    tn = float(((yv <= 0.5) & pred_smooth).sum())
    fp = float(((yv <= 0.5) & ~pred_smooth).sum())
    w = theta.cpu().numpy().astype(np.float32)
    os.makedirs(args.out, exist_ok=True)
    np.save(os.path.join(args.out, "gate_weights.npy"), w)
    summary = {
        "data": {"runs": args.runs, "val_runs": args.val_runs, "grid": [args.nx, args.ny], "steps": args.steps,
                 "every": args.every, "tau": args.tau, "train_samples": int(len(Y)),
                 "train_troubled": int((Y > 0.5).sum()), "val_samples": int(len(Yv)),
                 "troubled_fraction_of_all_samples": round(st["troubled_fraction"], 4),
                 "flat_fraction_of_all_samples": round(st["flat_fraction"], 4),
                 "round_off_floor": 1e-4},
        "training": {"epochs": args.epochs, "batch": args.batch, "lr": args.lr, "pos_weight": args.pos_weight,
                     "loss_per_epoch": [round(h, 5) for h in hist]},
        "heldout": {"decision_shift_logit": round(shift, 4), "recall_troubled": round(tp / max(tp + fn, 1), 5),
                    "specificity_smooth": round(tn / max(tn + fp, 1), 5),
                    "accuracy": round((tp + tn) / max(tp + tn + fp + fn, 1), 5)},
        "seconds": {"data": round(t_data, 1), "train": round(t_train, 1)},
    }
    with open(os.path.join(args.out, "gate_training.json"), "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
