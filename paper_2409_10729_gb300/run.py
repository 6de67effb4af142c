"""Run one of the seeded cases on the GPU and report its grind time.

  python -m paper_2409_10729_gb300.run --case droplets --n 160 --form fp64 --steps 2 --warmup 1

Used as the command under profilers (ncu) and for quick timing; prints one
line per run with the device time per RK3 step and the grind time in
ns per cell, equation and RHS evaluation.
"""
from __future__ import annotations

import argparse
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["droplets", "droplets3", "column", "tube"], default="droplets")
    ap.add_argument("--n", type=int, default=128, help="cells per dimension (column: ny, nx = 2 ny)")
    ap.add_argument("--form", choices=["fp64", "fp64_fast", "mixed", "gated"], default="fp64")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--weno-order", type=int, choices=[3, 5], default=5)
    ap.add_argument("--stretch", action="store_true",
                    help="tanh-refined grid in every direction (cells at the centre half as wide)")
    args = ap.parse_args()

    import torch

    from . import build as B
    from . import inputs as I
    from . import mfc

    B.build()
    if args.case == "droplets":
        p, w = I.shock_droplets(args.n)
    elif args.case == "droplets3":
        p, w = I.shock_droplets_3fluid(args.n)
    elif args.case == "column":
        p, w = I.shock_water_column(2 * args.n, args.n)
    else:
        p, w = I.air_water_shock_tube(args.n)
    p = dict(p, weno_order=args.weno_order)
    if args.stretch:
        p["edges"] = [I.tanh_edges(p["n"][d], p["lo"][d], p["hi"][d], 0.5 * (p["lo"][d] + p["hi"][d]),
                                   strength=8.0, refine=0.5) if d < p["ndim"] else None for d in range(3)]
    s = mfc.Solver(p, args.form)
    if args.form == "gated":
        import numpy as np
        import os
        s.set_mlp_weights(np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "gate_weights.npy")))
    s.set_state_prim(w)
    s.step_rk3(args.cfl, args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    t0 = time.perf_counter()
    t = s.step_rk3(args.cfl, args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ncell = p["n"][0] * p["n"][1] * p["n"][2]
    neq = I.neq_of(p)
    grind = ms * 1e6 / (args.steps * 3 * ncell * neq)
    print(f"case={args.case} n={args.n} form={args.form} steps={args.steps} ms/step={ms / args.steps:.3f} "
          f"grind_ns={grind:.5f} t={t:.6e} wall={time.perf_counter() - t0:.2f}s")
    s.close()


if __name__ == "__main__":
    main()
