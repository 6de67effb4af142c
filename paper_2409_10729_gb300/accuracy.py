"""Per-field error of the mixed-precision and gated forms against the FP64 form.

  python -m paper_2409_10729_gb300.accuracy --case droplets --n 512 --steps 100 --forms mixed
  python -m paper_2409_10729_gb300.accuracy --case droplets --n 256 --steps 100 --forms mixed gated

Runs the seeded case for the same number of CFL-0.4 SSP-RK3 steps in the FP64
form (reference operation order: plain WENO5-JS + HLLC, the oracle's
arithmetic) and in each listed form, and reports per field f of the
conservative state q = (a1 r1, a2 r2, r u.., r E, a1):

  rel_l1   = sum_cells |q_f - q_f^64| / sum_cells |q_f^64|
  rel_linf = max_cells |q_f - q_f^64| / max_cells |q_f^64|
             (the momentum rows share the largest momentum component)
  abs_l1   = mean_cells |q_f - q_f^64|,  abs_linf = max_cells |q_f - q_f^64|

plus the time each run advanced, its device time per step and, for the gated
form, the fractions of cell reconstructions gated linear and sent back to
WENO.  The SHA-256 of the FP64 final state is printed so that it can be set
against a stored oracle result of the same case.  One JSON object is
printed (and written to --out if given).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def case(name, n):
    from . import inputs as I
    if name == "droplets":
        return I.shock_droplets(n)
    if name == "column":
        return I.shock_water_column(2 * n, n)
    return I.air_water_shock_tube(n)


def run(p, w, form, steps, cfl, weights=None):
    """Final state (torch CUDA float64), time advanced, ms per step, gate stats."""
    import torch

    from . import mfc
    s = mfc.Solver(p, form)
    if form == "gated":
        s.set_mlp_weights(weights)
    s.set_state_prim(w)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    t = s.step_rk3(cfl, steps)
    e1.record()
    torch.cuda.synchronize()
    n = p["n"]
    q = torch.empty((p["ndim"] + 4, n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    s.get_state(q)
    torch.cuda.synchronize()
    gate = s.gate_stats() if form == "gated" else None
    s.close()
    return q, t, e0.elapsed_time(e1) / steps, gate


def field_errors(q, ref, ndim):
    import torch
    ne = ref.shape[0]
    d = (q - ref).abs().reshape(ne, -1)
    r = ref.abs().reshape(ne, -1)
    scale = r.amax(1)
    scale[2:2 + ndim] = scale[2:2 + ndim].max()
    return {"rel_l1": (d.sum(1) / r.sum(1)).tolist(),
            "rel_linf": (d.amax(1) / scale).tolist(),
            "abs_l1": d.mean(1).tolist(),
            "abs_linf": d.amax(1).tolist(),
            "finite": bool(torch.isfinite(q).all())}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["droplets", "column", "tube"], default="droplets")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--forms", nargs="+", default=["mixed", "gated"], choices=["mixed", "gated", "fp64_fast"])
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)

    import numpy as np
    import torch

    from . import build as B
    B.build()
    p, w = case(args.case, args.n)
    ndim = p["ndim"]
    weights = np.load(os.path.join(HERE, "gate_weights.npy")) if "gated" in args.forms else None
    ref, t_ref, ms_ref, _ = run(p, w, "fp64", args.steps, args.cfl)
    sha = hashlib.sha256(ref.cpu().numpy().tobytes()).hexdigest()
    out = {"case": args.case, "n": p["n"], "steps": args.steps, "cfl": args.cfl,
           "fields": ["a1r1", "a2r2"] + ["ru", "rv", "rw"][:ndim] + ["rE", "a1"],
           "fp64": {"t": t_ref, "ms_per_step": round(ms_ref, 3), "state_sha256": sha}}
    for form in args.forms:
        q, t, ms, gate = run(p, w, form, args.steps, args.cfl, weights)
        rec = {"t": t, "t_rel_err": abs(t - t_ref) / t_ref, "ms_per_step": round(ms, 3)}
        rec.update(field_errors(q, ref, ndim))
        if gate is not None:
            gated, fallback, recon = gate
            rec["fraction_gated"] = gated / recon
            rec["fraction_fallback"] = fallback / recon
        out[form] = rec
        del q
        torch.cuda.empty_cache()
    line = json.dumps(out)
    print(line)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
