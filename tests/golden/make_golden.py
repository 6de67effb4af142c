"""Write the stored oracle results the full-size GPU parity tests compare to.

Calls only the CPU oracle (oracle/) on the seeded inputs of
paper_2409_10729_gb300.inputs and records, for the final state after the
stated number of CFL-0.4 SSP-RK3 steps:
  - the SHA-256 of the initial primitive state (the tests regenerate it and
    refuse to compare if it differs),
  - the time advanced,
  - per-field max|q|, sum|q| and sum q over all cells,
  - the full state at ~1000 sampled cells (random + domain corners/edges),
  - the SHA-256 of the whole final state (float64, [field][z][y][x]).
Both the generators (only +, *, /, sqrt) and the oracle (-ffp-contract=off,
IEEE division and square root, no libm transcendentals) are bit-reproducible
across platforms, so these values hold on any machine.

  python tests/golden/make_golden.py column_1024x512   (about 6 minutes, one core)
  python tests/golden/make_golden.py droplets_128      (about 13 minutes, one core)
  python tests/golden/make_golden.py droplets_256      (about 115 minutes, one core)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2409_10729_gb300 import inputs as I  # noqa: E402

CASES = {
    "column_1024x512": (lambda: I.shock_water_column(1024, 512), 500),
    "droplets_128": (lambda: I.shock_droplets(128), 100),
    "droplets_256": (lambda: I.shock_droplets(256), 100),
}


def sample_cells(p, k=1000, seed=12345):
    rng = np.random.default_rng(seed)
    n = p["n"]
    cells = set(int(c) for c in rng.integers(0, n[0] * n[1] * n[2], size=k))
    for z in sorted({0, n[2] - 1}):
        for y in sorted({0, n[1] // 2, n[1] - 1}):
            for x in sorted({0, 1, 2, n[0] // 2, n[0] - 3, n[0] - 2, n[0] - 1}):
                cells.add(x + n[0] * (y + n[1] * z))
    return np.array(sorted(cells), dtype=np.int64)


def ic_hash(w):
    return hashlib.sha256(np.ascontiguousarray(w, dtype=np.float64).tobytes()).hexdigest()


def make(name):
    gen, steps = CASES[name]
    p, w = gen()
    q0 = O.prim_to_cons(p, w)
    t0 = time.time()
    q, t = O.run_cfl(p, q0, 0.4, steps)
    wall = time.time() - t0
    ne = q.shape[0]
    qf = q.reshape(ne, -1)
    cells = sample_cells(p)
    out = {
        "case": name, "steps": steps, "cfl": 0.4, "params": p, "ic_sha256": ic_hash(w),
        "t_final": repr(t), "field_max_abs": [repr(float(v)) for v in np.abs(qf).max(1)],
        "field_l1": [repr(float(v)) for v in np.abs(qf).sum(1)],
        "field_sum": [repr(float(v)) for v in qf.sum(1)],
        "state_sha256": hashlib.sha256(np.ascontiguousarray(q, dtype=np.float64).tobytes()).hexdigest(),
        "cells": cells.tolist(),
        "values": [[repr(float(v)) for v in qf[:, c]] for c in cells],
        "oracle_wall_s": round(wall, 1),
        "made_by": "tests/golden/make_golden.py " + name,
    }
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(f"{name}: {steps} steps, t = {t!r}, oracle {wall:.0f} s -> {path}")


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        make(name)
