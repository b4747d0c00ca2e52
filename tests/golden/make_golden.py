"""Writes the stored expected values used by the GPU parity tests and the benchmark.

Calls only the FP64 oracle (oracle/) and the seeded input generator; nothing here
touches the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [tiny medium autograd medium_100]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import ba_oracle as O  # noqa: E402
from paper_2605_30583_gb300 import synth  # noqa: E402

# LM settings per workload: 20 LM iterations of at most 50 PCG iterations, initial
# trust region 100 and CG tolerance 1e-3 (Sec. VI).
SETTINGS = {"tiny": dict(max_lm_iters=20, max_pcg_iters=50),
            "medium": dict(max_lm_iters=20, max_pcg_iters=50),
            "autograd": dict(max_lm_iters=20, max_pcg_iters=50)}


def run(name, f32_inputs):
    p = synth.make_config(name)
    if f32_inputs:
        p = synth.round_to_f32(p)
    opts = O.LMOptions(**SETTINGS[name])
    t0 = time.time()
    res = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, opts)
    dt = time.time() - t0
    return dict(config=name, inputs="fp32-rounded" if f32_inputs else "fp64",
                n_cams=p.n_cams, n_pts=p.n_pts, n_obs=p.n_obs,
                options=SETTINGS[name], initial_cost=res.initial_cost, final_cost=res.final_cost,
                lm_iters=res.lm_iters, accepted=res.accepted, pcg_iters_total=res.pcg_iters_total,
                history=[{k: (float(v) if not isinstance(v, bool) else v) for k, v in h.items()}
                         for h in res.history],
                oracle_seconds=dt, numpy=np.__version__)


def run_long(name, iters):
    """The same workload with a longer LM budget, FP64 inputs only (context for the
    headline's C*: how far 20 iterations are from where LM settles)."""
    p = synth.make_config(name)
    settings = dict(SETTINGS[name], max_lm_iters=iters)
    t0 = time.time()
    res = O.ba_solve(p.cams_init, p.pts_init, p.cam_idx, p.pt_idx, p.pixels, O.LMOptions(**settings))
    return dict(config=name, inputs="fp64", options=settings, initial_cost=res.initial_cost,
                final_cost=res.final_cost, lm_iters=res.lm_iters, accepted=res.accepted,
                pcg_iters_total=res.pcg_iters_total,
                costs=[float(h["cost"]) for h in res.history] + [float(res.final_cost)],
                oracle_seconds=time.time() - t0, numpy=np.__version__)


def main(names):
    for name in names:
        if name.endswith("_100"):   # e.g. medium_100: 100 LM iterations
            out = run_long(name[:-4], 100)
            with open(os.path.join(HERE, f"oracle_lm_{name}.json"), "w") as f:
                json.dump(out, f, indent=1)
            print(name, out["final_cost"], f"{out['oracle_seconds']:.1f}s")
            continue
        out = {"fp64": run(name, False), "fp32_inputs": run(name, True)}
        path = os.path.join(HERE, f"oracle_lm_{name}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(name, out["fp64"]["final_cost"], out["fp32_inputs"]["final_cost"],
              f"{out['fp64']['oracle_seconds']:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "medium", "autograd"])
