"""Per-kernel device times of one PCG-Aug step on a synthetic SUR workload.

    python -m paper_2510_14471_gb300.profile [--M 20000] [--G 64] [--k 16]
        [--precision fp32_refine|fp64] [--reps 10]

Sets the model up (TSQR), runs a two-step solve to size the workspace, then
times `reps` steps with CUDA events around every launch (glm_sur_profile_steps)
and prints one JSON line: mean milliseconds of the Sigma-apply step, the
projection partials, the reduction/scalar step, the projection update and the
whole step, with the algorithmic bytes of each.  Few launches precede the
timed ones, so the command is also the one to run under Nsight Compute.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=20000)
    ap.add_argument("--G", type=int, default=64)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64"])
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args(argv)
    import torch
    from synth import sur_inputs as S
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur

    p = S.config1(k=a.k, M=a.M, G=a.G)
    h = GlmSur(p.X_blocks, p.Omega, precision=a.precision, maxit=2, max_refine=1)
    h.solve(p.Y)
    torch.cuda.synchronize()
    ms = L.glm_sur_profile_steps(h.handle, a.reps, torch.cuda.current_stream().cuda_stream)
    pb = 4 if a.precision == "fp32_refine" else 8
    mk, Mn = p.m * p.k, p.M * p.n
    names = ["sigma_step", "proj_partial", "reduce", "proj_update", "step"]
    alg = [6 * pb * mk, pb * (Mn + mk), 0, pb * (Mn + 3 * mk), 2 * pb * Mn + 8 * pb * mk]
    out = {"workload": f"sur-singular-g{a.G}-m{a.M}-k{a.k}", "precision": a.precision,
           "ms": dict(zip(names, ms)), "algorithmic_bytes": dict(zip(names, alg)),
           "GBps": {nm: (b / (t * 1e-3) / 1e9 if t > 0 else None) for nm, b, t in zip(names, alg, ms)}}
    print(json.dumps(out))
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
