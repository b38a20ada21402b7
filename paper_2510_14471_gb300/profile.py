"""Per-kernel device times of one PCG-Aug step on a synthetic SUR workload.

    python -m paper_2510_14471_gb300.profile [--M 20000] [--G 64] [--k 16]
        [--precision fp32_refine|fp64] [--reps 10] [--nmin 8 --nmax 32 --rank 56]
    python -m paper_2510_14471_gb300.profile --batch 152 [--Mmax 600] [--k 8]

Sets the model up (TSQR), runs a two-step solve to size the workspace, then
times `reps` steps with CUDA events around every launch (glm_sur_profile_steps)
and prints one JSON line: mean milliseconds of the Sigma-apply step, the
projection partials, the reduction/scalar step, the projection update and the
whole step, with the algorithmic bytes of each.  Few launches precede the
timed ones, so the command is also the one to run under Nsight Compute.

With --batch N: N uneven instances of the batched workload (M up to --Mmax)
solved three times (the first tunes the tile height in at most three
launches; the later ones replay the tuned launch); prints the time of the last
solve and the per-instance work.
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
    ap.add_argument("--nmin", type=int, default=8)
    ap.add_argument("--nmax", type=int, default=32)
    ap.add_argument("--rank", type=int, default=56)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--Mmax", type=int, default=4000)
    ap.add_argument("--step-kernels", default="auto", choices=["auto", "simt"])
    a = ap.parse_args(argv)
    if a.batch:
        return profile_batch(a)
    import torch
    from synth import sur_inputs as S
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur

    p = S.singular_g64_m20000(k=a.k, M=a.M, G=a.G, rank=min(a.rank, a.G), nmin=a.nmin, nmax=a.nmax)
    h = GlmSur(p.X_blocks, p.Omega, precision=a.precision, maxit=2, max_refine=1, step_kernels=a.step_kernels)
    h.solve(p.Y)
    torch.cuda.synchronize()
    ms = L.glm_sur_profile_steps(h.handle, a.reps, torch.cuda.current_stream().cuda_stream)
    pb = 4 if a.precision == "fp32_refine" else 8
    mk, Mn = p.m * p.k, p.M * p.n
    if L.glm_sur_step_path(h.handle) == 1:
        # fused two-pass step, Sigma-apply on the tensor cores
        names = ["pass_a", "-", "reduce", "pass_b", "step"]
        alg = [pb * (Mn + 3 * mk), 0, 0, pb * (Mn + 5 * mk), 2 * pb * Mn + 8 * pb * mk]
    else:
        names = ["sigma_step", "proj_partial", "reduce", "proj_update", "step"]
        alg = [6 * pb * mk, pb * (Mn + mk), 0, pb * (Mn + 3 * mk), 2 * pb * Mn + 8 * pb * mk]
    out = {"workload": f"sur-singular-g{a.G}-m{a.M}-k{a.k}", "precision": a.precision,
           "ms": dict(zip(names, ms)), "algorithmic_bytes": dict(zip(names, alg)),
           "GBps": {nm: (b / (t * 1e-3) / 1e9 if t > 0 else None) for nm, b, t in zip(names, alg, ms)}}
    print(json.dumps(out))
    h.close()
    return 0


def profile_batch(a):
    import time
    import numpy as np
    import torch
    from synth import sur_inputs as S
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSurBatch

    k = a.k if a.k in (1, 2, 4, 8) else 8   # batched solves take k in {1, 2, 4, 8}
    probs = S.batched_uneven_instances(count=a.batch, k=k, Mmax=a.Mmax)
    bt = GlmSurBatch([(q.X_blocks, q.Omega) for q in probs])
    Y = bt.pack_y([q.Y for q in probs])
    count = len(probs)
    b = torch.empty(sum(bt.n) * k, dtype=torch.float64, device="cuda")
    iters = torch.zeros(count * k, dtype=torch.int32, device="cuda")
    relres = torch.zeros(count * k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ms = 0.0
    for _ in range(3):
        t0 = time.perf_counter()
        L.glm_sur_batch_solve(bt.handle, Y.data_ptr(), k, b.data_ptr(), iters.data_ptr(), relres.data_ptr(), stream)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
    steps, cycles = L.glm_sur_batch_get_work(bt.handle, count)
    tile, tune = L.glm_sur_batch_tile(bt.handle)
    print(json.dumps({"workload": f"batched-{count}-mmax{a.Mmax}-k{k}", "ms_last_solve": ms, "tile_rows": tile,
                      "tune_ms": tune, "steps_total": int(np.sum(steps)), "steps_max": int(np.max(steps)),
                      "cycles_max": int(np.max(cycles))}))
    bt.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
