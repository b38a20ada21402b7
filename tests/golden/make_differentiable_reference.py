"""Writes differentiable_g128_m40000_reference.json: reference values of the differentiable SUR
workload G = 128, M = 40000, n_i ~ U{4..24}, Omega = L L^T (cond ~ 1e6),
loss ||b - beta_target||^2, from the oracle's extended-precision iterative
refinement (``sur_gls_refined``).  Stored: b in full, and dL/dy = lam and the
symmetrised dL/dOmega at 512 seeded sample positions each, with their norms.
Calls only oracle/ and synth/.  numpy's longdouble is 80-bit extended on
x86-64 and IEEE quad on aarch64; either carries the residuals far below the
float64 rounding level, so the file does not depend on the machine beyond
the last few bits."""
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import sur_oracle as O  # noqa: E402
from synth import sur_inputs as S  # noqa: E402

N_SAMPLE = 512

if __name__ == "__main__":
    t0 = time.time()
    p, Lfac, target = S.differentiable_g128_m40000()
    fwd = O.sur_gls_refined(p.X_blocks, p.Omega, p.Y, steps=3)
    b = fwd["b"]
    gb = 2 * (b - target)
    adj = O.sur_gls_refined(p.X_blocks, p.Omega, p.Y, gb, steps=3)
    lam, gO = adj["lam"][:, 0], adj["dOmega"]
    gOs = 0.5 * (gO + gO.T)
    g = np.random.default_rng(2510)
    lam_idx = np.sort(g.choice(lam.size, N_SAMPLE, replace=False))
    om_idx = np.sort(g.choice(gOs.size, N_SAMPLE, replace=False))
    out = dict(workload=p.meta["name"], G=p.G, M=p.M, n=p.n, cond_omega=float(np.linalg.cond(p.Omega)),
               longdouble_eps=float(np.finfo(np.longdouble).eps), machine=platform.machine(),
               corrections=[fwd["corrections"][0], adj["corrections"][-1]],
               b=[float(v) for v in b[:, 0]],
               lam_norm=float(np.linalg.norm(lam)), lam_idx=[int(i) for i in lam_idx],
               lam=[float(lam[i]) for i in lam_idx],
               dOmega_sym_norm=float(np.linalg.norm(gOs)), dOmega_idx=[int(i) for i in om_idx],
               dOmega_sym=[float(gOs.reshape(-1)[i]) for i in om_idx],
               seconds=time.time() - t0)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "differentiable_g128_m40000_reference.json"), "w") as f:
        json.dump(out, f, indent=0)
    print({k: v for k, v in out.items() if not isinstance(v, list)}, out["corrections"])
