"""Writes singular_g64_m20000_oracle_iterations.json: the iteration counts the float64
reference PCG of the oracle (Algorithm glmpcg2, D = I) takes on the singular
SUR workload G = 64, M = 20000, n_i ~ U{8..32}, Omega = A A^T (A 64 x 56),
k = 16, tol 1e-13, W = 25.  Calls only oracle/ and synth/.  The benchmark's CPU
reference arm uses the counts to turn a timed sample of iterations into
solves per second."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import sur_oracle as O  # noqa: E402
from synth import sur_inputs as S  # noqa: E402

if __name__ == "__main__":
    p = S.singular_g64_m20000(k=16)
    t0 = time.time()
    res = O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=1e-13, stag_window=25)
    err = np.linalg.norm(res["b"] - p.beta, axis=0) / np.linalg.norm(p.beta, axis=0)
    out = dict(workload="sur-singular-g64-m20000-k16", tol=1e-13, stagnation_window=25,
               iters=[int(v) for v in res["iters"]], status=list(res["status"]),
               relres=[float(v) for v in res["relres"]],
               rel_err_vs_beta_true=[float(v) for v in err], seconds=time.time() - t0)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "singular_g64_m20000_oracle_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))
