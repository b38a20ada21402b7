"""Benchmark: SUR GLS solves/sec at <= 1e-9 relative error on the singular
SUR workload (G = 64 equations, M = 20000 observations, n_i ~ U{8..32},
Omega = A A^T with A 64 x 56, k = 16 right-hand sides), float32-bulk PCG-Aug
inside float64 iterative refinement, on one GB300.

One step = one complete glm_sur_solve call (all k right-hand sides) with the
inputs resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica (the single-instance path
has no exchange step: replicas only, weak scaling); value = total solves/s.
--impl reference times the float64 CPU oracle (the reference PCG of the
paper's algorithm) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SUR GLS solves/sec @ <=1e-9 rel err vs FP64 oracle; PCG-iter HBM GB/s vs roofline"
WORKLOAD = "sur-singular-g64-m20000-k16 (G=64, M=20000, n_i~U{8..32}, Omega=AA^T rank 56)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--M", type=int, default=20000)
    ap.add_argument("--G", type=int, default=64)
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 PCG comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-reduced", action="store_true", help="skip the row-reduced comparison solve")
    ap.add_argument("--profile-reps", type=int, default=20)
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the batched, constrained and differentiable summaries")
    ap.add_argument("--workload", default="singular",
                    choices=["singular", "batched", "constrained", "differentiable", "var"],
                    help="singular: the headline workload; the others measure the batched, restricted and "
                         "adjoint paths on their own workloads")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(args):
    from synth import sur_inputs as S
    return S.singular_g64_m20000(k=args.k, M=args.M, G=args.G)


def rel_err(b, ref):
    return float(np.max(np.linalg.norm(b - ref, axis=0) / np.linalg.norm(ref, axis=0)))


def oracle_iteration_sample(p, n_iter):
    """Time n_iter steps of the float64 reference PCG of the oracle (all host
    cores); returns seconds per step (setup QR excluded)."""
    from oracle import sur_oracle as O
    ops = O.SurOps(p.X_blocks, p.Omega)
    O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=2, stag_window=10 ** 9, ops=ops)   # warm
    t0 = time.perf_counter()
    O.sur_pcg_aug(p.X_blocks, p.Omega, p.Y, tol=0.0, maxit=n_iter, stag_window=10 ** 9, ops=ops)
    return (time.perf_counter() - t0) / n_iter


def oracle_iters_per_solve():
    path = os.path.join(ROOT, "tests", "golden", "singular_g64_m20000_oracle_iterations.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return int(max(d["iters"])), "oracle float64 PCG to tol 1e-13 (tests/golden/singular_g64_m20000_oracle_iterations.json)"
    return None, None


def aggregate(ms_local, pg, world, device="cpu"):
    """Replicas: the job's time per step is the slowest rank's; the job's
    throughput is every rank's solve over that time."""
    ms = ms_local
    if pg is not None:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * 1e3 / ms


NCU_SECTION = {"sigma_step": "k_sigma_step_tma", "proj_partial": "k_proj_partial_tma", "proj_update": "k_proj_update_bj",
               "pass_a": "k_tc_pass_a", "pass_b": "k_tc_pass_b"}


def ncu_traffic(args, kernel):
    """DRAM bytes per launch of `kernel` from the committed Nsight Compute
    summary of this workload (float32 bulk only), else None."""
    if args.precision != "fp32_refine" or kernel not in NCU_SECTION:
        return None
    path = os.path.join(ROOT, "profiles", f"step_kernels_sur-singular-g{args.G}-m{args.M}-k{args.k}.md")
    if not os.path.exists(path):
        return None
    cur = None
    for line in open(path):
        if line.startswith("## "):
            cur = line[3:].split("<")[0].strip()
        elif line.startswith("traffic_bytes_per_launch:") and cur == NCU_SECTION[kernel]:
            return int(line.split(":")[1])
    return None


EXTRA_WORKLOADS = ("batched", "constrained", "differentiable", "var")


def run_extras(timeout_s=420):
    """The other workloads, each run once (one warm-up, one timed solve) in a
    child process of this script; returns a summary of each one's JSON line."""
    import subprocess
    out = {}
    for w in EXTRA_WORKLOADS:
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", w, "--steps", "1", "--warmup", "1",
               "--no-cpu"]
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
            line = None
            for ln in r.stdout.splitlines():
                if ln.startswith("{"):
                    line = json.loads(ln)
            if r.returncode != 0 or line is None:
                out[w] = {"error": f"rc={r.returncode}: {r.stderr.strip().splitlines()[-1:] if r.stderr else ''}"}
                continue
        except subprocess.TimeoutExpired:
            out[w] = {"error": f"did not finish within {timeout_s} s"}
            continue
        keep = ["value", "unit", "ms_per_step", "dtype", "config", "roofline", "roofline_iter", "e2e", "gpu_launches",
                "clocks", "rel_err_sampled", "rel_err", "status_counts", "steps_per_instance", "iters_max", "k1",
                "grad_err", "b_err", "steps", "models", "row_reduced", "full_model", "rel_err_b",
                "rel_err_dOmega_sampled", "speedup_vs_full_model", "balance"]
        out[w] = {k2: line[k2] for k2 in keep if k2 in line}
        out[w]["wall_s"] = time.perf_counter() - t0
    return out


def run_reference(args, rank, world, pg):
    """CPU reference arm: the oracle's float64 PCG timed on the host cores."""
    if rank != 0:
        return 0
    p = make_problem(args)
    iters, src = oracle_iters_per_solve()
    n_iter = 8
    times = []
    for s in range(args.warmup + args.steps):
        t = oracle_iteration_sample(p, n_iter)
        if s >= args.warmup:
            times.append(t)
    t_iter = float(np.mean(times))
    if iters is None:
        iters, src = 500, "assumed 500 iterations per solve (no stored oracle count)"
    sps = 1.0 / (t_iter * iters)
    line = {"impl": "reference", "metric": METRIC, "value": sps, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * iters * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "k": args.k, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": sps, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{n_iter} float64 reference-PCG steps per timed step, "
                                       f"x {iters} steps per solve ({src})"},
            "e2e": {"value": sps, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args, rank, world, local, pg):
    import torch
    from paper_2510_14471_gb300 import build
    if rank == 0:
        build.build()
    if pg is not None:
        pg.barrier()
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = make_problem(args)
    m, n, k = p.m, p.n, p.k
    stream = torch.cuda.current_stream().cuda_stream

    # ---- setup (TSQR), timed separately
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = GlmSur(p.X_blocks, p.Omega, precision=args.precision, tol=1e-13, device=dev)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3   # includes the host->device copy of X
    Ycm = torch.as_tensor(p.Y.T.copy(), device=dev)                # column-major m x k
    b = torch.empty((k, n), dtype=torch.float64, device=dev)
    iters = torch.zeros(k, dtype=torch.int32, device=dev)
    relres = torch.zeros(k, dtype=torch.float64, device=dev)

    def solve():
        L.glm_sur_solve(h.handle, Ycm.data_ptr(), m, k, b.data_ptr(), n, iters.data_ptr(), relres.data_ptr(),
                        stream)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    status = L.glm_sur_get_status(h.handle, k)
    err = rel_err(b.t().cpu().numpy(), p.beta)
    it_used = iters.cpu().numpy()
    launches0 = L.glm_sur_launch_count(h.handle)

    # ---- timed region: K solves, inputs resident in HBM (working set > L2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            solve()
        ev1.record()
        torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = L.glm_sur_launch_count(h.handle) - launches0
    ms, value = aggregate(ms, pg, world, dev)

    # ---- end to end through the public API with host buffers
    Y_host = torch.as_tensor(p.Y.T.copy()).pin_memory()
    b_host = torch.empty((k, n), dtype=torch.float64).pin_memory()
    Ydev2 = torch.empty_like(Ycm)
    e2e_times = []
    for s in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ydev2.copy_(Y_host, non_blocking=True)
        L.glm_sur_solve(h.handle, Ydev2.data_ptr(), m, k, b.data_ptr(), n, iters.data_ptr(), relres.data_ptr(),
                        stream)
        b_host.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        if s >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_err = rel_err(b_host.t().numpy(), p.beta)
    e2e_sps = world / float(np.mean(e2e_times))

    # ---- per-kernel times of one float32 bulk step (dominant kernel roofline)
    prof = L.glm_sur_profile_steps(h.handle, args.profile_reps, stream)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    pb = 4 if args.precision == "fp32_refine" else 8
    M, G = args.M, args.G
    mk = m * k
    step_path = L.glm_sur_step_path(h.handle)
    if step_path == 1:
        # fused two-pass step, Sigma-apply on the tensor cores (S never stored)
        kbytes = {"pass_a": pb * M * n + 3 * pb * mk,    # read Q, g, u; write u
                  "-": 0, "reduce": 0,
                  "pass_b": pb * M * n + 5 * pb * mk}    # read Q, u, g, w; write g, w
        names = ["pass_a", "-", "reduce", "pass_b"]
    else:
        kbytes = {   # algorithmic bytes per launch of each kernel of a step
            "sigma_step": 6 * pb * mk,                 # read g, u, w; write u, w, S
            "proj_partial": pb * M * n + pb * mk,      # read Q, S
            "reduce": 0,
            "proj_update": pb * M * n + 3 * pb * mk,   # read Q, S, g; write g
        }
        names = ["sigma_step", "proj_partial", "reduce", "proj_update"]
    dom = max(range(4), key=lambda i: prof[i])
    dname = names[dom]
    ach = kbytes[dname] / (prof[dom] * 1e-3) / 1e9
    b_iter = 2 * pb * M * n + 8 * pb * mk
    ach_iter = b_iter / (prof[4] * 1e-3) / 1e9
    traffic = ncu_traffic(args, dname)

    # ---- float64 PCG on the same workload (comparison at the same accuracy)
    fp64 = None
    if not args.no_fp64:
        h64 = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=1e-13, device=dev)
        Lh = h64.handle
        L.glm_sur_solve(Lh, Ycm.data_ptr(), m, k, b.data_ptr(), n, iters.data_ptr(), relres.data_ptr(), stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.glm_sur_solve(Lh, Ycm.data_ptr(), m, k, b.data_ptr(), n, iters.data_ptr(), relres.data_ptr(), stream)
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        it64 = iters.cpu().numpy()
        prof64 = L.glm_sur_profile_steps(Lh, 5, stream)
        fp64 = {"solves_per_s": 1e3 / t64, "ms_per_solve": t64, "iters_max": int(it64.max()),
                "rel_err_vs_beta_true": rel_err(b.t().cpu().numpy(), p.beta),
                "status": L.glm_sur_get_status(Lh, k),
                "step_ms": prof64[4],
                "step_fp64_gflops": (2 * M * G * G * k + 4 * M * n * k) / (prof64[4] * 1e-3) / 1e9}
        h64.close()

    # ---- the same solves on the row-reduced model (Remark rem:reduction)
    reduced = None
    if not args.no_reduced:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hr = GlmSur(p.X_blocks, p.Omega, precision=args.precision, tol=1e-13, reduce_rows=True, device=dev)
        torch.cuda.synchronize()
        setup_r = (time.perf_counter() - t0) * 1e3
        Lr = hr.handle

        def solve_r():
            L.glm_sur_solve(Lr, Ycm.data_ptr(), m, k, b.data_ptr(), n, iters.data_ptr(), relres.data_ptr(), stream)

        solve_r()
        torch.cuda.synchronize()
        ms_r, _ = timed(solve_r, max(1, args.steps), 1, local, None)
        reduced = {"solves_per_s": 1e3 / ms_r, "ms_per_solve": ms_r, "setup_ms": setup_r,
                   "rel_err_vs_beta_true": rel_err(b.t().cpu().numpy(), p.beta),
                   "status": L.glm_sur_get_status(Lr, k), "iters_max": int(iters.cpu().numpy().max()),
                   "rows": int(n), "note": "rows of every equation rotated onto range([X_1 ... X_G]); "
                                           "one float64 product Q^T Y per solve"}
        hr.close()

    # ---- the float32 bulk alone: one float32 PCG run to its own floor, no
    # float64 refinement step after it (the "unrefined" error)
    unrefined = None
    if args.precision == "fp32_refine":
        hu = GlmSur(p.X_blocks, p.Omega, precision="fp32_refine", tol=1e-13, inner_tol=1e-13, max_refine=1,
                    device=dev)
        L.glm_sur_solve(hu.handle, Ycm.data_ptr(), m, k, b.data_ptr(), n, iters.data_ptr(), relres.data_ptr(), stream)
        torch.cuda.synchronize()
        unrefined = {"rel_err_vs_beta_true": rel_err(b.t().cpu().numpy(), p.beta),
                     "iters_max": int(iters.cpu().numpy().max()),
                     "note": "one float32 PCG run (inner tolerance 1e-13, stops at its float32 floor), "
                             "correction projected in float64, no refinement step"}
        hu.close()

    # ---- CPU oracle baseline (rank 0, bounded sample)
    cpu = None
    if rank == 0 and not args.no_cpu:
        n_iter = 6
        t_iter = oracle_iteration_sample(p, n_iter)
        iters_ref, src = oracle_iters_per_solve()
        if iters_ref is None and fp64 is not None:
            iters_ref, src = fp64["iters_max"], "float64 PCG step count of this run"
        if iters_ref is None:
            iters_ref, src = 500, "assumed"
        cpu = {"value": 1.0 / (t_iter * iters_ref), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n_iter} steps of the float64 reference PCG (numpy, k={k}) timed, "
                         f"x {iters_ref} steps per solve ({src}); setup QR excluded",
               "sec_per_step": t_iter}
        # the oracle's structured direct GLS (Remark rem:reduction + eigen-split of
        # Omega), timed on the whole workload: a measurement, not a projection
        from oracle import sur_oracle as O
        t0 = time.perf_counter()
        b_o2 = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y)
        t_o2 = time.perf_counter() - t0
        cpu["direct_structured"] = {"seconds": t_o2, "solves_per_s": 1.0 / t_o2,
                                    "rel_err_vs_beta_true": rel_err(b_o2, p.beta),
                                    "sample": f"one full solve, all k={k} right-hand sides"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.precision == "fp32_refine" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "G": G, "M": M, "n": n, "k": k, "precision": args.precision,
                       "tol": 1e-13, "l2": "inputs larger than L2 (Q 205 MB f64 + 102 MB f32, vectors 82-164 MB)",
                       "parallelism": f"replicas{world}"},
            "per_rhs_solves_per_s": value * k,
            "rel_err_max": err, "status": status, "iters_max": int(it_used.max()),
            "setup_ms": setup_ms,
            "roofline": {"bound": "hbm", "kernel": dname, "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": traffic, "peak_source": peak_src,
                         "algorithmic_bytes": kbytes[dname], "ms": prof[dom]},
            "roofline_iter": {"bound": "hbm", "achieved": ach_iter, "peak": hbm, "unit": "GB/s",
                              "frac": ach_iter / hbm, "B_iter": b_iter, "ms": prof[4],
                              "kernel_ms": {nm: t for nm, t in zip(names, prof[:4]) if nm != "-"},
                              "step_kernels": "tensor-core fused two-pass" if step_path == 1 else "simt four-launch"},
            "fp64_pcg": fp64,
            "row_reduced": reduced,
            "unrefined": unrefined,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_sps, "unit": "solves/s", "h2d_bytes_per_step": int(m * k * 8),
                    "d2h_bytes_per_step": int(n * k * 8), "rel_err_max": e2e_err},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_extras:
            h.close()
            h = None
            torch.cuda.empty_cache()
            line["workloads"] = run_extras()
        print(json.dumps(line))
    if h is not None:
        h.close()
    return 0


# ---------------------------------------------------------------------------
# Secondary workloads (--workload): the batched, restricted and adjoint paths,
# each timed the same way (inputs resident, CUDA events, clocks sampled) with
# its own roofline and CPU oracle sample.
# ---------------------------------------------------------------------------

def load_peaks():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    return hbm, ("measured" if "hbm_gbs" in peaks else "fallback")


FP64_PEAK_GFLOPS = 1250.0   # nominal float64 FMA rate of the part (dense, non-tensor)


def timed(fn, steps, warmup, local, pg):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(steps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    return ev0.elapsed_time(ev1) / steps, clk.summary()


def batch_balance(L, handle, count, ms, clocks):
    """Load balance of one persistent batch launch from the per-instance
    cycle counts the kernel records (SM clock): the longest instance, and the
    ideal time, the instances' total time spread evenly over the launch's
    CTAs (all resident at once: SMs x CTAs per SM)."""
    steps, cycles = L.glm_sur_batch_get_work(handle, count)
    grid = L.glm_sur_batch_grid(handle)
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    inst_ms = np.asarray(cycles, dtype=float) / (mhz * 1e3)
    ideal = float(inst_ms.sum()) / grid if grid > 0 else 0.0
    return {"batch_ms": ms, "longest_instance_ms": float(inst_ms.max()), "ideal_ms": ideal,
            "batch_over_ideal": ms / ideal if ideal > 0 else None, "ctas": grid, "sm_mhz_used": mhz,
            "note": "ideal = sum of the instances' own times / CTAs of the launch; times from clock64 per instance"}


def base_line(args, world, metric, workload, value, unit, ms, dtype, config):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": dict({"workload": workload, "parallelism": f"replicas{world}"}, **config)}


def run_batched(args, rank, world, local, pg):
    """2048 uneven instances, k = 8, one persistent launch per solve."""
    import torch
    from paper_2510_14471_gb300 import build
    if rank == 0:
        build.build()
    if pg is not None:
        pg.barrier()
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSurBatch
    from synth import sur_inputs as S
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    k, count = 8, 2048
    probs = S.batched_uneven_instances(count=count, k=k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = GlmSurBatch([(q.X_blocks, q.Omega) for q in probs], device=dev)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    Y = bt.pack_y([q.Y for q in probs])
    nb = sum(bt.n) * k
    b = torch.empty(nb, dtype=torch.float64, device=dev)
    iters = torch.zeros(count * k, dtype=torch.int32, device=dev)
    relres = torch.zeros(count * k, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def solve():
        L.glm_sur_batch_solve(bt.handle, Y.data_ptr(), k, b.data_ptr(), iters.data_ptr(), relres.data_ptr(), stream)

    solve()                                  # first solve: tile autotune + graph capture
    torch.cuda.synchronize()
    l0 = L.glm_sur_batch_launch_count(bt.handle)
    ms, clocks = timed(solve, args.steps, args.warmup, local, pg)
    launches = (L.glm_sur_batch_launch_count(bt.handle) - l0) // (args.steps + args.warmup)
    status = np.array(L.glm_sur_batch_get_status(bt.handle, count * k))
    balance = batch_balance(L, bt.handle, count, ms, clocks)
    it = iters.view(count, k).cpu().numpy()
    ms, value = aggregate(ms, pg, world, dev)
    value *= count                           # instances solved per second (all k right-hand sides each)
    tile, tune = L.glm_sur_batch_tile(bt.handle)
    # algorithmic bytes: every float32 step of instance j reads Q_j twice and
    # moves eight float32 vectors of m_j k values (as the single-instance step)
    steps_j = it.max(axis=1)
    bytes_j = 4 * (2 * np.array(bt.M) * np.array(bt.n) + 8 * np.array(bt.m) * k)
    alg = float(np.sum(steps_j * bytes_j))
    hbm, src = load_peaks()
    ach = alg / (ms * 1e-3) / 1e9
    # accuracy on sampled instances (structured direct GLS of the oracle)
    from oracle import sur_oracle as O
    bs, off, errs = b.cpu().numpy(), 0, {}
    offs = np.cumsum([0] + [nj * k for nj in bt.n])
    for j in (0, 1, 777, 2047):
        bj = bs[offs[j]:offs[j + 1]].reshape(k, bt.n[j]).T
        errs[j] = rel_err(bj, O.sur_gls_structured(probs[j].X_blocks, probs[j].Omega, probs[j].Y))
    # end to end: host Y in, b out
    Yh = Y.cpu().pin_memory()
    bh = torch.empty(nb, dtype=torch.float64).pin_memory()
    Y2 = torch.empty_like(Y)
    e2e = []
    for s in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Y2.copy_(Yh, non_blocking=True)
        L.glm_sur_batch_solve(bt.handle, Y2.data_ptr(), k, b.data_ptr(), iters.data_ptr(), relres.data_ptr(),
                              stream)
        bh.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        if s >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    cpu = None
    if rank == 0 and not args.no_cpu:
        t0 = time.perf_counter()
        nrun = 0
        while nrun < 64 and time.perf_counter() - t0 < 15.0:
            q = probs[nrun]
            O.sur_pcg_aug(q.X_blocks, q.Omega, q.Y, tol=1e-12)
            nrun += 1
        dt = time.perf_counter() - t0
        cpu = {"value": nrun / dt, "unit": "instance solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the float64 reference PCG of the oracle (k={k}, tol 1e-12) on the first {nrun} "
                         f"instances, {dt:.1f} s"}
    # the same batch on the row-reduced instances (Remark rem:reduction: every
    # instance with M >= 2n solved on its n rotated rows)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    btr = GlmSurBatch([(q.X_blocks, q.Omega) for q in probs], reduce_rows=True, device=dev)
    torch.cuda.synchronize()
    setup_r_ms = (time.perf_counter() - t0) * 1e3
    br = torch.empty(nb, dtype=torch.float64, device=dev)
    itr = torch.zeros(count * k, dtype=torch.int32, device=dev)
    rrr = torch.zeros(count * k, dtype=torch.float64, device=dev)

    def solve_r():
        L.glm_sur_batch_solve(btr.handle, Y.data_ptr(), k, br.data_ptr(), itr.data_ptr(), rrr.data_ptr(), stream)

    solve_r()
    torch.cuda.synchronize()
    ms_r, clocks_r = timed(solve_r, args.steps, args.warmup, local, pg)
    balance_r = batch_balance(L, btr.handle, count, ms_r, clocks_r)
    status_r = np.array(L.glm_sur_batch_get_status(btr.handle, count * k))
    ms_r, value_r = aggregate(ms_r, pg, world, dev)
    bsr, errs_r = br.cpu().numpy(), {}
    for j in (0, 1, 777, 2047):
        bj = bsr[offs[j]:offs[j + 1]].reshape(k, bt.n[j]).T
        errs_r[j] = rel_err(bj, O.sur_gls_structured(probs[j].X_blocks, probs[j].Omega, probs[j].Y))
    row_reduced = {"value": value_r * count, "unit": "instance solves/s", "ms": ms_r, "setup_ms": setup_r_ms,
                   "rel_err_sampled": errs_r,
                   "status_counts": {int(v): int(c) for v, c in zip(*np.unique(status_r, return_counts=True))},
                   "steps_max": int(itr.view(count, k).max().item()), "balance": balance_r,
                   "note": "every instance with M >= 2n on its n rows; one float64 product Q_W^T Y per instance"}
    btr.close()
    if rank == 0:
        line = base_line(args, world, METRIC, "batched-2048-uneven-k8 (G~U{2..12}, M~U{200..4000}, "
                         "n_i~U{2..10}, Omega Wishart(G,G+4)/trace)", value, "instance solves/s", ms, "f32+f64",
                         {"count": count, "k": k, "precision": "fp32_refine", "tol": 1e-12, "tile_rows": tile,
                          "tile_tune_ms": tune, "l2": "per-instance working set 0.5-5 MB; 2048 instances 1.9 GB"})
        line.update({
            "rel_err_sampled": errs, "status_counts": {int(v): int(c) for v, c in zip(*np.unique(status, return_counts=True))},
            "steps_per_instance": {"min": int(steps_j.min()), "median": float(np.median(steps_j)),
                                   "max": int(steps_j.max())},
            "setup_ms": setup_ms, "balance": balance,
            "roofline": {"bound": "hbm", "kernel": "k_batch_solve", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": None, "peak_source": src, "algorithmic_bytes": alg,
                         "ms": ms, "note": "lower bound of the work: steps per instance = max over its columns"},
            "cpu_baseline": cpu,
            "row_reduced": row_reduced,
            "e2e": {"value": world * count / float(np.mean(e2e)), "unit": "instance solves/s",
                    "h2d_bytes_per_step": int(Y.numel() * 8), "d2h_bytes_per_step": int(nb * 8)},
            "gpu_launches": int(launches), "clocks": clocks})
        print(json.dumps(line))
    bt.close()
    return 0


def run_constrained(args, rank, world, local, pg):
    """G = 32, M = 50000, n_i = 16, 64 restrictions C b = d, float64, k = 32 (and k = 1)."""
    import torch
    from paper_2510_14471_gb300 import build
    if rank == 0:
        build.build()
    if pg is not None:
        pg.barrier()
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur
    from synth import sur_inputs as S
    from oracle import sur_oracle as O
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    out = {}
    for k in (32, 1):
        p = S.constrained_g32_m50000(k=k)
        h = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=1e-13, device=dev)
        h.set_restrictions(p.C)
        m, n, kc = p.m, p.n, p.C.shape[0]
        Ycm = torch.as_tensor(p.Y.T.copy(), device=dev)
        dcm = torch.as_tensor(np.asarray(p.d).reshape(kc, k).T.copy(), device=dev)
        b = torch.empty((k, n), dtype=torch.float64, device=dev)
        iters = torch.zeros(k, dtype=torch.int32, device=dev)
        relres = torch.zeros(k, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream

        def solve():
            L.glm_sur_solve_restricted(h.handle, Ycm.data_ptr(), m, dcm.data_ptr(), kc, k, b.data_ptr(), n,
                                       iters.data_ptr(), relres.data_ptr(), stream)

        solve()
        torch.cuda.synchronize()
        l0 = L.glm_sur_launch_count(h.handle)
        ms, clocks = timed(solve, args.steps, args.warmup, local, pg)
        launches = (L.glm_sur_launch_count(h.handle) - l0) // (args.steps + args.warmup)
        it = iters.cpu().numpy()
        bb = b.t().cpu().numpy()
        # sampled accuracy: two columns against the structured direct solve with restrictions
        cols = [0, k - 1] if k > 1 else [0]
        ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y[:, cols], C=p.C, d=np.asarray(p.d).reshape(kc, k)[:, cols])
        err = rel_err(bb[:, cols], ref)
        prof = L.glm_sur_profile_steps(h.handle, 5, stream)
        G, M = p.G, p.M
        flops = 2 * M * G * G * k + 4 * M * n * k     # Sigma-apply + the two projections of one step
        out[k] = dict(ms=ms, clocks=clocks, launches=launches, iters_max=int(it.max()), err=err,
                      status=L.glm_sur_get_status(h.handle, k), step_ms=prof[4], kernel_ms=prof[:4],
                      step_gflops=flops / (prof[4] * 1e-3) / 1e9, sigma_gflops=2 * M * G * G * k / (prof[0] * 1e-3) / 1e9,
                      p=p, h=h, Ycm=Ycm, dcm=dcm, b=b, iters=iters, relres=relres, solve=solve)
    r = out[32]
    ms, value = aggregate(r["ms"], pg, world, dev)
    p, h = r["p"], r["h"]
    k, m, n, kc = 32, p.m, p.n, p.C.shape[0]
    Yh = torch.as_tensor(p.Y.T.copy()).pin_memory()
    bh = torch.empty((k, n), dtype=torch.float64).pin_memory()
    Y2 = torch.empty_like(r["Ycm"])
    e2e = []
    for s in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Y2.copy_(Yh, non_blocking=True)
        L.glm_sur_solve_restricted(h.handle, Y2.data_ptr(), m, r["dcm"].data_ptr(), kc, k, r["b"].data_ptr(), n,
                                   r["iters"].data_ptr(), r["relres"].data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
        bh.copy_(r["b"], non_blocking=True)
        torch.cuda.synchronize()
        if s >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    # the k = 32 solve on the row-reduced model (Remark rem:reduction)
    reduced = None
    if not args.no_reduced:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hr = GlmSur(p.X_blocks, p.Omega, precision="fp64", tol=1e-13, reduce_rows=True, device=dev)
        hr.set_restrictions(p.C)
        torch.cuda.synchronize()
        setup_r = (time.perf_counter() - t0) * 1e3

        def solve_r():
            L.glm_sur_solve_restricted(hr.handle, r["Ycm"].data_ptr(), m, r["dcm"].data_ptr(), kc, k,
                                       r["b"].data_ptr(), n, r["iters"].data_ptr(), r["relres"].data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)

        solve_r()
        torch.cuda.synchronize()
        ms_r, _ = timed(solve_r, max(1, args.steps), 1, local, None)
        bb = r["b"].t().cpu().numpy()
        cols = [0, k - 1]
        ref = O.sur_gls_structured(p.X_blocks, p.Omega, p.Y[:, cols], C=p.C, d=np.asarray(p.d).reshape(kc, k)[:, cols])
        reduced = {"solves_per_s": 1e3 / ms_r, "ms_per_solve": ms_r, "setup_ms": setup_r,
                   "rel_err_sampled": rel_err(bb[:, cols], ref), "status": L.glm_sur_get_status(hr.handle, k),
                   "iters_max": int(r["iters"].cpu().numpy().max()), "rows": int(n)}
        hr.close()
    cpu = None
    if rank == 0 and not args.no_cpu:
        q = S.constrained_g32_m50000(k=k)
        n_it = 3
        t0 = time.perf_counter()
        O.rglm_pcg_aug(q.X_blocks, q.Omega, q.Y, q.C, q.d, tol=0.0, maxit=n_it, stag_window=10 ** 9)
        dt = (time.perf_counter() - t0) / n_it
        cpu = {"value": 1.0 / (dt * r["iters_max"]), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n_it} steps of the oracle's restricted PCG (k={k}; setup included) timed, x "
                         f"{r['iters_max']} steps per solve (the GPU run's count)"}
    if rank == 0:
        line = base_line(args, world, METRIC, "constrained-g32-m50000-kc64-k32 (n_i=16, C 64x512 N(0,1), d=C beta, "
                         "Omega eigenvalues log-U[0.1,10])", value, "solves/s", ms, "f64",
                         {"G": 32, "M": 50000, "n": n, "kc": kc, "k": k, "precision": "fp64", "tol": 1e-13,
                          "l2": "Q 205 MB f64, vectors 410 MB at k=32"})
        line.update({
            "rel_err_sampled": r["err"], "status": r["status"], "iters_max": r["iters_max"],
            "k1": {"solves_per_s": 1e3 / out[1]["ms"], "ms": out[1]["ms"], "iters_max": out[1]["iters_max"],
                   "rel_err": out[1]["err"], "step_ms": out[1]["step_ms"]},
            "row_reduced": reduced,
            "roofline": {"bound": "alu", "kernel": "k_sigma_step", "achieved": r["sigma_gflops"],
                         "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": r["sigma_gflops"] / FP64_PEAK_GFLOPS,
                         "traffic": None, "peak_source": "nominal float64 FMA rate (1.25 TFLOP/s)",
                         "flops_per_launch": 2 * 50000 * 32 * 32 * k, "ms": r["kernel_ms"][0]},
            "roofline_iter": {"bound": "alu", "achieved": r["step_gflops"], "peak": FP64_PEAK_GFLOPS,
                              "unit": "GFLOP/s", "frac": r["step_gflops"] / FP64_PEAK_GFLOPS, "ms": r["step_ms"],
                              "kernel_ms": r["kernel_ms"]},
            "cpu_baseline": cpu,
            "e2e": {"value": world / float(np.mean(e2e)), "unit": "solves/s", "h2d_bytes_per_step": int(m * k * 8),
                    "d2h_bytes_per_step": int(n * k * 8)},
            "gpu_launches": int(r["launches"]), "clocks": r["clocks"]})
        print(json.dumps(line))
    for kk in out:
        out[kk]["h"].close()
    return 0


def run_differentiable(args, rank, world, local, pg):
    """G = 128, M = 40000, Omega = L L^T (cond ~ 3.5e6): forward solve plus the
    adjoint solve and the dL/dOmega reduction, loss ||b - beta_target||^2.
    The line's value is the row-reduced model (Remark rem:reduction: every
    equation on the n rotated rows of range([X_1 ... X_G])) with the
    preconditioner block D = diag(Sigma) (Sec. "Scaling of Sigma") in float64
    steps; the full M-row model in float32 steps with float64 refinement is
    timed beside it (key full_model)."""
    import torch
    from paper_2510_14471_gb300 import build
    if rank == 0:
        build.build()
    if pg is not None:
        pg.barrier()
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmSur
    from synth import sur_inputs as S
    from oracle import sur_oracle as O
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p, Lfac, target = S.differentiable_g128_m40000()
    m, n, G, M = p.m, p.n, p.G, p.M
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "differentiable_g128_m40000_reference.json")))
    Ycm = torch.as_tensor(p.Y.T.copy(), device=dev)
    tgt = torch.as_tensor(target[:, 0], device=dev)
    b = torch.empty((1, n), dtype=torch.float64, device=dev)
    gb = torch.empty((1, n), dtype=torch.float64, device=dev)
    dY = torch.empty((1, m), dtype=torch.float64, device=dev)
    dO = torch.empty((G, G), dtype=torch.float64, device=dev)
    it_f = torch.zeros(1, dtype=torch.int32, device=dev)
    it_b = torch.zeros(1, dtype=torch.int32, device=dev)
    rr = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def step_of(h):
        def step():
            L.glm_sur_solve(h.handle, Ycm.data_ptr(), m, 1, b.data_ptr(), n, it_f.data_ptr(), rr.data_ptr(), stream)
            torch.sub(b[0], tgt, out=gb[0]).mul_(2.0)          # dL/db of the loss (marshalling)
            L.glm_sur_backward(h.handle, gb.data_ptr(), n, 1, dY.data_ptr(), m, dO.data_ptr(), G, it_b.data_ptr(),
                               rr.data_ptr(), stream)
        return step

    def errors():
        bb = b[0].cpu().numpy()
        om = dO.cpu().numpy().reshape(-1)[gold["dOmega_idx"]]
        return (float(np.linalg.norm(bb - np.asarray(gold["b"])) / np.linalg.norm(gold["b"])),
                float(np.linalg.norm(om - np.asarray(gold["dOmega_sym"])) / np.linalg.norm(gold["dOmega_sym"])))

    # the full model: float32 steps, float64 refinement, D = I
    h = GlmSur(p.X_blocks, p.Omega, precision="fp32_refine", stagnation_window=1000, max_refine=20, device=dev)
    ms_f, clocks_f = timed(step_of(h), args.steps, args.warmup, local, pg)
    ms_f, value_f = aggregate(ms_f, pg, world, dev)
    err_b_f, err_om_f = errors()
    iters_full = (int(it_f.item()), int(it_b.item()))
    prof = L.glm_sur_profile_steps(h.handle, 20, stream)
    h.close()
    hbm, src = load_peaks()
    pb, k = 4, 1
    kbytes = {"sigma_step": 6 * pb * m * k, "proj_partial": pb * M * n + pb * m * k, "reduce": 0,
              "proj_update": pb * M * n + 3 * pb * m * k}
    names = ["sigma_step", "proj_partial", "reduce", "proj_update"]
    dom = max(range(4), key=lambda i: prof[i])
    ach = kbytes[names[dom]] / (prof[dom] * 1e-3) / 1e9
    b_iter = 2 * pb * M * n + 8 * pb * m * k
    ach_iter = b_iter / (prof[4] * 1e-3) / 1e9
    full_model = {"value": value_f, "unit": "forward+adjoint/s", "ms": ms_f, "rel_err_b": err_b_f,
                  "rel_err_dOmega_sampled": err_om_f, "iters_forward": iters_full[0], "iters_adjoint": iters_full[1],
                  "precision": "fp32_refine", "precond": "identity", "clocks": clocks_f,
                  "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": hbm, "unit": "GB/s",
                               "frac": ach / hbm, "traffic": None, "peak_source": src,
                               "algorithmic_bytes": kbytes[names[dom]], "ms": prof[dom]},
                  "roofline_iter": {"bound": "hbm", "achieved": ach_iter, "peak": hbm, "unit": "GB/s",
                                    "frac": ach_iter / hbm, "B_iter": b_iter, "ms": prof[4],
                                    "kernel_ms": dict(zip(names, prof[:4]))},
                  "l2": "Q 287 MB f32 + 573 MB f64, vectors 20-41 MB"}
    cpu = None
    if rank == 0 and not args.no_cpu:
        t0 = time.perf_counter()
        bo = O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, 0 * target)[0]
        O.sur_gls_gradient_kron(p.X_blocks, p.Omega, p.Y, 2 * (bo - target))
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "forward+adjoint/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the oracle's Kronecker-inverse GLS and adjoint (normal equations, float64), two calls, "
                         f"{dt:.1f} s"}
    # the row-reduced model with D = diag(Sigma), float64 steps: dL/dY = S Q dL/dy'~
    hr = GlmSur(p.X_blocks, p.Omega, precision="fp64", precond="diag", stagnation_window=1000, reduce_rows=True,
                device=dev)
    l0 = L.glm_sur_launch_count(hr.handle)
    ms, clocks = timed(step_of(hr), args.steps, args.warmup, local, pg)
    launches = (L.glm_sur_launch_count(hr.handle) - l0) // (args.steps + args.warmup)
    ms, value = aggregate(ms, pg, world, dev)
    err_b, err_om = errors()
    iters_fb = (int(it_f.item()), int(it_b.item()))
    # step kernels of the reduced model (n rows per equation, float64): the
    # Sigma-apply is 2 n G^2 flops per right-hand side on the FP64 pipe; the
    # projections read the n x n factor (25.7 MB, L2-resident) twice
    prof_r = L.glm_sur_profile_steps(hr.handle, 20, stream)
    sig_flops = 2 * n * G * G * k
    step_flops = sig_flops + 4 * n * n * k
    # end to end: Y from the host, b, dL/dY and dL/dOmega back
    Yh = torch.as_tensor(p.Y.T.copy()).pin_memory()
    Y2 = torch.empty_like(Ycm)
    bh = torch.empty((1, n), dtype=torch.float64).pin_memory()
    dYh = torch.empty((1, m), dtype=torch.float64).pin_memory()
    dOh = torch.empty((G, G), dtype=torch.float64).pin_memory()
    e2e = []
    for s in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Y2.copy_(Yh, non_blocking=True)
        L.glm_sur_solve(hr.handle, Y2.data_ptr(), m, 1, b.data_ptr(), n, it_f.data_ptr(), rr.data_ptr(), stream)
        torch.sub(b[0], tgt, out=gb[0]).mul_(2.0)
        L.glm_sur_backward(hr.handle, gb.data_ptr(), n, 1, dY.data_ptr(), m, dO.data_ptr(), G, it_b.data_ptr(),
                           rr.data_ptr(), stream)
        bh.copy_(b, non_blocking=True)
        dYh.copy_(dY, non_blocking=True)
        dOh.copy_(dO, non_blocking=True)
        torch.cuda.synchronize()
        if s >= 1:
            e2e.append(time.perf_counter() - t0)
    hr.close()
    if rank == 0:
        line = base_line(args, world, "SUR GLS forward+adjoint/sec @ <=1e-9 rel err vs refined FP64 oracle",
                         "differentiable-g128-m40000 (n_i~U{4..24}, Omega=LL^T cond ~3.5e6, loss ||b-t||^2)",
                         value, "forward+adjoint/s", ms, "f64",
                         {"G": G, "M": M, "n": n, "k": 1, "precision": "fp64", "precond": "diag",
                          "reduce_rows": True, "rows_per_equation": n, "tol": 1e-13, "stagnation_window": 1000,
                          "l2": "every solve reads the basis Q_W (574 MB, larger than L2) in its rotation; "
                                "reduced factor 25.7 MB L2-resident"})
        line.update({
            "rel_err_b": err_b, "rel_err_dOmega_sampled": err_om,
            "iters_forward": iters_fb[0], "iters_adjoint": iters_fb[1],
            "full_model": full_model,
            "speedup_vs_full_model": value / value_f,
            "roofline": {"bound": "alu", "kernel": "k_sigma_step (float64, reduced rows)",
                         "achieved": sig_flops / (prof_r[0] * 1e-3) / 1e9, "peak": FP64_PEAK_GFLOPS,
                         "unit": "GFLOP/s", "frac": sig_flops / (prof_r[0] * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                         "traffic": None, "peak_source": "nominal float64 FMA rate (1.25 TFLOP/s)",
                         "flops_per_launch": sig_flops, "ms": prof_r[0]},
            "roofline_iter": {"bound": "alu", "achieved": step_flops / (prof_r[4] * 1e-3) / 1e9,
                              "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                              "frac": step_flops / (prof_r[4] * 1e-3) / 1e9 / FP64_PEAK_GFLOPS, "ms": prof_r[4],
                              "kernel_ms": dict(zip(names, prof_r[:4]))},
            "cpu_baseline": cpu,
            "e2e": {"value": world / float(np.mean(e2e)), "unit": "forward+adjoint/s",
                    "h2d_bytes_per_step": int(m * 8), "d2h_bytes_per_step": int((n + m + G * G) * 8)},
            "gpu_launches": int(launches), "clocks": clocks})
        print(json.dumps(line))
    return 0


# the six restricted VAR models of the paper's second experiment (sparsity
# factor, largest root, condition number of Omega0), on synthetic data
VAR_MODELS = ((0.26, 0.90, 4.48), (0.26, 1.05, 4.48), (0.26, 0.90, 448.0), (0.26, 1.05, 448.0),
              (0.80, 0.90, 448.0), (0.80, 1.05, 448.0))


def run_var(args, rank, world, local, pg):
    """Restricted VAR(4) models, G = 12, M = 300, N = 60, k = 1: MVRGLM and
    PCG-Aug (the SUR model without the excluded regressors) with D = alpha I
    (K1) and D = diag(Sigma) (K2), and PCG-NE, each to tol 1e-10 (the
    explosive models floor near 1e-9 .. 1e-8 and end stagnated); steps, time
    per solve and the error against the oracle's structured GLS solve."""
    import torch
    from paper_2510_14471_gb300 import build
    if rank == 0:
        build.build()
    if pg is not None:
        pg.barrier()
    from paper_2510_14471_gb300 import _lib as L
    from paper_2510_14471_gb300.sur import GlmMvrglm, GlmSur
    from synth import var_inputs as V
    from oracle import sur_oracle as O
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    models = []
    launches = 0
    total_ms = 0.0
    total_solves = 0
    clocks_all = None
    for mi, (sp, lam, oc) in enumerate(VAR_MODELS):
        p = V.var_problem(sparsity=sp, lam_max=lam, omega_cond=oc, k=1, seed=2510014471 + 50 + mi)
        ref_free = O.sur_gls_structured(p.free_blocks(), p.Omega0, p.y_vec())
        ref = np.zeros((p.N, p.G))
        off = 0
        for i, f in enumerate(p.free):
            ref[f, i] = ref_free[off:off + f.size, 0]
            off += f.size
        row = {"sparsity": sp, "lam_max": lam, "omega_cond": oc, "restrictions": int(sum(p.k_i)),
               "cond_Z0": float(np.linalg.cond(p.Z0))}
        Yd = torch.as_tensor(p.Y, device=dev)
        yv = torch.as_tensor(p.y_vec(), device=dev)
        for name, make, call, to_b in (
                ("mvrglm_K1", lambda: GlmMvrglm(p.Z0, p.Omega0, p.C_list, precond="scaled", tol=1e-10,
                                                stagnation_window=1000, maxit=5000, device=dev),
                 lambda h: h.solve(Yd), lambda r: r.b[:, :, 0].cpu().numpy()),
                ("mvrglm_K2", lambda: GlmMvrglm(p.Z0, p.Omega0, p.C_list, precond="diag", tol=1e-10,
                                                stagnation_window=1000, maxit=5000, device=dev),
                 lambda h: h.solve(Yd), lambda r: r.b[:, :, 0].cpu().numpy()),
                ("pcg_aug_K1", lambda: GlmSur(p.free_blocks(), p.Omega0, precond="scaled", tol=1e-10,
                                              stagnation_window=1000, maxit=5000, device=dev),
                 lambda h: h.solve(yv), None),
                ("pcg_aug_K2", lambda: GlmSur(p.free_blocks(), p.Omega0, precond="diag", tol=1e-10,
                                              stagnation_window=1000, maxit=5000, device=dev),
                 lambda h: h.solve(yv), None),
                ("pcg_ne", lambda: GlmSur(p.free_blocks(), p.Omega0, tol=1e-10, maxit=20000, device=dev),
                 lambda h: h.solve_ne(yv), None)):
            h = make()
            r = call(h)
            torch.cuda.synchronize()
            l0 = L.glm_sur_launch_count(h.handle)
            ms, clocks = timed(lambda: call(h), args.steps, args.warmup, local, pg)
            launches += (L.glm_sur_launch_count(h.handle) - l0) * args.steps // (args.steps + args.warmup)
            clocks_all = clocks if clocks_all is None else clocks_all
            if to_b is not None:
                B = to_b(r)
            else:
                bf = r.b[:, 0].cpu().numpy()
                B = np.zeros((p.N, p.G))
                off = 0
                for i, f in enumerate(p.free):
                    B[f, i] = bf[off:off + f.size]
                    off += f.size
            row[name] = {"steps": int(r.iters.max().item()), "ms": float(ms), "status": [int(v) for v in r.status],
                         "rel_err": float(np.linalg.norm(B - ref) / np.linalg.norm(ref))}
            total_ms += float(ms)
            total_solves += 1
            h.close()
        models.append(row)
    if rank == 0:
        line = base_line(args, world, "restricted VAR solves/s (MVRGLM, PCG-Aug, PCG-NE)",
                         "var-g12-m300-n60 (six restricted VAR(4) models, k=1)",
                         1000.0 * total_solves / total_ms, "solves/s", total_ms / total_solves, "f64",
                         {"workload": "var-g12-m300-n60", "G": 12, "M": 300, "N": 60, "k": 1})
        line.update({"models": models, "gpu_launches": int(launches), "clocks": clocks_all})
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    rank, world, local, pg = dist_init(args)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world, pg)
        if args.workload == "batched":
            return run_batched(args, rank, world, local, pg)
        if args.workload == "constrained":
            return run_constrained(args, rank, world, local, pg)
        if args.workload == "differentiable":
            return run_differentiable(args, rank, world, local, pg)
        if args.workload == "var":
            return run_var(args, rank, world, local, pg)
        return run_ours(args, rank, world, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
