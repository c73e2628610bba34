"""Benchmark: SLR-preconditioned CG solves/s on one GB300 (and N replicas).

Workload (default): 3-D 7-point Laplacian 64^3 (n = 262,144), Dirichlet, 4x4x4
box partition (64 subdomains of 16^3), rank k = 32 from 5k Lanczos steps, one
right-hand side b = A x*, x* uniform[-1,1) from a seed, PCG to 1e-8 relative
residual.  A step is one full solve; the FP64 path is the headline (`value`),
the mixed path (FP32 apply, FP64 outer loop) is reported beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SLR-PCG solves/s to 1e-8 residual, mixed vs FP64; apply GB/s; p50/p99 latency"
L2_BYTES = 129 * 2 ** 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 FMA peak: 1.25 TFLOP/s nominal for the GB300 (152 SMs, 2070 MHz max),
# i.e. 2 FP64 FMA per SM per clock.
FP64_PEAK_TFLOPS = 1.25


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = []
        mx = 0.0
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
            except ValueError:
                continue
            for nm, v in zip(names, r[3:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def band_source_sha():
    """SHA-256 over the band kernel's sources (kernel template and both instantiation units)."""
    import hashlib
    hsh = hashlib.sha256()
    for f in ("slr_band_kernel.cuh", "slr_band.cu", "slr_band_half.cu"):
        hsh.update(open(os.path.join(ROOT, "paper_1505_04340_gb300", "csrc", f), "rb").read())
    return hsh.hexdigest()


def captured_traffic(summary):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel source changed since the capture (its SHA-256 is recorded there)."""
    try:
        kv = {}
        for line in open(os.path.join(ROOT, "profiles", summary)):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.split("#")[0].strip()
        sha = band_source_sha()
        return int(kv["traffic_bytes_per_launch"]) if kv.get("source_sha256") == sha else None
    except (OSError, KeyError, ValueError):
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(units, seconds, device=None):
    """Whole-job throughput over the ranks of the current process group.

    Returns (units summed over ranks / slowest rank's seconds, total units,
    max seconds).  Without an initialised group it is this process's own ratio.
    """
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units / seconds, units, seconds
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(u.item()), float(t.item())


def build_problem(name):
    import slrgen
    if name == "3d64":
        return slrgen.config2(), "3d-laplace-64^3-p64-k32"
    if name == "2d32":
        return slrgen.config1(), "2d-laplace-32x32-p4-k8"
    raise ValueError(name)


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_sample(P, iters_full, sample_its=3):
    """Time `sample_its` oracle PCG iterations (A product + SLR apply) on the full problem.

    The oracle's own Lanczos runs with k+1 steps here: the per-iteration cost of
    the apply depends on k, not on how converged the Ritz pairs are.
    """
    import scipy.sparse as sp
    from oracle.slr_oracle import SLR as OracleSLR
    t0 = time.perf_counter()
    ora = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, lanczos_steps=P.k + 1)
    t_setup = time.perf_counter() - t0
    b = ora.to_dd(P.b[:, 0])
    r = b.copy()
    p = ora.apply(r)
    t0 = time.perf_counter()
    for _ in range(sample_its):
        q = ora.App @ p
        r = r - 1e-3 * q
        z = ora.apply(r)
        p = z + 1e-3 * p
    t_it = (time.perf_counter() - t0) / sample_its
    return t_it, t_setup, t_it * iters_full


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    P, wname = build_problem(args.problem)
    # a full solve of this workload takes this many iterations with the same method
    iters_full = int(args.ref_iters)
    from oracle.slr_oracle import SLR as OracleSLR
    ora = OracleSLR(P.rowptr, P.colind, P.val, P.part, P.nparts, P.k, lanczos_steps=P.k + 1)
    b = ora.to_dd(P.b[:, 0])

    def step():
        r = b.copy()
        p = ora.apply(r)
        for _ in range(args.ref_sample_its):
            q = ora.App @ p
            r = r - 1e-3 * q
            p = ora.apply(r) + 1e-3 * p

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    per_it = dt / (args.ref_sample_its + 1)
    value = 1.0 / (per_it * iters_full)
    sample = (f"{args.ref_sample_its + 1} SLR applies + {args.ref_sample_its} A products per step on the full "
              f"workload, scaled to a {iters_full}-iteration solve")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": P.n, "nparts": P.nparts, "k": P.k, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_profile(args):
    """Setup, warm-up, then `steps` solves inside the NVTX range "timed" (for ncu)."""
    import torch
    import paper_1505_04340_gb300 as pkg
    from paper_1505_04340_gb300 import SLR
    pkg.load()
    P, _ = build_problem(args.problem)
    b = torch.tensor(P.b[:, 0], device="cuda")
    h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps,
            precision=args.precision, nrhs_max=1, flexible_cg=(args.precision == "mixed"),
            host_loop=args.host_loop, autotune=not args.no_autotune)   # the bench's kernel choices
    info = h.get_info()
    f = torch.randn(info["n_interior"], dtype=torch.float64, device="cuda")
    g = torch.randn(info["s"], dtype=torch.float64, device="cuda")
    r = torch.randn(P.n, dtype=torch.float64, device="cuda")
    step = {"pcg": lambda: h.pcg(b), "bsolve": lambda: h.bsolve(f), "csolve": lambda: h.csolve(g),
            "apply": lambda: h.apply(r)}[args.profile_kernel]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    x, its, rel, st = h.pcg(b)
    inf = h.get_info()
    print(json.dumps({"profile": args.precision, "kernel": args.profile_kernel, "iterations": int(its[0]),
                      "relres": float(rel[0]), "launches_total": pkg.slr.kernel_launches(),
                      "band_split": inf["band_split"], "band_threads": inf["band_threads"],
                      "band_source_sha256": band_source_sha()}))
    h.close()


def run_indefinite(args, dev):
    """Section 6's symmetric indefinite problem at the bench's size: the 3-D 64^3
    Laplacian shifted by s = 0.05 (-Laplacian u - c u = f), the same 4x4x4 boxes,
    SLR with an SPD interface and rank k, GMRES(40) to 1e-8.  Solves/s with the
    right-hand side resident on the device; setup reported apart, as in the paper."""
    import torch
    import slrgen
    from paper_1505_04340_gb300 import SLR
    P = slrgen.make_problem("3d-laplace-64^3-shift0.05-p64", (64, 64, 64), (4, 4, 4), args.indefinite_k,
                            shift=0.05)
    b = torch.tensor(np.ascontiguousarray(P.b[:, 0]), device=dev)
    out = {"workload": P.name, "k": P.k, "lanczos_steps": P.lanczos_steps, "restart": 40, "tol": 1e-8}
    for prec in ("fp64", "mixed"):
        t0 = time.perf_counter()
        h = SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps,
                precision=prec, indefinite=True, autotune=not args.no_autotune)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        x, its, rel, st = h.gmres(b, restart=40, check=False)          # warm-up, and the iteration count
        reps = 3
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            h.gmres(b, restart=40, check=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        err = float(np.linalg.norm(x.cpu().numpy() - P.xstar[:, 0]) / np.linalg.norm(P.xstar[:, 0]))
        out[prec] = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": int(its[0]),
                     "relres": float(rel[0]), "status": int(st), "x_rel_err": err, "setup_s": setup_s,
                     "theta": h.get_info()["theta"]}
        h.close()
    return out


def run_serving(args, dev):
    """Config-5 request stream through the solve server: a cold pass (each matrix
    set up on its first request) and a warm pass over the same stream (all resident)."""
    import torch
    import slrgen
    from paper_1505_04340_gb300 import serving
    specs = slrgen.serving_specs(32, seed=3)
    stream = slrgen.serving_requests(count=args.serving_requests, seed=3, nspecs=len(specs), rate=args.serving_rate)
    used = sorted({d["spec"] for d in stream})
    probs = {i: slrgen.serving_problem(specs[i]) for i in used}
    mats = {i: serving.MatrixSpec(p.rowptr, p.colind, p.val, p.part, p.nparts, k=p.k) for i, p in probs.items()}

    def requests():
        out = []
        for d in stream:
            _, b = slrgen.request_rhs(probs[d["spec"]], d["nrhs"], d["rhs_seed"])
            out.append(serving.Request(rid=d["rid"], matrix=d["spec"], b=b[:, 0] if d["nrhs"] == 1 else b,
                                       arrival=d["arrival"]))
        return out

    srv = serving.SolveServer(mats, precision="mixed", nrhs_max=8, tol=1e-8, maxit=300,
                              max_concurrent=args.serving_concurrency, log=sys.stderr)
    res = {}
    try:
        for name in ("cold", "warm"):
            reqs = requests()
            l0 = pkg_launches()
            torch.cuda.synchronize()
            srv.run(reqs, realtime=True)
            torch.cuda.synchronize()
            st = serving.latency_stats(reqs)
            worst = 0.0
            failed = [r for r in reqs if r.x is None]
            for r in failed:
                print(f"[serving] request {r.rid} (matrix {r.matrix}) failed: status {r.status}: {r.error}",
                      file=sys.stderr)
            for r in reqs:
                if r.x is None:
                    continue
                P = probs[r.matrix]
                A = sp.csr_matrix((P.val, P.colind, P.rowptr))
                B, X = r.b.reshape(P.n, -1), r.x.reshape(P.n, -1)
                worst = max(worst, float(np.max(np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0))))
            st.update(max_true_relres=worst, gpu_launches=pkg_launches() - l0,
                      unconverged=sum(r.status != 0 for r in reqs), failed=len(failed),
                      mean_batch_columns=float(np.mean([r.batch for r in reqs])))
            res[name] = st
        res.update(setups=srv.setups, evictions=srv.evictions, batches=srv.batches, matrices=len(mats),
                   requests=len(stream), rate_per_s=args.serving_rate, concurrency=args.serving_concurrency,
                   precision="f32 apply / f64 flexible CG", workload="fv-diffusion pool of %d specs, "
                   "1-8 RHS, Poisson arrivals, seed 3" % len(specs))
    finally:
        srv.close()
    return res


def pkg_launches():
    import paper_1505_04340_gb300 as pkg
    return pkg.slr.kernel_launches()


def run_ours(args):
    import torch
    import paper_1505_04340_gb300 as pkg
    from paper_1505_04340_gb300 import SLR

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.load()
    P, wname = build_problem(args.problem)
    dev = "cuda"
    b = torch.tensor(P.b[:, 0], device=dev)
    stream = torch.cuda.current_stream()

    def make(precision):
        return SLR(P.rowptr, P.colind, P.val, P.part, P.nparts, k=P.k, lanczos_steps=P.lanczos_steps,
                   precision=precision, nrhs_max=1, flexible_cg=(precision == "mixed"),
                   autotune=not args.no_autotune)

    results = {}
    for prec in ("fp64", "mixed"):
        t0 = time.perf_counter()
        h = make(prec)
        setup_s = time.perf_counter() - t0
        x, its, rel, st = h.pcg(b)
        assert st == 0, f"{prec} solve did not converge: {rel}"
        for _ in range(args.warmup):
            h.pcg(b)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(local) if (rank == 0 and prec == "fp64") else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        l0 = pkg.slr.kernel_launches()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        its_all = []
        for i in range(args.steps):
            x, its, rel, st = h.pcg(b)
            ev[i + 1].record(stream)
            its_all.append(int(its[0]))
        torch.cuda.synchronize()
        launches = pkg.slr.kernel_launches() - l0
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
        clocks = sampler.stop() if sampler else None
        job_rate, _, max_s = aggregate(args.steps, total_ms / 1e3, device=dev)
        total_ms = max_s * 1e3
        A_err = None
        if prec == "fp64":
            import scipy.sparse as sp
            A = sp.csr_matrix((P.val, P.colind, P.rowptr))
            xn = x.cpu().numpy()
            A_err = float(np.linalg.norm(P.b[:, 0] - A @ xn) / np.linalg.norm(P.b[:, 0]))
            results["x64"] = xn
        else:
            results["x_mixed_err"] = float(np.linalg.norm(x.cpu().numpy() - results["x64"]) /
                                           np.linalg.norm(results["x64"]))
        # apply alone (apply GB/s) and the dominant kernel alone (K1 band solve)
        info = h.get_info()
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        r = torch.randn(P.n, dtype=torch.float64, device=dev, generator=gen)
        z1 = h.apply(r).cpu().numpy()
        if prec == "fp64":
            results["z64"] = z1
        else:       # the FP32 apply against the FP64 apply on the same vector
            results["apply_rel_diff"] = float(np.abs(z1 - results["z64"]).max() / np.abs(results["z64"]).max())
        na = max(10, args.steps)
        for _ in range(3):
            h.apply(r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(na):
            h.apply(r)
        e1.record(stream)
        torch.cuda.synchronize()
        apply_us = e0.elapsed_time(e1) * 1e3 / na
        f = torch.randn(info["n_interior"], dtype=torch.float64, device=dev)
        out = torch.empty_like(f)
        for _ in range(3):
            h._lib.slr_bsolve(h._h, f.data_ptr(), out.data_ptr(), 1, info["n_interior"], stream.cuda_stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(na):
            h._lib.slr_bsolve(h._h, f.data_ptr(), out.data_ptr(), 1, info["n_interior"], stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        band_us = e0.elapsed_time(e1) * 1e3 / na
        wbytes = 8 if prec == "fp64" else 4
        # one B-solve reads the forward blocks (O_J, D_J) and the backward blocks (O_J^T, D_J^T):
        # band_entries = sum c_i W_i (W_i + 1) per pass
        band_bytes = 2 * info["band_entries"] * wbytes + 2 * info["n_interior"] * wbytes
        band_flops = 2 * 2 * info["band_entries"]
        results[prec] = dict(
            solves_per_s=job_rate, ms_per_step=total_ms / args.steps,
            p50_ms=float(np.percentile(per, 50)), p99_ms=float(np.percentile(per, 99)), iters=its_all[-1],
            setup_s=setup_s, launches=launches, clocks=clocks, relres=float(rel[0]), true_relres=A_err,
            apply_us=apply_us, apply_gbs=info["bytes_per_apply"] / apply_us / 1e3,
            bytes_per_apply=info["bytes_per_apply"], band_us=band_us, band_bytes=band_bytes,
            tuning={"band_split": info["band_split"], "band_slots": info["band_slots"],
                    "c_persistent": info["c_persistent"], "tuned": info["tuned"],
                    "tune_seconds": info["tune_seconds"]},
            band_flops=band_flops, device_bytes=info["device_bytes"], setup_parts=info["setup_seconds"],
            lanczos_parts=info["lanczos_seconds"], band_on_device=info["band_on_device"])
        # end to end through host buffers: pinned b -> device, solve, x -> pinned host
        if prec == "fp64":
            bh = torch.tensor(P.b[:, 0]).pin_memory()
            xh = torch.empty(P.n, dtype=torch.float64).pin_memory()
            bd = torch.empty(P.n, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                bd.copy_(bh, non_blocking=True)
                xd, _, _, _ = h.pcg(bd)
                xh.copy_(xd, non_blocking=True)
                torch.cuda.synchronize()
            e2e_rate, _, _ = aggregate(args.steps, time.perf_counter() - t0, device=dev)
            results["e2e"] = {"value": e2e_rate, "unit": "solves/s", "h2d_bytes_per_step": P.n * 8,
                              "d2h_bytes_per_step": P.n * 8}
        h.close()

    indef_res = run_indefinite(args, dev) if (args.indefinite_k > 0 and ws == 1 and args.problem == "3d64") else None
    serving_res = None
    if args.serving_requests > 0:
        serving_res = run_serving(args, dev)
        for key in ("cold", "warm"):
            st = serving_res[key]
            st["solves_per_s"], _, _ = aggregate(st["solves"], st["span_s"], device=dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    hbm, hbm_src = peaks()
    r64 = results["fp64"]
    # K1 FP64: compare its FMA rate with the FP64 peak and its bytes with HBM; report the binding one
    ach_gbs = r64["band_bytes"] / r64["band_us"] / 1e3
    ach_tf = r64["band_flops"] / r64["band_us"] / 1e6
    frac_hbm, frac_alu = ach_gbs / hbm, ach_tf / FP64_PEAK_TFLOPS
    traffic = captured_traffic("k_band_solve2_fp64_3d64.txt") if args.problem == "3d64" else None
    if frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": ach_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": frac_alu, "traffic": traffic, "kernel": "k_band_solve2<double> (K1, one B-solve)",
                "peak_source": "nominal FP64 (152 SMs x 2 FMA/clk x 2070 MHz); 1.20 measured",
                "hbm_frac": frac_hbm, "algorithmic_bytes": r64["band_bytes"]}
    else:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": frac_hbm,
                "traffic": traffic, "kernel": "k_band_solve2<double> (K1, one B-solve)", "peak_source": hbm_src}
    rm = results["mixed"]
    mixed_band_gbs = rm["band_bytes"] / rm["band_us"] / 1e3
    its_full = r64["iters"]
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        t_it, t_setup, t_solve = oracle_sample(P, its_full)
        cpu = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"3 oracle PCG iterations (A product + SLR apply) on the full workload, "
                         f"{t_it * 1e3:.0f} ms each, scaled to the {its_full}-iteration solve; "
                         f"oracle setup {t_setup:.1f} s excluded as in the metric"}
    line = {
        "metric": METRIC, "value": r64["solves_per_s"], "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": P.n, "nparts": P.nparts, "k": P.k, "lanczos_steps": P.lanczos_steps,
                   "tol": 1e-8, "precision": "fp64", "nrhs": 1,
                   "l2": "working set larger than L2 (band factor %.0f MB > 129 MB)" % (r64["band_bytes"] / 2e6),
                   "parallelism": f"replicas x{ws}", "tuning": r64["tuning"]},
        "iterations": its_full, "p50_ms": r64["p50_ms"], "p99_ms": r64["p99_ms"],
        "true_relres": r64["true_relres"], "setup_s": r64["setup_s"],
        "setup_phases_s": dict(zip(["analysis", "band_factor", "c_factor", "upload", "lanczos"],
                                   [round(x, 4) for x in r64["setup_parts"]]),
                               lanczos_h_apply=round(r64["lanczos_parts"][0], 4),
                               lanczos_reorth=round(r64["lanczos_parts"][1], 4),
                               lanczos_eig=round(r64["lanczos_parts"][2], 4),
                               band_on_device=r64["band_on_device"]),
        "apply": {"us": r64["apply_us"], "gbs": r64["apply_gbs"], "bytes": r64["bytes_per_apply"]},
        "mixed": {"value": rm["solves_per_s"], "ms_per_step": rm["ms_per_step"], "iterations": rm["iters"],
                  "p50_ms": rm["p50_ms"], "p99_ms": rm["p99_ms"], "x_rel_diff_vs_fp64": results["x_mixed_err"],
                  "apply_rel_diff_vs_fp64": results["apply_rel_diff"],
                  "apply_us": rm["apply_us"], "apply_gbs": rm["apply_gbs"],
                  "band_solve_us": rm["band_us"], "band_gbs": mixed_band_gbs,
                  "band_frac_hbm": mixed_band_gbs / hbm,
                  "band_traffic": (captured_traffic("k_band_solve2_fp32_3d64.txt") if args.problem == "3d64" else None),
                  "dtype": "f32 apply / f64 outer",
                  "tuning": rm["tuning"]},
        "roofline": roof,
        "band_solve_us": r64["band_us"],
        "cpu_baseline": cpu,
        "e2e": results["e2e"],
        "gpu_launches": r64["launches"],
        "clocks": r64["clocks"],
        "serving": serving_res,
        "indefinite": indef_res,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--problem", default="3d64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-iters", type=int, default=22,
                    help="iterations of a full solve of the workload (measured by the GPU arm)")
    ap.add_argument("--ref-sample-its", type=int, default=2)
    ap.add_argument("--profile", action="store_true", help="solves inside an NVTX range only (for ncu)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--profile-kernel", default="pcg", choices=["pcg", "bsolve", "csolve", "apply"])
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch choices")
    ap.add_argument("--serving-requests", type=int, default=256, help="config-5 request stream length (0: skip)")
    # the 256-request stream carries 4.4 right-hand sides per request on average; 12 requests/s
    # (about 53 solves/s) keeps the server below its measured capacity so latencies are service
    # plus queueing, not a growing backlog
    ap.add_argument("--serving-rate", type=float, default=12.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serving-concurrency", type=int, default=8)
    ap.add_argument("--indefinite-k", type=int, default=64,
                    help="rank of the shifted (indefinite) 3-D 64^3 GMRES(40) leg (0: skip)")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive CG from the host (profilers do not see kernels inside conditional graph nodes)")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
