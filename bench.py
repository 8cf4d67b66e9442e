#!/usr/bin/env python
"""BDDC-PCG on one GB300: time to rtol 1e-8 and M^-1 applies/s, mixed vs FP64.

Workload: 3D Q1 heterogeneous diffusion, 96^3 elements on the unit cube,
12^3 cube subdomains of 8^3 elements, sigma = exp(N(0,1)) per element,
corner + edge + face constraints, f ~ U[-1,1] per node, one right-hand side
(synthetic, seeded). One step = one whole BDDC-PCG solve to rtol 1e-8 (all
hot-path phases: restriction, local and interior solves, coarse residual,
coarse solve, prolongation, SpMV, dot products), inputs resident in HBM.

`value` is solves per second of the headline mixed form (bf16 local and
interior operators with float32 accumulation inside flexible PCG; everything
else float64). The FP64, FP32 and TF32 (tensor-core) forms are timed beside it.
`forms_cfg5` times the 192^3 workload (24^3 subdomains, 8 right-hand sides,
whole solve as one CUDA graph) in FP64 and in the mixed BF16 tensor-core form.
`forms_sparse_local` times the sparse local solver (A_II factorised, interior
solves as its sweeps) on the paper's 2D Poisson workloads: 10^4 dofs per
subdomain, and 6.35 million dofs in 9 x 9 subdomains.

`cpu_baseline` and `--impl reference` time the CPU oracle (the plain
NumPy/SciPy definitions of the paper's Sec. 2) on this same workload: its
setup untimed, then whole PCG solves to rtol 1e-8 (the reference arm times as
many whole solves as its time budget allows and reports that count as steps).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BDDC-PCG time to rtol 1e-8 & M^-1 applies/s, mixed vs FP64, 1 GB300"
WORKLOAD = "3d_q1_96cubed_12cubed_subdomains_lognormal_sigma_1rhs"
RTOL = 1e-8
# DRAM bytes (read + write) of the three operator passes of one apply, from
# ncu captures of the operator kernel on this workload in the bf16 form; no
# figure for other workloads or kernels (traffic is then null).
MEASURED_TRAFFIC = {(WORKLOAD, "bf16", "k_bgemv_tma"): 1.2897e9,   # full operators (full_operators=True)
                    (WORKLOAD, "bf16", "k_sgemv_tma"): 6.6318e8}   # lower triangles, block-row kernel (default)
WORKLOAD5 = "3d_q1_192cubed_24cubed_subdomains_lognormal_sigma_8rhs"
REF_BUDGET_S = 150.0      # reference arm: whole oracle solves are timed until this much time has passed


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"bddc_bench_clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """The largest x over the ranks of the process group (x itself when there
    is no group or one rank): step times are those of the slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, seconds_per_step: float) -> float:
    """Solves per second of the whole job: each of the ws replicas solves one
    problem per step; seconds_per_step is the slowest replica's."""
    return ws / seconds_per_step


def _blas_threads() -> int | None:
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads") or 0) for i in threadpool_info()) or None
    except Exception:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
            if os.environ.get(k):
                return int(os.environ[k])
        return None


def oracle_measure(budget_s: float, max_solves: int, warm_applies: int = 0) -> dict:
    """The CPU oracle on the benchmark workload itself (96^3 elements, 12^3
    subdomains): setup (untimed), then whole PCG solves to rtol 1e-8 until
    budget_s has passed or max_solves are done (at least one)."""
    import synth
    from oracle import Oracle
    p = synth.config(2)
    t0 = time.perf_counter()
    o = Oracle(p.dim, p.ne, p.elem_sigma, p.elem_subdomain, p.n_sub)
    setup_s = time.perf_counter() - t0
    b = o.rhs(p.f[:, 0])
    for _ in range(warm_applies):
        o.apply(o.to_free(b))
    times, iters = [], 0
    t_start = time.perf_counter()
    while not times or (len(times) < max_solves and time.perf_counter() - t_start < budget_s):
        t1 = time.perf_counter()
        _, h = o.pcg(b, RTOL)
        times.append(time.perf_counter() - t1)
        iters = h[0]["iters"]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"setup_s": setup_s, "solve_s": times, "iters": iters, "cores": cores, "blas_threads": _blas_threads()}


ORACLE_CORES = 4   # the oracle's host cores and BLAS threads: its dense LAPACK calls are small
                   # (one subdomain's saddle-point system each), and more threads only slow them


def start_oracle_worker(budget_s: float = 0.0, max_solves: int = 1, warm_applies: int = 0):
    """The oracle in a fresh interpreter (exec, not fork) on the last
    ORACLE_CORES host cores with as many BLAS threads; the GPU process keeps
    the others for its own host setup."""
    n = os.cpu_count() or 1
    env = dict(os.environ)
    cores = list(range(max(0, n - ORACLE_CORES), n))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(len(cores))
    env["BDDC_ORACLE_CORES"] = ",".join(map(str, cores))
    env["BDDC_ORACLE_RUN"] = f"{budget_s},{max_solves},{warm_applies}"
    return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker"], env=env,
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)


def read_oracle_worker(proc, timeout_s: float):
    """(result dict, None) or (None, reason)."""
    try:
        out, err = proc.communicate(timeout=timeout_s)
    except subprocess.TimeoutExpired:
        proc.kill()
        proc.communicate()
        return None, f"the oracle did not finish within {timeout_s:.0f} s"
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    if proc.returncode != 0 or not lines:
        return None, "oracle worker failed: " + (err.strip().splitlines() or ["?"])[-1][:200]
    return json.loads(lines[-1]), None


def collect_oracle_worker(proc, timeout_s: float) -> dict:
    r, why = read_oracle_worker(proc, timeout_s)
    if r is None:
        return {"value": None, "unit": "solves/s", "kind": "oracle", "sample": "not measured: " + why}
    per = float(np.mean(r["solve_s"]))
    return {"value": 1.0 / per, "unit": "solves/s", "cores": r["cores"], "kind": "oracle",
            "blas_threads": r["blas_threads"], "setup_s": r["setup_s"], "solve_s": per, "iters": r["iters"],
            "sample": f"one whole oracle PCG solve to rtol 1e-8 of this workload (96^3 elements, 12^3 subdomains, "
                      f"{r['iters']} iterations) after an untimed oracle setup of {r['setup_s']:.0f} s"}


def oracle_worker_main() -> int:
    cores = os.environ.get("BDDC_ORACLE_CORES")
    if cores and hasattr(os, "sched_setaffinity"):
        os.sched_setaffinity(0, {int(c) for c in cores.split(",")})
    budget, max_solves, warm = os.environ.get("BDDC_ORACLE_RUN", "0,1,0").split(",")
    print(json.dumps(oracle_measure(budget_s=float(budget), max_solves=int(max_solves), warm_applies=int(warm))))
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    r, why = read_oracle_worker(start_oracle_worker(REF_BUDGET_S, max(1, args.steps), 1), timeout_s=3000.0)
    if r is None:
        print(json.dumps({"impl": "reference", "unavailable": why}))
        return 0
    per = float(np.mean(r["solve_s"]))
    value = 1.0 / per
    n = len(r["solve_s"])
    sample = (f"whole oracle PCG solves to rtol 1e-8 of this workload ({r['iters']} iterations each): {n} timed "
              f"(as many as fit in {REF_BUDGET_S:.0f} s), after an untimed oracle setup of {r['setup_s']:.0f} s "
              f"and one untimed apply")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": n, "warmup": 1, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "elements": "96^3", "subdomains": 1728, "nrhs": 1,
                                            "rtol": RTOL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": r["cores"], "kind": "oracle",
                             "blas_threads": r["blas_threads"], "setup_s": r["setup_s"], "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gb300(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_2410_14786_gb300 import BDDC, build

    ws, rank, local = _dist()
    # the oracle baseline runs in its own process on the other host cores
    # while the GPU forms are timed (started before any CUDA call)
    oracle_proc = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.config == 2:
        oracle_proc = start_oracle_worker()
    if ws > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    build.build()

    p = synth.config(args.config, args.nrhs or None)
    nrhs = p.nrhs
    f = torch.from_numpy(np.ascontiguousarray(p.f if nrhs > 1 else p.f[:, 0])).cuda()
    forms = {}
    handles = {}
    precs = ["fp64", "fp32", "tf32", "bf16"] if not args.only else args.only.split(",")
    headline = args.precision if args.precision in precs else precs[-1]
    for prec in precs:
        g = BDDC.from_problem(p, precision=prec, nrhs_max=nrhs, graph=not args.no_graph, coarse=args.coarse,
                              tensor_cores={"auto": "auto", "on": True, "off": False}[args.tensor_cores]
                              if prec in ("bf16", "tf32") else "auto")
        handles[prec] = g
        gi = g.info()
        forms[prec] = {"setup_s": gi["setup_seconds"], "tensor_cores": gi["tensor_cores"],
                       "runs_as": ["fp64", "fp32", "bf16", "tf32"][gi["precision"]]}
        if not args.no_autotune:
            # launch parameters measured on this handle (part of setup, untimed)
            t0 = time.perf_counter()
            forms[prec]["tuning"] = g.autotune(nrhs)
            forms[prec]["autotune_s"] = time.perf_counter() - t0
    g64 = handles.get("fp64", handles[headline])
    b = g64.rhs(f)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    x_ref = None
    for prec in precs:
        g = handles[prec]
        x = torch.empty_like(b)
        for _ in range(args.warmup):
            g.pcg_solve(b, x, rtol=RTOL, maxit=500)
        barrier()
        launches0 = g.info()["kernel_launches"]
        sampler = ClockSampler(local) if prec == headline and rank == 0 else None
        if sampler:
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        iters = []
        for _ in range(args.steps):
            _, res = g.pcg_solve(b, x, rtol=RTOL, maxit=500)
            iters.append(int(res.iters.max()))
        e1.record(stream)
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps)
        launches = g.info()["kernel_launches"] - launches0
        tr = float(((b - g64.matvec(x)).norm() / b.norm()).item())
        forms[prec].update({"ms_per_solve": ms, "iters": iters[-1], "true_relres": tr,
                            "launches_per_solve": launches / args.steps})
        if args.coarse == "cg":
            forms[prec]["coarse_cg_iters_last"] = g.info()["coarse_cg_iters"]
        if prec == "fp64":
            x_ref = x.clone()
        elif x_ref is not None:
            forms[prec]["rel_diff_vs_fp64"] = float(((x - x_ref).norm() / x_ref.norm()).item())
        if clocks is not None:
            forms[prec]["clocks"] = clocks
        # standalone apply throughput (inputs larger than L2: each operator family > 129 MB)
        r = torch.rand_like(b)
        z = torch.empty_like(b)
        for _ in range(3):
            g.apply(r, z)
        n_ap = 20
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n_ap):
            g.apply(r, z)
        a1.record(stream)
        torch.cuda.synchronize()
        ams = a0.elapsed_time(a1) / n_ap
        inf = g.info()
        forms[prec]["apply_ms"] = ams
        forms[prec]["applies_per_s"] = 1e3 / ams
        forms[prec]["apply_GBps"] = inf["apply_bytes_1rhs"] / (ams * 1e-3) / 1e9
        prof = g.profile_apply(r, reps=10)
        forms[prec]["apply_launch_ms"] = prof
        forms[prec]["operator_bytes"] = inf["operator_bytes"]

    head = forms[headline]
    g = handles[headline]
    inf = g.info()
    peak, peak_kind = _peaks()
    prof = head["apply_launch_ms"]
    op_ms = prof["interior_op"] + prof["interface_op"] + prof["interior_op_final"]
    op_bytes = (2 * inf["interior_op_bytes"] + inf["interface_op_bytes"]
                + 8 * 2 * nrhs * (2 * inf["n_interior"] + inf["n_interface_copies"]))
    achieved = op_bytes / (op_ms * 1e-3) / 1e9
    kname = ("k_tc_gemm" if inf["tensor_cores"] else "k_sgemv_tma" if inf["symmetric_operators"]
             else "k_bgemv_tma")
    wl = WORKLOAD if args.config == 2 and nrhs == 1 else p.name
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": MEASURED_TRAFFIC.get((wl, headline, kname)), "peak_kind": peak_kind,
                "kernel": ("k_tc_gemm + k_tc_pack" if inf["tensor_cores"] else kname) + " (3 operator passes per apply"
                          + (", operators stored as lower triangles)" if inf["symmetric_operators"] else ")"),
                "bytes_per_apply": op_bytes}
    # the whole apply (every launch of M^-1 r) against the same peak
    apply_roofline = {"bytes_per_apply": inf["apply_bytes_1rhs"] * nrhs if nrhs == 1 else None,
                      "apply_ms": head["apply_ms"],
                      "achieved_GBps": inf["apply_bytes_1rhs"] / (head["apply_ms"] * 1e-3) / 1e9 if nrhs == 1 else None}
    if nrhs == 1:
        apply_roofline["frac"] = apply_roofline["achieved_GBps"] / peak

    # end to end through the public API with host buffers (pinned)
    bh = torch.empty(b.shape, dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    xh = torch.empty_like(bh)
    bn, xn = bh.numpy(), xh.numpy()
    for _ in range(2):
        g.pcg_solve_host(bn, rtol=RTOL, out=xn)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.pcg_solve_host(bn, rtol=RTOL, out=xn)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps)

    for gg in handles.values():
        gg.close()
    handles.clear()
    cfg5 = None
    if args.config == 2 and not args.no_cfg5:
        cfg5 = run_cfg5(args, barrier, peak, peak_kind)

    sparse_local = None
    if args.config == 2 and not args.no_sparse_local:
        sparse_local = run_sparse_local(args, barrier, peak, peak_kind)

    cpu = collect_oracle_worker(oracle_proc, timeout_s=1200.0) if oracle_proc is not None else None

    ms = head["ms_per_solve"]
    line = {
        "metric": METRIC, "value": whole_job_rate(ws, ms * 1e-3), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+" + headline if headline != "fp64" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.config == 2 and nrhs == 1 else p.name, "elements": f"{p.ne}^{p.dim}",
                   "subdomains": p.n_sub, "nrhs": nrhs, "n_c": inf["n_c"], "rtol": RTOL, "mixed_form": headline, "l2": f"inputs larger than L2 (operators {inf['operator_bytes'] / 1e9:.2f} GB)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roofline,
        "apply_roofline": apply_roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": whole_job_rate(ws, e2e_s), "unit": "solves/s", "h2d_bytes_per_step": int(b.numel() * 8),
                "d2h_bytes_per_step": int(b.numel() * 8)},
        "gpu_launches": int(head["launches_per_solve"] * args.steps),
        "clocks": head.get("clocks"),
        "forms": forms,
        "time_to_rtol_ms": {k: v["ms_per_solve"] for k, v in forms.items()},
        "applies_per_s": {k: v["applies_per_s"] for k, v in forms.items()},
        "forms_cfg5": cfg5,
        "forms_sparse_local": sparse_local,
    }
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_cfg5(args, barrier, peak, peak_kind) -> dict:
    """The 192^3 workload (24^3 subdomains of 8^3, 8 right-hand sides, whole
    solve as one CUDA graph): FP64 and the mixed BF16 form on the tensor
    cores, time to rtol 1e-8 per block of 8 solves (steps capped at 3 after
    one untimed solve: a FP64 solve takes seconds), iterations, true
    residual, difference from FP64, and the roofline of the tensor-core
    operator passes."""
    import torch

    import synth
    from paper_2410_14786_gb300 import BDDC
    p = synth.config(5)
    nrhs = p.nrhs
    f = torch.from_numpy(np.ascontiguousarray(p.f)).cuda()
    out = {"workload": WORKLOAD5, "elements": f"{p.ne}^{p.dim}", "subdomains": p.n_sub, "nrhs": nrhs, "rtol": RTOL,
           "steps": min(args.steps, 3), "warmup": 1, "forms": {}}
    x64 = None
    g64 = None
    for prec in ("fp64", "bf16"):
        g = BDDC.from_problem(p, precision=prec, nrhs_max=nrhs)
        fm = {"setup_s": g.info()["setup_seconds"], "tensor_cores": g.info()["tensor_cores"]}
        if not args.no_autotune:
            fm["tuning"] = g.autotune(nrhs)
        b = g.rhs(f)
        x = torch.empty_like(b)
        g.pcg_solve(b, x, rtol=RTOL, maxit=500)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(out["steps"]):
            _, res = g.pcg_solve(b, x, rtol=RTOL, maxit=500)
        e1.record()
        barrier()
        fm["ms_per_solve_block"] = e0.elapsed_time(e1) / out["steps"]
        fm["iters_max"] = int(res.iters.max())
        gm = g64 if g64 is not None else g
        fm["true_relres_max"] = float(((b - gm.matvec(x)).norm(dim=0) / b.norm(dim=0)).max().item())
        prof = g.profile_apply(torch.rand_like(b), reps=3)
        fm["apply_launch_ms"] = prof
        inf = g.info()
        if prec == "fp64":
            x64, g64 = x.clone(), g
        else:
            fm["rel_diff_vs_fp64"] = float(((x - x64).norm() / x64.norm()).item())
            op_ms = prof["interior_op"] + prof["interface_op"] + prof["interior_op_final"]
            op_bytes = (2 * inf["interior_op_bytes"] + inf["interface_op_bytes"]
                        + 8 * 2 * nrhs * (2 * inf["n_interior"] + inf["n_interface_copies"]))
            ach = op_bytes / (op_ms * 1e-3) / 1e9
            fm["roofline"] = {"bound": "hbm", "kernel": "k_tc_gemm + k_tc_pack (3 operator passes per apply)",
                              "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                              "peak_kind": peak_kind, "bytes_per_apply": op_bytes, "traffic": None}
            g.close()
        out["forms"][prec] = fm
    if g64 is not None:
        g64.close()
    out["mixed_speedup_vs_fp64"] = out["forms"]["fp64"]["ms_per_solve_block"] / out["forms"]["bf16"]["ms_per_solve_block"]
    return out


SPARSE_LOCAL_WORKLOADS = [
    # the paper's 2D Poisson workloads (Sec. 3, Fig. 1): 10^4 dofs per
    # subdomain (the local size of its BDDC vs CG comparison), and its
    # strong-scaling problem of 6.35 million dofs split into 9 x 9
    # subdomains of 280^2 elements (78,000 dofs each)
    ("paper_2d_800sq_8x8_subdomains_10k_dofs_each", 800, 8),
    ("paper_2d_2520sq_9x9_subdomains_6.35M_dofs", 2520, 9),
]


def run_sparse_local(args, barrier, peak, peak_kind) -> dict:
    """The sparse local solver on the paper's own 2D workloads (sigma = 1,
    corner and edge constraints, one right-hand side), where a dense A_II^-1
    does not fit (80 MB to 48 GB per subdomain in float64): FP64 and the
    mixed form (BF16 K_GG, float32 interior sweeps) to rtol 1e-8, with
    setup time, iterations, true residual, the apply's phases and the
    interior sweeps' bytes per solve against the HBM peak."""
    import torch

    import synth
    from paper_2410_14786_gb300 import BDDC
    out = {}
    for wi, (name, ne, nsub) in enumerate(SPARSE_LOCAL_WORKLOADS):
        if args.sparse_local_workload >= 0 and wi != args.sparse_local_workload:
            continue
        p = synth.make_problem(2, ne, nsub, "one", 1, k=6, name=name)
        f = torch.from_numpy(np.ascontiguousarray(p.f)).cuda()
        w = {"elements": f"{ne}^2", "subdomains": p.n_sub, "nrhs": 1, "rtol": RTOL, "constraints": "corners+edges",
             "steps": min(args.steps, 5), "warmup": 1, "forms": {}}
        x64 = None
        g64 = None
        for prec in ("fp64", "bf16"):
            g = BDDC.from_problem(p, precision=prec, constraints=3, local_solver="sparse")
            inf = g.info()
            fm = {"setup_s": inf["setup_seconds"], "interior_levels": inf["interior_levels"],
                  "interior_factor_entries": inf["interior_factor_entries"],
                  "interior_bytes_per_solve": inf["interior_op_bytes"], "device_gb": inf["device_bytes"] / 1e9}
            w["n_free"], w["n_c"], w["max_ni"] = inf["n_free"], inf["n_c"], inf["max_ni"]
            b = g.rhs(f[:, 0])
            if prec == "fp64":
                # the interior sweeps split at every height (gather form below
                # it, block form from it on): one interior solve's time each
                scan = {}
                rr = torch.rand_like(b)
                for k in range(inf["interior_levels"] + 1):
                    t = g.get_tuning()
                    t["interior_block_height"] = k
                    g.set_tuning(t)
                    scan[k] = g.profile_apply(rr, reps=3)["interior_op"]
                w["interior_split_scan_ms"] = scan
            fm["tuning"] = g.autotune(1)
            fm["interior_bytes_per_solve"] = g.info()["interior_op_bytes"]
            x = torch.empty_like(b)
            g.pcg_solve(b, x, rtol=RTOL, maxit=500)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(w["steps"]):
                _, res = g.pcg_solve(b, x, rtol=RTOL, maxit=500)
            e1.record()
            barrier()
            fm["ms_per_solve"] = e0.elapsed_time(e1) / w["steps"]
            fm["iters"] = int(res.iters[0])
            gm = g64 if g64 is not None else g
            fm["true_relres"] = float(((b - gm.matvec(x)).norm() / b.norm()).item())
            prof = g.profile_apply(torch.rand_like(b), reps=5)
            fm["apply_launch_ms"] = prof
            sweep_ms = prof["interior_op"] + prof["interior_op_final"]
            # two interior solves per apply: the gather form read once each,
            # plus the compact vectors (operand, two work vectors, result)
            sweep_bytes = 2 * (inf["interior_op_bytes"] + 8 * 4 * inf["n_interior"])
            ach = sweep_bytes / (sweep_ms * 1e-3) / 1e9
            fm["sweeps_roofline"] = {"bound": "hbm",
                                     "kernel": ("interior sweeps, 2 per apply: k_level_sweep per level"
                                                + (", k_block_fwd/bwd from the tuned split height on"
                                                   if prec == "fp64" else " (float32 coefficients)")),
                                     "note": ("bound by the float64 pipe, not HBM" if prec == "fp64" else
                                              "latency-bound: each operand load waits for its index load"),
                                     "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                     "peak_kind": peak_kind, "bytes_per_apply": sweep_bytes, "traffic": None}
            if prec == "fp64":
                x64, g64 = x.clone(), g
            else:
                fm["rel_diff_vs_fp64"] = float(((x - x64).norm() / x64.norm()).item())
                g.close()
            w["forms"][prec] = fm
        if g64 is not None:
            g64.close()
        w["mixed_speedup_vs_fp64"] = w["forms"]["fp64"]["ms_per_solve"] / w["forms"]["bf16"]["ms_per_solve"]
        out[name] = w
        del f
        torch.cuda.empty_cache()
    return out


def run_apply_only(args):
    """A short command for profilers: setup, N applies, one PCG solve."""
    import torch

    import synth
    from paper_2410_14786_gb300 import BDDC, build
    build.build()
    p = synth.config(args.config, args.nrhs or None)
    g = BDDC.from_problem(p, precision=args.precision, nrhs_max=p.nrhs, graph=not args.no_graph,
                          tensor_cores={"auto": "auto", "on": True, "off": False}[args.tensor_cores]
                          if args.precision in ("bf16", "tf32") else "auto")
    f = torch.from_numpy(np.ascontiguousarray(p.f if p.nrhs > 1 else p.f[:, 0])).cuda()
    b = g.rhs(f)
    z = torch.empty_like(b)
    for _ in range(args.apply_only):
        g.apply(b, z)
    x, res = g.pcg_solve(b, rtol=RTOL, maxit=500)
    torch.cuda.synchronize()
    print(json.dumps({"apply_only": args.apply_only, "precision": args.precision, "nrhs": p.nrhs,
                      "tensor_cores": g.info()["tensor_cores"], "iters": int(max(res.iters)),
                      "relres": float(max(res.relres))}))
    g.close()
    return 0


def run_adjoint(args):
    """Adjoint workload on the 96^3 grid and 12^3 partition (884736 element
    conductivities): J(sigma) = 1/2 ||u(sigma) - u_obs||^2, u_obs from the
    forward solve at sigma exp(0.1 N(0,1)). Times the forward solve (setup
    separately) and the backward pass (adjoint BDDC-PCG solve + element
    kernel) through torch.autograd; with --fd N, checks N seeded gradient
    entries against central differences (step 1e-6, each side a fresh setup
    and an FP64 solve to rtol 1e-13)."""
    import torch

    import synth
    from paper_2410_14786_gb300 import BDDC, adjoint, build
    build.build()
    p = synth.config(4)
    dim, ne = p.dim, p.ne
    opts = {"precision": args.only or "fp64"}
    g0 = BDDC.from_problem(p)
    f = torch.from_numpy(np.ascontiguousarray(p.f[:, 0])).cuda()
    b = g0.rhs(f)
    pert = p.elem_sigma * np.exp(0.1 * synth.normal(3004, p.elem_sigma.size))
    gp = BDDC(dim, ne, pert, p.elem_subdomain, p.n_sub)
    u_obs, _ = gp.pcg_solve(b, rtol=1e-13, maxit=2000)
    gp.close()
    n1 = ne + 1
    idx = np.arange(n1 ** dim)
    crd = [idx % n1, (idx // n1) % n1, idx // (n1 * n1)]
    free = torch.from_numpy(~np.any([(c == 0) | (c == ne) for c in crd], axis=0)).cuda()

    def objective(u):
        return 0.5 * ((u - u_obs)[free] ** 2).sum()

    rows = []
    for step in range(args.warmup + args.steps):
        sigma = torch.tensor(p.elem_sigma, dtype=torch.float64, requires_grad=True)
        t0 = time.perf_counter()
        u = adjoint.solve(sigma, b, dim, ne, p.elem_subdomain, p.n_sub, rtol=RTOL, **opts)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J = objective(u)
        J.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if step >= args.warmup:
            rows.append((t1 - t0, t2 - t1))
    fwd = statistics.median(r[0] for r in rows)
    bwd = statistics.median(r[1] for r in rows)
    grad = sigma.grad.numpy().copy()
    line = {"metric": "adjoint dJ/dsigma (forward incl. setup, backward)", "value": 1.0 / (fwd + bwd),
            "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * (fwd + bwd), "higher_is_better": True, "data": "synthetic",
            "dtype": "f64" if opts["precision"] == "fp64" else "f64+" + opts["precision"],
            "config": {"workload": p.name, "elements": f"{ne}^{dim}", "subdomains": p.n_sub, "rtol": RTOL},
            "forward_s": fwd, "backward_s": bwd, "J": float(J)}
    if args.fd:
        gf = BDDC.from_problem(p)
        picks = [int(v % np.uint64(p.elem_sigma.size)) for v in synth.splitmix64(5004, args.fd)]
        hstep = 1e-6

        def J_at(sig):
            gg = BDDC(dim, ne, sig, p.elem_subdomain, p.n_sub)
            uu, rr = gg.pcg_solve(b, rtol=1e-13, maxit=2000)
            gg.close()
            return float(objective(uu))
        errs = []
        for e in picks:
            sp_, sm_ = p.elem_sigma.copy(), p.elem_sigma.copy()
            sp_[e] += hstep
            sm_[e] -= hstep
            fd = (J_at(sp_) - J_at(sm_)) / (2 * hstep)
            errs.append(abs(fd - grad[e]) / max(abs(grad[e]), 1e-300))
        gf.close()
        line["fd_check"] = {"elements": args.fd, "step": hstep, "max_rel_err": max(errs),
                            "median_rel_err": statistics.median(errs)}
    print(json.dumps(line))
    g0.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp64", "fp32", "bf16", "tf32"])
    ap.add_argument("--only", default=None,
                    help="comma-separated forms to time (fp64, fp32, tf32, bf16); default all four")
    ap.add_argument("--nrhs", type=int, default=0,
                    help="development aid: override the workload's number of right-hand sides")
    ap.add_argument("--tensor-cores", default="auto", choices=["auto", "on", "off"],
                    help="where the bf16 / tf32 local operators run (auto: tf32 always, bf16 from 8 rhs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch parameters instead of measuring them at setup")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch each PCG iteration's kernels directly (for profilers); not for timing")
    ap.add_argument("--fd", type=int, default=0,
                    help="with --config 4: check this many gradient entries against central differences")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="workload (2 = the metric's configuration; others for development)")
    ap.add_argument("--apply-only", type=int, default=0,
                    help="profiling aid: set up the headline form, run this many applies and one solve, exit")
    ap.add_argument("--no-cfg5", action="store_true", help="skip the 192^3 workload (forms_cfg5)")
    ap.add_argument("--no-sparse-local", action="store_true",
                    help="skip the sparse local solver on the paper's 2D workloads (forms_sparse_local)")
    ap.add_argument("--sparse-local-only", action="store_true",
                    help="run only the sparse local solver on the paper's 2D workloads and print that section")
    ap.add_argument("--sparse-local-workload", type=int, default=-1,
                    help="with --sparse-local-only: run only this one of its workloads (0 or 1)")
    ap.add_argument("--coarse", default="auto", choices=["auto", "sparse", "dense", "cg"],
                    help="development aid: coarse solve (auto = sparse factorisation; cg = inexact, by plain CG)")
    ap.add_argument("--oracle-worker", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_worker:
        return oracle_worker_main()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.apply_only:
        return run_apply_only(args)
    if args.config == 4:
        return run_adjoint(args)
    if args.sparse_local_only:
        import torch
        torch.cuda.init()
        peak, peak_kind = _peaks()
        print(json.dumps({"forms_sparse_local": run_sparse_local(args, torch.cuda.synchronize, peak, peak_kind)}))
        return 0
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
