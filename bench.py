#!/usr/bin/env python
"""Throughput of the GB300 FEAST eigensolver: converged eigenpairs/s.

Workload: 7-point 3D Laplacian on a 64^3 grid plus a seeded diagonal potential
V ~ U[0, 0.5] (N = 262144), B = I, interval [0, Emax] around the lowest ~100
eigenvalues, M0 = 150, Ne = 8 Gauss nodes, stop at relative residual 1e-10.
One step = one complete FEAST solve (filter passes + Rayleigh-Ritz loops) with
the inputs resident in HBM.  The headline runs the complex-FP32 shifted solves
(fpm(42)=1); the FP64-solve run of the same problem is reported beside it.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl gb300|reference]

Under torchrun (N > 1) every rank solves its own replica of the workload (the
method's independent-interval parallelism, no data exchange); value = total
converged eigenpairs of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged eigenpairs/s at rel. residual 1e-10, mixed vs FP64 FEAST, 1 GB300"
UNIT = "eigenpairs/s"
RES_TOL = 1e-10
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per group-iteration of each COCG step from one ncu
# capture (profiles/cocg_steps_laplace3d_64cube.md), valid only for the kernel
# source they were measured on.
NCU_TRAFFIC = {"source_sha1": "d111b7a42e3d2659aeb3f935d8e05e73d221142c",
               "cocg_step_a": (1.108692e9 + 0.626872e9) / 5, "cocg_step_b": (1.181998e9 + 0.467095e9) / 5}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--side", type=int, default=None, help="grid side (default 64; 96 for --workload stencil27)")
    ap.add_argument("--workload", default="laplace3d", choices=["laplace3d", "stencil27", "batched", "grad48", "hermitian"],
                    help="laplace3d: 7-point 3D Laplacian + potential, B = I (the headline line); stencil27: "
                         "27-point generalized problem, B diagonal, lowest 200 eigenvalues, M0 = 300, Ne = 16; "
                         "batched: 512 2D problems in one batched solve; grad48: eigenvalue-loss forward and "
                         "backward at 48^3")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--inner-tol", type=int, default=2, help="fpm(45): inner solves to 10^-k relative residual")
    ap.add_argument("--inner-maxit", type=int, default=80, help="fpm(46): inner-solver iteration cap")
    ap.add_argument("--node-batch", type=int, default=0, help="fpm(50): contour nodes per inner-solver batch "
                                                                 "(0: the workload's default)")
    ap.add_argument("--rows-per-item", type=int, default=0, help="fpm(51): rows per work item of the COCG gather "
                                                                    "step (0: the library's choice)")
    return ap.parse_args()


def workload(side):
    import feast_workloads as fw

    # contour: Gauss, Ne = 8, ellipse ratio fpm(18) = 200 (vertical axis twice the
    # half-width: keeps the shifted systems better conditioned for COCG)
    return fw.laplace3d_potential(side=side, count=100, m0=150, ne=8, ratio=200, seed=1)


def config_dict(p, extra=None):
    d = {"workload": f"laplace3d_7pt_{round(p.n ** (1 / 3))}^3_potential_U[0,0.5]_seed1",
         "N": p.n, "nnz": p.A.nnz, "M0": p.m0, "Ne": p.ne, "contour_ratio_pct": p.ratio,
         "interval": [p.emin, round(p.emax, 6)], "B": "identity", "tol": RES_TOL,
         "inner_solver": f"COCG, fpm(45)={INNER[0]} (1e-{INNER[0]}), fpm(46)={INNER[1]}, one node per batch "
                         "(fpm(50)=1)",
         "l2": "inputs larger than L2 (each filter block vector 2.5 GB)"}
    if extra:
        d.update(extra)
    return d


ROWS_PER_ITEM = 0
INNER = (2, 80)  # fpm(45), fpm(46) of the 64^3 workload


def cocg_rates(pr, p):
    """Algorithmic GB/s of the two COCG launches of a profiled solve (per-launch
    CUDA events): step A gathers r and reads and writes p, q; step B reads r,
    p, q, writes r and updates the quadrature accumulator.  Padded lanes and
    the matrix's padding entries are not counted."""
    n, W, mt, sc, G = pr["n"], pr["W"], pr["mt"], pr["complex_bytes"], pr["groups"]
    nbp = W / mt  # node lanes per column in a tile
    live = (p.m0 * min(nbp, p.ne)) / (G * W)
    mat = p.A.nnz * (4 + (4 if sc == 8 else 8)) + (p.n + 1) * 4
    if p.B is not None:
        mat += p.n * (sc // 2)  # diagonal of B in the filter precision
    tile = n * W * sc * live
    qb = 4 if sc == 8 else 8  # quadrature accumulator: FP32 in mixed precision
    bytes_a = pr["group_iterations"] * 5 * tile + pr["cocg_a_launches"] * mat
    bytes_b = pr["group_iterations"] * (4 * tile + n * mt * 2 * qb * live)
    gbs_a = bytes_a / (pr["cocg_a_ms"] / 1e3) / 1e9
    gbs_b = bytes_b / (pr["cocg_b_ms"] / 1e3) / 1e9
    return gbs_a, gbs_b


def fpm_for(pkg, p, mixed, profile):
    f = pkg.feast_init()
    f[1], f[2], f[3], f[4], f[17] = p.ne, 10, 40, 1, p.ratio
    f[41] = 1 if mixed else 0
    f[44], f[45] = INNER
    f[49] = 1  # one contour node per batch: groups of a fast node stop early
    f[50] = ROWS_PER_ITEM
    f[52] = 1 if profile else 0
    return f


# ---------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- distributed helpers
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist

    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def _reduce(v, ws, op):
    if ws <= 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(v, ws):
    import torch.distributed as dist

    return _reduce(v, ws, dist.ReduceOp.MAX)


def sum_over_ranks(v, ws):
    import torch.distributed as dist

    return _reduce(v, ws, dist.ReduceOp.SUM)


def throughput(conv_per_rank, ms_per_rank, ws):
    """Whole-job converged eigenpairs/s: all ranks' pairs over the slowest rank's time."""
    return sum_over_ranks(conv_per_rank, ws) / (max_over_ranks(ms_per_rank, ws) / 1000.0)


# ---------------------------------------------------------------- CPU baseline (oracle)
FULL_SOLVE_RECORD = os.path.join(ROOT, "oracle", "full_solve_laplace3d_64.json")
COUNT_RECORD = os.path.join(ROOT, "tests", "golden", "laplace3d_64_count.json")


def oracle_solve_shape():
    """Filter passes and eigenvalue count of the oracle's own full solve of the
    64^3 workload: from the recorded full oracle run (oracle/
    full_solve_laplace3d_64.py) and the Sylvester-inertia count (tests/golden/
    make_laplace3d_64_count.py).  Returns (passes, M, record or None)."""
    rec = None
    if os.path.exists(FULL_SOLVE_RECORD):
        rec = json.load(open(FULL_SOLVE_RECORD))
    M = None
    if os.path.exists(COUNT_RECORD):
        M = int(json.load(open(COUNT_RECORD))["count_in_interval"])
    if rec is not None:
        return int(rec["filter_passes"]), int(M if M is not None else rec["M"]), rec
    return 7, (M if M is not None else 100), None


def cpu_baseline(p, seconds, passes, M):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload (oracle/cpu_sample.py: COCG shifted solves of `cores` start-block
    columns at two contour nodes, extrapolated to every solve of the oracle's
    own full solve, `passes` filter passes), for its M eigenpairs; scaled by
    the recorded ratio of a full oracle solve to the same sample on the same
    kind of host when that record exists.  Returns (eigenpairs/s, cores, text)."""
    import oracle as O  # noqa: F401
    from oracle.cpu_sample import sample_solve_seconds

    t_full, cores, text = sample_solve_seconds(p, seconds, passes)
    _, _, rec = oracle_solve_shape()
    cal = 1.0
    if rec is not None and rec.get("calibration"):
        cal = float(rec["calibration"])
        text += (f"; x {cal:.3f}, the ratio of a full oracle solve ({rec['wall_s']:.0f} s on {rec['cores']} "
                 f"{rec['host']} cores, {rec['filter_passes']} passes) to this sample's estimate on that host")
    return M / (t_full * cal), cores, text + f"; M = {M} (inertia count)"


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    import paper_2002_04807_gb300 as pkg
    from paper_2002_04807_gb300 import build

    rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    build.build()
    pkg.library()
    p = workload(args.side)
    dev = torch.device("cuda", local)
    ia = torch.as_tensor(p.A.indptr).to(dev)
    ja = torch.as_tensor(p.A.indices).to(dev)
    av = torch.as_tensor(p.A.data).to(dev)
    y0 = torch.as_tensor(np.ascontiguousarray(p.y0().T)).to(dev)  # column-major n x m0
    x = torch.empty_like(y0)
    stream = torch.cuda.Stream(device=dev)
    f_mixed = fpm_for(pkg, p, True, False)  # timed solves: no per-launch event profiling
    f_prof = fpm_for(pkg, p, True, True)  # one extra solve after the timed region, for the roofline
    work = torch.empty(pkg.feast_scsr_workspace_bytes(p.n, p.A.nnz, 0, p.m0, f_mixed), dtype=torch.uint8,
                       device=dev)

    def solve(fpm):
        x.copy_(y0)
        r = pkg.feast_scsr_solve_dev(p.n, ia, ja, av, fpm=fpm, emin=p.emin, emax=p.emax, m0=p.m0, x=x,
                                     work=work, stream=stream)
        if r.info != 0:
            raise RuntimeError(f"FEAST info {r.info}")
        conv = int(np.sum(r.res[: r.M] <= RES_TOL))
        return r, conv

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            solve(f_mixed)
        torch.cuda.synchronize()
        barrier(ws)
        clocks = Clocks(local)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        conv_total, n_launch, loops = 0, 0, []
        t_host0 = time.time()
        for _ in range(args.steps):
            r, conv = solve(f_mixed)
            conv_total += conv
            loops.append(r.loop)
            n_launch += int(pkg.feast_last_profile()["launches"])
        ev1.record(stream)
        torch.cuda.synchronize()
        host_s = time.time() - t_host0
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop()
        barrier(ws)
        # per-kernel CUDA-event timings from one more solve of the same problem
        rp, _ = solve(f_prof)
        prof_tot = dict(pkg.feast_last_profile())
        torch.cuda.synchronize()
    ms_max = max_over_ranks(ms, ws)
    value = throughput(conv_total, ms, ws)
    M = r.M

    # FP64 shifted solves on the same problem
    fp64 = None
    if args.fp64_steps > 0:
        f64 = fpm_for(pkg, p, False, False)
        w64 = pkg.feast_scsr_workspace_bytes(p.n, p.A.nnz, 0, p.m0, f64)
        if w64 > work.numel():
            work = torch.empty(w64, dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            solve(f64)
            torch.cuda.synchronize()
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c64 = 0
            for _ in range(args.fp64_steps):
                r64, c = solve(f64)
                c64 += c
            e1.record(stream)
            torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1), ws)
        v64 = sum_over_ranks(c64, ws) / (ms64 / 1000.0)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "loops": r64.loop,
                "M": r64.M, "mixed_over_fp64": value / v64,
                "max_rel_eig_diff_vs_mixed": float(np.max(np.abs(r64.E[:M] - r.E[:M]) / np.abs(r.E[:M])))}

    # roofline of the dominant kernel from the per-launch events of the profiled solve
    pr = prof_tot
    gbs_a, gbs_b = cocg_rates(pr, p)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = FALLBACK_HBM_GBS, "fallback"
    if os.path.exists(peaks_path):
        try:
            pk = json.load(open(peaks_path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in pk:
                    peak, peak_src = float(pk[key]), "measured"
                    break
        except (ValueError, OSError):
            pass
    dom = "cocg_step_a" if pr["cocg_a_ms"] >= pr["cocg_b_ms"] else "cocg_step_b"
    ach = gbs_b if dom == "cocg_step_b" else gbs_a
    import hashlib

    src = os.path.join(ROOT, "paper_2002_04807_gb300", "csrc", "k_filter.cu")
    traffic = None
    if (hashlib.sha1(open(src, "rb").read()).hexdigest() == NCU_TRAFFIC["source_sha1"] and args.side == 64
            and dom in NCU_TRAFFIC):
        launches = pr["cocg_a_launches"] if dom == "cocg_step_a" else pr["cocg_b_launches"]
        # per launch, averaged like `achieved`: per-group traffic x active groups per launch
        traffic = NCU_TRAFFIC[dom] * pr["group_iterations"] / max(launches, 1)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "peak_source": peak_src,
                "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
                "cocg_step_a_gbs": gbs_a, "cocg_step_b_gbs": gbs_b,
                "step_a_staged": int(pr.get("step_a_staged", 0)),
                "step_a_rows_per_item": int(pr.get("step_a_rows_per_item", 0)),
                "cocg_share_of_step": (pr["cocg_a_ms"] + pr["cocg_b_ms"]) / (ms / args.steps),
                "timing": "CUDA events around every COCG launch of one extra solve after the timed region "
                          f"({int(pr['cocg_a_launches'])} step-A launches, {pr['filter_ms']:.0f} ms of filter)"}

    # end to end through the host C ABI (pinned host buffers, copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        import torch as T

        a_h = T.as_tensor(p.A.data).pin_memory().numpy()
        ia_h = T.as_tensor(p.A.indptr).pin_memory().numpy()
        ja_h = T.as_tensor(p.A.indices).pin_memory().numpy()
        y_h = T.as_tensor(p.y0()).pin_memory().numpy()
        # the library's X block in pinned memory, used in place (column-major n x m0)
        x_h = T.empty((p.m0, p.n), dtype=T.float64).pin_memory().numpy().T
        f_host = fpm_for(pkg, p, True, False)
        pkg.feast_scsr_solve("F", p.n, a_h, ia_h, ja_h, fpm=f_host, emin=p.emin, emax=p.emax, m0=p.m0, x0=y_h,
                             x_out=x_h)
        barrier(ws)
        t0 = time.time()
        ce = 0
        e2e_steps = max(1, min(args.steps, 2))
        for _ in range(e2e_steps):
            rh = pkg.feast_scsr_solve("F", p.n, a_h, ia_h, ja_h, fpm=f_host, emin=p.emin, emax=p.emax, m0=p.m0,
                                      x0=y_h, x_out=x_h)
            ce += int(np.sum(rh.res[: rh.M] <= RES_TOL))
        t_e2e = max_over_ranks(time.time() - t0, ws)
        h2d = p.A.data.nbytes + p.A.indptr.nbytes + p.A.indices.nbytes + y_h.nbytes
        d2h = p.n * p.m0 * 8 + 2 * p.m0 * 8
        e2e = {"value": sum_over_ranks(ce, ws) / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "api": "feast_scsr_solve (host buffers)",
               "ms_per_step": 1e3 * t_e2e / e2e_steps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        passes, Mo, _ = oracle_solve_shape()
        v_cpu, cores, sample = cpu_baseline(p, args.cpu_sample_seconds, passes, Mo)
        cpu = {"value": v_cpu, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c32 solves + f64 Rayleigh-Ritz",
               "data": "synthetic (seeded generator, no dataset)",
               "config": config_dict(p, {"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                                         "M_found": M, "loops": loops, "precision": "mixed fpm(42)=1"}),
               "e2e": e2e, "gpu_launches": n_launch, "roofline": roofline, "cpu_baseline": cpu,
               "fp64": fp64, "clocks": clk,
               "phases_ms_per_solve": {k: pr[k] for k in ("filter_ms", "project_ms", "reduce_ms", "ritz_ms")},
               "host_wall_s": host_s}
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import feast_workloads  # noqa: F401
    import oracle as O

    p = workload(args.side)
    O.build()
    passes, Mo, _ = oracle_solve_shape()
    for _ in range(args.warmup):
        cpu_baseline(p, min(args.cpu_sample_seconds, 5.0), passes, Mo)
    vals, samples = [], ""
    t0 = time.time()
    for _ in range(args.steps):
        v, cores, samples = cpu_baseline(p, args.cpu_sample_seconds / max(1, args.steps), passes, Mo)
        vals.append(v)
    wall = time.time() - t0
    value = float(np.mean(vals))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator, no dataset)", "impl": "reference",
           "config": config_dict(p, {"precision": "FP64 oracle", "M": Mo, "filter_passes": passes}),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": samples},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- 27-point generalized workload
def run_stencil27(args):
    """The 27-point generalized problem (B diagonal): the interval holding the
    200 lowest eigenvalues comes from the library's extreme-eigenvalue mode
    (fpm(40) = -1, M0 = 400, timed apart), then mixed and FP64 solves with
    M0 = 300, Ne = 16 on it are timed.  The mixed result is checked on the CPU
    in FP64: residuals, X^T B X = I, eigenvalue count; and against the FP64
    solve."""
    import scipy.sparse as sps
    import torch

    import feast_workloads as fw
    import paper_2002_04807_gb300 as pkg
    from paper_2002_04807_gb300 import build

    rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    build.build()
    pkg.library()
    p = fw.stencil27_generalized(side=args.side)
    k = p.notes["target_count"]
    dev = torch.device("cuda", local)
    ia, ja, av = (torch.as_tensor(p.A.indptr).to(dev), torch.as_tensor(p.A.indices).to(dev),
                  torch.as_tensor(p.A.data).to(dev))
    ib, jb, bv = (torch.as_tensor(p.B.indptr).to(dev), torch.as_tensor(p.B.indices).to(dev),
                  torch.as_tensor(p.B.data).to(dev))
    stream = torch.cuda.Stream(device=dev)
    # interval: the k lowest eigenpairs by the extreme-eigenvalue search
    fx = fpm_for(pkg, p, True, False)
    fx[4], fx[39] = 0, -1
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.time()
        rx = pkg.feast_scsr_extreme_dev(p.n, ia, ja, av, ib=ib, jb=jb, b=bv, fpm=fx, m0=2 * k, stream=stream)
        torch.cuda.synchronize()
        t_search = time.time() - t0
    if rx.info != 0:
        raise RuntimeError(f"extreme-eigenvalue search info {rx.info}")
    # the searched interval holds exactly the k lowest eigenvalues; its lower
    # end (the Gershgorin bound of the scaled pencil) lies well below the
    # spectrum, which makes the contour taller and the inexact shifted solves
    # far better conditioned than Emin = 0 would (8 loops instead of 30)
    emin, emax = rx.emin, rx.emax
    del rx
    torch.cuda.empty_cache()
    y0 = torch.as_tensor(np.ascontiguousarray(p.y0().T)).to(dev)
    x = torch.empty_like(y0)

    def solve(f):
        x.copy_(y0)
        r = pkg.feast_scsr_solve_dev(p.n, ia, ja, av, ib=ib, jb=jb, b=bv, fpm=f, emin=emin, emax=emax, m0=p.m0,
                                     x=x, stream=stream)
        if r.info != 0:
            raise RuntimeError(f"FEAST info {r.info}")
        return r, int(np.sum(r.res[: r.M] <= RES_TOL))

    def timed(f, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                solve(f)
            torch.cuda.synchronize()
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            conv, prof = 0, None
            for _ in range(steps):
                r, c = solve(f)
                conv += c
                pr = pkg.feast_last_profile()
                if prof is None:
                    prof = dict(pr)
                else:
                    for kk in ("cocg_a_ms", "cocg_b_ms", "cocg_a_launches", "cocg_b_launches", "group_iterations",
                               "filter_ms", "project_ms", "reduce_ms", "ritz_ms", "launches"):
                        prof[kk] += pr[kk]
            e1.record(stream)
            torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), ws)
        return r, throughput(conv, e0.elapsed_time(e1), ws), ms, prof

    clocks = Clocks(local)
    clocks.start()
    r, value, ms, pr = timed(fpm_for(pkg, p, True, True), args.steps, args.warmup)
    clk = clocks.stop()
    M = r.M
    E = r.E[:M].copy()
    X = x.cpu().numpy().T[:, :M]  # column-major n x m0 block, first M columns
    fp64 = None
    if args.fp64_steps > 0:
        r64, v64, ms64, _ = timed(fpm_for(pkg, p, False, False), args.fp64_steps, 0)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "loops": r64.loop,
                "M": r64.M, "mixed_over_fp64": value / v64,
                "max_rel_eig_diff_vs_mixed": float(np.max(np.abs(r64.E[:M] - E) / np.abs(E)))}
    # FP64 a-posteriori checks on the CPU
    A = sps.csr_matrix((p.A.data, p.A.indices, p.A.indptr), shape=(p.n, p.n))
    Bd = p.B.data
    AX, BX = A @ X, Bd[:, None] * X
    alpha = max(abs(emin), abs(emax))
    res = np.linalg.norm(AX - BX * E[None, :], axis=0) / (alpha * np.linalg.norm(BX, axis=0))
    checks = {"M": M, "wanted": k, "max_residual_cpu_fp64": float(res.max()),
              "max_abs_XtBX_minus_I": float(np.abs(X.T @ BX - np.eye(M)).max())}
    gbs_a, gbs_b = cocg_rates(pr, p)
    peak = FALLBACK_HBM_GBS
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "c32 solves + f64 Rayleigh-Ritz",
               "data": "synthetic (seeded generator, no dataset)",
               "config": {"workload": f"stencil27_generalized_{args.side}^3_Bdiag_U[1,2]_seed2", "N": p.n,
                          "nnz": p.A.nnz, "M0": p.m0, "Ne": p.ne, "contour_ratio_pct": p.ratio,
                          "interval": [emin, emax], "B": "diagonal U[1,2]", "tol": RES_TOL,
                          "interval_from": "feast_scsr_extreme_dev, fpm(40)=-1, M0 = 2 x 200",
                          "interval_search_s": t_search, "loops": r.loop, "precision": "mixed fpm(42)=1"},
               "fp64": fp64, "checks": checks, "clocks": clk,
               "cocg_gbs": {"step_a": gbs_a, "step_b": gbs_b, "peak": peak,
                            "step_a_staged": int(pr.get("step_a_staged", 0))},
               "phases_ms_per_step": {kk: pr[kk] / args.steps for kk in ("filter_ms", "project_ms", "reduce_ms",
                                                                          "ritz_ms")},
               "gpu_launches": int(pr["launches"])}
        print(json.dumps(out))


# ---------------------------------------------------------------- batched and gradient workloads
def _lib_setup():
    import torch

    import paper_2002_04807_gb300 as pkg
    from paper_2002_04807_gb300 import build

    rank, ws, local = dist_setup()
    torch.cuda.set_device(local)
    build.build()
    pkg.library()
    return pkg, rank, ws


def run_batched(args):
    """512 independent 2D 5-point Laplacians + V ~ U[0,1] (sides log-uniform in
    [32, 256], 8-64 wanted eigenvalues each, M0 = 1.5 x count) in one call of
    the batched host entry point; timed on the host around the call (copies
    of the 512 CSRs in and of the results out included)."""
    import torch

    import feast_workloads as fw

    pkg, rank, ws = _lib_setup()
    t0 = time.time()
    probs = fw.batched_laplace2d()
    t_gen = time.time() - t0
    dicts = [dict(n=p.n, a=p.A.data, ia=p.A.indptr, ja=p.A.indices, emin=p.emin, emax=p.emax, m0=p.m0, x0=None)
             for p in probs]

    def fpm(mixed):
        f = pkg.feast_init()
        f[1], f[2], f[3], f[17], f[41], f[44], f[45] = 8, 10, 40, 200, mixed, 2, 80
        return f

    def run(mixed):
        torch.cuda.synchronize()
        t = time.time()
        st, res = pkg.feast_scsr_solve_batched(dicts, fpm(mixed))
        torch.cuda.synchronize()
        dt = time.time() - t
        if st != 0 or any(r.info != 0 for r in res):
            raise RuntimeError(f"batched FEAST status {st}, infos {sorted(set(r.info for r in res))}")
        return dt, sum(int(np.sum(r.res[: r.M] <= RES_TOL)) for r in res), res

    for _ in range(args.warmup):
        run(1)
    tt, conv = 0.0, 0
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for _ in range(args.steps):
        dt, c, res = run(1)
        tt += dt
        conv += c
    clk = clocks.stop()
    value = conv / tt
    fp64 = None
    if args.fp64_steps > 0:
        dt64, c64, _ = run(0)
        fp64 = {"value": c64 / dt64, "unit": UNIT, "ms_per_step": 1e3 * dt64, "mixed_over_fp64": value / (c64 / dt64)}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c32 solves + f64 Rayleigh-Ritz",
               "data": "synthetic (seeded generator, no dataset)",
               "config": {"workload": "batched_laplace2d_512_sides_32-256_seed3", "problems": len(probs),
                          "sum_N": int(sum(p.n for p in probs)), "sum_M0": int(sum(p.m0 for p in probs)),
                          "wanted": int(sum(p.notes.get("target_count", 0) for p in probs)),
                          "Ne": 8, "contour_ratio_pct": 200, "timing": "host clock around the batched call",
                          "generation_s": t_gen},
               "converged_pairs": conv // args.steps, "max_residual": float(max(r.res[: r.M].max() for r in res)),
               "fp64": fp64, "clocks": clk}
        print(json.dumps(out))


def run_grad(args):
    """The differentiation workload: lowest ~64 eigenvalues of the 48^3
    Laplacian + potential (M0 = 96) as a differentiable tensor, loss
    sum_k g_k lambda_k, backward over A's CSR values; forward and backward
    timed separately with CUDA events."""
    import torch

    import feast_workloads as fw
    from paper_2002_04807_gb300.autograd import feast_eigenvalues

    pkg, rank, ws = _lib_setup()
    p = fw.laplace3d_grad()
    dev = torch.device("cuda")
    ia, ja = torch.as_tensor(p.A.indptr).to(dev), torch.as_tensor(p.A.indices).to(dev)
    x0 = torch.as_tensor(np.ascontiguousarray(p.y0().T)).to(dev)
    f = pkg.feast_init()
    f[1], f[2], f[3], f[17], f[41], f[44], f[45], f[49] = 8, 12, 40, 200, 1, 2, 200, 1

    def step():
        av = torch.as_tensor(p.A.data).to(dev).requires_grad_(True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        ev = feast_eigenvalues(av, ia, ja, p.n, p.emin, p.emax, p.m0, f, x0=x0)
        e1.record()
        g = torch.as_tensor(fw.loss_weights(ev.numel(), 4), device=dev)
        (g * ev).sum().backward()
        e2.record()
        torch.cuda.synchronize()
        return ev.numel(), e0.elapsed_time(e1), e1.elapsed_time(e2)

    for _ in range(args.warmup):
        step()
    M, fw_ms, bw_ms = 0, 0.0, 0.0
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for _ in range(args.steps):
        M, a, b = step()
        fw_ms += a
        bw_ms += b
    clk = clocks.stop()
    if rank == 0:
        out = {"metric": METRIC, "value": M * args.steps / ((fw_ms + bw_ms) / 1e3), "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": (fw_ms + bw_ms) / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "c32 solves + f64 Rayleigh-Ritz and backward", "data": "synthetic (seeded generator, no dataset)",
               "config": {"workload": "laplace3d_7pt_48^3_potential_U[0,0.5]_seed4_eigenvalue_loss", "N": p.n,
                          "M0": p.m0, "M": M, "Ne": 8, "contour_ratio_pct": 200, "tol": 1e-12},
               "forward_ms": fw_ms / args.steps, "backward_ms": bw_ms / args.steps, "clocks": clk}
        print(json.dumps(out))


# ---------------------------------------------------------------- complex Hermitian workload
def run_hermitian(args):
    """The complex Hermitian driver on the bench's 64^3 Laplacian + potential
    with random gauge phases on every site (same ~100 lowest eigenvalues and
    interval as the real workload, every off-diagonal entry complex), M0 = 150,
    Ne = 8: both contour halves by BiCG, complex FP64 Rayleigh-Ritz.  Device
    entry point, CUDA events around each solve."""
    import torch

    import feast_workloads as fw

    pkg, rank, ws = _lib_setup()
    p = fw.laplace3d_gauge(side=args.side)
    dev = torch.device("cuda")
    ia = torch.as_tensor(p.A.indptr).to(dev, torch.int32)
    ja = torch.as_tensor(p.A.indices).to(dev, torch.int32)
    av = torch.as_tensor(p.A.data).to(dev, torch.complex128)
    x0 = torch.as_tensor(np.ascontiguousarray(p.y0().T)).to(dev)

    def fpm(mixed):
        f = pkg.feast_init()
        f[1], f[2], f[3], f[4], f[5], f[17], f[41], f[44], f[45] = p.ne, 10, 40, 1, 1, p.ratio, mixed, 2, 80
        f[49] = args.node_batch or 1  # one node per batch: the lanes of a fast node stop early
        return f

    def solve(mixed):
        x = x0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        r = pkg.feast_hcsr_solve_dev(p.n, ia, ja, av, fpm=fpm(mixed), emin=p.emin, emax=p.emax, m0=p.m0, x=x)
        e1.record()
        torch.cuda.synchronize()
        if r.info != 0:
            raise RuntimeError(f"Hermitian FEAST info {r.info}")
        return e0.elapsed_time(e1), int(np.sum(r.res[: r.M] <= RES_TOL)), r

    for _ in range(args.warmup):
        solve(1)
    ms, conv = 0.0, 0
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    for _ in range(args.steps):
        t, c, r = solve(1)
        ms += t
        conv += c
    clk = clocks.stop()
    value = conv / (ms / 1e3)
    fp64 = None
    if args.fp64_steps > 0:
        t64, c64, _ = solve(0)
        fp64 = {"value": c64 / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64,
                "mixed_over_fp64": value / (c64 / (t64 / 1e3))}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c32 BiCG solves + c64 Rayleigh-Ritz",
               "data": "synthetic (seeded generator, no dataset)",
               "config": {"workload": f"laplace3d_7pt_{args.side}^3_potential_U[0,0.5]_seed1_random_gauge_phases",
                          "N": p.n, "nnz": p.A.nnz, "M0": p.m0, "Ne": p.ne, "contour_ratio_pct": p.ratio,
                          "interval": [p.emin, round(p.emax, 6)], "node_batch": args.node_batch or 1,
                          "inner_solver": "BiCG with the conjugate-shift shadow system, 1e-2, 80 steps"},
               "M": r.M, "converged_pairs": conv // args.steps, "max_residual": float(r.res[: r.M].max()),
               "bicg_iterations": int(r.fpm[59]), "fp64": fp64, "clocks": clk}
        print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    ROWS_PER_ITEM = a.rows_per_item
    INNER = (a.inner_tol, a.inner_maxit)
    if a.side is None:
        a.side = 96 if a.workload == "stencil27" else 64
    if a.impl == "reference" and a.workload != "laplace3d":
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the laplace3d workload "
                              "only; --workload " + a.workload + " has no CPU reference line"}))
    elif a.impl == "reference":
        run_reference(a)
    elif a.workload == "stencil27":
        run_stencil27(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "grad48":
        run_grad(a)
    elif a.workload == "hermitian":
        run_hermitian(a)
    else:
        run_gpu(a)
