#!/usr/bin/env python
"""Ground-state throughput of the Augmented Lagrangian OF-DFT solver on GB300.

One step = one complete ground state of the 5x5x5-cell FCC cluster (666 atoms,
Z = 3, a = 7.6 bohr, seeded +-0.1 bohr displacements, 10 bohr vacuum, h = 0.5
bohr -> 128^3 grid, 12th-order FD): pseudocharge and starting guess,
Algorithm 1 around PR nonlinear CG with one CG Poisson solve per gradient
evaluation, then the forces.  Synthetic input (the paper's aluminium clusters
with Gaussian nuclei standing in for its pseudopotential).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded samples)

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ground states/s + p50/p99 latency at 1e-5 Ha/atom; stencil HBM GB/s vs peak"
UNIT = "ground states/s"
FP64_ALU_PEAK_GFLOPS = 152 * 2 * 2 * 2.070  # SMs x DFMA/clk/SM x 2 flop x GHz (sm_103a, 2070 MHz)
COUNTS_FILE = os.path.join(ROOT, "profiles", "c2_solve_counts.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")


def workload():
    from paper_1405_6456_gb300 import workloads as W
    return W.cluster_c2()


def workload_config(c, g, precision, extra=None):
    cfg = {"workload": f"{c.name}: {c.M} atoms, FCC 5x5x5 cells a=7.6 bohr, Z=3, seeded +-0.1 bohr, "
                       f"h={c.h} bohr, {c.fd_order}th-order FD, {c.vacuum} bohr vacuum, grid "
                       f"{g[0]}x{g[1]}x{g[2]}, AL+PR-NLCG ground state with a Poisson solve per evaluation, to 1e-6 "
                       f"Ha/atom, forces",
           "atoms": c.M, "grid": list(g), "fd_order": c.fd_order, "precision": precision,
           "l2": "flushed between steps (256 MB write); the 128^3 CG working set itself fits in L2"}
    if extra:
        cfg.update(extra)
    return cfg


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def src_hash():
    h = hashlib.sha256()
    for rel in ("paper_1405_6456_gb300/csrc/kernels.cuh", "paper_1405_6456_gb300/csrc/common.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        load = [s for s in sm if s > 0.5 * (max(sm) if sm else 1)]
        return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(backend=None):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        import torch
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


def replica_cluster(rank, ws):
    """The cluster rank `rank` of `ws` solves: replicas only, every rank its own
    independent seeded 666-atom cluster (no data-path collective)."""
    from paper_1405_6456_gb300 import workloads as W
    return W.cluster_c2(seed=2 + rank) if ws > 1 else W.cluster_c2()


def job_rate(pg, ws, units_per_rank, local_seconds, device):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    slowest = allreduce_max(pg, local_seconds, device)
    return ws * units_per_rank / slowest, slowest


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce_max(pg, x, device):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------- CPU oracle arm --
def oracle_sample(c, n_cg=4):
    """Time the FP64 CPU oracle on a bounded sample of the workload: n_cg CG
    iterations of the 128^3 Poisson problem and one functional evaluation.
    Returns (seconds per CG iteration, seconds per functional evaluation)."""
    import oracle as O
    O.build()
    g = O.grid_for_atoms(c.R, c.h, c.vacuum, 16)
    n = c.fd_order // 2
    b, es = O.pseudocharge(g, n, c.R, c.Z)
    u = O.initial_guess(g, c.R, c.Z)
    rho = u**2 + b
    t0 = time.perf_counter()
    O.poisson(g, n, rho, tol=1e-300, max_it=n_cg)
    t1 = time.perf_counter()
    O.poisson(g, n, rho, tol=1e-300, max_it=0)
    t2 = time.perf_counter()
    t_cg = ((t1 - t0) - (t2 - t1)) / n_cg
    p = O.default_params()
    phi = np.zeros(g.shape)
    t3 = time.perf_counter()
    O.functional(g, p, u, b, phi, es, -0.2, 1.0, c.N)
    t_fun = time.perf_counter() - t3
    return t_cg, t_fun


def read_counts():
    try:
        with open(COUNTS_FILE) as f:
            return json.load(f)
    except Exception:
        return None


def run_reference(args):
    ws, rank, local, pg = dist_setup()
    if rank != 0:
        return 0
    c = workload()
    counts = read_counts()
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": "profiles/c2_solve_counts.json missing: the "
                          "oracle cannot finish this ground state in minutes and needs the counts to scale"}))
        return 0
    cg_per, ev_per = counts["cg_iters"], counts["grad_evals"]
    for _ in range(args.warmup):
        oracle_sample(c, n_cg=2)
    times = []
    for _ in range(args.steps):
        t_cg, t_fun = oracle_sample(c, n_cg=3)
        times.append(t_cg * cg_per + t_fun * ev_per)
    sec = statistics.mean(times)
    val = 1.0 / sec
    g = counts.get("grid", [128, 128, 128])
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(c, g, "fp64"),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"per step: oracle pseudocharge + 3 CG iterations + 1 functional at 128^3, "
                                       f"scaled to {cg_per} CG iterations and {ev_per} gradient evaluations "
                                       f"per ground state (counts of the plain-CG FP64 GPU solve of this "
                                       f"workload, the oracle's own iteration)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm --
def run_gpu(args):
    import torch
    from paper_1405_6456_gb300 import build as B
    from paper_1405_6456_gb300 import ofdft as F
    ws, rank, local, pg = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    from paper_1405_6456_gb300 import workloads as W
    base = workload()
    # replicas only: every rank solves its own independent cluster
    c = replica_cluster(rank, ws)
    prec = F.PREC_MIXED if args.precision == "mixed" else F.PREC_FP64
    p = F.default_params(precision=prec, tol_E=1e-6, vacuum=c.vacuum, round_to=16)
    ctx = F.Context(local)
    if args.write_counts:  # the counts scale the oracle, which runs plain CG
        ctx.set_poisson_precond(F.PRECOND_NONE)
    stream = ctx.stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_solve():
        return ctx.solve(c.R, c.Z, c.h, p)

    for _ in range(args.warmup):
        E, Fv, st = one_solve()
    g = tuple(st.grid.n)
    G = g[0] * g[1] * g[2]
    # timed region (device time per step, L2 flushed between steps)
    dom = F.K_CG_DIR_STENCIL
    ctx.reset_counters()
    # events around the candidates for the dominant kernel only: the FP64
    # residual passes of the Poisson rounds, the persistent CG launches, else one
    # CG stencil pass in eight (inside the CG graphs)
    ctx.profile(((1 << dom) | (1 << F.K_CG_PERSISTENT) | (1 << F.K_RESIDUAL)) if args.profile_timed else 0)
    lat = []
    stats = []
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E, Fv, st = one_solve()
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1) / 1e3)
            stats.append(st)
    torch.cuda.synchronize()
    barrier(pg)
    cnt = ctx.counters()
    ctx.profile(False)
    total = sum(lat)
    value, total_max = job_rate(pg, ws, args.steps, total, dev)
    # e2e: the public C-ABI call with host buffers (atoms in, energy+forces out)
    ctx.reset_counters()
    barrier(pg)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E2, F2, st2 = one_solve()
        e2e_t.append(time.perf_counter() - t0)
    e2e_val, e2e_max = job_rate(pg, ws, args.steps, sum(e2e_t), dev)
    h2d = c.R.nbytes + c.Z.nbytes
    d2h = 8 + 3 * c.M * 8
    # roofline of the dominant kernel: the persistent CG kernel where the
    # library ran it, else the CG direction + stencil pass
    es = 4 if prec == F.PREC_MIXED else 8
    roof = None
    n = c.fd_order // 2
    pk = F.K_CG_PERSISTENT
    if cnt.timed_launches[pk] > 0 and cnt.persistent_cg_iters > 0:
        tl, tms, its = cnt.timed_launches[pk], cnt.timed_ms[pk], cnt.persistent_cg_iters
        avg_s = tms / tl / 1e3
        traffic = None
        try:
            with open(TRAFFIC_FILE) as f:
                tr = json.load(f)
            key = f"cg_persistent_{args.precision}"
            if tr.get("src_hash") == src_hash() and key in tr:
                traffic = tr[key]["bytes_per_iteration_full"] * its / tl
        except Exception:
            pass
        # per CG iteration: stencil half reads r, p, q and writes p, q; update
        # half reads x, p, q, r and writes x, r
        algo_it = 11 * G * es
        kname = "cg_coop_kernel<%s,%d,%d> (whole CG iterations: q = A r + beta q, p = r + beta p, p.q | " \
                "x += alpha p, r -= alpha q, r.r)" % ("float" if es == 4 else "double", n, 16 // es)
        common = {"traffic": traffic, "kernel": kname, "launches": tl, "avg_us": avg_s * 1e6,
                  "cg_iters_per_launch": its / tl,
                  "timing": "CUDA events on the solve's stream around every persistent CG launch, over the "
                            "whole timed region",
                  "algorithmic_bytes_per_launch": algo_it * its / tl}
        if prec == F.PREC_MIXED:
            peak, which = load_peaks()
            ach = algo_it * its / (tms / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "peak_source": which, **common}
        else:
            flops_it = G * (2 * (6 * n + 1) + 12)  # stencil, p, q, x, r updates, p.q, r.r
            ach = flops_it * its / (tms / 1e3) / 1e9
            roof = {"bound": "alu", "achieved": ach, "peak": FP64_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": ach / FP64_ALU_PEAK_GFLOPS,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz",
                    "algorithmic_flops_per_launch": flops_it * its / tl, **common}
    tl, tms = cnt.timed_launches[dom], cnt.timed_ms[dom]
    if roof is None and tl > 0:
        avg_s = tms / tl / 1e3
        traffic = None
        try:
            with open(TRAFFIC_FILE) as f:
                tr = json.load(f)
            key = f"cg_dir_stencil_{args.precision}"
            if tr.get("src_hash") == src_hash() and key in tr:
                traffic = tr[key]["bytes_per_launch_full"]
        except Exception:
            pass
        if prec == F.PREC_MIXED:
            peak, which = load_peaks()
            fold = 5 * G * es > 96 * (1 << 20)  # the library folds the x update into this pass
            algo = G * (7 if fold else 5) * es  # read r (stencil), p, q (, x); write p, q (, x)
            ach = algo / avg_s / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": traffic, "kernel": "zstream_kernel<float,6,LoadPlain,EpiCgA%s> (CG: q = A r + beta q, p = r + beta p, p.q%s)" % (("X", ", x += alpha p_old") if fold else ("", "")),
                    "launches": tl, "avg_us": avg_s * 1e6, "peak_source": which,
                    "timing": "CUDA events on the solve's stream around one stencil launch in 8 (recorded "
                              "inside the CG graphs), over the whole timed region",
                    "algorithmic_bytes_per_launch": algo}
        else:
            fold = 5 * G * es > 96 * (1 << 20)
            flops = G * (2 * (6 * n + 1) + 2 + 2 + 2 + (2 if fold else 0))  # stencil, p, q (, x) updates, p.q
            ach = flops / avg_s / 1e9
            roof = {"bound": "alu", "achieved": ach, "peak": FP64_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": ach / FP64_ALU_PEAK_GFLOPS, "traffic": traffic,
                    "kernel": "zstream_kernel<double,6,LoadPlain,EpiCgA%s> (CG: q = A r + beta q, p = r + beta p, p.q%s)" % (("X", ", x += alpha p_old") if fold else ("", "")), "launches": tl,
                    "avg_us": avg_s * 1e6, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz",
                    "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": G * (7 if fold else 5) * es}
    # the FP64 residual pass r = 4 pi rho + L_h phi of every Poisson round
    # (FP64 ALU-bound): 2(6n+1) stencil flops + u^2, 4 pi (u^2 + b), r and
    # three dot products per node
    roof_res = None
    kr = F.K_RESIDUAL
    if cnt.timed_launches[kr] > 0:
        avg_r = cnt.timed_ms[kr] / cnt.timed_launches[kr] / 1e3
        flops_r = G * (2 * (6 * n + 1) + 10)
        ach_r = flops_r / avg_r / 1e9
        traffic_r = None
        try:
            with open(TRAFFIC_FILE) as f:
                tr = json.load(f)
            key = f"residual_fp64_{args.precision}"
            if tr.get("src_hash") == src_hash() and key in tr:
                traffic_r = tr[key]["bytes_per_launch_full"]
        except Exception:
            pass
        roof_res = {"bound": "alu", "achieved": ach_r, "peak": FP64_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": ach_r / FP64_ALU_PEAK_GFLOPS, "traffic": traffic_r,
                    "kernel": "zstream_kernel<double,%d,2,LoadPlain,EpiResidual> (FP64 residual "
                              "4 pi (u^2 + b) + L_h phi of each Poisson round, with r.r, b.b, u.u)" % n,
                    "launches": int(cnt.timed_launches[kr]), "avg_us": avg_r * 1e6,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz",
                    "timing": "CUDA events on the solve's stream around every residual launch, over the whole "
                              "timed region",
                    "algorithmic_flops_per_launch": flops_r, "algorithmic_bytes_per_launch": G * 8 * 3,
                    "total_ms": cnt.timed_ms[kr]}
    if roof is not None and "launches" in roof and cnt.timed_launches[F.K_CG_PERSISTENT] == 0:
        # the stencil pass's total: its mean duration times the CG iterations run
        roof["total_ms_estimate"] = roof["avg_us"] / 1e3 * sum(s.cg_iters for s in stats)
    roof_other = None
    if roof_res is not None and (roof is None or roof_res["total_ms"] > roof.get("total_ms_estimate", 0.0)):
        roof, roof_other = roof_res, roof
    elif roof_res is not None:
        roof_other = roof_res
    kinds = {F.KIND_NAMES[k]: {"launches": int(cnt.kind_launches[k]),
                               "ms": round(cnt.timed_ms[k], 3)} for k in range(F.K_COUNT) if cnt.kind_launches[k]}
    st = stats[-1]
    lat_sorted = sorted(lat)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64acc" if prec == F.PREC_MIXED else "f64", "data": "synthetic",
           "config": workload_config(c, g, args.precision, {"parallelism": f"replicas x{ws}"}),
           "latency_s": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99))},
           "energy_per_atom": E / c.M, "eta": st.eta,
           "per_solve": {"cg_iters": st.cg_iters, "grad_evals": st.grad_evals, "nlcg_iters": st.nlcg_iters,
                         "outer_iters": st.outer_iters, "stencil_apps": st.stencil_apps},
           "gpu_launches": int(cnt.launches), "kernels": kinds,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "roofline": roof, "roofline_next": roof_other}
    # plain FP64 form for comparison (the chosen form is MIXED)
    if prec == F.PREC_MIXED and args.plain_steps > 0:
        p64 = F.default_params(precision=F.PREC_FP64, tol_E=1e-6, vacuum=c.vacuum, round_to=16)
        t64 = []
        for _ in range(args.plain_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E64, F64, st64 = ctx.solve(c.R, c.Z, c.h, p64)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1) / 1e3)
        out["plain_fp64"] = {"value": 1.0 / statistics.mean(t64), "unit": UNIT, "steps": args.plain_steps,
                             "ms_per_step": 1e3 * statistics.mean(t64), "energy_per_atom": E64 / c.M,
                             "mixed_minus_fp64_Ha_per_atom": (E - E64) / c.M,
                             "max_force_diff_Ha_per_bohr": float(np.abs(Fv - F64).max()),
                             "cg_iters": st64.cg_iters, "grad_evals": st64.grad_evals}
    if prec == F.PREC_FP64 and rank == 0 and args.write_counts:
        os.makedirs(os.path.dirname(COUNTS_FILE), exist_ok=True)
        with open(COUNTS_FILE, "w") as f:
            json.dump({"workload": c.name, "grid": list(g), "cg_iters": st.cg_iters, "grad_evals": st.grad_evals,
                       "stencil_apps": st.stencil_apps, "precision": "fp64"}, f, indent=1)
    ctx.close()
    out["clocks"] = clk.summary()
    if rank == 0 and ws == 1 and not args.no_cpu:
        t_cg, t_fun = oracle_sample(base, n_cg=4)
        # the oracle runs plain CG: scale by the plain-CG counts of this
        # workload (profiles/c2_solve_counts.json), not by the PCG iterations
        counts = read_counts()
        cg_n, ev_n, src = ((counts["cg_iters"], counts["grad_evals"], "the plain-CG FP64 solve of this workload")
                           if counts else (st.cg_iters, st.grad_evals, "this solve"))
        sec = t_cg * cg_n + t_fun * ev_n
        out["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"oracle pseudocharge + 4 CG iterations + 1 functional evaluation at "
                                         f"{g[0]}^3, scaled to {cg_n} CG iterations and {ev_n} gradient "
                                         f"evaluations per ground state (counts of {src}; {t_cg:.3f} s/CG "
                                         f"iteration, {t_fun:.3f} s/evaluation)"}
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()
    return 0


# ------------------------------------------------------ batch / serving modes --
def run_batch(args):
    """C4: count FCC cubes (m uniform in 1..5, h = 0.5, 12th order, 8 bohr vacuum,
    48^3..112^3 grids) solved together by the batch engine (MIXED)."""
    import torch
    from paper_1405_6456_gb300 import build as B
    from paper_1405_6456_gb300 import ofdft as F
    from paper_1405_6456_gb300 import workloads as W
    B.build()
    ctx = F.Context(0)
    cl = W.batch_c4(args.batch_count)
    p = F.default_params(precision=F.PREC_MIXED, vacuum=8.0, round_to=16)
    grids = [F.ofdft_grid_for_atoms(c.R, c.h, c.vacuum, 16) for c in cl]
    out = {"metric": METRIC, "mode": "batch", "unit": UNIT, "requests": len(cl),
           "grids": sorted({g.n[0] for g in grids}), "dtype": "f32+f64acc", "data": "synthetic"}
    for rep in range(2):  # warm-up pass, then the timed pass
        bt = F.Batch(ctx, F.PREC_MIXED, 200 << 30)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [bt.submit(c.R, c.Z, c.h, p) for c in cl]
        done_t = {}
        rounds = 0
        while len(done_t) < len(ids):
            bt.step()
            rounds += 1
            for rid in ids:
                if rid not in done_t and bt.poll(rid, allow_notconv=True) is not None:
                    done_t[rid] = time.perf_counter() - t0
        wall = time.perf_counter() - t0
        bt.close()
    lat = np.array(sorted(done_t.values()))
    out.update({"value": len(cl) / wall, "wall_s": wall, "rounds": rounds,
                "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))}})
    # the same requests one at a time through ofdft_solve (the plain form)
    t0 = time.perf_counter()
    for c in cl[: args.batch_solo]:
        ctx.solve(c.R, c.Z, c.h, p, want_forces=True, allow_notconv=True)
    solo = (time.perf_counter() - t0) / max(args.batch_solo, 1)
    out["one_at_a_time"] = {"value": 1.0 / solo, "unit": UNIT, "sample": f"first {args.batch_solo} requests"}
    ctx.close()
    print(json.dumps(out))
    return 0


def run_serve(args):
    """C5: Poisson arrivals of FCC cubes (m log-uniform in 1..8, h in {0.45, 0.5, 0.6},
    order in {8, 12}, 8 bohr vacuum) served with continuous batching (MIXED)."""
    from paper_1405_6456_gb300 import build as B
    from paper_1405_6456_gb300 import ofdft as F
    from paper_1405_6456_gb300 import serving as S
    from paper_1405_6456_gb300 import workloads as W
    B.build()
    ctx = F.Context(0)
    rates = [float(x) for x in args.rates.split(",")]
    res = []
    for rate in rates:
        reqs = W.serving_requests_c5(rate, args.requests, max_m=args.max_m)
        prm = lambda c: F.default_params(precision=F.PREC_MIXED, fd_order=c.fd_order, vacuum=c.vacuum, round_to=16)
        rep = S.serve(ctx, reqs, prm, precision=F.PREC_MIXED, hbm_budget_bytes=args.hbm_gb << 30)
        s = rep.summary()
        s["rate_per_s"] = rate
        res.append(s)
    ctx.close()
    print(json.dumps({"metric": METRIC, "mode": "serve", "unit": UNIT, "dtype": "f32+f64acc",
                      "data": "synthetic", "max_m": args.max_m, "rates": res}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--write-counts", action="store_true")
    ap.add_argument("--profile-timed", type=int, default=1)
    ap.add_argument("--mode", default="solve", choices=["solve", "batch", "serve"])
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-solo", type=int, default=4)
    ap.add_argument("--rates", default="1,5,20")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--max-m", type=int, default=8)
    ap.add_argument("--hbm-gb", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
