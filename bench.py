#!/usr/bin/env python
"""Ground-state throughput of the Augmented Lagrangian OF-DFT solver on GB300.

One step = one complete ground state of the 8x8x8-cell FCC cluster (2457 atoms,
Z = 3, a = 7.6 bohr, seeded +-0.1 bohr displacements, 10 bohr vacuum, h = 0.45
bohr -> 192^3 grid, 12th-order FD) in the mixed-precision form:
pseudocharge and starting guess, Algorithm 1 around PR nonlinear CG with one
Poisson solve per gradient evaluation, then the forces.  The plain FP64 form
of the same ground state is timed beside it.  Synthetic input (the paper's
aluminium clusters with Gaussian nuclei standing in for its pseudopotential).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--workload fcc8|fcc5]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded samples)
  python bench.py --mode batch|serve     (64-cluster batch / Poisson-arrival serving)

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
FP32_ALU_PEAK_GOPS = 152 * 128 * 2.070      # SMs x FP32 lanes x GHz: one FP32 instruction per lane and clock



def ff_residual_ops_per_node(n):
    """FP32 operations per node of the float-float residual pass at radius n,
    counted from the algorithm: 3n pair sums (TwoSum + 2 adds = 8 each), 3
    products at p = 1 and 3(n - 1) product-and-sum steps (FMA-exact product 4 +
    lazy sum 8), the centre product (4), 3 axis sums (8 each); epilogue:
    renormalisation (6), u^2 + b (2 + 11), 4 pi rho (7), + L_h phi (11), 9
    compensated dot terms (7 each) = 100.  464 at 12th order."""
    return 24 * n + 12 + 36 * (n - 1) + 4 + 24 + 100
GOLDEN = os.path.join(ROOT, "tests", "golden")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
CELLS = {"fcc8": 8, "fcc5": 5}


def workload(name="fcc8", seed=None):
    from paper_1405_6456_gb300 import workloads as W
    f = W.cluster_c3 if name == "fcc8" else W.cluster_c2
    return f() if seed is None else f(seed=seed)


def workload_config(c, g, precision, name, extra=None):
    m = CELLS[name]
    cfg = {"workload": f"{c.name}: {c.M} atoms, FCC {m}x{m}x{m} cells a=7.6 bohr, Z=3, seeded +-0.1 bohr, "
                       f"h={c.h} bohr, {c.fd_order}th-order FD, {c.vacuum} bohr vacuum, grid "
                       f"{g[0]}x{g[1]}x{g[2]}, AL+PR-NLCG ground state with a Poisson solve per evaluation, to 1e-6 "
                       f"Ha/atom, forces",
           "atoms": c.M, "grid": list(g), "fd_order": c.fd_order, "precision": precision,
           "l2": "flushed between steps (256 MB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def golden(c, tol):
    """The oracle's ground state of cluster c (tests/golden/, written by
    tests/golden/make_ground_states.py), or None."""
    try:
        with open(os.path.join(GOLDEN, f"ground_state_{c.name}_{tol}.json")) as f:
            return json.load(f)
    except Exception:
        return None


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


def replica_cluster(name, rank, ws):
    """The cluster rank `rank` of `ws` solves: replicas only, every rank its own
    independent seeded cluster of the workload (no data-path collective)."""
    if ws == 1:
        return workload(name)
    return workload(name, seed=(3 if name == "fcc8" else 2) + rank)


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
def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class OracleSampler:
    """Times the FP64 CPU oracle on a bounded sample of a workload: n_cg CG
    iterations of its Poisson problem and one functional evaluation (the
    pseudocharge and starting guess are set up once, untimed).  The oracle's
    whole ground state is then scaled from its own counts of CG iterations and
    gradient evaluations (tests/golden/, at the benchmark's tolerances)."""

    def __init__(self, c):
        import oracle as O
        O.build()
        self.O = O
        self.c = c
        self.g = O.grid_for_atoms(c.R, c.h, c.vacuum, 16)
        self.n = c.fd_order // 2
        O.set_threads(os.cpu_count() or 1)
        self.b, self.es = O.pseudocharge(self.g, self.n, c.R, c.Z)
        self.u = O.initial_guess(self.g, c.R, c.Z)
        self.rho = self.u**2 + self.b
        self.p = O.default_params(fd_n=self.n)

    def sample(self, threads, n_cg=3):
        """(seconds per CG iteration, seconds per functional evaluation, threads used)."""
        O = self.O
        O.set_threads(threads)
        used = O.threads()
        t0 = time.perf_counter()
        O.poisson(self.g, self.n, self.rho, tol=1e-300, max_it=n_cg)
        t1 = time.perf_counter()
        O.poisson(self.g, self.n, self.rho, tol=1e-300, max_it=0)
        t2 = time.perf_counter()
        t_cg = max((t1 - t0) - (t2 - t1), 0.0) / n_cg
        phi = np.zeros(self.g.shape)
        t3 = time.perf_counter()
        O.functional(self.g, self.p, self.u, self.b, phi, self.es, -0.2, 1.0, self.c.N)
        t_fun = time.perf_counter() - t3
        return t_cg, t_fun, used


def oracle_counts(c):
    """The oracle's own work per ground state at the benchmark's tolerances."""
    gd = golden(c, "product")
    if gd is None:
        return None
    return gd["counts"]["cg_iters"], gd["counts"]["grad_evals"]


def run_reference(args):
    ws, rank, local, pg = dist_setup("gloo")
    if rank != 0:
        return 0
    c = workload(args.workload)
    counts = oracle_counts(c)
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": f"tests/golden/ground_state_{c.name}_product.json "
                          "missing: the oracle's own iteration counts scale its timed sample"}))
        return 0
    cg_per, ev_per = counts
    smp = OracleSampler(c)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        smp.sample(threads, n_cg=1)
    times, walls = [], []
    used = threads
    for _ in range(args.steps):
        t0 = time.perf_counter()
        t_cg, t_fun, used = smp.sample(threads, n_cg=3)
        walls.append(time.perf_counter() - t0)
        times.append(t_cg * cg_per + t_fun * ev_per)
    sec = statistics.mean(times)
    val = 1.0 / sec
    g = [smp.g.n1, smp.g.n2, smp.g.n3]
    # a step is the bounded sample (its wall time is ms_per_step); value is the
    # oracle's ground states per second, the sample scaled to its own counts
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
            "ms_per_ground_state_scaled": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(c, g, args.precision, args.workload),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": used, "kind": "oracle",
                             "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "sample": f"per step: 3 oracle CG iterations + 1 functional evaluation on the "
                                       f"{g[0]}x{g[1]}x{g[2]} grid ({used} threads), scaled to the oracle's own "
                                       f"{cg_per} CG iterations and {ev_per} gradient evaluations per ground "
                                       f"state at the benchmark's tolerances (tests/golden/)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm --
def _traffic(key):
    """Per-launch DRAM bytes from the committed ncu summary, if it was measured on
    the current kernel sources."""
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if tr.get("src_hash") == src_hash() and key in tr:
            return tr[key]["bytes_per_launch_full"]
    except Exception:
        pass
    return None


def roofline_entries(cnt, sampled, G, n, prec_name, es, fold):
    """Rooflines of the hot kernels from CUDA-event durations of a profiled
    ground state: one entry per kernel with its algorithmic bytes (or flops) per
    launch over its mean launch duration, and its total time."""
    from paper_1405_6456_gb300 import ofdft as F
    peak_hbm, which = load_peaks()
    out = []
    # CG stencil pass (one launch in eight timed inside the CG graphs)
    k = F.K_CG_DIR_STENCIL
    if sampled.timed_launches[k] > 0:
        avg = sampled.timed_ms[k] / sampled.timed_launches[k] / 1e3
        algo = G * (7 if fold else 5) * es  # read r (stencil), p, q (, x); write p, q (, x)
        e = {"kernel": "zstream_kernel<%s,%d,LoadPlain,EpiCgA%s> (CG: q = A z + beta q, p = z + beta p, p.q%s)"
                       % ("float" if es == 4 else "double", n, "X" if fold else "", ", x += alpha p_old" if fold else ""),
             "launches_timed": int(sampled.timed_launches[k]), "avg_us": avg * 1e6,
             "total_ms": avg * 1e3 * cnt.kind_launches[k],
             "algorithmic_bytes_per_launch": algo, "traffic": _traffic(f"cg_dir_stencil_{prec_name}"),
             "timing": "CUDA events inside the CG graphs around one stencil launch in eight"}
        if es == 4:
            ach = algo / avg / 1e9
            e.update({"bound": "hbm", "achieved": ach, "peak": peak_hbm, "unit": "GB/s", "frac": ach / peak_hbm,
                      "peak_source": which})
        else:
            fl = G * (2 * (6 * n + 1) + 6 + (2 if fold else 0))
            ach = fl / avg / 1e9
            e.update({"bound": "alu", "achieved": ach, "peak": FP64_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                      "frac": ach / FP64_ALU_PEAK_GFLOPS, "algorithmic_flops_per_launch": fl,
                      "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz"})
        out.append(e)
    # residual pass of each Poisson round (every launch timed): float-float on
    # the FP32 pipes in MIXED (unless OFDFT_FF_RESIDUAL=0), FP64 otherwise
    k = F.K_RESIDUAL
    ff = es == 4 and os.environ.get("OFDFT_FF_RESIDUAL", "1") != "0"
    if sampled.timed_launches[k] > 0 and ff:
        avg = sampled.timed_ms[k] / sampled.timed_launches[k] / 1e3
        ops = G * ff_residual_ops_per_node(n)
        ach = ops / avg / 1e9
        out.append({"kernel": "zstream_kernel<float2,%d,2,LoadPlain<float2>,EpiResidualFF> (float-float residual "
                              "4 pi (u^2 + b) + L_h phi of each mixed Poisson round, with u.u, ||4 pi rho||^2, "
                              "r.r and the electrostatic sums)" % n,
                    "bound": "alu", "achieved": ach, "peak": FP32_ALU_PEAK_GOPS, "unit": "Gop/s",
                    "frac": ach / FP32_ALU_PEAK_GOPS,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz (one op per lane and clock)",
                    "launches_timed": int(sampled.timed_launches[k]), "avg_us": avg * 1e6,
                    "total_ms": sampled.timed_ms[k], "algorithmic_ops_per_launch": ops,
                    "algorithmic_bytes_per_launch": G * 28, "hbm_frac": G * 28 / avg / 1e9 / peak_hbm,
                    "traffic": _traffic(f"residual_ff_{prec_name}"),
                    "timing": "CUDA events around every residual launch"})
    elif sampled.timed_launches[k] > 0:
        avg = sampled.timed_ms[k] / sampled.timed_launches[k] / 1e3
        fl = G * (2 * (6 * n + 1) + 10)
        ach = fl / avg / 1e9
        out.append({"kernel": "zstream_kernel<double,%d,LoadPlain,EpiResidual> (FP64 residual 4 pi (u^2 + b) + "
                              "L_h phi of each Poisson round, with r.r, b.b, u.u)" % n,
                    "bound": "alu", "achieved": ach, "peak": FP64_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": ach / FP64_ALU_PEAK_GFLOPS, "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2070 MHz",
                    "launches_timed": int(sampled.timed_launches[k]), "avg_us": avg * 1e6,
                    "total_ms": sampled.timed_ms[k], "algorithmic_flops_per_launch": fl,
                    "algorithmic_bytes_per_launch": G * 28, "traffic": _traffic(f"residual_fp64_{prec_name}"),
                    "timing": "CUDA events around every residual launch"})
    # fused functional + gradient pass (every launch timed)
    k = F.K_FUNCTIONAL
    if sampled.timed_launches[k] > 0:
        avg = sampled.timed_ms[k] / sampled.timed_launches[k] / 1e3
        algo = G * 5 * es  # read u (stencil), phi, b, d; write G
        ach = algo / avg / 1e9
        out.append({"kernel": "zstream_kernel<%s,%d,LoadPlain,EpiFunctional> (fused TF + vW + XC + electrostatic "
                              "energy, gradient, preconditioner, 11 sums)" % ("float" if es == 4 else "double", n),
                    "bound": "hbm", "achieved": ach, "peak": peak_hbm, "unit": "GB/s", "frac": ach / peak_hbm,
                    "peak_source": which, "launches_timed": int(sampled.timed_launches[k]), "avg_us": avg * 1e6,
                    "total_ms": sampled.timed_ms[k], "algorithmic_bytes_per_launch": algo,
                    "traffic": _traffic(f"functional_{prec_name}"),
                    "timing": "CUDA events around every functional launch"})
    return out


def run_gpu(args):
    import torch
    from paper_1405_6456_gb300 import build as B
    from paper_1405_6456_gb300 import ofdft as F
    ws, rank, local, pg = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    # replicas only: every rank solves its own independent cluster
    c = replica_cluster(args.workload, rank, ws)
    prec = F.PREC_MIXED if args.precision == "mixed" else F.PREC_FP64
    over = {}
    for kv in args.param:  # solver-parameter experiments: --param name=value
        k, v = kv.split("=", 1)
        over[k] = type(getattr(F.default_params(), "lam" if k == "lambda" else k))(float(v))
    p = F.default_params(precision=prec, tol_E=1e-6, vacuum=c.vacuum, round_to=16, **over)
    ctx = F.Context(local)
    stream = ctx.stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_solve(pp):
        return ctx.solve(c.R, c.Z, c.h, pp, allow_notconv=False)

    g = tuple(F.ofdft_grid_for_atoms(c.R, c.h, c.vacuum, 16).n)
    for _ in range(args.warmup):
        one_solve(p)
    G = g[0] * g[1] * g[2]
    # timed region: device time per step, L2 flushed between steps, no event
    # instrumentation of the library's own (that runs in a separate pass below)
    ctx.profile(False)
    ctx.reset_counters()
    lat, stats = [], []
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E, Fv, st = one_solve(p)
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1) / 1e3)
            stats.append(st)
    torch.cuda.synchronize()
    barrier(pg)
    cnt = ctx.counters()
    total = sum(lat)
    value, total_max = job_rate(pg, ws, args.steps, total, dev)
    # e2e: the public C-ABI call with host buffers (atoms in, energy + forces out)
    barrier(pg)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E2, F2, st2 = one_solve(p)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val, e2e_max = job_rate(pg, ws, args.steps, sum(e2e_t), dev)
    h2d = c.R.nbytes + c.Z.nbytes
    d2h = 8 + 3 * c.M * 8
    st = stats[-1]
    lat_sorted = sorted(lat)
    es = 4 if prec == F.PREC_MIXED else 8
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64acc" if prec == F.PREC_MIXED else "f64", "data": "synthetic",
           "config": workload_config(c, g, args.precision, args.workload,
                                     {"parallelism": f"replicas x{ws}", **({"params": over} if over else {})}),
           "latency_s": {"p50": float(np.percentile(lat_sorted, 50)), "p99": float(np.percentile(lat_sorted, 99))},
           "energy_per_atom": E / c.M, "eta": st.eta, "converged": all(s.converged for s in stats),
           "per_solve": {"cg_iters": st.cg_iters, "grad_evals": st.grad_evals, "nlcg_iters": st.nlcg_iters,
                         "outer_iters": st.outer_iters, "stencil_apps": st.stencil_apps},
           "gpu_launches": int(cnt.launches), "tma_launches": int(cnt.tma_launches),
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}
    # the plain FP64 form of the same ground state (the chosen form is MIXED)
    E64 = F64 = None
    if prec == F.PREC_MIXED and args.plain_steps > 0:
        p64 = F.default_params(precision=F.PREC_FP64, tol_E=1e-6, vacuum=c.vacuum, round_to=16)
        one_solve(p64)  # warm-up: workspace, autotuner, graphs of the FP64 kernels
        t64 = []
        for _ in range(args.plain_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            E64, F64, st64 = one_solve(p64)
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1) / 1e3)
        med = statistics.median(t64)
        out["plain_fp64"] = {"value": 1.0 / med, "unit": UNIT, "steps": args.plain_steps, "warmup": 1,
                             "ms_per_step_median": 1e3 * med, "ms_per_step": [round(1e3 * t, 2) for t in t64],
                             "energy_per_atom": E64 / c.M,
                             "mixed_minus_fp64_Ha_per_atom": (E - E64) / c.M,
                             "max_force_diff_Ha_per_bohr": float(np.abs(Fv - F64).max()),
                             "cg_iters": st64.cg_iters, "grad_evals": st64.grad_evals,
                             "converged": bool(st64.converged)}
    # error against the FP64 oracle's ground state of the same cluster (tests/golden/)
    # (tightly converged where written, else at the benchmark's own tolerances)
    gd, gtol = None, None
    if ws == 1:
        for gtol in ("tight", "product"):
            gd = golden(c, gtol)
            if gd is not None:
                break
    if gd is not None:
        Fo = np.array(gd["forces_paper"])
        vs = {"source": f"tests/golden/ground_state_{c.name}_{gtol}.json", "E_per_atom": gd["E_per_atom"],
              args.precision: {"dE_Ha_per_atom": (E - gd["E"]) / c.M,
                               "max_dF_Ha_per_bohr": float(np.abs(Fv - Fo).max())}}
        if E64 is not None:
            vs["fp64"] = {"dE_Ha_per_atom": (E64 - gd["E"]) / c.M, "max_dF_Ha_per_bohr": float(np.abs(F64 - Fo).max())}
        out["vs_oracle"] = vs
    # profiled pass, after the timed region: (a) one ground state with CUDA
    # events around the residual and functional launches and one CG stencil
    # pass in eight (inside the CG graphs); (b) one with every launch timed
    # (no graphs) for the per-kind breakdown
    if args.profile_steps > 0:
        ctx.reset_counters()
        ctx.profile((1 << F.K_CG_DIR_STENCIL) | (1 << F.K_RESIDUAL) | (1 << F.K_FUNCTIONAL))
        for _ in range(args.profile_steps):
            flush.zero_()
            one_solve(p)
        sampled = ctx.counters()
        ctx.reset_counters()
        ctx.profile(True)
        for _ in range(args.profile_steps):
            flush.zero_()
            one_solve(p)
        allk = ctx.counters()
        ctx.profile(False)
        fold = 5 * G * es > 96 * (1 << 20)
        ents = roofline_entries(sampled, sampled, G, c.fd_order // 2, args.precision, es, fold)
        ents.sort(key=lambda e: -e["total_ms"])
        if ents:
            out["roofline"] = ents[0]
            out["roofline_others"] = ents[1:]
        tot = sum(allk.timed_ms[k] for k in range(F.K_COUNT))
        out["kernels"] = {F.KIND_NAMES[k]: {"launches": int(allk.kind_launches[k] // args.profile_steps),
                                            "ms": round(allk.timed_ms[k] / args.profile_steps, 3),
                                            "share": round(allk.timed_ms[k] / tot, 4) if tot > 0 else None}
                          for k in range(F.K_COUNT) if allk.kind_launches[k]}
        out["kernels_note"] = ("per ground state, every launch bracketed by CUDA events (no CUDA graphs) in a "
                               "profiled pass after the timed region; events add a few us per launch")
    ctx.close()
    out["clocks"] = clk.summary()
    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(c)
    if rank == 0:
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()
    return 0


def cpu_baseline(c):
    """The oracle timed on this machine's host cores at 1 thread and at all
    cores, scaled by its own work per ground state."""
    counts = oracle_counts(c)
    smp = OracleSampler(c)
    nproc = os.cpu_count() or 1
    res = {}
    for th in sorted({1, nproc}):
        t_cg, t_fun, used = smp.sample(th, n_cg=2 if th == 1 else 4)
        res[th] = (t_cg, t_fun, used)
    if counts is None:
        return {"value": None, "unit": UNIT, "cores": nproc, "kind": "oracle",
                "sample": "oracle counts for this workload missing from tests/golden/",
                "per_cg_iteration_s": {str(k): v[0] for k, v in res.items()}}
    cg_n, ev_n = counts
    sec = {th: v[0] * cg_n + v[1] * ev_n for th, v in res.items()}
    gg = smp.g
    return {"value": 1.0 / sec[nproc], "unit": UNIT, "cores": res[nproc][2], "kind": "oracle",
            "value_1_thread": 1.0 / sec[1], "nproc": nproc, "cpu_model": cpu_model(),
            "sample": f"oracle CG iterations (2 at 1 thread, 4 at {nproc}) + 1 functional evaluation on the "
                      f"{gg.n1}x{gg.n2}x{gg.n3} grid, scaled to the oracle's own {cg_n} CG iterations and {ev_n} "
                      f"gradient evaluations per ground state at the benchmark's tolerances (tests/golden/); "
                      f"s per CG iteration: {res[1][0]:.3f} (1 thread), {res[nproc][0]:.3f} ({nproc}); "
                      f"s per functional: {res[1][1]:.3f}, {res[nproc][1]:.3f}"}


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
        unconv = set()
        rounds = 0
        while len(done_t) < len(ids):
            bt.step()
            rounds += 1
            for rid in ids:
                if rid in done_t:
                    continue
                res = bt.poll(rid, allow_notconv=True)
                if res is not None:
                    done_t[rid] = time.perf_counter() - t0
                    if not res[2].converged:
                        unconv.add(rid)
        wall = time.perf_counter() - t0
        binfo = bt.info()
        if rep == 0:
            tuning = binfo  # the warm-up pass tunes each grid shape once for the context
        bt.close()
    lat = np.array(sorted(t for rid, t in done_t.items() if rid not in unconv))
    out.update({"value": (len(cl) - len(unconv)) / wall, "wall_s": wall, "rounds": rounds,
                "unconverged": len(unconv), "batch_launch_stats": binfo,
                "autotune_warmup_pass": tuning,
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
    prm = lambda c: F.default_params(precision=F.PREC_MIXED, fd_order=c.fd_order, vacuum=c.vacuum, round_to=16)
    if args.serve_warmup > 0:  # warm-up: workspaces, CUDA graphs and tuned shapes (discarded)
        S.serve(ctx, W.serving_requests_c5(100.0, args.serve_warmup, seed=99, max_m=args.max_m), prm,
                precision=F.PREC_MIXED, hbm_budget_bytes=args.hbm_gb << 30)
    res = []
    for rate in rates:
        reqs = W.serving_requests_c5(rate, args.requests, max_m=args.max_m)
        rep = S.serve(ctx, reqs, prm, precision=F.PREC_MIXED, hbm_budget_bytes=args.hbm_gb << 30)
        s = rep.summary()
        s["rate_per_s"] = rate
        res.append(s)
    ctx.close()
    print(json.dumps({"metric": METRIC, "mode": "serve", "unit": UNIT, "dtype": "f32+f64acc",
                      "data": "synthetic", "max_m": args.max_m, "rates": res}))
    return 0


def run_kernels(args):
    """Kernel microbenchmark on one n^3 grid (seeded random fields, through the
    C ABI): a Poisson solve with a fixed iteration count times the CG stencil
    pass, the CG update, the multigrid V-cycle and the residual pass; repeated
    functional evaluations at a fixed potential time the fused functional pass.
    Reports mean launch durations (CUDA events around each launch) with the
    algorithmic bytes each pass moves.  Grids of 256^3 in FP32 exceed the 129 MB
    L2, which makes a profiler's DRAM counters meaningful."""
    import torch
    from paper_1405_6456_gb300 import build as B
    from paper_1405_6456_gb300 import ofdft as F
    B.build()
    dt = torch.float64 if args.kprec == "fp64" else torch.float32
    es = 8 if args.kprec == "fp64" else 4
    prec = F.PREC_FP64 if args.kprec == "fp64" else F.PREC_MIXED
    ctx = F.Context(0)
    n = args.n
    g = F.make_grid(n, n, n, 0.5)
    G = g.size
    rng = np.random.default_rng(0)
    dev = "cuda:0"
    rho = torch.as_tensor(rng.standard_normal(g.shape), dtype=dt, device=dev)
    fold = 5 * G * es > 96 * (1 << 20)
    out = {"mode": "kernels", "grid": n, "order": args.order, "prec": args.kprec, "folded_update": fold}
    peak, which = load_peaks()
    out["hbm_peak_GBps"] = {"value": peak, "source": which}
    if args.which in ("all", "cg"):
        for _ in range(2):  # warm-up (autotuner, graphs), then the timed solve
            phi = torch.zeros(g.shape, dtype=dt, device=dev)
            ctx.reset_counters()
            ctx.profile((1 << F.K_CG_DIR_STENCIL) | (1 << F.K_CG_UPDATE) | (1 << F.K_MG) | (1 << F.K_RESIDUAL))
            st = ctx.poisson(g, args.order, phi, rho=rho, tol=1e-300, max_it=args.iters, allow_notconv=True)
            cnt = ctx.counters()
            ctx.profile(False)
        out["cg_iterations"] = st.iterations
        # per node: the stencil pass reads r, p, q and writes p, q (and moves x when folded); the update
        # reads x, r, p, q and writes x, r (folded: reads r, q, writes r)
        for k, name, acc in [(F.K_CG_DIR_STENCIL, "cg_dir_stencil", 7 if fold else 5),
                             (F.K_CG_UPDATE, "cg_update", 3 if fold else 6)]:
            nl = cnt.timed_launches[k]
            if nl:
                us = cnt.timed_ms[k] / nl * 1e3
                out[name] = {"launches": nl, "avg_us": us, "algorithmic_bytes": G * acc * es,
                             "GBps": G * acc * es / (us * 1e-6) / 1e9,
                             "frac_hbm": G * acc * es / (us * 1e-6) / 1e9 / peak}
        if cnt.timed_launches[F.K_MG]:
            out["mg_vcycle"] = {"launches": cnt.timed_launches[F.K_MG],
                                "launches_per_iteration": cnt.timed_launches[F.K_MG] / max(st.iterations, 1),
                                "us_per_iteration": cnt.timed_ms[F.K_MG] * 1e3 / max(st.iterations, 1)}
        if cnt.timed_launches[F.K_RESIDUAL]:
            nl = cnt.timed_launches[F.K_RESIDUAL]
            us = cnt.timed_ms[F.K_RESIDUAL] / nl * 1e3
            out["residual"] = {"launches": nl, "avg_us": us}
    if args.which in ("all", "functional"):
        u = torch.as_tensor(0.1 * np.abs(rng.standard_normal(g.shape)), dtype=dt, device=dev)
        b = torch.as_tensor(-0.1 * np.abs(rng.standard_normal(g.shape)), dtype=dt, device=dev)
        phi = torch.as_tensor(rng.standard_normal(g.shape), dtype=dt, device=dev)
        grad = torch.empty_like(u)
        sv = torch.empty_like(u)
        d = torch.as_tensor(rng.standard_normal(g.shape), dtype=dt, device=dev)
        pp = F.default_params(fd_order=args.order, precision=prec)
        for rep in range(2):
            ctx.reset_counters()
            ctx.profile(1 << F.K_FUNCTIONAL)
            for _ in range(args.iters):
                ctx.energy_grad(g, pp, u, b, phi, 0.0, -0.2, 1.0, 1.0, solve_poisson=False, grad=grad, s=sv,
                                d=d)
            cnt = ctx.counters()
            ctx.profile(False)
        nl = cnt.timed_launches[F.K_FUNCTIONAL]
        if nl:
            us = cnt.timed_ms[F.K_FUNCTIONAL] / nl * 1e3
            algo = G * 5 * es  # read u (stencil), phi, b, d; write G
            out["functional"] = {"launches": nl, "avg_us": us, "algorithmic_bytes": algo,
                                 "GBps": algo / (us * 1e-6) / 1e9, "frac_hbm": algo / (us * 1e-6) / 1e9 / peak}
    ctx.close()
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="fcc8", choices=sorted(CELLS))
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=1)
    ap.add_argument("--param", action="append", default=[])
    ap.add_argument("--mode", default="solve", choices=["solve", "batch", "serve", "kernels"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--order", type=int, default=12)
    ap.add_argument("--kprec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--which", default="all", choices=["all", "cg", "functional"])
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-solo", type=int, default=4)
    ap.add_argument("--rates", default="1,2,5,10,20,50,100,200")
    ap.add_argument("--requests", type=int, default=500)
    ap.add_argument("--serve-warmup", type=int, default=16)
    ap.add_argument("--max-m", type=int, default=8)
    ap.add_argument("--hbm-gb", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "kernels":
        return run_kernels(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
