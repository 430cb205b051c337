"""Times the library's Poisson CG (the hot loop of the method) on one grid.

  python -m paper_1405_6456_gb300.kernel_bench --n 256 --order 12 --prec mixed --iters 50

Solves (-L_h) phi = 4 pi rho for a seeded random rho with a fixed iteration
count (tolerance 0), through the C ABI, and reports the average duration of the
CG stencil pass (CUDA events around each launch), of the CG update and of the
multigrid preconditioner's V-cycle, with the algorithmic bytes moved.  Grids
above 200^3 in FP32 exceed the 129 MB L2, which makes the DRAM counters of a
profiler meaningful.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np


def main():
    import torch

    from paper_1405_6456_gb300 import build as B
    from paper_1405_6456_gb300 import ofdft as F

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--order", type=int, default=12)
    ap.add_argument("--prec", choices=["fp64", "fp32"], default="fp32")
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--h", type=float, default=0.5)
    args = ap.parse_args()
    B.build()
    dt = torch.float64 if args.prec == "fp64" else torch.float32
    ctx = F.Context(0)
    g = F.make_grid(args.n, args.n, args.n, args.h)
    rng = np.random.default_rng(0)
    rho = torch.as_tensor(rng.standard_normal(g.shape), dtype=dt, device="cuda:0")
    # warm-up, then the timed solve (FP32 fields go through the mixed path's FP32 CG
    # only when called with float tensors: here a plain FP32 CG is not exposed, so
    # the FP32 case times the mixed solve's FP32 correction iterations)
    # the default two-kernel iteration, then (a context created with
    # OFDFT_COOP=1) the persistent cooperative kernel where the grid's blocks fit
    # on the GPU at once
    for rep in range(2):
        phi = torch.zeros(g.shape, dtype=dt, device="cuda:0")
        ctx.reset_counters()
        ctx.profile((1 << F.K_CG_DIR_STENCIL) | (1 << F.K_CG_UPDATE) | (1 << F.K_MG))
        st = ctx.poisson(g, args.order, phi, rho=rho, tol=1e-300, max_it=args.iters, allow_notconv=True)
        cnt = ctx.counters()
        ctx.profile(False)
    os.environ["OFDFT_COOP"] = "1"
    ctxp = F.Context(0)
    ctxp.set_poisson_precond(F.PRECOND_NONE)  # the persistent kernel runs plain CG
    for rep in range(2):
        phi = torch.zeros(g.shape, dtype=dt, device="cuda:0")
        ctxp.reset_counters()
        ctxp.profile(1 << F.K_CG_PERSISTENT)
        ctxp.poisson(g, args.order, phi, rho=rho, tol=1e-300, max_it=args.iters, allow_notconv=True)
        cntp = ctxp.counters()
        ctxp.profile(False)
    ctxp.close()
    es = 4 if args.prec == "fp32" else 8
    G = g.size
    out = {"grid": args.n, "order": args.order, "prec": args.prec, "cg_iterations": st.iterations,
           "folded_update": bool(5 * g.size * es > 96 * (1 << 20))}
    # per node: the stencil pass reads r, p, q and writes p, q; the update reads x, r, p, q and writes
    # x, r -- or, when the five vectors exceed 96 MB, the stencil pass also moves x (folded update)
    # and the update only reads r, q and writes r
    fold = 5 * G * es > 96 * (1 << 20)
    for k, name, acc in [(F.K_CG_DIR_STENCIL, "cg_dir_stencil", 7 if fold else 5),
                         (F.K_CG_UPDATE, "cg_update", 3 if fold else 6)]:
        n = cnt.timed_launches[k]
        if n:
            us = cnt.timed_ms[k] / n * 1e3
            out[name] = {"launches": n, "avg_us": us, "algorithmic_bytes": G * acc * es,
                         "GBps": G * acc * es / (us * 1e-6) / 1e9}
    if cnt.timed_launches[F.K_MG]:
        # the multigrid preconditioner's passes (one V-cycle per CG iteration)
        out["mg_vcycle"] = {"launches": cnt.timed_launches[F.K_MG],
                            "launches_per_iteration": cnt.timed_launches[F.K_MG] / st.iterations,
                            "us_per_iteration": cnt.timed_ms[F.K_MG] * 1e3 / st.iterations}
    its = cntp.persistent_cg_iters
    if cntp.timed_launches[F.K_CG_PERSISTENT] and its:
        us_it = cntp.timed_ms[F.K_CG_PERSISTENT] / its * 1e3
        out["cg_persistent"] = {"launches": cntp.timed_launches[F.K_CG_PERSISTENT], "iterations": its,
                                "avg_us_per_iteration": us_it, "algorithmic_bytes_per_iteration": G * 11 * es,
                                "GBps": G * 11 * es / (us_it * 1e-6) / 1e9}
    print(json.dumps(out))
    ctx.close()


if __name__ == "__main__":
    main()
