"""Writes the oracle's ground states of the full-size cluster workloads to
tests/golden/ (energy, multiplier, constraint, forces and the oracle's own
iteration counts).  Calls only `oracle/` (and the seeded geometry generators of
`workloads.py`, which hold no method arithmetic); nothing here touches the CUDA
library.

Two tolerance sets:
  tight   - Algorithm 1 stops at |E_{q+1} - E_q| < 1e-9 Ha/atom, the NLCG at
            h^3 r.s < 1e-10 Ha/atom, every Poisson CG at a relative residual of
            1e-10: the reference values of the full-size parity tests;
  product - the library's default tolerances (1e-6 Ha/atom, 1e-8 Ha/atom,
            Poisson 1e-8): the oracle's own work (CG iterations, gradient
            evaluations) at the accuracy the benchmark runs at, which scales the
            timed CPU-baseline sample.

Usage: python tests/golden/make_ground_states.py fcc5 tight [--threads N]
       (clusters: fcc5 = 666 atoms at h = 0.5 on 128^3, fcc8 = 2457 atoms at
       h = 0.45 on 192^3; both 12th order)
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1405_6456_gb300 import workloads as W  # noqa: E402

CLUSTERS = {"fcc5": W.cluster_c2, "fcc8": W.cluster_c3}
TOLS = {
    "tight": dict(tol_E=1e-9, tol_inner=1e-10, tol_poisson=1e-10),
    "product": dict(tol_E=1e-6, tol_inner=1e-8, tol_poisson=1e-8),
}


def path_for(cluster_name: str, tol: str) -> str:
    return os.path.join(HERE, f"ground_state_{cluster_name}_{tol}.json")


def run(which: str, tol: str, threads: int) -> dict:
    c = CLUSTERS[which]()
    O.set_threads(threads)
    g = O.grid_for_atoms(c.R, c.h, c.vacuum, 16)
    t = TOLS[tol]
    M = c.M
    p = O.default_params(fd_n=c.fd_order // 2, tol_E=t["tol_E"] * M, tol_inner=t["tol_inner"] * M,
                         tol_poisson=t["tol_poisson"])
    t0 = time.perf_counter()
    res, _u, phi, _b = O.solve(g, p, c.R, c.Z)
    F = O.forces(g, c.fd_order // 2, c.R, c.Z, phi)
    wall = time.perf_counter() - t0
    return {
        "cluster": c.name,
        "source": "oracle/ (FP64 CPU), written by tests/golden/make_ground_states.py",
        "seed": c.seed,
        "M": M,
        "N": c.N,
        "h": c.h,
        "fd_order": c.fd_order,
        "vacuum": c.vacuum,
        "grid": [g.n1, g.n2, g.n3],
        "tolerances": {"tol_E_per_atom": t["tol_E"], "tol_inner_per_atom": t["tol_inner"],
                       "tol_poisson": t["tol_poisson"]},
        "E": res.E,
        "E_per_atom": res.E / M,
        "eta": res.eta,
        "C": res.C,
        "parts": {k: getattr(res.parts, k) for k in ("E_tf", "E_vw", "E_xc", "E_es", "E_self")},
        "forces_paper": F.tolist(),
        "converged": bool(res.converged),
        "counts": {"outer_iters": res.outer_iters, "nlcg_iters": res.nlcg_iters,
                   "grad_evals": res.grad_evals, "cg_iters": res.cg_iters,
                   "stencil_apps": int(res.stencil_apps)},
        "oracle_threads": O.threads(),
        "oracle_wall_s": round(wall, 1),
    }


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("cluster", choices=sorted(CLUSTERS))
    ap.add_argument("tol", choices=sorted(TOLS))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    out = run(a.cluster, a.tol, a.threads)
    with open(path_for(out["cluster"], a.tol), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("cluster", "E_per_atom", "eta", "C", "counts", "oracle_wall_s")}))


if __name__ == "__main__":
    main()
