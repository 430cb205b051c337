"""Continuous-batching request loop over the batch engine (ofdft_batch_*).

Requests (cluster solves of different sizes) arrive over time.  The loop
submits each one when its arrival time has passed; the engine admits queued
requests between rounds while their workspace fits the HBM budget, keeps every
admitted solve's u, phi, CG and NLCG vectors and (eta, mu) resident on the
device, and advances all of them together one evaluation round per step.  The
loop polls for finished requests and records their latency (finish - arrival)
and whether the solve converged: a request that hit an iteration cap
(OFDFT_ENOTCONV) is counted apart and left out of the throughput and latency
figures, which are stated at the solves' tolerances.  All numerical work happens
in the library; this module only schedules calls.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import ofdft as F


@dataclasses.dataclass
class RequestResult:
    rid: int
    arrival_s: float
    admit_s: float
    finish_s: float
    energy: float
    forces: np.ndarray
    stats: object
    name: str = ""
    converged: bool = True

    @property
    def latency_s(self) -> float:
        return self.finish_s - self.arrival_s


@dataclasses.dataclass
class ServeReport:
    results: list
    wall_s: float
    rounds: int

    def summary(self) -> dict:
        """Throughput and latency over the converged requests; requests that hit
        an iteration cap are counted in `unconverged` only."""
        ok = [r for r in self.results if r.converged]
        lat = np.array([r.latency_s for r in ok]) if ok else np.zeros(1)
        return {"requests": len(self.results), "converged": len(ok),
                "unconverged": len(self.results) - len(ok), "wall_s": self.wall_s,
                "throughput_per_s": len(ok) / self.wall_s if self.wall_s > 0 else 0.0,
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "latency_mean_s": float(lat.mean()), "rounds": self.rounds}


def serve(ctx: F.Context, requests, params_for, precision=F.PREC_MIXED, hbm_budget_bytes=64 << 30,
          grid_for=None, time_scale=1.0, strict=False) -> ServeReport:
    """Run the request loop.

    requests: iterable of (arrival_s, cluster) with cluster.R, cluster.Z, cluster.h;
    params_for(cluster) -> Params; grid_for(cluster) -> Grid or None (box rule).
    time_scale stretches (>1) or compresses (<1) the arrival times.
    strict: raise OfdftError when a request ends without converging (otherwise it
    is recorded with converged=False and reported apart).
    """
    pending = collections.deque(sorted(requests, key=lambda t: t[0]))
    bt = F.Batch(ctx, precision, hbm_budget_bytes)
    inflight = {}
    results = []
    rounds = 0
    t0 = time.perf_counter()
    try:
        while pending or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0][0] * time_scale <= now:
                arr, c = pending.popleft()
                grid = grid_for(c) if grid_for else None
                rid = bt.submit(c.R, c.Z, c.h, params_for(c), grid=grid)
                inflight[rid] = (arr * time_scale, c, now)
            if not inflight:
                wait = pending[0][0] * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
                continue
            bt.step()
            rounds += 1
            t_now = time.perf_counter() - t0
            for rid in list(inflight):
                out = bt.poll(rid, allow_notconv=not strict)
                if out is None:
                    continue
                arr, c, sub = inflight.pop(rid)
                E, Fv, st = out
                results.append(RequestResult(rid, arr, sub, t_now, E, Fv, st, getattr(c, "name", ""),
                                             bool(st.converged)))
    finally:
        bt.close()
    return ServeReport(results, time.perf_counter() - t0, rounds)
