"""Batched and continuously served solves (S11, S12) through the C ABI.

A solve's arithmetic in a batch depends only on its own grid (its tiles, its
reduction order), never on which other solves share the launches, so a request
must give the same result alone and in any mix: the test demands bit equality.
Against single solves (ofdft_solve, other launch shapes) and the oracle the
tolerances are the converged-solve ones.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1405_6456_gb300 import build as B
from paper_1405_6456_gb300 import ofdft as F
from paper_1405_6456_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GB = 1 << 30


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.Context(0)
    yield c
    c.close()


def _params(order, prec=F.PREC_FP64, **kw):
    base = dict(fd_order=order, precision=prec, tol_E=1e-10, tol_inner=1e-13, tol_poisson=1e-12,
                max_outer=40, max_nlcg=4000)
    base.update(kw)
    return F.default_params(**base)


def _mix():
    return [W.tiny_cluster("dimer", h=0.8, fd_order=6), W.tiny_cluster("trimer", h=0.7, fd_order=12),
            W.tiny_cluster("atom", h=0.6, fd_order=8), W.cluster_c1()]


def _grid(c):
    return F.ofdft_grid_for_atoms(c.R, c.h, c.vacuum, 2)


def test_batch_fp64_matches_single_solves_and_oracle(ctx):
    cases = _mix()
    bt = F.Batch(ctx, F.PREC_FP64, 8 * GB)
    ids = [bt.submit(c.R, c.Z, c.h, _params(c.fd_order), grid=_grid(c)) for c in cases]
    bt.run()
    for c, rid in zip(cases, ids):
        E, Fv, st = bt.poll(rid)
        assert st.converged
        E1, F1, st1 = ctx.solve(c.R, c.Z, c.h, _params(c.fd_order), grid=_grid(c))
        assert abs(E - E1) / c.M <= 1e-9, c.name
        assert np.abs(Fv - F1).max() <= 1e-7, c.name
    c = cases[0]
    g = _grid(c)
    po = O.default_params(fd_n=3, tol_E=1e-10 * c.M, tol_inner=1e-12, tol_poisson=1e-12, max_outer=40,
                          max_nlcg=4000)
    res, _, phi, _ = O.solve(O.make_grid(g.n[0], g.n[1], g.n[2], g.h, tuple(g.origin)), po, c.R, c.Z)
    rid = bt.submit(c.R, c.Z, c.h, _params(6), grid=g)
    bt.run()
    E, Fv, st = bt.poll(rid)
    assert abs(E - res.E) / c.M <= 1e-8
    bt.close()


@pytest.mark.parametrize("prec", [F.PREC_MIXED, F.PREC_FP64])
def test_request_is_identical_alone_and_in_the_mix(ctx, prec):
    cases = _mix()
    target = cases[3]
    p = _params(12, prec, tol_E=1e-8, tol_inner=1e-9, tol_poisson=1e-9)
    alone = F.Batch(ctx, prec, 8 * GB)
    rid = alone.submit(target.R, target.Z, target.h, p, grid=_grid(target))
    alone.run()
    Ea, Fa, sa = alone.poll(rid)
    alone.close()
    mix = F.Batch(ctx, prec, 8 * GB)
    others = [mix.submit(c.R, c.Z, c.h, _params(c.fd_order, prec, tol_E=1e-8, tol_inner=1e-9, tol_poisson=1e-9),
                         grid=_grid(c)) for c in cases[:3]]
    rid = mix.submit(target.R, target.Z, target.h, p, grid=_grid(target))
    mix.run()
    Em, Fm, sm = mix.poll(rid)
    for o in others:
        assert mix.poll(o) is not None
    mix.close()
    assert Em == Ea
    assert np.array_equal(Fm, Fa)
    assert (sm.grad_evals, sm.cg_iters, sm.nlcg_iters) == (sa.grad_evals, sa.cg_iters, sa.nlcg_iters)
    if prec == F.PREC_MIXED:
        # and the mixed result is within the stated 1e-5 Ha/atom of FP64
        E64, _, _ = ctx.solve(target.R, target.Z, target.h, _params(12, F.PREC_FP64, tol_E=1e-8, tol_inner=1e-9,
                                                                    tol_poisson=1e-9), grid=_grid(target))
        assert abs(Em - E64) / target.M <= 1e-5


def test_admission_by_hbm_budget_queues_and_completes(ctx):
    cases = _mix() * 2
    need = max(F.batch_bytes(_grid(c), F.PREC_MIXED) for c in cases)
    bt = F.Batch(ctx, F.PREC_MIXED, int(1.5 * need))  # room for about one solve at a time
    ids = [bt.submit(c.R, c.Z, c.h, _params(c.fd_order, F.PREC_MIXED, tol_E=1e-7, tol_inner=1e-8,
                                            tol_poisson=1e-8), grid=_grid(c)) for c in cases]
    na, nq = bt.step()
    assert nq > 0  # the budget holds some requests back
    bt.run()
    Es = [bt.poll(i)[0] for i in ids]
    n = len(cases) // 2
    np.testing.assert_array_equal(Es[:n], Es[n:])  # same request, same result, whatever the queueing
    bt.close()


def test_serving_loop_results_match_solo_and_report_latency(ctx):
    """Requests arriving while others run join the mix (continuous batching) and
    finish with the result they have alone (bit-identical), each with a latency."""
    from paper_1405_6456_gb300 import serving as S
    cases = _mix()[:3]
    prm = lambda c: _params(c.fd_order, F.PREC_MIXED, tol_E=1e-7, tol_inner=1e-8, tol_poisson=1e-8)
    solo = []
    for c in cases:
        bt = F.Batch(ctx, F.PREC_MIXED, 8 * GB)
        rid = bt.submit(c.R, c.Z, c.h, prm(c), grid=_grid(c))
        bt.run()
        solo.append(bt.poll(rid)[0])
        bt.close()
    reqs = [(0.0, cases[0]), (0.05, cases[1]), (0.1, cases[2])]
    rep = S.serve(ctx, reqs, prm, precision=F.PREC_MIXED, hbm_budget_bytes=8 * GB, grid_for=_grid)
    assert len(rep.results) == 3
    by_name = {r.name: r for r in rep.results}
    for c, Es in zip(cases, solo):
        r = by_name[c.name]
        assert r.energy == Es
        assert r.latency_s > 0 and r.finish_s >= r.admit_s >= r.arrival_s - 1e-9
    s = rep.summary()
    assert s["latency_p99_s"] >= s["latency_p50_s"] > 0
