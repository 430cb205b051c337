"""GPU tests of the rows beyond the core path: warm-started ground states
(ofdft_solve_from), geometry relaxation (ofdft_relax) and the binding-energy
workload, each checked against the FP64 CPU oracle or against the library's
own cold-start results.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1405_6456_gb300 import binding as BE
from paper_1405_6456_gb300 import build as B
from paper_1405_6456_gb300 import ofdft as F
from paper_1405_6456_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    c = F.Context(0)
    yield c
    c.close()


def _ogrid(g):
    return O.make_grid(g.n[0], g.n[1], g.n[2], g.h, tuple(g.origin))


def _params(**kw):
    base = dict(fd_order=6, tol_E=1e-10, tol_inner=1e-11, tol_poisson=1e-11, max_outer=40, max_nlcg=4000)
    base.update(kw)
    return F.default_params(**base)


@pytest.mark.parametrize("prec", [F.PREC_FP64, F.PREC_MIXED])
def test_warm_start_reaches_the_same_ground_state_faster(ctx, prec):
    c = W.tiny_cluster("dimer", h=0.8, fd_order=6)
    g = F.ofdft_grid_for_atoms(c.R, c.h, c.vacuum, 1)
    dt = torch.float64 if prec == F.PREC_FP64 else torch.float32
    p = _params(precision=prec) if prec == F.PREC_FP64 else _params(precision=prec, tol_E=1e-8, tol_inner=1e-8,
                                                                       tol_poisson=1e-9)
    u = torch.empty(g.shape, dtype=dt, device=DEV)
    phi = torch.empty_like(u)
    E0, F0, s0 = ctx.solve(c.R, c.Z, c.h, p, grid=g, u_out=u, phi_out=phi)
    # restart from the converged state (u, phi and the multipliers): same
    # minimum, a fraction of the work
    pw = F.Params.from_buffer_copy(p)
    pw.eta0 = s0.eta
    pw.mu0 = p.mu0 * p.kappa ** (s0.outer_iters - 1)
    E1, F1, s1 = ctx.solve_from(c.R, c.Z, c.h, pw, g, u_in=u, phi_in=phi, u_out=u, phi_out=phi)
    assert s0.converged and s1.converged
    tolE = 1e-9 if prec == F.PREC_FP64 else 1e-6
    assert abs(E1 - E0) / c.M <= tolE
    np.testing.assert_allclose(F1, F0, atol=1e-6 if prec == F.PREC_FP64 else 1e-4)
    # (with the multigrid-preconditioned Poisson CG a cold solve already needs
    # few iterations per evaluation, so the saving is smaller than with plain CG)
    assert s1.cg_iters < 0.6 * s0.cg_iters
    # a warm start needs the grid it was computed on
    with pytest.raises(F.OfdftError):
        ctx._check(ctx._lib.ofdft_solve_from(ctx.h, None, F._dp(np.ascontiguousarray(c.R)),
                                             F._dp(np.ascontiguousarray(c.Z)), c.M, c.h, F.C.byref(p),
                                             u.data_ptr(), None, None, None, F._dp(np.zeros(1)), None, None),
                   "ofdft_solve_from")


def test_relaxation_ends_where_the_oracle_sees_no_force(ctx):
    """Relax a stretched dimer on a fixed grid; the oracle's forces at the
    relaxed geometry (same grid, same parameters) are below the tolerance."""
    c = W.tiny_cluster("dimer", h=0.8, fd_order=6)
    R0 = np.array(c.R, copy=True)
    R0[0, 0] -= 0.3  # stretch the bond by 0.3 bohr
    g = F.ofdft_grid_for_atoms(R0, c.h, c.vacuum + 2.0, 1)
    p = _params()
    E_start, F_start, _ = ctx.solve(R0, c.Z, c.h, p, grid=g)
    f_tol = 1e-3
    R, E, Fr, st = ctx.relax(R0, c.Z, c.h, p, grid=g, max_steps=60, f_tol=f_tol, max_move=0.05)
    assert st.converged and st.steps >= 1 and st.solves >= 2 * st.steps
    assert np.linalg.norm(Fr, axis=1).max() < f_tol
    assert E < E_start
    assert np.linalg.norm(F_start, axis=1).max() > 5 * f_tol  # the start was not relaxed
    # the oracle at the relaxed geometry
    po = O.default_params(fd_n=3, tol_E=1e-10 * c.M, tol_inner=1e-12, tol_poisson=1e-12, max_outer=40,
                          max_nlcg=4000)
    res, _, phi, _ = O.solve(_ogrid(g), po, R, c.Z)
    Fo = O.forces(_ogrid(g), 3, R, c.Z, phi)
    assert np.linalg.norm(Fo, axis=1).max() < f_tol + 1e-5
    assert abs(res.E - E) / c.M <= 1e-8


def test_binding_energy_matches_oracle():
    """E_b = E*(14-atom FCC cube) / M - E*(atom), both on grids of the box rule."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    ctx = F.Context(0)
    try:
        h, vac = 0.8, 6.0
        p = F.default_params(fd_order=6, vacuum=vac, round_to=1, tol_E=1e-9, tol_inner=1e-10, tol_poisson=1e-11)
        E_atom, res = BE.binding_energies(ctx, [1], h=h, params=p)
        r = res[0]
        assert r.atoms == 14
        po = O.default_params(fd_n=3, tol_E=1e-9, tol_inner=1e-11, tol_poisson=1e-11, max_outer=40, max_nlcg=4000)
        Ra = np.zeros((1, 3))
        ga = O.grid_for_atoms(Ra, h, vac, 1)
        ea, _, _, _ = O.solve(ga, po, Ra, np.array([3.0]))
        Rc = W.fcc_cube_sites(1, 7.6)
        gc = O.grid_for_atoms(Rc, h, vac, 1)
        po_c = O.default_params(fd_n=3, tol_E=1e-9 * 14, tol_inner=1e-11, tol_poisson=1e-11, max_outer=40,
                                max_nlcg=4000)
        ec, _, _, _ = O.solve(gc, po_c, Rc, np.full(14, 3.0))
        assert E_atom == pytest.approx(ea.E, abs=1e-7)
        assert r.binding_per_atom == pytest.approx(ec.E / 14 - ea.E, abs=1e-7)
        assert r.binding_per_atom < 0  # the cluster binds
    finally:
        ctx.close()
