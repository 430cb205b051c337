"""CPU checks of the C-ABI library: it builds, loads, and exports every entry
point that include/ofdft.h declares; host-only calls behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1405_6456_gb300 import build as B
from paper_1405_6456_gb300 import ofdft as F
from paper_1405_6456_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ofdft_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.lib()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 12
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(F.exported_symbols()) <= declared


def test_default_params_follow_the_paper(lib):
    p = F.default_params()
    assert p.lam == 0.2  # Sec. 5
    assert (p.eta0, p.mu0, p.kappa) == (-0.2, 1.0, 0.1)  # Sec. 5.3.1
    assert p.fd_order == 12 and p.terms == F.TERM_ALL and p.method == F.METHOD_AL


def test_binding_struct_layouts_match_the_library(lib):
    lib.ofdft_struct_bytes.restype = ctypes.c_longlong
    lib.ofdft_struct_bytes.argtypes = [ctypes.c_char_p]
    for name, cls in [("ofdft_grid", F.Grid), ("ofdft_params", F.Params), ("ofdft_cg_stats", F.CgStats),
                      ("ofdft_energy", F.Energy), ("ofdft_solve_stats", F.SolveStats),
                      ("ofdft_counters", F.Counters), ("ofdft_relax_stats", F.RelaxStats),
                      ("ofdft_batch_stats", F.BatchStats)]:
        assert lib.ofdft_struct_bytes(name.encode()) == ctypes.sizeof(cls), name
    assert lib.ofdft_struct_bytes(b"nothing") == -1
    p = F.default_params()
    assert p.poisson_adapt == 1.0 and p.refine_every == 200 and p.tol_poisson == 1e-8


def test_box_rule_matches_oracle_box_rule(lib):
    for c in [W.cluster_c1(), W.cluster_c2(), W.tiny_cluster("dimer")] + W.batch_c4(6):
        for rt in (1, 2, 16):
            g = F.ofdft_grid_for_atoms(c.R, c.h, c.vacuum, rt)
            go = O.grid_for_atoms(c.R, c.h, c.vacuum, rt)
            assert tuple(g.n) == (go.n1, go.n2, go.n3)
            np.testing.assert_allclose(list(g.origin), list(go.origin), rtol=0, atol=1e-12)


def test_host_argument_checks(lib):
    g = F.Grid()
    R = np.zeros(3)
    assert lib.ofdft_grid_for_atoms(R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 0.5, 8.0,
                                    16, ctypes.byref(g)) == F.EINVAL
    assert lib.ofdft_grid_for_atoms(R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, -0.5, 8.0,
                                    16, ctypes.byref(g)) == F.EINVAL
    bad = np.array([0.0, np.nan, 0.0])
    assert lib.ofdft_grid_for_atoms(bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, 0.5, 8.0,
                                    16, ctypes.byref(g)) == F.ENONFINITE
    assert lib.ofdft_destroy(None) == F.OK
    assert lib.ofdft_last_error(None) == b"null context"
    assert lib.ofdft_set_poisson_precond(None, F.PRECOND_MG) == F.EINVAL
    gg = F.make_grid(128, 128, 128, 0.5)
    assert F.workspace_bytes(gg, 12, F.PREC_FP64) > F.workspace_bytes(gg, 12, F.PREC_MIXED) > 0


def _levels_by_rule(dims):
    """The coarsening rule written out: halve every extent (floor) while every
    extent is at least 4."""
    out = [tuple(dims)]
    while min(out[-1]) >= 4:
        out.append(tuple(n // 2 for n in out[-1]))
    return out


@pytest.mark.parametrize("dims", [(128, 128, 128), (192, 192, 192), (37, 29, 23), (48, 40, 36), (5, 70, 9),
                                  (3, 40, 40), (80, 80, 80), (1, 1, 1), (4, 4, 4), (400, 4, 400)])
@pytest.mark.parametrize("prec", [F.PREC_FP64, F.PREC_MIXED])
def test_multigrid_level_plan(lib, dims, prec):
    g = F.make_grid(*dims, 0.5)
    plan = F.mg_plan(g, prec)
    levels = _levels_by_rule(dims)
    assert plan["levels"] == levels
    nodes = [a * b * c for a, b, c in levels]
    small = [l for l, n in enumerate(nodes) if n <= 4096]
    es = 4 if prec == F.PREC_MIXED else 8
    if small:
        lc = small[0]
        assert plan["coarse_level"] == lc
        # z and one scratch vector at the finest level, r, z, t of levels 1..lc
        assert plan["bytes"] == (2 * nodes[0] + 3 * sum(nodes[1:lc + 1])) * es
        # the one-block coarse end keeps r, z, t of its levels in shared memory
        assert 3 * sum(nodes[lc:]) * es <= 200 * 1024
    else:
        assert plan["coarse_level"] == -1 and plan["bytes"] == 0
    if dims == (128, 128, 128):
        assert plan["coarse_level"] == 3 and len(levels) == 7  # 128 .. 2, the block from 16^3
    if dims == (3, 40, 40):
        assert plan["coarse_level"] == -1  # an extent below 4, 4800 nodes: plain CG


def test_multigrid_plan_rejects_bad_grids(lib):
    with pytest.raises(F.OfdftError):
        F.mg_plan(F.make_grid(0, 8, 8, 0.5))
    with pytest.raises(F.OfdftError):
        F.mg_plan(F.make_grid(8, 8, 8, -0.5))
