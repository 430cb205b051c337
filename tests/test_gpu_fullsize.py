"""Whole ground states at full size against the FP64 oracle's, through the C ABI.

The reference values are the oracle's ground states of the 666-atom cluster
(5x5x5 FCC cells, h = 0.5, 12th order, 128^3) and of the 2457-atom cluster
(8x8x8 cells, h = 0.45, 192^3), written to tests/golden/ by
tests/golden/make_ground_states.py, which calls only oracle/.  Targets:
  - FP64 path: 1e-6 Ha/atom in energy and 1e-5 Ha/bohr in forces, at
    tightened solver tolerances;
  - MIXED path: 1e-5 Ha/atom in energy; at tightened tolerances its forces
    (from the FP64 potential of the last residual correction) meet 1e-5 Ha/bohr
    as well;
  - at the library's default tolerances (the benchmark's) the energy targets
    hold; the forces, first order in the remaining density error where the
    energy is second order, are within 5e-5 Ha/bohr (measured 2.1e-5 FP64 and
    1.2e-5 MIXED on the 666-atom cluster), and within 1e-4 Ha/bohr for MIXED on
    the 2457-atom cluster (measured 6.4e-5; its energy is 2.7e-7 Ha/atom from
    the oracle's).  The 1e-5 Ha/bohr force bound is the FP64 path's.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1405_6456_gb300 import build as B
from paper_1405_6456_gb300 import ofdft as F
from paper_1405_6456_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    # the fixed launch shapes (no timing-based autotuning): the order of every
    # partial sum, and with it the solver's path, is the same on every run
    old = os.environ.get("OFDFT_AUTOTUNE")
    os.environ["OFDFT_AUTOTUNE"] = "0"
    try:
        c = F.Context(0)
    finally:
        if old is None:
            del os.environ["OFDFT_AUTOTUNE"]
        else:
            os.environ["OFDFT_AUTOTUNE"] = old
    yield c
    c.close()


def _golden(cluster, tol):
    path = os.path.join(GOLDEN, f"ground_state_{cluster.name}_{tol}.json")
    with open(path) as f:
        gd = json.load(f)
    assert gd["converged"] and gd["M"] == cluster.M
    return gd


def _check(ctx, c, gd, prec, tolE, tolF, **kw):
    p = F.default_params(precision=prec, vacuum=c.vacuum, round_to=16, **kw)
    E, Fv, st = ctx.solve(c.R, c.Z, c.h, p)
    assert st.converged
    assert list(st.grid.n) == gd["grid"]
    dE = abs(E - gd["E"]) / c.M
    dF = float(np.abs(Fv - np.array(gd["forces_paper"])).max())
    print(f"\n{c.name} {'MIXED' if prec == F.PREC_MIXED else 'FP64'}: |dE| = {dE:.2e} Ha/atom, "
          f"max |dF| = {dF:.2e} Ha/bohr, eta {st.eta:.9f} (oracle {gd['eta']:.9f})")
    assert dE <= tolE
    assert dF <= tolF
    return st


def test_fp64_ground_state_666_atoms_matches_oracle(ctx):
    """666 atoms, 128^3: FP64 at tightened tolerances against the oracle's
    tightly converged ground state."""
    c = W.cluster_c2()
    gd = _golden(c, "tight")
    st = _check(ctx, c, gd, F.PREC_FP64, 1e-6, 1e-5, tol_E=1e-8, tol_inner=1e-10, tol_poisson=1e-10)
    # the multiplier is first order in the remaining constraint violation C / mu,
    # which the two solves leave at different outer iterations
    assert st.eta == pytest.approx(gd["eta"], abs=5e-5)


def test_fp64_ground_state_666_atoms_product_tolerances(ctx):
    """The same at the library's default tolerances (the benchmark's)."""
    c = W.cluster_c2()
    _check(ctx, c, _golden(c, "tight"), F.PREC_FP64, 1e-6, 5e-5)


def test_mixed_ground_state_666_atoms_matches_oracle(ctx):
    """MIXED at the default tolerances."""
    c = W.cluster_c2()
    _check(ctx, c, _golden(c, "tight"), F.PREC_MIXED, 1e-5, 5e-5)


def test_mixed_ground_state_666_atoms_tight_tolerances(ctx):
    """MIXED at tightened tolerances: the forces meet the FP64 path's 1e-5 Ha/bohr."""
    c = W.cluster_c2()
    _check(ctx, c, _golden(c, "tight"), F.PREC_MIXED, 1e-5, 1e-5, tol_E=1e-8, tol_inner=1e-10, tol_poisson=1e-9)


def _fcc8_golden():
    c = W.cluster_c3()
    if not os.path.exists(os.path.join(GOLDEN, f"ground_state_{c.name}_product.json")):
        pytest.skip("2457-atom oracle ground state not written")
    return c, _golden(c, "product")


def test_mixed_ground_state_2457_atoms_matches_oracle(ctx):
    """The benchmark's workload (2457 atoms, 192^3) in the benchmark's form
    (MIXED, default tolerances) against the oracle's ground state at the same
    tolerances."""
    c, gd = _fcc8_golden()
    _check(ctx, c, gd, F.PREC_MIXED, 1e-5, 1e-4)


def test_fp64_ground_state_2457_atoms_matches_oracle(ctx):
    c, gd = _fcc8_golden()
    _check(ctx, c, gd, F.PREC_FP64, 1e-6, 5e-5)
