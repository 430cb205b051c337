"""Binding energies of the m x m x m FCC cluster series (Sec. 5, the binding
energy per atom against the isolated atom with the same discretisation).

  E_b(m) = E*(cluster m) / M - E*(isolated atom)

Every ground state is computed by the library (ofdft_solve); this module only
builds the geometries and combines the energies.  With Gaussian nuclei instead
of the paper's pseudopotential the values show the series' shape, not the
paper's numbers.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import ofdft as F
from . import workloads as W


@dataclasses.dataclass
class BindingResult:
    m: int
    atoms: int
    energy: float            # E* of the cluster (Ha)
    energy_per_atom: float   # E* / M
    binding_per_atom: float  # E* / M - E*(atom)
    grid: tuple
    cg_iters: int


def atom_energy(ctx: F.Context, h: float, params: F.Params, Z: float = 3.0):
    """E* of one isolated atom on a grid with the same spacing, order and vacuum
    (params.vacuum, params.round_to)."""
    R = np.zeros((1, 3))
    E, _, st = ctx.solve(R, np.array([Z]), h, params, want_forces=False)
    return E, st


def binding_energies(ctx: F.Context, ms, h: float = 0.5, a: float = 7.6, Z: float = 3.0, params: F.Params | None = None,
                     seed: int | None = None, amp: float = 0.1):
    """E_b per atom of the m x m x m FCC cubes (lattice constant a, seeded
    displacements of amplitude amp unless seed is None)."""
    p = params if params is not None else F.default_params()
    E_atom, _ = atom_energy(ctx, h, p, Z)
    out = []
    for m in ms:
        R = W.fcc_cube_sites(m, a)
        if seed is not None:
            R = W.displaced(R, amp, seed)
        Zs = np.full(len(R), Z)
        E, _, st = ctx.solve(R, Zs, h, p, want_forces=False)
        M = len(R)
        out.append(BindingResult(m, M, E, E / M, E / M - E_atom, tuple(st.grid.n), st.cg_iters))
    return E_atom, out
