"""Thin Python binding of the C ABI in include/ofdft.h (argument marshalling only).

Every numerical step runs in the CUDA library libofdft.so; this module converts
torch tensors to device pointers and ctypes structures.  There is no CPU
fallback: if the library cannot be loaded, every call raises.

Field tensors are CUDA tensors of shape (n3, n2, n1) (x fastest), float64 for
OFDFT_PREC_FP64 and float32 for OFDFT_PREC_MIXED.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libofdft.so")

OK, EINVAL, ENOMEM, ENOTCONV, ENONFINITE, ETIMEOUT, ECUDA = range(7)
PREC_FP64, PREC_MIXED = 0, 1
TERM_TF, TERM_VW, TERM_XC, TERM_ES, TERM_ALL = 1, 2, 4, 8, 15
METHOD_AL, METHOD_PENALTY, METHOD_LM = 0, 1, 2
FORCE_PAPER, FORCE_EXACT = 0, 1
_STATUS = {0: "OFDFT_OK", 1: "OFDFT_EINVAL", 2: "OFDFT_ENOMEM", 3: "OFDFT_ENOTCONV",
           4: "OFDFT_ENONFINITE", 5: "OFDFT_ETIMEOUT", 6: "OFDFT_ECUDA"}


class OfdftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double), ("origin", C.c_double * 3)]

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def size(self):
        return self.n[0] * self.n[1] * self.n[2]

    def __repr__(self):
        return f"Grid(n={tuple(self.n)}, h={self.h}, origin={tuple(round(o, 6) for o in self.origin)})"


class Params(C.Structure):
    _fields_ = [("fd_order", C.c_int), ("terms", C.c_int), ("method", C.c_int),
                ("precision", C.c_int), ("lam", C.c_double), ("eta0", C.c_double),
                ("mu0", C.c_double), ("kappa", C.c_double), ("sigma", C.c_double),
                ("rc", C.c_double), ("guess_sigma", C.c_double), ("guess_cut", C.c_double),
                ("tol_E", C.c_double), ("tol_inner", C.c_double), ("tol_poisson", C.c_double),
                ("max_outer", C.c_int), ("max_nlcg", C.c_int), ("max_cg", C.c_int),
                ("max_secant", C.c_int), ("sigma0", C.c_double), ("eps_secant", C.c_double),
                ("restart_every", C.c_int), ("force_variant", C.c_int),
                ("ezz_correction", C.c_int), ("vacuum", C.c_double), ("round_to", C.c_int),
                ("refine_every", C.c_int), ("trial_max_rel", C.c_double), ("max_backtrack", C.c_int),
                ("precond_rank1", C.c_int), ("poisson_adapt", C.c_double),
                ("trial_poisson_loosen", C.c_double)]


class CgStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double)]


class Energy(C.Structure):
    _fields_ = [("L", C.c_double), ("E", C.c_double), ("E_tf", C.c_double),
                ("E_vw", C.c_double), ("E_xc", C.c_double), ("E_es", C.c_double),
                ("E_self", C.c_double), ("E_zz_corr", C.c_double), ("C", C.c_double),
                ("gd", C.c_double), ("gs_old", C.c_double), ("gnorm2", C.c_double),
                ("rs", C.c_double), ("rs_pc", C.c_double), ("poisson", CgStats)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "poisson"}
        d["cg_iters"] = self.poisson.iterations
        d["cg_relres"] = self.poisson.rel_residual
        return d


K_STENCIL, K_CG_DIR_STENCIL, K_CG_UPDATE, K_RESIDUAL, K_FUNCTIONAL, K_VECTOR, K_ATOMS, K_CG_PERSISTENT, K_MG = range(9)
K_COUNT = 9
KIND_NAMES = ["stencil", "cg_dir_stencil", "cg_update", "residual", "functional", "vector", "atoms",
              "cg_persistent", "mg"]
PRECOND_NONE, PRECOND_MG = 0, 1


class Counters(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("kind_launches", C.c_longlong * K_COUNT),
                ("timed_launches", C.c_longlong * K_COUNT), ("timed_ms", C.c_double * K_COUNT),
                ("persistent_cg_iters", C.c_longlong), ("tma_launches", C.c_longlong)]


class SolveStats(C.Structure):
    _fields_ = [("E", C.c_double), ("eta", C.c_double), ("C", C.c_double), ("parts", Energy),
                ("outer_iters", C.c_int), ("nlcg_iters", C.c_int), ("grad_evals", C.c_int),
                ("cg_iters", C.c_int), ("energy_evals", C.c_int), ("stencil_apps", C.c_longlong),
                ("converged", C.c_int),
                ("grid", Grid)]


class RelaxStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("solves", C.c_int), ("cg_iters", C.c_longlong), ("max_force", C.c_double),
                ("energy", C.c_double), ("converged", C.c_int)]


class BatchStats(C.Structure):
    _fields_ = [("rounds", C.c_longlong), ("graph_captures", C.c_longlong), ("graph_replays", C.c_longlong),
                ("graph_iterations", C.c_longlong), ("eager_iterations", C.c_longlong), ("z_depth", C.c_int),
                ("z_tuned", C.c_int), ("tune_candidates", C.c_int), ("tune_depth", C.c_int * 8),
                ("tune_us", C.c_double * 8)]

    def as_dict(self):
        n = self.tune_candidates
        return {"rounds": self.rounds, "graph_captures": self.graph_captures,
                "graph_replays": self.graph_replays, "graph_iterations": self.graph_iterations,
                "eager_iterations": self.eager_iterations, "z_depth": self.z_depth, "z_tuned": self.z_tuned,
                "tuning_us_by_depth": {int(self.tune_depth[i]): round(float(self.tune_us[i]), 2) for i in range(n)}}


_lib = None


def lib():
    """Load libofdft.so (raises if it has not been built: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; run paper_1405_6456_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    L.ofdft_default_params.argtypes = [C.POINTER(Params)]
    L.ofdft_default_params.restype = None
    L.ofdft_create.argtypes = [C.POINTER(vp), ip, vp]
    L.ofdft_destroy.argtypes = [vp]
    L.ofdft_last_error.argtypes = [vp]
    L.ofdft_last_error.restype = C.c_char_p
    L.ofdft_grid_for_atoms.argtypes = [dp, ip, C.c_double, C.c_double, ip, C.POINTER(Grid)]
    L.ofdft_stencil.argtypes = [vp, C.POINTER(Grid), ip, ip, vp, vp]
    L.ofdft_pseudocharge.argtypes = [vp, C.POINTER(Grid), ip, dp, dp, ip, C.c_double, C.c_double, ip,
                                     vp, dp]
    L.ofdft_initial_guess.argtypes = [vp, C.POINTER(Grid), dp, dp, ip, C.c_double, C.c_double,
                                      C.c_double, ip, vp]
    L.ofdft_poisson.argtypes = [vp, C.POINTER(Grid), ip, ip, vp, vp, vp, vp, C.c_double, ip,
                                C.POINTER(CgStats)]
    L.ofdft_energy_grad.argtypes = [vp, C.POINTER(Grid), C.POINTER(Params), vp, vp, vp, C.c_double,
                                    C.c_double, C.c_double, C.c_double, ip, vp, vp, vp, vp,
                                    C.POINTER(Energy)]
    L.ofdft_forces.argtypes = [vp, C.POINTER(Grid), ip, dp, dp, ip, C.c_double, C.c_double, ip, ip,
                               vp, dp]
    L.ofdft_overlap_correction.argtypes = [vp, C.POINTER(Grid), ip, dp, dp, ip, C.c_double, C.c_double,
                                           C.c_double, C.c_double, C.c_double, dp, dp]
    L.ofdft_solve.argtypes = [vp, C.POINTER(Grid), dp, dp, ip, C.c_double, C.POINTER(Params), vp,
                              vp, dp, dp, C.POINTER(SolveStats)]
    L.ofdft_solve_from.argtypes = [vp, C.POINTER(Grid), dp, dp, ip, C.c_double, C.POINTER(Params), vp, vp,
                                   vp, vp, dp, dp, C.POINTER(SolveStats)]
    L.ofdft_relax.argtypes = [vp, C.POINTER(Grid), dp, dp, ip, C.c_double, C.POINTER(Params), ip, C.c_double,
                              C.c_double, dp, dp, C.POINTER(RelaxStats)]
    L.ofdft_struct_bytes.argtypes = [C.c_char_p]
    L.ofdft_struct_bytes.restype = C.c_longlong
    L.ofdft_profile.argtypes = [vp, ip]
    L.ofdft_set_poisson_precond.argtypes = [vp, ip]
    L.ofdft_get_counters.argtypes = [vp, C.POINTER(Counters)]
    L.ofdft_reset_counters.argtypes = [vp]
    L.ofdft_batch_create.argtypes = [vp, ip, C.c_longlong, C.POINTER(vp)]
    L.ofdft_batch_destroy.argtypes = [vp]
    L.ofdft_batch_submit.argtypes = [vp, dp, dp, ip, C.c_double, C.POINTER(Params), C.POINTER(Grid),
                                     C.POINTER(C.c_int)]
    L.ofdft_batch_step.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.ofdft_batch_poll.argtypes = [vp, ip, C.POINTER(C.c_int), dp, dp, C.POINTER(SolveStats)]
    L.ofdft_batch_run.argtypes = [vp]
    L.ofdft_batch_bytes.argtypes = [C.POINTER(Grid), ip]
    L.ofdft_batch_bytes.restype = C.c_longlong
    L.ofdft_batch_info.argtypes = [vp, C.POINTER(BatchStats)]
    L.ofdft_mg_plan.argtypes = [C.POINTER(Grid), ip, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
    L.ofdft_workspace_bytes.argtypes = [C.POINTER(Grid), ip, ip]
    L.ofdft_workspace_bytes.restype = C.c_longlong
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _host_f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("field tensors must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("field tensors must be contiguous")
    return C.c_void_p(t.data_ptr())


def prec_of(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return PREC_FP64
    if t.dtype == torch.float32:
        return PREC_MIXED
    raise ValueError(f"unsupported field dtype {t.dtype}")


def default_params(**kw) -> Params:
    p = Params()
    lib().ofdft_default_params(C.byref(p))
    for k, v in kw.items():
        k = "lam" if k == "lambda" else k
        if not any(k == f for f, _ in Params._fields_):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def ofdft_grid_for_atoms(R, h, vacuum, round_to=16) -> Grid:
    R = _host_f64(R).reshape(-1, 3)
    g = Grid()
    rc = lib().ofdft_grid_for_atoms(_dp(R), R.shape[0], h, vacuum, round_to, C.byref(g))
    if rc != OK:
        raise OfdftError(rc, "ofdft_grid_for_atoms")
    return g


def make_grid(n1, n2, n3, h, origin=(0.0, 0.0, 0.0)) -> Grid:
    g = Grid()
    g.n[0], g.n[1], g.n[2] = n1, n2, n3
    g.h = h
    for d in range(3):
        g.origin[d] = origin[d]
    return g


class Context:
    """An ofdft_ctx bound to a CUDA device and stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._lib = lib()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        rc = self._lib.ofdft_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise OfdftError(rc, "ofdft_create failed")
        self.h = h
        self._batches = weakref.WeakSet()

    def close(self):
        if self.h:
            for bt in list(self._batches):  # a batch must not outlive its context
                bt.close()
            self._lib.ofdft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what, allow=()):
        if rc != OK and rc not in allow:
            raise OfdftError(rc, f"{what}: {self._lib.ofdft_last_error(self.h).decode()}")
        return rc

    # tracing
    def set_poisson_precond(self, kind: int):
        """PRECOND_MG (default) or PRECOND_NONE for the Poisson CG of later calls."""
        return self._check(self._lib.ofdft_set_poisson_precond(self.h, int(kind)), "ofdft_set_poisson_precond")

    def profile(self, kinds=-1):
        """Time launches of the given kinds (bitmask of 1 << K_*; True/-1: all; False/0: none)."""
        mask = -1 if kinds is True else (0 if kinds is False else int(kinds))
        return self._check(self._lib.ofdft_profile(self.h, mask), "ofdft_profile")

    def counters(self) -> Counters:
        c = Counters()
        self._check(self._lib.ofdft_get_counters(self.h, C.byref(c)), "ofdft_get_counters")
        return c

    def reset_counters(self):
        return self._check(self._lib.ofdft_reset_counters(self.h), "ofdft_reset_counters")

    # S2
    def stencil(self, g: Grid, fd_order: int, f, out):
        return self._check(self._lib.ofdft_stencil(self.h, C.byref(g), fd_order, prec_of(f), _ptr(f),
                                                   _ptr(out)), "ofdft_stencil")

    # S1
    def pseudocharge(self, g: Grid, fd_order: int, R, Z, b, sigma=1.0, rc=7.0) -> float:
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        es = C.c_double()
        self._check(self._lib.ofdft_pseudocharge(self.h, C.byref(g), fd_order, _dp(R), _dp(Z), R.shape[0],
                                                 sigma, rc, prec_of(b), _ptr(b), C.byref(es)),
                    "ofdft_pseudocharge")
        return es.value

    def initial_guess(self, g: Grid, R, Z, u, guess_sigma=2.0, guess_cut=8.0, N=None):
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        N = float(Z.sum()) if N is None else float(N)
        self._check(self._lib.ofdft_initial_guess(self.h, C.byref(g), _dp(R), _dp(Z), R.shape[0],
                                                  guess_sigma, guess_cut, N, prec_of(u), _ptr(u)),
                    "ofdft_initial_guess")

    # S3
    def poisson(self, g: Grid, fd_order: int, phi, rho=None, u=None, b=None, tol=1e-10,
                max_it=20000, allow_notconv=False) -> CgStats:
        st = CgStats()
        rc = self._lib.ofdft_poisson(self.h, C.byref(g), fd_order, prec_of(phi), _ptr(rho), _ptr(u),
                                     _ptr(b), _ptr(phi), tol, max_it, C.byref(st))
        self._check(rc, "ofdft_poisson", allow=(ENOTCONV,) if allow_notconv else ())
        return st

    # S3 + S4
    def energy_grad(self, g: Grid, p: Params, u, b, phi, E_self, eta, mu, N, solve_poisson=True,
                    grad=None, s=None, d=None, s_old=None) -> Energy:
        e = Energy()
        self._check(self._lib.ofdft_energy_grad(self.h, C.byref(g), C.byref(p), _ptr(u), _ptr(b),
                                                _ptr(phi), E_self, eta, mu, N, 1 if solve_poisson else 0,
                                                _ptr(grad), _ptr(s), _ptr(d), _ptr(s_old), C.byref(e)),
                    "ofdft_energy_grad")
        return e

    # S9
    def forces(self, g: Grid, fd_order: int, R, Z, phi, sigma=1.0, rc=7.0, variant=FORCE_PAPER):
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        F = np.zeros((R.shape[0], 3))
        self._check(self._lib.ofdft_forces(self.h, C.byref(g), fd_order, _dp(R), _dp(Z), R.shape[0], sigma,
                                           rc, variant, prec_of(phi), _ptr(phi), _dp(F)), "ofdft_forces")
        return F

    # Appendix A, general form
    def overlap_correction(self, g: Grid, fd_order: int, R, Z, sigma=1.0, rc=7.0, sigma_ref=0.4, rc_ref=1.8,
                           tol=1e-12):
        """(E_c, F_c): the repulsive-energy and force corrections for overlapping
        pseudocharges with reference charges b~ (ofdft_overlap_correction)."""
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        E = C.c_double()
        F = np.zeros((R.shape[0], 3))
        self._check(self._lib.ofdft_overlap_correction(self.h, C.byref(g), fd_order, _dp(R), _dp(Z), R.shape[0],
                                                       sigma, rc, sigma_ref, rc_ref, tol, C.byref(E), _dp(F)),
                    "ofdft_overlap_correction")
        return E.value, F

    # S1..S9
    def solve(self, R, Z, h, p: Params, grid: Grid | None = None, u_out=None, phi_out=None,
              want_forces=True, allow_notconv=False):
        """Ground state; returns (energy, forces or None, SolveStats)."""
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        E = C.c_double()
        F = np.zeros((R.shape[0], 3)) if want_forces else None
        st = SolveStats()
        rc = self._lib.ofdft_solve(self.h, C.byref(grid) if grid is not None else None, _dp(R), _dp(Z),
                                   R.shape[0], h, C.byref(p), _ptr(u_out), _ptr(phi_out), C.byref(E),
                                   _dp(F) if F is not None else None, C.byref(st))
        self._check(rc, "ofdft_solve", allow=(ENOTCONV,) if allow_notconv else ())
        return E.value, F, st

    def solve_from(self, R, Z, h, p: Params, grid: Grid, u_in=None, phi_in=None, u_out=None, phi_out=None,
                   want_forces=True, allow_notconv=False):
        """Warm-started ground state (ofdft_solve_from); returns (energy, forces or None, SolveStats)."""
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        E = C.c_double()
        F = np.zeros((R.shape[0], 3)) if want_forces else None
        st = SolveStats()
        rc = self._lib.ofdft_solve_from(self.h, C.byref(grid), _dp(R), _dp(Z), R.shape[0], h, C.byref(p),
                                        _ptr(u_in), _ptr(phi_in), _ptr(u_out), _ptr(phi_out), C.byref(E),
                                        _dp(F) if F is not None else None, C.byref(st))
        self._check(rc, "ofdft_solve_from", allow=(ENOTCONV,) if allow_notconv else ())
        return E.value, F, st

    def relax(self, R, Z, h, p: Params, grid: Grid | None = None, max_steps=50, f_tol=1e-3, max_move=0.05,
              allow_notconv=False):
        """Geometry relaxation (ofdft_relax); returns (R*, energy, forces, RelaxStats)."""
        R = np.array(_host_f64(R).reshape(-1, 3), copy=True)
        Z = _host_f64(Z)
        E = C.c_double()
        F = np.zeros_like(R)
        st = RelaxStats()
        rc = self._lib.ofdft_relax(self.h, C.byref(grid) if grid is not None else None, _dp(R), _dp(Z),
                                   R.shape[0], h, C.byref(p), int(max_steps), float(f_tol), float(max_move),
                                   C.byref(E), _dp(F), C.byref(st))
        self._check(rc, "ofdft_relax", allow=(ENOTCONV,) if allow_notconv else ())
        return R, E.value, F, st


class Batch:
    """A batch of ground-state solves advanced together (ofdft_batch_*)."""

    def __init__(self, ctx: Context, precision: int, hbm_budget_bytes: int):
        self.ctx = ctx
        self.h = C.c_void_p()
        ctx._check(ctx._lib.ofdft_batch_create(ctx.h, precision, int(hbm_budget_bytes), C.byref(self.h)),
                   "ofdft_batch_create")
        self.M = {}
        ctx._batches.add(self)

    def close(self):
        if self.h:
            if self.ctx.h:  # the context frees the batch's device memory only through it
                self.ctx._lib.ofdft_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, R, Z, h, p: Params, grid: Grid | None = None) -> int:
        R, Z = _host_f64(R).reshape(-1, 3), _host_f64(Z)
        rid = C.c_int()
        self.ctx._check(self.ctx._lib.ofdft_batch_submit(self.h, _dp(R), _dp(Z), R.shape[0], h, C.byref(p),
                                                         C.byref(grid) if grid is not None else None,
                                                         C.byref(rid)), "ofdft_batch_submit")
        self.M[rid.value] = R.shape[0]
        return rid.value

    def step(self):
        na, nq = C.c_int(), C.c_int()
        self.ctx._check(self.ctx._lib.ofdft_batch_step(self.h, C.byref(na), C.byref(nq)), "ofdft_batch_step")
        return na.value, nq.value

    def poll(self, rid: int, allow_notconv=False):
        """None while running; (energy, forces, SolveStats) once finished."""
        done = C.c_int()
        E = C.c_double()
        F = np.zeros((self.M[rid], 3))
        st = SolveStats()
        rc = self.ctx._lib.ofdft_batch_poll(self.h, rid, C.byref(done), C.byref(E), _dp(F), C.byref(st))
        if not done.value:
            self.ctx._check(rc, "ofdft_batch_poll")
            return None
        self.ctx._check(rc, "ofdft_batch_poll", allow=(ENOTCONV,) if allow_notconv else ())
        return E.value, F, st

    def run(self):
        self.ctx._check(self.ctx._lib.ofdft_batch_run(self.h), "ofdft_batch_run")

    def info(self) -> dict:
        """Launch statistics: rounds, CG loop graphs captured and replayed, the
        autotuned z-tile depth and its timings (ofdft_batch_info)."""
        st = BatchStats()
        self.ctx._check(self.ctx._lib.ofdft_batch_info(self.h, C.byref(st)), "ofdft_batch_info")
        return st.as_dict()


def batch_bytes(g: Grid, prec: int) -> int:
    return int(lib().ofdft_batch_bytes(C.byref(g), prec))


def mg_plan(g: Grid, prec: int = PREC_MIXED) -> dict:
    """Levels of the multigrid Poisson preconditioner for grid g (host only):
    {"levels": [(n1, n2, n3), ...], "coarse_level": int (-1: plain CG), "bytes": int}."""
    nl, lc = C.c_int(), C.c_int()
    dims = (C.c_int * (3 * 24))()
    nb = C.c_longlong()
    rc = lib().ofdft_mg_plan(C.byref(g), prec, C.byref(nl), C.byref(lc), dims, C.byref(nb))
    if rc != OK:
        raise OfdftError(rc, "ofdft_mg_plan: invalid grid")
    return {"levels": [tuple(dims[3 * l:3 * l + 3]) for l in range(nl.value)], "coarse_level": lc.value,
            "bytes": nb.value}


def workspace_bytes(g: Grid, fd_order: int, prec: int) -> int:
    return int(lib().ofdft_workspace_bytes(C.byref(g), fd_order, prec))


def exported_symbols():
    """Names the header declares (for the load/export check)."""
    return ["ofdft_default_params", "ofdft_create", "ofdft_destroy", "ofdft_last_error",
            "ofdft_grid_for_atoms", "ofdft_stencil", "ofdft_pseudocharge", "ofdft_initial_guess",
            "ofdft_poisson", "ofdft_energy_grad", "ofdft_forces", "ofdft_overlap_correction", "ofdft_solve",
            "ofdft_workspace_bytes", "ofdft_profile", "ofdft_get_counters", "ofdft_reset_counters",
            "ofdft_set_poisson_precond", "ofdft_mg_plan",
            "ofdft_batch_create", "ofdft_batch_destroy", "ofdft_batch_submit", "ofdft_batch_step",
            "ofdft_batch_poll", "ofdft_batch_run", "ofdft_batch_bytes", "ofdft_batch_info"]

