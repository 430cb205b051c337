"""FP64 CPU oracle for the Augmented Lagrangian OF-DFT method (arXiv:1405.6456).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  The product path
(`paper_1405_6456_gb300`) never imports it, and the two share no code: the C
source here (`ofdft_oracle.c`) is compiled with gcc into its own library.

Every function follows a passage of the paper; see the C source for the
citation of each step and the list of readings taken where the paper is silent.
Functions with no independent pin are marked "parity unpinned" in their
docstring (none at present).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ofdft_oracle.c")
_HDR = os.path.join(_HERE, "ofdft_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TF, VW, XC, ES, ALL = 1, 2, 4, 8, 15
AL, PENALTY, LM = 0, 1, 2


class Grid(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("h", C.c_double),
                ("origin", C.c_double * 3)]

    @property
    def shape(self):
        """numpy shape (n3, n2, n1) of an x-fastest grid array."""
        return (self.n3, self.n2, self.n1)

    @property
    def size(self):
        return self.n1 * self.n2 * self.n3

    def __repr__(self):
        return (f"Grid(n=({self.n1},{self.n2},{self.n3}), h={self.h}, "
                f"origin=({self.origin[0]:.4f},{self.origin[1]:.4f},{self.origin[2]:.4f}))")


class Params(C.Structure):
    _fields_ = [("fd_n", C.c_int), ("terms", C.c_int), ("lam", C.c_double),
                ("eta0", C.c_double), ("mu0", C.c_double), ("kappa", C.c_double),
                ("method", C.c_int), ("tol_E", C.c_double), ("tol_inner", C.c_double),
                ("tol_poisson", C.c_double), ("max_outer", C.c_int), ("max_nlcg", C.c_int),
                ("max_cg", C.c_int), ("max_secant", C.c_int), ("sigma0", C.c_double),
                ("eps_secant", C.c_double), ("restart_every", C.c_int), ("sigma", C.c_double),
                ("rc", C.c_double), ("guess_sigma", C.c_double), ("guess_cut", C.c_double),
                ("ezz_correction", C.c_int), ("trial_max_rel", C.c_double), ("max_backtrack", C.c_int),
                ("precond_rank1", C.c_int)]


class Energy(C.Structure):
    _fields_ = [("L", C.c_double), ("E", C.c_double), ("E_tf", C.c_double),
                ("E_vw", C.c_double), ("E_xc", C.c_double), ("E_es", C.c_double),
                ("E_self", C.c_double), ("E_zz_corr", C.c_double), ("C", C.c_double),
                ("gnorm2", C.c_double), ("rs", C.c_double), ("rs_pc", C.c_double),
                ("cg_iters", C.c_int), ("cg_relres", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(C.Structure):
    _fields_ = [("E", C.c_double), ("eta", C.c_double), ("C", C.c_double),
                ("parts", Energy), ("outer_iters", C.c_int), ("nlcg_iters", C.c_int),
                ("grad_evals", C.c_int), ("energy_evals", C.c_int), ("cg_iters", C.c_int),
                ("stencil_apps", C.c_longlong), ("converged", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (idempotent)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR),
                                              os.path.getmtime(__file__)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                   _SRC, "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        L.orc_default_params.argtypes = [C.POINTER(Params)]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_lap_weights.argtypes = [C.c_int, C.c_double, dp]
        L.orc_grad_weights.argtypes = [C.c_int, C.c_double, dp]
        L.orc_laplacian.argtypes = [C.POINTER(Grid), C.c_int, dp, dp]
        L.orc_xc.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_grid_for_atoms.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_int,
                                         C.POINTER(Grid)]
        L.orc_gauss_potential.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_gauss_potential.restype = C.c_double
        L.orc_pseudocharge.argtypes = [C.POINTER(Grid), C.c_int, dp, dp, C.c_int, C.c_double,
                                       C.c_double, dp, C.POINTER(C.c_double)]
        L.orc_initial_guess.argtypes = [C.POINTER(Grid), dp, dp, C.c_int, C.c_double,
                                        C.c_double, C.c_double, dp]
        L.orc_poisson.argtypes = [C.POINTER(Grid), C.c_int, dp, dp, C.c_double, C.c_int,
                                  C.POINTER(C.c_double)]
        L.orc_functional.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, dp, dp, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                     C.POINTER(Energy)]
        L.orc_energy_grad.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, dp, dp, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                      C.POINTER(Energy)]
        L.orc_solve.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, dp, C.c_int, dp, dp, dp,
                                C.POINTER(Result)]
        L.orc_forces.argtypes = [C.POINTER(Grid), C.c_int, dp, dp, C.c_int, C.c_double,
                                 C.c_double, dp, C.c_int, dp]
        L.orc_ezz_correction.argtypes = [dp, dp, C.c_int, C.c_double, C.c_void_p]
        L.orc_ezz_correction.restype = C.c_double
        # one thread unless a caller asks for more (set_threads): the tests run
        # many small grids, where threads only add overhead
        L.orc_set_threads(1)
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads of the grid-sized loops (sums are independent of it)."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    """Threads the grid-sized loops use."""
    return int(lib().orc_get_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "lambda":
            k = "lam"
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def lap_weights(n: int, h: float) -> np.ndarray:
    """w_0..w_n of Sec. 4, Eq. FD:Laplacian (centre coefficient is 6 w_0)."""
    w = np.zeros(n + 1)
    if lib().orc_lap_weights(n, h, w) != 0:
        raise ValueError("bad stencil radius or spacing")
    return w


def grad_weights(n: int, h: float) -> np.ndarray:
    """w~_0..w~_n of Sec. 4 (w~_0 = 0)."""
    w = np.zeros(n + 1)
    if lib().orc_grad_weights(n, h, w) != 0:
        raise ValueError("bad stencil radius or spacing")
    return w


def make_grid(n1, n2, n3, h, origin=(0.0, 0.0, 0.0)) -> Grid:
    g = Grid()
    g.n1, g.n2, g.n3, g.h = n1, n2, n3, h
    for d in range(3):
        g.origin[d] = origin[d]
    return g


def grid_for_atoms(R, h, vacuum, round_to=16) -> Grid:
    g = Grid()
    R = _f64(R)
    if lib().orc_grid_for_atoms(R, R.shape[0], h, vacuum, round_to, C.byref(g)) != 0:
        raise ValueError("bad grid request")
    return g


def laplacian(g: Grid, n: int, f: np.ndarray) -> np.ndarray:
    """L_h f with zero Dirichlet values (Sec. 4); f has shape g.shape."""
    f = _f64(f).reshape(-1)
    out = np.zeros_like(f)
    lib().orc_laplacian(C.byref(g), n, f, out)
    return out.reshape(g.shape)


def xc(u: float):
    """(eps_xc, V_xc) at u = sqrt(rho) (Sec. 2 and Sec. 3)."""
    e, v = C.c_double(), C.c_double()
    lib().orc_xc(float(u), C.byref(e), C.byref(v))
    return e.value, v.value


def gauss_potential(Z, sigma, r) -> float:
    return lib().orc_gauss_potential(Z, sigma, r)


def pseudocharge(g: Grid, n: int, R, Z, sigma=1.0, rc=7.0):
    """(b, E_self): b = sum_J b_J (Sec. 4), E_self = (1/2) sum_J h^3 sum b_J V_J."""
    R, Z = _f64(R), _f64(Z)
    b = np.zeros(g.size)
    es = C.c_double()
    lib().orc_pseudocharge(C.byref(g), n, R, Z, R.shape[0], sigma, rc, b, C.byref(es))
    return b.reshape(g.shape), es.value


def initial_guess(g: Grid, R, Z, gsigma=2.0, gcut=8.0, N=None) -> np.ndarray:
    R, Z = _f64(R), _f64(Z)
    N = float(np.sum(Z)) if N is None else float(N)
    u = np.zeros(g.size)
    lib().orc_initial_guess(C.byref(g), R, Z, R.shape[0], gsigma, gcut, N, u)
    return u.reshape(g.shape)


def poisson(g: Grid, n: int, rho, phi0=None, tol=1e-11, max_it=20000):
    """Solve (-L_h) phi = 4 pi rho by CG from phi0 (Sec. 4). Returns (phi, iters, relres)."""
    rho = _f64(rho).reshape(-1)
    phi = np.zeros(g.size) if phi0 is None else _f64(phi0).reshape(-1).copy()
    rel = C.c_double()
    it = lib().orc_poisson(C.byref(g), n, rho, phi, tol, max_it, C.byref(rel))
    return phi.reshape(g.shape), it, rel.value


def functional(g: Grid, p: Params, u, b, phi, E_self, eta, mu, N, want_grad=True):
    """Energy parts, gradient G and Jacobi-preconditioned s = -G/M at fixed phi."""
    u, b, phi = (_f64(a).reshape(-1) for a in (u, b, phi))
    G = np.zeros(g.size) if want_grad else None
    s = np.zeros(g.size) if want_grad else None
    e = Energy()
    lib().orc_functional(C.byref(g), C.byref(p), u, b, phi, E_self, eta, mu, N, _ptr(G), _ptr(s),
                         C.byref(e))
    if want_grad:
        return e, G.reshape(g.shape), s.reshape(g.shape)
    return e, None, None


def energy_grad(g: Grid, p: Params, u, b, phi, E_self, eta, mu, N, ezz=0.0):
    """Poisson solve (warm start from phi, updated in place) + functional."""
    u, b = _f64(u).reshape(-1), _f64(b).reshape(-1)
    phi_w = _f64(phi).reshape(-1).copy()
    G = np.zeros(g.size)
    s = np.zeros(g.size)
    e = Energy()
    e.E_zz_corr = ezz
    lib().orc_energy_grad(C.byref(g), C.byref(p), u, b, phi_w, E_self, eta, mu, N, _ptr(G),
                          _ptr(s), C.byref(e))
    return e, G.reshape(g.shape), s.reshape(g.shape), phi_w.reshape(g.shape)


def solve(g: Grid, p: Params, R, Z, u0=None):
    """Ground state (AL / penalty / LM per p.method). Returns (Result, u, phi, b)."""
    R, Z = _f64(R), _f64(Z)
    u = np.zeros(g.size) if u0 is None else _f64(u0).reshape(-1).copy()
    phi = np.zeros(g.size)
    b = np.zeros(g.size)
    res = Result()
    lib().orc_solve(C.byref(g), C.byref(p), R, Z, R.shape[0], u, phi, b, C.byref(res))
    return res, u.reshape(g.shape), phi.reshape(g.shape), b.reshape(g.shape)


def forces(g: Grid, n: int, R, Z, phi, sigma=1.0, rc=7.0, exact=False) -> np.ndarray:
    """Forces of Eq. Force:Nuclei (paper FD-gradient form, or the exact derivative)."""
    R, Z = _f64(R), _f64(Z)
    F = np.zeros(R.shape[0] * 3)
    lib().orc_forces(C.byref(g), n, R, Z, R.shape[0], sigma, rc, _f64(phi).reshape(-1),
                     1 if exact else 0, F)
    return F.reshape(-1, 3)


def ezz_correction(R, Z, sigma=1.0):
    """(E_c, F_c) of the Gaussian-overlap repulsion correction (Appendix A)."""
    R, Z = _f64(R), _f64(Z)
    F = np.zeros(R.shape[0] * 3)
    E = lib().orc_ezz_correction(R, Z, R.shape[0], sigma, _ptr(F))
    return E, F.reshape(-1, 3)


def overlap_correction(g: Grid, n: int, R, Z, sigma=1.0, rc=7.0, sigma_ref=0.4, rc_ref=1.8, tol=1e-12):
    """(E_c, F_c) of Appendix A in its general form, on the grid: reference
    pseudocharges b~_J (Gaussian nuclei of width sigma_ref cut at rc_ref, whose
    balls must not overlap) next to the pseudocharges b_J of the method;
    V and V~ from (-1/4 pi) L_h V = b and (-1/4 pi) L_h V~ = b~ (so V_c = V~ - V
    solves (-1/4 pi) L_h V_c = b~ - b); Eq. RepulsiveCorrection2:
        E_c = 1/2 h^3 sum (b~ + b) V_c + E_self(b) - E_self(b~),
    E_self the self energies 1/2 h^3 sum_J sum b_J V_J of pseudocharge(); and the
    force correction -dE_c/dR_J,
        f_J = h^3 sum grad b~_J (V~ - V~_J) - h^3 sum grad b_J (V - V_J),
    each the paper-form force expression of forces() at the given potential."""
    R, Z = _f64(R), _f64(Z)
    b, es = pseudocharge(g, n, R, Z, sigma, rc)
    bt, est = pseudocharge(g, n, R, Z, sigma_ref, rc_ref)
    V, _, _ = poisson(g, n, b, tol=tol)
    Vt, _, _ = poisson(g, n, bt, tol=tol)
    h3 = g.h ** 3
    E = 0.5 * h3 * float(np.sum((bt + b) * (Vt - V))) + es - est
    F = forces(g, n, R, Z, Vt, sigma_ref, rc_ref) - forces(g, n, R, Z, V, sigma, rc)
    return E, F
