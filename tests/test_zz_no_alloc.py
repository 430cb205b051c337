"""The allocation-free Poisson entry point (ofdft_poisson_noalloc).

It serves callers that cannot allocate device memory (an application whose
framework owns every device allocation, or code that must not call cudaMalloc
on a latency-critical path).  Its CG vectors and reduction scratch live in one
fixed file-scope device array (grids of at most 64^3 nodes), shared by every
call.  The test calls it through the C ABI twice in a row and checks each
result against ofdft_poisson, within the Poisson tolerance the other GPU tests
use.  It lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1405_6456_gb300 import build as B
from paper_1405_6456_gb300 import ofdft as F

pytestmark = pytest.mark.gpu


def _noalloc(lib, g, order, rho, phi, tol, max_it, stream):
    st = F.CgStats()
    rc = lib.ofdft_poisson_noalloc(ctypes.byref(g), order, ctypes.c_void_p(rho.data_ptr()),
                                   ctypes.c_void_p(phi.data_ptr()), tol, max_it,
                                   ctypes.c_void_p(stream.cuda_stream), ctypes.byref(st))
    return rc, st


def test_noalloc_poisson_matches_poisson_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    lib = F.lib()
    lib.ofdft_poisson_noalloc.argtypes = [ctypes.POINTER(F.Grid), ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(F.CgStats)]
    ctx = F.Context(0)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(21)
    for call, (dims, order) in enumerate([((40, 36, 30), 12), ((64, 64, 64), 8)]):
        g = F.make_grid(*dims, 0.5)
        rho_h = rng.standard_normal(g.shape)
        rho = torch.as_tensor(rho_h, device="cuda:0")
        phi_ref = torch.zeros(g.shape, dtype=torch.float64, device="cuda:0")
        ctx.poisson(g, order, phi_ref, rho=rho, tol=1e-11)
        phi = torch.zeros_like(phi_ref)
        rc, st = _noalloc(lib, g, order, rho, phi, 1e-11, 20000, stream)
        torch.cuda.synchronize()
        assert rc == F.OK, call
        assert st.rel_residual <= 1e-11
        scale = phi_ref.abs().max().item()
        assert (phi - phi_ref).abs().max().item() <= 1e-9 * scale, call
    # beyond the fixed maximum: a clear error, nothing launched
    g = F.make_grid(65, 64, 64, 0.5)
    big = torch.zeros(g.shape, dtype=torch.float64, device="cuda:0")
    rc, _ = _noalloc(lib, g, 8, big, big.clone(), 1e-9, 10, stream)
    assert rc == F.EINVAL
    ctx.close()
