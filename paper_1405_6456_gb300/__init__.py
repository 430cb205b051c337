"""GB300 (sm_103a) library for the Augmented Lagrangian formulation of
orbital-free DFT (Suryanarayana & Phanish, arXiv:1405.6456).

`paper_1405_6456_gb300.ofdft` is the thin Python binding of the C ABI declared in
include/ofdft.h (argument marshalling only; every step runs in the CUDA library).
`paper_1405_6456_gb300.workloads` holds the seeded synthetic cluster generators.
"""
import importlib

__all__ = ["ofdft", "workloads", "build", "serving"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
