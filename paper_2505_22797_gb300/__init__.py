"""GB300-native equilibrium-model (Langevin) MPI reconstruction.

The compute path is the C-ABI library ``libmpi_recon.so`` (hand-written CUDA
for sm_103a, declared in ``include/mpi_recon.h``).  ``paper_2505_22797_gb300.api``
is a thin ctypes binding with the same entry-point names; importing this
package does not load the library, the first call does, and it raises if the
library is missing.
"""
import importlib

__all__ = ["api", "synthetic"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
