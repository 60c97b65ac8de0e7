"""GB300-native (sm_103a) volume-penalized lattice Boltzmann solver with the
momentum-exchange (MEM) and stress-integration (SIM) force estimators of
Liberge & Beghein (arXiv 2110.00967).

`vplbm` is the binding of the C ABI in include/vplbm.h; importing the package
does not load the CUDA library (that happens on first use, and fails loudly
when the library cannot be built or loaded).
"""
from . import vplbm  # noqa: F401

__all__ = ["vplbm"]
