"""GB300-native finite-volume hydrodynamics update (GenASiS, arXiv:1207.3392).

The compute path lives in the CUDA library ``_lib/libgenasis_hydro.so`` (built by
``paper_1207_3392_gb300.build``); ``paper_1207_3392_gb300.hydro`` is its thin
ctypes binding.  Importing this package loads nothing: the binding loads the
library on first use and raises if it is missing.
"""
__all__ = ["problems", "hydro", "build"]
