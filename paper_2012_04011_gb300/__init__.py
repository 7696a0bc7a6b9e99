"""GB300-native (sm_103a) time stepping of the 4D Hamilton-Jacobi reachability
PDE for the car of arxiv 2012.04011, behind the C-ABI library ``libhj``.

``scenes`` builds seeded inputs (grids, obstacles, V0).  The CUDA binding is
imported lazily so that input generation works on machines without the
built library.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes"]
