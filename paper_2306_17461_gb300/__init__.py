"""GB300-native exact edit distance (Landau-Vishkin BFS, Algorithm 1 of
"Efficient Parallel Output-Sensitive Edit Distance").

The compute path is the CUDA library libedgb300.so (include/ed.h); this
package holds its ctypes binding (``binding``), its build step (``build``)
and the seeded workload generators (``workloads``).
"""
from . import binding  # noqa: F401
from .binding import Context, EdError  # noqa: F401
