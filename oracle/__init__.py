"""Test infrastructure: the sequential CPU oracle for the global Curveball
super step (Def. "Undirected Global Trade", Section 3.3).

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The CUDA library never does.
"""
from .oracle import Oracle, build_oracle, philox4x32_10, successors, uniform_pair  # noqa: F401
