"""Brute-force CPU oracle (test infrastructure only; see oracle.py)."""
from .oracle import (build, default_threads, median2d, median2d_numpy, median3d,  # noqa: F401
                     median3d_numpy, points)
