"""FP64 CPU oracle for the boundary-integral JFNK scheme (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  The product path never does.  See bfs_oracle.c for the paper
passages each function follows and linear_fft.py for the exact linear solution.
"""
from .oracle import *  # noqa: F401,F403
