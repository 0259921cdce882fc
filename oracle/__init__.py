"""FP64 CPU oracle for the SCALE local-energy path (test infrastructure only).

Only the tests, the smoke check and the bench's CPU-baseline leg may import this package.
It shares no code with the CUDA library; see oracle.c for what it computes and where in
the paper each step comes from.
"""
from .oracle import *  # noqa: F401,F403
