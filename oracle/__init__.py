"""CPU oracle for the CCGPAK complex Krylov solvers.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use it.  The GPU library never imports it.
"""
from .oracle import *  # noqa: F401,F403
