"""Plain FP64 CPU oracle for the spectral Boltzmann collision operator.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the CPU-baseline leg of the benchmark.  The CUDA library and its Python
binding never import it.
"""
from .oracle import Kernel, FastKernel, build, load, gauss_legendre, radial_bhat, num_threads  # noqa: F401
