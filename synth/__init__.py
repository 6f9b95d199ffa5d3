"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds no arithmetic of randUTV itself.  It provides
  * the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw,
    "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller
    map that turn a seed into the Gaussian matrices G the method draws
    (randUTV Fig. 4, the ``randn`` of each randomized step), and
  * test matrices A = Q1 diag(sigma) Q2^T with Haar-distributed Q1, Q2 and a
    prescribed spectrum (the construction of Section 6.2, "Matrix 1").
"""
from .philox import philox4x32_10, PHILOX_M0, PHILOX_M1, PHILOX_W0, PHILOX_W1
from .gauss import step_gaussian, step_gaussian_f32, gaussian_stream, stream_layout, uniform52, uniform23
from .matrices import make_matrix, spectrum, haar_orthogonal
from . import batch

__all__ = [
    "philox4x32_10", "PHILOX_M0", "PHILOX_M1", "PHILOX_W0", "PHILOX_W1",
    "step_gaussian", "step_gaussian_f32", "gaussian_stream", "stream_layout", "uniform52", "uniform23", "batch",
    "make_matrix", "spectrum", "haar_orthogonal",
]
