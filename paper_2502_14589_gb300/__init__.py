"""GB300 (sm_103a) library for the explicit Cahn-Hilliard integrators of arXiv:2502.14589:
EE2 (exponential Euler with residual-time restarted Krylov phi) and LIM (Chebyshev local
iteration), constant and adaptive steps, on periodic 2D/3D grids.

The compute path is libch.so (hand-written CUDA behind the C ABI of include/ch.h); `ch`
is its thin Python binding and `inputs` the seeded synthetic-input generator.
"""
from . import inputs  # noqa: F401
