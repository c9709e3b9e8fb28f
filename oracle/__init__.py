"""CPU oracle for the WRI augmented-system hot path (test infrastructure only).

Plain, slow, complex128 numpy/scipy restatement of what the method computes,
written from the paper (arXiv 2410.18429, "GPU Accelerated 3D P-wave Source Free
Adaptive Wavefield Reconstruction Inversion").  It is imported only by the test
suite, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``; the product path never calls it and shares no code with it.

Pins (each function is checked against something other than itself in
``tests/test_oracle_*.py``): dense least squares, the textbook interior stencil,
symmetry/adjoint identities, the free-space Green's function, the lambda -> 0 and
lambda -> infinity limits, the data-consistency invariant, the joint (u, alpha)
block solve and central finite differences of the reduced objective.
"""
from .wri_oracle import *  # noqa: F401,F403
