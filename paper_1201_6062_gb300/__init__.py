"""GB300-native propagator for the laser-driven hydrogen TDSE in an eigenstate basis.

The hot path (Hamiltonian-vector product fused with RK4 stages or Taylor
terms, norm/populations, the discrete adjoint and the batched variants) runs in
hand-written sm_103a CUDA kernels behind the C ABI declared in
``include/tdse.h``.  ``paper_1201_6062_gb300.tdse`` is the thin ctypes binding
(argument marshalling only).  Importing this package does not load the CUDA
library; ``paper_1201_6062_gb300.tdse`` does, and raises if it is missing.
"""
__all__ = ["inputs"]
