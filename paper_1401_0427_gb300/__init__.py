"""GB300-native vectorial lattice Boltzmann schemes for the shallow-water equations.

The hot path (fused collide-and-stream steps of the D1Q3Q2 and D2Q5Q4Q4 schemes of
Dubois, "Simulation of strong nonlinear waves with vectorial lattice Boltzmann
schemes", sections 2 and 3) runs in hand-written CUDA kernels for sm_103a behind the
C ABI declared in ``include/lbm_sw.h``.  ``lbm_sw`` is the thin ctypes binding with
the same entry-point names; it loads ``csrc/_build/liblbm_sw.so`` and raises if the
library is missing: there is no CPU fallback.

``inputs`` holds the seeded synthetic workloads and imports nothing else.
"""

__all__ = ["inputs", "lbm_sw"]
