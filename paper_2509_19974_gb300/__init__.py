"""GB300-native time-difference estimator (arXiv 2509.19974, Algorithm 1).

Quantize two signals with a monotone integer map, correlate them exactly in
integers, take the tie-ruled argmax -- all in hand-written sm_103a kernels
behind the C ABI of ``libtde.so`` (``include/tde.h``).  ``tde`` is the Python
binding; ``synth`` draws the seeded synthetic workloads; ``build`` compiles
the library in-tree.
"""

__all__ = ["tde", "synth", "build"]
