"""GB300-native DGP particle-mesh hot path (Chan & Scoccimarro, brane-induced
gravity N-body with FFT-relaxation).

The compute path is the CUDA shared library built from ``csrc/`` and declared
in ``include/dgp.h``; ``paper_0906_4548_gb300.dgp`` is its thin ctypes binding.
Nothing is imported eagerly so that ``paper_0906_4548_gb300.inputs`` (the
seeded input generator) can be used without the library.
"""
