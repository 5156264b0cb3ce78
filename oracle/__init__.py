"""FP64 CPU oracle for the DGP particle-mesh hot path (Chan & Scoccimarro,
"Large-Scale Structure in Brane-Induced Gravity II. Numerical Simulations").

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method in numpy float64.  It exists to check the
CUDA library, and only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import or run it.  The product path never
calls into it, and it shares no code with the CUDA library: it has its own
FFT (``oracle.fft``), its own background cosmology, its own CIC and its own
relaxation solver.

Modules
-------
fft         mixed-radix Cooley-Tukey FFT (four-step form, DFT-matrix leaves)
background  DGP expansion history and the scalar coefficients (Sec. II)
field       the FFT-relaxation solve for the brane-bending mode and the
            modified Poisson equation for phi (Sec. III.B-C, Eqs. FullDGP1-2)
pm          CIC deposit / force interpolation and the leapfrog step (Sec. III.A)
estimators  power spectrum and bispectrum estimators (Secs. IV, VI)

Every function cites the passage it follows.  Functions without an
independent pin say "parity unpinned" in their docstring.
"""
