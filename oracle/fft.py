"""The oracle's own discrete Fourier transform (test infrastructure).

The paper transforms every field with FFTs (Sec. III.B, Sec. III.D: fifteen
transforms per relaxation iteration).  The oracle needs a transform that is
checkably the DFT

    X[k] = sum_j x[j] exp(-2 pi i j k / n)      (forward)
    x[j] = (1/n) sum_k X[k] exp(+2 pi i j k / n) (inverse)

so it is written here as the textbook Cooley-Tukey split n = n1 * n2
("four-step" form): n2-strided length-n1 DFTs, a twiddle multiply, length-n2
DFTs and an index transpose.  Lengths <= 32, or lengths with no split, are the
dense DFT matrix applied by a matmul (a library primitive used as one step).
Any length works; the meshes in use are 2^a 3^b.

Pins (tests/test_oracle_fft.py): brute-force O(N^6) DFT on 8^3, 6^3 and 12^3
meshes, and numpy.fft (an independent library) on larger meshes.
"""

import numpy as np

_LEAF = 32


def _dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


def _split(n):
    """Largest divisor n1 <= sqrt(n); returns (n1, n // n1) or None."""
    best = None
    d = 2
    while d * d <= n:
        if n % d == 0:
            best = d
        d += 1
    return None if best is None else (best, n // best)


def _fft_last(x, sign):
    """DFT along the last axis of a C-contiguous complex array."""
    n = x.shape[-1]
    sp = None if n <= _LEAF else _split(n)
    if sp is None:
        # X[..., k] = sum_j x[..., j] W[j, k]
        return x @ _dft_matrix(n, sign)
    n1, n2 = sp
    lead = x.shape[:-1]
    # input index j = n2*j1 + j2  ->  view [j1, j2]
    v = x.reshape(lead + (n1, n2))
    # length-n1 DFTs over j1 (k1 <- j1) for each j2: move j1 last
    v = np.ascontiguousarray(np.swapaxes(v, -1, -2))          # [..., j2, j1]
    v = v @ _dft_matrix(n1, sign)                              # [..., j2, k1]
    # twiddle w_n^{j2 k1}
    j2 = np.arange(n2)[:, None]
    k1 = np.arange(n1)[None, :]
    v = v * np.exp(sign * 2j * np.pi * j2 * k1 / n)
    # length-n2 DFTs over j2 (k2 <- j2) for each k1: move j2 last
    v = np.ascontiguousarray(np.swapaxes(v, -1, -2))          # [..., k1, j2]
    v = _fft_last(v, sign)                                     # [..., k1, k2]
    # output index k = k1 + n1*k2  ->  order [k2, k1]
    v = np.swapaxes(v, -1, -2)
    return np.ascontiguousarray(v).reshape(lead + (n,))


def fft_axis(x, axis, inverse=False):
    """DFT of ``x`` along ``axis`` (unnormalised forward, 1/n inverse)."""
    x = np.asarray(x, dtype=np.complex128)
    v = np.ascontiguousarray(np.moveaxis(x, axis, -1))
    v = _fft_last(v, +1 if inverse else -1)
    if inverse:
        v = v / x.shape[axis]
    return np.moveaxis(v, -1, axis)


def fft3(x):
    """Forward 3D DFT of a (possibly real) N1 x N2 x N3 array, full spectrum."""
    v = np.asarray(x, dtype=np.complex128)
    for ax in range(3):
        v = fft_axis(v, ax)
    return v


def ifft3(X):
    """Inverse 3D DFT (with 1/M), full complex result."""
    v = np.asarray(X, dtype=np.complex128)
    for ax in range(3):
        v = fft_axis(v, ax, inverse=True)
    return v


def ifft3_real(X):
    """Inverse 3D DFT of a Hermitian spectrum; returns the real part."""
    return ifft3(X).real
