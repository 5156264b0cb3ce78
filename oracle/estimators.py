"""Power spectrum and bispectrum estimators of the oracle.

Test infrastructure: see ``oracle/__init__.py``.

Sec. IV: P(k) of the mesh density contrast.  Convention (the paper states
none): P(k) = L^3 < |delta_k / M|^2 > over shells of width k_f = 2 pi / L
centred on n k_f, n = 1 .. N/2 (a mode belongs to shell round(|k| / k_f));
no CIC deconvolution and no shot-noise subtraction.  Every mode of the full
N^3 grid except k = 0 counts once.

Sec. VI: reduced bispectrum Q_123 = B_123 / (P1 P2 + P2 P3 + P3 P1) (Eq. Qdef).
The paper does not say how B is estimated; the oracle uses the FFT
shell-filter estimator.  With <delta(k1) delta(k2) delta(k3)> = V B for
closed triangles and delta(k) = (V/M) delta_k, the average of
delta_k1 delta_k2 delta_k3 over the closed triangles with k_i in shell S_i
(|k| within dk/2 of k_i) gives
    B(k1,k2,k3) = V^2 / M^3 * sum_x d1 d2 d3 / sum_x I1 I2 I3,
d_i = IFFT(delta_k on S_i), I_i = IFFT(1 on S_i): both sums are M^-2 times
the sums over closed triangles, so their ratio is the triangle average.  Pinned against that
average taken by brute force over the closed triangles of an 8^3 field
(tests/test_oracle_estimators.py).
"""

import numpy as np

from . import background as bg
from .fft import fft3, ifft3_real
from .field import KGrid


def power_spectrum(delta, box, nbins=None):
    """(k_mean, P, n_modes) per shell n = 1..nbins (default N/2)."""
    n = delta.shape[0]
    m = n ** 3
    nb = n // 2 if nbins is None else nbins
    grid = KGrid(n, box)
    kf = 2.0 * np.pi / box
    dk = fft3(delta)
    p = box ** 3 * np.abs(dk / m) ** 2
    b = np.floor(grid.kmag / kf + 0.5).astype(np.int64) * np.ones((n, n, n), np.int64)
    sel = (b >= 1) & (b <= nb)
    bs = b[sel] - 1
    cnt = np.bincount(bs, minlength=nb)
    ks = np.bincount(bs, weights=(grid.kmag * np.ones((n, n, n)))[sel], minlength=nb)
    ps = np.bincount(bs, weights=p[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ks / cnt, ps / cnt, cnt


def brane_spectra(D, a, box, omega_m0, rc_H0, nbins=None):
    """Spectra of the brane-bending mode from D = lapbar^2 C (Sec. IV):
    P_c of the normalised mode c = alpha eta / (3 (eta - 1)) D (Eq. cdef),
    P_C of C itself, C(k) = -D(k) / kbar^2 with kbar = C_H |k| / (a E), and the
    dimensionless spectrum of g_4i = grad_i C, Delta(k) = 4 pi k^5 P_C(k)
    (Eq. DGradC, k the shell's mean |k| in h/Mpc, C dimensionless).  Shells and
    normalisation as power_spectrum.  Returns (k_mean, P_c, P_C, Delta, n_modes)."""
    n = D.shape[0]
    m = n ** 3
    nb = n // 2 if nbins is None else nbins
    coef = bg.coefficients(a, omega_m0, rc_H0)
    grid = KGrid(n, box)
    kf = 2.0 * np.pi / box
    Dk = fft3(D)
    kbar = bg.C_H * np.where(grid.zero, 1.0, grid.kmag) / (a * coef["E"])
    fac_c = coef["alpha"] * coef["eta"] / (3.0 * (coef["eta"] - 1.0))
    pc = box ** 3 * np.abs(fac_c * Dk / m) ** 2
    pC = box ** 3 * np.abs(Dk / kbar ** 2 / m) ** 2
    b = np.floor(grid.kmag / kf + 0.5).astype(np.int64) * np.ones((n, n, n), np.int64)
    sel = (b >= 1) & (b <= nb)
    bs = b[sel] - 1
    cnt = np.bincount(bs, minlength=nb)
    ks = np.bincount(bs, weights=(grid.kmag * np.ones((n, n, n)))[sel], minlength=nb)
    sc = np.bincount(bs, weights=pc[sel], minlength=nb)
    sC = np.bincount(bs, weights=pC[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = ks / cnt
        PC = sC / cnt
        return kmean, sc / cnt, PC, 4.0 * np.pi * kmean ** 5 * PC, cnt


def _shell(grid, k, dk):
    return (np.abs(grid.kmag - k) < 0.5 * dk).astype(np.float64)


def bispectrum(delta, box, k1, k2, thetas, dk=None):
    """B and Q for triangles (k1, k2, theta), k3 = |k1 + k2| with
    k3^2 = k1^2 + k2^2 + 2 k1 k2 cos(theta) (theta is the angle between k1
    and k2, Sec. VI, Fig. 10).  Returns (B, Q, P1, P2, P3) arrays."""
    n = delta.shape[0]
    m = n ** 3
    grid = KGrid(n, box)
    dk = 2.0 * np.pi / box if dk is None else dk
    d = fft3(delta)
    d[grid.zero] = 0.0

    def filt(k):
        sh = _shell(grid, k, dk)
        return ifft3_real(d * sh), ifft3_real(sh.astype(complex)), sh

    def pk(sh):
        return box ** 3 * float(np.sum(np.abs(d / m) ** 2 * sh)) / float(np.sum(sh))

    d1, i1, s1 = filt(k1)
    d2, i2, s2 = filt(k2)
    P1, P2 = pk(s1), pk(s2)
    B, Q, P3s = [], [], []
    for th in thetas:
        k3 = float(np.sqrt(k1 * k1 + k2 * k2 + 2 * k1 * k2 * np.cos(th)))
        d3, i3, s3 = filt(k3)
        P3 = pk(s3)
        ntri = float(np.sum(i1 * i2 * i3))
        b = box ** 6 / m ** 3 * float(np.sum(d1 * d2 * d3)) / ntri
        B.append(b)
        Q.append(b / (P1 * P2 + P2 * P3 + P3 * P1))
        P3s.append(P3)
    return np.array(B), np.array(Q), P1, P2, np.array(P3s)
