"""Pins of the oracle's P(k) and bispectrum estimators (Secs. IV, VI)."""
import itertools

import numpy as np

from oracle import background as bg
from oracle import estimators as est
from oracle import field
from oracle.field import KGrid
from paper_0906_4548_gb300 import inputs


def test_pk_parseval_and_mode_counts():
    n, box = 16, 100.0
    d = np.random.default_rng(4).standard_normal((n, n, n))
    k, P, cnt = est.power_spectrum(d, box)
    grid = KGrid(n, box)
    b = np.floor(grid.kmag / (2 * np.pi / box) + 0.5) * np.ones((n, n, n))
    excluded = (b > n // 2)
    dk = np.fft.fftn(d) / n ** 3
    assert cnt.sum() == n ** 3 - 1 - excluded.sum()
    # Parseval: binned power plus modes beyond the last shell = mesh variance
    total = np.sum(P * cnt) / box ** 3 + np.sum(np.abs(dk[excluded]) ** 2)
    assert abs(total - d.var()) < 1e-12 * d.var()


def test_pk_recovers_input_power_law():
    n, box, ns = 64, 200.0, -1.5
    d, A = inputs.linear_field(n, box, ns, 0.5, seed=3)
    k, P, cnt = est.power_spectrum(d, box)
    sel = (cnt > 200) & (np.arange(1, n // 2 + 1) < n // 2 - 1)
    # Gaussian field: relative scatter of a shell estimate is sqrt(2 / cnt)
    z = (P[sel] / (A * k[sel] ** ns) - 1) / np.sqrt(2 / cnt[sel])
    assert np.all(np.abs(z) < 4.5) and abs(np.mean(z)) < 3 / np.sqrt(z.size) + 0.5


def test_bispectrum_matches_brute_force_triangle_average():
    """B = V^2/M^3 <delta_k1 delta_k2 delta_k3> over closed triangles in the shells."""
    n, box = 8, 10.0
    kf = 2 * np.pi / box
    d = np.random.default_rng(8).standard_normal((n, n, n))
    dk = np.fft.fftn(d)
    grid = KGrid(n, box)
    kmag = (grid.kmag * np.ones((n, n, n)))
    k1, k2, th = 1.0 * kf, 2.0 * kf, np.pi / 3
    k3 = np.sqrt(k1 ** 2 + k2 ** 2 + 2 * k1 * k2 * np.cos(th))
    B, Q, P1, P2, P3 = est.bispectrum(d, box, k1, k2, [th])
    idx = list(np.ndindex(n, n, n))
    in1 = [i for i in idx if abs(kmag[i] - k1) < 0.5 * kf]
    in2 = [i for i in idx if abs(kmag[i] - k2) < 0.5 * kf]
    acc, cnt = 0.0, 0
    for i1, i2 in itertools.product(in1, in2):
        i3 = tuple((-np.array(i1) - np.array(i2)) % n)
        if abs(kmag[i3] - k3) < 0.5 * kf:
            acc += (dk[i1] * dk[i2] * dk[i3]).real
            cnt += 1
    assert cnt > 0
    want = box ** 6 / n ** 9 * acc / cnt
    assert abs(B[0] - want) < 1e-10 * abs(want)


def test_brane_spectra_of_a_plane_wave():
    """P_c, P_C and Delta of D = A cos(2 k_f x) from their definitions (Eqs. cdef,
    DGradC): only the +-k modes of shell 2 carry power."""
    n, box, a, A = 16, 80.0, 0.5, 0.7
    x = np.arange(n) * box / n
    D = A * np.cos(2 * 2 * np.pi / box * x)[:, None, None] * np.ones((n, n, n))
    k, Pc, PC, Dl, cnt = est.brane_spectra(D, a, box, 0.27, 1.0)
    coef = bg.coefficients(a, 0.27, 1.0)
    kk = 2 * 2 * np.pi / box
    kbar = bg.C_H * kk / (a * coef["E"])
    fac = coef["alpha"] * coef["eta"] / (3 * (coef["eta"] - 1))
    # |D_k / M|^2 = A^2 / 4 at each of the two modes
    assert np.isclose(Pc[1], box ** 3 * fac ** 2 * A ** 2 / 2 / cnt[1], rtol=1e-12)
    assert np.isclose(PC[1], box ** 3 * (A / kbar ** 2) ** 2 / 2 / cnt[1], rtol=1e-12)
    assert np.isclose(Dl[1], 4 * np.pi * k[1] ** 5 * PC[1], rtol=1e-12)
    assert np.all(Pc[np.arange(len(Pc)) != 1] < 1e-25)


def test_brane_spectrum_linear_theory_ratio():
    """In linear theory c_k / delta_k = alpha (1 - beta/kbar) / (alpha - c2/kbar)
    (Sec. IV: P_c / P_m -> 1 once kbar >> 1), here for a plane wave delta."""
    from oracle.fft import fft3, ifft3_real
    n, box, a = 16, 60.0, 0.6
    grid = KGrid(n, box)
    coef = bg.coefficients(a, 0.27, 1.0)
    kk = 3 * 2 * np.pi / box
    x = np.arange(n) * box / n
    d = 0.1 * np.cos(kk * x)[None, :, None] * np.ones((n, n, n))
    D = ifft3_real(field.linear_D_spectrum(field.source_spectrum(fft3(d), grid, coef), grid, coef))
    k, Pc, PC, Dl, cnt = est.brane_spectra(D, a, box, 0.27, 1.0)
    _, Pd, _ = est.power_spectrum(d, box)
    kbar = bg.C_H * kk / (a * coef["E"])
    ratio = (coef["alpha"] * (1 - coef["beta"] / kbar) / (coef["alpha"] - coef["c2"] / kbar)) ** 2
    assert abs(Pc[2] / Pd[2] - ratio) < 1e-12 * ratio
