"""Pins of the oracle's P(k) and bispectrum estimators (Secs. IV, VI)."""
import itertools

import numpy as np

from oracle import estimators as est
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
