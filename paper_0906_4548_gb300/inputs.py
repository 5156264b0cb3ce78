"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

This module holds no arithmetic of the solver or of the particle-mesh step:
it only draws random numbers and shapes them into the initial state that
both sides are fed.  Anything the method computes (the growth rate, E(a),
coefficients) is passed in by the caller.

Recipe (the paper's runs used CMBFAST transfer functions and 2LPT initial
conditions, Sec. III.A; those are replaced by a seeded power law):
  * white noise: counter-based SplitMix64 of (seed, cell index, draw) -> two
    uniforms -> Box-Muller -> unit-variance real white noise w(x) on the mesh;
  * delta_L(k) = W_k sqrt(M P(k) / L^3) with W_k the unnormalised DFT of w,
    P(k) = A k^n_s, so that P = L^3 <|delta_k / M|^2>; k = 0 and every mode with
    a component on the Nyquist index are set to zero;
  * A is fixed so that the ensemble rms of delta_L on the mesh is ``rms``:
    A = rms^2 L^3 / sum_k k^n_s over the retained modes;
  * Zel'dovich particles: one per cell on the lattice q = i d,
    Psi(k) = i k delta_L(k) / k^2, x = q + Psi (wrapped), p = vel_factor Psi,
    where ``vel_factor`` (a^2 E f for the growing mode) comes from the caller.
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z):
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniforms(seed, index, draw):
    """Uniform [0, 1) double for counter (seed, index, draw), draw in {0, 1}."""
    key = splitmix64_mix(np.uint64(seed))
    ctr = np.asarray(index, dtype=np.uint64) * np.uint64(2) + np.uint64(draw) + np.uint64(1)
    with np.errstate(over="ignore"):
        z = splitmix64_mix(key + ctr * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def white_noise(n, seed):
    """Unit-variance Gaussian white noise on an n^3 mesh (Box-Muller)."""
    idx = np.arange(n ** 3, dtype=np.uint64)
    u1 = uniforms(seed, idx, 0)
    u2 = uniforms(seed, idx, 1)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return (r * np.cos(2.0 * np.pi * u2)).reshape(n, n, n)


def _kvec(n, box):
    i = np.arange(n)
    m = np.where(i < n // 2, i, i - n)
    k1 = 2.0 * np.pi * m / box
    keep1 = i != n // 2
    return k1, keep1


def power_law_amplitude(n, box, n_s, rms):
    """A such that the ensemble rms of delta_L on the mesh equals ``rms``."""
    k1, keep1 = _kvec(n, box)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    keep = keep1[:, None, None] & keep1[None, :, None] & keep1[None, None, :]
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    keep &= k > 0
    return rms ** 2 * box ** 3 / float(np.sum(k[keep] ** n_s))


def linear_field_k(n, box, n_s, rms, seed):
    """delta_L(k) on the full n^3 grid (numpy FFT layout) and the amplitude A."""
    A = power_law_amplitude(n, box, n_s, rms)
    Wk = np.fft.fftn(white_noise(n, seed))
    k1, keep1 = _kvec(n, box)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    keep = keep1[:, None, None] & keep1[None, :, None] & keep1[None, None, :] & (k > 0)
    ksafe = np.where(k > 0, k, 1.0)
    amp = np.where(keep, np.sqrt(n ** 3 * A * ksafe ** n_s / box ** 3), 0.0)
    return Wk * amp, A


def linear_field(n, box, n_s, rms, seed):
    """Real-space Gaussian random field delta_L (float64 n^3) and A."""
    dk, A = linear_field_k(n, box, n_s, rms, seed)
    return np.fft.ifftn(dk).real, A


def zeldovich_particles(n, box, n_s, rms, seed, vel_factor):
    """One particle per cell displaced by Zel'dovich from the lattice.

    Returns (pos, mom, A): pos and mom float64 arrays of shape (3, n^3) in
    lattice order (x index slowest), positions wrapped into [0, box)."""
    dk, A = linear_field_k(n, box, n_s, rms, seed)
    pos, mom = _zeldovich(dk, n, box, vel_factor)
    return pos, mom, A


def zeldovich_from_field(delta_l, box, vel_factor):
    """The same map from a real linear field delta_L (n^3): Psi = IFFT(i k / k^2 delta_L(k)),
    the Nyquist component of each k_j dropped; pos = q + Psi (wrapped), mom = vel_factor Psi."""
    n = delta_l.shape[0]
    return _zeldovich(np.fft.fftn(delta_l), n, box, vel_factor)


def _zeldovich(dk, n, box, vel_factor):
    k1, _ = _kvec(n, box)
    k1z = np.where(np.arange(n) == n // 2, 0.0, k1)  # i k_j is odd: drop Nyquist
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2s = np.where(k2 > 0, k2, 1.0)
    grads = np.meshgrid(k1z, k1z, k1z, indexing="ij")
    d = box / n
    q = np.arange(n) * d
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    psi = [np.fft.ifftn(1j * g * dk / k2s).real for g in grads]
    pos = np.stack([(qq + p).reshape(-1) for qq, p in zip((qx, qy, qz), psi)]) % box
    mom = vel_factor * np.stack([p.reshape(-1) for p in psi])
    return pos, mom


def lattice_particles(n, box):
    """Unperturbed lattice q = i d (uniform density), zero momenta."""
    d = box / n
    q = np.arange(n) * d
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    pos = np.stack([qx.reshape(-1), qy.reshape(-1), qz.reshape(-1)])
    return pos, np.zeros_like(pos)
