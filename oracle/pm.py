"""Particle-mesh layer of the oracle: CIC deposit, force interpolation, KDK.

Test infrastructure: see ``oracle/__init__.py``.

Sec. III.A.  Mesh: N^3 points at x = i d, d = box / N, periodic.  CIC window
W(x) = 1 - |x|/d for |x| < d (Eq. CIC gives rho_grid as the convolution of
W(x)W(y)W(z) with the particles); forces are interpolated back with the same
window.  Particles carry x (comoving, Mpc/h) and p = a^2 dx/dt (code units),
so the equations of motion dx/dt = u, du/dt = -2 H u - grad(phi)/a^2 become
    dp/dlna = -grad(phi) / E,    dx/dlna = p / (a^2 E).
The time step is uniform in ln a and second-order leapfrog; the oracle takes
the kick-drift-kick form with one force evaluation per step (the paper names
only "second-order leapfrog"), and the kick / drift factors are the exact
integrals of 1/E and 1/(a^2 E) over the step (8-point Gauss-Legendre).
"""

import math

import numpy as np

from . import background as bg
from . import field


def _cic_cells(pos, n, box):
    """Lower grid index and fractional offset along each axis (x = i d)."""
    d = box / n
    out = []
    for ax in range(3):
        u = pos[ax] / d
        i = np.floor(u)
        f = u - i
        i = i.astype(np.int64) % n
        out.append((i, f))
    return out


def cic_deposit(pos, n, box, mass=None):
    """rho_grid(i) = sum_p W(x_i - x_p) W(y_i - y_p) W(z_i - z_p)  (Eq. CIC).

    pos: (3, Np) float64 positions in [0, box) (wrapped here anyway).
    Returns the N^3 particle count per grid point (mass 1 per particle)."""
    pos = np.asarray(pos, dtype=np.float64)
    m = np.ones(pos.shape[1]) if mass is None else np.asarray(mass, float)
    (ix, fx), (iy, fy), (iz, fz) = _cic_cells(pos, n, box)
    rho = np.zeros(n * n * n)
    for dx in (0, 1):
        wx = fx if dx else 1.0 - fx
        jx = (ix + dx) % n
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            jy = (iy + dy) % n
            for dz in (0, 1):
                wz = fz if dz else 1.0 - fz
                jz = (iz + dz) % n
                rho += np.bincount((jx * n + jy) * n + jz, weights=m * wx * wy * wz,
                                   minlength=n ** 3)
    return rho.reshape(n, n, n)


def cell_index(pos, n, box):
    """Cell of the lower CIC corner of each particle, (ix n + iy) n + iz with
    i = floor(x / d) mod n per axis (the point that receives weight
    (1 - fx)(1 - fy)(1 - fz) in Eq. CIC).  int64 array of length Np."""
    (ix, _), (iy, _), (iz, _) = _cic_cells(np.asarray(pos, dtype=np.float64), n, box)
    return (ix * n + iy) * n + iz


def cell_sort(pos, n, box):
    """Counting sort of particles by cell_index: (order, cell_start) with
    order a stable permutation putting the keys in nondecreasing order and
    cell_start[c] = number of particles with key < c, for c = 0 .. n^3."""
    key = cell_index(pos, n, box)
    counts = np.bincount(key, minlength=n ** 3)
    start = np.zeros(n ** 3 + 1, dtype=np.int64)
    start[1:] = np.cumsum(counts)
    order = np.empty(key.size, dtype=np.int64)
    cursor = start[:-1].copy()
    for p in range(key.size):  # scatter in input order: stable
        order[cursor[key[p]]] = p
        cursor[key[p]] += 1
    return order, start


def density_contrast(rho):
    """delta = rho / rho_bar - 1 with rho_bar the mean of the mesh (Sec. III.A)."""
    return rho / float(np.mean(rho)) - 1.0


def cic_interpolate(field_xyz, pos, box):
    """Value of a mesh field at the particles with the same CIC window (Sec. III.A)."""
    n = field_xyz.shape[0]
    (ix, fx), (iy, fy), (iz, fz) = _cic_cells(np.asarray(pos, float), n, box)
    flat = field_xyz.reshape(-1)
    out = np.zeros(ix.shape[0])
    for dx in (0, 1):
        wx = fx if dx else 1.0 - fx
        jx = (ix + dx) % n
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            jy = (iy + dy) % n
            for dz in (0, 1):
                wz = fz if dz else 1.0 - fz
                jz = (iz + dz) % n
                out += wx * wy * wz * flat[(jx * n + jy) * n + jz]
    return out


class PMState:
    """Particle state of the oracle run plus the carried solver state."""

    def __init__(self, pos, mom, a, n, box, omega_m0, rc_H0, w=1.0 / 3.0, tol=1e-12,
                 max_iter=500, gravity="nl", local_only=False, a_nonlinear=0.0):
        self.pos = np.array(pos, dtype=np.float64) % box
        self.mom = np.array(mom, dtype=np.float64)
        self.a = float(a)
        self.n, self.box = n, box
        self.omega_m0, self.rc_H0 = omega_m0, rc_H0
        self.w, self.tol, self.max_iter = w, tol, max_iter
        self.gravity, self.local_only = gravity, local_only
        # Sec. III.D: the linearised DGP equation before a_nonlinear, the full one after
        self.a_nonlinear = a_nonlinear
        self.D = None          # warm start: last accepted nonlinear solution
        self.g_part = None     # force at the particles at self.a
        self.solves = []       # info of each field solve

    def forces_at_particles(self):
        """Deposit -> delta -> field solve -> g = -grad(phi) on the mesh -> CIC gather."""
        delta = density_contrast(cic_deposit(self.pos, self.n, self.box))
        gravity = "ldgp" if (self.gravity == "nl" and self.a < self.a_nonlinear) else self.gravity
        _, g, D, info = field.solve_phi(delta, self.a, self.box, self.omega_m0, self.rc_H0,
                                        self.w, self.tol, self.max_iter, self.D,
                                        self.local_only, gravity)
        if D is not None:
            self.D = D
        self.solves.append(dict(a=self.a, iters=info.get("iters", 0),
                                norm_res=info.get("norm_res", 0.0),
                                converged=info.get("converged", True)))
        return np.stack([cic_interpolate(g[i], self.pos, self.box) for i in range(3)])

    def step(self, da):
        """One KDK step a -> a + da, uniform in ln a (Sec. III.A)."""
        a0, a1 = self.a, self.a + da
        ah = math.exp(0.5 * (math.log(a0) + math.log(a1)))
        if self.g_part is None:
            self.g_part = self.forces_at_particles()
        self.mom += bg.kick_factor(a0, ah, self.omega_m0, self.rc_H0) * self.g_part
        self.pos = (self.pos + bg.drift_factor(a0, a1, self.omega_m0, self.rc_H0) * self.mom) \
            % self.box
        self.a = a1
        self.g_part = self.forces_at_particles()
        self.mom += bg.kick_factor(ah, a1, self.omega_m0, self.rc_H0) * self.g_part


def run(pos, mom, a_start, a_end, nsteps, n, box, omega_m0, rc_H0, **kw):
    """nsteps KDK steps uniform in ln a from a_start to a_end; returns the state."""
    st = PMState(pos, mom, a_start, n, box, omega_m0, rc_H0, **kw)
    dlna = (math.log(a_end) - math.log(a_start)) / nsteps
    for i in range(nsteps):
        a_next = a_start * math.exp((i + 1) * dlna)
        st.step(a_next - st.a)
    return st
