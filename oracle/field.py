"""FFT-relaxation solve for the brane-bending mode and phi (oracle).

Test infrastructure: see ``oracle/__init__.py``.

Notation (Sec. II):  lapbar = lap / (a H),  kbar = c k / (a H) = C_H |k| / (a E).
The unknown is D = lapbar C (the paper solves Eq. FullDGP2 for it, Sec. III.B).
In Fourier space (Sec. III.B: nabla_ij C(k) = -k_i k_j C(k)) every other field
the equations need is a real multiplier on D(k):
    H_ij = lapbar_ij C  ->  (k_i k_j / k^2) D(k)
    N    = sqrt(-lapbar) C  ->  kbar C(k) = -D(k) / kbar
    S    = s (1 - beta lapbar^-1) delta  ->  s (1 - beta / kbar) delta(k)

Eq. FullDGP2 then reads, pointwise on the mesh,
    R = D^2 + alpha D - sum_ij H_ij^2 + c2 N - S = 0.

Readings of the paper used here (the paper is silent on them):
  * k = 0: D(0) = N(0) = S(0) = phi(0) = 0, delta(0) ignored; the real-space
    D used in the pointwise formulas is the mean-free one (the iteration
    projects D(0) = 0 each time it transforms D).
  * Nyquist: a multiplier odd in a component at the Nyquist index would make
    the inverse transform non-Hermitian.  Forces (i k_i) are set to zero
    there.  For the off-diagonal Hessian multipliers the oracle uses
    |k_i k_j| / k^2 when k_i or k_j is at Nyquist, which keeps
    sum_ij m_ij(k)^2 = 1 at every k != 0 (so <D^2> = <sum H_ij^2> exactly,
    the mesh form of Eq. NLFourier having no monopole for mean-free D) and
    lets R -> 0 at the fixed point.
  * The residual norm is the mean of |R| (the signed mean is zero, see above)
    divided by eps = <|S|> (Eq. normres).
  * Bad points (Delta < 0, Sec. III.C) take Delta = 0.
  * The accepted iterate is the one whose residual met the tolerance (the
    residual certifies the incoming D); without convergence, the iterate of
    minimum residual (Sec. III.C, Fig. 4 discussion).
"""

import numpy as np

from . import background as bg
from .fft import fft3, ifft3_real


class KGrid:
    """Wave vectors of an N^3 periodic mesh of side ``box`` (grid point i at x = i d)."""

    def __init__(self, n, box):
        self.n, self.box = n, box
        i = np.arange(n)
        m = np.where(i < n // 2, i, i - n)  # the Nyquist index n/2 maps to -n/2
        k1 = 2.0 * np.pi * m / box
        nyq1 = (i == n // 2) if n % 2 == 0 else np.zeros(n, bool)
        self.k = [k1[:, None, None], k1[None, :, None], k1[None, None, :]]
        self.nyq = [nyq1[:, None, None], nyq1[None, :, None], nyq1[None, None, :]]
        self.k2 = self.k[0] ** 2 + self.k[1] ** 2 + self.k[2] ** 2
        self.kmag = np.sqrt(self.k2)
        self.zero = self.k2 == 0.0
        self.k2_safe = np.where(self.zero, 1.0, self.k2)

    def hessian_multiplier(self, i, j):
        """m_ij(k) = k_i k_j / k^2 (Sec. III.B), 0 at k = 0; |k_i k_j|/k^2 on a
        Nyquist plane of i or j when i != j (see module docstring)."""
        num = self.k[i] * self.k[j]
        if i != j:
            num = np.where(self.nyq[i] | self.nyq[j], np.abs(num), num)
        return np.where(self.zero, 0.0, num / self.k2_safe)

    def gradient_multiplier(self, i):
        """i k_i with the Nyquist component of axis i set to zero."""
        return np.where(self.nyq[i], 0.0, 1j * self.k[i]) * np.ones_like(self.k2)


PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _kbar_inv(grid, coef, local_only):
    """1 / kbar = a E / (C_H |k|), 0 at k = 0; identically 0 when local_only
    (the local form Eq. FullDGP2simp of the Appendix)."""
    if local_only:
        return np.zeros_like(grid.k2)
    kb = np.where(grid.zero, 1.0, bg.C_H * grid.kmag / (coef["a"] * coef["E"]))
    return np.where(grid.zero, 0.0, 1.0 / kb)


def source_spectrum(delta_k, grid, coef, local_only=False):
    """S(k) = s (1 - beta / kbar) delta(k): RHS of Eq. FullDGP2; S(0) = 0."""
    ikb = _kbar_inv(grid, coef, local_only)
    out = coef["s"] * (1.0 - coef["beta"] * ikb) * delta_k
    out[grid.zero] = 0.0
    return out


def linear_D_spectrum(S_k, grid, coef, local_only=False):
    """Linearised Eq. FullDGP2 in Fourier space (Sec. III.B):
    -alpha kbar^2 C + c2 kbar C = S  with D = -kbar^2 C  gives
    D(k) = S(k) / (alpha - c2 / kbar).  This is the first trial solution."""
    ikb = _kbar_inv(grid, coef, local_only)
    out = S_k / (coef["alpha"] - coef["c2"] * ikb)
    out[grid.zero] = 0.0
    return out


def derived_fields(D_k, grid, coef, local_only=False):
    """Real-space D (mean-free), the six H_ij and N from D(k)."""
    D_k = D_k.copy()
    D_k[grid.zero] = 0.0
    D = ifft3_real(D_k)
    H = {p: ifft3_real(grid.hessian_multiplier(*p) * D_k) for p in PAIRS}
    Nf = ifft3_real(-_kbar_inv(grid, coef, local_only) * D_k)
    return D, H, Nf


def sum_hessian_sq(H):
    """(lapbar_ij C)^2 summed over i, j (symmetric: off-diagonals twice)."""
    return (H[(0, 0)] ** 2 + H[(1, 1)] ** 2 + H[(2, 2)] ** 2
            + 2.0 * (H[(0, 1)] ** 2 + H[(0, 2)] ** 2 + H[(1, 2)] ** 2))


def residual(D, H, Nf, S, coef):
    """R = LHS - RHS of Eq. FullDGP2 (Sec. III.B, residual paragraph)."""
    return D * D + coef["alpha"] * D - sum_hessian_sq(H) + coef["c2"] * Nf - S


def relax_update(D, H, Nf, S, coef, w):
    """One pointwise update, Eqs. nabla^2Cwpara and Bwpara (Sec. III.C):
    B' = sum H^2 - w D^2 - c2 N + S,  Delta = alpha^2 + 4 (1-w) B',
    D_new = (-alpha + sqrt(Delta)) / (2 (1-w))  ('+' root, Sec. III.B);
    points with Delta < 0 are bad points and take Delta = 0.
    Returns (D_new, number of bad points)."""
    alpha = coef["alpha"]
    Bp = sum_hessian_sq(H) - w * D * D - coef["c2"] * Nf + S
    Delta = alpha * alpha + 4.0 * (1.0 - w) * Bp
    bad = Delta < 0.0
    Delta = np.where(bad, 0.0, Delta)
    return (-alpha + np.sqrt(Delta)) / (2.0 * (1.0 - w)), int(bad.sum())


def solve_brane_bending(delta, a, box, omega_m0, rc_H0, w=1.0 / 3.0, tol=1e-12,
                        max_iter=500, D_init=None, local_only=False, patience=10):
    """Solve Eq. FullDGP2 for D = lapbar^2 C by FFT-relaxation (Secs. III.B-C).

    delta : real N^3 density contrast at scale factor ``a`` (its mean is ignored)
    D_init: previous nonlinear solution (warm start, Sec. III.B last paragraph);
            None -> the linear solution.
    Stops when <|R|>/eps < tol; otherwise after ``max_iter`` updates, or when
    bad points are present and the residual rises, or after ``patience``
    updates without a new minimum, returning the minimum-residual iterate.

    Returns (D, info): D is the accepted mean-free iterate (real N^3) and info
    holds D_k, delta_k, S, eps, iters (updates before the accepted iterate),
    history (normalised residual per iterate), bad (bad points per update),
    converged.
    """
    n = delta.shape[0]
    grid = KGrid(n, box)
    coef = bg.coefficients(a, omega_m0, rc_H0)
    delta_k = fft3(delta)
    delta_k[grid.zero] = 0.0
    S_k = source_spectrum(delta_k, grid, coef, local_only)
    S = ifft3_real(S_k)
    eps = float(np.mean(np.abs(S)))
    if D_init is None:
        D = ifft3_real(linear_D_spectrum(S_k, grid, coef, local_only))
    else:
        D = np.array(D_init, dtype=np.float64)

    history, bads = [], []
    best = (np.inf, None, None, -1)
    converged = False
    for it in range(max_iter + 1):
        D_k = fft3(D)
        D_k[grid.zero] = 0.0
        D, H, Nf = derived_fields(D_k, grid, coef, local_only)
        # Eq. normres divides by eps; with a zero source (uniform density) there
        # is no scale and the absolute mean residual is monitored instead.
        r = float(np.mean(np.abs(residual(D, H, Nf, S, coef)))) / (eps if eps > 0 else 1.0)
        history.append(r)
        if r < best[0]:
            best = (r, D, D_k, it)
        if r < tol:
            converged = True
            break
        if it == max_iter:
            break
        if bads and bads[-1] > 0 and len(history) > 1 and r > history[-2]:
            break
        if it - best[3] >= patience:
            break
        D, nbad = relax_update(D, H, Nf, S, coef, w)
        bads.append(nbad)
    r, D, D_k, it = best
    info = dict(D_k=D_k, delta_k=delta_k, S=S, eps=eps, iters=it, history=history,
                bad=bads, converged=converged, norm_res=r, coef=coef, grid=grid)
    return D, info


def spherical_D(delta_k, grid, coef, local_only=False):
    """Spherical approximation of Eq. FullDGP2 (Sec. IV, Eq. FullDGP2sph): the
    w = 1/3 relaxation update from C = 0.  There every H_ij and N vanish, so
    B' = S and the '+' root is D = (-alpha + sqrt(alpha^2 + (8/3) S)) / (4/3)
    (bad points, Delta < 0, take Delta = 0); S = s (1 - beta/kbar) delta keeps
    its nonlocal factor.  Returns (D mean-free, D_k, number of bad points)."""
    S = ifft3_real(source_spectrum(delta_k, grid, coef, local_only))
    z = np.zeros_like(S)
    D, nbad = relax_update(z, {p: z for p in PAIRS}, z, S, coef, 1.0 / 3.0)
    D_k = fft3(D)
    D_k[grid.zero] = 0.0
    return ifft3_real(D_k), D_k, nbad


def phi_spectrum(delta_k, D_k, grid, coef, local_only=False, gravity="nl"):
    """phi(k) in code units from Eq. FullDGP1 (Sec. II) given delta(k), D(k).

    Fourier form with lapbar -> -kbar^2, sqrt(-lapbar) -> kbar, and
    kbar C = -D / kbar:
        -kbar^2 (1 + 1/(eta kbar)) phi = (3/2)(eta-1)/eta delta - D/(2 eta) + c3 D / kbar
    and phi_code = C_H^2 phi, C_H^2 / kbar^2 = (a E)^2 / k^2.
    gravity="grh": GR with the DGP expansion, Eq. GRPoisson;
    gravity="ldgp": linearised DGP, Eq. LinearDGP with G_eff of Eq. Geff.
    """
    a, E, eta = coef["a"], coef["E"], coef["eta"]
    pref = -(a * E) ** 2 / grid.k2_safe
    om = (eta - 1.0) / eta  # = Omega_m(a)
    if gravity == "grh":
        out = pref * 1.5 * om * delta_k
    elif gravity == "ldgp":
        out = pref * 1.5 * om * _geff(grid, coef) * delta_k
    else:
        ikb = _kbar_inv(grid, coef, local_only)
        rhs = 1.5 * om * delta_k - D_k / (2.0 * eta) + coef["c3"] * D_k * ikb
        out = pref * rhs / (1.0 + ikb / eta)
    out = np.where(grid.zero, 0.0, out)
    return out


def _geff(grid, coef):
    """G_eff/G of Eq. Geff on the mesh (r_c H0 = eta / E)."""
    eta, q, a = coef["eta"], coef["q"], coef["a"]
    rc = eta / coef["E"]
    kk = np.where(grid.zero, 1.0, grid.kmag)
    inv = (2 * eta * (2 + q) - 3) / (2 * eta * (2 + q) - 4) \
        + (3.0 * a / (kk * rc * bg.C_H)) * ((eta * (1 + q) - 1) / (eta * (2 + q) - 2)) ** 2
    return 1.0 / inv


def phi_and_forces(delta_k, D_k, grid, coef, local_only=False, gravity="nl"):
    """phi (real) and the force field g_i = -d_i phi (Sec. III.A: grad phi is
    i k phi in Fourier space, transformed back to the mesh)."""
    pk = phi_spectrum(delta_k, D_k, grid, coef, local_only, gravity)
    phi = ifft3_real(pk)
    g = [ifft3_real(-grid.gradient_multiplier(i) * pk) for i in range(3)]
    return phi, g


def solve_phi(delta, a, box, omega_m0, rc_H0, w=1.0 / 3.0, tol=1e-12, max_iter=500,
              D_init=None, local_only=False, gravity="nl"):
    """delta -> (phi, forces, D, info): the full field solve of one PM step."""
    if gravity == "nl":
        D, info = solve_brane_bending(delta, a, box, omega_m0, rc_H0, w, tol, max_iter,
                                      D_init, local_only)
        D_k = info["D_k"]
        grid, coef, delta_k = info["grid"], info["coef"], info["delta_k"]
    elif gravity == "sph":
        grid = KGrid(delta.shape[0], box)
        coef = bg.coefficients(a, omega_m0, rc_H0)
        delta_k = fft3(delta)
        delta_k[grid.zero] = 0.0
        D, D_k, nbad = spherical_D(delta_k, grid, coef, local_only)
        info = dict(iters=1, converged=True, bad=[nbad])
        gravity = "nl"  # Eq. FullDGP1 with the spherical D
    else:
        grid = KGrid(delta.shape[0], box)
        coef = bg.coefficients(a, omega_m0, rc_H0)
        delta_k = fft3(delta)
        delta_k[grid.zero] = 0.0
        D, D_k, info = None, None, dict(iters=0, converged=True)
    phi, g = phi_and_forces(delta_k, D_k, grid, coef, local_only, gravity)
    return phi, g, D, info
