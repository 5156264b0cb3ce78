"""Adjoint of the converged field solve (delta -> phi) in the oracle.

Test infrastructure: see ``oracle/__init__.py``.

The forward solve (Secs. III.B-C) defines D implicitly by R(D, delta) = 0 on
mean-free fields, with
    R(D, delta) = D^2 + alpha D - sum_ij H_ij(D)^2 + c2 N[D] - S[delta]  (Eq. FullDGP2),
and phi = A delta + B D from Eq. FullDGP1, A and B real even Fourier
multipliers (phi_spectrum with D = 0, resp. delta = 0).  For a cotangent
phibar of phi (gradient of a scalar L = <phibar, phi>, <.,.> the sum over
mesh points), the implicit function theorem gives
    Dbar = B phibar,   J^T lam = Dbar,   deltabar = A phibar + S lam,
with J = dR/dD and S = -dR/ddelta the source multiplier s (1 - beta/kbar).
H_ij, N, A, B and S are real even multipliers, hence symmetric, so
    J^T lam = (2 D + alpha) lam - 2 sum_ij H_ij[H_ij(D) lam] + c2 N[lam]
(the sum over all nine i, j).  J^T lam = g is solved by the w-splitting the
forward solve uses (Sec. III.C): the diagonal (2 (1 - w) D + alpha) lam is
taken implicitly and the rest from the previous iterate,
    lam_new = (g - 2 w D lam + 2 sum_ij H_ij[H_ij(D) lam] - c2 N[lam] + c) / (2 (1 - w) D + alpha).
The solve lives on mean-free fields: J maps them to mean-free fields (the
nonlinear terms' mean vanishes since sum_ij (k_i k_j / k^2)^2 = 1), so the
system is P J^T lam = P g with P the mean projection and lam mean-free; the
constant c (the free mean of J^T lam - g) is the one that makes lam_new
mean-free.  At a converged D the divisor equals sqrt(Delta) of Eq. nabla^2Cwpara.

A cotangent of the forces g_i = -d_i phi enters as phibar = sum_i d_i gbar_i
(i k_i in Fourier space, the Nyquist component set to zero), the transpose of
the force multiplier -i k_i.

The particle side (deposit, force interpolation, the kick-drift-kick step)
is differentiated below by hand from the CIC weights' derivatives.

The crossover scale r_c H0 enters the converged solve through the scalar
coefficients and E(a) (in 1/kbar and the prefactor (a E)^2 / k^2).  With D, lam
and delta held at the solution, its explicit derivative is
    rcbar = <phibar, A' delta + B' D> - <lam, dR/d(r_c H0)>,
    dR/d(r_c H0) = alpha' D + c2' N[D] + c2 N'[D] - S' delta,
(' = d/d(r_c H0)); a step adds the derivatives of its kick and drift factors.

Parity pins (tests/test_oracle_adjoint.py): central finite differences of
<phibar, phi(delta)> through the oracle's own nonlinear solve; the identity
<u, J v> = <J^T u, v> with J v taken by finite differences of the forward
residual; the D = 0 limit, where J^T = alpha + c2 N is diagonal in k; and
central differences of the deposit, the particle forces and a whole step.
"""

import numpy as np

from . import background as bg
from . import field
from .fft import fft3, ifft3_real

_ALL_PAIRS = [(i, j) for i in range(3) for j in range(3)]


def _mult(grid, coef, local_only):
    """Real even multipliers of Eq. FullDGP1 and Eq. FullDGP2: A, B (phi = A delta + B D),
    S (source), the N operator n(k) = -1/kbar."""
    a, E, eta = coef["a"], coef["E"], coef["eta"]
    ikb = field._kbar_inv(grid, coef, local_only)
    pref = -(a * E) ** 2 / grid.k2_safe
    den = 1.0 + ikb / eta
    A = np.where(grid.zero, 0.0, pref * 1.5 * (eta - 1.0) / eta / den)
    B = np.where(grid.zero, 0.0, pref * (-1.0 / (2.0 * eta) + coef["c3"] * ikb) / den)
    S = np.where(grid.zero, 0.0, coef["s"] * (1.0 - coef["beta"] * ikb))
    Nm = -ikb
    return A, B, S, Nm


def _mult_drc(grid, coef, dcoef, local_only):
    """d/d(r_c H0) of the multipliers of _mult (dcoef from background.coefficient_derivatives)."""
    a, E, eta = coef["a"], coef["E"], coef["eta"]
    dE, deta = dcoef["E"], dcoef["eta"]
    ikb = field._kbar_inv(grid, coef, local_only)
    dikb = ikb * dE / E                                  # 1/kbar = a E / (C_H |k|)
    pref = -(a * E) ** 2 / grid.k2_safe
    dpref = 2.0 * pref * dE / E
    den = 1.0 + ikb / eta
    dden = dikb / eta - ikb * deta / (eta * eta)
    om, dom = (eta - 1.0) / eta, deta / (eta * eta)
    dA = 1.5 * (dpref * om / den + pref * dom / den - pref * om * dden / (den * den))
    b = -1.0 / (2.0 * eta) + coef["c3"] * ikb
    db = deta / (2.0 * eta * eta) + dcoef["c3"] * ikb + coef["c3"] * dikb
    dB = dpref * b / den + pref * db / den - pref * b * dden / (den * den)
    dS = dcoef["s"] * (1.0 - coef["beta"] * ikb) - coef["s"] * (dcoef["beta"] * ikb + coef["beta"] * dikb)
    z = grid.zero
    return (np.where(z, 0.0, dA), np.where(z, 0.0, dB), np.where(z, 0.0, dS), np.where(z, 0.0, -dikb))


def rc_bar_solve(phibar, lam, delta, D, grid, coef, dcoef, local_only=False):
    """Explicit d<phibar, phi>/d(r_c H0) of a converged solve (module docstring)."""
    _, _, _, Nm = _mult(grid, coef, local_only)
    dA, dB, dS, dN = _mult_drc(grid, coef, dcoef, local_only)
    dR = dcoef["alpha"] * D + dcoef["c2"] * _apply(Nm, D) + coef["c2"] * _apply(dN, D) - _apply(dS, delta)
    return float(np.sum(phibar * (_apply(dA, delta) + _apply(dB, D))) - np.sum(lam * dR))


def _apply(mult, f):
    return ifft3_real(mult * fft3(f))


def _mean_free(f):
    return f - np.mean(f)


def jt_apply(lam, D, H, grid, coef, local_only=False):
    """J^T lam for the converged D with Hessian fields H (dict over field.PAIRS)."""
    _, _, _, Nm = _mult(grid, coef, local_only)
    out = (2.0 * D + coef["alpha"]) * lam + coef["c2"] * _apply(Nm, lam)
    for (i, j) in _ALL_PAIRS:
        p = (min(i, j), max(i, j))
        out -= 2.0 * _apply(grid.hessian_multiplier(i, j), H[p] * lam)
    return out


def solve_adjoint(D, H, g, grid, coef, w=1.0 / 3.0, tol=1e-12, max_iter=500, local_only=False):
    """Solve J^T lam = g (mean-free g) by the w-split iteration; returns (lam, info)."""
    _, _, _, Nm = _mult(grid, coef, local_only)
    diag = 2.0 * (1.0 - w) * D + coef["alpha"]
    if np.any(diag <= 0.0):
        raise ValueError("2 (1 - w) D + alpha must be positive (no bad points at the solution)")
    gn = float(np.mean(np.abs(g)))
    scale = gn if gn > 0 else 1.0
    inv_diag_mean = float(np.mean(1.0 / diag))

    def update(rhs):  # rhs = g - rest; the constant making the result mean-free
        c = -float(np.mean(rhs / diag)) / inv_diag_mean
        return (rhs + c) / diag

    lam = update(g)
    history = []
    for it in range(max_iter + 1):
        r = float(np.mean(np.abs(_mean_free(jt_apply(lam, D, H, grid, coef, local_only) - g)))) / scale
        history.append(r)
        if r < tol or it == max_iter:
            break
        rest = 2.0 * w * D * lam + coef["c2"] * _apply(Nm, lam)
        for (i, j) in _ALL_PAIRS:
            p = (min(i, j), max(i, j))
            rest -= 2.0 * _apply(grid.hessian_multiplier(i, j), H[p] * lam)
        lam = update(g - rest)
    return lam, dict(iters=len(history) - 1, history=history, converged=history[-1] < tol)


def phibar_from_forces(gbar, grid):
    """phibar = sum_i d_i gbar_i: the transpose of g_i = -d_i phi (Nyquist component zero)."""
    out = np.zeros_like(gbar[0])
    for i in range(3):
        out += ifft3_real(grid.gradient_multiplier(i) * fft3(gbar[i]))
    return out


def phi_vjp(delta, a, box, omega_m0, rc_H0, phibar, w=1.0 / 3.0, tol=1e-13, adj_tol=1e-12,
            max_iter=500, local_only=False):
    """deltabar = d<phibar, phi(delta)>/d delta through the converged nonlinear solve.
    Returns (deltabar, info) with the forward solve's D and the adjoint's lam."""
    D, finfo = field.solve_brane_bending(delta, a, box, omega_m0, rc_H0, w, tol, max_iter,
                                         local_only=local_only)
    grid, coef = finfo["grid"], finfo["coef"]
    _, H, _ = field.derived_fields(finfo["D_k"], grid, coef, local_only)
    A, B, S, _ = _mult(grid, coef, local_only)
    Dbar = _apply(B, phibar)
    lam, ainfo = solve_adjoint(D, H, Dbar, grid, coef, w, adj_tol, max_iter, local_only)
    deltabar = _apply(A, phibar) + _apply(S, lam)
    dcoef = bg.coefficient_derivatives(a, omega_m0, rc_H0)
    rcbar = rc_bar_solve(phibar, lam, delta, D, grid, coef, dcoef, local_only)
    return deltabar, dict(D=D, lam=lam, forward=finfo, adjoint=ainfo, rcbar=rcbar)


# ---------------------------------------------------------------- particles
# CIC (Eq. CIC) is piecewise linear in the positions: for the corner c of a
# particle the weight is W = w_x w_y w_z with w = 1 - f or f per axis, and
# dW/dx_a = (+-1/d) times the other two factors (- for the lower corner).

def _corner_terms(pos, n, box):
    """Yield (flat corner index, W, dW/dx, dW/dy, dW/dz) for the 8 corners of every particle."""
    from . import pm
    d = box / n
    (ix, fx), (iy, fy), (iz, fz) = pm._cic_cells(np.asarray(pos, float), n, box)
    for dx in (0, 1):
        wx, sx, jx = (fx, 1.0 / d, (ix + 1) % n) if dx else (1.0 - fx, -1.0 / d, ix)
        for dy in (0, 1):
            wy, sy, jy = (fy, 1.0 / d, (iy + 1) % n) if dy else (1.0 - fy, -1.0 / d, iy)
            for dz in (0, 1):
                wz, sz, jz = (fz, 1.0 / d, (iz + 1) % n) if dz else (1.0 - fz, -1.0 / d, iz)
                yield (jx * n + jy) * n + jz, wx * wy * wz, sx * wy * wz, wx * sy * wz, wx * wy * sz


def deposit_vjp(pos, n, box, rhobar):
    """Transpose of the Jacobian of rho(x) = sum_p W(x - x_p) in the positions:
    xbar_p = sum_c grad W(x_p - c) rhobar_c, shape (3, Np)."""
    flat = np.asarray(rhobar, float).reshape(-1)
    out = np.zeros((3, np.asarray(pos).shape[1]))
    for idx, _, gx, gy, gz in _corner_terms(pos, n, box):
        v = flat[idx]
        out[0] += gx * v
        out[1] += gy * v
        out[2] += gz * v
    return out


def gather_vjp(grids, pos, box, fbar):
    """F_p,i = sum_c W(x_p - c) G_i(c) (the force interpolation of Sec. III.A): for the
    particle cotangents fbar (3, Np) returns (Gbar, xbar): Gbar_i = sum_p W fbar_i,p (the
    deposit of fbar) and xbar_p = sum_c grad W(x_p - c) (G(c) . fbar_p)."""
    from . import pm
    n = grids[0].shape[0]
    Gbar = [pm.cic_deposit(pos, n, box, mass=fbar[i]) for i in range(3)]
    flats = [np.asarray(g, float).reshape(-1) for g in grids]
    xbar = np.zeros((3, np.asarray(pos).shape[1]))
    for idx, _, gx, gy, gz in _corner_terms(pos, n, box):
        v = flats[0][idx] * fbar[0] + flats[1][idx] * fbar[1] + flats[2][idx] * fbar[2]
        xbar[0] += gx * v
        xbar[1] += gy * v
        xbar[2] += gz * v
    return Gbar, xbar


def force_vjp(pos, a, n, box, omega_m0, rc_H0, fbar, w=1.0 / 3.0, tol=1e-13, adj_tol=1e-12,
              with_rc=False):
    """xbar for the particle forces F(x) = gather(g(delta(x)), x) of Sec. III.A: the
    direct term of the gather, plus deposit of fbar -> force cotangent grids -> the solve's
    adjoint -> deltabar -> rhobar = deltabar M / Np (delta = rho M / Np - 1, the particle
    count being conserved) -> the deposit's transpose.  with_rc: returns (xbar, rcbar,
    <fbar, F>), rcbar the explicit d<fbar, F>/d(r_c H0) of the solve."""
    from . import pm
    pos = np.asarray(pos, float) % box
    npart = pos.shape[1]
    delta = pm.density_contrast(pm.cic_deposit(pos, n, box))
    _, g, _, _ = field.solve_phi(delta, a, box, omega_m0, rc_H0, w, tol)
    Gbar, xbar = gather_vjp(g, pos, box, fbar)
    grid = field.KGrid(n, box)
    dbar, info = phi_vjp(delta, a, box, omega_m0, rc_H0, phibar_from_forces(Gbar, grid), w, tol, adj_tol)
    xbar = xbar + deposit_vjp(pos, n, box, dbar * (n ** 3 / npart))
    if not with_rc:
        return xbar
    F = np.stack([pm.cic_interpolate(g[i], pos, box) for i in range(3)])
    return xbar, info["rcbar"], float(np.sum(np.asarray(fbar) * F))


def step_vjp(pos0, mom0, a, da, xbar1, pbar1, n, box, omega_m0, rc_H0, w=1.0 / 3.0, tol=1e-13,
             with_rc=False):
    """Transpose of the Jacobian of one kick-drift-kick step (Sec. III.A, as PMState.step):
    p_h = p0 + K1 F(x0), x1 = x0 + Dr p_h (mod box), p1 = p_h + K2 F(x1).
    Returns (xbar0, pbar0) for the cotangents (xbar1, pbar1) of (x1, p1); with_rc also
    the step's explicit derivative in r_c H0 (xbar0, pbar0, rcbar):
        K2' <pbar1, F(x1)> + rcbar_solve(x1) + Dr' <xbar1_tot, p_h>
        + K1' <pbar_h, F(x0)> + rcbar_solve(x0),
    xbar1_tot the cotangent of x1 after the second kick's transpose."""
    if with_rc:
        return _step_vjp_rc(pos0, mom0, a, da, xbar1, pbar1, n, box, omega_m0, rc_H0, w, tol)
    a1 = a + da
    ah = np.exp(0.5 * (np.log(a) + np.log(a1)))
    k1 = bg.kick_factor(a, ah, omega_m0, rc_H0)
    k2 = bg.kick_factor(ah, a1, omega_m0, rc_H0)
    dr = bg.drift_factor(a, a1, omega_m0, rc_H0)
    from . import pm
    st = pm.PMState(pos0, mom0, a, n, box, omega_m0, rc_H0, w=w, tol=tol)
    f0 = st.forces_at_particles()
    ph = st.mom + k1 * f0
    x1 = (st.pos + dr * ph) % box
    xbar = xbar1 + force_vjp(x1, a1, n, box, omega_m0, rc_H0, k2 * pbar1, w, tol)
    phbar = pbar1 + dr * xbar
    xbar0 = xbar + force_vjp(st.pos, a, n, box, omega_m0, rc_H0, k1 * phbar, w, tol)
    return xbar0, phbar


def _step_vjp_rc(pos0, mom0, a, da, xbar1, pbar1, n, box, omega_m0, rc_H0, w, tol):
    from . import pm
    a1 = a + da
    ah = np.exp(0.5 * (np.log(a) + np.log(a1)))
    k1 = bg.kick_factor(a, ah, omega_m0, rc_H0)
    k2 = bg.kick_factor(ah, a1, omega_m0, rc_H0)
    dr = bg.drift_factor(a, a1, omega_m0, rc_H0)
    dk1 = bg.kick_factor_drc(a, ah, omega_m0, rc_H0)
    dk2 = bg.kick_factor_drc(ah, a1, omega_m0, rc_H0)
    ddr = bg.drift_factor_drc(a, a1, omega_m0, rc_H0)
    st = pm.PMState(pos0, mom0, a, n, box, omega_m0, rc_H0, w=w, tol=tol)
    f0 = st.forces_at_particles()
    ph = st.mom + k1 * f0
    x1 = (st.pos + dr * ph) % box
    pbar1 = np.asarray(pbar1, float)
    xb, rc1, pf1 = force_vjp(x1, a1, n, box, omega_m0, rc_H0, k2 * pbar1, w, tol, with_rc=True)
    xbar = np.asarray(xbar1, float) + xb
    phbar = pbar1 + dr * xbar
    xb0, rc0, pf0 = force_vjp(st.pos, a, n, box, omega_m0, rc_H0, k1 * phbar, w, tol, with_rc=True)
    rcbar = dk2 * pf1 / k2 + rc1 + ddr * float(np.sum(xbar * ph)) + dk1 * pf0 / k1 + rc0
    return xbar + xb0, phbar, rcbar


# ---------------------------------------------------------------- estimator and initial conditions
def pk_vjp(delta, box, nbins, dldp):
    """deltabar for L(P) with the P(k) estimator of Sec. IV (estimators.power_spectrum):
    P_b = box^3 / (M^2 n_b) sum_{k in b} |delta_k|^2, so dL/ddelta(x) =
    2 sum_k c(k) Re(delta_k e^{i k x}) with c(k) = dL/dP_b box^3 / (M^2 n_b) on shell b."""
    from .estimators import power_spectrum
    n = delta.shape[0]
    m = n ** 3
    grid = field.KGrid(n, box)
    kf = 2.0 * np.pi / box
    _, _, cnt = power_spectrum(delta, box, nbins)
    b = np.floor(grid.kmag / kf + 0.5).astype(np.int64) * np.ones((n, n, n), np.int64)
    c = np.zeros((n, n, n))
    sel = (b >= 1) & (b <= nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        cb = np.where(cnt > 0, np.asarray(dldp, float) * box ** 3 / (m * m * np.maximum(cnt, 1)), 0.0)
    c[sel] = cb[b[sel] - 1]
    return 2.0 * m * ifft3_real(c * fft3(delta))


def zeldovich_vjp(xbar, pbar, n, box, vel_factor):
    """deltaL_bar for (pos, mom) = (q + Psi, vel_factor Psi), Psi_j = IFFT(i k_j / k^2 delta_L(k))
    (Nyquist component of k_j dropped): sum_j Psi_j^T (xbar_j + vel_factor pbar_j), the transpose of
    the multiplier i k_j / k^2 being -i k_j / k^2."""
    grid = field.KGrid(n, box)
    out = np.zeros((n, n, n))
    for j in range(3):
        psibar = (np.asarray(xbar[j]) + vel_factor * np.asarray(pbar[j])).reshape(n, n, n)
        mult = np.where(grid.zero, 0.0, -grid.gradient_multiplier(j) / grid.k2_safe)
        out += ifft3_real(mult * fft3(psibar))
    return out


def zeldovich_displacement(delta_l, box):
    """Psi_j = IFFT(i k_j / k^2 delta_L(k)), the Nyquist component of k_j dropped (three n^3 fields)."""
    n = delta_l.shape[0]
    grid = field.KGrid(n, box)
    dk = fft3(np.asarray(delta_l, float))
    return [ifft3_real(np.where(grid.zero, 0.0, grid.gradient_multiplier(j) / grid.k2_safe) * dk)
            for j in range(3)]


def zeldovich_vf_bar(pbar, delta_l, box):
    """Cotangent of vel_factor in mom = vel_factor Psi: sum_j <pbar_j, Psi_j>."""
    psi = zeldovich_displacement(delta_l, box)
    return float(sum(np.sum(np.asarray(pbar[j]).reshape(psi[j].shape) * psi[j]) for j in range(3)))
