"""Pins of the oracle's field solve (Secs. II, III.B-C, Appendix) against closed
forms and invariants that do not come from the oracle itself."""
import math

import numpy as np
import pytest

from oracle import background as bg
from oracle import field
from oracle.fft import fft3, ifft3_real
from paper_0906_4548_gb300 import inputs

OM = 0.27


def _mode_amp(f, n, idx):
    return fft3(f)[idx]


@pytest.mark.parametrize("a,rc", [(1.0, 1.0), (0.5, 2.0)])
def test_linear_phi_matches_geff_to_first_order(a, rc):
    """Eq. Geff is Eq. FullDGP1+2 linearised and expanded to first order in
    1/kbar (Sec. II): the exact linear phi must differ from it by O(1/kbar^2)."""
    n, box = 16, 2000.0
    coef = bg.coefficients(a, OM, rc)
    errs, kbars = [], []
    for m in (1, 2, 4):
        i = np.arange(n)
        delta = 1e-7 * np.cos(2 * np.pi * m * i / n)[:, None, None] * np.ones((n, n, n))
        phi, _, D, info = field.solve_phi(delta, a, box, OM, rc, tol=1e-12)
        k = 2 * np.pi * m / box
        ratio = (fft3(phi)[m, 0, 0] / fft3(delta)[m, 0, 0]).real
        want = -(a * coef["E"]) ** 2 / k ** 2 * 1.5 * coef["omega_m"] * bg.geff_over_G(k, a, OM, rc)
        errs.append(abs(ratio / want - 1))
        kbars.append(bg.C_H * k / (a * coef["E"]))
    kbars = np.array(kbars)
    errs = np.array(errs)
    assert np.all(errs * kbars ** 2 < 5.0)
    # second-order scaling: doubling kbar divides the error by ~4
    r = errs[:-1] / errs[1:]
    assert np.all((r > 3.0) & (r < 5.5)), (errs, kbars)


def _line_field(n, direction, rng, band_limited=False):
    i, j, k = np.indices((n, n, n))
    u = (direction[0] * i + direction[1] * j + direction[2] * k) % n
    f = rng.standard_normal(n)
    if band_limited:
        F = np.fft.fft(f)
        F[n // 2] = 0
        f = np.fft.ifft(F).real
    d = f[u]
    return 0.9 * (d - d.mean()) / np.abs(d - d.mean()).max()


@pytest.mark.parametrize("direction,bl", [((1, 0, 0), False), ((0, 1, 1), False),
                                          ((1, 1, 1), False), ((1, -1, 0), True)])
def test_one_dimensional_field_has_no_nonlinear_term(direction, bl):
    """Sec. VI / Eq. NLFourier: the kernel (1 - mu^2) vanishes when all modes are
    collinear, so the nonlinear solution is the linear one and phi is linear."""
    n, box, a = 16, 64.0, 0.5
    d = _line_field(n, direction, np.random.default_rng(7), bl)
    D, info = field.solve_brane_bending(d, a, box, OM, 1.0, tol=1e-13)
    coef = bg.coefficients(a, OM, 1.0)
    grid = field.KGrid(n, box)
    dk = fft3(d)
    dk[grid.zero] = 0
    Dlin = ifft3_real(field.linear_D_spectrum(field.source_spectrum(dk, grid, coef), grid, coef))
    assert info["converged"] and info["iters"] == 0
    assert np.max(np.abs(D - Dlin)) <= 1e-12 * np.max(np.abs(Dlin))


def test_two_plane_waves_nonlinear_term_closed_form():
    """Eq. NLFourier for D = D1 cos(k1.x) + D2 cos(k2.x):
    (lapbar C)^2 - (lapbar_ij C)^2 = 2 D1 D2 cos(k1.x) cos(k2.x) (1 - mu^2)."""
    n, box = 16, 100.0
    grid = field.KGrid(n, box)
    coef = bg.coefficients(0.5, OM, 1.0)
    x = np.indices((n, n, n)) * (box / n)
    n1, n2 = np.array([1, 2, 0]), np.array([0, -1, 3])
    k1, k2 = 2 * np.pi * n1 / box, 2 * np.pi * n2 / box
    c1 = np.cos(np.tensordot(k1, x, 1))
    c2 = np.cos(np.tensordot(k2, x, 1))
    D1, D2 = 0.7, -1.3
    Dx = D1 * c1 + D2 * c2
    D, H, _ = field.derived_fields(fft3(Dx), grid, coef)
    mu = k1 @ k2 / np.linalg.norm(k1) / np.linalg.norm(k2)
    want = 2 * D1 * D2 * c1 * c2 * (1 - mu ** 2)
    assert np.max(np.abs(D * D - field.sum_hessian_sq(H) - want)) < 1e-12


def test_parseval_no_monopole_with_nyquist_content():
    """<D^2> = <sum H_ij^2> for any mean-free D (sum_ij m_ij^2 = 1 on every k != 0)."""
    n = 12
    grid = field.KGrid(n, 50.0)
    coef = bg.coefficients(0.5, OM, 1.0)
    Dk = fft3(np.random.default_rng(3).standard_normal((n, n, n)))
    D, H, _ = field.derived_fields(Dk, grid, coef)
    assert abs(np.mean(D * D) - np.mean(field.sum_hessian_sq(H))) < 1e-13 * np.mean(D * D)
    # trace of the Hessian is D
    assert np.max(np.abs(H[(0, 0)] + H[(1, 1)] + H[(2, 2)] - D)) < 1e-13


def test_first_w13_update_is_spherical_approximation():
    """Sec. IV: with w = 1/3 the first relaxation step from C = 0 solves Eq.
    FullDGP2sph; locally that is Eq. SphPoi for phi."""
    n = 8
    rng = np.random.default_rng(5)
    d = rng.uniform(-1, 4, (n, n, n))  # pointwise: any delta >= -1
    a = 0.3
    coef = bg.coefficients(a, OM, 1.0)
    eta, alpha = coef["eta"], coef["alpha"]
    z = np.zeros_like(d)
    H = {p: z for p in field.PAIRS}
    D1, nbad = field.relax_update(z, H, z, coef["s"] * d, coef, 1.0 / 3.0)
    lap_phi = 1.5 * (eta - 1) / eta * d - D1 / (2 * eta)  # local Eq. FullDGP1
    sph = 1.5 * (eta - 1) / eta * d - (1 / (2 * eta)) * (3 * alpha / 4) * (
        np.sqrt(1 + 8 / alpha ** 2 * (eta - 1) / eta * d) - 1)
    assert nbad == 0
    assert np.max(np.abs(lap_phi - sph)) < 1e-13


def test_spherical_profile_matches_radial_solution():
    """Local Eq. FullDGP2 in spherical symmetry: (2/r^2)(r C'^2)' + alpha lap C = s delta
    integrates to 2 g^2 + alpha g = s m(r)/r^3 with g = C'/r, so D = 3 g + r g'."""
    from scipy.special import erf
    n, box, a = 64, 64.0, 0.3
    coef = bg.coefficients(a, OM, 1.0)
    s, alpha = coef["s"], coef["alpha"]
    sig, A = box / 20, 6.0
    x = (np.indices((n, n, n)) - n // 2) * (box / n)
    r = np.sqrt((x ** 2).sum(0))
    dg = A * np.exp(-r ** 2 / (2 * sig ** 2))
    dbar = dg.mean()
    D, info = field.solve_brane_bending(dg - dbar, a, box, OM, 1.0, tol=1e-12, local_only=True)
    assert info["converged"]

    def g_of(rr):
        mg = sig ** 3 * (np.sqrt(np.pi / 2) * erf(rr / (np.sqrt(2) * sig))
                         - rr / sig * np.exp(-rr ** 2 / (2 * sig ** 2)))
        m = A * mg - dbar * rr ** 3 / 3
        return (-alpha + np.sqrt(alpha ** 2 + 8 * s * m / rr ** 3)) / 4

    sel = (r > 0) & (r < 2 * sig)
    rr = r[sel]
    h = 1e-4
    Dsph = 3 * g_of(rr) + rr * (g_of(rr + h) - g_of(rr - h)) / (2 * h)
    err = np.max(np.abs(D[sel] - Dsph)) / np.max(np.abs(Dsph))
    assert err < 5e-4, err
    # deep nonlinear regime: the linear answer s delta / alpha is far off at the centre
    c = (n // 2, n // 2, n // 2)
    assert abs(D[c] - s * (dg[c] - dbar) / alpha) > 0.3 * abs(D[c])


@pytest.fixture(scope="module")
def realistic():
    from paper_0906_4548_gb300 import inputs
    from oracle import pm
    n, box, a = 32, 100.0, 0.3
    vf = bg.zeldovich_velocity_factor(a, OM, 1.0)
    pos, mom, _ = inputs.zeldovich_particles(n, box, -2.0, 0.7, 11, vf)
    delta = pm.density_contrast(pm.cic_deposit(pos, n, box))
    return n, box, a, delta


def test_w_invariance_of_converged_solution(realistic):
    """Eq. FullDGP2wpara is Eq. FullDGP2 for every w (Sec. III.C): converged D
    does not depend on w."""
    n, box, a, delta = realistic
    D3, i3 = field.solve_brane_bending(delta, a, box, OM, 1.0, w=1 / 3, tol=1e-13)
    D5, i5 = field.solve_brane_bending(delta, a, box, OM, 1.0, w=0.5, tol=1e-13)
    assert i3["converged"] and i5["converged"]
    assert np.max(np.abs(D3 - D5)) < 1e-11 * np.max(np.abs(D3))


def test_ellipticity_of_converged_solution(realistic):
    """Appendix A: F_{lapbar_ij C} = (2 D + alpha) delta_ij - 2 H_ij has eigenvalues
    of one sign at every point for the w = 1/3 solution; the residual vanishes."""
    n, box, a, delta = realistic
    D, info = field.solve_brane_bending(delta, a, box, OM, 1.0, tol=1e-13)
    coef = info["coef"]
    _, H, Nf = field.derived_fields(info["D_k"], info["grid"], coef)
    R = field.residual(D, H, Nf, info["S"], coef)
    assert np.mean(np.abs(R)) / info["eps"] < 1e-13
    M = np.zeros((n, n, n, 3, 3))
    for (i, j) in field.PAIRS:
        M[..., i, j] = M[..., j, i] = -2 * H[(i, j)]
    for i in range(3):
        M[..., i, i] += 2 * D + coef["alpha"]
    ev = np.linalg.eigvalsh(M)
    assert np.all(ev > 0)
    assert max(info["bad"] or [0]) == 0


def test_monge_ampere_reduction_in_2d():
    """Appendix A, Eqs. MA and Det2D: for delta independent of z the local
    equation is 2 (Hxx Hyy - Hxy^2) + alpha (Hxx + Hyy) = s delta and the
    determinant alpha^2 + 6 (eta-1)/eta delta is positive for delta >= -1."""
    n, box, a = 32, 64.0, 0.4
    rng = np.random.default_rng(9)
    d2 = ifft3_real(fft3(rng.standard_normal((n, n, 1))) * 1.0).real
    d2 = np.exp(1.2 * (d2 - d2.mean()) / d2.std())
    d = np.repeat(d2 / d2.mean() - 1.0, n, axis=2)
    D, info = field.solve_brane_bending(d, a, box, OM, 1.0, tol=1e-13, local_only=True)
    coef = info["coef"]
    _, H, _ = field.derived_fields(info["D_k"], info["grid"], coef, local_only=True)
    for p in [(2, 2), (0, 2), (1, 2)]:
        assert np.max(np.abs(H[p])) < 1e-12
    lhs = 2 * (H[(0, 0)] * H[(1, 1)] - H[(0, 1)] ** 2) + coef["alpha"] * (H[(0, 0)] + H[(1, 1)])
    assert np.max(np.abs(lhs - coef["s"] * (d - d.mean()))) < 1e-10
    eta = coef["eta"]
    assert coef["alpha"] ** 2 + 6 * (eta - 1) / eta * (-1.0) > 0


def test_grh_phi_is_comoving_poisson():
    """Eq. GRPoisson in code units (H0 = 1): lap phi = (3/2) Om0 / a delta."""
    n, box, a = 16, 80.0, 0.25
    d = np.random.default_rng(2).standard_normal((n, n, n))
    phi, g, _, _ = field.solve_phi(d, a, box, OM, 1.0, gravity="grh")
    grid = field.KGrid(n, box)
    want = -1.5 * OM / a * fft3(d) / grid.k2_safe
    want[grid.zero] = 0
    assert np.max(np.abs(phi - ifft3_real(want))) < 1e-12 * np.max(np.abs(phi))


def test_force_is_minus_gradient_of_phi_single_mode():
    n, box, a = 16, 80.0, 0.4
    i = np.arange(n)
    m = 3
    d = 0.2 * np.cos(2 * np.pi * m * i / n)[None, :, None] * np.ones((n, n, n))
    phi, g, _, _ = field.solve_phi(d, a, box, OM, 1.0, tol=1e-13)
    k = 2 * np.pi * m / box
    amp = phi[0, 0, 0]  # phi = amp cos(k y)
    y = i * box / n
    want = amp * k * np.sin(k * y)[None, :, None] * np.ones((n, n, n))  # -d/dy
    assert np.max(np.abs(g[1] - want)) < 1e-12 * abs(amp * k)
    assert np.max(np.abs(g[0])) < 1e-14 and np.max(np.abs(g[2])) < 1e-14


def test_spherical_mode_local_is_sphpoi():
    """Sec. IV: with the nonlocal terms dropped, phi of the spherical mode obeys
    Eq. SphPoi pointwise (for the mean-free density the solver sees)."""
    n, box, a = 16, 50.0, 0.4
    rng = np.random.default_rng(3)
    d = rng.uniform(0.0, 1.6, (n, n, n))  # delta - mean >= -1: no bad points for w = 1/3 (Sec. III.C)
    phi, g, D, info = field.solve_phi(d, a, box, OM, 1.0, local_only=True, gravity="sph")
    coef = bg.coefficients(a, OM, 1.0)
    eta, alpha, E = coef["eta"], coef["alpha"], coef["E"]
    assert info["bad"] == [0]
    dm = d - d.mean()
    sph = 1.5 * (eta - 1) / eta * dm - (1 / (2 * eta)) * (3 * alpha / 4) * (
        np.sqrt(1 + 8 / alpha ** 2 * (eta - 1) / eta * dm) - 1)
    grid = field.KGrid(n, box)
    lap = -grid.k2 * fft3(phi) / (a * E) ** 2   # = FFT of lapbar^2 phi in these units
    want = fft3(sph)
    want[grid.zero] = 0.0
    assert np.max(np.abs(lap - want)) < 1e-10 * np.max(np.abs(want))


def test_spherical_mode_is_first_w13_update_with_nonlocal_source():
    """Sec. IV: including the nonlocal terms, the spherical D is the first
    iterate of the full w = 1/3 FFT-relaxation started from C = 0."""
    n, box, a = 16, 50.0, 0.3
    d, _ = inputs.linear_field(n, box, -1.5, 0.2, seed=4)  # min delta > -1: no bad points
    coef = bg.coefficients(a, OM, 1.0)
    grid = field.KGrid(n, box)
    dk = fft3(d)
    dk[grid.zero] = 0
    Dsph, _, nbad = field.spherical_D(dk, grid, coef)
    D1, info = field.solve_brane_bending(d, a, box, OM, 1.0, D_init=np.zeros_like(d), max_iter=1, tol=0.0)
    assert nbad == 0 and info["iters"] == 1  # the update lowered the residual of C = 0
    assert np.max(np.abs(D1 - Dsph)) < 1e-13 * np.max(np.abs(Dsph))


def test_large_crossover_scale_tends_to_gr():
    """r_c -> infinity (eta = r_c H -> infinity): alpha -> 3, beta -> 1, c2 -> 3/2, c3 -> 0 and
    Eq. FullDGP1 becomes the GR Poisson equation, so the nonlinear DGP phi approaches the GR phi
    of the same expansion history with a difference falling as 1/r_c (Sec. II)."""
    n, box, a = 16, 100.0, 0.5
    d, _ = inputs.linear_field(n, box, -1.5, 0.5, seed=3)
    diffs = []
    for rc in (1e2, 1e3, 1e4):
        c = bg.coefficients(a, OM, rc)
        assert abs(c["alpha"] - 3.0) < 2.0 / c["eta"] and abs(c["beta"] - 1.0) < 1.0 / c["eta"]
        assert abs(c["c2"] - 1.5) < 2.0 / c["eta"] and abs(c["c3"]) < 1.0 / c["eta"]
        p_nl = field.solve_phi(d, a, box, OM, rc, tol=1e-12)[0]
        p_gr = field.solve_phi(d, a, box, OM, rc, gravity="grh")[0]
        diffs.append(np.linalg.norm(p_nl - p_gr) / np.linalg.norm(p_gr))
    assert diffs[0] < 1e-2
    for lo, hi in zip(diffs[1:], diffs[:-1]):
        assert 9.0 < hi / lo < 11.0
