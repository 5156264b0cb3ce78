"""Pins of the oracle's adjoint of the field solve (oracle/adjoint.py): finite
differences through the nonlinear solve, the transpose identity against a
finite-difference Jacobian of the forward residual, and the D = 0 limit."""
import numpy as np

from oracle import adjoint as adj
from oracle import background as bg
from oracle import field
from oracle.fft import fft3, ifft3_real
from paper_0906_4548_gb300 import inputs

OM = 0.27


def _mean_free(f):
    return f - f.mean()


def _converged(n, box, a, rms, seed):
    d, _ = inputs.linear_field(n, box, -1.5, rms, seed=seed)
    D, info = field.solve_brane_bending(d, a, box, OM, 1.0, tol=1e-13)  # no bad points at rms 0.25
    assert info["converged"]
    _, H, _ = field.derived_fields(info["D_k"], info["grid"], info["coef"])
    return d, D, H, info


def test_jt_is_the_transpose_of_the_residual_jacobian():
    """R is quadratic in D, so the central difference (R(D + e v) - R(D - e v)) / 2e is J v exactly
    (up to rounding); <u, J v> must equal <J^T u, v>."""
    n, box, a = 16, 60.0, 0.6
    d, D, H, info = _converged(n, box, a, 0.25, 3)
    grid, coef = info["grid"], info["coef"]
    S = info["S"]
    rng = np.random.default_rng(1)
    u, v = _mean_free(rng.standard_normal((n, n, n))), _mean_free(rng.standard_normal((n, n, n)))

    def R(Dx):
        Dm, Hx, Nx = field.derived_fields(fft3(Dx), grid, coef)
        return field.residual(Dm, Hx, Nx, S, coef)

    e = 1e-3 * np.max(np.abs(D))
    Jv = (R(D + e * v) - R(D - e * v)) / (2 * e)
    lhs = np.sum(u * Jv)
    rhs = np.sum(adj.jt_apply(u, D, H, grid, coef) * v)
    assert abs(lhs - rhs) < 1e-9 * (np.sum(np.abs(u * Jv)))


def test_adjoint_solve_at_zero_D_is_diagonal_in_k():
    """At D = 0 (every H_ij = 0), J^T = alpha + c2 N, i.e. lam(k) = g(k) / (alpha - c2 / kbar)."""
    n, box, a = 16, 40.0, 0.4
    grid = field.KGrid(n, box)
    coef = bg.coefficients(a, OM, 1.0)
    z = np.zeros((n, n, n))
    H = {p: z for p in field.PAIRS}
    g = _mean_free(np.random.default_rng(2).standard_normal((n, n, n)))
    lam, info = adj.solve_adjoint(z, H, g, grid, coef, tol=1e-14)
    assert info["converged"]
    ikb = field._kbar_inv(grid, coef, False)
    want = ifft3_real(np.where(grid.zero, 0.0, fft3(g) / (coef["alpha"] - coef["c2"] * ikb)))
    assert np.max(np.abs(lam - want)) < 1e-12 * np.max(np.abs(want))


def test_phi_vjp_matches_central_differences():
    n, box, a = 16, 60.0, 0.6
    d, _ = inputs.linear_field(n, box, -1.5, 0.25, seed=4)
    rng = np.random.default_rng(5)
    phibar = rng.standard_normal((n, n, n))
    dbar, info = adj.phi_vjp(d, a, box, OM, 1.0, phibar)
    assert info["adjoint"]["converged"]
    for seed in (6, 7):
        u = _mean_free(np.random.default_rng(seed).standard_normal((n, n, n)))
        e = 1e-4
        lp = np.sum(phibar * field.solve_phi(d + e * u, a, box, OM, 1.0, tol=1e-13)[0])
        lm = np.sum(phibar * field.solve_phi(d - e * u, a, box, OM, 1.0, tol=1e-13)[0])
        fd = (lp - lm) / (2 * e)
        assert abs(fd - np.sum(dbar * u)) < 1e-6 * abs(fd)


def test_force_cotangent_through_finite_differences():
    """L = sum_i <gbar_i, g_i(delta)>: phibar from the forces' transpose, then the solve's VJP."""
    n, box, a = 16, 60.0, 0.6
    d, _ = inputs.linear_field(n, box, -1.5, 0.25, seed=8)
    rng = np.random.default_rng(9)
    gbar = [rng.standard_normal((n, n, n)) for _ in range(3)]
    grid = field.KGrid(n, box)
    dbar, _ = adj.phi_vjp(d, a, box, OM, 1.0, adj.phibar_from_forces(gbar, grid))
    u = _mean_free(rng.standard_normal((n, n, n)))
    e = 1e-4

    def L(x):
        g = field.solve_phi(x, a, box, OM, 1.0, tol=1e-13)[1]
        return sum(np.sum(gbar[i] * g[i]) for i in range(3))

    fd = (L(d + e * u) - L(d - e * u)) / (2 * e)
    assert abs(fd - np.sum(dbar * u)) < 1e-6 * abs(fd)


# ---------------------------------------------------------------- particle side
from oracle import pm  # noqa: E402


def _particles(n, box, sig, seed):
    pos, mom = inputs.lattice_particles(n, box)
    rng = np.random.default_rng(seed)
    pos = (pos + rng.normal(0, sig * box / n, pos.shape)) % box
    mom = rng.normal(0, 0.5, pos.shape)
    return pos, mom


def test_deposit_vjp_central_differences():
    n, box = 8, 16.0
    pos, _ = _particles(n, box, 0.3, 1)
    rng = np.random.default_rng(2)
    rbar = rng.standard_normal((n, n, n))
    u = rng.standard_normal(pos.shape)
    e = 1e-7
    fd = (np.sum(rbar * pm.cic_deposit(pos + e * u, n, box)) - np.sum(rbar * pm.cic_deposit(pos - e * u, n, box))) / (2 * e)
    assert abs(fd - np.sum(adj.deposit_vjp(pos, n, box, rbar) * u)) < 1e-7 * abs(fd)


def test_gather_vjp_central_differences():
    n, box = 8, 16.0
    pos, _ = _particles(n, box, 0.3, 3)
    rng = np.random.default_rng(4)
    grids = [rng.standard_normal((n, n, n)) for _ in range(3)]
    fbar = rng.standard_normal(pos.shape)
    u = rng.standard_normal(pos.shape)
    dg = [rng.standard_normal((n, n, n)) for _ in range(3)]

    def L(x, gs):
        return sum(np.sum(fbar[i] * pm.cic_interpolate(gs[i], x, box)) for i in range(3))

    Gbar, xbar = adj.gather_vjp(grids, pos, box, fbar)
    e = 1e-7
    fd_x = (L(pos + e * u, grids) - L(pos - e * u, grids)) / (2 * e)
    assert abs(fd_x - np.sum(xbar * u)) < 1e-7 * abs(fd_x)
    fd_g = (L(pos, [g + e * h for g, h in zip(grids, dg)]) - L(pos, [g - e * h for g, h in zip(grids, dg)])) / (2 * e)
    assert abs(fd_g - sum(np.sum(Gbar[i] * dg[i]) for i in range(3))) < 1e-7 * abs(fd_g)


def test_force_vjp_central_differences():
    """Particle forces through deposit, density contrast, the nonlinear solve and the gather."""
    n, box, a = 16, 80.0, 0.5
    pos, _ = _particles(n, box, 0.25, 5)
    rng = np.random.default_rng(6)
    fbar = rng.standard_normal(pos.shape)
    u = rng.standard_normal(pos.shape)

    def L(x):
        st = pm.PMState(x, np.zeros_like(x), a, n, box, OM, 1.0, tol=1e-13)
        return np.sum(fbar * st.forces_at_particles())

    e = 1e-5
    fd = (L(pos + e * u) - L(pos - e * u)) / (2 * e)
    got = np.sum(adj.force_vjp(pos, a, n, box, OM, 1.0, fbar) * u)
    assert abs(fd - got) < 1e-6 * abs(fd)


def test_step_vjp_central_differences():
    n, box, a, da = 16, 80.0, 0.5, 0.02
    pos, mom = _particles(n, box, 0.25, 7)
    rng = np.random.default_rng(8)
    xb1, pb1 = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    u, v = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)

    def L(x, p):
        st = pm.PMState(x, p, a, n, box, OM, 1.0, tol=1e-13)
        st.step(da)
        # positions enter through their increments (x1 - x0 is smooth; the wrap is not)
        return np.sum(xb1 * ((st.pos - x + box / 2) % box)) + np.sum(pb1 * st.mom)

    xb0, pb0 = adj.step_vjp(pos, mom, a, da, xb1, pb1, n, box, OM, 1.0)
    e = 1e-5
    fd = (L(pos + e * u, mom + e * v) - L(pos - e * u, mom - e * v)) / (2 * e)
    got = np.sum((xb0 - xb1) * u) + np.sum(pb0 * v)
    assert abs(fd - got) < 1e-6 * abs(fd)


def test_pk_vjp_central_differences():
    from oracle import estimators as est
    n, box, nb = 16, 60.0, 8
    d, _ = inputs.linear_field(n, box, -1.5, 0.5, seed=11)
    rng = np.random.default_rng(12)
    w, target = rng.uniform(0.5, 1.5, nb), rng.uniform(0.5, 1.5, nb) * est.power_spectrum(d, box, nb)[1]

    def L(x):
        P = est.power_spectrum(x, box, nb)[1]
        return np.sum(w * (P - target) ** 2)

    P = est.power_spectrum(d, box, nb)[1]
    dbar = adj.pk_vjp(d, box, nb, 2 * w * (P - target))
    u = rng.standard_normal((n, n, n))
    e = 1e-5
    fd = (L(d + e * u) - L(d - e * u)) / (2 * e)
    assert abs(fd - np.sum(dbar * u)) < 1e-7 * abs(fd)


def test_zeldovich_vjp_central_differences():
    n, box, vf = 16, 60.0, 0.7
    d, _ = inputs.linear_field(n, box, -1.5, 0.3, seed=13)
    rng = np.random.default_rng(14)
    xb, pb = rng.standard_normal((3, n ** 3)), rng.standard_normal((3, n ** 3))
    u = rng.standard_normal((n, n, n))
    e = 1e-6

    def L(x):
        pos, mom = inputs.zeldovich_from_field(x, box, vf)
        q, _ = inputs.lattice_particles(n, box)
        return np.sum(xb * ((pos - q + box / 2) % box)) + np.sum(pb * mom)

    fd = (L(d + e * u) - L(d - e * u)) / (2 * e)
    assert abs(fd - np.sum(adj.zeldovich_vjp(xb, pb, n, box, vf) * u)) < 1e-7 * abs(fd)


# ---------------------------------------------------------------- r_c H0
def test_background_derivatives_central_differences():
    """Chain-rule derivatives in r_c H0 against central differences of the pinned background."""
    for a, rc in ((0.5, 1.2), (0.05, 0.8), (1.0, 2.5)):
        d = bg.coefficient_derivatives(a, OM, rc)
        h = 1e-6 * rc
        cp, cm = bg.coefficients(a, OM, rc + h), bg.coefficients(a, OM, rc - h)
        for k in ("E", "eta", "alpha", "beta", "s", "c2", "c3", "q", "omega_m"):
            fd = (cp[k] - cm[k]) / (2 * h)
            assert abs(d[k] - fd) < 1e-7 * abs(fd) + 1e-12, k
        for f, df in ((bg.kick_factor, bg.kick_factor_drc), (bg.drift_factor, bg.drift_factor_drc)):
            fd = (f(a * 0.9, a, OM, rc + h) - f(a * 0.9, a, OM, rc - h)) / (2 * h)
            assert abs(df(a * 0.9, a, OM, rc) - fd) < 1e-7 * abs(fd)


def test_velocity_factor_derivative_central_differences():
    """d(a^2 E f)/d(r_c H0) from the RK4 sensitivity equations against differences of the
    growth ODE itself; the value matches zeldovich_velocity_factor."""
    for a, rc in ((0.02, 1.0), (0.5, 0.7)):
        vf, dvf = bg.zeldovich_velocity_factor_drc(a, OM, rc)
        assert abs(vf - bg.zeldovich_velocity_factor(a, OM, rc)) < 1e-14 * vf
        h = 1e-4 * rc
        fd = (bg.zeldovich_velocity_factor(a, OM, rc + h) - bg.zeldovich_velocity_factor(a, OM, rc - h)) / (2 * h)
        assert abs(dvf - fd) < 1e-6 * abs(fd)


def test_phi_vjp_rc_central_differences():
    """d<phibar, phi>/d(r_c H0) through the converged nonlinear solve (delta fixed)."""
    n, box, a, rc = 16, 60.0, 0.6, 1.0
    d, _ = inputs.linear_field(n, box, -1.5, 0.25, seed=4)
    phibar = np.random.default_rng(15).standard_normal((n, n, n))
    _, info = adj.phi_vjp(d, a, box, OM, rc, phibar)
    h = 1e-5
    lp = np.sum(phibar * field.solve_phi(d, a, box, OM, rc + h, tol=1e-13)[0])
    lm = np.sum(phibar * field.solve_phi(d, a, box, OM, rc - h, tol=1e-13)[0])
    fd = (lp - lm) / (2 * h)
    assert abs(fd - info["rcbar"]) < 1e-6 * abs(fd)


def test_step_vjp_rc_central_differences():
    n, box, a, da, rc = 16, 80.0, 0.5, 0.02, 1.0
    pos, mom = _particles(n, box, 0.25, 7)
    rng = np.random.default_rng(16)
    xb1, pb1 = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)

    def L(r):
        st = pm.PMState(pos, mom, a, n, box, OM, r, tol=1e-13)
        st.step(da)
        return np.sum(xb1 * ((st.pos - pos + box / 2) % box)) + np.sum(pb1 * st.mom)

    xb0, pb0, rcbar = adj.step_vjp(pos, mom, a, da, xb1, pb1, n, box, OM, rc, with_rc=True)
    xr, pr = adj.step_vjp(pos, mom, a, da, xb1, pb1, n, box, OM, rc)
    assert np.array_equal(xb0, xr) and np.array_equal(pb0, pr)
    h = 1e-5
    fd = (L(rc + h) - L(rc - h)) / (2 * h)
    assert abs(fd - rcbar) < 1e-6 * abs(fd)


def test_zeldovich_vf_bar_central_differences():
    n, box, vf = 16, 60.0, 0.7
    d, _ = inputs.linear_field(n, box, -1.5, 0.3, seed=13)
    pb = np.random.default_rng(17).standard_normal((3, n ** 3))
    e = 1e-6
    fd = (np.sum(pb * inputs.zeldovich_from_field(d, box, vf + e)[1])
          - np.sum(pb * inputs.zeldovich_from_field(d, box, vf - e)[1])) / (2 * e)
    assert abs(fd - adj.zeldovich_vf_bar(pb, d, box)) < 1e-7 * abs(fd)
