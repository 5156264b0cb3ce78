"""DGP background and the scalar coefficients of the field equations (oracle).

Test infrastructure: see ``oracle/__init__.py``.

Units: lengths in Mpc/h, time in 1/H0 (so H0 = 1), c/H0 = C_H Mpc/h.

Sec. II, Eq. DGPFriedmann:  H^2 = H / r_c + (8 pi G / 3) rho_m.
With E = H/H0, eps = 1/(r_c H0) and rho_m proportional to a^-3 this is the
quadratic E^2 - eps E - Omega_m0 a^-3 = 0, whose self-accelerating root is
E = [eps + sqrt(eps^2 + 4 Omega_m0 a^-3)] / 2.  r_c H0 is an input; the
paper's flat relation r_c H0 = 1/(1 - Omega_m0) (Sec. II) is one choice of it.

Coefficients (Sec. II, Eqs. FullDGP1, FullDGP2 and the definitions of eta,
alpha, beta, q that follow them):
    eta   = r_c H
    alpha = 3 (2 eta^2 - 2 eta + 1) / (eta (2 eta - 1))
    beta  = (2 eta^2 - 2 eta - 1) / (eta (2 eta - 1))
    s     = 3 (eta - 1) / eta                     (RHS factor of FullDGP2)
    c2    = 3 beta (eta - 1) / (2 eta - 1)        (sqrt(-lap) C term of FullDGP2)
    c3    = (3 eta^2 - 5 eta + 1) / (2 eta^2 (2 eta - 1))   (same term of FullDGP1)
    q     = (2 - eta) / (2 eta - 1)               (acceleration parameter)
"""

import math

import numpy as np

C_H = 2997.92458  # c / H0 in Mpc/h


def hubble_E(a, omega_m0, rc_H0):
    """E(a) = H/H0, self-accelerating root of Eq. DGPFriedmann."""
    eps = 1.0 / rc_H0
    return 0.5 * (eps + np.sqrt(eps * eps + 4.0 * omega_m0 * np.asarray(a, float) ** -3))


def eta_of_a(a, omega_m0, rc_H0):
    """eta = r_c H (Sec. II)."""
    return rc_H0 * hubble_E(a, omega_m0, rc_H0)


def coefficients(a, omega_m0, rc_H0):
    """All scalar coefficients at scale factor ``a`` as a dict (Sec. II)."""
    E = float(hubble_E(a, omega_m0, rc_H0))
    eta = rc_H0 * E
    den = eta * (2.0 * eta - 1.0)
    alpha = 3.0 * (2.0 * eta * eta - 2.0 * eta + 1.0) / den
    beta = (2.0 * eta * eta - 2.0 * eta - 1.0) / den
    s = 3.0 * (eta - 1.0) / eta
    c2 = 3.0 * beta * (eta - 1.0) / (2.0 * eta - 1.0)
    c3 = (3.0 * eta * eta - 5.0 * eta + 1.0) / (2.0 * eta * eta * (2.0 * eta - 1.0))
    q = (2.0 - eta) / (2.0 * eta - 1.0)
    return dict(a=float(a), E=E, eta=eta, alpha=alpha, beta=beta, s=s, c2=c2, c3=c3, q=q,
                omega_m=omega_m0 * float(a) ** -3 / (E * E))


def geff_over_G(k, a, omega_m0, rc_H0):
    """Linearised G_eff/G of Eq. Geff (Sec. II); k in h/Mpc.

    (G_eff/G)^-1 = [2 eta (2+q) - 3] / [2 eta (2+q) - 4]
                   + (3 a / (k r_c)) ([eta (1+q) - 1] / [eta (2+q) - 2])^2
    with r_c = rc_H0 * c/H0 in Mpc/h.
    """
    c = coefficients(a, omega_m0, rc_H0)
    eta, q = c["eta"], c["q"]
    rc = rc_H0 * C_H
    inv = (2 * eta * (2 + q) - 3) / (2 * eta * (2 + q) - 4) \
        + (3.0 * a / (np.asarray(k, float) * rc)) * ((eta * (1 + q) - 1) / (eta * (2 + q) - 2)) ** 2
    return 1.0 / inv


def geff_local_over_G(a, omega_m0, rc_H0):
    """k -> infinity limit of Eq. Geff (first term only)."""
    c = coefficients(a, omega_m0, rc_H0)
    eta, q = c["eta"], c["q"]
    return (2 * eta * (2 + q) - 4) / (2 * eta * (2 + q) - 3)


def w_zero_discriminant(a, omega_m0, rc_H0):
    """Eq. ZeroDis (Sec. III.C): w that zeroes Delta at delta = -1 with no C terms."""
    c = coefficients(a, omega_m0, rc_H0)
    eta, alpha = c["eta"], c["alpha"]
    return 1.0 - alpha * alpha * eta / (12.0 * (eta - 1.0))


def discriminant_C_free(a, omega_m0, rc_H0, w, delta=-1.0):
    """C-independent part of Delta, Eq. NewDis (Eq. Discweq0 at w = 0):
    alpha^2 + 4 (1 - w) 3 (eta - 1)/eta delta   (Fig. 2 plots it at delta = -1)."""
    c = coefficients(a, omega_m0, rc_H0)
    return c["alpha"] ** 2 + 4.0 * (1.0 - w) * c["s"] * delta


def _dlnE_dlna(a, omega_m0, rc_H0):
    # differentiate E^2 - eps E - Om a^-3 = 0 implicitly in ln a:
    # (2E - eps) dE/dlna = -3 Om a^-3
    eps = 1.0 / rc_H0
    E = float(hubble_E(a, omega_m0, rc_H0))
    return -3.0 * omega_m0 * a ** -3 / ((2.0 * E - eps) * E)


def growth(a_out, omega_m0, rc_H0, geff="local", a_start=1e-5, steps_per_efold=400):
    """Linear growth D+ and rate f = dlnD+/dlna at ``a_out``.

    ODE in ln a:  D'' + (2 + dlnE/dlna) D' = (3/2) Omega_m(a) (G_eff/G) D,
    which is the linearised form of the particle equations of Sec. III.A with
    the linearised Poisson equation Eq. LinearDGP (k -> infinity limit of
    Eq. Geff for ``geff="local"``, G_eff = G for ``geff="GR"``).  Started on the
    growing mode D = a, D' = a deep in matter domination; classical RK4 with a
    fixed step in ln a.  Returns (D+(a_out), f(a_out)) with D+ normalised to
    D+ = a at a_start.
    """
    def rhs(lna, y):
        a = math.exp(lna)
        c = coefficients(a, omega_m0, rc_H0)
        g = geff_local_over_G(a, omega_m0, rc_H0) if geff == "local" else 1.0
        D, dD = y
        return np.array([dD, -(2.0 + _dlnE_dlna(a, omega_m0, rc_H0)) * dD
                         + 1.5 * c["omega_m"] * g * D])

    x0, x1 = math.log(a_start), math.log(a_out)
    n = max(1, int(math.ceil((x1 - x0) * steps_per_efold)))
    h = (x1 - x0) / n
    y = np.array([a_start, a_start])
    x = x0
    for _ in range(n):
        k1 = rhs(x, y)
        k2 = rhs(x + 0.5 * h, y + 0.5 * h * k1)
        k3 = rhs(x + 0.5 * h, y + 0.5 * h * k2)
        k4 = rhs(x + h, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        x += h
    return float(y[0]), float(y[1] / y[0])


def zeldovich_velocity_factor(a, omega_m0, rc_H0, geff="local"):
    """p = a^2 dx/dt = a^2 E f Psi for Zel'dovich displacements Psi (Sec. III.A
    variables: dx/dt = u, so u = f H Psi for a growing-mode displacement)."""
    _, f = growth(a, omega_m0, rc_H0, geff)
    return a * a * float(hubble_E(a, omega_m0, rc_H0)) * f


def _gauss_legendre(fn, x0, x1, order=8):
    t, wts = np.polynomial.legendre.leggauss(order)
    xm, xr = 0.5 * (x1 + x0), 0.5 * (x1 - x0)
    return xr * float(np.sum(wts * np.array([fn(xm + xr * ti) for ti in t])))


def kick_factor(a0, a1, omega_m0, rc_H0):
    """int_{ln a0}^{ln a1} dlna / E(a): p = a^2 dx/dt obeys dp/dlna = -grad(phi)/E
    (Sec. III.A: du/dt = -2 H u - grad(phi)/a^2)."""
    return _gauss_legendre(lambda x: 1.0 / float(hubble_E(math.exp(x), omega_m0, rc_H0)),
                           math.log(a0), math.log(a1))


def drift_factor(a0, a1, omega_m0, rc_H0):
    """int_{ln a0}^{ln a1} dlna / (a^2 E(a)): dx/dlna = p / (a^2 E) (Sec. III.A)."""
    return _gauss_legendre(
        lambda x: 1.0 / (math.exp(2 * x) * float(hubble_E(math.exp(x), omega_m0, rc_H0))),
        math.log(a0), math.log(a1))


# ---------------------------------------------------------------- derivatives in r_c H0
# d/d(r_c H0) of the quantities above, written out by the chain rule (the
# gradient of a loss with respect to the crossover scale goes through E(a),
# eta = r_c H and every coefficient of Eqs. FullDGP1-2).

def hubble_E_drc(a, omega_m0, rc_H0):
    """dE/d(r_c H0): differentiating E^2 - eps E - Om a^-3 = 0 with eps = 1/(r_c H0)
    gives (2E - eps) dE = E d eps, d eps = -d(r_c H0) / (r_c H0)^2."""
    E = float(hubble_E(a, omega_m0, rc_H0))
    eps = 1.0 / rc_H0
    return -E / (rc_H0 * rc_H0 * (2.0 * E - eps))


def coefficient_derivatives(a, omega_m0, rc_H0):
    """d/d(r_c H0) of E, eta, alpha, beta, s, c2, c3, q and Omega_m(a), as a dict
    with the same keys as coefficients()."""
    c = coefficients(a, omega_m0, rc_H0)
    E, eta, beta = c["E"], c["eta"], c["beta"]
    dE = hubble_E_drc(a, omega_m0, rc_H0)
    deta = E + rc_H0 * dE
    den = 2.0 * eta * eta - eta            # eta (2 eta - 1)
    dden = 4.0 * eta - 1.0
    a_num, b_num = 2.0 * eta * eta - 2.0 * eta + 1.0, 2.0 * eta * eta - 2.0 * eta - 1.0
    dalpha = 3.0 * ((4.0 * eta - 2.0) * den - a_num * dden) / (den * den)
    dbeta = ((4.0 * eta - 2.0) * den - b_num * dden) / (den * den)
    ds = 3.0 / (eta * eta)
    t = 2.0 * eta - 1.0
    dc2 = 3.0 * (dbeta * (eta - 1.0) / t + beta / (t * t))
    c3_num, c3_den = 3.0 * eta * eta - 5.0 * eta + 1.0, 4.0 * eta ** 3 - 2.0 * eta * eta
    dc3 = ((6.0 * eta - 5.0) * c3_den - c3_num * (12.0 * eta * eta - 4.0 * eta)) / (c3_den * c3_den)
    dq = -3.0 / (t * t)
    out = dict(E=dE, eta=deta, alpha=dalpha * deta, beta=dbeta * deta, s=ds * deta, c2=dc2 * deta,
               c3=dc3 * deta, q=dq * deta, omega_m=-2.0 * c["omega_m"] * dE / E)
    return out


def kick_factor_drc(a0, a1, omega_m0, rc_H0):
    """d/d(r_c H0) of kick_factor: the same 8-point rule applied to -E'/E^2."""
    def fn(x):
        a = math.exp(x)
        E = float(hubble_E(a, omega_m0, rc_H0))
        return -hubble_E_drc(a, omega_m0, rc_H0) / (E * E)
    return _gauss_legendre(fn, math.log(a0), math.log(a1))


def drift_factor_drc(a0, a1, omega_m0, rc_H0):
    """d/d(r_c H0) of drift_factor: the same 8-point rule applied to -E'/(a^2 E^2)."""
    def fn(x):
        a = math.exp(x)
        E = float(hubble_E(a, omega_m0, rc_H0))
        return -hubble_E_drc(a, omega_m0, rc_H0) / (a * a * E * E)
    return _gauss_legendre(fn, math.log(a0), math.log(a1))


def growth_drc(a_out, omega_m0, rc_H0, a_start=1e-5, steps_per_efold=400):
    """(D+, f, dD+/d(r_c H0), df/d(r_c H0)) with the local G_eff: the growth ODE of
    growth() integrated together with its sensitivity equations
        z' = (dF/dy) z + dF/d(r_c H0),  z = dy/d(r_c H0),  z(a_start) = 0,
    by the same classical RK4 steps (forward-mode differentiation of the RK4 map)."""
    eps = 1.0 / rc_H0

    def rhs(lna, y):
        a = math.exp(lna)
        c = coefficients(a, omega_m0, rc_H0)
        dc = coefficient_derivatives(a, omega_m0, rc_H0)
        E, eta, q = c["E"], c["eta"], c["q"]
        G = (2.0 * E - eps) * E
        dG = (2.0 * dc["E"] + eps * eps) * E + (2.0 * E - eps) * dc["E"]   # d eps = -eps^2
        L = -3.0 * omega_m0 * a ** -3 / G
        dL = 3.0 * omega_m0 * a ** -3 * dG / (G * G)
        u = 2.0 * eta * (2.0 + q)
        du = 2.0 * dc["eta"] * (2.0 + q) + 2.0 * eta * dc["q"]
        g = (u - 4.0) / (u - 3.0)
        dg = du / ((u - 3.0) ** 2)
        src = 1.5 * c["omega_m"] * g
        dsrc = 1.5 * (dc["omega_m"] * g + c["omega_m"] * dg)
        D, dD, zD, zdD = y
        return np.array([dD, -(2.0 + L) * dD + src * D,
                         zdD, -(2.0 + L) * zdD - dL * dD + src * zD + dsrc * D])

    x0, x1 = math.log(a_start), math.log(a_out)
    n = max(1, int(math.ceil((x1 - x0) * steps_per_efold)))
    h = (x1 - x0) / n
    y = np.array([a_start, a_start, 0.0, 0.0])
    x = x0
    for _ in range(n):
        k1 = rhs(x, y)
        k2 = rhs(x + 0.5 * h, y + 0.5 * h * k1)
        k3 = rhs(x + 0.5 * h, y + 0.5 * h * k2)
        k4 = rhs(x + h, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        x += h
    D, dD, zD, zdD = (float(v) for v in y)
    return D, dD / D, zD, (zdD * D - dD * zD) / (D * D)


def zeldovich_velocity_factor_drc(a, omega_m0, rc_H0):
    """(vf, dvf/d(r_c H0)) for vf = a^2 E f (local G_eff)."""
    _, f, _, df = growth_drc(a, omega_m0, rc_H0)
    E = float(hubble_E(a, omega_m0, rc_H0))
    return a * a * E * f, a * a * (hubble_E_drc(a, omega_m0, rc_H0) * f + E * df)
