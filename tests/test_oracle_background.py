"""Pins of the oracle's background cosmology and coefficients (Sec. II)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import background as bg

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("rc", [0.5, 1.0, 2.0, 1 / 0.73])
@pytest.mark.parametrize("a", [0.02, 0.05, 0.3, 1.0, 5.0])
def test_friedmann_equation_holds(a, rc):
    # Eq. DGPFriedmann with H0 = 1: E^2 = E / rc + Om a^-3
    E = float(bg.hubble_E(a, 0.27, rc))
    assert abs(E * E - E / rc - 0.27 * a ** -3) <= 1e-13 * E * E
    assert E > 1 / rc  # self-accelerating root: eta = rc E > 1


def test_de_sitter_limit():
    # Sec. II: when matter is diluted, H -> 1 / r_c
    assert abs(float(bg.hubble_E(1e4, 0.27, 1.3)) - 1 / 1.3) < 1e-9


def test_flat_relation_gives_E1_equal_1():
    # Sec. II: r_c H0 = 1/(1 - Om) is the relation that makes H(a=1) = H0
    assert abs(float(bg.hubble_E(1.0, 0.27, 1 / 0.73)) - 1.0) < 1e-14


@pytest.mark.parametrize("a", [0.04, 0.2, 0.7, 1.0])
def test_q_is_acceleration_parameter(a):
    # q = a a'' / a'^2 = 1 + dlnH/dlna ; compare Sec. II closed form by finite differences of E
    h = 1e-5
    dlnE = (math.log(bg.hubble_E(a * math.exp(h), 0.27, 1.0))
            - math.log(bg.hubble_E(a * math.exp(-h), 0.27, 1.0))) / (2 * h)
    c = bg.coefficients(a, 0.27, 1.0)
    assert abs((1 + dlnE) - c["q"]) < 1e-8


@pytest.mark.parametrize("a", [0.02, 0.5, 1.0])
def test_omega_m_is_eta_minus_one_over_eta(a):
    c = bg.coefficients(a, 0.27, 1.0)
    assert abs(c["omega_m"] - (c["eta"] - 1) / c["eta"]) < 1e-14


def test_w_zero_discriminant_paper_value():
    g = GOLD["w_zero_discriminant_z24"]
    om = g["omega_m0"]
    w = bg.w_zero_discriminant(1.0 / (1 + g["z"]), om, 1.0 / (1 - om))
    assert abs(w - g["value"]) <= g["abs_tol"]


def test_discriminant_sign_change_w0_and_w13_positive():
    g = GOLD["discriminant_w0_sign_change_z"]
    om = g["omega_m0"]
    rc = 1.0 / (1 - om)
    zs = np.linspace(0.0, 30.0, 3001)
    d0 = np.array([bg.discriminant_C_free(1 / (1 + z), om, rc, 0.0) for z in zs])
    d13 = np.array([bg.discriminant_C_free(1 / (1 + z), om, rc, 1 / 3) for z in zs])
    z_cross = zs[np.argmax(d0 < 0)]
    assert d0[0] > 0 and np.all(d0[zs > 1.2] < 0)
    assert abs(z_cross - g["value"]) <= g["abs_tol"]
    assert np.all(d13 > 0)


def test_geff_below_G_and_local_limit():
    for a in (0.1, 0.5, 1.0):
        c = bg.coefficients(a, 0.27, 1.0)
        eta = c["eta"]
        loc = bg.geff_local_over_G(a, 0.27, 1.0)
        # k -> infinity limit of Eq. Geff written with q eliminated
        assert abs(loc - 2 * (3 * eta ** 2 - 4 * eta + 2) / (3 * (2 * eta ** 2 - 2 * eta + 1))) < 1e-13
        ks = np.array([1e-3, 1e-2, 0.1, 10.0])
        ge = bg.geff_over_G(ks, a, 0.27, 1.0)
        assert np.all(ge < 1) and np.all(np.diff(ge) > 0) and abs(ge[-1] - loc) < 1e-4


def test_growth_eds_closed_form():
    # Om = 1 and r_c -> infinity: E = a^-3/2, D = a, f = 1 exactly
    D, f = bg.growth(0.5, 1.0, 1e12, geff="GR")
    assert abs(D - 0.5) < 1e-7 and abs(f - 1.0) < 1e-7


def test_kick_drift_eds_closed_forms():
    a0, a1 = 0.2, 0.31
    k = bg.kick_factor(a0, a1, 1.0, 1e12)
    d = bg.drift_factor(a0, a1, 1.0, 1e12)
    assert abs(k - (2 / 3) * (a1 ** 1.5 - a0 ** 1.5)) < 1e-13
    assert abs(d - 2 * (a0 ** -0.5 - a1 ** -0.5)) < 1e-12


def test_growth_suppressed_in_dgp():
    # Sec. III.A: with equal initial amplitude DGP ends with sigma8 0.715 vs 0.9 (ratio 0.79):
    # here only check the sign and the rough size of the suppression vs GR with the same H(a).
    Dd, _ = bg.growth(1.0, 0.27, 1 / 0.73, geff="local")
    Dg, _ = bg.growth(1.0, 0.27, 1 / 0.73, geff="GR")
    assert 0.8 < Dd / Dg < 0.95
