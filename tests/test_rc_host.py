"""Host side of the derivatives in r_c H0: dgp_velocity_factor (complex-step differentiation of
the library's growth ODE) against the oracle's RK4 sensitivity equations (pinned by central
differences in test_oracle_adjoint.py)."""
import pytest

from oracle import background as obg
from paper_0906_4548_gb300 import dgp

OM = 0.27


@pytest.mark.parametrize("a,rc", [(0.02, 1.0), (0.3, 0.7), (1.0, 2.0), (0.05, 0.5)])
def test_velocity_factor_and_derivative(a, rc):
    vf, dvf = dgp.dgp_velocity_factor(OM, rc, a)
    ovf, odvf = obg.zeldovich_velocity_factor_drc(a, OM, rc)
    assert abs(vf - ovf) < 1e-13 * ovf
    assert abs(dvf - odvf) < 1e-11 * abs(odvf)


def test_velocity_factor_rejects_bad_arguments():
    for a, rc in ((0.0, 1.0), (0.5, 0.0), (-1.0, 1.0)):
        with pytest.raises(dgp.DgpError):
            dgp.dgp_velocity_factor(OM, rc, a)


@pytest.mark.parametrize("a0,a1,rc", [(0.02, 0.0204, 1.0), (0.3, 0.35, 0.7), (0.9, 1.0, 2.0)])
def test_time_factors_and_derivatives_match_the_oracle(a0, a1, rc):
    """The library's kick and drift factors (the ones pm_step uses) and their complex-step
    derivatives against the oracle's quadrature and its chain-rule derivatives."""
    k, dr, dk, ddr = dgp.dgp_time_factors(OM, rc, a0, a1)
    assert abs(k - obg.kick_factor(a0, a1, OM, rc)) < 1e-14 * abs(k)
    assert abs(dr - obg.drift_factor(a0, a1, OM, rc)) < 1e-14 * abs(dr)
    assert abs(dk - obg.kick_factor_drc(a0, a1, OM, rc)) < 1e-11 * abs(dk)
    assert abs(ddr - obg.drift_factor_drc(a0, a1, OM, rc)) < 1e-11 * abs(ddr)


def test_time_factors_reject_bad_arguments():
    for a0, a1, rc in ((0.0, 0.5, 1.0), (0.5, float("inf"), 1.0), (0.5, 0.6, -1.0)):
        with pytest.raises(dgp.DgpError):
            dgp.dgp_time_factors(OM, rc, a0, a1)


@pytest.mark.parametrize("a,rc", [(0.5, 1.2), (0.05, 0.8), (1.0, 2.5)])
def test_coefficient_derivatives_match_the_oracle(a, rc):
    """The library's complex-step derivatives of the coefficients (the scalars of the r_c
    contraction) against the oracle's chain rule; growth f against the RK4 sensitivities."""
    d = dgp.dgp_background_drc(OM, rc, a)
    o = obg.coefficient_derivatives(a, OM, rc)
    for k in ("E", "eta", "alpha", "beta", "s", "c2", "c3", "q", "omega_m"):
        assert abs(d[k] - o[k]) < 1e-11 * abs(o[k]) + 1e-15, k
    _, _, dD, df = obg.growth_drc(a, OM, rc)
    assert abs(d["growth_D"] - dD) < 1e-10 * abs(dD)
    assert abs(d["growth_f"] - df) < 1e-10 * abs(df)
    h = 1e-6 * rc   # geff_local has no oracle derivative: central differences of the library's value
    fd = (dgp.dgp_background(OM, rc + h, a)["geff_local"] - dgp.dgp_background(OM, rc - h, a)["geff_local"]) / (2 * h)
    assert abs(d["geff_local"] - fd) < 1e-6 * abs(fd)
