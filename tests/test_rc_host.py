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
