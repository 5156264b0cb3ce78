"""The arithmetic of the pointwise residual against the FP32 data's own floor (CPU).

The mixed arithmetic of the 256^3 workload evaluates the residual R of Eq. FullDGP2 in FP32 on
FP32 mesh fields.  On a strongly nonlinear state (an oracle run to a = 1, delta in the hundreds)
at the oracle's converged solution, this checks, with numpy's float32 arithmetic standing in
for the GPU's:
  * rounding the converged fields to FP32 already leaves a mean |R| of order 1e-8 of <|S|>,
    which no evaluation of R can go below;
  * evaluating R in FP32 (the order of the GPU's mixed policy) adds an error of the same order;
  * both stay far below the relaxation tolerance 1e-6 of the workloads;
  * summing q's products exactly and only its assembly in FP32, or the reverse, changes the
    error by less than a factor of two, so wider residual arithmetic buys nothing at 1e-6.
"""
import numpy as np
import pytest

from oracle import background as obg
from oracle import field as ofield
from oracle import pm as opm
from paper_0906_4548_gb300 import inputs

OM = 0.27


def f32(x):
    return np.asarray(x, np.float32)


def fma32(x, y, z):
    """float32 fused multiply-add: the product of two floats is exact in float64."""
    return f32(np.asarray(x, np.float64) * np.asarray(y, np.float64) + np.asarray(z, np.float64))


@pytest.fixture(scope="module")
def converged_state():
    n, box, a = 32, 50.0, 1.0
    vf = obg.zeldovich_velocity_factor(0.02, OM, 1.0)
    pos, mom, _ = inputs.zeldovich_particles(n, box, -1.5, 0.5, 7, vf)
    st = opm.run(pos, mom, 0.02, a, 12, n, box, OM, 1.0, tol=1e-7, max_iter=200)
    delta = opm.density_contrast(opm.cic_deposit(st.pos, n, box))
    D, info = ofield.solve_brane_bending(delta, a, box, OM, 1.0, tol=1e-12, max_iter=400)
    Dm, H, Nf = ofield.derived_fields(info["D_k"], info["grid"], info["coef"])
    return delta, Dm, H, Nf, info["S"], info["coef"]


def test_fp32_residual_sits_at_the_fp32_data_floor(converged_state):
    delta, D, H, Nf, S, coef = converged_state
    assert delta.max() > 50.0  # strongly nonlinear
    eps = np.mean(np.abs(S))
    al, c2 = coef["alpha"], coef["c2"]
    r_exact = np.mean(np.abs(ofield.residual(D, H, Nf, S, coef))) / eps
    assert r_exact < 1e-10  # the oracle's converged solution
    d, a, b = f32(D), f32(H[(0, 0)]), f32(H[(1, 1)])
    hxy, hxz, hyz, nn, s = f32(H[(0, 1)]), f32(H[(0, 2)]), f32(H[(1, 2)]), f32(Nf), f32(S)
    # R of the FP32 data, exactly (float64 products of floats are exact)
    d64, a64, b64 = (v.astype(np.float64) for v in (d, a, b))
    c64 = d64 - a64 - b64
    q64 = (hxy.astype(np.float64) ** 2 + hxz.astype(np.float64) ** 2 + hyz.astype(np.float64) ** 2
           - a64 * b64 - (a64 + b64) * c64)
    r_data = al * d64 - 2.0 * q64 + c2 * nn.astype(np.float64) - s.astype(np.float64)
    floor = np.mean(np.abs(r_data)) / eps
    # the GPU's FP32 evaluation (the same order of operations as the mixed policy)
    u = f32(a + b)
    c = f32(d - u)
    r = fma32(f32(-2 * hxy), hxy, f32(f32(-2 * hxz) * hxz))
    r = fma32(f32(-2 * hyz), hyz, fma32(np.float32(c2), nn, r))
    r32 = fma32(f32(2 * a), b, fma32(f32(2 * u), c, fma32(np.float32(al), d, f32(r - s))))
    err32 = np.mean(np.abs(r32.astype(np.float64) - r_data)) / eps
    # q in FP32, the assembly exact
    q32 = f32(f32(f32(hxy * hxy) + f32(hxz * hxz)) + f32(hyz * hyz))
    q32 = f32(f32(q32 - f32(a * b)) - f32(u * c))
    rq = al * d64 - 2.0 * q32.astype(np.float64) + c2 * nn.astype(np.float64) - s.astype(np.float64)
    errq = np.mean(np.abs(rq - r_data)) / eps
    assert 1e-9 < floor < 3e-7
    assert err32 < 3 * floor and err32 < 1e-7
    assert errq < 3 * floor and errq > err32 / 2
