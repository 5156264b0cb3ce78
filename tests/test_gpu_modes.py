"""Gravity modes and diagnostics beyond the default path, through the C ABI,
against the FP64 oracle: the spherical approximation (Sec. IV), the spectra of
the brane-bending mode (Eqs. cdef, DGradC) and the linear-to-nonlinear switch
epoch of the time evolution (Sec. III.D)."""
import math

import numpy as np
import pytest

from oracle import estimators as oest
from oracle import field as ofield
from oracle import pm as opm
from paper_0906_4548_gb300 import inputs

from test_gpu_parity import OM, np_dtype, prec_dtype, rel_l2, to_dev, zel  # noqa: F401
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,prec,local_only,tol", [(32, 2, False, 1e-10), (32, 1, False, 1e-5),
                                                   (64, 3, True, 1e-5), (32, 0, False, 1e-5)])
def test_spherical_mode_parity(dgp, torch_dev, n, prec, local_only, tol):
    torch, dev = torch_dev
    box, a = 100.0, 0.5
    pos, _, _ = zel(n, box, a, -1.5, 0.8, 12)
    delta = opm.density_contrast(opm.cic_deposit(pos, n, box)).astype(np_dtype(prec, dgp))
    phi_o, g_o, D_o, info_o = ofield.solve_phi(delta.astype(np.float64), a, box, OM, 1.0, local_only=local_only,
                                               gravity="sph")
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec, gravity=dgp.DGP_GRAVITY_SPH, local_only=local_only)
    try:
        dd = to_dev(torch_dev, delta, prec_dtype(torch, prec, dgp))
        phi = torch.empty_like(dd)
        g = [torch.empty_like(dd) for _ in range(3)]
        st, info = dgp.dgp_solve_forces(ctx, a, dd, phi, *g, 0.0)
    finally:
        dgp.dgp_destroy(ctx)
    assert st == dgp.DGP_OK and info["iters"] == 1
    # the bad-point test Delta < 0 is taken in the kernel's precision: exact for FP64
    nbad = round(info["bad_fraction"] * n ** 3)
    assert nbad == info_o["bad"][0] if prec == dgp.DGP_FP64 else abs(nbad - info_o["bad"][0]) <= 2
    assert rel_l2(phi.cpu().numpy(), phi_o) < tol
    for i in range(3):
        assert rel_l2(g[i].cpu().numpy(), g_o[i]) < tol


@pytest.mark.parametrize("n,prec,tol", [(32, 2, 1e-9), (64, 3, 2e-5)])
def test_brane_spectra_parity(dgp, torch_dev, n, prec, tol):
    torch, dev = torch_dev
    box, a = 200.0, 0.7
    pos, _, _ = zel(n, box, a, -1.5, 0.8, 5)
    delta = opm.density_contrast(opm.cic_deposit(pos, n, box)).astype(np_dtype(prec, dgp))
    _, _, D_o, info_o = ofield.solve_phi(delta.astype(np.float64), a, box, OM, 1.0, tol=1e-12)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec, tol=1e-10 if prec == 2 else 1e-6)
    try:
        with pytest.raises(dgp.DgpError):
            dgp.dgp_brane_spectra(ctx, n // 2)  # no solution yet
        dd = to_dev(torch_dev, delta, prec_dtype(torch, prec, dgp))
        dgp.dgp_solve_phi(ctx, a, dd, None, 1e-10 if prec == 2 else 1e-6)
        k, pc, pC, dl, nm = dgp.dgp_brane_spectra(ctx, n // 2)
    finally:
        dgp.dgp_destroy(ctx)
    ko, pco, pCo, dlo, nmo = oest.brane_spectra(D_o, a, box, OM, 1.0)
    assert np.array_equal(nm, nmo)
    assert np.allclose(k, ko, rtol=1e-12)
    for got, want in ((pc, pco), (pC, pCo), (dl, dlo)):
        assert np.max(np.abs(got / want - 1)) < tol


def test_pm_run_with_linear_switch_matches_oracle(dgp, torch_dev):
    """FP64, 32^3, six steps from a = 0.08 to 0.16 with the nonlinear solve from a = 0.11."""
    torch, dev = torch_dev
    n, box, a0, a1, ns, a_nl = 32, 100.0, 0.08, 0.16, 6, 0.11
    pos, mom, _ = zel(n, box, a0, -2.0, 0.5, 3)
    st = opm.run(pos, mom, a0, a1, ns, n, box, OM, 1.0, tol=1e-10, max_iter=300, a_nonlinear=a_nl)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64, tol=1e-10, max_iter=300, a_nonlinear=a_nl)
    iters = []
    try:
        t = [to_dev(torch_dev, v, torch.float64) for v in (*pos, *mom)]
        parts = dgp.particles(*t)
        a = a0
        dl = (math.log(a1) - math.log(a0)) / ns
        for i in range(ns):
            a_next = a0 * math.exp((i + 1) * dl)
            iters.append(dgp.pm_step(ctx, parts, a, a_next - a)["iters"])
            a = a_next
        x = np.stack([v.cpu().numpy() for v in t[:3]])
        p = np.stack([v.cpu().numpy() for v in t[3:]])
    finally:
        dgp.dgp_destroy(ctx)
    assert rel_l2(x, st.pos) < 1e-12 and rel_l2(p, st.mom) < 1e-9
    # the step infos describe the solve at the step's end: linear before a_nl
    ends = [a0 * math.exp((i + 1) * (math.log(a1) - math.log(a0)) / ns) for i in range(ns)]
    assert all((it == 0) == (ae < a_nl) for it, ae in zip(iters, ends))
