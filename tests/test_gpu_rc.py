"""Derivatives in r_c H0 on the GPU (dgp_solve_adjoint_rc, pm_step_adjoint_rc,
dgp_zeldovich_vf_adjoint and the autograd chain) against the oracle's
(oracle/adjoint.py, oracle/background.py) and against central differences of GPU runs."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import background as obg
from oracle import field as ofield
from paper_0906_4548_gb300 import inputs

from test_gpu_parity import OM, rel_l2, to_dev  # noqa: F401
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)
from test_gpu_adjoint import _field, _particles

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,prec,rc,use_forces,tol", [(16, 2, 1.0, False, 1e-9), (32, 2, 0.8, True, 1e-9),
                                                      (48, 2, 1.3, False, 1e-9), (64, 3, 1.0, False, 2e-4),
                                                      (64, 0, 1.0, True, 2e-3)])
def test_solve_rc_bar_matches_oracle(dgp, torch_dev, n, prec, rc, use_forces, tol):
    torch, dev = torch_dev
    box, a = 100.0, 0.6
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    d = _field(n, box, 0.25, 4)
    rng = np.random.default_rng(21)
    if use_forces:
        gbar = [rng.standard_normal((n, n, n)) for _ in range(3)]
        phibar = oadj.phibar_from_forces(gbar, ofield.KGrid(n, box))
    else:
        phibar = rng.standard_normal((n, n, n))
    want_db, oinfo = oadj.phi_vjp(d, a, box, OM, rc, phibar)
    ctx = dgp.dgp_init(box, n, rc, OM, precision=prec, tol=1e-12 if prec == 2 else 1e-6, max_iter=200)
    try:
        dd = to_dev(torch_dev, d, td)
        dgp.dgp_solve_phi(ctx, a, dd, None, 1e-12 if prec == 2 else 1e-6)
        out = torch.empty_like(dd)
        atol = 1e-12 if prec == 2 else 1e-6
        if use_forces:
            st, info, rcbar = dgp.dgp_solve_adjoint_rc(ctx, None, out, atol,
                                                       gbar=[to_dev(torch_dev, g, td) for g in gbar])
        else:
            st, info, rcbar = dgp.dgp_solve_adjoint_rc(ctx, to_dev(torch_dev, phibar, td), out, atol)
        got_db = out.double().cpu().numpy()
        # without the r_c output the same call gives the same deltabar
        out2 = torch.empty_like(dd)
        if not use_forces:
            dgp.dgp_solve_adjoint(ctx, to_dev(torch_dev, phibar, td), out2, atol)
            assert torch.equal(out, out2)
    finally:
        dgp.dgp_destroy(ctx)
    assert st == dgp.DGP_OK
    assert rel_l2(got_db, want_db) < max(tol, 1e-9 if prec == 2 else 1e-4)
    assert abs(rcbar - oinfo["rcbar"]) < tol * abs(oinfo["rcbar"])


def test_solve_rc_bar_needs_a_nonlinear_delta(dgp, torch_dev):
    """After a solve in another gravity mode the accepted D's delta is gone: DGP_E_STATE."""
    torch, dev = torch_dev
    n, box = 16, 60.0
    d = to_dev(torch_dev, _field(n, box, 0.25, 4), torch.float64)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64, tol=1e-12, a_nonlinear=0.5)
    try:
        out = torch.empty_like(d)
        dgp.dgp_solve_phi(ctx, 0.6, d, None, 1e-12)
        st, _, _ = dgp.dgp_solve_adjoint_rc(ctx, d, out, 1e-12)
        assert st == dgp.DGP_OK
        dgp.dgp_solve_phi(ctx, 0.4, d, None, 1e-12)  # before a_nonlinear: linearised DGP
        with pytest.raises(dgp.DgpError) as e:
            dgp.dgp_solve_adjoint_rc(ctx, d, out, 1e-12)
        assert e.value.status == dgp.DGP_E_STATE
    finally:
        dgp.dgp_destroy(ctx)


@pytest.mark.parametrize("n,prec,rc,tol", [(16, 2, 1.0, 1e-8), (32, 2, 0.7, 1e-8), (32, 3, 1.0, 5e-3)])
def test_step_rc_bar_matches_oracle(dgp, torch_dev, n, prec, rc, tol):
    torch, dev = torch_dev
    box, a, da = 80.0 * n / 16, 0.5, 0.02
    pos, mom = _particles(n, box, 0.25, 7)
    rng = np.random.default_rng(22)
    xb1, pb1 = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    xb0, pb0, want = oadj.step_vjp(pos, mom, a, da, xb1, pb1, n, box, OM, rc, with_rc=True)
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    ctx = dgp.dgp_init(box, n, rc, OM, precision=prec, tol=1e-12 if prec == 2 else 1e-6, max_iter=300)
    try:
        st = [to_dev(torch_dev, v, td) for v in (*pos, *mom)]
        cot = [to_dev(torch_dev, v, td) for v in (*xb1, *pb1)]
        got = dgp.pm_step_adjoint_rc(ctx, dgp.particles(*st), a, da, dgp.particles(*cot))
        gcot = np.stack([v.double().cpu().numpy() for v in cot])
    finally:
        dgp.dgp_destroy(ctx)
    assert rel_l2(gcot[:3], xb0) < max(tol, 1e-8) and rel_l2(gcot[3:], pb0) < max(tol, 1e-8)
    assert abs(got - want) < tol * abs(want)


@pytest.mark.parametrize("prec", [2, 3])
def test_zeldovich_vf_bar_matches_oracle(dgp, torch_dev, prec):
    torch, dev = torch_dev
    n, box = 32, 100.0
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    dl = _field(n, box, 0.3, 23)
    pb = np.random.default_rng(24).standard_normal((3, n ** 3))
    want = oadj.zeldovich_vf_bar(pb, dl, box)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec)
    try:
        cot = [to_dev(torch_dev, v, td) for v in (*pb, *pb)]
        got = dgp.dgp_zeldovich_vf_adjoint(ctx, to_dev(torch_dev, dl, td), dgp.particles(*cot))
    finally:
        dgp.dgp_destroy(ctx)
    assert abs(got - want) < (1e-11 if prec == 2 else 1e-5) * abs(want)


def _oracle_rc_gradient(dl, n, box, rc, sched, nb, target, w):
    """L and dL/d(r_c H0) of delta_L -> Zel'dovich(vf(rc)) -> KDK steps -> P(k) loss, the oracle's
    step VJPs chained backwards, plus vf_bar * dvf/drc."""
    from oracle import estimators as oest
    from oracle import pm as opm
    vf, dvf = obg.zeldovich_velocity_factor_drc(sched[0], OM, rc)
    pos, mom = inputs.zeldovich_from_field(dl, box, vf)
    st = opm.PMState(pos, mom, sched[0], n, box, OM, rc, tol=1e-13)
    starts = []
    for i in range(len(sched) - 1):
        starts.append((st.pos.copy(), st.mom.copy()))
        st.step(sched[i + 1] - sched[i])
    delta = opm.density_contrast(opm.cic_deposit(st.pos, n, box))
    P = oest.power_spectrum(delta, box, nb)[1]
    L = np.sum(w * (P - target) ** 2)
    xb = oadj.deposit_vjp(st.pos, n, box, oadj.pk_vjp(delta, box, nb, 2 * w * (P - target)) * (n ** 3 / pos.shape[1]))
    pb = np.zeros_like(xb)
    total = 0.0
    for i in reversed(range(len(sched) - 1)):
        xb, pb, r = oadj.step_vjp(*starts[i], sched[i], sched[i + 1] - sched[i], xb, pb, n, box, OM, rc, with_rc=True)
        total += r
    return L, total + oadj.zeldovich_vf_bar(pb, dl, box) * dvf


def test_gradient_of_pk_loss_wrt_rc(dgp, torch_dev):
    """d L / d(r_c H0) through the velocity factor, the Zel'dovich map, 3 KDK steps and the P(k) loss,
    FP64 16^3: autograd against the oracle's chain and against central differences of GPU runs
    (a fresh context per r_c)."""
    from paper_0906_4548_gb300 import autodiff
    torch, dev = torch_dev
    n, box, a0, a1, ns, nb, rc = 16, 64.0, 0.3, 0.4, 3, 8, 1.0
    dl = _field(n, box, 0.25, 13)
    sched = [a0 * (a1 / a0) ** (i / ns) for i in range(ns + 1)]
    rng = np.random.default_rng(25)
    w = rng.uniform(0.5, 1.5, nb)
    target = 0.8 * _oracle_rc_gradient(dl, n, box, rc, sched, nb, np.zeros(nb), w)[0] ** 0.5 * np.ones(nb) / nb

    def run(r, grad):
        ctx = dgp.dgp_init(box, n, r, OM, precision=dgp.DGP_FP64, tol=1e-12, max_iter=300, sort_every=0)
        try:
            rt = torch.tensor(r, dtype=torch.float64, requires_grad=grad)
            vf = autodiff.VelocityFactor.apply(rt, OM, sched[0])
            d = to_dev(torch_dev, dl, torch.float64)
            x, p = autodiff.ZeldovichIC.apply(d, ctx, vf)
            x, p = autodiff.PMRun.apply(x, p, ctx, sched, 2, rt)
            L = autodiff.PkLoss.apply(x, ctx, n, target, w)
            if grad:
                L.backward()
                return float(L.detach()), float(rt.grad)
            return float(L), None
        finally:
            dgp.dgp_destroy(ctx)

    L, g = run(rc, True)
    Lo, go = _oracle_rc_gradient(dl, n, box, rc, sched, nb, target, w)
    assert abs(L / Lo - 1) < 1e-9
    assert abs(g - go) < 1e-6 * abs(go)
    h = 1e-5
    fd = (run(rc + h, False)[0] - run(rc - h, False)[0]) / (2 * h)
    assert abs(fd - g) < 1e-5 * abs(fd)
