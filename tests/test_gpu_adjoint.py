"""Adjoint of the converged field solve on the GPU (dgp_solve_adjoint) against
the oracle's (oracle/adjoint.py) and against central differences of GPU solves."""
import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import field as ofield
from paper_0906_4548_gb300 import inputs

from test_gpu_parity import OM, rel_l2, to_dev  # noqa: F401
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu


def _field(n, box, rms, seed):
    d, _ = inputs.linear_field(n, box, -1.5, rms, seed=seed)  # min delta > -1: no bad points
    return d


@pytest.mark.parametrize("n,prec,tol,use_forces", [(32, 2, 1e-9, False), (32, 2, 1e-9, True), (48, 2, 1e-9, False),
                                                   (64, 3, 1e-4, False), (64, 0, 1e-4, True)])
def test_adjoint_matches_oracle(dgp, torch_dev, n, prec, tol, use_forces):
    torch, dev = torch_dev
    box, a = 100.0, 0.6
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    d = _field(n, box, 0.25, 4)
    rng = np.random.default_rng(5)
    if use_forces:
        gbar = [rng.standard_normal((n, n, n)) for _ in range(3)]
        phibar = oadj.phibar_from_forces(gbar, ofield.KGrid(n, box))
    else:
        phibar = rng.standard_normal((n, n, n))
    want, oinfo = oadj.phi_vjp(d, a, box, OM, 1.0, phibar)
    assert oinfo["adjoint"]["converged"]
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec, tol=1e-12 if prec == 2 else 1e-6, max_iter=200)
    try:
        dd = to_dev(torch_dev, d, td)
        dgp.dgp_solve_phi(ctx, a, dd, None, 1e-12 if prec == 2 else 1e-6)
        out = torch.empty_like(dd)
        if use_forces:
            st, info = dgp.dgp_solve_adjoint(ctx, None, out, 1e-12 if prec == 2 else 1e-6,
                                             gbar=[to_dev(torch_dev, g, td) for g in gbar])
        else:
            st, info = dgp.dgp_solve_adjoint(ctx, to_dev(torch_dev, phibar, td), out, 1e-12 if prec == 2 else 1e-6)
        got = out.double().cpu().numpy()
    finally:
        dgp.dgp_destroy(ctx)
    assert st == dgp.DGP_OK and info["iters"] >= 1
    assert rel_l2(got, want) < tol


def test_adjoint_directional_derivative_of_gpu_solves(dgp, torch_dev):
    """<deltabar, u> against (L(delta + e u) - L(delta - e u)) / 2e with L = <phibar, phi> from GPU solves (FP64)."""
    torch, dev = torch_dev
    n, box, a = 32, 100.0, 0.6
    d = _field(n, box, 0.25, 6)
    rng = np.random.default_rng(7)
    phibar = rng.standard_normal((n, n, n))
    u = rng.standard_normal((n, n, n))
    u -= u.mean()
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64, tol=1e-13, max_iter=300)
    try:
        pb = to_dev(torch_dev, phibar, torch.float64)
        phi = torch.empty((n, n, n), dtype=torch.float64, device=dev)

        def L(x):
            dgp.dgp_reset(ctx)
            dgp.dgp_solve_phi(ctx, a, to_dev(torch_dev, x, torch.float64), phi, 1e-13)
            return float((phi * pb).sum())

        e = 1e-4
        fd = (L(d + e * u) - L(d - e * u)) / (2 * e)
        dgp.dgp_reset(ctx)
        dgp.dgp_solve_phi(ctx, a, to_dev(torch_dev, d, torch.float64), None, 1e-13)
        out = torch.empty_like(phi)
        st, info = dgp.dgp_solve_adjoint(ctx, pb, out, 1e-12)
        ad = float((out * to_dev(torch_dev, u, torch.float64)).sum())
    finally:
        dgp.dgp_destroy(ctx)
    assert abs(fd - ad) < 1e-6 * abs(fd)


def test_adjoint_states_and_arguments(dgp, torch_dev):
    torch, dev = torch_dev
    n, box = 16, 50.0
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_MIXED)
    try:
        z = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
        out = torch.empty_like(z)
        with pytest.raises(dgp.DgpError) as e:
            dgp.dgp_solve_adjoint(ctx, z, out, 1e-6)
        assert e.value.status == dgp.DGP_E_STATE
        dgp.dgp_solve_phi(ctx, 0.5, to_dev(torch_dev, _field(n, box, 0.2, 1), torch.float32), None, 1e-6)
        with pytest.raises(dgp.DgpError) as e:
            dgp.dgp_solve_adjoint(ctx, None, out, 1e-6)
        assert e.value.status == dgp.DGP_E_INVALID
        st, info = dgp.dgp_solve_adjoint(ctx, z, out, 1e-6)  # zero cotangent: zero gradient
        assert float(out.abs().max()) == 0.0
    finally:
        dgp.dgp_destroy(ctx)


def _particles(n, box, sig, seed):
    pos, _ = inputs.lattice_particles(n, box)
    rng = np.random.default_rng(seed)
    pos = (pos + rng.normal(0, sig * box / n, pos.shape)) % box
    mom = rng.normal(0, 0.5, pos.shape)
    return pos, mom


@pytest.mark.parametrize("n,prec,tol", [(16, 2, 1e-8), (32, 2, 1e-8), (32, 3, 2e-3)])
def test_step_adjoint_matches_oracle(dgp, torch_dev, n, prec, tol):
    torch, dev = torch_dev
    box, a, da = 80.0 * n / 16, 0.5, 0.02
    pos, mom = _particles(n, box, 0.25, 7)
    rng = np.random.default_rng(8)
    xb1, pb1 = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    xb0, pb0 = oadj.step_vjp(pos, mom, a, da, xb1, pb1, n, box, OM, 1.0)
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec, tol=1e-12 if prec == 2 else 1e-6, max_iter=300)
    try:
        st = [to_dev(torch_dev, v, td) for v in (*pos, *mom)]
        cot = [to_dev(torch_dev, v, td) for v in (*xb1, *pb1)]
        dgp.pm_step_adjoint(ctx, dgp.particles(*st), a, da, dgp.particles(*cot))
        got = np.stack([v.double().cpu().numpy() for v in cot])
        unchanged = np.stack([v.double().cpu().numpy() for v in st])
    finally:
        dgp.dgp_destroy(ctx)
    assert np.array_equal(unchanged, np.concatenate([pos, mom]).astype(unchanged.dtype) if prec == 2 else
                          np.concatenate([pos, mom]).astype(np.float32).astype(np.float64))
    assert rel_l2(got[:3], xb0) < tol and rel_l2(got[3:], pb0) < tol


def test_pk_adjoint_matches_oracle(dgp, torch_dev):
    from oracle import estimators as oest
    from oracle import pm as opm
    torch, dev = torch_dev
    n, box, nb = 32, 100.0, 16
    pos, _ = _particles(n, box, 0.3, 9)
    rng = np.random.default_rng(10)
    dldp = rng.standard_normal(nb)
    delta = opm.density_contrast(opm.cic_deposit(pos, n, box))
    want = oadj.deposit_vjp(pos, n, box, oadj.pk_vjp(delta, box, nb, dldp) * (n ** 3 / pos.shape[1]))
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64)
    try:
        x = [to_dev(torch_dev, v, torch.float64) for v in pos]
        cot = [torch.zeros_like(x[0]) for _ in range(6)]
        dgp.dgp_power_spectrum_adjoint(ctx, dgp.particles(*x, *x), dldp, dgp.particles(*cot))
        got = np.stack([c.cpu().numpy() for c in cot[:3]])
        assert all(float(c.abs().max()) == 0.0 for c in cot[3:])
    finally:
        dgp.dgp_destroy(ctx)
    assert rel_l2(got, want) < 1e-10


def test_zeldovich_map_and_transpose(dgp, torch_dev):
    torch, dev = torch_dev
    n, box, vf = 32, 100.0, 0.8
    dl = _field(n, box, 0.3, 11)
    pos, mom = inputs.zeldovich_from_field(dl, box, vf)
    rng = np.random.default_rng(12)
    xb, pb = rng.standard_normal((3, n ** 3)), rng.standard_normal((3, n ** 3))
    want_bar = oadj.zeldovich_vjp(xb, pb, n, box, vf)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64)
    try:
        out = [torch.empty(n ** 3, dtype=torch.float64, device=dev) for _ in range(6)]
        dgp.dgp_zeldovich(ctx, to_dev(torch_dev, dl, torch.float64), vf, dgp.particles(*out))
        got = np.stack([o.cpu().numpy() for o in out])
        cot = [to_dev(torch_dev, v, torch.float64) for v in (*xb, *pb)]
        bar = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        dgp.dgp_zeldovich_adjoint(ctx, dgp.particles(*cot), vf, bar)
    finally:
        dgp.dgp_destroy(ctx)
    dpos = (got[:3] - pos + box / 2) % box - box / 2  # equal up to the periodic wrap
    assert np.max(np.abs(dpos)) < 1e-11 and rel_l2(got[3:], mom) < 1e-12
    assert rel_l2(bar.cpu().numpy(), want_bar) < 1e-11


def _run_loss_oracle(dl, n, box, vf, sched, nb, target, w):
    from oracle import estimators as oest
    from oracle import pm as opm
    pos, mom = inputs.zeldovich_from_field(dl, box, vf)
    st = opm.PMState(pos, mom, sched[0], n, box, OM, 1.0, tol=1e-13)
    starts = []
    for i in range(len(sched) - 1):
        starts.append((st.pos.copy(), st.mom.copy()))
        st.step(sched[i + 1] - sched[i])
    delta = opm.density_contrast(opm.cic_deposit(st.pos, n, box))
    P = oest.power_spectrum(delta, box, nb)[1]
    L = np.sum(w * (P - target) ** 2)
    xb = oadj.deposit_vjp(st.pos, n, box, oadj.pk_vjp(delta, box, nb, 2 * w * (P - target)) * (n ** 3 / pos.shape[1]))
    pb = np.zeros_like(xb)
    for i in reversed(range(len(sched) - 1)):
        xb, pb = oadj.step_vjp(*starts[i], sched[i], sched[i + 1] - sched[i], xb, pb, n, box, OM, 1.0)
    return L, oadj.zeldovich_vjp(xb, pb, n, box, vf)


def test_gradient_of_pk_loss_wrt_initial_field(dgp, torch_dev):
    """delta_L -> Zel'dovich ICs -> 4 KDK steps (checkpoint every 2) -> P(k) loss, FP64 16^3:
    the autograd gradient against the oracle's chained VJPs and against central differences
    of GPU runs along single Fourier modes of delta_L."""
    from oracle import background as obg
    from paper_0906_4548_gb300 import autodiff
    torch, dev = torch_dev
    n, box, a0, a1, ns, nb = 16, 64.0, 0.3, 0.4, 4, 8
    dl = _field(n, box, 0.25, 13)
    vf = obg.zeldovich_velocity_factor(a0, OM, 1.0)
    sched = [a0 * (a1 / a0) ** (i / ns) for i in range(ns + 1)]
    rng = np.random.default_rng(14)
    w = rng.uniform(0.5, 1.5, nb)
    target = 0.8 * _run_loss_oracle(dl, n, box, vf, sched, nb, np.zeros(nb), w)[0] ** 0.5 * np.ones(nb) / nb
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64, tol=1e-12, max_iter=300, sort_every=0)
    try:
        def loss(field, grad):
            d = to_dev(torch_dev, field, torch.float64).requires_grad_(grad)
            x, p = autodiff.ZeldovichIC.apply(d, ctx, vf)
            x, p = autodiff.PMRun.apply(x, p, ctx, sched, 2)
            return autodiff.PkLoss.apply(x, ctx, n, target, w), d

        L, d = loss(dl, True)
        L.backward()
        g = d.grad.cpu().numpy()
        Lo, go = _run_loss_oracle(dl, n, box, vf, sched, nb, target, w)
        assert abs(float(L) / Lo - 1) < 1e-9
        assert rel_l2(g, go) < 1e-6
        x = np.arange(n) * box / n
        for t in range(6):
            k = rng.integers(1, n // 2, 3)
            u = np.cos(2 * np.pi / box * (k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :])
                       + rng.uniform(0, 2 * np.pi))
            e = 1e-5
            fd = (float(loss(dl + e * u, False)[0]) - float(loss(dl - e * u, False)[0])) / (2 * e)
            assert abs(fd - np.sum(g * u)) < 1e-4 * max(abs(fd), 1e-3 * np.sum(np.abs(g * u)))
    finally:
        dgp.dgp_destroy(ctx)
