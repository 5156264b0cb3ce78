"""Whole runs and full-size steps of the GPU path against the FP64 oracle.

* A whole run from a = 0.02 to 1 at 32^3, in the arithmetic the 256^3 benchmark uses (FP32
  residual, exact discriminant, FP64 norms and reductions), with error-free pairs, and in plain
  FP32: P(k) after the run within 1e-3 of the oracle's.
* One step of the 256^3 benchmark workload: the gather-kick-drift of the GPU's own force
  meshes against the oracle's CIC interpolation and kick/drift factors (Sec. III.A).
* The Zel'dovich map against the oracle's displacement field.
* A batch of realisations in FP64 against the oracle's runs.
* pm_step_host on alternating host particle sets against fresh contexts.
* The iteration replay as CUDA graphs (contexts on a non-default stream) against the oracle.
* P(k) is the same bits on every call.
"""
import math

import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import background as obg
from oracle import estimators as oest
from oracle import field as ofield
from oracle import pm as opm
from test_gpu_parity import OM, rel_l2, to_dev, zel
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu

# 32^3 particles in 50 Mpc/h (the 128^3, 200 Mpc/h resolution), n_s = -1.5, rms 0.5 at a = 0.02,
# 50 steps uniform in ln a to a = 1, relaxation tolerance 1e-6 (oracle 1e-8)
RUN = dict(n=32, box=50.0, a0=0.02, a1=1.0, steps=50, seed=7)


def _sched(a0, a1, ns):
    dl = (math.log(a1) - math.log(a0)) / ns
    return [a0 * math.exp(i * dl) for i in range(ns + 1)]


@pytest.fixture(scope="module")
def full_run_oracle():
    n, box = RUN["n"], RUN["box"]
    pos, mom, _ = zel(n, box, RUN["a0"], -1.5, 0.5, RUN["seed"])
    pos, mom = pos.astype(np.float32).astype(np.float64), mom.astype(np.float32).astype(np.float64)
    st = opm.run(pos, mom, RUN["a0"], RUN["a1"], RUN["steps"], n, box, OM, 1.0, tol=1e-8, max_iter=300)
    assert all(s["converged"] for s in st.solves)
    pk = oest.power_spectrum(opm.density_contrast(opm.cic_deposit(st.pos, n, box)), box)
    return pos, mom, pk


@pytest.mark.parametrize("prec_name", ["DGP_MIXED_F32R", "DGP_MIXED_EFT", "DGP_FP32"])
def test_full_run_pk_matches_oracle(dgp, torch_dev, full_run_oracle, prec_name):
    torch, dev = torch_dev
    n, box = RUN["n"], RUN["box"]
    pos, mom, (ko, Po, co) = full_run_oracle
    sched = _sched(RUN["a0"], RUN["a1"], RUN["steps"])
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=getattr(dgp, prec_name), tol=1e-6, max_iter=100, sort_every=8)
    try:
        t = [to_dev(torch_dev, v, torch.float32) for v in (*pos, *mom)]
        parts = dgp.particles(*t)
        infos = [dgp.pm_step(ctx, parts, sched[i], sched[i + 1] - sched[i]) for i in range(RUN["steps"])]
        delta = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        dgp.dgp_deposit(ctx, parts, delta)
        k, P, cnt = dgp.power_spectrum(ctx, delta, n // 2)
    finally:
        dgp.dgp_destroy(ctx)
    assert all(i["status"] == dgp.DGP_OK and i["norm_res"] < 1e-6 for i in infos)
    assert np.array_equal(cnt, co)
    assert np.max(np.abs(P / Po - 1)) < 1e-3


def test_gather_kick_drift_full_size_matches_oracle(dgp, torch_dev):
    """256^3 particles and mesh, 400 Mpc/h, the first step of the 200-step run: positions after the
    drift and momenta after both kicks, on a sample of 200k particles, against the oracle's CIC
    interpolation of the GPU's force meshes with the oracle's kick and drift factors."""
    torch, dev = torch_dev
    n, box, a0 = 256, 400.0, 0.02
    a1 = a0 * math.exp(math.log(1.0 / a0) / 200)
    ah = math.exp(0.5 * (math.log(a0) + math.log(a1)))
    pos, mom, _ = zel(n, box, a0, -1.5, 0.5, 3)
    x0, p0 = pos.astype(np.float32), mom.astype(np.float32)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_MIXED_EFT, tol=1e-6, max_iter=100)
    try:
        t = [to_dev(torch_dev, v, torch.float32) for v in (*x0, *p0)]
        parts = dgp.particles(*t)
        delta = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        g0 = [torch.empty_like(delta) for _ in range(3)]
        dgp.dgp_deposit(ctx, parts, delta)
        dgp.dgp_solve_forces(ctx, a0, delta, None, g0[0], g0[1], g0[2], 1e-6)
        dgp.dgp_reset(ctx)
        dgp.pm_step(ctx, parts, a0, a1 - a0)
        x1 = np.stack([v.cpu().numpy() for v in t[:3]]).astype(np.float64)
        p1 = np.stack([v.cpu().numpy() for v in t[3:]]).astype(np.float64)
        dgp.dgp_deposit(ctx, parts, delta)
        g1 = [torch.empty_like(delta) for _ in range(3)]
        dgp.dgp_solve_forces(ctx, a1, delta, None, g1[0], g1[1], g1[2], 1e-6)
        G0 = [g.double().cpu().numpy() for g in g0]
        G1 = [g.double().cpu().numpy() for g in g1]
    finally:
        dgp.dgp_destroy(ctx)
    sel = np.random.default_rng(0).choice(n ** 3, 200000, replace=False)
    xs0, ps0 = x0[:, sel].astype(np.float64), p0[:, sel].astype(np.float64)
    k1 = obg.kick_factor(a0, ah, OM, 1.0)
    k2 = obg.kick_factor(ah, a1, OM, 1.0)
    dr = obg.drift_factor(a0, a1, OM, 1.0)
    ph = ps0 + k1 * np.stack([opm.cic_interpolate(G0[c], xs0, box) for c in range(3)])
    x_want = (xs0 + dr * ph) % box
    dx = (x1[:, sel] - x_want + box / 2) % box - box / 2
    step = dr * np.abs(ph)
    # float positions near 400 Mpc/h carry ~3e-5 Mpc/h of rounding
    assert np.max(np.abs(dx) - 1e-5 * step) < 4 * np.spacing(np.float32(box))
    p_want = ph + k2 * np.stack([opm.cic_interpolate(G1[c], x1[:, sel], box) for c in range(3)])
    assert rel_l2(p1[:, sel] - ps0, p_want - ps0) < 1e-5


def test_zeldovich_matches_oracle_displacement(dgp, torch_dev):
    torch, dev = torch_dev
    n, box, vf = 48, 120.0, 0.7
    rng = np.random.default_rng(21)
    dl = rng.standard_normal((n, n, n)) * 0.3
    psi = oadj.zeldovich_displacement(dl, box)
    d = box / n
    i = np.arange(n)
    q = [np.broadcast_to(v * d, (n, n, n)).reshape(-1) for v in
         (i[:, None, None], i[None, :, None], i[None, None, :])]
    pos_want = np.stack([(q[j] + psi[j].reshape(-1)) % box for j in range(3)])
    mom_want = np.stack([vf * psi[j].reshape(-1) for j in range(3)])
    for prec, tol in ((dgp.DGP_FP64, 1e-12), (dgp.DGP_FP32, 1e-5)):
        td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
        ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec)
        try:
            out = [torch.empty(n ** 3, dtype=td, device=dev) for _ in range(6)]
            dgp.dgp_zeldovich(ctx, to_dev(torch_dev, dl, td), vf, dgp.particles(*out))
            got = np.stack([o.double().cpu().numpy() for o in out])
        finally:
            dgp.dgp_destroy(ctx)
        dpos = (got[:3] - pos_want + box / 2) % box - box / 2
        disp = np.stack([psi[j].reshape(-1) for j in range(3)])
        assert np.linalg.norm(dpos) / np.linalg.norm(disp) < tol
        assert rel_l2(got[3:], mom_want) < tol


def test_batch_fp64_matches_oracle(dgp, torch_dev):
    """Two realisations of different meshes, boxes and r_c in one batch, FP64, 3 steps each,
    against the oracle's runs."""
    torch, dev = torch_dev
    cases = [(48, 120.0, 0.6, 2), (32, 80.0, 1.4, 5)]
    a0, a1, ns = 0.2, 0.3, 3
    sched = _sched(a0, a1, ns)
    ics = [zel(n, box, a0, -1.5, 0.5, seed, rc)[:2] for n, box, rc, seed in cases]
    plist = [dgp.params(box, n, rc, precision=dgp.DGP_FP64, tol=1e-12, max_iter=300) for n, box, rc, _ in cases]
    b, _ = dgp.dgp_batch_create(plist, OM)
    try:
        tb = [[to_dev(torch_dev, v, torch.float64) for v in (*p, *m)] for p, m in ics]
        parts = [dgp.particles(*t) for t in tb]
        for i in range(ns):
            dgp.dgp_batch_step(b, parts, [sched[i]] * len(cases), [sched[i + 1] - sched[i]] * len(cases))
        got = [np.stack([v.cpu().numpy() for v in t]) for t in tb]
    finally:
        dgp.dgp_batch_destroy(b)
    for (n, box, rc, _), (p, m), g in zip(cases, ics, got):
        st = opm.run(p, m, a0, a1, ns, n, box, OM, rc, tol=1e-12, max_iter=300)
        dx = (g[:3] - st.pos + box / 2) % box - box / 2
        disp = (st.pos - p + box / 2) % box - box / 2
        assert np.linalg.norm(dx) / np.linalg.norm(disp) < 1e-9
        assert rel_l2(g[3:], st.mom) < 1e-9


def test_pm_step_host_on_alternating_sets_matches_fresh_contexts(dgp, torch_dev):
    """Set A steps a0 -> a1 on one context; set B, A's state at a1 with every particle moved by up
    to a tenth of a cell, then steps a1 -> a2 on the same context, and A again a1 -> a2.  The
    start force must be computed for B and for A's second step, not taken over from the previous
    call (the mesh force of another particle set differs at the cell scale).  FP64 at tol 1e-12
    against fresh contexts, so the warm start (close in both cases) does not show."""
    torch, dev = torch_dev
    n, box = 32, 100.0
    a0, a1, a2 = 0.3, 0.32, 0.34
    pos, mom, _ = zel(n, box, a0, -1.5, 0.3, 31)
    ha = [np.ascontiguousarray(v) for v in (*pos, *mom)]

    def fresh(arrs, a, da):
        c = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64, tol=1e-12, max_iter=300)
        try:
            t = [to_dev(torch_dev, v, torch.float64) for v in arrs]
            info = dgp.pm_step(c, dgp.particles(*t), a, da)
            return np.stack([v.cpu().numpy() for v in t]), info
        finally:
            dgp.dgp_destroy(c)

    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP64, tol=1e-12, max_iter=300)
    try:
        dgp.pm_step_host(ctx, dgp.particles(*ha), a0, a1 - a0)
        a_mid = [v.copy() for v in ha]
        jit = np.random.default_rng(5).uniform(-0.1, 0.1, (3, n ** 3)) * box / n
        hb = [np.ascontiguousarray((a_mid[j] + jit[j]) % box) for j in range(3)] + [v.copy() for v in a_mid[3:]]
        b_start = [v.copy() for v in hb]
        ib = dgp.pm_step_host(ctx, dgp.particles(*hb), a1, a2 - a1)
        b_got = np.stack(hb).copy()
        ia = dgp.pm_step_host(ctx, dgp.particles(*ha), a1, a2 - a1)
        a_got = np.stack(ha).copy()
    finally:
        dgp.dgp_destroy(ctx)
    b_want, ib_f = fresh(b_start, a1, a2 - a1)
    a_want, ia_f = fresh(a_mid, a1, a2 - a1)
    for i in (ib, ia, ib_f, ia_f):
        assert i["status"] == dgp.DGP_OK and i["norm_res"] < 1e-12, i
    assert rel_l2(b_got, b_want) < 1e-10
    assert rel_l2(a_got, a_want) < 1e-10


@pytest.mark.parametrize("prec,tol", [(2, 1e-9), (3, 1e-5), (4, 1e-5)])
def test_graph_replayed_solve_matches_oracle(dgp, torch_dev, prec, tol):
    """A context on a non-default stream replays the relaxation iterations as CUDA graphs."""
    torch, dev = torch_dev
    n, box, a = 64, 200.0, 0.5
    pos, _, _ = zel(n, box, a, -1.5, 0.5, 9)
    delta = opm.density_contrast(opm.cic_deposit(pos, n, box))
    phi_o, _, _, info_o = ofield.solve_phi(delta, a, box, OM, 1.0, tol=1e-12, max_iter=300)
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    s = torch.cuda.Stream(device=dev)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec, tol=1e-10 if prec == 2 else 1e-6, max_iter=200,
                       stream=s.cuda_stream)
    try:
        d = to_dev(torch_dev, delta, td)
        phi = torch.empty_like(d)
        torch.cuda.synchronize()
        st, info = dgp.dgp_solve_phi(ctx, a, d, phi, 1e-10 if prec == 2 else 1e-6)
        torch.cuda.synchronize()
        # a second solve from the warm start goes through the cached graph
        st2, info2 = dgp.dgp_solve_phi(ctx, a, d, phi, 1e-10 if prec == 2 else 1e-6)
        torch.cuda.synchronize()
        got = phi.double().cpu().numpy()
    finally:
        dgp.dgp_destroy(ctx)
    assert st == dgp.DGP_OK and st2 == dgp.DGP_OK and info["iters"] >= 3
    assert rel_l2(got, phi_o) < tol


def test_power_spectrum_same_bits_every_call(dgp, torch_dev):
    torch, dev = torch_dev
    n, box = 64, 150.0
    d = to_dev(torch_dev, np.random.default_rng(5).standard_normal((n, n, n)), torch.float32)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_FP32)
    try:
        runs = [dgp.power_spectrum(ctx, d, n // 2) for _ in range(3)]
    finally:
        dgp.dgp_destroy(ctx)
    for k, P, c in runs[1:]:
        assert np.array_equal(k, runs[0][0]) and np.array_equal(P, runs[0][1]) and np.array_equal(c, runs[0][2])
