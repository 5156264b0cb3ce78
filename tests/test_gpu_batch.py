"""Batches of independent realisations (dgp_batch_*): every realisation of a
mixed-size batch steps exactly as the same realisation stepped alone."""
import math

import numpy as np
import pytest

from test_gpu_parity import OM, rel_l2, to_dev, zel  # noqa: F401
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu

CASES = [(32, 80.0, 1.0, 1), (48, 120.0, 0.6, 2), (64, 200.0, 1.7, 3), (32, 60.0, 1.2, 4), (96, 150.0, 0.9, 5)]


def _ics(n, box, rc, seed, a0):
    pos, mom, _ = zel(n, box, a0, -1.5, 0.5, seed, rc)
    return pos, mom


@pytest.mark.parametrize("prec,tol,sort_every", [(2, 1e-11, 2), (3, 2e-5, 0)])
def test_batch_matches_individual_contexts(dgp, torch_dev, prec, tol, sort_every):
    """FP64 with the cell sort: compared after ordering by position.  FP32 runs
    differ at the 1e-6 level (float atomics), where ordering by position would
    pair up different particles, so that case keeps the input order."""
    torch, dev = torch_dev
    td = torch.float64 if prec == dgp.DGP_FP64 else torch.float32
    a0, a1, ns = 0.2, 0.3, 3
    dl = (math.log(a1) - math.log(a0)) / ns
    sched = [a0 * math.exp(i * dl) for i in range(ns + 1)]
    ics = [_ics(n, box, rc, seed, a0) for n, box, rc, seed in CASES]
    plist = [dgp.params(box, n, rc, precision=prec, tol=1e-9 if prec == 2 else 1e-6, max_iter=200,
                        sort_every=sort_every) for n, box, rc, _ in CASES]
    # batch
    b, ctxs = dgp.dgp_batch_create(plist, OM)
    try:
        tb = [[to_dev(torch_dev, v, td) for v in (*p, *m)] for p, m in ics]
        parts = [dgp.particles(*t) for t in tb]
        binfo = []
        for i in range(ns):
            binfo.append(dgp.dgp_batch_step(b, parts, [sched[i]] * len(CASES),
                                            [sched[i + 1] - sched[i]] * len(CASES)))
        got = [np.stack([v.cpu().numpy() for v in t]) for t in tb]
    finally:
        dgp.dgp_batch_destroy(b)
    # the same realisations, one context at a time
    for k, ((n, box, rc, _), (p, m)) in enumerate(zip(CASES, ics)):
        ctx = dgp.dgp_init(box, n, rc, OM, precision=prec, tol=1e-9 if prec == 2 else 1e-6, max_iter=200,
                           sort_every=sort_every)
        try:
            t = [to_dev(torch_dev, v, td) for v in (*p, *m)]
            pp = dgp.particles(*t)
            for i in range(ns):
                inf = dgp.pm_step(ctx, pp, sched[i], sched[i + 1] - sched[i])
                assert inf["iters"] == binfo[i][k]["iters"] or prec != dgp.DGP_FP64
            want = np.stack([v.cpu().numpy() for v in t])
        finally:
            dgp.dgp_destroy(ctx)
        if sort_every:
            # the cell sort orders particles within a cell arbitrarily: compare sorted by position
            og = np.lexsort(got[k][:3][::-1])
            ow = np.lexsort(want[:3][::-1])
            assert rel_l2(got[k][:, og], want[:, ow]) < tol, k
        else:
            assert rel_l2(got[k], want) < tol, k


def test_batch_reports_a_failing_realisation(dgp, torch_dev):
    torch, dev = torch_dev
    plist = [dgp.params(60.0, 32, 1.0), dgp.params(60.0, 48, 1.0)]
    b, ctxs = dgp.dgp_batch_create(plist, OM)
    try:
        p, m = _ics(32, 60.0, 1.0, 3, 0.2)
        t = [to_dev(torch_dev, v, torch.float32) for v in (*p, *m)]
        empty = [torch.empty(0, dtype=torch.float32, device=dev) for _ in range(6)]
        x0 = t[0].clone()
        with pytest.raises(dgp.DgpError) as e:
            dgp.dgp_batch_step(b, [dgp.particles(*t), dgp.particles(*empty)], [0.2, 0.2], [0.01, 0.01])
        assert e.value.status == dgp.DGP_E_INVALID
        assert not torch.equal(t[0], x0)  # the valid realisation stepped
        with pytest.raises(dgp.DgpError):
            dgp.dgp_batch_create([dgp.params(60.0, 40, 1.0)], OM)  # invalid size: nothing leaks
    finally:
        dgp.dgp_batch_destroy(b)


@pytest.mark.parametrize("prec", [4, 0])
def test_class_step_matches_individual_contexts_and_oracle(dgp, torch_dev, prec):
    """Four 48^3 realisations with different boxes and r_c form one class: every kernel stage of
    their step is one launch for all four, and they iterate in lockstep.  Each realisation must end
    where its own context stepped alone ends (float atomics of the deposit aside) and follow the FP64
    oracle's run."""
    from oracle import pm as opm
    torch, dev = torch_dev
    cases = [(48, 120.0, 0.6, 2), (48, 90.0, 1.3, 3), (48, 150.0, 1.9, 4), (48, 60.0, 0.8, 5)]
    a0, a1, ns = 0.2, 0.3, 3
    dl = (math.log(a1) - math.log(a0)) / ns
    sched = [a0 * math.exp(i * dl) for i in range(ns + 1)]
    ics = [_ics(n, box, rc, seed, a0) for n, box, rc, seed in cases]
    ics = [(p.astype(np.float32).astype(np.float64), m.astype(np.float32).astype(np.float64)) for p, m in ics]
    plist = [dgp.params(box, n, rc, precision=prec, tol=1e-6, max_iter=200) for n, box, rc, _ in cases]
    b, ctxs = dgp.dgp_batch_create(plist, OM)
    try:
        cls, ncls = dgp.dgp_batch_classes(b, len(cases))
        assert ncls == 1 and cls == [0] * len(cases)
        tb = [[to_dev(torch_dev, v, torch.float32) for v in (*p, *m)] for p, m in ics]
        parts = [dgp.particles(*t) for t in tb]
        infos = []
        for i in range(ns):
            infos.append(dgp.dgp_batch_step(b, parts, [sched[i]] * len(cases), [sched[i + 1] - sched[i]] * len(cases)))
        got = [np.stack([v.cpu().numpy() for v in t]).astype(np.float64) for t in tb]
    finally:
        dgp.dgp_batch_destroy(b)
    assert all(inf["status"] == dgp.DGP_OK and inf["norm_res"] < 1e-6 for step in infos for inf in step)
    for k, ((n, box, rc, _), (p, m)) in enumerate(zip(cases, ics)):
        ctx = dgp.dgp_init(box, n, rc, OM, precision=prec, tol=1e-6, max_iter=200)
        try:
            t = [to_dev(torch_dev, v, torch.float32) for v in (*p, *m)]
            pp = dgp.particles(*t)
            for i in range(ns):
                inf = dgp.pm_step(ctx, pp, sched[i], sched[i + 1] - sched[i])
                assert abs(inf["iters"] - infos[i][k]["iters"]) <= 1  # float atomics of the deposit
            want = np.stack([v.cpu().numpy() for v in t]).astype(np.float64)
        finally:
            dgp.dgp_destroy(ctx)
        assert rel_l2(got[k], want) < 2e-5, k
        st = opm.run(p, m, a0, a1, ns, n, box, OM, rc, tol=1e-10, max_iter=300)
        dx = (got[k][:3] - st.pos + box / 2) % box - box / 2
        disp = (st.pos - p + box / 2) % box - box / 2
        assert np.linalg.norm(dx) / np.linalg.norm(disp) < 1e-4, k
        assert rel_l2(got[k][3:], st.mom) < 1e-4, k


@pytest.mark.parametrize("n,box", [(16, 40.0), (32, 70.0), (48, 110.0), (64, 160.0), (96, 150.0)])
def test_plane_pass_matches_separate_passes_and_oracle(dgp, torch_dev, n, box):
    """A class of three realisations stepped with the plane-resident Hessian pass and with the
    separate x and y passes: both are the same spectra up to rounding, so the two runs agree to
    the FP32 level, with the same evaluation counts to within one; the plane run follows the FP64
    oracle (n <= 64)."""
    from oracle import pm as opm
    torch, dev = torch_dev
    cases = [(n, box * f, rc, seed) for f, rc, seed in ((1.0, 0.7, 11), (0.8, 1.4, 12), (1.3, 1.9, 13))]
    a0, a1, ns = 0.25, 0.4, 3
    dl = (math.log(a1) - math.log(a0)) / ns
    sched = [a0 * math.exp(i * dl) for i in range(ns + 1)]
    ics = [_ics(nn, bx, rc, seed, a0) for nn, bx, rc, seed in cases]
    ics = [(p.astype(np.float32).astype(np.float64), m.astype(np.float32).astype(np.float64)) for p, m in ics]
    plist = [dgp.params(bx, nn, rc, precision=dgp.DGP_FP32, tol=1e-6, max_iter=200) for nn, bx, rc, _ in cases]
    runs = {}
    for plane in (True, False):
        b, ctxs = dgp.dgp_batch_create(plist, OM)
        try:
            dgp.dgp_batch_set_plane_pass(b, plane)
            cls, ncls = dgp.dgp_batch_classes(b, len(cases))
            assert ncls == 1
            tb = [[to_dev(torch_dev, v, torch.float32) for v in (*p, *m)] for p, m in ics]
            parts = [dgp.particles(*t) for t in tb]
            infos = [dgp.dgp_batch_step(b, parts, [sched[i]] * len(cases), [sched[i + 1] - sched[i]] * len(cases))
                     for i in range(ns)]
            runs[plane] = ([np.stack([v.cpu().numpy() for v in t]).astype(np.float64) for t in tb], infos)
        finally:
            dgp.dgp_batch_destroy(b)
    (gp, ip), (gs, is_) = runs[True], runs[False]
    for step_p, step_s in zip(ip, is_):
        for x, y in zip(step_p, step_s):
            assert x["status"] == dgp.DGP_OK and x["norm_res"] < 1e-6
            assert abs(x["iters"] - y["iters"]) <= 1
    for k, ((nn, bx, rc, _), (p, m)) in enumerate(zip(cases, ics)):
        assert rel_l2(gp[k], gs[k]) < 2e-5, k
        if nn > 64:  # the separate passes' 96^3 runs are checked against the oracle elsewhere
            continue
        st = opm.run(p, m, a0, a1, ns, nn, bx, OM, rc, tol=1e-10, max_iter=300)
        dx = (gp[k][:3] - st.pos + bx / 2) % bx - bx / 2
        disp = (st.pos - p + bx / 2) % bx - bx / 2
        assert np.linalg.norm(dx) / np.linalg.norm(disp) < 1e-4, k
        assert rel_l2(gp[k][3:], st.mom) < 1e-4, k
