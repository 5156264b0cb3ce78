"""The fused Hessian pass (Hessian x pass and six-field inverse y pass in one clustered launch,
FP32 mesh data at 128^3 and 256^3) against the separate passes on the same inputs: the same
spectra up to rounding order, so the solves agree to the FP32 level with the same iteration
counts (within one).  The separate passes are the ones the oracle checks in test_gpu_parity
exercise (the fused pass is opt-in)."""
import math

import numpy as np
import pytest

from test_gpu_parity import OM, rel_l2, to_dev, zel  # noqa: F401
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,box,prec", [(128, 200.0, 4), (256, 400.0, 4), (128, 150.0, 0), (128, 250.0, 3)])
def test_fused_solve_matches_separate_passes(dgp, torch_dev, n, box, prec):
    torch, dev = torch_dev
    a = 0.4
    pos, mom, _ = zel(n, box, a, -1.5, 1.0, 5)
    got = {}
    for fused in (True, False):
        ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec, tol=1e-6, max_iter=100)
        try:
            dgp.dgp_set_hessian_fusion(ctx, fused)
            assert dgp.dgp_hessian_fusion(ctx) == fused
            t = [to_dev(torch_dev, v, torch.float32) for v in (*pos, *mom)]
            delta = torch.empty((n, n, n), dtype=torch.float32, device=dev)
            dgp.dgp_deposit(ctx, dgp.particles(*t), delta)
            phi = torch.empty_like(delta)
            st, info = dgp.dgp_solve_phi(ctx, a, delta, phi, 1e-6)
            D = torch.empty_like(delta)
            dgp.dgp_get_solution(ctx, D)
            got[fused] = (phi.double().cpu().numpy(), D.double().cpu().numpy(), info, dgp.dgp_solve_history(ctx))
        finally:
            dgp.dgp_destroy(ctx)
    (pf, Df, inf_f, hf), (ps, Ds, inf_s, hs) = got[True], got[False]
    assert inf_f["norm_res"] < 1e-6 and inf_s["norm_res"] < 1e-6
    assert abs(inf_f["iters"] - inf_s["iters"]) <= 1
    k = min(len(hf), len(hs))
    big = hs[:k] > 1e-4  # above the FP32 rounding floor of the residual
    assert np.allclose(hf[:k][big], hs[:k][big], rtol=2e-3, atol=0)
    assert rel_l2(Df, Ds) < 1e-5
    assert rel_l2(pf, ps) < 1e-5


def test_fused_pass_in_a_class_of_128cube(dgp, torch_dev):
    """Two 128^3 realisations form a class (no plane pass at this size): their class step uses
    the batched fused pass and must end where the separate passes end."""
    torch, dev = torch_dev
    cases = [(128, 180.0, 0.8, 21), (128, 240.0, 1.6, 22)]
    a0, a1, ns = 0.3, 0.4, 2
    dl = (math.log(a1) - math.log(a0)) / ns
    sched = [a0 * math.exp(i * dl) for i in range(ns + 1)]
    ics = [zel(n, bx, a0, -1.5, 0.8, seed, rc) for n, bx, rc, seed in cases]
    plist = [dgp.params(bx, n, rc, precision=dgp.DGP_MIXED_F32R, tol=1e-6, max_iter=200) for n, bx, rc, _ in cases]
    runs = {}
    for fused in (True, False):
        b, ctxs = dgp.dgp_batch_create(plist, OM)
        try:
            assert dgp.dgp_batch_classes(b, 2)[1] == 1
            for c in ctxs:
                dgp.dgp_set_hessian_fusion(c, fused)
                assert dgp.dgp_hessian_fusion(c) == fused
            tb = [[to_dev(torch_dev, v, torch.float32) for v in (*p, *m)] for p, m, _ in ics]
            parts = [dgp.particles(*t) for t in tb]
            infos = [dgp.dgp_batch_step(b, parts, [sched[i]] * 2, [sched[i + 1] - sched[i]] * 2) for i in range(ns)]
            runs[fused] = ([np.stack([v.cpu().numpy() for v in t]).astype(np.float64) for t in tb], infos)
        finally:
            dgp.dgp_batch_destroy(b)
    (gf, i_f), (gs, i_s) = runs[True], runs[False]
    for sf, ss in zip(i_f, i_s):
        for x, y in zip(sf, ss):
            assert x["status"] == dgp.DGP_OK and x["norm_res"] < 1e-6
            assert abs(x["iters"] - y["iters"]) <= 1
    for k in range(2):
        assert rel_l2(gf[k], gs[k]) < 2e-5, k
