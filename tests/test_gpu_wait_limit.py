"""Bounded waits inside the relaxation kernel.

The FP32-data relaxation pass waits on its own asynchronous tile copies.  Each wait has a time
bound; when it runs out the kernel records a fault, waits for the copies it did issue, and returns,
and the solve reports DGP_E_TIMEOUT.  The test makes a wait run out without any fault on the GPU:
the test hook leaves one copy unissued (so its barrier is never completed), with a 1 ms bound.
The context must then solve normally again, to the oracle's phi.
"""
import numpy as np
import pytest

from oracle import field as ofield
from oracle import pm as opm
from test_gpu_parity import OM, rel_l2, to_dev, zel
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("side_stream", [False, True])
def test_wait_runs_out_then_context_solves_again(dgp, torch_dev, side_stream):
    torch, dev = torch_dev
    n, box, a = 64, 200.0, 0.5
    pos, _, _ = zel(n, box, a, -1.5, 0.5, 13)
    delta = opm.density_contrast(opm.cic_deposit(pos, n, box))
    phi_o, _, _, _ = ofield.solve_phi(delta, a, box, OM, 1.0, tol=1e-12, max_iter=300)
    s = torch.cuda.Stream(device=dev) if side_stream else None
    kw = {"stream": s.cuda_stream} if s is not None else {}
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_MIXED_EFT, tol=1e-6, max_iter=100, **kw)
    try:
        d = to_dev(torch_dev, delta, torch.float32)
        phi = torch.zeros_like(d)
        torch.cuda.synchronize()
        dgp.dgp_set_wait_limit(ctx, 1e-3, True)
        with pytest.raises(dgp.DgpError) as e:
            dgp.dgp_solve_phi(ctx, a, d, phi, 1e-6)
        assert e.value.status == dgp.DGP_E_TIMEOUT
        dgp.dgp_set_wait_limit(ctx, 2.0, False)
        st, info = dgp.dgp_solve_phi(ctx, a, d, phi, 1e-6)
        torch.cuda.synchronize()
        got = phi.double().cpu().numpy()
    finally:
        dgp.dgp_destroy(ctx)
    assert st == dgp.DGP_OK and info["norm_res"] < 1e-6
    assert rel_l2(got, phi_o) < 1e-5


def test_wait_limit_rejects_bad_bounds(dgp, torch_dev):
    ctx = dgp.dgp_init(100.0, 16, 1.0, OM, precision=dgp.DGP_FP32)
    try:
        for bad in (0.0, -1.0, 61.0, float("nan")):
            with pytest.raises(dgp.DgpError) as e:
                dgp.dgp_set_wait_limit(ctx, bad)
            assert e.value.status == dgp.DGP_E_INVALID
    finally:
        dgp.dgp_destroy(ctx)
