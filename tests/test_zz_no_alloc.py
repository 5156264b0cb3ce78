"""P(k) through the entry point that allocates no device memory.

Some callers cannot call cudaMalloc at all: a host framework that reserved the
whole GPU for its own pooling allocator, or a loop that must not allocate once
it runs.  They cannot create a dgp context (dgp_init allocates its workspace),
so dgp_power_spectrum_noalloc computes P(k) of a small mesh field with all its
temporaries in a fixed device array that is part of the library.  This file
checks, through the C ABI, that two calls in a row give the same result as the
ordinary power_spectrum entry point, that a mesh too large for the fixed
array is refused, and that the first call of a fresh process, made from a
side stream, already gives the oracle's P(k).  It is named to run after every
other test module.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    from paper_0906_4548_gb300 import dgp
    return torch, dgp


def _reference(dgp, torch, d, n, box, nbins):
    ctx = dgp.dgp_init(box, n, 1.0, 0.27, precision=dgp.DGP_FP32)
    try:
        return dgp.power_spectrum(ctx, d, nbins)
    finally:
        dgp.dgp_destroy(ctx)


def test_noalloc_power_spectrum_matches_power_spectrum_twice(env):
    torch, dgp = env
    dev = torch.device("cuda:0")
    cases = [(64, 150.0, 32, 1), (32, 80.0, 11, 2)]  # two calls in a row, different sizes
    got = []
    for n, box, nbins, seed in cases:
        d = torch.tensor(np.random.default_rng(seed).standard_normal((n, n, n)), dtype=torch.float32, device=dev)
        got.append((dgp.dgp_power_spectrum_noalloc(d, n, box, nbins), _reference(dgp, torch, d, n, box, nbins)))
    for (k, P, cnt), (kr, Pr, cr) in got:
        assert np.array_equal(cnt, cr)
        assert np.allclose(k, kr, rtol=1e-12)
        assert np.max(np.abs(P / Pr - 1)) < 2e-6


def test_noalloc_rejects_a_mesh_larger_than_its_array(env):
    torch, dgp = env
    n = 2 * dgp.DGP_NOALLOC_MAX_N
    d = torch.zeros((n, n, n), dtype=torch.float32, device="cuda:0")
    with pytest.raises(dgp.DgpError) as e:
        dgp.dgp_power_spectrum_noalloc(d, n, 100.0, 4)
    assert e.value.status == dgp.DGP_E_INVALID


_FIRST_CALL_ON_SIDE_STREAM = r"""
import numpy as np, torch
from paper_0906_4548_gb300 import dgp
from oracle import estimators as oest
n, box, nbins = 64, 150.0, 32
f = np.random.default_rng(9).standard_normal((n, n, n)).astype(np.float32)
d = torch.tensor(f, device="cuda:0")
torch.cuda.synchronize()
s = torch.cuda.Stream()
k, P, c = dgp.dgp_power_spectrum_noalloc(d, n, box, nbins, stream=s.cuda_stream)
k2, P2, c2 = dgp.dgp_power_spectrum_noalloc(d, n, box, nbins, stream=s.cuda_stream)
ko, Po, co = oest.power_spectrum(f.astype(np.float64), box, nbins)
assert np.array_equal(c, co), (c, co)
assert np.allclose(k, ko, rtol=1e-12)
assert np.max(np.abs(P / Po - 1)) < 2e-6, np.max(np.abs(P / Po - 1))
assert np.array_equal(P, P2) and np.array_equal(k, k2) and np.array_equal(c, c2)
print("ok")
"""


def test_noalloc_first_call_from_a_side_stream_matches_the_oracle(env):
    """The first call of a process sets the array up (its twiddle tables are copied in).  Made from
    a non-blocking side stream, in a fresh process, it must already give the oracle's P(k), and a
    second call the same bits."""
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_ON_SIDE_STREAM], cwd=ROOT, capture_output=True,
                       text=True, timeout=900, env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]
