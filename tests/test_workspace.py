"""dgp_workspace_size (host-only): the device bytes of a context from its parameters, checked
against the sizes of the buffers the context allocates (fields F = 4 N^3 bytes for FP32 data,
half spectra (N/2 + 1) N^2 complex), without a GPU."""
import pytest

from paper_0906_4548_gb300 import dgp


@pytest.mark.parametrize("n", [16, 48, 96, 256])
def test_base_is_14_fields_and_9_spectra_plus_small_buffers(n):
    m, spec = n ** 3, (n // 2 + 1) * n * n
    for prec, t in ((dgp.DGP_MIXED, 4), (dgp.DGP_FP64, 8)):
        w = dgp.dgp_workspace_size(n, prec, max_iter=100)
        big = 14 * t * m + 9 * 2 * t * spec
        assert big <= w["base"] < big + 8 * 4 * (n // 2) * (n // 8 + 1) * (n // 2 + 1) + (1 << 20)
        assert w["sort"] == 3 * 4 * m + 4 * ((m + 2047) // 2048)          # no particles yet
        assert w["host_step"] == 0


def test_particle_terms_scale_with_np():
    n, npart = 64, 123457
    w0 = dgp.dgp_workspace_size(n, dgp.DGP_FP32)
    w1 = dgp.dgp_workspace_size(n, dgp.DGP_FP32, np_particles=npart)
    assert w1["base"] == w0["base"]
    assert w1["sort"] - w0["sort"] == (4 + 6 * 4) * npart
    assert w1["adjoint"] - w0["adjoint"] == 6 * 4 * npart
    assert w1["host_step"] == 6 * 4 * npart
    w64 = dgp.dgp_workspace_size(n, dgp.DGP_FP64, np_particles=npart)
    assert w64["host_step"] == 2 * w1["host_step"]


def test_256_context_is_about_1_5_gb():
    w = dgp.dgp_workspace_size(256, dgp.DGP_MIXED_EFT)
    assert 1.50e9 < w["base"] < 1.56e9


def test_invalid_arguments():
    for n, prec in ((40, dgp.DGP_MIXED), (64, 7), (64, -1)):
        with pytest.raises(dgp.DgpError):
            dgp.dgp_workspace_size(n, prec)
    with pytest.raises(dgp.DgpError):
        dgp.dgp_workspace_size(64, dgp.DGP_FP32, np_particles=-1)
