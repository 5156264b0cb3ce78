"""The C-ABI library loads and exports every symbol include/dgp.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dgp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\**\s*([a-z_0-9]+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_0906_4548_gb300 import dgp
    return dgp


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("dgp_init", "dgp_solve_phi", "pm_step", "power_spectrum", "bispectrum", "dgp_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib._LIB_PATH)
    for name in _declared():
        assert hasattr(so, name), name
    assert sorted(lib.EXPORTED) == _declared()


def test_host_only_calls_without_gpu(lib):
    # dgp_background is host code: compare with the oracle's background
    from oracle import background as bg
    for a in (0.02, 0.3, 1.0):
        b = lib.dgp_background(0.27, 1.0, a)
        c = bg.coefficients(a, 0.27, 1.0)
        for k in ("E", "eta", "alpha", "beta", "s", "c2", "c3", "q", "omega_m"):
            assert abs(b[k] - c[k]) <= 1e-13 * max(1.0, abs(c[k])), k
        assert abs(b["geff_local"] - bg.geff_local_over_G(a, 0.27, 1.0)) < 1e-13
        D, f = bg.growth(a, 0.27, 1.0)
        assert abs(b["growth_f"] - f) < 1e-10 and abs(b["growth_D"] / D - 1) < 1e-10
    assert lib.strerror(0) == "ok"
    with pytest.raises(lib.DgpError):
        lib.dgp_background(0.27, -1.0, 0.5)


def test_init_rejects_bad_parameters_before_touching_the_gpu(lib):
    for kw in (dict(n=40), dict(n=24), dict(n=0), dict(w=1.0), dict(rc_H0=0.0), dict(precision=7), dict(precision=-1),
               dict(sort_every=-1), dict(gravity=4), dict(a_nonlinear=-0.5)):
        args = dict(box=100.0, n=32, rc_H0=1.0, precision=lib.DGP_MIXED)
        args.update(kw)
        with pytest.raises(lib.DgpError) as e:
            lib.dgp_init(args.pop("box"), args.pop("n"), args.pop("rc_H0"), stream=0, **args)
        assert e.value.status == lib.DGP_E_INVALID
