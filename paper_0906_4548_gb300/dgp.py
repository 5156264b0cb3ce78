"""Thin ctypes binding of the DGP CUDA library (include/dgp.h).

Argument marshalling only: every computation runs in libdgp.so.  Functions
carry the C names; device buffers are passed as torch CUDA tensors (their
data_ptr), host outputs come back as numpy arrays.  Importing this module
raises if the library has not been built: there is no fallback.
"""

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libdgp.so")

DGP_OK, DGP_E_INVALID, DGP_E_CUDA, DGP_E_NOMEM, DGP_E_NONFINITE = 0, 1, 2, 3, 4
DGP_E_NOT_CONVERGED, DGP_E_BAD_POINTS, DGP_E_TIMEOUT, DGP_E_STATE = 5, 6, 7, 8
DGP_FP32, DGP_MIXED, DGP_FP64, DGP_MIXED_EFT, DGP_MIXED_F32R = 0, 1, 2, 3, 4
DGP_GRAVITY_NL, DGP_GRAVITY_LDGP, DGP_GRAVITY_GRH, DGP_GRAVITY_SPH = 0, 1, 2, 3
C_OVER_H0 = 2997.92458

EXPORTED = ["dgp_background", "dgp_init", "dgp_destroy", "dgp_strerror", "dgp_reset", "dgp_solve_phi",
            "dgp_solve_forces", "dgp_solve_history", "dgp_get_solution", "dgp_deposit", "pm_step", "pm_step_host", "power_spectrum", "bispectrum",
            "dgp_profile", "dgp_profile_read", "dgp_kernel_name", "dgp_power_spectrum_noalloc",
            "dgp_sort_particles", "dgp_profile_kinds", "dgp_brane_spectra", "dgp_set_blocking_sync",
            "dgp_batch_create", "dgp_batch_context", "dgp_batch_step", "dgp_batch_destroy",
            "dgp_solve_adjoint", "pm_step_adjoint", "dgp_zeldovich", "dgp_zeldovich_adjoint",
            "dgp_power_spectrum_adjoint", "dgp_tile_config", "dgp_set_tile_config",
            "dgp_solve_adjoint_rc", "pm_step_adjoint_rc", "dgp_zeldovich_vf_adjoint", "dgp_velocity_factor",
            "dgp_workspace_size", "dgp_time_factors", "dgp_background_drc", "dgp_profile_sampled",
            "dgp_set_wait_limit", "dgp_batch_classes", "dgp_batch_set_plane_pass", "dgp_set_hessian_fusion",
            "dgp_hessian_fusion"]
DGP_NOALLOC_MAX_N = 64
DGP_KERNEL_KINDS = 11


class DgpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, strerror(status), status))


class Cosmology(ctypes.Structure):
    _fields_ = [("omega_m0", ctypes.c_double), ("c_over_H0", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("n", ctypes.c_int), ("rc_H0", ctypes.c_double),
                ("w", ctypes.c_double), ("precision", ctypes.c_int), ("gravity", ctypes.c_int),
                ("local_only", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("sort_every", ctypes.c_int), ("a_nonlinear", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("norm_res", ctypes.c_double), ("min_norm_res", ctypes.c_double),
                ("bad_fraction", ctypes.c_double), ("eps", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Workspace(ctypes.Structure):
    _fields_ = [("base", ctypes.c_size_t), ("sort", ctypes.c_size_t), ("adjoint", ctypes.c_size_t),
                ("host_step", ctypes.c_size_t)]


class Particles(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("px", ctypes.c_void_p), ("py", ctypes.c_void_p), ("pz", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class Background(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in
                ("E", "eta", "alpha", "beta", "s", "c2", "c3", "q", "omega_m", "geff_local", "growth_D",
                 "growth_f")]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libdgp.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    vp, d, i, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "dgp_background": (i, [P(Cosmology), d, d, P(Background)]),
        "dgp_init": (i, [P(vp), P(Params), P(Cosmology), vp]),
        "dgp_destroy": (None, [vp]),
        "dgp_strerror": (ctypes.c_char_p, [i]),
        "dgp_reset": (i, [vp]),
        "dgp_solve_phi": (i, [vp, d, vp, vp, d, P(SolveInfo)]),
        "dgp_solve_forces": (i, [vp, d, vp, vp, vp, vp, vp, d, P(SolveInfo)]),
        "dgp_get_solution": (i, [vp, vp]),
        "dgp_solve_history": (i, [vp, P(d), i]),
        "dgp_deposit": (i, [vp, P(Particles), vp]),
        "pm_step": (i, [vp, P(Particles), d, d, P(SolveInfo)]),
        "pm_step_host": (i, [vp, P(Particles), d, d, P(SolveInfo)]),
        "power_spectrum": (i, [vp, vp, i, P(d), P(d), P(i64)]),
        "bispectrum": (i, [vp, vp, d, d, i, P(d), d, P(d), P(d)]),
        "dgp_profile": (i, [vp, i]),
        "dgp_profile_kinds": (i, [vp, ctypes.c_uint]),
        "dgp_profile_sampled": (i, [vp, ctypes.c_uint]),
        "dgp_set_wait_limit": (i, [vp, d, i]),
        "dgp_batch_classes": (i, [vp, P(i), P(i)]),
        "dgp_batch_set_plane_pass": (i, [vp, i]),
        "dgp_set_hessian_fusion": (i, [vp, i]),
        "dgp_hessian_fusion": (i, [vp, P(i)]),
        "dgp_profile_read": (i, [vp, i, P(i64), P(d), P(i64), P(d), P(d)]),
        "dgp_kernel_name": (ctypes.c_char_p, [i]),
        "dgp_power_spectrum_noalloc": (i, [vp, i, d, i, P(d), P(d), P(i64), vp]),
        "dgp_sort_particles": (i, [vp, P(Particles), vp]),
        "dgp_brane_spectra": (i, [vp, i, P(d), P(d), P(d), P(d), P(i64)]),
        "dgp_set_blocking_sync": (i, [vp, i]),
        "dgp_tile_config": (i, [vp, P(i)]),
        "dgp_set_tile_config": (i, [vp, i]),
        "dgp_solve_adjoint": (i, [vp, vp, vp, vp, vp, vp, d, P(SolveInfo)]),
        "pm_step_adjoint": (i, [vp, P(Particles), d, d, P(Particles)]),
        "dgp_solve_adjoint_rc": (i, [vp, vp, vp, vp, vp, vp, d, P(d), P(SolveInfo)]),
        "pm_step_adjoint_rc": (i, [vp, P(Particles), d, d, P(Particles), P(d)]),
        "dgp_zeldovich_vf_adjoint": (i, [vp, vp, P(Particles), P(d)]),
        "dgp_velocity_factor": (i, [P(Cosmology), d, d, P(d), P(d)]),
        "dgp_workspace_size": (i, [P(Params), ctypes.c_int64, P(Workspace)]),
        "dgp_time_factors": (i, [P(Cosmology), d, d, d, P(d)]),
        "dgp_background_drc": (i, [P(Cosmology), d, d, P(Background)]),
        "dgp_zeldovich": (i, [vp, vp, d, P(Particles)]),
        "dgp_zeldovich_adjoint": (i, [vp, P(Particles), d, vp]),
        "dgp_power_spectrum_adjoint": (i, [vp, P(Particles), i, P(d), P(Particles)]),
        "dgp_batch_create": (i, [P(vp), i, P(Params), P(Cosmology)]),
        "dgp_batch_context": (i, [vp, i, P(vp)]),
        "dgp_batch_step": (i, [vp, P(Particles), P(d), P(d), P(SolveInfo), vp]),
        "dgp_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def strerror(status):
    return lib.dgp_strerror(int(status)).decode()


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _check(status, where, allow=(DGP_OK,)):
    if status not in allow:
        raise DgpError(status, where)
    return status


def dgp_background(omega_m0, rc_H0, a, c_over_H0=C_OVER_H0):
    out = Background()
    _check(lib.dgp_background(ctypes.byref(Cosmology(omega_m0, c_over_H0)), rc_H0, a, ctypes.byref(out)),
           "dgp_background")
    return {f: getattr(out, f) for f, _ in Background._fields_}


def dgp_init(box, n, rc_H0, omega_m0=0.27, w=1.0 / 3.0, precision=DGP_MIXED, gravity=DGP_GRAVITY_NL,
             local_only=False, max_iter=100, tol=1e-6, stream=None, c_over_H0=C_OVER_H0, sort_every=0,
             a_nonlinear=0.0):
    """Returns an opaque context handle (ctypes.c_void_p)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    ctx = ctypes.c_void_p()
    p = Params(box, n, rc_H0, w, precision, gravity, 1 if local_only else 0, max_iter, tol, sort_every,
               a_nonlinear)
    _check(lib.dgp_init(ctypes.byref(ctx), ctypes.byref(p), ctypes.byref(Cosmology(omega_m0, c_over_H0)),
                        ctypes.c_void_p(stream)), "dgp_init")
    return ctx


def params(box, n, rc_H0, w=1.0 / 3.0, precision=DGP_MIXED, gravity=DGP_GRAVITY_NL, local_only=False,
           max_iter=100, tol=1e-6, sort_every=0, a_nonlinear=0.0):
    return Params(box, n, rc_H0, w, precision, gravity, 1 if local_only else 0, max_iter, tol, sort_every,
                  a_nonlinear)


def dgp_background_drc(omega_m0, rc_H0, a, c_over_H0=C_OVER_H0):
    """d/d(r_c H0) of every member of dgp_background (host)."""
    out = Background()
    _check(lib.dgp_background_drc(ctypes.byref(Cosmology(omega_m0, c_over_H0)), rc_H0, a, ctypes.byref(out)),
           "dgp_background_drc")
    return {f: getattr(out, f) for f, _ in Background._fields_}


def dgp_time_factors(omega_m0, rc_H0, a0, a1, c_over_H0=C_OVER_H0):
    """(kick, drift, d kick / d(r_c H0), d drift / d(r_c H0)) between a0 and a1 (host)."""
    out = (ctypes.c_double * 4)()
    _check(lib.dgp_time_factors(ctypes.byref(Cosmology(omega_m0, c_over_H0)), rc_H0, a0, a1, out),
           "dgp_time_factors")
    return tuple(out)


def dgp_workspace_size(n, precision=DGP_MIXED, max_iter=100, np_particles=0):
    """Device bytes a context requests (host-only, see dgp.h): {"base", "sort", "adjoint", "host_step"}."""
    out = Workspace()
    _check(lib.dgp_workspace_size(ctypes.byref(params(1.0, n, 1.0, precision=precision, max_iter=max_iter)),
                                  int(np_particles), ctypes.byref(out)), "dgp_workspace_size")
    return {f: getattr(out, f) for f, _ in Workspace._fields_}


def dgp_batch_create(param_list, omega_m0=0.27, c_over_H0=C_OVER_H0):
    """A batch of len(param_list) contexts (see params()); returns (handle, [contexts])."""
    arr = (Params * len(param_list))(*param_list)
    b = ctypes.c_void_p()
    _check(lib.dgp_batch_create(ctypes.byref(b), len(param_list), arr, ctypes.byref(Cosmology(omega_m0, c_over_H0))),
           "dgp_batch_create")
    ctxs = []
    for i in range(len(param_list)):
        c = ctypes.c_void_p()
        _check(lib.dgp_batch_context(b, i, ctypes.byref(c)), "dgp_batch_context")
        ctxs.append(c)
    return b, ctxs


def dgp_batch_step(batch, parts_list, a, da, stream=None):
    """pm_step of every realisation; returns the list of solve infos."""
    import torch
    n = len(parts_list)
    parts = (Particles * n)(*parts_list)
    av = np.ascontiguousarray(a, dtype=np.float64)
    dv = np.ascontiguousarray(da, dtype=np.float64)
    infos = (SolveInfo * n)()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.dgp_batch_step(batch, parts, av.ctypes.data_as(dp), dv.ctypes.data_as(dp), infos,
                              ctypes.c_void_p(stream)), "dgp_batch_step")
    return [x.as_dict() for x in infos]


def dgp_batch_classes(batch, count):
    """(class of each realisation, number of classes and lone contexts)."""
    cls = (ctypes.c_int * count)()
    nc = ctypes.c_int()
    _check(lib.dgp_batch_classes(batch, cls, ctypes.byref(nc)), "dgp_batch_classes")
    return list(cls), nc.value


def dgp_set_hessian_fusion(ctx, on):
    """Fused Hessian x pass and inverse y pass (n = 128 or 256, FP32 data) on or off (the default)."""
    _check(lib.dgp_set_hessian_fusion(ctx, 1 if on else 0), "dgp_set_hessian_fusion")


def dgp_hessian_fusion(ctx):
    """True when the context's solves use the fused Hessian pass."""
    v = ctypes.c_int()
    _check(lib.dgp_hessian_fusion(ctx, ctypes.byref(v)), "dgp_hessian_fusion")
    return bool(v.value)


def dgp_batch_set_plane_pass(batch, on):
    """Plane-resident Hessian pass for the classes of n <= 96 (on, the default) or the separate passes."""
    _check(lib.dgp_batch_set_plane_pass(batch, 1 if on else 0), "dgp_batch_set_plane_pass")


def dgp_batch_destroy(batch):
    lib.dgp_batch_destroy(batch)


def dgp_destroy(ctx):
    lib.dgp_destroy(ctx)


def dgp_reset(ctx):
    _check(lib.dgp_reset(ctx), "dgp_reset")


def dgp_solve_phi(ctx, a, delta, phi, tol):
    info = SolveInfo()
    st = _check(lib.dgp_solve_phi(ctx, a, _ptr(delta), _ptr(phi), tol, ctypes.byref(info)), "dgp_solve_phi",
                (DGP_OK, DGP_E_NOT_CONVERGED))
    return st, info.as_dict()


def dgp_solve_forces(ctx, a, delta, phi, gx, gy, gz, tol):
    info = SolveInfo()
    st = _check(lib.dgp_solve_forces(ctx, a, _ptr(delta), _ptr(phi), _ptr(gx), _ptr(gy), _ptr(gz), tol,
                                     ctypes.byref(info)), "dgp_solve_forces", (DGP_OK, DGP_E_NOT_CONVERGED))
    return st, info.as_dict()


def dgp_solve_history(ctx):
    n = lib.dgp_solve_history(ctx, None, 0)
    if n < 0:
        raise DgpError(-n, "dgp_solve_history")
    out = np.zeros(n)
    lib.dgp_solve_history(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
    return out


def dgp_solve_adjoint(ctx, phibar, deltabar, tol, gbar=None):
    """deltabar for a cotangent phibar (and/or gbar = (gx, gy, gz)) of the last accepted solve."""
    info = SolveInfo()
    g = gbar if gbar is not None else (None, None, None)
    st = _check(lib.dgp_solve_adjoint(ctx, _ptr(phibar), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(deltabar), tol,
                                      ctypes.byref(info)), "dgp_solve_adjoint", (DGP_OK, DGP_E_NOT_CONVERGED))
    return st, info.as_dict()


def dgp_solve_adjoint_rc(ctx, phibar, deltabar, tol, gbar=None):
    """dgp_solve_adjoint plus the solve's explicit derivative in r_c H0: (status, info, rc_bar)."""
    info = SolveInfo()
    rc = ctypes.c_double()
    g = gbar if gbar is not None else (None, None, None)
    st = _check(lib.dgp_solve_adjoint_rc(ctx, _ptr(phibar), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(deltabar),
                                         tol, ctypes.byref(rc), ctypes.byref(info)),
                "dgp_solve_adjoint_rc", (DGP_OK, DGP_E_NOT_CONVERGED))
    return st, info.as_dict(), rc.value


def pm_step_adjoint(ctx, start, a, da, cot):
    """cot (Particles of cotangents (xbar1, pbar1)) <- (xbar0, pbar0) for the step from `start` at a."""
    _check(lib.pm_step_adjoint(ctx, ctypes.byref(start), a, da, ctypes.byref(cot)), "pm_step_adjoint")


def pm_step_adjoint_rc(ctx, start, a, da, cot):
    """pm_step_adjoint; returns the step's explicit derivative in r_c H0."""
    rc = ctypes.c_double()
    _check(lib.pm_step_adjoint_rc(ctx, ctypes.byref(start), a, da, ctypes.byref(cot), ctypes.byref(rc)),
           "pm_step_adjoint_rc")
    return rc.value


def dgp_zeldovich_vf_adjoint(ctx, delta_l, cot):
    """sum_j <pbar_j, Psi_j(delta_L)>: the cotangent of vel_factor in dgp_zeldovich."""
    v = ctypes.c_double()
    _check(lib.dgp_zeldovich_vf_adjoint(ctx, _ptr(delta_l), ctypes.byref(cot), ctypes.byref(v)),
           "dgp_zeldovich_vf_adjoint")
    return v.value


def dgp_velocity_factor(omega_m0, rc_H0, a, c_over_H0=C_OVER_H0):
    """(vf, d vf / d(r_c H0)) for the Zel'dovich velocity factor vf = a^2 E f (host)."""
    vf, dvf = ctypes.c_double(), ctypes.c_double()
    _check(lib.dgp_velocity_factor(ctypes.byref(Cosmology(omega_m0, c_over_H0)), rc_H0, a, ctypes.byref(vf),
                                   ctypes.byref(dvf)), "dgp_velocity_factor")
    return vf.value, dvf.value


def dgp_zeldovich(ctx, delta_l, vel_factor, out):
    _check(lib.dgp_zeldovich(ctx, _ptr(delta_l), vel_factor, ctypes.byref(out)), "dgp_zeldovich")


def dgp_zeldovich_adjoint(ctx, cot, vel_factor, delta_l_bar):
    _check(lib.dgp_zeldovich_adjoint(ctx, ctypes.byref(cot), vel_factor, _ptr(delta_l_bar)), "dgp_zeldovich_adjoint")


def dgp_power_spectrum_adjoint(ctx, parts, dl_dp, cot):
    g = np.ascontiguousarray(dl_dp, dtype=np.float64)
    _check(lib.dgp_power_spectrum_adjoint(ctx, ctypes.byref(parts), g.size,
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cot)),
           "dgp_power_spectrum_adjoint")


def dgp_tile_config(ctx):
    v = ctypes.c_int()
    _check(lib.dgp_tile_config(ctx, ctypes.byref(v)), "dgp_tile_config")
    return {"y_threads": v.value}


def dgp_set_tile_config(ctx, y_threads):
    _check(lib.dgp_set_tile_config(ctx, int(y_threads)), "dgp_set_tile_config")


def dgp_set_wait_limit(ctx, seconds, withhold_first_copy=False):
    """Bound of the relaxation kernel's waits; withhold_first_copy is the test hook of dgp.h."""
    _check(lib.dgp_set_wait_limit(ctx, float(seconds), 1 if withhold_first_copy else 0), "dgp_set_wait_limit")


def dgp_get_solution(ctx, D):
    _check(lib.dgp_get_solution(ctx, _ptr(D)), "dgp_get_solution")


def particles(x, y, z, px, py, pz):
    return Particles(_ptr(x), _ptr(y), _ptr(z), _ptr(px), _ptr(py), _ptr(pz), int(x.numel() if hasattr(x, "numel") else x.size))


def dgp_deposit(ctx, parts, delta):
    _check(lib.dgp_deposit(ctx, ctypes.byref(parts), _ptr(delta)), "dgp_deposit")


def dgp_sort_particles(ctx, parts, cell_start=None):
    """Cell-sorts the particle arrays in place; cell_start: None or a device int32 tensor of n^3 + 1."""
    _check(lib.dgp_sort_particles(ctx, ctypes.byref(parts), _ptr(cell_start)), "dgp_sort_particles")


def pm_step(ctx, parts, a, da):
    info = SolveInfo()
    _check(lib.pm_step(ctx, ctypes.byref(parts), a, da, ctypes.byref(info)), "pm_step")
    return info.as_dict()


def pm_step_host(ctx, parts, a, da):
    info = SolveInfo()
    _check(lib.pm_step_host(ctx, ctypes.byref(parts), a, da, ctypes.byref(info)), "pm_step_host")
    return info.as_dict()


def power_spectrum(ctx, delta, nbins):
    k = np.zeros(nbins)
    pk = np.zeros(nbins)
    nm = np.zeros(nbins, dtype=np.int64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.power_spectrum(ctx, _ptr(delta), nbins, k.ctypes.data_as(dp), pk.ctypes.data_as(dp),
                              nm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "power_spectrum")
    return k, pk, nm


def dgp_brane_spectra(ctx, nbins):
    """(k, P_c, P_C, Delta_gradC, nmodes) of the accepted nonlinear solution."""
    out = [np.zeros(nbins) for _ in range(4)]
    nm = np.zeros(nbins, dtype=np.int64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.dgp_brane_spectra(ctx, nbins, *[o.ctypes.data_as(dp) for o in out],
                                 nm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "dgp_brane_spectra")
    return (*out, nm)


def bispectrum(ctx, delta, k1, k2, thetas, dk=0.0):
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    b = np.zeros(th.size)
    q = np.zeros(th.size)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.bispectrum(ctx, _ptr(delta), k1, k2, th.size, th.ctypes.data_as(dp), dk, b.ctypes.data_as(dp),
                          q.ctypes.data_as(dp)), "bispectrum")
    return b, q


def dgp_profile(ctx, timing, kinds=None):
    """Reset the kernel counters; time every kind (timing true), none, or only
    the kinds named in `kinds` (kernel names as returned by dgp_profile_read)."""
    if kinds is None:
        _check(lib.dgp_profile(ctx, 1 if timing else 0), "dgp_profile")
        return
    names = [lib.dgp_kernel_name(k).decode() for k in range(DGP_KERNEL_KINDS)]
    mask = 0
    for kname in kinds:
        mask |= 1 << names.index(kname)
    _check(lib.dgp_profile_kinds(ctx, mask), "dgp_profile_kinds")


def dgp_profile_sampled(ctx, kinds):
    """Reset the kernel counters and time, with graph replay kept on, the launches of the named kinds
    that run outside graphs and are sure to do their work (see dgp.h)."""
    names = [lib.dgp_kernel_name(k).decode() for k in range(DGP_KERNEL_KINDS)]
    mask = 0
    for kname in kinds:
        mask |= 1 << names.index(kname)
    _check(lib.dgp_profile_sampled(ctx, mask), "dgp_profile_sampled")


def dgp_profile_read(ctx):
    """{kernel name: dict(launches, bytes, timed, ms, timed_bytes)} since the last dgp_profile."""
    out = {}
    for kind in range(DGP_KERNEL_KINDS):
        l, t = ctypes.c_int64(), ctypes.c_int64()
        b, ms, tb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib.dgp_profile_read(ctx, kind, ctypes.byref(l), ctypes.byref(b), ctypes.byref(t), ctypes.byref(ms),
                                    ctypes.byref(tb)), "dgp_profile_read")
        out[lib.dgp_kernel_name(kind).decode()] = dict(launches=l.value, bytes=b.value, timed=t.value, ms=ms.value,
                                                       timed_bytes=tb.value)
    return out


def dgp_power_spectrum_noalloc(delta, n, box, nbins, stream=None):
    """P(k) of an FP32 n^3 device field without a context and without any device
    allocation (n <= DGP_NOALLOC_MAX_N); same outputs as power_spectrum."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    k = np.zeros(nbins)
    pk = np.zeros(nbins)
    nm = np.zeros(nbins, dtype=np.int64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.dgp_power_spectrum_noalloc(_ptr(delta), n, box, nbins, k.ctypes.data_as(dp), pk.ctypes.data_as(dp),
                                          nm.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.c_void_p(stream)),
           "dgp_power_spectrum_noalloc")
    return k, pk, nm
