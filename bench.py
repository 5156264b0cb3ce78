"""PM steps/s at 256^3 including the converged nonlinear DGP phi solve.

Workload (the 256^3 run): 256^3 particles on a 256^3 mesh in a 400 Mpc/h box,
seeded n_s = -1.5 power-law Gaussian field with mesh rms 0.5 at a = 0.02,
Zel'dovich initial conditions, r_c H0 = 1, Omega_m0 = 0.27, w = 1/3, steps
uniform in ln a from a = 0.02 to a = 1 in 200 steps, relaxation tolerance 1e-6
on <|R|>/eps every step, FP32 mesh/particles with FP64 residual, discriminant
and reductions (the residual R, split source B' and discriminant Delta are
evaluated on pairs of floats with error-free transformations, ~48 bits;
--precision mixed-fp64 evaluates them on the FP64 pipe instead).  A "step" is
one pm_step call (deposit, field solve, forces,
gather, kick-drift-kick).  The timed region runs K consecutive steps from
a = 0.02 (K = 200 is the whole run) after W warm-up steps and a reset to the
initial conditions.  Inputs (403 MB of particles, 64 MB mesh fields) exceed
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun, one process per GPU): independent replicas with distinct
seeds, no data-path collective; value = all ranks' steps / max rank time.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WL = dict(n=256, box=400.0, n_s=-1.5, rms=0.5, seed=3, a_start=0.02, a_end=1.0, run_steps=200, rc_H0=1.0,
          omega_m0=0.27, w=1.0 / 3.0, tol=1e-6, max_iter=100)
METRIC = "PM steps/s at 256³ incl. converged DGP φ solve; % HBM roofline; vs FP64 oracle"
UNIT = "steps/s"
# Mean residual evaluations per solve of this workload as measured on GB300
# (used by the oracle reference arm, which has no GPU run to read it from).
E_PER_SOLVE_REF = 20.8
# Cell sort cadence of the particles (pm_step sorts after every K-th drift; 0 = never).
SORT_EVERY = 8
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel kind from one ncu capture (summarised under profiles/), with the
# SHA-256 of the sources the captured kernel was built from: when they have
# changed since, the traffic is reported as null.
NCU_TRAFFIC = {
    "relax": {"bytes": 653.6e6, "sources": ["fused_relax.cu", "fft_core.cuh", "kernels.cuh", "common.cuh"],
              "sha256": "93c8181dd253cac10354af47bf0135d5395797029e7bb5097ebb2c03bc3b2efa",
              "profile": "profiles/k_fused_relax_256cube.md"},
}


def sources_sha256(names):
    import hashlib
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_0906_4548_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kind):
    rec = NCU_TRAFFIC.get(kind)
    if not rec or rec["bytes"] is None or rec["sha256"] != sources_sha256(rec["sources"]):
        return None
    return rec["bytes"]


PRECISION_DESC = {
    "mixed": "mixed: fp32 mesh/FFT/particles; residual, B', discriminant as error-free fp32 pairs "
             "(~48-bit); norms and reductions fp64",
    "mixed-fp64": "mixed: fp32 mesh/FFT/particles; residual, B', discriminant, norms and reductions fp64",
    "fp32": "fp32 throughout (fp64 cross-block sums only)",
}


def config(n_gpus, prec="mixed", sort_every=SORT_EVERY):
    return {"workload": "dgp_pm_%dcube_box%g_ns%g_rms%g_a%g-%g_%dsteps_tol%g" % (
        WL["n"], WL["box"], WL["n_s"], WL["rms"], WL["a_start"], WL["a_end"], WL["run_steps"], WL["tol"]),
        "mesh": WL["n"], "particles": WL["n"] ** 3, "box_mpc_h": WL["box"], "rc_H0": WL["rc_H0"],
        "w": WL["w"], "tol": WL["tol"], "precision": PRECISION_DESC[prec],
        "parallelism": "replicas" if n_gpus > 1 else "single", "cell_sort_every": sort_every,
        "l2": "inputs larger than L2 (particles 403 MB, fields 64 MB each); no flush"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_fft_sample_seconds(nsamples, n=None):
    """Time the FP64 oracle's FFT on the workload's mesh: each sample is one
    axis pass of its four-step DFT over a quarter of a 256^3 field (one
    twelfth of a 3D transform).  Runs in this process."""
    import numpy as np
    from oracle.fft import fft_axis
    n = WL["n"] if n is None else n
    rng = np.random.default_rng(0)
    f = rng.standard_normal((n, n, n))
    q = n // 4
    slabs = [(f[:q], 2), (f[:q], 1), (f[:, :q], 0)]
    fft_axis(slabs[0][0], slabs[0][1])  # untimed warm-up
    ts = []
    for j in range(nsamples):
        s, ax = slabs[j % 3]
        t0 = time.perf_counter()
        fft_axis(s, ax)
        ts.append(time.perf_counter() - t0)
    return ts


def oracle_steps_per_s(t_sample, e_per_solve):
    """An oracle PM step of this workload does one field solve with 6 + 9 E 3D
    transforms (E residual evaluations, each 1 forward + 8 inverse; plus delta,
    the source, phi and 3 forces); a 3D transform is 12 samples."""
    return 1.0 / (t_sample * 12.0 * (6.0 + 9.0 * e_per_solve))


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only)."""
    rank = replica_env()[1]
    if rank != 0:
        return 0
    cores = os.cpu_count()
    ts = oracle_fft_sample_seconds(args.warmup + args.steps)[args.warmup:]
    t = sum(ts) / len(ts)
    v = oracle_steps_per_s(t, E_PER_SOLVE_REF)
    sample = ("FP64 oracle four-step FFT, one axis pass over a quarter of the 256^3 field per step (%.3f s); "
              "steps/s = 1 / (12 x (6 + 9 x %.1f) x that): FFT work of one PM step with %.1f residual "
              "evaluations per solve; deposit, gather and pointwise work not counted (upper bound)"
              % (t, E_PER_SOLVE_REF, E_PER_SOLVE_REF))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config(args.gpus, "mixed"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# Batched workload: independent realisations of uneven meshes stepped together.
WB = dict(sizes=[48] * 16 + [64] * 16 + [96] * 16, box_range=(50.0, 200.0), rc_range=(0.5, 2.0), n_s=-1.5,
          rms=0.5, seed=100, a_start=0.02, a_end=1.0, run_steps=50, omega_m0=0.27, tol=1e-6, max_iter=100)


def run_batched(args):
    """48 realisations (16 x 48^3, 16 x 64^3, 16 x 96^3, particles = mesh cells), boxes and r_c H0
    drawn uniformly, distinct seeds, FP32, 50 steps each: the batch path (one context and stream per
    realisation, all stepped together) and the plain path (the same realisations stepped one after
    another on one stream).  value = realisation-steps per second of the batch path."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_0906_4548_gb300 import dgp, inputs
    rng = np.random.default_rng(WB["seed"])
    nr = len(WB["sizes"])
    boxes = rng.uniform(*WB["box_range"], nr)
    rcs = rng.uniform(*WB["rc_range"], nr)
    dev = torch.device("cuda", 0)
    ics = []
    for i, n in enumerate(WB["sizes"]):
        bgi = dgp.dgp_background(WB["omega_m0"], rcs[i], WB["a_start"])
        vf = WB["a_start"] ** 2 * bgi["E"] * bgi["growth_f"]
        pos, mom, _ = inputs.zeldovich_particles(n, boxes[i], WB["n_s"], WB["rms"], WB["seed"] + i, vf)
        ics.append([torch.tensor(v.astype(np.float32), device=dev) for v in (*pos, *mom)])
    cur = [[t.clone() for t in ic] for ic in ics]
    parts = [dgp.particles(*c) for c in cur]
    prec = dgp.DGP_FP32
    plist = [dgp.params(boxes[i], n, rcs[i], precision=prec, tol=WB["tol"], max_iter=WB["max_iter"],
                        sort_every=SORT_EVERY) for i, n in enumerate(WB["sizes"])]
    dlna = math.log(WB["a_end"] / WB["a_start"]) / WB["run_steps"]
    sched = [WB["a_start"] * math.exp(i * dlna) for i in range(WB["run_steps"] + 1)]
    steps = min(args.steps, WB["run_steps"])

    def restart(ctxs):
        for c, ic in zip(cur, ics):
            for x, y in zip(c, ic):
                x.copy_(y)
        for c in ctxs:
            dgp.dgp_reset(c)
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    b, ctxs = dgp.dgp_batch_create(plist, WB["omega_m0"])
    infos = []
    try:
        restart(ctxs)
        for i in range(args.warmup):
            dgp.dgp_batch_step(b, parts, [sched[i]] * nr, [sched[i + 1] - sched[i]] * nr)
        restart(ctxs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            time.sleep(0.3)
            e0.record(stream)
            t0 = time.perf_counter()
            for i in range(steps):
                infos.append(dgp.dgp_batch_step(b, parts, [sched[i]] * nr, [sched[i + 1] - sched[i]] * nr))
            e1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
        pk_batch = []
        for k in (0, 16, 32):
            dl = torch.empty((WB["sizes"][k],) * 3, dtype=torch.float32, device=dev)
            dgp.dgp_deposit(ctxs[k], parts[k], dl)
            pk_batch.append(dgp.power_spectrum(ctxs[k], dl, WB["sizes"][k] // 2)[1])
    finally:
        dgp.dgp_batch_destroy(b)
    # plain path: the same realisations, one context at a time on the current stream
    seq = [dgp.dgp_init(boxes[i], n, rcs[i], WB["omega_m0"], precision=prec, tol=WB["tol"],
                        max_iter=WB["max_iter"], sort_every=SORT_EVERY) for i, n in enumerate(WB["sizes"])]
    try:
        restart(seq)
        for i in range(args.warmup):
            for k in range(nr):
                dgp.pm_step(seq[k], parts[k], sched[i], sched[i + 1] - sched[i])
        restart(seq)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(steps):
            for k in range(nr):
                dgp.pm_step(seq[k], parts[k], sched[i], sched[i + 1] - sched[i])
        f1.record(stream)
        torch.cuda.synchronize()
        ms_seq = f0.elapsed_time(f1)
        diffs = []
        for j, k in enumerate((0, 16, 32)):
            dl = torch.empty((WB["sizes"][k],) * 3, dtype=torch.float32, device=dev)
            dgp.dgp_deposit(seq[k], parts[k], dl)
            pk = dgp.power_spectrum(seq[k], dl, WB["sizes"][k] // 2)[1]
            diffs.append(float(np.max(np.abs(pk_batch[j] / pk - 1))))
    finally:
        for c in seq:
            dgp.dgp_destroy(c)
    evals = [i["iters"] + 1 for step in infos for i in step]
    line = {"metric": "PM realisation-steps/s, 48 realisations (16 x 48^3, 16 x 64^3, 16 x 96^3) incl. "
                      "converged DGP phi solves", "value": nr * steps / (ms / 1000.0), "unit": "realisation-steps/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "dgp_pm_batched_48x(48,64,96)cube_box50-200_rc0.5-2_a0.02-1_50steps_tol1e-6",
                       "realisations": nr, "precision": PRECISION_DESC["fp32"], "cell_sort_every": SORT_EVERY,
                       "l2": "realisations' fields and particles (about 1.5 GB in total) exceed L2; no flush"},
            "wall_s": wall, "clocks": clk.summary(),
            "plain_path": {"value": nr * steps / (ms_seq / 1000.0), "ms_per_step": ms_seq / steps,
                           "how": "the same 48 contexts stepped one after another on one stream"},
            "end_pk_max_rel_diff_batch_vs_plain": max(diffs),
            "solver": {"evals_per_solve_mean": sum(evals) / len(evals), "max_evals": max(evals),
                       "not_converged": sum(1 for step in infos for i in step if i["status"] != 0)}}
    print(json.dumps(line))
    return 0


# Gradient workload: a P(k) loss after a 128^3 run, differentiated with respect to the linear field.
WA = dict(n=128, box=200.0, n_s=-1.5, rms=0.5, seed=3, target_seed=4, a_start=0.02, a_end=1.0, run_steps=100,
          every=10, omega_m0=0.27, rc_H0=1.0, tol=1e-6, max_iter=100)


def run_adjoint(args):
    """128^3 mesh and particles, FP32, 100 steps from a = 0.02 to 1 with a checkpoint every 10 steps:
    L = sum_k [P(k) - P_target(k)]^2 (target from a second seed), its gradient with respect to the
    128^3 linear field (initial Fourier modes) and to r_c H0 by the adjoint kernels, timed, and
    checked against central differences of the loss along --fd-modes random single Fourier modes
    and in r_c H0 (fresh contexts at r_c H0 +- h)."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_0906_4548_gb300 import autodiff, dgp, inputs
    n, box = WA["n"], WA["box"]
    dev = torch.device("cuda", 0)
    vf = dgp.dgp_velocity_factor(WA["omega_m0"], WA["rc_H0"], WA["a_start"])[0]
    dl = torch.tensor(inputs.linear_field(n, box, WA["n_s"], WA["rms"], WA["seed"])[0], dtype=torch.float32,
                      device=dev)
    dl_t = torch.tensor(inputs.linear_field(n, box, WA["n_s"], WA["rms"], WA["target_seed"])[0],
                        dtype=torch.float32, device=dev)
    dlna = math.log(WA["a_end"] / WA["a_start"]) / WA["run_steps"]
    nsteps = args.adjoint_steps if args.adjoint_steps else WA["run_steps"]
    sched = [WA["a_start"] * math.exp(i * dlna) for i in range(nsteps + 1)]
    nb = n // 2
    fd64 = args.fd_precision == "fp64"
    ctx = dgp.dgp_init(box, n, WA["rc_H0"], WA["omega_m0"], precision=dgp.DGP_FP32, tol=WA["tol"],
                       max_iter=WA["max_iter"], sort_every=0)
    stream = torch.cuda.current_stream()
    try:
        def final_pk(field):
            x, p = autodiff.ZeldovichIC.apply(field, ctx, vf)
            dgp.dgp_reset(ctx)
            x, p = autodiff.PMRun.apply(x, p, ctx, sched, WA["every"])
            delta = torch.empty((n, n, n), dtype=field.dtype, device=dev)
            xc = x.detach().contiguous()
            dgp.dgp_deposit(ctx, dgp.particles(xc[0], xc[1], xc[2], xc[0], xc[1], xc[2]), delta)
            return dgp.power_spectrum(ctx, delta, nb)[1]

        target = final_pk(dl_t)
        w = np.ones(nb)

        def loss(field, grad, c=None, rc=WA["rc_H0"]):
            c = ctx if c is None else c
            d = field.clone().requires_grad_(grad)
            rt = torch.tensor(rc, dtype=torch.float64, requires_grad=grad)
            vfr = autodiff.VelocityFactor.apply(rt, WA["omega_m0"], WA["a_start"])
            x, p = autodiff.ZeldovichIC.apply(d, c, vfr)
            dgp.dgp_reset(c)
            x, p = autodiff.PMRun.apply(x, p, c, sched, WA["every"], rt)
            loss.rt = rt
            return autodiff.PkLoss.apply(x, c, n, target, w), d

        for _ in range(max(1, min(args.warmup, 1))):   # one untimed forward + backward
            L, d = loss(dl, True)
            L.backward()
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        with ClockSampler(0) as clk:
            time.sleep(0.3)
            e0.record(stream)
            L, d = loss(dl, True)
            e1.record(stream)
            L.backward()
            e2.record(stream)
            torch.cuda.synchronize()
        ms_fwd, ms_bwd = e0.elapsed_time(e1), e1.elapsed_time(e2)
        loss_value = float(L.detach())
        grad = d.grad.detach().double().cpu().numpy()
        rc_grad = float(loss.rt.grad)
        prec_fd = dgp.DGP_FP32
        if fd64:
            # the accuracy check in FP64 (tolerance 1e-10): FP32 rounding and a 1e-6 solver
            # tolerance, amplified over 100 steps, swamp small central differences
            dgp.dgp_destroy(ctx)
            ctx = dgp.dgp_init(box, n, WA["rc_H0"], WA["omega_m0"], precision=dgp.DGP_FP64, tol=1e-10,
                               max_iter=300, sort_every=0)
            dl, dl_t = dl.double(), dl_t.double()
            target = final_pk(dl_t)
            L64, d64 = loss(dl, True)
            L64.backward()
            grad = d64.grad.detach().cpu().numpy()
            rc_grad = float(loss.rt.grad)
            prec_fd = dgp.DGP_FP64
        # central differences along random single modes of the linear field
        rng = np.random.default_rng(0)
        xg = np.arange(n) * box / n
        fd = []
        for t in range(args.fd_modes):
            k = rng.integers(1, n // 4, 3)
            u = np.cos(2 * np.pi / box * (k[0] * xg[:, None, None] + k[1] * xg[None, :, None]
                                          + k[2] * xg[None, None, :]) + rng.uniform(0, 2 * np.pi))
            e = (1e-4 if fd64 else 2e-3) * WA["rms"]
            ut = torch.tensor(u, dtype=dl.dtype, device=dev)
            lp = float(loss(dl + e * ut, False)[0])
            lm = float(loss(dl - e * ut, False)[0])
            f = (lp - lm) / (2 * e)
            a_ = float(np.sum(grad * u))
            fd.append({"mode": [int(v) for v in k], "central_difference": f, "adjoint": a_,
                       "rel_diff": abs(f - a_) / max(abs(f), 1e-300)})
        # central difference in r_c H0 (r_c is a constant of a context: one context per value)
        h = (1e-4 if fd64 else 1e-3) * WA["rc_H0"]
        lrc = []
        for r in (WA["rc_H0"] + h, WA["rc_H0"] - h):
            c2 = dgp.dgp_init(box, n, r, WA["omega_m0"], precision=prec_fd, tol=1e-10 if fd64 else WA["tol"],
                              max_iter=300 if fd64 else WA["max_iter"], sort_every=0)
            try:
                lrc.append(float(loss(dl, False, c2, r)[0]))
            finally:
                dgp.dgp_destroy(c2)
        fd_rc = (lrc[0] - lrc[1]) / (2 * h)
    finally:
        dgp.dgp_destroy(ctx)
    rel = [x["rel_diff"] for x in fd]
    line = {"metric": "gradient evaluations/s of a P(k) loss after a 128^3, 100-step DGP PM run (adjoint kernels, "
                      "checkpoint every 10 steps)", "value": 1000.0 / (ms_fwd + ms_bwd),
            "unit": "gradients/s", "n_gpus": 1, "steps": nsteps, "warmup": 1,
            "ms_per_step": (ms_fwd + ms_bwd) / nsteps, "final_a": sched[-1], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "dgp_pm_adjoint_128cube_box200_ns-1.5_a0.02-1_100steps_every10_tol1e-6",
                       "gradient_wrt": "the 128^3 linear field delta_L (initial Fourier modes) and r_c H0",
                       "l2": "particles (25 MB per array) and fields (8 MB each) partly fit L2; no flush"},
            "forward_ms": ms_fwd, "backward_ms": ms_bwd, "backward_over_forward": ms_bwd / ms_fwd,
            "loss": loss_value, "clocks": clk.summary(),
            "rc_gradient": {"adjoint": rc_grad, "central_difference": fd_rc, "h": h,
                            "rel_diff": abs(fd_rc - rc_grad) / max(abs(fd_rc), 1e-300)},
            "fd_check": {"modes": len(fd), "precision": "fp64, tol 1e-10" if fd64 else "fp32, tol 1e-6",
                         "max_rel_diff": max(rel) if rel else None,
                         "median_rel_diff": float(np.median(rel)) if rel else None, "cases": fd}}
    print(json.dumps(line))
    return 0


def fp64_path_error(dgp, torch, np, n, box, delta_end, a_end, sched, steps, pos, mom, pk_main, dev,
                    sort_every):
    """Error of the mixed path against the FP64 GPU path: phi and forces of one solve on the run's
    end-state density (a fresh context per precision, tol as the run), and P(k) at the end of the
    same 200-step run done entirely in FP64 (the mixed run's P(k) is pk_main)."""
    fields = {}
    for name, prec, dt in (("mixed", dgp.DGP_MIXED_EFT, torch.float32), ("fp64", dgp.DGP_FP64, torch.float64)):
        c = dgp.dgp_init(box, n, WL["rc_H0"], WL["omega_m0"], w=WL["w"], precision=prec, max_iter=WL["max_iter"],
                         tol=WL["tol"])
        try:
            d = delta_end.to(dt).contiguous()
            phi = torch.empty_like(d)
            g = [torch.empty_like(d) for _ in range(3)]
            dgp.dgp_solve_forces(c, a_end, d, phi, g[0], g[1], g[2], WL["tol"])
            fields[name] = [phi.double()] + [x.double() for x in g]
        finally:
            dgp.dgp_destroy(c)

    def rl2(a, b):
        return float((a - b).norm() / b.norm())

    out = {"phi_rel_l2": rl2(fields["mixed"][0], fields["fp64"][0]),
           "force_rel_l2": max(rl2(fields["mixed"][i], fields["fp64"][i]) for i in (1, 2, 3))}
    del fields
    t = [torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev) for v in (*pos, *mom)]
    c = dgp.dgp_init(box, n, WL["rc_H0"], WL["omega_m0"], w=WL["w"], precision=dgp.DGP_FP64,
                     max_iter=WL["max_iter"], tol=WL["tol"], sort_every=sort_every)
    try:
        parts = dgp.particles(*t)
        for i in range(steps):
            dgp.pm_step(c, parts, sched[i], sched[i + 1] - sched[i])
        dl = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        dgp.dgp_deposit(c, parts, dl)
        pk64 = dgp.power_spectrum(c, dl, n // 2)[1]
    finally:
        dgp.dgp_destroy(c)
    out["pk_max_rel_diff"] = float(np.max(np.abs(pk_main / pk64 - 1)))
    out["note"] = ("mixed (error-free pairs) vs the FP64 GPU path: phi and forces of one solve on the "
                   "end-state density of the run at a = %.3f; P(k) after %d steps" % (a_end, steps))
    return out


# ---------------------------------------------------------------- replicas (one process per GPU)
def replica_env():
    """(world, rank, local_rank) from the torchrun environment; (1, 0, 0) without one."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(seed, rank):
    """Each replica runs its own realisation: the base seed offset by the rank."""
    return seed + rank


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (barrier, then a MAX all-reduce of one scalar); the replicas
    share no data, so this is the only collective."""
    if dist is None:
        return ms
    import torch
    dist.barrier()
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, steps, ms):
    """Steps of all replicas per second of the slowest replica's time."""
    return world * steps / (ms / 1000.0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--precision", default="mixed", choices=sorted(PRECISION_DESC))
    ap.add_argument("--no-compare", action="store_true", help="skip the precision comparison runs")
    ap.add_argument("--workload", default="pm256", choices=["pm256", "batched", "adjoint"],
                    help="pm256: the 256^3 PM run (default); batched: 48 small realisations; adjoint: the "
                         "gradient of a P(k) loss after a 128^3 run")
    ap.add_argument("--fd-modes", type=int, default=20, help="adjoint workload: central-difference checks")
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="adjoint workload: run only the first K of the 100 steps (0: all)")
    ap.add_argument("--fd-precision", default="fp32", choices=["fp32", "fp64"],
                    help="adjoint workload: precision of the gradient and differences that are compared")
    ap.add_argument("--sort-every", type=int, default=SORT_EVERY,
                    help="cell-sort the particles after every K-th drift (0: never)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "adjoint":
        return run_adjoint(args)

    import numpy as np
    import torch

    world, rank, local = replica_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__ as g
    g.build()
    from paper_0906_4548_gb300 import dgp, inputs

    n, box = WL["n"], WL["box"]
    bgi = dgp.dgp_background(WL["omega_m0"], WL["rc_H0"], WL["a_start"])
    vf = WL["a_start"] ** 2 * bgi["E"] * bgi["growth_f"]
    pos, mom, amp = inputs.zeldovich_particles(n, box, WL["n_s"], WL["rms"], replica_seed(WL["seed"], rank), vf)
    dev = torch.device("cuda", local)
    ic = [torch.tensor(v.astype(np.float32), device=dev) for v in (*pos, *mom)]
    cur = [t.clone() for t in ic]
    parts = dgp.particles(*cur)
    pcode = {"mixed": dgp.DGP_MIXED_EFT, "mixed-fp64": dgp.DGP_MIXED, "fp32": dgp.DGP_FP32}
    ctx = dgp.dgp_init(box, n, WL["rc_H0"], WL["omega_m0"], w=WL["w"], precision=pcode[args.precision],
                       max_iter=WL["max_iter"], tol=WL["tol"], sort_every=args.sort_every)
    dlna = math.log(WL["a_end"] / WL["a_start"]) / WL["run_steps"]
    sched = [WL["a_start"] * math.exp(i * dlna) for i in range(max(args.steps, args.warmup) + 1)]

    def restart():
        for c, s in zip(cur, ic):
            c.copy_(s)
        dgp.dgp_reset(ctx)

    def steps(k, infos=None):
        for i in range(k):
            inf = dgp.pm_step(ctx, parts, sched[i], sched[i + 1] - sched[i])
            if infos is not None:
                infos.append(inf)

    restart()
    steps(args.warmup)
    # per-kernel breakdown: the same run with every launch bracketed by events
    restart()
    dgp.dgp_profile(ctx, True)
    steps(args.steps)
    prof_all = dgp.dgp_profile_read(ctx)
    dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    # timed region: events only around the dominant kernel (its roofline)
    restart()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        dgp.dgp_profile(ctx, True, kinds=[dom])
        e0.record(stream)
        steps(args.steps, infos)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = dgp.dgp_profile_read(ctx)
    dgp.dgp_profile(ctx, False)
    ms = max_over_ranks(ms, dist, dev)
    value = whole_job_value(world, args.steps, ms)

    # end to end through the public C ABI with host buffers (copies inside the timed region)
    ne = args.steps if args.e2e_steps is None else args.e2e_steps
    host = [torch.empty(n ** 3, dtype=torch.float32, pin_memory=True) for _ in range(6)]
    for h, s in zip(host, ic):
        h.copy_(s)
    harr = [h.numpy() for h in host]
    hparts = dgp.particles(*harr)
    dgp.dgp_reset(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(ne):
        dgp.pm_step_host(ctx, hparts, sched[i], sched[i + 1] - sched[i])
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ne / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 6 * 4 * n ** 3,
           "d2h_bytes_per_step": 6 * 4 * n ** 3}

    # roofline of the dominant kernel (algorithmic bytes / event-timed duration in the timed region)
    peak, peak_kind = measured_peaks()
    d = prof[dom]
    achieved = d["timed_bytes"] / (d["ms"] / 1000.0) / 1e9 if d["ms"] > 0 else 0.0
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "gbs": round(v["timed_bytes"] / (v["ms"] / 1000.0) / 1e9, 1) if v["ms"] > 0 else None}
               for k, v in prof_all.items() if v["launches"]}
    evals = [i["iters"] + 1 for i in infos]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"mixed": "f32+eft", "mixed-fp64": "f32+f64", "fp32": "f32"}[args.precision],
            "data": "synthetic", "config": config(world, args.precision, args.sort_every),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": recorded_traffic(dom), "kernel": dom,
                         "algorithmic_bytes_per_launch": round(d["timed_bytes"] / max(d["timed"], 1)),
                         "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                         "peak_source": peak_kind},
            "e2e": e2e, "gpu_launches": int(sum(v["launches"] for v in prof.values())),
            "clocks": clk.summary(),
            "solver": {"evals_per_solve_mean": sum(evals) / len(evals), "max_evals": max(evals),
                       "final_a": sched[args.steps],
                       "not_converged_steps": sum(1 for i in infos if i["status"] != 0),
                       "max_norm_res": max(i["norm_res"] for i in infos), "amplitude_A": amp},
            "kernels": kernels, "tiles": dgp.dgp_tile_config(ctx),
            "kernels_note": "per-kind event times from a separate pass of the same run with every launch "
                            "bracketed by events; the timed region brackets only the dominant kind"}
    # the same run under the other precisions (same accuracy target): steps/s,
    # evaluations and P(k) of the end state relative to this run's
    if rank == 0 and not args.no_compare:
        def end_pk(c):
            dl = torch.empty((n, n, n), dtype=torch.float32, device=dev)
            dgp.dgp_deposit(c, parts, dl)
            return dgp.power_spectrum(c, dl, n // 2)[1]
        pk_main = end_pk(ctx)
        delta_end = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        dgp.dgp_deposit(ctx, parts, delta_end)
        comp = {}
        for name in sorted(pcode):
            if name == args.precision:
                comp[name] = {"value": value, "evals_per_solve_mean": sum(evals) / len(evals)}
                continue
            c2 = dgp.dgp_init(box, n, WL["rc_H0"], WL["omega_m0"], w=WL["w"], precision=pcode[name],
                              max_iter=WL["max_iter"], tol=WL["tol"], sort_every=args.sort_every)
            for cc, s0 in zip(cur, ic):
                cc.copy_(s0)
            infs = []
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for i in range(args.steps):
                infs.append(dgp.pm_step(c2, parts, sched[i], sched[i + 1] - sched[i]))
            f1.record(stream)
            torch.cuda.synchronize()
            pk2 = end_pk(c2)
            comp[name] = {"value": args.steps / (f0.elapsed_time(f1) / 1000.0),
                          "evals_per_solve_mean": sum(i["iters"] + 1 for i in infs) / len(infs),
                          "pk_max_rel_diff_vs_main": float(np.max(np.abs(pk2 / pk_main - 1)))}
            dgp.dgp_destroy(c2)
        line["precision_comparison"] = comp
        if args.precision == "mixed":
            try:
                line["fp64_path_error"] = fp64_path_error(dgp, torch, np, n, box, delta_end, sched[args.steps], sched,
                                                          args.steps, pos, mom, pk_main, dev, args.sort_every)
            except Exception as e:  # the comparison must not cost the measurement
                line["fp64_path_error"] = {"unavailable": repr(e)[:200]}
    dgp.dgp_destroy(ctx)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ts = oracle_fft_sample_seconds(96)
        t = sum(ts) / len(ts)
        e_mean = sum(evals) / len(evals)
        line["cpu_baseline"] = {
            "value": oracle_steps_per_s(t, e_mean), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "96 axis passes of the FP64 oracle FFT over a quarter of the 256^3 field (%.3f s each); "
                      "scaled to the FFT work of one PM step at the measured %.2f residual evaluations per "
                      "solve (deposit, gather and pointwise work not counted: an upper bound)" % (t, e_mean)}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
