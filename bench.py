"""PM steps/s at 256^3 including the converged nonlinear DGP phi solve.

Workload (the 256^3 run): 256^3 particles on a 256^3 mesh in a 400 Mpc/h box,
seeded n_s = -1.5 power-law Gaussian field with mesh rms 0.5 at a = 0.02,
Zel'dovich initial conditions, r_c H0 = 1, Omega_m0 = 0.27, w = 1/3, steps
uniform in ln a from a = 0.02 to a = 1 in 200 steps, relaxation tolerance 1e-6
on <|R|>/eps every step.  Arithmetic (--precision mixed, the default): FP32
mesh fields, FFTs, particles and pointwise residual, with the discriminant
formed exactly for its FP32 operands (its sign is the bad-point test) and the
residual norms, means and reductions in FP64.  The FP32 data's own rounding
leaves a residual floor near 1e-8 of <|S|>, 100 times below the tolerance, so
the residual gains nothing from wider arithmetic.  The run is repeated with R
and Delta on error-free FP32 pairs (--precision mixed-eft), on the FP64 pipe
(mixed-fp64; its rate is printed beside the headline) and in plain FP32, each
compared with this one.  A "step" is one pm_step call (deposit, field solve,
forces, gather, kick-drift-kick).

Timing: after W warm-up steps the whole 200-step run is started again from the
initial conditions and always run to the end; K of its steps, the middle step
of each of K equal strata of the run, are timed (each bracketed by a device
synchronisation, a barrier for N > 1, and CUDA events on the context's stream).
The context runs on its own stream, where the relaxation iterations replay as
CUDA graphs.  Inputs (403 MB of particles, 64 MB mesh fields) exceed L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun, one process per GPU): independent replicas with distinct
seeds, no data-path collective; value = all ranks' timed steps / max rank time.
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
    "relax": {"bytes": 652.6e6, "sources": ['relax_tma.cu', 'tma.cuh', 'eft.cuh', 'fft_core.cuh', 'kernels.cuh', 'common.cuh'],
              "sha256": "10664cba0c3d40605d047d2a008a8b42e05d6ce3eb56a750e3edaab2f3750327",
              "profile": "profiles/k_relax_tma_256cube.md"},
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
    "fp64": "fp64 throughout (the oracle)",
    "mixed": "mixed (the 256^3 workload's): fp32 mesh fields, FFTs, particles and pointwise residual R, B' "
             "and D_new; the discriminant Delta formed exactly (float pair) for its fp32 operands, so the "
             "bad-point sign test is exact; residual-norm and mean-of-D sums as float pairs within a thread "
             "and fp64 across threads and blocks, as every global mean and reduction",
    "mixed-eft": "mixed: fp32 mesh/FFT/particles; the residual R and discriminant Delta as unevaluated pairs "
                 "of fp32 (error-free transformations, ~48-bit significand) in place of fp64; B' fp32 from the "
                 "pair R; norms, means and reductions fp64",
    "mixed-fp64": "mixed: fp32 mesh/FFT/particles; residual, B', discriminant, norms and reductions fp64 "
                  "(the fp64 pipe)",
    "fp32": "fp32 throughout (fp64 cross-block sums only)",
}
DTYPE = {"mixed": "f32+f64", "mixed-eft": "f32+eft", "mixed-fp64": "f32+f64pipe", "fp32": "f32"}


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


def oracle_threads():
    """Host threads the oracle uses: its matmul steps run on the BLAS thread pool (all cores unless
    limited by the environment); its elementwise numpy steps on one thread."""
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(k)
        if v and v.isdigit():
            return int(v)
    return os.cpu_count()


# Residual evaluations per solve of each of the 200 steps of the 256^3 run, as measured on GB300
# (solver.evals_per_step of a bench run; every precision variant follows the same iterates): the
# reference arm has no GPU run to read them from, and times the oracle at the mean over the same
# timed steps as the GPU arm.
EVALS_PER_STEP_256 = [
    6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7, 7,
    7, 7, 7, 7, 7, 7, 7, 7, 7, 7, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 9, 9, 9,
    9, 9, 9, 9, 9, 9, 9, 10, 10, 10, 10, 10, 10, 10, 11, 11, 11, 11, 11, 11, 12, 12, 12, 12, 12,
    12, 13, 13, 13, 13, 13, 14, 14, 14, 14, 15, 15, 15, 15, 16, 16, 16, 16, 17, 17, 17, 18, 18, 18, 19,
    19, 19, 20, 20, 20, 21, 21, 22, 22, 22, 23, 23, 24, 24, 24, 25, 25, 26, 26, 26, 27, 27, 28, 28, 29,
    29, 29, 30, 30, 31, 31, 31, 32, 32, 33, 33, 33, 34, 35, 35, 36, 36, 36, 37, 37, 37, 37, 38, 38, 38,
    38, 38, 38, 38, 38, 38, 38, 38, 38, 38, 38, 37, 37, 37, 37, 37, 37, 37, 36, 36, 36, 36, 36, 36, 35,
    35, 35, 35, 34, 34, 34, 34, 34, 34, 33, 34, 33, 33, 32, 31, 31, 30, 30, 30, 30, 29, 29, 29, 28, 28,
]


def reference_evals(idx):
    if EVALS_PER_STEP_256 is None:
        return E_PER_SOLVE_REF
    return sum(EVALS_PER_STEP_256[i] for i in idx) / len(idx)


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only).  Each of the W + K steps
    is one real call of a piece of the oracle's PM step (deposit, forward transform, source,
    residual evaluation, update, phi and forces, interpolation, in turn) on the 256^3 workload's
    initial state; the K timed calls give each piece's time, and value = 1 / (the oracle's step
    time at E residual evaluations per solve), E the mean over the GPU arm's timed steps."""
    rank = replica_env()[1]
    if rank != 0:
        return 0
    model = OracleStepModel()
    pieces = OracleStepModel.PIECES
    # the pieces depend on one another's results: the warm-up calls run them in order
    for j in range(max(args.warmup, len(pieces))):
        model._run(pieces[j % len(pieces)])
    t0 = time.perf_counter()
    k = max(args.steps, 1)
    for j in range(k):
        model.time_piece(pieces[j % len(pieces)])
    wall = time.perf_counter() - t0
    for piece in pieces:  # a piece the K calls did not reach is timed once more
        if not model.times[piece]:
            model.time_piece(piece)
    idx = sampled_steps(WL["run_steps"], args.steps)
    e = reference_evals(idx)
    t_step = model.step_seconds(e)
    v = 1.0 / t_step
    sample = model.describe(e)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(config(args.gpus, "fp64"), precision=PRECISION_DESC["fp64"]),
            "timing": {"how": "each step is one real oracle call of one piece of a PM step (cycling through "
                              "%s); the PM step time is the sum of the pieces' mean times at E = %.2f residual "
                              "evaluations per solve, the mean over the GPU arm's timed steps of the 200-step "
                              "run" % (", ".join(pieces), e),
                       "timed_calls_s": wall, "pm_step_equivalents_timed": wall / t_step},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# Batched workload: independent realisations of uneven meshes stepped together.
WB = dict(sizes=[48] * 16 + [64] * 16 + [96] * 16, box_range=(50.0, 200.0), rc_range=(0.5, 2.0), n_s=-1.5,
          rms=0.5, seed=100, a_start=0.02, a_end=1.0, run_steps=50, omega_m0=0.27, tol=1e-6, max_iter=100)


def run_batched(args):
    """48 realisations (16 x 48^3, 16 x 64^3, 16 x 96^3, particles = mesh cells), boxes and r_c H0
    drawn uniformly, distinct seeds, FP32, 50 steps each from a = 0.02 to 1: the batch path (the
    realisations of one mesh size stepped as a class, every kernel stage launched once for all of
    them) and the plain path (the same realisations stepped one after another on one stream).  Both
    are timed over the whole 50-step run (--steps does not shorten it).  value = realisation-steps
    per second of the batch path."""
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
    # the whole run is timed: the early, nearly linear steps need far fewer evaluations per solve
    # than the late ones, so a prefix of the run would not measure the stated workload
    steps = WB["run_steps"]

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
    if args.no_plain:
        evals = [i["iters"] + 1 for step in infos for i in step]
        print(json.dumps({"metric": "PM realisation-steps/s, 48 realisations (16 x 48^3, 16 x 64^3, 16 x 96^3)",
                          "value": nr * steps / (ms / 1000.0), "unit": "realisation-steps/s", "steps": steps,
                          "ms_per_step": ms / steps, "evals_per_solve_mean": sum(evals) / len(evals)}))
        return 0
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
            "timing": {"how": "the whole run (a = 0.02 -> 1) between two CUDA events on the calling stream; "
                              "each batch step returns after all its classes finished"},
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
            e = (args.fd_eps if args.fd_eps else (1e-4 if fd64 else 2e-3)) * WA["rms"]
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
                         "eps_over_rms": args.fd_eps if args.fd_eps else (1e-4 if fd64 else 2e-3),
                         "max_rel_diff": max(rel) if rel else None,
                         "median_rel_diff": float(np.median(rel)) if rel else None, "cases": fd}}
    print(json.dumps(line))
    return 0


def fp64_path_error(dgp, torch, np, n, box, delta_end, a_end, sched, pos, mom, pk_main, dev, sort_every,
                    stream):
    """Error of the mixed path against the FP64 GPU path: phi and forces of one solve on the run's
    end-state density (a fresh context per precision, tol as the run), and P(k) at the end of the
    same whole run done entirely in FP64 (the mixed run's P(k) is pk_main)."""
    fields = {}
    for name, prec, dt in (("mixed", dgp.DGP_MIXED_F32R, torch.float32), ("fp64", dgp.DGP_FP64, torch.float64)):
        c = dgp.dgp_init(box, n, WL["rc_H0"], WL["omega_m0"], w=WL["w"], precision=prec, max_iter=WL["max_iter"],
                         tol=WL["tol"], stream=stream.cuda_stream)
        try:
            d = delta_end.to(dt).contiguous()
            phi = torch.empty_like(d)
            g = [torch.empty_like(d) for _ in range(3)]
            torch.cuda.synchronize()
            dgp.dgp_solve_forces(c, a_end, d, phi, g[0], g[1], g[2], WL["tol"])
            torch.cuda.synchronize()
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
                     max_iter=WL["max_iter"], tol=WL["tol"], sort_every=sort_every, stream=stream.cuda_stream)
    try:
        torch.cuda.synchronize()
        parts = dgp.particles(*t)
        for i in range(len(sched) - 1):
            dgp.pm_step(c, parts, sched[i], sched[i + 1] - sched[i])
        dl = torch.empty((n, n, n), dtype=torch.float64, device=dev)
        dgp.dgp_deposit(c, parts, dl)
        pk64 = dgp.power_spectrum(c, dl, n // 2)[1]
    finally:
        dgp.dgp_destroy(c)
    out["pk_max_rel_diff"] = float(np.max(np.abs(pk_main / pk64 - 1)))
    out["note"] = ("mixed vs the FP64 GPU path: phi and forces of one solve on the "
                   "end-state density of the run at a = %.3f; P(k) after the whole %d-step run"
                   % (a_end, len(sched) - 1))
    return out


def sampled_steps(run_steps, k):
    """The K timed steps of a run of run_steps steps: the middle step of each of K equal strata
    of the run (all steps when K >= run_steps)."""
    k = max(1, min(int(k), run_steps))
    return [min(run_steps - 1, int((j + 0.5) * run_steps / k)) for j in range(k)]


def oracle_sample_inputs(n, box, a, seed):
    """Workload-shaped inputs of the oracle sample: the Zel'dovich particles of the run's
    initial conditions at a (FP32 positions, as the GPU run starts from)."""
    import numpy as np
    from oracle import background as obg
    from paper_0906_4548_gb300 import inputs
    vf = obg.zeldovich_velocity_factor(a, WL["omega_m0"], WL["rc_H0"])
    pos, _, _ = inputs.zeldovich_particles(n, box, WL["n_s"], WL["rms"], seed, vf)
    return pos.astype(np.float32).astype(np.float64)


class OracleStepModel:
    """The FP64 oracle's PM step, timed on real oracle calls on one workload-shaped state.

    One oracle PM step (oracle.pm.PMState.step, the start force carried over) is
        deposit + density contrast + fft3(delta) + source (one inverse transform)
        + E evaluations (fft3(D), the eight inverse transforms of derived_fields, residual)
        + (E - 1) updates (relax_update) + phi and forces (four inverse transforms)
        + 3 CIC interpolations,
    with E the residual evaluations of the step's solve.  Each piece is one call of the oracle
    as it stands; the step time is their sum for a given E."""

    PIECES = ("deposit", "forward", "source", "evaluation", "update", "phi_forces", "interpolate")

    def __init__(self, n=None, box=None, a=None, seed=None, pos=None):
        import numpy as np
        from oracle import background as obg
        from oracle import field as ofield
        from oracle import pm as opm
        from oracle.fft import fft3, ifft3_real
        self.np, self.opm, self.ofield, self.fft3, self.ifft3_real = np, opm, ofield, fft3, ifft3_real
        self.n = WL["n"] if n is None else n
        self.box = WL["box"] if box is None else box
        self.a = WL["a_start"] if a is None else a
        self.pos = (oracle_sample_inputs(self.n, self.box, self.a, WL["seed"] if seed is None else seed)
                    if pos is None else np.asarray(pos, dtype=np.float32).astype(np.float64))
        self.grid = ofield.KGrid(self.n, self.box)
        self.coef = obg.coefficients(self.a, WL["omega_m0"], WL["rc_H0"])
        self.state = {}
        self.times = {k: [] for k in self.PIECES}

    def _run(self, piece):
        st, np, of, g, c = self.state, self.np, self.ofield, self.grid, self.coef
        if piece == "deposit":
            st["delta"] = self.opm.density_contrast(self.opm.cic_deposit(self.pos, self.n, self.box))
        elif piece == "forward":
            dk = self.fft3(st["delta"])
            dk[g.zero] = 0.0
            st["dk"] = dk
        elif piece == "source":
            st["Sk"] = of.source_spectrum(st["dk"], g, c)
            st["S"] = self.ifft3_real(st["Sk"])
        elif piece == "evaluation":
            if "D" not in st:
                st["D"] = self.ifft3_real(of.linear_D_spectrum(st["Sk"], g, c))
            D_k = self.fft3(st["D"])
            D_k[g.zero] = 0.0
            D, H, Nf = of.derived_fields(D_k, g, c)
            st["r"] = float(np.mean(np.abs(of.residual(D, H, Nf, st["S"], c))))
            st["DHN"], st["Dk"] = (D, H, Nf), D_k
        elif piece == "update":
            D, H, Nf = st["DHN"]
            st["D"], _ = of.relax_update(D, H, Nf, st["S"], c, WL["w"])
        elif piece == "phi_forces":
            _, st["g"] = of.phi_and_forces(st["dk"], st["Dk"], g, c)
        elif piece == "interpolate":
            self.opm.cic_interpolate(st["g"][0], self.pos, self.box)

    def time_piece(self, piece):
        t0 = time.perf_counter()
        self._run(piece)
        dt = time.perf_counter() - t0
        self.times[piece].append(dt)
        return dt

    def time_all(self):
        for piece in self.PIECES:
            self.time_piece(piece)

    def step_seconds(self, e):
        m = {k: sum(v) / len(v) for k, v in self.times.items() if v}
        return (m["deposit"] + m["forward"] + m["source"] + e * m["evaluation"] + max(e - 1.0, 0.0) * m["update"]
                + m["phi_forces"] + 3.0 * m["interpolate"])

    def describe(self, e):
        m = {k: round(sum(v) / len(v), 3) for k, v in self.times.items() if v}
        return ("real FP64 oracle calls on the %d^3 workload's initial state (%d particles, a = %g), seconds "
                "per call %s; one oracle PM step = deposit + forward + source + E evaluations + (E - 1) updates "
                "+ phi_forces + 3 interpolations at E = %.2f residual evaluations per solve"
                % (self.n, self.n ** 3, self.a, json.dumps(m), e))


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
    ap.add_argument("--steps", type=int, default=20,
                    help="timed steps K, spread evenly over the whole run (which always runs in full)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=sorted(k for k in PRECISION_DESC if k != "fp64"))
    ap.add_argument("--no-compare", action="store_true", help="skip the precision comparison runs")
    ap.add_argument("--no-kernel-table", action="store_true", help="skip the per-kind event pass")
    ap.add_argument("--workload", default="pm256", choices=["pm256", "batched", "adjoint"],
                    help="pm256: the 256^3 PM run (default); batched: 48 small realisations; adjoint: the "
                         "gradient of a P(k) loss after a 128^3 run")
    ap.add_argument("--fd-modes", type=int, default=20, help="adjoint workload: central-difference checks")
    ap.add_argument("--adjoint-steps", type=int, default=0,
                    help="adjoint workload: run only the first K of the 100 steps (0: all)")
    ap.add_argument("--fd-eps", type=float, default=0.0,
                    help="adjoint workload: central-difference step in units of the field rms (0: 1e-4 in FP64, "
                         "2e-3 in FP32)")
    ap.add_argument("--fd-precision", default="fp32", choices=["fp32", "fp64"],
                    help="adjoint workload: precision of the gradient and differences that are compared")
    ap.add_argument("--no-plain", action="store_true", help="batched workload: skip the one-by-one comparison")
    ap.add_argument("--sort-every", type=int, default=SORT_EVERY,
                    help="cell-sort the particles after every K-th drift (0: never)")
    ap.add_argument("--run-steps", type=int, default=WL["run_steps"],
                    help="steps of the run (the workload is 200; smaller only for quick checks)")
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
    R = args.run_steps
    bgi = dgp.dgp_background(WL["omega_m0"], WL["rc_H0"], WL["a_start"])
    vf = WL["a_start"] ** 2 * bgi["E"] * bgi["growth_f"]
    pos, mom, amp = inputs.zeldovich_particles(n, box, WL["n_s"], WL["rms"], replica_seed(WL["seed"], rank), vf)
    dev = torch.device("cuda", local)
    ic = [torch.tensor(v.astype(np.float32), device=dev) for v in (*pos, *mom)]
    cur = [t.clone() for t in ic]
    parts = dgp.particles(*cur)
    # the context runs on its own stream: the relaxation iterations replay as CUDA graphs there
    # (stream capture is not available on the legacy default stream)
    bs = torch.cuda.Stream(device=dev)
    pcode = {"mixed": dgp.DGP_MIXED_F32R, "mixed-eft": dgp.DGP_MIXED_EFT, "mixed-fp64": dgp.DGP_MIXED,
             "fp32": dgp.DGP_FP32}

    def make_ctx(prec):
        return dgp.dgp_init(box, n, WL["rc_H0"], WL["omega_m0"], w=WL["w"], precision=pcode[prec],
                            max_iter=WL["max_iter"], tol=WL["tol"], sort_every=args.sort_every,
                            stream=bs.cuda_stream)

    ctx = make_ctx(args.precision)
    dlna = math.log(WL["a_end"] / WL["a_start"]) / WL["run_steps"]
    sched = [WL["a_start"] * math.exp(i * dlna) for i in range(R + 1)]
    idx = sampled_steps(R, args.steps)
    K = len(idx)
    sel = set(idx)

    def restart(c):
        for x, s0 in zip(cur, ic):
            x.copy_(s0)
        dgp.dgp_reset(c)
        torch.cuda.synchronize()

    def run(c, nsteps=R, infos=None, timed=None, launches=None, dom=None, roof=None):
        """Steps 0 .. nsteps-1 of the schedule; each step in `sel` is bracketed by a barrier and a
        device synchronisation on both sides and timed with CUDA events on the context's stream."""
        for i in range(nsteps):
            if timed is not None and i in sel:
                torch.cuda.synchronize()
                if dist:
                    dist.barrier()
                before = dgp.dgp_profile_read(c) if launches is not None else None
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(bs)
                inf = dgp.pm_step(c, parts, sched[i], sched[i + 1] - sched[i])
                e1.record(bs)
                torch.cuda.synchronize()
                timed.append(e0.elapsed_time(e1))
                if launches is not None:
                    after = dgp.dgp_profile_read(c)
                    launches.append(sum(after[k]["launches"] - before[k]["launches"] for k in after))
                    if dom is not None:
                        for f in ("ms", "timed", "timed_bytes"):
                            roof[f] += after[dom][f] - before[dom][f]
            else:
                inf = dgp.pm_step(c, parts, sched[i], sched[i + 1] - sched[i])
            if infos is not None:
                infos.append(inf)

    restart(ctx)
    run(ctx, min(args.warmup, R))
    # per-kind breakdown over the whole run: every launch bracketed by events (graphs off)
    prof_all = None
    dom = "relax"
    if not args.no_kernel_table:
        restart(ctx)
        dgp.dgp_profile(ctx, True)
        run(ctx)
        prof_all = dgp.dgp_profile_read(ctx)
        dom = max(prof_all, key=lambda k: prof_all[k]["ms"])
    # timed pass: the whole run on the production path (graph replay on); K steps spread over the
    # run are timed, and inside them the dominant kind's launches outside graphs carry events
    restart(ctx)
    if dist:
        dist.barrier()
    timed, launches, infos = [], [], []
    roof = {"ms": 0.0, "timed": 0, "timed_bytes": 0.0}
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        dgp.dgp_profile_sampled(ctx, [dom])
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(bs)
        run(ctx, R, infos, timed, launches, dom, roof)
        f1.record(bs)
        torch.cuda.synchronize()
    full_ms = f0.elapsed_time(f1)
    dgp.dgp_profile(ctx, False)
    ms = max_over_ranks(sum(timed), dist, dev)
    value = whole_job_value(world, K, ms)

    # roofline of the dominant kernel: algorithmic bytes / event-timed duration of its launches
    # inside the timed steps
    peak, peak_kind = measured_peaks()
    achieved = roof["timed_bytes"] / (roof["ms"] / 1000.0) / 1e9 if roof["ms"] > 0 else 0.0
    ev_t = [infos[i]["iters"] + 1 for i in idx]
    ev_all = [x["iters"] + 1 for x in infos]
    kernels = None
    if prof_all is not None:
        kernels = {}
        for k, v in prof_all.items():
            if not v["launches"]:
                continue
            gbs = v["timed_bytes"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] > 0 else None
            kernels[k] = {"launches": v["launches"], "ms": round(v["ms"], 3),
                          "ms_per_step": round(v["ms"] / R, 4), "gbs": round(gbs, 1) if gbs else None,
                          "frac_of_peak": round(gbs / peak, 3) if gbs else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic", "config": config(world, args.precision, args.sort_every),
            "timing": {"how": "the whole %d-step run (a = %g -> %g) runs every time; the K = %d timed steps are the "
                              "middle step of each of K equal strata of the run, each bracketed by a device "
                              "synchronisation (and a barrier for N > 1) and CUDA events on the context's "
                              "stream, with the relaxation iterations replayed as CUDA graphs"
                              % (R, sched[0], sched[R], K),
                       "timed_step_indices": idx, "timed_a_range": [sched[idx[0]], sched[idx[-1] + 1]],
                       "full_run": {"steps": R, "ms": full_ms, "steps_per_s": R / (full_ms / 1000.0),
                                    "note": "the same pass end to end, including the K synchronisations"}},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": recorded_traffic(dom), "kernel": dom,
                         "launches_timed": roof["timed"],
                         "algorithmic_bytes_per_launch": round(roof["timed_bytes"] / max(roof["timed"], 1)),
                         "how": "launches of this kind outside CUDA graphs inside the timed steps (the first "
                                "iteration of each solve), CUDA events on the launch stream",
                         "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                         "peak_source": peak_kind},
            "gpu_launches": int(sum(launches)),
            "clocks": clk.summary(),
            "solver": {"evals_per_solve_timed_steps": sum(ev_t) / len(ev_t),
                       "evals_per_solve_run": sum(ev_all) / len(ev_all), "max_evals": max(ev_all),
                       "final_a": sched[R], "not_converged_steps": sum(1 for i in infos if i["status"] != 0),
                       "max_norm_res": max(i["norm_res"] for i in infos), "amplitude_A": amp,
                       "evals_per_step": ev_all},
            "tiles": dgp.dgp_tile_config(ctx)}
    if kernels is not None:
        line["kernels"] = kernels
        line["kernels_note"] = ("per-kind event times over the whole run from a separate pass with every launch "
                                "bracketed by events (graph replay off); frac_of_peak against the measured "
                                "copy bandwidth")

    # end to end through the public C ABI with host buffers (copies inside the timed steps)
    if not args.no_e2e:
        host = [torch.empty(n ** 3, dtype=torch.float32, pin_memory=True) for _ in range(6)]
        for h, s0 in zip(host, ic):
            h.copy_(s0)
        hparts = dgp.particles(*[h.numpy() for h in host])
        dgp.dgp_reset(ctx)
        torch.cuda.synchronize()
        te = []
        t_all = time.perf_counter()
        for i in range(R):
            if i in sel:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                dgp.pm_step_host(ctx, hparts, sched[i], sched[i + 1] - sched[i])
                te.append(time.perf_counter() - t0)
            else:
                dgp.pm_step_host(ctx, hparts, sched[i], sched[i + 1] - sched[i])
        t_all = time.perf_counter() - t_all
        line["e2e"] = {"value": world * K / max_over_ranks(sum(te), dist, dev), "unit": UNIT,
                       "h2d_bytes_per_step": 6 * 4 * n ** 3, "d2h_bytes_per_step": 6 * 4 * n ** 3,
                       "how": "pm_step_host on pinned host arrays over the whole run, the same K steps timed "
                              "with the host clock (each call returns after its copies back)",
                       "full_run_steps_per_s": R / t_all}

    # the same run under the other precisions (same accuracy target): steps/s over the same timed
    # steps, evaluations and P(k) of the end state relative to this run's
    if rank == 0 and not args.no_compare:
        def end_pk(c):
            dl = torch.empty((n, n, n), dtype=torch.float32, device=dev)
            dgp.dgp_deposit(c, parts, dl)
            return dgp.power_spectrum(c, dl, n // 2)[1]
        restart(ctx)
        run(ctx)
        pk_main = end_pk(ctx)
        delta_end = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        dgp.dgp_deposit(ctx, parts, delta_end)
        torch.cuda.synchronize()
        comp = {}
        for name in sorted(pcode):
            if name == args.precision:
                comp[name] = {"value": value, "evals_per_solve_timed_steps": sum(ev_t) / len(ev_t),
                              "precision": PRECISION_DESC[name]}
                continue
            c2 = make_ctx(name)
            try:
                restart(c2)
                t2, inf2 = [], []
                run(c2, R, inf2, t2)
                comp[name] = {"value": K / (sum(t2) / 1000.0),
                              "evals_per_solve_timed_steps": sum(inf2[i]["iters"] + 1 for i in idx) / K,
                              "pk_max_rel_diff_vs_main": float(np.max(np.abs(end_pk(c2) / pk_main - 1))),
                              "precision": PRECISION_DESC[name]}
            finally:
                dgp.dgp_destroy(c2)
        line["precision_comparison"] = comp
        if "mixed-fp64" in comp and args.precision != "mixed-fp64":
            line["fp64_pipe_variant"] = {"value": comp["mixed-fp64"]["value"], "unit": UNIT,
                                         "precision": PRECISION_DESC["mixed-fp64"]}
        if args.precision == "mixed":
            try:
                line["fp64_path_error"] = fp64_path_error(dgp, torch, np, n, box, delta_end, sched[R], sched, pos,
                                                          mom, pk_main, dev, args.sort_every, bs)
            except Exception as e:  # the comparison must not cost the measurement
                line["fp64_path_error"] = {"unavailable": repr(e)[:200]}
    dgp.dgp_destroy(ctx)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        model = OracleStepModel(pos=pos)
        model.time_all()
        e_mean = sum(ev_t) / len(ev_t)
        t_step = model.step_seconds(e_mean)
        line["cpu_baseline"] = {"value": 1.0 / t_step, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                                "sample": model.describe(e_mean)}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
