"""Cell sort of the particles and the deposit on sorted particles (Sec. III.A),
through the C ABI, against the oracle's cell_index / cell_sort / cic_deposit.

The cell of a particle is an integer, so it is compared exactly.  Both sides
take floor(x n / box): the oracle in FP64, the FP32 path on an unevaluated
float pair (~48 bits); a coordinate whose x n / box lies within 1e-9 of an
integer may fall on either side, and there either neighbouring cell is accepted.
"""
import functools
import math

import numpy as np
import pytest

from oracle import estimators as oest
from oracle import pm as opm
from paper_0906_4548_gb300 import inputs

from test_gpu_parity import OM, np_dtype, prec_dtype, rel_l2, to_dev, zel  # noqa: F401
from test_gpu_parity import dgp, torch_dev  # noqa: F401  (fixtures)

pytestmark = pytest.mark.gpu


def check_slot_cells(xs, start, n, box, eps=1e-9):
    """Every sorted slot holds a particle of the slot's cell (cell_start gives
    the slot ranges).  A coordinate with x n / box within eps of an integer may
    be keyed to either neighbouring cell; returns how many such particles."""
    xs = np.asarray(xs, np.float64)
    slot_cell = np.repeat(np.arange(n ** 3), np.diff(start))
    key = opm.cell_index(xs, n, box)
    u = xs * (n / box)
    amb = np.abs(u - np.round(u)) < eps
    for p in np.nonzero(slot_cell != key)[0]:
        assert amb[:, p].any(), p
        options = []
        for ax in range(3):
            r = int(np.round(u[ax, p]))
            options.append({r % n, (r - 1) % n} if amb[ax, p] else {int(np.floor(u[ax, p])) % n})
        cells = {(ix * n + iy) * n + iz for ix in options[0] for iy in options[1] for iz in options[2]}
        assert slot_cell[p] in cells, p
    return int(amb.any(axis=0).sum())


def clustered(n, box, npart, seed, frac_halo=0.3, width_cells=0.7):
    """Uniform background plus a compact Gaussian clump holding frac_halo of the particles."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, box, (3, npart))
    nh = int(frac_halo * npart)
    c = rng.uniform(0, box, (3, 1))
    pos[:, :nh] = np.mod(c + rng.normal(0, width_cells * box / n, (3, nh)), box)
    return pos


def run_sort(dgp, torch_dev, n, box, prec, pos, mom, want_start=True):
    torch, dev = torch_dev
    td = prec_dtype(torch, prec, dgp)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec)
    try:
        t = [to_dev(torch_dev, v, td) for v in (*pos, *mom)]
        cs = torch.full((n ** 3 + 1,), -7, dtype=torch.int32, device=dev) if want_start else None
        dgp.dgp_sort_particles(ctx, dgp.particles(*t), cs)
        arr = np.stack([v.cpu().numpy() for v in t])
        start = cs.cpu().numpy().astype(np.int64) if want_start else None
    finally:
        dgp.dgp_destroy(ctx)
    return arr, start


def check_sorted(arr, start, pos_in, mom_in, n, box):
    """Returns True when no particle sat on a cell boundary, in which case
    cell_start must equal the oracle's exactly."""
    npart = pos_in.shape[1]
    rows_in = np.concatenate([pos_in, mom_in]).T
    # the six arrays were permuted together: same multiset of rows, bit for bit
    a = rows_in[np.lexsort(rows_in.T[::-1])]
    b = arr.T[np.lexsort(arr[::-1])]
    assert np.array_equal(a, b)
    assert start[0] == 0 and start[-1] == npart and np.all(np.diff(start) >= 0)
    namb = check_slot_cells(arr[:3], start, n, box)
    if namb == 0:
        _, ostart = opm.cell_sort(pos_in.astype(np.float64), n, box)
        assert np.array_equal(start, ostart)
    return namb == 0


@pytest.mark.parametrize("n,prec,kind", [(32, 1, "zel"), (32, 2, "zel"), (16, 1, "clump"), (64, 0, "clump"),
                                         (32, 2, "clump")])
def test_cell_sort_matches_oracle(dgp, torch_dev, n, prec, kind):
    box = 100.0
    nd = np_dtype(prec, dgp)
    if kind == "zel":
        pos, mom, _ = zel(n, box, 0.3, -1.5, 1.0, 11)
        npart = n ** 3 - 45  # ragged
        pos, mom = pos[:, :npart], mom[:, :npart]
    else:
        npart = n ** 3 + 101
        pos = clustered(n, box, npart, 12)
        mom = np.random.default_rng(13).normal(0, 1, (3, npart))
    pos, mom = pos.astype(nd), mom.astype(nd)
    arr, start = run_sort(dgp, torch_dev, n, box, prec, pos, mom)
    check_sorted(arr, start, pos, mom, n, box)


def test_cell_sort_on_lattice_boundaries(dgp, torch_dev):
    """Particles exactly on mesh points (x n / box integer): either side of the
    boundary is a valid cell, everything else is still checked."""
    n, box = 16, 50.0
    pos, mom = inputs.lattice_particles(n, box)
    pos = pos.astype(np.float32)
    mom = np.random.default_rng(2).normal(0, 1, pos.shape).astype(np.float32)
    arr, start = run_sort(dgp, torch_dev, n, box, 1, pos, mom)
    check_sorted(arr, start, pos, mom, n, box)


def test_cell_sort_empty_and_repeat(dgp, torch_dev):
    torch, dev = torch_dev
    n, box = 16, 40.0
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=1)
    try:
        e = [torch.empty(0, dtype=torch.float32, device=dev) for _ in range(6)]
        cs = torch.full((n ** 3 + 1,), 5, dtype=torch.int32, device=dev)
        dgp.dgp_sort_particles(ctx, dgp.particles(*e), cs)
        assert int(cs.abs().sum()) == 0
        # sorting twice gives the same cells; a larger set after a smaller one regrows the workspace
        for npart in (100, 5000, 5000):
            pos = clustered(n, box, npart, npart).astype(np.float32)
            t = [to_dev(torch_dev, v, torch.float32) for v in (*pos, *pos)]
            dgp.dgp_sort_particles(ctx, dgp.particles(*t), cs)
            s1 = cs.cpu().numpy().copy()
            dgp.dgp_sort_particles(ctx, dgp.particles(*t), cs)
            assert np.array_equal(s1, cs.cpu().numpy())
            assert s1[-1] == npart
    finally:
        dgp.dgp_destroy(ctx)


@pytest.mark.parametrize("n,prec,kind", [(32, 1, "clump"), (32, 2, "clump"), (64, 0, "sparse"), (32, 1, "zel")])
def test_deposit_on_sorted_particles(dgp, torch_dev, n, prec, kind):
    """Deposit after the sort: the shared-memory tiles (dense blocks) and the
    direct atomics (blocks spanning more cells than a tile) agree with Eq. CIC."""
    torch, dev = torch_dev
    box = 100.0
    nd = np_dtype(prec, dgp)
    td = prec_dtype(torch, prec, dgp)
    if kind == "zel":
        pos, _, _ = zel(n, box, 0.3, -1.5, 1.0, 4)
    elif kind == "sparse":
        pos = np.random.default_rng(3).uniform(0, box, (3, n ** 3 // 20 + 3))
    else:
        pos = clustered(n, box, n ** 3 - 9, 21, frac_halo=0.5)
    pos = pos.astype(nd)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=prec)
    try:
        t = [to_dev(torch_dev, v, td) for v in (*pos, *pos)]
        parts = dgp.particles(*t)
        dgp.dgp_sort_particles(ctx, parts)
        delta = torch.empty((n, n, n), dtype=td, device=dev)
        dgp.dgp_deposit(ctx, parts, delta)
        got = delta.double().cpu().numpy()
    finally:
        dgp.dgp_destroy(ctx)
    want = opm.density_contrast(opm.cic_deposit(pos.astype(np.float64), n, box))
    assert rel_l2(got, want) < (1e-13 if prec == dgp.DGP_FP64 else 1e-6)


@functools.lru_cache(maxsize=1)
def _oracle_run_64():
    n, box, a0, a1, ns = 64, 200.0, 0.1, 0.3, 8
    pos, mom, _ = zel(n, box, a0, -1.5, 0.5, 2)
    pos, mom = pos.astype(np.float32).astype(np.float64), mom.astype(np.float32).astype(np.float64)
    st = opm.run(pos, mom, a0, a1, ns, n, box, OM, 1.0, tol=1e-10, max_iter=300)
    ko, Po, co = oest.power_spectrum(opm.density_contrast(opm.cic_deposit(st.pos, n, box)), box)
    return (n, box, a0, a1, ns, pos, mom), Po, co


@pytest.mark.parametrize("sort_every", [1, 3])
def test_pm_run_with_sorting_matches_oracle(dgp, torch_dev, sort_every):
    """pm_step with the cell sort every K steps: P(k) of the end state within
    1e-3 of the oracle run (which keeps the particles in their input order)."""
    torch, dev = torch_dev
    (n, box, a0, a1, ns, pos, mom), Po, co = _oracle_run_64()
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_MIXED_EFT, tol=1e-6, max_iter=100,
                       sort_every=sort_every)
    try:
        t = [to_dev(torch_dev, v, torch.float32) for v in (*pos, *mom)]
        parts = dgp.particles(*t)
        a = a0
        dl = (math.log(a1) - math.log(a0)) / ns
        for i in range(ns):
            a_next = a0 * math.exp((i + 1) * dl)
            dgp.pm_step(ctx, parts, a, a_next - a)
            a = a_next
        delta = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        dgp.dgp_deposit(ctx, parts, delta)
        k, P, cnt = dgp.power_spectrum(ctx, delta, n // 2)
        xs = np.stack([v.cpu().numpy() for v in t[:3]]).astype(np.float64)
    finally:
        dgp.dgp_destroy(ctx)
    assert np.array_equal(cnt, co)
    assert np.max(np.abs(P / Po - 1)) < 1e-3
    if sort_every == 1:
        # sorted after the last drift, and the closing half-kick moves no particle
        key = opm.cell_index(xs, n, box)
        u = xs * (n / box)
        namb = int(np.any(np.abs(u - np.round(u)) < 1e-9, axis=0).sum())
        assert int(np.sum(np.diff(key) < 0)) <= namb


# ---------------------------------------------------------------- full size
def test_full_size_sort_and_tiled_deposit(dgp, torch_dev):
    """256^3 particles in 400 Mpc/h at a = 0.3 (the PM-step workload): cell
    counts exact for all 16.8M particles, cells of a sample of slots, and the
    tiled deposit against Eq. CIC."""
    torch, dev = torch_dev
    n, box = 256, 400.0
    pos, mom, _ = zel(n, box, 0.3, -1.5, 1.0, 3)
    pos, mom = pos.astype(np.float32), mom.astype(np.float32)
    ctx = dgp.dgp_init(box, n, 1.0, OM, precision=dgp.DGP_MIXED_EFT)
    try:
        t = [to_dev(torch_dev, v, torch.float32) for v in (*pos, *mom)]
        parts = dgp.particles(*t)
        cs = torch.empty(n ** 3 + 1, dtype=torch.int32, device=dev)
        dgp.dgp_sort_particles(ctx, parts, cs)
        delta = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        dgp.dgp_deposit(ctx, parts, delta)
        start = cs.cpu().numpy().astype(np.int64)
        xs = np.stack([v.cpu().numpy() for v in t[:3]])
        dg = delta.double().cpu().numpy()
    finally:
        dgp.dgp_destroy(ctx)
    p64 = pos.astype(np.float64)
    assert start[0] == 0 and start[-1] == pos.shape[1] and np.all(np.diff(start) >= 0)
    namb = check_slot_cells(xs, start, n, box)
    if namb == 0:
        assert np.array_equal(np.diff(start), np.bincount(opm.cell_index(p64, n, box), minlength=n ** 3))
    # the sorted positions are the input positions, permuted
    for ax in range(3):
        assert np.array_equal(np.sort(xs[ax]), np.sort(pos[ax]))
    do = opm.density_contrast(opm.cic_deposit(p64, n, box))
    assert rel_l2(dg, do) < 1e-6
