"""Pins of the oracle's PM layer (Sec. III.A): CIC identities, brute-force
weights, and linear growth of a low-amplitude run."""
import math

import numpy as np
import pytest

from oracle import background as bg
from oracle import field, pm
from paper_0906_4548_gb300 import inputs

OM = 0.27


def test_uniform_lattice_gives_zero_delta_and_zero_force():
    n, box = 16, 50.0
    pos, mom = inputs.lattice_particles(n, box)
    rho = pm.cic_deposit(pos, n, box)
    assert np.all(rho == 1.0)
    delta = pm.density_contrast(rho)
    phi, g, D, info = field.solve_phi(delta, 0.3, box, OM, 1.0)
    assert np.all(delta == 0) and np.all(phi == 0) and all(np.all(gi == 0) for gi in g)


def test_mass_conservation_and_constant_gather():
    n, box = 12, 30.0
    rng = np.random.default_rng(1)
    pos = rng.uniform(0, box, (3, 5000))
    rho = pm.cic_deposit(pos, n, box)
    assert abs(rho.sum() - 5000) < 1e-9
    f = np.full((n, n, n), 2.5)
    assert np.allclose(pm.cic_interpolate(f, pos, box), 2.5, atol=1e-13)


def test_deposit_gather_adjoint():
    n, box = 10, 20.0
    rng = np.random.default_rng(2)
    pos = rng.uniform(0, box, (3, 777))
    f = rng.standard_normal((n, n, n))
    lhs = np.sum(pm.cic_deposit(pos, n, box) * f)
    rhs = np.sum(pm.cic_interpolate(f, pos, box))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_single_particle_brute_force_weights():
    """Eq. CIC with W(x) = 1 - |x|/d summed over every grid point (periodic images)."""
    n, box = 6, 12.0
    d = box / n
    p = np.array([[11.3], [0.7], [5.0]])
    rho = pm.cic_deposit(p, n, box)
    want = np.zeros((n, n, n))
    for idx in np.ndindex(n, n, n):
        w = 1.0
        for ax in range(3):
            dx = (idx[ax] * d - p[ax, 0] + box / 2) % box - box / 2
            w *= max(0.0, 1 - abs(dx) / d)
        want[idx] = w
    assert np.max(np.abs(rho - want)) < 1e-14


def test_cell_index_hand_values_and_wrap():
    """Key = (ix n + iy) n + iz, i = floor(x / d) mod n, checked on values worked by hand (n = 4, d = 2)."""
    n, box = 4, 8.0
    pos = np.array([[3.0, -0.5, 8.0, 7.999, 0.0],
                    [0.5, 2.0, 1.99, 4.0, 6.0],
                    [7.9, 0.0, 3.0, 2.0, 5.5]])
    want = [(1 * 4 + 0) * 4 + 3, (3 * 4 + 1) * 4 + 0, (0 * 4 + 0) * 4 + 1, (3 * 4 + 2) * 4 + 1, (0 * 4 + 3) * 4 + 2]
    assert pm.cell_index(pos, n, box).tolist() == want


def test_cell_index_is_the_full_weight_corner():
    """The keyed point receives (1 - fx)(1 - fy)(1 - fz) of the particle in the deposit (Eq. CIC)."""
    n, box = 8, 16.0
    d = box / n
    rng = np.random.default_rng(5)
    for _ in range(20):
        p = rng.uniform(0, box, (3, 1))
        key = int(pm.cell_index(p, n, box)[0])
        f = p[:, 0] / d - np.floor(p[:, 0] / d)
        rho = pm.cic_deposit(p, n, box).reshape(-1)
        assert abs(rho[key] - np.prod(1 - f)) < 1e-14


def test_cell_sort_matches_a_stable_comparison_sort():
    n, box = 6, 12.0
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, box, (3, 900))
    pos[:, 100:200] = pos[:, 0:1]  # a crowded cell
    key = pm.cell_index(pos, n, box)
    order, start = pm.cell_sort(pos, n, box)
    assert order.tolist() == sorted(range(pos.shape[1]), key=lambda p: key[p])
    assert start[0] == 0 and start[-1] == pos.shape[1]
    for c in range(n ** 3):
        assert start[c + 1] - start[c] == int(np.sum(key == c))


@pytest.mark.parametrize("gravity,geff", [("grh", "GR"), ("nl", "local")])
def test_linear_growth_of_low_amplitude_wave(gravity, geff):
    """A long plane wave of tiny amplitude grows like D+(a) (the linearised
    dynamics of Sec. III.A with Eq. GRPoisson / Eq. LinearDGP); the PM force at
    k_f is weakened by the CIC window squared (~0.2% on 64^3), so 5e-3."""
    n, box = 64, 200.0
    a0, a1, nsteps = 0.05, 0.1, 20
    D0, f0 = bg.growth(a0, OM, 1.0, geff)
    D1, _ = bg.growth(a1, OM, 1.0, geff)
    # 1D Zel'dovich wave along x: Psi_x = A sin(k q)
    d = box / n
    q = np.arange(n) * d
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    k = 2 * np.pi / box
    amp = 1e-3 / k
    psi = amp * np.sin(k * qx)
    pos = np.stack([(qx + psi).reshape(-1), qy.reshape(-1), qz.reshape(-1)]) % box
    vf = a0 * a0 * float(bg.hubble_E(a0, OM, 1.0)) * f0
    mom = np.stack([vf * psi.reshape(-1), 0 * psi.reshape(-1), 0 * psi.reshape(-1)])
    st = pm.run(pos, mom, a0, a1, nsteps, n, box, OM, 1.0, gravity=gravity, tol=1e-10)
    disp = ((st.pos[0] - qx.reshape(-1) + box / 2) % box) - box / 2
    growth_sim = np.sum(disp * np.sin(k * qx.reshape(-1))) / np.sum(psi.reshape(-1) * np.sin(k * qx.reshape(-1)))
    assert abs(growth_sim / (D1 / D0) - 1) < 5e-3, (growth_sim, D1 / D0)


def test_linear_switch_epoch():
    """Sec. III.D: before a_nonlinear the linearised DGP equation is used; a
    switch after the run's end reproduces the lDGP run, a switch at a = 0 the
    nonlinear run, and a switch inside it solves nonlinearly only from there."""
    n, box = 16, 60.0
    pos, mom = inputs.lattice_particles(n, box)
    rng = np.random.default_rng(3)
    pos = (pos + rng.normal(0, 1.0, pos.shape)) % box
    kw = dict(tol=1e-10, max_iter=200)
    late = pm.run(pos, mom, 0.1, 0.2, 3, n, box, OM, 1.0, a_nonlinear=1.0, **kw)
    ldgp = pm.run(pos, mom, 0.1, 0.2, 3, n, box, OM, 1.0, gravity="ldgp", **kw)
    assert np.array_equal(late.pos, ldgp.pos) and np.array_equal(late.mom, ldgp.mom)
    early = pm.run(pos, mom, 0.1, 0.2, 3, n, box, OM, 1.0, a_nonlinear=0.0, **kw)
    nl = pm.run(pos, mom, 0.1, 0.2, 3, n, box, OM, 1.0, **kw)
    assert np.array_equal(early.pos, nl.pos)
    mid = pm.run(pos, mom, 0.1, 0.2, 3, n, box, OM, 1.0, a_nonlinear=0.15, **kw)
    assert [s["a"] < 0.15 for s in mid.solves] == [s["iters"] == 0 for s in mid.solves]
    assert not np.array_equal(mid.pos, nl.pos) and not np.array_equal(mid.pos, ldgp.pos)
