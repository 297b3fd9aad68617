"""Pins for the oracle's time stepping and observables.

- free flight (no pair inside r_s): velocity-Verlet moves x by v t exactly;
- the O-step: with no forces the velocities follow the Ornstein-Uhlenbeck law,
  mean c1^n v0, variance T (1 - c1^(2n)), c1 = exp(-gamma dt);
- a bound dimer: velocity-Verlet energy error shrinks as dt^2;
- momentum: the net-force correction keeps the total momentum fixed (gamma = 0);
- tail corrections against numerical quadrature of the LJ tail integrals;
- g(r) counts of a perfect FCC crystal against its coordination shells.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2105_04884_gb300 import inputs


def _sparse_lattice(n_side, spacing):
    g = np.stack(np.meshgrid(*[np.arange(n_side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.5) * spacing
    return x.astype(np.float64), np.full(3, n_side * spacing)


def test_free_flight_velocity_verlet():
    x, L = _sparse_lattice(4, 9.0)  # spacing 9 > r_s + skin: no pairs at all
    v = np.random.default_rng(1).normal(size=x.shape)
    dt, n = 0.005, 50
    x2, v2, F, stats = oracle.run(x, v, L, 1.5, 3.5, 0.3, 10, dt, 1.0, 0.0, 1, n, subtract_mean=False)
    assert np.all(F == 0.0) and np.array_equal(v2, v)
    want = np.mod(x + n * dt * v, L)
    d = x2 - want
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-12


def test_ornstein_uhlenbeck_statistics():
    x, L = _sparse_lattice(16, 9.0)  # 4096 non-interacting particles
    v0 = np.full_like(x, 1.0)
    gamma, dt, T, n = 1.0, 0.01, 1.7, 60
    _, v, _, _ = oracle.run(x, v0, L, 1.5, 3.5, 0.3, 10, dt, T, gamma, 3, n, subtract_mean=False)
    c1 = math.exp(-gamma * dt)
    mean = c1**n
    var = T * (1 - c1 ** (2 * n))
    m = v.size
    assert abs(v.mean() - mean) < 5 * math.sqrt(var / m)
    assert abs(v.var() / var - 1) < 5 * math.sqrt(2 / m)


def _dimer_energy_error(dt, t_end=5.0):
    L = np.full(3, 20.0)
    x = np.array([[5.0, 5.0, 5.0], [6.2, 5.0, 5.0]])
    v = np.array([[0.3, 0.1, 0.0], [-0.3, -0.1, 0.0]])

    def energy(x, v):
        r = np.linalg.norm(x[0] - x[1])
        return 4 * (r**-12 - r**-6) + 0.5 * (v * v).sum()

    e0 = energy(x, v)
    worst = 0.0
    steps = int(round(t_end / dt))
    chunk = max(1, steps // 50)
    for _ in range(steps // chunk):
        x, v, _, _ = oracle.run(x, v, L, 1.5, 3.5, 0.3, 10, dt, 1.0, 0.0, 1, chunk, subtract_mean=False)
        worst = max(worst, abs(energy(x, v) - e0))
    return worst


def test_velocity_verlet_second_order():
    e1 = _dimer_energy_error(0.004)
    e2 = _dimer_energy_error(0.002)
    assert 3.0 < e1 / e2 < 5.0


def test_momentum_conserved_with_correction():
    x, L = inputs.fcc(500, 0.8, 0.05, seed=2)
    v = inputs.maxwell_boltzmann(500, 1.5, seed=2)
    _, v2, F, _ = oracle.run(x, v, L, 1.5, 3.5, 0.3, 5, 0.005, 1.5, 0.0, 1, 20, subtract_mean=True)
    assert np.abs(v2.sum(0)).max() < 1e-10
    assert np.abs(F.sum(0)).max() < 1e-9


def test_tail_corrections_by_quadrature():
    rho, rs = 0.8, 3.5

    def u(r):
        return 4 * (r**-12 - r**-6)

    def du(r):
        return -48 * r**-13 + 24 * r**-7

    ut = 2 * math.pi * rho * integrate.quad(lambda r: u(r) * r * r, rs, np.inf)[0]
    pt = -2 * math.pi / 3 * rho * rho * integrate.quad(lambda r: du(r) * r**3, rs, np.inf)[0]
    got = oracle.tail(rho, rs)
    assert abs(got[0] - ut) < 1e-10 and abs(got[1] - pt) < 1e-10


def test_ideal_gas_pressure():
    v = inputs.maxwell_boltzmann(1000, 2.0, seed=4)
    L = np.array([10.0, 11.0, 12.0])
    k, t, p = oracle.thermo(v, L, 0.0)
    assert abs(k - 0.5 * (v * v).sum()) < 1e-9
    assert abs(p - 1000 / L.prod() * t) < 1e-12


def test_rdf_counts_on_fcc():
    x, L = inputs.fcc(500, 1.0, 0.0)  # 5x5x5 cells
    a = L[0] / 5
    dr = 0.01
    nb = int(0.5 * L[0] / dr)
    h = oracle.rdf_counts(x, L, dr, nb)
    bas = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    shells = {}
    for v in itertools.product(range(-3, 4), repeat=3):
        for b in bas:
            q = (np.array(v) + b) * a
            r = math.sqrt(q @ q)
            if 0 < r < 0.5 * L[0]:
                k = round(r, 9)
                shells[k] = shells.get(k, 0) + 1
    for r, z in shells.items():
        assert h[int(r / dr)] == 500 * z, (r, z)
    assert h.sum() == 500 * sum(shells.values())


def test_density_profile_counts():
    """Profile counts: all particles counted; bins agree with floor(x nbins / L)
    away from bin edges; a liquid-vapour slab shows its two densities."""
    x, L = inputs.fcc(3000, 0.8, 0.3, seed=4)
    for axis, nb in ((0, 7), (2, 40)):
        h = oracle.density_profile(x, L, axis, nb)
        assert h.sum() == len(x)
        t = x[:, axis] / L[axis] * nb
        safe = np.abs(t - np.round(t)) > 1e-6
        ref = np.bincount(np.floor(t[safe]).astype(int), minlength=nb)
        h_safe = oracle.density_profile(x[safe], L, axis, nb)
        assert np.array_equal(h_safe, ref)
    V = 30.0 * 30.0 * 120.0
    N = int(round(0.75 * 0.4 * V + 0.01 * 0.6 * V))  # liquid over 40% of z, vapour elsewhere
    x, L = inputs.slab(N, 30.0, 120.0, 0.75, 0.01, seed=3)
    nb = 240  # 0.5 sigma bins (single bins alias with the start's lattice planes: average regions)
    h = oracle.density_profile(x, L, 2, nb)
    rho = h / (L[0] * L[1] * (L[2] / nb))
    z = (np.arange(nb) + 0.5) * L[2] / nb
    liquid = np.abs(z - L[2] / 2) < 0.15 * L[2]
    vapour = np.abs(z - L[2] / 2) > 0.3 * L[2]
    assert abs(rho[liquid].mean() - 0.75) < 0.02
    assert rho[vapour].mean() < 0.05
