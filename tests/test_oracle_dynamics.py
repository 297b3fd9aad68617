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


# ---------------------------------------------------------------------------
# BAOAB positions with friction (gamma > 0).  One step of the splitting is
# B: v += dt/2 F; A: x += dt/2 v; O: v = c1 v + c2 xi; A: x += dt/2 v; B: v += dt/2 F
# (Leimkuhler & Matthews; the underdamped Langevin equation, Eq. (2)).  The pins
# below follow from that sequence alone and fail for a dropped or doubled half
# drift, a single full-dt drift, or an O step outside the two A steps.
# ---------------------------------------------------------------------------
def _min_image(d, L):
    return d - L * np.round(d / L)


def test_baoab_free_particles_zero_temperature_closed_form():
    """T = 0, no pair inside r_s: v_n = c1^n v0 and
    x_n = x0 + (dt/2)(1 + c1) v0 (1 - c1^n) / (1 - c1)."""
    x, L = _sparse_lattice(4, 9.0)
    v0 = np.random.default_rng(5).normal(size=x.shape)
    gamma, dt, n = 1.3, 0.01, 37
    x2, v2, F, _ = oracle.run(x, v0, L, 1.5, 3.5, 0.3, 10, dt, 0.0, gamma, 2, n, subtract_mean=False)
    assert np.all(F == 0.0)
    c1 = math.exp(-gamma * dt)
    assert np.abs(v2 - c1**n * v0).max() < 1e-13
    want = x + 0.5 * dt * (1.0 + c1) * v0 * (1.0 - c1**n) / (1.0 - c1)
    assert np.abs(_min_image(x2 - want, L)).max() < 1e-12
    # the alternatives differ from it by far more than the tolerance
    for wrong in (0.5 * dt * c1, 0.5 * dt, dt, dt * c1):
        alt = x + wrong * v0 * (1.0 - c1**n) / (1.0 - c1)
        assert np.abs(_min_image(x2 - alt, L)).max() > 1e-4


def test_baoab_free_particles_trapezoid_drift_with_noise():
    """T > 0, free particles, one step per call: the two half drifts straddle the
    O step, so x_{k+1} - x_k = (dt/2)(v_k + v_{k+1}) for every particle, whatever
    the noise drew; the noise itself changes v (v_{k+1} != c1 v_k)."""
    x, L = _sparse_lattice(8, 9.0)
    v = inputs.maxwell_boltzmann(len(x), 1.2, seed=6)
    gamma, dt, T = 1.0, 0.005, 1.7
    c1 = math.exp(-gamma * dt)
    for k in range(6):
        x2, v2, _, _ = oracle.run(x, v, L, 1.5, 3.5, 0.3, 10, dt, T, gamma, 4, 1, step0=k, subtract_mean=False)
        d = _min_image(x2 - x, L)
        # two drifts, each rounded at the position's magnitude (up to L)
        assert np.abs(d - 0.5 * dt * (v + v2)).max() < 8 * np.spacing(L.max())
        assert np.abs(v2 - c1 * v).max() > 1e-3
        x, v = x2, v2


def test_baoab_free_particles_position_variance():
    """T > 0, v0 = 0, n steps: x_n - x0 = sum_m a_m xi_m with
    a_m = (dt/2) c2 [1 + (1 + c1)(1 - c1^(n-1-m)) / (1 - c1)], c2 = sqrt((1 - c1^2) T),
    so each component has variance sum_m a_m^2 (derived from the splitting)."""
    x, L = _sparse_lattice(16, 9.0)
    gamma, dt, T, n = 2.0, 0.05, 1.5, 4
    c1 = math.exp(-gamma * dt)
    c2 = math.sqrt((1 - c1 * c1) * T)
    a = [0.5 * dt * c2 * (1 + (1 + c1) * (1 - c1 ** (n - 1 - m)) / (1 - c1)) for m in range(n)]
    var = sum(t * t for t in a)
    x2, _, _, _ = oracle.run(x, np.zeros_like(x), L, 1.5, 3.5, 0.3, 10, dt, T, gamma, 7, n, subtract_mean=False)
    d = _min_image(x2 - x, L).ravel()
    m = d.size
    assert abs(d.mean()) < 5 * math.sqrt(var / m)
    assert abs(d.var() / var - 1) < 5 * math.sqrt(2 / m)
    # an O step before both drifts (x += dt v after O) would give sum of (dt c2 ...)^2
    alt = sum((dt * c2 * (1 - c1 ** (n - m)) / (1 - c1)) ** 2 for m in range(n))
    assert abs(alt / var - 1) > 10 * math.sqrt(2 / m)


def test_baoab_drift_with_forces():
    """Interacting LJ fluid, gamma > 0, one step per call: the drift uses the
    velocity after the opening half kick and after the O step, so
    x_{k+1} - x_k = (dt/2)[v_k + v_{k+1} + (dt/2)(F_k - F_{k+1})], F_k the force the
    step opens with (a call of zero steps at the same state and step returns it:
    each call builds its lists at its start) and F_{k+1} the one it closes with."""
    x, L = inputs.fcc(500, 0.8, 0.05, seed=8)
    v = inputs.maxwell_boltzmann(500, 1.5, seed=8)
    dt, T, gamma = 0.005, 1.5, 1.0
    for k in range(5):
        _, _, F, _ = oracle.run(x, v, L, 1.5, 3.5, 0.3, 10, dt, T, gamma, 3, 0, step0=k)
        assert np.abs(F).max() > 1.0
        x2, v2, F2, _ = oracle.run(x, v, L, 1.5, 3.5, 0.3, 10, dt, T, gamma, 3, 1, step0=k)
        d = _min_image(x2 - x, L)
        want = 0.5 * dt * (v + v2 + 0.5 * dt * (F - F2))
        assert np.abs(d - want).max() < 8 * np.spacing(L.max())
        # a drift from the kicked velocity alone (O after both drifts) is far off
        alt = 0.5 * dt * (2 * v + dt * F)
        assert np.abs(d - alt).max() > 1e-5
        x, v = x2, v2
