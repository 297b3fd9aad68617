"""Pins for the oracle's LJ pair, RBL force estimator and net-force correction.

- closed forms of the LJ 12-6 pair (Sec. 2, Eq. (1));
- a two-body system whose force is known exactly;
- the all-pairs O(N^2) sum, which uses no lists at all;
- the identity 'N_s <= p reduces to the classical cutoff scheme' (Algorithm 1);
- unbiasedness and the without-replacement variance of the shell estimator
  (Appendix A), over many seeds;
- lattice symmetry (zero force) and lattice sums counted from integer vectors.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

RC, RS, SKIN = 1.5, 3.5, 0.3


def test_lj_closed_forms():
    u, f = oracle.lj(np.array([1.0, 2 ** (1 / 6), 1.5]))
    assert u[0] == 0.0 and abs(u[1] + 1.0) < 1e-15
    assert f[0] == 24.0 and abs(f[1]) < 1e-13
    r = 1.5
    assert abs(u[2] - 4 * (r**-12 - r**-6)) < 1e-15
    assert abs(f[2] - 24 * (2 * r**-13 - r**-7)) < 1e-15


def test_two_body_force():
    L = np.array([20.0, 20.0, 20.0])
    for r in (0.95, 1.3, 2.0, 3.2):
        x = np.array([[1.0, 5.0, 5.0], [1.0 + r, 5.0, 5.0]])
        F, ev = oracle.brute_forces(x, L, RS)
        mag = 24 * (2 * r**-13 - r**-7)
        assert np.allclose(F[0], [-mag, 0, 0], rtol=1e-13, atol=1e-14)
        assert np.allclose(F[1], [mag, 0, 0], rtol=1e-13, atol=1e-14)
        assert abs(ev[0] - 4 * (r**-12 - r**-6)) < 1e-14
    # across the periodic face
    x = np.array([[0.3, 5.0, 5.0], [19.5, 5.0, 5.0]])
    F, _ = oracle.brute_forces(x, L, RS)
    r = 0.8
    assert np.allclose(F[0], [24 * (2 * r**-13 - r**-7), 0, 0], rtol=1e-12)


@pytest.fixture(scope="module")
def fluid():
    x, L = inputs.fcc(1000, 0.8, 0.15, seed=1)
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=2)
    return x, L, lists


def test_full_list_equals_all_pairs(fluid):
    x, L, lists = fluid
    Fb, evb = oracle.brute_forces(x, L, RS)
    Ff, evf = oracle.full_forces(x, L, RS, lists)
    assert np.allclose(Ff, Fb, rtol=0, atol=1e-12 * np.abs(Fb).max())
    assert np.allclose(evf, evb, rtol=1e-12)
    # Newton's third law: the total force vanishes
    assert np.all(np.abs(Fb.sum(0)) < 1e-9)


def test_rbl_with_large_batch_is_classical_cutoff(fluid):
    """p >= max N_s: every shell neighbour is in the batch with scale 1."""
    x, L, lists = fluid
    p = int(lists.n_shell.max())
    F, ev, _, _ = oracle.rbl_forces(x, L, RC, RS, SKIN, p, 1, 0, lists)
    Fb, evb = oracle.brute_forces(x, L, RS)
    assert np.allclose(F, Fb, rtol=0, atol=1e-12 * np.abs(Fb).max())
    assert np.allclose(ev, evb, rtol=1e-12)


def test_perfect_fcc_has_zero_force():
    x, L = inputs.fcc(864, 1.0, 0.0)
    F, _ = oracle.brute_forces(x, L, RS)
    assert np.abs(F).max() < 1e-10
    lists = oracle.build_lists(x, L, RC, RS, SKIN)
    F2, _, _, _ = oracle.rbl_forces(x, L, RC, RS, SKIN, 10_000, 1, 0, lists)
    assert np.abs(F2).max() < 1e-10


def test_fcc_lattice_energy_and_virial():
    """Energy and virial per particle of a perfect FCC crystal = half the lattice sums
    over neighbours inside r_s, counted from integer vectors."""
    rho = 1.0
    x, L = inputs.fcc(864, rho, 0.0)
    a = L[0] / 6
    _, ev = oracle.brute_forces(x, L, RS)
    bas = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    e = w = 0.0
    for v in itertools.product(range(-4, 5), repeat=3):
        for b in bas:
            q = (np.array(v) + b) * a
            r = math.sqrt(q @ q)
            if 0 < r < RS:
                e += 4 * (r**-12 - r**-6)
                w += 24 * (2 * r**-12 - r**-6)
    assert abs(ev[0] / 864 - e / 2) < 1e-10 * abs(e)
    assert abs(ev[1] / 864 - w / 2) < 1e-10 * abs(w)


def test_subtract_mean():
    F = np.random.default_rng(0).normal(size=(100, 3))
    G = oracle.subtract_mean(F)
    assert np.all(np.abs(G.sum(0)) < 1e-12)
    assert np.allclose(G - F, -F.mean(0))


def _shell_terms(x, L, lists, i, rc, rs):
    """y_j: the masked pair force f~_ij for every entry of i's shell row (0 outside
    r_c <= r < r_s), computed here in FP64 from the positions."""
    row = lists.row("shell", i)
    u = oracle.quantize(x, L)
    r2f = oracle.pair_r2f(u, L, np.full(row.size, i, np.int32), row.astype(np.int32))
    d = x[i] - x[row]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(1)
    mask = (r2f >= np.float32(rc * rc)) & (r2f < np.float32(rs * rs))
    coef = 24 * (2 * r2**-6 - r2**-3) / r2
    return np.where(mask[:, None], coef[:, None] * d, 0.0)


@pytest.mark.parametrize("rs_,skin_", [(RS, SKIN), (2.0, 0.1)])
def test_shell_estimator_unbiased_and_srswor_variance(rs_, skin_):
    """Over M seeds: mean of F~_s -> F_s (Appendix A, E[F~_s] = F_s) and variance ->
    N_s (N_s - p) / p * S^2, the simple-random-sampling-without-replacement variance
    equivalent to Appendix A's second moment with its (p-1)/(N-1) factor."""
    x, L = inputs.fcc(500, 0.8, 0.15, seed=5)
    p = 10
    lists = oracle.build_lists(x, L, RC, rs_, skin_, K=2)
    # core part is deterministic: isolate the shell estimate
    Fcore, _, _, _ = oracle.rbl_forces(x, L, RC, RC, skin_, 1, 0, 0, lists)  # r_s = r_c: shell masked out
    M = 3000
    samples = np.zeros((M, 500, 3))
    for m in range(M):
        F, _, _, _ = oracle.rbl_forces(x, L, RC, rs_, skin_, p, 1000 + m, 7, lists)
        samples[m] = F - Fcore
    idx = [i for i in range(0, 500, 25) if lists.n_shell[i] > p]
    zmax = 0.0
    for i in idx:
        y = _shell_terms(x, L, lists, i, RC, rs_)
        ns = y.shape[0]
        exact = y.sum(0)
        var = ns * (ns - p) / p * y.var(0, ddof=1)
        mean = samples[:, i].mean(0)
        z = np.abs(mean - exact) / np.sqrt(var / M)
        zmax = max(zmax, float(z.max()))
        emp = samples[:, i].var(0, ddof=1)
        # variance ratio: sampling error of a variance estimate ~ sqrt(2/M) (plus kurtosis)
        assert np.all(np.abs(emp / var - 1) < 0.25), (i, emp / var)
    assert zmax < 4.5


def test_sample_equals_full_system_oracle():
    """Per-particle sampling (rows by testing all pairs, batch, force) reproduces the
    whole-system oracle exactly for the sampled particles."""
    rc, rs, skin, p, seed, step = 1.5, 3.5, 0.3, 10, 7, 13
    x, L = inputs.fcc(1500, 0.8, 0.2, seed=21)
    lists = oracle.build_lists(x, L, rc, rs, skin, K=2)
    F, _, batch, bn = oracle.rbl_forces(x, L, rc, rs, skin, p, seed, step, lists, want_batch=True)
    idx = np.array([0, 1, 17, 512, 777, 1499])
    smp = oracle.sample(x, L, rc, rs, skin, p, seed, step, idx, K=2)
    for k, i in enumerate(idx):
        assert np.array_equal(smp.row("core", k), lists.row("core", i))
        assert np.array_equal(smp.row("shell", k), lists.row("shell", i))
        assert smp.n_batch[k] == bn[i]
        assert np.array_equal(smp.batch[k, : bn[i]], batch[i, : bn[i]])
        assert np.array_equal(smp.F[k], F[i])
