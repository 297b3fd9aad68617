"""Pins for the oracle's paper-literal sampling pool (Sec. 2): the pool of particle
i is every other particle in the (2m+1)^3 cells around i's cell, m = floor(r_s/r_c)
+ 1, on cells of edge >= r_c + skin; the batch is drawn from it and scaled by N_I/p.

Checked against numpy cell arithmetic written here, the all-pairs force, and the
sampling law over seeds."""
import math

import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

RC, RS, SKIN = 1.5, 3.5, 0.3


@pytest.fixture(scope="module")
def fluid():
    x, L = inputs.fcc(1200, 0.8, 0.2, seed=11)
    return x, L, oracle.build_pool(x, L, RC, RS, SKIN)


def test_pool_is_the_stencil_of_cells(fluid):
    m = math.floor(RS / RC) + 1
    x, L = inputs.fcc(4000, 0.8, 0.2, seed=12)  # 9 cells per axis >= 2m + 1
    pl = oracle.build_pool(x, L, RC, RS, SKIN)
    n = np.floor(L / (RC + SKIN)).astype(int)
    assert np.array_equal(pl.grid, n) and np.all(n >= 2 * m + 1)
    u = oracle.quantize(x, L).astype(np.uint64)
    c = ((u * n.astype(np.uint64)) >> np.uint64(32)).astype(np.int64)
    for i in range(0, len(x), 97):
        d = (c - c[i]) % n
        d = np.where(d > n // 2, d - n, d)
        want = set(np.nonzero(np.all(np.abs(d) <= m, axis=1))[0].tolist()) - {i}
        assert set(pl.row("shell", i).tolist()) == want, i
    # fewer than 2m + 1 cells per axis: every cell once, so the pool is everyone else
    x, L, small = fluid
    assert np.all(small.grid < 2 * m + 1) and np.all(small.n_shell == len(x) - 1)


def test_pool_covers_the_shell_and_core_rows_match(fluid):
    x, L, pl = fluid
    sh = oracle.build_lists(x, L, RC, RS, SKIN, K=2)
    dx = x[:, None, :] - x[None, :, :]
    dx -= L * np.round(dx / L)
    r = np.sqrt((dx * dx).sum(-1))
    for i in range(0, len(x), 41):
        within = set(np.nonzero((r[i] < RS) & (np.arange(len(x)) != i))[0].tolist())
        assert within <= set(pl.row("shell", i).tolist()), i
        assert set(pl.row("core", i).tolist()) == set(sh.row("core", i).tolist()), i


def test_whole_pool_is_the_classical_cutoff(fluid):
    """p >= N_I: every pool member is taken with scale 1, which is the cutoff force."""
    x, L, pl = fluid
    F, ev, _, _ = oracle.rbl_forces(x, L, RC, RS, SKIN, 100000, 1, 0, pl)
    Fb, evb = oracle.brute_forces(x, L, RS)
    assert np.allclose(F, Fb, rtol=0, atol=1e-12 * np.abs(Fb).max())
    assert np.allclose(ev, evb, rtol=1e-12)


def test_pool_estimator_unbiased():
    """Mean over seeds of the pool estimate of the shell force -> the exact shell force
    (E over uniform p-subsets of the pool, with zero terms outside r_c <= r < r_s)."""
    x, L = inputs.fcc(500, 0.8, 0.15, seed=5)
    pl = oracle.build_pool(x, L, RC, RS, SKIN)
    p = 10
    Fcore, _, _, _ = oracle.rbl_forces(x, L, RC, RC, SKIN, 1, 0, 0, pl)  # r_s = r_c: shell masked out
    Fexact, _ = oracle.brute_forces(x, L, RS)
    Fc_only, _ = oracle.brute_forces(x, L, RC)
    M = 3000
    acc = np.zeros((500, 3))
    acc2 = np.zeros((500, 3))
    for k in range(M):
        F, _, _, _ = oracle.rbl_forces(x, L, RC, RS, SKIN, p, 2000 + k, 3, pl)
        y = F - Fcore
        acc += y
        acc2 += y * y
    mean = acc / M
    var = acc2 / M - mean ** 2
    exact = Fexact - Fc_only
    z = np.abs(mean - exact) / np.sqrt(var / M + 1e-30)
    assert np.max(z) < 5.0
