"""Pins for the oracle's charged pair: LJ plus the Ewald real-space term
q_i q_j erfc(alpha r) / r, the short-range Coulomb kernel to which the RBL extends
(Sec. 2, closing remarks; Sec. 4).

- alpha -> 0 reduces the term to Coulomb's law q_i q_j / r (force q_i q_j / r^2);
  alpha r -> infinity removes it;
- the term equals its integral representation (2 / sqrt(pi)) int_alpha^inf
  exp(-r^2 t^2) dt, evaluated by quadrature (independent of libm's erfc);
- the force is minus the gradient of the energy (pair and many-body, by Richardson
  finite differences);
- the rock-salt Madelung constant: the oracle's real-space energy plus a reciprocal-
  space sum and the self term written here reproduce -N M / (2 r0);
- the full list and RBL with p >= max N_s equal the all-pairs sum with charges.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

MADELUNG_NACL = 1.747564594633182  # rock salt, referred to the nearest-neighbour distance


def test_alpha_zero_is_coulomb_and_large_alpha_is_lj():
    r = np.array([0.9, 1.0, 1.3, 2.0, 3.1])
    u0, f0 = oracle.lj(r)
    for qq in (1.0, -1.0, 0.25):
        u, f = oracle.pair(r, qq, 0.0)
        assert np.allclose(u, u0 + qq / r, rtol=1e-14, atol=1e-14)
        assert np.allclose(f, f0 + qq / r**2, rtol=1e-14, atol=1e-14)
    u, f = oracle.pair(r, -1.0, 40.0)  # erfc(36) underflows to 0
    assert np.array_equal(u, u0) and np.array_equal(f, f0)


def test_erfc_term_equals_its_integral():
    quad = pytest.importorskip("scipy.integrate").quad
    r = np.array([0.95, 1.4, 2.2, 3.3])
    for alpha in (0.4, 1.0, 1.7):
        u, _ = oracle.pair(r, 1.0, alpha)
        u0, _ = oracle.lj(r)
        for k, rk in enumerate(r):
            integral, _ = quad(lambda t: math.exp(-(rk * t) ** 2), alpha, np.inf, epsabs=1e-15, epsrel=1e-13)
            assert abs((u[k] - u0[k]) - 2.0 / math.sqrt(math.pi) * integral) < 1e-12


def _richardson(fun, x0, h):
    d1 = (fun(x0 + h) - fun(x0 - h)) / (2 * h)
    d2 = (fun(x0 + h / 2) - fun(x0 - h / 2)) / h
    return (4 * d2 - d1) / 3


def test_pair_force_is_minus_energy_gradient():
    for qq, alpha in ((1.0, 0.8), (-1.0, 1.3), (0.3, 2.0)):
        for r in (0.92, 1.17, 1.6, 2.5, 3.4):
            _, f = oracle.pair(np.array([r]), qq, alpha)
            du = _richardson(lambda s: oracle.pair(np.array([s]), qq, alpha)[0][0], r, 1e-4)
            assert abs(f[0] + du) < 1e-7 * max(1.0, abs(f[0])), (qq, alpha, r)


def test_many_body_force_is_minus_energy_gradient():
    rs, alpha = 3.0, 1.0
    x, L = inputs.fcc(256, 0.6, 0.2, seed=9)
    q = inputs.charges(256, 1.0, seed=9)
    F, _ = oracle.brute_forces(x, L, rs, q=q, alpha=alpha)
    checked = 0
    for i in range(0, 256, 17):
        d = x - x[i]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        if np.min(np.abs(r - rs)) < 2e-3:  # no pair may cross the cutoff under the displacement
            continue
        for a in range(3):
            def energy(s, i=i, a=a):
                y = x.copy()
                y[i, a] = s
                return oracle.brute_forces(y, L, rs, q=q, alpha=alpha)[1][0]

            g = _richardson(energy, x[i, a], 1e-4)
            assert abs(F[i, a] + g) < 1e-6 * max(1.0, abs(F[i, a])), (i, a, F[i, a], -g)
        checked += 1
    assert checked >= 10


def test_rock_salt_madelung_energy():
    """Real-space part from the oracle, reciprocal part (2 pi / V) sum_k exp(-k^2 /
    4 alpha^2) / k^2 |S(k)|^2 and self term -alpha / sqrt(pi) sum q^2 computed here:
    the Ewald total is the lattice energy -N M / (2 r0)."""
    n, r0, rs, alpha = 8, 1.1, 3.5, 1.2
    x, L, q = inputs.rock_salt(n, r0)
    N = x.shape[0]
    _, ev_q = oracle.brute_forces(x, L, rs, q=q, alpha=alpha)
    _, ev_0 = oracle.brute_forces(x, L, rs)
    u_real = ev_q[0] - ev_0[0]
    V = float(np.prod(L))
    mmax = 20
    m = np.arange(-mmax, mmax + 1)
    mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
    mv = np.stack([mx.ravel(), my.ravel(), mz.ravel()], 1)
    m2 = (mv * mv).sum(1)
    mv = mv[(m2 > 0) & (m2 <= mmax * mmax)]
    k = 2 * np.pi * mv / L
    k2 = (k * k).sum(1)
    u_rec = 0.0
    for s in range(0, k.shape[0], 4096):
        phase = k[s : s + 4096] @ x.T
        S = (np.cos(phase) @ q) ** 2 + (np.sin(phase) @ q) ** 2
        u_rec += float(np.sum(np.exp(-k2[s : s + 4096] / (4 * alpha**2)) / k2[s : s + 4096] * S))
    u_rec *= 2 * np.pi / V
    u_self = -alpha / math.sqrt(math.pi) * float(np.sum(q * q))
    exact = -N * MADELUNG_NACL / (2 * r0)
    assert abs(u_real + u_rec + u_self - exact) < 2e-8 * abs(exact)
    # a wrong real-space term (a missing factor or sign) moves the total by O(1)
    assert abs(u_real) > 0.1 * abs(exact)


@pytest.fixture(scope="module")
def charged():
    rc, rs, skin, alpha = 1.5, 3.5, 0.3, 1.0
    x, L = inputs.fcc(1000, 0.8, 0.15, seed=3)
    q = inputs.charges(1000, 1.0, seed=3)
    lists = oracle.build_lists(x, L, rc, rs, skin, K=2)
    return x, L, q, lists, rc, rs, skin, alpha


def test_charged_full_list_and_large_batch_equal_all_pairs(charged):
    x, L, q, lists, rc, rs, skin, alpha = charged
    Fb, evb = oracle.brute_forces(x, L, rs, q=q, alpha=alpha)
    Ff, evf = oracle.full_forces(x, L, rs, lists, q=q, alpha=alpha)
    assert np.allclose(Ff, Fb, rtol=0, atol=1e-12 * np.abs(Fb).max())
    assert np.allclose(evf, evb, rtol=1e-12)
    p = int(lists.n_shell.max())
    Fr, evr, _, _ = oracle.rbl_forces(x, L, rc, rs, skin, p, 1, 0, lists, q=q, alpha=alpha)
    assert np.allclose(Fr, Fb, rtol=0, atol=1e-12 * np.abs(Fb).max())
    assert np.allclose(evr, evb, rtol=1e-12)
    assert np.all(np.abs(Fb.sum(0)) < 1e-9)
    # the charges matter: the LJ-only force differs
    F0, _ = oracle.brute_forces(x, L, rs)
    assert np.abs(F0 - Fb).max() > 0.1


def test_charged_sample_equals_full_system_oracle(charged):
    x, L, q, lists, rc, rs, skin, alpha = charged
    p, seed, step = 10, 4, 9
    F, _, batch, bn = oracle.rbl_forces(x, L, rc, rs, skin, p, seed, step, lists, want_batch=True, q=q,
                                        alpha=alpha)
    idx = np.array([0, 5, 333, 999])
    smp = oracle.sample(x, L, rc, rs, skin, p, seed, step, idx, K=2, q=q, alpha=alpha)
    for k, i in enumerate(idx):
        assert np.array_equal(smp.batch[k, : bn[i]], batch[i, : bn[i]])
        assert np.array_equal(smp.F[k], F[i])


def test_charged_shell_estimator_unbiased(charged):
    """Mean over seeds of the RBL force approaches the classical-cutoff force (the
    estimator is unbiased for any pair kernel, Appendix A)."""
    x, L, q, lists, rc, rs, skin, alpha = charged
    Fb, _ = oracle.full_forces(x, L, rs, lists, q=q, alpha=alpha)
    M = 400
    acc = np.zeros_like(Fb)
    acc2 = np.zeros_like(Fb)
    for m in range(M):
        F, _, _, _ = oracle.rbl_forces(x, L, rc, rs, skin, 10, 500 + m, 3, lists, q=q, alpha=alpha)
        acc += F
        acc2 += F * F
    mean = acc / M
    var = acc2 / M - mean**2
    z = np.abs(mean - Fb) / np.sqrt(var / M + 1e-30)
    live = var > 1e-12
    assert live.sum() > 1000
    assert np.quantile(z[live], 0.99) < 3.5 and z[live].max() < 6.0


def test_charged_inputs():
    """The seeded charge generators: neutral, half +q and half -q (one 0 for odd N), a
    seed-dependent order; the rock-salt lattice has opposite charges on nearest neighbours."""
    for N in (10, 11, 1000):
        q = inputs.charges(N, 2.0, seed=4)
        assert q.sum() == 0.0 and (q == 2.0).sum() == N // 2 and (q == -2.0).sum() == N // 2
    assert not np.array_equal(inputs.charges(100, 1.0, seed=1), inputs.charges(100, 1.0, seed=2))
    x, L, q = inputs.rock_salt(4, 1.1)
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    nn = np.isclose(r, 1.1)
    assert nn.sum() == 6 * len(x)  # six nearest neighbours each
    assert np.all((q[:, None] * q[None, :])[nn] == -1.0)
