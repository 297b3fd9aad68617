"""Parity at the full sizes of the two other timed workloads, on sampled particles
checked one by one against the oracle (which tests every other particle of the
system for each of them): core and shell rows and the batch bit-exact, the
un-subtracted force within the FP32 bar (1e-5 relative global norm over the sample).

- liquid-vapour slab: N = 4,194,304 in Lx = Ly, Lz = 4 Lx, liquid rho* = 0.75 over
  the central 40% of z, vapour rho* = 0.01 elsewhere, T* = 0.9, r_c = 1.5, r_s = 4.0,
  skin 0.3, p = 20, FP32, capacities from the liquid density; after 10 graph-path
  steps; particles sampled in the liquid, at the interfaces and in the vapour;
- ensemble: 256 replicas, N log-uniform in [500, 20000], rho* in [0.6, 0.9], T* in
  [1, 2], r_c = 1.5, r_s = 3.5, skin 0.3, p = 10, FP32; after 10 steps of the one-graph
  ensemble step; the smallest and the largest replica and six others, 16 particles each.
"""
import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402


def _check(sm, rows_c, nc, rows_s, ns, batch, nb, F):
    assert np.array_equal(nc, sm.n_core) and np.array_equal(ns, sm.n_shell)
    for k in range(len(nc)):
        assert np.array_equal(rows_c[k, : nc[k]], sm.row("core", k)), k
        assert np.array_equal(rows_s[k, : ns[k]], sm.row("shell", k)), k
    assert np.array_equal(nb, sm.n_batch)
    for k in range(len(nb)):
        assert np.array_equal(batch[k, : nb[k]], sm.batch[k, : sm.n_batch[k]]), k
    assert np.linalg.norm(F - sm.F) <= 1e-5 * np.linalg.norm(sm.F)


def test_slab_full_size_sampled():
    N, rho_l, rho_v, frac = 4194304, 0.75, 0.01, 0.4
    rc, rs, skin, p, dt, T = 1.5, 4.0, 0.3, 20, 0.005, 0.9
    V = N / (rho_l * frac + rho_v * (1.0 - frac))
    Lx = (V / 4.0) ** (1.0 / 3.0)
    x, L = inputs.slab(N, Lx, 4.0 * Lx, rho_l, rho_v, frac, seed=1)
    v = inputs.maxwell_boltzmann(len(x), T, seed=1)
    common = dict(T=T, gamma=1.0, seed=1, precision=rbl.RBL_FP32, cells_per_cutoff=2, rho_cap=rho_l)
    s = rbl.System(x, v, L, rc, rs, skin, p, dt, **common)
    s.step(10)
    x1, v1, step = s.get_state()
    del s
    torch.cuda.empty_cache()
    # a context loaded with the stepped state builds its lists at these positions
    raw = rbl.System(x1, v1, L, rc, rs, skin, p, dt, subtract_net_force=False, step=step, **common)
    F = raw.forces()
    dz = np.abs(x1[:, 2] - L[2] / 2)
    half = frac * L[2] / 2
    rng = np.random.default_rng(7)
    idx = np.sort(np.concatenate([rng.choice(np.nonzero(dz < half - 3.0)[0], 48, replace=False),
                                  rng.choice(np.nonzero(np.abs(dz - half) < 2.0)[0], 48, replace=False),
                                  rng.choice(np.nonzero(dz > half + 5.0)[0], 32, replace=False)]))
    sm = oracle.sample(x1, L, rc, rs, skin, p, 1, step, idx, K=2)
    rows_c, nc = raw.get_rows(0, idx)
    rows_s, ns = raw.get_rows(1, idx)
    batch, nb = raw.get_batch(step)
    _check(sm, rows_c, nc, rows_s, ns, batch[idx], nb[idx], F[idx])
    # the sample spans the density contrast: full shells in the liquid, nearly empty in the vapour
    assert ns[dz[idx] < half - 3.0].mean() > 5 * max(ns[dz[idx] > half + 5.0].mean(), 1.0)
    del raw
    torch.cuda.empty_cache()


def test_ensemble_full_size_sampled():
    shared = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, gamma=1.0, cells_per_cutoff=2,
                  precision=rbl.RBL_FP32)
    reps = inputs.ensemble(256, seed=1)
    ens = rbl.Ensemble(reps, **shared)
    ens.step(10)
    x, v, step = ens.get_state()
    xs, vs = ens.split(x), ens.split(v)
    del ens
    torch.cuda.empty_cache()
    reps1 = [inputs.Replica(rp.N, rp.rho, rp.T, rp.seed, xs[r], vs[r], rp.L) for r, rp in enumerate(reps)]
    raw = rbl.Ensemble(reps1, subtract_net_force=False, step=step, **shared)
    F = raw.forces()
    batch, nb = raw.get_batch(step)
    sizes = np.array([rp.N for rp in reps])
    rng = np.random.default_rng(8)
    others = rng.choice(np.setdiff1d(np.arange(256), [sizes.argmin(), sizes.argmax()]), 6, replace=False)
    for r in [int(sizes.argmin()), int(sizes.argmax())] + [int(k) for k in others]:
        rp = reps1[r]
        idx = np.sort(rng.choice(rp.N, 16, replace=False))
        rows = raw.offsets[r] + idx
        sm = oracle.sample(rp.x, rp.L, 1.5, 3.5, 0.3, 10, rp.seed, step, idx, K=2)
        rows_c, nc = raw.get_rows(0, rows)
        rows_s, ns = raw.get_rows(1, rows)
        _check(sm, rows_c, nc, rows_s, ns, batch[rows], nb[rows], F[rows])
    del raw
    torch.cuda.empty_cache()
