"""Batched ensemble (many independent replicas of uneven N, density and temperature
advanced by one launch per kernel) against the same replicas run one by one, and
one replica against the oracle.

Each replica of an ensemble must evolve exactly as a context of its own: the same
lists and batches (bit-exact), the same forces (bit-exact: every sum is taken in
the same canonical order, and each replica starts on a tile boundary so its block
partition is the same), the same trajectory and the same rebuild decisions."""
import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

SHARED = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, gamma=1.0)


def _replicas():
    # uneven sizes (ragged tiles), densities and temperatures, one box with fewer
    # than 2K + 1 cells per axis (N = 500 at rho* = 0.9: L = 8.22)
    spec = [(500, 0.9, 1.0), (1000, 0.8, 1.5), (2113, 0.6, 2.0), (777, 0.75, 1.2), (3001, 0.85, 1.8)]
    out = []
    for r, (N, rho, T) in enumerate(spec):
        # jitter 0.05: larger jitter puts pairs near 0.5 sigma, where a dt = 0.005 step blows up
        x, L = inputs.fcc(N, rho, 0.05, seed=40 + r)
        v = inputs.maxwell_boltzmann(N, T, seed=40 + r)
        out.append(inputs.Replica(N, rho, T, 40 + r, x, v, L))
    return out


def _single(rp, precision, **kw):
    return rbl.System(rp.x, rp.v, rp.L, T=rp.T, seed=rp.seed, precision=precision, **dict(SHARED, **kw))


@pytest.fixture(scope="module")
def reps():
    return _replicas()


@pytest.mark.parametrize("precision", [rbl.RBL_FP32, rbl.RBL_FP64])
def test_lists_batches_forces_match_single_contexts(reps, precision):
    ens = rbl.Ensemble(reps, precision=precision, **SHARED)
    F = ens.split(ens.forces())
    core, nc = ens.get_lists(0)
    shell, ns = ens.get_lists(1)
    batch, nb = ens.get_batch(5)
    core, nc, shell, ns = ens.split(core), ens.split(nc), ens.split(shell), ens.split(ns)
    batch, nb = ens.split(batch), ens.split(nb)
    obs = ens.observables()
    for r, rp in enumerate(reps):
        s = _single(rp, precision)
        assert np.array_equal(F[r], s.forces()), r
        c1, n1 = s.get_lists(0, cap=core[r].shape[1])
        s1, m1 = s.get_lists(1, cap=shell[r].shape[1])
        assert np.array_equal(nc[r], n1) and np.array_equal(core[r], c1), r
        assert np.array_equal(ns[r], m1) and np.array_equal(shell[r], s1), r
        b1, k1 = s.get_batch(5)
        assert np.array_equal(nb[r], k1) and np.array_equal(batch[r], b1), r
        o1 = s.observables()
        assert obs[r]["U_est"] == o1["U_est"] and obs[r]["W_est"] == o1["W_est"], r
        assert obs[r]["Ns_mean"] == o1["Ns_mean"] and obs[r]["Nc_max"] == o1["Nc_max"], r


def test_trajectories_and_rebuilds_match_single_contexts(reps):
    """60 BAOAB steps: each replica rebuilds on its own schedule."""
    ens = rbl.Ensemble(reps, precision=rbl.RBL_FP32, **SHARED)
    ens.step(60)
    x, v, step = ens.get_state()
    assert step == 60
    xs, vs = ens.split(x), ens.split(v)
    obs = ens.observables()
    nreb = [o["n_rebuild"] for o in obs]
    for r, rp in enumerate(reps):
        s = _single(rp, rbl.RBL_FP32)
        s.step(60)
        x1, v1, _ = s.get_state()
        assert np.array_equal(xs[r], x1) and np.array_equal(vs[r], v1), r
        assert nreb[r] == s.observables()["n_rebuild"], r
    assert len(set(nreb)) > 1, nreb  # the schedules differ between replicas


def test_exact_energy_and_rdf_per_replica(reps):
    ens = rbl.Ensemble(reps, precision=rbl.RBL_FP64, **SHARED)
    U, W = ens.exact_energy()
    h = ens.rdf(0.05, 69)  # bins below r_s (the top edge is the cutoff itself)
    for r, rp in enumerate(reps):
        lists = oracle.build_lists(rp.x, rp.L, SHARED["r_c"], SHARED["r_s"], SHARED["skin"], K=2, method="cells")
        _, ev = oracle.full_forces(rp.x, rp.L, SHARED["r_s"], lists)
        assert abs(U[r] - ev[0]) <= 1e-11 * abs(ev[0]), r
        assert abs(W[r] - ev[1]) <= 1e-11 * abs(ev[1]), r
        assert np.array_equal(h[r], oracle.rdf_counts(rp.x, rp.L, 0.05, 69)), r


def test_replica_forces_match_oracle(reps):
    ens = rbl.Ensemble(reps, precision=rbl.RBL_FP32, **SHARED)
    F = ens.split(ens.forces())
    for r in (0, 2):
        rp = reps[r]
        lists = oracle.build_lists(rp.x, rp.L, SHARED["r_c"], SHARED["r_s"], SHARED["skin"], K=2, method="cells")
        Fo, _, _, _ = oracle.rbl_forces(rp.x, rp.L, SHARED["r_c"], SHARED["r_s"], SHARED["skin"], SHARED["p"],
                                        rp.seed, 0, lists)
        Fo = oracle.subtract_mean(Fo)
        assert np.linalg.norm(F[r] - Fo) / np.linalg.norm(Fo) <= 1e-5, r


def test_ensemble_workload_matches_single_contexts():
    """The 256-replica ensemble (N log-uniform 500-20000, rho* 0.6-0.9, T* 1-2), 50
    steps under the graph: sampled replicas, including the smallest and the largest,
    equal standalone runs bit for bit, with the same rebuild counts."""
    reps = inputs.ensemble(256, seed=1)
    ens = rbl.Ensemble(reps, precision=rbl.RBL_FP32, **SHARED)
    ens.step(50)
    x, v, _ = ens.get_state()
    xs, vs = ens.split(x), ens.split(v)
    obs = ens.observables()
    sizes = [rp.N for rp in reps]
    pick = sorted({0, 17, 128, 255, int(np.argmin(sizes)), int(np.argmax(sizes))})
    for r in pick:
        s = _single(reps[r], rbl.RBL_FP32)
        s.step(50)
        x1, v1, _ = s.get_state()
        assert np.array_equal(xs[r], x1) and np.array_equal(vs[r], v1), r
        assert obs[r]["n_rebuild"] == s.observables()["n_rebuild"], r
    assert all(np.isfinite(o["T_kin"]) for o in obs)


@pytest.mark.parametrize("precision", [rbl.RBL_FP64, rbl.RBL_FP32])
def test_multi_chunk_replica_matches_single_context(precision):
    """A replica with more than one chunk of 256 sixty-four-thread groups (N = 40,000:
    3 chunks) beside small ones: its FP64 force sums (mean force) and energy sums go
    through the two-stage reduction and must equal a standalone context's bit for bit."""
    spec = [(900, 0.8, 1.2), (40000, 0.8, 1.5), (1500, 0.7, 1.0)]
    reps = []
    for r, (N, rho, T) in enumerate(spec):
        x, L = inputs.fcc(N, rho, 0.05, seed=70 + r)
        reps.append(rbl.Replica(x, inputs.maxwell_boltzmann(N, T, seed=70 + r), L, T, 70 + r))
    ens = rbl.Ensemble(reps, precision=precision, **SHARED)
    ens.step(12)
    xs = ens.split(ens.get_state()[0])
    F = ens.split(ens.forces())
    obs = ens.observables()
    for r, rp in enumerate(reps):
        s = _single(rp, precision)
        s.step(12)
        assert np.array_equal(xs[r], s.get_state()[0]), r
        assert np.array_equal(F[r], s.forces()), r
        o = s.observables()
        assert obs[r]["U_est"] == o["U_est"] and obs[r]["W_est"] == o["W_est"], r
        assert obs[r]["K"] == o["K"], r
