"""Degenerate inputs on the GPU against the oracle, through the C ABI (Sec. 2, Algorithm 1).

- the smallest system the library takes, N = 2: one pair inside the core, inside the
  shell, in the skin band beyond r_s, beyond r_s + skin (no neighbour at all: empty
  rows, no batch, a force of exactly zero), and a core pair through the periodic face;
- two small clusters in a large box, one of them split by the box corner, so that
  nearly every cell is empty and the cell stencils wrap (the local density is passed
  as rho_cap, which sizes the candidate tables);
- particles exactly on the box faces: coordinates 0 and the largest double below L,
  whose fixed-point image rounds to 2^32, i.e. 0 (R10's image of a periodic box);
- the largest batch, p = 128, below every shell size of a dense fluid;
- all of these as the replicas of one ensemble, against each run on its own.

Each case: core, shell and full rows and the batches at two steps bit-exact; forces
within 1e-12 (FP64 path) and 1e-5 (FP32 path) of the oracle's in relative global norm
(exactly zero where the oracle's are); a 30-step FP64 velocity-Verlet trajectory within
1e-9 of the oracle's, with the same number of list builds.
"""
import numpy as np
import pytest

import oracle
from degenerate_cases import CASES
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

RC, RS, SKIN, P, DT = 1.5, 3.5, 0.3, 10, 0.005


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    x, v, L, kw = CASES[request.param]()
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=2, method="cells")
    return request.param, x, v, L, kw, lists


def _system(x, v, L, kw, **more):
    args = dict(T=1.0, gamma=0.0, seed=3, cells_per_cutoff=2)
    args.update(kw)
    args.update(more)
    return rbl.System(x, v, L, RC, RS, SKIN, P, DT, **args)


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_lists_bit_exact(case):
    name, x, v, L, kw, lists = case
    s = _system(x, v, L, kw)
    for kind, row in ((0, "core"), (1, "shell")):
        rows, counts = s.get_lists(kind)
        assert np.array_equal(counts, getattr(lists, "n_" + row)), (name, row)
        for i in range(len(x)):
            assert np.array_equal(rows[i, : counts[i]], lists.row(row, i)), (name, row, i)
    f = _system(x, v, L, kw, full_list=True)
    rows, counts = f.get_lists(1)
    assert np.array_equal(counts, lists.n_full), name
    for i in range(len(x)):
        assert np.array_equal(rows[i, : counts[i]], lists.row("full", i)), (name, i)
    if name == "pair_beyond":
        assert counts.sum() == 0 and lists.n_core.sum() == 0


@pytest.mark.parametrize("step", [0, 5])
def test_batches_bit_exact(case, step):
    name, x, v, L, kw, lists = case
    s = _system(x, v, L, kw)
    batch, counts = s.get_batch(step)
    _, _, ob, obn = oracle.rbl_forces(x, L, RC, RS, SKIN, P, 3, step, lists, want_batch=True)
    assert np.array_equal(counts, obn), name
    for i in range(len(x)):
        assert np.array_equal(batch[i, : counts[i]], ob[i, : obn[i]]), (name, i)


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_forces(case, precision, tol):
    name, x, v, L, kw, lists = case
    s = _system(x, v, L, kw, precision=precision)
    F = s.forces()
    Fo, _, _, _ = oracle.rbl_forces(x, L, RC, RS, SKIN, P, 3, 0, lists)
    Fo = oracle.subtract_mean(Fo)
    norm = np.linalg.norm(Fo)
    if norm == 0.0:
        assert not F.any(), name
    else:
        assert np.linalg.norm(F - Fo) <= tol * norm, name


def test_trajectory_fp64(case):
    name, x, v, L, kw, lists = case
    n = 30
    s = _system(x, v, L, kw, precision=rbl.RBL_FP64)
    s.step(n)
    xg, vg, step = s.get_state()
    obs = s.observables()
    xo, vo, _, stats = oracle.run(x, v, L, RC, RS, SKIN, P, DT, 1.0, 0.0, 3, n)
    assert step == n
    assert obs["n_rebuild"] == int(stats[2]), name
    assert np.abs(_min_image(xg - xo, L)).max() < 1e-9, name
    assert np.abs(vg - vo).max() < 1e-8, name
    assert (xg >= 0.0).all() and (xg < L).all(), name


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_largest_batch(precision, tol):
    """p = 128, the largest batch, below the shell sizes of a dense fluid (N_s ~ 177):
    batches bit-exact at two steps, forces at the bars."""
    p = 128
    x, L = inputs.fcc(2000, 0.8, 0.05, seed=13)
    v = inputs.maxwell_boltzmann(2000, 1.5, seed=13)
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=2, method="cells")
    assert lists.n_shell.min() > p
    s = rbl.System(x, v, L, RC, RS, SKIN, p, DT, T=1.5, seed=13, precision=precision)
    for step in (0, 7):
        batch, counts = s.get_batch(step)
        _, _, ob, obn = oracle.rbl_forces(x, L, RC, RS, SKIN, p, 13, step, lists, want_batch=True)
        assert np.array_equal(counts, obn) and (counts == p).all()
        for i in range(len(x)):
            assert np.array_equal(batch[i], ob[i]), (step, i)
    F = s.forces()
    Fo, _, _, _ = oracle.rbl_forces(x, L, RC, RS, SKIN, p, 13, 0, lists)
    Fo = oracle.subtract_mean(Fo)
    assert np.linalg.norm(F - Fo) <= tol * np.linalg.norm(Fo)


def test_degenerate_replicas_in_one_ensemble():
    """Every case above as one replica of an ensemble (uneven sizes from 2 to 500,
    boxes from 8.5 to 25, the local density passed as rho_cap for all): forces and 30
    FP32 steps bit-identical to each case run as a context of its own."""
    reps = []
    for k, name in enumerate(sorted(CASES)):
        x, v, L, _ = CASES[name]()
        reps.append(inputs.Replica(len(x), 0.0, 1.0, 3 + k, x, v, L))
    kw = dict(r_c=RC, r_s=RS, skin=SKIN, p=P, dt=DT, gamma=0.0, rho_cap=1.0)
    ens = rbl.Ensemble(reps, **kw)
    F = ens.split(ens.forces())
    singles = [rbl.System(rp.x, rp.v, rp.L, T=rp.T, seed=rp.seed, **kw) for rp in reps]
    for r, s in enumerate(singles):
        assert np.array_equal(F[r], s.forces()), r
    ens.step(30)
    x, v, _ = ens.get_state()
    xs, vs = ens.split(x), ens.split(v)
    nreb = [o["n_rebuild"] for o in ens.observables()]
    for r, s in enumerate(singles):
        s.step(30)
        x1, v1, _ = s.get_state()
        assert np.array_equal(xs[r], x1) and np.array_equal(vs[r], v1), r
        assert nreb[r] == s.observables()["n_rebuild"], r
