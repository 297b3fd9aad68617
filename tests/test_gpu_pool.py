"""The paper's own sampling pool on the GPU (RBL_SAMPLE_STENCIL) against the oracle:
core rows and batches bit-exact, forces within the FP64 / FP32 bars, unsampled
energy and g(r) counts, and pool sizes, on a box with fewer than 2m + 1 cells per
axis (the pool is everyone) and on boxes where the stencil is a proper sub-box."""
import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

CASES = {
    "n1000_whole_box": dict(N=1000, rho=0.8, rc=1.5, p=10, seed=1),
    "n4000": dict(N=4000, rho=0.8, rc=1.5, p=10, seed=2),
    "n5001_rc1.2_p20": dict(N=5001, rho=0.85, rc=1.2, p=20, seed=3),
}
RS, SKIN = 3.5, 0.3


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = CASES[request.param]
    x, L = inputs.fcc(c["N"], c["rho"], 0.2, seed=c["seed"])
    v = inputs.maxwell_boltzmann(c["N"], 1.5, seed=c["seed"])
    return c, x, v, L, oracle.build_pool(x, L, c["rc"], RS, SKIN)


def _system(c, x, v, L, **kw):
    return rbl.System(x, v, L, c["rc"], RS, SKIN, c["p"], 0.005, T=1.5, gamma=1.0, seed=c["seed"],
                      sampling=rbl.RBL_SAMPLE_STENCIL, **kw)


def test_core_rows_and_pool_sizes(case):
    c, x, v, L, pl = case
    s = _system(c, x, v, L)
    rows, counts = s.get_lists(0)
    assert np.array_equal(counts, pl.n_core)
    for i in range(c["N"]):
        assert np.array_equal(rows[i, : counts[i]], pl.row("core", i)), i
    assert s.observables()["Ns_mean"] == pl.n_shell.mean()
    with pytest.raises(rbl.RblError):
        s.get_lists(1)  # no shell rows in this mode


@pytest.mark.parametrize("step", [0, 1, 977])
def test_batches_bit_exact(case, step):
    c, x, v, L, pl = case
    s = _system(c, x, v, L)
    batch, counts = s.get_batch(step)
    _, _, ob, obn = oracle.rbl_forces(x, L, c["rc"], RS, SKIN, c["p"], c["seed"], step, pl, want_batch=True)
    assert np.array_equal(counts, obn)
    for i in range(c["N"]):
        assert np.array_equal(batch[i, : counts[i]], ob[i, : obn[i]]), i


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_forces(case, precision, tol):
    c, x, v, L, pl = case
    s = _system(c, x, v, L, precision=precision)
    F = s.forces()
    Fo, ev, _, _ = oracle.rbl_forces(x, L, c["rc"], RS, SKIN, c["p"], c["seed"], 0, pl)
    Fo = oracle.subtract_mean(Fo)
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) <= tol
    obs = s.observables()
    assert abs(obs["U_est"] - ev[0]) <= 10 * tol * abs(ev[0])


def test_exact_energy_and_rdf(case):
    c, x, v, L, pl = case
    s = _system(c, x, v, L, precision=rbl.RBL_FP64)
    U, W = s.exact_energy()
    _, evb = oracle.brute_forces(x, L, RS)
    assert abs(U - evb[0]) <= 1e-11 * abs(evb[0]) and abs(W - evb[1]) <= 1e-11 * abs(evb[1])
    nb = int(RS / 0.05) - 1
    assert np.array_equal(s.rdf(0.05, nb), oracle.rdf_counts(x, L, 0.05, nb))


def test_steps_run(case):
    c, x, v, L, pl = case
    # a start that steps (the parity cases' jitter puts pairs near 0.5 sigma)
    x, L = inputs.fcc(c["N"], c["rho"], 0.05, seed=c["seed"])
    s = _system(c, x, v, L)
    s.step(40)
    o = s.observables()
    assert np.isfinite(o["T_kin"]) and o["n_rebuild"] >= 1
