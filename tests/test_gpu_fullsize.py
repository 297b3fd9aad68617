"""Parity at the full size of the throughput workload: LJ fluid N = 2^20 (FCC
64^3 x 4), rho* = 0.8, T* = 1.5, r_c = 1.5, r_s = 3.5, skin 0.3, p = 10, FP32,
Langevin gamma = 1, dt = 0.005, K = 2 -- the launch configuration bench.py times.

After 20 steps on the graph path, sampled particles are checked one by one against
the oracle (which tests every other particle for each of them): core and shell
rows and batches bit-exact, un-subtracted forces within the FP32 bar.  Properties
that hold at any size are checked on every particle: the corrected force sums to
exactly zero and differs from the raw force by the fixed-point mean."""
import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

N = 1 << 20
RC, RS, SKIN, P, DT, T, GAMMA, SEED = 1.5, 3.5, 0.3, 10, 0.005, 1.5, 1.0, 1
M = 256  # sampled particles


@pytest.fixture(scope="module")
def run():
    x, L = inputs.fcc(N, 0.8, 0.01, seed=SEED)
    v = inputs.maxwell_boltzmann(N, T, seed=SEED)
    common = dict(T=T, gamma=GAMMA, seed=SEED, precision=rbl.RBL_FP32, cells_per_cutoff=2)
    s = rbl.System(x, v, L, RC, RS, SKIN, P, DT, **common)
    s.step(20)
    x20, v20, step = s.get_state()
    s.build_lists()  # lists of the current positions, as the oracle builds them
    F_sub = s.forces()
    del s
    torch.cuda.empty_cache()
    raw = rbl.System(x20, v20, L, RC, RS, SKIN, P, DT, subtract_net_force=False, step=step, **common)
    F_raw = raw.forces()
    idx = np.sort(np.random.default_rng(5).choice(N, M, replace=False))
    return dict(x=x20, L=L, step=step, F_sub=F_sub, F_raw=F_raw, sys=raw, idx=idx)


def test_sampled_rows_batches_forces(run):
    s, idx, step = run["sys"], run["idx"], run["step"]
    smp = oracle.sample(run["x"], run["L"], RC, RS, SKIN, P, SEED, step, idx, K=2)
    core, nc = s.get_rows(0, idx)
    shell, ns = s.get_rows(1, idx)
    assert np.array_equal(nc, smp.n_core) and np.array_equal(ns, smp.n_shell)
    for k in range(M):
        assert np.array_equal(core[k, : nc[k]], smp.row("core", k)), k
        assert np.array_equal(shell[k, : ns[k]], smp.row("shell", k)), k
    batch, nb = s.get_batch(step)
    assert np.array_equal(nb[idx], smp.n_batch)
    for k, i in enumerate(idx):
        assert np.array_equal(batch[i, : nb[i]], smp.batch[k, : smp.n_batch[k]]), k
    F = run["F_raw"][idx]
    # FP32 bar: relative global norm over the sample
    assert np.linalg.norm(F - smp.F) / np.linalg.norm(smp.F) <= 1e-5


def test_net_force_properties(run):
    """The net force is removed exactly in fixed point (units of 2^-24): the corrected
    forces sum to zero exactly, and each differs from the raw force by the mean
    rounded down or up to the fixed-point grid (the remainder spread over the
    particles of lowest tag)."""
    F_sub, F_raw = run["F_sub"], run["F_raw"]
    unit = 2.0 ** -24
    assert np.all(F_sub.sum(axis=0) == 0.0)
    d = F_raw - F_sub
    lo = np.floor(F_raw.sum(axis=0) / unit / N) * unit
    assert np.all((d == lo) | (d == lo + unit))
    assert np.all(np.abs(d.mean(axis=0) - F_raw.mean(axis=0)) <= 1e-12)
