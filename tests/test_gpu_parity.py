"""GPU <-> oracle parity through the C ABI (librbl), on seeded LJ-fluid inputs.

Bars (each stated where it is asserted):
- cell/list membership and canonical row order: bit-exact;
- sampled batches: bit-exact (same Philox stream, same Floyd draws);
- forces: relative global norm ||F_gpu - F_orc|| / ||F_orc|| <= 1e-12 (FP64 path)
  and <= 1e-5 (FP32 path);
- energy and virial sums (RBL estimates, exact sums): |X_gpu - X_orc| <= tol * S, S the
  magnitude of the summed pair terms (1/2 sum |term|), tol as for the forces;
- p >= max N_s reproduces the full-list force (FP32: up to summation order).
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

CASES = {
    # the N=1000 parity workload: rho* = 0.8, FCC + 0.01 jitter, r_c 1.5, r_s 3.5, skin 0.3, p 10
    "n1000": dict(N=1000, rho=0.8, jitter=0.01, rc=1.5, rs=3.5, skin=0.3, p=10, K=2, seed=1),
    # 2 cells per axis (stencil de-duplicated), disordered
    "n1000_K1": dict(N=1000, rho=0.8, jitter=0.2, rc=1.5, rs=3.5, skin=0.3, p=10, K=1, seed=2),
    # 4 < 2K+1 cells per axis at K = 2
    "n500_small_box": dict(N=500, rho=0.8, jitter=0.3, rc=1.5, rs=3.5, skin=0.3, p=10, K=2, seed=3),
    # ragged tail (N not a multiple of the block), r_c = 1.2, dense
    "n4001_rc1.2": dict(N=4001, rho=0.8442, jitter=0.25, rc=1.2, rs=3.5, skin=0.3, p=5, K=2, seed=4),
    # r_c = 2.0, p = 20, K = 3 (7^3 stencil)
    "n3000_rc2_K3": dict(N=3000, rho=0.7, jitter=0.3, rc=2.0, rs=3.5, skin=0.3, p=20, K=3, seed=5),
    # p = 1
    "n2000_p1": dict(N=2000, rho=0.8, jitter=0.3, rc=1.5, rs=3.5, skin=0.3, p=1, K=2, seed=6),
    # the paper's Table 1 system: dilute, r_s = 6, r_c = 2, p = 100 (general batch path)
    "n2000_rho0.2_rs6_p100": dict(N=2000, rho=0.2, jitter=0.3, rc=2.0, rs=6.0, skin=0.3, p=100, K=2, seed=7),
    # non-cubic boxes: a different fixed-point unit per axis in the pair rule and the
    # list build's bounding-box cull; 5 cells along x (fewer than 2K + 3), and at K = 3
    # 6 (fewer than 2K + 1: the stencil takes every x cell once)
    "n2000_aniso": dict(N=2000, rho=0.8, jitter=0.15, rc=1.5, rs=3.5, skin=0.3, p=10, K=2, seed=8,
                        L=(10.0, 12.5, 20.0)),
    "n1500_aniso_K3": dict(N=1500, rho=0.8, jitter=0.15, rc=1.5, rs=3.5, skin=0.3, p=10, K=3, seed=9,
                           L=(8.2, 11.0, 20.8)),
    # K = 1 in the first non-cubic box: 2 x 3 x 5 cells, every x cell once
    "n2000_aniso_K1": dict(N=2000, rho=0.8, jitter=0.15, rc=1.5, rs=3.5, skin=0.3, p=10, K=1, seed=10,
                           L=(10.0, 12.5, 20.0)),
}


def _state(c):
    x, L = inputs.fcc(c["N"], c["rho"], c["jitter"], seed=c["seed"], L=c.get("L"))
    v = inputs.maxwell_boltzmann(c["N"], 1.5, seed=c["seed"])
    return x, v, L


def _system(c, x, v, L, **kw):
    args = dict(r_c=c["rc"], r_s=c["rs"], skin=c["skin"], p=c["p"], dt=0.005, T=1.5, gamma=0.0, seed=c["seed"],
                cells_per_cutoff=c["K"])
    args.update(kw)
    return rbl.System(x, v, L, **args)


def _relnorm(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pair_uw(x, L, I, J):
    """LJ energy and virial terms 4(r^-12 - r^-6), 24(2 r^-12 - r^-6) of pairs (I, J)
    and their r^2 (minimum image, FP64)."""
    d = x[J] - x[I]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(1)
    ir6 = r2**-3
    return 4 * (ir6 * ir6 - ir6), 24 * (2 * ir6 * ir6 - ir6), r2


def _rows(lists, name, N):
    I = np.concatenate([np.full(len(lists.row(name, i)), i) for i in range(N)]).astype(np.int64)
    J = np.concatenate([lists.row(name, i) for i in range(N)]).astype(np.int64)
    return I, J


def _scale_exact(x, L, rs, lists):
    """1/2 sum over pairs r < r_s of |u| and of |w|: the magnitude of the terms the
    exact energy and virial add up, the scale of a rounded sum's error."""
    I, J = _rows(lists, "full", len(x))
    u, w, r2 = _pair_uw(x, L, I, J)
    m = r2 < rs * rs
    return 0.5 * np.abs(u[m]).sum(), 0.5 * np.abs(w[m]).sum()


def _scale_estimate(x, L, rc, rs, p, lists, batch, nb):
    """The same magnitude for the RBL estimates: core pairs r < r_c, and the batch
    pairs r_c <= r < r_s times s_i = N_s / p."""
    N = len(x)
    I, J = _rows(lists, "core", N)
    u, w, r2 = _pair_uw(x, L, I, J)
    m = r2 < rc * rc
    su, sw = np.abs(u[m]).sum(), np.abs(w[m]).sum()
    ns = lists.n_shell
    scale = np.where(ns > p, ns / p, 1.0)
    Ib = np.concatenate([np.full(nb[i], i) for i in range(N)]).astype(np.int64)
    Jb = np.concatenate([batch[i, : nb[i]] for i in range(N)]).astype(np.int64)
    u, w, r2 = _pair_uw(x, L, Ib, Jb)
    m = (r2 >= rc * rc) & (r2 < rs * rs)
    su += (scale[Ib[m]] * np.abs(u[m])).sum()
    sw += (scale[Ib[m]] * np.abs(w[m])).sum()
    return 0.5 * su, 0.5 * sw


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = CASES[request.param]
    x, v, L = _state(c)
    lists = oracle.build_lists(x, L, c["rc"], c["rs"], c["skin"], K=c["K"], method="cells")
    return c, x, v, L, lists


def test_lists_bit_exact(case):
    c, x, v, L, lists = case
    s = _system(c, x, v, L)
    for kind, name in ((0, "core"), (1, "shell")):
        rows, counts = s.get_lists(kind)
        assert np.array_equal(counts, getattr(lists, "n_" + name)), name
        for i in range(c["N"]):
            assert np.array_equal(rows[i, : counts[i]], lists.row(name, i)), (name, i)


def test_full_list_bit_exact(case):
    c, x, v, L, lists = case
    s = _system(c, x, v, L, full_list=True)
    rows, counts = s.get_lists(1)
    assert np.array_equal(counts, lists.n_full)
    for i in range(c["N"]):
        assert np.array_equal(rows[i, : counts[i]], lists.row("full", i))


@pytest.mark.parametrize("step", [0, 1, 977])
def test_batches_bit_exact(case, step):
    c, x, v, L, lists = case
    s = _system(c, x, v, L)
    batch, counts = s.get_batch(step)
    _, _, ob, obn = oracle.rbl_forces(x, L, c["rc"], c["rs"], c["skin"], c["p"], c["seed"], step, lists,
                                      want_batch=True)
    assert np.array_equal(counts, obn)
    for i in range(c["N"]):
        assert np.array_equal(batch[i, : counts[i]], ob[i, : obn[i]]), i


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_forces_and_estimates(case, precision, tol):
    c, x, v, L, lists = case
    s = _system(c, x, v, L, precision=precision)
    F = s.forces()
    Fo, ev, ob, obn = oracle.rbl_forces(x, L, c["rc"], c["rs"], c["skin"], c["p"], c["seed"], 0, lists,
                                        want_batch=True)
    Fo = oracle.subtract_mean(Fo)
    assert _relnorm(F, Fo) <= tol
    obs = s.observables()
    # the estimates are sums of pair terms of both signs (the virial nearly cancels:
    # W ~ 500 out of terms summing to ~10^4 in magnitude), so their bar is the
    # tolerance times the magnitude of the summed terms, as for any rounded sum
    su, sw = _scale_estimate(x, L, c["rc"], c["rs"], c["p"], lists, ob, obn)
    assert abs(obs["U_est"] - ev[0]) <= tol * su
    assert abs(obs["W_est"] - ev[1]) <= tol * sw


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_full_list_forces(case, precision, tol):
    c, x, v, L, lists = case
    s = _system(c, x, v, L, precision=precision, full_list=True)
    F = s.forces()
    Fo, ev = oracle.full_forces(x, L, c["rs"], lists)
    assert _relnorm(F, oracle.subtract_mean(Fo)) <= tol
    obs = s.observables()
    su, sw = _scale_exact(x, L, c["rs"], lists)
    assert abs(obs["U_est"] - ev[0]) <= tol * su
    assert abs(obs["W_est"] - ev[1]) <= tol * sw


@pytest.mark.parametrize("full", [False, True])
@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_exact_energy(case, precision, tol, full):
    """The unsampled energy and virial (every pair with r < r_s, from the core and
    shell lists, or the full list) equal the oracle's full-list sums; the call leaves
    the force state and the RBL estimates untouched."""
    c, x, v, L, lists = case
    s = _system(c, x, v, L, precision=precision, full_list=full)
    F0 = s.forces()
    est0 = s.observables()
    U, W = s.exact_energy()
    _, ev = oracle.full_forces(x, L, c["rs"], lists)
    # per-pair terms (binary32 on the FP32 path) summed per particle (~200 terms):
    # the bar is the tolerance times the magnitude of the summed terms
    su, sw = _scale_exact(x, L, c["rs"], lists)
    assert abs(U - ev[0]) <= tol * su
    assert abs(W - ev[1]) <= tol * sw
    est1 = s.observables()
    assert est1["U_est"] == est0["U_est"] and est1["W_est"] == est0["W_est"]
    assert np.array_equal(s.forces(), F0)


@pytest.mark.parametrize("N,rho,seed", [(1000, 0.8, 11), (2501, 0.9, 12), (800, 0.6, 13)])
def test_fp32_large_batch_is_full_list(N, rho, seed):
    """p >= max N_s takes every shell neighbour with scale 1, so the RBL force equals
    the full-list force up to binary32 summation order (core and shell summed
    separately vs one full row); both match the oracle's cutoff force.  The total
    force of the full list (no mean subtraction) is zero up to rounding, and its
    fixed-point representation is exact: every force is an integer multiple of
    2^-24.  r_s is small here so that whole shell rows fit in one batch (p <= 64)."""
    c = dict(N=N, rho=rho, jitter=0.3, rc=1.5, rs=2.2, skin=0.1, p=64, K=2, seed=seed)
    x, v, L = _state(c)
    lists = oracle.build_lists(x, L, c["rc"], c["rs"], c["skin"], K=2)
    assert lists.n_shell.max() <= 64
    a = _system(c, x, v, L, subtract_net_force=False).forces()
    b = _system(c, x, v, L, full_list=True, subtract_net_force=False).forces()
    assert _relnorm(a, b) <= 1e-6
    q = np.rint(b * 2.0**24).astype(np.int64)
    assert np.array_equal(q.astype(np.float64) / 2.0**24, b)
    rms = np.sqrt((b * b).sum() / N)
    assert np.all(np.abs(q.sum(0)) * 2.0**-24 <= 1e-6 * rms * N)
    Fo, _ = oracle.full_forces(x, L, c["rs"], lists)
    assert _relnorm(a, Fo) <= 1e-5 and _relnorm(b, Fo) <= 1e-5


def test_rdf_counts_exact(case):
    c, x, v, L, lists = case
    dr, nb = 0.02, int(c["rs"] / 0.02) - 1
    for full in (False, True):
        s = _system(c, x, v, L, full_list=full)
        h = s.rdf(dr, nb)
        assert np.array_equal(h, oracle.rdf_counts(x, L, dr, nb))


def test_density_profile_exact(case):
    c, x, v, L, lists = case
    s = _system(c, x, v, L)
    for axis, nb in ((0, 13), (2, 50)):
        assert np.array_equal(s.density_profile(axis, nb), oracle.density_profile(x, L, axis, nb))
