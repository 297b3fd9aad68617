"""The LJ + Ewald real-space pair (q_i q_j erfc(alpha r) / r added to the LJ pair,
the RBL's extension to the short-range part of the Coulomb interaction; Sec. 2
closing remarks, Sec. 4) through the C ABI, against the oracle on the same seeded
charged LJ fluid (FCC start, neutral random +-1 charges).

Bars: forces ||F_gpu - F_orc|| / ||F_orc|| <= 1e-12 (FP64 path) and <= 1e-5 (FP32
path: the kernel's own erfc fit is within about 1e-7); exact energy 1e-11 (FP64); trajectories
as in the LJ dynamics test; ensembles and reloads bit-exact.
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

EW = dict(potential=rbl.RBL_POT_LJ_EWALD)
CASES = {
    # the charged-fluid parity workload: rho* = 0.8, r_c 1.5, r_s 3.5, p 10, alpha 1 (erfc(alpha r_s) = 7e-7)
    "n1000": dict(N=1000, rho=0.8, jitter=0.15, rc=1.5, rs=3.5, skin=0.3, p=10, K=2, alpha=1.0, seed=1),
    # ragged tail, r_c = 1.2, p = 5, weaker screening
    "n4001_rc1.2_a0.8": dict(N=4001, rho=0.8442, jitter=0.25, rc=1.2, rs=3.5, skin=0.3, p=5, K=2, alpha=0.8,
                             seed=4),
    # r_c = 2, p = 20, K = 3
    "n3000_rc2_K3_a1.2_q2": dict(N=3000, rho=0.7, jitter=0.3, rc=2.0, rs=3.5, skin=0.3, p=20, K=3, alpha=1.2,
                                 seed=5, q=2.0),
    # general batch path (p = 100)
    "n2000_p100_q1.5": dict(N=2000, rho=0.5, jitter=0.3, rc=1.5, rs=4.0, skin=0.3, p=100, K=2, alpha=0.9, seed=7,
                            q=1.5),
}


def _state(c):
    x, L = inputs.fcc(c["N"], c["rho"], c["jitter"], seed=c["seed"])
    v = inputs.maxwell_boltzmann(c["N"], 1.5, seed=c["seed"])
    q = inputs.charges(c["N"], c.get("q", 1.0), seed=c["seed"])
    return x, v, L, q


def _system(c, x, v, L, q, **kw):
    args = dict(r_c=c["rc"], r_s=c["rs"], skin=c["skin"], p=c["p"], dt=0.005, T=1.5, gamma=0.0, seed=c["seed"],
                cells_per_cutoff=c["K"], alpha=c["alpha"], charges=q, **EW)
    args.update(kw)
    return rbl.System(x, v, L, **args)


def _relnorm(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pair_uw(x, L, q, alpha, I, J):
    """Pair energy LJ + q_i q_j erfc(alpha r)/r and virial r . f of pairs (I, J), and r^2."""
    from scipy.special import erfc

    d = x[J] - x[I]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(1)
    r = np.sqrt(r2)
    ir6 = r2**-3
    qq = q[I] * q[J]
    ec = erfc(alpha * r) / r
    u = 4 * (ir6 * ir6 - ir6) + qq * ec
    w = 24 * (2 * ir6 * ir6 - ir6) + qq * (ec + 2 * alpha / np.sqrt(np.pi) * np.exp(-alpha * alpha * r2))
    return u, w, r2


def _scale_estimate(c, x, L, q, lists, batch, nb):
    """1/2 the magnitude of the summed terms of the RBL energy and virial estimates:
    core pairs r < r_c, batch pairs r_c <= r < r_s times s_i = N_s / p (the scale of a
    rounded sum's error; the virial nearly cancels)."""
    N, rc, rs, p = len(x), c["rc"], c["rs"], c["p"]
    I = np.concatenate([np.full(len(lists.row("core", i)), i) for i in range(N)]).astype(np.int64)
    J = np.concatenate([lists.row("core", i) for i in range(N)]).astype(np.int64)
    u, w, r2 = _pair_uw(x, L, q, c["alpha"], I, J)
    m = r2 < rc * rc
    su, sw = np.abs(u[m]).sum(), np.abs(w[m]).sum()
    ns = lists.n_shell
    scale = np.where(ns > p, ns / p, 1.0)
    Ib = np.concatenate([np.full(nb[i], i) for i in range(N)]).astype(np.int64)
    Jb = np.concatenate([batch[i, : nb[i]] for i in range(N)]).astype(np.int64)
    u, w, r2 = _pair_uw(x, L, q, c["alpha"], Ib, Jb)
    m = (r2 >= rc * rc) & (r2 < rs * rs)
    su += (scale[Ib[m]] * np.abs(u[m])).sum()
    sw += (scale[Ib[m]] * np.abs(w[m])).sum()
    return 0.5 * su, 0.5 * sw


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = CASES[request.param]
    x, v, L, q = _state(c)
    lists = oracle.build_lists(x, L, c["rc"], c["rs"], c["skin"], K=c["K"], method="cells")
    return c, x, v, L, q, lists


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_rbl_forces_and_estimates(case, precision, tol):
    c, x, v, L, q, lists = case
    s = _system(c, x, v, L, q, precision=precision)
    F = s.forces()
    Fo, ev, ob, obn = oracle.rbl_forces(x, L, c["rc"], c["rs"], c["skin"], c["p"], c["seed"], 0, lists, q=q,
                                        alpha=c["alpha"], want_batch=True)
    Fo = oracle.subtract_mean(Fo)
    assert _relnorm(F, Fo) <= tol
    obs = s.observables()
    # the estimates' bar: tol times the magnitude of the summed pair terms
    su, sw = _scale_estimate(c, x, L, q, lists, ob, obn)
    assert abs(obs["U_est"] - ev[0]) <= tol * su
    assert abs(obs["W_est"] - ev[1]) <= tol * sw


@pytest.mark.parametrize("full_list", [False, True])
@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-10), (rbl.RBL_FP32, 1e-5)])
def test_coulomb_part_alone(precision, tol, full_list):
    """The charged term by itself, on a nearly perfect lattice where the LJ pair forces
    are small and the Coulomb forces of the random charges are a large part of the
    total (most of it with the full list), so the total's rounding cannot hide an
    error in the Ewald term.  Zero charges give the LJ kernel's result bit for bit
    (same batch), so the difference is the charged term."""
    rc, rs, skin, p, seed, alpha = 1.5, 3.5, 0.3, 10, 11, 1.0
    x, L = inputs.fcc(2048, 0.8, 0.005, seed=seed)
    q = inputs.charges(2048, 1.0, seed=seed)
    s = rbl.System(x, None, L, rc, rs, skin, p, 0.005, seed=seed, precision=precision, alpha=alpha, charges=q,
                   full_list=full_list, **EW)
    F = s.forces()
    s.set_charges(np.zeros_like(q))
    dF = F - s.forces()
    lists = oracle.build_lists(x, L, rc, rs, skin, K=2)
    if full_list:
        Fo, _ = oracle.full_forces(x, L, rs, lists, q=q, alpha=alpha)
        F0, _ = oracle.full_forces(x, L, rs, lists)
    else:
        Fo, _, _, _ = oracle.rbl_forces(x, L, rc, rs, skin, p, seed, 0, lists, q=q, alpha=alpha)
        F0, _, _, _ = oracle.rbl_forces(x, L, rc, rs, skin, p, seed, 0, lists)
    dFo = oracle.subtract_mean(Fo) - oracle.subtract_mean(F0)
    assert np.linalg.norm(dFo) > 0.1 * np.linalg.norm(Fo)
    assert _relnorm(dF, dFo) <= tol


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_full_list_and_exact_energy(case, precision, tol):
    c, x, v, L, q, lists = case
    s = _system(c, x, v, L, q, precision=precision, full_list=True)
    F = s.forces()
    Fo, ev = oracle.full_forces(x, L, c["rs"], lists, q=q, alpha=c["alpha"])
    assert _relnorm(F, oracle.subtract_mean(Fo)) <= tol
    if precision == rbl.RBL_FP64:
        s2 = _system(c, x, v, L, q, precision=precision)
        U, W = s2.exact_energy()
        _, evb = oracle.brute_forces(x, L, c["rs"], q=q, alpha=c["alpha"])
        assert abs(U - evb[0]) <= 1e-11 * abs(evb[0]) and abs(W - evb[1]) <= 1e-11 * abs(evb[1])


@pytest.mark.parametrize("precision,tol", [(rbl.RBL_FP64, 1e-12), (rbl.RBL_FP32, 1e-5)])
def test_stencil_pool_forces(precision, tol):
    c = CASES["n1000"]
    x, v, L, q = _state(c)
    pl = oracle.build_pool(x, L, c["rc"], c["rs"], c["skin"])
    s = _system(c, x, v, L, q, precision=precision, sampling=rbl.RBL_SAMPLE_STENCIL)
    F = s.forces()
    Fo, _, _, _ = oracle.rbl_forces(x, L, c["rc"], c["rs"], c["skin"], c["p"], c["seed"], 0, pl, q=q,
                                    alpha=c["alpha"])
    assert _relnorm(F, oracle.subtract_mean(Fo)) <= tol


def test_nve_trajectory_fp64_charges_follow_particles():
    """40 velocity-Verlet steps with list rebuilds (each rebuild re-sorts the particles
    and their charges into cell order) against the oracle's trajectory."""
    c = CASES["n1000"]
    x, v, L, q = _state(c)
    n = 40
    s = _system(c, x, v, L, q, precision=rbl.RBL_FP64)
    s.step(n)
    xg, vg, step = s.get_state()
    obs = s.observables()
    xo, vo, _, stats = oracle.run(x, v, L, c["rc"], c["rs"], c["skin"], c["p"], 0.005, 1.5, 0.0, c["seed"], n,
                                  q=q, alpha=c["alpha"])
    assert step == n
    assert obs["n_rebuild"] == int(stats[2]) and stats[2] > 1
    d = xg - xo
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9
    assert np.abs(vg - vo).max() < 1e-8
    assert abs(obs["U_est"] - stats[0]) < 1e-8 * abs(stats[0])


def test_reload_and_recharge():
    """Charges stay with their tags across set_state (positions reloaded in tag order)
    and set_charges after rebuilds; forces after a reload equal those before bit for
    bit (FP32)."""
    c = CASES["n1000"]
    x, v, L, q = _state(c)
    s = _system(c, x, v, L, q, gamma=1.0)
    s.step(60)
    assert s.observables()["n_rebuild"] > 1
    x1, v1, step = s.get_state()
    s.build_lists()  # lists of the current positions, as a reload builds them
    F1 = s.forces()
    s.set_state(x1, v1, step)
    assert np.array_equal(s.forces(), F1)
    s.set_charges(q)  # same charges, set while the particles are in cell order
    assert np.array_equal(s.forces(), F1)
    lists = oracle.build_lists(x1, L, c["rc"], c["rs"], c["skin"], K=c["K"])
    Fo, _, _, _ = oracle.rbl_forces(x1, L, c["rc"], c["rs"], c["skin"], c["p"], c["seed"], step, lists, q=q,
                                    alpha=c["alpha"])
    assert _relnorm(F1, oracle.subtract_mean(Fo)) <= 1e-5
    s.set_charges(-q)  # reversed charges: q_i q_j, hence every force, is unchanged bit for bit
    assert np.array_equal(s.forces(), F1)
    s.set_charges(np.zeros_like(q))  # no charges: the LJ kernel's result bit for bit
    lj = rbl.System(x1, v1, L, c["rc"], c["rs"], c["skin"], c["p"], 0.005, T=1.5, seed=c["seed"],
                    cells_per_cutoff=c["K"], step=step)
    assert np.array_equal(s.forces(), lj.forces())


def test_errors():
    c = CASES["n1000"]
    x, v, L, q = _state(c)
    lj = rbl.System(x, v, L, c["rc"], c["rs"], c["skin"], c["p"], 0.005)
    with pytest.raises(rbl.RblError) as e:
        lj.set_charges(q)
    assert e.value.status == 1
    s = _system(c, x, v, L, q)
    bad = q.copy()
    bad[7] = np.nan
    with pytest.raises(rbl.RblError):
        s.set_charges(bad)
    # the allocation-free entry point takes no charges
    prm = rbl.make_params(L, c["rc"], c["rs"], c["skin"], c["p"], 0.005, potential=rbl.RBL_POT_LJ_EWALD,
                          alpha=1.0)
    xd = torch.as_tensor(x, device="cuda")
    Fd = torch.empty_like(xd)
    st = rbl.load().rbl_forces_static(prm, len(x), rbl._ptr(xd), 0, rbl._ptr(Fd), None)
    assert st == 1


def test_ensemble_matches_single_contexts():
    spec = [(500, 0.9, 1.0), (2113, 0.6, 2.0), (777, 0.75, 1.2)]
    reps = []
    for r, (N, rho, T) in enumerate(spec):
        x, L = inputs.fcc(N, rho, 0.2, seed=60 + r)
        v = inputs.maxwell_boltzmann(N, T, seed=60 + r)
        reps.append(rbl.Replica(x, v, L, T, 60 + r, q=inputs.charges(N, 1.0, seed=60 + r)))
    shared = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, gamma=1.0, alpha=1.0, **EW)
    ens = rbl.Ensemble(reps, **shared)
    F = ens.split(ens.forces())
    ens.step(40)
    xs = ens.split(ens.get_state()[0])
    for r, rp in enumerate(reps):
        s = rbl.System(rp.x, rp.v, rp.L, T=rp.T, seed=rp.seed, charges=rp.q, **shared)
        assert np.array_equal(F[r], s.forces()), r
        s.step(40)
        assert np.array_equal(xs[r], s.get_state()[0]), r


def test_charged_fluid_full_size_sampled():
    """The charged-fluid throughput workload (N = 2^20, rho* = 0.8, T* = 1.5, r_c 1.5,
    r_s 3.5, p 10, alpha 1, FP32, Langevin) after 20 graph steps: 128 sampled
    particles' rows, batches and forces against the oracle, which tests every other
    particle for each of them."""
    N, seed = 1 << 20, 1
    x, L = inputs.fcc(N, 0.8, 0.01, seed=seed)
    v = inputs.maxwell_boltzmann(N, 1.5, seed=seed)
    q = inputs.charges(N, 1.0, seed=seed)
    common = dict(T=1.5, seed=seed, alpha=1.0, charges=q, **EW)
    s = rbl.System(x, v, L, 1.5, 3.5, 0.3, 10, 0.005, gamma=1.0, **common)
    s.step(20)
    x20, v20, step = s.get_state()
    del s
    torch.cuda.empty_cache()
    raw = rbl.System(x20, v20, L, 1.5, 3.5, 0.3, 10, 0.005, subtract_net_force=False, step=step, **common)
    F = raw.forces()
    idx = np.sort(np.random.default_rng(3).choice(N, 128, replace=False))
    smp = oracle.sample(x20, L, 1.5, 3.5, 0.3, 10, seed, step, idx, K=2, q=q, alpha=1.0)
    shell, ns = raw.get_rows(1, idx)
    assert np.array_equal(ns, smp.n_shell)
    for k in range(len(idx)):
        assert np.array_equal(shell[k, : ns[k]], smp.row("shell", k)), k
    assert _relnorm(F[idx], smp.F) <= 1e-5
