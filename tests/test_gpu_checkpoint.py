"""Checkpoint and resume through the C ABI.

Algorithm 1 draws each step's batches from the rows of the last list build with
random numbers keyed by (seed, step, tag), so a resumed run reproduces the
uninterrupted one only if it resumes with those rows.  A checkpoint carries the
images the lists were built from; the tests run 2n steps in one call against n
steps, a checkpoint, a new context that loads it, and n more steps, and require
positions, velocities, step counter and rebuild counts to be bit-identical.  The
same holds for a run split into calls in one context, with observations between
them: a call leaves its last closing half kick pending for the next call's first
step, as between the steps inside a call."""
import numpy as np
import pytest

from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

SHARED = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, gamma=1.0)


def _system(precision, N=3000, seed=11):
    x, L = inputs.fcc(N, 0.8, 0.05, seed=seed)  # a start that steps without blowing up
    v = inputs.maxwell_boltzmann(N, 1.5, seed=seed)
    return lambda: rbl.System(x, v, L, T=1.5, seed=seed, precision=precision, **SHARED)


def _ensemble(precision):
    spec = [(500, 0.9, 1.0), (2113, 0.6, 2.0), (1777, 0.8, 1.5)]
    reps = []
    for r, (N, rho, T) in enumerate(spec):
        x, L = inputs.fcc(N, rho, 0.05, seed=60 + r)
        reps.append(rbl.Replica(x, inputs.maxwell_boltzmann(N, T, seed=60 + r), L, T, 60 + r))
    return lambda: rbl.Ensemble(reps, precision=precision, **SHARED)


def _rebuilds(ctx):
    o = ctx._observables()
    return [int(x["n_rebuild"]) for x in o]


def _check_resume(make, n, device):
    # the reference runs the 2n steps in one call (a run's trajectory does not depend
    # on how it is split into calls)
    ref = make()
    ref.step(2 * n)
    x_ref, v_ref, step_ref = ref.get_state()
    nr_ref = _rebuilds(ref)
    assert nr_ref[0] >= 4  # the segment crosses several rebuilds

    a = make()
    a.step(n)
    buf = a.save_checkpoint(device=device)
    nr_saved = _rebuilds(a)
    del a
    b = make()
    b.step(3)  # a context with a different trajectory: everything must be replaced
    b.load_checkpoint(buf)
    assert _rebuilds(b) == nr_saved  # no extra rebuild at the resume step
    b.step(n)
    x, v, step = b.get_state()
    assert step == step_ref
    assert np.array_equal(x, x_ref)
    assert np.array_equal(v, v_ref)
    assert _rebuilds(b) == nr_ref


@pytest.mark.parametrize("precision", [rbl.RBL_FP32, rbl.RBL_FP64])
@pytest.mark.parametrize("device", [False, True])
def test_resume_single_system_bit_identical(precision, device):
    _check_resume(_system(precision), 30, device)


@pytest.mark.parametrize("precision", [rbl.RBL_FP32, rbl.RBL_FP64])
def test_resume_ensemble_bit_identical(precision):
    _check_resume(_ensemble(precision), 30, False)


def test_resume_right_after_set_state():
    """A checkpoint taken before any step (lists not built yet) resumes to the same
    trajectory: the first step of both builds the lists."""
    make = _system(rbl.RBL_FP32, N=2000, seed=12)
    ref = make()
    ref.step(25)
    a = make()
    buf = a.save_checkpoint()
    b = make()
    b.step(7)
    b.load_checkpoint(buf)
    b.step(25)
    xr, vr, _ = ref.get_state()
    x, v, _ = b.get_state()
    assert np.array_equal(x, xr) and np.array_equal(v, vr)
    assert _rebuilds(b) == _rebuilds(ref)


def test_checkpoint_of_other_sizes_rejected():
    a = _system(rbl.RBL_FP32, N=2000)()
    buf = a.save_checkpoint()
    b = _system(rbl.RBL_FP32, N=2001)()
    with pytest.raises(rbl.RblError) as e:
        b.load_checkpoint(buf)
    assert e.value.status == 1  # RBL_EINVAL
    bad = buf.copy()
    bad[:8] = 0
    with pytest.raises(rbl.RblError):
        a.load_checkpoint(bad)
    c = _system(rbl.RBL_FP64, N=2000)()
    with pytest.raises(rbl.RblError):
        c.load_checkpoint(buf)


@pytest.mark.parametrize("precision", [rbl.RBL_FP32, rbl.RBL_FP64])
def test_call_splitting_does_not_change_the_trajectory(precision):
    make = _system(precision, N=2000, seed=13)
    a = make()
    a.step(24)
    b = make()  # split, with state and observables read in between
    b.step(10)
    b.get_state()
    b.observables()
    b.step(13)
    b.get_state()
    b.step(1)
    c = make()  # one step per call, as an end-to-end loop runs
    for _ in range(24):
        c.step_async(1)
        c.observables()
    xa, va, sa = a.get_state()
    for other in (b, c):
        x, v, st = other.get_state()
        assert st == sa
        assert np.array_equal(x, xa) and np.array_equal(v, va)
        assert _rebuilds(other) == _rebuilds(a)
    assert a.observables()["K"] == c.observables()["K"]


def test_pending_kick_applied_before_charges_change():
    """rbl_set_charges applies the pending half kick with the force it is due with
    (the old charges'), so setting the same charges again changes nothing."""
    N, seed = 1500, 14
    x, L = inputs.fcc(N, 0.8, 0.05, seed=seed)
    v = inputs.maxwell_boltzmann(N, 1.5, seed=seed)
    q = inputs.charges(N, 1.0, seed=seed)
    args = dict(T=1.5, seed=seed, potential=rbl.RBL_POT_LJ_EWALD, alpha=1.0, charges=q, **SHARED)
    a = rbl.System(x, v, L, **args)
    a.step(12)
    b = rbl.System(x, v, L, **args)
    b.step(6)
    b.set_charges(q)
    b.step(6)
    xa, va, _ = a.get_state()
    xb, vb, _ = b.get_state()
    # the kick is applied separately (two roundings instead of one fused kick of dt),
    # so the trajectories agree to rounding, not bit for bit
    assert np.abs(xa - xb).max() < 1e-9 and np.abs(va - vb).max() < 1e-9
