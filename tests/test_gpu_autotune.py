"""Launch shapes change nothing: every force-kernel block size and list-build
block shape gives bit-identical forces, lists and trajectories, for one system and
for an ensemble; the autotuner picks among them and leaves the run as it was."""
import itertools

import numpy as np
import pytest

from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

ARGS = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, T=1.5, gamma=1.0, seed=9)
CONFIGS = list(itertools.product((64, 128, 256), (2, 4, 8)))


def _run(make, cfg, steps=30):
    s = make()
    s.set_launch_config(*cfg)
    F = s.forces()
    rows, counts = s.get_lists(1, cap=400)
    s.step(steps)
    x, v, _ = s.get_state()
    return F, rows, counts, x, v


@pytest.mark.parametrize("precision", [rbl.RBL_FP32, rbl.RBL_FP64])
def test_single_system_results_do_not_depend_on_launch_shape(precision):
    x, L = inputs.fcc(3001, 0.8, 0.05, seed=9)  # a start velocity-Verlet at dt = 0.005 can step
    v = inputs.maxwell_boltzmann(3001, 1.5, seed=9)
    ref = None
    for cfg in CONFIGS:
        out = _run(lambda: rbl.System(x, v, L, precision=precision, **ARGS), cfg)
        if ref is None:
            ref = out
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), cfg


def test_ensemble_results_do_not_depend_on_launch_shape():
    reps = inputs.ensemble(6, n_min=500, n_max=3000, seed=4)
    shared = {k: ARGS[k] for k in ("r_c", "r_s", "skin", "p", "dt", "gamma")}
    ref = None
    for cfg in [(64, 2), (256, 8), (128, 4)]:
        out = _run(lambda: rbl.Ensemble(reps, **shared), cfg)
        if ref is None:
            ref = out
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), cfg


def test_autotune_leaves_the_run_unchanged():
    x, L = inputs.fcc(20000, 0.8, 0.01, seed=2)
    v = inputs.maxwell_boltzmann(20000, 1.5, seed=2)
    s = rbl.System(x, v, L, **ARGS)
    ref = rbl.System(x, v, L, **ARGS)
    s.step(10)
    ref.step(10)
    before = s.observables()
    pick = s.autotune(trials=2)
    assert pick["force_threads"] in (64, 128, 256) and pick["build_warps"] in (2, 4, 8)
    after = s.observables()
    assert after["n_rebuild"] == before["n_rebuild"] and after["U_est"] == before["U_est"]
    assert np.array_equal(s.get_state()[0], ref.get_state()[0])
    s.step(10)
    ref.step(10)
    xs, vs, _ = s.get_state()
    xr, vr, _ = ref.get_state()
    assert np.array_equal(xs, xr) and np.array_equal(vs, vr)


def test_tune_cells_picks_the_fastest_cell_size():
    """rbl_tune_cells times K = 1, 2, 3 on the caller's system, each in a context of
    its own inside one workspace, and returns the K of the smallest time; the caller's
    arrays are not touched, and a context at the chosen K runs from the same state."""
    N = 8000
    x, L = inputs.fcc(N, 0.8, 0.05, seed=11)
    v = inputs.maxwell_boltzmann(N, 1.5, seed=11)
    x0, v0 = x.copy(), v.copy()
    args = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005)
    K, ms = rbl.tune_cells(x, v, L, steps=10, T=1.5, gamma=1.0, seed=11, **args)
    assert np.array_equal(x, x0) and np.array_equal(v, v0)
    assert all(t > 0 for t in ms), ms  # L = 21.5 allows every K
    assert K == 1 + int(np.argmin(ms)), (K, ms)
    s = rbl.System(x, v, L, T=1.5, gamma=1.0, seed=11, cells_per_cutoff=K, **args)
    s.step(10)
    assert np.isfinite(s.observables()["T_kin"])


def test_tune_cells_skips_cell_sizes_the_box_does_not_allow():
    """A K whose workspace does not fit is reported as -1 and never chosen."""
    import ctypes

    import torch

    N = 4000
    x, L = inputs.fcc(N, 0.8, 0.05, seed=12)
    v = inputs.maxwell_boltzmann(N, 1.5, seed=12)
    lib = rbl.load()
    sizes = []
    for k in (1, 2, 3):
        prm = rbl.make_params(L, 1.5, 3.5, 0.3, 10, 0.005, T=1.5, seed=12, cells_per_cutoff=k)
        b = ctypes.c_size_t()
        assert lib.rbl_workspace_size(ctypes.byref(prm), N, ctypes.byref(b)) == 0
        sizes.append(b.value)
    room = sorted(sizes)[1]  # fits the two smaller workspaces only
    ws = torch.empty(room + 256, dtype=torch.uint8, device="cuda")
    aligned = (ws.data_ptr() + 255) & ~255
    prm = rbl.make_params(L, 1.5, 3.5, 0.3, 10, 0.005, T=1.5, seed=12)
    Kb = ctypes.c_int()
    ms = (ctypes.c_float * 3)()
    stream = torch.cuda.Stream()
    xs = np.ascontiguousarray(x)
    vs = np.ascontiguousarray(v)
    st = lib.rbl_tune_cells(ctypes.byref(prm), N, xs.ctypes.data_as(ctypes.c_void_p),
                            vs.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(aligned), room,
                            ctypes.c_void_p(stream.cuda_stream), 10, ctypes.byref(Kb), ms)
    assert st == 0
    big = int(np.argmax(sizes))
    assert ms[big] == -1.0 and Kb.value != big + 1
    assert all(ms[k] > 0 for k in range(3) if k != big)
