"""rbl_observables and rbl_observables_async through the C ABI: the scalars against
their definitions computed here from the state the library returns, and the
asynchronous form equal to the synchronous one bit for bit (both assemble rbl_obs on
the device from the same sums).

- K = sum v^2 / 2, T_kin = 2K / (3N), net momentum = sum v (FP64, to rounding);
- P = rho T_kin + W_est / (3V);
- tail terms equal to the oracle's tail corrections (Sec. 3), themselves pinned by
  quadrature;
- list statistics equal to the row lengths the library returns.
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

RC, RS, SKIN, P, DT = 1.5, 3.5, 0.3, 10, 0.005


def test_scalars_match_their_definitions():
    x, L = inputs.fcc(3000, 0.8, 0.1, seed=3)
    v = inputs.maxwell_boltzmann(3000, 1.5, seed=3)
    s = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.5, gamma=1.0, seed=3)
    s.step(25)
    o = s.observables()
    xs, vs, step = s.get_state()
    N, V = len(xs), float(np.prod(L))
    K = 0.5 * float((vs * vs).sum())
    assert o["step"] == step == 25
    assert abs(o["K"] - K) <= 1e-12 * K
    assert abs(o["T_kin"] - 2 * K / (3 * N)) <= 1e-12 * o["T_kin"]
    assert np.allclose(o["net_momentum"], vs.sum(0), rtol=0, atol=1e-10)
    rho = N / V
    assert abs(o["P"] - (rho * o["T_kin"] + o["W_est"] / (3 * V))) <= 1e-12 * abs(o["P"])
    tail = oracle.tail(rho, RS)
    assert abs(o["U_tail"] - tail[0]) <= 1e-13 * abs(tail[0])
    assert abs(o["P_tail"] - tail[1]) <= 1e-13 * abs(tail[1])
    core, nc = s.get_lists(0)
    shell, ns = s.get_lists(1)
    assert o["Nc_max"] == nc.max() and o["Ns_max"] == ns.max()
    assert o["Nc_mean"] == nc.sum() / N and o["Ns_mean"] == ns.sum() / N


def test_async_equals_sync():
    reps = []
    for r, (N, rho, T) in enumerate([(700, 0.8, 1.2), (1500, 0.7, 1.8), (2049, 0.85, 1.0)]):
        x, L = inputs.fcc(N, rho, 0.05, seed=90 + r)
        reps.append(rbl.Replica(x, inputs.maxwell_boltzmann(N, T, seed=90 + r), L, T, 90 + r))
    ens = rbl.Ensemble(reps, r_c=RC, r_s=RS, skin=SKIN, p=P, dt=DT, gamma=1.0)
    buf = ens.obs_buffer()
    for n in (1, 7):
        ens.step(n)
        ens.observables_async(buf)
        ens.synchronize()
        assert ens.read_obs(buf) == ens.observables()
    # device destination
    dbuf = torch.empty(len(buf), dtype=torch.uint8, device="cuda")
    ens.observables_async(dbuf)
    ens.synchronize()
    assert ens.read_obs(dbuf.cpu()) == ens.observables()


def test_step_async_equals_step():
    """rbl_step_async enqueues exactly what rbl_step runs: 30 one-step calls of each give
    the same trajectory bit for bit, and the observables read after them agree."""
    x, L = inputs.fcc(2000, 0.8, 0.1, seed=5)
    v = inputs.maxwell_boltzmann(2000, 1.5, seed=5)
    a = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.5, gamma=1.0, seed=5)
    b = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.5, gamma=1.0, seed=5)
    buf = b.obs_buffer()
    for _ in range(30):
        a.step(1)
        b.step_async(1)
        b.observables_async(buf)
    xa, va, sa = a.get_state()
    xb, vb, sb = b.get_state()
    assert sa == sb == 30
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert b.read_obs(buf)[0] == a.observables()


def test_state_through_page_locked_buffers():
    """rbl_set_state / rbl_get_state with page-locked host buffers (read and written by
    the kernels themselves, no staging copy) give exactly what pageable host buffers and
    device buffers give, for an ensemble with a pending half kick."""
    import ctypes

    reps = []
    for r, (N, rho, T) in enumerate([(700, 0.8, 1.2), (1500, 0.7, 1.8)]):
        x, L = inputs.fcc(N, rho, 0.05, seed=60 + r)
        reps.append(rbl.Replica(x, inputs.maxwell_boltzmann(N, T, seed=60 + r), L, T, 60 + r))
    ens = rbl.Ensemble(reps, r_c=RC, r_s=RS, skin=SKIN, p=P, dt=DT, gamma=1.0)
    ens.step(7)  # leaves a half kick pending
    x0, v0, step0 = ens.get_state()  # pageable host buffers
    xd, vd, _ = ens.get_state(device=True)
    assert np.array_equal(xd.cpu().numpy(), x0) and np.array_equal(vd.cpu().numpy(), v0)
    xp = torch.empty(x0.shape, dtype=torch.float64).pin_memory()
    vp = torch.empty_like(xp).pin_memory()
    st = ctypes.c_longlong()
    ens._check(ens.lib.rbl_get_state(ens.h, ctypes.c_void_p(xp.data_ptr()), ctypes.c_void_p(vp.data_ptr()),
                                     ctypes.byref(st), 0))
    assert st.value == step0
    assert np.array_equal(xp.numpy(), x0) and np.array_equal(vp.numpy(), v0)
    # the same state loaded from page-locked and from pageable buffers steps identically
    ens._check(ens.lib.rbl_set_state(ens.h, ctypes.c_void_p(xp.data_ptr()), ctypes.c_void_p(vp.data_ptr()),
                                     step0, 0))
    ens.step(5)
    xa, va, _ = ens.get_state()
    ens.set_state(x0, v0, step0)
    ens.step(5)
    xb, vb, _ = ens.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
