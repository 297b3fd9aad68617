"""The allocation-free entry point rbl_forces_static, through the C ABI.

It exists for callers that may not allocate device memory when they need forces:
a plugin called inside another engine's time step, whose host application owns all
device memory and forbids cudaMalloc there (it can fail, or synchronise the device,
in the middle of a run), or code that may only allocate while it initialises.  Its
working memory is a fixed device array inside the library.  This file runs last so
that a failure here never hides the other GPU tests; it passes both alone in a fresh
process and after them (the first call on a device sets the array up)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

RADII = (1.5, 3.5, 0.3, 10)  # r_c, r_s, skin, p
LIMIT = 48 << 20  # bytes of the library's fixed array


def _relnorm(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _call(lib, prm, N, xd, step, Fd):
    stream = torch.cuda.current_stream()
    return lib.rbl_forces_static(ctypes.byref(prm), N, ctypes.c_void_p(xd.data_ptr()), step,
                                 ctypes.c_void_p(Fd.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_static_entry_matches_oracle_and_context():
    """Two calls in a row (different systems and step counters) each give the oracle's
    mean-subtracted RBL force within the FP32-path tolerance (1e-5 relative norm)
    and the force rbl_forces gives on a context."""
    lib = rbl.load()
    rc, rs, skin, p = RADII
    for N, seed, step in ((3000, 3, 0), (4096, 4, 17)):
        x, L = inputs.fcc(N, 0.8, 0.2, seed=seed)
        v = inputs.maxwell_boltzmann(N, 1.5, seed=seed)
        prm = rbl.make_params(L, rc, rs, skin, p, 0.005, T=1.5, gamma=1.0, seed=seed)
        xd = torch.from_numpy(x).cuda()
        Fd = torch.full_like(xd, float("nan"))
        torch.cuda.synchronize()
        st = _call(lib, prm, N, xd, step, Fd)
        assert st == 0, rbl.STATUS.get(st, st)
        got = Fd.cpu().numpy()
        assert np.all(np.isfinite(got))
        lists = oracle.build_lists(x, L, rc, rs, skin, K=2)
        Fo, _, _, _ = oracle.rbl_forces(x, L, rc, rs, skin, p, seed, step, lists)
        assert _relnorm(got, oracle.subtract_mean(Fo)) <= 1e-5
        ref = rbl.System(x, v, L, rc, rs, skin, p, 0.005, T=1.5, gamma=1.0, seed=seed, step=step).forces()
        assert _relnorm(got, ref) <= 1e-5


def test_static_entry_allocates_nothing():
    """A call after the first one leaves the device's free memory unchanged."""
    lib = rbl.load()
    rc, rs, skin, p = RADII
    x, L = inputs.fcc(5000, 0.8, 0.2, seed=5)
    prm = rbl.make_params(L, rc, rs, skin, p, 0.005, seed=5)
    xd = torch.from_numpy(x).cuda()
    Fd = torch.empty_like(xd)
    assert _call(lib, prm, 5000, xd, 0, Fd) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _call(lib, prm, 5000, xd, 1, Fd) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def _largest_fitting_N(rho):
    """The largest N whose workspace (rbl_workspace_size) fits the fixed array."""
    lib = rbl.load()
    rc, rs, skin, p = RADII

    def need(N):
        L = (N / rho) ** (1 / 3)
        prm = rbl.make_params([L] * 3, rc, rs, skin, p, 0.005)
        out = ctypes.c_size_t()
        assert lib.rbl_workspace_size(ctypes.byref(prm), N, ctypes.byref(out)) == 0
        return out.value

    lo, hi = 1000, 2_000_000
    assert need(lo) <= LIMIT < need(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if need(mid) <= LIMIT else (lo, mid)
    return lo


def test_static_entry_size_limit():
    """The largest system whose workspace fits the array runs; one particle more
    (same density) is refused with RBL_ENOMEM before any work."""
    lib = rbl.load()
    rc, rs, skin, p = RADII
    rho = 0.8
    N = _largest_fitting_N(rho)
    assert 40_000 < N < 80_000
    for n, want in ((N, 0), (N + 1, 2)):
        x, L = inputs.fcc(n, rho, 0.2, seed=6)
        prm = rbl.make_params(L, rc, rs, skin, p, 0.005, seed=6)
        xd = torch.from_numpy(x).cuda()
        Fd = torch.full_like(xd, float("nan"))
        assert _call(lib, prm, n, xd, 0, Fd) == want
        if want == 0:
            assert np.all(np.isfinite(Fd.cpu().numpy()))
