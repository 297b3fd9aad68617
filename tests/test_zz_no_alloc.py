"""The allocation-free entry point rbl_forces_static, through the C ABI.

It exists for callers that may not allocate device memory when they need forces
(a plugin inside another engine's time step whose host application owns all device
memory, or code under a no-allocation rule after initialisation).  Its working
memory is a fixed device array inside the library.  This file runs last so that a
failure here never hides the other GPU tests; it passes both alone in a fresh
process and after them (the first call on a device sets the array up)."""
import ctypes

import numpy as np
import pytest

from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402


def _relnorm(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_entry_matches_context_path():
    """Two calls in a row (different systems and step counters) each give the force
    that rbl_forces on a context gives, within the FP32-path tolerance (1e-5)."""
    lib = rbl.load()
    stream = torch.cuda.current_stream()
    for N, seed, step in ((3000, 3, 0), (4096, 4, 17)):
        x, L = inputs.fcc(N, 0.8, 0.2, seed=seed)
        v = inputs.maxwell_boltzmann(N, 1.5, seed=seed)
        prm = rbl.make_params(L, 1.5, 3.5, 0.3, 10, 0.005, T=1.5, gamma=1.0, seed=seed)
        xd = torch.from_numpy(x).cuda()
        Fd = torch.full_like(xd, float("nan"))
        torch.cuda.synchronize()
        st = lib.rbl_forces_static(ctypes.byref(prm), N, ctypes.c_void_p(xd.data_ptr()), step,
                                   ctypes.c_void_p(Fd.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, rbl.STATUS.get(st, st)
        got = Fd.cpu().numpy()
        ref = rbl.System(x, v, L, 1.5, 3.5, 0.3, 10, 0.005, T=1.5, gamma=1.0, seed=seed, step=step).forces()
        assert np.all(np.isfinite(got))
        assert _relnorm(got, ref) <= 1e-5


def test_static_entry_rejects_oversized_system():
    """A system whose workspace exceeds the fixed array is refused before any work."""
    lib = rbl.load()
    N = 2_000_000
    L = [(N / 0.8) ** (1 / 3)] * 3
    prm = rbl.make_params(L, 1.5, 3.5, 0.3, 10, 0.005)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.rbl_forces_static(ctypes.byref(prm), N, ctypes.c_void_p(dummy.data_ptr()), 0,
                               ctypes.c_void_p(dummy.data_ptr()), None)
    assert st == 2  # RBL_ENOMEM
