"""Liquid-vapour slab (the slab workload at reduced size): Lx = Ly = 30, Lz = 4 Lx,
liquid rho* = 0.75 over the central 40% of z, vapour rho* = 0.01 elsewhere,
T* = 0.9, r_c = 1.5, r_s = 4.0, p = 20, FP32, capacities sized for the liquid
(rho_cap).  The density profile is exact against the oracle, the run stays within
its capacities through the 75x density contrast, and RBL keeps the liquid and
vapour densities of the full Verlet list."""
import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

LX, LZ, RHO_L, RHO_V = 30.0, 120.0, 0.75, 0.01
COMMON = dict(r_c=1.5, r_s=4.0, skin=0.3, p=20, dt=0.005, T=0.9, gamma=1.0, seed=3, rho_cap=RHO_L)
NB = 240  # 0.5 sigma bins


def _slab():
    V = LX * LX * LZ
    N = int(round(RHO_L * 0.4 * V + RHO_V * 0.6 * V))
    x, L = inputs.slab(N, LX, LZ, RHO_L, RHO_V, seed=3)
    v = inputs.maxwell_boltzmann(len(x), 0.9, seed=3)
    return x, v, L


def _densities(h, L, nsamp):
    rho = h / nsamp / (L[0] * L[1] * (L[2] / NB))
    z = (np.arange(NB) + 0.5) * L[2] / NB
    liquid = np.abs(z - L[2] / 2) < 0.12 * L[2]
    vapour = np.abs(z - L[2] / 2) > 0.35 * L[2]
    return rho[liquid].mean(), rho[vapour].mean()


def test_profile_exact_on_slab():
    x, v, L = _slab()
    s = rbl.System(x, v, L, **COMMON)
    assert np.array_equal(s.density_profile(2, NB), oracle.density_profile(x, L, 2, NB))
    s.step(50)
    x1, _, _ = s.get_state()
    assert np.array_equal(s.density_profile(2, NB), oracle.density_profile(x1, L, 2, NB))


def test_rbl_keeps_slab_densities():
    x, v, L = _slab()
    out = {}
    for full in (False, True):
        s = rbl.System(x, v, L, full_list=full, **COMMON)
        s.step(200)
        h = np.zeros(NB, np.int64)
        for _ in range(10):
            s.step(20)
            s.density_profile(2, NB, h)
        out[full] = _densities(h, L, 10)
    (lr, vr), (lf, vf) = out[False], out[True]
    assert abs(lr - lf) < 0.02, (lr, lf)
    assert abs(lf - 0.75) < 0.05
    assert vr < 0.05 and vf < 0.05
