"""GPU time stepping against the oracle from the same state, through the C ABI.

- FP64 path, gamma = 0: 40 velocity-Verlet steps with list rebuilds stay within
  1e-9 (positions) of the oracle's trajectory: both integrate the same FP64
  arithmetic up to rounding order, and 0.2 time units are too short for chaos to
  amplify 1e-16 differences past that; the number of list builds must agree exactly.
- gamma > 0: one BAOAB step; the thermostat noise is drawn in binary32 on the GPU and
  FP64 in the oracle from the same Philox words, so velocities agree to the binary32
  accuracy of the noise term (|dv| <= 5e-7), positions to dt/2 of that.
- momentum: with the mean force subtracted and gamma = 0 the total momentum stays
  at its initial value to rounding.
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


def _min_image(d, L):
    return d - L * np.round(d / L)


@pytest.mark.parametrize("full_list", [False, True])
def test_nve_trajectory_fp64(full_list):
    x, L = inputs.fcc(1000, 0.8, 0.01, seed=1)
    v = inputs.maxwell_boltzmann(1000, 1.5, seed=1)
    n = 40
    s = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.5, gamma=0.0, seed=1, precision=rbl.RBL_FP64,
                   full_list=full_list)
    s.step(n)
    xg, vg, step = s.get_state()
    obs = s.observables()
    xo, vo, Fo, stats = oracle.run(x, v, L, RC, RS, SKIN, P, DT, 1.5, 0.0, 1, n, full_list=full_list)
    assert step == n
    assert obs["n_rebuild"] == int(stats[2]) and stats[2] > 2
    assert np.abs(_min_image(xg - xo, L)).max() < 1e-9
    assert np.abs(vg - vo).max() < 1e-8
    assert abs(obs["U_est"] - stats[0]) < 1e-8 * abs(stats[0])
    # the observables launch's kinetic sums against the oracle's own velocities
    Ko = 0.5 * float((vo * vo).sum())
    assert abs(obs["K"] - Ko) < 1e-8 * Ko
    assert abs(obs["T_kin"] - 2 * Ko / (3 * len(xo))) < 1e-8 * obs["T_kin"]
    assert np.abs(np.asarray(obs["net_momentum"]) - vo.sum(0)).max() < 1e-7


@pytest.mark.parametrize("precision", [rbl.RBL_FP64, rbl.RBL_FP32])
def test_baoab_single_step(precision):
    x, L = inputs.fcc(1000, 0.8, 0.05, seed=2)
    v = inputs.maxwell_boltzmann(1000, 1.5, seed=2)
    s = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.5, gamma=1.0, seed=7, precision=precision, step=5)
    s.step(1)
    xg, vg, step = s.get_state()
    xo, vo, _, _ = oracle.run(x, v, L, RC, RS, SKIN, P, DT, 1.5, 1.0, 7, 1, step0=5)
    assert step == 6
    # force error enters v with dt/2 per half kick (FP32 path: 1e-5 relative)
    ftol = 0.0 if precision == rbl.RBL_FP64 else 1e-4
    assert np.abs(vg - vo).max() < 5e-7 + ftol
    assert np.abs(_min_image(xg - xo, L)).max() < 5e-9 + DT * ftol


def test_momentum_conserved_fp32():
    x, L = inputs.fcc(4000, 0.8, 0.01, seed=3)
    v = inputs.maxwell_boltzmann(4000, 1.5, seed=3)
    s = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.5, gamma=0.0, seed=3)
    p0 = v.sum(0)
    s.step(50)
    _, vg, _ = s.get_state()
    assert np.abs(vg.sum(0) - p0).max() < 1e-9
    obs = s.observables()
    assert obs["n_rebuild"] >= 2


def test_langevin_temperature_fp32():
    """BAOAB at gamma = 1 holds <T_kin> near T (short run from an FCC start)."""
    x, L = inputs.fcc(8000, 0.8, 0.01, seed=4)
    v = inputs.maxwell_boltzmann(8000, 1.2, seed=4)
    s = rbl.System(x, v, L, RC, RS, SKIN, P, DT, T=1.2, gamma=1.0, seed=4)
    s.step(400)
    temps = []
    for _ in range(20):
        s.step(20)
        temps.append(s.observables()["T_kin"])
    assert abs(np.mean(temps) - 1.2) < 0.05
