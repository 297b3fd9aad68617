"""Matched physics on the GPU: block-averaged pressure, energy and g(r) of RBL
trajectories against the full Verlet list (LJ fluid N = 32,000, rho* = 0.8442,
T* = 1.2, Langevin gamma = 1, dt = 0.005, r_s = 3.5), and the numerical heating the
batch estimator causes (Sec. 2: extra force variance heats the system; under a
Langevin thermostat the kinetic temperature settles dt <|chi|^2> / (6 gamma) above
the bath, chi the per-particle force error of the estimator).

Trajectories are deterministic for a given seed, so each bar below either always
holds or never does; the bars are 3 combined block-average standard errors."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import bench  # noqa: E402
from paper_2105_04884_gb300 import rbl  # noqa: E402

CFG = dict(bench.PHYS)  # 10^4 steps, first 2000 discarded, 16 blocks of 500


@pytest.fixture(scope="module")
def runs():
    x, v, L = bench.physics_inputs(cfg=CFG)
    full = bench.physics_run(x, v, L, 1.5, 10, rbl.RBL_FP32, True, 1, CFG)
    rc2 = bench.physics_run(x, v, L, 2.0, 20, rbl.RBL_FP32, False, 1, CFG)
    rc15 = bench.physics_run(x, v, L, 1.5, 10, rbl.RBL_FP32, False, 1, CFG)
    return full, rc2, rc15


def test_rbl_matches_full_list_at_rc2(runs):
    full, rc2, _ = runs
    c = bench.physics_compare(rc2, full, CFG["dr"])
    for k in ("P_bath", "U", "T"):
        assert abs(c[k]["z"]) < 3.0, (k, c[k])
    assert c["g"]["chi2_per_bin"] < 2.5, c["g"]


def test_heating_follows_estimator_variance(runs):
    """At r_c = 1.5, p = 10 the RBL run is measurably hotter than the full list, by
    the amount the estimator's force variance predicts."""
    full, _, rc15 = runs
    dT = rc15["T"][0] - full["T"][0]
    pred = rc15["heating"]["dT_predicted"]
    assert dT > 10 * (rc15["T"][1] + full["T"][1])
    assert abs(dT - pred) < 0.3 * pred, (dT, pred)


@pytest.fixture(scope="module")
def charged_runs():
    """The same system with neutral random +-1 charges and the Ewald real-space term
    (alpha = 1): full list, RBL at r_c = 2.5 and at r_c = 1.5 (p = 10)."""
    from paper_2105_04884_gb300 import inputs

    x, v, L = bench.physics_inputs(cfg=CFG)
    ch = dict(charges=inputs.charges(len(x), 1.0, seed=1), alpha=1.0)
    full = bench.physics_run(x, v, L, 1.5, 10, rbl.RBL_FP32, True, 1, CFG, **ch)
    rc25 = bench.physics_run(x, v, L, 2.5, 10, rbl.RBL_FP32, False, 1, CFG, **ch)
    rc15 = bench.physics_run(x, v, L, 1.5, 10, rbl.RBL_FP32, False, 1, CFG, **ch)
    return full, rc25, rc15


def test_charged_fluid_matches_full_list_at_rc25(charged_runs):
    full, rc25, _ = charged_runs
    c = bench.physics_compare(rc25, full, CFG["dr"])
    for k in ("P_bath", "U", "T"):
        assert abs(c[k]["z"]) < 3.0, (k, c[k])
    assert c["g"]["chi2_per_bin"] < 2.5, c["g"]


def test_charged_fluid_heating_follows_estimator_variance(charged_runs):
    full, _, rc15 = charged_runs
    dT = rc15["T"][0] - full["T"][0]
    pred = rc15["heating"]["dT_predicted"]
    assert dT > 10 * (rc15["T"][1] + full["T"][1])
    assert abs(dT - pred) < 0.3 * pred, (dT, pred)
