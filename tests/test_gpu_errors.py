"""Failure detection through the C ABI, with no GPU fault: the kernels record a
problem in the context's device flags and keep every access inside the arrays (rows
are written only up to their capacity; a cell whose culled candidate table exceeds
its capacity gets empty rows), and the next synchronising call turns the flag into a
status.

- a core row longer than its capacity -> RBL_EOVERFLOW (rows truncated, counts kept);
- a culled candidate table beyond its capacity (cap_stencil) -> RBL_EOVERFLOW;
- non-finite input positions -> RBL_ENONFINITE at rbl_set_state;
- finite input that turns bad during a step (two particles 0.05 sigma apart, or at
  the same place): the binary32 force leaves the fixed-point range or is NaN (FP32
  path), or the kicked particle jumps more than a box length (FP64 path) ->
  RBL_ENONFINITE from rbl_step, with every kernel still inside its arrays (images are
  32-bit integers whatever the positions, so cells and rows stay in range);
- the capacities sized for the density pass (the same system with derived caps).
"""
import numpy as np
import pytest

from paper_2105_04884_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2105_04884_gb300 import rbl  # noqa: E402

ARGS = dict(r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, T=1.5, seed=1)


@pytest.fixture(scope="module")
def fluid():
    x, L = inputs.fcc(2000, 0.8, 0.1, seed=2)
    v = inputs.maxwell_boltzmann(2000, 1.5, seed=2)
    return x, v, L


def test_core_row_overflow(fluid):
    x, v, L = fluid
    s = rbl.System(x, v, L, cap_core=4, **ARGS)  # ~19 core entries per particle
    with pytest.raises(rbl.RblError) as e:
        s.forces()
    assert e.value.status == 3 and "capacity" in str(e.value)


def test_stencil_overflow(fluid):
    x, v, L = fluid
    s = rbl.System(x, v, L, cap_stencil=64, **ARGS)  # ~350 culled candidates per home cell
    with pytest.raises(rbl.RblError) as e:
        s.step(2)
    assert e.value.status == 3


def test_nonfinite_input(fluid):
    x, v, L = fluid
    bad = x.copy()
    bad[17, 1] = np.nan
    with pytest.raises(rbl.RblError) as e:
        rbl.System(bad, v, L, **ARGS)
    assert e.value.status == 4


def test_derived_capacities_pass(fluid):
    x, v, L = fluid
    s = rbl.System(x, v, L, **ARGS)
    s.step(5)
    assert np.isfinite(s.forces()).all()


@pytest.mark.parametrize("precision", [rbl.RBL_FP32, rbl.RBL_FP64])
@pytest.mark.parametrize("gap", [0.05, 0.0])
def test_overlap_mid_run(fluid, precision, gap):
    """Finite positions are accepted; the first step reports the blow-up."""
    x, v, L = fluid
    y = x.copy()
    y[1] = y[0] + np.array([gap, 0.0, 0.0])  # particle 1 moved next to (or onto) particle 0
    s = rbl.System(y, v, L, precision=precision, **ARGS)
    with pytest.raises(rbl.RblError) as e:
        s.step(1)
    assert e.value.status == 4, str(e.value)
    # the context still answers: a new state loads and steps
    s.set_state(x, v)
    s.step(2)
    assert np.isfinite(s.forces()).all()
