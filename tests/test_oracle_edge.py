"""The oracle on degenerate inputs (no GPU): the cell-list builder against the
all-pairs builder where most cells are empty, stencils wrap or particles sit exactly
on the faces; the fixed-point image of the largest coordinate below L (R10: the
image of x is rint(x 2^32 / L) mod 2^32, so it wraps to 0, the image of 0); and the
two-particle system against the closed-form LJ pair (Sec. 2 with N_s <= p: the whole
shell is the batch, scale 1)."""
import numpy as np
import pytest

import oracle
from degenerate_cases import CASES

RC, RS, SKIN, P = 1.5, 3.5, 0.3, 10


@pytest.mark.parametrize("name", sorted(CASES))
def test_cell_builder_equals_brute(name):
    x, _, L, _ = CASES[name]()
    a = oracle.build_lists(x, L, RC, RS, SKIN, K=2, method="brute")
    b = oracle.build_lists(x, L, RC, RS, SKIN, K=2, method="cells")
    for kind in ("core", "shell", "full"):
        assert np.array_equal(getattr(a, "n_" + kind), getattr(b, "n_" + kind)), kind
        for i in range(len(x)):
            assert np.array_equal(a.row(kind, i), b.row(kind, i)), (kind, i)


@pytest.mark.parametrize("Lv", [8.549879733383484, 10.0, 25.0, 603.0493035782765])
def test_largest_coordinate_wraps_to_image_zero(Lv):
    L = np.full(3, Lv)
    x = np.array([[0.0, np.nextafter(Lv, 0.0), Lv / 2], [np.nextafter(Lv, 0.0), 0.0, np.nextafter(Lv / 2, 0.0)]])
    u = oracle.quantize(x, L)
    assert u[0, 0] == 0 and u[0, 1] == 0 and u[1, 0] == 0 and u[1, 1] == 0
    assert u[0, 2] == 2**31 and u[1, 2] == 2**31  # L/2 less one ulp rounds to the half-box image


@pytest.mark.parametrize("name,d", [("pair_core", 1.2), ("pair_shell", 2.5), ("pair_skin_band", 3.65),
                                    ("pair_beyond", 4.5), ("pair_core_through_face", 1.2)])
def test_pair_forces_closed_form(name, d):
    x, _, L, _ = CASES[name]()
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=2)
    F, ev, _, nb = oracle.rbl_forces(x, L, RC, RS, SKIN, P, 3, 0, lists, want_batch=True)
    r = x[0] - x[1]
    r -= L * np.round(r / L)
    rr = np.sqrt((r * r).sum())
    assert abs(rr - d) < 1e-12
    if d < RS:
        ir6 = rr**-6
        f = 24.0 * (2.0 * ir6 * ir6 - ir6) / (rr * rr)  # F_0 = f (x_0 - x_1)
        u = 4.0 * (ir6 * ir6 - ir6)
    else:
        f = u = 0.0
    expect = np.array([f * r, -f * r])
    assert np.allclose(F, expect, rtol=1e-12, atol=1e-300)
    assert abs(ev[0] - u) <= 1e-12 * max(abs(u), 1e-300)
    # the whole shell is the batch when N_s <= p; the core is summed directly
    in_shell = RC <= d < RS + SKIN
    assert list(nb) == ([1, 1] if in_shell else [0, 0])
