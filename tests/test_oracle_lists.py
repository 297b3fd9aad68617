"""Pins for the oracle's fixed-point pair rule, linked cells and two-level lists.

Lists are pinned by (a) exact lattice-shell counts computed here from integer vectors,
(b) the all-pairs brute-force builder, and (c) FP64 distances away from the
thresholds (the binary32 rule may only differ from exact arithmetic within rounding
of a threshold)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2105_04884_gb300 import inputs

RC, RS, SKIN = 1.5, 3.5, 0.3


def _minimg(x, L, i, j):
    d = x[i] - x[j]
    return d - L * np.round(d / L)


def test_quantize_and_min_image():
    L = np.array([10.0, 12.0, 30.0])
    x = np.array([[0.0, 0.0, 0.0], [5.0, 6.0, 15.0], [9.9, 11.5, 0.25], [0.2, 0.5, 29.75]])
    u = oracle.quantize(x, L)
    assert list(u[0]) == [0, 0, 0]
    assert list(u[1]) == [2**31, 2**31, 2**31]
    # across the periodic face: separation (0.3, 1.0, 0.5)
    r2 = oracle.pair_r2f(u, L, np.array([2]), np.array([3]))[0]
    assert abs(r2 - (0.3**2 + 1.0**2 + 0.5**2)) < 1e-5


def test_pair_rule_matches_fp64_distance():
    """Binary32 r2 from the fixed-point image agrees with the FP64 minimum-image r2."""
    x, L = inputs.fcc(2000, 0.8, 0.3, seed=3)
    u = oracle.quantize(x, L)
    rng = np.random.default_rng(0)
    i = rng.integers(0, 2000, 5000).astype(np.int32)
    j = rng.integers(0, 2000, 5000).astype(np.int32)
    r2 = oracle.pair_r2f(u, L, i, j).astype(np.float64)
    d = x[i] - x[j]
    d -= L * np.round(d / L)
    r2e = (d * d).sum(1)
    assert np.all(np.abs(r2 - r2e) <= 1e-6 * np.maximum(r2e, 1.0))


def test_cells_match_floor():
    x, L = inputs.fcc(3000, 0.8, 0.3, seed=4)
    u = oracle.quantize(x, L)
    for K in (1, 2, 3):
        n = oracle.cell_grid(L, RS, SKIN, K)
        assert list(n) == [int(math.floor(L[0] * K / (RS + SKIN)))] * 3
        c = oracle.cells(u, L, RS, SKIN, K)
        f = np.floor(x / L * n).astype(np.int64)
        lin = (f[:, 2] * n[1] + f[:, 1]) * n[0] + f[:, 0]
        # away from cell faces the exact-integer rule equals floor(x n / L)
        frac = (x / L * n) % 1.0
        ok = np.all((frac > 1e-6) & (frac < 1 - 1e-6), axis=1)
        assert ok.mean() > 0.99
        assert np.array_equal(c[ok], lin[ok])


def _lattice_count(vectors_scale, basis, lo2, hi2, reach):
    """Number of lattice points q != 0 with lo2 <= |q|^2 < hi2 (integer enumeration)."""
    cnt = 0
    for v in itertools.product(range(-reach, reach + 1), repeat=3):
        for b in basis:
            q = (np.array(v) + b) * vectors_scale
            r2 = float(q @ q)
            if r2 > 0 and lo2 <= r2 < hi2:
                cnt += 1
    return cnt


@pytest.mark.parametrize("lattice", ["sc", "fcc"])
def test_list_lengths_on_perfect_lattice(lattice):
    """Every row of a perfect lattice has the lattice-shell count of its window."""
    if lattice == "sc":
        n, a = 12, 1.02
        g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
        x = (g + 0.5) * a
        basis = [np.zeros(3)]
    else:
        n, a = 6, 1.66
        g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
        bas = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
        x = ((g[:, None, :] + bas[None] + 0.25) * a).reshape(-1, 3)
        basis = list(bas)
    L = np.full(3, n * a)
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=2, method="brute")
    expect_core = _lattice_count(a, basis, 0.0, (RC + SKIN) ** 2, 5)
    expect_shell = _lattice_count(a, basis, (RC - SKIN) ** 2, (RS + SKIN) ** 2, 5)
    assert np.all(lists.n_core == expect_core)
    assert np.all(lists.n_shell == expect_shell)
    assert np.all(lists.n_full == _lattice_count(a, basis, 0.0, (RS + SKIN) ** 2, 5))


@pytest.mark.parametrize("N,rho,K", [(1000, 0.8, 1), (1000, 0.8, 2), (1200, 0.5, 3), (800, 0.9, 2)])
def test_cell_builder_equals_brute(N, rho, K):
    x, L = inputs.fcc(N, rho, 0.2, seed=N + K)
    a = oracle.build_lists(x, L, RC, RS, SKIN, K=K, method="brute")
    b = oracle.build_lists(x, L, RC, RS, SKIN, K=K, method="cells")
    for kind in ("core", "shell", "full"):
        assert np.array_equal(getattr(a, "n_" + kind), getattr(b, "n_" + kind))
        for i in range(N):
            assert np.array_equal(a.row(kind, i), b.row(kind, i)), (kind, i)


def test_list_membership_against_fp64():
    """Rows contain exactly the pairs inside each window, judged in FP64 wherever the
    FP64 distance is not within rounding of a window edge."""
    x, L = inputs.fcc(1500, 0.8, 0.25, seed=9)
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=2, method="cells")
    n = x.shape[0]
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    edges = [(RC + SKIN) ** 2, (RC - SKIN) ** 2, (RS + SKIN) ** 2]
    safe = np.ones_like(r2, dtype=bool)
    for e in edges:
        safe &= np.abs(r2 - e) > 1e-5 * e
    for i in range(0, n, 7):
        core = set(lists.row("core", i).tolist())
        shell = set(lists.row("shell", i).tolist())
        want_core = set(np.nonzero(r2[i] < edges[0])[0].tolist())
        want_shell = set(np.nonzero((r2[i] >= edges[1]) & (r2[i] < edges[2]))[0].tolist())
        s = set(np.nonzero(safe[i])[0].tolist())
        assert core & s == want_core & s
        assert shell & s == want_shell & s


def test_canonical_row_order_is_slot_x_then_tag():
    """Row order: by the neighbour cell's stencil slot, then by the neighbour's x
    image, then by tag (checked against a direct recomputation from the cells)."""
    x, L = inputs.fcc(1000, 0.8, 0.2, seed=2)
    K = 2
    lists = oracle.build_lists(x, L, RC, RS, SKIN, K=K, method="cells")
    n3 = oracle.cell_grid(L, RS, SKIN, K)
    u = oracle.quantize(x, L)
    c = (u.astype(np.uint64) * n3.astype(np.uint64)) >> np.uint64(32)
    c = c.astype(np.int64)

    def offsets(n):
        return list(range(-K, K + 1)) if n >= 2 * K + 1 else list(range(n))

    for i in range(0, 1000, 37):
        for kind in ("core", "shell", "full"):
            keys = []
            for j in lists.row(kind, i):
                idx = []
                for a in range(3):
                    offs = offsets(int(n3[a]))
                    idx.append([(c[i, a] + o) % n3[a] for o in offs].index(c[j, a]))
                slot = (idx[2] * len(offsets(int(n3[1]))) + idx[1]) * len(offsets(int(n3[0]))) + idx[0]
                keys.append((slot, int(u[j, 0]), int(j)))
            assert keys == sorted(keys)
