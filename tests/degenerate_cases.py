"""Degenerate configurations for the edge-case tests (inputs only, no method arithmetic):
the smallest system (N = 2) with its pair at several distances, two clusters in a large
box with nearly every cell empty, and particles exactly on the box faces.  Each builder
returns (x, v, L, extra keyword arguments for the context)."""
import numpy as np

from paper_2105_04884_gb300 import inputs


def pair(d, face=False):
    """Two particles at distance d along the body diagonal (or, face=True, along x
    through the periodic face), in a box of 10, with opposite velocities."""
    L = np.full(3, 10.0)
    u = np.ones(3) / np.sqrt(3.0)
    if face:
        x = np.array([[0.3, 5.0, 5.0], [10.0 - (d - 0.3), 5.0, 5.0]])
    else:
        x = np.array([[2.0, 3.0, 4.0], [2.0, 3.0, 4.0] + d * u])
    v = np.array([[0.5, -0.2, 0.1], [-0.5, 0.2, -0.1]])
    return x, v, L, {}


def clusters():
    """Two 4 x 4 x 4 simple-cubic clusters (spacing 1.12, jitter 0.05) in a box of 25:
    one in the middle, one around the box corner."""
    g = np.stack(np.meshgrid(*[np.arange(4) * 1.12] * 3, indexing="ij"), -1).reshape(-1, 3) - 1.68
    rng = np.random.default_rng(12)
    L = np.full(3, 25.0)
    x = np.concatenate([g + 12.5, g]) + rng.uniform(-0.05, 0.05, (128, 3))
    x = np.mod(x, L)
    v = inputs.maxwell_boltzmann(128, 0.3, seed=12)
    return x, v, L, {"rho_cap": 1.0}


def faces():
    """FCC (N = 500, rho* = 0.8) moved so that lattice planes lie on the faces; of the
    particles within 0.06 of a face, every other one is put exactly on it: at 0 on the
    low side, at the largest double below L on the high side."""
    x, L = inputs.fcc(500, 0.8, 0.05, seed=11)
    x = np.mod(x - L / 5 / 4, L)
    for a in range(3):
        lo = np.nonzero(x[:, a] < 0.06)[0][::2]
        hi = np.nonzero(x[:, a] > L[a] - 0.06)[0][::2]
        assert len(lo) > 0 and len(hi) > 0
        x[lo, a] = 0.0
        x[hi, a] = np.nextafter(L[a], 0.0)
    v = inputs.maxwell_boltzmann(500, 1.5, seed=11)
    return x, v, L, {}


CASES = {
    "pair_core": lambda: pair(1.2),
    "pair_shell": lambda: pair(2.5),
    "pair_skin_band": lambda: pair(3.65),
    "pair_beyond": lambda: pair(4.5),
    "pair_core_through_face": lambda: pair(1.2, face=True),
    "clusters_empty_cells": clusters,
    "particles_on_faces": faces,
}
