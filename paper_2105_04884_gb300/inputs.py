"""Seeded synthetic inputs for LJ-fluid workloads (no method arithmetic here).

This module is the only code shared by the CUDA path's tests and benches and by the
CPU oracle's tests: it draws initial configurations, nothing else.  Random numbers
come from numpy's PCG64 seeded with the workload seed.

Workloads follow the LJ-fluid set-ups of the paper's Sec. 3 (reduced units,
sigma = epsilon = m = 1, periodic cubic box), widened to the sizes the library is
benchmarked at:

* ``fcc(N, rho, ...)``: face-centred cubic start, n = ceil((N/4)^(1/3)) unit cells a
  side, sites in lexicographic (ix, iy, iz, basis) order; when N < 4 n^3 the sites
  floor(k 4 n^3 / N), k = 0..N-1, are kept (evenly spread, so the start has the
  nominal density everywhere); lattice constant a = L/n with L = (N/rho)^(1/3),
  shifted by a/4 off the box faces, plus a uniform jitter of half-width ``jitter``
  per coordinate.
* ``maxwell_boltzmann(N, T, ...)``: N(0, sqrt(T)) components, mean removed, rescaled to
  exactly T with 3N - 3 degrees of freedom.
* ``slab(...)``: liquid FCC slab over the central fraction of z plus a uniform vapour.
* ``ensemble(...)``: independent replicas with log-uniform sizes and uniform densities
  and temperatures.
* ``charges(N, ...)``: a neutral set of charges +q / -q (half each, one 0 when N is
  odd) in random order, for the charged LJ fluid of the Ewald real-space workload.
* ``rock_salt(n, r0)``: the NaCl lattice, n^3 sites of a simple cubic lattice of
  spacing r0 with alternating unit charges.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def box_for(N: int, rho: float) -> float:
    return (N / rho) ** (1.0 / 3.0)


def fcc(N: int, rho: float, jitter: float = 0.01, seed: int = 1, L=None) -> tuple[np.ndarray, np.ndarray]:
    """(x[N,3] in [0, L), box lengths L[3]) for an FCC start with uniform jitter."""
    if L is None:
        L = np.full(3, box_for(N, rho))
    L = np.asarray(L, dtype=np.float64)
    n = int(math.ceil((N / 4.0) ** (1.0 / 3.0) - 1e-9))
    a = L / n
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    keep = (np.arange(N, dtype=np.int64) * sites.shape[0]) // N  # evenly spread subset
    sites = sites[keep]
    x = (sites + 0.25) * a
    if jitter > 0:
        x = x + _rng(seed, 2).uniform(-jitter, jitter, size=x.shape)
    x = np.mod(x, L)
    x[x >= L] -= L[np.nonzero(x >= L)[1]]
    return np.ascontiguousarray(x), L


def maxwell_boltzmann(N: int, T: float, seed: int = 1) -> np.ndarray:
    v = _rng(seed, 3).normal(0.0, math.sqrt(T), size=(N, 3))
    v -= v.mean(axis=0)
    t_now = (v * v).sum() / (3 * N - 3)
    if t_now > 0:
        v *= math.sqrt(T / t_now)
    return np.ascontiguousarray(v)


def uniform_gas(N: int, L, seed: int = 1) -> np.ndarray:
    L = np.asarray(L, dtype=np.float64)
    return np.ascontiguousarray(_rng(seed, 4).uniform(0.0, 1.0, size=(N, 3)) * L)


def slab(N: int, Lx: float, Lz: float, rho_liquid: float, rho_vapour: float, frac: float = 0.4,
         seed: int = 1, min_sep: float = 0.9) -> tuple[np.ndarray, np.ndarray]:
    """Liquid FCC slab over |z - Lz/2| < frac Lz / 2, vapour elsewhere.

    The liquid lattice constant gives density rho_liquid.  Vapour particles are a
    random subset of a simple cubic lattice of spacing 1.2 sigma (so no two start
    closer than 1 sigma), kept min_sep away from the slab faces.  The first N
    particles are kept (liquid first).
    """
    L = np.array([Lx, Lx, Lz], dtype=np.float64)
    a = (4.0 / rho_liquid) ** (1.0 / 3.0)
    n_xy = max(1, int(round(Lx / a)))
    a_xy = Lx / n_xy
    a_z = 4.0 / (rho_liquid * a_xy * a_xy)
    z_lo, z_hi = Lz / 2 - frac * Lz / 2, Lz / 2 + frac * Lz / 2
    n_z = int((z_hi - z_lo) / a_z)
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    ix, iy, iz = np.meshgrid(np.arange(n_xy), np.arange(n_xy), np.arange(n_z), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) + 0.25
    liquid = sites * np.array([a_xy, a_xy, a_z]) + np.array([0.0, 0.0, z_lo])
    rng = _rng(seed, 2)
    liquid += rng.uniform(-0.01, 0.01, size=liquid.shape)
    n_vap = max(0, N - liquid.shape[0])
    vap = np.zeros((0, 3))
    if n_vap:
        sp = 1.2
        gx = (np.arange(int(Lx / sp)) + 0.5) * (Lx / int(Lx / sp))
        gz = (np.arange(int(Lz / sp)) + 0.5) * (Lz / int(Lz / sp))
        gz = gz[(gz < z_lo - min_sep) | (gz > z_hi + min_sep)]
        gxx, gyy, gzz = np.meshgrid(gx, gx, gz, indexing="ij")
        grid = np.stack([gxx.ravel(), gyy.ravel(), gzz.ravel()], axis=1)
        pick = rng.choice(grid.shape[0], size=min(n_vap, grid.shape[0]), replace=False)
        vap = grid[np.sort(pick)] + rng.uniform(-0.1, 0.1, size=(len(pick), 3))
    x = np.concatenate([liquid, vap])[:N]
    x = np.mod(x, L)
    return np.ascontiguousarray(x), L


@dataclass
class Replica:
    N: int
    rho: float
    T: float
    seed: int
    x: np.ndarray = field(repr=False)
    v: np.ndarray = field(repr=False)
    L: np.ndarray = field(repr=False)


def ensemble(R: int = 256, n_min: int = 500, n_max: int = 20000, rho=(0.6, 0.9), T=(1.0, 2.0),
             seed: int = 1) -> list[Replica]:
    """R independent replicas: N log-uniform in [n_min, n_max], rho and T uniform; replica r
    uses seed + r for its own lattice jitter and velocities."""
    rng = _rng(seed, 5)
    out = []
    for r in range(R):
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        rh = float(rng.uniform(*rho))
        t = float(rng.uniform(*T))
        x, L = fcc(N, rh, 0.01, seed + r)
        v = maxwell_boltzmann(N, t, seed + r)
        out.append(Replica(N, rh, t, seed + r, x, v, L))
    return out


def charges(N: int, q: float = 1.0, seed: int = 1) -> np.ndarray:
    """Neutral charges: +q on half the particles, -q on the other half (and 0 on one
    particle when N is odd), in a seeded random order."""
    out = np.zeros(N, np.float64)
    h = N // 2
    out[:h] = q
    out[h : 2 * h] = -q
    return out[_rng(seed, 5).permutation(N)]


def rock_salt(n: int, r0: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(x, L, q): n^3 sites (n even) of a simple cubic lattice of spacing r0, offset
    by r0/2 from the box faces, with charge (-1)^(ix + iy + iz)."""
    if n % 2:
        raise ValueError("n must be even for a periodic rock-salt lattice")
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    idx = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1)
    x = (idx + 0.5) * r0
    q = np.where(idx.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return np.ascontiguousarray(x, dtype=np.float64), np.full(3, n * r0), q
