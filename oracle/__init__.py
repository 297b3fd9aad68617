"""FP64 CPU oracle for the random-batch list (RBL) force step (arXiv 2105.04884).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library.  The arithmetic lives in
``rbl_oracle.c`` (plain C, compiled with ``-ffp-contract=off``); this module only
builds it and marshals numpy arrays.  It shares nothing with the CUDA path.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``.  The
BAOAB step with friction is pinned step by step (the drift is the trapezoid of the
velocities around the O step, with and without forces; the zero-temperature free
flight has a closed form; the free-particle position variance is derived from the
splitting); long noisy trajectories are checked statistically (<v^2> -> T), since
their individual paths have nothing independent to compare with.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbl_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librbl_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (oracle/_build/)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["cc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
F = ctypes.c_float


def _declare(L):
    L.orc_set_threads.argtypes = [I]
    L.orc_set_threads.restype = None
    L.orc_max_threads.argtypes = []
    L.orc_max_threads.restype = I
    L.orc_philox4x32_10.argtypes = [P, P, P]
    L.orc_stream_words.argtypes = [U64, U64, U32, U32, I, P]
    L.orc_stream_uniform_below.argtypes = [U64, U64, U32, U32, U32, I, P]
    L.orc_batch_positions.argtypes = [U64, U64, U32, I, I, P]
    L.orc_batch_positions.restype = I
    L.orc_floyd_from_draws.argtypes = [I, I, P, P]
    L.orc_floyd_from_draws.restype = I
    L.orc_gaussians.argtypes = [U64, U64, U32, P]
    L.orc_quantize.argtypes = [I, P, P, P]
    L.orc_pair_r2f.argtypes = [I, P, P, P, P, P]
    L.orc_cell_grid.argtypes = [P, D, D, I, P]
    L.orc_cells.argtypes = [I, P, P, D, D, I, P]
    sig_lists = [I, P, P, D, D, D, I, I, I, I, P, P, P, P, P, P]
    L.orc_build_lists_brute.argtypes = sig_lists
    L.orc_build_lists_brute.restype = I
    L.orc_build_lists_cells.argtypes = sig_lists
    L.orc_build_lists_cells.restype = I
    L.orc_lj.argtypes = [I, P, P, P]
    L.orc_pair.argtypes = [I, P, D, D, P, P]
    L.orc_rbl_forces.argtypes = [I, P, P, D, D, D, I, U64, U64, P, P, I, P, P, I, P, P, P, P, P, D]
    L.orc_rbl_forces.restype = I
    L.orc_build_pool.argtypes = [I, P, P, D, D, D, I, I, P, P, P, P, P]
    L.orc_build_pool.restype = I
    L.orc_sample.argtypes = [I, P, P, D, D, D, I, I, U64, U64, I, P, I, I, P, P, P, P, P, P, P, P, D]
    L.orc_sample.restype = I
    L.orc_full_forces.argtypes = [I, P, P, D, P, P, I, P, P, P, D]
    L.orc_full_forces.restype = I
    L.orc_brute_forces.argtypes = [I, P, P, D, P, P, P, D]
    L.orc_subtract_mean.argtypes = [I, P]
    L.orc_run.argtypes = [I, P, P, P, P, D, D, D, I, I, D, D, D, U64, U64, I, I, I, I, I, I, P, P, D]
    L.orc_run.restype = I
    L.orc_tail.argtypes = [D, D, P]
    L.orc_thermo.argtypes = [I, P, P, D, P]
    L.orc_rdf_counts.argtypes = [I, P, P, F, I, P]
    L.orc_density_profile.argtypes = [I, P, P, I, I, P]


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# --------------------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def stream_words(seed, step, tag, stream, n):
    out = np.zeros(n, np.uint32)
    lib().orc_stream_words(seed, step, tag, stream, n, _p(out))
    return out


def stream_uniform_below(seed, step, tag, stream, s, n):
    out = np.zeros(n, np.uint32)
    lib().orc_stream_uniform_below(seed, step, tag, stream, s, n, _p(out))
    return out


def batch_positions(seed, step, tag, n_s, p):
    """Ascending Floyd sample of min(p, n_s) positions in [0, n_s)."""
    out = np.zeros(max(p, 1), np.int32)
    m = lib().orc_batch_positions(seed, step, tag, n_s, p, _p(out))
    return out[:m].copy()


def floyd_from_draws(n_s, p, draws):
    d = np.ascontiguousarray(draws, dtype=np.int32)
    out = np.zeros(p, np.int32)
    m = lib().orc_floyd_from_draws(n_s, p, _p(d), _p(out))
    return out[:m].copy()


def gaussians(seed, step, tag):
    out = np.zeros(3, np.float64)
    lib().orc_gaussians(seed, step, tag, _p(out))
    return out


# ------------------------------------------------------------------ geometry
def quantize(x, L):
    x = _f64(x, (-1, 3))
    Lv = _f64(L)
    u = np.zeros(x.shape, np.uint32)
    lib().orc_quantize(x.shape[0], _p(x), _p(Lv), _p(u))
    return u


def pair_r2f(u, L, i, j):
    u = np.ascontiguousarray(u, dtype=np.uint32)
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    Lv = _f64(L)
    out = np.zeros(i.shape[0], np.float32)
    lib().orc_pair_r2f(i.shape[0], _p(u), _p(Lv), _p(i), _p(j), _p(out))
    return out


def cell_grid(L, rs, skin, K):
    out = np.zeros(3, np.int32)
    lib().orc_cell_grid(_p(_f64(L)), rs, skin, K, _p(out))
    return out


def cells(u, L, rs, skin, K):
    u = np.ascontiguousarray(u, dtype=np.uint32)
    out = np.zeros(u.shape[0], np.int32)
    lib().orc_cells(u.shape[0], _p(u), _p(_f64(L)), rs, skin, K, _p(out))
    return out


class Lists:
    """Fixed-stride neighbour rows (tags), canonical (stencil slot, tag) order."""

    def __init__(self, core, n_core, shell, n_shell, full=None, n_full=None):
        self.core, self.n_core = core, n_core
        self.shell, self.n_shell = shell, n_shell
        self.full, self.n_full = full, n_full

    def row(self, kind, i):
        arr, cnt = getattr(self, kind), getattr(self, "n_" + kind)
        return arr[i, : cnt[i]]


def build_lists(x, L, rc, rs, skin, K=2, method="cells", cap_core=160, cap_shell=640, cap_full=640, full=True):
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    core = np.full((n, cap_core), -1, np.int32)
    shell = np.full((n, cap_shell), -1, np.int32)
    ncore = np.zeros(n, np.int32)
    nshell = np.zeros(n, np.int32)
    fl = np.full((n, cap_full), -1, np.int32) if full else None
    nfl = np.zeros(n, np.int32) if full else None
    fn = lib().orc_build_lists_brute if method == "brute" else lib().orc_build_lists_cells
    st = fn(n, _p(x), _p(_f64(L)), rc, rs, skin, K, cap_core, cap_shell, cap_full, _p(core), _p(ncore),
            _p(shell), _p(nshell), _p(fl), _p(nfl))
    if st != 0:
        raise OverflowError("oracle list row exceeded its capacity")
    return Lists(core, ncore, shell, nshell, fl, nfl)


# --------------------------------------------------------------------- forces
def lj(r):
    r = _f64(r)
    u = np.zeros_like(r)
    f = np.zeros_like(r)
    lib().orc_lj(r.shape[0], _p(r), _p(u), _p(f))
    return u, f


def _charges(q, n):
    """Charges as a contiguous float64 array of n, or None (LJ only)."""
    if q is None:
        return None
    q = _f64(q).reshape(-1)
    if q.shape[0] != n:
        raise ValueError("one charge per particle")
    return q


def pair(r, qq=0.0, alpha=0.0):
    """Energy and radial force magnitude of a pair at distances r: LJ plus, for
    qq = q_i q_j != 0, the Ewald real-space term qq erfc(alpha r) / r."""
    r = _f64(r)
    u = np.zeros_like(r)
    f = np.zeros_like(r)
    lib().orc_pair(r.shape[0], _p(r), float(qq), float(alpha), _p(u), _p(f))
    return u, f


def rbl_forces(x, L, rc, rs, skin, p, seed, step, lists, want_batch=False, q=None, alpha=0.0):
    """F_i = F_i,c + F~_i,s (no mean subtraction); returns (F, (U_est, W_est), batch, batch_n).
    q: per-particle charges for the LJ + Ewald real-space pair (None: LJ only)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    q = _charges(q, n)
    F = np.zeros((n, 3))
    ev = np.zeros(2)
    batch = np.full((n, max(p, 1)), -1, np.int32) if want_batch else None
    bn = np.zeros(n, np.int32) if want_batch else None
    lib().orc_rbl_forces(n, _p(x), _p(_f64(L)), rc, rs, skin, p, seed, step, _p(lists.core), _p(lists.n_core),
                         lists.core.shape[1], _p(lists.shell), _p(lists.n_shell), lists.shell.shape[1], _p(F),
                         _p(ev), _p(batch), _p(bn), _p(q), float(alpha))
    return F, ev, batch, bn


def build_pool(x, L, rc, rs, skin, cap_core=160, cap_pool=6000):
    """The paper's own sampling (Sec. 2): core rows and the stencil pool of every
    particle on the grid of edge >= r_c + skin; returned as Lists whose shell rows
    are the pools, so rbl_forces() evaluates the paper-literal estimator."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    core = np.full((n, cap_core), -1, np.int32)
    pool = np.full((n, cap_pool), -1, np.int32)
    nc = np.zeros(n, np.int32)
    npl = np.zeros(n, np.int32)
    gn = np.zeros(3, np.int32)
    st = lib().orc_build_pool(n, _p(x), _p(_f64(L)), rc, rs, skin, cap_core, cap_pool, _p(core), _p(nc), _p(pool),
                              _p(npl), _p(gn))
    if st != 0:
        raise OverflowError("oracle row exceeded its capacity")
    out = Lists(core, nc, pool, npl)
    out.grid = gn
    return out


class Sample:
    """Rows, batches and forces of sampled particles (see sample())."""

    def __init__(self, idx, core, n_core, shell, n_shell, batch, n_batch, F):
        self.idx = idx
        self.core, self.n_core, self.shell, self.n_shell = core, n_core, shell, n_shell
        self.batch, self.n_batch, self.F = batch, n_batch, F

    def row(self, kind, k):
        arr, cnt = getattr(self, kind), getattr(self, "n_" + kind)
        return arr[k, : cnt[k]]


def sample(x, L, rc, rs, skin, p, seed, step, idx, K=2, cap_core=160, cap_shell=640, q=None, alpha=0.0):
    """Core and shell rows (canonical order), batch at `step` and un-subtracted RBL
    force of the particles idx, each computed on its own against all the others."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    q = _charges(q, n)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    m = idx.shape[0]
    core = np.full((m, cap_core), -1, np.int32)
    shell = np.full((m, cap_shell), -1, np.int32)
    nc = np.zeros(m, np.int32)
    ns = np.zeros(m, np.int32)
    batch = np.full((m, max(p, 1)), -1, np.int32)
    nb = np.zeros(m, np.int32)
    F = np.zeros((m, 3))
    st = lib().orc_sample(n, _p(x), _p(_f64(L)), rc, rs, skin, K, p, seed, step, m, _p(idx), cap_core, cap_shell,
                          _p(core), _p(nc), _p(shell), _p(ns), _p(batch), _p(nb), _p(F), _p(q), float(alpha))
    if st != 0:
        raise OverflowError("oracle row exceeded its capacity")
    return Sample(idx, core, nc, shell, ns, batch, nb, F)


def full_forces(x, L, rs, lists, q=None, alpha=0.0):
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    q = _charges(q, n)
    F = np.zeros((n, 3))
    ev = np.zeros(2)
    lib().orc_full_forces(n, _p(x), _p(_f64(L)), rs, _p(lists.full), _p(lists.n_full), lists.full.shape[1],
                          _p(F), _p(ev), _p(q), float(alpha))
    return F, ev


def brute_forces(x, L, rs, q=None, alpha=0.0):
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    q = _charges(q, n)
    F = np.zeros((n, 3))
    ev = np.zeros(2)
    lib().orc_brute_forces(n, _p(x), _p(_f64(L)), rs, _p(F), _p(ev), _p(q), float(alpha))
    return F, ev


def subtract_mean(F):
    F = _f64(F, (-1, 3)).copy()
    lib().orc_subtract_mean(F.shape[0], _p(F))
    return F


def set_threads(n):
    """OpenMP threads for the oracle's loops (timing only)."""
    lib().orc_set_threads(int(n))


def max_threads():
    return int(lib().orc_max_threads())


def run(x, v, L, rc, rs, skin, p, dt, T, gamma, seed, n_steps, step0=0, K=2, subtract_mean=True,
        full_list=False, cap_core=160, cap_shell=640, cap_full=640, q=None, alpha=0.0):
    """Advance (x, v) by n_steps; returns (x, v, F, (U, W, n_rebuild))."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    n = x.shape[0]
    q = _charges(q, n)
    F = np.zeros((n, 3))
    stats = np.zeros(3)
    st = lib().orc_run(n, _p(x), _p(v), _p(F), _p(_f64(L)), rc, rs, skin, p, K, dt, T, gamma, seed, step0,
                       n_steps, int(subtract_mean), int(full_list), cap_core, cap_shell, cap_full, _p(stats),
                       _p(q), float(alpha))
    if st != 0:
        raise OverflowError("oracle list row exceeded its capacity")
    return x, v, F, stats


# ----------------------------------------------------------------- observables
def tail(rho, rs):
    out = np.zeros(2)
    lib().orc_tail(rho, rs, _p(out))
    return out


def thermo(v, L, W):
    v = _f64(v, (-1, 3))
    out = np.zeros(3)
    lib().orc_thermo(v.shape[0], _p(v), _p(_f64(L)), W, _p(out))
    return out


def rdf_counts(x, L, dr, nbins):
    x = _f64(x, (-1, 3))
    h = np.zeros(nbins, np.int64)
    lib().orc_rdf_counts(x.shape[0], _p(x), _p(_f64(L)), dr, nbins, _p(h))
    return h


def density_profile(x, L, axis, nbins):
    """Particle counts in nbins equal slabs along axis (fixed-point binning)."""
    x = _f64(x, (-1, 3))
    hist = np.zeros(nbins, np.int64)
    lib().orc_density_profile(x.shape[0], _p(x), _p(_f64(L)), int(axis), int(nbins), _p(hist))
    return hist
