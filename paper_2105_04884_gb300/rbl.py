"""Thin ctypes binding of librbl (include/rbl.h): same names, argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies the device workspace
and the stream.  If the library has not been built the first call raises -- there
is no fallback path.

    sys = System(x, v, L, r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005, T=1.5, gamma=1.0)
    sys.step(100); obs = sys.observables(); F = sys.forces()

    ens = Ensemble([Replica(x0, v0, L0, T0, seed0), ...], r_c=1.5, r_s=3.5, skin=0.3, p=10, dt=0.005)
    ens.step(100); obs = ens.observables()  # one dict per replica

    # LJ plus the Ewald real-space term q_i q_j erfc(alpha r) / r
    sys = System(x, v, L, 1.5, 3.5, 0.3, 10, 0.005, potential=RBL_POT_LJ_EWALD, alpha=1.0, charges=q)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

RBL_FP64, RBL_FP32 = 0, 1
RBL_SAMPLE_SHELL, RBL_SAMPLE_STENCIL = 0, 1
RBL_POT_LJ, RBL_POT_LJ_EWALD = 0, 1
STATUS = {0: "RBL_OK", 1: "RBL_EINVAL", 2: "RBL_ENOMEM", 3: "RBL_EOVERFLOW", 4: "RBL_ENONFINITE",
          5: "RBL_ETIMEOUT", 6: "RBL_ECUDA"}


class RblError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class rbl_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3), ("r_c", ctypes.c_double), ("r_s", ctypes.c_double),
                ("skin", ctypes.c_double), ("p", ctypes.c_int), ("dt", ctypes.c_double), ("T", ctypes.c_double),
                ("gamma", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("precision", ctypes.c_int),
                ("full_list", ctypes.c_int), ("subtract_net_force", ctypes.c_int),
                ("cells_per_cutoff", ctypes.c_int), ("cap_core", ctypes.c_int), ("cap_stencil", ctypes.c_int),
                ("rho_cap", ctypes.c_double), ("sampling", ctypes.c_int), ("potential", ctypes.c_int),
                ("alpha", ctypes.c_double)]


class rbl_obs(ctypes.Structure):
    _fields_ = [("U_est", ctypes.c_double), ("W_est", ctypes.c_double), ("K", ctypes.c_double),
                ("T_kin", ctypes.c_double), ("P", ctypes.c_double), ("U_tail", ctypes.c_double),
                ("P_tail", ctypes.c_double), ("net_momentum", ctypes.c_double * 3), ("step", ctypes.c_longlong),
                ("n_rebuild", ctypes.c_longlong), ("Ns_mean", ctypes.c_double), ("Nc_mean", ctypes.c_double),
                ("Mc_mean", ctypes.c_double),
                ("Ns_max", ctypes.c_int), ("Nc_max", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["net_momentum"] = list(self.net_momentum)
        return d


EXPORTS = ["rbl_params_default", "rbl_workspace_size", "rbl_workspace_size_batch", "rbl_create",
           "rbl_create_batch", "rbl_replicas", "rbl_set_state", "rbl_set_charges", "rbl_get_state",
           "rbl_build_lists", "rbl_forces", "rbl_step", "rbl_step_async", "rbl_observables",
           "rbl_observables_async", "rbl_exact_energy", "rbl_get_lists", "rbl_get_rows", "rbl_get_batch",
           "rbl_rdf", "rbl_density_profile", "rbl_set_launch_config", "rbl_autotune", "rbl_set_phase_timing",
           "rbl_phase_times", "rbl_forces_static", "rbl_checkpoint_size", "rbl_save_checkpoint",
           "rbl_load_checkpoint", "rbl_destroy", "rbl_last_error", "rbl_status_string",
           "rbl_tune_cells_workspace_size", "rbl_tune_cells", "rbl_rebuild_times"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load librbl.so (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"librbl is not built ({path}); run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    L.rbl_params_default.argtypes = [ctypes.POINTER(rbl_params)]
    L.rbl_params_default.restype = None
    L.rbl_workspace_size.argtypes = [ctypes.POINTER(rbl_params), I, ctypes.POINTER(ctypes.c_size_t)]
    L.rbl_create.argtypes = [ctypes.POINTER(rbl_params), I, P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    L.rbl_workspace_size_batch.argtypes = [ctypes.POINTER(rbl_params), I, P, ctypes.POINTER(ctypes.c_size_t)]
    L.rbl_create_batch.argtypes = [ctypes.POINTER(rbl_params), I, P, P, ctypes.c_size_t, P, ctypes.POINTER(P)]
    L.rbl_replicas.argtypes = [P]
    L.rbl_set_state.argtypes = [P, P, P, LL, I]
    L.rbl_set_charges.argtypes = [P, P]
    L.rbl_get_state.argtypes = [P, P, P, ctypes.POINTER(LL), I]
    L.rbl_build_lists.argtypes = [P]
    L.rbl_forces.argtypes = [P, P, I]
    L.rbl_step.argtypes = [P, I]
    L.rbl_step_async.argtypes = [P, I]
    L.rbl_observables.argtypes = [P, ctypes.POINTER(rbl_obs)]
    L.rbl_observables_async.argtypes = [P, P, I]
    L.rbl_exact_energy.argtypes = [P, P, P]
    L.rbl_get_lists.argtypes = [P, I, P, I, P]
    L.rbl_get_rows.argtypes = [P, I, P, I, P, I, P]
    L.rbl_get_batch.argtypes = [P, LL, P, P]
    L.rbl_rdf.argtypes = [P, ctypes.c_float, I, P]
    L.rbl_density_profile.argtypes = [P, I, I, P]
    L.rbl_set_launch_config.argtypes = [P, I, I]
    L.rbl_autotune.argtypes = [P, I, P, P]
    L.rbl_set_phase_timing.argtypes = [P, I]
    L.rbl_phase_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(LL), I]
    L.rbl_rebuild_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(LL), I]
    L.rbl_forces_static.argtypes = [ctypes.POINTER(rbl_params), I, P, LL, P, P]
    L.rbl_checkpoint_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.rbl_save_checkpoint.argtypes = [P, P, I]
    L.rbl_load_checkpoint.argtypes = [P, P, I]
    L.rbl_destroy.argtypes = [P]
    L.rbl_destroy.restype = None
    L.rbl_last_error.argtypes = [P]
    L.rbl_last_error.restype = ctypes.c_char_p
    L.rbl_tune_cells_workspace_size.argtypes = [ctypes.POINTER(rbl_params), I, ctypes.POINTER(ctypes.c_size_t)]
    L.rbl_tune_cells.argtypes = [ctypes.POINTER(rbl_params), I, P, P, P, ctypes.c_size_t, P, I,
                                 ctypes.POINTER(ctypes.c_int), P]
    L.rbl_status_string.argtypes = [I]
    L.rbl_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("rbl_params_default", "rbl_destroy", "rbl_last_error", "rbl_status_string"):
            getattr(L, name).restype = I
    _lib = L
    return L


def make_params(L, r_c, r_s, skin, p, dt, T=1.0, gamma=0.0, seed=1, precision=RBL_FP32, full_list=False,
                subtract_net_force=True, cells_per_cutoff=2, cap_core=0, cap_stencil=0, rho_cap=0.0,
                sampling=RBL_SAMPLE_SHELL, potential=RBL_POT_LJ, alpha=0.0) -> rbl_params:
    prm = rbl_params()
    load().rbl_params_default(ctypes.byref(prm))
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,))
    for a in range(3):
        prm.L[a] = float(Lv[a])
    prm.r_c, prm.r_s, prm.skin, prm.p = r_c, r_s, skin, int(p)
    prm.dt, prm.T, prm.gamma, prm.seed = dt, T, gamma, int(seed)
    prm.precision = int(precision)
    prm.full_list = int(bool(full_list))
    prm.subtract_net_force = int(bool(subtract_net_force))
    prm.cells_per_cutoff = int(cells_per_cutoff)
    prm.cap_core, prm.cap_stencil = int(cap_core), int(cap_stencil)
    prm.rho_cap = float(rho_cap)
    prm.sampling = int(sampling)
    prm.potential = int(potential)
    prm.alpha = float(alpha)
    return prm


def tune_cells(x, v, L, r_c, r_s, skin, p, dt, steps=20, stream=None, device=None, **kw):
    """rbl_tune_cells: time the given system (host arrays x, v [N][3], tag order) at
    cells_per_cutoff K = 1, 2, 3 and return (fastest K, [ms per step for K = 1, 2, 3],
    -1 where a K does not apply).  The workspace is allocated here, as for a context;
    other keyword arguments are make_params's."""
    import torch

    lib = load()
    kw.pop("cells_per_cutoff", None)
    prm = make_params(L, r_c, r_s, skin, p, dt, **kw)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    N = int(x.shape[0])
    size = ctypes.c_size_t()
    st = lib.rbl_tune_cells_workspace_size(ctypes.byref(prm), N, ctypes.byref(size))
    if st != 0:
        raise RblError(st, lib.rbl_status_string(st).decode())
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    strm = stream if stream is not None else torch.cuda.Stream(dev)
    ws = torch.empty(int(size.value) + 256, dtype=torch.uint8, device=dev)
    aligned = (ws.data_ptr() + 255) & ~255
    K = ctypes.c_int()
    ms = (ctypes.c_float * 3)()
    st = lib.rbl_tune_cells(ctypes.byref(prm), N, _ptr(x), _ptr(v), ctypes.c_void_p(aligned), int(size.value),
                            ctypes.c_void_p(strm.cuda_stream), int(steps), ctypes.byref(K), ms)
    if st != 0:
        raise RblError(st, lib.rbl_status_string(st).decode())
    return K.value, [float(t) for t in ms]


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class _Context:
    """A librbl context on one CUDA device and a stream of its own; R replicas whose
    particle rows are packed one replica after another."""

    def _create(self, prms, Ns, stream, device):
        import torch

        self._torch = torch
        self.lib = load()
        self.R = len(prms)
        self.Ns = [int(n) for n in Ns]
        self.N = int(sum(self.Ns))
        self.prm = prms[0]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        # a stream of its own (the legacy default stream cannot host graph replays)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        arr = (rbl_params * self.R)(*prms)
        nn = (ctypes.c_int * self.R)(*self.Ns)
        size = ctypes.c_size_t()
        self.h = None
        self._check(self.lib.rbl_workspace_size_batch(arr, self.R, nn, ctypes.byref(size)))
        self.workspace = torch.empty(int(size.value) + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        h = ctypes.c_void_p()
        st = self.lib.rbl_create_batch(arr, self.R, nn, ctypes.c_void_p(aligned), int(size.value),
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        self.h = h
        if st != 0:
            msg = self.lib.rbl_last_error(h).decode() if h else ""
            self.lib.rbl_destroy(h)
            self.h = None
            raise RblError(st, msg)

    # -- plumbing
    def _check(self, st):
        if st != 0:
            msg = self.lib.rbl_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise RblError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.rbl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _is_dev(a):
        return hasattr(a, "data_ptr") and a.is_cuda

    # -- C-ABI calls
    def set_state(self, x, v=None, step=0):
        dev = self._is_dev(x)
        if dev:
            self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
        else:
            x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
            v = None if v is None else np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        self._check(self.lib.rbl_set_state(self.h, _ptr(x), _ptr(v), int(step), int(dev)))

    def set_charges(self, q):
        """Charges in tag order (packed over replicas), host array."""
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
        if q.shape[0] != self.N:
            raise ValueError(f"need {self.N} charges (got {q.shape[0]})")
        self._check(self.lib.rbl_set_charges(self.h, _ptr(q)))

    def get_state(self, device=False):
        if device:
            x = self._torch.empty((self.N, 3), dtype=self._torch.float64, device=self.device)
            v = self._torch.empty_like(x)
        else:
            x = np.empty((self.N, 3))
            v = np.empty((self.N, 3))
        step = ctypes.c_longlong()
        self._check(self.lib.rbl_get_state(self.h, _ptr(x), _ptr(v), ctypes.byref(step), int(device)))
        if device:
            self._torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return x, v, step.value

    def build_lists(self):
        self._check(self.lib.rbl_build_lists(self.h))

    def save_checkpoint(self, device=False):
        """The context's checkpoint (state, build-time images, step, rebuild counts) as a
        uint8 numpy array, or a uint8 tensor on the context's device."""
        n = ctypes.c_size_t()
        self._check(self.lib.rbl_checkpoint_size(self.h, ctypes.byref(n)))
        if device:
            buf = self._torch.empty(n.value, dtype=self._torch.uint8, device=self.device)
        else:
            buf = np.empty(n.value, np.uint8)
        self._check(self.lib.rbl_save_checkpoint(self.h, _ptr(buf), int(device)))
        return buf

    def load_checkpoint(self, buf):
        """Restore a checkpoint saved by a context of the same parameters and sizes."""
        dev = self._is_dev(buf)
        if dev:
            self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
        else:
            buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.rbl_load_checkpoint(self.h, _ptr(buf), int(dev)))

    def forces(self, out=None):
        if out is None:
            out = np.empty((self.N, 3))
        dev = self._is_dev(out)
        self._check(self.lib.rbl_forces(self.h, _ptr(out), int(dev)))
        if dev:
            self._torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out

    def step(self, n=1):
        self._check(self.lib.rbl_step(self.h, int(n)))

    def step_async(self, n=1):
        """Enqueue n steps without waiting (errors surface at the next synchronising call)."""
        self._check(self.lib.rbl_step_async(self.h, int(n)))

    def _observables(self):
        o = (rbl_obs * self.R)()
        self._check(self.lib.rbl_observables(self.h, o))
        return [o[r].as_dict() for r in range(self.R)]

    def observables_async(self, out):
        """Enqueue the observables into `out` (a page-locked uint8 tensor or array of
        R * sizeof(rbl_obs) bytes, e.g. from obs_buffer()) without waiting; read it
        with read_obs() after the stream has synchronised."""
        dev = self._is_dev(out)
        self._check(self.lib.rbl_observables_async(self.h, _ptr(out), int(dev)))

    def obs_buffer(self, pinned=True):
        """A host buffer for observables_async (page-locked by default)."""
        return self._torch.empty(self.R * ctypes.sizeof(rbl_obs), dtype=self._torch.uint8, pin_memory=pinned)

    def read_obs(self, buf):
        """Dicts from a buffer filled by observables_async (call after synchronising)."""
        raw = bytes(buf.numpy().tobytes()) if hasattr(buf, "numpy") else bytes(buf)
        arr = (rbl_obs * self.R).from_buffer_copy(raw)
        return [arr[r].as_dict() for r in range(self.R)]

    def synchronize(self):
        self.stream.synchronize()

    def _exact_energy(self):
        U = np.zeros(self.R)
        W = np.zeros(self.R)
        self._check(self.lib.rbl_exact_energy(self.h, _ptr(U), _ptr(W)))
        return U, W

    def get_lists(self, kind, cap=None):
        if cap is None:
            cap = max(int(o["Nc_max" if kind == 0 else "Ns_max"]) for o in self._observables()) + 1
        rows = np.full((self.N, cap), -1, np.int32)
        counts = np.zeros(self.N, np.int32)
        self._check(self.lib.rbl_get_lists(self.h, int(kind), _ptr(rows), int(cap), _ptr(counts)))
        return rows, counts

    def get_rows(self, kind, which, cap=None):
        """Rows of the particles `which` (packed row indices) only."""
        which = np.ascontiguousarray(which, dtype=np.int64)
        if cap is None:
            cap = max(int(o["Nc_max" if kind == 0 else "Ns_max"]) for o in self._observables()) + 1
        rows = np.full((len(which), cap), -1, np.int32)
        counts = np.zeros(len(which), np.int32)
        self._check(self.lib.rbl_get_rows(self.h, int(kind), _ptr(which), len(which), _ptr(rows), int(cap),
                                          _ptr(counts)))
        return rows, counts

    def get_batch(self, step):
        p = self.prm.p
        batch = np.full((self.N, p), -1, np.int32)
        counts = np.zeros(self.N, np.int32)
        self._check(self.lib.rbl_get_batch(self.h, int(step), _ptr(batch), _ptr(counts)))
        return batch, counts

    def set_launch_config(self, force_threads=128, build_warps=4):
        self._check(self.lib.rbl_set_launch_config(self.h, int(force_threads), int(build_warps)))

    def autotune(self, trials=5):
        """Pick the fastest launch shapes on the current state; returns them."""
        ft = ctypes.c_int()
        bw = ctypes.c_int()
        self._check(self.lib.rbl_autotune(self.h, int(trials), ctypes.byref(ft), ctypes.byref(bw)))
        return {"force_threads": ft.value, "build_warps": bw.value}

    def set_phase_timing(self, enable=True):
        self._check(self.lib.rbl_set_phase_timing(self.h, int(bool(enable))))

    def rebuild_times(self, reset=False):
        """(ms [cell sort chain, list build] summed over the rebuilds timed outside the
        step loop, their number)."""
        ms = (ctypes.c_double * 2)()
        n = ctypes.c_longlong()
        self._check(self.lib.rbl_rebuild_times(self.h, ms, ctypes.byref(n), int(bool(reset))))
        return list(ms), n.value

    def phase_times(self, reset=False):
        """(ms per phase [integrate, cell sort, list build, force kernel, force reduction],
        timed steps)."""
        ms = (ctypes.c_double * 5)()
        n = ctypes.c_longlong()
        self._check(self.lib.rbl_phase_times(self.h, ms, ctypes.byref(n), int(bool(reset))))
        return list(ms), n.value

    def _profile(self, axis, nbins, hist):
        self._check(self.lib.rbl_density_profile(self.h, int(axis), int(nbins), _ptr(hist)))
        return hist

    def _rdf(self, dr, nbins, hist):
        self._check(self.lib.rbl_rdf(self.h, float(dr), int(nbins), _ptr(hist)))
        return hist


class System(_Context):
    """One RBL (or full-list) system on the current CUDA device and stream."""

    def __init__(self, x, v, L, r_c, r_s, skin, p, dt, T=1.0, gamma=0.0, seed=1, precision=RBL_FP32,
                 full_list=False, subtract_net_force=True, cells_per_cutoff=2, cap_core=0, cap_stencil=0, step=0,
                 stream=None, device=None, rho_cap=0.0, sampling=RBL_SAMPLE_SHELL, potential=RBL_POT_LJ,
                 alpha=0.0, charges=None):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3) if not hasattr(x, "data_ptr") else x
        prm = make_params(L, r_c, r_s, skin, p, dt, T, gamma, seed, precision, full_list, subtract_net_force,
                          cells_per_cutoff, cap_core, cap_stencil, rho_cap, sampling, potential, alpha)
        self._create([prm], [int(x.shape[0])], stream, device)
        self.set_state(x, v, step)
        if charges is not None:
            self.set_charges(charges)

    def observables(self) -> dict:
        return self._observables()[0]

    def exact_energy(self):
        """(U, W): unsampled energy and virial sums over all pairs with r < r_s."""
        U, W = self._exact_energy()
        return float(U[0]), float(W[0])

    def rdf(self, dr, nbins, hist=None):
        if hist is None:
            hist = np.zeros(nbins, np.int64)
        return self._rdf(dr, nbins, hist)

    def density_profile(self, axis, nbins, hist=None):
        """Particle counts in nbins equal slabs along axis."""
        if hist is None:
            hist = np.zeros(nbins, np.int64)
        return self._profile(axis, nbins, hist)


class Replica:
    """One member of an ensemble: its state, box, bath temperature and seed."""

    def __init__(self, x, v, L, T, seed, q=None):
        self.x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        self.v = None if v is None else np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        self.L, self.T, self.seed = L, T, seed
        self.q = None if q is None else np.ascontiguousarray(q, dtype=np.float64).reshape(-1)


class Ensemble(_Context):
    """R independent replicas (own N, box, T and seed; shared radii, p, dt, gamma,
    precision) advanced together: one launch per kernel for all of them."""

    def __init__(self, replicas, r_c, r_s, skin, p, dt, gamma=0.0, precision=RBL_FP32, full_list=False,
                 subtract_net_force=True, cells_per_cutoff=2, cap_core=0, cap_stencil=0, step=0, stream=None,
                 device=None, rho_cap=0.0, sampling=RBL_SAMPLE_SHELL, potential=RBL_POT_LJ, alpha=0.0):
        prms = [make_params(rp.L, r_c, r_s, skin, p, dt, rp.T, gamma, rp.seed, precision, full_list,
                            subtract_net_force, cells_per_cutoff, cap_core, cap_stencil, rho_cap, sampling,
                            potential, alpha)
                for rp in replicas]
        self._create(prms, [len(rp.x) for rp in replicas], stream, device)
        self.offsets = np.concatenate([[0], np.cumsum(self.Ns)])
        x = np.concatenate([rp.x for rp in replicas])
        v = np.concatenate([rp.v if rp.v is not None else np.zeros_like(rp.x) for rp in replicas])
        self.set_state(x, v, step)
        if potential == RBL_POT_LJ_EWALD:  # replicas without charges (q None) get zeros
            q = [getattr(rp, "q", None) for rp in replicas]
            self.set_charges(np.concatenate([qr if qr is not None else np.zeros(len(rp.x))
                                             for qr, rp in zip(q, replicas)]))

    def split(self, a):
        """Packed per-particle rows -> list of per-replica arrays."""
        return [a[self.offsets[r]:self.offsets[r + 1]] for r in range(self.R)]

    def observables(self) -> list:
        return self._observables()

    def exact_energy(self):
        return self._exact_energy()

    def rdf(self, dr, nbins, hist=None):
        if hist is None:
            hist = np.zeros((self.R, nbins), np.int64)
        return self._rdf(dr, nbins, hist)

    def density_profile(self, axis, nbins, hist=None):
        if hist is None:
            hist = np.zeros((self.R, nbins), np.int64)
        return self._profile(axis, nbins, hist)
