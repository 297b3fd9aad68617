#!/usr/bin/env python3
"""Benchmark: particle-steps/s of the RBL step vs the full Verlet list on one GB300.

Workload (default): LJ fluid N = 1,048,576 (FCC 64^3 x 4), rho* = 0.8, T* = 1.5,
r_c = 1.5, r_s = 3.5, skin 0.3, p = 10, Langevin gamma = 1 (NVT), dt = 0.005,
FP32 pair math with int64 fixed-point force sums, FP64 integration.  One "step" is
one pass of the whole hot path: kick/drift/thermostat, device-conditional list
rebuild (cell hash, counting sort, scan, permute, two-level list build), RBL force,
force reduction.  Inputs are synthetic (seeded FCC start + Maxwell-Boltzmann).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle on the host
cores on the same workload (the paper's own implementation is unpublished).
Multi-GPU: independent replicas (one per rank, seed 1 + rank), weak scaling, no
collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s, RBL vs full Verlet list on 1 GB300 at matched pressure/g(r)"
WORKLOAD = dict(name="lj_fluid_N1048576_rho0.8_T1.5_rc1.5_rs3.5_skin0.3_p10_nvt", N=1048576, rho=0.8, T=1.5,
                rc=1.5, rs=3.5, skin=0.3, p=10, dt=0.005, gamma=1.0, K=2)
FORCE_KERNEL = "k_force<0, true, false, 10, false>"  # RBL, FP32, no energy, p = 10, LJ
FORCE_KERNEL_EWALD = "k_force<0, true, false, 10, true>"  # the same with the Ewald real-space term
EWALD_ALPHA = 1.0  # the charged fluid's splitting parameter: erfc(alpha r_s) = 7e-7 at r_s = 3.5
# Untimed steps between the start (FCC lattice) and every timed region, on top of
# --warmup: the rebuild rate settles within ~100 steps (one rebuild every ~5 steps at
# T* = 1.5), so the timed steps measure the steady state whatever --warmup is.
EQUIL_STEPS = 200


def phase_dict(pm, n):
    """Per-step milliseconds of the five timed phases (rbl_phase_times)."""
    names = ("integrate", "cell_sort", "list_build", "force_kernel", "force_reduce")
    return {k: pm[q] / n for q, k in enumerate(names)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-full-list", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune-cells", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=30)
    ap.add_argument("--no-physics", action="store_true", help="skip the matched-physics block")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble block")
    ap.add_argument("--no-slab", action="store_true", help="skip the liquid-vapour slab block")
    ap.add_argument("--no-ewald", action="store_true", help="skip the charged-fluid (Ewald real-space) block")
    ap.add_argument("--potential", default="lj", choices=["lj", "ewald"],
                    help="pair kernel of the timed workload: LJ, or LJ + Ewald real-space on the charged fluid")
    ap.add_argument("--ensemble-steps", type=int, default=200)
    ap.add_argument("--variance", action="store_true",
                    help="run the force-error variance study against the paper's Appendix A estimate")
    ap.add_argument("--table1", action="store_true",
                    help="run the paper's Table 1 study (g(r) first peak and MSD slope, classical cutoffs vs RBL)")
    ap.add_argument("--table1-scale", type=float, default=1.0, help="fraction of the paper's step counts")
    ap.add_argument("--ewald-physics", action="store_true",
                    help="run the matched-physics comparison for the charged fluid (Ewald real-space term)")
    ap.add_argument("--physics", action="store_true",
                    help="run the full matched-physics sweep (r_c x p x precision vs the full list) instead")
    ap.add_argument("--N", type=int, default=WORKLOAD["N"], help="override particle count (debug only)")
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    return a


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Multi-GPU: one independent replica per rank (weak scaling, no collective on the data
# path); the only collectives are the barriers around the timed region and the max of
# the ranks' times.
def replica_seed(rank):
    return 1 + rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(t, world, device):
    """The slowest rank's time (every rank gets it)."""
    if world == 1:
        return t
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(n_per_rank, steps, world, ms):
    """Particle-steps per second of the whole job: every rank's particles over the
    slowest rank's time."""
    return n_per_rank * steps * world / (ms * 1e-3)


class Clocks:
    """nvidia-smi sampler during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def step_roofline(alg_force, alg_build, N, ms_step, long_steps, ms_long, long_rebuilds, peak, world):
    """The fused step's algorithmic bytes per particle-step (alg_force - 24 + 96 + 16)
    and the list build's per-rebuild bytes amortised over the rebuild interval, against
    the HBM peak, for the timed K steps and the steady-state run."""
    step_bytes = alg_force - 24 + 96 + 16
    interval = long_steps / max(long_rebuilds, 1)
    amort = alg_build / interval
    out = {"algorithmic_bytes_per_particle_step": step_bytes, "rebuild_interval_steps": interval,
           "rebuild_bytes_amortised_per_step": amort, "peak": peak, "unit": "GB/s"}
    for key, ms in (("timed", ms_step), ("steady_state", ms_long / long_steps)):
        achieved = (step_bytes + amort) * N / (ms * 1e-3) / 1e9
        out[key] = {"ms_per_step": ms, "achieved": achieved, "frac": achieved / peak}
    out["ceiling_particle_steps_per_s"] = peak * 1e9 / (step_bytes + amort) * world
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic(N, name="force_kernel_traffic.json"):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if it was taken
    on the current sources of that kernel (the record names the digest it depends on:
    _build.force_digest by default, or _build.build_digest), else None.  The figure is
    per particle: traffic grows in proportion to N."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as fh:
            d = json.load(fh)
        from paper_2105_04884_gb300 import _build

        digest = getattr(_build, d.get("digest", "force_digest"))
        if d.get("source_sha") != digest():
            return None
        return float(d["dram_bytes_per_particle"]) * N
    except Exception:
        return None


# Matched-physics study: LJ fluid N = 32,000 (FCC 20^3 x 4), rho* = 0.8442, T* = 1.2,
# Langevin gamma = 1, dt = 0.005, r_s = 3.5, skin 0.3; 10^4 steps, the first 2000
# discarded, block averages over blocks of 500 steps.
PHYS = dict(N=32000, rho=0.8442, T=1.2, rs=3.5, skin=0.3, dt=0.005, gamma=1.0, K=2, steps=10000, discard=2000,
            block=500, stride=10, rdf_every=5, dr=0.02)


def physics_run(x, v, L, rc, p, precision, full, seed, cfg=PHYS, sampling=0, charges=None, alpha=0.0):
    """Block-averaged observables of one NVT trajectory.  Pressure and energy are the
    exact (unsampled) ones of the configurations the dynamics visits: P = rho T_kin +
    W / (3V) and U / N with W, U over every pair with r < r_s; the RBL estimates of the
    same quantities are reported beside them.  g(r) from ordered-pair counts.
    charges: the charged fluid (pair LJ + q_i q_j erfc(alpha r) / r)."""
    import numpy as np

    from paper_2105_04884_gb300 import rbl

    N = len(x)
    V = float(np.prod(L))
    rho = N / V
    pot = {} if charges is None else dict(potential=rbl.RBL_POT_LJ_EWALD, alpha=alpha, charges=charges)
    s = rbl.System(x, v, L, r_c=rc, r_s=cfg["rs"], skin=cfg["skin"], p=p, dt=cfg["dt"], T=cfg["T"],
                   gamma=cfg["gamma"], seed=seed, cells_per_cutoff=cfg["K"], precision=precision, full_list=full,
                   sampling=0 if full else sampling, **pot)
    nbins = int(round(cfg["rs"] / cfg["dr"]))
    s.step(cfg["discard"])
    nblk = (cfg["steps"] - cfg["discard"]) // cfg["block"]
    per = cfg["block"] // cfg["stride"]
    blocks = {k: [] for k in ("P", "P_bath", "U", "T", "P_est", "U_est")}
    g_blocks = []
    shell = 4.0 / 3.0 * math.pi * (np.arange(1, nbins + 1) ** 3 - np.arange(nbins) ** 3) * cfg["dr"] ** 3
    t0 = time.perf_counter()
    for _ in range(nblk):
        acc = {k: 0.0 for k in blocks}
        h = np.zeros(nbins, np.int64)
        nr = 0
        for k in range(per):
            s.step(cfg["stride"])
            U, W = s.exact_energy()
            o = s.observables()
            acc["P"] += rho * o["T_kin"] + W / (3 * V)
            acc["P_bath"] += rho * cfg["T"] + W / (3 * V)  # Sec. 3: rho / beta + virial
            acc["U"] += U / N
            acc["T"] += o["T_kin"]
            acc["P_est"] += rho * o["T_kin"] + o["W_est"] / (3 * V)
            acc["U_est"] += o["U_est"] / N
            if (k + 1) % cfg["rdf_every"] == 0:
                s.rdf(cfg["dr"], nbins, h)
                nr += 1
        for k in blocks:
            blocks[k].append(acc[k] / per)
        g_blocks.append(h / (nr * N * rho * shell))
    wall = time.perf_counter() - t0
    heating = None
    if not full:
        # numerical heating check: the per-particle variance of the RBL force error
        # chi = F_rbl - F_exact at the final configuration predicts, for BAOAB with
        # friction gamma, a kinetic temperature excess dT = dt <|chi|^2> / (6 gamma)
        xs, vs, _ = s.get_state()
        F_rbl = s.forces()
        ref = rbl.System(xs, vs, L, r_c=rc, r_s=cfg["rs"], skin=cfg["skin"], p=p, dt=cfg["dt"], T=cfg["T"],
                         gamma=cfg["gamma"], seed=seed, cells_per_cutoff=cfg["K"], precision=precision,
                         full_list=True, **pot)
        F_ex = ref.forces()
        var = float(np.mean(np.sum((F_rbl - F_ex) ** 2, axis=1)))
        heating = {"force_err_var": var, "dT_predicted": cfg["dt"] * var / (6.0 * cfg["gamma"])}
        del ref
    out = {"heating": heating}
    for k, b in blocks.items():
        b = np.asarray(b)
        out[k] = [float(b.mean()), float(b.std(ddof=1) / math.sqrt(len(b)))]
    g = np.asarray(g_blocks)
    out["g"] = g.mean(0)
    out["g_err"] = g.std(0, ddof=1) / math.sqrt(len(g))
    out["wall_s"] = wall
    out["n_rebuild"] = s.observables()["n_rebuild"]
    return out


def physics_compare(a, b, dr):
    """z-scores of the scalar differences (combined block-average errors) and the
    reduced chi^2 of the g(r) difference over bins where g > 0.05."""
    import numpy as np

    res = {}
    for k in ("P", "P_bath", "U", "T"):
        d = a[k][0] - b[k][0]
        e = math.hypot(a[k][1], b[k][1])
        res[k] = {"rbl": a[k], "full": b[k], "z": d / e if e > 0 else None}
    m = (a["g"] > 0.05) | (b["g"] > 0.05)
    var = a["g_err"][m] ** 2 + b["g_err"][m] ** 2
    ok = var > 0
    chi2 = float(np.mean((a["g"][m][ok] - b["g"][m][ok]) ** 2 / var[ok]))
    ia, ib = int(np.argmax(a["g"])), int(np.argmax(b["g"]))
    res["g"] = {"chi2_per_bin": chi2, "bins": int(ok.sum()), "dr": dr,
                "peak_rbl": [float(a["g"][ia]), float(a["g_err"][ia]), (ia + 0.5) * dr],
                "peak_full": [float(b["g"][ib]), float(b["g_err"][ib]), (ib + 0.5) * dr],
                "max_abs_diff": float(np.max(np.abs(a["g"] - b["g"])))}
    return res


ENSEMBLE = dict(R=256, rc=1.5, rs=3.5, skin=0.3, p=10, dt=0.005, gamma=1.0, K=2)


def ensemble_bench(a, rank, world, timed):
    """Batched ensemble: 256 replicas, N log-uniform in [500, 20000], rho* in
    [0.6, 0.9], T* in [1, 2], FP32, one launch per kernel for all replicas and one
    graph per step; beside it the same replicas as 256 separate contexts stepped
    one after another (the unbatched alternative, fewer steps)."""
    import torch

    from paper_2105_04884_gb300 import inputs, rbl

    e = ENSEMBLE
    reps = inputs.ensemble(e["R"], seed=replica_seed(rank))
    shared = dict(r_c=e["rc"], r_s=e["rs"], skin=e["skin"], p=e["p"], dt=e["dt"], gamma=e["gamma"],
                  cells_per_cutoff=e["K"], precision=rbl.RBL_FP32)
    ntot = sum(rp.N for rp in reps)
    ens = rbl.Ensemble(reps, **shared)
    ens.step(a.warmup + EQUIL_STEPS)
    ens_cfg = ens.autotune(trials=3)
    K = a.ensemble_steps
    ms, _ = timed(ens, K, phases=False)
    obs = ens.observables()
    del ens
    torch.cuda.empty_cache()
    # unbatched: one context per replica, each stepped k times in turn
    k = max(3, K // 10)
    singles = [rbl.System(rp.x, rp.v, rp.L, T=rp.T, seed=rp.seed, **shared) for rp in reps]
    for s1 in singles:
        s1.step(a.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s1 in singles:
        s1.step(k)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    del singles
    torch.cuda.empty_cache()
    return {"workload": "lj_ensemble_R256_N500-20000_rho0.6-0.9_T1-2_rc1.5_rs3.5_p10_nvt", "replicas": e["R"],
            "particles": ntot, "steps": K, "value": whole_job_rate(ntot, K, world, ms), "unit": "particle-steps/s",
            "ms_per_step": ms / K, "rebuilds_per_replica_mean": sum(o["n_rebuild"] for o in obs) / e["R"],
            "launch_config": ens_cfg,
            "separate_contexts": {"value": ntot * k / t_single, "steps": k,
                                  "ms_per_step": t_single * 1e3 / k}}


SLAB = dict(N=4194304, rho_l=0.75, rho_v=0.01, frac=0.4, T=0.9, rc=1.5, rs=4.0, skin=0.3, p=20, dt=0.005,
            gamma=1.0, K=2, steps=500, dz=0.5)


def slab_bench(a, rank, world, timed):
    """Liquid-vapour slab: N = 4,194,304 in Lx = Ly, Lz = 4 Lx, liquid rho* = 0.75
    over the central 40% of z, vapour 0.01 elsewhere, T* = 0.9, r_c = 1.5, r_s = 4.0,
    p = 20, FP32; 500 steps of RBL and of the full list from the same start, then
    the z density profile (0.5 sigma bins) of both, averaged over 5 more samples
    10 steps apart."""
    import numpy as np
    import torch

    from paper_2105_04884_gb300 import inputs, rbl

    c = SLAB
    V = c["N"] / (c["rho_l"] * c["frac"] + c["rho_v"] * (1.0 - c["frac"]))
    Lx = (V / 4.0) ** (1.0 / 3.0)
    x, L = inputs.slab(c["N"], Lx, 4.0 * Lx, c["rho_l"], c["rho_v"], c["frac"], seed=replica_seed(rank))
    v = inputs.maxwell_boltzmann(len(x), c["T"], seed=replica_seed(rank))
    nb = int(round(L[2] / c["dz"]))
    common = dict(r_c=c["rc"], r_s=c["rs"], skin=c["skin"], p=c["p"], dt=c["dt"], T=c["T"], gamma=c["gamma"],
                  seed=replica_seed(rank), cells_per_cutoff=c["K"], precision=rbl.RBL_FP32, rho_cap=c["rho_l"])
    out = {"workload": "lj_slab_N4194304_rhoL0.75_rhoV0.01_T0.9_rc1.5_rs4.0_p20_nvt", "N": len(x),
           "box": [float(L[0]), float(L[1]), float(L[2])], "steps": c["steps"]}
    prof = {}
    for name, full in (("rbl", False), ("full_list", True)):
        s = rbl.System(x, v, L, full_list=full, **common)
        s.step(3)
        s.autotune(trials=2)
        ms, _ = timed(s, c["steps"], phases=False)
        h = np.zeros(nb, np.int64)
        for _ in range(5):
            s.step(10)
            s.density_profile(2, nb, h)
        prof[name] = h / 5.0 / (L[0] * L[1] * c["dz"])
        out[name] = {"value": whole_job_rate(len(x), c["steps"], world, ms), "unit": "particle-steps/s",
                     "ms_per_step": ms / c["steps"], "T_kin": s.observables()["T_kin"]}
        del s
        torch.cuda.empty_cache()
    z = (np.arange(nb) + 0.5) * c["dz"]
    liquid = np.abs(z - L[2] / 2) < 0.3 * c["frac"] * L[2]
    vapour = np.abs(z - L[2] / 2) > (0.5 * c["frac"] + 0.1) * L[2]
    for name in prof:
        out[name]["rho_liquid"] = float(prof[name][liquid].mean())
        out[name]["rho_vapour"] = float(prof[name][vapour].mean())
    # per-bin difference in units of the bins' counting noise (Poisson, both runs)
    cnt = L[0] * L[1] * c["dz"] * 5.0
    sig = np.sqrt((prof["rbl"] + prof["full_list"]) / cnt + 1e-12)
    out["profile_max_abs_diff"] = float(np.max(np.abs(prof["rbl"] - prof["full_list"])))
    out["profile_rms_z"] = float(np.sqrt(np.mean(((prof["rbl"] - prof["full_list"]) / sig) ** 2)))
    out["speedup_vs_full_list"] = out["rbl"]["value"] / out["full_list"]["value"]
    return out


def physics_inputs(seed=1, cfg=PHYS):
    from paper_2105_04884_gb300 import inputs

    x, L = inputs.fcc(cfg["N"], cfg["rho"], 0.01, seed=seed)
    v = inputs.maxwell_boltzmann(cfg["N"], cfg["T"], seed=seed)
    return x, v, L


def matched_physics_pair(rc=1.5, p=10, cfg=PHYS, full=None, sampling=0):
    """RBL (FP32, r_c, p; shell list or stencil pool) against the full list (FP32)
    on the same start."""
    from paper_2105_04884_gb300 import rbl

    x, v, L = physics_inputs(cfg=cfg)
    a = physics_run(x, v, L, rc, p, rbl.RBL_FP32, False, 1, cfg, sampling=sampling)
    b = full if full is not None else physics_run(x, v, L, rc, p, rbl.RBL_FP32, True, 1, cfg)
    res = physics_compare(a, b, cfg["dr"])
    res["workload"] = "lj_fluid_N32000_rho0.8442_T1.2_rs3.5_nvt"
    res["r_c"], res["p"] = rc, p
    res["sampling"] = "stencil_pool" if sampling else "shell_list"
    res["steps"], res["discard"], res["block"] = cfg["steps"], cfg["discard"], cfg["block"]
    res["P_est_rbl"] = a["P_est"]
    res["U_est_rbl"] = a["U_est"]
    if a["heating"]:
        res["heating"] = dict(a["heating"], dT_measured=a["T"][0] - b["T"][0])
    res["wall_s"] = a["wall_s"] + b["wall_s"]
    return res, b


def ewald_physics_sweep(alpha=EWALD_ALPHA):
    """The matched-physics comparison for the charged fluid (the matched-physics system
    with neutral random +-1 charges, pair LJ + q_i q_j erfc(alpha r) / r): RBL at
    r_c in {1.5, 2.0, 2.5} x p in {10, 20} against the full list, FP32.  One JSON line
    per run."""
    from paper_2105_04884_gb300 import inputs, rbl

    x, v, L = physics_inputs()
    q = inputs.charges(len(x), 1.0, seed=1)
    ch = dict(charges=q, alpha=alpha)
    ref = physics_run(x, v, L, 1.5, 10, rbl.RBL_FP32, True, 1, **ch)
    print(json.dumps({"potential": "lj+ewald", "alpha": alpha, "method": "full", "P": ref["P"], "U": ref["U"],
                      "T": ref["T"], "wall_s": ref["wall_s"]}), flush=True)
    for rc in (1.5, 2.0, 2.5):
        for p in (10, 20):
            r = physics_run(x, v, L, rc, p, rbl.RBL_FP32, False, 1, **ch)
            c = physics_compare(r, ref, PHYS["dr"])
            c.update({"potential": "lj+ewald", "alpha": alpha, "method": "rbl", "r_c": rc, "p": p,
                      "wall_s": r["wall_s"], "n_rebuild": r["n_rebuild"],
                      "heating": dict(r["heating"], dT_measured=r["T"][0] - ref["T"][0])})
            print(json.dumps(c), flush=True)


def physics_sweep():
    """The full study: r_c in {1.2, 1.5, 2.0} x p in {1, 2, 5, 10, 20}, FP32 and FP64,
    each against the full list of the same precision.  One JSON line per run."""
    from paper_2105_04884_gb300 import rbl

    x, v, L = physics_inputs()
    for prec, name in ((rbl.RBL_FP32, "fp32"), (rbl.RBL_FP64, "fp64")):
        ref = physics_run(x, v, L, 1.5, 10, prec, True, 1)
        print(json.dumps({"precision": name, "method": "full", "P": ref["P"], "U": ref["U"], "T": ref["T"],
                          "wall_s": ref["wall_s"]}), flush=True)
        for rc in (1.2, 1.5, 2.0):
            for p in (1, 2, 5, 10, 20):
                r = physics_run(x, v, L, rc, p, prec, False, 1)
                c = physics_compare(r, ref, PHYS["dr"])
                c.update({"precision": name, "method": "rbl", "r_c": rc, "p": p, "P_est": r["P_est"],
                          "U_est": r["U_est"], "wall_s": r["wall_s"], "n_rebuild": r["n_rebuild"],
                          "heating": dict(r["heating"], dT_measured=r["T"][0] - ref["T"][0])})
                print(json.dumps(c), flush=True)
        # the paper's own pool (every particle of the cell stencil), same comparison
        for rc in (1.2, 1.5, 2.0):
            for p in (10, 20):
                r = physics_run(x, v, L, rc, p, prec, False, 1, sampling=rbl.RBL_SAMPLE_STENCIL)
                c = physics_compare(r, ref, PHYS["dr"])
                c.update({"precision": name, "method": "rbl_stencil_pool", "r_c": rc, "p": p, "P_est": r["P_est"],
                          "U_est": r["U_est"], "wall_s": r["wall_s"], "n_rebuild": r["n_rebuild"],
                          "heating": dict(r["heating"], dT_measured=r["T"][0] - ref["T"][0])})
                print(json.dumps(c), flush=True)


# The paper's Table 1 study (Sec. 3): N = 2000, rho* = 0.2, T* = 0.9 (gas-liquid
# coexistence), tau = 0.002, Langevin gamma = 1, 2x10^5 equilibration and 10^5
# production steps, 10 runs; g(r) first peak and MSD slope for classical cutoffs
# r_s = 6, 3, 2 and for RBL with r_s = 6, r_c = 2, p = 10, 20, 50, 100.  The ten
# runs are one ensemble of ten replicas (seeds 100..109).
TABLE1 = dict(N=2000, rho=0.2, T=0.9, dt=0.002, gamma=1.0, skin=0.3, runs=10, equil=200000, prod=100000,
              stride=100, rdf_every=10, dr=0.02, rmax=1.98)
TABLE1_PAPER = {  # Table 1 of the paper: (g(r) first peak, MSD slope)
    "DT r_s=6": (7.0196, 2.1117), "DT r_s=3": (6.1095, 2.4668), "DT r_s=2": (2.6592, 3.7144),
    "RBL p=10": (7.1532, 2.2367), "RBL p=20": (7.0849, 2.0303), "RBL p=50": (7.0366, 2.1669),
    "RBL p=100": (7.0141, 2.1348)}


def table1_study(scale=1.0):
    import numpy as np

    from paper_2105_04884_gb300 import inputs, rbl

    c = TABLE1
    reps = []
    for r in range(c["runs"]):
        x, L = inputs.fcc(c["N"], c["rho"], 0.01, seed=100 + r)
        v = inputs.maxwell_boltzmann(c["N"], c["T"], seed=100 + r)
        reps.append(rbl.Replica(x, v, L, c["T"], 100 + r))
    L = reps[0].L
    V = float(np.prod(L))
    rho = c["N"] / V
    nb = int(round(c["rmax"] / c["dr"]))
    shell = 4.0 / 3.0 * math.pi * (np.arange(1, nb + 1) ** 3 - np.arange(nb) ** 3) * c["dr"] ** 3
    configs = [("DT r_s=6", dict(full_list=True, r_c=1.0, r_s=6.0, p=10)),
               ("DT r_s=3", dict(full_list=True, r_c=1.0, r_s=3.0, p=10)),
               ("DT r_s=2", dict(full_list=True, r_c=1.0, r_s=2.0, p=10))]
    configs += [(f"RBL p={p}", dict(full_list=False, r_c=2.0, r_s=6.0, p=p)) for p in (10, 20, 50, 100)]
    n_eq = int(c["equil"] * scale)
    n_pr = int(c["prod"] * scale) // c["stride"] * c["stride"]
    for name, cfg in configs:
        t0 = time.perf_counter()
        # the gas condenses into liquid droplets (rho* ~ 0.75): size the rows for them
        ens = rbl.Ensemble(reps, skin=c["skin"], dt=c["dt"], gamma=c["gamma"], precision=rbl.RBL_FP32,
                           rho_cap=0.8, **cfg)
        ens.step(n_eq)
        x0 = ens.get_state()[0]
        prev, unwrapped = x0.copy(), x0.copy()
        hist = np.zeros((c["runs"], nb), np.int64)
        nrdf = 0
        msd = []
        for k in range(n_pr // c["stride"]):
            ens.step(c["stride"])
            x = ens.get_state()[0]
            d = x - prev
            d -= L * np.round(d / L)
            unwrapped += d
            prev = x
            disp = ((unwrapped - x0) ** 2).sum(axis=1).reshape(c["runs"], c["N"]).mean(axis=1)
            msd.append(disp)
            if (k + 1) % c["rdf_every"] == 0:
                ens.rdf(c["dr"], nb, hist)
                nrdf += 1
        msd = np.asarray(msd)                                 # [samples][runs]
        t = (np.arange(1, len(msd) + 1) * c["stride"]) * c["dt"]
        keep = t >= 0.1 * t[-1]                               # past the ballistic start
        slopes = np.array([np.polyfit(t[keep], msd[keep, r], 1)[0] for r in range(c["runs"])])
        g = hist / (nrdf * c["N"] * rho * shell)              # [runs][bins]
        peaks = g.max(axis=1)
        out = {"config": name, "runs": c["runs"], "equil_steps": n_eq, "prod_steps": n_pr,
               "g_peak": [float(peaks.mean()), float(peaks.std(ddof=1) / math.sqrt(c["runs"]))],
               "g_peak_r": float((np.argmax(g.mean(axis=0)) + 0.5) * c["dr"]),
               "msd_slope": [float(slopes.mean()), float(slopes.std(ddof=1) / math.sqrt(c["runs"]))],
               "paper_g_peak": TABLE1_PAPER[name][0], "paper_msd_slope": TABLE1_PAPER[name][1],
               "wall_s": time.perf_counter() - t0}
        print(json.dumps(out), flush=True)
        del ens


def variance_study(draws=8):
    """Variance of the force error chi_i = F~_i - F_i (Appendix A) on one equilibrated
    liquid configuration (the matched-physics system: N = 32,000, rho* = 0.8442,
    T* = 1.2, r_s = 3.5), for r_c in {1.2, 1.5, 2.0, 2.5}, p in {5, 10, 20} and both
    pools, over `draws` independent batches (different step counters), FP64.  Beside
    the measurement: Appendix A's leading term (N - p)/p * int_{r_c}^{r_s} 4 pi rho r^2
    f(r)^2 dr with N the mean pool (N_s or N_I) and g = 1 as the paper assumes, and the
    same integral weighted by the measured g(r)."""
    import numpy as np

    from paper_2105_04884_gb300 import rbl

    cfg = PHYS
    x, v, L = physics_inputs()
    rho = len(x) / float(np.prod(L))
    eq = rbl.System(x, v, L, r_c=1.5, r_s=cfg["rs"], skin=cfg["skin"], p=10, dt=cfg["dt"], T=cfg["T"],
                    gamma=cfg["gamma"], seed=1, full_list=True, precision=rbl.RBL_FP64)
    eq.step(2000)
    xs, vs, _ = eq.get_state()
    F_full = eq.forces()
    dr = 0.01
    nb = int(round(cfg["rs"] / dr)) - 1
    h = eq.rdf(dr, nb)
    r = (np.arange(nb) + 0.5) * dr
    g = h / (len(x) * rho * 4.0 / 3.0 * np.pi * ((r + dr / 2) ** 3 - (r - dr / 2) ** 3))
    f2 = (24.0 * (2.0 * r ** -13 - r ** -7)) ** 2
    del eq
    for mode, name in ((rbl.RBL_SAMPLE_SHELL, "shell_list"), (rbl.RBL_SAMPLE_STENCIL, "stencil_pool")):
        for rc in (1.2, 1.5, 2.0, 2.5):
            for p in (5, 10, 20):
                s = rbl.System(xs, vs, L, r_c=rc, r_s=cfg["rs"], skin=cfg["skin"], p=p, dt=cfg["dt"], T=cfg["T"],
                               gamma=cfg["gamma"], seed=7, precision=rbl.RBL_FP64, sampling=mode)
                acc = 0.0
                for k in range(draws):
                    s.set_state(xs, vs, step=1000 + k)
                    acc += float(np.mean(np.sum((s.forces() - F_full) ** 2, axis=1)))
                meas = acc / draws
                npool = s.observables()["Ns_mean"]
                win = (r >= rc) & (r < cfg["rs"])
                integ = np.sum(4.0 * np.pi * rho * r[win] ** 2 * f2[win]) * dr
                integ_g = np.sum(4.0 * np.pi * rho * r[win] ** 2 * g[win] * f2[win]) * dr
                fac = (npool - p) / p
                print(json.dumps({"sampling": name, "r_c": rc, "p": p, "pool_mean": npool, "var_chi": meas,
                                  "appendix_g1": fac * integ, "appendix_with_g": fac * integ_g,
                                  "ratio_meas_over_g": meas / (fac * integ_g)}), flush=True)
                del s


def ewald_bench(a, world, x, v, L, common, timed):
    """The Ewald real-space extension on the headline workload's positions: the same
    fluid with neutral random +-1 charges, pair LJ + q_i q_j erfc(alpha r) / r; RBL
    against the full list, both autotuned."""
    import torch

    from paper_2105_04884_gb300 import inputs, rbl

    N = len(x)
    q = inputs.charges(N, 1.0, seed=common["seed"])
    ew = dict(common, potential=rbl.RBL_POT_LJ_EWALD, alpha=EWALD_ALPHA)
    out = {"workload": "charged LJ fluid: headline positions + neutral random +-1 charges", "alpha": EWALD_ALPHA}
    for name, kw in (("rbl", {}), ("full_list", {"full_list": True})):
        s = rbl.System(x, v, L, charges=q, **dict(ew, **kw))
        s.step(a.warmup + EQUIL_STEPS)
        s.autotune(trials=3)
        _, (pm, n) = timed(s, a.steps, phases=True)
        ms, _ = timed(s, a.steps, phases=False)
        out[name] = {"value": whole_job_rate(N, a.steps, world, ms), "ms_per_step": ms / a.steps,
                     "force_kernel_ms": pm[3] / n, "rebuild_chain_ms": (pm[1] + pm[2]) / n}
        del s
        torch.cuda.empty_cache()
    out["speedup_vs_full_list"] = out["rbl"]["value"] / out["full_list"]["value"]
    return out


def make_workload(N, seed):
    from paper_2105_04884_gb300 import inputs

    w = WORKLOAD
    x, L = inputs.fcc(N, w["rho"], 0.01, seed=seed)
    v = inputs.maxwell_boltzmann(N, w["T"], seed=seed)
    return x, v, L


def run_ours(a, rank, world, local):
    import numpy as np
    import torch

    from paper_2105_04884_gb300 import rbl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    w = WORKLOAD
    N = a.N
    x, v, L = make_workload(N, replica_seed(rank))
    sync_all = lambda: barrier(world)  # noqa: E731
    slowest = lambda t: max_over_ranks(t, world, dev)  # noqa: E731

    def timed(system, K, phases=True):
        system.set_phase_timing(phases)
        system.phase_times(reset=True)
        stream = system.stream
        sync_all()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("timed")  # profilers can restrict captures to this range
        system.step(K)
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        sync_all()
        ms = e0.elapsed_time(e1)
        return slowest(ms), system.phase_times()

    common = dict(r_c=w["rc"], r_s=w["rs"], skin=w["skin"], p=w["p"], dt=w["dt"], T=w["T"], gamma=w["gamma"],
                  seed=replica_seed(rank), cells_per_cutoff=w["K"], precision=rbl.RBL_FP32)
    ewald = a.potential == "ewald"
    wname, kname, qself = w["name"], FORCE_KERNEL, 0
    if ewald:  # the charged fluid is the timed workload (every block below runs it)
        from paper_2105_04884_gb300 import inputs

        common.update(potential=rbl.RBL_POT_LJ_EWALD, alpha=EWALD_ALPHA,
                      charges=inputs.charges(N, 1.0, seed=replica_seed(rank)))
        wname = "charged_" + w["name"] + "_ewald_alpha%g" % EWALD_ALPHA
        kname, qself = FORCE_KERNEL_EWALD, 4
    s = rbl.System(x, v, L, **common)
    s.step(a.warmup + EQUIL_STEPS)
    tuned = s.autotune(trials=3)  # launch shapes only: no result depends on them
    # per-phase breakdown (direct launches bracketed by CUDA events) for the roofline,
    # then the headline: the same K steps as the library runs them, graph replays
    obs0 = s.observables()
    ms_phase, (phase_ms, nsteps) = timed(s, a.steps, phases=True)
    obs1 = s.observables()
    # clocks: sampled every 20 ms from just before the timed region through a 1000-step
    # steady-state run of the same workload right after it (the timed region alone is
    # ~10 ms); the steady-state run is reported beside the K-step value (a K-step window
    # holds whichever rebuilds fall in it)
    clocks = Clocks(local)
    clocks.start()
    obs_pre = s.observables()  # rebuild count at the start of the timed steps
    ms, _ = timed(s, a.steps, phases=False)
    obs_post = s.observables()
    LONG = 1000
    ms_long, _ = timed(s, LONG, phases=False)
    clk = clocks.stop()
    clk["window"] = "the %d timed steps and the %d-step steady-state run right after them" % (a.steps, LONG)
    obs_long = s.observables()
    # the list build timed on forced rebuilds of the equilibrated state (the phase-timed
    # steps' list-build phase also carries the build's skipped launches on the steps that
    # do not rebuild)
    s.set_phase_timing(True)
    s.rebuild_times(reset=True)
    for _ in range(4):
        s.build_lists()
    (rb_sort, rb_lists), rb_n = s.rebuild_times()
    s.set_phase_timing(False)
    obs = obs_post
    value = whole_job_rate(N, a.steps, world, ms)
    rebuilds = obs["n_rebuild"] - obs_pre["n_rebuild"]
    rebuilds_phase = obs1["n_rebuild"] - obs0["n_rebuild"]
    ph = phase_dict(phase_ms, nsteps)
    peak, peak_kind = load_peaks()
    nc, ns, p = obs["Nc_mean"], obs["Ns_mean"], w["p"]
    # Roofline of the RBL force kernel (K4).  Algorithmic bytes per particle, the data
    # the method must move: own position 16, core row 4 n_c, N_s 4, the p sampled shell
    # entries 4 p, force out 24.  The DRAM traffic ncu measured for this data layout
    # (row counts and home cell, core row, the shell mask words over the home cell's
    # culled table, one 32-byte sector of that table per drawn entry, force) is reported
    # beside it, with the fraction it gives.
    alg_force = 16 + 4 * nc + 4 + 4 * p + 24 + qself
    t_force = ph["force_kernel"] * 1e-3
    traffic_f = load_traffic(N, "force_kernel_traffic_ewald.json" if ewald else "force_kernel_traffic.json")
    roof_force = {"kernel": kname, "bound": "hbm", "achieved": alg_force * N / t_force / 1e9, "peak": peak,
                  "unit": "GB/s", "frac": alg_force * N / t_force / 1e9 / peak, "peak_source": peak_kind,
                  "algorithmic_bytes_per_particle": alg_force,
                  "traffic": traffic_f, "traffic_per": "launch", "ms_per_launch": ph["force_kernel"]}
    if traffic_f is not None:
        roof_force["traffic_frac"] = traffic_f / t_force / 1e9 / peak
    # Roofline of the list build (K3), per rebuild: own position 16 and the rows, core
    # and shell, as 4-byte entries 4 (n_c + N_s) (~800 B per particle per rebuild).
    # Timed on forced rebuilds of the equilibrated state; the step phases' figure (the
    # phase total over the rebuilds, which also carries the build's launches on the
    # phase-timed steps that do not rebuild) is reported beside it.
    alg_build = 16 + 4 * (nc + ns)
    t_build_phase = ph["list_build"] * nsteps / max(rebuilds_phase, 1) * 1e-3
    t_build = rb_lists / rb_n * 1e-3
    traffic_b = load_traffic(N, "list_build_traffic.json")
    roof_build = {"kernel": "k_build_culled<0> (bounding-box cull into the cell's candidate table, then core row + "
                            "shell mask; one warp per home cell)", "bound": "hbm",
                  "achieved": alg_build * N / t_build / 1e9, "peak": peak, "unit": "GB/s",
                  "frac": alg_build * N / t_build / 1e9 / peak, "peak_source": peak_kind,
                  "algorithmic_bytes_per_particle": alg_build, "traffic": traffic_b, "traffic_per": "launch",
                  "ms_per_launch": t_build * 1e3, "launches_timed": rb_n,
                  "timed_on": "forced rebuilds of the equilibrated state (rbl_build_lists under phase timing)",
                  "cell_sort_ms_per_rebuild": rb_sort / rb_n,
                  "ms_per_rebuild_from_step_phases": t_build_phase * 1e3,
                  "share_of_step": ph["list_build"] / sum(ph.values())}
    if traffic_b is not None:
        roof_build["traffic_frac"] = traffic_b / t_build / 1e9 / peak
    dominant = roof_build if ph["list_build"] >= ph["force_kernel"] else roof_force
    result = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded FCC start + Maxwell-Boltzmann velocities)",
        "config": {"workload": wname, "N": N, "rho": w["rho"], "T": w["T"], "r_c": w["rc"], "r_s": w["rs"],
                   "skin": w["skin"], "p": p, "dt": w["dt"], "gamma": w["gamma"], "cells_per_cutoff": w["K"],
                   "pair_math": "fp32 + int64 fixed-point sums", "integration": "fp64 BAOAB",
                   "parallelism": "replicas" if world > 1 else "single",
                   "equilibration_steps": a.warmup + EQUIL_STEPS,
                   "l2": "working set > L2 (lists %.0f MB)" % (4 * N * (nc + ns) / 1e6),
                   "timed_path": "rbl_step(K): CUDA graph replays, one per step (the rebuild chain behind a "
                                 "device-side IF node)"},
        # per step: integrate, the rebuild condition, force kernel and its reduction;
        # the 12 rebuild-chain kernels on the steps that rebuild
        "gpu_launches": 4 * a.steps + 12 * rebuilds,
        "phases_ms_per_step": ph,
        "phase_timed_ms_per_step": ms_phase / a.steps,
        "rebuilds_in_timed_region": rebuilds,
        "steady_state": {"steps": LONG, "ms_per_step": ms_long / LONG,
                         "value": whole_job_rate(N, LONG, world, ms_long),
                         "rebuilds": obs_long["n_rebuild"] - obs_post["n_rebuild"],
                         "path": "the same rbl_step graph path, timed right after the K timed steps"},
        "rows": {"core_mean": nc, "shell_mean": ns, "core_max": obs["Nc_max"], "shell_max": obs["Ns_max"],
                 "stencil_mean": obs["Mc_mean"]},
        "roofline": dominant,
        # the whole step against the same peak: the method's bytes per particle-step
        # (force kernel K4 without its own force write, the FP64 x and v read and written
        # 96, the fixed-point image written 16) plus the list build's bytes amortised over
        # the steady-state rebuild interval
        "step_roofline": step_roofline(alg_force, alg_build, N, ms / a.steps, LONG, ms_long,
                                       obs_long["n_rebuild"] - obs_post["n_rebuild"], peak, world),
        # pair terms the force kernel evaluates per particle-step: the whole core row
        # (r < r_c + skin at the build) and the p sampled shell entries
        "pairs": {"pair_terms_per_particle_step": nc + p,
                  "pair_terms_per_s": (nc + p) * N * world / t_force,
                  "pair_flops_per_s_approx": 20.0 * (nc + p) * N * world / t_force},
        "rooflines": {"k_build_culled": roof_build, "k_force": roof_force},
        "clocks": clk,
        "launch_config": tuned,
    }
    x_tune, v_tune = None, None
    if not a.no_tune_cells and not ewald:  # (the tuner's contexts carry no charges)
        x_tune, v_tune, _ = s.get_state()  # the equilibrated state, for the cell-size tuner below
    # full Verlet list on the same GPU and workload
    if not a.no_full_list:
        del s
        torch.cuda.empty_cache()
        sf = rbl.System(x, v, L, full_list=True, **common)
        sf.step(a.warmup + EQUIL_STEPS)
        sf.autotune(trials=3)
        _, (pmf, nf) = timed(sf, a.steps, phases=True)
        msf, _ = timed(sf, a.steps, phases=False)
        vf = whole_job_rate(N, a.steps, world, msf)
        of = sf.observables()
        # the full-list force kernel's roofline: own position 16, the row 4 N_full, force 24
        alg_full = 16 + 4 * of["Ns_mean"] + 24
        t_full = pmf[3] / nf * 1e-3
        result["full_list"] = {"value": vf, "ms_per_step": msf / a.steps, "phases_ms_per_step": phase_dict(pmf, nf),
                               "force_kernel_ms": pmf[3] / nf, "full_mean": of["Ns_mean"],
                               "pairs_per_s": N * of["Ns_mean"] / t_full,
                               "roofline": {"kernel": "k_force<1, true, false, 0, false> (explicit full rows)",
                                            "bound": "hbm", "achieved": alg_full * N / t_full / 1e9, "peak": peak,
                                            "unit": "GB/s", "frac": alg_full * N / t_full / 1e9 / peak,
                                            "algorithmic_bytes_per_particle": alg_full,
                                            "traffic": load_traffic(N, "full_list_force_traffic.json"),
                                            "traffic_per": "launch"}}
        result["speedup_vs_full_list"] = value / vf
        del sf
        torch.cuda.empty_cache()
        # the same workload at r_c = 2.0, where the block-averaged P, U and g(r) of the
        # RBL trajectory match the full list's (the metric's "matched pressure/g(r)")
        s2 = rbl.System(x, v, L, **dict(common, r_c=2.0))
        s2.step(a.warmup + EQUIL_STEPS)
        s2.autotune(trials=3)
        _, (pm2, n2) = timed(s2, a.steps, phases=True)
        ms2, _ = timed(s2, a.steps, phases=False)
        v2 = whole_job_rate(N, a.steps, world, ms2)
        result["rbl_rc2.0"] = {"value": v2, "ms_per_step": ms2 / a.steps, "force_kernel_ms": pm2[3] / n2,
                               "phases_ms_per_step": phase_dict(pm2, n2), "speedup_vs_full_list": v2 / vf}
        result["value_matched_physics"] = v2
        result["speedup_matched_physics"] = v2 / vf
        result["matched_physics_setting"] = ("r_c = 2.0, p = 10 (block-averaged P, U and g(r) within error bars of "
                                             "the full list; r_c = 1.5 heats the system)")
        del s2
        torch.cuda.empty_cache()
        # the paper's own sampling pool on the same workload: no shell list (the list
        # build tests only the 27 nearest cells), batch from the whole cell stencil
        s3 = rbl.System(x, v, L, **dict(common, sampling=rbl.RBL_SAMPLE_STENCIL))
        s3.step(a.warmup + EQUIL_STEPS)
        s3.autotune(trials=3)
        _, (pm3, n3) = timed(s3, a.steps, phases=True)
        ms3, _ = timed(s3, a.steps, phases=False)
        o3 = s3.observables()
        v3 = whole_job_rate(N, a.steps, world, ms3)
        result["rbl_stencil_pool"] = {"value": v3, "ms_per_step": ms3 / a.steps,
                                      "phases_ms_per_step": phase_dict(pm3, n3),
                                      "pool_mean": o3["Ns_mean"], "speedup_vs_full_list": v3 / vf,
                                      "speedup_vs_shell_list": v3 / value}
        del s3
        torch.cuda.empty_cache()
    # end to end through the C ABI with host buffers: upload once, K x (one step + that
    # step's observables into host memory), download the final state.  e2e: the
    # observables of every step copied asynchronously into a page-locked ring that the
    # host reads after the final download; e2e_sync: rbl_observables, which waits, each step.
    if not a.no_e2e:
        import ctypes

        se = rbl.System(x, v, L, **common)
        se.set_phase_timing(False)
        se.step(a.warmup + EQUIL_STEPS)
        se.autotune(trials=3)
        xe, ve, step_e = se.get_state()  # the equilibrated state is what a user's loop uploads
        xh = torch.from_numpy(xe).pin_memory()
        vh = torch.from_numpy(ve).pin_memory()
        xo = torch.empty_like(xh).pin_memory()
        vo = torch.empty_like(vh).pin_memory()
        osz = ctypes.sizeof(rbl.rbl_obs)
        ring = torch.empty(a.steps * osz, dtype=torch.uint8).pin_memory()
        obs_c = rbl.rbl_obs()
        e2e = {}
        for mode in ("async", "sync"):
            sync_all()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            se._check(se.lib.rbl_set_state(se.h, ctypes.c_void_p(xh.data_ptr()), ctypes.c_void_p(vh.data_ptr()),
                                           step_e, 0))
            for k in range(a.steps):
                if mode == "async":
                    se._check(se.lib.rbl_step_async(se.h, 1))
                    se._check(se.lib.rbl_observables_async(se.h, ctypes.c_void_p(ring.data_ptr() + k * osz), 0))
                else:
                    se._check(se.lib.rbl_step(se.h, 1))
                    se._check(se.lib.rbl_observables(se.h, ctypes.byref(obs_c)))
            step = ctypes.c_longlong()
            se._check(se.lib.rbl_get_state(se.h, ctypes.c_void_p(xo.data_ptr()), ctypes.c_void_p(vo.data_ptr()),
                                           ctypes.byref(step), 0))
            if mode == "async":  # the host reads every step's scalars
                obs_all = (rbl.rbl_obs * a.steps).from_buffer_copy(ring.numpy().tobytes())
                t_mean = sum(o.T_kin for o in obs_all) / a.steps
            torch.cuda.synchronize()
            e2e[mode] = slowest(time.perf_counter() - t0)
            sync_all()
        te = e2e["async"]
        result["e2e"] = {"value": whole_job_rate(N, a.steps, world, te * 1e3), "unit": "particle-steps/s",
                         "h2d_bytes_per_step": 48 * N / a.steps,
                         "d2h_bytes_per_step": 48 * N / a.steps + osz,
                         "path": "rbl_set_state(host) + steps x (rbl_step_async(1) + rbl_observables_async into "
                                 "a page-locked ring) + rbl_get_state(host, waits and reports device flags) + host "
                                 "read of every step's rbl_obs",
                         "T_kin_mean": t_mean}
        result["e2e_sync"] = {"value": whole_job_rate(N, a.steps, world, e2e["sync"] * 1e3),
                              "unit": "particle-steps/s",
                              "path": "as e2e with rbl_step(1) and rbl_observables, each of which waits"}
        del se
    if x_tune is not None:
        # cells_per_cutoff by measurement (rbl_tune_cells): K decides which batches are
        # drawn, so it is a choice made before a run; the workload's K = 2 is its result
        torch.cuda.empty_cache()
        kw = {k: v for k, v in common.items() if k not in ("cells_per_cutoff", "r_c", "r_s", "skin", "p", "dt")}
        K_best, ms_k = rbl.tune_cells(x_tune, v_tune, L, common["r_c"], common["r_s"], common["skin"], common["p"],
                                      common["dt"], steps=20, **kw)
        result["cell_size_tuning"] = {"K_best": K_best, "ms_per_step_K1_K2_K3": ms_k,
                                      "workload_K": w["K"], "steps": 20,
                                      "path": "rbl_tune_cells on the equilibrated state, each K in its own context"}
        del x_tune, v_tune
    if not a.no_ewald and not ewald:
        result["ewald"] = ewald_bench(a, world, x, v, L, common, timed)
    if not a.no_ensemble:
        result["ensemble"] = ensemble_bench(a, rank, world, timed)
    if not a.no_slab:
        result["slab"] = slab_bench(a, rank, world, timed)
    if rank == 0 and not a.no_physics:
        # the bench workload's (r_c, p) and r_c = 2.0 (the matched setting), each
        # against one full-list trajectory
        mp, full_run = matched_physics_pair(1.5, 10)
        mp2, _ = matched_physics_pair(2.0, 10, full=full_run)
        mp3, _ = matched_physics_pair(1.5, 10, full=full_run, sampling=1)
        mp4, _ = matched_physics_pair(2.0, 10, full=full_run, sampling=1)
        result["matched_physics"] = [mp, mp2, mp3, mp4]
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(x, v, L, a.cpu_steps, q=common.get("charges"),
                                              alpha=common.get("alpha", 0.0))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return result


def cpu_baseline(x, v, L, steps, steps_single=3, q=None, alpha=0.0):
    """The oracle timed on the host cores: OpenMP over every core, and single-threaded
    (the paper's own setting, one core).  Each sample starts from the workload's
    initial state, so it includes one list build.  q: charges of the charged fluid."""
    import oracle

    w = WORKLOAD
    cores = os.cpu_count() or 1
    args = (L, w["rc"], w["rs"], w["skin"], w["p"], w["dt"], w["T"], w["gamma"], 1)
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    oracle.run(x, v, *args, steps, q=q, alpha=alpha)
    t = time.perf_counter() - t0
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.run(x, v, *args, steps_single, q=q, alpha=alpha)
    t1 = time.perf_counter() - t1
    # the small parity system (N = 1000, rho* = 0.8, FP64 NVE, 100 steps), 1 thread and
    # every core
    from paper_2105_04884_gb300 import inputs

    xs, Ls = inputs.fcc(1000, 0.8, 0.01, seed=1)
    vs = inputs.maxwell_boltzmann(1000, 1.5, seed=1)
    small = {}
    for th in (1, cores):
        oracle.set_threads(th)
        t2 = time.perf_counter()
        oracle.run(xs, vs, Ls, w["rc"], w["rs"], w["skin"], w["p"], w["dt"], 1.5, 0.0, 1, 100)
        small[th] = 1000 * 100 / (time.perf_counter() - t2)
    oracle.set_threads(cores)
    return {"value": len(x) * steps / t, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of the same N={len(x)} workload from its start (includes the initial list "
                      f"build), FP64 C oracle with OpenMP on {cores} threads",
            "single_thread": {"value": len(x) * steps_single / t1, "unit": "particle-steps/s", "cores": 1,
                              "sample": f"{steps_single} steps of the same workload from its start, 1 thread"},
            "parity_system_N1000": {"unit": "particle-steps/s", "single_thread": small[1], "all_cores": small[cores],
                                    "sample": "100 FP64 velocity-Verlet steps of N = 1000, rho* = 0.8"}}


REF_BUDGET_S = 120.0  # timed oracle work of the reference arm


def run_reference(a, rank, world):
    """The oracle as the reference arm: warm-up steps, then as many of the requested
    timed steps as fit in REF_BUDGET_S (estimated from the warm-up), on every host
    core.  Ranks other than 0 exit without work."""
    if rank != 0:
        return None
    import oracle

    w = WORKLOAD
    N = a.N
    x, v, L = make_workload(N, 1)
    cores = os.cpu_count() or 1
    oracle.build()
    oracle.set_threads(cores)
    args = (L, w["rc"], w["rs"], w["skin"], w["p"], w["dt"], w["T"], w["gamma"], 1)
    tw = time.perf_counter()
    x, v, _, _ = oracle.run(x, v, *args, a.warmup)
    tw = (time.perf_counter() - tw) / a.warmup
    k = max(1, min(a.steps, int(REF_BUDGET_S / max(tw, 1e-9))))
    t0 = time.perf_counter()
    oracle.run(x, v, *args, k, step0=a.warmup)
    t = time.perf_counter() - t0
    value = N * k / t
    sample = (f"{k} of the {a.steps} requested steps of the full N={N} workload after {a.warmup} warm-up steps "
              f"(lists rebuilt at the start of the timed call), bounded to ~{REF_BUDGET_S:.0f} s of CPU time")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3 / k, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "N": N},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    rank, world, local = dist_info()
    if a.physics:
        if rank == 0:
            physics_sweep()
        return
    if a.ewald_physics:
        if rank == 0:
            ewald_physics_sweep()
        return
    if a.table1:
        if rank == 0:
            table1_study(a.table1_scale)
        return
    if a.variance:
        if rank == 0:
            variance_study()
        return
    if a.impl == "reference":
        res = run_reference(a, rank, world)
    else:
        res = run_ours(a, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
