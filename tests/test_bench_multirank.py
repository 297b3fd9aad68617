"""The N > 1 path of bench.py on the CPU: two ranks over gloo (127.0.0.1), as torchrun
launches them (RANK / WORLD_SIZE / LOCAL_RANK in the environment).

The path shards by independent replicas: each rank draws its own workload (seed
1 + rank), nothing is exchanged on the data path, and the only collectives are the
barriers around the timed region and the max of the ranks' times.  Checked here:
the ranks' workloads differ, every rank gets the slowest rank's time, the whole-job
rate counts every rank's particles over that time, and the reference arm does no
work on ranks other than 0.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench

    r, w, local = bench.dist_info()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        x, v, L = bench.make_workload(4000, bench.replica_seed(r))
        bench.barrier(w)
        t = 0.010 * (1 + r)  # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, w, "cpu")
        rate = bench.whole_job_rate(4000, 100, w, tmax * 1e3)

        class A:
            N, steps, warmup = 4000, 10, 3

        ref = bench.run_reference(A, r, w) if r != 0 else "skipped"
        gathered = [None] * w
        dist.all_gather_object(gathered, (r, local, float(x[:8].sum()), tmax, rate, ref))
        if r == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, l0, s0, t0, v0, ref0), (r1, l1, s1, t1, v1, ref1) = sorted(res)
    assert (r0, r1) == (0, 1) and (l0, l1) == (0, 1)
    assert s0 != s1  # independent replicas: seed 1 + rank
    assert t0 == t1 == pytest.approx(0.020)  # every rank holds the slowest time
    assert v0 == v1 == pytest.approx(4000 * 100 * 2 / 0.020)
    assert ref1 is None  # the reference arm runs on rank 0 only


def test_single_rank_helpers():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.replica_seed(0) == 1 and bench.replica_seed(3) == 4
    assert bench.max_over_ranks(1.5, 1, "cpu") == 1.5
    bench.barrier(1)  # no process group needed
    assert bench.whole_job_rate(1000, 10, 1, 5.0) == pytest.approx(2e6)
    x1, _, L = bench.make_workload(2000, 1)
    x2, _, _ = bench.make_workload(2000, 2)
    assert x1.shape == (2000, 3) and not np.array_equal(x1, x2)


def test_traffic_figure_only_for_matching_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu figure only while the force
    kernel's and the list build's sources are the ones it was measured on."""
    import json
    import sys

    sys.path.insert(0, ROOT)
    import bench
    from paper_2105_04884_gb300 import _build

    prof = tmp_path / "profiles"
    prof.mkdir()
    fig = {"dram_bytes_per_particle": 270.0, "source_sha": _build.force_digest()}
    (prof / "force_kernel_traffic.json").write_text(json.dumps(fig))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic(1000) == pytest.approx(270.0 * 1000)
    fig["source_sha"] = "0" * 16
    (prof / "force_kernel_traffic.json").write_text(json.dumps(fig))
    assert bench.load_traffic(1000) is None
    # the measured peak, else the documented fallback
    assert bench.load_peaks()[1] == "fallback" and bench.load_peaks()[0] == 6800.0


def test_step_roofline_arithmetic():
    """The whole step's bytes: the force kernel's algorithmic bytes without its force
    write (24), plus the FP64 x and v read and written (96) and the image written (16),
    plus the list build's bytes over the rebuild interval; the fraction is the bytes moved
    per second over the peak, and two ranks double the ceiling."""
    import sys

    sys.path.insert(0, ROOT)
    import bench

    nc, p, ns, N = 17.5, 10, 177.0, 1 << 20
    alg_force = 16 + 4 * nc + 4 + 4 * p + 24
    alg_build = 16 + 4 * (nc + ns)
    r = bench.step_roofline(alg_force, alg_build, N, 0.5, 1000, 500.0, 200, 6693.8, 1)
    assert r["algorithmic_bytes_per_particle_step"] == pytest.approx(16 + 4 * nc + 4 + 4 * p + 96 + 16)
    assert r["rebuild_interval_steps"] == pytest.approx(5.0)
    assert r["rebuild_bytes_amortised_per_step"] == pytest.approx(alg_build / 5.0)
    per_step = r["algorithmic_bytes_per_particle_step"] + r["rebuild_bytes_amortised_per_step"]
    assert r["timed"]["achieved"] == pytest.approx(per_step * N / 0.5e-3 / 1e9)
    assert r["steady_state"]["frac"] == pytest.approx(per_step * N / 0.5e-3 / 1e9 / 6693.8)
    r2 = bench.step_roofline(alg_force, alg_build, N, 0.5, 1000, 500.0, 200, 6693.8, 2)
    assert r2["ceiling_particle_steps_per_s"] == pytest.approx(2 * r["ceiling_particle_steps_per_s"])
    assert bench.step_roofline(alg_force, alg_build, N, 0.5, 10, 5.0, 0, 6693.8, 1)["rebuild_interval_steps"] == 10
