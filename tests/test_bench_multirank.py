"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, the job
time is the slowest rank's, throughput counts every rank's units, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.aggregate_ms(times[rank], world)
    out[rank] = (t, bench.throughput(1000, t, 10, world))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    port = _free_port()
    times = [12.5, 20.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, times, out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for r in (0, 1):
        t, thr = res[r]
        assert t == 20.0
        # 2 ranks x 1000 units x 10 steps in 20 ms
        assert thr == pytest.approx(2 * 1000 * 10 / 0.020)


def test_single_rank_is_identity():
    import bench

    assert bench.aggregate_ms(7.25, 1) == 7.25
    assert bench.throughput(5, 10.0, 4, 1) == pytest.approx(5 * 4 / 0.010)


def test_reference_arm_other_ranks_do_no_work():
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.reference_arm(args, rank=1, world=2) is None


def test_mesh_stage_bytes():
    """The mesh stages' minimum traffic: a 256^3 real mesh is 64 MiB, its half
    spectrum 256 x 256 x 129 complex values; ik adds two spectra and writes
    the four-component field."""
    import bench

    m, mh = 256 ** 3, 256 * 256 * 129
    ad = bench.mesh_stage_gbs((256, 256, 256), {"fft_fwd": 1.0, "green": 0.5, "fft_inv": 2.0})
    assert ad["fft_fwd"]["bytes"] == 4 * m + 8 * mh
    assert ad["green"]["bytes"] == 20 * mh and ad["fft_inv"]["bytes"] == 8 * mh + 4 * m
    assert ad["green"]["gbs"] == round(20 * mh / 0.5e-3 / 1e9, 1)
    ik = bench.mesh_stage_gbs((64, 64, 64), {"fft_fwd": 0.01, "green": 0.01, "fft_inv": 0.01}, ik=True)
    assert ik["green"]["bytes"] == 36 * 64 * 64 * 33 and ik["fft_inv"]["bytes"] == 24 * 64 * 64 * 33 + 16 * 64 ** 3
    assert bench.mesh_stage_gbs((8, 8, 8), {"fft_fwd": 0.0}) == {}


def test_cpu_baseline_object():
    """The reported baseline is the all-cores figure when replicas ran, with
    the one-core figure beside it."""
    import bench

    one = {"value": 0.01, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": "s1"}
    o = bench.cpu_baseline_obj({"one_core": one})
    assert o["value"] == 0.01 and o["cores"] == 1 and o["host_cores"] == os.cpu_count()
    allc = {"value": 0.1, "unit": "steps/s", "cores": 12, "kind": "oracle", "sample": "s12"}
    o = bench.cpu_baseline_obj({"one_core": one, "all_cores": allc})
    assert o["value"] == 0.1 and o["cores"] == 12 and o["one_core"] == one and o["sample"] == "s12"


def test_algorithmic_bytes_follow_the_scope_table():
    """Per-launch algorithmic bytes on the 2,048,001-charge 256^3 workload:
    make_rho 16N + 8M, ad fieldforce 4M + 32N, ik fieldforce 16M + 32N,
    sort 40N, ad green 4M + 2M + 4M (half spectrum)."""
    import bench

    n, mesh = 2048001, (256, 256, 256)
    M, mh = 256 ** 3, 256 * 256 * 129
    assert bench.alg_bytes("make_rho", n, mesh, False) == 16 * n + 8 * M
    assert bench.alg_bytes("fieldforce", n, mesh, False) == 4 * M + 32 * n
    assert bench.alg_bytes("fieldforce", n, mesh, True) == 16 * M + 32 * n
    assert bench.alg_bytes("sort", n, mesh, False) == 40 * n
    assert bench.alg_bytes("green", n, mesh, False) == 20 * mh
    assert abs(bench.alg_bytes("make_rho", n, mesh, False) / 1e6 - 167.0) < 0.5  # 167 MB
    assert abs(bench.alg_bytes("fieldforce", n, mesh, False) / 1e6 - 132.6) < 0.5


def test_sampled_oracle_step_is_the_oracle_step():
    """The timed CPU sample runs the oracle's own stages: its subsampled
    forces, energy and virial equal OraclePPPM.compute on the same inputs,
    and the estimate scales only the fieldforce time."""
    import numpy as np

    import bench
    from paper_1702_04250_gb300.workloads import config

    w = config("c1")
    for mode in ("ik", "ad"):
        o = bench.oracle_setup(w, mode)
        est, sample_s, out = bench.oracle_sampled_step(o, w.x, w.q, 7)
        ref = o.compute(w.x, w.q, subset=np.arange(0, w.n, 7))
        assert np.allclose(out["f_sub"], ref["f"], rtol=0, atol=1e-12 * np.abs(ref["f"]).max())
        assert abs(out["ev"][0] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
        assert np.allclose(out["ev"][1:], ref["virial"], rtol=1e-12, atol=0)
        st = out["stage_s"]
        assert est >= sample_s - 0.01
        assert abs(est - (st["make_rho"] + st["poisson"] + st["energy_virial"] + 7 * st["fieldforce_sample"])) < 0.01


def test_oracle_replicas_respect_the_memory_budget(monkeypatch):
    """No replica run when two do not fit in the memory budget."""
    import bench

    monkeypatch.setattr(bench, "host_memory_budget", lambda: bench.ORACLE_REPLICA_BYTES + 1)
    assert bench.oracle_all_cores(None, None, 100) is None
