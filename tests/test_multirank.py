"""The N > 1 host path of bench.py on CPU: two gloo ranks (replicas only; rays are independent,
so the replicas exchange nothing but their timings)."""
import os
import sys
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank times different work; every rank must see the slowest replica's times
    mine = [10.0 + 5.0 * rank, 2.0 - rank]
    got = bench.max_over_ranks(mine, world, device="cpu")
    value = bench.aggregate_rays_per_s(8192, 20, world, got[0])
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array(got + [value, bench.replica_seed(rank)]))


def test_two_gloo_ranks_take_the_max_time_and_aggregate(tmp_path):
    world, port = 2, 29400 + os.getpid() % 500
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert list(r0[:2]) == [15.0, 2.0] and list(r1[:2]) == [15.0, 2.0]
    assert r0[2] == r1[2] == pytest.approx(8192 * 20 * 2 / 0.015)
    assert r0[3] != r1[3]  # each replica samples its own rays


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks([3.5, 1.25], 1) == [3.5, 1.25]
    assert bench.aggregate_rays_per_s(8192, 10, 1, 1000.0) == pytest.approx(81920.0)


def test_replica_seeds_sample_different_rays():
    """The oracle's sampler with two replicas' seeds draws different pixels (the replicas'
    batches are independent), and the same seed reproduces its batch."""
    import bench
    import oracle as oc
    import scenegen as sg
    w = sg.WORKLOADS["cube-1024x64"]
    cfg, F = oc.make_config(w), oc.OcFramesHolder(sg.make_frames(w))
    a = oc.sample_rays(cfg, F, bench.replica_seed(0), 0, 256)
    b = oc.sample_rays(cfg, F, bench.replica_seed(1), 0, 256)
    c = oc.sample_rays(cfg, F, bench.replica_seed(1), 0, 256)
    assert np.array_equal(b["pix"], c["pix"]) and (a["pix"] != b["pix"]).mean() > 0.9


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, frames, warmup, steps = "room-8192x96", 1, 0, 1
    assert bench.run_reference(Args()) is None


class _RefArgs:
    workload, frames, warmup, steps = "cube-1024x64", None, 1, 2
    recompute = no_pipeline = poses = split = eikonal = False
    prop_pretrain = 300


def test_reference_arm_times_the_steps_it_prints(monkeypatch):
    """Rank 0 of the reference arm runs W + K full oracle steps of the GPU arm's workload and
    prints K, the GPU arm's config and a per-step time that covers K steps."""
    import bench
    import scenegen as sg
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    calls = []
    real = bench._oracle_steps

    def spy(w, fr, R, P, n_steps, **kw):
        calls.append((R, P, n_steps))
        return real(w, fr, R, P, n_steps, **kw)

    monkeypatch.setattr(bench, "_oracle_steps", spy)
    t0 = time.perf_counter()
    line = bench.run_reference(_RefArgs())
    wall = time.perf_counter() - t0
    w = sg.WORKLOADS["cube-1024x64"]
    assert calls == [(w.rays, w.n_smooth, 1), (w.rays, w.n_smooth, 2)]
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["config"] == bench.step_config(w, _RefArgs(), 1, 1)
    assert 2 * line["ms_per_step"] / 1e3 <= wall
    assert abs(line["value"] - w.rays / (line["ms_per_step"] / 1e3)) <= 1e-3 * line["value"] + 0.01
