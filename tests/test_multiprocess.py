"""The multi-rank logic of bench.py on CPU ranks (gloo, world sizes 2 and 3): every
rank evolves an independent replica (seed = rank), the timing is the max over
ranks after a barrier, and the whole-job rate counts every replica; under
torchrun the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        out[rank] = (ms, bench.replica_seed(rank), bench.whole_job_rate(64 ** 3, 10, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_count_every_replica():
    world = 2
    mgr = mp.get_context("spawn").Manager()  # no fork of this multi-threaded process
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    assert out[0][0] == out[1][0] == 15.0  # both ranks see the slowest time
    assert out[0][1] != out[1][1]  # independent replicas
    assert out[0][2] == pytest.approx(2 * 64 ** 3 * 10 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    import sys
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""  # the non-zero rank exits without work or output



def test_reference_arm_prints_the_contract_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 times the oracle (a small lattice here) and prints one JSON line with
    the reference arm's keys: impl, the metric of the ours arm, a cpu_baseline
    describing the run and an e2e entry that moves no bytes."""
    import json
    import sys

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1", "--N", "16"])
    bench.run_reference(bench.parse())
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "site-updates/s" and d["unit"] == "site-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}

def _scan_rank_main(rank, world, port, n, out):
    import numpy as np
    import torch.distributed as dist

    from paper_2006_15122_gb300 import scan

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        block = scan.partition(n, world, rank)
        # each run's "observations": its index and a few derived numbers, as the ensemble would return
        local = np.array([[i, 2.0 * i, -float(i)] for i in block], dtype=np.float32).reshape(len(block), 1, 3)
        if not block:  # fewer runs than ranks: this rank's ensemble call returns nothing
            spec = scan.ScanSpec(n_slices=1)
            local = scan.ensemble_observations(spec, [], [], [])[0][:, :, :3]
        out[rank] = (block, scan.gather_runs(local, n, dist, "cpu"))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 7), (2, 8), (3, 2)])
def test_gloo_ranks_split_the_scan_and_gather_every_run_in_order(world, n):
    """The scan's run list is split into contiguous blocks, one per rank (no
    data-path exchange while the lattices evolve); one gather assembles every
    run's observations in run order on every rank, also when some rank's block
    is empty (fewer runs than ranks)."""
    import numpy as np

    mgr = mp.get_context("spawn").Manager()  # no fork of this multi-threaded process
    out = mgr.dict()
    mp.start_processes(_scan_rank_main, args=(world, _free_port(), n, out), nprocs=world, join=True,
                       start_method="spawn")
    blocks = [out[r][0] for r in range(world)]
    assert sorted(sum(blocks, [])) == list(range(n)) and sum(map(len, blocks)) == n
    for r in range(world):
        g = out[r][1]
        assert g.shape == (n, 1, 3)
        assert np.array_equal(g[:, 0, 0], np.arange(n, dtype=np.float32))
        assert np.array_equal(g[:, 0, 2], -np.arange(n, dtype=np.float32))


def test_partition_without_a_process_group_is_the_whole_scan():
    import numpy as np

    from paper_2006_15122_gb300 import scan

    for n, world in ((10, 3), (3, 4), (512, 8)):
        blocks = [scan.partition(n, world, r) for r in range(world)]
        assert sum(blocks, []) == list(range(n))
        assert max(map(len, blocks)) - min(map(len, blocks)) <= 1
    a = np.zeros((5, 2))
    assert scan.gather_runs(a, 5) is not None


def test_clock_samples_are_summarized_with_their_throttle_reasons():
    """The nvidia-smi rows sampled during the timed region (index, clocks.sm,
    clocks.max.sm, power, active mask, then hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap as Active / Not Active) reduce to the
    median SM clock, the max clock and the reasons seen Active."""
    import bench

    text = ("0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
            "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
            "garbage line\n"
            "0, 2055, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    d = bench.ClockSampler.summarize(text)
    assert d == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler.summarize("")["sm_mhz"] is None


def test_clock_sampler_without_nvidia_smi_reports_unavailable_and_cleans_up(monkeypatch):
    import os
    import subprocess

    import bench

    def no_smi(*a, **k):
        raise FileNotFoundError("nvidia-smi")

    monkeypatch.setattr(subprocess, "Popen", no_smi)
    c = bench.ClockSampler(0)
    c.start()
    d = c.stop()
    assert d["sm_mhz"] is None and d["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(c.f.name)
    assert c.stop() is d  # a second stop returns the same summary
