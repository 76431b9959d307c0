"""The multi-GPU path of bench.py on CPU: two gloo ranks.

The method runs one lattice per GPU with no exchange between them (replicas),
so the only multi-rank logic is the max-over-ranks time and the whole-job
value; both are checked here with world_size 2 over gloo.  Also on CPU: which
clock samples the bench reports for its timed region, and that it reports ncu
records only for the kernel source they were taken on.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.reduce_max(10.0 + 5.0 * rank, torch.device("cpu"))
    value = bench.replica_value(2048 * 2048, 100, world, slowest / 1e3)
    dist.barrier()
    out[rank] = (slowest, value)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        slowest, value = res[r]
        assert slowest == 15.0
        assert value == pytest.approx(2048 * 2048 * 100 * 2 / 0.015 / 1e6)



def _clock_line(mhz, *reasons):
    flags = ["Active" if nm in reasons else "Not Active"
             for nm in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
    return ", ".join(["0", str(mhz), "2070", "900.0", "0x0"] + flags)


def test_clock_summary_takes_the_samples_of_the_timed_region():
    # samples inside [start, stop] when there are any; for a region shorter
    # than the sampling period the samples just before and just after it;
    # throttle reasons from those samples only
    import bench
    clk = bench.ClockSampler(0)
    clk.lines = [(0.0, _clock_line(1200, "hw_slowdown")), (1.0, _clock_line(2070)),
                 (1.1, _clock_line(2040, "sw_power_cap")), (1.2, _clock_line(2070)),
                 (2.0, _clock_line(900, "hw_thermal_slowdown"))]
    clk.t0, clk.t1 = 0.95, 1.15
    s = clk.summary()
    assert s["samples"] == 2 and s["samples_taken"] == "inside"
    assert s["sm_mhz"] == 2055.0 and s["reasons"] == ["sw_power_cap"]
    clk.t0, clk.t1 = 1.15, 1.16
    s = clk.summary()
    assert s["samples_taken"] == "bracketing" and s["samples"] == 2
    assert s["sm_mhz"] == 2055.0 and s["reasons"] == ["sw_power_cap"]
    assert abs(s["region_ms"] - 10.0) < 1e-6


def test_profile_records_are_reported_only_for_the_source_they_were_taken_on(tmp_path, monkeypatch):
    # the bench's DRAM and instruction figures per node come from ncu records
    # that name the kernel source they were measured on; a different source
    # gives no figure (the line reports null rather than a stale number)
    import hashlib
    import json
    import bench
    csrc = tmp_path / "paper_2501_04920_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = b"// kernels\n"
    (csrc / "ehdlb_kernels.cuh").write_bytes(src)
    digest = hashlib.sha256(src).hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
        {"k_main": {"dram_bytes_per_node": 256.4, "source_sha256_16": digest}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_record("k_main", "dram_bytes_per_node") == 256.4
    assert bench.measured_traffic("k_main", 2048) == 256.4 * 2048 * 2048
    assert bench.profile_record("k_prep", "dram_bytes_per_node") is None
    (csrc / "ehdlb_kernels.cuh").write_bytes(src + b"// changed\n")
    assert bench.profile_record("k_main", "dram_bytes_per_node") is None
    assert bench.measured_traffic("k_main", 2048) is None
