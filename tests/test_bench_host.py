"""Host-side logic of bench.py, without a GPU: the whole-job figures of a
multi-rank run (world size 2 over gloo on 127.0.0.1), the clock summary,
the hash-keyed DRAM traffic record and the reference arm's JSON line."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed (100 + 50 r) ms for (1 + r) * 1e9 units of its own
        ms, value = bench.combine_ranks(100.0 + 50.0 * rank, (1 + rank) * 1e9, world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_takes_slowest_rank_and_all_units():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 150.0  # the slowest rank
        assert value == pytest.approx(3e9 / 0.150)  # units of both ranks / slowest time


def test_combine_ranks_single_process():
    assert bench.combine_ranks(200.0, 4e9, 1) == (200.0, pytest.approx(2e10))


def test_clock_summary_reports_throttle_reasons():
    lines = [
        "GPU-abc, 2070 MHz, 2070 MHz, 900.00 W, 0x0, Not Active, Not Active, Not Active, Not Active",
        "GPU-abc, 2040 MHz, 2070 MHz, 1300.00 W, 0x4, Not Active, Not Active, Not Active, Active",
        "GPU-abc, 1980 MHz, 2070 MHz, 1390.00 W, 0x4, Not Active, Not Active, Not Active, Active",
        "GPU-other, 900 MHz, 2070 MHz, 100.00 W, 0x0, Active, Not Active, Not Active, Not Active",
    ]
    c = bench.ClockSampler.summarize(lines, "GPU-abc")
    assert c["sm_mhz"] == 2040.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]  # the other GPU's hw_slowdown is not ours


def test_traffic_record_is_keyed_by_kernel_source(tmp_path, monkeypatch):
    rec = tmp_path / "profiles"
    rec.mkdir()
    (rec / os.path.basename(bench.TRAFFIC_RECORD)).write_text(
        "text\nrecord-lattice: 1024\nrecord-precision: fp32\n"
        f"record-source-sha256: {bench.step_kernel_hash()}\nrecord-dram-bytes-per-launch-w64: 1.5e11\n"
        "record-dram-bytes-per-launch-w256: 1.4e11\n")
    for rel in bench.STEP_KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(1024, "fp32", 64) == 1.5e11
    assert bench.recorded_traffic(512, "fp32", 64) is None
    assert bench.recorded_traffic(1024, "fp64", 64) is None
    assert bench.recorded_traffic(1024, "fp32", 256) == 1.4e11
    assert bench.recorded_traffic(1024, "fp32", 32) is None  # a z-chunking without a record
    # any change to the kernel's sources voids the record
    src = tmp_path / bench.STEP_KERNEL_SOURCES[0]
    src.write_bytes(src.read_bytes() + b"\n")
    assert bench.recorded_traffic(1024, "fp32", 64) is None


def test_launch_count_per_detection_period():
    """One period at 1024^3 on the tiled path: 16 step launches, windings,
    cell bits, overlap and the two finalize stages (the launch list of the
    benchmark shows 21 per period); small lattices skip the first stage."""
    assert bench.launches_per_period(1024, 16, True) == 21
    assert bench.measure_partials(1024, True) == 16384 + 34 * 147 * 2
    assert bench.launches_per_period(64, 16, True) == 20
    assert bench.launches_per_period(64, 16, False) == 19


def _run_bench(args, env_extra=None):
    import subprocess
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_the_contract_line():
    """`--impl reference` times the FP64 oracle on the host cores (one step =
    one detection period of the sample) and prints one JSON line with the
    benchmark's metric and unit, `impl`, a `cpu_baseline` describing the run
    and an `e2e` with no host-device bytes."""
    import json
    r = _run_bench(["--impl", "reference", "--ref-n", "16", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "site-updates/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert abs(d["value"] - 2 * 16 * 16 ** 3 / (2 * d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "16^3" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs and prints the reference arm."""
    r = _run_bench(["--impl", "reference", "--ref-n", "16", "--steps", "1", "--warmup", "1"], {"RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
