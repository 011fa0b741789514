"""The multi-process paths of bench.py on CPU (gloo, world size 2): the barrier and
the max-over-ranks reduction of the step time, and the reference arm under
torchrun, where rank 0 alone runs and prints one line and the other rank exits 0."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w = bench.dist_setup(None)
    bench.barrier(w)
    q.put((r, w, bench.max_over_ranks(1.5 + r, w)))
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks_with_gloo():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_reference_arm_under_torchrun_prints_one_line():
    pytest.importorskip("torch")
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--nel", "32"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    # the requested warm-up and timed oracle steps, the time per timed step
    assert line["steps"] == 2 and line["warmup"] == 1 and line["ms_per_step"] > 0


def test_clock_samples_are_taken_from_the_timed_region():
    """The clock summary keeps the nvidia-smi samples whose timestamps fall between
    the two marks around the timed region (median SM clock, throttle reasons, power
    of those), and falls back to all samples, flagged by samples_in_region = 0, when
    none does."""
    import datetime
    sys.path.insert(0, ROOT)
    import bench
    t = lambda s: datetime.datetime.strptime(s, "%Y/%m/%d %H:%M:%S.%f")
    text = "\n".join([
        "2026/12/03 09:12:46.100, 0, 1980, 2070, 150.2, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 09:12:46.300, 0, 2070, 2070, 600.5, 0x4, Not Active, Not Active, Not Active, Active",
        "2026/12/03 09:12:46.500, 0, 2055, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 09:12:46.700, 0, 1500, 2070, 120.0, 0x0, Not Active, Active, Not Active, Not Active"])
    c = bench.ClockSampler.parse(text, [t("2026/12/03 09:12:46.250"), t("2026/12/03 09:12:46.600")])
    assert c["samples_in_region"] == 2 and c["sm_mhz"] == 2062.5 and c["reasons"] == ["sw_power_cap"]
    assert c["power_w_max"] == 700.0 and c["sm_max_mhz"] == 2070.0
    c = bench.ClockSampler.parse(text, [t("2026/12/03 09:12:47.000"), t("2026/12/03 09:12:47.100")])
    assert c["samples_in_region"] == 0 and c["samples"] == 4 and "hw_thermal_slowdown" in c["reasons"]
    assert bench.ClockSampler.parse("", [])["reasons"] == ["no samples"]
