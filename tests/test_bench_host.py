"""Host-side logic of bench.py, on the CPU: the clock record that decides
whether a timed run is kept, the DRAM-traffic lookup behind the roofline
line, and the multi-rank path (replicas, max over ranks) as two gloo ranks."""

import os
import socket
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _smi(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    # one line of nvidia-smi --format=csv,noheader,nounits for ClockSampler.QUERY
    return f"0, {sm}, {mx}, 812.40, 0x0000000000000000, {hw}, {hwt}, {swt}, {pcap}"


def test_clock_summary_median_max_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [_smi(2070, 2070), _smi(2055, 2070, pcap="Active"), _smi(1980, 2070),
                "garbage", "0, [N/A], 2070, 1, 0, a, b, c, d", _smi(2070, 2070)]
    s = cs.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == pytest.approx(2062.5)
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_throttle_reason():
    cs = bench.ClockSampler(0)
    cs.lines = [_smi(1500, 2070, hw="Active"), _smi(1400, 2070, hwt="Active", swt="Active")]
    assert cs.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_known_for_every_stage_kernel():
    for stage, kernel in bench.KERNEL_OF_STAGE.items():
        t = bench.load_traffic(kernel)
        assert t is not None and t > 0, (stage, kernel)
    assert bench.load_traffic("no_such_kernel") is None
    assert bench.load_traffic(None) is None


def test_single_rank_reduce_is_identity(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.reduce_max(3.25, 1) == 3.25


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench as b
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        r, w, local = b.dist_env()
        # each rank's timed region; the job's time is the slowest rank's
        slowest = b.reduce_max(100.0 + 25.0 * rank, w)
        dist.barrier()
        q.put((rank, r, w, local, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0, 0], codes
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, r, w, local, slowest in got:
        assert (r, w, local) == (rank, 2, rank)
        assert slowest == 125.0
    # whole-job rate as bench.py reports it: all ranks' steps over that time
    K = 10
    assert 2 * K / (slowest / 1e3) == pytest.approx(160.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "2", "--warmup", "3"],
                         env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr[-2000:]
    assert res.stdout.strip() == ""
