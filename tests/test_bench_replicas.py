"""The multi-rank (replica) path of the benchmark on CPU ranks over gloo: each rank runs its
own replica, the ranks exchange only the max of their timed-region durations, and the
whole-job value counts every rank's node updates over the slowest rank's time. Rank 0
alone prints; the reference arm runs on rank 0 only."""
import json
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms_local = [12.5, 20.0][rank]
    ms_max = bench.max_over_ranks(ms_local, world, "cpu")
    value = bench.job_mflups(1_000_000, 100, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, value))


def test_max_over_ranks_and_job_value_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in out:
        assert ms_max == 20.0                     # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 1_000_000 * 100 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.job_mflups(5_000_000, 10, 1, 50.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MFLUPS" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["n_gpus"] == 1 and line["higher_is_better"] is True and line["steps"] == 1


def test_traffic_figures_are_keyed_to_the_library_code():
    """The bench reports its stored DRAM traffic only while the library code matches the
    code it was captured with; comments do not count."""
    import bench
    assert bench._code_only("int a; // note\n/* block\n comment */ int b;  \n\n") == "int a;\n int b;"
    assert len(bench.step_source_hash()) == 16
    assert set(bench.TRAFFIC_PER_LAUNCH_256) == {"sources", "f64", "f32", "f16s"}
