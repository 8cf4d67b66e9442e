"""Several ranks (bench.py --gpus N under torchrun) on the CPU: the path does
not shard, so N ranks run independent replicas; their step times are reduced
to the slowest one and the whole-job rate counts every replica's solves. The
reference arm runs on rank 0 alone. World size 2, gloo, 127.0.0.1."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        # ms per step differ by rank; every rank gets the slowest
        ms = bench.max_over_ranks(12.5 + 7.0 * rank, device="cpu")
        dist.barrier()
        e2e = bench.max_over_ranks(0.020 - 0.005 * rank, device="cpu")
        out[rank] = (ms, e2e, bench.whole_job_rate(ws, ms * 1e-3))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_replica, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        ms, e2e, rate = res[rank]
        assert ms == 19.5 and e2e == 0.020
        assert rate == pytest.approx(2 / 0.0195)


def test_one_rank_without_a_group_is_unchanged():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(3.25, device="cpu") == 3.25
    assert bench.whole_job_rate(1, 0.5) == 2.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
