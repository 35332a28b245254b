"""The N > 1 path of bench.py runs independent replicas (one instance per
rank, no collective on the data path); its only cross-rank step is the
timing reduction: the job's time is the slowest rank's, its throughput the
units of all ranks over that time.  Checked with 2 gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seconds = [0.25, 0.40][rank]                  # rank 1 is the slower replica
    t = bench.max_over_ranks(seconds, world, device="cpu")
    v = bench.job_throughput(2, seconds, world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, v))


@pytest.mark.timeout(120)
def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == pytest.approx(0.40)           # every rank sees the max
        assert v == pytest.approx(2 * 2 / 0.40)   # 2 ranks x 2 rhs over the slowest time


def test_single_rank_is_its_own_time():
    import bench
    assert bench.max_over_ranks(0.3, 1) == 0.3
    assert bench.job_throughput(2, 0.5, 1) == pytest.approx(4.0)


def test_algorithmic_bytes_are_per_launch():
    """The streaming kernels process at most 4 right-hand sides per launch:
    the roofline's algorithmic bytes count one launch, so they stop growing
    past 4 right-hand sides; the split-sphere figures are the stored entries
    plus inputs and piece sums."""
    import bench
    Ns, n = [2178] * 3, 13068
    assert bench._stream_bytes("matvec32", Ns, n, 2) == 3 * 2178 ** 2 * 16 + n * 8 * 2 + 3 * 2178 * 9 * 16 * 4
    assert bench._stream_bytes("matvec32", Ns, n, 64) == bench._stream_bytes("matvec32", Ns, n, 4)
    assert bench._stream_bytes("osrc_apply", Ns, n, 2) == 3 * 2178 * 2180 * 4 + n * 8 * 2 + 3 * 2178 * 4 * 8 * 4
