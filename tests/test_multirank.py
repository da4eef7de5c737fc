"""The N > 1 benchmark path runs independent replicas, one per rank; its only
collective work is the whole-job aggregation (sum of atom-steps, max of
times).  Checked here on CPU with two gloo ranks."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r processed 100 (r + 1) units in 10 + r ms
    value, ms = bench.job_throughput(100.0 * (rank + 1), 10.0 + rank, dist, "cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, ms = out[r]
        assert ms == 11.0
        assert value == pytest.approx(300.0 / 0.011)


def test_single_rank_aggregation():
    import bench
    value, ms = bench.job_throughput(500.0, 20.0)
    assert ms == 20.0 and value == pytest.approx(25000.0)


def test_kernel_source_hash_ignores_comments_and_whitespace():
    # the ncu summaries name the kernel source they were taken on by this
    # hash; a comment or layout edit must keep it, a code edit must change it
    import bench
    code = 'int a = 1;  // one\n/* two\n */ const char* s = "x // y";\nchar q = \'/\';'
    same = "int a = 1;\n\n const char* s = \"x // y\"; /* note */ char q = '/';"
    other = 'int a = 2; const char* s = "x // y"; char q = \'/\';'
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)
    assert '"x // y"' in bench._code_only(code)
