"""Host logic of bench.py's N-replica mode on CPU: two gloo ranks, max-over-ranks timing and the whole-job
throughput (no GPU, no data-path collective: the replicas only agree on the slowest step time)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [3.0, 5.0][rank]
    m = bench.reduce_max(ms)
    out[rank] = (m, bench.aggregate_rays_per_s(world, 1 << 18, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_timing_and_aggregate():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 5.0
    assert abs(v - 2 * (1 << 18) / 5e-3) < 1e-6


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(4.5) == 4.5
    assert bench.aggregate_rays_per_s(1, 1000, 2.0) == 500000.0


def test_one_gpu_configs_run_on_rank_zero_only(monkeypatch):
    """The precision, serving, apartment, fusion, query and CRF measurements are one-GPU runs: under a
    multi-process launch every rank but 0 returns without measuring."""
    import sys
    import bench
    called = []
    for name in ("run_precision", "run_serve", "run_apartment", "run_fusion", "run_query", "run_crf"):
        monkeypatch.setattr(bench, name, lambda args, n=name: called.append(n))
    monkeypatch.setenv("WORLD_SIZE", "2")
    for cfg in ("room_bf16_sem", "serve", "apartment", "fusion", "query", "crf"):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--config", cfg])
        monkeypatch.setenv("RANK", "1")
        bench.main()
        assert called == []
        monkeypatch.setenv("RANK", "0")
        bench.main()
        assert len(called) == 1
        called.clear()
