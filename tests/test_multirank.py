"""The multi-GPU bench path on CPU: two gloo ranks (127.0.0.1) each price
their own book (weak scaling, independent options, no collective on the data
path); the step time is the slowest rank's and the whole-job rate counts the
options of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(100.0 + 50.0 * rank, world)      # rank 1 is the slow one
    rate = bench.whole_job_rate(512, world, ms)
    dist.barrier()
    out.put((rank, ms, rate))
    dist.destroy_process_group()


def test_two_ranks_slowest_time_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 150.0
        assert abs(rate - 2 * 512 / 0.150) < 1e-9


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(42.0, 1) == 42.0
    assert bench.whole_job_rate(512, 1, 500.0) == 1024.0


def test_captured_traffic_only_for_the_captured_sources(monkeypatch):
    """The roofline's DRAM traffic is reported only while the pricing kernel's
    sources hash to the value recorded with the ncu capture."""
    import bench
    sha = bench.kernel_sources_sha256()
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", {"sources_sha256": sha, "bytes_per_launch": {"df32": 123}})
    assert bench.captured_traffic("df32") == 123
    assert bench.captured_traffic("fft64") is None
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", {"sources_sha256": "0" * 64, "bytes_per_launch": {"df32": 123}})
    assert bench.captured_traffic("df32") is None


def test_lattice_cells_and_stencil_floor():
    """The plain stencil's cell count: T(T+1)/2 binomial cells, T^2 trinomial
    or BSM cells; its relative distance skips near-zero prices (below 1e-3 K)."""
    import numpy as np
    import bench
    from paper_2303_02317_gb300 import workloads as wl
    T = 100
    assert bench.lattice_cells(wl.fixed_call(0, T)) == T * (T + 1) / 2
    assert bench.lattice_cells(wl.fixed_call(1, T)) == T * T
    assert bench.lattice_cells(wl.fixed_bsm_put(T)) == T * T
    reqs = [wl.fixed_call(0, T), wl.fixed_call(1, T)]
    ref = np.array([10.0, 1e-9])
    got = np.array([10.0 * (1 + 1e-9), 2e-9])
    ok = np.array([True, True])
    assert abs(bench.max_rel_floor(ref, got, ok, reqs) - 1e-9) < 1e-15
