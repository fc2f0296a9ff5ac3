"""The N > 1 host logic of bench.py on CPU, two gloo ranks.

Receivers are independent (Eqs. 1-4 per receiver), so the evaluation shards
across ranks with no data-path exchange: one job's receivers split into
contiguous ranges of the same size, each rank writes its own output slice
(gathered into the single-rank layout afterwards), the job's time is the
slowest rank's, and the job's throughput is all ranks' samples over that
time.  No GPU is used here.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2310_10578_gb300 import shard
        sc = bench.make_scene(rank, world)
        # a rank-dependent "time": the reduction must return the slowest rank's
        ms, e2e = bench.max_over_ranks([1.0 + rank, 10.0 - rank])
        # stand-in for the rank's field slice: a function of each receiver's
        # coordinates in the evaluation's layout [n_f][3][n][2]
        E = torch.tensor(_fake_fields(sc.rx, len(sc.freqs)))
        full = shard.gather_fields(E, 256 * 256 * world)
        # the reference arm runs on rank 0 only; other ranks return without work
        rc = bench.run_reference(None) if rank != 0 else 0
        q.put((rank, ms, e2e, sc.n_rx, len(sc.freqs), sc.rx.copy(), None if full is None else full.numpy(), rc))
    finally:
        dist.destroy_process_group()


def _fake_fields(rx, n_f):
    x, y, z = (rx[:, k].astype(np.float64) for k in range(3))
    E = np.empty((n_f, 3, len(rx), 2), dtype=np.float32)
    for f in range(n_f):
        for c in range(3):
            E[f, c, :, 0] = x * (1 + f) + c * y
            E[f, c, :, 1] = y * (2 + c) - z * f
    return E


def test_two_gloo_ranks_shard_one_job_without_exchange():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, n_rx, n_f, rx, full, rc in res:
        assert ms == 2.0 and e2e == 10.0          # max over ranks, on every rank
        assert n_rx == 65536 and n_f == 3          # same per-rank work (weak scaling)
        assert rc == 0
        assert (full is None) == (rank != 0)       # gathered on rank 0 only
    # one job: the ranks' receivers are the contiguous halves of the job's grid
    from paper_2310_10578_gb300 import scenes
    job = scenes.room(nx=256, ny=512)
    assert np.array_equal(np.concatenate([res[0][5], res[1][5]]), job.rx)
    # the gather gives the single-rank layout of the whole job
    assert np.array_equal(res[0][6], _fake_fields(job.rx, 3))


def test_single_process_reduction_and_throughput():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.5]) == [3.0, 4.5]
    assert bench.job_throughput(196608, 4, 0.5) == pytest.approx(4 * 196608 / 0.5)


def _adjoint_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2310_10578_gb300 import adjoint
        # stand-in for each receiver's contribution to the parameter gradient
        # (the adjoint is a sum over receivers): the rank's share, then the sum
        contrib = np.random.default_rng(0).standard_normal((4097, 9))
        lo, hi = adjoint.shard(len(contrib), rank, world)
        g = torch.tensor(contrib[lo:hi].sum(axis=0))
        adjoint.allreduce_gradients([g])
        q.put((rank, lo, hi, g.numpy()))
    finally:
        dist.destroy_process_group()


def test_adjoint_gradient_sum_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_adjoint_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = np.random.default_rng(0).standard_normal((4097, 9)).sum(axis=0)
    assert [(lo, hi) for _, lo, hi, _ in res] == [(0, 2049), (2049, 4097)]
    for _, _, _, g in res:
        assert np.allclose(g, full, rtol=1e-12, atol=1e-12)


def test_shards_cover_every_receiver_once():
    from paper_2310_10578_gb300 import adjoint
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            ranges = [adjoint.shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
