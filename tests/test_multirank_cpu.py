"""The multi-rank logic of bench.py on CPU: two gloo ranks (world_size 2)
combine their step times by the maximum and report the whole job's samples/s
(weak scaling: each rank works on its own samples, no data-path collective);
each rank draws its own seeded samples; the reference arm runs on rank 0 only;
data-parallel step-size training sums the loss and gradient over the ranks."""
import os
import socket

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


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1905_11071_gb300 import synth
    ms = [3.0, 5.0][rank]
    got = bench.max_over_ranks(ms, world, "cpu")
    val = bench.job_throughput(10000, world, got)
    w = synth.slista_64x256(seed=rank, N=16, T=2)
    args = type("A", (), {"N": 16, "T": 2, "cpu_samples": 1, "warmup": 0, "steps": 1, "prec": "bf16x3",
                          "oista_prec": "bf16x3", "backward": "traj", "cpu_cores": 1})()
    ref = bench.run_reference(args, rank, world)
    out[rank] = (got, val, float(w.X[0, 0]), ref is None)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_by_max():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, val, x00, ref_none = res[r]
        assert got == 5.0
        assert val == pytest.approx(10000 * 2 / 5e-3)
        assert ref_none == (r != 0)
    # weak scaling: the ranks draw different samples
    assert res[0][2] != res[1][2]


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_throughput(100, 1, 1000.0) == pytest.approx(100.0)
    assert np.isfinite(bench.job_throughput(1, 8, 1e-3))


# --- data-parallel step-size training: the loss and its gradient summed over ranks

def _shard(rank, world, T=6, N=40):
    """Rank r's samples of a fixed least-squares problem in the steps (a
    stand-in for the Step-LISTA loss, which needs a GPU): rows r, r + world, ..."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((N, T))
    y = A @ np.linspace(0.5, 1.5, T) + 0.1 * rng.standard_normal(N)
    return A[rank::world], y[rank::world]


def _loss_fn(A, y):
    At, yt = torch.from_numpy(A), torch.from_numpy(y)

    def f(a):  # a sum over the samples, like the Step-LISTA loss (non-smooth too)
        r = At @ a - yt
        return (0.5 * r * r + 0.05 * r.abs()).sum()
    return f


def _train_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1905_11071_gb300 import api
    A, y = _shard(rank, world)
    a0 = torch.full((A.shape[1],), 0.2, dtype=torch.float64)
    alpha, hist = api.train_step_sizes(a0, None, 0.0, steps=25, group=dist.group.WORLD, loss_fn=_loss_fn(A, y))
    out[rank] = (alpha.numpy().tolist(), hist)
    dist.barrier()
    dist.destroy_process_group()


def test_data_parallel_step_training_matches_one_process():
    """Two gloo ranks, each with half the samples, train the steps with the
    loss and gradient summed over the ranks: both end with the same steps
    (bit for bit) and follow the same trajectory as one process holding all
    the samples (up to the order of the sums)."""
    from paper_1905_11071_gb300 import api
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_train_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]
    A, y = _shard(0, 1)
    a0 = torch.full((A.shape[1],), 0.2, dtype=torch.float64)
    alpha, hist = api.train_step_sizes(a0, None, 0.0, steps=25, loss_fn=_loss_fn(A, y))
    assert len(hist) == len(res[0][1])
    np.testing.assert_allclose(res[0][0], alpha.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(res[0][1], hist, rtol=1e-10)
    assert hist[-1] < hist[0]  # the trainer made progress
