"""Shot-sharded gradient reduction on CPU ranks (gloo, world size 2).

Each rank computes the FP64 oracle gradient of its shard of shots; one
all-reduce sums gradients and misfits; the result must equal the single-rank
gradient over all shots.  The solver per rank is the oracle, so no GPU is
needed; this checks the sharding and reduction logic the benchmark uses."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_14189_gb300 import inputs, shots


def _case():
    rng = np.random.default_rng(4)
    nz, nx, nt = 20, 26, 60
    v = rng.uniform(1800.0, 2800.0, (nz, nx))
    src = np.array([[1, 3], [2, 12], [1, 20], [3, 7], [2, 25]], dtype=np.int32)
    rec = inputs.surface_line(5, 0, np.arange(0, nx, 3))
    w = np.stack([inputs.ricker(15.0 + k, 1e-3, nt) for k in range(5)])
    d_obs = 0.01 * rng.standard_normal((5, rec.shape[1], nt))
    return nz, nx, nt, v, src, rec, w, d_obs


def _oracle_grad(sl):
    import oracle
    nz, nx, nt, v, src, rec, w, d_obs = _case()
    n = len(range(*sl.indices(5)))
    p = oracle.make_problem(0, nz, nx, 5, 10.0, 1e-3, nt, n, rec.shape[1], 15.0, v_pml=2800.0)
    return oracle.acoustic_gradient(p, v, w[sl], src[sl], rec[sl], d_obs[sl])


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, J = _oracle_grad(shots.shard(5, rank, world))
        gt = torch.tensor(g)
        Jt = torch.tensor(J, dtype=torch.float64)
        shots.reduce_gradient(gt, Jt)
        if rank == 0:
            np.save(out + "_g.npy", gt.numpy())
            np.save(out + "_J.npy", Jt.numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_all_shots():
    for n in (0, 1, 5, 20, 21):
        for world in (1, 2, 3, 8):
            parts = [range(*shots.shard(n, r, world).indices(n)) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_two_rank_gradient_equals_single_rank(tmp_path):
    out = str(tmp_path / "res")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    g2, J2 = np.load(out + "_g.npy"), float(np.load(out + "_J.npy"))
    g1, J1 = _oracle_grad(slice(0, 5))
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-14 * np.abs(g1).max())
    assert abs(J2 - J1) <= 1e-12 * J1


def _survey_case():
    """The benchmark's acquisition layout on a small grid: a surface survey
    of 2 x 3 shots (3 per rank at world size 2), receivers every 3 cells."""
    rng = np.random.default_rng(9)
    nz, nx, nt = 18, 31, 50
    v = rng.uniform(1900.0, 2700.0, (nz, nx))
    src, rec = inputs.surface_survey(nx, 6)
    w = np.stack([inputs.ricker(18.0, 1e-3, nt)] * 6)
    d_obs = 0.01 * rng.standard_normal((6, rec.shape[1], nt))
    return nz, nx, nt, v, src, rec, w, d_obs


def _survey_grad(sl):
    import oracle
    nz, nx, nt, v, src, rec, w, d_obs = _survey_case()
    n = len(range(*sl.indices(6)))
    p = oracle.make_problem(0, nz, nx, 4, 10.0, 1e-3, nt, n, rec.shape[1], 18.0, v_pml=2700.0)
    return oracle.acoustic_gradient(p, v, w[sl], src[sl], rec[sl], d_obs[sl])


def _survey_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, J = _survey_grad(shots.shard(6, rank, world))
        gt = torch.tensor(g)
        Jt = torch.tensor(J, dtype=torch.float64)
        shots.reduce_gradient(gt, Jt)
        if rank == 0:
            np.save(out + "_g.npy", gt.numpy())
            np.save(out + "_J.npy", Jt.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_survey_shards_equal_the_whole_survey(tmp_path):
    """Each rank models its own block of one survey (the benchmark's layout
    under torchrun), not a copy of the same shots: the all-reduced gradient
    and misfit are those of the whole survey on one rank."""
    assert [shots.shard(6, r, 2) for r in range(2)] == [slice(0, 3), slice(3, 6)]
    src, _ = inputs.surface_survey(31, 6)
    assert list(src[:, 1]) == [0, 6, 12, 18, 24, 30]
    out = str(tmp_path / "survey")
    mp.start_processes(_survey_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    g2, J2 = np.load(out + "_g.npy"), float(np.load(out + "_J.npy"))
    g1, J1 = _survey_grad(slice(0, 6))
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-14 * np.abs(g1).max())
    assert abs(J2 - J1) <= 1e-12 * J1


def test_bench_workload_shards_one_survey():
    """Under torchrun the benchmark's ranks take disjoint blocks of one
    20 N-shot survey; at N = 1 it is the 20-shot single-GPU workload."""
    w1 = inputs.workload_marmousi(nt=10)
    assert w1["src"].shape == (20, 2) and w1["src"][-1, 1] == 900
    parts = [inputs.workload_marmousi(nt=10, total_shots=40, shots=shots.shard(40, r, 2))
             for r in range(2)]
    xs = np.concatenate([p["src"][:, 1] for p in parts])
    assert len(xs) == 40 and len(set(xs.tolist())) == 40
    assert parts[0]["src"].shape == (20, 2) and parts[1]["rec"].shape == (20, 301, 2)
