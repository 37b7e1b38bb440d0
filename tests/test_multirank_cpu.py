"""Multi-rank logic on CPU (gloo, world size 2, 127.0.0.1): the subject
sharding of Algorithm 1 (D-SRM) with its one exchange per iteration gives the
single-process EM result, and bench.py's max-over-ranks timing agrees on all
ranks.  No GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1608_04647_gb300.shard import imbalance, shard_subjects


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_plan_balanced_and_complete():
    vox = synth.draw_voxel_counts(synth.config_spec(2))
    for world in (1, 2, 3, 8):
        plan = shard_subjects(vox, world)
        flat = sorted(i for p in plan for i in p)
        assert flat == list(range(len(vox)))
        assert imbalance(vox, plan) < 1.15
    assert shard_subjects([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]


def _sharded_em(rank, world, port, X, W0, n_iter, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = len(X)
    plan = shard_subjects([x.shape[0] for x in X], world)
    mine = plan[rank]
    Xh = {i: oracle.center(X[i])[0] for i in mine}
    sq = {i: float(np.sum(Xh[i] ** 2)) for i in mine}
    W = {i: W0[i].astype(np.float64) for i in mine}
    rho2 = np.ones(N)
    k, T = W0[0].shape[1], X[0].shape[1]
    Sigma = np.eye(k)
    V = float(sum(x.shape[0] for x in X))
    lls = []
    for _ in range(n_iter):
        # local part of the reduction y = sum_i rho_i^-2 W_i^T X_i and the scalars
        y = np.zeros((k, T))
        s = np.zeros(3)  # sum rho^-2, sum v ln rho^2, sum ||X||^2 / rho^2
        for i in mine:
            y += W[i].T @ Xh[i] / rho2[i]
            s += [1.0 / rho2[i], Xh[i].shape[0] * np.log(rho2[i]), sq[i] / rho2[i]]
        ty, ts = torch.from_numpy(y), torch.from_numpy(s)
        dist.all_reduce(ty)
        dist.all_reduce(ts)
        y, s = ty.numpy(), ts.numpy()
        rho0 = s[0]
        est = {"y": y, "rho0": rho0, "Phi": np.linalg.inv(np.linalg.inv(Sigma) + rho0 * np.eye(k))}
        est["ES"] = Sigma @ (np.eye(k) - rho0 * est["Phi"]) @ y
        ld = np.linalg.slogdet(np.eye(k) + rho0 * Sigma)[1]
        lls.append(-0.5 * (T * V * np.log(2 * np.pi) + T * s[1] + T * ld + s[2] - np.sum(y * (est["Phi"] @ y))))
        Sigma = oracle.sigma_update(est, T)
        Wl, rl = oracle.mstep([Xh[i] for i in mine], [sq[i] for i in mine], est["ES"], Sigma)
        new_rho = np.zeros(N)
        for j, i in enumerate(mine):
            W[i] = Wl[j]
            new_rho[i] = rl[j]
        tr = torch.from_numpy(new_rho)
        dist.all_reduce(tr)
        rho2 = tr.numpy()
    if rank == 0:
        out.put((np.array(lls), rho2, Sigma))
    dist.destroy_process_group()


def test_sharded_em_equals_single_process():
    case = synth.PlantedSpec("shard", 5, ("fixed", 0, 0), 60, 4, 4, (0.2, 1.0), 21)
    d = synth.planted_dataset(case, voxel_counts=[80, 130, 95, 110, 70])
    ref = oracle.fit(d["X"], d["W0"], case.n_iter)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_em, args=(r, 2, port, d["X"], d["W0"], case.n_iter, q)) for r in range(2)]
    for p in procs:
        p.start()
    lls, rho2, Sigma = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    np.testing.assert_allclose(lls, ref["ll"], rtol=1e-10)
    np.testing.assert_allclose(rho2, ref["rho2"], rtol=1e-9)
    np.testing.assert_allclose(Sigma, ref["Sigma_s"], rtol=1e-8, atol=1e-12)


def _bench_max(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out.put((rank, bench.max_over_ranks(10.0 + rank, world, device="cpu")))
    dist.destroy_process_group()


def test_bench_time_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_max, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 11.0, 1: 11.0}
