"""Multi-rank logic on CPU (gloo, world size 2, 127.0.0.1): the subject
sharding of Algorithm 1 (D-SRM) with its one exchange per iteration gives the
single-process EM result, and bench.py's max-over-ranks timing agrees on all
ranks.  No GPU is used.  The sharded fit runs through the library's host
driver (shard.fit_sharded) and the contract of its sharded E-step calls; an
oracle-backed stand-in implements that contract on the CPU."""
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


class OracleShard:
    """The sharded E-step contract of the library (srm_estep_partial /
    srm_estep_finish / srm_mstep, include/srm.h) over one process's subjects,
    with the FP64 oracle's arithmetic on CPU tensors: test infrastructure
    that lets the host driver (shard.fit_sharded) and its all-reduce run over
    gloo without a GPU."""

    def __init__(self, X, W0, mine):
        self.mine = list(mine)
        self.Xh = [oracle.center(X[i])[0] for i in self.mine]
        self.sq = [float(np.sum(x * x)) for x in self.Xh]
        self.W = [W0[i].astype(np.float64) for i in self.mine]
        self.rho2 = np.ones(len(self.mine))
        self.k, self.T = W0[0].shape[1], X[0].shape[1]
        self.Sigma = np.eye(self.k)
        self.ll = []

    def shard_buffers(self):
        return torch.zeros((self.k, self.T), dtype=torch.float64), torch.zeros(4, dtype=torch.float64)

    def estep_partial(self, y, sums):
        yl = np.zeros((self.k, self.T))
        for x, w, r in zip(self.Xh, self.W, self.rho2):
            yl += (w.T @ x) / r
        y.copy_(torch.from_numpy(yl))
        v = np.array([x.shape[0] for x in self.Xh], dtype=np.float64)
        sums.copy_(torch.tensor([np.sum(1.0 / self.rho2), np.sum(v * np.log(self.rho2)),
                                 np.sum(np.array(self.sq) / self.rho2), np.sum(v)]))

    def estep_finish(self, y, sums):
        y, s = y.numpy(), sums.numpy()
        k, T = self.k, self.T
        rho0 = s[0]
        Phi = np.linalg.inv(np.linalg.inv(self.Sigma) + rho0 * np.eye(k))
        est = {"y": y, "rho0": rho0, "Phi": Phi, "ES": self.Sigma @ (np.eye(k) - rho0 * Phi) @ y}
        ld = np.linalg.slogdet(np.eye(k) + rho0 * self.Sigma)[1]
        self.ll.append(-0.5 * (T * s[3] * np.log(2 * np.pi) + T * s[1] + T * ld + s[2] - np.sum(y * (Phi @ y))))
        self.est = est

    def mstep(self):
        self.Sigma = oracle.sigma_update(self.est, self.T)
        self.W, self.rho2 = oracle.mstep(self.Xh, self.sq, self.est["ES"], self.Sigma)


def _sharded_em(rank, world, port, X, W0, n_iter, out):
    from paper_1608_04647_gb300.shard import fit_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = shard_subjects([x.shape[0] for x in X], world)
    model = OracleShard(X, W0, plan[rank])
    fit_sharded(model, n_iter, dist.all_reduce)
    out.put((rank, np.array(model.ll), dict(zip(model.mine, model.rho2)), model.Sigma))
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
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rho2 = np.zeros(len(d["X"]))
    for rank, lls, r, Sigma in res:
        # every rank holds the whole likelihood trace and Sigma_s
        np.testing.assert_allclose(lls, ref["ll"], rtol=1e-10)
        np.testing.assert_allclose(Sigma, ref["Sigma_s"], rtol=1e-8, atol=1e-12)
        for i, v in r.items():
            rho2[i] = v
    np.testing.assert_allclose(rho2, ref["rho2"], rtol=1e-9)


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
