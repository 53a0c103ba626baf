"""Multi-rank paths on the CPU (gloo, world size 2).

* The replica bookkeeping of `bench.py --gpus N`: every rank sees the slowest
  rank's time and the whole-job rows/s.
* The row-sharded form of the algorithm that a multi-GPU run would use (the
  paper's distributed structure, Sec. 1 and Sec. 7.1): each rank owns a block
  of rows, forms its partial Gram matrix, the partials are summed by an
  allreduce, every rank factors the same n x n matrix and solves its own rows.
  The result must be the unsharded factorization.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _run(fn, world=2, timeout=120):
    """Start `world` gloo ranks; read every rank's result before joining (a child
    that put data on a queue cannot exit until the data has been read)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    pc = mp.start_processes(fn, args=(world, port, q), nprocs=world, join=False, start_method="spawn")
    out = [q.get(timeout=timeout) for _ in range(world)]
    while not pc.join(timeout=timeout):
        pass
    return out


def _replica_worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    _init(rank, world, port)
    ms = [120.0, 175.5][rank]
    slow = bench.max_over_ranks(ms, dist, "cpu")
    q.put((rank, slow, bench.replica_value(1000, world, slow)))
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    res = sorted(_run(_replica_worker))
    for rank, slow, value in res:
        assert slow == 175.5
        assert value == pytest.approx(2 * 1000 / 0.1755)


def _sharded_worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import oracle
    from paper_1809_11085_gb300.testmat import testmat

    _init(rank, world, port)
    m, n = 3000, 12
    X = testmat(m, n, 1e11, seed=99)
    rows = np.array_split(np.arange(m), world)[rank]
    Qk = X[rows].copy()
    R = np.eye(n)
    plain = 0
    shifted = []
    for p in range(6):
        A = torch.from_numpy(oracle.gram(Qk))
        dist.all_reduce(A, op=dist.ReduceOp.SUM)  # the only exchange: n x n per pass
        A = A.numpy()
        if p == 0:
            Rt, fail = oracle.chol(A, oracle.shift(m, n, float(np.trace(A))))
            sh = 1
        else:
            Rt, fail = oracle.chol(A, 0.0)
            sh = 0
            if fail:
                Rt, fail = oracle.chol(A, oracle.shift(m, n, float(np.trace(A))))
                sh = 1
        assert fail == 0
        shifted.append(sh)
        Qk = oracle.trsm(Qk, Rt)
        R = oracle.trmm(Rt, R)
        plain = 0 if sh else plain + 1
        if plain == 2:
            break
    q.put((rank, rows, Qk, R, shifted))
    dist.destroy_process_group()


def test_row_sharded_factorization_equals_unsharded():
    import oracle
    from paper_1809_11085_gb300.testmat import testmat

    parts = sorted(_run(_sharded_worker), key=lambda t: t[0])
    m, n = 3000, 12
    X = testmat(m, n, 1e11, seed=99)
    Q = np.empty((m, n))
    for rank, rows, Qk, R, shifted in parts:
        Q[rows] = Qk
    R0 = parts[0][3]
    assert np.array_equal(R0, parts[1][3])  # every rank holds the same R
    assert parts[0][4] == parts[1][4]
    Qo, Ro, st, tr = oracle.scqr3(X)
    assert st == 0 and tr["shifted"] == parts[0][4]
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) < 1e-14
    assert np.linalg.norm(X - Q @ R0) / np.linalg.norm(X) < 1e-15
    assert np.linalg.norm(R0 - Ro) / np.linalg.norm(Ro) < 1e-4  # kappa = 1e11: rounding-order level
