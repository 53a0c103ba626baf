"""The row-partitioned calls (scqr3_gram_partial, scqr3_apply_pass): the
data-parallel structure of the method (Sec. 1: the Gram matrix of a
row-partitioned X is the sum of its blocks' Gram matrices; Sec. 7.1, Table 8:
one reduction of n(n+1)/2 values per pass, the Cholesky replicated, each block
solved locally).

X is split into uneven row blocks; each block gets its own workspace (one
"rank"), the Gram vectors are summed between the calls, and the stacked Q and
the common R are compared with scqr3_factor on the whole X and with the CPU
oracle, at the FP64 parity tolerances (the blocks' partial sums add in another
order than the single call's, so the results agree to rounding, not bit for
bit). One test runs two gloo processes on the GPU, each driving the library on
its own rows, with the sums going through torch.distributed; their kernels
never wait on each other (the reduction is on the host)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1809_11085_gb300 import scqr3  # noqa: E402
from paper_1809_11085_gb300.testmat import block_diag_spd, testmat  # noqa: E402

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1809_11085_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_shards(X, bounds, B=None, normb=0.0, **kw):
    """The partitioned calls for row blocks [bounds[i], bounds[i+1]) of X, in
    one process: the 'allreduce' sums the blocks' Gram vectors on the device."""
    m, n = X.shape
    parts = [(a, b) for a, b in zip(bounds[:-1], bounds[1:])]
    Xs = [X[a:b] for a, b in parts]
    Bs = [None if B is None else B[a // B.shape[1]:b // B.shape[1]] for a, b in parts]
    wss = [scqr3.ShardWorkspace(b - a, n, Bi, normb, kw.get("precision", 0), kw.get("max_passes", 0))
           for (a, b), Bi in zip(parts, Bs)]
    Qs = [torch.empty_like(x) for x in Xs]
    Rs = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in parts]
    for x, ws, Bi in zip(Xs, wss, Bs):
        scqr3.gram_partial(x, ws, Bi, normb=normb, **kw)
    G = sum(ws.G for ws in wss)
    for ws in wss:
        ws.G.copy_(G)
    infos = None
    for k in range(kw.get("max_passes", 0) or 6):
        for x, q, r, ws, Bi in zip(Xs, Qs, Rs, wss, Bs):
            scqr3.apply_pass(k, m, x, q, r, ws, Bi, normb=normb, **kw)
        torch.cuda.synchronize()
        infos = [scqr3.Info.from_bytes(ws.info.cpu().numpy().tobytes()) for ws in wss]
        assert len({(i.status, i.passes, i.more) for i in infos}) == 1, infos  # the same decisions
        if not infos[0].more:
            break
        G = sum(ws.G_next for ws in wss)
        for ws in wss:
            ws.G.copy_(G)
    for r in Rs[1:]:
        assert torch.equal(r, Rs[0])  # the Cholesky is replicated bit for bit
    return torch.cat(Qs), Rs[0], infos[0]


@pytest.mark.parametrize("precision", [scqr3.PREC_FP64, scqr3.PREC_TC])
@pytest.mark.parametrize("n", [8, 40, 64, 100])
def test_shards_match_single_call_and_oracle(precision, n):
    m, kappa = 60011, 1e8
    Xh = testmat(m, n, kappa, seed=9900 + n)
    X = torch.from_numpy(Xh).cuda()
    Qs, Rs, inf = run_shards(X, [0, 20000, 20007, 47000, m], precision=precision)
    Q1, R1, i1 = scqr3.factor(X, precision=precision)
    torch.cuda.synchronize()
    assert inf.status == 0 and inf.passes == i1.passes == 3
    Qs, Rs, R1 = Qs.cpu().numpy(), Rs.cpu().numpy(), R1.cpu().numpy()
    Qo, Ro, st, tr = oracle.scqr3(Xh)
    assert st == 0
    assert np.linalg.norm(Rs - R1) / np.linalg.norm(R1) <= 1e-12
    assert np.linalg.norm(Rs - Ro) / np.linalg.norm(Ro) <= 1e-12
    # Q itself is determined only to about kappa u (Q = X R^-1 with R known to
    # u kappa in its small singular directions); its defining properties are
    # held to the FP64 tolerances below
    assert np.linalg.norm(Qs - Q1.cpu().numpy()) / np.linalg.norm(Q1.cpu().numpy()) <= 10 * n * kappa * U
    assert np.linalg.norm(Qs.T @ Qs - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Qs @ Rs) / np.linalg.norm(Xh) <= 1e-13


def test_shards_wide_and_ill_conditioned():
    """n = 200 (the 256-padded FP64 kernels), and kappa = 1e15 where the
    breakdown rule adds shifted passes: every block takes the same ones."""
    for (m, n, kappa, seed) in ((30000, 200, 1e6, 9950), (60000, 64, 1e15, 9951)):
        Xh = testmat(m, n, kappa, seed=seed)
        X = torch.from_numpy(Xh).cuda()
        Qs, Rs, inf = run_shards(X, [0, 11111, 29000, m])
        Q1, R1, i1 = scqr3.factor(X)
        torch.cuda.synchronize()
        assert inf.status == 0 and inf.passes == i1.passes
        Qs, Rs = Qs.cpu().numpy(), Rs.cpu().numpy()
        assert np.linalg.norm(Qs.T @ Qs - np.eye(n), 2) <= 1e-13
        assert np.linalg.norm(Xh - Qs @ Rs) / np.linalg.norm(Xh) <= 1e-13
        assert np.linalg.norm(Rs - R1.cpu().numpy()) / np.linalg.norm(R1.cpu().numpy()) <= 100 * n * kappa * U


@pytest.mark.parametrize("precision", [scqr3.PREC_FP64, scqr3.PREC_TC])
def test_shards_oblique_block_diagonal(precision):
    """Block-diagonal B with each block's rows whole B blocks and the caller's
    ||B||_2 (the same on every rank): Q is B-orthonormal and R matches the
    oracle."""
    m, n, bs = 48000, 64, 8
    Xh = testmat(m, n, 1e8, seed=9960)
    Bh = block_diag_spd(m, bs, seed=9961)
    normb = float(max(np.linalg.eigvalsh(Bh).max(axis=1)))
    X, B = torch.from_numpy(Xh).cuda(), torch.from_numpy(Bh).cuda()
    Qs, Rs, inf = run_shards(X, [0, 8000, 30008, m], B=B, normb=normb, precision=precision)
    Qo, Ro, st, tr = oracle.scqr3(Xh, Bblk=Bh, normb=normb)
    assert st == 0 and inf.status == 0 and inf.passes == tr["passes"]
    Q, R = Qs.cpu().numpy(), Rs.cpu().numpy()
    BQ = np.einsum("kij,kjn->kin", Bh, Q.reshape(-1, bs, n)).reshape(Q.shape)
    assert np.linalg.norm(Q.T @ BQ - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(R - Ro) / np.linalg.norm(Ro) <= 1e-12


def test_shard_rejections():
    X = torch.zeros((1000, 16), dtype=torch.float64, device="cuda")
    ws = scqr3.ShardWorkspace(1000, 16)
    with pytest.raises(scqr3.ScqrError) as e:  # mixed forms are not partitioned
        scqr3.ShardWorkspace(1000, 16, precision=scqr3.PREC_MIXED)
    assert e.value.code == scqr3.E_UNSUPPORTED
    B = torch.from_numpy(block_diag_spd(1000, 8, seed=1)).cuda()
    with pytest.raises(scqr3.ScqrError) as e:  # B without the caller's ||B||_2
        scqr3.gram_partial(X, ws, B)
    assert e.value.code == -5
    Q = torch.empty_like(X)
    R = torch.empty((16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(scqr3.ScqrError) as e:  # global m below the block's rows
        scqr3.apply_pass(0, 999, X, Q, R, ws)
    assert e.value.code == -3
    with pytest.raises(scqr3.ScqrError) as e:
        scqr3.apply_pass(6, 5000, X, Q, R, ws)
    assert e.value.code == -1


def _rank_main(rank, world, port, m, n, kappa, seed, outdir):
    import torch.distributed as dist

    from paper_1809_11085_gb300 import scqr3 as lib

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    Xh = testmat(m, n, kappa, seed=seed)
    bounds = [0, m // 3, m]  # uneven blocks
    a, b = bounds[rank], bounds[rank + 1]
    X = torch.from_numpy(Xh[a:b].copy()).cuda()

    def allreduce(t):
        h = t.cpu()
        dist.all_reduce(h)
        t.copy_(h)

    Q, R, info = lib.factor_sharded(X, m, allreduce, precision=lib.PREC_TC)
    torch.cuda.synchronize()
    np.save(os.path.join(outdir, "q%d.npy" % rank), Q.cpu().numpy())
    np.save(os.path.join(outdir, "r%d.npy" % rank), R.cpu().numpy())
    np.save(os.path.join(outdir, "i%d.npy" % rank), np.array([info.status, info.passes]))
    dist.destroy_process_group()


def test_two_gloo_processes_drive_the_library(tmp_path):
    import socket

    import torch.multiprocessing as mp

    m, n, kappa, seed = 40000, 48, 1e10, 9970
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.spawn(_rank_main, args=(2, port, m, n, kappa, seed, str(tmp_path)), nprocs=2, join=True)
    Q = np.concatenate([np.load(tmp_path / ("q%d.npy" % r)) for r in range(2)])
    R0, R1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    i0, i1 = np.load(tmp_path / "i0.npy"), np.load(tmp_path / "i1.npy")
    assert np.array_equal(R0, R1) and np.array_equal(i0, i1) and i0[0] == 0
    Xh = testmat(m, n, kappa, seed=seed)
    Qo, Ro, st, tr = oracle.scqr3(Xh)
    assert st == 0
    assert np.linalg.norm(Q.T @ Q - np.eye(n), 2) <= 1e-13
    assert np.linalg.norm(Xh - Q @ R0) / np.linalg.norm(Xh) <= 1e-13
    assert np.linalg.norm(R0 - Ro) / np.linalg.norm(Ro) <= 100 * n * kappa * U
