"""The N > 1 bench path on CPU (gloo, world size 2): every rank gets the
slowest rank's time, the whole-job value counts all ranks' units, and the
reference arm prints on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    v = bench.weak_scaling_value(world, 8, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 8 / 15.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.weak_scaling_value(1, 8, 2.0) == 4.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import argparse

    import bench
    bench.run_reference(argparse.Namespace(steps=1, warmup=0), 1, 2)
    assert capsys.readouterr().out == ""


# ------------------------------------------- HCovMtrx sharded over row blocks

def test_row_block_shares_cover_every_block_once():
    from paper_2305_17341_gb300.sharding import row_blocks_of_rank
    for nrb in range(1, 20):
        for world in range(1, 9):
            shares = [row_blocks_of_rank(nrb, r, world) for r in range(world)]
            got = [l for lo, hi in shares for l in range(lo, hi)]
            assert got == list(range(nrb))
            sizes = [hi - lo for lo, hi in shares]
            assert max(sizes) - min(sizes) <= 1


def _cov_setup():
    """The small HCovMtrx case both ranks and the parent build identically:
    logN 10, q 60 + 7x40, p 60, 8x8 blocks, a ragged 20 x 16 dataset (3 row
    blocks, the last zero-padded; 2 feature blocks)."""
    import numpy as np

    from oracle.ckks import CKKS, Params
    from oracle.hmm import matmul_rot_steps, transpose_rot_steps
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    P = Params(10, [60] + [40] * 7, [60])
    he = CKKS(P, 5)
    n, n1 = 8, 2
    steps = set(matmul_rot_steps(n, n1, n1, P.S)) | set(transpose_rot_steps(n, n1, P.S))
    i = 1
    while i < n * n:
        steps |= {i % (n * n), (-i) % (n * n)}
        i <<= 1
    for st in sorted(steps - {0}):
        he.gen_rotation_key(st)
    he.gen_relin_key()
    X = lowrank_dataset(20, 16, 9)
    s, k = X.shape[0], 2
    nrb = -(-s // n)
    Xp = np.zeros((nrb * n, k * n))
    Xp[:s] = X
    blocks = []
    for l in range(nrb):
        row = []
        for j in range(k):
            z = np.zeros(P.S)
            z[: n * n] = Xp[l * n:(l + 1) * n, j * n:(j + 1) * n].ravel()
            row.append(he.encrypt_slots(z, P.L, obj=100 + l * k + j))
        blocks.append(row)
    return P, he, n, n1, X, s, k, nrb, blocks


def _cov_worker(rank, world, port, q):
    """One rank of the sharded HCovMtrx on the CPU: the oracle stands in for
    the GPU part of each rank (its share of the row blocks), the product's
    sharding module does the partition and the modular all-reduce, the
    oracle finishes."""
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.ckks import Ct
        from oracle.pca import PCA
        from paper_2305_17341_gb300.sharding import modular_allreduce, row_blocks_of_rank
        P, he, n, n1, X, s, k, nrb, blocks = _cov_setup()
        lo, hi = row_blocks_of_rank(nrb, rank, world)
        pca = PCA(he)
        upper, sums = pca.covariance_partial(blocks[lo:hi], s, n, n1, n1)
        # this rank's part alone, finished without the others'
        alone = pca.covariance_finish(upper, sums, s, n, n1, blocks[0][0].level)

        def summed(ct):
            r = modular_allreduce(np.stack([ct.c0, ct.c1]), P.q[: ct.level + 1])
            return Ct(r[0], r[1], ct.level, ct.scale, ct.period)

        upper = {key: summed(ct) for key, ct in sorted(upper.items())}
        sums = [summed(ct) for ct in sums]
        C = pca.covariance_finish(upper, sums, s, n, n1, blocks[0][0].level)
        q.put((rank, (lo, hi), [[np.stack([C[a][b].c0, C[a][b].c1]) for b in range(k)] for a in range(k)],
               np.stack([alone[0][0].c0, alone[0][0].c1])))
    finally:
        dist.destroy_process_group()


def test_sharded_covariance_equals_single_process():
    """HCovMtrx with its 3 row blocks split over two gloo ranks (2 + 1): the
    modular all-reduce of the partial X^T X and column-sum residues gives,
    on every rank, the single-process covariance word for word, which
    decrypts to FP64 Xc^T Xc / s within 1e-4; one rank's part finished
    alone does not."""
    import numpy as np

    from oracle.pca import PCA
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_cov_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(2)), key=lambda r: r[0])
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [(0, 2), (2, 3)]
    P, he, n, n1, X, s, k, nrb, blocks = _cov_setup()
    whole = PCA(he).covariance(blocks, s, n, n1, n1)
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / s
    for rank, _, C, alone in res:
        for a in range(k):
            for b in range(k):
                assert np.array_equal(C[a][b], np.stack([whole[a][b].c0, whole[a][b].c1])), (rank, a, b)
        assert not np.array_equal(alone, np.stack([whole[0][0].c0, whole[0][0].c1]))
    for a in range(k):
        for b in range(k):
            d = he.decrypt_slots(whole[a][b]).real[: n * n].reshape(n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4
