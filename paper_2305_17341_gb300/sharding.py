"""HCovMtrx with its row blocks spread over several GPUs.

The block products of HCovMtrx for different row blocks are independent
(Sec. 5.2 runs them in parallel over the row blocks); only their sum over
the row blocks -- and, for the mean, the sum of the blocks themselves -- is
needed afterwards.  So each rank (one process per GPU, the rotation keys of
the covariance on every GPU) takes a contiguous share of the row blocks and
runs he_covariance_partial on it; one all-reduce adds the parts residue by
residue modulo each prime; he_covariance_finish then gives the covariance
blocks, word for word those of he_covariance on all row blocks at once
(modular addition is exact and the transforms between the residue forms
are linear).

The residues of a part are below 2^60, so the sum over at most 8 ranks
stays below 2^63 and is carried exactly by a signed 64-bit all-reduce
before the reduction modulo each prime.
"""
import numpy as np

from . import _lib

MAX_RANKS = 8


def row_blocks_of_rank(n_row_blocks, rank, world):
    """The contiguous share [lo, hi) of `n_row_blocks` row blocks that rank
    `rank` of `world` takes: the first n_row_blocks % world ranks one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of %d" % (rank, world))
    base, extra = divmod(n_row_blocks, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def modular_allreduce(residues, moduli, group=None):
    """Sum over the ranks of `residues` (uint64, shape [..., limbs, N], every
    word below the modulus of its limb), reduced limb by limb modulo
    `moduli` (one per limb).  Runs on the process group's backend: CUDA
    tensors for NCCL, host tensors otherwise.  Returns uint64 [..., limbs, N]."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if world > MAX_RANKS:
        raise ValueError("at most %d ranks (sums of 60-bit residues must stay below 2^63)" % MAX_RANKS)
    moduli = np.asarray(moduli, dtype=np.uint64)
    if int(moduli.max()) >= 1 << 60:
        raise ValueError("moduli must be below 2^60")
    r = np.ascontiguousarray(residues, dtype=np.uint64)
    if r.shape[-2] != len(moduli):
        raise ValueError("one modulus per limb")
    device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(r.view(np.int64).copy()).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    s = t.cpu().numpy().view(np.uint64)
    return s % moduli[:, None]


def covariance_sharded(ctx, blocks, n_row_blocks, k, n, s, centered, n1z, n1t, group=None, relin_once=False,
                       dcd_z=0, dcd_t=0):
    """HCovMtrx over this rank's row blocks ([l][j] order, l-major; at least
    one row block per rank; s = the dataset's total row count), summed with
    the other ranks' parts: returns the k*k covariance blocks (every rank
    gets them)."""
    if n_row_blocks < 1:
        raise ValueError("every rank needs at least one row block")
    upper, colsum = _lib.he_covariance_partial(ctx, blocks, n_row_blocks, k, n, s, centered, n1z, n1t,
                                               relin_once, dcd_z, dcd_t)
    q, _ = _lib.he_ctx_primes(ctx)

    def summed(h):
        level, scale, period = _lib.he_ct_info(h)
        r = _lib.he_ct_export(ctx, h)
        _lib.he_ct_free(h)
        r = modular_allreduce(r, [int(x) for x in q[: level + 1]], group)
        return _lib.he_ct_import(ctx, r, level, scale, period)

    upper = [summed(h) for h in upper]
    colsum = [summed(h) for h in colsum]
    block_level = _lib.he_ct_info(blocks[0])[0]
    try:
        return _lib.he_covariance_finish(ctx, upper, colsum, k, n, s, centered, n1z, n1t, block_level, relin_once,
                                         dcd_z, dcd_t)
    finally:
        for h in upper + colsum:
            _lib.he_ct_free(h)
