"""The Omega split of one problem over several GPUs (host plumbing).

Eq. sd sums independent terms over (W, q); every (q, W) ladder needs only
G~ and its own bosonic plane.  So each rank owns a contiguous range of
bosonic planes (a handle created with ``w_range``), runs the bubble and the
ladders of its planes, and the per-rank shares of Eq. sd are summed by one
all-reduce of Sigma~ [n_w][N] (complex128) per pass; every rank then applies
the mixing, the residual and Eq. dyson to the same sum (df_sigma_finish), so
G~ stays replicated.  The reduction goes through ``torch.distributed``
(NCCL on GPUs, gloo on the host); this module does none of the method's
arithmetic.
"""
from __future__ import annotations

from typing import Tuple


def omega_partition(n_bos: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous bosonic range [lo, hi) of `rank`: n_bos planes over `world`
    ranks, sizes differing by at most one (the first n_bos % world ranks take
    one more).  A rank beyond n_bos gets an empty range (lo == hi)."""
    if n_bos < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("need n_bos >= 1, world >= 1 and 0 <= rank < world")
    base, extra = divmod(n_bos, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def allreduce_sum(x, group=None):
    """Sum a complex128 array over the ranks of `group`, in place.

    x is a torch tensor (complex128, contiguous; a CUDA tensor under NCCL, a
    CPU tensor under gloo); the sum runs on its float64 view.  Without an
    initialised process group (one rank) x is already the sum."""
    import torch
    import torch.distributed as dist
    if not x.is_contiguous():
        raise ValueError("allreduce_sum needs a contiguous tensor")
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(torch.view_as_real(x), op=dist.ReduceOp.SUM, group=group)
    return x


def split_pass(d, group=None):
    """One loop pass of a range handle ``d`` (paper_1507_00895_gb300.df.DualFermion
    created with ``w_range``): the bubble and the ladders of its planes, its share
    of Eq. sd on the device, the all-reduce, then mixing, residual and Dyson.
    Returns the residual (the same on every rank)."""
    import torch
    part = torch.empty((d.n_w, d.N), dtype=torch.complex128, device="cuda")
    d.bubble()
    d.bse(3)
    d.sigma_partial(part)
    allreduce_sum(part, group)
    return d.sigma_finish(part)
