"""Coil sharding of one problem over several ranks (host logic, torch.distributed).

E = (I kron A) S sums over coils (Sec. II-G), and so do the products built on it:
grad_omega = sum_c Re{conj(v_c) (-i) A(s_c . x . r^[d])} and grad_x = sum_c conj(s_c) A' v_c
(Eq. (e,jac,Ax,v)).  A problem with many coils can therefore be split by coils: every
rank runs the VJP on its own contiguous block of coils (its maps and its rows of v),
and one all-reduce (sum) of grad_omega ([D][M] floats) and grad_x ([N] complex) gives
the all-coil result.  The forward y = E x needs no exchange: each rank owns its coils'
rows of y.
"""
import torch


def coil_slice(C, rank, world):
    """The contiguous block of coils rank `rank` of `world` owns (sizes differ by at most one)."""
    if not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(int(C), int(world))
    lo = rank * base + min(rank, extra)
    return slice(lo, lo + base + (1 if rank < extra else 0))


def allreduce_vjp(grad_omega, grad_x, group=None):
    """Sums the per-rank coil-block gradients in place over the group and returns them.

    grad_x is complex; it is reduced as its real view, so every backend that sums floats
    (gloo, nccl) can carry it."""
    import torch.distributed as dist
    if grad_omega is not None:
        dist.all_reduce(grad_omega, op=dist.ReduceOp.SUM, group=group)
    if grad_x is not None:
        view = torch.view_as_real(grad_x) if grad_x.is_complex() else grad_x
        dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
    return grad_omega, grad_x
