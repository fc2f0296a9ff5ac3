"""Receiver sharding over several GPUs (one process per GPU).

The field at a receiver depends on the scene and the transmitter only
(Eqs. 1-4 are evaluated per receiver), so one workload's receivers split into
contiguous ranges, one per rank, with no exchange during the evaluation:
each rank evaluates its range into its own output slice.  An optional
gather assembles the ranks' slices into the single-rank layout
[n_f][3][n_rx][2] on one rank.  The adjoint adds one sum of the parameter
gradients over the ranks (allreduce_gradients).
"""
import torch


def shard(n_rx, rank, world):
    """The contiguous receiver range [lo, hi) of `rank` of `world` ranks:
    sizes differ by at most one, ranks in order, every receiver once."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank %d of %d" % (rank, world))
    base, extra = divmod(int(n_rx), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def local_receivers(rx_soa, rank, world):
    """This rank's receivers of the [3][n_rx] array (a contiguous copy)."""
    lo, hi = shard(rx_soa.shape[1], rank, world)
    return rx_soa[:, lo:hi].contiguous() if isinstance(rx_soa, torch.Tensor) else rx_soa[:, lo:hi].copy()


def _dist():
    import torch.distributed as dist
    return dist if (dist.is_available() and dist.is_initialized()) else None


def gather_fields(E_local, n_rx, dst=0, group=None):
    """The ranks' field slices [n_f][3][hi - lo][2] assembled on rank `dst`
    into [n_f][3][n_rx][2] (the layout a single rank writes); None on the
    other ranks; the input itself on one process.  Slices are padded to the
    largest range for the collective and trimmed again."""
    dist = _dist()
    if dist is None or dist.get_world_size(group) == 1:
        return E_local
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    lo, hi = shard(n_rx, rank, world)
    if E_local.shape[2] != hi - lo:
        raise ValueError("rank %d holds %d receivers, its range is %d" % (rank, E_local.shape[2], hi - lo))
    width = shard(n_rx, 0, world)[1]          # rank 0's range is the largest
    pad = E_local.new_zeros((E_local.shape[0], E_local.shape[1], width, E_local.shape[3]))
    pad[:, :, :hi - lo] = E_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    if rank != dst:
        return None
    out = []
    for r in range(world):
        a, b = shard(n_rx, r, world)
        out.append(parts[r][:, :, :b - a])
    return torch.cat(out, dim=2)


def allreduce_gradients(tensors, group=None):
    """Sum each tensor over the ranks in place (no-op on one process)."""
    dist = _dist()
    if dist is None or dist.get_world_size(group) == 1:
        return tensors
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors
