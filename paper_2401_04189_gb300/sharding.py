"""Sharding of the exchange apply over ranks (one process per GPU).

Every (target i, occupied j) pair is independent and W_i sums over j only (Eq. hadam), so the
targets are split across the ranks with the occupied block replicated on each: a rank applies
K to its own targets and needs no data-path exchange.  The exchange energy
E_x = 1/2 sum_i sum_x w(x) psi_i(x) W_i(x) is the sum of the ranks' shares, combined with one
float64 all-reduce, the only collective of the sharded path.
"""
import torch


def target_range(n_tgt: int, world: int, rank: int):
    """Contiguous, balanced [start, stop) slice of the targets owned by `rank` (the first
    n_tgt % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world or n_tgt < 0:
        raise ValueError(f"invalid sharding: n_tgt={n_tgt}, world={world}, rank={rank}")
    base, extra = divmod(n_tgt, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def energy_share(ctx, psi_tgt: torch.Tensor, W_tgt: torch.Tensor) -> torch.Tensor:
    """This rank's share 1/2 sum_i sum_x w(x) psi_i(x) W_i(x) over its targets, computed by the
    library (tx_exchange_energy_from_w) as a float64 device scalar."""
    from ._lib import tx_exchange_energy_from_w
    return tx_exchange_energy_from_w(ctx, psi_tgt, W_tgt)


def combine_energy(e_local: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the ranks' energy shares (float64 all-reduce over `group`); a copy of e_local
    when no process group with more than one rank is initialised."""
    import torch.distributed as dist
    t = e_local.detach().clone().to(torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def exchange_apply_sharded(ctx, psi_occ: torch.Tensor, world: int, rank: int):
    """K applied to this rank's targets psi_occ[start:stop] with every occupied orbital:
    returns (start, stop, W_local)."""
    from ._lib import tx_exchange_apply
    a, b = target_range(psi_occ.shape[0], world, rank)
    if b == a:
        return a, b, psi_occ.new_empty((0,) + tuple(psi_occ.shape[1:]))
    return a, b, tx_exchange_apply(ctx, psi_occ, psi_occ[a:b])
