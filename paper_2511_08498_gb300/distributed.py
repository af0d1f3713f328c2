"""Wavelength-sharded Lambda iteration over several GPUs (one process per GPU).

Wavelength batches are independent in the formal solution (the paper batches
them, Section 4.1), so each rank solves a contiguous range of whole batches.
The radiative-rate reduction Jbar_l = sum_k w_k phi_k J_k is linear in J with
weights fixed by the full wavelength grid, so each rank reduces its own J
(zero at the other ranks' wavelengths) over the full grid and one float64
sum-allreduce of the [n_line][n_cells] rates gives every rank the exact total;
the statistical-equilibrium solve then runs on every rank, leaving identical
populations everywhere.  That allreduce is the only exchange.  Emissivity and
opacity are evaluated for the full grid on every rank (a cheap elementwise
kernel whose line-profile normalisation needs every sample of a line).

With one rank (or without an initialised process group) the reduction is a no-op.
"""

from __future__ import annotations

import numpy as np
import torch

from . import api


def wavelength_shard(n_lambda: int, W: int, rank: int, world: int):
    """Contiguous wavelength range [l0, l1) of whole batches of W for this rank;
    batches are split as evenly as possible (the first ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    n_batch = -(-n_lambda // W)
    base, extra = divmod(n_batch, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return min(b0 * W, n_lambda), min(b1 * W, n_lambda)


def allreduce_sum_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over the ranks of the default (or given) process group; a no-op
    for one rank or when torch.distributed is not initialised."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def reduce_scalar(x: float, op: str = "sum", group=None) -> float:
    """A Python number reduced over the ranks ("sum" or "max"); the value itself for
    one rank.  The tensor lives where the group's backend wants it (CUDA for NCCL)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1):
        return x
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX, group=group)
    return float(t.item())


def lambda_iteration_sharded(ctx, atom, lam_nm, tag, T, ne, nh, nx: int, nz: int, dirs, weights, n_iter: int,
                             rank: int = 0, world: int = 1, W: int = 8, max_mip: int = 3, iod: float = 1e-2,
                             chi_ds_min: float = 0.25, band=None, storage: int = api.STORE_F32, reduce=None,
                             pops=None):
    """The accelerated Lambda iteration of :func:`api.lambda_iteration` with this
    rank's wavelength batches only; ``reduce`` (default :func:`allreduce_sum_`)
    sums the float64 rates over the ranks.  Returns the float64 populations."""
    reduce = allreduce_sum_ if reduce is None else reduce
    lam_nm = np.asarray(lam_nm, dtype=np.float64)
    tag = np.asarray(tag, dtype=np.int32)
    L = lam_nm.size
    l0, l1 = wavelength_shard(L, W, rank, world)
    n = nx * nz
    if pops is None:
        pops = api.lte_populations(ctx, atom, T, nh)
    eta = torch.empty((L, n), dtype=torch.float32, device=T.device)
    chi = torch.empty_like(eta)
    J = torch.zeros_like(eta)  # zero outside [l0, l1) for good
    grid = mips = jbar = None
    for _ in range(n_iter):
        api.atom_eta_chi(ctx, atom, lam_nm, tag, T, ne, pops, eta, chi)
        if l1 > l0:
            e, c = eta[l0:l1], chi[l0:l1]
            grid = api.grid_build(ctx, nx, nz, e, c, out=grid)
            mips = api.mips_build(ctx, grid, e, c, W, max_mip, iod, iod, chi_ds_min, out=mips, storage=storage)
            api.formal_solve_hdda(ctx, grid, mips, dirs, weights, J=J[l0:l1], band=band)
        jbar = api.rates_accumulate(ctx, atom, lam_nm, tag, T, J, out=jbar)
        reduce(jbar)
        pops = api.se_solve(ctx, atom, T, ne, nh, jbar, out=pops)
    return pops
