"""LED sharding of the Elfpie iteration across processes (one per GPU, or several on one GPU).

The fidelity gradient is a sum over LEDs (Eq. 9 for Psi, Eq. 18 for P) whose terms each
need one LED's image and crop (Sec. 3.4).  Every rank holds a handle of the same problem
with all measurements and the same state; per iteration it runs the tile work of its own
contiguous block of LEDs (``elf_shard_tiles``), the ranks all-gather the blocks' per-LED
results (tile gradients on the pupil support and fidelity cost partials; one exchange, no
reduction), every rank imports the other blocks and finishes the iteration
(``elf_shard_finish``: the sums over LEDs in LED order, the Hessian term, Eq. 19).  The
state after each iteration is therefore bitwise equal on every rank to a single handle's
``elf_step(h, 1)``.

The exchange goes through ``torch.distributed``: with NCCL the device buffers are gathered
in place on the current stream (the handle must have been created on it); with gloo they
are staged through host memory.  This module only partitions, moves bytes and calls the
library; every step of the method runs in the library's kernels.
"""
from __future__ import annotations

from . import elfpie as E


def led_blocks(n_led: int, world: int) -> list[tuple[int, int]]:
    """Contiguous, near-equal [k0, k1) LED ranges in rank order (the first ranks one LED longer;
    ranks beyond n_led get an empty range)."""
    if n_led < 0 or world < 1:
        raise ValueError("n_led >= 0 and world >= 1 required")
    q, r = divmod(n_led, world)
    out, k0 = [], 0
    for rank in range(world):
        k1 = k0 + q + (1 if rank < r else 0)
        out.append((k0, k1))
        k0 = k1
    return out


def all_gather_blocks(send, world: int, group=None):
    """All-gather equal-sized 1D tensors in rank order: returns a tensor [world, len(send)] whose
    row r is rank r's ``send``.  CUDA tensors with a non-NCCL backend are staged through host
    memory (gloo)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return send.reshape(1, -1)
    staged = send.is_cuda and dist.get_backend(group) != "nccl"
    src = send.cpu() if staged else send
    out = torch.empty((world, src.numel()), dtype=src.dtype, device=src.device)
    dist.all_gather(list(out.unbind(0)), src, group=group)
    return out.to(send.device) if staged else out


class ShardedElf:
    """Runs iterations of one problem with its LEDs split over the ranks of a process group.

    elf: this rank's handle (same problem, measurements and state on every rank).
    rank, world: this rank's place in the group (default: torch.distributed's).
    device: where the exchange buffer lives ("cuda": the library exports into device memory).
    """

    def __init__(self, elf: E.Elf, rank: int | None = None, world: int | None = None, group=None,
                 device: str = "cuda"):
        import torch
        import torch.distributed as dist
        if rank is None or world is None:
            if dist.is_available() and dist.is_initialized():
                rank, world = dist.get_rank(group), dist.get_world_size(group)
            else:
                rank, world = 0, 1
        self.elf, self.rank, self.world, self.group = elf, int(rank), int(world), group
        self.blocks = led_blocks(elf.K, self.world)
        self.k0, self.k1 = self.blocks[self.rank]
        self.row = elf.shard_row_floats()
        self.bmax = max(k1 - k0 for k0, k1 in self.blocks)
        self.send = torch.zeros(self.bmax * self.row, dtype=torch.float32, device=device)
        self.exchanged_bytes = 0

    def step(self, n_iter: int = 1):
        for _ in range(int(n_iter)):
            self.elf.shard_tiles(self.k0, self.k1)
            nl = self.k1 - self.k0
            if nl:
                self.elf.shard_export(self.k0, self.k1, self.send[:nl * self.row])
            allb = all_gather_blocks(self.send, self.world, self.group)
            self.exchanged_bytes += allb.numel() * 4
            for r, (k0, k1) in enumerate(self.blocks):
                if r != self.rank and k1 > k0:
                    self.elf.shard_import(k0, k1, allb[r, :(k1 - k0) * self.row].contiguous())
            self.elf.shard_finish()


def exchange_bytes_per_iteration(n_led: int, S: int, cluster: int) -> int:
    """Bytes one rank contributes to the exchange of one iteration, summed over ranks: every LED's
    tile gradients on the support (S complex) and its cost partials (one float pair per CTA of
    its cluster)."""
    return int(n_led) * 8 * (int(S) + int(cluster))


__all__ = ["led_blocks", "all_gather_blocks", "ShardedElf", "exchange_bytes_per_iteration"]
