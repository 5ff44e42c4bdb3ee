"""Several GPUs: replicas, and one graph sharded over ranks.

Independent graphs need nothing but a split of the work (each rank reorders
its own graphs).  One graph too large for a device shards by edges: each rank
computes first-occurrence keys over its edge range with global positions
(``boba_first_keys``), the key arrays are merged by an elementwise MIN
(all-reduce), and every rank then derives the same labels
(``boba_labels_from_keys``) and rewrites its own edges (``boba_relabel``).
The merge is the only exchange: 4n bytes per rank.

Keys are unsigned 32-bit with 0xFFFFFFFF for "not seen".  Collectives reduce
signed int32, so keys travel with their top bit flipped, which maps unsigned
order onto signed order (MIN commutes with the flip).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

FLIP = -0x80000000          # int32 with only the top bit set


def shard_bounds(total: int, rank: int, world: int):
    """Contiguous split of [0, total) into `world` near-equal ranges."""
    return total * rank // world, total * (rank + 1) // world


def keys_to_wire(key_i32: torch.Tensor) -> torch.Tensor:
    return torch.bitwise_xor(key_i32, FLIP)


def wire_to_keys(w: torch.Tensor) -> torch.Tensor:
    return torch.bitwise_xor(w, FLIP)


def merge_keys_min(key_i32: torch.Tensor, group=None) -> torch.Tensor:
    """Elementwise unsigned MIN of every rank's keys (int32 tensors holding uint32 bits)."""
    w = keys_to_wire(key_i32)
    dist.all_reduce(w, op=dist.ReduceOp.MIN, group=group)
    return wire_to_keys(w)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest value over all ranks (timing: the slowest rank sets the job time)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_reorder(src_shard, dst_shard, m_total: int, n: int, e0: int, group=None,
                    stream=None):
    """BOBA of one graph whose edges [e0, e0 + len) live on this rank.

    Returns (perm, src_out_shard, dst_out_shard); perm is the same on every rank.
    """
    from . import _p, _s, check, load, _ws
    lib = load()
    dev = src_shard.device
    key = torch.empty(n, dtype=torch.int32, device=dev)
    check(lib.boba_first_keys(_p(src_shard), _p(dst_shard), src_shard.numel(), e0, m_total + e0,
                              n, _p(key), 1, _s(stream)), "boba_first_keys")
    if dist.is_available() and dist.is_initialized():
        key = merge_keys_min(key, group)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    label = torch.empty(n, dtype=torch.int32, device=dev)
    buf = _ws(None, lib.boba_labels_workspace_bytes(m_total, n), dev)
    check(lib.boba_labels_from_keys(_p(key), m_total, n, _p(perm), _p(label), _p(buf), buf.numel(),
                                    _s(stream)), "boba_labels_from_keys")
    so, do = torch.empty_like(src_shard), torch.empty_like(dst_shard)
    check(lib.boba_relabel(_p(src_shard), _p(dst_shard), src_shard.numel(), n, _p(label), _p(so),
                           _p(do), _s(stream)), "boba_relabel")
    return perm, so, do
