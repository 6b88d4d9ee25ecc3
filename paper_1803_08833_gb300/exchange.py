"""The two-step spike exchange between shards on separate processes.

The paper's processes exchange spikes every time step in two steps (Sec. II-E):
each process first tells every process it can reach how many spikes it
emitted, then sends the spikes themselves (AER ids), so that every receiver
can size its buffers before the payload arrives; only processes whose tiles
lie within the stencil's reach talk to each other.  Here a process owns one
shard (a stripe of module rows, include/snn.h snn_shard_*): after
snn_shard_integrate its outbox holds the step's spike ids, the exchange below
moves them to the peer ranks over torch.distributed point-to-point messages
(any backend: gloo on CPU, NCCL between GPUs), and snn_shard_deliver
arborizes the received lists into the local ring.

Peers: shard q is a peer of shard k when some module row of q lies within the
stencil's row radius R of k's stripe; the relation is symmetric, so a rank
sends to exactly the ranks it receives from.
"""
from __future__ import annotations

import math


def stencil_row_radius(cfg: dict) -> int:
    """Largest |dy| of the cut-off disc dx^2 + dy^2 <= floor((cutoff / spacing)^2)."""
    q = float(cfg["cutoff_um"]) / float(cfg["spacing_um"])
    R2 = int(math.floor(q * q + 1e-9))
    R = 0
    while (R + 1) * (R + 1) <= R2:
        R += 1
    return R


def shard_rows(grid_h: int, n_shards: int, k: int):
    """Module rows [row0, row1) of shard k of an n-way split."""
    return grid_h * k // n_shards, grid_h * (k + 1) // n_shards


def peers(cfg: dict, n_shards: int, k: int):
    """Shards (k included) whose spikes can reach shard k, in index order."""
    H = int(cfg["grid_h"])
    R = stencil_row_radius(cfg)
    r0, r1 = shard_rows(H, n_shards, k)
    lo, hi = max(0, r0 - R), min(H, r1 + R)
    out = []
    for q in range(n_shards):
        a, b = shard_rows(H, n_shards, q)
        if a < hi and b > lo:
            out.append(q)
    return out


def exchange_spikes(ids, peer_ranks, group=None):
    """Sends this rank's spike ids (a 1-D int32 tensor on the backend's device)
    to every rank in peer_ranks and receives theirs: first the counts, then
    the ids.  Returns {rank: int32 tensor of its ids}; this rank is skipped if
    listed.  Non-blocking sends and receives are posted together and waited
    on, so no pairing order can deadlock."""
    import torch
    import torch.distributed as dist
    me = dist.get_rank(group)
    others = [q for q in peer_ranks if q != me]
    dev = ids.device
    n = torch.tensor([ids.numel()], dtype=torch.int64, device=dev)
    counts = {q: torch.zeros(1, dtype=torch.int64, device=dev) for q in others}
    reqs = [dist.isend(n, q, group=group) for q in others]
    reqs += [dist.irecv(counts[q], q, group=group) for q in others]
    for r in reqs:
        r.wait()
    out = {q: torch.empty(int(counts[q].item()), dtype=torch.int32, device=dev) for q in others}
    reqs = []
    if ids.numel() > 0:
        reqs += [dist.isend(ids, q, group=group) for q in others]
    reqs += [dist.irecv(out[q], q, group=group) for q in others if out[q].numel() > 0]
    for r in reqs:
        r.wait()
    return out
