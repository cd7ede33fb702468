"""Spatial decomposition of one scene over several ranks (slabs along x).

The dual-grid step couples particles only through grid nodes within one cell
of them, so a scene splits into slabs of cells along x, one per rank, with
three exchanges per step:

  1. after P2G, a reverse halo sum: a rank's particles in cells [lo, hi) add
     to nodes lo - 1 .. hi + 1 (G- and G+ nodes of the compact kernel, the
     27-node quadratic stencil alike), so the node layers outside [lo, hi)
     are sent to the ranks that own them and added there;
  2. after the grid update, a halo fill: each rank receives the updated
     velocities of the node layers it touches but does not own;
  3. after G2P, a migration: particles whose new cell lies in another slab
     move to its owner.

Node layer i (along x) is owned by the rank whose cell range [lo, hi)
contains i; the last rank also owns the layer at res.  Slabs are multiples
of 4 cells (whole particle blocks).  Everything here is bookkeeping on
tensors with the node layers along the last-but-one axis of a
(grids, nz, ny, nx, components) array, exchanged with torch.distributed
point-to-point calls (gloo on the host, NCCL between GPUs: plain copies, no
multicast).  The arithmetic of the step itself is the caller's.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import torch
import torch.distributed as dist

HALO_BELOW = 1  # node layers below a slab its particles touch
HALO_ABOVE = 2  # and above


def slab_ranges(res: int, world: int) -> List[Tuple[int, int]]:
    """Cell ranges [lo, hi) along x, one per rank, in whole 4-cell blocks and
    as even as the block count allows."""
    nblk = -(-res // 4)
    if world > nblk:
        raise ValueError("more ranks than particle blocks along x")
    out, b0 = [], 0
    for r in range(world):
        b1 = b0 + nblk // world + (1 if r < nblk % world else 0)
        out.append((4 * b0, min(res, 4 * b1)))
        b0 = b1
    return out


def owner_of_cells(cx: torch.Tensor, ranges: Sequence[Tuple[int, int]]) -> torch.Tensor:
    """Rank owning each cell index along x."""
    his = torch.tensor([hi for _, hi in ranges], dtype=cx.dtype, device=cx.device)
    return torch.searchsorted(his, cx, right=True).clamp_(max=len(ranges) - 1)


def owned_layers(rank: int, ranges: Sequence[Tuple[int, int]], res: int) -> Tuple[int, int]:
    """Node layers [a, b) along x owned by rank."""
    lo, hi = ranges[rank]
    return lo, (res + 1 if rank == len(ranges) - 1 else hi)


def _exchange(sends: Dict[int, torch.Tensor], recv_shapes: Dict[int, Tuple[int, ...]], like: torch.Tensor,
              group=None) -> Dict[int, torch.Tensor]:
    """Post every send and receive, then wait: peer -> received tensor."""
    reqs, got = [], {}
    for peer, shape in recv_shapes.items():
        got[peer] = torch.empty(shape, dtype=like.dtype, device=like.device)
        reqs.append(dist.irecv(got[peer], src=peer, group=group))
    for peer, t in sends.items():
        reqs.append(dist.isend(t.contiguous(), dst=peer, group=group))
    for r in reqs:
        r.wait()
    return got


def halo_sum(grid: torch.Tensor, rank: int, ranges: Sequence[Tuple[int, int]], res: int, group=None) -> torch.Tensor:
    """Reverse halo exchange after P2G.  grid: this rank's contributions on
    the full node range, shape (..., nx = res + 1, C) with x the second last
    axis.  Layers this rank does not own are sent to their owners; what the
    neighbours send for this rank's layers is added.  Returns grid with the
    owned layers complete (the others are left as they were)."""
    world = len(ranges)
    a, b = owned_layers(rank, ranges, res)
    sends, shapes = {}, {}
    for peer in (rank - 1, rank + 1):
        if 0 <= peer < world:
            pa, pb = owned_layers(peer, ranges, res)
            # layers of peer this rank's particles reach, and the reverse
            lo_t, hi_t = max(pa, a - HALO_BELOW), min(pb, b + HALO_ABOVE)
            sends[peer] = grid[..., lo_t:hi_t, :]
            lo_r, hi_r = max(a, pa - HALO_BELOW), min(b, pb + HALO_ABOVE)
            shapes[peer] = tuple(grid.shape[:-2]) + (max(0, hi_r - lo_r), grid.shape[-1])
    got = _exchange(sends, shapes, grid, group)
    out = grid.clone()
    for peer, t in got.items():
        pa, pb = owned_layers(peer, ranges, res)
        lo_r, hi_r = max(a, pa - HALO_BELOW), min(b, pb + HALO_ABOVE)
        out[..., lo_r:hi_r, :] += t
    return out


def halo_fill(grid: torch.Tensor, rank: int, ranges: Sequence[Tuple[int, int]], res: int, group=None) -> torch.Tensor:
    """Forward halo exchange after the grid update: each rank receives from
    its neighbours the layers it touches but does not own (and sends them
    the layers of its own they touch).  Returns grid with those layers filled."""
    world = len(ranges)
    a, b = owned_layers(rank, ranges, res)
    sends, shapes = {}, {}
    for peer in (rank - 1, rank + 1):
        if 0 <= peer < world:
            pa, pb = owned_layers(peer, ranges, res)
            lo_s, hi_s = max(a, pa - HALO_BELOW), min(b, pb + HALO_ABOVE)  # own layers peer touches
            sends[peer] = grid[..., lo_s:hi_s, :]
            lo_r, hi_r = max(pa, a - HALO_BELOW), min(pb, b + HALO_ABOVE)  # peer's layers this rank touches
            shapes[peer] = tuple(grid.shape[:-2]) + (max(0, hi_r - lo_r), grid.shape[-1])
    got = _exchange(sends, shapes, grid, group)
    out = grid.clone()
    for peer, t in got.items():
        pa, pb = owned_layers(peer, ranges, res)
        lo_r, hi_r = max(pa, a - HALO_BELOW), min(pb, b + HALO_ABOVE)
        out[..., lo_r:hi_r, :] = t
    return out


def migrate(fields: Dict[str, torch.Tensor], cell_x: torch.Tensor, rank: int, ranges: Sequence[Tuple[int, int]],
            group=None) -> Dict[str, torch.Tensor]:
    """After G2P: particles whose cell index along x (cell_x) lies in another
    rank's slab move there.  fields: per-particle tensors with the particle
    index first (positions, velocities, B, F, material, global id ...), all
    moved together.  A particle crosses at most into the neighbouring slab per
    step (one cell of travel at most, slabs are at least four cells wide).
    Returns this rank's fields: the particles that stayed, then those
    received from the lower neighbour, then from the upper one."""
    world = len(ranges)
    own = owner_of_cells(cell_x, ranges)
    if bool(((own - rank).abs() > 1).any()):
        raise ValueError("a particle moved more than one slab in one step")
    keep = own == rank
    peers = [p for p in (rank - 1, rank + 1) if 0 <= p < world]
    sel = {p: own == p for p in peers}
    counts = _exchange({p: torch.tensor([int(sel[p].sum())], dtype=torch.int64) for p in peers},
                       {p: (1,) for p in peers}, torch.zeros(1, dtype=torch.int64), group)
    n_in = {p: int(counts[p][0]) for p in peers}
    out = {}
    for k, v in fields.items():  # the same field order on every rank
        sends = {p: v[sel[p]] for p in peers if int(sel[p].sum()) > 0}
        got = _exchange(sends, {p: (n_in[p],) + tuple(v.shape[1:]) for p in peers if n_in[p] > 0}, v, group)
        out[k] = torch.cat([v[keep]] + [got[p] for p in peers if p in got], 0)
    return out


def layer_counts(cell_x: torch.Tensor, res: int, group=None) -> torch.Tensor:
    """Particles per cell layer along x over all ranks (int64, length res):
    each rank counts its own particles, then one sum over the group."""
    c = torch.bincount(cell_x.clamp(0, res - 1).to(torch.int64), minlength=res)[:res].to(torch.int64)
    if dist.is_initialized():
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    return c


def balanced_slab_ranges(counts: torch.Tensor, world: int) -> List[Tuple[int, int]]:
    """Cell ranges [lo, hi) along x in whole 4-cell blocks, one per rank, with
    about the same number of particles each: counts holds the particles of
    each cell layer (length res).  Boundary r is the block edge where the
    running count first reaches r / world of the total, moved where needed so
    that every rank keeps at least one block.  Where no boundary had to move,
    a rank's load exceeds total / world by at most the particles of one block
    layer.  With no particles the slabs are the even ones of slab_ranges."""
    res = int(counts.numel())
    nblk = -(-res // 4)
    if world > nblk:
        raise ValueError("more ranks than particle blocks along x")
    per_blk = torch.zeros(nblk, dtype=torch.int64)
    per_blk.index_add_(0, torch.arange(res) // 4, counts.to(torch.int64))
    total = int(per_blk.sum())
    if total == 0:
        return slab_ranges(res, world)
    cum = torch.cumsum(per_blk, 0)  # particles in blocks [0, b]
    edges = [0]
    for r in range(1, world):
        target = (total * r + world - 1) // world
        b = int(torch.searchsorted(cum, torch.tensor(target), right=False)) + 1  # first block edge with cum >= target
        b = max(b, edges[-1] + 1)  # every rank keeps at least one block
        b = min(b, nblk - (world - r))  # and leaves one for each rank above
        edges.append(b)
    edges.append(nblk)
    return [(4 * edges[r], min(res, 4 * edges[r + 1])) for r in range(world)]


def repartition(fields: Dict[str, torch.Tensor], cell_x: torch.Tensor, rank: int,
                ranges: Sequence[Tuple[int, int]], group=None) -> Dict[str, torch.Tensor]:
    """Move every particle to the rank whose slab holds its cell (any
    distance: after new slab boundaries, where migrate only moves between
    neighbours).  fields as for migrate.  Returns this rank's particles: the
    ones it kept, then those received, in rank order."""
    world = len(ranges)
    own = owner_of_cells(cell_x, ranges)
    peers = [p for p in range(world) if p != rank]
    sel = {p: own == p for p in peers}
    counts = _exchange({p: torch.tensor([int(sel[p].sum())], dtype=torch.int64) for p in peers},
                       {p: (1,) for p in peers}, torch.zeros(1, dtype=torch.int64), group)
    n_in = {p: int(counts[p][0]) for p in peers}
    keep = own == rank
    out = {}
    for k, v in fields.items():  # the same field order on every rank
        sends = {p: v[sel[p]] for p in peers if int(sel[p].sum()) > 0}
        got = _exchange(sends, {p: (n_in[p],) + tuple(v.shape[1:]) for p in peers if n_in[p] > 0}, v, group)
        out[k] = torch.cat([v[keep]] + [got[p] for p in peers if p in got], 0)
    return out


def load_imbalance(counts: torch.Tensor, ranges: Sequence[Tuple[int, int]]) -> float:
    """Largest rank's particle count over the mean (1.0 when balanced or empty)."""
    loads = [int(counts[a:b].sum()) for a, b in ranges]
    total = sum(loads)
    return max(loads) * len(loads) / total if total else 1.0


def rebalance(fields: Dict[str, torch.Tensor], cell_x: torch.Tensor, rank: int,
              ranges: Sequence[Tuple[int, int]], res: int, tolerance: float = 0.1,
              group=None) -> Tuple[Dict[str, torch.Tensor], List[Tuple[int, int]], bool]:
    """Between steps: when the largest rank holds more than (1 + tolerance)
    times the mean and particle-balanced slabs would hold less, move to those
    slabs (repartition).  Every rank calls it with the same ranges; all take
    the same decision from the summed layer counts.  Returns (fields, ranges,
    whether they changed)."""
    counts = layer_counts(cell_x, res, group)
    now = load_imbalance(counts, ranges)
    if now <= 1.0 + tolerance:
        return fields, list(ranges), False
    new = balanced_slab_ranges(counts, len(ranges))
    if load_imbalance(counts, new) >= now:
        return fields, list(ranges), False
    return repartition(fields, cell_x, rank, new, group), new, True
