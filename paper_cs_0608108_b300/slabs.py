"""Slab decomposition of the all-agents radius query over ranks.

The lattice's z planes are split into P contiguous slabs, one per rank.  A
rank owns the queries of the points whose cell plane lies in its slab; every
neighbor of such a point lies within `reach` planes of the slab (reach =
floor(r_max / s) + 2: the floor(r_max / s) + 1 planes a sphere of radius
r_max can span beyond its own cell's plane, Sec. II.A, and one more for a
coordinate that float32 binning puts a few ulps across a plane), so a rank
needs the points of its slab plus a halo of `reach` planes on each side.  On a cyclic
z axis the halo wraps around the box (the first slab's lower halo is the
last planes, Sec. II.B); on a non-cyclic one it stops at the region, and a
point outside the region in z belongs to the slab of the nearest plane.

After each binning step the ranks exchange points once: every rank sends the
points of its shard that fall in another rank's slab or halo (an all-gather
of the boundary planes); then each rank queries on its own GPU with the
global lattice descriptor (same cell size, origin and cyclic mask), over its
local points only.  The local points are kept in ascending global index, so
local lists sorted by local index are sorted by global index, and a rank's
lists are exactly the global lists of its owned points: the union over ranks
is the single-GPU result.  The batched configuration needs no exchange: its
scenes are independent and are partitioned whole across ranks.

Host bookkeeping only (numpy and torch.distributed): the query itself is a
callable, the library's si_query_radius on a GPU rank.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class SlabPlan:
    """Slab of one rank on a lattice of gz planes (z cell index)."""
    gz: int           # planes of the lattice along z
    ranks: int
    rank: int
    z0: int           # owned planes [z0, z1)
    z1: int
    reach: int        # halo planes on each side
    cyclic: bool      # z wraps

    def halo_planes(self) -> list:
        """Planes of the lower and upper halo, in order (wrapped on a cyclic
        axis, clipped to the region otherwise; never a plane of the slab)."""
        lo = [self.z0 - k for k in range(self.reach, 0, -1)]
        hi = [self.z1 - 1 + k for k in range(1, self.reach + 1)]
        out = []
        for z in lo + hi:
            if self.cyclic:
                z %= self.gz
            elif z < 0 or z >= self.gz:
                continue
            if not (self.z0 <= z < self.z1) and z not in out:
                out.append(z)
        return out


def reach_planes(r_max: float, cell_size: float) -> int:
    """Halo width in planes: floor(r_max / s) + 2."""
    return int(math.floor(float(r_max) / float(cell_size))) + 2


def plan(gz: int, ranks: int, rank: int, r_max: float, cell_size: float, cyclic: bool) -> SlabPlan:
    """Slab of `rank`: planes split as evenly as possible, lower ranks first.
    A cyclic z axis needs every slab's halos to stay disjoint from the slab
    itself and from each other's wrap: 2 reach + slab <= gz."""
    if ranks < 1 or not 0 <= rank < ranks:
        raise ValueError("bad rank")
    if ranks > gz:
        raise ValueError("more ranks than z planes")
    base, extra = divmod(gz, ranks)
    z0 = rank * base + min(rank, extra)
    z1 = z0 + base + (1 if rank < extra else 0)
    reach = reach_planes(r_max, cell_size)
    if cyclic and 2 * reach + (z1 - z0) > gz and ranks > 1:
        raise ValueError("halo wraps onto the slab: too few z planes for this radius and rank count")
    return SlabPlan(gz, ranks, rank, z0, z1, reach, cyclic)


def planes_of(z: np.ndarray, origin_z: float, cell_size: float) -> np.ndarray:
    """Unclamped cell plane of each z coordinate (float32 arithmetic, as the
    binning does: (z - origin) * (1 / s), then floor)."""
    rel = (np.asarray(z, np.float32) - np.float32(origin_z)) * np.float32(1.0 / np.float32(cell_size))
    return np.floor(rel.astype(np.float64)).astype(np.int64)


def owned_mask(planes: np.ndarray, p: SlabPlan) -> np.ndarray:
    """Points whose (clamped, or wrapped on a cyclic axis) plane is in the slab."""
    zc = np.mod(planes, p.gz) if p.cyclic else np.clip(planes, 0, p.gz - 1)
    return (zc >= p.z0) & (zc < p.z1)


def local_mask(planes: np.ndarray, p: SlabPlan) -> np.ndarray:
    """Points a rank needs: its slab and its halo planes (a point outside a
    non-cyclic region counts at its clamped plane, and also at its true plane
    when that lies in the halo window)."""
    m = owned_mask(planes, p)
    for z in p.halo_planes():
        zc = np.mod(planes, p.gz) if p.cyclic else np.clip(planes, 0, p.gz - 1)
        m |= zc == z
    if not p.cyclic:
        m |= (planes >= p.z0 - p.reach) & (planes < p.z1 + p.reach)
    return m


def exchange(shard_ids: np.ndarray, shard_pos: np.ndarray, plans: list, origin_z: float, cell_size: float,
             group=None):
    """One exchange after binning: every rank sends, to every rank, the
    points of its shard that rank needs (an all-gather of fixed-size padded
    blocks, one per rank, over torch.distributed).  Returns this rank's local
    points in ascending global index: (ids int64[k], pos float32[k, 4])."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    planes = planes_of(shard_pos[:, 2], origin_z, cell_size)
    # per destination rank: the rows it needs, packed as [id, x, y, z, w]
    send = []
    for r in range(world):
        sel = local_mask(planes, plans[r])
        rows = np.zeros((int(sel.sum()), 5), np.float64)
        rows[:, 0] = shard_ids[sel]
        rows[:, 1:] = shard_pos[sel].astype(np.float64)
        send.append(rows)
    counts = torch.tensor([len(x) for x in send], dtype=torch.int64)
    all_counts = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(all_counts, counts, group=group)
    width = max(1, int(max(int(c.max()) for c in all_counts)))
    block = torch.zeros((world, width, 5), dtype=torch.float64)
    for r in range(world):
        block[r, : len(send[r])] = torch.from_numpy(send[r])
    gathered = [torch.zeros_like(block) for _ in range(world)]
    dist.all_gather(gathered, block, group=group)
    parts = [gathered[src][me, : int(all_counts[src][me])].numpy() for src in range(world)]
    rows = np.concatenate(parts) if parts else np.zeros((0, 5))
    order = np.argsort(rows[:, 0], kind="stable")
    rows = rows[order]
    ids = rows[:, 0].astype(np.int64)
    pos = rows[:, 1:].astype(np.float32)
    return ids, pos


def rank_query(local_ids: np.ndarray, local_pos: np.ndarray, p: SlabPlan, origin_z: float, cell_size: float,
               query):
    """The owned queries of one rank over its local points.  query(pos, q)
    returns (offsets int64[len(q)+1], ids int32) for local query indices q,
    neighbors as local indices, ascending, each query's own index excluded.
    Returns (global ids of the owned points, ascending; offsets; global
    neighbor ids)."""
    planes = planes_of(local_pos[:, 2], origin_z, cell_size)
    q = np.nonzero(owned_mask(planes, p))[0]
    off, lids = query(local_pos, q)
    return local_ids[q], np.asarray(off, np.int64), local_ids[np.asarray(lids, np.int64)].astype(np.int64)
