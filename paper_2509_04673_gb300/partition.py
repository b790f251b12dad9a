"""Host-side work partitioning over ranks (one process per GPU).

Two decompositions of the stage's work:

* independent instances (the batched form): a deterministic disjoint split
  whose union is every instance, balanced by DOF; the ranks never exchange
  data;
* one mesh: a 2D block decomposition of the elements over a px x py process
  grid.  A rank owns the nodes of its element block (a shared interface
  node belongs to the block whose element has it as its lower-left local
  node; on a non-periodic mesh the last node row and column belong to the
  last blocks).  Before a stage it needs the nodal coefficients of a halo of
  H elements around its block: one stage reads at most five elements away
  (sensor neighbours, the g_h and udot Richardson sweeps, the neighbours'
  low-order averages of the flux limiter, the node gather), so H = 6 lets a
  rank compute its owned nodes of the stage from its extended block alone,
  with one exchange per stage, and the global dt = omega_CFL min_e dt_e is a
  min-reduction over the ranks' owned elements once per step.

The exchange plan lists, per peer, the owned node ranges a rank sends and
the ranges it receives; `exchange` runs it with point-to-point messages of
torch.distributed (gloo on the host; a device implementation would copy the
same ranges peer to peer).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# independent instances
# --------------------------------------------------------------------------
def partition_instances(sizes, world):
    """Split instance indices over `world` ranks: largest first, each to the
    rank with the least DOF so far (lowest rank on ties).  Returns one sorted
    index list per rank; together they hold every index exactly once."""
    if world < 1:
        raise ValueError("world >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


# --------------------------------------------------------------------------
# 2D block decomposition of one mesh
# --------------------------------------------------------------------------
def process_grid(world, nx, ny):
    """px x py = world with the blocks as square as possible (ties: more
    ranks along x)."""
    best = None
    for px in range(1, world + 1):
        if world % px:
            continue
        py = world // px
        if px > nx or py > ny:
            continue
        cost = abs(np.log((nx / px) / (ny / py)))
        if best is None or cost < best[0] - 1e-12:
            best = (cost, px, py)
    if best is None:
        raise ValueError("more ranks than elements along a direction")
    return best[1], best[2]


def split_range(n, parts, k):
    """Element range of part k of n elements split into `parts` near-equal parts."""
    return (k * n) // parts, ((k + 1) * n) // parts


@dataclass(frozen=True)
class Block:
    rank: int
    ex0: int
    ex1: int
    ey0: int
    ey1: int


def blocks(world, nx, ny):
    px, py = process_grid(world, nx, ny)
    out = []
    for r in range(world):
        ix, iy = r % px, r // px
        ex0, ex1 = split_range(nx, px, ix)
        ey0, ey1 = split_range(ny, py, iy)
        out.append(Block(r, ex0, ex1, ey0, ey1))
    return out


def owned_nodes(b: Block, nx, ny, p, periodic_x, periodic_y):
    """Global node ranges [gx0, gx1) x [gy0, gy1) owned by block b."""
    gx0, gx1 = b.ex0 * p, b.ex1 * p
    gy0, gy1 = b.ey0 * p, b.ey1 * p
    if b.ex1 == nx and not periodic_x:
        gx1 += 1
    if b.ey1 == ny and not periodic_y:
        gy1 += 1
    return gx0, gx1, gy0, gy1


def window_periodic(b: Block, nx, ny, periodic_x, periodic_y):
    """A direction stays periodic in the window of block b when the mesh is
    periodic in it and the block spans the whole direction (one rank along
    it): then the window is the full periodic direction, without a halo."""
    return (periodic_x and b.ex0 == 0 and b.ex1 == nx), (periodic_y and b.ey0 == 0 and b.ey1 == ny)


def extended_elements(b: Block, nx, ny, halo, periodic_x, periodic_y):
    """Element range of block b grown by `halo` elements: clipped at a
    non-periodic boundary, unclipped (wrapping) on a periodic direction
    split over ranks, unchanged on a periodic direction the block spans."""
    wpx, wpy = window_periodic(b, nx, ny, periodic_x, periodic_y)

    def grow(a0, a1, n, per, whole):
        if whole:
            return a0, a1
        lo, hi = a0 - halo, a1 + halo
        if per:
            if hi - lo >= n:
                raise ValueError("halo wider than the periodic direction: use fewer ranks along it")
            return lo, hi
        return max(0, lo), min(n, hi)
    ex0, ex1 = grow(b.ex0, b.ex1, nx, periodic_x, wpx)
    ey0, ey1 = grow(b.ey0, b.ey1, ny, periodic_y, wpy)
    return ex0, ex1, ey0, ey1


def extended_nodes(ext, nx, ny, p, periodic_x, periodic_y, whole_x=False, whole_y=False):
    """Node index lists (global, wrapped) of an extended element range: the
    window holds every node of its elements (a direction kept periodic in
    the window holds its n p nodes once)."""
    ex0, ex1, ey0, ey1 = ext
    nnx = nx * p + (0 if periodic_x else 1)
    nny = ny * p + (0 if periodic_y else 1)
    gx = np.arange(nnx) if whole_x else np.arange(ex0 * p, ex1 * p + 1)
    gy = np.arange(nny) if whole_y else np.arange(ey0 * p, ey1 * p + 1)
    if periodic_x:
        gx = gx % nnx
    if periodic_y:
        gy = gy % nny
    return gx, gy


def halo_plan(world, nx, ny, p, halo, periodic_x, periodic_y):
    """For every rank: the (peer, gx list, gy list) pieces it receives, each
    piece a product of owned-node index lists of the peer (the local part
    included as the peer == rank piece)."""
    bl = blocks(world, nx, ny)
    owned = [owned_nodes(b, nx, ny, p, periodic_x, periodic_y) for b in bl]
    plan = []
    for b in bl:
        ext = extended_elements(b, nx, ny, halo, periodic_x, periodic_y)
        wpx, wpy = window_periodic(b, nx, ny, periodic_x, periodic_y)
        gx, gy = extended_nodes(ext, nx, ny, p, periodic_x, periodic_y, wpx, wpy)
        pieces = []
        for q, (ox0, ox1, oy0, oy1) in enumerate(owned):
            sx = np.nonzero((gx >= ox0) & (gx < ox1))[0]
            sy = np.nonzero((gy >= oy0) & (gy < oy1))[0]
            if sx.size and sy.size:
                pieces.append((q, sx, sy, gx[sx] - ox0, gy[sy] - oy0))
        plan.append(dict(block=b, ext=ext, gx=gx, gy=gy, pieces=pieces, owned=owned[b.rank],
                         periodic=(wpx, wpy)))
    return plan


def exchange(plan, rank, local, dist=None):
    """Assemble the extended window of `rank` from the ranks' owned arrays.

    local: this rank's owned coefficients, shape (nc, gy1 - gy0, gx1 - gx0).
    Sends every peer the pieces it needs, receives its own pieces, and
    returns the window of shape (nc, len(gy), len(gx)).  Blocking gloo
    point-to-point messages, sends posted before receives (isend)."""
    import torch
    me = plan[rank]
    nc = local.shape[0]
    win = np.zeros((nc, me["gy"].size, me["gx"].size), dtype=local.dtype)
    reqs = []
    sendbufs = []
    for q, pq in enumerate(plan):
        for (owner, sx, sy, lx, ly) in pq["pieces"]:
            if owner != rank:
                continue
            piece = np.ascontiguousarray(local[:, ly][:, :, lx])
            if q == rank:
                win[:, sy[:, None], sx[None, :]] = piece
            else:
                t = torch.from_numpy(piece.reshape(-1).copy())
                sendbufs.append(t)
                reqs.append(dist.isend(t, dst=q))
    for (owner, sx, sy, lx, ly) in me["pieces"]:
        if owner == rank:
            continue
        t = torch.empty(nc * sy.size * sx.size, dtype=torch.float64)
        dist.recv(t, src=owner)
        win[:, sy[:, None], sx[None, :]] = t.numpy().reshape(nc, sy.size, sx.size)
    for r in reqs:
        r.wait()
    return win


def owned_slice_of_window(plan, rank):
    """Index arrays (iy, ix) of the rank's owned nodes inside its window, in
    owned-array order."""
    me = plan[rank]
    ox0, ox1, oy0, oy1 = me["owned"]
    ix = np.array([np.nonzero(me["gx"] == g)[0][0] for g in range(ox0, ox1)])
    iy = np.array([np.nonzero(me["gy"] == g)[0][0] for g in range(oy0, oy1)])
    return iy, ix
