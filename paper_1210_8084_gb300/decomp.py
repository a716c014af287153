"""Host logic of the x-slab domain decomposition of one instance over ranks.

Locality of the pair decision (scattering detection, criteria 1-3, and the
unambiguous-pair rule of Sect. "Implementation"): a particle picks its closest
candidate among the particles of its 3^D neighbourhood of c-bins, and a pair
forms only when both particles pick each other.  The choice of a particle in
c-bin column c therefore depends on the columns c - 1 .. c + 1, and the choice
of its partner on c - 2 .. c + 2.  A rank that owns the columns [c0, c1) and
also holds the particles of the HALO = 2 columns on either side decides every
pair of its own particles exactly as the undivided system does, provided that
the tie-break and the random keys use global particle ids and the contact
distance is the global one (the mean density of the whole instance).  Halo
particles are read only; their own results are discarded.  After the move, the
particles that left [c0, c1) migrate to the rank that owns their new column.

This module holds the integer bookkeeping (slab bounds, owners, halo columns,
send lists) and the exchange over torch.distributed.  The per-rank step is
the caller's: any implementation of the step on a subset of particles with
global ids and global geometry.  Column indices come from the caller too.
"""
import numpy as np

HALO = 2


def slab_bounds(n_x, world, col_weight=None):
    """Split the columns 0 .. n_x - 1 into `world` contiguous slabs of at least
    one column each.  With col_weight (per-column cost, e.g. particle counts
    or candidate counts) each cut is the column boundary whose prefix sum is
    nearest to an equal share; without it
    the slabs are as equal in width as possible.  Returns bounds (world + 1,),
    slab r = [bounds[r], bounds[r + 1])."""
    if world < 1 or n_x < world:
        raise ValueError(f"cannot split {n_x} columns over {world} ranks")
    if col_weight is None:
        return np.array([(r * n_x) // world for r in range(world + 1)], dtype=np.int64)
    w = np.asarray(col_weight, dtype=np.float64)
    if w.shape != (n_x,) or np.any(w < 0):
        raise ValueError("col_weight must be n_x non-negative numbers")
    cum = np.concatenate(([0.0], np.cumsum(w)))
    total = cum[-1]
    b = [0]
    for r in range(1, world):
        target = total * r / world
        cut = int(np.searchsorted(cum, target, side="left"))
        if cut > 0 and (cut > n_x or target - cum[cut - 1] <= cum[cut] - target):
            cut -= 1                            # the nearer of the two prefix sums
        cut = max(cut, b[-1] + 1)               # at least one column per slab
        cut = min(cut, n_x - (world - r))       # leave one for each later slab
        b.append(cut)
    b.append(n_x)
    return np.array(b, dtype=np.int64)


def owner(cx, bounds):
    """Rank that owns each column index (int array; -1 for columns outside
    [0, n_x), e.g. absorbed particles)."""
    cx = np.asarray(cx, dtype=np.int64)
    r = np.searchsorted(bounds, cx, side="right") - 1
    return np.where((cx >= 0) & (cx < bounds[-1]), r, -1)


def halo_columns(rank, bounds, periodic, width=HALO):
    """Columns within `width` of slab `rank` that other ranks own: wrapped
    around the box when x is periodic, cut at the walls otherwise."""
    n_x = int(bounds[-1])
    c0, c1 = int(bounds[rank]), int(bounds[rank + 1])
    cols = set()
    for c in list(range(c0 - width, c0)) + list(range(c1, c1 + width)):
        if periodic:
            c %= n_x
        elif c < 0 or c >= n_x:
            continue
        if not (c0 <= c < c1):
            cols.add(c)
    return np.array(sorted(cols), dtype=np.int64)


def halo_sends(cx, rank, bounds, periodic, width=HALO):
    """For the particles of `rank` (column indices cx), the indices to send to
    each rank as its halo: a list of `world` int arrays (empty for `rank`)."""
    cx = np.asarray(cx, dtype=np.int64)
    world = len(bounds) - 1
    out = []
    for q in range(world):
        if q == rank:
            out.append(np.zeros(0, dtype=np.int64))
            continue
        out.append(np.flatnonzero(np.isin(cx, halo_columns(q, bounds, periodic, width))))
    return out


def migration_sends(cx_new, rank, bounds):
    """After the move: indices of the particles of `rank` (new column indices
    cx_new) that each rank now owns, and the mask of those that stay.
    Particles with no owner (cx_new < 0: absorbed) go nowhere."""
    own = owner(cx_new, bounds)
    world = len(bounds) - 1
    out = [np.flatnonzero(own == q) if q != rank else np.zeros(0, dtype=np.int64) for q in range(world)]
    return out, own == rank


def exchange(rows, group=None):
    """All-to-all of variable-length row blocks over torch.distributed: rows[q]
    (a 2-D float64 array, the same number of columns on every rank) goes to
    rank q; returns the list of blocks received from each rank (rows[self]
    comes back unchanged).  Counts travel first by all_gather, then one
    isend/irecv per non-empty block, so the gloo backend suffices."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    if len(rows) != world:
        raise ValueError("one block per rank")
    ncol = rows[0].shape[1]
    counts = torch.tensor([r.shape[0] for r in rows], dtype=torch.int64)
    table = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(table, counts, group=group)
    reqs, recv = [], [None] * world
    for q in range(world):
        if q != me and rows[q].shape[0]:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(rows[q], dtype=np.float64)), q, group=group))
    for q in range(world):
        if q == me:
            recv[q] = np.asarray(rows[q], dtype=np.float64)
            continue
        n = int(table[q][me])
        buf = torch.empty((n, ncol), dtype=torch.float64)
        if n:
            reqs.append(dist.irecv(buf, q, group=group))
        recv[q] = buf
    for r in reqs:
        r.wait()
    return [b if isinstance(b, np.ndarray) else b.numpy() for b in recv]


def allreduce_min(x, group=None):
    """Global minimum of a float (the adaptive timestep: dt = dx / v_max over
    the whole instance is the minimum of the ranks' dx / v_max,r, because a
    correctly rounded quotient does not increase as the divisor grows)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t[0])
