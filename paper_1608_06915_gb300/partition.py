"""Slab partition of a level along x and the halo exchange of the pull stream.

The update is node-local except for the pull f_i(x) = f'_i(x - c_i) (Eq. 1,
left-hand side), so a level split into slabs along x needs, per substep, one
exchange: each slab receives, into a ghost layer on either side, the nine
post-collision populations that cross that face -- c_x = +1 from the left
neighbour's last layer, c_x = -1 from the right neighbour's first layer.  The
rest of the step stays on the rank that owns the node.

This module holds the host-side logic: slab bounds, which populations cross a
face, packing and unpacking them, the exchange over torch.distributed
(point-to-point send/recv, so any backend), and the local pull over a slab
with its ghost layers.  For refined layouts it also gives the slabs of every
level, aligned with the coarse slabs so that coarse/fine twins stay on one
rank, the parent halo the interface coupling needs beyond a slab edge, and
a deterministic FP64 all-reduce for the diagnostics.  Populations are arrays [27][nz][ny][nx] (x fastest),
velocity order i = (cx+1) + 3(cy+1) + 9(cz+1); y and z are periodic within
every slab.
"""
import numpy as np

Q = 27
CX = np.array([(i % 3) - 1 for i in range(Q)])
CY = np.array([((i // 3) % 3) - 1 for i in range(Q)])
CZ = np.array([(i // 9) - 1 for i in range(Q)])

# populations crossing an x-face, in increasing index order
TO_RIGHT = np.flatnonzero(CX == 1)   # leave through the +x face, enter the right neighbour
TO_LEFT = np.flatnonzero(CX == -1)   # leave through the -x face, enter the left neighbour


def slab_bounds(nx: int, ranks: int, rank: int) -> tuple:
    """[x0, x1) of rank's slab: nx split as evenly as possible, lower ranks
    taking the remainder; every slab at least one layer thick."""
    if ranks < 1 or not 0 <= rank < ranks:
        raise ValueError("bad rank")
    if nx < ranks:
        raise ValueError("fewer x layers than ranks")
    base, extra = divmod(nx, ranks)
    x0 = rank * base + min(rank, extra)
    return x0, x0 + base + (1 if rank < extra else 0)


def pack_faces(f: np.ndarray) -> tuple:
    """Face buffers of a slab's post-collision populations [27][nz][ny][nx]:
    (to_left [9][nz][ny] of the first layer, to_right [9][nz][ny] of the last)."""
    return (np.ascontiguousarray(f[TO_LEFT, :, :, 0]), np.ascontiguousarray(f[TO_RIGHT, :, :, -1]))


def with_ghosts(f: np.ndarray, from_left: np.ndarray, from_right: np.ndarray) -> np.ndarray:
    """The slab extended by one ghost layer on each side along x; ghosts hold
    only the populations that cross into the slab (the others are never read
    by the pull of an owned node and are left at zero)."""
    q, nz, ny, nx = f.shape
    g = np.zeros((q, nz, ny, nx + 2), dtype=f.dtype)
    g[:, :, :, 1:-1] = f
    g[TO_RIGHT, :, :, 0] = from_left
    g[TO_LEFT, :, :, -1] = from_right
    return g


def pull_local(g: np.ndarray) -> np.ndarray:
    """Pull stream of the owned nodes from a ghost-extended slab: f_i(x) =
    f'_i(x - c_i), x - c_i within the slab plus ghosts along x, periodic in
    y and z."""
    q, nz, ny, nxg = g.shape
    nx = nxg - 2
    out = np.empty((q, nz, ny, nx), dtype=g.dtype)
    for i in range(q):
        src = g[i, :, :, 1 - CX[i]:1 - CX[i] + nx]
        out[i] = np.roll(np.roll(src, CY[i], axis=1), CZ[i], axis=0)
    return out


def exchange(f: np.ndarray, rank: int, ranks: int, dist) -> tuple:
    """Ghost data (from_left, from_right) for rank's slab, ring-periodic in x.
    Sends and receives are posted as non-blocking pairs, so every rank can
    send before it receives."""
    import torch
    to_left, to_right = pack_faces(f)
    left, right = (rank - 1) % ranks, (rank + 1) % ranks
    from_left = torch.empty(to_right.shape, dtype=torch.float64)
    from_right = torch.empty(to_left.shape, dtype=torch.float64)
    if ranks == 1:
        return to_right.copy(), to_left.copy()
    # tag 1: data moving towards +x, tag 2: towards -x (two ranks are each
    # other's left and right neighbour)
    reqs = [dist.isend(torch.from_numpy(to_right), right, tag=1), dist.isend(torch.from_numpy(to_left), left, tag=2),
            dist.irecv(from_left, left, tag=1), dist.irecv(from_right, right, tag=2)]
    for r in reqs:
        r.wait()
    return from_left.numpy(), from_right.numpy()


# ---------------------------------------------------------------------------
# Refined layouts

def level_slab(nx: int, ranks: int, rank: int, level: int) -> tuple:
    """[x0, x1) of rank's slab on ``level`` in that level's node coordinates:
    the coarse slab of slab_bounds scaled by 2^level, so every level-l node
    that coincides with a coarse node lies on the rank owning that coarse node
    (twins of the coupling, Sec. III.A, stay on one rank)."""
    a, b = slab_bounds(nx, ranks, rank)
    s = 1 << level
    return a * s, b * s


def owner(x_level: int, nx: int, ranks: int, level: int) -> int:
    """Rank owning the level node with x coordinate ``x_level`` (periodic in x)."""
    period = nx << level
    x = x_level % period
    for r in range(ranks):
        a, b = level_slab(nx, ranks, r, level)
        if a <= x < b:
            return r
    raise ValueError("no owner")


# Reconstruction samples sit at +-1/2 and +-3/2 parent spacings from a
# reconstructed child node along each off-lattice axis (the centred four-point
# Lagrange rule, Eq. interp), and each sample is a parent (or coinciding child)
# node; the pull of every sample node reaches one parent spacing further.
SAMPLE_OFFSETS = (-1.5, -0.5, 0.5, 1.5)


def parent_halo() -> tuple:
    """Parent layers (below, above) a slab that the coupling of the slab's
    child nodes reads, with level slabs as level_slab gives them: a child
    slab [2a, 2b) starts on parent node a and ends half a parent spacing past
    parent node b - 1.  The first off-lattice child node (a + 1/2) samples
    down to parent node a - 1, the last (b - 1/2) up to b + 1, and each
    sample is the pulled state of its node, one layer further."""
    first, last = 0.5, -0.5  # parent coordinates relative to a and to b
    below = -(first + min(SAMPLE_OFFSETS)) + 1  # a - 1, then its pull
    above = (last + max(SAMPLE_OFFSETS)) + 1 + 1  # b + 1 is layer 2 past b - 1, then its pull
    return int(below), int(above)


def allreduce_sums(values, dist) -> np.ndarray:
    """FP64 sums of per-rank partial values, identical on every rank and equal
    to the serial sum in rank order: all-gather, then add rank by rank (an
    all-reduce's own order of additions may differ between ranks and runs)."""
    import torch
    v = torch.as_tensor(np.asarray(values, dtype=np.float64))
    parts = [torch.empty_like(v) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, v)
    total = np.zeros(v.shape, dtype=np.float64)
    for p in parts:
        total = total + p.numpy()
    return total
