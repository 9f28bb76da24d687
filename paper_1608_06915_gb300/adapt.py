"""Refinement boxes from the stabiliser gamma.

The paper observes (Sec. IV, channel) that the KBC stabiliser gamma of Eq.
gamma_min_approx tends to its LBGK value 2 where the flow is resolved, so
that |gamma - 2| measures under-resolution, and its conclusion proposes this
as the criterion of adaptive refinement.  ``lbm_gamma_blocks`` computes the
largest |gamma - 2| per block of nodes on the GPU; this module turns the
flagged blocks of a patch into candidate boxes of the next level in the
layout's coarse units, widened to the layout's minimum width and merged
until they satisfy the layout rules that ``lbm_grid_create`` checks; ``regrid`` then moves the state onto the new
layout (``lbm_transfer``).

Host logic only (numpy): clustering, conversion to coarse units, merging.
"""
import numpy as np


def clusters(flags: np.ndarray) -> list:
    """Face-connected clusters of True entries of a 3-D array [z][y][x]:
    a list of (lo, hi) index bounding boxes, each a tuple (x, y, z), closed."""
    flags = np.asarray(flags, dtype=bool)
    seen = np.zeros_like(flags)
    out = []
    nz, ny, nx = flags.shape
    for start in zip(*np.nonzero(flags)):
        if seen[start]:
            continue
        seen[start] = True
        stack, lo, hi = [start], list(start), list(start)
        while stack:
            z, y, x = stack.pop()
            for a in range(3):
                lo[a] = min(lo[a], (z, y, x)[a])
                hi[a] = max(hi[a], (z, y, x)[a])
            for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                q = (z + dz, y + dy, x + dx)
                if 0 <= q[0] < nz and 0 <= q[1] < ny and 0 <= q[2] < nx and flags[q] and not seen[q]:
                    seen[q] = True
                    stack.append(q)
        out.append(((lo[2], lo[1], lo[0]), (hi[2], hi[1], hi[0])))
    return out


def block_box_to_coarse(info: dict, block: int, lo_b, hi_b, margin: int, n) -> tuple:
    """Coarse-unit closed box [lo, hi] covering blocks lo_b..hi_b of a patch
    (storage-box block indices, x y z), grown by ``margin`` coarse units and
    clipped to the domain [0, n - 1]."""
    s = 1 << info["level"]
    lo, hi = [], []
    for a in range(3):
        i0 = lo_b[a] * block
        i1 = min((hi_b[a] + 1) * block, info["dim"][a]) - 1
        c0 = (info["org"][a] + i0) // s - margin
        c1 = -((-(info["org"][a] + i1)) // s) + margin  # ceil
        lo.append(max(0, c0))
        hi.append(min(int(n[a]) - 1, c1))
    return tuple(lo), tuple(hi)


def widen(box, min_width: float, n) -> tuple:
    """A closed box (lo, hi) grown about its centre to at least ``min_width``
    per axis (hi - lo), shifted back inside the domain [0, n - 1]."""
    lo, hi = list(box[0]), list(box[1])
    for a in range(3):
        w = hi[a] - lo[a]
        if w < min_width:
            extra = int(np.ceil(min_width - w))
            lo[a] -= extra // 2
            hi[a] += extra - extra // 2
        if lo[a] < 0:
            hi[a] = min(int(n[a]) - 1, hi[a] - lo[a])
            lo[a] = 0
        if hi[a] > int(n[a]) - 1:
            lo[a] = max(0, lo[a] - (hi[a] - (int(n[a]) - 1)))
            hi[a] = int(n[a]) - 1
    return tuple(lo), tuple(hi)


def merge_boxes(boxes: list, gap: float) -> list:
    """Merge closed boxes (lo, hi) until no two of them overlap or lie within
    ``gap`` of each other on every axis; a merged pair becomes its bounding box."""
    boxes = [(tuple(lo), tuple(hi)) for lo, hi in boxes]
    changed = True
    while changed:
        changed = False
        for i in range(len(boxes)):
            for j in range(i + 1, len(boxes)):
                (alo, ahi), (blo, bhi) = boxes[i], boxes[j]
                near = all(not (ahi[a] + gap < blo[a] or bhi[a] + gap < alo[a]) for a in range(3))
                if near:
                    boxes[i] = (tuple(min(alo[a], blo[a]) for a in range(3)),
                                tuple(max(ahi[a], bhi[a]) for a in range(3)))
                    del boxes[j]
                    changed = True
                    break
            if changed:
                break
    return boxes


def parent_region(info: dict, n) -> tuple:
    """The coarse-unit closed box a next-level box must lie in to nest in the
    level-l patch ``info``: the patch's box, less 4 level-l spacings on each
    face that does not reach the domain's edge (an interface face), rounded
    inwards to whole coarse units.  Level 0: the whole domain."""
    if info["level"] == 0:
        return tuple(0 for _ in range(3)), tuple(int(v) - 1 for v in n)
    s = 1 << info["level"]
    inset = -(-4 // s)  # ceil(4 / s) coarse units
    lo, hi = [], []
    for a in range(3):
        plo = -(-info["org"][a] // s)
        phi = (info["org"][a] + info["dim"][a] - 1) // s
        lo.append(plo + inset if plo > 0 else plo)
        hi.append(phi - inset if phi < int(n[a]) - 1 else phi)
    return tuple(lo), tuple(hi)


def _inside(box, region) -> bool:
    return all(region[0][a] <= box[0][a] and box[1][a] <= region[1][a] for a in range(3))


def _fit(box, region) -> tuple:
    """A closed box moved inside ``region`` along each axis where it fits,
    and clipped to it where it is wider."""
    lo, hi = list(box[0]), list(box[1])
    for a in range(3):
        if hi[a] > region[1][a]:
            lo[a] -= hi[a] - region[1][a]
            hi[a] = region[1][a]
        if lo[a] < region[0][a]:
            hi[a] = min(region[1][a], hi[a] + region[0][a] - lo[a])
            lo[a] = region[0][a]
    return tuple(lo), tuple(hi)


def boxes_from_flags(flags: np.ndarray, info: dict, block: int, case: dict, margin: int = 1,
                     storage: str = "fp32"):
    """The full box list (all levels) of a layout that covers the flagged
    blocks ([z][y][x] bools over a level-l patch's storage box, ``info`` as
    in Grid.patches) with level-(l+1) boxes, or None when nothing is flagged
    or no valid layout is found.  The new boxes are widened to the layout's
    minimum width, moved into the region where they nest in this patch
    (parent_region), and merged with each other and with the existing
    level-(l+1) boxes inside that region while closer than 8 parent spacings;
    level-(l+1) boxes under other patches are kept as they are.  If that
    layout is rejected, one bounding box of the merged ones is tried."""
    from . import lbm as L
    cl = clusters(flags)
    if not cl:
        return None
    spacing = 8.0 / (1 << info["level"])  # 8 parent spacings in coarse units
    lev = info["level"] + 1
    region = parent_region(info, case["n"])
    new = [_fit(widen(block_box_to_coarse(info, block, lo, hi, margin, case["n"]), spacing, case["n"]), region)
           for lo, hi in cl]
    new = [b for b in new if all(b[0][a] <= b[1][a] for a in range(3))]
    if not new:
        return None
    mine = [(tuple(b[1]), tuple(b[2])) for b in case.get("boxes", []) if b[0] == lev
            and _inside((tuple(b[1]), tuple(b[2])), region)]
    keep = [b for b in case.get("boxes", []) if not (b[0] == lev and _inside((tuple(b[1]), tuple(b[2])), region))]
    merged = merge_boxes(mine + new, spacing)
    candidates = [merged]
    if len(merged) > 1:
        lo = tuple(min(b[0][a] for b in merged) for a in range(3))
        hi = tuple(max(b[1][a] for b in merged) for a in range(3))
        candidates.append([(lo, hi)])
    for cand in candidates:
        boxes = keep + [(lev, lo, hi) for lo, hi in cand]
        try:
            L.Grid(dict(case, boxes=boxes), storage, bind=False)
        except L.LbmError:  # the layout validation rejected these boxes
            continue
        return boxes
    return None


def refinement_boxes(grid, case: dict, patch: int, block: int = 4, threshold: float = 0.1, margin: int = 1):
    """The full box list of a layout refining the blocks of ``patch`` whose
    largest |gamma - 2| (lbm_gamma_blocks) exceeds ``threshold``; non-finite
    values count as flagged.  None when nothing is flagged or no valid layout
    is found (boxes_from_flags).  The grid's state is read, not changed."""
    dev = grid.gamma_blocks(patch, block).cpu().numpy()
    return boxes_from_flags(~(dev <= threshold), grid.patches[patch], block, case, margin, grid.storage)


def regrid(grid, case: dict, boxes: list):
    """A new grid of ``case`` with ``boxes`` (the full list, all levels) in
    the storage of ``grid``, holding ``grid``'s state (lbm_transfer).
    Returns (new grid, number of fluid nodes no source level held)."""
    from . import lbm as L
    new = L.Grid(dict(case, boxes=list(boxes)), grid.storage, device=grid.buffer.device)
    missing = new.transfer_from(grid)
    return new, missing
