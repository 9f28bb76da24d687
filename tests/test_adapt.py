"""Refinement boxes from the stabiliser gamma (Sec. IV channel discussion and
the conclusion's adaptive-refinement criterion): the host logic that turns
flagged blocks into layout boxes (CPU), and the GPU indicator against the
oracle's gamma (gpu)."""
import numpy as np
import pytest

from paper_1608_06915_gb300 import adapt as A
from paper_1608_06915_gb300 import inputs as I


def test_clusters_are_face_connected_components():
    f = np.zeros((6, 5, 7), dtype=bool)
    f[1, 1, 1:4] = True          # a run along x
    f[2, 1, 3] = True            # joined to it through a face
    f[4, 3, 5] = True            # a separate single block
    f[4, 4, 6] = True            # diagonal neighbour of the last: separate
    got = sorted(A.clusters(f))
    assert got == sorted([((1, 1, 1), (3, 1, 2)), ((5, 3, 4), (5, 3, 4)), ((6, 4, 4), (6, 4, 4))])
    assert A.clusters(np.zeros((2, 2, 2), dtype=bool)) == []


def test_block_box_to_coarse_units():
    # a level-1 patch whose storage box starts at level coordinate 8 (coarse 4)
    info = dict(level=1, org=(8, 8, 8), dim=(17, 17, 17))
    lo, hi = A.block_box_to_coarse(info, 4, (0, 1, 4), (1, 1, 4), 0, (32, 32, 32))
    # x: nodes 0..7 -> level 8..15 -> coarse 4..7.5 -> [4, 8]; y: nodes 4..7 -> [6, 8];
    # z: block 4 is node 16 only (the box has 17 nodes) -> level 24 -> coarse [12, 12]
    assert (lo, hi) == ((4, 6, 12), (8, 8, 12))
    lo, hi = A.block_box_to_coarse(info, 4, (0, 0, 0), (4, 4, 4), 2, (12, 12, 12))
    assert lo == (2, 2, 2) and hi == (11, 11, 11)  # grown by 2, clipped to the domain


def test_merge_boxes_until_separated():
    b = [((0, 0, 0), (3, 3, 3)), ((10, 0, 0), (12, 3, 3)), ((30, 0, 0), (31, 3, 3))]
    assert A.merge_boxes(b, 8) == [((0, 0, 0), (12, 3, 3)), ((30, 0, 0), (31, 3, 3))]
    assert len(A.merge_boxes(b, 20)) == 1
    # separated along one axis only is enough
    assert len(A.merge_boxes([((0, 0, 0), (3, 3, 3)), ((0, 20, 0), (3, 23, 3))], 8)) == 2


def test_boxes_from_flags_merges_with_existing_boxes():
    """Flagged blocks next to an existing level-1 box join it; far ones get a
    box of their own; the resulting layouts pass the validation."""
    from paper_1608_06915_gb300 import lbm as L
    case = I.tgv_case(n=48, box=(8, 18))  # one level-1 box [8, 18]^3
    info = dict(level=0, org=(0, 0, 0), dim=(48, 48, 48))
    f = np.zeros((12, 12, 12), dtype=bool)  # blocks of 4 nodes
    f[4, 4, 5] = True  # x 20..23, y 16..19, z 16..19: within 8 of the existing box
    boxes = A.boxes_from_flags(f, info, 4, case)
    assert boxes is not None and len(boxes) == 1
    lev, lo, hi = boxes[0]
    assert lev == 1 and lo[0] <= 8 and hi[0] >= 23 and lo[1] <= 8 and hi[1] >= 19
    f = np.zeros((12, 12, 12), dtype=bool)
    f[9, 9, 9] = True  # x, y, z 36..39: far from it
    boxes = A.boxes_from_flags(f, info, 4, case)
    assert boxes is not None and len(boxes) == 2 and (1, (8, 8, 8), (18, 18, 18)) in boxes
    L.Grid(dict(case, boxes=boxes), "fp32", bind=False)
    assert A.boxes_from_flags(np.zeros((12, 12, 12), dtype=bool), info, 4, case) is None


def test_boxes_from_flags_keeps_to_the_parent_patch():
    """Blocks flagged at the face of a level-1 patch: widened to the minimum
    width, their level-2 box would stick out of the patch, which the layout
    rules reject.  It is moved back inside the region where it nests; the
    level-2 box under the other level-1 patch is kept as it was."""
    from paper_1608_06915_gb300 import lbm as L
    case = I.tgv_case(n=64, refined=False)
    case["boxes"] = [(1, (4, 4, 4), (24, 24, 24)), (1, (34, 4, 4), (56, 26, 26)),
                     (2, (36, 10, 10), (42, 20, 20))]
    g = L.Grid(case, "fp32", bind=False)
    info = g.patches[1]
    assert info["level"] == 1 and tuple(info["org"]) == (8, 8, 8)
    assert A.parent_region(info, case["n"]) == ((6, 6, 6), (22, 22, 22))
    nb = [-(-d // 4) for d in info["dim"]]  # blocks of 4 level-1 nodes
    f = np.zeros((nb[2], nb[1], nb[0]), dtype=bool)
    f[5, 5, nb[0] - 1] = True  # the last block along x: coarse x 24
    boxes = A.boxes_from_flags(f, info, 4, case)
    assert boxes is not None
    assert (2, (36, 10, 10), (42, 20, 20)) in boxes and (1, (34, 4, 4), (56, 26, 26)) in boxes
    lev2 = [b for b in boxes if b[0] == 2 and b != (2, (36, 10, 10), (42, 20, 20))]
    assert len(lev2) == 1
    _, lo, hi = lev2[0]
    assert all(6 <= lo[a] and hi[a] <= 22 and hi[a] - lo[a] >= 4 for a in range(3)) and hi[0] == 22
    L.Grid(dict(case, boxes=boxes), "fp32", bind=False)


def test_widen_keeps_boxes_inside_the_domain():
    assert A.widen(((10, 10, 10), (12, 10, 11)), 8, (32, 32, 32)) == ((7, 6, 7), (15, 14, 15))
    assert A.widen(((0, 0, 29), (1, 2, 31)), 8, (32, 32, 32)) == ((0, 0, 23), (8, 8, 31))


def test_widened_merged_boxes_pass_the_layout_validation():
    from paper_1608_06915_gb300 import lbm as L
    case = I.tgv_case(n=32, refined=False)
    raw = [((6, 6, 6), (10, 10, 10)), ((14, 6, 6), (16, 10, 10))]
    boxes = A.merge_boxes([A.widen(b, 8.0, case["n"]) for b in raw], 8.0)
    assert len(boxes) == 1
    L.Grid(dict(case, boxes=[(1, lo, hi) for lo, hi in boxes]), "fp32", bind=False)
    with pytest.raises(L.LbmError):  # as they came, the boxes are too narrow and too close
        L.Grid(dict(case, boxes=[(1, lo, hi) for lo, hi in raw]), "fp32", bind=False)


def _ball(n=16, nu0=0.002):
    """Single-level periodic box with a solid ball: bulk and boundary-class nodes only."""
    return dict(name="ball", n=(n, n, n), periodic=(1, 1, 1), walls=(0,) * 6, inflow_axis=-1, u_in=(0, 0, 0),
                boxes=[], solid=I.sphere_mask(0, (n / 2, n / 2, n / 2), 6.0), nu0=nu0, accel0=(0, 0, 0),
                mirror_lbgk=False, thermal=None)


@pytest.mark.gpu
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_gamma_blocks_match_the_oracle(storage):
    """The GPU indicator against the oracle's own gamma: the GPU reads the
    oracle's state after three steps and gives the block maxima of |gamma - 2|
    for the next collision; the oracle takes that step and reports the gamma
    of each node's collision.  Single level with a solid ball, so every fluid
    node is a bulk or boundary-class node."""
    import torch
    from oracle import oracle as O
    from paper_1608_06915_gb300 import lbm as L
    case = _ball()
    o = O.Oracle(case)
    g = L.Grid(case, storage)
    rng = np.random.default_rng(41)
    info = g.patches[0]
    x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
    rho = 1.0 + 0.02 * rng.standard_normal(x.shape)
    u = 0.04 * rng.standard_normal((3,) + x.shape)  # rough: gamma far from 2 in places
    o.init_equilibrium(0, rho, u)
    o.step(3)
    g.set_populations(0, torch.from_numpy(o.get_pop(0)).cuda())
    block = 3
    got = g.gamma_blocks(0, block).cpu().numpy()
    o.step(1)
    m = o.mask(0) == 1
    gam = o.moments(0)[3]
    dev = np.where(m, np.abs(gam - 2.0), 0.0)
    nb = [(s + block - 1) // block for s in m.shape]
    ref = np.zeros(nb)
    for idx in np.ndindex(*m.shape):
        b = tuple(i // block for i in idx)
        ref[b] = max(ref[b], dev[idx])
    assert got.shape == ref.shape
    assert ref.max() > 0.05, ref.max()
    tol = 1e-6 if storage == "fp64" else 1e-3
    assert np.max(np.abs(got - ref)) < tol * max(1.0, ref.max()), np.max(np.abs(got - ref))


@pytest.mark.gpu
def test_refinement_boxes_cover_the_rough_region():
    """A fluid at rest but for one rough region: the suggested level-1 box
    covers that region, stays local, and the layout accepts it."""
    import torch
    from paper_1608_06915_gb300 import lbm as L
    case = I.tgv_case(n=32, refined=False, nu=0.002)
    g = L.Grid(case, "fp64")
    info = g.patches[0]
    x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
    rng = np.random.default_rng(42)
    rough = (np.abs(x - 20) < 3) & (np.abs(y - 12) < 3) & (np.abs(z - 16) < 3)
    # fluid at rest (gamma exactly 2: no non-equilibrium part) but for the rough region
    u = 0.04 * rough * rng.standard_normal((3,) + x.shape)
    g.init_equilibrium(0, torch.ones(x.shape, dtype=torch.float64).cuda(), torch.from_numpy(u).cuda())
    g.step(2)
    dev = g.gamma_blocks(0, 4).cpu().numpy()
    # every flagged block touches the rough region (x 18..22, y 10..14, z 14..18) grown by three
    # nodes (two steps and the pull of the next): the rest state elsewhere has gamma = 2 exactly
    assert (dev > 0).any()
    for bz, by, bx in zip(*np.nonzero(dev > 0)):
        assert 4 * bx <= 25 and 4 * bx + 3 >= 15 and 4 * by <= 17 and 4 * by + 3 >= 7 and 4 * bz <= 21 \
            and 4 * bz + 3 >= 11, (bx, by, bz)
    boxes = A.refinement_boxes(g, case, 0, block=4, threshold=0.5 * float(dev.max()))
    assert len(boxes) == 1
    lev, lo, hi = boxes[0]
    assert lev == 1
    assert lo[0] <= 18 and hi[0] >= 22 and lo[1] <= 10 and hi[1] >= 14 and lo[2] <= 14 and hi[2] >= 18, boxes
    assert all(hi[a] - lo[a] < 24 for a in range(3)), boxes  # not the whole domain


def _load_from_oracle(g, o):
    import torch
    for p in range(len(o.patches)):
        g.set_populations(p, torch.from_numpy(o.get_pop(p)).cuda())


@pytest.mark.gpu
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_transfer_matches_the_oracle_and_steps_on(storage, tol):
    """A two-level state (after four oracle steps) moved onto a layout with
    the level-1 box shifted and a level-2 box added: every node against the
    oracle's own transfer (reading R9), then two more coarse steps on both."""
    from oracle import oracle as O
    from paper_1608_06915_gb300 import lbm as L
    src_case = I.tgv_case(n=16, box=(4, 12), nu=0.005)
    o_src = O.Oracle(src_case)
    for p, info in enumerate(o_src.patches):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        o_src.init_equilibrium(p, *I.tgv_fields(x, y, z, n=16))
    o_src.step(4)
    g_src = L.Grid(src_case, storage)
    _load_from_oracle(g_src, o_src)
    dst_case = dict(src_case, boxes=[(1, (6, 5, 6), (15, 13, 14)), (2, (8, 7, 8), (12, 11, 12))])
    o_dst = O.Oracle(dst_case)
    g_dst = L.Grid(dst_case, storage)
    assert o_dst.transfer_from(o_src) == 0
    assert g_dst.transfer_from(g_src) == 0
    for step in range(3):
        for p in range(len(o_dst.patches)):
            m = o_dst.mask(p) == 1
            d = np.max(np.abs(g_dst.get_populations(p).cpu().numpy()[:, m] - o_dst.get_pop(p)[:, m]))
            assert d < tol, (step, p, d)
        o_dst.step(1)
        g_dst.step(1)


@pytest.mark.gpu
def test_regrid_from_the_indicator():
    """Indicator, boxes and transfer together: a rough region gets a level-1
    box, the state moves onto the new layout with no node left without a
    source, and the new grid steps on, its mass kept."""
    import torch
    from paper_1608_06915_gb300 import lbm as L
    case = I.tgv_case(n=32, refined=False, nu=0.002)
    g = L.Grid(case, "fp64")
    info = g.patches[0]
    x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
    rng = np.random.default_rng(43)
    rough = (np.abs(x - 16) < 3) & (np.abs(y - 16) < 3) & (np.abs(z - 16) < 3)
    u = 0.04 * rough * rng.standard_normal((3,) + x.shape)
    g.init_equilibrium(0, torch.ones(x.shape, dtype=torch.float64).cuda(), torch.from_numpy(u).cuda())
    g.step(2)
    dev = g.gamma_blocks(0, 4).cpu().numpy()
    boxes = A.refinement_boxes(g, case, 0, block=4, threshold=0.5 * float(dev.max()))
    assert len(boxes) == 1
    new, missing = A.regrid(g, case, boxes)
    assert missing == 0 and len(new.patches) == 2
    m0 = new.diagnostics()["mass"]  # on the new layout (the level weighting differs from the old one)
    new.step(5)
    d = new.diagnostics()
    assert d["status"] == 0
    assert abs(d["mass"] - m0) < 1e-4 * m0, (d["mass"], m0)
