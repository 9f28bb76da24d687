"""Slab partition along x with halo exchange (the multi-GPU decomposition of
a level, exercised on CPU ranks): a split run, each rank pulling from its
slab plus ghost layers and colliding its own nodes with the oracle's
collision, is bitwise equal to the unsplit oracle."""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_06915_gb300 import partition as PT

N = (12, 6, 5)  # x, y, z


def _case():
    return dict(name="box", n=N, periodic=(1, 1, 1), walls=(0,) * 6, inflow_axis=-1, u_in=(0, 0, 0), boxes=[],
                solid=None, nu0=0.02, accel0=(0, 0, 0), mirror_lbgk=False, thermal=None)


def _initial(o):
    rng = np.random.default_rng(11)
    shp = o.shape(0)
    rho = 1.0 + 0.02 * rng.standard_normal(shp)
    u = 0.04 * rng.standard_normal((3,) + shp)
    o.init_equilibrium(0, rho, u)
    return o.get_pop(0)


def _collide_all(f, beta):
    out = np.empty_like(f)
    q, nz, ny, nx = f.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                out[:, z, y, x], _ = O.collide(f[:, z, y, x], beta)
    return out


def test_slab_bounds_cover_the_level():
    for nx in (5, 12, 13):
        for P in (1, 2, 3, 5):
            spans = [PT.slab_bounds(nx, P, r) for r in range(P)]
            assert spans[0][0] == 0 and spans[-1][1] == nx
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
    with pytest.raises(ValueError):
        PT.slab_bounds(2, 3, 0)


def test_nine_populations_cross_each_face():
    assert len(PT.TO_RIGHT) == 9 and len(PT.TO_LEFT) == 9
    assert all(PT.CX[i] == 1 for i in PT.TO_RIGHT) and all(PT.CX[i] == -1 for i in PT.TO_LEFT)
    assert sorted(26 - i for i in PT.TO_RIGHT) == sorted(PT.TO_LEFT)


def test_three_slabs_in_one_process_match_the_oracle():
    """Ghost data passed by hand between three uneven slabs."""
    o = O.Oracle(_case())
    f = _initial(o)
    beta = o.patches[0]["beta"]
    P = 3
    spans = [PT.slab_bounds(N[0], P, r) for r in range(P)]
    local = [f[..., a:b].copy() for a, b in spans]
    for _ in range(2):
        packs = [PT.pack_faces(s) for s in local]
        nxt = []
        for r in range(P):
            from_left = packs[(r - 1) % P][1]
            from_right = packs[(r + 1) % P][0]
            nxt.append(_collide_all(PT.pull_local(PT.with_ghosts(local[r], from_left, from_right)), beta))
        local = nxt
        o.step(1)
    assert np.array_equal(np.concatenate(local, axis=-1), o.get_pop(0))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        o = O.Oracle(_case())
        f = _initial(o)
        beta = o.patches[0]["beta"]
        a, b = PT.slab_bounds(N[0], world, rank)
        mine = f[..., a:b].copy()
        for _ in range(3):
            from_left, from_right = PT.exchange(mine, rank, world, dist)
            mine = _collide_all(PT.pull_local(PT.with_ghosts(mine, from_left, from_right)), beta)
        np.save(os.path.join(out_dir, "slab%d.npy" % rank), mine)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_the_unsplit_oracle(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    o = O.Oracle(_case())
    _initial(o)
    o.step(3)
    split = np.concatenate([np.load(tmp_path / ("slab%d.npy" % r)) for r in range(world)], axis=-1)
    assert np.array_equal(split, o.get_pop(0))


# ---------------------------------------------------------------------------
# Refined layouts: aligned level slabs, the coupling's parent halo, FP64 sums

def test_level_slabs_keep_twins_on_one_rank():
    nx = 13
    for P in (1, 2, 3, 4):
        for level in (1, 2):
            spans = [PT.level_slab(nx, P, r, level) for r in range(P)]
            assert spans[0][0] == 0 and spans[-1][1] == nx << level
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            for x in range(nx << level):
                r = PT.owner(x, nx, P, level)
                if x % (1 << level) == 0:  # coincides with a coarse node: same rank
                    assert r == PT.owner(x >> level, nx, P, 0)


def test_parent_halo_covers_every_reconstruction_sample():
    """Brute force over the child nodes of each slab: every parent sample of
    the four-point rule, and every pull source of it, lies within the
    parent_halo() layers below and above the slab, and both bounds are reached."""
    hl, hh = PT.parent_halo()
    assert (hl, hh) == (2, 3)
    nx, P = 12, 3
    for r in range(P):
        a, b = PT.slab_bounds(nx, P, r)  # parent (coarse) slab [a, b)
        lo, hi = a, b - 1
        for xc in range(2 * a, 2 * b):  # the slab's child nodes, child units
            if xc % 2 == 0:
                continue  # on the parent lattice along x: no interpolation along x
            for off in PT.SAMPLE_OFFSETS:
                xs = xc / 2.0 + off  # parent node of the sample
                assert xs == int(xs)
                for pull in (-1, 0, 1):  # the sample is the pulled state of that node
                    lo, hi = min(lo, xs + pull), max(hi, xs + pull)
        assert (lo, hi) == (a - hl, b - 1 + hh), (r, lo, hi)


def _sum_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        mine = rng.standard_normal(8) * 10.0 ** rng.integers(-8, 8, 8)
        tot = PT.allreduce_sums(mine, dist)
        np.save(os.path.join(out_dir, "sum%d.npy" % rank), tot)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_allreduce_sums_equal_the_serial_sum_on_every_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_sum_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    parts = [np.random.default_rng(100 + r) for r in range(world)]
    serial = np.zeros(8)
    for g in parts:
        serial = serial + g.standard_normal(8) * 10.0 ** g.integers(-8, 8, 8)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / ("sum%d.npy" % r)), serial)
