"""CPU tests of the C ABI: the library loads and exports every declared entry
point; the layout builder (host code of liblbm.so) agrees node by node with
the oracle's independent geometry; full-size node counts; invalid layouts are
rejected.  No compute call is made (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1608_06915_gb300 import build as B
from paper_1608_06915_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_1608_06915_gb300 import lbm
    return lbm


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    names = declared_symbols()
    assert "lbm_grid_create" in names and "lbm_step" in names
    for n in names:
        assert hasattr(lib, n), n


def iso(case):
    c = dict(case)
    c["thermal"] = None
    return c


CASES = {
    "tgv2": lambda: I.tgv_case(),
    "tgv3": lambda: dict(I.tgv_case(n=32, box=(4, 28)),
                         boxes=[(1, (4, 4, 4), (28, 28, 28)), (2, (10, 10, 10), (22, 22, 22))]),
    "channel_small": I.channel_small_case,
    "sphere_small": lambda: I.sphere_case(scale=8),
    "rbc_small_iso": lambda: iso(I.rbc_small_case()),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_layout_matches_oracle(L, name):
    case = CASES[name]()
    g = L.Grid(case, "fp32", bind=False)
    o = O.Oracle(case)
    assert len(g.patches) == len(o.patches)
    for p, (a, b) in enumerate(zip(g.patches, o.patches)):
        assert a["level"] == b["level"] and a["parent"] == b["parent"]
        assert a["org"] == b["org"] and a["dim"] == b["dim"], (p, a, b)
        assert abs(a["beta"] - b["beta"]) < 1e-15
        assert np.array_equal(g.mask(p), o.mask(p)), p
    assert g.node_updates() == o.node_updates_per_step()


def test_full_size_node_counts(L):
    # node updates per coarse step, sum over levels of fluid nodes * 2^level
    assert L.Grid(I.tgv_case(), bind=False).node_updates() == 30571 + 2 * 35937
    assert L.Grid(I.channel_case(), bind=False).node_updates() == 1638400 + 2 * 2621440 + 4 * 17825792
    assert L.Grid(I.adjoint_case(), bind=False).node_updates() == (64 ** 3 - 13 ** 3) + 2 * 33 ** 3
    g5 = L.Grid(iso(I.rbc_case()), bind=False)
    assert g5.node_updates() == 256 * 256 * 106 + 2 * 2 * 512 * 512 * 14 + 4 * 2 * 1024 * 1024 * 25
    g3 = L.Grid(I.sphere_case(), "fp32", bind=False)
    assert [p["level"] for p in g3.patches] == [0, 1, 2, 3]
    assert 30e6 < g3.node_updates() < 45e6


@pytest.mark.parametrize("boxes,msg", [
    ([(1, (8, 8, 8), (12, 24, 24))], "narrower"),
    ([(1, (8, 8, 8), (24, 24, 24)), (2, (9, 9, 9), (20, 20, 20))], "child node"),
    ([(1, (2, 2, 2), (14, 14, 14)), (1, (12, 2, 2), (28, 14, 14))], "overlap"),
    ([(2, (8, 8, 8), (24, 24, 24))], "nest"),
    ([(1, (8, 8, 8), (40, 24, 24))], "outside"),
])
def test_invalid_layouts_rejected(L, boxes, msg):
    case = I.tgv_case()
    case["boxes"] = boxes
    with pytest.raises(L.LbmError) as e:
        L.Grid(case, bind=False)
    assert e.value.status in (-1, -2)
    assert msg in str(e.value), str(e.value)


def test_bad_arguments(L):
    case = I.tgv_case()
    case["nu0"] = -1.0
    with pytest.raises(L.LbmError):
        L.Grid(case, bind=False)
    case = I.tgv_case()
    case["periodic"] = (0, 1, 1)
    with pytest.raises(L.LbmError):
        L.Grid(case, bind=False)


def test_thermal_parameters_validated(L):
    """Both Prandtl regimes are accepted (Table I), with the relaxation
    parameters swapped for Pr > 1; Pr <= 0 and T0 != 1/3 are rejected."""
    g07 = L.Grid(I.rbc_small_case(pr=0.7), bind=False)
    g2 = L.Grid(I.rbc_small_case(pr=2.0), bind=False)
    t0 = 1.0 / 3.0
    for g, pr in ((g07, 0.7), (g2, 2.0)):
        b, b1 = g.patches[0]["beta"], g.patches[0]["beta1"]
        b_nu, b_al = (b, b1) if pr <= 1 else (b1, b)
        assert abs(((0.5 / b_nu - 0.5) * t0) / ((0.5 / b_al - 0.5) * t0) - pr) < 1e-12
    for bad in (dict(pr=0.0), dict(pr=-1.0), dict(t0=0.3)):
        case = I.rbc_small_case()
        case["thermal"] = dict(case["thermal"], **bad)
        with pytest.raises(L.LbmError):
            L.Grid(case, bind=False)


def test_indicator_and_transfer_refuse_unbound_grids(L):
    """lbm_gamma_blocks and lbm_transfer check their arguments before any
    device work: an unbound grid is LBM_ERR_STATE, a bad block or patch
    LBM_ERR_ARG (no GPU needed)."""
    import ctypes
    lib = L.lib()
    a = L.Grid(I.tgv_case(n=16, box=(4, 12)), bind=False)
    b = L.Grid(I.tgv_case(n=16, refined=False), bind=False)
    assert lib.lbm_gamma_blocks(a.handle, 0, 4, ctypes.c_void_p(16)) == -7  # LBM_ERR_STATE: unbound
    assert lib.lbm_gamma_blocks(a.handle, 5, 4, ctypes.c_void_p(16)) == -1  # no patch 5
    n = ctypes.c_int64(-1)
    assert lib.lbm_transfer(a.handle, b.handle, ctypes.byref(n)) == -7
    assert lib.lbm_transfer(a.handle, a.handle, ctypes.byref(n)) == -1
    assert lib.lbm_transfer(None, b.handle, ctypes.byref(n)) == -1
    assert n.value == -1
