"""The allocation-free diagnostics entry point.

lbm_diagnostics_noalloc gives callers that cannot allocate device memory the
same FP64 sums as lbm_diagnostics, with its partial sums in a fixed array
inside the library instead of the grid's bound buffer.  This file sorts last
so that a run stopping at the first failure has run every other test first;
it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1608_06915_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_06915_gb300 import build as B
    B.build()


def _grid(case, storage, fields):
    import torch
    from paper_1608_06915_gb300 import lbm as L
    g = L.Grid(case, storage)
    for p, info in enumerate(g.patches):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        rho, u = fields(x, y, z, info)
        g.init_equilibrium(p, torch.from_numpy(np.ascontiguousarray(rho)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(u)).cuda())
    return g


def _close(a, b, tol=1e-12):
    for k in ("mass", "kinetic_energy", "fluid_nodes", "min_rho"):
        assert abs(a[k] - b[k]) <= tol * max(1.0, abs(b[k])), (k, a[k], b[k])
    for x, y in zip(a["momentum"], b["momentum"]):
        assert abs(x - y) <= tol * max(1.0, abs(a["mass"])), (x, y)
    assert a["status"] == b["status"]


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_noalloc_matches_diagnostics_two_calls(storage):
    case = I.channel_small_case()
    g = _grid(case, storage, lambda x, y, z, info: I.channel_fields(case, info["level"], info["org"], info["dim"]))
    g.step(2)
    for _ in range(2):  # two calls in a row: the shared array keeps the last call's contents
        ref = g.diagnostics()
        got = g.diagnostics_noalloc()
        _close(got, ref)
        g.step(1)


def test_noalloc_allocates_nothing_after_the_first_call():
    # The first call on a device may be where CUDA's lazy module loading
    # places the library's module, and the array with it, on the device; from
    # then on a call must leave the device's memory as it found it: nothing
    # through torch's allocator and nothing through the driver.
    # Python's cycle collector is held off while measuring, so that tensors
    # of earlier tests freed meanwhile do not move the counts.
    import gc

    import torch
    case = I.channel_small_case()
    g = _grid(case, "fp32", lambda x, y, z, info: I.channel_fields(case, info["level"], info["org"], info["dim"]))
    g.step(1)
    g.diagnostics_noalloc()
    torch.cuda.synchronize()
    gc.collect()
    gc.disable()
    try:
        alloc0 = torch.cuda.memory_allocated()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            g.diagnostics_noalloc()
            torch.cuda.synchronize()
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
    finally:
        gc.enable()


def test_noalloc_rejects_too_many_patches():
    from paper_1608_06915_gb300 import lbm as L
    case = I.tgv_case(n=64)
    # 27 small level-1 boxes: more patches than the fixed array covers
    boxes = []
    for i in range(3):
        for j in range(3):
            for k in range(3):
                lo = (4 + 20 * i, 4 + 20 * j, 4 + 20 * k)
                boxes.append((1, lo, tuple(v + 10 for v in lo)))
    case["boxes"] = boxes
    g = _grid(case, "fp32", lambda x, y, z, info: I.uniform_fields(x, (0.01, 0.0, 0.0)))
    assert len(g.patches) > 16
    g.diagnostics()
    with pytest.raises(L.LbmError) as e:
        g.diagnostics_noalloc()
    assert "at most 16 patches" in str(e.value)
