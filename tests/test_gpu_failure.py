"""Failure detection on the GPU, made without faulting it.

* A bounded wait that runs out: the stage waits of the TMA stream-collide
  passes take their bound from the host (lbm_wait_limit).  With a bound of
  zero the consumers test each stage once, find the first tile's loads still
  in flight, flag bit 1 of the status word, wait with the full bound for the
  copies in flight and return; lbm_diagnostics then reports LBM_ERR_TIMEOUT,
  clears the bit, and with the default bound the grid steps on normally.
* A non-finite population written from the host: lbm_diagnostics reports
  LBM_ERR_UNSTABLE.
"""
import math

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


def _grid(case, storage="fp32"):
    import torch
    from paper_1608_06915_gb300 import lbm as L
    g = L.Grid(case, storage)
    for p, info in enumerate(g.patches):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        rho, u = I.tgv_fields(x, y, z, n=case["n"][0])
        g.init_equilibrium(p, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    return g


@pytest.mark.parametrize("thermal", [False, True])
def test_expired_wait_is_reported_and_the_grid_recovers(thermal):
    import torch
    from paper_1608_06915_gb300 import lbm as L
    if thermal:
        case = I.rbc_small_case()
        g = L.Grid(case, "fp32")
        for p, info in enumerate(g.patches):
            rho, u, T = I.rbc_fields(case, info["level"], info["org"], info["dim"])
            g.init_equilibrium(p, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(),
                               torch.from_numpy(T).cuda())
    else:
        g = _grid(I.tgv_case(n=32))
    g.step(1)
    assert g.diagnostics()["status"] == 0
    g.wait_limit(0)
    seen = None
    for _ in range(4):  # the first tile's loads are in flight when a consumer first tests its stage
        g.step(1)
        try:
            g.diagnostics()
        except L.LbmError as e:
            seen = e
            break
    assert seen is not None and seen.status == -6, seen
    # the bit was cleared when reported; the default bound steps on normally
    g.wait_limit(1 << 21)
    g.step(2)
    d = g.diagnostics()
    assert d["status"] == 0 and math.isfinite(d["mass"]) and d["min_rho"] > 0


def test_host_written_nan_is_reported_as_unstable():
    import torch
    from paper_1608_06915_gb300 import lbm as L
    g = _grid(I.tgv_case(n=24, box=(6, 18), nu=0.02))
    g.step(1)
    f = g.get_populations(1)
    nz, ny, nx = g.shape(1)
    f[5, nz // 2, ny // 2, nx // 2] = float("nan")
    g.set_populations(1, f)
    with pytest.raises(L.LbmError) as e:
        g.diagnostics()
    assert e.value.status == -5
    with pytest.raises(L.LbmError) as e:
        g.diagnostics_noalloc()
    assert e.value.status == -5
