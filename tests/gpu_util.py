"""Shared helpers of the GPU parity tests: build the same seeded case on the
CUDA path and in the oracle, and compare them."""
import numpy as np

from oracle import oracle as O
from paper_1608_06915_gb300 import inputs as I

C = np.array([[(i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], dtype=np.int64)


def twin(case, storage, fields, oracle=True):
    """GPU grid and oracle initialised from the same fields(x, y, z, p, info)."""
    import torch
    from paper_1608_06915_gb300 import lbm as L
    g = L.Grid(case, storage)
    o = O.Oracle(case) if oracle else None
    for p, info in enumerate(g.patches):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        out = fields(x, y, z, p, info)
        rho, u = out[0], out[1]
        T = out[2] if len(out) > 2 else None
        if o is not None:
            o.init_equilibrium(p, rho, u, T)
        g.init_equilibrium(p, torch.from_numpy(np.ascontiguousarray(rho)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(u)).cuda(),
                           None if T is None else torch.from_numpy(np.ascontiguousarray(T)).cuda())
    return g, o


def pop_diff(g, o, which=0):
    """Largest |f_gpu - f_oracle| over the fluid nodes of every patch."""
    worst = 0.0
    for p in range(len(o.patches)):
        fg = g.get_populations(p, which).cpu().numpy()
        fo = o.get_pop(p, which)
        m = o.mask(p) == 1
        worst = max(worst, float(np.max(np.abs(fg[:, m] - fo[:, m]))))
    return worst


def macro_rel_l2(g, o):
    """Relative L2 errors of rho and u over all fluid nodes of all patches."""
    nr = dr = nu = du = 0.0
    for p in range(len(o.patches)):
        rg, ug, _, _ = g.moments(p)
        ro, uo, _, _ = o.moments(p)
        m = o.mask(p) == 1
        rg, ug = rg.cpu().numpy(), ug.cpu().numpy()
        nr += float(np.sum((rg[m] - ro[m]) ** 2))
        dr += float(np.sum(ro[m] ** 2))
        nu += float(np.sum((ug[:, m] - uo[:, m]) ** 2))
        du += float(np.sum(uo[:, m] ** 2))
    return (nr / dr) ** 0.5, (nu / max(du, 1e-300)) ** 0.5
