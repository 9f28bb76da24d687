"""Discrete adjoint: the FP64 reference gradient (PyTorch autograd of a plain
restatement of the refined step, pinned to the C oracle) and the CUDA adjoint
(lbm_adjoint_step) against it and against finite differences."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import torch_oracle as T
from paper_1608_06915_gb300 import inputs as I

N, A, B, NU = 16, 4, 12, 0.02


def small_case():
    return I.tgv_case(n=N, box=(A, B), nu=NU)


def initial_fields(seed=4):
    modes = I.divfree_modes(n=N, kmax=3.0, rms=0.03, seed=seed)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    _, uc = I.divfree_fields(x * 1.0, y * 1.0, z * 1.0, modes)
    m = 2 * (B - A) + 1
    z, y, x = np.meshgrid(*[np.arange(m) + 2 * A] * 3, indexing="ij")
    _, uf = I.divfree_fields(x * 0.5, y * 0.5, z * 0.5, modes)
    return uc, uf  # [3][z][y][x]


def to_rows(u):
    return torch.tensor(u.reshape(3, -1).T.copy(), dtype=torch.float64)


# --- pins of the reference (CPU)
def test_torch_oracle_forward_matches_c_oracle():
    uc, uf = initial_fields()
    m = T.TwoLevel(N, A, B, NU)
    fc = T.feq(torch.ones(N ** 3, dtype=torch.float64), to_rows(uc))
    ff = T.feq(torch.ones(m.m ** 3, dtype=torch.float64), to_rows(uf))
    o = O.Oracle(small_case())
    o.init_equilibrium(0, np.ones(uc.shape[1:]), uc)
    o.init_equilibrium(1, np.ones(uf.shape[1:]), uf)
    for _ in range(3):
        fc, ff = m.step(fc, ff)
        o.step(1)
    gc = o.get_pop(0).reshape(27, -1).T
    gf = o.get_pop(1).reshape(27, -1).T
    mc = o.mask(0).ravel() == 1
    assert np.max(np.abs(fc.numpy()[mc] - gc[mc])) < 1e-13
    assert np.max(np.abs(ff.numpy() - gf)) < 1e-13


def test_torch_oracle_gradient_matches_central_differences():
    """autograd gradient vs FP64 central differences of the C oracle's forward."""
    uc, uf = initial_fields()
    m = T.TwoLevel(N, A, B, NU)
    tc, tf = to_rows(uc).requires_grad_(True), to_rows(uf).requires_grad_(True)
    ke, _, _ = m.run(tc, tf, 3)
    ke.backward()
    rng = np.random.default_rng(100)

    def c_oracle_ke(duc, duf):
        o = O.Oracle(small_case())
        o.init_equilibrium(0, np.ones(uc.shape[1:]), uc + duc)
        o.init_equilibrium(1, np.ones(uf.shape[1:]), uf + duf)
        o.step(3)
        fc = torch.tensor(o.get_pop(0).reshape(27, -1).T)
        ff = torch.tensor(o.get_pop(1).reshape(27, -1).T)
        return float(m.kinetic_energy(fc, ff))

    for _ in range(2):
        dc, df = rng.normal(size=uc.shape), rng.normal(size=uf.shape)
        eps = 1e-6  # truncation error ~ eps^2 along white-noise directions (measured 2.5e-8 here)
        fd = (c_oracle_ke(eps * dc, eps * df) - c_oracle_ke(-eps * dc, -eps * df)) / (2 * eps)
        ad = float((tc.grad * to_rows(dc)).sum() + (tf.grad * to_rows(df)).sum())
        assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


# --- CUDA adjoint
def _gpu_grad(storage, steps, K, uc, uf):
    from paper_1608_06915_gb300 import lbm as L
    g = L.Grid(small_case(), storage)
    u0 = [torch.tensor(uc).cuda().requires_grad_(True), torch.tensor(uf).cuda().requires_grad_(True)]
    J = L.kinetic_energy_run(g, u0, steps, K)
    J.backward()
    return float(J), u0[0].grad.cpu().numpy(), u0[1].grad.cpu().numpy()


def _ref_grad(steps, uc, uf):
    m = T.TwoLevel(N, A, B, NU)
    tc, tf = to_rows(uc).requires_grad_(True), to_rows(uf).requires_grad_(True)
    ke, _, _ = m.run(tc, tf, steps)
    ke.backward()
    return float(ke), tc.grad.numpy().T.reshape(uc.shape), tf.grad.numpy().T.reshape(uf.shape)


@pytest.mark.gpu
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_cuda_adjoint_matches_reference_gradient(storage, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    uc, uf = initial_fields()
    jr, gcr, gfr = _ref_grad(6, uc, uf)
    jg, gcg, gfg = _gpu_grad(storage, 6, 3, uc, uf)
    scale = max(np.abs(gcr).max(), np.abs(gfr).max())
    err = max(np.abs(gcg - gcr).max(), np.abs(gfg - gfr).max()) / scale
    print("adjoint %s: J %.12e vs %.12e, max gradient error / max gradient %.3e" % (storage, jg, jr, err))
    assert abs(jg - jr) < (1e-12 if storage == "fp64" else 1e-5) * abs(jr)
    assert err < tol


@pytest.mark.gpu
def test_cuda_adjoint_full_case_finite_differences():
    """64^3 box with [24,40]^3 refined, objective after 200 coarse steps,
    checkpoints every 20, 16 seeded smooth directions, central differences of
    the FP64 forward: the FP64 adjoint within 1e-6 relative per direction; the
    FP32-storage adjoint (FP64 gradient reduction) within 1e-4 of the
    gradient's norm (a direction with a small derivative measures the FP32
    trajectory's rounding, not the adjoint)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_06915_gb300 import lbm as L
    case = I.adjoint_case()
    g32 = L.Grid(case, "fp32")
    g64 = L.Grid(case, "fp64")
    modes = I.divfree_modes(n=64, kmax=4.0, rms=0.03, seed=4)
    u0 = []
    for info in g32.patches:
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        u0.append(torch.tensor(I.divfree_fields(x, y, z, modes)[1]).cuda())
    steps, K = 200, 20
    grads = {}
    for name, g in (("fp32", g32), ("fp64", g64)):
        x0 = [u.clone().requires_grad_(True) for u in u0]
        L.kinetic_energy_run(g, x0, steps, K).backward()
        grads[name] = [u.grad for u in x0]
    gnorm = math.sqrt(sum(float((v * v).sum()) for v in grads["fp64"]))
    norm = math.sqrt(sum(float((u * u).sum()) for u in u0))
    worst64 = worst32 = 0.0
    for seed in range(100, 116):
        # smooth seeded directions (divergence-free Fourier fields, |k| <= 4)
        dm = I.divfree_modes(n=64, kmax=4.0, rms=0.03, seed=seed)
        d = []
        for info in g32.patches:
            x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
            d.append(torch.tensor(I.divfree_fields(x, y, z, dm)[1]).cuda())
        dn = math.sqrt(sum(float((v * v).sum()) for v in d))
        d = [v / dn for v in d]
        eps = 1e-4 * norm
        jp = float(L.kinetic_energy_run(g64, [u + eps * v for u, v in zip(u0, d)], steps, K))
        jm = float(L.kinetic_energy_run(g64, [u - eps * v for u, v in zip(u0, d)], steps, K))
        fd = (jp - jm) / (2 * eps)
        a64 = sum(float((gr * v).sum()) for gr, v in zip(grads["fp64"], d))
        a32 = sum(float((gr * v).sum()) for gr, v in zip(grads["fp32"], d))
        r64, r32 = abs(fd - a64) / abs(fd), abs(fd - a32) / gnorm
        worst64, worst32 = max(worst64, r64), max(worst32, r32)
        print("direction %d: finite difference %.10e adjoint fp64 %.10e (rel %.1e) fp32 %.10e (/|grad| %.1e)" % (
            seed, fd, a64, r64, a32, r32))
    assert worst64 < 1e-6, worst64
    assert worst32 < 1e-4, worst32


@pytest.mark.gpu
def test_cuda_adjoint_three_levels_finite_differences():
    """32^3 periodic box, [4,28]^3 refined once and [10,22]^3 (level-1 units)
    twice, FP64, 6 coarse steps with a checkpoint every 3: directional
    derivatives along 3 smooth seeded directions against central differences,
    then a forward run after the adjoint reproduces the first one."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_06915_gb300 import lbm as L
    case = dict(I.tgv_case(n=32, box=(4, 28)), boxes=[(1, (4, 4, 4), (28, 28, 28)), (2, (10, 10, 10), (22, 22, 22))])
    g = L.Grid(case, "fp64")

    def fields(seed):
        m = I.divfree_modes(n=32, kmax=3.0, rms=0.03, seed=seed)
        out = []
        for info in g.patches:
            x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
            out.append(torch.tensor(I.divfree_fields(x, y, z, m)[1]).cuda())
        return out

    u0 = fields(7)
    steps, K = 6, 3
    x0 = [u.clone().requires_grad_(True) for u in u0]
    J = L.kinetic_energy_run(g, x0, steps, K)
    J.backward()
    grads = [u.grad for u in x0]
    assert float(L.kinetic_energy_run(g, u0, steps, K)) == float(J)
    norm = math.sqrt(sum(float((u * u).sum()) for u in u0))
    worst = 0.0
    for seed in range(200, 203):
        d = fields(seed)
        dn = math.sqrt(sum(float((v * v).sum()) for v in d))
        d = [v / dn for v in d]
        eps = 1e-6 * norm
        jp = float(L.kinetic_energy_run(g, [u + eps * v for u, v in zip(u0, d)], steps, K))
        jm = float(L.kinetic_energy_run(g, [u - eps * v for u, v in zip(u0, d)], steps, K))
        fd = (jp - jm) / (2 * eps)
        ad = sum(float((gr * v).sum()) for gr, v in zip(grads, d))
        rel = abs(fd - ad) / abs(ad)
        worst = max(worst, rel)
        print("three levels, direction %d: finite difference %.12e adjoint %.12e rel %.2e" % (seed, fd, ad, rel))
    assert worst < 1e-6, worst


@pytest.mark.gpu
@pytest.mark.parametrize("levels", [2, 3])
def test_cuda_adjoint_graph_sweeps_match_direct_sweeps(levels):
    """The reverse walks of lbm_adjoint_step run directly (graphs off), then
    captured as CUDA graphs, then replayed from the graph cache: the three
    lambdas are the same bits.  Every lambda entry takes one store and at
    most one addition, in stream order, and the transposed interpolation
    gathers over fixed consumer lists, so nothing depends on scheduling."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_06915_gb300 import lbm as L
    if levels == 2:
        case = small_case()
    else:
        case = dict(I.tgv_case(n=32, box=(4, 28)),
                    boxes=[(1, (4, 4, 4), (28, 28, 28)), (2, (10, 10, 10), (22, 22, 22))])
    g = L.Grid(case, "fp64")
    n = case["n"][0] if isinstance(case["n"], (tuple, list)) else case["n"]
    m = I.divfree_modes(n=n, kmax=3.0, rms=0.03, seed=11)
    for p, info in enumerate(g.patches):
        x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
        rho, u = I.divfree_fields(x, y, z, m)
        g.init_equilibrium(p, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    K = 3
    ck = torch.empty(g.checkpoint_bytes(), dtype=torch.uint8, device="cuda")
    g.checkpoint(ck, save=True)
    lam, ws = g.adjoint_buffers(K)
    out = []
    for graphs in (False, True, True):
        g.graphs(graphs)
        g.step(K)
        g.adjoint_seed(lam, ws)
        g.adjoint_step(ck, K, lam, ws)
        out.append(lam.view(torch.float64).cpu().numpy().copy())
    scale = np.abs(out[0]).max()
    assert scale > 0
    for o in out[1:]:
        assert np.array_equal(o, out[0]), np.abs(o - out[0]).max() / scale


@pytest.mark.gpu
def test_cuda_adjoint_is_bitwise_reproducible_fp32():
    """Two grids with the same FP32 state: the same lambda bits after an
    adjoint segment, and again after a second segment replayed from graphs."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1608_06915_gb300 import lbm as L
    case = small_case()
    m = I.divfree_modes(n=N, kmax=3.0, rms=0.03, seed=13)
    runs = []
    for _ in range(2):
        g = L.Grid(case, "fp32")
        for p, info in enumerate(g.patches):
            x, y, z = I.node_positions(info["level"], info["org"], info["dim"])
            rho, u = I.divfree_fields(x, y, z, m)
            g.init_equilibrium(p, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        K = 4
        ck = torch.empty(g.checkpoint_bytes(), dtype=torch.uint8, device="cuda")
        g.checkpoint(ck, save=True)
        lam, ws = g.adjoint_buffers(K)
        outs = []
        for _ in range(2):
            g.step(K)
            g.adjoint_seed(lam, ws)
            g.adjoint_step(ck, K, lam, ws)
            outs.append(lam.view(torch.float32).cpu().numpy().copy())
        runs.append(outs)
    assert np.abs(runs[0][0]).max() > 0
    for a, b in zip(runs[0] + runs[1][1:], runs[1] + runs[0][1:]):
        assert np.array_equal(a, b)
