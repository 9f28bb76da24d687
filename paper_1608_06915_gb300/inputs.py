"""Seeded synthetic inputs: case geometries and initial macroscopic fields.

This module holds no lattice Boltzmann arithmetic.  It describes the
workloads (domain, refinement boxes, walls, solid mask, viscosity, forcing)
as plain dictionaries and evaluates initial density, velocity and
temperature fields at node positions.  Both the CUDA path and the FP64
oracle are fed from here, each computing its own equilibria from these
fields.

Workloads (coarse lattice units throughout):

* ``tgv``      -- periodic 32^3 box, centred box [8,24]^3 refined 2x,
                  2-D Taylor-Green vortex extruded in z, u0 = 0.05, nu = 0.01.
* ``channel``  -- 256x64x128, periodic x/z, half-way walls in y, bands of
                  2x (y in [0,8], [55,63]) and 4x (y in [0,4], [59,63])
                  refinement, body force for Re_tau = 180, laminar profile
                  plus seeded uniform +-5% velocity perturbations.
* ``sphere``   -- 384x192x192, equilibrium inlet at x = 0, zero-gradient
                  outlet, periodic y/z, 4 nested levels, bounce-back sphere
                  of diameter 64 finest-level nodes, Re = 3700.
* ``adjoint``  -- periodic 64^3 box with the box [24,40]^3 refined 2x,
                  seeded divergence-free random velocity (rms 0.03).
* ``rbc``      -- 256x256x128, periodic x/y, isothermal plates in z with 2x
                  and 4x refined layers, Ra = 1e7, Pr = 0.7, linear
                  temperature with seeded +-1% noise.

Each has a reduced variant with the same structure that the oracle finishes
in seconds (used by the parity tests and the CPU baseline).
"""
from __future__ import annotations

import math

import numpy as np

T0 = 1.0 / 3.0


# ---------------------------------------------------------------------------
# case geometries

def tgv_case(n: int = 32, box=(8, 24), nu: float = 0.01, refined: bool = True, lbgk: bool = False) -> dict:
    boxes = [(1, (box[0],) * 3, (box[1],) * 3)] if refined else []
    return dict(name="tgv", n=(n, n, n), periodic=(1, 1, 1), walls=(0,) * 6, inflow_axis=-1, u_in=(0, 0, 0),
                boxes=boxes, solid=None, nu0=nu, accel0=(0, 0, 0), mirror_lbgk=lbgk, thermal=None)


def channel_case(n=(256, 64, 128), l1=8, l2=4, re_tau: float = 180.0, u_tau: float = 0.0045) -> dict:
    """Channel with walls in y.  The first finest-level node sits half a finest
    spacing (1/8 coarse) from each wall, so the height is n_y - 1 + 1/4."""
    nx, ny, nz = n
    H = (ny - 1) + 0.25
    delta = H / 2.0
    nu0 = u_tau * delta / re_tau
    accel = u_tau * u_tau / delta  # g = Re_tau^2 nu^2 / delta^3
    boxes = [
        (1, (0, 0, 0), (nx - 1, l1, nz - 1)),
        (1, (0, ny - 1 - l1, 0), (nx - 1, ny - 1, nz - 1)),
        (2, (0, 0, 0), (nx - 1, l2, nz - 1)),
        (2, (0, ny - 1 - l2, 0), (nx - 1, ny - 1, nz - 1)),
    ]
    return dict(name="channel", n=n, periodic=(1, 0, 1), walls=(0, 0, 1, 1, 0, 0), inflow_axis=-1,
                u_in=(0, 0, 0), boxes=boxes, solid=None, nu0=nu0, accel0=(accel, 0, 0), mirror_lbgk=False,
                thermal=None, height=H, wall_lo=-0.125)


def channel_small_case() -> dict:
    """Same structure as ``channel_case`` at 16x32x8 coarse nodes."""
    return channel_case(n=(16, 32, 8), l1=8, l2=4)


def sphere_mask(level: int, centre, diameter_fine: float):
    """Solid mask (uint8, [z][y][x]) of a sphere on the given level's lattice.

    ``centre`` is in coarse units; a node is solid when its distance from the
    centre is below half the diameter (finest-level spacing units)."""
    s = 1 << level
    c = [ci * s for ci in centre]
    r = diameter_fine / 2.0
    lo = [int(math.floor(ci - r)) - 1 for ci in c]
    hi = [int(math.ceil(ci + r)) + 1 for ci in c]
    z, y, x = np.meshgrid(*[np.arange(lo[a], hi[a] + 1) for a in (2, 1, 0)], indexing="ij")
    d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    mask = (d2 < r * r).astype(np.uint8)
    return dict(level=level, lo=tuple(lo), mask=mask)


def sphere_case(scale: int = 1, re: float = 3700.0, u: float = 0.05, curved: bool = False) -> dict:
    """Flow past a sphere, 4 levels.  scale=1 is the full 384x192x192 case;
    scale=8 gives a 48x24x24 coarse grid with the same nesting.  With
    ``curved`` the sphere itself is the analytic surface of the wall
    (interpolated bounce-back), else the staircase of its solid nodes."""
    if scale == 1:
        n = (384, 192, 192)
        boxes = [(1, (80, 80, 80), (160, 112, 112)), (2, (86, 86, 86), (132, 106, 106)),
                 (3, (90, 89, 89), (110, 103, 103))]
        centre, d_fine = (96, 96, 96), 64.0
    else:
        n = (48, 24, 24)
        boxes = [(1, (8, 4, 4), (36, 20, 20)), (2, (10, 6, 6), (30, 18, 18)), (3, (12, 8, 8), (24, 16, 16))]
        centre, d_fine = (18, 12, 12), 24.0
    nu_fine = u * d_fine / re
    nu0 = nu_fine / 8.0
    case = dict(name="sphere", n=n, periodic=(0, 1, 1), walls=(0,) * 6, inflow_axis=0, u_in=(u, 0, 0),
                boxes=boxes, solid=sphere_mask(3, centre, d_fine), nu0=nu0, accel0=(0, 0, 0), mirror_lbgk=False,
                thermal=None)
    if curved:
        case["wall_shape"] = dict(kind="sphere", c=tuple(float(c) for c in centre), r=d_fine / 16.0,
                                  solid_inside=True)
    return case


def adjoint_case(n: int = 64, box=(24, 40), nu: float = 0.01) -> dict:
    c = tgv_case(n=n, box=box, nu=nu)
    c["name"] = "adjoint"
    return c


def rbc_case(n=(256, 256, 128), l1=12, l2=6, ra: float = 1e7, pr: float = 0.7, u_ff: float = 0.05,
             dT: float = 0.01) -> dict:
    """Rayleigh-Benard cell with plates at z (half a finest spacing outside the
    first and last node)."""
    nx, ny, nz = n
    H = (nz - 1) + 0.25
    nu0 = u_ff * H * math.sqrt(pr / ra)
    glambda = u_ff * u_ff / (dT * H)  # U_ff = sqrt(g lambda dT H)
    boxes = [
        (1, (0, 0, 0), (nx - 1, ny - 1, l1)),
        (1, (0, 0, nz - 1 - l1), (nx - 1, ny - 1, nz - 1)),
        (2, (0, 0, 0), (nx - 1, ny - 1, l2)),
        (2, (0, 0, nz - 1 - l2), (nx - 1, ny - 1, nz - 1)),
    ]
    th = dict(pr=pr, t0=T0, glambda=glambda, t_ref=T0, dT=dT,
              wall_T=(0, 0, 0, 0, T0 + dT / 2, T0 - dT / 2))
    return dict(name="rbc", n=n, periodic=(1, 1, 0), walls=(0, 0, 0, 0, 1, 1), inflow_axis=-1, u_in=(0, 0, 0),
                boxes=boxes, solid=None, nu0=nu0, accel0=(0, 0, 0), mirror_lbgk=False, thermal=th, height=H,
                wall_lo=-0.125)


def rbc_small_case(pr: float = 0.7) -> dict:
    return rbc_case(n=(8, 8, 32), l1=8, l2=4, ra=1e5, pr=pr)


def heated_slab_case(n=(4, 4, 16), slab: int = 3, refined: bool = False, pr: float = 0.7, nu0: float = 0.02,
                     dT: float = 0.01) -> dict:
    """Conduction between an isothermal solid slab and a cold plate: walls at
    z, a solid slab filling the first ``slab`` coarse layers at T0 + dT/2 (the
    wall below it is never seen by the fluid and held at T0 - dT), the top
    plate at T0 - dT/2, no buoyancy.  With ``refined`` a level-1 band covers
    the slab and the layers above it, and the slab is given on level 1."""
    nx, ny, nz = n
    boxes = []
    if refined:
        boxes = [(1, (0, 0, 0), (nx - 1, ny - 1, slab + 6))]
        lev, s = 1, 2
    else:
        lev, s = 0, 1
    mask = np.ones((slab * s, ny * s, nx * s), dtype=np.uint8)
    th = dict(pr=pr, t0=T0, glambda=0.0, t_ref=T0, dT=dT,
              wall_T=(0, 0, 0, 0, T0 - dT, T0 - dT / 2), solid_T=T0 + dT / 2)
    # fluid between the slab surface (half a level-lev spacing above its top
    # layer) and the top plate (half a coarse spacing above the last node)
    z_lo = (slab * s - 0.5) / s
    z_hi = nz - 0.5
    return dict(name="slab", n=n, periodic=(1, 1, 0), walls=(0, 0, 0, 0, 1, 1), inflow_axis=-1, u_in=(0, 0, 0),
                boxes=boxes, solid=dict(level=lev, lo=(0, 0, 0), mask=mask), nu0=nu0, accel0=(0, 0, 0),
                mirror_lbgk=False, thermal=th, z_lo=z_lo, z_hi=z_hi)


def heated_slab_profile(case: dict, z):
    """Linear conduction profile of heated_slab_case at coarse height z."""
    th = case["thermal"]
    return th["solid_T"] + (th["wall_T"][5] - th["solid_T"]) * (z - case["z_lo"]) / (case["z_hi"] - case["z_lo"])


def pipe_case(R: float = 10.0, nu: float = 0.1, u_max: float = 0.01, curved: bool = True, nz: int = 4) -> dict:
    """Flow through a circular pipe along z driven by a body force: periodic
    box of 2R + 4 nodes across, solid outside the radius R about the box
    centre (the mask holds the nodes at r >= R; with ``curved`` the cylinder
    itself is the analytic surface of the wall).  The force gives a centreline
    velocity u_max: a = 4 nu u_max / R^2."""
    n = int(2 * R + 4)
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    mask = (((x - c) ** 2 + (y - c) ** 2) >= R * R).astype(np.uint8)
    case = dict(name="pipe", n=(n, n, nz), periodic=(1, 1, 1), walls=(0,) * 6, inflow_axis=-1, u_in=(0, 0, 0),
                boxes=[], solid=dict(level=0, lo=(0, 0, 0), mask=mask), nu0=nu,
                accel0=(0, 0, 4.0 * nu * u_max / (R * R)), mirror_lbgk=False, thermal=None, radius=R, centre=c)
    if curved:
        case["wall_shape"] = dict(kind="cylinder", c=(c, c, 0.0), r=R, axis=2, solid_inside=False)
    return case


def offset_slab_case(z_s: float, n=(4, 4, 16), curved: bool = True, pr: float = 0.7, nu0: float = 0.05,
                     dT: float = 0.01) -> dict:
    """Conduction between an isothermal solid (the nodes below z_s, held at
    T0 + dT/2) and the cold top plate (T0 - dT/2, half a spacing above the last
    node), no buoyancy.  The solid surface is the plane z = z_s, anywhere
    between two node layers; with ``curved`` it is the analytic surface of the
    wall, else the mask's staircase (half a spacing above its top layer)."""
    nx, ny, nz = n
    top = int(math.floor(z_s))
    mask = np.ones((top + 1, ny, nx), dtype=np.uint8)
    th = dict(pr=pr, t0=T0, glambda=0.0, t_ref=T0, dT=dT,
              wall_T=(0, 0, 0, 0, T0 - dT, T0 - dT / 2), solid_T=T0 + dT / 2)
    case = dict(name="offset_slab", n=n, periodic=(1, 1, 0), walls=(0, 0, 0, 0, 1, 1), inflow_axis=-1,
                u_in=(0, 0, 0), boxes=[], solid=dict(level=0, lo=(0, 0, 0), mask=mask), nu0=nu0, accel0=(0, 0, 0),
                mirror_lbgk=False, thermal=th, z_lo=z_s, z_hi=nz - 0.5)
    if curved:
        case["wall_shape"] = dict(kind="plane", c=(0.0, 0.0, z_s), axis=2, solid_inside=True)
    return case


# ---------------------------------------------------------------------------
# initial fields, evaluated at node positions given in coarse units

def node_positions(level: int, org, dim):
    """Coarse-unit positions (x, y, z), each [z][y][x], of a storage box."""
    s = 1.0 / (1 << level)
    z, y, x = np.meshgrid(*[np.arange(org[a], org[a] + dim[a]) for a in (2, 1, 0)], indexing="ij")
    return x * s, y * s, z * s


def tgv_fields(x, y, z, n: int = 32, u0: float = 0.05, pressure: bool = False):
    """2-D Taylor-Green vortex extruded in z (an exact Navier-Stokes solution
    whose amplitude decays as exp(-2 nu k^2 t)).  With ``pressure`` the density
    carries the vortex's pressure field at c_s^2 = 1/3."""
    k = 2.0 * math.pi / n
    ux = u0 * np.sin(k * x) * np.cos(k * y)
    uy = -u0 * np.cos(k * x) * np.sin(k * y)
    uz = np.zeros_like(ux)
    rho = np.ones_like(ux)
    if pressure:
        rho = 1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    return rho, np.stack([ux, uy, uz])


def uniform_fields(x, u=(0.05, 0.02, 0.0), rho: float = 1.0):
    shp = np.shape(x)
    return np.full(shp, rho), np.stack([np.full(shp, float(v)) for v in u])


def _rng(seed: int, level: int, org) -> np.random.Generator:
    """Counter-based (Philox) generator keyed by seed, level and patch origin."""
    key = [int(seed), int(level)] + [int(o) & 0xFFFFFFFF for o in org]
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(key)))


def channel_fields(case: dict, level: int, org, dim, seed: int = 1, u_bulk: float = 0.07, amp: float = 0.05):
    """Laminar parabola with bulk velocity u_bulk plus i.i.d. uniform +-amp
    perturbations of the local velocity on each component (seeded per patch)."""
    x, y, z = node_positions(level, org, dim)
    H = case["height"]
    yw = y - case["wall_lo"]
    prof = 6.0 * u_bulk * yw * (H - yw) / (H * H)
    rng = _rng(seed, level, org)
    pert = rng.uniform(-amp, amp, size=(3,) + prof.shape)
    ux = prof * (1.0 + pert[0])
    uy = prof * pert[1]
    uz = prof * pert[2]
    return np.ones_like(prof), np.stack([ux, uy, uz])


def divfree_modes(n: int = 64, kmax: float = 4.0, rms: float = 0.03, seed: int = 4):
    """Random Fourier modes |k| <= kmax (units of 2 pi / n) with amplitudes
    projected perpendicular to k, scaled to the requested rms velocity."""
    rng = np.random.default_rng(seed)
    ks = []
    r = int(math.floor(kmax))
    for kx in range(-r, r + 1):
        for ky in range(-r, r + 1):
            for kz in range(0, r + 1):
                if kz == 0 and (ky < 0 or (ky == 0 and kx <= 0)):
                    continue  # one of each +-k pair, no k = 0
                if kx * kx + ky * ky + kz * kz <= kmax * kmax:
                    ks.append((kx, ky, kz))
    ks = np.array(ks, dtype=np.float64)
    amp = rng.normal(size=(len(ks), 3)) + 1j * rng.normal(size=(len(ks), 3))
    kh = ks / np.linalg.norm(ks, axis=1, keepdims=True)
    amp -= kh * np.sum(amp * kh, axis=1, keepdims=True)
    # u = sum 2 Re(a e^{ikx}); mean of |u|^2 over the box = sum 2 |a|^2
    ms = 2.0 * np.sum(np.abs(amp) ** 2) / 3.0
    amp *= rms / math.sqrt(ms)
    return dict(n=n, k=ks, a=amp)


def divfree_fields(x, y, z, modes: dict):
    k = 2.0 * math.pi / modes["n"]
    u = np.zeros((3,) + np.shape(x))
    for kv, av in zip(modes["k"], modes["a"]):
        ph = k * (kv[0] * x + kv[1] * y + kv[2] * z)
        c, s = np.cos(ph), np.sin(ph)
        for a in range(3):
            u[a] += 2.0 * (av[a].real * c - av[a].imag * s)
    return np.ones(np.shape(x)), u


def rbc_fields(case: dict, level: int, org, dim, seed: int = 5, amp: float = 0.01):
    """Linear conduction profile between the plates plus i.i.d. uniform
    +-amp relative noise on the temperature deviation scale dT; fluid at rest."""
    x, y, z = node_positions(level, org, dim)
    th = case["thermal"]
    H = case["height"]
    zw = z - case["wall_lo"]
    t_hot, t_cold = th["wall_T"][4], th["wall_T"][5]
    T = t_hot + (t_cold - t_hot) * zw / H
    rng = _rng(seed, level, org)
    T = T + amp * th["dT"] * rng.uniform(-1.0, 1.0, size=T.shape)
    return np.ones_like(T), np.zeros((3,) + T.shape), T
