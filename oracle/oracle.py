"""ctypes wrapper around the FP64 oracle in ``oracle.cpp``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never does.  It
imports nothing from the product package.  Cases are plain dictionaries
(see ``paper_1608_06915_gb300.inputs`` for the ones the tests use).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 27


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrcBox(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("lo", ctypes.c_int32 * 3), ("hi", ctypes.c_int32 * 3)]


class OrcDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("periodic", ctypes.c_uint32),
        ("walls", ctypes.c_uint32),
        ("inflow_axis", ctypes.c_int32),
        ("u_in", ctypes.c_double * 3),
        ("boxes", ctypes.POINTER(OrcBox)),
        ("n_boxes", ctypes.c_int32),
        ("solid", ctypes.POINTER(ctypes.c_uint8)),
        ("solid_level", ctypes.c_int32),
        ("solid_lo", ctypes.c_int32 * 3),
        ("solid_dims", ctypes.c_int32 * 3),
        ("nu0", ctypes.c_double),
        ("accel0", ctypes.c_double * 3),
        ("mirror_lbgk", ctypes.c_int32),
        ("thermal", ctypes.c_int32),
        ("pr", ctypes.c_double),
        ("t0", ctypes.c_double),
        ("glambda", ctypes.c_double),
        ("t_ref", ctypes.c_double),
        ("wall_T", ctypes.c_double * 6),
        ("solid_T", ctypes.c_double),
        ("solid_isothermal", ctypes.c_int32),
        ("shape_kind", ctypes.c_int32),
        ("shape_c", ctypes.c_double * 3),
        ("shape_r", ctypes.c_double),
        ("shape_axis", ctypes.c_int32),
        ("shape_solid_inside", ctypes.c_int32),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(OrcDesc)]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_last_error.restype = ctypes.c_char_p
            L.orc_num_patches.argtypes = [ctypes.c_void_p]
            L.orc_patch_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64), dp, dp]
            L.orc_patch_mask.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)]
            L.orc_init_equilibrium.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, dp, dp, dp]
            L.orc_get_pop.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            L.orc_set_pop.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_moments.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, dp, dp]
            L.orc_node_updates_per_step.restype = ctypes.c_double
            L.orc_node_updates_per_step.argtypes = [ctypes.c_void_p]
            L.orc_drag.argtypes = [ctypes.c_void_p, dp]
            L.orc_feq.argtypes = [ctypes.c_double, dp, dp]
            L.orc_split.argtypes = [dp, dp, dp, dp]
            L.orc_collide.restype = ctypes.c_double
            L.orc_collide.argtypes = [dp, ctypes.c_double, dp, ctypes.c_int, ctypes.c_double, dp]
            L.orc_geq.argtypes = [ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp]
            L.orc_thermal_collide.restype = ctypes.c_double
            L.orc_thermal_collide.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
            L.orc_lagrange_weights.argtypes = [dp]
            L.orc_rescale.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_transfer.restype = ctypes.c_long
            L.orc_transfer.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- single-node functions -------------------------------------------------

def feq(rho: float, u) -> np.ndarray:
    out = np.empty(Q)
    lib().orc_feq(float(rho), _dp(_f64(u)), _dp(out))
    return out


def split(f) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    f = _f64(f)
    k, s, h = np.empty(Q), np.empty(Q), np.empty(Q)
    lib().orc_split(_dp(f), _dp(k), _dp(s), _dp(h))
    return k, s, h


def collide(f, beta: float, du=(0.0, 0.0, 0.0), lbgk: bool = False, gamma=None) -> tuple[np.ndarray, float]:
    f = _f64(f)
    out = np.empty(Q)
    g = lib().orc_collide(_dp(f), float(beta), _dp(_f64(du)), int(lbgk),
                          float("nan") if gamma is None else float(gamma), _dp(out))
    return out, g


def geq(rho: float, u, T: float, t0: float = 1.0 / 3.0) -> np.ndarray:
    out = np.empty(Q)
    lib().orc_geq(float(rho), _dp(_f64(u)), float(T), float(t0), _dp(out))
    return out


def thermal_collide(f, g, beta, beta1, t0=1.0 / 3.0, glambda=0.0, t_ref=0.0, pr_gt1=False):
    """One thermal collision of (f, g); pr_gt1 selects the Pr > 1 row of Table I."""
    fo, go = np.empty(Q), np.empty(Q)
    gm = lib().orc_thermal_collide(_dp(_f64(f)), _dp(_f64(g)), float(beta), float(beta1), float(t0),
                                   float(glambda), float(t_ref), 1 if pr_gt1 else 0, _dp(fo), _dp(go))
    return fo, go, gm


def rescale(f, g, beta_s, beta_t, beta1_s=1.0, beta1_t=1.0, r=2.0, thermal=False, pr_gt1=False,
            t0=1.0 / 3.0):
    """Interface rescaling of one node's populations from a level with
    (beta_s, beta1_s) to one with (beta_t, beta1_t), r = dx_s / dx_t
    (Sec. III.A).  Returns (f, g); g is None for the isothermal model."""
    fo, go = np.empty(Q), np.empty(Q)
    gin = _f64(g) if g is not None else np.zeros(Q)
    lib().orc_rescale(_dp(_f64(f)), _dp(gin), float(beta_s), float(beta_t), float(beta1_s), float(beta1_t),
                      float(r), int(bool(thermal)), int(bool(pr_gt1)), float(t0), _dp(fo), _dp(go))
    return fo, (go if thermal else None)


def lagrange_weights() -> np.ndarray:
    w = np.empty(4)
    lib().orc_lagrange_weights(_dp(w))
    return w


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---- whole simulations -----------------------------------------------------

def _walls_bits(walls) -> int:
    bits = 0
    for k, w in enumerate(walls):
        if w:
            bits |= 1 << k
    return bits


class Oracle:
    """An FP64 multi-level simulation described by a case dictionary.

    Keys: ``n`` (coarse extents), ``periodic`` (3 flags), ``walls`` (6 flags:
    -x,+x,-y,+y,-z,+z), ``inflow_axis``, ``u_in``, ``boxes`` (list of
    ``(level, lo, hi)`` in coarse units), ``solid`` (None or dict with
    ``level``, ``lo`` and a uint8 ``mask`` indexed [z][y][x]), ``nu0``,
    ``accel0``, ``mirror_lbgk``, ``thermal`` (None or dict with ``pr``,
    ``t0``, ``glambda``, ``t_ref``, ``wall_T`` and, for isothermal solid
    surfaces, ``solid_T``) and ``wall_shape`` (None or dict with ``kind``
    sphere / cylinder / plane, ``c``, ``r``, ``axis``, ``solid_inside``: the
    analytic solid surface of curved walls, coarse units).
    """

    def __init__(self, case: dict):
        L = lib()
        d = OrcDesc()
        d.n[:] = [int(v) for v in case["n"]]
        d.periodic = sum((1 << a) for a in range(3) if case.get("periodic", (1, 1, 1))[a])
        d.walls = _walls_bits(case.get("walls", (0,) * 6))
        d.inflow_axis = int(case.get("inflow_axis", -1))
        d.u_in[:] = [float(v) for v in case.get("u_in", (0, 0, 0))]
        boxes = case.get("boxes", [])
        self._boxes = (OrcBox * max(1, len(boxes)))()
        for k, (lev, lo, hi) in enumerate(boxes):
            self._boxes[k].level = int(lev)
            self._boxes[k].lo[:] = [int(v) for v in lo]
            self._boxes[k].hi[:] = [int(v) for v in hi]
        d.boxes = self._boxes
        d.n_boxes = len(boxes)
        solid = case.get("solid")
        self._solid = None
        if solid is not None:
            self._solid = np.ascontiguousarray(solid["mask"], dtype=np.uint8)
            d.solid = self._solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
            d.solid_level = int(solid["level"])
            d.solid_lo[:] = [int(v) for v in solid["lo"]]
            d.solid_dims[:] = [int(self._solid.shape[2]), int(self._solid.shape[1]), int(self._solid.shape[0])]
        else:
            d.solid_level = -1
        shape = case.get("wall_shape")
        if shape is not None:  # curved solid surface (reading R10)
            d.shape_kind = {"sphere": 1, "cylinder": 2, "plane": 3}[shape["kind"]]
            d.shape_c[:] = [float(v) for v in shape["c"]]
            d.shape_r = float(shape.get("r", 0.0))
            d.shape_axis = int(shape.get("axis", 0))
            d.shape_solid_inside = int(bool(shape.get("solid_inside", True)))
        d.nu0 = float(case["nu0"])
        d.accel0[:] = [float(v) for v in case.get("accel0", (0, 0, 0))]
        d.mirror_lbgk = int(bool(case.get("mirror_lbgk", False)))
        th = case.get("thermal")
        if th is not None:
            d.thermal = 1
            d.pr = float(th["pr"])
            d.t0 = float(th.get("t0", 1.0 / 3.0))
            d.glambda = float(th["glambda"])
            d.t_ref = float(th["t_ref"])
            d.wall_T[:] = [float(v) for v in th["wall_T"]]
            if th.get("solid_T") is not None:  # isothermal solid surfaces
                d.solid_T = float(th["solid_T"])
                d.solid_isothermal = 1
        else:
            d.t0 = 1.0 / 3.0
        self.thermal = th is not None
        h = L.orc_create(ctypes.byref(d))
        if not h:
            raise ValueError("oracle rejected the case: " + L.orc_last_error().decode())
        self._h = ctypes.c_void_p(h)
        self.patches = []
        for p in range(L.orc_num_patches(self._h)):
            lev, par = ctypes.c_int32(), ctypes.c_int32()
            org, dim = (ctypes.c_int64 * 3)(), (ctypes.c_int64 * 3)()
            b, b1 = ctypes.c_double(), ctypes.c_double()
            L.orc_patch_info(self._h, p, ctypes.byref(lev), ctypes.byref(par), org, dim, ctypes.byref(b),
                             ctypes.byref(b1))
            self.patches.append(dict(level=lev.value, parent=par.value, org=tuple(org), dim=tuple(dim),
                                     beta=b.value, beta1=b1.value))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def shape(self, p: int) -> tuple[int, int, int]:
        dx, dy, dz = self.patches[p]["dim"]
        return (dz, dy, dx)

    def coords(self, p: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Node positions of patch p in coarse units, each shaped [z][y][x]."""
        info = self.patches[p]
        s = 1.0 / (1 << info["level"])
        ox, oy, oz = info["org"]
        dx, dy, dz = info["dim"]
        z, y, x = np.meshgrid(np.arange(oz, oz + dz), np.arange(oy, oy + dy), np.arange(ox, ox + dx), indexing="ij")
        return x * s, y * s, z * s

    def mask(self, p: int) -> np.ndarray:
        out = np.empty(self.shape(p), dtype=np.uint8)
        lib().orc_patch_mask(self._h, p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return out

    def init_equilibrium(self, p: int, rho, u, T=None) -> None:
        shp = self.shape(p)
        rho = _f64(np.broadcast_to(rho, shp))
        u = [_f64(np.broadcast_to(u[a], shp)) for a in range(3)]
        Tp = None if T is None else _f64(np.broadcast_to(T, shp))
        rc = lib().orc_init_equilibrium(self._h, p, _dp(rho), _dp(u[0]), _dp(u[1]), _dp(u[2]),
                                        None if Tp is None else _dp(Tp))
        if rc:
            raise RuntimeError("orc_init_equilibrium failed")

    def get_pop(self, p: int, which: int = 0) -> np.ndarray:
        out = np.empty((Q,) + self.shape(p))
        if lib().orc_get_pop(self._h, p, which, _dp(out)):
            raise RuntimeError("orc_get_pop failed")
        return out

    def set_pop(self, p: int, arr, which: int = 0) -> None:
        a = _f64(arr)
        if lib().orc_set_pop(self._h, p, which, _dp(a)):
            raise RuntimeError("orc_set_pop failed")

    def transfer_from(self, src: "Oracle") -> int:
        """Take the state of another oracle of the same domain onto this
        layout (reading R9); returns the number of fluid nodes no source
        level holds."""
        n = lib().orc_transfer(self._h, src._h)
        if n < 0:
            raise ValueError("oracle transfer between incompatible grids")
        return int(n)

    def step(self, n: int = 1) -> None:
        if lib().orc_step(self._h, int(n)):
            raise RuntimeError("oracle step failed: " + lib().orc_last_error().decode())

    def moments(self, p: int):
        shp = self.shape(p)
        rho, T, gam = np.empty(shp), np.empty(shp), np.empty(shp)
        u = np.empty((3,) + shp)
        lib().orc_moments(self._h, p, _dp(rho), _dp(u), _dp(T), _dp(gam))
        return rho, u, T, gam

    def node_updates_per_step(self) -> float:
        return float(lib().orc_node_updates_per_step(self._h))

    def drag(self) -> np.ndarray:
        """Momentum-exchange force on the solid nodes of the current state (coarse units)."""
        F = np.zeros(3)
        lib().orc_drag(self._h, _dp(F))
        return F
