"""Thin ctypes binding of liblbm.so (the C ABI declared in include/lbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device memory (one uint8 buffer per grid)
and the CUDA stream.  If the library is missing the import fails loudly;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_LAYOUT", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_OOM",
          -5: "LBM_ERR_UNSTABLE", -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_STATE"}
STORAGE = {"fp64": 0, "fp32": 1, "fp16s": 2, "bf16s": 3}


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class lbm_box(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("lo", ctypes.c_int32 * 3), ("hi", ctypes.c_int32 * 3)]


class lbm_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("periodic", ctypes.c_uint32),
        ("walls", ctypes.c_uint32),
        ("inflow_axis", ctypes.c_int32),
        ("u_in", ctypes.c_double * 3),
        ("boxes", ctypes.POINTER(lbm_box)),
        ("n_boxes", ctypes.c_int32),
        ("solid", ctypes.POINTER(ctypes.c_uint8)),
        ("solid_level", ctypes.c_int32),
        ("solid_lo", ctypes.c_int32 * 3),
        ("solid_dims", ctypes.c_int32 * 3),
        ("nu0", ctypes.c_double),
        ("accel0", ctypes.c_double * 3),
        ("model", ctypes.c_int32),
        ("pr", ctypes.c_double),
        ("t0", ctypes.c_double),
        ("glambda", ctypes.c_double),
        ("t_ref", ctypes.c_double),
        ("wall_T", ctypes.c_double * 6),
        ("storage", ctypes.c_int32),
        ("mirror_lbgk", ctypes.c_int32),
        ("solid_T", ctypes.c_double),
        ("solid_isothermal", ctypes.c_int32),
        ("shape_kind", ctypes.c_int32),
        ("shape_c", ctypes.c_double * 3),
        ("shape_r", ctypes.c_double),
        ("shape_axis", ctypes.c_int32),
        ("shape_solid_inside", ctypes.c_int32),
    ]


_lib = None


def lib():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblbm.so not built: run __graft_entry__.build() (no fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        sig = {
            "lbm_grid_create": [ctypes.POINTER(lbm_desc), ctypes.POINTER(vp)],
            "lbm_grid_bytes": [vp, ctypes.POINTER(ctypes.c_size_t)],
            "lbm_grid_bind": [vp, vp, ctypes.c_size_t, vp],
            "lbm_grid_destroy": [vp],
            "lbm_num_patches": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)],
            "lbm_patch_info": [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64),
                               ctypes.POINTER(i64), dp, dp],
            "lbm_patch_mask": [vp, i32, ctypes.POINTER(ctypes.c_uint8)],
            "lbm_node_updates": [vp, dp],
            "lbm_init_equilibrium": [vp, i32, vp, vp, vp, i32],
            "lbm_step": [vp, i64],
            "lbm_moments": [vp, i32, vp, vp, vp, vp, i32],
            "lbm_gamma_blocks": [vp, i32, i32, vp],
            "lbm_transfer": [vp, vp, ctypes.POINTER(i64)],
            "lbm_get_populations": [vp, i32, i32, vp, i32],
            "lbm_set_populations": [vp, i32, i32, vp, i32],
            "lbm_force": [vp, dp, dp],
            "lbm_diagnostics": [vp, dp],
            "lbm_diagnostics_noalloc": [vp, dp],
            "lbm_checkpoint_bytes": [vp, ctypes.POINTER(ctypes.c_size_t)],
            "lbm_checkpoint": [vp, vp, i32],
            "lbm_collide_nodes": [vp, vp, vp, i64, ctypes.c_double, dp, i32, i32, vp],
            "lbm_timing": [vp, i32],
            "lbm_graphs": [vp, i32],
            "lbm_wait_limit": [vp, i32],
            "lbm_autotune": [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float), i32,
                             ctypes.POINTER(ctypes.c_int32)],
            "lbm_set_variant": [vp, i32],
            "lbm_adjoint_workspace_bytes": [vp, i32, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
            "lbm_adjoint_seed": [vp, vp, vp, dp],
            "lbm_adjoint_step": [vp, vp, i32, vp, vp, ctypes.c_size_t],
            "lbm_adjoint_grad_u0": [vp, vp, i32, vp],
            "lbm_timing_report": [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                  ctypes.POINTER(i64), dp, dp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, handle=None) -> None:
    if rc != LBM_OK:
        msg = lib().lbm_last_error(handle)
        raise LbmError(rc, msg.decode() if msg else "")


def make_desc(case: dict, storage: str = "fp32"):
    """lbm_desc from a case dictionary (see paper_1608_06915_gb300.inputs).
    Returns (desc, keepalive) -- keepalive holds the host arrays it points to."""
    d = lbm_desc()
    d.n[:] = [int(v) for v in case["n"]]
    d.periodic = sum((1 << a) for a in range(3) if case.get("periodic", (1, 1, 1))[a])
    d.walls = sum((1 << k) for k, w in enumerate(case.get("walls", (0,) * 6)) if w)
    d.inflow_axis = int(case.get("inflow_axis", -1))
    d.u_in[:] = [float(v) for v in case.get("u_in", (0, 0, 0))]
    boxes = case.get("boxes", [])
    barr = (lbm_box * max(1, len(boxes)))()
    for k, (lev, lo, hi) in enumerate(boxes):
        barr[k].level = int(lev)
        barr[k].lo[:] = [int(v) for v in lo]
        barr[k].hi[:] = [int(v) for v in hi]
    d.boxes = barr
    d.n_boxes = len(boxes)
    keep = [barr]
    solid = case.get("solid")
    if solid is not None:
        m = np.ascontiguousarray(solid["mask"], dtype=np.uint8)
        keep.append(m)
        d.solid = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        d.solid_level = int(solid["level"])
        d.solid_lo[:] = [int(v) for v in solid["lo"]]
        d.solid_dims[:] = [int(m.shape[2]), int(m.shape[1]), int(m.shape[0])]
    else:
        d.solid_level = -1
    d.nu0 = float(case["nu0"])
    d.accel0[:] = [float(v) for v in case.get("accel0", (0, 0, 0))]
    th = case.get("thermal")
    d.model = 1 if th is not None else 0
    d.t0 = 1.0 / 3.0
    if th is not None:
        d.pr, d.t0, d.glambda, d.t_ref = float(th["pr"]), float(th.get("t0", 1 / 3)), float(th["glambda"]), \
            float(th["t_ref"])
        d.wall_T[:] = [float(v) for v in th["wall_T"]]
        if th.get("solid_T") is not None:  # isothermal solid surfaces
            d.solid_T = float(th["solid_T"])
            d.solid_isothermal = 1
    shape = case.get("wall_shape")
    if shape is not None:  # analytic surface of curved solid walls
        d.shape_kind = {"sphere": 1, "cylinder": 2, "plane": 3}[shape["kind"]]
        d.shape_c[:] = [float(v) for v in shape["c"]]
        d.shape_r = float(shape.get("r", 0.0))
        d.shape_axis = int(shape.get("axis", 0))
        d.shape_solid_inside = int(bool(shape.get("solid_inside", True)))
    d.storage = STORAGE[storage]
    d.mirror_lbgk = int(bool(case.get("mirror_lbgk", False)))
    return d, keep


def lbm_grid_create(case: dict, storage: str = "fp32") -> ctypes.c_void_p:
    d, keep = make_desc(case, storage)
    h = ctypes.c_void_p()
    _check(lib().lbm_grid_create(ctypes.byref(d), ctypes.byref(h)))
    return h


class Grid:
    """A refined grid bound to torch-owned device memory on the current stream."""

    def __init__(self, case: dict, storage: str = "fp32", device=None, bind: bool = True):
        self.case = case
        self.storage = storage
        self.handle = lbm_grid_create(case, storage)
        L = lib()
        n, nl = ctypes.c_int32(), ctypes.c_int32()
        L.lbm_num_patches(self.handle, ctypes.byref(n), ctypes.byref(nl))
        self.n_levels = nl.value
        self.patches = []
        for p in range(n.value):
            lev, par = ctypes.c_int32(), ctypes.c_int32()
            org, dim = (ctypes.c_int64 * 3)(), (ctypes.c_int64 * 3)()
            b, b1 = ctypes.c_double(), ctypes.c_double()
            _check(L.lbm_patch_info(self.handle, p, ctypes.byref(lev), ctypes.byref(par), org, dim,
                                    ctypes.byref(b), ctypes.byref(b1)), self.handle)
            self.patches.append(dict(level=lev.value, parent=par.value, org=tuple(org), dim=tuple(dim),
                                     beta=b.value, beta1=b1.value))
        nb = ctypes.c_size_t()
        L.lbm_grid_bytes(self.handle, ctypes.byref(nb))
        self.device_bytes = nb.value
        self.buffer = None
        if bind:
            self.bind(device)

    def bind(self, device=None):
        import torch
        dev = torch.device("cuda") if device is None else torch.device(device)
        self.buffer = torch.empty(self.device_bytes, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev)
        _check(lib().lbm_grid_bind(self.handle, ctypes.c_void_p(self.buffer.data_ptr()), self.device_bytes,
                                   ctypes.c_void_p(self.stream.cuda_stream)), self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.lbm_grid_destroy(h)
            self.handle = None

    # ---- host-side queries
    def shape(self, p: int):
        dx, dy, dz = self.patches[p]["dim"]
        return (dz, dy, dx)

    def gamma_blocks(self, p: int, block: int):
        """Refinement indicator of patch p: the largest |gamma - 2| over the
        fluid nodes of each block^3 block of its storage box, a device float
        tensor [nbz][nby][nbx] (lbm_gamma_blocks)."""
        import torch
        dx, dy, dz = self.patches[p]["dim"]
        nb = [(d + block - 1) // block for d in (dz, dy, dx)]
        out = torch.empty(nb, dtype=torch.float32, device=self.buffer.device)
        _check(lib().lbm_gamma_blocks(self.handle, int(p), int(block), self._ptr(out)), self.handle)
        return out

    def transfer_from(self, src: "Grid") -> int:
        """Take the state of another grid of the same domain onto this layout
        (lbm_transfer); returns the number of fluid nodes no source level holds."""
        n = ctypes.c_int64()
        _check(lib().lbm_transfer(self.handle, src.handle, ctypes.byref(n)), self.handle)
        return n.value

    def mask(self, p: int) -> np.ndarray:
        out = np.empty(self.shape(p), dtype=np.uint8)
        _check(lib().lbm_patch_mask(self.handle, p, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
               self.handle)
        return out

    def node_updates(self) -> float:
        v = ctypes.c_double()
        _check(lib().lbm_node_updates(self.handle, ctypes.byref(v)), self.handle)
        return v.value

    # ---- device calls
    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else None

    def _need(self, t, shape, what):
        if t is None:
            return
        if tuple(t.shape) != tuple(shape) or not t.is_cuda:
            raise ValueError("%s: expected a CUDA tensor of shape %s, got %s" % (what, shape, tuple(t.shape)))

    def init_equilibrium(self, p: int, rho, u, T=None):
        import torch
        shp = self.shape(p)
        self._need(rho, shp, "rho")
        self._need(u, (3,) + shp, "u")
        self._need(T, shp, "T")
        dt = torch.float64 if rho.dtype == torch.float64 else torch.float32
        rho = rho.to(dtype=dt).contiguous()
        u = u.to(dtype=dt).contiguous()
        T = None if T is None else T.to(dtype=dt).contiguous()
        self._keep = (rho, u, T)
        _check(lib().lbm_init_equilibrium(self.handle, p, self._ptr(rho), self._ptr(u), self._ptr(T),
                                          1 if dt == torch.float64 else 0), self.handle)

    def step(self, n: int = 1):
        _check(lib().lbm_step(self.handle, int(n)), self.handle)

    def moments(self, p: int, dtype=None, gamma: bool = False):
        import torch
        dtype = dtype or torch.float64
        shp = self.shape(p)
        dev = self.buffer.device
        rho = torch.empty(shp, dtype=dtype, device=dev)
        u = torch.empty((3,) + shp, dtype=dtype, device=dev)
        T = torch.empty(shp, dtype=dtype, device=dev)
        g = torch.empty(shp, dtype=dtype, device=dev) if gamma else None
        _check(lib().lbm_moments(self.handle, p, self._ptr(rho), self._ptr(u), self._ptr(T), self._ptr(g),
                                 1 if dtype == torch.float64 else 0), self.handle)
        return rho, u, T, g

    def get_populations(self, p: int, which: int = 0, dtype=None):
        import torch
        dtype = dtype or torch.float64
        out = torch.empty((27,) + self.shape(p), dtype=dtype, device=self.buffer.device)
        _check(lib().lbm_get_populations(self.handle, p, which, self._ptr(out), 1 if dtype == torch.float64 else 0),
               self.handle)
        return out

    def set_populations(self, p: int, src, which: int = 0):
        import torch
        self._need(src, (27,) + self.shape(p), "populations")
        if src.dtype not in (torch.float32, torch.float64):
            raise ValueError("populations must be float32 or float64")
        src = src.contiguous()
        _check(lib().lbm_set_populations(self.handle, p, which, self._ptr(src),
                                         1 if src.dtype == torch.float64 else 0), self.handle)
        self._keep = src

    def diagnostics(self):
        out = (ctypes.c_double * 8)()
        rc = lib().lbm_diagnostics(self.handle, out)
        vals = list(out)
        if rc != LBM_OK:
            raise LbmError(rc, lib().lbm_last_error(self.handle).decode())
        return dict(mass=vals[0], momentum=vals[1:4], kinetic_energy=vals[4], fluid_nodes=vals[5],
                    min_rho=vals[6], status=int(vals[7]))

    def diagnostics_noalloc(self):
        """lbm_diagnostics_noalloc: the same sums without the grid's workspace."""
        out = (ctypes.c_double * 8)()
        rc = lib().lbm_diagnostics_noalloc(self.handle, out)
        vals = list(out)
        if rc != LBM_OK:
            raise LbmError(rc, lib().lbm_last_error(self.handle).decode())
        return dict(mass=vals[0], momentum=vals[1:4], kinetic_energy=vals[4], fluid_nodes=vals[5],
                    min_rho=vals[6], status=int(vals[7]))

    def set_force(self, accel0):
        a = (ctypes.c_double * 3)(*[float(v) for v in accel0])
        _check(lib().lbm_force(self.handle, a, None), self.handle)

    def drag(self):
        """FP64 momentum-exchange force on the solid nodes of the current state
        (coarse units, summed over levels); synchronises the stream."""
        out = (ctypes.c_double * 3)()
        _check(lib().lbm_force(self.handle, None, out), self.handle)
        return [out[0], out[1], out[2]]

    def autotune(self, trials: int = 2):
        """Times each variant (TMA kernel x schedule of the reconstruction
        samples) over `trials` coarse steps as step() runs them, then the two
        fastest over 3 * trials steps, and keeps the faster of those:
        dict(chosen, ms_per_step).  The state advances by
        1 + variants * (2 + trials) + 2 * (2 + 3 * trials) coarse steps."""
        chosen, n = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * 16)()
        _check(lib().lbm_autotune(self.handle, int(trials), ctypes.byref(chosen), ms, 16, ctypes.byref(n)),
               self.handle)
        return dict(chosen=chosen.value, ms_per_step=[ms[i] for i in range(n.value)])

    def set_variant(self, v: int):
        _check(lib().lbm_set_variant(self.handle, int(v)), self.handle)

    def graphs(self, enable: bool):
        _check(lib().lbm_graphs(self.handle, 1 if enable else 0), self.handle)

    def wait_limit(self, sleeps: int):
        """lbm_wait_limit: bound of the TMA passes' stage waits (0.5 us units)."""
        _check(lib().lbm_wait_limit(self.handle, int(sleeps)), self.handle)

    def timing(self, enable: bool):
        _check(lib().lbm_timing(self.handle, 1 if enable else 0), self.handle)

    def timing_report(self):
        """Per kernel class: dict(kind, level, launches, ms, nodes)."""
        m = 64
        n = ctypes.c_int32()
        kind, lev = (ctypes.c_int32 * m)(), (ctypes.c_int32 * m)()
        cnt, ms, nodes = (ctypes.c_int64 * m)(), (ctypes.c_double * m)(), (ctypes.c_double * m)()
        _check(lib().lbm_timing_report(self.handle, m, ctypes.byref(n), kind, lev, cnt, ms, nodes), self.handle)
        names = {0: "stream_collide", 1: "coalesce", 2: "samples", 3: "explode", 4: "stream_collide_tma"}
        return [dict(kind=names[kind[k]], level=lev[k], launches=cnt[k], ms=ms[k], nodes=nodes[k])
                for k in range(min(n.value, m))]

    # ---- discrete adjoint
    def adjoint_buffers(self, K: int):
        """(lambda, workspace) device buffers for segments of K coarse steps."""
        import torch
        lb, wb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().lbm_adjoint_workspace_bytes(self.handle, int(K), ctypes.byref(lb), ctypes.byref(wb)),
               self.handle)
        dev = self.buffer.device
        return (torch.empty(lb.value, dtype=torch.uint8, device=dev),
                torch.empty(wb.value, dtype=torch.uint8, device=dev))

    def adjoint_seed(self, lam, ws) -> float:
        ke = ctypes.c_double()
        _check(lib().lbm_adjoint_seed(self.handle, self._ptr(lam), self._ptr(ws), ctypes.byref(ke)), self.handle)
        return ke.value

    def adjoint_step(self, ckpt, K: int, lam, ws):
        _check(lib().lbm_adjoint_step(self.handle, self._ptr(ckpt), int(K), self._ptr(lam), self._ptr(ws),
                                      ws.numel()), self.handle)

    def adjoint_grad_u0(self, lam, p: int):
        import torch
        out = torch.empty((3,) + self.shape(p), dtype=torch.float64, device=self.buffer.device)
        _check(lib().lbm_adjoint_grad_u0(self.handle, self._ptr(lam), int(p), self._ptr(out)), self.handle)
        return out

    def checkpoint_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().lbm_checkpoint_bytes(self.handle, ctypes.byref(n)), self.handle)
        return n.value

    def checkpoint(self, buf, save: bool):
        _check(lib().lbm_checkpoint(self.handle, self._ptr(buf), 1 if save else 0), self.handle)


def lbm_collide_nodes(f_in, beta: float, du=(0.0, 0.0, 0.0), lbgk: bool = False):
    """One KBC collision of n independent nodes, f_in a CUDA tensor [27, n]."""
    import torch
    f_in = f_in.contiguous()
    n = f_in.shape[1]
    f_out = torch.empty_like(f_in)
    gam = torch.empty(n, dtype=f_in.dtype, device=f_in.device)
    d = (ctypes.c_double * 3)(*[float(v) for v in du])
    rc = lib().lbm_collide_nodes(ctypes.c_void_p(f_in.data_ptr()), ctypes.c_void_p(f_out.data_ptr()),
                                 ctypes.c_void_p(gam.data_ptr()), n, float(beta), d, int(lbgk),
                                 1 if f_in.dtype == torch.float64 else 0,
                                 ctypes.c_void_p(torch.cuda.current_stream(f_in.device).cuda_stream))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_collide_nodes")
    return f_out, gam


def kinetic_energy_run(grid: "Grid", u0, n_steps: int, K: int):
    """J = kinetic energy after n_steps coarse steps from f = f^eq(1, u0), as a
    differentiable function of the initial velocity fields u0 (one CUDA
    tensor [3][z][y][x] per patch).  The backward pass runs the library's
    discrete adjoint with a checkpoint every K coarse steps."""
    import torch

    class _Run(torch.autograd.Function):
        @staticmethod
        def forward(ctx, *u0s):
            dev = grid.buffer.device
            for p, u in enumerate(u0s):
                grid.init_equilibrium(p, torch.ones(grid.shape(p), dtype=torch.float64, device=dev),
                                      u.detach().to(torch.float64))
            nb = grid.checkpoint_bytes()
            ckpts = []
            done = 0
            while done < n_steps:
                ck = torch.empty(nb, dtype=torch.uint8, device=dev)
                grid.checkpoint(ck, save=True)
                k = min(K, n_steps - done)
                ckpts.append((ck, k))
                grid.step(k)
                done += k
            lam, ws = grid.adjoint_buffers(K)
            ke = grid.adjoint_seed(lam, ws)
            ctx.ckpts, ctx.lam, ctx.ws = ckpts, lam, ws
            return torch.tensor(ke, dtype=torch.float64, device=dev)

        @staticmethod
        def backward(ctx, gJ):
            lam, ws = ctx.lam, ctx.ws
            for ck, k in reversed(ctx.ckpts):
                grid.adjoint_step(ck, k, lam, ws)
            scale = gJ.to(torch.float64)
            return tuple(grid.adjoint_grad_u0(lam, p) * scale for p in range(len(grid.patches)))

    return _Run.apply(*u0)
