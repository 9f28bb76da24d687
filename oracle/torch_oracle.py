"""FP64 reference gradient for the discrete adjoint (test infrastructure only).

A plain PyTorch (CPU, float64) restatement of the refined KBC step for the
case the adjoint targets -- a periodic box with one level-1 box -- written
node-set by node-set from the paper, so that torch.autograd gives the exact
gradient of the kinetic-energy objective with respect to the initial velocity.
Its forward is pinned to the C oracle (``tests/test_adjoint.py``); it imports
nothing from the product package.

Follows, in order: equilibrium Eq. (feq_iso); KBC split and mirror with the
stabiliser Eqs. (popSplit), (f_mirr), (gamma_min_approx); the five steps of
Sec. III.C with r = 2: fine stream + collide on depth >= 1, stream both
levels, twin rescaling Eq. (f_neq_rescaling_iso) both ways, four-point
reconstruction Eq. (interp) of rho, u and the non-equilibrium part, collide all.
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64
C_NP = np.array([[(i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], dtype=np.int64)
C = torch.tensor(C_NP, dtype=DT)
_W1 = {0: 2.0 / 3.0, -1: 1.0 / 6.0, 1: 1.0 / 6.0}
W = torch.tensor([_W1[a] * _W1[b] * _W1[c] for a, b, c in C_NP], dtype=DT)


def feq(rho: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """rho [N], u [N,3] -> [N,27], Eq. (feq_iso)."""
    s = torch.sqrt(1.0 + 3.0 * u * u)
    base = (2.0 * u + s) / (1.0 - u)
    out = rho[:, None] * W[None, :]
    for a in range(3):
        c = C[:, a]
        fac = (2.0 - s[:, a])[:, None] * torch.where(c[None, :] > 0, base[:, a:a + 1],
                                                       torch.where(c[None, :] < 0, 1.0 / base[:, a:a + 1],
                                                                   torch.ones_like(base[:, a:a + 1])))
        out = out * fac
    return out


def macro(f: torch.Tensor):
    rho = f.sum(1)
    u = (f @ C) / rho[:, None]
    return rho, u


# natural-moment map (Eq. moments) and its tensor-product inverse
def _moment_matrix():
    M = np.zeros((27, 27))
    for p in range(3):
        for q in range(3):
            for r in range(3):
                M[p + 3 * q + 9 * r] = C_NP[:, 0] ** p * C_NP[:, 1] ** q * C_NP[:, 2] ** r
    return M


_M = torch.tensor(_moment_matrix(), dtype=DT)
_MI = torch.linalg.inv(_M)


def split(f: torch.Tensor):
    """k, s, h of Eq. (popSplit): conserved moments, deviatoric stress, rest."""
    m = f @ _M.T
    mk = torch.zeros_like(m)
    ms = torch.zeros_like(m)
    for j in (0, 1, 3, 9):
        mk[:, j] = m[:, j]
    tr = m[:, 2] + m[:, 6] + m[:, 18]
    for j in (2, 6, 18):
        ms[:, j] = m[:, j] - tr / 3.0
    for j in (4, 10, 12):
        ms[:, j] = m[:, j]
    k = mk @ _MI.T
    s = ms @ _MI.T
    return k, s, f - k - s


def collide(f: torch.Tensor, beta: float, lbgk: bool = False) -> torch.Tensor:
    rho, u = macro(f)
    fe = feq(rho, u)
    if lbgk:
        fm = 2.0 * fe - f
    else:
        k, s, h = split(f)
        ke, se, he = split(fe)
        ds, dh = s - se, h - he
        sh = (ds * dh / fe).sum(1)
        hh = (dh * dh / fe).sum(1)
        guard = hh > 1e-30 * rho * rho
        gamma = torch.where(guard, 1.0 / beta - (2.0 - 1.0 / beta) * sh / torch.where(guard, hh, torch.ones_like(hh)),
                            torch.full_like(hh, 2.0))
        fm = k + (2.0 * se - s) + ((1.0 - gamma)[:, None] * h + gamma[:, None] * he)
    return (1.0 - beta) * f + beta * fm


class TwoLevel:
    """Periodic n^3 coarse box with the level-1 box [a, b]^3 (coarse units)."""

    def __init__(self, n: int, a: int, b: int, nu0: float, lbgk: bool = False):
        self.n, self.a, self.b, self.lbgk = n, a, b, lbgk
        self.beta_c = 1.0 / (6.0 * nu0 + 1.0)
        self.beta_f = 1.0 / (1.0 + 2.0 * (1.0 / self.beta_c - 1.0))
        # coarse nodes (all n^3 stored, x fastest); hole and twins (Sec. III layout)
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        self.cX = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
        inside = lambda P, lo, hi: np.all((P >= lo) & (P <= hi), axis=1)
        self.c_hole = inside(self.cX, a + 2, b - 2)
        self.c_twin = inside(self.cX, a + 1, b - 1) & ~self.c_hole
        self.c_exist = ~self.c_hole
        # fine nodes: (2(b-a)+1)^3 at fine coordinates 2a..2b
        m = 2 * (b - a) + 1
        self.m = m
        z, y, x = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
        self.fY = np.stack([x.ravel(), y.ravel(), z.ravel()], 1) + 2 * a
        self.depth = np.min(np.minimum(self.fY - 2 * a, 2 * b - self.fY), axis=1)
        # stream sources (pull: x - c_i)
        cidx = lambda P: (P[..., 2] * n + P[..., 1]) * n + P[..., 0]
        src = (self.cX[:, None, :] - C_NP[None, :, :]) % n
        self.c_src = torch.tensor(cidx(src), dtype=torch.long)
        fs = self.fY[:, None, :] - C_NP[None, :, :] - 2 * a
        self.f_src_ok = np.all((fs >= 0) & (fs < m), axis=2)
        fsc = np.clip(fs, 0, m - 1)
        self.f_src = torch.tensor((fsc[..., 2] * m + fsc[..., 1]) * m + fsc[..., 0], dtype=torch.long)
        self.fidx = lambda Y: ((Y[..., 2] - 2 * a) * m + (Y[..., 1] - 2 * a)) * m + (Y[..., 0] - 2 * a)
        self.cidx = cidx
        self.sel = lambda mask: torch.tensor(np.nonzero(mask)[0], dtype=torch.long)
        # reconstruction tables: per interface node, samples (coarse or fine source, weight)
        w4 = np.array([-1.0, 9.0, 9.0, -1.0]) / 16.0
        tgt, srcs, kinds, wts = [], [], [], []
        twin_t, twin_s = [], []
        for j in np.nonzero(self.depth <= 1)[0]:
            Y = self.fY[j]
            odd = Y % 2 == 1
            if not odd.any():
                twin_t.append(j)
                twin_s.append(cidx(Y // 2))
                continue
            axes = []
            for ax in range(3):
                if odd[ax]:
                    axes.append([((Y[ax] - 3 + 2 * k) // 2, w4[k]) for k in range(4)])
                else:
                    axes.append([(Y[ax] // 2, 1.0)])
            for px, wx in axes[0]:
                for py, wy in axes[1]:
                    for pz, wz in axes[2]:
                        P = np.array([px, py, pz])
                        tgt.append(j)
                        wts.append(wx * wy * wz)
                        if inside(P[None], a + 2, b - 2)[0]:
                            # inside the coarse hole: the fine node at 2P
                            kinds.append(1)
                            srcs.append(self.fidx(2 * P))
                        else:
                            kinds.append(0)
                            srcs.append(cidx(P % n))
        self.twin_t = torch.tensor(twin_t, dtype=torch.long)
        self.twin_s = torch.tensor(twin_s, dtype=torch.long)
        self.rec_t = torch.tensor(tgt, dtype=torch.long)
        self.rec_s = torch.tensor(srcs, dtype=torch.long)
        self.rec_k = torch.tensor(kinds, dtype=torch.long)
        self.rec_w = torch.tensor(wts, dtype=DT)
        self.rec_nodes = torch.tensor(sorted(set(tgt)), dtype=torch.long)
        self.cf_c = self.sel(self.c_twin)
        self.cf_f = torch.tensor(self.fidx(2 * self.cX[self.c_twin]), dtype=torch.long)

    # ---- steps
    def stream_fine(self, post, nodes):
        ii = torch.arange(27)
        return post[self.f_src[nodes][:, ii], ii[None, :].expand(len(nodes), 27)]

    def stream_coarse(self, post, nodes):
        ii = torch.arange(27)
        return post[self.c_src[nodes][:, ii], ii[None, :].expand(len(nodes), 27)]

    def rescale(self, f, factor):
        rho, u = macro(f)
        fe = feq(rho, u)
        return fe + factor * (f - fe)

    def step(self, fc, ff):
        """One coarse step: fc [n^3,27], ff [m^3,27] post-collision -> post-collision."""
        bc, bf = self.beta_c, self.beta_f
        d1 = self.sel(self.depth >= 1)
        d2 = self.sel(self.depth >= 2)
        # 1. fine stream + collide on depth >= 1
        ff1 = ff.index_put((d1,), collide(self.stream_fine(ff, d1), bf, self.lbgk))
        # 2. stream both levels
        pre_f = ff1.index_put((d2,), self.stream_fine(ff1, d2))
        cvalid = self.sel(self.c_exist & ~self.c_twin)
        pre_c = fc.index_put((cvalid,), self.stream_coarse(fc, cvalid))
        # 3. twins: coarse <- fine (factor r beta_f / beta_c), fine <- coarse (inverse)
        pre_c = pre_c.index_put((self.cf_c,), self.rescale(pre_f[self.cf_f], 2.0 * bf / bc))
        pre_f = pre_f.index_put((self.twin_t,), self.rescale(pre_c[self.twin_s], bc / (2.0 * bf)))
        # 4. reconstruction: rho, u and fine-scale non-equilibrium interpolated
        cf_vals = pre_c[self.rec_s.clamp(max=pre_c.shape[0] - 1)]
        ff_vals = pre_f[self.rec_s.clamp(max=pre_f.shape[0] - 1)]
        sv = torch.where((self.rec_k == 0)[:, None], cf_vals, ff_vals)
        rho, u = macro(sv)
        factor = torch.where(self.rec_k == 0, torch.full_like(rho, bc / (2.0 * bf)), torch.ones_like(rho))
        neq = factor[:, None] * (sv - feq(rho, u))
        nrec = pre_f.shape[0]
        acc_r = torch.zeros(nrec, dtype=DT).index_add(0, self.rec_t, self.rec_w * rho)
        acc_u = torch.zeros(nrec, 3, dtype=DT).index_add(0, self.rec_t, self.rec_w[:, None] * u)
        acc_n = torch.zeros(nrec, 27, dtype=DT).index_add(0, self.rec_t, self.rec_w[:, None] * neq)
        r = self.rec_nodes
        pre_f = pre_f.index_put((r,), feq(acc_r[r], acc_u[r]) + acc_n[r])
        # 5. collide all
        call = self.sel(self.c_exist)
        fc2 = fc.index_put((call,), collide(pre_c[call], bc, self.lbgk))
        ff2 = collide(pre_f, bf, self.lbgk)
        return fc2, ff2

    def kinetic_energy(self, fc, ff):
        """1/2 sum rho |u|^2 8^-level; the coarse level owns nodes outside [a+1, b-1]^3,
        the fine level its nodes of depth >= 2."""
        own_c = self.sel(self.c_exist & ~self.c_twin)
        own_f = self.sel(self.depth >= 2)
        rc, uc = macro(fc[own_c])
        rf, uf = macro(ff[own_f])
        return 0.5 * (rc * (uc * uc).sum(1)).sum() + 0.125 * 0.5 * (rf * (uf * uf).sum(1)).sum()

    def run(self, uc, uf, steps):
        """uc [n^3,3], uf [m^3,3] initial velocities -> kinetic energy after `steps`."""
        fc = feq(torch.ones(uc.shape[0], dtype=DT), uc)
        ff = feq(torch.ones(uf.shape[0], dtype=DT), uf)
        for _ in range(steps):
            fc, ff = self.step(fc, ff)
        return self.kinetic_energy(fc, ff), fc, ff
