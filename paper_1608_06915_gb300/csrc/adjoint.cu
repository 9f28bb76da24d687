// Discrete adjoint of the refined isothermal KBC step (periodic layouts
// without walls, solids, inflow or body force).
//
// Every forward kernel maps the previous states (pulled) to the nodes it
// writes; its adjoint takes the adjoint of those nodes (lambda_new), recomputes
// the forward pre-collision state from the restored previous state, applies
// the transposed Jacobian of the node map and sends the result back along the
// pull (a push to lambda_old[x - c_i][i]).  Each entry of lambda_old has one
// puller, so it takes one store from the stream-collide adjoint and at most
// one addition from a coupling adjoint, in stream order; the transposed
// interpolation gathers over fixed consumer lists.  Results do not depend on
// scheduling.
//
// Vector-Jacobian products used here (all per node, in registers):
//   * KBC collision f' = f^eq + (1 - beta gamma) df + beta (gamma - 2) ds with
//     df = f - f^eq(f), ds = S df (shear part), dh = df - ds and
//     gamma = 1/beta - (2 - 1/beta) <ds|dh>/<dh|dh>, <x|y> = sum x y / f^eq
//     (Eqs. f_mirr, gamma_min_approx), differentiated through gamma and the
//     weights 1/f^eq; gamma held at 2 in the LBGK mirror and in the 0/0 guard;
//   * f^eq(rho, u) (Eq. feq_iso): d f^eq_i / d rho = f^eq_i / rho and
//     d f^eq_i / d u_a = f^eq_i L_a(c_ia), L the log-derivative of the axis factor;
//   * rho = sum f, u = j / rho;
//   * non-equilibrium rescaling f -> f^eq + r (f - f^eq) and the four-point
//     tensor interpolation (linear).
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "device.cuh"
#include "kernels.h"
#include "warp.cuh"

namespace lbmk {

// Log-derivatives of the axis factors ghat(c) w.r.t. u (c = -1, 0, +1):
// L(0) = A'/A, L(+1) = A'/A + B'/B, L(-1) = A'/A - B'/B with
// A = 2 - s, A' = -3u/s, B = (2u + s)/(1 - u), B' = ((2 + 3u/s)(1 - u) + 2u + s)/(1 - u)^2.
template <typename R>
__device__ __forceinline__ void axis_logderiv(R u, const AxisEq<R>& e, R (&L)[3]) {
  const R s = e.s;
  const R A = R(1) + e.d[1];
  const R u_s = R(3) * u * rcp_fast(s);  // 3u / s
  const R dA = -u_s;
  const R om = R(1) - u;
  const R iom = rcp_fast(om);
  const R dB = ((R(2) + u_s) * om + R(2) * u + s) * (iom * iom);
  const R la = dA * rcp_fast(A), lb = dB * rcp_fast(e.B);
  L[1] = la;
  L[2] = la + lb;
  L[0] = la - lb;
}

// VJP of f^eq(rho, u) at (rho, u): given xbar (27) with fe_full_i = f^eq_i (full
// value), returns rhobar = sum xbar_i fe_i / rho and ubar_a = sum xbar_i fe_i L_a.
template <typename R>
__device__ __forceinline__ void feq_vjp_rho_u(const R (&xbar)[27], const R (&fefull)[27], R rho, const R (&Lx)[3],
                                              const R (&Ly)[3], const R (&Lz)[3], R& rhobar, R (&ubar)[3]) {
  R sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, sz[3] = {0, 0, 0}, tot = 0;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const R q = xbar[i] * fefull[i];
    tot += q;
    sx[CX(i) + 1] += q;
    sy[CY(i) + 1] += q;
    sz[CZ(i) + 1] += q;
  });
  rhobar = tot * rcp_fast(rho);
  ubar[0] = sx[0] * Lx[0] + sx[1] * Lx[1] + sx[2] * Lx[2];
  ubar[1] = sy[0] * Ly[0] + sy[1] * Ly[1] + sy[2] * Ly[2];
  ubar[2] = sz[0] * Lz[0] + sz[1] * Lz[1] + sz[2] * Lz[2];
}

// Forward quantities of f^eq at the state of f (deviation populations).
template <typename R>
struct EqState {
  R rho_t, rho, u[3];
  AxisEq<R> e[3];
  R L[3][3];
  R fe[27];      // f^eq - W (deviation)
  R fefull[27];  // f^eq
};

template <typename R>
__device__ __forceinline__ void eq_state_from_moments(R rho_t, R rho, R ux, R uy, R uz, EqState<R>& q,
                                                      bool want_inverse) {
  q.rho_t = rho_t;
  q.rho = rho;
  q.u[0] = ux, q.u[1] = uy, q.u[2] = uz;
  for (int a = 0; a < 3; ++a) {
    axis_eq<R>(q.u[a], q.e[a], want_inverse);
    axis_logderiv<R>(q.u[a], q.e[a], q.L[a]);
  }
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    q.fe[i] = R(WI(i)) * (rho_t + rho * qprod<i>(q.e[0], q.e[1], q.e[2]));
    q.fefull[i] = R(WI(i)) + q.fe[i];
  });
}

// fbar += J_feq(f)^T xbar, f^eq as a function of f through rho = sum f and j = sum c f.
template <typename R>
__device__ __forceinline__ void add_feq_f_vjp(const EqState<R>& q, const R (&xbar)[27], R (&fbar)[27]) {
  R rb, ub[3];
  feq_vjp_rho_u<R>(xbar, q.fefull, q.rho, q.L[0], q.L[1], q.L[2], rb, ub);
  // u = j / rho: jbar = ubar / rho, rhobar -= ubar . u / rho
  const R ir = rcp_fast(q.rho);
  const R jb[3] = {ub[0] * ir, ub[1] * ir, ub[2] * ir};
  rb -= (ub[0] * q.u[0] + ub[1] * q.u[1] + ub[2] * q.u[2]) * ir;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    fbar[i] += rb + R(CX(i)) * jb[0] + R(CY(i)) * jb[1] + R(CZ(i)) * jb[2];
  });
}

// lam: in = adjoint of the post-collision state, out = adjoint of the
// pre-collision state f (deviation populations, unchanged).
//
// Written to keep few arrays live (this is register-bound): f^eq - W and df
// are kept, while the shear part, dh and the weights 1/f^eq are recomputed
// in each pass, and the adjoints of ds, df and f^eq are reduced on the fly.
template <typename R>
__device__ void kbc_vjp(const R (&f)[27], R (&lam)[27], R beta, bool lbgk) {
  R rho_t, rho, ux, uy, uz;
  macro(f, rho_t, rho, ux, uy, uz);
  EqState<R> q;
  eq_state_from_moments<R>(rho_t, rho, ux, uy, uz, q, true);
  R df[27];
  R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const R d = f[i] - q.fe[i];
    df[i] = d;
    if constexpr (CX(i) != 0) pxx += d;
    if constexpr (CY(i) != 0) pyy += d;
    if constexpr (CZ(i) != 0) pzz += d;
    if constexpr (CX(i) * CY(i) != 0) pxy += R(CX(i) * CY(i)) * d;
    if constexpr (CX(i) * CZ(i) != 0) pxz += R(CX(i) * CZ(i)) * d;
    if constexpr (CY(i) * CZ(i) != 0) pyz += R(CY(i) * CZ(i)) * d;
  });
  const R tr3 = (pxx + pyy + pzz) * R(1.0 / 3.0);
  const R nxx = pxx - tr3, nyy = pyy - tr3, nzz = pzz - tr3;
  R gamma = R(2), sh = 0, hh = 0;
  bool use_gamma = false;
  const R ib = rcp_fast(beta);
  // entropic weights 1 / f^eq_i in product form: (1/rho) ig_x(c_x) ig_y(c_y) ig_z(c_z)
  R wxy[3][3], wz[3];
  {
    const R irho = rcp_fast(q.rho);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      wz[a] = irho * q.e[2].ig[a];
#pragma unroll
      for (int b2 = 0; b2 < 3; ++b2) wxy[a][b2] = q.e[0].ig[a] * q.e[1].ig[b2];
    }
  }
  auto wgt = [&](auto I) -> R {
    constexpr int i = decltype(I)::value;
    return wxy[CX(i) + 1][CY(i) + 1] * wz[CZ(i) + 1];
  };
  if (!lbgk) {
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const R w = wgt(I);  // entropic weight 1 / f^eq_i
      const R ds = shear_part<i>(nxx, nyy, nzz, pxy, pxz, pyz);
      const R dh = df[i] - ds;
      sh += ds * dh * w;
      hh += dh * dh * w;
    });
    if (hh > R(1e-30) * rho * rho) {
      use_gamma = true;
      gamma = ib - (R(2) - ib) * fdiv(sh, hh);
    }
  }
  const R a = R(1) - beta * gamma, b = beta * (gamma - R(2));
  // reverse of f' = fe + a df + b ds; G = dL/dgamma = -beta lam . dh
  R G = 0;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    G -= beta * lam[i] * (df[i] - shear_part<i>(nxx, nyy, nzz, pxy, pxz, pyz));
  });
  R Lsh = 0, Lhh = 0;
  if (use_gamma) {
    const R c = R(2) - ib;
    const R ihh = rcp_fast(hh);
    Lsh = -G * c * ihh;
    Lhh = G * c * sh * ihh * ihh;
  }
  // pass 1: adjoint of ds reduced to the adjoint of the second moments
  R Sx = 0, Sy = 0, Sz = 0, Exy = 0, Exz = 0, Eyz = 0;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int ax = CX(i) != 0, ay = CY(i) != 0, az = CZ(i) != 0;
    if constexpr (ax + ay + az == 1 || ax + ay + az == 2) {
      const R ds = shear_part<i>(nxx, nyy, nzz, pxy, pxz, pyz);
      R dsb = b * lam[i];
      if (use_gamma) {
        const R dh = df[i] - ds;
        const R w = wgt(I);
        const R dhb = (Lsh * ds + R(2) * Lhh * dh) * w;
        dsb += Lsh * dh * w - dhb;
      }
      if constexpr (ax + ay + az == 1) {
        if constexpr (ax) Sx += dsb;
        else if constexpr (ay) Sy += dsb;
        else Sz += dsb;
      } else {
        if constexpr (!az) Exy += R(CX(i) * CY(i)) * dsb;
        else if constexpr (!ay) Exz += R(CX(i) * CZ(i)) * dsb;
        else Eyz += R(CY(i) * CZ(i)) * dsb;
      }
    }
  });
  // face: ds = (1/3) Pxx - (1/6) Pyy - (1/6) Pzz (for x); edge: ds = c c P / 4
  const R Pbxx = R(1.0 / 3.0) * Sx - R(1.0 / 6.0) * (Sy + Sz);
  const R Pbyy = R(1.0 / 3.0) * Sy - R(1.0 / 6.0) * (Sx + Sz);
  const R Pbzz = R(1.0 / 3.0) * Sz - R(1.0 / 6.0) * (Sx + Sy);
  const R Pbxy = R(0.25) * Exy, Pbxz = R(0.25) * Exz, Pbyz = R(0.25) * Eyz;
  // pass 2: adjoint of df (to f directly) and of f^eq (reduced to rho, u)
  R tot = 0, sx[3] = {0, 0, 0}, sy[3] = {0, 0, 0}, sz[3] = {0, 0, 0};
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const R fefull = R(WI(i)) + q.fe[i];
    R dfb = a * lam[i];
    R feb = lam[i];
    if (use_gamma) {
      const R ds = shear_part<i>(nxx, nyy, nzz, pxy, pxz, pyz);
      const R dh = df[i] - ds;
      const R w = wgt(I);
      dfb += (Lsh * ds + R(2) * Lhh * dh) * w;
      feb -= (Lsh * ds * dh + Lhh * dh * dh) * w * w;  // d(1/fe) = -w^2
    }
    if constexpr (CX(i) != 0) dfb += Pbxx;
    if constexpr (CY(i) != 0) dfb += Pbyy;
    if constexpr (CZ(i) != 0) dfb += Pbzz;
    if constexpr (CX(i) * CY(i) != 0) dfb += R(CX(i) * CY(i)) * Pbxy;
    if constexpr (CX(i) * CZ(i) != 0) dfb += R(CX(i) * CZ(i)) * Pbxz;
    if constexpr (CY(i) * CZ(i) != 0) dfb += R(CY(i) * CZ(i)) * Pbyz;
    feb -= dfb;  // df = f - fe
    lam[i] = dfb;
    const R qv = feb * fefull;
    tot += qv;
    sx[CX(i) + 1] += qv;
    sy[CY(i) + 1] += qv;
    sz[CZ(i) + 1] += qv;
  });
  // f^eq(rho, u): rho-bar = sum feb fe / rho, u-bar_a = sum feb fe L_a; then
  // through rho = sum f and u = j / rho
  R rb = tot * rcp_fast(q.rho);
  const R ub[3] = {sx[0] * q.L[0][0] + sx[1] * q.L[0][1] + sx[2] * q.L[0][2],
                   sy[0] * q.L[1][0] + sy[1] * q.L[1][1] + sy[2] * q.L[1][2],
                   sz[0] * q.L[2][0] + sz[1] * q.L[2][1] + sz[2] * q.L[2][2]};
  const R ir = rcp_fast(q.rho);
  const R jb[3] = {ub[0] * ir, ub[1] * ir, ub[2] * ir};
  rb -= (ub[0] * q.u[0] + ub[1] * q.u[1] + ub[2] * q.u[2]) * ir;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    lam[i] += rb + R(CX(i)) * jb[0] + R(CY(i)) * jb[1] + R(CZ(i)) * jb[2];
  });
}

// ---------------------------------------------------------------------------
// Pull sources, replicated from the forward pull for the scatter of the adjoint.
template <typename R>
__device__ __forceinline__ void push_adjoint(const PatchDev& p, R* __restrict__ lam_old, int x, int y, int z,
                                             const R (&fb)[27]) {
  const long long own = node_index(p, x, y, z);
  const bool bulk = p.type[own] == T_BULK;
  const int X[3] = {x, y, z};
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int c[3] = {CX(i), CY(i), CZ(i)};
    int s[3];
    bool bounce = false;
    unroll<3>([&](auto A) {
      constexpr int a = decltype(A)::value;
      s[a] = X[a] - c[a];
      if (s[a] < 0 || s[a] >= p.dim[a]) {
        if (bulk || p.span[a]) s[a] += s[a] < 0 ? p.dim[a] : -p.dim[a];
        else bounce = true;  // not produced by the layouts the adjoint accepts
      }
    });
    long long src = own;
    int comp = 26 - i;
    if (!bounce) {
      src = node_index(p, s[0], s[1], s[2]);
      comp = i;
    }
    atomicAdd(lam_old + (long long)comp * p.plane + src, fb[i]);
  });
}

template <typename R>
__device__ __forceinline__ void load_lam(const PatchDev& p, const R* __restrict__ lam, long long n, R (&l)[27]) {
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    l[i] = lam[(long long)i * p.plane + n];
  });
}

// Scatter of the adjoint to the sources pull_bulk reads.
template <typename R>
__device__ __forceinline__ void push_bulk(const PatchDev& p, R* __restrict__ lam_old, int x, int y, int z,
                                          const R (&fb)[27]) {
  const int xm = x == 0 ? p.dim[0] - 1 : x - 1, xp = x == p.dim[0] - 1 ? 0 : x + 1;
  const int ym = y == 0 ? p.dim[1] - 1 : y - 1, yp = y == p.dim[1] - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.dim[2] - 1 : z - 1, zp = z == p.dim[2] - 1 ? 0 : z + 1;
  const long long row = p.nxp, sl = (long long)p.nxp * p.dim[1];
  const long long xs[3] = {xp, x, xm};  // source x for cx = -1, 0, +1
  const long long ys[3] = {yp * row, y * row, ym * row};
  const long long zs[3] = {zp * sl, z * sl, zm * sl};
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    atomicAdd(lam_old + (long long)i * p.plane + zs[CZ(i) + 1] + ys[CY(i) + 1] + xs[CX(i) + 1], fb[i]);
  });
}

// stream-collide, two kernels over the stored nodes: bulk nodes and (odd
// substeps) depth-1 nodes pull and scatter along the plain neighbour pattern,
// whose sources all lie in the patch in the layouts the adjoint accepts;
// boundary-class nodes take the node-by-node pull in a kernel of their own, so
// that the hot kernel's code and registers stay those of the plain path.
template <typename R, bool PLAIN>
__global__ void __launch_bounds__(128, 3) k_adj_sc(PatchDev p, const R* __restrict__ fin, const R* __restrict__ lam_new,
                                                R* __restrict__ lam_old, R beta, int odd, int lbgk, int* status) {
  // one thread per stored node (no padding lanes)
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)p.dim[0] * p.dim[1] * p.dim[2]) return;
  const int x = (int)(k % p.dim[0]), y = (int)((k / p.dim[0]) % p.dim[1]);
  const int z = (int)(k / ((long long)p.dim[0] * p.dim[1]));
  const long long own = node_index(p, x, y, z);
  const uint8_t t = p.type[own];
  R f[27], l[27];
  if constexpr (PLAIN) {
    if (!(t == T_BULK || (t == T_D1 && odd))) return;
    pull_bulk<R, R>(p, fin, x, y, z, f);
  } else {
    if (t != T_BC) return;
    pull_generic<R, R>(p, fin, x, y, z, f, status);
  }
  load_lam<R>(p, lam_new, own, l);
  kbc_vjp<R>(f, l, beta, lbgk != 0);
  if constexpr (PLAIN) push_bulk<R>(p, lam_old, x, y, z, l);
  else push_adjoint<R>(p, lam_old, x, y, z, l);
}

// Stream-collide adjoint with plain stores, for patches without boundary-class
// nodes: every entry (y, i) of lambda_old has exactly one pusher, the node
// x = y + c_i (wrapped on spanned axes).  A node updated in the substep pushes
// the adjoint of its pre-collision state; any other stored node pushes zeros;
// an entry whose pusher lies beyond a non-spanned face of the storage box is
// zeroed by its own node.  So the kernel writes every entry once, needs no
// clearing beforehand, and its result does not depend on the order threads
// run in.  The coupling adjoints add to lambda_old after it.
template <typename R>
__global__ void __launch_bounds__(128, 4) k_adj_sc_st(PatchDev p, const R* __restrict__ fin,
                                                   const R* __restrict__ lam_new, R* __restrict__ lam_old, R beta,
                                                   int odd, int lbgk) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)p.dim[0] * p.dim[1] * p.dim[2]) return;
  const int x = (int)(k % p.dim[0]), y = (int)((k / p.dim[0]) % p.dim[1]);
  const int z = (int)(k / ((long long)p.dim[0] * p.dim[1]));
  const long long own = node_index(p, x, y, z);
  const uint8_t t = p.type[own];
  R l[27];
  if (t == T_BULK || (t == T_D1 && odd)) {
    R f[27];
    pull_bulk<R, R>(p, fin, x, y, z, f);
    load_lam<R>(p, lam_new, own, l);
    kbc_vjp<R>(f, l, beta, lbgk != 0);
  } else {
    unroll<27>([&](auto I) { l[decltype(I)::value] = R(0); });
  }
  // source coordinate along an axis for shift -c (the pull source), -1 if
  // beyond a non-spanned face
  const int X[3] = {x, y, z};
  int src[3][3], dst_in[3][3];
  unroll<3>([&](auto A) {
    constexpr int a = decltype(A)::value;
    unroll<3>([&](auto C) {
      constexpr int c = (int)decltype(C)::value - 1;
      int v = X[a] - c;
      if (v < 0 || v >= p.dim[a]) v = p.span[a] ? (v < 0 ? v + p.dim[a] : v - p.dim[a]) : -1;
      src[a][c + 1] = v;
      const int w = X[a] + c;  // the pusher of this node's entry along the axis
      dst_in[a][c + 1] = (w >= 0 && w < p.dim[a]) || p.span[a];
    });
  });
  const long long row = p.nxp, sl = (long long)p.nxp * p.dim[1];
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int sx = src[0][CX(i) + 1], sy = src[1][CY(i) + 1], sz = src[2][CZ(i) + 1];
    if (sx >= 0 && sy >= 0 && sz >= 0) lam_old[(long long)i * p.plane + sz * sl + sy * row + sx] = l[i];
    if (!(dst_in[0][CX(i) + 1] && dst_in[1][CY(i) + 1] && dst_in[2][CZ(i) + 1]))
      lam_old[(long long)i * p.plane + own] = R(0);
  });
}

__device__ __forceinline__ void node_xyz(const PatchDev& p, long long n, int& x, int& y, int& z) {
  x = (int)(n % p.nxp);
  y = (int)((n / p.nxp) % p.dim[1]);
  z = (int)(n / ((long long)p.nxp * p.dim[1]));
}

template <typename R>
__device__ __forceinline__ void pull_node(const PatchDev& p, const R* __restrict__ fin, int x, int y, int z,
                                          R (&f)[27], int* status) {
  if (p.type[node_index(p, x, y, z)] == T_BULK) pull_bulk<R, R>(p, fin, x, y, z, f);
  else pull_generic<R, R>(p, fin, x, y, z, f, status);
}

// ---------------------------------------------------------------------------
// Warp-cooperative node maps for the coalesce and sample adjoints.  Their
// node sets are small (a few thousand nodes) and each node's VJP is a long
// serial chain, so one warp takes one node: lane i < 27 holds population i,
// lanes 27..31 hold zeros, and every sum over the populations is a butterfly
// reduction across the warp.

// Equilibrium quantities of one node, the lane's share: f^eq - W and f^eq of
// its direction and the log-derivatives L_a(c_ia) of its axis factors.
template <typename R>
struct WEq {
  R rho_t, rho, ir, u[3];
  R fe, fefull, Ld[3];
};

template <typename R>
__device__ __forceinline__ void weq_from_moments(R rho_t, R rho, R ux, R uy, R uz, const Lane& d, WEq<R>& q) {
  q.rho_t = rho_t;
  q.rho = rho;
  q.ir = rcp_fast(rho);
  q.u[0] = ux, q.u[1] = uy, q.u[2] = uz;
  R dv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    AxisEq<R> e;
    axis_eq<R>(q.u[a], e, false);
    R L[3];
    axis_logderiv<R>(q.u[a], e, L);
    dv[a] = sel3(d.c[a], e.d);
    q.Ld[a] = sel3(d.c[a], L);
  }
  const R t = dv[0] + dv[1] + dv[0] * dv[1];
  const R qp = t + dv[2] + t * dv[2];
  const R W = R(wi_rt(d.i));
  q.fe = W * (rho_t + rho * qp);
  q.fefull = W + q.fe;
}

// rho~ = sum f, u = j / rho, reduced over the warp, then the equilibrium.
template <typename R>
__device__ __forceinline__ void weq_of(R f, const Lane& d, WEq<R>& q) {
  R m[4] = {f, R(d.c[0]) * f, R(d.c[1]) * f, R(d.c[2]) * f};
  wsum<4>(m);
  const R rho = R(1) + m[0];
  const R ir = rcp_fast(rho);
  weq_from_moments<R>(m[0], rho, m[1] * ir, m[2] * ir, m[3] * ir, d, q);
}

// VJP of f^eq(rho, u) at q: given the lane's xbar, returns rhobar and ubar
// (sum_i xbar_i f^eq_i / rho, sum_i xbar_i f^eq_i L_a(c_ia)).
template <typename R>
__device__ __forceinline__ void wfeq_vjp_rho_u(R xbar, const Lane& d, const WEq<R>& q, R& rb, R (&ub)[3]) {
  const R x = d.on ? xbar * q.fefull : R(0);
  R v[4] = {x, x * q.Ld[0], x * q.Ld[1], x * q.Ld[2]};
  wsum<4>(v);
  rb = v[0] * q.ir;
  ub[0] = v[1], ub[1] = v[2], ub[2] = v[3];
}

// fbar += (J_feq(f)^T xbar)_i, f^eq through rho = sum f and u = j / rho.
template <typename R>
__device__ __forceinline__ R wadd_feq_f_vjp(R xbar, const Lane& d, const WEq<R>& q) {
  R rb, ub[3];
  wfeq_vjp_rho_u<R>(xbar, d, q, rb, ub);
  const R jb[3] = {ub[0] * q.ir, ub[1] * q.ir, ub[2] * q.ir};
  rb -= (ub[0] * q.u[0] + ub[1] * q.u[1] + ub[2] * q.u[2]) * q.ir;
  return rb + R(d.c[0]) * jb[0] + R(d.c[1]) * jb[1] + R(d.c[2]) * jb[2];
}

// The KBC collision VJP of kbc_vjp, one node per warp: f and lam are the
// lane's pre-collision population and post-collision adjoint; returns the
// lane's pre-collision adjoint (garbage on idle lanes).
template <typename R>
__device__ R wkbc_vjp(R f, R lam, const Lane& d, R beta, bool lbgk) {
  WEq<R> q;
  weq_of<R>(f, d, q);
  const R df = d.on ? f - q.fe : R(0);
  const int cx = d.c[0], cy = d.c[1], cz = d.c[2];
  R m[6] = {cx ? df : R(0), cy ? df : R(0), cz ? df : R(0), R(cx * cy) * df, R(cx * cz) * df, R(cy * cz) * df};
  wsum<6>(m);
  const R tr3 = (m[0] + m[1] + m[2]) * R(1.0 / 3.0);
  const R nxx = m[0] - tr3, nyy = m[1] - tr3, nzz = m[2] - tr3;
  const R pxy = m[3], pxz = m[4], pyz = m[5];
  // shear part of the lane's direction (zero at rest and corners)
  R ds = R(0);
  if (d.na == 1) ds = R(0.5) * (cx ? nxx : (cy ? nyy : nzz));
  else if (d.na == 2) ds = R(0.25) * (cz == 0 ? R(cx * cy) * pxy : (cy == 0 ? R(cx * cz) * pxz : R(cy * cz) * pyz));
  const R dh = df - ds;
  const R w = rcp_fast(q.fefull);  // entropic weight 1 / f^eq_i
  R t3[3] = {ds * dh * w, dh * dh * w, d.on ? lam * dh : R(0)};
  wsum<3>(t3);
  const R sh = t3[0], hh = t3[1];
  const R G = -beta * t3[2];  // dL/dgamma
  const R ib = rcp_fast(beta);
  R gamma = R(2);
  bool use_gamma = false;
  if (!lbgk && hh > R(1e-30) * q.rho * q.rho) {
    use_gamma = true;
    gamma = ib - (R(2) - ib) * fdiv(sh, hh);
  }
  const R a = R(1) - beta * gamma, b = beta * (gamma - R(2));
  R Lsh = 0, Lhh = 0;
  if (use_gamma) {
    const R c = R(2) - ib;
    const R ihh = rcp_fast(hh);
    Lsh = -G * c * ihh;
    Lhh = G * c * sh * ihh * ihh;
  }
  // adjoint of ds, reduced to the adjoint of the second moments
  R dsb = b * lam, gw = R(0);
  if (use_gamma) {
    gw = (Lsh * ds + R(2) * Lhh * dh) * w;
    dsb += Lsh * dh * w - gw;
  }
  const bool face = d.on && d.na == 1, edge = d.on && d.na == 2;
  R S[6] = {face && cx ? dsb : R(0),
            face && cy ? dsb : R(0),
            face && cz ? dsb : R(0),
            edge && cz == 0 ? R(cx * cy) * dsb : R(0),
            edge && cy == 0 ? R(cx * cz) * dsb : R(0),
            edge && cx == 0 ? R(cy * cz) * dsb : R(0)};
  wsum<6>(S);
  const R Pbxx = R(1.0 / 3.0) * S[0] - R(1.0 / 6.0) * (S[1] + S[2]);
  const R Pbyy = R(1.0 / 3.0) * S[1] - R(1.0 / 6.0) * (S[0] + S[2]);
  const R Pbzz = R(1.0 / 3.0) * S[2] - R(1.0 / 6.0) * (S[0] + S[1]);
  const R Pbxy = R(0.25) * S[3], Pbxz = R(0.25) * S[4], Pbyz = R(0.25) * S[5];
  // adjoint of df (to f directly) and of f^eq (reduced to rho, u)
  R dfb = a * lam + gw;
  if (cx) dfb += Pbxx;
  if (cy) dfb += Pbyy;
  if (cz) dfb += Pbzz;
  dfb += R(cx * cy) * Pbxy + R(cx * cz) * Pbxz + R(cy * cz) * Pbyz;
  R feb = lam;
  if (use_gamma) feb -= (Lsh * ds * dh + Lhh * dh * dh) * w * w;  // d(1/fe) = -w^2
  feb -= dfb;                                                     // df = f - fe
  return dfb + wadd_feq_f_vjp<R>(feb, d, q);
}

// The lane's population of the pull of node (x, y, z): pull_generic for one
// runtime direction (bulk nodes wrap, as pull_bulk does).
template <typename R>
__device__ __forceinline__ R pull_one(const PatchDev& p, const R* __restrict__ fin, int x, int y, int z, const Lane& d,
                                      int* status) {
  const long long own = node_index(p, x, y, z);
  const bool bulk = p.type[own] == T_BULK;
  const int X[3] = {x, y, z};
  int s[3];
  bool bounce = false, bad = false;
  unroll<3>([&](auto A) {
    constexpr int a = decltype(A)::value;
    s[a] = X[a] - d.c[a];
    if (s[a] < 0 || s[a] >= p.dim[a]) {
      if (bulk || p.span[a]) {
        s[a] += s[a] < 0 ? p.dim[a] : -p.dim[a];
      } else if (!p.periodic[a]) {
        const int Gc = p.org[a] + s[a];
        if (Gc < 0) {
          if (p.walls & (1u << (2 * a))) bounce = true;
          else bad = true;
        } else if (Gc > p.maxc[a]) {
          if (p.walls & (1u << (2 * a + 1))) bounce = true;
          else if (p.inflow == a) s[a] = p.maxc[a] - p.org[a];
          else bad = true;
        } else {
          bad = true;
        }
      } else {
        bad = true;
      }
    }
  });
  long long src = own;
  if (!bounce && !bad) {
    src = node_index(p, s[0], s[1], s[2]);
    if (!bulk) {
      const uint8_t t = p.type[src];
      if (t == T_SOLID) bounce = true;
      else if (t == T_SKIP) bad = true;
    }
  }
  if (bad) {
    atomicOr(status, 1);
    bounce = true;
  }
  if (bounce) return __ldg(fin + (long long)(26 - d.i) * p.plane + own);
  return __ldg(fin + (long long)d.i * p.plane + src);
}

// Scatter of the lane's adjoint along the reversed pull (push_adjoint for one
// runtime direction).
template <typename R>
__device__ __forceinline__ void push_one(const PatchDev& p, R* __restrict__ lam_old, int x, int y, int z, const Lane& d,
                                         R v) {
  const long long own = node_index(p, x, y, z);
  const bool bulk = p.type[own] == T_BULK;
  const int X[3] = {x, y, z};
  int s[3];
  bool bounce = false;
  unroll<3>([&](auto A) {
    constexpr int a = decltype(A)::value;
    s[a] = X[a] - d.c[a];
    if (s[a] < 0 || s[a] >= p.dim[a]) {
      if (bulk || p.span[a]) s[a] += s[a] < 0 ? p.dim[a] : -p.dim[a];
      else bounce = true;  // not produced by the layouts the adjoint accepts
    }
  });
  if (bounce) atomicAdd(lam_old + (long long)(26 - d.i) * p.plane + own, v);
  else atomicAdd(lam_old + (long long)d.i * p.plane + node_index(p, s[0], s[1], s[2]), v);
}


// coalesce: parent twin <- collide_parent(f^eq + r (f_child - f^eq)); one warp per twin
template <typename R>
__global__ void __launch_bounds__(128) k_adj_coalesce(PatchDev pc, const R* __restrict__ fin_c, PatchDev pp,
                                                      const R* __restrict__ lam_new_p, R* __restrict__ lam_old_c,
                                                      const uint32_t* __restrict__ cf_parent,
                                                      const uint32_t* __restrict__ cf_child, long long n, R r,
                                                      R beta_p, int lbgk, int* status) {
  const long long k = warp_id();
  if (k >= n) return;  // whole warp
  const Lane d = lane_dir();
  int x, y, z;
  node_xyz(pc, cf_child[k], x, y, z);
  const R f = d.on ? pull_one<R>(pc, fin_c, x, y, z, d, status) : R(0);
  WEq<R> q;
  weq_of<R>(f, d, q);
  const R fc = d.on ? q.fe + r * (f - q.fe) : R(0);
  R l = d.on ? lam_new_p[(long long)d.i * pp.plane + cf_parent[k]] : R(0);
  l = wkbc_vjp<R>(fc, l, d, beta_p, lbgk != 0);
  // fc = r f + (1 - r) fe(f)
  const R fb = r * l + wadd_feq_f_vjp<R>((R(1) - r) * l, d, q);
  if (d.on) push_one<R>(pc, lam_old_c, x, y, z, d, fb);
}

// explode: child node <- collide_child(f^eq(rho~, u~) + neq~), (rho~, u~, neq~)
// one point of the reconstruction point space or the four-point interpolation
// of four; writes the adjoint of the 31 values to tbar [31][targets].  One
// thread per node: the explode set is large enough (about ten thousand nodes)
// that a warp per node would be bound by instruction issue.
template <typename R>
__global__ void __launch_bounds__(128) k_adj_explode(PatchDev pc, const R* __restrict__ lam_new_c,
                                                     const uint32_t* __restrict__ ex_node,
                                                     const uint4* __restrict__ ex_src, long long n_one, long long n,
                                                     const R* __restrict__ val, R* __restrict__ tbar, long long ld,
                                                     R beta_c, int lbgk) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint4 s = ex_src[k];
  const bool one = k < n_one;
  const R w0 = R(-1.0 / 16.0), w1 = R(9.0 / 16.0);
  auto ip = [&](int c) {
    const R* v = val + (long long)c * ld;
    if (one) return v[s.x];
    return w0 * (v[s.x] + v[s.w]) + w1 * (v[s.y] + v[s.z]);
  };
  R v[4], neq[27];
  for (int c = 0; c < 4; ++c) v[c] = ip(c);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    neq[i] = ip(4 + i);
  });
  EqState<R> q;
  eq_state_from_moments<R>(v[0], R(1) + v[0], v[1], v[2], v[3], q, false);
  R f[27];
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = q.fe[i] + neq[i];
  });
  R l[27];
  load_lam<R>(pc, lam_new_c, ex_node[k], l);
  kbc_vjp<R>(f, l, beta_c, lbgk != 0);
  // f = fe(rho, u) + neq: neq-bar = l; (rho-bar, u-bar) from fe directly
  R rb, ub[3];
  feq_vjp_rho_u<R>(l, q.fefull, q.rho, q.L[0], q.L[1], q.L[2], rb, ub);
  const R vb[4] = {rb, ub[0], ub[1], ub[2]};  // rho~ enters as rho = 1 + rho~
  // the adjoint of the target's interpolated values, tbar[c][k]; the point
  // columns gather them (k_adj_gather)
  for (int c = 0; c < 4; ++c) tbar[(long long)c * n + k] = vb[c];
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    tbar[(long long)(4 + i) * n + k] = l[i];
  });
}

// The transpose of the interpolation passes in gather form: each point column
// j in [j0, j1) sums w * (adjoint of its consumer) over its consumer list --
// targets (tbar) and points of later stages (vbar) -- in a fixed order, so
// the result does not depend on scheduling.  One thread per (column, value).
template <typename R>
__global__ void __launch_bounds__(128) k_adj_gather(const uint32_t* __restrict__ use_ptr,
                                                    const uint32_t* __restrict__ use_ent, long long j0, long long j1,
                                                    R* __restrict__ vbar, long long ld, const R* __restrict__ tbar,
                                                    long long nt) {
  const long long j = j0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j1) return;
  const int c = blockIdx.y;
  const R w[4] = {R(-1.0 / 16.0), R(9.0 / 16.0), R(9.0 / 16.0), R(-1.0 / 16.0)};
  R acc = R(0);
  for (uint32_t e = use_ptr[j]; e < use_ptr[j + 1]; ++e) {
    const uint32_t u = use_ent[e];
    const uint32_t id = u & ((1u << 28) - 1);
    const R x = (u >> 31) ? vbar[(long long)c * ld + id] : tbar[(long long)c * nt + id];
    acc += ((u >> 30) & 1u) ? x : w[(u >> 28) & 3u] * x;
  }
  vbar[(long long)c * ld + j] = acc;
}

// samples: (rho~, u, factor (f - f^eq)) of the pulled state of a parent or
// child node; one warp per sample
template <typename R>
__global__ void __launch_bounds__(128) k_adj_samples(PatchDev pp, const R* __restrict__ fin_p, R* __restrict__ lam_p,
                                                     PatchDev pc, const R* __restrict__ fin_c, R* __restrict__ lam_c,
                                                     const uint32_t* __restrict__ smp_node,
                                                     const uint8_t* __restrict__ smp_kind, long long ns,
                                                     const R* __restrict__ sbar, long long ld, R rescale_p,
                                                     int* status) {
  const long long s = warp_id();
  if (s >= ns) return;  // whole warp
  const Lane d = lane_dir();
  const bool par = smp_kind[s] == 0;
  const PatchDev& q = par ? pp : pc;
  int x, y, z;
  node_xyz(q, smp_node[s], x, y, z);
  const R f = d.on ? pull_one<R>(q, par ? fin_p : fin_c, x, y, z, d, status) : R(0);
  const R factor = par ? rescale_p : R(1);
  WEq<R> e;
  weq_of<R>(f, d, e);
  const R rb = sbar[s], ub[3] = {sbar[ld + s], sbar[2 * ld + s], sbar[3 * ld + s]};
  const R nb = d.on ? sbar[(4 + d.i) * ld + s] : R(0);
  // neq = factor (f - fe(f))
  R fb = factor * nb + wadd_feq_f_vjp<R>(-factor * nb, d, e);
  // rho~ = sum f, u = j / rho
  fb += rb + ((R(d.c[0]) - e.u[0]) * ub[0] + (R(d.c[1]) - e.u[1]) * ub[1] + (R(d.c[2]) - e.u[2]) * ub[2]) * e.ir;
  if (d.on) push_one<R>(q, par ? lam_p : lam_c, x, y, z, d, fb);
}

// Objective: kinetic energy 1/2 sum rho |u|^2 8^-level over owned nodes (a parent
// owns its nodes outside every child's [a+1, b-1] box: classes BULK, BC, D0, D1,
// INLET; a child owns its nodes of depth >= 2: BULK and BC).  Writes dKE/df and
// FP64 partial sums of KE.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_seed(PatchDev p, const R* __restrict__ fin, R* __restrict__ lam,
                                                  double vw, int child_level, double* __restrict__ partial) {
  double acc = 0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < p.plane;
       n += (long long)gridDim.x * blockDim.x) {
    const uint8_t t = p.type[n];
    bool owned;
    if (child_level) owned = (t == T_BULK || t == T_BC);
    else owned = (t == T_BULK || t == T_BC || t == T_D0 || t == T_D1 || t == T_INLET);
    R l[27];
    if (owned) {
      R f[27];
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = fin[(long long)i * p.plane + n];
      });
      R rho_t, rho, ux, uy, uz;
      macro(f, rho_t, rho, ux, uy, uz);
      const double r = 1.0 + (double)rho_t;
      const double u2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
      acc += vw * 0.5 * r * u2;
      // d/df_i (1/2 |j|^2 / rho) = c_i . u - |u|^2 / 2
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        l[i] = (R)(vw * ((double)(CX(i) * ux + CY(i) * uy + CZ(i) * uz) - 0.5 * u2));
      });
    } else {
      unroll<27>([&](auto I) { l[decltype(I)::value] = R(0); });
    }
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      lam[(long long)i * p.plane + n] = l[i];
    });
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < n; ++k) s += partial[k];
    *out = s;
  }
}

// dJ/du0 at each node of a state f = f^eq(1, u0): sum_i lam_i f^eq_i L_a(c_ia), in FP64.
template <typename R>
__global__ void k_adj_grad_u0(PatchDev p, const R* __restrict__ fin, const R* __restrict__ lam, double* __restrict__ g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const long long d = ((long long)z * p.dim[1] + y) * p.dim[0] + x;
  const long long nd = (long long)p.dim[0] * p.dim[1] * p.dim[2];
  const uint8_t t = p.type[own];
  double out[3] = {0, 0, 0};
  if (t != T_SKIP && t != T_SOLID && t != T_INLET) {
    double f[27], l[27];
    for (int i = 0; i < 27; ++i) {
      f[i] = (double)fin[(long long)i * p.plane + own];
      l[i] = (double)lam[(long long)i * p.plane + own];
    }
    double rho_t, rho, ux, uy, uz;
    macro(f, rho_t, rho, ux, uy, uz);
    EqState<double> q;
    eq_state_from_moments<double>(rho_t, rho, ux, uy, uz, q, false);
    double rb, ub[3];
    feq_vjp_rho_u<double>(l, q.fefull, q.rho, q.L[0], q.L[1], q.L[2], rb, ub);
    out[0] = ub[0], out[1] = ub[1], out[2] = ub[2];
  }
  for (int a = 0; a < 3; ++a) g[a * nd + d] = out[a];
}

// ---------------------------------------------------------------------------
template <typename F>
cudaError_t adj_dispatch(int storage, F&& f) {
  if (storage == LBM_FP64) return f((double)0);
  if (storage == LBM_FP32) return f((float)0);
  return cudaErrorInvalidValue;
}

cudaError_t launch_adj_sc(int storage, const PatchDev& p, const void* fin, const void* lam_new, void* lam_old,
                          double beta, int odd, int lbgk, bool with_bc, int* status, cudaStream_t st) {
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    const long long n = (long long)p.dim[0] * p.dim[1] * p.dim[2];
    dim3 block(128), grid((unsigned)((n + 127) / 128));
    if (!with_bc) {  // plain stores, lambda_old needs no clearing
      k_adj_sc_st<R><<<grid, block, 0, st>>>(p, (const R*)fin, (const R*)lam_new, (R*)lam_old, (R)beta, odd, lbgk);
      return cudaGetLastError();
    }
    k_adj_sc<R, true><<<grid, block, 0, st>>>(p, (const R*)fin, (const R*)lam_new, (R*)lam_old, (R)beta, odd, lbgk,
                                              status);
    cudaError_t e = cudaGetLastError();
    if (e || !with_bc) return e;
    k_adj_sc<R, false><<<grid, block, 0, st>>>(p, (const R*)fin, (const R*)lam_new, (R*)lam_old, (R)beta, odd,
                                               lbgk, status);
    return cudaGetLastError();
  });
}

cudaError_t launch_adj_coalesce(int storage, const PatchDev& child, const void* fin_c, const PatchDev& parent,
                                const void* lam_new_p, void* lam_old_c, const uint32_t* cf_parent,
                                const uint32_t* cf_child, int64_t n, double r, double beta_p, int lbgk, int* status,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_adj_coalesce<R><<<(unsigned)((n + 3) / 4), 128, 0, st>>>(child, (const R*)fin_c, parent,
                                                                   (const R*)lam_new_p, (R*)lam_old_c, cf_parent,
                                                                   cf_child, n, (R)r, (R)beta_p, lbgk, status);
    return cudaGetLastError();
  });
}

cudaError_t launch_adj_explode(int storage, const PatchDev& child, const void* lam_new_c, const uint32_t* ex_node,
                               const uint32_t* ex_src, int64_t n_one, int64_t n, const void* val, void* tbar,
                               int64_t ld, double beta_c, int lbgk, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_adj_explode<R><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(child, (const R*)lam_new_c, ex_node,
                                                                  (const uint4*)ex_src, n_one, n, (const R*)val,
                                                                  (R*)tbar, ld, (R)beta_c, lbgk);
    return cudaGetLastError();
  });
}

cudaError_t launch_adj_gather(int storage, const uint32_t* use_ptr, const uint32_t* use_ent, int64_t j0, int64_t j1,
                              void* vbar, int64_t ld, const void* tbar, int64_t nt, cudaStream_t st) {
  if (j1 <= j0) return cudaSuccess;
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_adj_gather<R><<<dim3((unsigned)((j1 - j0 + 127) / 128), 31), 128, 0, st>>>(use_ptr, use_ent, j0, j1, (R*)vbar,
                                                                                 ld, (const R*)tbar, nt);
    return cudaGetLastError();
  });
}

cudaError_t launch_adj_samples(int storage, const PatchDev& parent, const void* fin_p, void* lam_p,
                               const PatchDev& child, const void* fin_c, void* lam_c, const uint32_t* smp_node,
                               const uint8_t* smp_kind, int64_t ns, const void* sbar, int64_t ld, double rescale_p,
                               int* status, cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_adj_samples<R><<<(unsigned)((ns + 3) / 4), 128, 0, st>>>(parent, (const R*)fin_p, (R*)lam_p, child,
                                                                   (const R*)fin_c, (R*)lam_c, smp_node, smp_kind, ns,
                                                                   (const R*)sbar, ld, (R)rescale_p, status);
    return cudaGetLastError();
  });
}

cudaError_t launch_adj_seed(int storage, const PatchDev& p, const void* fin, void* lam, double vol_weight,
                            int child_level, double* partial, int blocks, cudaStream_t st) {
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_adj_seed<R><<<blocks, 256, 0, st>>>(p, (const R*)fin, (R*)lam, vol_weight, child_level, partial);
    return cudaGetLastError();
  });
}

cudaError_t launch_sum_partials(const double* partial, int n, double* out, cudaStream_t st) {
  k_sum_partials<<<1, 32, 0, st>>>(partial, n, out);
  return cudaGetLastError();
}

cudaError_t launch_adj_grad_u0(int storage, const PatchDev& p, const void* fin, const void* lam, double* grad,
                               cudaStream_t st) {
  return adj_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_adj_grad_u0<R><<<grid, block, 0, st>>>(p, (const R*)fin, (const R*)lam, grad);
    return cudaGetLastError();
  });
}

}  // namespace lbmk
