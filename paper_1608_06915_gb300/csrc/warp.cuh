// One node per warp: lane i < 27 holds population i of the node, lanes
// 27 .. 31 take the rest direction and stay out of every sum and store, and
// every sum over the populations is a butterfly reduction across the warp.
// For node sets too small to fill the GPU with a thread per node: the
// thread-per-node code, unrolled over the 27 populations, is long, and a few
// warps per SM walking it stall on instruction fetch (on the fix-up nodes of
// the sphere, ncu counts 11 no-instruction stalls per issued instruction);
// the warp form is short and keeps 27 lanes busy per node.
// Shared by the forward fix-up kernels (sc_tma.cuh) and the coupling adjoints
// (adjoint.cu).
#pragma once
#include "device.cuh"

namespace lbmk {

constexpr unsigned kFullMask = 0xffffffffu;

// Sums over the warp of N values at once (the N butterflies interleaved).
template <int N, typename R>
__device__ __forceinline__ void wsum(R (&v)[N]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] += __shfl_xor_sync(kFullMask, v[j], o);
  }
}

template <typename R>
__device__ __forceinline__ R sel3(int c, const R (&a)[3]) {
  return c < 0 ? a[0] : (c == 0 ? a[1] : a[2]);
}

// The lane's direction: idle lanes take the rest direction (finite
// equilibrium values) and are masked out of every sum and store.
struct Lane {
  int i, c[3], na;  // direction, velocity, number of non-zero components
  bool on;
};

__device__ __forceinline__ Lane lane_dir() {
  Lane d;
  const int l = threadIdx.x & 31;
  d.on = l < 27;
  d.i = d.on ? l : 13;
  d.c[0] = d.i % 3 - 1, d.c[1] = (d.i / 3) % 3 - 1, d.c[2] = d.i / 9 - 1;
  d.na = (d.c[0] != 0) + (d.c[1] != 0) + (d.c[2] != 0);
  return d;
}

__device__ __forceinline__ long long warp_id() {
  return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

// The generic pull (pull_generic) of the lane's population: the source node
// along -c, or the bounce rule at walls and solids (interpolated along the
// link where the patch carries wall fractions); sets *bad for a source that
// resolves to no node (the caller reports it).
template <typename S, typename R>
__device__ __forceinline__ R wpull_generic(const PatchDev& p, const S* __restrict__ fin, int x, int y, int z,
                                           const Lane& d, bool& bad) {
  const long long own = node_index(p, x, y, z);
  const int X[3] = {x, y, z};
  int s[3];
  bool bounce = false;
  bad = false;
  unroll<3>([&](auto A) {
    constexpr int a = decltype(A)::value;
    s[a] = X[a] - d.c[a];
    if (s[a] < 0 || s[a] >= p.dim[a]) {
      if (p.span[a]) {
        s[a] += s[a] < 0 ? p.dim[a] : -p.dim[a];
      } else if (!p.periodic[a]) {
        const int G = p.org[a] + s[a];
        if (G < 0) {
          if (p.walls & (1u << (2 * a))) bounce = true;
          else bad = true;
        } else if (G > p.maxc[a]) {
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
  const int ib = 26 - d.i;
  const R own_ib = Stor<S>::ld(fin + (long long)ib * p.plane + own);
  if (bounce || bad) return own_ib;
  const long long src = node_index(p, s[0], s[1], s[2]);
  const uint8_t t = p.type[src];
  if (t == T_SKIP) {
    bad = true;
    return own_ib;
  }
  if (t != T_SOLID) return Stor<S>::ld(fin + (long long)d.i * p.plane + src);
  const int wk = p.wq_idx ? p.wq_idx[own] : -1;
  if (wk < 0) return own_ib;
  // curved surface (returning): the wall at fraction q of the link along c_ib
  const R q = R(p.wq[27 * wk + ib]);
  if (q < R(0.5)) {
    int b[3];
    bool ok = true;
    unroll<3>([&](auto A) {
      constexpr int a = decltype(A)::value;
      b[a] = X[a] + d.c[a];
      if (b[a] < 0 || b[a] >= p.dim[a]) {
        if (p.span[a]) b[a] += b[a] < 0 ? p.dim[a] : -p.dim[a];
        else ok = false;
      }
    });
    if (ok) {
      const long long bi = node_index(p, b[0], b[1], b[2]);
      const uint8_t tb = p.type[bi];
      if (tb != T_SOLID && tb != T_SKIP)
        return R(2) * q * own_ib + (R(1) - R(2) * q) * Stor<S>::ld(fin + (long long)ib * p.plane + bi);
    }
    return own_ib;
  }
  const R i2q = R(1) / (R(2) * q);
  return own_ib * i2q + (R(2) * q - R(1)) * i2q * Stor<S>::ld(fin + (long long)d.i * p.plane + own);
}

// The lane's deviation of f^eq(rho, u) from the per-axis factors (Eq.
// feq_iso in deviation form): W_i (rho~ + rho q_i), q_i = prod (1 + d_a) - 1.
template <typename R>
__device__ __forceinline__ R wfeq_dev(R rho_t, R rho, R ux, R uy, R uz, const Lane& d) {
  const R u[3] = {ux, uy, uz};
  R dv[3];
  unroll<3>([&](auto A) {
    constexpr int a = decltype(A)::value;
    AxisEq<R> e;
    axis_eq<R>(u[a], e, false);
    dv[a] = sel3(d.c[a], e.d);
  });
  const R t = dv[0] + dv[1] + dv[0] * dv[1];
  const R qp = t + dv[2] + t * dv[2];
  return R(wi_rt(d.i)) * (rho_t + rho * qp);
}

// The KBC collision with the exact-difference force (kbc_collide), one node
// per warp: f is the lane's pre-collision deviation population; returns its
// post-collision deviation (garbage on idle lanes).  Same arithmetic as the
// thread-per-node collision, summed in another order.
template <typename R>
__device__ __forceinline__ R wkbc_collide(R f, const Lane& d, R beta, R dux, R duy, R duz, bool lbgk) {
  R m[4] = {d.on ? f : R(0), d.on ? R(d.c[0]) * f : R(0), d.on ? R(d.c[1]) * f : R(0), d.on ? R(d.c[2]) * f : R(0)};
  wsum<4>(m);
  const R rho_t = m[0], rho = R(1) + m[0];
  const R ir = rcp_fast(rho);
  const R ux = m[1] * ir, uy = m[2] * ir, uz = m[3] * ir;
  const R fe = wfeq_dev<R>(rho_t, rho, ux, uy, uz, d);
  const R df = d.on ? f - fe : R(0);
  const int cx = d.c[0], cy = d.c[1], cz = d.c[2];
  R P[6] = {cx ? df : R(0), cy ? df : R(0), cz ? df : R(0), R(cx * cy) * df, R(cx * cz) * df, R(cy * cz) * df};
  wsum<6>(P);
  const R tr3 = (P[0] + P[1] + P[2]) * R(1.0 / 3.0);
  R ds = R(0);
  if (d.na == 1) ds = R(0.5) * ((cx ? P[0] : (cy ? P[1] : P[2])) - tr3);
  else if (d.na == 2) ds = R(0.25) * (cz == 0 ? R(cx * cy) * P[3] : (cy == 0 ? R(cx * cz) * P[4] : R(cy * cz) * P[5]));
  R gamma = R(2);
  if (!lbgk) {
    const R dh = df - ds;
    const R w = rcp_fast(R(wi_rt(d.i)) + fe);  // entropic weight 1 / f^eq_i
    R t2[2] = {d.on ? ds * dh * w : R(0), d.on ? dh * dh * w : R(0)};
    wsum<2>(t2);
    const R ib = rcp_fast(beta);
    if (t2[1] > R(1e-30) * rho * rho) gamma = ib - (R(2) - ib) * fdiv(t2[0], t2[1]);
  }
  const R a = R(1) - beta * gamma, b = beta * (gamma - R(2));
  // f' = f^eq(rho, u + du) + a df + b ds (the exact difference method)
  const R fe1 = (dux != R(0) || duy != R(0) || duz != R(0)) ? wfeq_dev<R>(rho_t, rho, ux + dux, uy + duy, uz + duz, d)
                                                           : fe;
  return fe1 + a * df + b * ds;
}

}  // namespace lbmk
