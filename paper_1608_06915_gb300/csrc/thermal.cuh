// Device functions of the two-population thermal model (Sec. II.B, both regimes of Table I),
// shared by the node-by-node kernels (thermal.cu) and the TMA tile pass
// (thermal_tma.cu).  The model and storage conventions are stated in thermal.cu.
#pragma once
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "collide.cuh"
#include "device.cuh"
#include "kernels.h"

namespace lbmk {

template <int i>
__host__ __device__ constexpr int C2() {
  return CX(i) * CX(i) + CY(i) * CY(i) + CZ(i) * CZ(i);
}

template <typename R>
struct ThState {
  R rho_t, rho, ux, uy, uz;
  R e_t;    // 2 rho E - 1
  R T_d;    // T - T0
};

template <typename R>
__device__ __forceinline__ void thermal_state(const R (&f)[27], const R (&g)[27], ThState<R>& s) {
  macro(f, s.rho_t, s.rho, s.ux, s.uy, s.uz);
  R e[3] = {0, 0, 0};
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    e[CZ(i) + 1] += g[i];
  });
  s.e_t = (e[0] + e[2]) + e[1];
  // T = (2E - u^2)/3 with 2E = (1 + e_t)/rho  =>  T - 1/3 = ((e_t - rho_t)/rho - u^2)/3
  const R u2 = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
  s.T_d = (fdiv(s.e_t - s.rho_t, s.rho) - u2) * R(1.0 / 3.0);
}

// g^eq - W_i c_i^2 for (rho, u, 2 rho E); see the header comment.
template <typename R>
__device__ __forceinline__ void geq_dev(R rho_t, R rho, R ux, R uy, R uz, R e_t, R (&ge)[27]) {
  const R E2 = R(1) + e_t;
  const R u2 = ux * ux + uy * uy + uz * uz;
  const R a1 = R(3) * (E2 + R(2.0 / 3.0) * rho);
  const R a2 = R(4.5) * (E2 + R(4.0 / 3.0) * rho);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const R cu = R(CX(i)) * ux + R(CY(i)) * uy + R(CZ(i)) * uz;
    ge[i] = R(WI(i)) * (e_t + rho_t * R(C2<i>() - 1) + a1 * cu + a2 * (cu * cu - u2 * R(1.0 / 3.0)));
  });
}

// Non-equilibrium pressure tensor P1 = sum c c (f - f^eq) from f and its equilibrium.
template <typename R>
__device__ __forceinline__ void p1_tensor(const R (&f)[27], const R (&fe)[27], R (&P)[6]) {
  for (int k = 0; k < 6; ++k) P[k] = 0;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const R d = f[i] - fe[i];
    if constexpr (CX(i) != 0) P[0] += d;
    if constexpr (CY(i) != 0) P[1] += d;
    if constexpr (CZ(i) != 0) P[2] += d;
    if constexpr (CX(i) * CY(i) != 0) P[3] += R(CX(i) * CY(i)) * d;
    if constexpr (CX(i) * CZ(i) != 0) P[4] += R(CX(i) * CZ(i)) * d;
    if constexpr (CY(i) * CZ(i) != 0) P[5] += R(CY(i) * CZ(i)) * d;
  });
}

// W_i c_i . V / T0 for a vector V
template <int i, typename R>
__device__ __forceinline__ R wcv3(R vx, R vy, R vz) {
  return R(3.0 * WI(i)) * (R(CX(i)) * vx + R(CY(i)) * vy + R(CZ(i)) * vz);
}

// One thermal collision of deviation populations: f in place, g read through
// gget(I) (the pre-collision g_i, any number of times) and written through
// gput(I, g'_i) once per population after every read; returns gamma.
// Pr <= 1: f* = f^eq and g* carries q - 2 u.(P - P^eq) (Table I); Pr > 1:
// f* - f^eq is the Grad term W_i (P - P^eq)_ab (c_ia c_ib - T0 d_ab)/(2 T0^2)
// and g* carries q^eq + 2 u.(P - P^eq), with the closed-form P^eq.  The g
// update of each population needs only the node's moments.
template <typename R, typename GGet, typename GPut>
__device__ __forceinline__ R thermal_collide_acc(R (&f)[27], GGet&& gget, GPut&& gput, R beta, R beta1, R glam,
                                                 R tref_d, bool lbgk, bool pr_gt1) {
  ThState<R> s;
  macro(f, s.rho_t, s.rho, s.ux, s.uy, s.uz);
  {
    R e[3] = {0, 0, 0};
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      e[CZ(i) + 1] += gget(I);
    });
    s.e_t = (e[0] + e[2]) + e[1];
    // T = (2E - u^2)/3 with 2E = (1 + e_t)/rho  =>  T - 1/3 = ((e_t - rho_t)/rho - u^2)/3
    const R u2 = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
    s.T_d = (fdiv(s.e_t - s.rho_t, s.rho) - u2) * R(1.0 / 3.0);
  }
  // pre-collision moments: P - P^eq = P~ + T0 d - rho T0 d - rho u u, q = sum c g
  R P[6] = {0, 0, 0, 0, 0, 0}, q[3] = {0, 0, 0};
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (CX(i) != 0) P[0] += f[i];
    if constexpr (CY(i) != 0) P[1] += f[i];
    if constexpr (CZ(i) != 0) P[2] += f[i];
    if constexpr (CX(i) * CY(i) != 0) P[3] += R(CX(i) * CY(i)) * f[i];
    if constexpr (CX(i) * CZ(i) != 0) P[4] += R(CX(i) * CZ(i)) * f[i];
    if constexpr (CY(i) * CZ(i) != 0) P[5] += R(CY(i) * CZ(i)) * f[i];
  });
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (CX(i) != 0 || CY(i) != 0 || CZ(i) != 0) {
      const R gi = gget(I);
      if constexpr (CX(i) != 0) q[0] += R(CX(i)) * gi;
      if constexpr (CY(i) != 0) q[1] += R(CY(i)) * gi;
      if constexpr (CZ(i) != 0) q[2] += R(CZ(i)) * gi;
    }
  });
  const R u[3] = {s.ux, s.uy, s.uz};
  const R rt3 = s.rho_t * R(1.0 / 3.0);
  const R Pd[3][3] = {{P[0] - rt3 - s.rho * u[0] * u[0], P[3] - s.rho * u[0] * u[1], P[4] - s.rho * u[0] * u[2]},
                      {P[3] - s.rho * u[1] * u[0], P[1] - rt3 - s.rho * u[1] * u[1], P[5] - s.rho * u[1] * u[2]},
                      {P[4] - s.rho * u[2] * u[0], P[5] - s.rho * u[2] * u[1], P[2] - rt3 - s.rho * u[2] * u[2]}};
  const R qc = R(1) + s.e_t + R(2.0 / 3.0) * s.rho;  // q^eq = (2 rho E + 2 rho T0) u
  R X[3];  // (g* - g^eq) first moment
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R Pu2 = R(2) * (Pd[a][0] * u[0] + Pd[a][1] * u[1] + Pd[a][2] * u[2]);
    X[a] = pr_gt1 ? Pu2 : q[a] - qc * u[a] - Pu2;
  }
  // g^eq - W_i c_i^2 for (rho, u, 2 rho E) (geq_dev), population by population
  {
    const R E2 = R(1) + s.e_t;
    const R u2 = s.ux * s.ux + s.uy * s.uy + s.uz * s.uz;
    const R a1 = R(3) * (E2 + R(2.0 / 3.0) * s.rho);
    const R a2 = R(4.5) * (E2 + R(4.0 / 3.0) * s.rho);
    const R b2 = R(2) * beta, b12 = R(2) * (beta - beta1);
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const R cu = R(CX(i)) * s.ux + R(CY(i)) * s.uy + R(CZ(i)) * s.uz;
      const R ge = R(WI(i)) * (s.e_t + s.rho_t * R(C2<i>() - 1) + a1 * cu + a2 * (cu * cu - u2 * R(1.0 / 3.0)));
      const R gi = gget(I);
      gput(I, gi + b2 * (ge - gi) + b12 * wcv3<i>(X[0], X[1], X[2]));
    });
  }
  const R duz = glam * (s.T_d - tref_d);
  // f is still the pre-collision state: its moments are those computed above
  const R gamma = kbc_collide_m<R, 4>(f, s.rho_t, s.rho, s.ux, s.uy, s.uz, beta, R(0), R(0), duz, lbgk);
  if (pr_gt1) {
    // 2 (beta - beta1)(f* - f^eq) at T0 = 1/3: 9 (beta - beta1) W_i Pd_ab (c_ia c_ib - d_ab / 3)
    const R k9 = R(9) * (beta - beta1);
    const R tr3 = (Pd[0][0] + Pd[1][1] + Pd[2][2]) * R(1.0 / 3.0);
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      R v = -tr3;
      if constexpr (CX(i) != 0) v += Pd[0][0];
      if constexpr (CY(i) != 0) v += Pd[1][1];
      if constexpr (CZ(i) != 0) v += Pd[2][2];
      if constexpr (CX(i) * CY(i) != 0) v += R(2 * CX(i) * CY(i)) * Pd[0][1];
      if constexpr (CX(i) * CZ(i) != 0) v += R(2 * CX(i) * CZ(i)) * Pd[0][2];
      if constexpr (CY(i) * CZ(i) != 0) v += R(2 * CY(i) * CZ(i)) * Pd[1][2];
      f[i] += k9 * R(WI(i)) * v;
    });
  }
  return gamma;
}

// The same collision with g held in registers (in place).
template <typename R>
__device__ __forceinline__ R thermal_collide(R (&f)[27], R (&g)[27], R beta, R beta1, R glam, R tref_d, bool lbgk,
                                             bool pr_gt1) {
  return thermal_collide_acc<R>(
      f, [&](auto I) -> R { return g[decltype(I)::value]; }, [&](auto I, R v) { g[decltype(I)::value] = v; }, beta,
      beta1, glam, tref_d, lbgk, pr_gt1);
}

// Non-equilibrium rescaling of a thermal pair from a level with (beta_s, beta1_s)
// to one with (beta_t, beta1_t): factors ff = beta_s/(r beta_t), fg = beta1_s/(r beta1_t).
// Writes the rescaled non-equilibrium parts and the state's (rho~, u, T - T0).
template <typename R>
__device__ __forceinline__ void thermal_neq(const R (&f)[27], const R (&g)[27], R ff, R fg, R (&fneq)[27],
                                            R (&gneq)[27], ThState<R>& s) {
  thermal_state(f, g, s);
  R fe[27], ge[27];
  feq_dev(s.rho_t, s.rho, s.ux, s.uy, s.uz, fe);
  geq_dev(s.rho_t, s.rho, s.ux, s.uy, s.uz, s.e_t, ge);
  R P1[6];
  p1_tensor(f, fe, P1);
  const R Y[3] = {R(2) * (P1[0] * s.ux + P1[3] * s.uy + P1[4] * s.uz),
                  R(2) * (P1[3] * s.ux + P1[1] * s.uy + P1[5] * s.uz),
                  R(2) * (P1[4] * s.ux + P1[5] * s.uy + P1[2] * s.uz)};
  const R fd = ff - fg;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    fneq[i] = ff * (f[i] - fe[i]);
    gneq[i] = fg * (g[i] - ge[i]) + fd * wcv3<i>(Y[0], Y[1], Y[2]);
  });
}

// Generic pull of f and g: walls (f bounce-back, g anti-bounce-back to the wall
// equilibrium at rest, temperature T_w, density of the node's own state), solid
// nodes (f bounce-back; g bounce-back when adiabatic, else anti-bounce-back to
// the solid temperature twd[6] as at the walls), outlet (clamped source),
// spanned-axis wrap.
template <typename R>
__device__ __forceinline__ void pull_generic_th(const PatchDev& p, const R* __restrict__ fin,
                                                const R* __restrict__ gin, int x, int y, int z, R (&f)[27],
                                                R (&g)[27], const R* twd, bool solid_iso, int* status) {
  const long long own = node_index(p, x, y, z);
  const int X[3] = {x, y, z};
  const int wk = p.wq_idx ? p.wq_idx[own] : -1;  // this node's row of wall fractions
  R rho_own_t = 0;
  bool have_rho = false, any_bad = false;  // an unresolved source is reported once, after the loads
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int c[3] = {CX(i), CY(i), CZ(i)};
    int s[3];
    bool bounce = false, bad = false;
    int wall_face = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s[a] = X[a] - c[a];
      if (s[a] < 0 || s[a] >= p.dim[a]) {
        if (p.span[a]) {
          s[a] += s[a] < 0 ? p.dim[a] : -p.dim[a];
        } else if (!p.periodic[a]) {
          const int G = p.org[a] + s[a];
          if (G < 0) {
            if (p.walls & (1u << (2 * a))) bounce = true, wall_face = 2 * a;
            else bad = true;
          } else if (G > p.maxc[a]) {
            if (p.walls & (1u << (2 * a + 1))) bounce = true, wall_face = 2 * a + 1;
            else if (p.inflow == a) s[a] = p.maxc[a] - p.org[a];
            else bad = true;
          } else {
            bad = true;
          }
        } else {
          bad = true;
        }
      }
    }
    long long src = own;
    bool solid = false;
    if (!bounce && !bad) {
      src = node_index(p, s[0], s[1], s[2]);
      const uint8_t t = p.type[src];
      if (t == T_SOLID) {
        bounce = solid = true;
        if (solid_iso) wall_face = 6;  // isothermal solid surface at twd[6]
      }
      else if (t == T_SKIP) bad = true;
    }
    if (bad) {
      any_bad = true;
      bounce = true;
    }
    if (bounce) {
      // the wall term of an isothermal face or surface, in deviation form:
      // g^w_i + g^w_ibar - 2 W_i c_i^2 = 2 W_i (3 rho T_w' + rho~ c_i^2),
      // T_w' = T_w - T0, g^w_i = W_i rho (3 T_w + c_i^2 - 1)
      R w = 0;
      if (wall_face >= 0) {
        if (!have_rho) {
          for (int k = 0; k < 27; ++k) rho_own_t += fin[(long long)k * p.plane + own];
          have_rho = true;
        }
        w = R(2 * WI(i)) * (R(3) * (R(1) + rho_own_t) * twd[wall_face] + rho_own_t * R(C2<i>()));
      }
      if (solid && wk >= 0) {
        // curved surface: interpolated along the link
        const R q = R(p.wq[27 * wk + 26 - i]);
        f[i] = returning<i, R, R>(p, fin, own, X, q, false, R(0));
        g[i] = returning<i, R, R>(p, gin, own, X, q, wall_face >= 0, w);
      } else {
        f[i] = fin[(long long)(26 - i) * p.plane + own];
        const R gb = gin[(long long)(26 - i) * p.plane + own];
        g[i] = wall_face >= 0 ? w - gb : gb;
      }
    } else {
      f[i] = fin[(long long)i * p.plane + src];
      g[i] = gin[(long long)i * p.plane + src];
    }
  });
  if (any_bad) atomicOr(status, 1);
}

template <typename R>
__device__ __forceinline__ void pull_th(const PatchDev& p, const R* __restrict__ fin, const R* __restrict__ gin,
                                        int x, int y, int z, R (&f)[27], R (&g)[27], const R* twd, bool solid_iso,
                                        int* status) {
  if (p.type[node_index(p, x, y, z)] == T_BULK) {
    pull_bulk<R, R>(p, fin, x, y, z, f);
    pull_bulk<R, R>(p, gin, x, y, z, g);
  } else {
    pull_generic_th<R>(p, fin, gin, x, y, z, f, g, twd, solid_iso, status);
  }
}

template <typename R>
struct ThParams {
  R twd[7];  // wall temperature - T0 per wall face; [6]: isothermal solid surfaces
  R glam;    // g lambda / 2^level (coarse acceleration per unit T, per level step)
  R tref_d;  // T_ref - T0
  R beta, beta1;
  int lbgk;
  int pr_gt1;     // Pr > 1 rows of Table I
  int solid_iso;  // solid surfaces held at twd[6] (else adiabatic)
  int wait_sleeps;  // bound of the TMA pass's waits for a loaded stage
};

template <typename R>
__device__ __forceinline__ void store2(const PatchDev& p, R* __restrict__ fo, R* __restrict__ go, long long n,
                                       const R (&f)[27], const R (&g)[27]) {
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    fo[(long long)i * p.plane + n] = f[i];
    go[(long long)i * p.plane + n] = g[i];
  });
}

template <typename R>
ThParams<R> th_params(const ThermalLevel& L) {
  ThParams<R> t;
  for (int k = 0; k < 7; ++k) t.twd[k] = (R)L.twd[k];
  t.solid_iso = L.solid_iso;
  t.glam = (R)L.glam;
  t.tref_d = (R)L.tref_d;
  t.beta = (R)L.beta;
  t.beta1 = (R)L.beta1;
  t.lbgk = L.lbgk;
  t.pr_gt1 = L.pr_gt1;
  t.wait_sleeps = L.wait_sleeps;
  return t;
}

template <typename F>
cudaError_t th_dispatch(int storage, F&& f) {
  if (storage == LBM_FP64) return f((double)0);
  if (storage == LBM_FP32) return f((float)0);
  return cudaErrorInvalidValue;
}

}  // namespace lbmk
