// Two-population thermal model (Sec. II.B, both Prandtl regimes of Table I)
// on the refined grid.
//
// f follows the isothermal KBC collision with the Boussinesq acceleration
// g*lambda*(T - T_ref) e_z through the exact difference method, plus, for
// Pr > 1, 2 (beta - beta1)(f* - f^eq) with the Grad term of P - P^eq; g relaxes as
//   g' = g + 2 beta (g^eq - g) + 2 (beta - beta1) (g* - g^eq)
// (Eq. kinetics_g_entr), where the quasi-equilibrium differs from the
// equilibrium only in its first moment (Table I):
//   Pr <= 1: g*_i - g^eq_i = W_i c_i . (q - q^eq - 2 (P - P^eq) u) / T0,
//   Pr > 1:  g*_i - g^eq_i = W_i c_i . (2 (P - P^eq) u) / T0.
// g^eq is the Grad form (Eq. grad_general) with (2 rho E, q^eq, R^eq), T0 = 1/3.
// At rest at the reference state g^eq_i = W_i c_i^2; g is stored as the
// deviation from that, f as the deviation from W_i.
//
// Interface (Sec. III.A, thermal model): f non-equilibrium scaled by
// ff = beta_s / (r beta_t); g by
//   g_t = g^eq + fg (g - g^eq) + (ff - fg) W_i c_i . (2 P1 u) / T0,
//   fg = beta1_s / (r beta1_t),  P1 = sum c c (f - f^eq)  (Eqs. for P1 and g^neq_f);
// for Pr > 1 the two ratios swap (the host passes them).
// Reconstruction interpolates rho, u, T and both non-equilibrium parts.
// Walls: f half-way bounce-back, g anti-bounce-back to the wall equilibrium at
// rest, temperature T_w; solids likewise at their temperature when isothermal,
// else bounce-back of g.  Every kernel here pulls node by node.
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "device.cuh"
#include "kernels.h"
#include "thermal.cuh"

namespace lbmk {

// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) k_th_tiles(PatchDev p, const R* __restrict__ fin, const R* __restrict__ gin,
                                                  R* __restrict__ fout, R* __restrict__ gout,
                                                  const uint32_t* __restrict__ tiles, int ntx, ThParams<R> tp, int odd,
                                                  int* status) {
  const uint32_t t = tiles[blockIdx.x];
  const int x = (int)(t % (uint32_t)ntx) * 128 + threadIdx.x;
  const int y = (int)((t / (uint32_t)ntx) % (uint32_t)p.dim[1]);
  const int z = (int)(t / ((uint32_t)ntx * (uint32_t)p.dim[1]));
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const uint8_t ty = p.type[own];
  if (!(ty == T_BULK || ty == T_BC || (ty == T_D1 && odd))) return;
  R f[27], g[27];
  pull_th<R>(p, fin, gin, x, y, z, f, g, tp.twd, tp.solid_iso != 0, status);
  thermal_collide<R>(f, g, tp.beta, tp.beta1, tp.glam, tp.tref_d, tp.lbgk != 0, tp.pr_gt1 != 0);
  store2(p, fout, gout, own, f, g);
}

template <typename R>
__global__ void __launch_bounds__(128) k_th_coalesce(PatchDev pc, const R* __restrict__ fin_c,
                                                     const R* __restrict__ gin_c, PatchDev pp, R* __restrict__ fo_p,
                                                     R* __restrict__ go_p, const uint32_t* __restrict__ cf_parent,
                                                     const uint32_t* __restrict__ cf_child, long long n, R ff, R fg,
                                                     ThParams<R> tc, ThParams<R> tpar, int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t cn = cf_child[k];
  const int x = (int)(cn % pc.nxp), y = (int)((cn / pc.nxp) % pc.dim[1]);
  const int z = (int)(cn / ((long long)pc.nxp * pc.dim[1]));
  R f[27], g[27];
  pull_th<R>(pc, fin_c, gin_c, x, y, z, f, g, tc.twd, tc.solid_iso != 0, status);
  R fn[27], gn[27];
  ThState<R> s;
  thermal_neq<R>(f, g, ff, fg, fn, gn, s);
  R fe[27], ge[27];
  feq_dev(s.rho_t, s.rho, s.ux, s.uy, s.uz, fe);
  geq_dev(s.rho_t, s.rho, s.ux, s.uy, s.uz, s.e_t, ge);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = fe[i] + fn[i];
    g[i] = ge[i] + gn[i];
  });
  thermal_collide<R>(f, g, tpar.beta, tpar.beta1, tpar.glam, tpar.tref_d, tpar.lbgk != 0, tpar.pr_gt1 != 0);
  store2(pp, fo_p, go_p, cf_parent[k], f, g);
}

// samples: [59][ld] = rho - 1, ux, uy, uz, T - T0, fneq_0..26, gneq_0..26 (child
// scale), columns [0, ns) of the point space
template <typename R>
__global__ void __launch_bounds__(128, 4) k_th_samples(PatchDev pp, const R* __restrict__ fin_p,
                                                    const R* __restrict__ gin_p, PatchDev pc,
                                                    const R* __restrict__ fin_c, const R* __restrict__ gin_c,
                                                    const uint32_t* __restrict__ smp_node,
                                                    const uint8_t* __restrict__ smp_kind, long long ns,
                                                    R* __restrict__ out, long long ld, R ff, R fg, ThParams<R> tpar,
                                                    ThParams<R> tc, int* status) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  R f[27], g[27];
  const uint32_t n = smp_node[s];
  const bool par = smp_kind[s] == 0;
  const PatchDev& q = par ? pp : pc;
  const int x = (int)(n % q.nxp), y = (int)((n / q.nxp) % q.dim[1]);
  const int z = (int)(n / ((long long)q.nxp * q.dim[1]));
  if (par) pull_th<R>(pp, fin_p, gin_p, x, y, z, f, g, tpar.twd, tpar.solid_iso != 0, status);
  else pull_th<R>(pc, fin_c, gin_c, x, y, z, f, g, tc.twd, tc.solid_iso != 0, status);
  R fn[27], gn[27];
  ThState<R> st;
  thermal_neq<R>(f, g, par ? ff : R(1), par ? fg : R(1), fn, gn, st);
  out[s] = st.rho_t;
  out[ld + s] = st.ux;
  out[2 * ld + s] = st.uy;
  out[3 * ld + s] = st.uz;
  out[4 * ld + s] = st.T_d;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    out[(5 + i) * ld + s] = fn[i];
    out[(32 + i) * ld + s] = gn[i];
  });
}

// Targets [0, n_one) read one point of the reconstruction point space, the
// others interpolate four (the last separable Lagrange pass, Eq. interp).
template <typename R>
__global__ void __launch_bounds__(128, 4) k_th_explode(PatchDev pc, R* __restrict__ fo_c, R* __restrict__ go_c,
                                                    const uint32_t* __restrict__ ex_node,
                                                    const uint4* __restrict__ ex_src, long long n_one, long long n,
                                                    const R* __restrict__ val, long long ld, ThParams<R> tc) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint4 s = __ldg(ex_src + k);
  const bool one = k < n_one;
  const R w0 = R(-1.0 / 16.0), w1 = R(9.0 / 16.0);
  auto ip = [&](int c) {
    const R* v = val + (long long)c * ld;
    if (one) return __ldg(v + s.x);
    return w0 * (__ldg(v + s.x) + __ldg(v + s.w)) + w1 * (__ldg(v + s.y) + __ldg(v + s.z));
  };
  R m[5], f[27], g[27];
#pragma unroll
  for (int c = 0; c < 5; ++c) m[c] = ip(c);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = ip(5 + i);
    g[i] = ip(32 + i);
  });
  const R rho_t = m[0], rho = R(1) + rho_t, ux = m[1], uy = m[2], uz = m[3], T_d = m[4];
  // 2 rho E - 1 = rho (3 T + u^2) - 1 = rho_t + rho (3 (T - T0) + u^2)
  const R e_t = rho_t + rho * (R(3) * T_d + ux * ux + uy * uy + uz * uz);
  R fe[27], ge[27];
  feq_dev(rho_t, rho, ux, uy, uz, fe);
  geq_dev(rho_t, rho, ux, uy, uz, e_t, ge);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] += fe[i];
    g[i] += ge[i];
  });
  thermal_collide<R>(f, g, tc.beta, tc.beta1, tc.glam, tc.tref_d, tc.lbgk != 0, tc.pr_gt1 != 0);
  store2(pc, fo_c, go_c, ex_node[k], f, g);
}

template <typename R>
__global__ void k_th_init(PatchDev p, R* __restrict__ f0, R* __restrict__ f1, R* __restrict__ g0,
                          R* __restrict__ g1, const void* rho_in, const void* u_in, const void* T_in, int dtype,
                          R uix, R uiy, R uiz) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const long long d = ((long long)z * p.dim[1] + y) * p.dim[0] + x;
  const long long nd = (long long)p.dim[0] * p.dim[1] * p.dim[2];
  const uint8_t t = p.type[own];
  R rho = 1, ux = 0, uy = 0, uz = 0, T = R(1.0 / 3.0);
  auto ld = [&](const void* a, long long i) -> R {
    return dtype == 1 ? (R)((const double*)a)[i] : (R)((const float*)a)[i];
  };
  if (t == T_INLET) {
    ux = uix, uy = uiy, uz = uiz;
  } else if (t != T_SKIP && t != T_SOLID) {
    rho = ld(rho_in, d);
    ux = ld(u_in, d), uy = ld(u_in, nd + d), uz = ld(u_in, 2 * nd + d);
    if (T_in) T = ld(T_in, d);
  }
  const R rho_t = rho - R(1);
  const R e_t = rho_t + rho * (R(3) * (T - R(1.0 / 3.0)) + ux * ux + uy * uy + uz * uz);
  R fe[27], ge[27];
  feq_dev(rho_t, rho, ux, uy, uz, fe);
  geq_dev(rho_t, rho, ux, uy, uz, e_t, ge);
  store2(p, f0, g0, own, fe, ge);
  store2(p, f1, g1, own, fe, ge);
}

template <typename R>
__global__ void k_th_moments(PatchDev p, const R* __restrict__ fin, const R* __restrict__ gin, void* rho_o,
                             void* u_o, void* T_o, void* gamma_o, int dtype, ThParams<R> tp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const long long d = ((long long)z * p.dim[1] + y) * p.dim[0] + x;
  const long long nd = (long long)p.dim[0] * p.dim[1] * p.dim[2];
  const uint8_t t = p.type[own];
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (t != T_SKIP && t != T_SOLID) {
    R f[27], g[27];
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      f[i] = fin[(long long)i * p.plane + own];
      g[i] = gin[(long long)i * p.plane + own];
    });
    ThState<R> s;
    thermal_state(f, g, s);
    const double duz = (double)tp.glam * ((double)s.T_d - (double)tp.tref_d);
    v[0] = 1.0 + (double)s.rho_t;
    v[1] = s.ux;
    v[2] = s.uy;
    v[3] = (double)s.uz + 0.5 * duz;
    v[4] = 1.0 / 3.0 + (double)s.T_d;
    if (gamma_o) v[5] = thermal_collide<R>(f, g, tp.beta, tp.beta1, tp.glam, tp.tref_d, tp.lbgk != 0, tp.pr_gt1 != 0);
  }
  auto st = [&](void* a, long long i, double val) {
    if (!a) return;
    if (dtype == 1) ((double*)a)[i] = val;
    else ((float*)a)[i] = (float)val;
  };
  st(rho_o, d, v[0]);
  if (u_o)
    for (int a = 0; a < 3; ++a) st(u_o, a * nd + d, v[1 + a]);
  st(T_o, d, v[4]);
  st(gamma_o, d, v[5]);
}

// ---------------------------------------------------------------------------
cudaError_t launch_th_tiles(int storage, const PatchDev& p, const void* fin, const void* gin, void* fout, void* gout,
                            const uint32_t* tiles, int64_t ntiles, int ntx, const ThermalLevel& L, int odd,
                            int* status, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_th_tiles<R><<<(unsigned)ntiles, 128, 0, st>>>(p, (const R*)fin, (const R*)gin, (R*)fout, (R*)gout, tiles, ntx,
                                                    th_params<R>(L), odd, status);
    return cudaGetLastError();
  });
}

cudaError_t launch_th_coalesce(int storage, const PatchDev& child, const void* fin_c, const void* gin_c,
                               const PatchDev& parent, void* fo_p, void* go_p, const uint32_t* cf_parent,
                               const uint32_t* cf_child, int64_t n, double ff, double fg, const ThermalLevel& Lc,
                               const ThermalLevel& Lp, int* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_th_coalesce<R><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
        child, (const R*)fin_c, (const R*)gin_c, parent, (R*)fo_p, (R*)go_p, cf_parent, cf_child, n, (R)ff, (R)fg,
        th_params<R>(Lc), th_params<R>(Lp), status);
    return cudaGetLastError();
  });
}

cudaError_t launch_th_samples(int storage, const PatchDev& parent, const void* fin_p, const void* gin_p,
                              const PatchDev& child, const void* fin_c, const void* gin_c, const uint32_t* smp_node,
                              const uint8_t* smp_kind, int64_t ns, void* smp_val, int64_t ld, double ff, double fg,
                              const ThermalLevel& Lp, const ThermalLevel& Lc, int* status, cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_th_samples<R><<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(
        parent, (const R*)fin_p, (const R*)gin_p, child, (const R*)fin_c, (const R*)gin_c, smp_node, smp_kind, ns,
        (R*)smp_val, ld, (R)ff, (R)fg, th_params<R>(Lp), th_params<R>(Lc), status);
    return cudaGetLastError();
  });
}

cudaError_t launch_th_explode(int storage, const PatchDev& child, void* fo_c, void* go_c, const uint32_t* ex_node,
                              const uint32_t* ex_src, int64_t n_one, int64_t n, const void* val, int64_t ld,
                              const ThermalLevel& Lc, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_th_explode<R><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(child, (R*)fo_c, (R*)go_c, ex_node,
                                                                 (const uint4*)ex_src, n_one, n, (const R*)val, ld,
                                                                 th_params<R>(Lc));
    return cudaGetLastError();
  });
}

cudaError_t launch_th_init(int storage, const PatchDev& p, void* f0, void* f1, void* g0, void* g1, const void* rho,
                           const void* u, const void* T, int dtype, const double u_in[3], cudaStream_t st) {
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_th_init<R><<<grid, block, 0, st>>>(p, (R*)f0, (R*)f1, (R*)g0, (R*)g1, rho, u, T, dtype, (R)u_in[0],
                                         (R)u_in[1], (R)u_in[2]);
    return cudaGetLastError();
  });
}

cudaError_t launch_th_moments(int storage, const PatchDev& p, const void* fin, const void* gin, void* rho, void* u,
                              void* T, void* gamma, int dtype, const ThermalLevel& L, cudaStream_t st) {
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_th_moments<R><<<grid, block, 0, st>>>(p, (const R*)fin, (const R*)gin, rho, u, T, gamma, dtype,
                                            th_params<R>(L));
    return cudaGetLastError();
  });
}

}  // namespace lbmk
