// CUDA kernels of the refined KBC step (isothermal model).
//
// One instant of the refined step runs, per active patch:
//   k_stream_collide  pull-stream + KBC collide + force of every node whose
//                     pull sources are valid (Eq. f_equations; Sec. III.C step 1
//                     and the stream+collide of steps 2 and 5 fused),
//   k_coalesce        parent twins x_t,cf <- child state rescaled fine->coarse
//                     (Eq. f_neq_rescaling_iso inverted), then collide,
//   k_samples         reconstruction samples: pre-collision rho, u and the
//                     child-scale non-equilibrium part at parent positions,
//   k_points          intermediate points of the separable tensor interpolation,
//   k_explode         child twins x_t,fc and reconstruction nodes x_r
//                     (Eq. interp, tensor four-point Lagrange), then collide.
// Kernels of one instant read only the previous states and write disjoint
// nodes of the next-state buffers, so they need no ordering among themselves
// except samples, then the point stages, before explode.
#include <type_traits>

#include "../../include/lbm.h"
#include "collide.cuh"
#include "device.cuh"
#include "kernels.h"

namespace lbmk {

template <typename T>
struct tag {
  using type = T;
};

template <typename F>
cudaError_t dispatch(int storage, F&& f) {
  switch (storage) {
    case LBM_FP64:
      return f(tag<double>{}, tag<double>{});
    case LBM_FP32:
      return f(tag<float>{}, tag<float>{});
    case LBM_FP16_SHIFT:
      return f(tag<__half>{}, tag<float>{});
    case LBM_BF16_SHIFT:
      return f(tag<__nv_bfloat16>{}, tag<float>{});
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename S, typename R>
__device__ __forceinline__ void store_node(const PatchDev& p, S* __restrict__ fout, long long own, const R (&f)[27]) {
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Stor<S>::st(fout + (long long)i * p.plane + own, f[i]);
  });
}

template <typename S, typename R>
__device__ __forceinline__ void pull_any(const PatchDev& p, const S* __restrict__ fin, long long node, R (&f)[27],
                                         int* status) {
  const int x = (int)(node % p.nxp);
  const int y = (int)((node / p.nxp) % p.dim[1]);
  const int z = (int)(node / ((long long)p.nxp * p.dim[1]));
  if (p.type[node] == T_BULK) pull_bulk<S, R>(p, fin, x, y, z, f);
  else pull_generic<S, R>(p, fin, x, y, z, f, status);
}

// ---------------------------------------------------------------------------
// Fine -> coarse twin coupling: pre-collision child state at the coinciding
// node, non-equilibrium scaled by r beta_f / beta_c, collided with beta_c.
template <typename S, typename R, int FM>
__global__ void __launch_bounds__(128) k_coalesce(PatchDev pc, const S* __restrict__ fin_c, PatchDev pp,
                                                  S* __restrict__ fout_p, const uint32_t* __restrict__ cf_parent,
                                                  const uint32_t* __restrict__ cf_child, long long n, R rescale,
                                                  R beta_p, R dux, R duy, R duz, int lbgk, int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  R f[27];
  pull_any<S, R>(pc, fin_c, cf_child[k], f, status);
  R rho_t, rho, ux, uy, uz, fe[27];
  macro(f, rho_t, rho, ux, uy, uz);
  feq_dev(rho_t, rho, ux, uy, uz, fe);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = fe[i] + rescale * (f[i] - fe[i]);
  });
  kbc_collide<R, FM>(f, beta_p, dux, duy, duz, lbgk != 0);
  store_node<S, R>(pp, fout_p, cf_parent[k], f);
}

cudaError_t launch_coalesce(int storage, const PatchDev& child, const void* fin_child, const PatchDev& parent,
                            void* fout_parent, const uint32_t* cf_parent, const uint32_t* cf_child, int64_t n,
                            double rescale, double beta_parent, const Force& Fp, int lbgk, int* status,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((unsigned)((n + 127) / 128));
    auto go = [&](auto kern) {
      kern<<<grid, block, 0, st>>>(child, (const S*)fin_child, parent, (S*)fout_parent, cf_parent, cf_child, n,
                                   (R)rescale, (R)beta_parent, (R)Fp.du[0], (R)Fp.du[1], (R)Fp.du[2], lbgk, status);
    };
    switch (Fp.mask()) {
      case 0: go(k_coalesce<S, R, 0>); break;
      case 1: go(k_coalesce<S, R, 1>); break;
      case 4: go(k_coalesce<S, R, 4>); break;
      default: go(k_coalesce<S, R, 7>);
    }
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// Reconstruction samples: [31][ld] = rho - 1, ux, uy, uz, neq_0..26 (child
// scale), columns [0, ns) of the point space.
template <typename S, typename R>
__global__ void __launch_bounds__(128) k_samples(PatchDev pp, const S* __restrict__ fin_p, PatchDev pc,
                                                 const S* __restrict__ fin_c, const uint32_t* __restrict__ smp_node,
                                                 const uint8_t* __restrict__ smp_kind, long long ns,
                                                 R* __restrict__ out, long long ld, R rescale_p, int* status) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  R f[27];
  R factor;
  if (smp_kind[s] == 0) {
    pull_any<S, R>(pp, fin_p, smp_node[s], f, status);
    factor = rescale_p;
  } else {
    pull_any<S, R>(pc, fin_c, smp_node[s], f, status);
    factor = R(1);
  }
  R rho_t, rho, ux, uy, uz, fe[27];
  macro(f, rho_t, rho, ux, uy, uz);
  feq_dev(rho_t, rho, ux, uy, uz, fe);
  out[s] = rho_t;
  out[ld + s] = ux;
  out[2 * ld + s] = uy;
  out[3 * ld + s] = uz;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    out[(4 + i) * ld + s] = factor * (f[i] - fe[i]);
  });
}

cudaError_t launch_samples(int storage, const PatchDev& parent, const void* fin_parent, const PatchDev& child,
                           const void* fin_child, const uint32_t* smp_node, const uint8_t* smp_kind, int64_t ns,
                           void* smp_val, int64_t ld, double rescale_parent, int* status, cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((unsigned)((ns + 127) / 128));
    k_samples<S, R><<<grid, block, 0, st>>>(parent, (const S*)fin_parent, child, (const S*)fin_child, smp_node,
                                            smp_kind, ns, (R*)smp_val, ld, (R)rescale_parent, status);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// Intermediate reconstruction points: four-point Lagrange (Eq. interp,
// weights (-1, 9, 9, -1)/16) along one axis of NC values per point,
// val[c][out0 + q] = sum_k w_k val[c][src[4q + k]].  The tensor interpolation
// over two or three off-lattice axes is this one-axis pass applied axis after
// axis (stage 1 from the samples, stage 2 from stage 1, the targets last).
// Large passes: one thread per point, all its values (enough points to fill
// the GPU, and the four source indices are read once).
template <typename R, int NC>
__global__ void __launch_bounds__(128) k_points(const uint4* __restrict__ src, long long n, R* __restrict__ val,
                                                long long ld, long long out0) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint4 s = __ldg(src + q);
  const R w0 = R(-1.0 / 16.0), w1 = R(9.0 / 16.0);
#pragma unroll 4
  for (int c = 0; c < NC; ++c) {
    // the columns read are never written by this pass: read-only cache path
    const R* v = val + (long long)c * ld;
    const R a = __ldg(v + s.x), b = __ldg(v + s.y), d = __ldg(v + s.z), e = __ldg(v + s.w);
    val[(long long)c * ld + out0 + q] = w0 * (a + e) + w1 * (b + d);
  }
}

// Small passes: one thread per (point, value), a single round trip to the
// four sources, so that a pass of a few thousand points is not latency-bound.
template <typename R>
__global__ void __launch_bounds__(128) k_points_small(const uint4* __restrict__ src, long long n,
                                                      R* __restrict__ val, long long ld, long long out0) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint4 s = __ldg(src + q);
  const R w0 = R(-1.0 / 16.0), w1 = R(9.0 / 16.0);
  R* v = val + (long long)blockIdx.y * ld;
  const R a = __ldg(v + s.x), b = __ldg(v + s.y), d = __ldg(v + s.z), e = __ldg(v + s.w);
  v[out0 + q] = w0 * (a + e) + w1 * (b + d);
}

cudaError_t launch_points(int storage, int ncomp, const uint32_t* pt_src, int64_t n, void* val, int64_t ld,
                          int64_t out0, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (ncomp != 31 && ncomp != 59) return cudaErrorInvalidValue;
  return dispatch(storage, [&](auto, auto tr) {
    using R = typename decltype(tr)::type;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    if (n < 65536) {
      k_points_small<R><<<dim3(blocks, (unsigned)ncomp), 128, 0, st>>>((const uint4*)pt_src, n, (R*)val, ld, out0);
    } else if (ncomp == 31) {
      k_points<R, 31><<<blocks, 128, 0, st>>>((const uint4*)pt_src, n, (R*)val, ld, out0);
    } else {
      k_points<R, 59><<<blocks, 128, 0, st>>>((const uint4*)pt_src, n, (R*)val, ld, out0);
    }
    return cudaGetLastError();
  });
}

// Child twins and reconstruction nodes: the last interpolation pass (or the
// point itself), f = f^eq(rho~, u~) + neq~, then collide.  The collision
// starts from df = neq~ and the moments (rho~, u~) directly: f^eq(rho~, u~) +
// neq~ has these moments (the product-form equilibrium carries the node's mass
// and momentum exactly, and neq~ interpolates states without any), so its
// df is neq~ up to rounding.  Targets [0, n_one) read one point, the others
// interpolate four; a thread block takes targets of one kind only.
template <int K, typename S, typename R, int FM>
__device__ __forceinline__ void explode_node(const PatchDev& pc, S* __restrict__ fout_c,
                                             const uint32_t* __restrict__ ex_node, const uint4* __restrict__ ex_src,
                                             long long k, const R* __restrict__ val, long long ld, R beta_c, R dux,
                                             R duy, R duz, int lbgk) {
  const uint4 s = __ldg(ex_src + k);
  R m[4], f[27];
  if constexpr (K == 1) {
#pragma unroll
    for (int c = 0; c < 4; ++c) m[c] = __ldg(val + c * ld + s.x);
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      f[i] = __ldg(val + (4 + i) * ld + s.x);
    });
  } else {
    const R w0 = R(-1.0 / 16.0), w1 = R(9.0 / 16.0);
    auto ip = [&](int c) {
      const R* v = val + (long long)c * ld;
      return w0 * (__ldg(v + s.x) + __ldg(v + s.w)) + w1 * (__ldg(v + s.y) + __ldg(v + s.z));
    };
#pragma unroll
    for (int c = 0; c < 4; ++c) m[c] = ip(c);
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      f[i] = ip(4 + i);
    });
  }
  kbc_collide_m<R, FM, true>(f, m[0], R(1) + m[0], m[1], m[2], m[3], beta_c, dux, duy, duz, lbgk != 0);
  store_node<S, R>(pc, fout_c, __ldg(ex_node + k), f);
}

template <typename S, typename R, int FM>
__global__ void __launch_bounds__(128, 7) k_explode(PatchDev pc, S* __restrict__ fout_c,
                                                 const uint32_t* __restrict__ ex_node,
                                                 const uint4* __restrict__ ex_src, long long n_one, long long n,
                                                 unsigned blocks_one, const R* __restrict__ val, long long ld,
                                                 R beta_c, R dux, R duy, R duz, int lbgk) {
  if (blockIdx.x < blocks_one) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_one) explode_node<1, S, R, FM>(pc, fout_c, ex_node, ex_src, k, val, ld, beta_c, dux, duy, duz, lbgk);
  } else {
    const long long k = n_one + (long long)(blockIdx.x - blocks_one) * blockDim.x + threadIdx.x;
    if (k < n) explode_node<4, S, R, FM>(pc, fout_c, ex_node, ex_src, k, val, ld, beta_c, dux, duy, duz, lbgk);
  }
}

cudaError_t launch_explode(int storage, const PatchDev& child, void* fout_child, const uint32_t* ex_node,
                           const uint32_t* ex_src, int64_t n_one, int64_t n, const void* val, int64_t ld,
                           double beta_child, const Force& Fc, int lbgk, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned b1 = (unsigned)((n_one + 127) / 128), b4 = (unsigned)((n - n_one + 127) / 128);
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid(b1 + b4);
    auto go = [&](auto kern) {
      kern<<<grid, block, 0, st>>>(child, (S*)fout_child, ex_node, (const uint4*)ex_src, n_one, n, b1, (const R*)val,
                                   ld, (R)beta_child, (R)Fc.du[0], (R)Fc.du[1], (R)Fc.du[2], lbgk);
    };
    switch (Fc.mask()) {
      case 0: go(k_explode<S, R, 0>); break;
      case 1: go(k_explode<S, R, 1>); break;
      case 4: go(k_explode<S, R, 4>); break;
      default: go(k_explode<S, R, 7>);
    }
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ double ldv(const void* p, long long i) {
  return (double)((const V*)p)[i];
}

template <typename S, typename R>
__global__ void k_init(PatchDev p, S* __restrict__ f0, S* __restrict__ f1, const void* rho_in, const void* u_in,
                       int dtype, R uix, R uiy, R uiz) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const long long d = ((long long)z * p.dim[1] + y) * p.dim[0] + x;
  const long long nd = (long long)p.dim[0] * p.dim[1] * p.dim[2];
  const uint8_t t = p.type[own];
  R rho = 1, ux = 0, uy = 0, uz = 0;
  if (t == T_INLET) {
    ux = uix;
    uy = uiy;
    uz = uiz;
  } else if (t != T_SKIP && t != T_SOLID) {
    if (dtype == 1) {
      rho = (R)ldv<double>(rho_in, d);
      ux = (R)ldv<double>(u_in, d);
      uy = (R)ldv<double>(u_in, nd + d);
      uz = (R)ldv<double>(u_in, 2 * nd + d);
    } else {
      rho = (R)ldv<float>(rho_in, d);
      ux = (R)ldv<float>(u_in, d);
      uy = (R)ldv<float>(u_in, nd + d);
      uz = (R)ldv<float>(u_in, 2 * nd + d);
    }
  }
  R fe[27];
  feq_dev(rho - R(1), rho, ux, uy, uz, fe);
  store_node<S, R>(p, f0, own, fe);
  store_node<S, R>(p, f1, own, fe);
}

cudaError_t launch_init(int storage, const PatchDev& p, void* f0, void* f1, const void* rho, const void* u,
                        int dtype, const double u_in[3], cudaStream_t st) {
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_init<S, R><<<grid, block, 0, st>>>(p, (S*)f0, (S*)f1, rho, u, dtype, (R)u_in[0], (R)u_in[1], (R)u_in[2]);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
template <typename S, typename R>
__device__ __forceinline__ void load_node(const PatchDev& p, const S* __restrict__ fin, long long own,
                                          R (&f)[27]) {
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = Stor<S>::ld(fin + (long long)i * p.plane + own);
  });
}

// ---------------------------------------------------------------------------
// State transfer onto another layout (regridding; the paper leaves adaptive
// refinement to future work).  Each node of the destination patch takes the
// state of the source level nearest its own that holds it (the host orders
// the source patches: own level, finer nearest first, coarser nearest first):
// the coinciding node when that level is as fine or finer, else a trilinear
// interpolation of rho, u and f - f^eq over the corners of non-zero weight of
// the source cell around it.  The stored (post-collision) f - f^eq is scaled
// by (1 - 2 beta_t)/(1 - 2 beta_s) beta_s/(r beta_t), r = dx_s / dx_t (Eq.
// f_neq_rescaling_iso for the pre-collision part, times the post-collision
// factor of each level), and dropped where 1 - 2 beta_s vanishes.  Solid and
// hole nodes take the rest state, inlet nodes the inflow equilibrium; both
// destination buffers are written.  Nodes no source level holds take the rest
// state and are counted in *missing.
template <typename S, typename R>
__device__ __forceinline__ bool src_node(const TransferSrc& T, int k, long long Y0, long long Y1, long long Y2,
                                         long long& idx) {
  const PatchDev& q = T.p[k];
  long long Y[3] = {Y0, Y1, Y2};
  for (int a = 0; a < 3; ++a) {
    if (T.periodic[a]) {
      const long long P = (long long)T.n[a] << T.level[k];
      Y[a] = ((Y[a] % P) + P) % P;
    }
    Y[a] -= q.org[a];
    if (Y[a] < 0 || Y[a] >= q.dim[a]) return false;
  }
  idx = node_index(q, (int)Y[0], (int)Y[1], (int)Y[2]);
  const uint8_t t = q.type[idx];
  return t != T_SKIP && t != T_SOLID;
}

template <typename S, typename R>
__global__ void __launch_bounds__(128) k_transfer(PatchDev p, S* __restrict__ f0, S* __restrict__ f1, int level,
                                                  R beta_t, R uix, R uiy, R uiz, TransferSrc T,
                                                  unsigned long long* missing) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const uint8_t t = p.type[own];
  R fo[27];
  if (t == T_SKIP || t == T_SOLID || t == T_INLET) {
    const bool in = t == T_INLET;
    feq_dev(R(0), R(1), in ? uix : R(0), in ? uiy : R(0), in ? uiz : R(0), fo);
    store_node<S, R>(p, f0, own, fo);
    store_node<S, R>(p, f1, own, fo);
    return;
  }
  const long long X[3] = {(long long)p.org[0] + x, (long long)p.org[1] + y, (long long)p.org[2] + z};
  bool done = false;
  for (int o = 0; o < T.n_src && !done; ++o) {
    const int k = T.order[o];
    const int dl = T.level[k] - level;
    R rt = 0, ux = 0, uy = 0, uz = 0, neq[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) neq[i] = 0;
    bool ok = true;
    if (dl >= 0) {
      long long n;
      const long long sc = 1LL << dl;
      ok = src_node<S, R>(T, k, X[0] * sc, X[1] * sc, X[2] * sc, n);
      if (ok) {
        R f[27], fe[27];
        load_node<S, R>(T.p[k], static_cast<const S*>(T.f[k]), n, f);
        R rho;
        macro(f, rt, rho, ux, uy, uz);
        feq_dev(rt, rho, ux, uy, uz, fe);
#pragma unroll
        for (int i = 0; i < 27; ++i) neq[i] = f[i] - fe[i];
      }
    } else {
      const long long sdiv = 1LL << (-dl);
      long long base[3];
      R fr[3];
      for (int a = 0; a < 3; ++a) {
        base[a] = X[a] >= 0 ? X[a] / sdiv : -((-X[a] + sdiv - 1) / sdiv);
        fr[a] = (R)(double)(X[a] - base[a] * sdiv) / (R)(double)sdiv;
      }
      for (int c = 0; c < 8 && ok; ++c) {
        R w = 1;
        long long Y[3];
        for (int a = 0; a < 3; ++a) {
          const int bit = (c >> a) & 1;
          w *= bit ? fr[a] : R(1) - fr[a];
          Y[a] = base[a] + bit;
        }
        if (w == R(0)) continue;
        long long n;
        if (!src_node<S, R>(T, k, Y[0], Y[1], Y[2], n)) {
          ok = false;
          break;
        }
        R f[27], fe[27], r1, rho1, u1x, u1y, u1z;
        load_node<S, R>(T.p[k], static_cast<const S*>(T.f[k]), n, f);
        macro(f, r1, rho1, u1x, u1y, u1z);
        feq_dev(r1, rho1, u1x, u1y, u1z, fe);
        rt += w * r1;
        ux += w * u1x;
        uy += w * u1y;
        uz += w * u1z;
#pragma unroll
        for (int i = 0; i < 27; ++i) neq[i] += w * (f[i] - fe[i]);
      }
    }
    if (!ok) continue;
    const double r = ldexp(1.0, -dl);  // dx_s / dx_t
    const double bs = T.beta[k], post_s = 1.0 - 2.0 * bs, post_t = 1.0 - 2.0 * (double)beta_t;
    const R factor = fabs(post_s) < 1e-12 ? R(0) : (R)((post_t / post_s) * bs / (r * (double)beta_t));
    feq_dev(rt, R(1) + rt, ux, uy, uz, fo);
#pragma unroll
    for (int i = 0; i < 27; ++i) fo[i] += factor * neq[i];
    done = true;
  }
  if (!done) {
    feq_dev(R(0), R(1), R(0), R(0), R(0), fo);
    atomicAdd(missing, 1ull);
  }
  store_node<S, R>(p, f0, own, fo);
  store_node<S, R>(p, f1, own, fo);
}

cudaError_t launch_transfer(int storage, const PatchDev& p, void* f0, void* f1, int level, double beta,
                            const double u_in[3], const TransferSrc& T, unsigned long long* missing,
                            cudaStream_t st) {
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_transfer<S, R><<<grid, block, 0, st>>>(p, (S*)f0, (S*)f1, level, (R)beta, (R)u_in[0], (R)u_in[1],
                                             (R)u_in[2], T, missing);
    return cudaGetLastError();
  });
}

template <typename V>
__device__ __forceinline__ void stv(void* p, long long i, double v) {
  ((V*)p)[i] = (V)v;
}

template <typename S, typename R>
__global__ void k_moments(PatchDev p, const S* __restrict__ fin, void* rho_o, void* u_o, void* gamma_o, int dtype,
                          R beta, R dux, R duy, R duz, int lbgk) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const long long d = ((long long)z * p.dim[1] + y) * p.dim[0] + x;
  const long long nd = (long long)p.dim[0] * p.dim[1] * p.dim[2];
  const uint8_t t = p.type[own];
  double vals[5] = {0, 0, 0, 0, 0};
  if (t != T_SKIP && t != T_SOLID) {
    R f[27];
    load_node<S, R>(p, fin, own, f);
    R rho_t, rho, ux, uy, uz;
    macro(f, rho_t, rho, ux, uy, uz);
    vals[0] = (double)rho_t + 1.0;
    vals[1] = ux + R(0.5) * dux;
    vals[2] = uy + R(0.5) * duy;
    vals[3] = uz + R(0.5) * duz;
    if (gamma_o) vals[4] = kbc_collide<R, 0>(f, beta, R(0), R(0), R(0), lbgk != 0);
  }
  if (dtype == 1) {
    if (rho_o) stv<double>(rho_o, d, vals[0]);
    if (u_o)
      for (int a = 0; a < 3; ++a) stv<double>(u_o, a * nd + d, vals[1 + a]);
    if (gamma_o) stv<double>(gamma_o, d, vals[4]);
  } else {
    if (rho_o) stv<float>(rho_o, d, vals[0]);
    if (u_o)
      for (int a = 0; a < 3; ++a) stv<float>(u_o, a * nd + d, vals[1 + a]);
    if (gamma_o) stv<float>(gamma_o, d, vals[4]);
  }
}

cudaError_t launch_moments(int storage, const PatchDev& p, const void* fin, void* rho, void* u, void* gamma,
                           int dtype, double beta, const Force& F, int lbgk, cudaStream_t st) {
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_moments<S, R><<<grid, block, 0, st>>>(p, (const S*)fin, rho, u, gamma, dtype, (R)beta, (R)F.du[0],
                                            (R)F.du[1], (R)F.du[2], lbgk);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// Refinement indicator: per block of B^3 nodes of the storage box, the largest
// |gamma - 2| over its bulk and boundary-class nodes, gamma from Eq.
// gamma_min_approx for the state the next stream-collide collides there (the
// pull of the stored post-collision state; a post-collision state itself has
// gamma = 2 exactly).  The stabiliser tends to its LBGK value 2 where the flow
// is resolved, so its deviation measures under-resolution (Sec. IV, channel;
// the conclusion proposes it as the criterion of adaptive refinement).
// Interface nodes, whose next state comes from the coupling, are left out.
// out [nbz][nby][nbx] is zeroed first; maxima of non-negative floats combine
// as integer maxima of their bits.
template <typename S, typename R>
__global__ void __launch_bounds__(128) k_gamma_blocks(PatchDev p, const S* __restrict__ fin, R beta, int lbgk, int B,
                                                      int nbx, int nby, float* __restrict__ out, int* status) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  float dev = 0.0f;
  if (x < p.dim[0]) {
    const long long own = node_index(p, x, y, z);
    const uint8_t t = p.type[own];
    if (t == T_BULK || t == T_BC) {
      R f[27];
      if (t == T_BULK) pull_bulk<S, R>(p, fin, x, y, z, f);
      else pull_generic<S, R>(p, fin, x, y, z, f, status);
      const R gamma = kbc_collide<R, 0>(f, beta, R(0), R(0), R(0), lbgk != 0);
      dev = (float)fabs((double)gamma - 2.0);
    }
  }
  // lanes of a warp share y and z; reduce the runs of equal x-block first
  const int bx = x / B;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int bx0 = __shfl_sync(full, bx, 0);
  const int bx31 = __shfl_sync(full, bx, 31);
  if (bx0 == bx31) {
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(full, dev, o));
    if (lane != 0) return;
  }
  if (x >= p.dim[0] || dev <= 0.0f) return;
  const long long b = ((long long)(z / B) * nby + (y / B)) * nbx + bx;
  atomicMax(reinterpret_cast<int*>(out) + b, __float_as_int(dev));
}

cudaError_t launch_gamma_blocks(int storage, const PatchDev& p, const void* fin, double beta, int lbgk, int B,
                                float* out, int* status, cudaStream_t st) {
  const int nbx = (p.dim[0] + B - 1) / B, nby = (p.dim[1] + B - 1) / B, nbz = (p.dim[2] + B - 1) / B;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)nbx * nby * nbz, st);
  if (e) return e;
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_gamma_blocks<S, R><<<grid, block, 0, st>>>(p, (const S*)fin, (R)beta, lbgk, B, nbx, nby, out, status);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
template <typename S, typename R>
__global__ void k_copy_pop(PatchDev p, S* fstore, void* dense, int dtype, int to_dense, int gset) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const long long d = ((long long)z * p.dim[1] + y) * p.dim[0] + x;
  const long long nd = (long long)p.dim[0] * p.dim[1] * p.dim[2];
  for (int i = 0; i < 27; ++i) {
    const int c2 = (i % 3 != 1) + ((i / 3) % 3 != 1) + (i / 9 != 1);
    const double w = gset ? wi_rt(i) * c2 : wi_rt(i);
    if (to_dense) {
      const double v = (double)Stor<S>::ld(fstore + (long long)i * p.plane + own) + w;
      if (dtype == 1) ((double*)dense)[i * nd + d] = v;
      else ((float*)dense)[i * nd + d] = (float)v;
    } else {
      const double v = dtype == 1 ? ((const double*)dense)[i * nd + d] : (double)((const float*)dense)[i * nd + d];
      Stor<S>::st(fstore + (long long)i * p.plane + own, (R)(v - w));
    }
  }
}

cudaError_t launch_copy_pop(int storage, const PatchDev& p, void* fstore, void* dense, int dtype, int to_dense,
                            int gset, cudaStream_t st) {
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    dim3 block(128), grid((p.dim[0] + 127) / 128, p.dim[1], p.dim[2]);
    k_copy_pop<S, R><<<grid, block, 0, st>>>(p, (S*)fstore, dense, dtype, to_dense, gset);
    return cudaGetLastError();
  });
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: fixed grid of blocks, fixed-order reductions (deterministic).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

template <typename S, typename R>
__global__ void __launch_bounds__(256) k_diag(PatchDev p, const S* __restrict__ fin, double vw, R dux, R duy,
                                              R duz, double* __restrict__ partial) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  double mn = 1e300;
  double bad = 0;
  const long long total = p.plane;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < total;
       n += (long long)gridDim.x * blockDim.x) {
    const uint8_t t = p.type[n];
    if (!(t == T_BULK || t == T_BC || t == T_D1 || t == T_INLET)) continue;
    R f[27];
    load_node<S, R>(p, fin, n, f);
    R rho_t, rho, ux, uy, uz;
    macro(f, rho_t, rho, ux, uy, uz);
    const double r = 1.0 + (double)rho_t;
    const double u[3] = {(double)ux + 0.5 * (double)dux, (double)uy + 0.5 * (double)duy,
                         (double)uz + 0.5 * (double)duz};
    if (!(r > 0.0) || !isfinite(r)) bad += 1.0;
    acc[0] += vw * r;
    acc[1] += vw * r * u[0];
    acc[2] += vw * r * u[1];
    acc[3] += vw * r * u[2];
    acc[4] += vw * 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    acc[5] += 1.0;
    mn = fmin(mn, r);
  }
  __shared__ double sh[8][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v[8];
  for (int k = 0; k < 6; ++k) v[k] = warp_sum(acc[k]);
  v[6] = warp_min(mn);
  v[7] = warp_sum(bad);
  if (lane == 0)
    for (int k = 0; k < 8; ++k) sh[wid][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    double s = (k == 6) ? 1e300 : 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = (k == 6) ? fmin(s, sh[w][k]) : s + sh[w][k];
    partial[blockIdx.x * 8 + k] = s;
  }
}

cudaError_t launch_diag(int storage, const PatchDev& p, const void* fin, double vol_weight, const Force& F,
                        double* partial, int blocks, cudaStream_t st) {
  return dispatch(storage, [&](auto ts, auto tr) {
    using S = typename decltype(ts)::type;
    using R = typename decltype(tr)::type;
    k_diag<S, R><<<blocks, 256, 0, st>>>(p, (const S*)fin, vol_weight, (R)F.du[0], (R)F.du[1], (R)F.du[2],
                                          partial);
    return cudaGetLastError();
  });
}

__global__ void k_diag_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  if (threadIdx.x >= 8) return;
  const int k = threadIdx.x;
  double s = (k == 6) ? 1e300 : 0.0;
  for (int b = 0; b < nb; ++b) s = (k == 6) ? fmin(s, partial[b * 8 + k]) : s + partial[b * 8 + k];
  out[k] = s;
}

__global__ void k_status_clear(int* status, int bits) { atomicAnd(status, ~bits); }

cudaError_t launch_status_clear(int* status, int bits, cudaStream_t st) {
  k_status_clear<<<1, 1, 0, st>>>(status, bits);
  return cudaGetLastError();
}

cudaError_t launch_diag_final(const double* partial, int total_blocks, double* out8, cudaStream_t st) {
  k_diag_final<<<1, 32, 0, st>>>(partial, total_blocks, out8);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Momentum exchange of half-way bounce-back (drag of Sec. IV A 2): every link
// from a fluid node x to a solid neighbour x + c_j hands the solid 2 c_j f'_j(x)
// per substep; scale = 4^-level converts to coarse units.  FP64 per-block sums.
template <typename S>
__global__ void __launch_bounds__(256) k_drag(PatchDev p, const S* __restrict__ fin,
                                              const uint32_t* __restrict__ node, const uint32_t* __restrict__ mask,
                                              long long n, double scale, double* __restrict__ partial) {
  const long long plane = p.plane;
  double acc[3] = {0, 0, 0};
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = mask[k];
    const long long nd = node[k];
    const int X[3] = {(int)(nd % p.nxp), (int)((nd / p.nxp) % p.dim[1]), (int)(nd / ((long long)p.nxp * p.dim[1]))};
    unroll<27>([&](auto J) {
      constexpr int j = decltype(J)::value;
      if ((m >> j) & 1u) {
        // f'_j leaves along c_j, f_{-j} of the next pull comes back: c_j (f'_j + f_{-j})
        const double out = WI(j) + (double)Stor<S>::ld(fin + (long long)j * plane + nd);
        const double back = p.wq ? WI(j) + (double)returning<26 - j, S, double>(p, fin, nd, X, p.wq[27 * k + j],
                                                                                 false, 0.0)
                                 : out;
        const double f = out + back;
        if constexpr (CX(j) != 0) acc[0] += CX(j) * f;
        if constexpr (CY(j) != 0) acc[1] += CY(j) * f;
        if constexpr (CZ(j) != 0) acc[2] += CZ(j) * f;
      }
    });
  }
  __shared__ double sh[8][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double v[3];
  for (int a = 0; a < 3; ++a) v[a] = warp_sum(acc[a]);
  if (lane == 0)
    for (int a = 0; a < 3; ++a) sh[wid][a] = v[a];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    partial[blockIdx.x * 3 + threadIdx.x] = scale * t;
  }
}

__global__ void k_drag_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  if (threadIdx.x >= 3) return;
  double t = 0;
  for (int b = 0; b < nb; ++b) t += partial[b * 3 + threadIdx.x];
  out[threadIdx.x] = t;
}

cudaError_t launch_drag(int storage, const PatchDev& p, const void* fin, const uint32_t* node, const uint32_t* mask,
                        int64_t n, double scale, double* partial, int blocks, cudaStream_t st) {
  return dispatch(storage, [&](auto ts, auto) {
    using S = typename decltype(ts)::type;
    k_drag<S><<<blocks, 256, 0, st>>>(p, (const S*)fin, node, mask, n, scale, partial);
    return cudaGetLastError();
  });
}

cudaError_t launch_drag_final(const double* partial, int total_blocks, double* out3, cudaStream_t st) {
  k_drag_final<<<1, 32, 0, st>>>(partial, total_blocks, out3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_collide_nodes(const R* __restrict__ fin, R* __restrict__ fout, R* __restrict__ gam, long long n,
                                R beta, R dux, R duy, R duz, int lbgk, int force) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  R f[27];
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = fin[i * n + k] - R(WI(i));
  });
  R g = force ? kbc_collide<R, 7>(f, beta, dux, duy, duz, lbgk != 0)
              : kbc_collide<R, 0>(f, beta, dux, duy, duz, lbgk != 0);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    fout[i * n + k] = f[i] + R(WI(i));
  });
  if (gam) gam[k] = g;
}

cudaError_t launch_collide_nodes(const void* fin, void* fout, void* gamma, int64_t n, double beta, const Force& F,
                                 int lbgk, int dtype, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  dim3 block(128), grid((unsigned)((n + 127) / 128));
  if (dtype == 1)
    k_collide_nodes<double><<<grid, block, 0, st>>>((const double*)fin, (double*)fout, (double*)gamma, n, beta,
                                                    F.du[0], F.du[1], F.du[2], lbgk, F.on());
  else
    k_collide_nodes<float><<<grid, block, 0, st>>>((const float*)fin, (float*)fout, (float*)gamma, n, (float)beta,
                                                   (float)F.du[0], (float)F.du[1], (float)F.du[2], lbgk, F.on());
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Segmented device copy: blockIdx.y picks the segment; the widest access the
// segment's addresses and size allow (16, 8, 4 or 1 bytes), grid-stride.
template <typename V>
__device__ __forceinline__ void copy_words(V* __restrict__ d, const V* __restrict__ s, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    d[k] = __ldg(s + k);
}

__global__ void __launch_bounds__(256) k_copy(CopySegs segs) {
  const int j = blockIdx.y;
  void* dst = segs.rel ? (void*)(uintptr_t)(*segs.rel + (uintptr_t)segs.dst[j]) : segs.dst[j];
  const uintptr_t a = (uintptr_t)dst | (uintptr_t)segs.src[j] | (uintptr_t)segs.bytes[j];
  const size_t n = segs.bytes[j];
  if ((a & 15) == 0) copy_words((uint4*)dst, (const uint4*)segs.src[j], n / 16);
  else if ((a & 7) == 0) copy_words((uint2*)dst, (const uint2*)segs.src[j], n / 8);
  else if ((a & 3) == 0) copy_words((unsigned*)dst, (const unsigned*)segs.src[j], n / 4);
  else copy_words((unsigned char*)dst, (const unsigned char*)segs.src[j], n);
  if (segs.done) {
    // the last block advances the base word: all blocks read it before this
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned total = gridDim.x * gridDim.y;
      if (atomicAdd(segs.done, 1u) == total - 1) {
        *segs.rel += segs.advance;
        *segs.done = 0;
      }
    }
  }
}

__global__ void k_word(unsigned long long* word, unsigned long long value, int advance) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *word = advance ? *word + value : value;
    if (!advance) *reinterpret_cast<unsigned*>(word + 1) = 0;  // the copy-completion count beside it
  }
}

cudaError_t launch_word(unsigned long long* word, unsigned long long value, int advance, cudaStream_t st) {
  k_word<<<1, 32, 0, st>>>(word, value, advance);
  return cudaGetLastError();
}

cudaError_t launch_copy(const CopySegs& segs, cudaStream_t st) {
  if (segs.n <= 0) return cudaSuccess;
  if (segs.n > kCopySegs) return cudaErrorInvalidValue;
  size_t most = 0;
  for (int j = 0; j < segs.n; ++j) most = segs.bytes[j] > most ? segs.bytes[j] : most;
  if (most == 0) return cudaSuccess;
  // about four 16-byte words per thread for the largest segment, at most
  // 8 blocks per SM (152 SMs)
  size_t blocks = (most / 16 + 1023) / 1024;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_copy<<<dim3((unsigned)blocks, (unsigned)segs.n), 256, 0, st>>>(segs);
  return cudaGetLastError();
}

}  // namespace lbmk
