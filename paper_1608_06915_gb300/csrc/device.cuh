// Device-side lattice, storage conversion, pull-streaming and the KBC collision.
//
// Velocity order: i = (cx+1) + 3(cy+1) + 9(cz+1), rest 13, opposite 26 - i.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

enum : uint8_t { T_SKIP = 0, T_BULK = 1, T_BC = 2, T_D1 = 3, T_D0 = 4, T_CF = 5, T_INLET = 6, T_SOLID = 7 };

__host__ __device__ constexpr int CX(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int CY(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int i) { return i / 9 - 1; }
__host__ __device__ constexpr double W1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double WI(int i) { return W1(CX(i)) * W1(CY(i)) * W1(CZ(i)); }

// ---------------------------------------------------------------------------
// Storage: every type holds the deviation f_i - W_i from the rest state at
// unit density (16-bit types need it for their few mantissa bits; float and
// double keep 100x more absolute resolution that way).  The compute type R is
// double for double storage and float otherwise.
template <typename S>
struct Stor;
template <>
struct Stor<double> {
  static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <>
struct Stor<float> {
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Stor<__half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Stor<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

__device__ __forceinline__ double wi_rt(int i) {
  // W_i for a runtime direction index
  const int c[3] = {i % 3, (i / 3) % 3, i / 9};
  double w = 1.0;
  for (int a = 0; a < 3; ++a) w *= c[a] == 1 ? 2.0 / 3.0 : 1.0 / 6.0;
  return w;
}

// compile-time loop
template <int N, typename F, int I = 0>
__device__ __forceinline__ void unroll(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    unroll<N, F, I + 1>(static_cast<F&&>(f));
  }
}

// ---------------------------------------------------------------------------
// Patch view passed by value to kernels.
struct PatchDev {
  int dim[3];
  int org[3];
  int maxc[3];       // last domain coordinate on non-periodic axes (this level)
  int nxp;
  long long plane;   // nodes per population plane
  unsigned char span[3];
  unsigned char periodic[3];
  unsigned walls;
  int inflow;
  const uint8_t* type;
  // curved solid surface (null without one): wq_idx over the storage box, and
  // wq[27 k + j] the wall fraction of the link along c_j of node k
  const int32_t* wq_idx;
  const double* wq;
};

__device__ __forceinline__ long long node_index(const PatchDev& p, int x, int y, int z) {
  return ((long long)z * p.dim[1] + y) * p.nxp + x;
}

// ---------------------------------------------------------------------------
// Product-form equilibrium, Eq. (feq_iso), per axis and in deviation form:
//   f_i^eq = rho W_i prod_a ghat_a(c_ia),  ghat(0) = A,  ghat(+1) = A B,
//   ghat(-1) = A / B,  A = 2 - s,  B = (2u + s)/(1 - u),  s = sqrt(1 + 3u^2).
// With e = s - 1 = 3u^2/(s + 1), the deviations d = ghat - 1 are
//   d(0)  = -e,
//   d(+1) = (u (3 - 3u - 2e) + 2e) / (1 - u),
//   d(-1) = (u (e - 3) - 2e) / (2u + s),
// free of cancellation, so f^eq - W_i = W_i (rho~ + rho q_i) with
// q_i = prod_a (1 + d_a) - 1 and rho~ = rho - 1 keeps full relative accuracy.
// Division and square root: IEEE in double; in float the hardware reciprocal
// and reciprocal square root (about 2 ulp), ample for the well-conditioned
// quotients of the collision (denominators near 1).
template <typename R>
__device__ __forceinline__ R rcp_fast(R x) {
  return R(1) / x;
}
template <>
__device__ __forceinline__ float rcp_fast<float>(float x) {
  return __fdividef(1.0f, x);
}
template <typename R>
__device__ __forceinline__ R fdiv(R a, R b) {
  return a / b;
}
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) {
  return __fdividef(a, b);
}
template <typename R>
__device__ __forceinline__ R fsqrt1(R x) {  // x >= 1
  return sqrt(x);
}
template <>
__device__ __forceinline__ float fsqrt1<float>(float x) {
  return x * rsqrtf(x);
}

template <typename R>
struct AxisEq {
  R d[3];   // ghat - 1 for c = -1, 0, +1
  R ig[3];  // 1 / (W1(c) ghat(c)), weights of the entropic scalar product
  R s, B;   // s = sqrt(1 + 3u^2), B as above (for the force increment)
};

// The entropic weights need 1/ghat(c): with A = 1 - e and 1/B = (1 - u)/(2u + s),
// 1/ghat(0) = 1/A, 1/ghat(+1) = (1/A)(1/B), 1/ghat(-1) = B/A.
template <typename R>
__device__ __forceinline__ void axis_eq(R u, AxisEq<R>& a, bool want_inverse) {
  const R u2 = u * u;
  const R s = fsqrt1(R(1) + R(3) * u2);
  const R e = fdiv(R(3) * u2, s + R(1));
  const R i1mu = rcp_fast(R(1) - u);
  const R i2us = rcp_fast(R(2) * u + s);
  a.s = s;
  a.B = (R(2) * u + s) * i1mu;
  a.d[1] = -e;
  a.d[2] = (u * (R(3) - R(3) * u - R(2) * e) + R(2) * e) * i1mu;
  a.d[0] = (u * (e - R(3)) - R(2) * e) * i2us;
  if (want_inverse) {
    const R iA = rcp_fast(R(1) - e);
    a.ig[1] = R(1.5) * iA;
    a.ig[2] = R(6) * iA * ((R(1) - u) * i2us);
    a.ig[0] = R(6) * iA * a.B;
  }
}

// Increment of the per-axis factors ghat when u -> u + du, evaluated without
// cancellation: ds = 3 du (2u + du)/(s' + s), dA = -ds,
// dB = ((2 du + ds)(1 - u) + (2u + s) du) / ((1 - u - du)(1 - u)),
// d[A B] = dA B' + A dB,  d[A/B] = (dA B - A dB) / (B B').
template <typename R>
__device__ __forceinline__ void axis_eq_increment(R u, R du, const AxisEq<R>& a, R (&g1)[3], R (&dg)[3]) {
  if (du == R(0)) {  // no force along this axis
    for (int c = 0; c < 3; ++c) {
      dg[c] = R(0);
      g1[c] = R(1) + a.d[c];
    }
    return;
  }
  const R u1 = u + du;
  const R s1 = fsqrt1(R(1) + R(3) * u1 * u1);
  const R ds = fdiv(R(3) * du * (R(2) * u + du), s1 + a.s);
  const R dA = -ds;
  const R dB = fdiv((R(2) * du + ds) * (R(1) - u) + (R(2) * u + a.s) * du, (R(1) - u1) * (R(1) - u));
  const R A = R(1) + a.d[1];
  const R B1 = a.B + dB;
  dg[1] = dA;
  dg[2] = dA * B1 + A * dB;
  dg[0] = fdiv(dA * a.B - A * dB, a.B * B1);
  for (int c = 0; c < 3; ++c) g1[c] = R(1) + a.d[c] + dg[c];
}

// Mass deviation rho~ = sum f~, density and velocity from deviation populations.
// Sums run as three independent partial sums (one per z-layer of the lattice)
// to keep the dependency chains short.
template <typename R>
__device__ __forceinline__ void macro(const R (&f)[27], R& rho_t, R& rho, R& ux, R& uy, R& uz) {
  R r[3] = {0, 0, 0}, jx[3] = {0, 0, 0}, jy[3] = {0, 0, 0}, jz = 0;
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int l = CZ(i) + 1;
    r[l] += f[i];
    if constexpr (CX(i) == 1) jx[l] += f[i];
    if constexpr (CX(i) == -1) jx[l] -= f[i];
    if constexpr (CY(i) == 1) jy[l] += f[i];
    if constexpr (CY(i) == -1) jy[l] -= f[i];
  });
  jz = r[2] - r[0];
  rho_t = (r[0] + r[2]) + r[1];
  rho = R(1) + rho_t;
  const R ir = rcp_fast(rho);
  ux = ((jx[0] + jx[2]) + jx[1]) * ir;
  uy = ((jy[0] + jy[2]) + jy[1]) * ir;
  uz = jz * ir;
}

// q_i = prod_a (1 + d_a(c_ia)) - 1 for all i, from the three axes.
template <int i, typename R>
__device__ __forceinline__ R qprod(const AxisEq<R>& ex, const AxisEq<R>& ey, const AxisEq<R>& ez) {
  const R dx = ex.d[CX(i) + 1], dy = ey.d[CY(i) + 1], dz = ez.d[CZ(i) + 1];
  const R t = dx + dy + dx * dy;
  return t + dz + t * dz;
}

// Deviation equilibrium fe~_i = f_i^eq - W_i.
template <typename R>
__device__ __forceinline__ void feq_dev(R rho_t, R rho, R ux, R uy, R uz, R (&fe)[27]) {
  AxisEq<R> ex, ey, ez;
  axis_eq<R>(ux, ex, false);
  axis_eq<R>(uy, ey, false);
  axis_eq<R>(uz, ez, false);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    fe[i] = R(WI(i)) * (rho_t + rho * qprod<i>(ex, ey, ez));
  });
}

// Shear part ds_i of a non-equilibrium vector from its second moments
// (reading: natural-moment basis; face directions carry half the deviatoric
// normal stress, edge directions a quarter of the off-diagonal stress with
// sign cx*cy, rest and corners none).
template <int i, typename R>
__device__ __forceinline__ R shear_part(R nxx, R nyy, R nzz, R pxy, R pxz, R pyz) {
  constexpr int ax = CX(i) != 0, ay = CY(i) != 0, az = CZ(i) != 0;
  if constexpr (ax + ay + az == 1) {
    if constexpr (ax) return R(0.5) * nxx;
    else if constexpr (ay) return R(0.5) * nyy;
    else return R(0.5) * nzz;
  } else if constexpr (ax + ay + az == 2) {
    if constexpr (!az) return R(0.25 * CX(i) * CY(i)) * pxy;
    else if constexpr (!ay) return R(0.25 * CX(i) * CZ(i)) * pxz;
    else return R(0.25 * CY(i) * CZ(i)) * pyz;
  } else {
    return R(0);
  }
}

// The KBC collision itself is in collide.cuh.

// ---------------------------------------------------------------------------
// Pull-streaming: f_i(x) = f'_i(x - c_i) from the previous state.
// Fast path for T_BULK nodes: every source is a stored fluid node, periodic
// wrap only on spanned axes.
template <typename S, typename R>
__device__ __forceinline__ void pull_bulk(const PatchDev& p, const S* __restrict__ fin, int x, int y, int z,
                                          R (&f)[27]) {
  const int xm = x == 0 ? p.dim[0] - 1 : x - 1, xp = x == p.dim[0] - 1 ? 0 : x + 1;
  const int ym = y == 0 ? p.dim[1] - 1 : y - 1, yp = y == p.dim[1] - 1 ? 0 : y + 1;
  const int zm = z == 0 ? p.dim[2] - 1 : z - 1, zp = z == p.dim[2] - 1 ? 0 : z + 1;
  const long long row = p.nxp, sl = (long long)p.nxp * p.dim[1];
  const long long xs[3] = {xp, x, xm};  // source x for cx = -1, 0, +1
  const long long ys[3] = {yp * row, y * row, ym * row};
  const long long zs[3] = {zp * sl, z * sl, zm * sl};
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    f[i] = Stor<S>::ld(fin + (long long)i * p.plane + zs[CZ(i) + 1] + ys[CY(i) + 1] + xs[CX(i) + 1]);
  });
}

// Population i returning to node own (coordinates X) from a solid neighbour
// X - c_i, with the wall at fraction q of the link from X along c_ib
// (ib = 26 - i): the particle that leaves along c_ib and comes back along c_i
// within one step, interpolated linearly along the link (Bouzidi, Firdaouss
// & Lallemand 2001).  For q < 1/2 it left from between X and the fluid node
// X + c_i behind it: 2q a'(X) + (1 - 2q) a'(X + c_i) along ib; for q >= 1/2 it
// lands between X and the wall and X takes (1/(2q)) a + ((2q - 1)/(2q)) a'_i(X)
// with a the reflected value.  a is a'_ib (bounce-back) or, with anti,
// -a'_ib + w (anti-bounce-back of an isothermal surface, w its wall term).  A
// missing node behind gives half-way bounce-back.  arr holds deviations from
// a weight that is the same for i and ib, and the weights of each formula
// sum to one, so deviations map to deviations.
template <int i, typename S, typename R>
__device__ __forceinline__ R returning(const PatchDev& p, const S* __restrict__ arr, long long own, const int X[3],
                                       R q, bool anti, R w) {
  constexpr int ib = 26 - i;
  constexpr int c[3] = {CX(i), CY(i), CZ(i)};
  const R own_ib = Stor<S>::ld(arr + (long long)ib * p.plane + own);
  if (q < R(0.5)) {
    int b[3];
    bool ok = true;
    unroll<3>([&](auto A) {
      constexpr int a = decltype(A)::value;
      b[a] = X[a] + c[a];
      if (b[a] < 0 || b[a] >= p.dim[a]) {
        if (p.span[a]) b[a] += b[a] < 0 ? p.dim[a] : -p.dim[a];
        else ok = false;
      }
    });
    long long bi = 0;
    if (ok) {
      bi = node_index(p, b[0], b[1], b[2]);
      const uint8_t t = p.type[bi];
      ok = t != T_SOLID && t != T_SKIP;
    }
    if (ok) {
      const R mix = R(2) * q * own_ib + (R(1) - R(2) * q) * Stor<S>::ld(arr + (long long)ib * p.plane + bi);
      return anti ? w - mix : mix;
    }
    return anti ? w - own_ib : own_ib;
  }
  const R a = anti ? w - own_ib : own_ib;
  const R i2q = R(1) / (R(2) * q);
  return a * i2q + (R(2) * q - R(1)) * i2q * Stor<S>::ld(arr + (long long)i * p.plane + own);
}

// Generic path: walls (half-way bounce-back), solid nodes (bounce-back,
// interpolated along the link at a curved surface),
// outlet (source clamped to the last node), periodic wrap on spanned axes.
// A source that resolves to no node sets bit 0 of *status and falls back to
// bounce-back (never produced by a validated layout).
// TWO: in two passes, so that the loads of each pass are independent of each
// other -- first every source node (or the bounce rule) and its class, then
// the populations: two memory round trips for the node instead of up to one
// per population, for the kernels whose few nodes leave the GPU waiting on
// latency (the fix-up nodes); at the cost of registers, which throughput
// kernels keep for occupancy.
template <typename S, typename R, bool TWO = false>
__device__ __forceinline__ void pull_generic(const PatchDev& p, const S* __restrict__ fin, int x, int y, int z,
                                             R (&f)[27], int* status) {
  const long long own = node_index(p, x, y, z);
  const int X[3] = {x, y, z};
  const int wk = p.wq_idx ? p.wq_idx[own] : -1;  // this node's row of wall fractions
  constexpr int kBounce = 0x100, kBad = 0x200;
  // the source of population i (or the bounce rule) and its class
  auto source = [&](auto I, long long& src) -> int {
    constexpr int i = decltype(I)::value;
    constexpr int c[3] = {CX(i), CY(i), CZ(i)};
    int s[3];
    bool bounce = false, bad = false;
    unroll<3>([&](auto A) {
      constexpr int a = decltype(A)::value;
      s[a] = X[a] - c[a];
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
    src = own;
    if (bad) return kBad;
    if (bounce) return kBounce;
    src = node_index(p, s[0], s[1], s[2]);
    return p.type[src];
  };
  // population i from its source class; an unresolved source is reported
  // once, after the loads (an atomic between them would order them)
  bool any_bad = false;
  auto take = [&](auto I, int t, long long src) {
    constexpr int i = decltype(I)::value;
    const bool solid = t == T_SOLID, bad = t == kBad || t == T_SKIP;
    any_bad |= bad;
    if (solid && wk >= 0) f[i] = returning<i, S, R>(p, fin, own, X, R(p.wq[27 * wk + 26 - i]), false, R(0));
    else if (solid || bad || t == kBounce) f[i] = Stor<S>::ld(fin + (long long)(26 - i) * p.plane + own);
    else f[i] = Stor<S>::ld(fin + (long long)i * p.plane + src);
  };
  if constexpr (TWO) {
    long long src[27];
    int cls[27];
    unroll<27>([&](auto I) { cls[decltype(I)::value] = source(I, src[decltype(I)::value]); });
    unroll<27>([&](auto I) { take(I, cls[decltype(I)::value], src[decltype(I)::value]); });
  } else {
    unroll<27>([&](auto I) {
      long long src;
      const int t = source(I, src);
      take(I, t, src);
    });
  }
  if (any_bad) atomicOr(status, 1);
}

}  // namespace lbmk
