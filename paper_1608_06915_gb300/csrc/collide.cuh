// The KBC collision (Eqs. f_equations, f_mirr, gamma_min_approx) with the
// exact-difference-method force, written once over an arithmetic type V:
//
//   double  one node in FP64 (native operators);
//   F1      one node in FP32, every operation rounded as written (no
//           contraction of a multiply and an add into one fused operation);
//   F2      two nodes in FP32 through the packed FP32x2 instructions of
//           sm_100 and later (one instruction computes both nodes' operation).
//
// F1 and F2 run the same sequence of IEEE-rounded operations per node, and
// the reciprocal and square-root approximations are taken per node, so a
// node collided as the half of a pair gets exactly the bits it gets alone.
// The TMA tile pass collides node pairs (F2); every other FP32 kernel
// collides single nodes (F1).
#pragma once

#include <type_traits>

#include "device.cuh"

namespace lbmk {

// The FP32 reciprocal and reciprocal square root: the hardware approximations
// (rcp.approx, rsqrt.approx; about 1 ulp), issued as written so that the
// compiler cannot fold them into neighbouring operations differently for
// single nodes and pairs.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

struct F1 {
  float v;
  F1() = default;
  __host__ __device__ constexpr explicit F1(float x) : v(x) {}
};
// F1 issues its operations as PTX with the rounding written out (.rn): the
// optimizer contracts no such scalar instruction into a fused one, so a node
// runs exactly the operations written here, whatever surrounds them.
__device__ __forceinline__ F1 operator+(F1 a, F1 b) {
  float r;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a.v), "f"(b.v));
  return F1(r);
}
__device__ __forceinline__ F1 operator-(F1 a, F1 b) {
  float r;
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a.v), "f"(b.v));
  return F1(r);
}
__device__ __forceinline__ F1 operator*(F1 a, F1 b) {
  float r;
  asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a.v), "f"(b.v));
  return F1(r);
}
__device__ __forceinline__ F1 operator-(F1 a) { return F1(-a.v); }
__device__ __forceinline__ F1 vfma(F1 a, F1 b, F1 c) {
  float r;
  asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a.v), "f"(b.v), "f"(c.v));
  return F1(r);
}
__device__ __forceinline__ F1 vrcp(F1 a) { return F1(rcp_approx(a.v)); }
__device__ __forceinline__ F1 vrsqrt(F1 a) { return F1(rsqrt_approx(a.v)); }
__device__ __forceinline__ F1 vsel_gt(F1 a, F1 b, F1 x, F1 y) { return F1(a.v > b.v ? x.v : y.v); }

struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float x) : v(make_float2(x, x)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
};
__device__ __forceinline__ unsigned long long f2bits(float2 a) {
  return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 bitsf2(unsigned long long r) {
  return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
// The packed operations are all issued as fused multiply-adds with the
// rounding written out: a + b = fma(a, 1, b), a - b = fma(b, -1, a),
// a b = fma(a, b, -0), each rounded once exactly as the plain operation.
// Written as packed add, sub or mul (.rn), ptxas contracts a multiply into a
// following add or subtract, which it does not for the scalar forms, so a
// node's result would depend on whether it was collided alone or in a pair;
// with immediate constants it turns these fused forms back into the plain
// ones and contracts them likewise.  The constants 1, -1 and -0 therefore
// come from constant memory, whose contents ptxas cannot assume.
static __constant__ float2 kPackedOne = {1.0f, 1.0f};
static __constant__ float2 kPackedMinusOne = {-1.0f, -1.0f};
static __constant__ float2 kPackedMinusZero = {-0.0f, -0.0f};
__device__ __forceinline__ F2 pfma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2bits(a)), "l"(f2bits(b)), "l"(f2bits(c)));
  return F2(bitsf2(r));
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return pfma(a.v, kPackedOne, b.v); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return pfma(b.v, kPackedMinusOne, a.v); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return pfma(a.v, b.v, kPackedMinusZero); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return pfma(a.v, b.v, c.v); }
__device__ __forceinline__ F2 vrcp(F2 a) { return F2(rcp_approx(a.v.x), rcp_approx(a.v.y)); }
__device__ __forceinline__ F2 vrsqrt(F2 a) { return F2(rsqrt_approx(a.v.x), rsqrt_approx(a.v.y)); }
__device__ __forceinline__ F2 vsel_gt(F2 a, F2 b, F2 x, F2 y) {
  return F2(a.v.x > b.v.x ? x.v.x : y.v.x, a.v.y > b.v.y ? x.v.y : y.v.y);
}

__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double vrcp(double a) { return 1.0 / a; }
__device__ __forceinline__ double vsel_gt(double a, double b, double x, double y) { return a > b ? x : y; }

// Constants of the arithmetic type (FP32 types round the double value once).
template <typename V>
struct VC;
template <>
struct VC<double> {
  static __device__ __forceinline__ double c(double x) { return x; }
};
template <>
struct VC<F1> {
  static __device__ __forceinline__ F1 c(double x) { return F1((float)x); }
};
template <>
struct VC<F2> {
  static __device__ __forceinline__ F2 c(double x) { return F2((float)x); }
};
template <typename V>
__device__ __forceinline__ V K(double x) {
  return VC<V>::c(x);
}

// sqrt(x) for x >= 1: IEEE in double, x * rsqrt(x) in FP32.
__device__ __forceinline__ double vsqrt1(double x) { return sqrt(x); }
template <typename V>
__device__ __forceinline__ V vsqrt1(V x) {
  return x * vrsqrt(x);
}

// ---------------------------------------------------------------------------
// Per-axis factors of the product-form equilibrium, Eq. (feq_iso), in
// deviation form: ghat(0) = A, ghat(+1) = A B, ghat(-1) = A / B with
// s = sqrt(1 + 3u^2), A = 2 - s, B = (2u + s)/(1 - u).  With e = s - 1 =
// 3u^2/(s + 1) the deviations d = ghat - 1 are
//   d(0) = -e,  d(+1) = (u (3 - 3u - 2e) + 2e)/(1 - u),
//   d(-1) = (u (e - 3) - 2e)/(2u + s),
// free of cancellation.  The entropic weights take 1/(W1(c) ghat(c)):
// 1/ghat(0) = 1/A, 1/ghat(+1) = (1/A)(1/B), 1/ghat(-1) = B/A, and 1 - e = A.
// The four reciprocals come from two: 1/((1 - u)(2u + s)) and 1/((s + 1) A).
template <typename V>
struct AxisV {
  V d[3];   // ghat - 1 for c = -1, 0, +1
  V ig[3];  // 1 / (W1(c) ghat(c))
  V s, B;
};

template <typename V>
__device__ __forceinline__ void axis_eq_v(V u, AxisV<V>& a, bool want_inverse) {
  const V one = K<V>(1.0), two = K<V>(2.0), three = K<V>(3.0);
  const V u2 = u * u;
  const V s = vsqrt1(vfma(three, u2, one));
  const V om = one - u;
  const V tus = vfma(two, u, s);
  const V r1 = vrcp(om * tus);
  const V i1mu = tus * r1, i2us = om * r1;
  const V sp1 = s + one, A = two - s;
  const V r2 = vrcp(sp1 * A);
  const V e = (three * u2) * (A * r2);
  const V e2 = e + e;
  a.s = s;
  a.B = tus * i1mu;
  a.d[1] = -e;
  a.d[2] = vfma(u, vfma(-three, u, three - e2), e2) * i1mu;
  a.d[0] = vfma(u, e - three, -e2) * i2us;
  if (want_inverse) {
    const V iA = sp1 * r2;
    const V iA6 = K<V>(6.0) * iA;
    a.ig[1] = K<V>(1.5) * iA;
    a.ig[2] = iA6 * (om * i2us);
    a.ig[0] = iA6 * a.B;
  }
}

// Mass deviation rho~ = sum f~, density and velocity of deviation
// populations, summed row by row along x: per (c_y, c_z) the row sum and
// the row's x-momentum, then per layer c_z.
template <typename V>
__device__ __forceinline__ void macro_v(const V (&f)[27], V& rho_t, V& rho, V& ux, V& uy, V& uz) {
  V L[3], X[3], Y[3];
#pragma unroll
  for (int z = 0; z < 3; ++z) {
    V s[3], m[3];
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      const V lo = f[9 * z + 3 * y], mid = f[9 * z + 3 * y + 1], hi = f[9 * z + 3 * y + 2];
      s[y] = (lo + hi) + mid;
      m[y] = hi - lo;
    }
    L[z] = (s[0] + s[2]) + s[1];
    X[z] = (m[0] + m[2]) + m[1];
    Y[z] = s[2] - s[0];
  }
  rho_t = (L[0] + L[2]) + L[1];
  rho = K<V>(1.0) + rho_t;
  const V ir = vrcp(rho);
  ux = ((X[0] + X[2]) + X[1]) * ir;
  uy = ((Y[0] + Y[2]) + Y[1]) * ir;
  uz = (L[2] - L[0]) * ir;
}

template <int i>
__host__ __device__ constexpr int wclass() {
  return (CX(i) != 0) + (CY(i) != 0) + (CZ(i) != 0);
}

// Shear class of direction i: 0 none (rest, corners), 1..3 face along x, y, z
// (ds = 1/2 of the deviatoric normal stress), 4..9 edge in the xy, xz, yz
// planes with sign c_a c_b positive (4..6) or negative (7..9), ds = c_a c_b
// P_ab / 4.
template <int i>
__host__ __device__ constexpr int shear_class() {
  constexpr int ax = CX(i) != 0, ay = CY(i) != 0, az = CZ(i) != 0;
  if constexpr (ax + ay + az == 1) return ax ? 1 : (ay ? 2 : 3);
  if constexpr (ax + ay + az == 2) {
    constexpr int plane = !az ? 0 : (!ay ? 1 : 2);
    constexpr int sg = !az ? CX(i) * CY(i) : (!ay ? CX(i) * CZ(i) : CY(i) * CZ(i));
    return 4 + plane + (sg < 0 ? 3 : 0);
  }
  return 0;
}

// The collision of Eqs. f_equations, f_mirr, gamma_min_approx in delta form,
//   f'_i = f^eq_i + (1 - beta gamma) df_i + beta (gamma - 2) ds_i,
// df = f - f^eq, ds the shear part (reading: natural-moment basis), with the
// exact-difference-method force f'_i += f^eq(rho, u + du) - f^eq(rho, u), and
// the 0/0 guard gamma = 2 when <dh|dh> <= 1e-30 rho^2.  f holds deviation
// populations f - W, the moments (rho~, rho, u) are those of f; f is replaced
// by the post-collision deviations; returns gamma.  With DF, f holds df itself
// on entry (a state assembled as f^eq(rho, u) + df, whose df is known).  FM:
// compile-time mask of the axes along which du may be nonzero (0: no force).
// beta and du are the same for every node of V (a pair of nodes shares its
// patch).
//
// Every per-direction quantity is a product of per-axis factors, so the loops
// read small tables: q_i from (1 + q_xy)(1 + d_z) - 1, rho W_i from the four
// weight classes, the second moments from the three z-columns of each
// (c_x, c_y) pair, the entropic weights 1/f^eq_i as 1/(g_x g_y) per column
// times 1/(rho g_z) per layer.  The tables of f^eq are built twice (before
// and after gamma) rather than held, which keeps few values live.
template <typename V, int FM, bool DF = false>
__device__ __forceinline__ V kbc_collide_v(V (&f)[27], V rho_t, V rho, V ux, V uy, V uz, V beta, V dux, V duy,
                                           V duz, bool du_x, bool du_y, bool du_z, bool lbgk) {
  AxisV<V> ex, ey, ez;
  axis_eq_v<V>(ux, ex, !lbgk);
  axis_eq_v<V>(uy, ey, !lbgk);
  axis_eq_v<V>(uz, ez, !lbgk);
  // f^eq_i - W_i = W_i (rho~ + rho q_i), q_i = (1 + q_xy)(1 + d_z) - 1, from
  // the per-axis deviations; f becomes df = f - f^eq
  constexpr double WK[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  if constexpr (!DF) {
    V wr[4], wrt[4], qxy[3][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      wr[k] = K<V>(WK[k]) * rho;
      wrt[k] = K<V>(WK[k]) * rho_t;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) qxy[a][b] = vfma(ex.d[a], ey.d[b], ex.d[a] + ey.d[b]);
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const V t = qxy[CX(i) + 1][CY(i) + 1], dz = ez.d[CZ(i) + 1];
      f[i] = f[i] - vfma(wr[wclass<i>()], vfma(t, dz, t + dz), wrt[wclass<i>()]);
    });
  }
  // second moments of df: per (c_x, c_y) column, z0 = sum over c_z,
  // z1 = sum c_z df, z2 = sum c_z^2 df
  V pxx, pyy, pzz, pxy, pxz, pyz;
  {
    V z0[3][3], z1[3][3], z2[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const V lo = f[a + 3 * b], mid = f[a + 3 * b + 9], hi = f[a + 3 * b + 18];
        z2[a][b] = lo + hi;
        z1[a][b] = hi - lo;
        z0[a][b] = z2[a][b] + mid;
      }
    pxx = ((z0[0][0] + z0[2][0]) + (z0[0][1] + z0[2][1])) + (z0[0][2] + z0[2][2]);
    pyy = ((z0[0][0] + z0[0][2]) + (z0[1][0] + z0[1][2])) + (z0[2][0] + z0[2][2]);
    pzz = ((z2[0][0] + z2[1][0]) + (z2[2][0] + z2[0][1])) + ((z2[1][1] + z2[2][1]) + (z2[0][2] + z2[1][2])) +
          z2[2][2];
    pxy = (z0[0][0] + z0[2][2]) - (z0[2][0] + z0[0][2]);
    pxz = ((z1[2][0] - z1[0][0]) + (z1[2][1] - z1[0][1])) + (z1[2][2] - z1[0][2]);
    pyz = ((z1[0][2] - z1[0][0]) + (z1[1][2] - z1[1][0])) + (z1[2][2] - z1[2][0]);
  }
  // shear part per class (shear_class): faces 1/2 of the deviatoric normal
  // stress, edges +-1/4 of the off-diagonal stress
  V ds[10];
  {
    const V tr3 = (pxx + pyy + pzz) * K<V>(1.0 / 3.0);
    const V half = K<V>(0.5), quarter = K<V>(0.25);
    ds[0] = K<V>(0.0);
    ds[1] = half * (pxx - tr3);
    ds[2] = half * (pyy - tr3);
    ds[3] = half * (pzz - tr3);
    ds[4] = quarter * pxy;
    ds[5] = quarter * pxz;
    ds[6] = quarter * pyz;
    ds[7] = -ds[4];
    ds[8] = -ds[5];
    ds[9] = -ds[6];
  }
  V gamma = K<V>(2.0);
  if (!lbgk) {
    V wxy[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) wxy[a][b] = ex.ig[a] * ey.ig[b];
    V shl[3] = {K<V>(0.0), K<V>(0.0), K<V>(0.0)}, hhl[3] = {K<V>(0.0), K<V>(0.0), K<V>(0.0)};
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int l = CZ(i) + 1, sc = shear_class<i>();
      if constexpr (sc == 0) {
        const V dhw = f[i] * wxy[CX(i) + 1][CY(i) + 1];
        hhl[l] = vfma(f[i], dhw, hhl[l]);
      } else {
        const V dh = f[i] - ds[sc];
        const V dhw = dh * wxy[CX(i) + 1][CY(i) + 1];
        shl[l] = vfma(ds[sc], dhw, shl[l]);
        hhl[l] = vfma(dh, dhw, hhl[l]);
      }
    });
    // layer weights 1/(rho g_z) applied once per layer
    const V irho = vrcp(rho);
    const V w0 = irho * ez.ig[0], w1 = irho * ez.ig[1], w2 = irho * ez.ig[2];
    const V sh = vfma(w1, shl[1], vfma(w0, shl[0], w2 * shl[2]));
    const V hh = vfma(w1, hhl[1], vfma(w0, hhl[0], w2 * hhl[2]));
    const V ib = vrcp(beta);
    const V g = ib - (K<V>(2.0) - ib) * (sh * vrcp(hh));
    gamma = vsel_gt(hh, K<V>(1e-30) * rho * rho, g, gamma);
  }
  // f' = f^eq(rho, u + du) + (1 - beta gamma) df + beta (gamma - 2) ds: the
  // exact difference method adds f^eq(rho, u + du) - f^eq(rho, u) to the
  // collided state, whose equilibrium part is f^eq(rho, u), so the force
  // enters as the shifted equilibrium, in deviation form like f^eq itself
  // (axes without force keep their factors)
  const V a = K<V>(1.0) - beta * gamma;
  const V b = beta * (gamma - K<V>(2.0));
  V bds[10];
#pragma unroll
  for (int k = 1; k < 10; ++k) bds[k] = b * ds[k];
  V dx[3], dy[3], dzz[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dx[c] = ex.d[c], dy[c] = ey.d[c], dzz[c] = ez.d[c];
  if constexpr (FM != 0) {
    AxisV<V> sh;
    if ((FM & 1) && du_x) {
      axis_eq_v<V>(ux + dux, sh, false);
#pragma unroll
      for (int c = 0; c < 3; ++c) dx[c] = sh.d[c];
    }
    if ((FM & 2) && du_y) {
      axis_eq_v<V>(uy + duy, sh, false);
#pragma unroll
      for (int c = 0; c < 3; ++c) dy[c] = sh.d[c];
    }
    if ((FM & 4) && du_z) {
      axis_eq_v<V>(uz + duz, sh, false);
#pragma unroll
      for (int c = 0; c < 3; ++c) dzz[c] = sh.d[c];
    }
  }
  V wr[4], wrt[4], qxy[3][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    wr[k] = K<V>(WK[k]) * rho;
    wrt[k] = K<V>(WK[k]) * rho_t;
  }
#pragma unroll
  for (int ca = 0; ca < 3; ++ca)
#pragma unroll
    for (int cb = 0; cb < 3; ++cb) qxy[ca][cb] = vfma(dx[ca], dy[cb], dx[ca] + dy[cb]);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int sc = shear_class<i>();
    const V t = qxy[CX(i) + 1][CY(i) + 1], dz = dzz[CZ(i) + 1];
    const V e = vfma(wr[wclass<i>()], vfma(t, dz, t + dz), wrt[wclass<i>()]);
    if constexpr (sc == 0) f[i] = vfma(a, f[i], e);
    else f[i] = vfma(a, f[i], e + bds[sc]);
  });
  return gamma;
}

// The collision for the scalar storage types of the kernels: float runs as F1,
// double natively.  Moments given (kbc_collide_m) or taken from f.
template <typename R>
struct CollideType {
  using V = double;
};
template <>
struct CollideType<float> {
  using V = F1;
};

// DF: f holds df = f - f^eq(rho, u) on entry (kbc_collide_v).
template <typename R, int FM, bool DF = false>
__device__ __forceinline__ R kbc_collide_m(R (&f)[27], R rho_t, R rho, R ux, R uy, R uz, R beta, R dux, R duy,
                                           R duz, bool lbgk) {
  using V = typename CollideType<R>::V;
  V fv[27];
  unroll<27>([&](auto I) { fv[decltype(I)::value] = V(f[decltype(I)::value]); });
  const V g = kbc_collide_v<V, FM, DF>(fv, V(rho_t), V(rho), V(ux), V(uy), V(uz), V(beta), V(dux), V(duy),
                                       V(duz), dux != R(0), duy != R(0), duz != R(0), lbgk);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (std::is_same<V, R>::value) f[i] = fv[i];
    else f[i] = fv[i].v;
  });
  if constexpr (std::is_same<V, R>::value) return g;
  else return g.v;
}

template <typename R, int FM>
__device__ __forceinline__ R kbc_collide(R (&f)[27], R beta, R dux, R duy, R duz, bool lbgk) {
  using V = typename CollideType<R>::V;
  V fv[27];
  unroll<27>([&](auto I) { fv[decltype(I)::value] = V(f[decltype(I)::value]); });
  V rho_t, rho, ux, uy, uz;
  macro_v<V>(fv, rho_t, rho, ux, uy, uz);
  const V g = kbc_collide_v<V, FM>(fv, rho_t, rho, ux, uy, uz, V(beta), V(dux), V(duy), V(duz), dux != R(0),
                                   duy != R(0), duz != R(0), lbgk);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (std::is_same<V, R>::value) f[i] = fv[i];
    else f[i] = fv[i].v;
  });
  if constexpr (std::is_same<V, R>::value) return g;
  else return g.v;
}

}  // namespace lbmk
