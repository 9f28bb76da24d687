// Oracle for the grid-refined entropic lattice Boltzmann method of
// Dorschner, Frapolli, Chikatamarla & Karlin, "Grid refinement for entropic
// lattice Boltzmann models" (arXiv:1608.06915).
//
// TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
// the method, written to be checked against the paper by eye.  Only the test
// suite, the smoke check and the CPU-baseline leg of the benchmark load it;
// the product path (the CUDA library) shares no code, header, table or
// helper with it, and neither side includes or links the other.
//
// What it computes, in the paper's order and notation:
//   * D3Q27 lattice, W_i = prod_a W_{c_ia}, W_0 = 2/3, W_{+-1} = 1/6   (Sec. II.A, after Eq. feq_iso)
//   * product-form entropic equilibrium                                (Sec. II.A, Eq. feq_iso)
//   * natural moments rho*M_pqr                                        (Sec. II.A, Eq. moments)
//   * KBC split f = k + s + h, mirror state, stabiliser gamma          (Sec. II.A, Eqs. popSplit, f_mirr, gamma_min_approx)
//   * post-collision state (1-beta) f + beta f^mirr                    (Sec. II, Eq. f_equations)
//   * exact-difference-method body force, du_f = du_c / r              (Sec. III.A, force paragraph)
//   * two-population thermal kinetics, Pr <= 1 and Pr > 1              (Sec. II.B, Eqs. kinetics_f_KBC_thermal,
//                                                                        kinetics_g_entr, grad_general, Table I)
//   * multi-domain refinement: twin-node non-equilibrium rescaling,
//     centred four-point Lagrange reconstruction, the five-step
//     algorithm with r = 2 and no time interpolation                 (Sec. III, Eqs. f_neq_rescaling_iso,
//                                                                        thermal g rescaling, interp; Sec. III.C)
//
// Every node carries a validity flag: streaming from a node that holds no
// valid state, or sampling such a node during the coupling, is an error.
// After each coarse step every fluid node must hold a valid post-collision
// state.  These checks make the oracle verify the layout reading as it runs.
//
// Readings taken where the paper is silent (the same readings the CUDA path
// implements independently):
//   R1  s is the part of f spanned by the deviatoric second-order natural
//       moments, k by the conserved ones, h = f - k - s (trace of P in h).
//   R2  gamma = 2 when <dh|dh> <= 1e-30 rho^2 (0/0 guard); no clamp.
//   R3  layout: a level-(l+1) box [a,b] (parent coordinates) holds child
//       nodes at every half-integer position of [a,b]; the child interface is
//       child-distance 0..1 from a box face that is neither a wall face nor a
//       periodic span; the parent hole is [a+2,b-2]; parent interface nodes
//       (twins x_t,cf) are the non-hole parent nodes of [a+1,b-1].
//   R4  reconstruction samples sit at parent positions +-1/2, +-3/2 along
//       each off-lattice axis; a sample inside the parent hole is taken from
//       the child node at that position; parent samples are rescaled to the
//       fine scale before interpolation.
//   R5  forcing: u = j/rho in the collision; reported velocity u + du/2.
//   R6  walls: half-way bounce-back; inlet: fixed equilibrium nodes;
//       outlet: zero-gradient (pull source clamped to the last node).
//   R7  thermal: T0 = 1/3; f* = f^eq for Pr <= 1; g* from Table I with the
//       closed-form P^eq; Boussinesq acceleration g*lambda*(T - T_ref) e_z;
//       thermal walls by anti-bounce-back of g to the wall equilibrium.
//   R9  state transfer onto another layout (not in the paper; see
//       Sim::transfer_from): the source level nearest the node's own that
//       holds it (own, then finer, then coarser), coinciding node or trilinear
//       cell corners, f - f^eq rescaled by beta_s/(r beta_t).
//   R8  thermal, Pr > 1: f* differs from f^eq only by the Grad term of the
//       non-equilibrium stress, f*_i - f^eq_i = W_i P1_ab (c_ia c_ib -
//       T0 d_ab) / (2 T0^2) with P1 = P - P^eq (Table I row f* for Pr > 1,
//       read consistently with R7, where the same Grad form with P^eq is
//       f^eq itself); the same tensor P1 enters g* (Table I row g*).
//
//   R10 curved solid surfaces (the heated sphere of Sec. IV): an analytic
//       sphere, cylinder or plane gives the fraction q of each solid link at
//       which the wall lies; the population returning from it is interpolated
//       linearly along the link (Bouzidi, Firdaouss & Lallemand 2001) -- for g
//       of an isothermal surface the same construction on the anti-bounce-back
//       rule -- and the drag takes the returning value; q = 1/2 without a
//       surface (half-way bounce-back, the staircase of the solid mask).
// Parity status: every function above is pinned by tests under tests/
// (closed forms, invariants, special cases, brute force, a two-level run
// against a uniform run at the fine spacing, and the Chapman-Enskog state of
// a shear flow through the interface rescaling).

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

constexpr int Q = 27;
using Pop = std::array<double, Q>;

// Velocity ordering: i = (cx+1) + 3(cy+1) + 9(cz+1); rest = 13; opposite = 26 - i.
inline int cvel(int i, int a) {
  int v = (a == 0) ? i % 3 : (a == 1) ? (i / 3) % 3 : i / 9;
  return v - 1;
}
inline int opposite(int i) { return Q - 1 - i; }
inline double W1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
inline double Wi(int i) { return W1(cvel(i, 0)) * W1(cvel(i, 1)) * W1(cvel(i, 2)); }

// ---------------------------------------------------------------------------
// Equilibrium, Eq. (feq_iso):
//   f_i^eq = rho W_i prod_a (2 - sqrt(1+3u_a^2)) ((2u_a + sqrt(1+3u_a^2))/(1-u_a))^{c_ia}
Pop feq(double rho, const double u[3]) {
  double s[3], base[3];
  for (int a = 0; a < 3; ++a) {
    s[a] = std::sqrt(1.0 + 3.0 * u[a] * u[a]);
    base[a] = (2.0 * u[a] + s[a]) / (1.0 - u[a]);
  }
  Pop f;
  for (int i = 0; i < Q; ++i) {
    double prod = rho * Wi(i);
    for (int a = 0; a < 3; ++a) {
      int c = cvel(i, a);
      double power = c == 0 ? 1.0 : (c == 1 ? base[a] : 1.0 / base[a]);  // base^{c_ia}
      prod *= (2.0 - s[a]) * power;
    }
    f[i] = prod;
  }
  return f;
}

struct Macro {
  double rho;
  double u[3];
};

// Conservation laws, Sec. II: sum_i {1, c_i} f_i = {rho, rho u}.
Macro macro(const Pop& f) {
  Macro m{};
  double j[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) {
    m.rho += f[i];
    for (int a = 0; a < 3; ++a) j[a] += cvel(i, a) * f[i];
  }
  for (int a = 0; a < 3; ++a) m.u[a] = j[a] / m.rho;
  return m;
}

// Natural moments, Eq. (moments): rho M_pqr = sum_i f_i cx^p cy^q cz^r, index p + 3q + 9r.
using Mom = std::array<double, Q>;
inline double ipow(int c, int p) { return p == 0 ? 1.0 : (p == 1 ? (double)c : (double)(c * c)); }

// Matrix of the moment map, MT[p+3q+9r][i] = cx^p cy^q cz^r.
struct MomentTable {
  double M[Q][Q];
  MomentTable() {
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q)
        for (int r = 0; r < 3; ++r)
          for (int i = 0; i < Q; ++i)
            M[p + 3 * q + 9 * r][i] = ipow(cvel(i, 0), p) * ipow(cvel(i, 1), q) * ipow(cvel(i, 2), r);
  }
};
static const MomentTable kMT;

Mom natural_moments(const Pop& f) {
  Mom m{};
  for (int k = 0; k < Q; ++k) {
    double acc = 0;
    for (int i = 0; i < Q; ++i) acc += kMT.M[k][i] * f[i];
    m[k] = acc;
  }
  return m;
}

// Populations from natural moments: the moment map is a tensor product of the
// one-dimensional map (m0, m1, m2) = (f_-1 + f_0 + f_1, f_1 - f_-1, f_1 + f_-1),
// whose inverse is f_0 = m0 - m2, f_+-1 = (+-m1 + m2)/2.
inline double inv1(int c, int p) {
  if (c == 0) return p == 0 ? 1.0 : (p == 1 ? 0.0 : -1.0);
  return p == 0 ? 0.0 : (p == 1 ? 0.5 * c : 0.5);
}

struct InverseTable {
  double A[Q][Q];  // A[i][p+3q+9r] = inv1(cx,p) inv1(cy,q) inv1(cz,r)
  InverseTable() {
    for (int i = 0; i < Q; ++i)
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
          for (int r = 0; r < 3; ++r)
            A[i][p + 3 * q + 9 * r] = inv1(cvel(i, 0), p) * inv1(cvel(i, 1), q) * inv1(cvel(i, 2), r);
  }
};
static const InverseTable kIT;

Pop from_moments(const Mom& m) {
  Pop f;
  for (int i = 0; i < Q; ++i) {
    double acc = 0;
    for (int k = 0; k < Q; ++k) acc += kIT.A[i][k] * m[k];
    f[i] = acc;
  }
  return f;
}

// KBC split, Eq. (popSplit): k from the conserved moments, s from the
// deviatoric stress P' = P - Tr(P)/D I and the off-diagonal P, h the rest
// (reading R1).
void kbc_split(const Pop& f, Pop& k, Pop& s, Pop& h) {
  Mom m = natural_moments(f);
  Mom mk{}, ms{};
  mk[0] = m[0];
  mk[1] = m[1];
  mk[3] = m[3];
  mk[9] = m[9];
  double trace = m[2] + m[6] + m[18];
  ms[2] = m[2] - trace / 3.0;
  ms[6] = m[6] - trace / 3.0;
  ms[18] = m[18] - trace / 3.0;
  ms[4] = m[4];
  ms[10] = m[10];
  ms[12] = m[12];
  k = from_moments(mk);
  s = from_moments(ms);
  for (int i = 0; i < Q; ++i) h[i] = f[i] - k[i] - s[i];
}

constexpr double kGammaTiny = 1e-30;

// One KBC collision, Eqs. (f_equations), (f_mirr), (gamma_min_approx), plus the
// exact-difference-method force (Sec. III.A).  Returns the stabiliser gamma.
double kbc_collide(const Pop& f, double beta, const double* du, bool lbgk, double gamma_forced, Pop& out) {
  Macro mc = macro(f);
  Pop fe = feq(mc.rho, mc.u);
  Pop fm;
  double gamma = 2.0;
  if (lbgk) {
    for (int i = 0; i < Q; ++i) fm[i] = 2.0 * fe[i] - f[i];  // Eq. (fmirr)
  } else {
    Pop k, s, h, ke, se, he;
    kbc_split(f, k, s, h);
    kbc_split(fe, ke, se, he);
    double sh = 0, hh = 0;
    for (int i = 0; i < Q; ++i) {
      double ds = s[i] - se[i], dh = h[i] - he[i];
      sh += ds * dh / fe[i];
      hh += dh * dh / fe[i];
    }
    if (hh > kGammaTiny * mc.rho * mc.rho) gamma = 1.0 / beta - (2.0 - 1.0 / beta) * sh / hh;
    if (!std::isnan(gamma_forced)) gamma = gamma_forced;
    for (int i = 0; i < Q; ++i) fm[i] = k[i] + (2.0 * se[i] - s[i]) + ((1.0 - gamma) * h[i] + gamma * he[i]);
  }
  for (int i = 0; i < Q; ++i) out[i] = (1.0 - beta) * f[i] + beta * fm[i];
  if (du && (du[0] != 0 || du[1] != 0 || du[2] != 0)) {
    double us[3] = {mc.u[0] + du[0], mc.u[1] + du[1], mc.u[2] + du[2]};
    Pop fs = feq(mc.rho, us);
    for (int i = 0; i < Q; ++i) out[i] += fs[i] - fe[i];
  }
  return gamma;
}

// ---------------------------------------------------------------------------
// Thermal two-population model, Sec. II.B, Pr <= 1 (reading R7).

// General Grad form, Eq. (grad_general), from moments (M0, M_a, M_ab).
Pop grad_form(double M0, const double Ma[3], const double Mab[3][3], double T0) {
  Pop G;
  for (int i = 0; i < Q; ++i) {
    double c[3] = {(double)cvel(i, 0), (double)cvel(i, 1), (double)cvel(i, 2)};
    double lin = 0, quad = 0;
    for (int a = 0; a < 3; ++a) lin += Ma[a] * c[a];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double d = (a == b) ? 1.0 : 0.0;
        quad += (Mab[a][b] - M0 * T0 * d) * (c[a] * c[b] - T0 * d);
      }
    G[i] = Wi(i) * (M0 + lin / T0 + quad / (2.0 * T0 * T0));
  }
  return G;
}

struct ThermalMacro {
  double rho, u[3], E2rho, T;  // E2rho = 2 rho E = sum g
};

ThermalMacro thermal_macro(const Pop& f, const Pop& g) {
  Macro m = macro(f);
  ThermalMacro t{};
  t.rho = m.rho;
  for (int a = 0; a < 3; ++a) t.u[a] = m.u[a];
  double s = 0;
  for (int i = 0; i < Q; ++i) s += g[i];
  t.E2rho = s;
  // E = (D/2) T + u^2/2  =>  T = (2E - u^2)/D with 2E = sum g / rho
  double u2 = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
  t.T = (s / m.rho - u2) / 3.0;
  return t;
}

// Equilibrium of g from Table I row g^eq with q^eq, R^eq of Eqs. (qeq_expression), (Req_expression).
Pop geq(double rho, const double u[3], double E2rho, double T0) {
  double q[3], R[3][3];
  for (int a = 0; a < 3; ++a) q[a] = E2rho * u[a] + 2.0 * rho * T0 * u[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double d = (a == b) ? 1.0 : 0.0;
      R[a][b] = E2rho * (T0 * d + u[a] * u[b]) + 2.0 * rho * T0 * (T0 * d + 2.0 * u[a] * u[b]);
    }
  return grad_form(E2rho, q, R, T0);
}

// Quasi-equilibrium g* for Pr <= 1, Table I: moments (2 rho E, q - 2u_b(P_ab - P^eq_ab), R^eq).
Pop gstar(const Pop& f, const Pop& g, double rho, const double u[3], double E2rho, double T0) {
  double q[3] = {0, 0, 0}, P[3][3] = {{0}}, R[3][3];
  for (int i = 0; i < Q; ++i)
    for (int a = 0; a < 3; ++a) {
      q[a] += cvel(i, a) * g[i];
      for (int b = 0; b < 3; ++b) P[a][b] += cvel(i, a) * cvel(i, b) * f[i];
    }
  double Mq[3];
  for (int a = 0; a < 3; ++a) {
    double corr = 0;
    for (int b = 0; b < 3; ++b) {
      double Peq = rho * T0 * (a == b ? 1.0 : 0.0) + rho * u[a] * u[b];
      corr += 2.0 * u[b] * (P[a][b] - Peq);
    }
    Mq[a] = q[a] - corr;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double d = (a == b) ? 1.0 : 0.0;
      R[a][b] = E2rho * (T0 * d + u[a] * u[b]) + 2.0 * rho * T0 * (T0 * d + 2.0 * u[a] * u[b]);
    }
  return grad_form(E2rho, Mq, R, T0);
}

// Non-equilibrium pressure tensor P1 = P - P^eq of f, with the closed-form
// P^eq = rho T0 delta + rho u u (Sec. II.B, after Table I).
void noneq_stress(const Pop& f, double rho, const double u[3], double T0, double P1[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double P = 0;
      for (int i = 0; i < Q; ++i) P += cvel(i, a) * cvel(i, b) * f[i];
      P1[a][b] = P - (rho * T0 * (a == b ? 1.0 : 0.0) + rho * u[a] * u[b]);
    }
}

// f* - f^eq for Pr > 1 (Table I row f*, reading R8): the Grad-form term of
// the non-equilibrium stress, W_i P1_ab (c_ia c_ib - T0 d_ab) / (2 T0^2).
Pop fstar_minus_feq_gt1(const Pop& f, double rho, const double u[3], double T0) {
  double P1[3][3];
  noneq_stress(f, rho, u, T0, P1);
  Pop d;
  for (int i = 0; i < Q; ++i) {
    double quad = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) quad += P1[a][b] * (cvel(i, a) * cvel(i, b) - T0 * (a == b ? 1.0 : 0.0));
    d[i] = Wi(i) * quad / (2.0 * T0 * T0);
  }
  return d;
}

// Quasi-equilibrium g* for Pr > 1, Table I: moments (2 rho E, q^eq + 2u_b(P_ab - P^eq_ab), R^eq).
Pop gstar_gt1(const Pop& f, double rho, const double u[3], double E2rho, double T0) {
  double P1[3][3], Mq[3], R[3][3];
  noneq_stress(f, rho, u, T0, P1);
  for (int a = 0; a < 3; ++a) {
    double corr = 0;
    for (int b = 0; b < 3; ++b) corr += 2.0 * u[b] * P1[a][b];
    Mq[a] = E2rho * u[a] + 2.0 * rho * T0 * u[a] + corr;  // q^eq (Eq. qeq_expression) + correction
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double d = (a == b) ? 1.0 : 0.0;
      R[a][b] = E2rho * (T0 * d + u[a] * u[b]) + 2.0 * rho * T0 * (T0 * d + 2.0 * u[a] * u[b]);
    }
  return grad_form(E2rho, Mq, R, T0);
}

// One thermal collision (Eqs. kinetics_f_KBC_thermal and kinetics_g_entr).
// With Pr <= 1, f* = f^eq (reading R7), so the f equation is the isothermal
// one; with Pr > 1 it adds 2 (beta - beta1) (f* - f^eq) (reading R8).  The
// Boussinesq acceleration enters through the exact difference method.
double thermal_collide(const Pop& f, const Pop& g, double beta, double beta1, double T0, double glambda,
                       double t_ref, double accel_scale, bool lbgk, bool pr_gt1, Pop& fo, Pop& go) {
  ThermalMacro tm = thermal_macro(f, g);
  double du[3] = {0, 0, glambda * (tm.T - t_ref) * accel_scale};
  double gamma = kbc_collide(f, beta, du, lbgk, NAN, fo);
  if (pr_gt1) {
    Pop d = fstar_minus_feq_gt1(f, tm.rho, tm.u, T0);
    for (int i = 0; i < Q; ++i) fo[i] += 2.0 * (beta - beta1) * d[i];
  }
  Pop ge = geq(tm.rho, tm.u, tm.E2rho, T0);
  Pop gs = pr_gt1 ? gstar_gt1(f, tm.rho, tm.u, tm.E2rho, T0) : gstar(f, g, tm.rho, tm.u, tm.E2rho, T0);
  for (int i = 0; i < Q; ++i) go[i] = g[i] + 2.0 * beta * (ge[i] - g[i]) + 2.0 * (beta - beta1) * (gs[i] - ge[i]);
  return gamma;
}

// Non-equilibrium moments for the thermal g rescaling: P1 = sum cc (f - f^eq) (Sec. III.A, thermal).
void p1_tensor(const Pop& f, const Pop& fe, double P1[3][3]) {
for (int a = 0; a < 3; ++a)
  for (int b = 0; b < 3; ++b) {
    double acc = 0;
    for (int i = 0; i < Q; ++i) acc += cvel(i, a) * cvel(i, b) * (f[i] - fe[i]);
    P1[a][b] = acc;
  }
}

// Interface rescaling of Sec. III.A: the non-equilibrium part of (f, g) moves
// from a level with (beta_s, beta1_s) to one with (beta_t, beta1_t);
// factor = beta_s / (r_st beta_t), r_st = dx_s / dx_t (2 for coarse-to-fine,
// 1/2 for fine-to-coarse).  Isothermal model: Eq. f_neq_rescaling_iso on the
// whole f - f^eq.  Thermal model: f as Eq. f_neq_rescaling_iso (Pr <= 1) or
// Eq. f_neq_rescaling_thr_Prgr1 (Pr > 1); g by the thermal rule of Sec. III.A,
// the part W_i 2 u_b P1_ab c_ia / T0 taken out, the rest rescaled with the
// other ratio, and the part added back with the rescaled P1.
void interface_rescale(bool thermal, bool pr_gt1, double t0, const Pop& f, const Pop& g, double beta_s,
                     double beta_t, double beta1_s, double beta1_t, double r_st, Pop& fo, Pop& go,
                     Pop* fneq_out, Pop* gneq_out, Macro* mac_out, ThermalMacro* tmac_out) {
  double ff = beta_s / (r_st * beta_t);
  if (!thermal) {
    Macro mc = macro(f);
    Pop fe = feq(mc.rho, mc.u);
    for (int i = 0; i < Q; ++i) fo[i] = fe[i] + ff * (f[i] - fe[i]);
    if (fneq_out)
      for (int i = 0; i < Q; ++i) (*fneq_out)[i] = ff * (f[i] - fe[i]);
    if (mac_out) *mac_out = mc;
    return;
  }
  ThermalMacro tm = thermal_macro(f, g);
  Pop fe = feq(tm.rho, tm.u);
  Pop ge = geq(tm.rho, tm.u, tm.E2rho, t0);
  // Sec. III.A thermal model: for Pr <= 1, f^neq and P1 scale with the beta
  // ratio and the rest of g^neq with the beta1 ratio; for Pr > 1 the two
  // ratios swap (Eq. f_neq_rescaling_thr_Prgr1 and the g rescaling after it)
  double fg = beta1_s / (r_st * beta1_t);
  if (pr_gt1) std::swap(ff, fg);
  for (int i = 0; i < Q; ++i) fo[i] = fe[i] + ff * (f[i] - fe[i]);
  double P1s[3][3], P1t[3][3];
  p1_tensor(f, fe, P1s);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) P1t[a][b] = ff * P1s[a][b];
  Pop gneq;
  for (int i = 0; i < Q; ++i) {
    double ts = 0, tt = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        ts += 2.0 * tm.u[b] * P1s[a][b] * cvel(i, a);
        tt += 2.0 * tm.u[b] * P1t[a][b] * cvel(i, a);
      }
    gneq[i] = fg * ((g[i] - ge[i]) - Wi(i) * ts / t0) + Wi(i) * tt / t0;
    go[i] = ge[i] + gneq[i];
  }
  if (fneq_out)
    for (int i = 0; i < Q; ++i) (*fneq_out)[i] = ff * (f[i] - fe[i]);
  if (gneq_out) *gneq_out = gneq;
  if (mac_out) {
    mac_out->rho = tm.rho;
    for (int a = 0; a < 3; ++a) mac_out->u[a] = tm.u[a];
  }
  if (tmac_out) *tmac_out = tm;
}

// ---------------------------------------------------------------------------
// Multi-domain layout (Sec. III, reading R3).

struct Box {
  int32_t level;
  int32_t lo[3], hi[3];
};

struct Desc {
  int32_t n[3];
  uint32_t periodic;
  uint32_t walls;  // bit 2a: wall at the min face of axis a, bit 2a+1: at the max face
  int32_t inflow_axis;
  double u_in[3];
  const Box* boxes;
  int32_t n_boxes;
  const uint8_t* solid;
  int32_t solid_level;
  int32_t solid_lo[3];
  int32_t solid_dims[3];
  double nu0;
  double accel0[3];
  int32_t mirror_lbgk;
  int32_t thermal;
  double pr, t0, glambda, t_ref;
  double wall_T[6];
  double solid_T;            // thermal: temperature of solid surfaces
  int32_t solid_isothermal;  // thermal: 1 = solid surfaces held at solid_T, 0 = adiabatic
  // curved solid surface (reading R10): 0 none (half-way, staircase), 1 sphere,
  // 2 cylinder along shape_axis, 3 plane normal to shape_axis; centre (a point
  // of the plane) and radius in coarse units; shape_solid_inside: the solid
  // is inside the sphere or cylinder (below the plane), else outside (above)
  int32_t shape_kind;
  double shape_c[3];
  double shape_r;
  int32_t shape_axis;
  int32_t shape_solid_inside;
};

struct Patch {
  int level = 0, parent = -1;
  std::vector<int> kids;
  long blo[3]{}, bhi[3]{};  // box in parent coordinates (level >= 1)
  bool span[3]{};           // spans a periodic axis completely
  bool flo[3]{}, fhi[3]{};  // faces that are interfaces toward the parent
  long rlo[3]{}, rhi[3]{};  // region, this level's coordinates, inclusive
  long org[3]{}, dim[3]{};  // storage box
  double beta = 0, beta1 = 0;
  std::vector<uint8_t> exists, solid, inlet, vpre, vpost;
  std::vector<Pop> pre, post, gpre, gpost;
  std::vector<double> gamma;
  long size() const { return dim[0] * dim[1] * dim[2]; }
};

struct Sim {
  Desc d{};
  std::vector<uint8_t> solid_mask;
  std::vector<Patch> P;
  int nlev = 1;
  std::string err;
  bool thermal = false;

  bool periodic(int a) const { return (d.periodic >> a) & 1u; }
  bool wall(int a, int side) const { return (d.walls >> (2 * a + side)) & 1u; }
  long period(int lev, int a) const { return (long)d.n[a] << lev; }
  long maxc(int lev, int a) const { return (long)(d.n[a] - 1) << lev; }

  void wrap(int lev, long X[3]) const {
    for (int a = 0; a < 3; ++a)
      if (periodic(a)) {
        long N = period(lev, a);
        X[a] = ((X[a] % N) + N) % N;
      }
  }

  static bool in_range(long v, long lo, long hi) { return v >= lo && v <= hi; }

  bool in_region(const Patch& p, const long X[3]) const {
    for (int a = 0; a < 3; ++a)
      if (!in_range(X[a], p.rlo[a], p.rhi[a])) return false;
    return true;
  }

  // Parent hole of child c, X in parent coordinates (reading R3).
  bool in_hole(const Patch& c, const long X[3]) const {
    for (int a = 0; a < 3; ++a) {
      if (c.span[a]) continue;
      long lo = c.flo[a] ? c.blo[a] + 2 : LONG_MIN;
      long hi = c.fhi[a] ? c.bhi[a] - 2 : LONG_MAX;
      if (!in_range(X[a], lo, hi)) return false;
    }
    return true;
  }

  // Parent interface (twin nodes x_t,cf) of child c.
  bool in_iface(const Patch& c, const long X[3]) const {
    for (int a = 0; a < 3; ++a) {
      if (c.span[a]) continue;
      long lo = c.flo[a] ? c.blo[a] + 1 : LONG_MIN;
      long hi = c.fhi[a] ? c.bhi[a] - 1 : LONG_MAX;
      if (!in_range(X[a], lo, hi)) return false;
    }
    return !in_hole(c, X);
  }

  // Child-distance to the nearest interface face (child coordinates).
  long depth(const Patch& c, const long Y[3]) const {
    long d = LONG_MAX;
    for (int a = 0; a < 3; ++a) {
      if (c.span[a]) continue;
      if (c.flo[a]) d = std::min(d, Y[a] - 2 * c.blo[a]);
      if (c.fhi[a]) d = std::min(d, 2 * c.bhi[a] - Y[a]);
    }
    return d;
  }

  bool exists_at(const Patch& p, const long X[3]) const {
    if (!in_region(p, X)) return false;
    for (int k : p.kids)
      if (in_hole(P[k], X)) return false;
    return true;
  }

  bool solid_at(int lev, const long X[3]) const {
    if (solid_mask.empty() || lev != d.solid_level) return false;
    long o[3];
    for (int a = 0; a < 3; ++a) {
      o[a] = X[a] - d.solid_lo[a];
      if (o[a] < 0 || o[a] >= d.solid_dims[a]) return false;
    }
    return solid_mask[(size_t)((o[2] * d.solid_dims[1] + o[1]) * d.solid_dims[0] + o[0])] != 0;
  }

  long index_of(const Patch& p, const long X[3]) const {
    long o[3];
    for (int a = 0; a < 3; ++a) {
      o[a] = X[a] - p.org[a];
      if (o[a] < 0 || o[a] >= p.dim[a]) return -1;
    }
    long n = (o[2] * p.dim[1] + o[1]) * p.dim[0] + o[0];
    return p.exists[n] ? n : -1;
  }

  void coords(const Patch& p, long n, long X[3]) const {
    X[0] = p.org[0] + n % p.dim[0];
    X[1] = p.org[1] + (n / p.dim[0]) % p.dim[1];
    X[2] = p.org[2] + n / (p.dim[0] * p.dim[1]);
  }

  void fail(const std::string& m) const { throw std::runtime_error(m); }

  // Failures inside OpenMP loops are recorded and raised after the loop.
  std::string perr;
  void pfail(const char* m) {
#pragma omp critical(orc_perr)
    if (perr.empty()) perr = m;
  }
  void raise_pending() {
    if (!perr.empty()) {
      std::string m = perr;
      perr.clear();
      fail(m);
    }
  }

  // ---- state transfer onto another layout (regridding) ---------------------
  // Not in the paper, which leaves adaptive refinement to future work (its
  // conclusion); reading R9.  Every fluid node of this layout takes the state
  // of the source level nearest its own that holds it, trying its own level,
  // then finer levels (nearest first), then coarser ones (nearest first): from
  // the coinciding node when that level is as fine or finer, else trilinearly
  // from the corners of the source cell around it (rho, u and f - f^eq
  // interpolated; only corners of non-zero weight are needed).
  // The stored states are post-collision, whose f - f^eq is (1 - 2 beta) times
  // the pre-collision one in the shear part (the whole of it with the LBGK
  // mirror); the pre-collision part scales between levels with the ratio of
  // Eq. f_neq_rescaling_iso, beta_s / (r beta_t), r = dx_s / dx_t.  So the
  // stored f - f^eq is scaled by (1 - 2 beta_t)/(1 - 2 beta_s) beta_s/(r beta_t),
  // and dropped where 1 - 2 beta_s vanishes (a fully relaxed state keeps none).
  // Solid nodes take the rest state and inlet nodes the inflow equilibrium, as
  // at initialisation.  Returns the number of fluid nodes no source level
  // holds (they take the rest state).
  long transfer_from(const Sim& src) {
    long missing = 0;
    const double rest[3] = {0, 0, 0};
    for (Patch& p : P) {
      std::vector<int> order(src.P.size());
      for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
      auto rank = [&](int k) {
        const int dl = src.P[k].level - p.level;
        return dl >= 0 ? dl : 1000 - dl;
      };
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rank(a) < rank(b); });
      for (long m = 0; m < p.size(); ++m) {
        if (!p.exists[m]) continue;
        if (p.solid[m]) {
          p.post[m] = feq(1.0, rest);
          p.vpost[m] = 0;
          continue;
        }
        if (p.inlet[m]) {
          p.post[m] = feq(1.0, d.u_in);
          p.vpost[m] = 1;
          continue;
        }
        long X[3];
        coords(p, m, X);
        bool done = false;
        for (int qi : order) {
          const Patch& q = src.P[qi];
          const int dl = q.level - p.level;
          double rho = 0, u[3] = {0, 0, 0};
          Pop neq{};
          if (dl >= 0) {
            const long sc = 1L << dl;
            long Y[3] = {X[0] * sc, X[1] * sc, X[2] * sc};
            src.wrap(q.level, Y);
            long n = src.index_of(q, Y);
            if (n < 0 || q.solid[n] || !q.vpost[n]) continue;
            Macro mc = macro(q.post[n]);
            Pop fe = feq(mc.rho, mc.u);
            rho = mc.rho;
            for (int a = 0; a < 3; ++a) u[a] = mc.u[a];
            for (int i = 0; i < Q; ++i) neq[i] = q.post[n][i] - fe[i];
          } else {
            const long sdiv = 1L << (-dl);
            long base[3];
            double fr[3];
            for (int a = 0; a < 3; ++a) {
              base[a] = X[a] >= 0 ? X[a] / sdiv : -((-X[a] + sdiv - 1) / sdiv);
              fr[a] = (double)(X[a] - base[a] * sdiv) / (double)sdiv;
            }
            bool ok = true;
            for (int c = 0; c < 8 && ok; ++c) {
              double w = 1.0;
              long Y[3];
              for (int a = 0; a < 3; ++a) {
                const int bit = (c >> a) & 1;
                w *= bit ? fr[a] : 1.0 - fr[a];
                Y[a] = base[a] + bit;
              }
              if (w == 0.0) continue;
              src.wrap(q.level, Y);
              long n = src.index_of(q, Y);
              if (n < 0 || q.solid[n] || !q.vpost[n]) {
                ok = false;
                break;
              }
              Macro mc = macro(q.post[n]);
              Pop fe = feq(mc.rho, mc.u);
              rho += w * mc.rho;
              for (int a = 0; a < 3; ++a) u[a] += w * mc.u[a];
              for (int i = 0; i < Q; ++i) neq[i] += w * (q.post[n][i] - fe[i]);
            }
            if (!ok) continue;
          }
          const double r = std::ldexp(1.0, -dl);  // dx_s / dx_t = 2^(level_t - level_s)
          const double post_s = 1.0 - 2.0 * q.beta, post_t = 1.0 - 2.0 * p.beta;
          const double factor = std::fabs(post_s) < 1e-12 ? 0.0 : (post_t / post_s) * q.beta / (r * p.beta);
          Pop fe = feq(rho, u);
          for (int i = 0; i < Q; ++i) p.post[m][i] = fe[i] + factor * neq[i];
          p.vpost[m] = 1;
          done = true;
          break;
        }
        if (!done) {
          p.post[m] = feq(1.0, rest);
          p.vpost[m] = 1;
          ++missing;
        }
      }
    }
    return missing;
  }

  // ---- construction -------------------------------------------------------
  bool pr_gt1() const { return thermal && d.pr > 1.0; }

  void build(const Desc& desc) {
    d = desc;
    thermal = d.thermal != 0;
    if (thermal && !(d.pr > 0.0)) fail("Prandtl number must be positive");
    for (int a = 0; a < 3; ++a)
      if (d.n[a] < 4) fail("domain extent below 4");
    for (int a = 0; a < 3; ++a) {
      if (periodic(a) && (wall(a, 0) || wall(a, 1))) fail("periodic axis with walls");
      if (!periodic(a) && a != d.inflow_axis && !(wall(a, 0) && wall(a, 1)))
        fail("non-periodic axis needs walls on both faces or the inflow");
    }
    if (d.inflow_axis >= 0 && (periodic(d.inflow_axis) || wall(d.inflow_axis, 0) || wall(d.inflow_axis, 1)))
      fail("inflow axis must be open");
    // level 0
    Patch root;
    root.level = 0;
    for (int a = 0; a < 3; ++a) {
      root.span[a] = periodic(a);
      root.rlo[a] = 0;
      root.rhi[a] = periodic(a) ? period(0, a) - 1 : maxc(0, a);
    }
    P.push_back(root);
    // refinement boxes, sorted by level (boxes of level l nest in a box of level l-1)
    int maxlev = 0;
    for (int b = 0; b < d.n_boxes; ++b) maxlev = std::max(maxlev, (int)d.boxes[b].level);
    for (int lev = 1; lev <= maxlev; ++lev)
      for (int b = 0; b < d.n_boxes; ++b) {
        const Box& bx = d.boxes[b];
        if (bx.level != lev) continue;
        Patch c;
        c.level = lev;
        for (int a = 0; a < 3; ++a) {
          if (bx.lo[a] > bx.hi[a]) fail("empty box");
          c.span[a] = periodic(a) && bx.lo[a] == 0 && bx.hi[a] == d.n[a] - 1;
          c.blo[a] = (long)bx.lo[a] << (lev - 1);
          c.bhi[a] = (long)bx.hi[a] << (lev - 1);
          if (c.span[a]) {
            c.rlo[a] = 0;
            c.rhi[a] = period(lev, a) - 1;
          } else {
            c.rlo[a] = 2 * c.blo[a];
            c.rhi[a] = 2 * c.bhi[a];
            c.flo[a] = !(bx.lo[a] == 0 && wall(a, 0));
            c.fhi[a] = !(bx.hi[a] == d.n[a] - 1 && wall(a, 1));
            if ((c.flo[a] || c.fhi[a]) && c.bhi[a] - c.blo[a] < 8) fail("box narrower than 8 parent nodes");
          }
        }
        // parent: the level-(lev-1) patch whose region contains the box
        int par = -1;
        for (size_t q = 0; q < P.size(); ++q) {
          if (P[q].level != lev - 1) continue;
          bool inside = true;
          for (int a = 0; a < 3; ++a) {
            if (c.span[a]) {
              if (!P[q].span[a]) inside = false;
              continue;
            }
            if (c.blo[a] < P[q].rlo[a] || c.bhi[a] > P[q].rhi[a]) inside = false;
          }
          if (inside) par = (int)q;
        }
        if (par < 0) fail("box does not nest in a parent patch");
        c.parent = par;
        P.push_back(c);
        P[par].kids.push_back((int)P.size() - 1);
        nlev = std::max(nlev, lev + 1);
      }
    // relaxation parameters: beta_0 from Eq. (visc) with c_s^2 = 1/3, then
    // beta_f = 1/(1 + r(1/beta_c - 1)) per level, r = 2 (Sec. III.A).
    double beta = 1.0 / (6.0 * d.nu0 + 1.0);
    double beta1 = 0.0;
    if (thermal) {
      // Sec. II.B: Pr <= 1: nu = (1/(2 beta) - 1/2) T0, alpha_th = (1/(2 beta1) - 1/2) T0;
      // Pr > 1: the roles of beta and beta1 swap
      double nu = d.nu0;
      double alpha = nu / d.pr;
      const double b_nu = 1.0 / (2.0 * nu / d.t0 + 1.0), b_alpha = 1.0 / (2.0 * alpha / d.t0 + 1.0);
      beta = pr_gt1() ? b_alpha : b_nu;
      beta1 = pr_gt1() ? b_nu : b_alpha;
    }
    std::vector<double> betas(nlev), betas1(nlev);
    for (int l = 0; l < nlev; ++l) {
      betas[l] = beta;
      betas1[l] = beta1;
      beta = 1.0 / (1.0 + 2.0 * (1.0 / beta - 1.0));
      if (thermal) beta1 = 1.0 / (1.0 + 2.0 * (1.0 / beta1 - 1.0));
    }
    if (d.solid && d.solid_dims[0] > 0) {
      size_t ns = (size_t)d.solid_dims[0] * d.solid_dims[1] * d.solid_dims[2];
      solid_mask.assign(d.solid, d.solid + ns);
    }
    for (auto& p : P) {
      p.beta = betas[p.level];
      p.beta1 = betas1[p.level];
      // storage box = bounding box of existing nodes of the region
      long lo[3] = {LONG_MAX, LONG_MAX, LONG_MAX}, hi[3] = {LONG_MIN, LONG_MIN, LONG_MIN};
      long X[3];
      for (X[2] = p.rlo[2]; X[2] <= p.rhi[2]; ++X[2])
        for (X[1] = p.rlo[1]; X[1] <= p.rhi[1]; ++X[1])
          for (X[0] = p.rlo[0]; X[0] <= p.rhi[0]; ++X[0]) {
            if (!exists_at(p, X)) continue;
            for (int a = 0; a < 3; ++a) {
              lo[a] = std::min(lo[a], X[a]);
              hi[a] = std::max(hi[a], X[a]);
            }
          }
      if (lo[0] > hi[0]) fail("patch with no nodes");
      for (int a = 0; a < 3; ++a) {
        p.org[a] = lo[a];
        p.dim[a] = hi[a] - lo[a] + 1;
      }
      long n = p.size();
      p.exists.assign(n, 0);
      p.solid.assign(n, 0);
      p.inlet.assign(n, 0);
      p.vpre.assign(n, 0);
      p.vpost.assign(n, 0);
      p.pre.assign(n, Pop{});
      p.post.assign(n, Pop{});
      p.gamma.assign(n, 2.0);
      if (thermal) {
        p.gpre.assign(n, Pop{});
        p.gpost.assign(n, Pop{});
      }
      for (long m = 0; m < n; ++m) {
        coords(p, m, X);
        p.exists[m] = exists_at(p, X);
        p.solid[m] = p.exists[m] && solid_at(p.level, X);
        p.inlet[m] = p.exists[m] && p.level == 0 && d.inflow_axis >= 0 && X[d.inflow_axis] == 0;
      }
      if (d.inflow_axis >= 0 && p.level > 0 && p.rlo[d.inflow_axis] < 2)
        fail("refinement box too close to the inflow face");
    }
  }

  // ---- curved solid surfaces (reading R10) ----------------------------------
  // Fraction q in (0, 1] of the link from node X (level lev) along c_k at which
  // it enters the solid side of the analytic surface: the root of
  // |P + t D - C|^2 = R^2 (sphere; cylinder without the axis component) or of
  // P_a + t D_a = C_a (plane), P = X h, D = c_k h, h = 2^-lev.  Without a
  // surface, or without a root in (0, 1], q = 1/2: half-way bounce-back.
  double wall_q(int lev, const long X[3], int k) const {
    if (d.shape_kind == 0) return 0.5;
    const double h = 1.0 / (double)(1L << lev);
    double P[3], D[3];
    for (int a = 0; a < 3; ++a) {
      P[a] = (double)X[a] * h;
      D[a] = (double)cvel(k, a) * h;
    }
    double t = -1.0;
    if (d.shape_kind == 3) {
      const int a = d.shape_axis;
      if (D[a] != 0.0) t = (d.shape_c[a] - P[a]) / D[a];
    } else {
      double A = 0, B = 0, C = -d.shape_r * d.shape_r;
      for (int a = 0; a < 3; ++a) {
        if (d.shape_kind == 2 && a == d.shape_axis) continue;
        const double pc = P[a] - d.shape_c[a];
        A += D[a] * D[a];
        B += 2.0 * D[a] * pc;
        C += pc * pc;
      }
      const double disc = B * B - 4.0 * A * C;
      if (A > 0.0 && disc >= 0.0) {
        // entering the body from outside: the first root; leaving a cavity: the second
        const double sq = std::sqrt(disc);
        t = d.shape_solid_inside ? (-B - sq) / (2.0 * A) : (-B + sq) / (2.0 * A);
      }
    }
    return (t > 0.0 && t <= 1.0) ? t : 0.5;
  }

  // Population i arriving at fluid node m (coordinates X) from a solid
  // neighbour X - c_i, from the post-collision state (reading R10): with the
  // wall at fraction q of the link from X along c_ib (ib the opposite of i),
  // follow the particle that leaves along c_ib and returns along c_i within
  // one step, and interpolate linearly along the link (Bouzidi, Firdaouss &
  // Lallemand 2001):
  //   q < 1/2: it left from X - (1 - 2q) c_ib, between X and the fluid node
  //            X + c_i behind:  a = 2q a'(X) + (1 - 2q) a'(X + c_i), along ib;
  //   q >= 1/2: it lands at X + (2q - 1) c_ib; with the population along i
  //            that X sends to X + c_i:
  //            f_i(X) = (1/(2q)) a + ((2q - 1)/(2q)) f'_i(X),  a = f'_ib(X);
  // where a is the reflected value: f'_ib for bounce-back, -g'_ib + w for the
  // anti-bounce-back of a surface at a fixed temperature (w the wall term).
  // q = 1/2 is half-way bounce-back; without a usable node behind, q < 1/2
  // falls back to it.
  double incoming(const Patch& p, long m, const long X[3], int i, double q, const std::vector<Pop>& post,
                  bool anti, double w) const {
    const int ib = opposite(i);
    if (q < 0.5) {
      long Bk[3];
      for (int a = 0; a < 3; ++a) Bk[a] = X[a] + cvel(i, a);
      bool in = true;
      for (int a = 0; a < 3; ++a)
        if (!periodic(a) && (Bk[a] < 0 || Bk[a] > maxc(p.level, a))) in = false;
      long b = -1;
      if (in) {
        wrap(p.level, Bk);
        b = index_of(p, Bk);
      }
      if (b >= 0 && !p.solid[b] && p.vpost[b]) {
        const double mix = 2.0 * q * post[m][ib] + (1.0 - 2.0 * q) * post[b][ib];
        return anti ? -mix + w : mix;
      }
      return anti ? -post[m][ib] + w : post[m][ib];
    }
    const double a = anti ? -post[m][ib] + w : post[m][ib];
    return a / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * post[m][i];
  }

  // ---- streaming (left-hand side of Eq. f_equations) ----------------------
  // pre(X)_i = post(X - c_i)_i, with the boundary rules of reading R6.
  void stream(Patch& p) {
    const int lev = p.level;
    const long n = p.size();
#pragma omp parallel for schedule(static)
    for (long m = 0; m < n; ++m) {
      if (!p.exists[m] || p.solid[m]) {
        p.vpre[m] = 0;
        continue;
      }
      if (p.inlet[m]) {  // fixed equilibrium node
        p.pre[m] = p.post[m];
        if (thermal) p.gpre[m] = p.gpost[m];
        p.vpre[m] = p.vpost[m];
        continue;
      }
      long X[3];
      coords(p, m, X);
      bool ok = true;
      for (int i = 0; i < Q && ok; ++i) {
        long S[3];
        int wall_axis = -1, wall_side = 0;
        for (int a = 0; a < 3; ++a) S[a] = X[a] - cvel(i, a);
        for (int a = 0; a < 3; ++a) {
          if (periodic(a)) continue;
          if (S[a] < 0) {
            if (wall(a, 0)) { wall_axis = a; wall_side = 0; }
            else ok = false;
          } else if (S[a] > maxc(lev, a)) {
            if (wall(a, 1)) { wall_axis = a; wall_side = 1; }
            else if (a == d.inflow_axis) S[a] = maxc(lev, a);  // zero-gradient outlet
            else ok = false;
          }
        }
        if (!ok) break;
        bool bounce = wall_axis >= 0, solid_wall = false;
        if (!bounce) {
          wrap(lev, S);
          bounce = solid_wall = solid_at(lev, S);
        }
        if (bounce) {
          if (!p.vpost[m]) { ok = false; break; }
          // domain walls: half-way; solid surfaces: at the fraction q of the
          // analytic surface (half-way without one)
          const double q = solid_wall ? wall_q(lev, X, opposite(i)) : 0.5;
          p.pre[m][i] = incoming(p, m, X, i, q, p.post, false, 0.0);
          if (thermal) {
            if (wall_axis >= 0 || (solid_wall && d.solid_isothermal)) {
              // anti-bounce-back to the wall equilibrium at rest, temperature
              // wall_T of the face, or solid_T of an isothermal solid surface
              double Tw = wall_axis >= 0 ? d.wall_T[2 * wall_axis + wall_side] : d.solid_T;
              double rho = 0;
              for (int k = 0; k < Q; ++k) rho += p.post[m][k];
              double zero[3] = {0, 0, 0};
              double E2 = rho * 3.0 * Tw;  // 2 rho E with u = 0
              Pop gw = geq(rho, zero, E2, d.t0);
              p.gpre[m][i] = incoming(p, m, X, i, q, p.gpost, true, gw[i] + gw[opposite(i)]);
            } else {
              p.gpre[m][i] = incoming(p, m, X, i, q, p.gpost, false, 0.0);
            }
          }
          continue;
        }
        long s = index_of(p, S);
        if (s < 0 || !p.vpost[s]) { ok = false; break; }
        p.pre[m][i] = p.post[s][i];
        if (thermal) p.gpre[m][i] = p.gpost[s][i];
      }
      p.vpre[m] = ok;
    }
  }

  // ---- collision (right-hand side of Eq. f_equations) ---------------------
  void collide(Patch& p) {
    const long n = p.size();
    double du[3];
    double scale = 1.0 / (double)(1L << p.level);  // du_f = du_c / r per level
    for (int a = 0; a < 3; ++a) du[a] = d.accel0[a] * scale;
#pragma omp parallel for schedule(static)
    for (long m = 0; m < n; ++m) {
      if (!p.exists[m] || p.solid[m]) { p.vpost[m] = 0; continue; }
      if (p.inlet[m]) { p.vpost[m] = 1; continue; }
      if (!p.vpre[m]) { p.vpost[m] = 0; continue; }
      if (thermal)
        p.gamma[m] = thermal_collide(p.pre[m], p.gpre[m], p.beta, p.beta1, d.t0, d.glambda, d.t_ref, scale,
                                     d.mirror_lbgk != 0, pr_gt1(), p.post[m], p.gpost[m]);
      else
        p.gamma[m] = kbc_collide(p.pre[m], p.beta, du, d.mirror_lbgk != 0, NAN, p.post[m]);
      p.vpost[m] = 1;
    }
  }

  // ---- coupling (Sec. III.A, III.B; algorithm steps 3 and 4) ---------------
  // Rescale the non-equilibrium part of (f, g) from a level with (beta_s, beta1_s)
  // to one with (beta_t, beta1_t): interface_rescale with this simulation's model.
  void rescale(const Pop& f, const Pop& g, double beta_s, double beta_t, double beta1_s, double beta1_t,
               double r_st, Pop& fo, Pop& go, Pop* fneq_out, Pop* gneq_out, Macro* mac_out,
               ThermalMacro* tmac_out) const {
    interface_rescale(thermal, pr_gt1(), d.t0, f, g, beta_s, beta_t, beta1_s, beta1_t, r_st, fo, go, fneq_out,
                      gneq_out, mac_out, tmac_out);
  }

  // Centred four-point Lagrange weights at the midpoint of nodes x = -3,-1,1,3
  // (units of half a parent spacing), from the Lagrange basis polynomials.
  static void lagrange4(double w[4]) {
    const double x[4] = {-3.0, -1.0, 1.0, 3.0};
    for (int k = 0; k < 4; ++k) {
      double l = 1.0;
      for (int m = 0; m < 4; ++m)
        if (m != k) l *= (0.0 - x[m]) / (x[k] - x[m]);
      w[k] = l;
    }
  }

  void couple(Patch& par, Patch& ch) {
    const Pop zero{};
    // (i) parent twins x_t,cf <- rescaled child state at the same position
    {
      const long n = par.size();
#pragma omp parallel for schedule(static)
      for (long m = 0; m < n; ++m) {
        if (!par.exists[m]) continue;
        long X[3];
        coords(par, m, X);
        if (!in_iface(ch, X)) continue;
        long Y[3] = {2 * X[0], 2 * X[1], 2 * X[2]};
        wrap(ch.level, Y);
        long s = index_of(ch, Y);
        if (s < 0 || !ch.vpre[s]) { pfail("coarse twin without a valid fine twin"); continue; }
        Pop go;
        rescale(ch.pre[s], thermal ? ch.gpre[s] : zero, ch.beta, par.beta, ch.beta1, par.beta1, 0.5, par.pre[m],
                go, nullptr, nullptr, nullptr, nullptr);
        if (thermal) par.gpre[m] = go;
        par.vpre[m] = 1;
      }
      raise_pending();
    }
    // (ii) fine twins x_t,fc and (iii) reconstruction nodes x_r
    double w4[4];
    lagrange4(w4);
    const long n = ch.size();
#pragma omp parallel for schedule(dynamic, 64)
    for (long m = 0; m < n; ++m) {
      if (!ch.exists[m]) continue;
      long Y[3];
      coords(ch, m, Y);
      if (depth(ch, Y) > 1) continue;
      bool odd[3];
      int noff = 0;
      for (int a = 0; a < 3; ++a) {
        odd[a] = (Y[a] & 1) != 0;
        noff += odd[a];
      }
      if (noff == 0) {  // twin node: rescale the parent state
        long X[3] = {Y[0] / 2, Y[1] / 2, Y[2] / 2};
        wrap(par.level, X);
        long s = index_of(par, X);
        if (s < 0 || !par.vpre[s]) { pfail("fine twin without a valid coarse twin"); continue; }
        Pop go;
        rescale(par.pre[s], thermal ? par.gpre[s] : zero, par.beta, ch.beta, par.beta1, ch.beta1, 2.0, ch.pre[m],
                go, nullptr, nullptr, nullptr, nullptr);
        if (thermal) ch.gpre[m] = go;
        ch.vpre[m] = 1;
        continue;
      }
      // reconstruction: tensor four-point Lagrange over the off-lattice axes of
      // rho, u (and 2 rho E) and of the fine-scale non-equilibrium parts
      double rho = 0, u[3] = {0, 0, 0}, T = 0;
      bool bad = false;
      Pop fneq{}, gneq{};
      long pos[3][4];
      double wt[3][4];
      int cnt[3];
      for (int a = 0; a < 3; ++a) {
        if (odd[a]) {
          cnt[a] = 4;
          for (int k = 0; k < 4; ++k) {
            pos[a][k] = (Y[a] + 2 * k - 3) / 2;  // Y/2 - 3/2, -1/2, +1/2, +3/2
            wt[a][k] = w4[k];
          }
        } else {
          cnt[a] = 1;
          pos[a][0] = Y[a] / 2;
          wt[a][0] = 1.0;
        }
      }
      for (int kz = 0; kz < cnt[2]; ++kz)
        for (int ky = 0; ky < cnt[1]; ++ky)
          for (int kx = 0; kx < cnt[0]; ++kx) {
            double w = wt[0][kx] * wt[1][ky] * wt[2][kz];
            long X[3] = {pos[0][kx], pos[1][ky], pos[2][kz]};
            wrap(par.level, X);
            Pop sf, sg, sfneq, sgneq;
            Macro mc;
            ThermalMacro tm{};
            long s = index_of(par, X);
            if (s >= 0) {
              if (!par.vpre[s]) { pfail("reconstruction sample on an invalid coarse node"); bad = true; continue; }
              rescale(par.pre[s], thermal ? par.gpre[s] : zero, par.beta, ch.beta, par.beta1, ch.beta1, 2.0, sf,
                      sg, &sfneq, &sgneq, &mc, &tm);
            } else {
              if (!in_hole(ch, X)) { pfail("reconstruction sample outside both levels"); bad = true; continue; }
              long Ys[3] = {2 * X[0], 2 * X[1], 2 * X[2]};
              wrap(ch.level, Ys);
              long t = index_of(ch, Ys);
              if (t < 0 || !ch.vpre[t]) { pfail("reconstruction sample on an invalid fine node"); bad = true; continue; }
              // already in fine units: factor 1
              rescale(ch.pre[t], thermal ? ch.gpre[t] : zero, ch.beta, ch.beta, ch.beta1, ch.beta1, 1.0, sf, sg,
                      &sfneq, &sgneq, &mc, &tm);
            }
            rho += w * mc.rho;
            for (int a = 0; a < 3; ++a) u[a] += w * mc.u[a];
            for (int i = 0; i < Q; ++i) fneq[i] += w * sfneq[i];
            if (thermal) {
              T += w * tm.T;
              for (int i = 0; i < Q; ++i) gneq[i] += w * sgneq[i];
            }
          }
      if (bad) continue;
      Pop fe = feq(rho, u);
      for (int i = 0; i < Q; ++i) ch.pre[m][i] = fe[i] + fneq[i];
      if (thermal) {
        double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        Pop ge = geq(rho, u, rho * (3.0 * T + u2), d.t0);
        for (int i = 0; i < Q; ++i) ch.gpre[m][i] = ge[i] + gneq[i];
      }
      ch.vpre[m] = 1;
    }
    raise_pending();
  }

  // ---- time stepping (Sec. III.C, generalised recursively to L levels) ------
  void collide_from(int lev) {
    for (auto& p : P)
      if (p.level >= lev) collide(p);
  }

  void advance(int lev) {
    if (lev + 1 < nlev) {
      advance(lev + 1);
      collide_from(lev + 1);
      advance(lev + 1);
    }
    for (auto& p : P)
      if (p.level == lev) stream(p);
    if (lev + 1 < nlev)
      for (auto& c : P)
        if (c.level == lev + 1) couple(P[c.parent], c);
  }

  void step() {
    advance(0);
    collide_from(0);
    for (auto& p : P)
      for (long m = 0; m < p.size(); ++m)
        if (p.exists[m] && !p.solid[m] && !p.vpost[m]) {
          long X[3];
          coords(p, m, X);
          fail("node without a valid state after a coarse step: level " + std::to_string(p.level) + " at (" +
               std::to_string(X[0]) + "," + std::to_string(X[1]) + "," + std::to_string(X[2]) + ")");
        }
  }

  // Drag F_d of Sec. IV A 2 (flow past a sphere), read as the momentum-exchange
  // force of the solid links: a post-collision population f'_j at a fluid
  // node x whose neighbour x + c_j is solid leaves along c_j and f_{-j}(x) of
  // the next pull arrives back (half-way bounce-back: f'_j itself, so 2 c_j
  // f'_j; curved surfaces: the interpolated value of reading R10), handing
  // the solid c_j (f'_j + f_{-j}) per substep.  Coarse units: a level-l node
  // carries 8^-l of a coarse volume and a level-l substep lasts 2^-l of a
  // coarse step, so each link counts 4^-l.  Evaluated on the current
  // post-collision state (what the next substep streams).
  void drag(double F[3]) const {
    F[0] = F[1] = F[2] = 0;
    for (const auto& p : P) {
      const double scale = 1.0 / (double)(1L << (2 * p.level));
      for (long m = 0; m < p.size(); ++m) {
        if (!p.exists[m] || p.solid[m] || !p.vpost[m]) continue;
        long X[3];
        coords(p, m, X);
        for (int j = 0; j < Q; ++j) {
          long S[3];
          bool inside = true;
          for (int a = 0; a < 3; ++a) {
            S[a] = X[a] + cvel(j, a);
            if (!periodic(a) && (S[a] < 0 || S[a] > maxc(p.level, a))) inside = false;
          }
          if (!inside) continue;
          wrap(p.level, S);
          if (!solid_at(p.level, S)) continue;
          const int i = opposite(j);
          const double back = incoming(p, m, X, i, wall_q(p.level, X, j), p.post, false, 0.0);
          for (int a = 0; a < 3; ++a) F[a] += (double)cvel(j, a) * (p.post[m][j] + back) * scale;
        }
      }
    }
  }

  double node_updates_per_step() const {
    double s = 0;
    for (auto& p : P) {
      long c = 0;
      for (long m = 0; m < p.size(); ++m) c += p.exists[m] && !p.solid[m];
      s += (double)c * (double)(1L << p.level);
    }
    return s;
  }
};

}  // namespace orc

// ---------------------------------------------------------------------------
// C interface (consumed by oracle/oracle.py through ctypes).

using namespace orc;

extern "C" {

typedef struct {
  int32_t level;
  int32_t lo[3], hi[3];
} orc_box;

typedef struct {
  int32_t n[3];
  uint32_t periodic;
  uint32_t walls;
  int32_t inflow_axis;
  double u_in[3];
  const orc_box* boxes;
  int32_t n_boxes;
  const uint8_t* solid;
  int32_t solid_level;
  int32_t solid_lo[3];
  int32_t solid_dims[3];
  double nu0;
  double accel0[3];
  int32_t mirror_lbgk;
  int32_t thermal;
  double pr, t0, glambda, t_ref;
  double wall_T[6];
  double solid_T;
  int32_t solid_isothermal;
  int32_t shape_kind;
  double shape_c[3];
  double shape_r;
  int32_t shape_axis;
  int32_t shape_solid_inside;
} orc_desc;

static std::string g_last_error;

const char* orc_last_error(void) { return g_last_error.c_str(); }

// Interface rescaling of one node (Sec. III.A): thermal 0/1, pr_gt1 0/1;
// g and go may be NULL for the isothermal model.
void orc_rescale(const double* f, const double* g, double beta_s, double beta_t, double beta1_s, double beta1_t,
                 double r_st, int thermal, int pr_gt1, double t0, double* fo, double* go) {
  Pop F{}, G{}, FO{}, GO{};
  for (int i = 0; i < Q; ++i) {
    F[i] = f[i];
    G[i] = g ? g[i] : 0.0;
  }
  interface_rescale(thermal != 0, pr_gt1 != 0, t0, F, G, beta_s, beta_t, beta1_s, beta1_t, r_st, FO, GO, nullptr,
                    nullptr, nullptr, nullptr);
  for (int i = 0; i < Q; ++i) {
    fo[i] = FO[i];
    if (go) go[i] = GO[i];
  }
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void* orc_create(const orc_desc* cd) {
  try {
    Sim* s = new Sim();
    Desc d{};
    std::memcpy(d.n, cd->n, sizeof d.n);
    d.periodic = cd->periodic;
    d.walls = cd->walls;
    d.inflow_axis = cd->inflow_axis;
    std::memcpy(d.u_in, cd->u_in, sizeof d.u_in);
    d.boxes = reinterpret_cast<const Box*>(cd->boxes);
    d.n_boxes = cd->n_boxes;
    d.solid = cd->solid;
    d.solid_level = cd->solid_level;
    std::memcpy(d.solid_lo, cd->solid_lo, sizeof d.solid_lo);
    std::memcpy(d.solid_dims, cd->solid_dims, sizeof d.solid_dims);
    d.nu0 = cd->nu0;
    std::memcpy(d.accel0, cd->accel0, sizeof d.accel0);
    d.mirror_lbgk = cd->mirror_lbgk;
    d.thermal = cd->thermal;
    d.pr = cd->pr;
    d.t0 = cd->t0;
    d.glambda = cd->glambda;
    d.t_ref = cd->t_ref;
    std::memcpy(d.wall_T, cd->wall_T, sizeof d.wall_T);
    d.solid_T = cd->solid_T;
    d.solid_isothermal = cd->solid_isothermal;
    d.shape_kind = cd->shape_kind;
    std::memcpy(d.shape_c, cd->shape_c, sizeof d.shape_c);
    d.shape_r = cd->shape_r;
    d.shape_axis = cd->shape_axis;
    d.shape_solid_inside = cd->shape_solid_inside;
    try {
      s->build(d);
    } catch (...) {
      delete s;
      throw;
    }
    s->d.boxes = nullptr;
    s->d.solid = nullptr;
    return s;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return nullptr;
  }
}

void orc_destroy(void* h) { delete static_cast<Sim*>(h); }

int orc_num_patches(void* h) { return (int)static_cast<Sim*>(h)->P.size(); }

int orc_patch_info(void* h, int p, int32_t* level, int32_t* parent, int64_t org[3], int64_t dim[3], double* beta,
                   double* beta1) {
  Sim* s = static_cast<Sim*>(h);
  if (p < 0 || p >= (int)s->P.size()) return -1;
  const Patch& q = s->P[p];
  *level = q.level;
  *parent = q.parent;
  for (int a = 0; a < 3; ++a) {
    org[a] = q.org[a];
    dim[a] = q.dim[a];
  }
  *beta = q.beta;
  *beta1 = q.beta1;
  return 0;
}

// mask: 1 fluid node, 0 not a node of this patch (hole or outside), 2 solid node
int orc_patch_mask(void* h, int p, uint8_t* out) {
  Sim* s = static_cast<Sim*>(h);
  if (p < 0 || p >= (int)s->P.size()) return -1;
  const Patch& q = s->P[p];
  for (long m = 0; m < q.size(); ++m) out[m] = q.exists[m] ? (q.solid[m] ? 2 : 1) : 0;
  return 0;
}

// Sets f = f^eq(rho, u) (and g = g^eq(rho, u, T)) on all fluid nodes; inlet nodes
// take the inflow equilibrium; arrays are [z][y][x] over the storage box.
int orc_init_equilibrium(void* h, int p, const double* rho, const double* ux, const double* uy, const double* uz,
                         const double* T) {
  Sim* s = static_cast<Sim*>(h);
  if (p < 0 || p >= (int)s->P.size()) return -1;
  Patch& q = s->P[p];
  for (long m = 0; m < q.size(); ++m) {
    if (!q.exists[m]) continue;
    double r = rho[m];
    double u[3] = {ux[m], uy[m], uz[m]};
    double Tm = T ? T[m] : s->d.t0;
    if (q.solid[m]) {
      r = 1.0;
      u[0] = u[1] = u[2] = 0.0;
    }
    if (q.inlet[m]) {
      r = 1.0;
      for (int a = 0; a < 3; ++a) u[a] = s->d.u_in[a];
    }
    q.post[m] = feq(r, u);
    if (s->thermal) {
      double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
      double E2 = r * (3.0 * Tm + u2);
      q.gpost[m] = geq(r, u, E2, s->d.t0);
    }
    q.vpost[m] = !q.solid[m];
  }
  return 0;
}

// Populations as [27][z][y][x]; which = 0 for f, 1 for g.
int orc_get_pop(void* h, int p, int which, double* out) {
  Sim* s = static_cast<Sim*>(h);
  if (p < 0 || p >= (int)s->P.size()) return -1;
  Patch& q = s->P[p];
  if (which == 1 && !s->thermal) return -1;
  const long n = q.size();
  for (long m = 0; m < n; ++m)
    for (int i = 0; i < Q; ++i) out[i * n + m] = (which ? q.gpost[m][i] : q.post[m][i]);
  return 0;
}

int orc_set_pop(void* h, int p, int which, const double* in) {
  Sim* s = static_cast<Sim*>(h);
  if (p < 0 || p >= (int)s->P.size()) return -1;
  Patch& q = s->P[p];
  if (which == 1 && !s->thermal) return -1;
  const long n = q.size();
  for (long m = 0; m < n; ++m) {
    for (int i = 0; i < Q; ++i) (which ? q.gpost[m][i] : q.post[m][i]) = in[i * n + m];
    if (q.exists[m] && !q.solid[m]) q.vpost[m] = 1;
  }
  return 0;
}

// State transfer from another oracle with the same domain (reading R9);
// returns the number of fluid nodes no source level holds, or -1.
long orc_transfer(void* dst, void* src) {
  Sim* a = static_cast<Sim*>(dst);
  Sim* b = static_cast<Sim*>(src);
  if (!a || !b || a->thermal || b->thermal) return -1;
  for (int k = 0; k < 3; ++k)
    if (a->d.n[k] != b->d.n[k] || a->periodic(k) != b->periodic(k)) return -1;
  return a->transfer_from(*b);
}

int orc_step(void* h, int64_t n) {
  Sim* s = static_cast<Sim*>(h);
  try {
    for (int64_t k = 0; k < n; ++k) s->step();
    return 0;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return -1;
  }
}

// rho, u (= j/rho + du/2, reading R5), T and the last gamma per node; [z][y][x].
int orc_moments(void* h, int p, double* rho, double* u, double* T, double* gamma) {
  Sim* s = static_cast<Sim*>(h);
  if (p < 0 || p >= (int)s->P.size()) return -1;
  Patch& q = s->P[p];
  const long n = q.size();
  double scale = 1.0 / (double)(1L << q.level);
  for (long m = 0; m < n; ++m) {
    Macro mc = macro(q.post[m]);
    double du[3] = {s->d.accel0[0] * scale, s->d.accel0[1] * scale, s->d.accel0[2] * scale};
    double Tm = 0;
    if (s->thermal) {
      ThermalMacro tm = thermal_macro(q.post[m], q.gpost[m]);
      Tm = tm.T;
      du[0] = du[1] = 0;
      du[2] = s->d.glambda * (tm.T - s->d.t_ref) * scale;
    }
    if (rho) rho[m] = mc.rho;
    if (u)
      for (int a = 0; a < 3; ++a) u[a * n + m] = mc.u[a] + 0.5 * du[a];
    if (T) T[m] = Tm;
    if (gamma) gamma[m] = q.gamma[m];
  }
  return 0;
}

double orc_node_updates_per_step(void* h) { return static_cast<Sim*>(h)->node_updates_per_step(); }

// Momentum-exchange force on the solid nodes of the current state (coarse units).
void orc_drag(void* h, double* F) { static_cast<Sim*>(h)->drag(F); }

// ---- single-node functions for the pins -----------------------------------
void orc_feq(double rho, const double* u, double* out) {
  Pop f = feq(rho, u);
  std::memcpy(out, f.data(), sizeof(double) * Q);
}

void orc_split(const double* f, double* k, double* s, double* h) {
  Pop pf, pk, ps, ph;
  std::memcpy(pf.data(), f, sizeof(double) * Q);
  kbc_split(pf, pk, ps, ph);
  std::memcpy(k, pk.data(), sizeof(double) * Q);
  std::memcpy(s, ps.data(), sizeof(double) * Q);
  std::memcpy(h, ph.data(), sizeof(double) * Q);
}

double orc_collide(const double* f, double beta, const double* du, int lbgk, double gamma_forced, double* out) {
  Pop pf, po;
  std::memcpy(pf.data(), f, sizeof(double) * Q);
  double g = kbc_collide(pf, beta, du, lbgk != 0, gamma_forced, po);
  std::memcpy(out, po.data(), sizeof(double) * Q);
  return g;
}

void orc_geq(double rho, const double* u, double T, double t0, double* out) {
  double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  Pop g = geq(rho, u, rho * (3.0 * T + u2), t0);
  std::memcpy(out, g.data(), sizeof(double) * Q);
}

double orc_thermal_collide(const double* f, const double* g, double beta, double beta1, double t0, double glambda,
                           double t_ref, int pr_gt1, double* fo, double* go) {
  Pop pf, pg, pfo, pgo;
  std::memcpy(pf.data(), f, sizeof(double) * Q);
  std::memcpy(pg.data(), g, sizeof(double) * Q);
  double gm = thermal_collide(pf, pg, beta, beta1, t0, glambda, t_ref, 1.0, false, pr_gt1 != 0, pfo, pgo);
  std::memcpy(fo, pfo.data(), sizeof(double) * Q);
  std::memcpy(go, pgo.data(), sizeof(double) * Q);
  return gm;
}

void orc_lagrange_weights(double* w) { Sim::lagrange4(w); }

}  // extern "C"
