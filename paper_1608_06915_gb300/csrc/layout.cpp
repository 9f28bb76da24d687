// Layout builder: patches, node classes and interface tables of a refined grid.
//
// Geometry (Sec. III, the overlap layout of Fig. 1, which the text describes
// but does not draw): a level-(l+1) box [a,b] (in level-l coordinates) holds
// child nodes at every half-integer position of [a,b].  Across each box face
// that is neither a wall face nor a periodic span, the child interface is two
// child nodes wide (depth 0 and 1) and the parent keeps one interface layer:
// parent nodes of [a+1,b-1] outside the hole [a+2,b-2] are the twins x_t,cf.
// Child interface nodes whose three coordinates fall on the parent lattice are
// the fine twins x_t,fc; the others are reconstruction nodes x_r, rebuilt by
// the centred four-point Lagrange rule (Eq. interp) along each off-lattice
// axis from samples at parent positions +-1/2 and +-3/2 parent spacings away.
// A sample under a parent twin or inside the parent hole is taken from the
// child node at that position.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_map>

#include "grid.h"

namespace lbm {
namespace {

constexpr int64_t kLo = INT64_MIN / 4;
constexpr int64_t kHi = INT64_MAX / 4;

inline int cvel(int i, int a) { return (a == 0 ? i % 3 : a == 1 ? (i / 3) % 3 : i / 9) - 1; }

// Fraction q in (0, 1] of the link from node X (level lev) along c_j at which
// it crosses into the solid side of the descriptor's analytic surface (the
// first crossing into a body, the way out of a cavity); 1/2 when the surface
// does not cross the link there.  Positions in coarse units: X 2^-lev.
double wall_fraction(const lbm_desc& d, int lev, const int64_t X[3], int j) {
  const double h = std::ldexp(1.0, -lev);
  double from[3], step[3];
  for (int a = 0; a < 3; ++a) {
    from[a] = (double)X[a] * h;
    step[a] = (double)cvel(j, a) * h;
  }
  double t = -1.0;
  if (d.shape_kind == 3) {
    const int a = d.shape_axis;
    if (step[a] != 0.0) t = (d.shape_c[a] - from[a]) / step[a];
  } else if (d.shape_kind == 1 || d.shape_kind == 2) {
    // |from + t step - c|^2 = r^2 over the axes of the shape
    double qa = 0.0, qb = 0.0, qc = -d.shape_r * d.shape_r;
    for (int a = 0; a < 3; ++a) {
      if (d.shape_kind == 2 && a == d.shape_axis) continue;
      const double rel = from[a] - d.shape_c[a];
      qa += step[a] * step[a];
      qb += 2.0 * step[a] * rel;
      qc += rel * rel;
    }
    const double disc = qb * qb - 4.0 * qa * qc;
    if (qa > 0.0 && disc >= 0.0) {
      const double root = std::sqrt(disc);
      t = (d.shape_solid_inside ? -qb - root : -qb + root) / (2.0 * qa);
    }
  }
  return (t > 0.0 && t <= 1.0) ? t : 0.5;
}

struct Geo {
  HostGrid& g;

  void wrap(int lev, int64_t X[3]) const {
    for (int a = 0; a < 3; ++a)
      if (g.periodic(a)) {
        int64_t N = g.period(lev, a);
        X[a] = ((X[a] % N) + N) % N;
      }
  }
  bool in_region(const HostPatch& p, const int64_t X[3]) const {
    for (int a = 0; a < 3; ++a)
      if (X[a] < p.rlo[a] || X[a] > p.rhi[a]) return false;
    return true;
  }
  // X in the parent's coordinates
  bool in_hole(const HostPatch& c, const int64_t X[3]) const {
    for (int a = 0; a < 3; ++a) {
      if (c.span[a]) continue;
      int64_t lo = c.flo[a] ? c.blo[a] + 2 : kLo, hi = c.fhi[a] ? c.bhi[a] - 2 : kHi;
      if (X[a] < lo || X[a] > hi) return false;
    }
    return true;
  }
  bool in_cf(const HostPatch& c, const int64_t X[3]) const {
    for (int a = 0; a < 3; ++a) {
      if (c.span[a]) continue;
      int64_t lo = c.flo[a] ? c.blo[a] + 1 : kLo, hi = c.fhi[a] ? c.bhi[a] - 1 : kHi;
      if (X[a] < lo || X[a] > hi) return false;
    }
    return !in_hole(c, X);
  }
  int64_t depth(const HostPatch& c, const int64_t Y[3]) const {
    int64_t d = kHi;
    for (int a = 0; a < 3; ++a) {
      if (c.span[a]) continue;
      if (c.flo[a]) d = std::min(d, Y[a] - 2 * c.blo[a]);
      if (c.fhi[a]) d = std::min(d, 2 * c.bhi[a] - Y[a]);
    }
    return d;
  }
  bool exists(const HostPatch& p, const int64_t X[3]) const {
    if (!in_region(p, X)) return false;
    for (int k : p.kids)
      if (in_hole(g.P[k], X)) return false;
    return true;
  }
  bool solid_at(int lev, const int64_t X[3]) const {
    if (g.solid.empty() || lev != g.desc.solid_level) return false;
    int64_t o[3];
    for (int a = 0; a < 3; ++a) {
      o[a] = X[a] - g.desc.solid_lo[a];
      if (o[a] < 0 || o[a] >= g.desc.solid_dims[a]) return false;
    }
    return g.solid[(size_t)((o[2] * g.desc.solid_dims[1] + o[1]) * g.desc.solid_dims[0] + o[0])] != 0;
  }
  // storage index of a global coordinate, -1 outside the storage box
  int64_t index(const HostPatch& p, const int64_t X[3]) const {
    int64_t o[3];
    for (int a = 0; a < 3; ++a) {
      o[a] = X[a] - p.org[a];
      if (o[a] < 0 || o[a] >= p.dim[a]) return -1;
    }
    return (o[2] * p.dim[1] + o[1]) * p.nxp + o[0];
  }
  void coords(const HostPatch& p, int64_t n, int64_t X[3]) const {
    X[0] = p.org[0] + n % p.nxp;
    X[1] = p.org[1] + (n / p.nxp) % p.dim[1];
    X[2] = p.org[2] + n / (p.nxp * p.dim[1]);
  }

  // Pull source of direction i at node X: 0 plain (src set), 1 bounce-back,
  // 2 outlet clamp (src set), 3 missing.
  int resolve(const HostPatch& p, const int64_t X[3], int i, int64_t* src) const {
    int64_t S[3];
    bool clamp = false;
    for (int a = 0; a < 3; ++a) S[a] = X[a] - cvel(i, a);
    for (int a = 0; a < 3; ++a) {
      if (g.periodic(a)) continue;
      if (S[a] < 0) {
        if (g.wall(a, 0)) return 1;
        return 3;
      }
      if (S[a] > g.maxc(p.level, a)) {
        if (g.wall(a, 1)) return 1;
        if (a == g.desc.inflow_axis) {
          S[a] = g.maxc(p.level, a);
          clamp = true;
        } else {
          return 3;
        }
      }
    }
    wrap(p.level, S);
    int64_t j = index(p, S);
    if (j < 0) return 3;
    uint8_t t = p.type[j];
    if (t == T_SKIP) return 3;
    if (t == T_SOLID) return 1;
    *src = j;
    return clamp ? 2 : 0;
  }
};

std::string fmt_node(const char* what, int lev, const int64_t X[3]) {
  return std::string(what) + " at level " + std::to_string(lev) + " node (" + std::to_string(X[0]) + "," +
         std::to_string(X[1]) + "," + std::to_string(X[2]) + ")";
}

}  // namespace

std::string build_layout(HostGrid& g) {
  const lbm_desc& d = g.desc;
  Geo geo{g};
  for (int a = 0; a < 3; ++a) {
    if (d.n[a] < 4) return "domain extent below 4 nodes";
    if (g.periodic(a) && (g.wall(a, 0) || g.wall(a, 1))) return "periodic axis with walls";
    if (!g.periodic(a) && a != d.inflow_axis && !(g.wall(a, 0) && g.wall(a, 1)))
      return "a non-periodic axis needs walls on both faces, or the inflow";
  }
  if (d.inflow_axis >= 3) return "inflow axis out of range";
  if (d.inflow_axis >= 0 &&
      (g.periodic(d.inflow_axis) || g.wall(d.inflow_axis, 0) || g.wall(d.inflow_axis, 1)))
    return "inflow axis must be non-periodic and without walls";
  if (d.nu0 <= 0) return "nu0 must be positive";
  if (g.thermal && !(d.pr > 0)) return "Prandtl number must be positive";
  if (g.thermal && std::fabs(d.t0 - 1.0 / 3.0) > 1e-12) return "thermal model needs T0 = 1/3 (D3Q27)";
  g.pr_gt1 = g.thermal && d.pr > 1.0;

  g.P.clear();
  HostPatch root;
  for (int a = 0; a < 3; ++a) {
    root.span[a] = g.periodic(a);
    root.rlo[a] = 0;
    root.rhi[a] = g.periodic(a) ? g.period(0, a) - 1 : g.maxc(0, a);
  }
  g.P.push_back(root);
  int maxlev = 0;
  for (auto& b : g.boxes) {
    if (b.level < 1 || b.level > 12) return "box level out of range";
    maxlev = std::max(maxlev, (int)b.level);
  }
  g.nlev = maxlev + 1;
  for (int lev = 1; lev <= maxlev; ++lev)
    for (auto& bx : g.boxes) {
      if (bx.level != lev) continue;
      HostPatch c;
      c.level = lev;
      for (int a = 0; a < 3; ++a) {
        if (bx.lo[a] > bx.hi[a] || bx.lo[a] < 0 || bx.hi[a] > d.n[a] - 1) return "box outside the domain";
        c.span[a] = g.periodic(a) && bx.lo[a] == 0 && bx.hi[a] == d.n[a] - 1;
        c.blo[a] = (int64_t)bx.lo[a] << (lev - 1);
        c.bhi[a] = (int64_t)bx.hi[a] << (lev - 1);
        if (c.span[a]) {
          c.rlo[a] = 0;
          c.rhi[a] = g.period(lev, a) - 1;
        } else {
          c.rlo[a] = 2 * c.blo[a];
          c.rhi[a] = 2 * c.bhi[a];
          c.flo[a] = !(bx.lo[a] == 0 && g.wall(a, 0));
          c.fhi[a] = !(bx.hi[a] == d.n[a] - 1 && g.wall(a, 1));
          if ((c.flo[a] || c.fhi[a]) && c.bhi[a] - c.blo[a] < 8)
            return "refinement box narrower than 8 parent spacings";
          if (a == d.inflow_axis && (bx.lo[a] < 2 || bx.hi[a] > d.n[a] - 3))
            return "refinement box too close to the inflow or outflow face";
        }
      }
      int par = -1;
      for (size_t q = 0; q < g.P.size(); ++q) {
        const HostPatch& pp = g.P[q];
        if (pp.level != lev - 1) continue;
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
          if (c.span[a]) {
            inside = inside && pp.span[a];
            continue;
          }
          inside = inside && c.blo[a] >= pp.rlo[a] && c.bhi[a] <= pp.rhi[a];
        }
        if (inside) {
          if (par >= 0) return "box nests in two parent boxes";
          par = (int)q;
        }
      }
      if (par < 0) return "refinement box does not nest in a box of the level below";
      c.parent = par;
      g.P.push_back(c);
      g.P[par].kids.push_back((int)g.P.size() - 1);
    }
  // sibling boxes must not overlap (holes and interfaces are per child)
  for (size_t q = 1; q < g.P.size(); ++q)
    for (size_t r = q + 1; r < g.P.size(); ++r) {
      if (g.P[q].level != g.P[r].level) continue;
      bool overlap = true;
      for (int a = 0; a < 3; ++a)
        overlap = overlap && !(g.P[q].rhi[a] + 16 < g.P[r].rlo[a] || g.P[r].rhi[a] + 16 < g.P[q].rlo[a]);
      if (overlap) return "boxes of one level overlap or lie within 8 parent spacings";
    }

  // relaxation parameters (Eq. visc, Sec. II.B, Sec. III.A)
  double beta, beta1 = 0;
  if (g.thermal) {
    // Sec. II.B: for Pr <= 1 beta sets nu and beta1 alpha_th; for Pr > 1 they swap
    const double b_nu = 1.0 / (2.0 * d.nu0 / d.t0 + 1.0);
    const double b_alpha = 1.0 / (2.0 * (d.nu0 / d.pr) / d.t0 + 1.0);
    beta = g.pr_gt1 ? b_alpha : b_nu;
    beta1 = g.pr_gt1 ? b_nu : b_alpha;
  } else {
    beta = 1.0 / (6.0 * d.nu0 + 1.0);
  }
  std::vector<double> bl(g.nlev), bl1(g.nlev);
  for (int l = 0; l < g.nlev; ++l) {
    bl[l] = beta;
    bl1[l] = beta1;
    beta = 1.0 / (1.0 + 2.0 * (1.0 / beta - 1.0));
    if (g.thermal) beta1 = 1.0 / (1.0 + 2.0 * (1.0 / beta1 - 1.0));
  }

  // storage boxes and first-pass classes
  for (auto& p : g.P) {
    p.beta = bl[p.level];
    p.beta1 = bl1[p.level];
    int64_t lo[3] = {kHi, kHi, kHi}, hi[3] = {kLo, kLo, kLo};
    // bounding box of the nodes: a node exists unless it lies in a child hole;
    // the region minus holes is scanned axis by axis on its extreme lines
    int64_t X[3];
    for (X[2] = p.rlo[2]; X[2] <= p.rhi[2]; ++X[2])
      for (X[1] = p.rlo[1]; X[1] <= p.rhi[1]; ++X[1]) {
        // on one x-row the existing nodes form at most a few runs; test both ends of
        // every run cheaply by scanning the row only when a hole touches it
        bool row_has_hole = false;
        for (int k : p.kids) {
          const HostPatch& c = g.P[k];
          bool hit = true;
          for (int a = 1; a < 3; ++a) {
            if (c.span[a]) continue;
            int64_t l2 = c.flo[a] ? c.blo[a] + 2 : kLo, h2 = c.fhi[a] ? c.bhi[a] - 2 : kHi;
            hit = hit && X[a] >= l2 && X[a] <= h2;
          }
          row_has_hole = row_has_hole || hit;
        }
        if (!row_has_hole) {
          lo[0] = std::min(lo[0], p.rlo[0]);
          hi[0] = std::max(hi[0], p.rhi[0]);
          for (int a = 1; a < 3; ++a) {
            lo[a] = std::min(lo[a], X[a]);
            hi[a] = std::max(hi[a], X[a]);
          }
          continue;
        }
        for (X[0] = p.rlo[0]; X[0] <= p.rhi[0]; ++X[0]) {
          if (!geo.exists(p, X)) continue;
          for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], X[a]);
            hi[a] = std::max(hi[a], X[a]);
          }
        }
      }
    if (lo[0] > hi[0]) return "a patch has no nodes";
    for (int a = 0; a < 3; ++a) {
      p.org[a] = lo[a];
      p.dim[a] = hi[a] - lo[a] + 1;
      if (p.span[a] && p.dim[a] != g.period(p.level, a)) return "periodic span broken by a refinement hole";
      if (p.dim[a] > (1 << 24)) return "patch extent too large";
    }
    p.nxp = (p.dim[0] + 31) / 32 * 32;
    p.plane = p.nxp * p.dim[1] * p.dim[2];
    if (p.plane >= (int64_t)UINT32_MAX) return "patch has too many nodes for 32-bit indices";
    p.type.assign((size_t)p.plane, T_SKIP);
  }
  // first pass: classes from geometry (independent per node)
  for (auto& p : g.P) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t z = 0; z < p.dim[2]; ++z) {
      int64_t X[3];
      for (int64_t y = 0; y < p.dim[1]; ++y)
        for (int64_t x = 0; x < p.dim[0]; ++x) {
          const int64_t n = (z * p.dim[1] + y) * p.nxp + x;
          X[0] = p.org[0] + x;
          X[1] = p.org[1] + y;
          X[2] = p.org[2] + z;
          if (!geo.exists(p, X)) continue;
          uint8_t t = T_BULK;  // provisional fluid class
          if (geo.solid_at(p.level, X)) t = T_SOLID;
          else if (p.level == 0 && d.inflow_axis >= 0 && X[d.inflow_axis] == 0) t = T_INLET;
          else {
            for (int k : p.kids)
              if (geo.in_cf(g.P[k], X)) t = T_CF;
            if (t != T_CF && p.level > 0) {
              int64_t dp = geo.depth(p, X);
              if (dp == 0) t = T_D0;
              else if (dp == 1) t = T_D1;
            }
          }
          p.type[n] = t;
        }
    }
  }
  // second pass: resolve pull sources of fluid nodes.  Nodes away from the
  // storage edges (or on spanned axes) only need their 26 neighbours' classes;
  // edge nodes go through the full resolution (walls, outlet, wrap).
  for (auto& p : g.P) {
    std::vector<uint8_t> mark((size_t)p.plane, 0);
    std::string perr;
    int64_t fluid = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : fluid)
    for (int64_t z = 0; z < p.dim[2]; ++z) {
      int64_t X[3];
      for (int64_t y = 0; y < p.dim[1]; ++y)
        for (int64_t x = 0; x < p.dim[0]; ++x) {
          const int64_t n = (z * p.dim[1] + y) * p.nxp + x;
          const uint8_t t = p.type[n];
          if (t == T_SKIP || t == T_SOLID) continue;
          ++fluid;
          if (t != T_BULK && t != T_D1) continue;
          const int64_t L[3] = {x, y, z};
          bool interior = true;
          for (int a = 0; a < 3; ++a) interior = interior && (p.span[a] || (L[a] > 0 && L[a] < p.dim[a] - 1));
          bool special = false, missing = false;
          if (interior) {
            for (int i = 0; i < 27 && !missing; ++i) {
              int64_t S[3];
              for (int a = 0; a < 3; ++a) {
                S[a] = L[a] - cvel(i, a);
                if (S[a] < 0) S[a] += p.dim[a];
                else if (S[a] >= p.dim[a]) S[a] -= p.dim[a];
              }
              const uint8_t tt = p.type[(S[2] * p.dim[1] + S[1]) * p.nxp + S[0]];
              if (tt == T_SKIP) missing = true;
              else if (tt == T_SOLID) special = true;
            }
          }
          if (!interior || missing) {
            special = false;
            X[0] = p.org[0] + x;
            X[1] = p.org[1] + y;
            X[2] = p.org[2] + z;
            for (int i = 0; i < 27; ++i) {
              int64_t s;
              int r = geo.resolve(p, X, i, &s);
              if (r == 3) {
#pragma omp critical(lbm_layout_err)
                if (perr.empty()) perr = fmt_node("unresolved pull source", p.level, X);
                break;
              }
              if (r != 0) special = true;
            }
          }
          if (t == T_BULK && special) mark[n] = 1;
        }
    }
    if (!perr.empty()) return perr;
    for (int64_t n = 0; n < p.plane; ++n)
      if (mark[n]) p.type[n] = T_BC;
    p.n_fluid = fluid;
    if (p.level > 0 && g.P[p.parent].level != p.level - 1) return "internal: parent level";
  }
  // stream-collide tiles
  //
  // A tile is 128 nodes along x at one (y, z).  The TMA path updates every
  // node of a tile from one rule per source row j = (c_y + 1) + 3 (c_z + 1):
  // pull from the neighbour row (wrapping only on spanned axes), or bounce back
  // when that row lies beyond a wall across y or z (bit j of the tile's bounce
  // mask); the first node of a row may be a fixed inlet node (written back
  // unchanged) and the last the zero-gradient outlet.  Nodes that are not
  // updated in the substep -- depth-0 and, on even substeps, depth-1 interface
  // nodes, parent twins, hole and solid nodes -- are overwritten too: explode
  // and coalesce rewrite the interface nodes later in the same instant, and no
  // valid node ever reads the others.  Updated nodes whose pulls the row rule
  // does not give (solid neighbours, x walls) are recomputed node by node
  // right after the tile pass (fix-up list); a tile with more such nodes than
  // regular ones goes to the node-by-node path whole.
  // Source of population i at patch-local L: 0 plain neighbour, 1 bounce-back
  // from a y or z wall, 3 the zero-gradient outlet across x (the node itself
  // along x), 2 anything else (solid, x wall).
  auto outcome = [&](const HostPatch& p, const int64_t L[3], int i) -> int {
    const int64_t X[3] = {p.org[0] + L[0], p.org[1] + L[1], p.org[2] + L[2]};
    int64_t src;
    const int r = geo.resolve(p, X, i, &src);
    if (r == 0 || r == 2) {
      const bool clamp = r == 2;
      if (clamp && !(d.inflow_axis == 0 && cvel(i, 0) == -1 && X[0] == g.maxc(p.level, 0) &&
                     L[0] == p.dim[0] - 1))
        return 2;
      int64_t S[3];
      for (int a = 0; a < 3; ++a) {
        S[a] = L[a] - (clamp && a == 0 ? 0 : cvel(i, a));
        if (S[a] < 0 || S[a] >= p.dim[a]) {
          if (!p.span[a]) return 2;
          S[a] += S[a] < 0 ? p.dim[a] : -p.dim[a];
        }
      }
      if (src != (S[2] * p.dim[1] + S[1]) * p.nxp + S[0]) return 2;
      return clamp ? 3 : 0;
    }
    if (r != 1) return 2;
    bool yz = false;
    for (int a = 1; a < 3; ++a) {
      const int64_t sa = X[a] - cvel(i, a);
      if (!g.periodic(a) && ((sa < 0 && g.wall(a, 0)) || (sa > g.maxc(p.level, a) && g.wall(a, 1)))) yz = true;
    }
    const int64_t sx = X[0] - cvel(i, 0);
    return yz && (g.periodic(0) || (sx >= 0 && sx <= g.maxc(p.level, 0))) ? 1 : 2;
  };
  for (auto& p : g.P) {
    p.ntx = (p.dim[0] + 127) / 128;
    for (int k = 0; k < 2; ++k) {
      p.tiles_pure[k].clear();
      p.tiles_half[k].clear();
      p.tiles_mixed[k].clear();
      p.tiles_all[k].clear();
      p.fix_nodes[k].clear();
    }
    struct Rows {
      std::vector<uint64_t> pure[2];
      std::vector<uint32_t> mixed[2], all[2], fix[2];
      double ntma[2] = {0, 0};
    };
    std::vector<Rows> rows(p.dim[2]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t z = 0; z < p.dim[2]; ++z) {
      Rows& R = rows[z];
      for (int64_t y = 0; y < p.dim[1]; ++y) {
        // the row rule: source rows beyond a wall across y or z bounce back
        uint32_t bm = 0;
        for (int j = 0; j < 9; ++j) {
          const int64_t sy = p.org[1] + y - ((j % 3) - 1), sz = p.org[2] + z - ((j / 3) - 1);
          const bool by = !g.periodic(1) && ((sy < 0 && g.wall(1, 0)) || (sy > g.maxc(p.level, 1) && g.wall(1, 1)));
          const bool bz = !g.periodic(2) && ((sz < 0 && g.wall(2, 0)) || (sz > g.maxc(p.level, 2) && g.wall(2, 1)));
          if (by || bz) bm |= 1u << j;
        }
        for (int64_t tx = 0; tx < p.ntx; ++tx) {
          int active[2] = {0, 0};
          bool inlet = false, outlet = false;
          std::vector<uint32_t> odd_nodes[2];  // updated nodes the row rule does not give
          for (int64_t x = tx * 128; x < std::min<int64_t>(p.dim[0], tx * 128 + 128); ++x) {
            const int64_t m = (z * p.dim[1] + y) * p.nxp + x;
            const uint8_t t = p.type[m];
            if (t == T_INLET && d.inflow_axis == 0 && x == 0 && p.org[0] == 0) inlet = true;
            bool act[2];
            act[0] = t == T_BULK || t == T_BC;
            act[1] = act[0] || t == T_D1;
            if (!act[1]) continue;
            for (int k = 0; k < 2; ++k) active[k] += act[k];
            bool regular = true;
            if (t != T_BULK) {
              const int64_t L[3] = {x, y, z};
              for (int i = 0; i < 27 && regular; ++i) {
                const int o = outcome(p, L, i);
                if ((bm >> (i / 3)) & 1u) regular = o == 1;
                else if (o == 3) outlet = true;  // the outlet node reads itself along x
                else regular = o == 0;
              }
            }
            if (!regular)
              for (int k = 0; k < 2; ++k)
                if (act[k]) odd_nodes[k].push_back((uint32_t)m);
          }
          const uint32_t id = (uint32_t)((z * p.dim[1] + y) * p.ntx + tx);
          // the TMA path fetches the periodic wrap of x-spanning rows as 16-byte
          // boxes at x = dim - H: row-edge tiles need dim a multiple of 8 nodes
          const bool edge = tx == 0 || (tx + 1) * 128 >= p.dim[0];
          const bool wrap_ok = !p.span[0] || !edge || p.dim[0] % 8 == 0;
          for (int k = 0; k < 2; ++k) {
            if (active[k] == 0) continue;
            R.all[k].push_back(id);
            const int nodd = (int)odd_nodes[k].size();
            // the thermal tile pass has no inlet or outlet rule: such tiles go node by node
            const bool rule_ok = !g.thermal || (!inlet && !outlet);
            if (wrap_ok && rule_ok && 2 * nodd <= active[k]) {
              const uint64_t fl = (inlet ? 1ull : 0ull) | (outlet ? 2ull : 0ull);
              R.pure[k].push_back((uint64_t)tx | ((uint64_t)y << 16) | ((uint64_t)z << 32) | ((uint64_t)bm << 48) |
                                  (fl << 57));
              R.fix[k].insert(R.fix[k].end(), odd_nodes[k].begin(), odd_nodes[k].end());
              R.ntma[k] += active[k] - nodd;
            } else {
              R.mixed[k].push_back(id);
            }
          }
        }
      }
    }
    p.n_tma[0] = p.n_tma[1] = 0;
    for (auto& R : rows)
      for (int k = 0; k < 2; ++k) {
        p.n_tma[k] += R.ntma[k];
        p.tiles_pure[k].insert(p.tiles_pure[k].end(), R.pure[k].begin(), R.pure[k].end());
        for (uint64_t t : R.pure[k]) {
          const uint64_t tx = t & 0xffffu, rest = t & ~(uint64_t)0xffffu;
          p.tiles_half[k].push_back(rest | (2 * tx));
          if ((int64_t)(2 * tx + 1) * 64 < p.dim[0]) p.tiles_half[k].push_back(rest | (2 * tx + 1));
        }
        p.tiles_mixed[k].insert(p.tiles_mixed[k].end(), R.mixed[k].begin(), R.mixed[k].end());
        p.tiles_all[k].insert(p.tiles_all[k].end(), R.all[k].begin(), R.all[k].end());
        p.fix_nodes[k].insert(p.fix_nodes[k].end(), R.fix[k].begin(), R.fix[k].end());
      }
  }
  // momentum-exchange links of patches holding solid nodes
  for (auto& p : g.P) {
    p.drag_node.clear();
    p.drag_mask.clear();
    bool any = false;
    for (int64_t n = 0; n < p.plane && !any; ++n) any = p.type[n] == T_SOLID;
    if (!any) continue;
    int64_t X[3];
    for (int64_t n = 0; n < p.plane; ++n) {
      const uint8_t t = p.type[n];
      if (t == T_SKIP || t == T_SOLID) continue;
      geo.coords(p, n, X);
      uint32_t m = 0;
      for (int j = 0; j < 27; ++j) {
        int64_t S[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
          S[a] = X[a] + cvel(j, a);
          if (!g.periodic(a) && (S[a] < 0 || S[a] > g.maxc(p.level, a))) inside = false;
        }
        if (!inside) continue;
        geo.wrap(p.level, S);
        const int64_t s = geo.index(p, S);
        if (s >= 0 && p.type[s] == T_SOLID) m |= 1u << j;
      }
      if (m) {
        p.drag_node.push_back((uint32_t)n);
        p.drag_mask.push_back(m);
      }
    }
    // curved surface: the wall fraction of every solid link of the drag nodes
    p.wq.clear();
    p.wq_idx.clear();
    if (g.desc.shape_kind != 0 && !p.drag_node.empty()) {
      p.wq_idx.assign((size_t)p.plane, -1);
      p.wq.assign(27 * p.drag_node.size(), 0.5);
      for (size_t k = 0; k < p.drag_node.size(); ++k) {
        p.wq_idx[p.drag_node[k]] = (int32_t)k;
        geo.coords(p, p.drag_node[k], X);
        for (int j = 0; j < 27; ++j)
          if ((p.drag_mask[k] >> j) & 1u) p.wq[27 * k + j] = wall_fraction(g.desc, p.level, X, j);
      }
    }
  }
  // interface tables, stored on the child
  for (size_t ci = 1; ci < g.P.size(); ++ci) {
    HostPatch& c = g.P[ci];
    HostPatch& par = g.P[c.parent];
    std::unordered_map<uint64_t, uint32_t> ids;
    auto sample_id = [&](uint8_t kind, int64_t node) -> uint32_t {
      uint64_t key = ((uint64_t)kind << 40) | (uint64_t)node;
      auto it = ids.find(key);
      if (it != ids.end()) return it->second;
      uint32_t id = (uint32_t)c.smp_node.size();
      ids.emplace(key, id);
      c.smp_node.push_back((uint32_t)node);
      c.smp_kind.push_back(kind);
      return id;
    };
    // Reconstruction (Eq. interp) as separable four-point passes: a target
    // off-lattice along the axes of mask m interpolates, along the last of
    // them in the pass order below, four points at the coarse positions of
    // that axis -- samples when
    // no other axis is off-lattice, else intermediate points of mask m minus
    // that axis, built the same way.  Points are keyed by (mask, fine
    // position); ids carry their stage in the top two bits until numbered.
    constexpr uint32_t kStage1 = 1u << 30, kStage2 = 2u << 30, kIdMask = (1u << 30) - 1;
    // Axis order of the passes: axes with interface faces first, the others
    // after.  Then the last pass runs along a tangential axis, and the points
    // it combines lie on the interface layers themselves (they are targets),
    // not in rows reaching into the parent.
    int order_pos[3];
    {
      int pos = 0;
      for (int pass = 0; pass < 2; ++pass)
        for (int a = 0; a < 3; ++a) {
          const bool normal = c.flo[a] || c.fhi[a];
          if (normal == (pass == 0)) order_pos[a] = pos++;
        }
    }
    auto top_axis = [&](int m) {
      int t = -1;
      for (int a = 0; a < 3; ++a)
        if ((m >> a) & 1)
          if (t < 0 || order_pos[a] > order_pos[t]) t = a;
      return t;
    };
    std::unordered_map<uint64_t, uint32_t> pts[2];
    std::vector<uint32_t> psrc[2];   // 4 tagged sources per point
    std::vector<uint64_t> ppos[2];   // position key of each point (ordering)
    std::string err;
    auto pkey = [](int m, const int64_t Q[3]) -> uint64_t {
      const uint64_t o = 1ull << 19;
      return ((uint64_t)m << 60) | ((uint64_t)(Q[2] + o) << 40) | ((uint64_t)(Q[1] + o) << 20) | (uint64_t)(Q[0] + o);
    };
    std::function<uint32_t(int, const int64_t*)> point = [&](int m, const int64_t* Qin) -> uint32_t {
      int64_t Q[3] = {Qin[0], Qin[1], Qin[2]};
      geo.wrap(c.level, Q);
      if (m == 0) {
        int64_t X[3] = {Q[0] / 2, Q[1] / 2, Q[2] / 2};
        geo.wrap(par.level, X);
        const int64_t pj = geo.index(par, X);
        const bool parent_node = pj >= 0 && par.type[pj] != T_SKIP;
        if (parent_node && !geo.in_cf(c, X)) {
          const uint8_t pt = par.type[pj];
          if (pt != T_BULK && pt != T_BC) {
            if (err.empty()) err = fmt_node("reconstruction sample on a non-bulk parent node", par.level, X);
            return 0;
          }
          return sample_id(S_PARENT, pj);
        }
        if (!parent_node && !geo.in_hole(c, X)) {
          if (err.empty()) err = fmt_node("reconstruction sample outside both levels", par.level, X);
          return 0;
        }
        int64_t Ys[3] = {2 * X[0], 2 * X[1], 2 * X[2]};
        geo.wrap(c.level, Ys);
        const int64_t cj = geo.index(c, Ys);
        if (cj < 0 || (c.type[cj] != T_BULK && c.type[cj] != T_BC)) {
          if (err.empty()) err = fmt_node("reconstruction sample on a non-bulk child node", c.level, Ys);
          return 0;
        }
        return sample_id(S_CHILD, cj);
      }
      const int st = __builtin_popcount((unsigned)m) - 1;  // stage 0 or 1 (masks of one or two axes)
      const uint64_t key = pkey(m, Q);
      auto it = pts[st].find(key);
      if (it != pts[st].end()) return it->second;
      const int top = top_axis(m);
      uint32_t src[4];
      for (int k = 0; k < 4; ++k) {
        int64_t R[3] = {Q[0], Q[1], Q[2]};
        R[top] = Q[top] - 3 + 2 * k;
        src[k] = point(m & ~(1 << top), R);
      }
      const uint32_t id = (uint32_t)ppos[st].size() | (st == 0 ? kStage1 : kStage2);
      pts[st].emplace(key, id);
      ppos[st].push_back(key);
      for (int k = 0; k < 4; ++k) psrc[st].push_back(src[k]);
      return id;
    };
    std::vector<uint32_t> tnode, tsrc;  // targets: node, 4 tagged sources (a single source: others ~0)
    std::vector<uint8_t> tmask;
    int64_t Y[3];
    for (int64_t n = 0; n < c.plane; ++n) {
      const uint8_t t = c.type[n];
      if (t != T_D0 && t != T_D1) continue;
      geo.coords(c, n, Y);
      int m = 0;
      for (int a = 0; a < 3; ++a)
        if (Y[a] & 1) m |= 1 << a;
      tnode.push_back((uint32_t)n);
      tmask.push_back((uint8_t)m);
      if (m == 0) {
        tsrc.push_back(point(0, Y));
        for (int k = 0; k < 3; ++k) tsrc.push_back(~0u);
      } else {
        const int top = top_axis(m);
        for (int k = 0; k < 4; ++k) {
          int64_t R[3] = {Y[0], Y[1], Y[2]};
          R[top] = Y[top] - 3 + 2 * k;
          tsrc.push_back(point(m & ~(1 << top), R));
        }
      }
      if (!err.empty()) return err;
    }
    // a target that is itself an intermediate point reads that point
    for (size_t e = 0; e < tnode.size(); ++e) {
      const int m = tmask[e], pc = __builtin_popcount((unsigned)m);
      if (pc < 1 || pc > 2) continue;
      geo.coords(c, tnode[e], Y);
      int64_t Q[3] = {Y[0], Y[1], Y[2]};
      geo.wrap(c.level, Q);
      auto it = pts[pc - 1].find(pkey(m, Q));
      if (it == pts[pc - 1].end()) continue;
      tsrc[4 * e] = it->second;
      for (int k = 1; k < 4; ++k) tsrc[4 * e + k] = ~0u;
    }
    // number samples in storage order (kind, node) and points by position, so
    // that neighbouring nodes read neighbouring values
    const size_t ns = c.smp_node.size();
    std::vector<uint32_t> srank(ns), prank[2];
    {
      std::vector<uint32_t> order(ns);
      for (size_t k = 0; k < ns; ++k) order[k] = (uint32_t)k;
      std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        if (c.smp_kind[a] != c.smp_kind[b]) return c.smp_kind[a] < c.smp_kind[b];
        return c.smp_node[a] < c.smp_node[b];
      });
      std::vector<uint32_t> node(ns);
      std::vector<uint8_t> kind(ns);
      for (size_t k = 0; k < ns; ++k) {
        srank[order[k]] = (uint32_t)k;
        node[k] = c.smp_node[order[k]];
        kind[k] = c.smp_kind[order[k]];
      }
      c.smp_node.swap(node);
      c.smp_kind.swap(kind);
    }
    for (int st = 0; st < 2; ++st) {
      const size_t np = ppos[st].size();
      std::vector<uint32_t> order(np);
      for (size_t k = 0; k < np; ++k) order[k] = (uint32_t)k;
      // position order: z, y, x (the key's low 60 bits), then mask
      std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        const uint64_t ka = ppos[st][a], kb = ppos[st][b];
        const uint64_t m60 = (1ull << 60) - 1;
        if ((ka & m60) != (kb & m60)) return (ka & m60) < (kb & m60);
        return ka < kb;
      });
      prank[st].assign(np, 0);
      for (size_t k = 0; k < np; ++k) prank[st][order[k]] = (uint32_t)k;
      c.n_pt[st] = (uint32_t)np;
    }
    auto final_id = [&](uint32_t t) -> uint32_t {
      const uint32_t tag = t & ~kIdMask, v = t & kIdMask;
      if (tag == 0) return srank[v];
      if (tag == kStage1) return (uint32_t)ns + prank[0][v];
      return (uint32_t)ns + c.n_pt[0] + prank[1][v];
    };
    c.pt_src.assign(4 * ((size_t)c.n_pt[0] + c.n_pt[1]), 0);
    for (int st = 0; st < 2; ++st)
      for (size_t q = 0; q < ppos[st].size(); ++q) {
        const size_t row = (st == 0 ? 0 : c.n_pt[0]) + prank[st][q];
        for (int k = 0; k < 4; ++k) c.pt_src[4 * row + k] = final_id(psrc[st][4 * q + k]);
      }
    // entries: one-source targets first, then four-source targets, node order inside each
    c.ex_node.clear();
    c.ex_src.clear();
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) c.ex_one = (uint32_t)c.ex_node.size();
      for (size_t e = 0; e < tnode.size(); ++e) {
        const bool one = tsrc[4 * e + 1] == ~0u;
        if (one != (pass == 0)) continue;
        c.ex_node.push_back(tnode[e]);
        for (int k = 0; k < 4; ++k) c.ex_src.push_back(one && k > 0 ? 0u : final_id(tsrc[4 * e + k]));
      }
    }
    // consumers of each point column (the transpose of the two tables), by
    // counting sort: targets first, then points, each in index order
    {
      const size_t np = c.n_points(), nt = c.ex_node.size(), nq = (size_t)c.n_pt[0] + c.n_pt[1];
      c.use_ptr.assign(np + 1, 0);
      for (size_t k = 0; k < nt; ++k)
        for (int j = 0; j < (k < c.ex_one ? 1 : 4); ++j) ++c.use_ptr[c.ex_src[4 * k + j] + 1];
      for (size_t q = 0; q < nq; ++q)
        for (int j = 0; j < 4; ++j) ++c.use_ptr[c.pt_src[4 * q + j] + 1];
      for (size_t j = 0; j < np; ++j) c.use_ptr[j + 1] += c.use_ptr[j];
      c.use_ent.assign(c.use_ptr[np], 0);
      std::vector<uint32_t> fill(c.use_ptr.begin(), c.use_ptr.end() - 1);
      for (size_t k = 0; k < nt; ++k) {
        const bool one = k < c.ex_one;
        for (int j = 0; j < (one ? 1 : 4); ++j)
          c.use_ent[fill[c.ex_src[4 * k + j]]++] = (uint32_t)k | (one ? (1u << 30) : ((uint32_t)j << 28));
      }
      for (size_t q = 0; q < nq; ++q)
        for (int j = 0; j < 4; ++j)
          c.use_ent[fill[c.pt_src[4 * q + j]]++] = (uint32_t)(ns + q) | (1u << 31) | ((uint32_t)j << 28);
    }
    // coalesce pairs: parent twins x_t,cf and the coinciding child node
    int64_t X[3];
    for (int64_t n = 0; n < par.plane; ++n) {
      if (par.type[n] != T_CF) continue;
      geo.coords(par, n, X);
      if (!geo.in_cf(c, X)) continue;
      int64_t Yc[3] = {2 * X[0], 2 * X[1], 2 * X[2]};
      geo.wrap(c.level, Yc);
      int64_t cj = geo.index(c, Yc);
      if (cj < 0 || (c.type[cj] != T_BULK && c.type[cj] != T_BC))
        return fmt_node("parent twin without a bulk child twin", par.level, X);
      c.cf_parent.push_back((uint32_t)n);
      c.cf_child.push_back((uint32_t)cj);
    }
  }
  // parent twins that are also interface nodes of the parent's own parent
  for (auto& p : g.P)
    for (int64_t n = 0; n < p.plane; ++n)
      if (p.type[n] == T_CF && p.level > 0) {
        int64_t X[3];
        geo.coords(p, n, X);
        if (geo.depth(p, X) <= 1) return fmt_node("child box too close to its parent's interface", p.level, X);
      }
  return std::string();
}

size_t plan_memory(HostGrid& g) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t ncomp = g.thermal ? 59 : 31;
  for (auto& p : g.P) {
    size_t pop = 27 * (size_t)p.plane * g.pop_bytes;
    p.off_f[0] = take(pop);
    p.off_f[1] = take(pop);
    if (g.thermal) {
      p.off_g[0] = take(pop);
      p.off_g[1] = take(pop);
    }
    p.off_type = take((size_t)p.plane);
    p.off_tiles_pure[0] = take(8 * p.tiles_pure[0].size());
    p.off_tiles_pure[1] = take(8 * p.tiles_pure[1].size());
    p.off_tiles_half[0] = take(8 * p.tiles_half[0].size());
    p.off_tiles_half[1] = take(8 * p.tiles_half[1].size());
    p.off_tiles_all[0] = take(4 * p.tiles_all[0].size());
    p.off_tiles_all[1] = take(4 * p.tiles_all[1].size());
    p.off_tiles_mixed[0] = take(4 * p.tiles_mixed[0].size());
    p.off_tiles_mixed[1] = take(4 * p.tiles_mixed[1].size());
    p.off_fix_nodes[0] = take(4 * p.fix_nodes[0].size());
    p.off_fix_nodes[1] = take(4 * p.fix_nodes[1].size());
    p.off_ex_node = take(4 * p.ex_node.size());
    p.off_ex_src = take(4 * p.ex_src.size());
    p.off_pt_src = take(4 * p.pt_src.size());
    p.off_use_ptr = take(4 * p.use_ptr.size());
    p.off_use_ent = take(4 * p.use_ent.size());
    p.off_smp_node = take(4 * p.smp_node.size());
    p.off_smp_kind = take(p.smp_kind.size());
    p.off_smp_val = take(ncomp * p.n_points() * g.real_bytes);
    p.off_cf_parent = take(4 * p.cf_parent.size());
    p.off_cf_child = take(4 * p.cf_child.size());
    p.off_drag_node = take(4 * p.drag_node.size());
    p.off_drag_mask = take(4 * p.drag_mask.size());
    p.off_wq = take(8 * p.wq.size());
    p.off_wq_idx = take(4 * p.wq_idx.size());
  }
  return off;
}

}  // namespace lbm
