// C ABI of liblbm.so (declared in include/lbm.h) and the refined-step scheduler.
//
// Time stepping (Sec. III.C, generalised to L levels with r = 2): a coarse step
// is 2^(L-1) instants; level l is active at every 2^(L-1-l)-th instant, i.e.
// it takes 2^l steps.  At an instant every active patch is streamed and
// collided from its previous state into its other buffer; the patch's twin
// nodes toward each child are coalesced from the child's previous state; and
// when the patch's parent is active in the same instant (the patch's even
// steps), its interface layers (depth 0 and 1) are rebuilt from the parent by
// twin rescaling and reconstruction, then collided -- the explode step.  At
// the patch's odd steps its depth-1 layer is streamed normally and its depth-0
// layer is not needed.  This realises steps 1-5 of Sec. III.C without time
// interpolation: nothing ever reads a parent state between its own steps.
//
// Execution of an instant: one batched TMA tile pass over every active patch
// (isothermal model), then the node-by-node remainder, the coalesces and the
// explode chains on side streams, joined before the next instant; a coarse
// step is captured once per set of buffer indices and replayed as a CUDA
// graph.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "device.cuh"
#include "grid.h"
#include "kernels.h"

using lbm::HostGrid;
using lbm::HostPatch;

namespace {
constexpr int kDiagBlocks = 296;  // 2 per SM on 148+ SM parts; fixed for determinism
constexpr size_t kTmaBatchMax = 8;  // patches per TMA launch
std::string g_create_error;
}  // namespace

struct lbm_grid {
  HostGrid hg;
  std::string err;
  size_t need = 0, bytes = 0;
  uint8_t* base = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  size_t off_status = 0, off_partial = 0, off_diag_out = 0;
  double accel[3] = {0, 0, 0};
  // measurement: CUDA events around each launch of lbm_step while enabled
  struct Rec {
    int kind, level;
    double nodes;
    cudaEvent_t e0, e1;
  };
  bool timing = false;
  int variant = 0;         // TMA kernel variant (lbm_autotune)
  int wait_sleeps = 1 << 21;  // bound of the TMA passes' stage waits (lbm_wait_limit)
  int device = -1;         // device of the bound buffer
  bool presample = false;  // reconstruction samples beside the TMA pass (lbm_autotune)
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  // CUDA graphs of one coarse step, keyed by the buffer index of every patch;
  // the first step after binding runs directly, so that capture finds every
  // kernel loaded and configured
  bool graphs = true;
  bool stepped = false;
  cudaStream_t cap_stream = nullptr;
  struct StepGraph {
    std::vector<uint8_t> cur;
    cudaGraphExec_t exec;
  };
  std::vector<StepGraph> gcache;
  // CUDA graphs of the adjoint's reverse walk over a segment, keyed by the
  // buffer indices of lambda, the segment length and the caller's buffers;
  // they hold the indices the walk leaves behind
  struct AdjGraph {
    std::vector<uint8_t> lcur, lcur_after;
    int K;
    const void *lam, *ws;
    cudaGraphExec_t exec;
  };
  std::vector<AdjGraph> acache;
  bool adj_swept = false;
  // CUDA graphs of n recording steps of the adjoint's recompute, keyed by the
  // buffer indices, the record's device word, the record's size and n
  struct RecGraph {
    std::vector<uint8_t> cur;
    const unsigned long long* slot;
    size_t step_bytes;
    int n;
    cudaGraphExec_t exec;
  };
  std::vector<RecGraph> rcache;
  bool rec_warm = false;
  void drop_graphs() {
    for (auto& x : gcache) cudaGraphExecDestroy(x.exec);
    gcache.clear();
    for (auto& x : acache) cudaGraphExecDestroy(x.exec);
    acache.clear();
    for (auto& x : rcache) cudaGraphExecDestroy(x.exec);
    rcache.clear();
  }
  // side streams of the adjoint: coupling adjoints run beside the
  // stream-collide adjoint (their writes are reductions that commute)
  cudaStream_t adj_side[2] = {nullptr, nullptr};
  cudaEvent_t adj_fork = nullptr, adj_join[2] = {nullptr, nullptr};
  cudaEvent_t adj_sc = nullptr, adj_cf = nullptr;  // stream-collide and coalesce adjoints of an instant done
  cudaEvent_t adj_s0 = nullptr;                     // side stream 0's work so far

  // side streams of the forward step: [0] node-by-node remainders, [1], [2]
  // coupling chains, all beside each other after the TMA pass of an instant
  cudaStream_t fwd_side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fwd_fork = nullptr, fwd_join[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fwd_pre = nullptr;  // the instant's pre-states are ready (before its TMA pass)
  std::vector<cudaEvent_t> patch_done;  // thermal model: a patch's stream-collide has been issued
  // the adjoint's recording step: its snapshot copies run on rec_side beside
  // the instants; rec_ev[k] marks instant k issued, rec_cp[k] copy k done;
  // level 0's outer snapshot runs on rec_side0 (rec_l0: done)
  cudaStream_t rec_side = nullptr, rec_side0 = nullptr;
  cudaEvent_t rec_l0 = nullptr;
  std::vector<cudaEvent_t> rec_ev, rec_cp;
  ~lbm_grid() {
    if (rec_side) cudaStreamDestroy(rec_side);
    if (rec_side0) cudaStreamDestroy(rec_side0);
    if (rec_l0) cudaEventDestroy(rec_l0);
    for (auto& x : rec_ev)
      if (x) cudaEventDestroy(x);
    for (auto& x : rec_cp)
      if (x) cudaEventDestroy(x);
    for (auto& x : fwd_side)
      if (x) cudaStreamDestroy(x);
    if (fwd_fork) cudaEventDestroy(fwd_fork);
    if (fwd_pre) cudaEventDestroy(fwd_pre);
    for (auto& x : fwd_join)
      if (x) cudaEventDestroy(x);
    for (auto& x : patch_done)
      if (x) cudaEventDestroy(x);
    for (auto& x : adj_side)
      if (x) cudaStreamDestroy(x);
    if (adj_fork) cudaEventDestroy(adj_fork);
    if (adj_sc) cudaEventDestroy(adj_sc);
    if (adj_s0) cudaEventDestroy(adj_s0);
    if (adj_cf) cudaEventDestroy(adj_cf);

    for (auto& x : adj_join)
      if (x) cudaEventDestroy(x);
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (auto e : pool) cudaEventDestroy(e);
  }
};

namespace {

// Side streams take the highest priority: their kernels (coupling chains,
// short and latency-bound) are scheduled ahead of the remaining blocks of a
// large kernel on the bound stream.  Graphs keep the priority per node.
cudaError_t side_stream(cudaStream_t* s) {
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  return e ? e : cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, greatest);
}

lbm_status fail(lbm_grid* g, lbm_status s, const std::string& m) {
  if (g) g->err = m;
  else g_create_error = m;
  return s;
}

lbm_status cuda_check(lbm_grid* g, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return LBM_OK;
  return fail(g, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

lbmk::PatchDev view(const lbm_grid* g, const HostPatch& p) {
  lbmk::PatchDev v{};
  for (int a = 0; a < 3; ++a) {
    v.dim[a] = (int)p.dim[a];
    v.org[a] = (int)p.org[a];
    v.maxc[a] = (int)g->hg.maxc(p.level, a);
    v.span[a] = p.span[a];
    v.periodic[a] = g->hg.periodic(a);
  }
  v.nxp = (int)p.nxp;
  v.plane = p.plane;
  v.walls = g->hg.desc.walls;
  v.inflow = g->hg.desc.inflow_axis;
  v.type = g->base + p.off_type;
  v.wq_idx = p.wq_idx.empty() ? nullptr : reinterpret_cast<const int32_t*>(g->base + p.off_wq_idx);
  v.wq = p.wq.empty() ? nullptr : reinterpret_cast<const double*>(g->base + p.off_wq);
  return v;
}

template <typename T>
T* at(const lbm_grid* g, size_t off) {
  return reinterpret_cast<T*>(g->base + off);
}

lbmk::Force level_force(const lbm_grid* g, int level) {
  lbmk::Force F{};
  const double s = 1.0 / (double)(1LL << level);  // du_f = du_c / r per level
  for (int a = 0; a < 3; ++a) F.du[a] = g->accel[a] * s;
  return F;
}

int* status_ptr(const lbm_grid* g) { return at<int>(g, g->off_status); }

lbmk::ThermalLevel thermal_level(const lbm_grid* g, const HostPatch& p) {
  lbmk::ThermalLevel L{};
  const lbm_desc& d = g->hg.desc;
  for (int k = 0; k < 6; ++k) L.twd[k] = d.wall_T[k] - d.t0;
  L.twd[6] = d.solid_T - d.t0;
  L.solid_iso = d.solid_isothermal ? 1 : 0;
  L.glam = d.glambda / (double)(1LL << p.level);  // du_f = du_c / r per level
  L.tref_d = d.t_ref - d.t0;
  L.beta = p.beta;
  L.beta1 = p.beta1;
  L.lbgk = d.mirror_lbgk;
  L.pr_gt1 = g->hg.pr_gt1 ? 1 : 0;
  L.wait_sleeps = g->wait_sleeps;
  return L;
}

cudaEvent_t next_event(lbm_grid* g) {
  if (g->pool_used == g->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g->pool.push_back(e);
  }
  return g->pool[g->pool_used++];
}

// Brackets one launch with events when timing is on.
template <typename F>
cudaError_t timed(lbm_grid* g, int kind, int level, double nodes, F&& launch) {
  if (!g->timing) return launch();
  lbm_grid::Rec r{kind, level, nodes, next_event(g), next_event(g)};
  if (!r.e0 || !r.e1) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(r.e0, g->stream);
  if (!e) e = launch();
  if (!e) e = cudaEventRecord(r.e1, g->stream);
  g->recs.push_back(r);
  return e;
}

double count_types(const HostPatch& p, bool with_d1) { return p.n_bulk + (with_d1 ? p.n_d1 : 0.0); }

lbm_status check_patch(lbm_grid* g, int32_t patch) {
  if (!g) return LBM_ERR_ARG;
  if (patch < 0 || patch >= (int32_t)g->hg.P.size()) return fail(g, LBM_ERR_ARG, "patch index out of range");
  return LBM_OK;
}

lbm_status check_bound(lbm_grid* g) {
  if (!g) return LBM_ERR_ARG;
  if (!g->bound) return fail(g, LBM_ERR_STATE, "grid has no bound device memory");
  return LBM_OK;
}

// Intermediate points of the separable reconstruction, stage 1 then stage 2.
cudaError_t point_passes(lbm_grid* g, const HostPatch& p, int ncomp, cudaStream_t st) {
  const int64_t ld = (int64_t)p.n_points(), ns = (int64_t)p.smp_node.size();
  const uint32_t* src = at<uint32_t>(g, p.off_pt_src);
  cudaError_t e = lbmk::launch_points(g->hg.desc.storage, ncomp, src, p.n_pt[0], g->base + p.off_smp_val, ld, ns, st);
  if (!e)
    e = lbmk::launch_points(g->hg.desc.storage, ncomp, src + 4 * (size_t)p.n_pt[0], p.n_pt[1],
                            g->base + p.off_smp_val, ld, ns + p.n_pt[0], st);
  return e;
}

// One instant k (1 .. 2^(L-1)) of the refined step.
lbm_status run_instant(lbm_grid* g, int k) {
  HostGrid& hg = g->hg;
  const int L = hg.nlev;
  const int storage = hg.desc.storage;
  const int lbgk = hg.desc.mirror_lbgk;
  std::vector<int> active;
  const bool side = !g->timing;
  if (side) {
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 3 && !e; ++q)
      if (!g->fwd_side[q]) e = side_stream(&g->fwd_side[q]);
    if (!e && !g->fwd_fork) e = cudaEventCreateWithFlags(&g->fwd_fork, cudaEventDisableTiming);
    if (!e && !g->fwd_pre) e = cudaEventCreateWithFlags(&g->fwd_pre, cudaEventDisableTiming);
    for (int q = 0; q < 3 && !e; ++q)
      if (!g->fwd_join[q]) e = cudaEventCreateWithFlags(&g->fwd_join[q], cudaEventDisableTiming);
    if (e) return cuda_check(g, e, "forward side streams");
  }
  // The reconstruction samples and their point passes read only pre-states:
  // in the isothermal model they may start on the coupling streams before the
  // TMA pass and run beside it, the explode after the pass finding them done.
  // That pays where the pass leaves the GPU idle (small grids) and costs where
  // the pass fills it, so it is a schedule variant that lbm_autotune times.
  const bool presample = side && !hg.thermal && g->presample;
  if (presample) {
    cudaError_t e = cudaEventRecord(g->fwd_pre, g->stream);
    for (int q = 1; q < 3 && !e; ++q) e = cudaStreamWaitEvent(g->fwd_side[q], g->fwd_pre, 0);
    for (int lev = 1; lev < L && !e; ++lev) {
      const int stride = 1 << (L - 1 - lev);
      if (k % stride || (k / stride) % 2) continue;  // stepped, with the parent active
      for (size_t pi = 0; pi < hg.P.size() && !e; ++pi) {
        HostPatch& p = hg.P[pi];
        if (p.level != lev) continue;
        HostPatch& q = hg.P[p.parent];
        cudaStream_t cs = g->fwd_side[1 + pi % 2];
        e = lbmk::launch_samples(storage, view(g, q), g->base + q.off_f[q.cur], view(g, p), g->base + p.off_f[p.cur],
                                 at<uint32_t>(g, p.off_smp_node), at<uint8_t>(g, p.off_smp_kind),
                                 (int64_t)p.smp_node.size(), g->base + p.off_smp_val, (int64_t)p.n_points(),
                                 q.beta / (2.0 * p.beta), status_ptr(g), cs);
        if (!e) e = point_passes(g, p, 31, cs);
      }
    }
    if (e) return cuda_check(g, e, "samples");
  }
  if (!hg.thermal) {
    // TMA tile pass of every patch stepped at this instant: one persistent
    // launch per 8 patches, whatever their levels and sizes
    // (the 64-node tile variant takes the half-tile lists and their load descriptors)
    std::vector<lbmk::TmaLaunchPatch> batch;
    const bool half = lbmk::sc_tma_tile_nodes(storage, g->variant) == 64;
    double nodes = 0;
    for (int lev = 0; lev < L; ++lev) {
      const int stride = 1 << (L - 1 - lev);
      if (k % stride) continue;
      const int odd = (lev > 0 && (k / stride) % 2) ? 1 : 0;
      for (auto& p : hg.P) {
        if (p.level != lev || p.tiles_pure[odd].empty()) continue;
        batch.push_back({half ? p.tmap64[p.cur] : p.tmap[p.cur], p.tmapo[1 - p.cur], p.tmapw[p.cur], view(g, p),
                         g->base + p.off_f[p.cur],
                         at<unsigned long long>(g, half ? p.off_tiles_half[odd] : p.off_tiles_pure[odd]),
                         (int64_t)(half ? p.tiles_half[odd].size() : p.tiles_pure[odd].size()), p.beta,
                         level_force(g, lev)});
        nodes += p.n_tma[odd];
      }
    }
    for (size_t b0 = 0; b0 < batch.size(); b0 += kTmaBatchMax) {
      const int nb = (int)std::min(batch.size() - b0, kTmaBatchMax);
      if (lbm_status st = cuda_check(g,
                                     timed(g, 4, -1, b0 == 0 ? nodes : 0.0,
                                           [&] {
                                             return lbmk::launch_sc_tma(storage, batch.data() + b0, nb,
                                                                        g->variant, lbgk, g->wait_sleeps,
                                                                        status_ptr(g), g->stream);
                                           }),
                                     "stream_collide (TMA)"))
        return st;
    }
  }
  // After the TMA pass the rest of the instant splits into independent chains:
  // the node-by-node remainder of the stream-collide (fix-up nodes, mixed
  // tiles) writes updated nodes only; each coalesce writes its parent's twin
  // nodes and each explode chain its child's interface nodes, which are never
  // updated in the same substep; all of them read the previous state.  So they
  // run on side streams beside each other, joined before the instant ends
  // (not under per-launch timing).
  // The thermal model issues each patch's stream-collide inside the loop
  // below; its coupling chains then start on the side streams once that
  // patch's stream-collide has been issued (one event per patch).
  cudaStream_t rest = g->stream, cpl[2] = {g->stream, g->stream};
  const bool forked = side && !hg.thermal;
  if (side) {
    cudaError_t e = cudaSuccess;
    if (hg.thermal && g->patch_done.size() != hg.P.size()) {
      g->patch_done.assign(hg.P.size(), nullptr);
      for (auto& x : g->patch_done)
        if (!e) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    }
    if (forked) {
      if (!e) e = cudaEventRecord(g->fwd_fork, g->stream);
      for (int q = 0; q < 3 && !e; ++q) e = cudaStreamWaitEvent(g->fwd_side[q], g->fwd_fork, 0);
      rest = g->fwd_side[0];
    }
    if (e) return cuda_check(g, e, "forward side streams");
    cpl[0] = g->fwd_side[1];
    cpl[1] = g->fwd_side[2];
  }
  for (int lev = 0; lev < L; ++lev) {
    const int stride = 1 << (L - 1 - lev);
    if (k % stride) continue;
    const int s = k / stride;
    const bool parent_active = (s % 2) == 0;
    for (size_t pi = 0; pi < hg.P.size(); ++pi) {
      HostPatch& p = hg.P[pi];
      if (p.level != lev) continue;
      active.push_back((int)pi);
      const lbmk::PatchDev pv = view(g, p);
      const lbmk::Force F = level_force(g, lev);
      void* fin = g->base + p.off_f[p.cur];
      void* fout = g->base + p.off_f[1 - p.cur];
      const int odd = (lev > 0 && !parent_active) ? 1 : 0;
      lbm_status st;
      if (hg.thermal) {
        st = cuda_check(g,
                        timed(g, 0, lev, g->timing ? count_types(p, odd) : 0.0,
                              [&] {
                                // TMA tile pass, then fix-up nodes and the node-by-node tiles
                                const void* maps[6] = {p.tmap[p.cur], p.tmapo[1 - p.cur], p.tmapw[p.cur],
                                                       p.tmapg[p.cur], p.tmapgo[1 - p.cur], p.tmapgw[p.cur]};
                                const lbmk::ThermalLevel TL = thermal_level(g, p);
                                void* gin = g->base + p.off_g[p.cur];
                                void* gout = g->base + p.off_g[1 - p.cur];
                                cudaError_t e = lbmk::launch_th_tma(storage, g->variant, maps, pv, fin, fout, gout,
                                                                   at<unsigned long long>(g, p.off_tiles_pure[odd]),
                                                                   (int64_t)p.tiles_pure[odd].size(), TL,
                                                                   status_ptr(g), g->stream);
                                if (!e)
                                  e = lbmk::launch_th_nodes(storage, pv, fin, gin, fout, gout,
                                                            at<uint32_t>(g, p.off_fix_nodes[odd]),
                                                            (int64_t)p.fix_nodes[odd].size(), TL, status_ptr(g),
                                                            g->stream);
                                if (!e)
                                  e = lbmk::launch_th_tiles(storage, pv, fin, gin, fout, gout,
                                                            at<uint32_t>(g, p.off_tiles_mixed[odd]),
                                                            (int64_t)p.tiles_mixed[odd].size(), (int)p.ntx, TL, odd,
                                                            status_ptr(g), g->stream);
                                return e;
                              }),
                        "thermal stream_collide");
      } else {
        // the nodes the TMA pass does not give: fix-up list, then mixed tiles
        st = cuda_check(
            g,
            timed(g, 0, lev, g->timing ? count_types(p, odd) - p.n_tma[odd] : 0.0,
                  [&] {
                    cudaError_t e = lbmk::launch_sc_nodes(storage, pv, fin, fout, at<uint32_t>(g, p.off_fix_nodes[odd]),
                                              (int64_t)p.fix_nodes[odd].size(), p.beta, F, lbgk, status_ptr(g),
                                              rest);
                    if (e) return e;
                    return lbmk::launch_sc_tiles(storage, pv, fin, fout, at<uint32_t>(g, p.off_tiles_mixed[odd]),
                                                 (int64_t)p.tiles_mixed[odd].size(), (int)p.ntx, p.beta, F, odd,
                                                 lbgk, status_ptr(g), rest);
                  }),
            "stream_collide");
      }
      if (st) return st;
      if (side && hg.thermal) {
        // this patch's coupling chains wait for its stream-collide only
        cudaError_t e = cudaEventRecord(g->patch_done[pi], g->stream);
        for (int q = 0; q < 2 && !e; ++q) e = cudaStreamWaitEvent(cpl[q], g->patch_done[pi], 0);
        if (e) return cuda_check(g, e, "thermal side streams");
      }
      for (int ci : p.kids) {
        HostPatch& c = hg.P[ci];
        const lbmk::PatchDev cv = view(g, c);
        if (hg.thermal) {
          st = cuda_check(g,
                          timed(g, 1, lev, (double)c.cf_parent.size(),
                                [&] {
                                  double ff = 2.0 * c.beta / p.beta, fg = 2.0 * c.beta1 / p.beta1;
                                  if (hg.pr_gt1) std::swap(ff, fg);  // Sec. III.A, Pr > 1
                                  return lbmk::launch_th_coalesce(
                                      storage, cv, g->base + c.off_f[c.cur], g->base + c.off_g[c.cur], pv, fout,
                                      g->base + p.off_g[1 - p.cur], at<uint32_t>(g, c.off_cf_parent),
                                      at<uint32_t>(g, c.off_cf_child), (int64_t)c.cf_parent.size(), ff, fg,
                                      thermal_level(g, c), thermal_level(g, p), status_ptr(g), cpl[(pi + 1) % 2]);
                                }),
                          "thermal coalesce");
          if (st) return st;
          continue;
        }
        st = cuda_check(g,
                        timed(g, 1, lev, (double)c.cf_parent.size(),
                              [&] {
                                return lbmk::launch_coalesce(storage, cv, g->base + c.off_f[c.cur], pv, fout,
                                                             at<uint32_t>(g, c.off_cf_parent),
                                                             at<uint32_t>(g, c.off_cf_child),
                                                             (int64_t)c.cf_parent.size(), 2.0 * c.beta / p.beta,
                                                             p.beta, F, lbgk, status_ptr(g), cpl[(pi + 1) % 2]);
                              }),
                        "coalesce");
        if (st) return st;
      }
      if (lev > 0 && parent_active && hg.thermal) {
        HostPatch& q = hg.P[p.parent];
        const lbmk::PatchDev qv = view(g, q);
        st = cuda_check(g,
                        timed(g, 2, lev, (double)p.n_points(),
                              [&] {
                                double ff = q.beta / (2.0 * p.beta), fg = q.beta1 / (2.0 * p.beta1);
                                if (hg.pr_gt1) std::swap(ff, fg);  // Sec. III.A, Pr > 1
                                cudaError_t e = lbmk::launch_th_samples(
                                    storage, qv, g->base + q.off_f[q.cur], g->base + q.off_g[q.cur], pv, fin,
                                    g->base + p.off_g[p.cur], at<uint32_t>(g, p.off_smp_node),
                                    at<uint8_t>(g, p.off_smp_kind), (int64_t)p.smp_node.size(),
                                    g->base + p.off_smp_val, (int64_t)p.n_points(), ff, fg, thermal_level(g, q),
                                    thermal_level(g, p), status_ptr(g), cpl[pi % 2]);
                                return e ? e : point_passes(g, p, 59, cpl[pi % 2]);
                              }),
                        "thermal samples");
        if (st) return st;
        st = cuda_check(g,
                        timed(g, 3, lev, (double)p.ex_node.size(),
                              [&] {
                                return lbmk::launch_th_explode(
                                    storage, pv, fout, g->base + p.off_g[1 - p.cur], at<uint32_t>(g, p.off_ex_node),
                                    at<uint32_t>(g, p.off_ex_src), (int64_t)p.ex_one, (int64_t)p.ex_node.size(),
                                    g->base + p.off_smp_val, (int64_t)p.n_points(), thermal_level(g, p),
                                    cpl[pi % 2]);
                              }),
                        "thermal explode");
        if (st) return st;
      } else if (lev > 0 && parent_active) {
        HostPatch& q = hg.P[p.parent];
        const lbmk::PatchDev qv = view(g, q);
        if (!presample) {  // (otherwise issued before the TMA pass)
          st = cuda_check(g,
                          timed(g, 2, lev, (double)p.n_points(),
                                [&] {
                                  cudaError_t e = lbmk::launch_samples(
                                      storage, qv, g->base + q.off_f[q.cur], pv, fin, at<uint32_t>(g, p.off_smp_node),
                                      at<uint8_t>(g, p.off_smp_kind), (int64_t)p.smp_node.size(),
                                      g->base + p.off_smp_val, (int64_t)p.n_points(), q.beta / (2.0 * p.beta),
                                      status_ptr(g), cpl[pi % 2]);
                                  return e ? e : point_passes(g, p, 31, cpl[pi % 2]);
                                }),
                          "samples");
          if (st) return st;
        }
        st = cuda_check(g,
                        timed(g, 3, lev, (double)p.ex_node.size(),
                              [&] {
                                return lbmk::launch_explode(storage, pv, fout, at<uint32_t>(g, p.off_ex_node),
                                                            at<uint32_t>(g, p.off_ex_src), (int64_t)p.ex_one,
                                                            (int64_t)p.ex_node.size(), g->base + p.off_smp_val,
                                                            (int64_t)p.n_points(), p.beta, F, lbgk, cpl[pi % 2]);
                              }),
                        "explode");
        if (st) return st;
      }
    }
  }
  if (side) {
    // join the side streams used in this instant (the remainder stream only
    // when it was forked)
    cudaError_t e = cudaSuccess;
    for (int q = forked ? 0 : 1; q < 3 && !e; ++q) {
      e = cudaEventRecord(g->fwd_join[q], g->fwd_side[q]);
      if (!e) e = cudaStreamWaitEvent(g->stream, g->fwd_join[q], 0);
    }
    if (e) return cuda_check(g, e, "forward side stream join");
  }
  for (int pi : active) hg.P[pi].cur ^= 1;
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_grid_create(const lbm_desc* desc, lbm_grid_t* out) {
  if (!desc || !out) return fail(nullptr, LBM_ERR_ARG, "null argument");
  *out = nullptr;
  if (desc->storage < LBM_FP64 || desc->storage > LBM_BF16_SHIFT) return fail(nullptr, LBM_ERR_ARG, "bad storage");
  if (desc->model != LBM_ISO_KBC && desc->model != LBM_THERMAL_KBC) return fail(nullptr, LBM_ERR_ARG, "unknown model");
  if (desc->model == LBM_THERMAL_KBC) {
    if (desc->storage != LBM_FP32 && desc->storage != LBM_FP64)
      return fail(nullptr, LBM_ERR_ARG, "thermal model: FP32 or FP64 storage");
    if (desc->t0 < 1.0 / 3.0 - 1e-12 || desc->t0 > 1.0 / 3.0 + 1e-12)
      return fail(nullptr, LBM_ERR_ARG, "thermal model implemented for T0 = 1/3");
  }
  if (desc->n_boxes < 0 || (desc->n_boxes > 0 && !desc->boxes)) return fail(nullptr, LBM_ERR_ARG, "bad boxes");
  lbm_grid* g = new lbm_grid();
  HostGrid& hg = g->hg;
  hg.desc = *desc;
  hg.boxes.assign(desc->boxes, desc->boxes + desc->n_boxes);
  hg.desc.boxes = nullptr;
  if (desc->solid) {
    for (int a = 0; a < 3; ++a)
      if (desc->solid_dims[a] <= 0) {
        delete g;
        return fail(nullptr, LBM_ERR_ARG, "solid mask with empty extent");
      }
    size_t ns = (size_t)desc->solid_dims[0] * desc->solid_dims[1] * desc->solid_dims[2];
    hg.solid.assign(desc->solid, desc->solid + ns);
  }
  hg.desc.solid = nullptr;
  hg.thermal = desc->model == LBM_THERMAL_KBC;
  hg.pop_bytes = desc->storage == LBM_FP64 ? 8 : desc->storage == LBM_FP32 ? 4 : 2;
  hg.real_bytes = desc->storage == LBM_FP64 ? 8 : 4;
  for (int a = 0; a < 3; ++a) g->accel[a] = desc->accel0[a];
  std::string e = lbm::build_layout(hg);
  if (!e.empty()) {
    delete g;
    return fail(nullptr, LBM_ERR_LAYOUT, e);
  }
  for (auto& p : hg.P)
    if (p.dim[1] > 65535 || p.dim[2] > 65535) {
      delete g;
      return fail(nullptr, LBM_ERR_LAYOUT, "patch extent in y or z above 65535 nodes");
    }
  for (auto& p : hg.P)
    for (uint8_t t : p.type) {
      p.n_bulk += (t == lbm::T_BULK || t == lbm::T_BC);
      p.n_d1 += (t == lbm::T_D1);
      p.n_bc += (t == lbm::T_BC);
    }
  size_t off = lbm::plan_memory(hg);
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) / 256 * 256;
    return o;
  };
  g->off_status = take(64);
  g->off_partial = take(sizeof(double) * 8 * kDiagBlocks * hg.P.size());
  g->off_diag_out = take(sizeof(double) * 8);
  g->need = off;
  *out = g;
  return LBM_OK;
}

lbm_status lbm_grid_bytes(lbm_grid_t g, size_t* device_bytes) {
  if (!g || !device_bytes) return LBM_ERR_ARG;
  *device_bytes = g->need;
  return LBM_OK;
}

lbm_status lbm_grid_bind(lbm_grid_t g, void* dev_ptr, size_t bytes, void* cuda_stream) {
  if (!g || !dev_ptr) return fail(g, LBM_ERR_ARG, "null argument");
  if (bytes < g->need) return fail(g, LBM_ERR_OOM, "bound buffer smaller than lbm_grid_bytes");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 256) return fail(g, LBM_ERR_ARG, "device buffer not 256-byte aligned");
  cudaPointerAttributes pa{};
  if (cudaError_t e = cudaPointerGetAttributes(&pa, dev_ptr)) return cuda_check(g, e, "cudaPointerGetAttributes");
  if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
    return fail(g, LBM_ERR_ARG, "bound buffer is not device memory");
  g->device = pa.device;
  g->drop_graphs();  // the captured launches name the previous buffer and stream
  g->stepped = false;
  g->base = static_cast<uint8_t*>(dev_ptr);
  g->bytes = bytes;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaStream_t s = g->stream;
  auto up = [&](size_t off, const void* src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(g->base + off, src, n, cudaMemcpyHostToDevice, s);
  };
  cudaError_t e = cudaSuccess;
  for (auto& p : g->hg.P) {
    if (!e) e = up(p.off_type, p.type.data(), p.type.size());
    if (!e) e = up(p.off_ex_node, p.ex_node.data(), 4 * p.ex_node.size());
    if (!e) e = up(p.off_ex_src, p.ex_src.data(), 4 * p.ex_src.size());
    if (!e) e = up(p.off_pt_src, p.pt_src.data(), 4 * p.pt_src.size());
    if (!e) e = up(p.off_use_ptr, p.use_ptr.data(), 4 * p.use_ptr.size());
    if (!e) e = up(p.off_use_ent, p.use_ent.data(), 4 * p.use_ent.size());
    if (!e) e = up(p.off_smp_node, p.smp_node.data(), 4 * p.smp_node.size());
    if (!e) e = up(p.off_smp_kind, p.smp_kind.data(), p.smp_kind.size());
    if (!e) e = up(p.off_cf_parent, p.cf_parent.data(), 4 * p.cf_parent.size());
    if (!e) e = up(p.off_cf_child, p.cf_child.data(), 4 * p.cf_child.size());
    if (!e) e = up(p.off_drag_node, p.drag_node.data(), 4 * p.drag_node.size());
    if (!e) e = up(p.off_drag_mask, p.drag_mask.data(), 4 * p.drag_mask.size());
    if (!e) e = up(p.off_wq, p.wq.data(), 8 * p.wq.size());
    if (!e) e = up(p.off_wq_idx, p.wq_idx.data(), 4 * p.wq_idx.size());
    for (int k = 0; k < 2; ++k)
      if (!e) e = up(p.off_tiles_pure[k], p.tiles_pure[k].data(), 8 * p.tiles_pure[k].size());
    for (int k = 0; k < 2; ++k)
      if (!e) e = up(p.off_tiles_half[k], p.tiles_half[k].data(), 8 * p.tiles_half[k].size());
    for (int k = 0; k < 2; ++k) {
      if (!e) e = up(p.off_tiles_mixed[k], p.tiles_mixed[k].data(), 4 * p.tiles_mixed[k].size());
      if (!e) e = up(p.off_fix_nodes[k], p.fix_nodes[k].data(), 4 * p.fix_nodes[k].size());
      if (!e) e = up(p.off_tiles_all[k], p.tiles_all[k].data(), 4 * p.tiles_all[k].size());
    }
    p.cur = 0;
  }
  for (auto& p : g->hg.P)
    for (int k = 0; k < 2 && !e; ++k) {
      e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmap[k], g->base + p.off_f[k], view(g, p), 0);
      if (!e) e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmapo[k], g->base + p.off_f[k], view(g, p), 1);
      if (!e) e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmapw[k], g->base + p.off_f[k], view(g, p), 2);
      if (!e) e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmap64[k], g->base + p.off_f[k], view(g, p), 3);
      if (g->hg.thermal) {
        if (!e) e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmapg[k], g->base + p.off_g[k], view(g, p), 0);
        if (!e) e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmapgo[k], g->base + p.off_g[k], view(g, p), 1);
        if (!e) e = lbmk::make_tensor_map(g->hg.desc.storage, p.tmapgw[k], g->base + p.off_g[k], view(g, p), 2);
      }
    }
  if (!e) e = cudaMemsetAsync(g->base + g->off_status, 0, 64, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return cuda_check(g, e, "lbm_grid_bind");
  g->bound = true;
  return LBM_OK;
}

lbm_status lbm_grid_destroy(lbm_grid_t g) {
  delete g;
  return LBM_OK;
}

lbm_status lbm_num_patches(lbm_grid_t g, int32_t* n_patches, int32_t* n_levels) {
  if (!g) return LBM_ERR_ARG;
  if (n_patches) *n_patches = (int32_t)g->hg.P.size();
  if (n_levels) *n_levels = g->hg.nlev;
  return LBM_OK;
}

lbm_status lbm_patch_info(lbm_grid_t g, int32_t patch, int32_t* level, int32_t* parent, int64_t org[3],
                          int64_t dim[3], double* beta, double* beta1) {
  if (lbm_status s = check_patch(g, patch)) return s;
  const HostPatch& p = g->hg.P[patch];
  if (level) *level = p.level;
  if (parent) *parent = p.parent;
  for (int a = 0; a < 3; ++a) {
    if (org) org[a] = p.org[a];
    if (dim) dim[a] = p.dim[a];
  }
  if (beta) *beta = p.beta;
  if (beta1) *beta1 = p.beta1;
  return LBM_OK;
}

lbm_status lbm_patch_mask(lbm_grid_t g, int32_t patch, uint8_t* host_out) {
  if (lbm_status s = check_patch(g, patch)) return s;
  if (!host_out) return fail(g, LBM_ERR_ARG, "null output");
  const HostPatch& p = g->hg.P[patch];
  size_t d = 0;
  for (int64_t z = 0; z < p.dim[2]; ++z)
    for (int64_t y = 0; y < p.dim[1]; ++y)
      for (int64_t x = 0; x < p.dim[0]; ++x) {
        uint8_t t = p.type[(size_t)((z * p.dim[1] + y) * p.nxp + x)];
        host_out[d++] = t == lbm::T_SKIP ? 0 : (t == lbm::T_SOLID ? 2 : 1);
      }
  return LBM_OK;
}

lbm_status lbm_node_updates(lbm_grid_t g, double* per_coarse_step) {
  if (!g || !per_coarse_step) return LBM_ERR_ARG;
  double s = 0;
  for (auto& p : g->hg.P) s += (double)p.n_fluid * (double)(1LL << p.level);
  *per_coarse_step = s;
  return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_grid_t g, int32_t patch, const void* rho, const void* u, const void* T,
                                int32_t dtype) {
  if (lbm_status s = check_patch(g, patch)) return s;
  if (lbm_status s = check_bound(g)) return s;
  if (!rho || !u || (dtype != 0 && dtype != 1)) return fail(g, LBM_ERR_ARG, "bad rho/u/dtype");
  HostPatch& p = g->hg.P[patch];
  if (g->hg.thermal)
    return cuda_check(g,
                      lbmk::launch_th_init(g->hg.desc.storage, view(g, p), g->base + p.off_f[0], g->base + p.off_f[1],
                                           g->base + p.off_g[0], g->base + p.off_g[1], rho, u, T, dtype,
                                           g->hg.desc.u_in, g->stream),
                      "lbm_init_equilibrium");
  (void)T;
  return cuda_check(g,
                    lbmk::launch_init(g->hg.desc.storage, view(g, p), g->base + p.off_f[0], g->base + p.off_f[1],
                                      rho, u, dtype, g->hg.desc.u_in, g->stream),
                    "lbm_init_equilibrium");
}

namespace {

lbm_status coarse_step_eager(lbm_grid* g) {
  const int K = 1 << (g->hg.nlev - 1);
  for (int k = 1; k <= K; ++k)
    if (lbm_status s = run_instant(g, k)) return s;
  return LBM_OK;
}

constexpr size_t kMaxStepGraphs = 8;

std::vector<uint8_t> cur_key(const lbm_grid* g) {
  std::vector<uint8_t> k;
  for (auto& p : g->hg.P) k.push_back((uint8_t)p.cur);
  return k;
}

// Captures one coarse step from the current buffer indices; the host-side
// indices are put back afterwards (capture launches nothing).
lbm_status capture_step(lbm_grid* g, const std::vector<uint8_t>& key, cudaGraphExec_t* out) {
  if (!g->cap_stream) {
    if (cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking))
      return cuda_check(g, e, "capture stream");
  }
  cudaStream_t keep = g->stream;
  g->stream = g->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed);
  lbm_status st = e ? LBM_OK : coarse_step_eager(g);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = e ? cudaSuccess : cudaStreamEndCapture(g->cap_stream, &graph);
  g->stream = keep;
  for (size_t i = 0; i < g->hg.P.size(); ++i) g->hg.P[i].cur = key[i];
  if (e) return cuda_check(g, e, "cudaStreamBeginCapture");
  if (st || e2) {
    if (graph) cudaGraphDestroy(graph);
    return st ? st : cuda_check(g, e2, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(out, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  return cuda_check(g, e, "cudaGraphInstantiate");
}

}  // namespace

lbm_status lbm_step(lbm_grid_t g, int64_t n_coarse_steps) {
  if (lbm_status s = check_bound(g)) return s;
  if (n_coarse_steps < 0) return fail(g, LBM_ERR_ARG, "negative step count");
  const int L = g->hg.nlev, K = 1 << (L - 1);
  for (int64_t n = 0; n < n_coarse_steps; ++n) {
    if (!g->graphs || g->timing || !g->stepped) {
      if (lbm_status s = coarse_step_eager(g)) return s;
      g->stepped = true;
      continue;
    }
    const std::vector<uint8_t> key = cur_key(g);
    cudaGraphExec_t exec = nullptr;
    for (auto& x : g->gcache)
      if (x.cur == key) exec = x.exec;
    if (!exec) {
      if (g->gcache.size() >= kMaxStepGraphs) g->drop_graphs();
      if (lbm_status s = capture_step(g, key, &exec)) return s;
      g->gcache.push_back({key, exec});
    }
    if (cudaError_t e = cudaGraphLaunch(exec, g->stream)) return cuda_check(g, e, "cudaGraphLaunch");
    // the buffer flips of the replayed step
    for (auto& p : g->hg.P)
      if ((K >> (L - 1 - p.level)) & 1) p.cur ^= 1;
  }
  return LBM_OK;
}

constexpr int kAutotuneWarm = 2;
constexpr int kAutotuneLong = 3;  // the two fastest variants are timed again over this many times the trials

lbm_status lbm_autotune(lbm_grid_t g, int32_t trials, int32_t* chosen, float* ms_per_step, int32_t max_variants,
                        int32_t* n_variants) {
  if (lbm_status s = check_bound(g)) return s;
  if (trials < 1) return fail(g, LBM_ERR_ARG, "autotune needs at least one trial step");
  // isothermal: TMA kernel variant x sample schedule; thermal: TMA kernel variant
  const int nt = g->hg.thermal ? lbmk::th_tma_variants() : lbmk::sc_tma_variants(g->hg.desc.storage);
  const int nv = g->hg.thermal ? nt : 2 * nt;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (!e) e = cudaEventCreate(&e1);
  std::vector<float> ms(nv, 0.0f);
  // one untimed step first: the first launches of a kernel pay for loading it
  g->variant = 0;
  g->presample = false;
  lbm_status st = e ? LBM_OK : coarse_step_eager(g);
  g->stepped = true;
  auto trial = [&](int v, int n) {
    g->variant = v % nt;
    g->presample = v >= nt;
    g->drop_graphs();
    // timed the way lbm_step runs: two untimed steps capture the step graphs
    // of both buffer parities of level 0 (or run directly without graphs)
    st = lbm_step(g, kAutotuneWarm);
    if (!st) e = cudaEventRecord(e0, g->stream);
    if (!e && !st) st = lbm_step(g, n);
    if (!e && !st) e = cudaEventRecord(e1, g->stream);
    if (!e && !st) e = cudaEventSynchronize(e1);
    if (!e && !st) e = cudaEventElapsedTime(&ms[v], e0, e1);
    ms[v] /= (float)n;
  };
  for (int v = 0; v < nv && !e && !st; ++v) trial(v, trials);
  // the two fastest again, over three times the steps: short trials of
  // schedules that differ by a few percent do not separate them reliably
  int best = 0, second = nv > 1 ? 1 : 0;
  if (ms[second] < ms[best]) std::swap(best, second);
  for (int v = 2; v < nv; ++v) {
    if (ms[v] < ms[best]) second = best, best = v;
    else if (ms[v] < ms[second]) second = v;
  }
  if (nv > 1)
    for (int v : {best, second})
      if (!e && !st) trial(v, kAutotuneLong * trials);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) return st;
  if (e) return cuda_check(g, e, "lbm_autotune");
  if (nv > 1 && ms[second] < ms[best]) best = second;
  g->variant = best % nt;
  g->presample = best >= nt;
  g->stepped = true;
  g->drop_graphs();
  if (chosen) *chosen = best;
  if (n_variants) *n_variants = nv;
  if (ms_per_step)
    for (int v = 0; v < nv && v < max_variants; ++v) ms_per_step[v] = ms[v];
  return LBM_OK;
}

lbm_status lbm_set_variant(lbm_grid_t g, int32_t variant) {
  if (!g) return LBM_ERR_ARG;
  const int nt = g->hg.thermal ? lbmk::th_tma_variants() : lbmk::sc_tma_variants(g->hg.desc.storage);
  const int nv = g->hg.thermal ? nt : 2 * nt;
  if (variant < 0 || variant >= nv) return fail(g, LBM_ERR_ARG, "variant out of range");
  g->variant = variant % nt;
  g->presample = variant >= nt;
  g->drop_graphs();
  return LBM_OK;
}

lbm_status lbm_wait_limit(lbm_grid_t g, int32_t sleeps) {
  if (!g) return LBM_ERR_ARG;
  if (sleeps < 0) return fail(g, LBM_ERR_ARG, "negative wait limit");
  g->wait_sleeps = sleeps;
  g->drop_graphs();  // the bound is baked into the captured launches
  return LBM_OK;
}

lbm_status lbm_graphs(lbm_grid_t g, int32_t enable) {
  if (!g) return LBM_ERR_ARG;
  g->graphs = enable != 0;
  if (!g->graphs) g->drop_graphs();
  return LBM_OK;
}

lbm_status lbm_moments(lbm_grid_t g, int32_t patch, void* rho, void* u, void* T, void* gamma, int32_t dtype) {
  if (lbm_status s = check_patch(g, patch)) return s;
  if (lbm_status s = check_bound(g)) return s;
  if (dtype != 0 && dtype != 1) return fail(g, LBM_ERR_ARG, "bad dtype");
  HostPatch& p = g->hg.P[patch];
  if (g->hg.thermal)
    return cuda_check(g,
                      lbmk::launch_th_moments(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur],
                                              g->base + p.off_g[p.cur], rho, u, T, gamma, dtype, thermal_level(g, p),
                                              g->stream),
                      "lbm_moments");
  (void)T;
  return cuda_check(g,
                    lbmk::launch_moments(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur], rho, u, gamma,
                                         dtype, p.beta, level_force(g, p.level), g->hg.desc.mirror_lbgk, g->stream),
                    "lbm_moments");
}

lbm_status lbm_transfer(lbm_grid_t dst, lbm_grid_t src, int64_t* missing) {
  if (!dst || !src || dst == src) return dst ? fail(dst, LBM_ERR_ARG, "transfer needs two grids") : LBM_ERR_ARG;
  if (lbm_status s = check_bound(dst)) return s;
  if (lbm_status s = check_bound(src)) return fail(dst, s, "source grid not bound");
  const lbm_desc &a = dst->hg.desc, &b = src->hg.desc;
  if (dst->hg.thermal || src->hg.thermal) return fail(dst, LBM_ERR_ARG, "transfer is for the isothermal model");
  if (a.storage != b.storage) return fail(dst, LBM_ERR_ARG, "transfer between different storages");
  for (int k = 0; k < 3; ++k)
    if (a.n[k] != b.n[k] || dst->hg.periodic(k) != src->hg.periodic(k))
      return fail(dst, LBM_ERR_ARG, "transfer between different domains");
  if ((int)src->hg.P.size() > lbmk::kTransferMax) return fail(dst, LBM_ERR_ARG, "too many source patches");
  // the source state must be complete before the destination reads it
  if (cudaError_t e = cudaStreamSynchronize(src->stream)) return cuda_check(dst, e, "lbm_transfer");
  lbmk::TransferSrc T{};
  T.n_src = (int)src->hg.P.size();
  for (int k = 0; k < 3; ++k) T.n[k] = a.n[k], T.periodic[k] = dst->hg.periodic(k) ? 1 : 0;
  for (int q = 0; q < T.n_src; ++q) {
    const HostPatch& sp = src->hg.P[q];
    T.p[q] = view(src, sp);
    T.f[q] = src->base + sp.off_f[sp.cur];
    T.level[q] = sp.level;
    T.beta[q] = sp.beta;
  }
  auto* count = at<unsigned long long>(dst, dst->off_partial);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), dst->stream);
  for (auto& p : dst->hg.P) {
    // own level first, then finer levels nearest first, then coarser nearest first
    std::vector<int> order(T.n_src);
    for (int q = 0; q < T.n_src; ++q) order[q] = q;
    auto rank = [&](int q) {
      const int dl = T.level[q] - p.level;
      return dl >= 0 ? dl : 1000 - dl;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rank(x) < rank(y); });
    for (int q = 0; q < T.n_src; ++q) T.order[q] = order[q];
    if (!e)
      e = lbmk::launch_transfer(a.storage, view(dst, p), dst->base + p.off_f[0], dst->base + p.off_f[1], p.level,
                                p.beta, a.u_in, T, count, dst->stream);
  }
  unsigned long long host = 0;
  if (!e) e = cudaMemcpyAsync(&host, count, sizeof host, cudaMemcpyDeviceToHost, dst->stream);
  if (!e) e = cudaStreamSynchronize(dst->stream);
  if (e) return cuda_check(dst, e, "lbm_transfer");
  if (missing) *missing = (int64_t)host;
  return LBM_OK;
}

lbm_status lbm_gamma_blocks(lbm_grid_t g, int32_t patch, int32_t block, float* out) {
  if (lbm_status s = check_patch(g, patch)) return s;
  if (lbm_status s = check_bound(g)) return s;
  if (block < 1 || !out) return fail(g, LBM_ERR_ARG, "block must be >= 1 and out non-null");
  HostPatch& p = g->hg.P[patch];
  return cuda_check(g,
                    lbmk::launch_gamma_blocks(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur], p.beta,
                                              g->hg.desc.mirror_lbgk, block, out, status_ptr(g), g->stream),
                    "lbm_gamma_blocks");
}

static lbm_status copy_pop(lbm_grid_t g, int32_t patch, int32_t which, void* dense, int32_t dtype, int to_dense) {
  if (lbm_status s = check_patch(g, patch)) return s;
  if (lbm_status s = check_bound(g)) return s;
  if (!dense || (dtype != 0 && dtype != 1)) return fail(g, LBM_ERR_ARG, "bad buffer/dtype");
  if (which != 0 && !(which == 1 && g->hg.thermal)) return fail(g, LBM_ERR_ARG, "bad population set");
  HostPatch& p = g->hg.P[patch];
  const size_t* off = which ? p.off_g : p.off_f;
  const lbmk::PatchDev pv = view(g, p);
  cudaError_t e = lbmk::launch_copy_pop(g->hg.desc.storage, pv, g->base + off[p.cur], dense, dtype, to_dense,
                                        which, g->stream);
  if (!e && !to_dense)
    e = lbmk::launch_copy_pop(g->hg.desc.storage, pv, g->base + off[1 - p.cur], dense, dtype, 0, which, g->stream);
  return cuda_check(g, e, "population copy");
}

lbm_status lbm_get_populations(lbm_grid_t g, int32_t patch, int32_t which, void* dst, int32_t dtype) {
  return copy_pop(g, patch, which, dst, dtype, 1);
}

lbm_status lbm_set_populations(lbm_grid_t g, int32_t patch, int32_t which, const void* src, int32_t dtype) {
  return copy_pop(g, patch, which, const_cast<void*>(src), dtype, 0);
}

namespace {
// Common ending of both diagnostics calls: out from the FP64 sums, the
// status word in out[7].  Bit 1 of the status word (a bounded wait of a TMA
// pass expired, so nodes of that pass kept stale values) gives
// LBM_ERR_TIMEOUT and is cleared once reported; k_diag's slot 7 (nodes with
// non-finite or non-positive density) gives LBM_ERR_UNSTABLE.
lbm_status diag_result(lbm_grid* g, const double host[8], int status, double out[8]) {
  for (int k = 0; k < 6; ++k) out[k] = host[k];
  out[6] = host[6];
  out[7] = (double)status;
  if (status & 2) {
    if (cudaError_t e = lbmk::launch_status_clear(status_ptr(g), 2, g->stream))
      return cuda_check(g, e, "status clear");
    return fail(g, LBM_ERR_TIMEOUT, "a bounded wait of the TMA pass expired; the state is not valid");
  }
  if (host[7] > 0 || !(host[6] > 0)) {
    out[6] = host[7] > 0 ? NAN : host[6];
    return fail(g, LBM_ERR_UNSTABLE, "non-finite or non-positive density");
  }
  return LBM_OK;
}
}  // namespace

lbm_status lbm_diagnostics(lbm_grid_t g, double out[8]) {
  if (lbm_status s = check_bound(g)) return s;
  if (!out) return fail(g, LBM_ERR_ARG, "null output");
  double* partial = at<double>(g, g->off_partial);
  int nb = 0;
  cudaError_t e = cudaSuccess;
  for (auto& p : g->hg.P) {
    if (!e)
      e = lbmk::launch_diag(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur],
                            1.0 / (double)(1LL << (3 * p.level)), level_force(g, p.level), partial + 8 * nb,
                            kDiagBlocks, g->stream);
    nb += kDiagBlocks;
  }
  double* dout = at<double>(g, g->off_diag_out);
  if (!e) e = lbmk::launch_diag_final(partial, nb, dout, g->stream);
  double host[8];
  int status = 0;
  if (!e) e = cudaMemcpyAsync(host, dout, sizeof host, cudaMemcpyDeviceToHost, g->stream);
  if (!e) e = cudaMemcpyAsync(&status, status_ptr(g), sizeof status, cudaMemcpyDeviceToHost, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_check(g, e, "lbm_diagnostics");
  return diag_result(g, host, status, out);
}

// ---------------------------------------------------------------------------
// Discrete adjoint (isothermal, periodic layouts).
namespace {

lbm_status adjoint_supported(lbm_grid* g) {
  const lbm_desc& d = g->hg.desc;
  if (g->hg.thermal || d.walls || d.inflow_axis >= 0 || !g->hg.solid.empty() || g->accel[0] != 0 ||
      g->accel[1] != 0 || g->accel[2] != 0)
    return fail(g, LBM_ERR_STATE,
                "the adjoint covers isothermal layouts without walls, solids, inflow or body force");
  if (d.storage != LBM_FP32 && d.storage != LBM_FP64) return fail(g, LBM_ERR_STATE, "adjoint: FP32 or FP64 storage");
  return LBM_OK;
}

// Workspace of lbm_adjoint_step: the second lambda buffer, the sample
// adjoints, and per coarse step of the segment one record of the recompute:
// the state of every patch at the step's start (outer snapshot), then, after
// each inner instant k = 1 .. 2^(L-1) - 1, the state of the levels >= 1 (inner
// snapshot k), so that the adjoint of every instant finds its pre-states
// without replaying the forward.
struct AdjLayout {
  std::vector<size_t> lam_off;   // per patch, in the packed lambda (and in the second buffer)
  std::vector<size_t> sbar_off;  // per patch (children), in the workspace
  std::vector<size_t> tbar_off;  // per patch (children): the explode targets' adjoints [31][targets]
  std::vector<size_t> snap_patch_off;   // per patch, within an outer snapshot
  std::vector<size_t> inner_patch_off;  // per patch of level >= 1, within an inner snapshot
  // per patch and instant k: offset of the reconstruction values recorded when
  // the patch exploded at k (its parent stepped too), (size_t)-1 otherwise
  std::vector<std::vector<size_t>> smp_rec_off;
  size_t lam_bytes = 0, second_off = 0, snap_off = 0, snap_bytes = 0, inner_bytes = 0, step_bytes = 0;
  size_t slot_off = 0, partial_off = 0, total = 0;
  int inner = 0;  // inner instants per coarse step
};

AdjLayout adjoint_layout(const lbm_grid* g, int K) {
  AdjLayout a;
  const size_t rb = g->hg.real_bytes;
  size_t off = 0;
  for (auto& p : g->hg.P) {
    a.lam_off.push_back(off);
    off += 27 * (size_t)p.plane * rb;
  }
  a.lam_bytes = off;
  size_t w = 0;
  auto take = [&](size_t b) {
    size_t o = w;
    w += (b + 255) / 256 * 256;
    return o;
  };
  a.second_off = take(a.lam_bytes);
  for (auto& p : g->hg.P) a.sbar_off.push_back(take(31 * p.n_points() * rb));
  for (auto& p : g->hg.P) a.tbar_off.push_back(take(31 * p.ex_node.size() * rb));
  a.snap_bytes = 0;
  for (auto& p : g->hg.P) {
    a.snap_patch_off.push_back(a.snap_bytes);
    a.inner_patch_off.push_back(a.inner_bytes);
    const size_t n = 27 * (size_t)p.plane * g->hg.pop_bytes;
    a.snap_bytes += n;
    if (p.level > 0) a.inner_bytes += n;
  }
  a.inner = (1 << (g->hg.nlev - 1)) - 1;
  size_t rec = a.snap_bytes + (size_t)a.inner * a.inner_bytes;
  const int L = g->hg.nlev, KI = 1 << (L - 1);
  for (auto& p : g->hg.P) {
    std::vector<size_t> offs(KI + 1, (size_t)-1);
    if (p.level > 0)
      for (int k = 1; k <= KI; ++k) {
        const int stride = 1 << (L - 1 - p.level);
        if (k % stride || (k / stride) % 2) continue;  // stepped, with the parent active
        rec = (rec + 255) / 256 * 256;
        offs[k] = rec;
        rec += 31 * p.n_points() * g->hg.real_bytes;
      }
    a.smp_rec_off.push_back(offs);
  }
  a.step_bytes = (rec + 255) / 256 * 256;
  // a spare record, where the first step's copy 0 puts the values of a
  // previous step that does not exist, then the K records
  a.snap_off = take(a.step_bytes * (size_t)(K + 1)) + a.step_bytes;
  a.slot_off = take(2 * sizeof(unsigned long long));  // the record's base word, then the copy-completion count
  a.partial_off = take(sizeof(double) * (kDiagBlocks * g->hg.P.size() + 1));
  a.total = w;
  return a;
}

// Pre-state of patch pi before instant k (1 .. 2^(L-1)) of the coarse step
// recorded at `step`: level 0 and every level at k = 1 from the outer
// snapshot, the others from inner snapshot k - 1 (the state after instant
// k - 1, which is the patch's state before its step at k).
uint8_t* pre_state(const lbm_grid* g, const AdjLayout& a, uint8_t* step, int pi, int k) {
  const HostPatch& p = g->hg.P[pi];
  if (p.level == 0 || k == 1) return step + a.snap_patch_off[pi];
  return step + a.snap_bytes + (size_t)(k - 2) * a.inner_bytes + a.inner_patch_off[pi];
}

// One coarse step of the recompute, recording its snapshots through the
// device word at `slot`, so that one captured graph serves every step of the
// segment.  The copies run on their own stream beside the instants (on the
// bound stream under per-launch timing).  Copy 0, beside instant 1, takes the
// previous step's last reconstruction values (instant 2^(L-1)) into the
// previous record, then this step's outer snapshot (every patch at the step's
// start) into the next one, and advances the word to it.  Copy k, after
// instant k < 2^(L-1), takes the reconstruction values of instant k and inner
// snapshot k (the levels >= 1 after instant k), beside instant k + 1.
// Ordering: instant 1 writes neither a step-start state nor a reconstruction
// value (no patch explodes at an odd instant), and instant k + 1 writes
// neither the states after instant k nor the values copy k reads (a patch's
// state buffer is rewritten at its second step after k, its values at its
// next explode, both at k + 2 or later); so instant m waits for copy m - 2
// only, and the step ends after its last copy.  Level 0 steps once per
// coarse step, so its step-start state stays unwritten through the step: with
// refined levels, its part of copy 0 runs on a second stream once copy 0 has
// advanced the word, beside the instants, and only the step's end waits for it.
lbm_status recording_step(lbm_grid* g, const AdjLayout& a, unsigned long long* slot) {
  const int L = g->hg.nlev, KI = 1 << (L - 1);
  const bool side = !g->timing;
  cudaError_t e = cudaSuccess;
  const bool split = L > 1;  // level 0's outer snapshot apart from copy 0
  if (side) {
    if (!g->rec_side) e = cudaStreamCreateWithFlags(&g->rec_side, cudaStreamNonBlocking);
    if (!e && !g->rec_side0) e = cudaStreamCreateWithFlags(&g->rec_side0, cudaStreamNonBlocking);
    if (!e && !g->rec_l0) e = cudaEventCreateWithFlags(&g->rec_l0, cudaEventDisableTiming);
    for (auto* v : {&g->rec_ev, &g->rec_cp})
      while (!e && v->size() < (size_t)KI + 1) {
        cudaEvent_t x = nullptr;
        e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (!e) v->push_back(x);
      }
    if (e) return cuda_check(g, e, "adjoint record stream");
  }
  cudaStream_t cs = side ? g->rec_side : g->stream;
  lbmk::CopySegs segs{};
  segs.rel = slot;
  unsigned* done = reinterpret_cast<unsigned*>(slot + 1);  // completion count beside the word
  auto add = [&](size_t off, const void* src, size_t n) {
    if (segs.n == lbmk::kCopySegs) {
      if (!e) e = lbmk::launch_copy(segs, cs);
      segs.n = 0;
    }
    segs.dst[segs.n] = reinterpret_cast<void*>(off);
    segs.src[segs.n] = src;
    segs.bytes[segs.n] = n;
    ++segs.n;
  };
  // copy k, issued once instant k (k = 0: the previous step) has been issued
  auto copy = [&](int k, bool advance) {
    if (side && !e) e = cudaEventRecord(g->rec_ev[k], g->stream);
    if (side && !e) e = cudaStreamWaitEvent(cs, g->rec_ev[k], 0);
    const int kv = k ? k : KI;  // the instant whose reconstruction values copy k takes
    for (size_t pi = 0; pi < g->hg.P.size(); ++pi)
      if (a.smp_rec_off[pi][kv] != (size_t)-1)
        add(a.smp_rec_off[pi][kv], g->base + g->hg.P[pi].off_smp_val,
            31 * g->hg.P[pi].n_points() * g->hg.real_bytes);
    for (size_t pi = 0; pi < g->hg.P.size(); ++pi) {
      const HostPatch& p = g->hg.P[pi];
      if (k == 0 && !(split && p.level == 0))
        add(a.step_bytes + a.snap_patch_off[pi], g->base + p.off_f[p.cur], 27 * (size_t)p.plane * g->hg.pop_bytes);
      else if (p.level > 0)
        add(a.snap_bytes + (size_t)(k - 1) * a.inner_bytes + a.inner_patch_off[pi], g->base + p.off_f[p.cur],
            27 * (size_t)p.plane * g->hg.pop_bytes);
    }
    // the advancing copy's last block moves the word on when it is done
    segs.done = advance ? done : nullptr;
    segs.advance = advance ? a.step_bytes : 0;
    if (!e) e = lbmk::launch_copy(segs, cs);
    segs.n = 0;
    segs.done = nullptr;
    if (side && !e) e = cudaEventRecord(g->rec_cp[k], cs);
  };
  copy(0, true);
  if (split) {
    // level 0's outer snapshot, into the record the word now holds
    cudaStream_t c0 = side ? g->rec_side0 : g->stream;
    lbmk::CopySegs s0{};
    s0.rel = slot;
    if (side && !e) e = cudaStreamWaitEvent(c0, g->rec_cp[0], 0);
    for (size_t pi = 0; pi < g->hg.P.size() && !e; ++pi) {
      const HostPatch& p = g->hg.P[pi];
      if (p.level != 0) continue;
      if (s0.n == lbmk::kCopySegs) {
        e = lbmk::launch_copy(s0, c0);
        s0.n = 0;
      }
      s0.dst[s0.n] = reinterpret_cast<void*>(a.snap_patch_off[pi]);
      s0.src[s0.n] = g->base + p.off_f[p.cur];
      s0.bytes[s0.n] = 27 * (size_t)p.plane * g->hg.pop_bytes;
      ++s0.n;
    }
    if (!e) e = lbmk::launch_copy(s0, c0);
    if (side && !e) e = cudaEventRecord(g->rec_l0, c0);
  }
  for (int k = 1; k <= KI && !e; ++k) {
    if (side && k >= 2) e = cudaStreamWaitEvent(g->stream, g->rec_cp[k - 2], 0);
    if (e) break;
    if (lbm_status st = run_instant(g, k)) return st;
    if (k < KI) copy(k, false);
  }
  if (side && !e) e = cudaStreamWaitEvent(g->stream, g->rec_cp[KI - 1], 0);
  if (side && split && !e) e = cudaStreamWaitEvent(g->stream, g->rec_l0, 0);
  return cuda_check(g, e, "adjoint snapshot");
}

// The reconstruction values of the segment's last step at its last instant,
// which no next step's copy 0 takes.
cudaError_t last_values(lbm_grid* g, const AdjLayout& a, unsigned long long* slot) {
  const int KI = 1 << (g->hg.nlev - 1);
  lbmk::CopySegs segs{};
  segs.rel = slot;
  cudaError_t e = cudaSuccess;
  for (size_t pi = 0; pi < g->hg.P.size() && !e; ++pi) {
    if (a.smp_rec_off[pi][KI] == (size_t)-1) continue;
    if (segs.n == lbmk::kCopySegs) {
      e = lbmk::launch_copy(segs, g->stream);
      segs.n = 0;
    }
    segs.dst[segs.n] = reinterpret_cast<void*>(a.smp_rec_off[pi][KI]);
    segs.src[segs.n] = g->base + g->hg.P[pi].off_smp_val;
    segs.bytes[segs.n] = 31 * g->hg.P[pi].n_points() * g->hg.real_bytes;
    ++segs.n;
  }
  if (!e) e = lbmk::launch_copy(segs, g->stream);
  return e;
}

// Copies the state of every patch to/from a packed buffer (restore: the current
// buffer only unless both are asked for).
cudaError_t copy_state(lbm_grid* g, uint8_t* dst_or_src, bool save, bool both = true, int min_level = 0) {
  cudaError_t e = cudaSuccess;
  uint8_t* d = dst_or_src;
  lbmk::CopySegs segs{};
  auto add = [&](void* dst, const void* src, size_t n) {
    if (segs.n == lbmk::kCopySegs) {
      if (!e) e = lbmk::launch_copy(segs, g->stream);
      segs.n = 0;
    }
    segs.dst[segs.n] = dst, segs.src[segs.n] = src, segs.bytes[segs.n] = n;
    ++segs.n;
  };
  for (auto& p : g->hg.P) {
    const size_t n = 27 * (size_t)p.plane * g->hg.pop_bytes;
    if (p.level < min_level) {
      d += n;
      continue;
    }
    if (save) {
      add(d, g->base + p.off_f[p.cur], n);
    } else {
      add(g->base + p.off_f[p.cur], d, n);
      if (both) add(g->base + p.off_f[1 - p.cur], d, n);
    }
    d += n;
  }
  if (!e) e = lbmk::launch_copy(segs, g->stream);
  return e;
}

// Patches active at instant k of a coarse step.
void flip_instant(lbm_grid* g, int k) {
  const int L = g->hg.nlev;
  for (auto& p : g->hg.P)
    if (k % (1 << (L - 1 - p.level)) == 0) p.cur ^= 1;
}

// Adjoint of instant k: lambda of the states after k -> lambda of the states before k.
lbm_status adjoint_instant(lbm_grid* g, int k, uint8_t* lam[2], std::vector<int>& lcur, const AdjLayout& a,
                           uint8_t* ws, uint8_t* step) {
  HostGrid& hg = g->hg;
  // pre-states of the instant, from the record of its coarse step
  auto state = [&](int pi) -> uint8_t* { return pre_state(g, a, step, pi, k); };
  const int L = hg.nlev, storage = hg.desc.storage, lbgk = hg.desc.mirror_lbgk;
  const size_t rb = hg.real_bytes;
  auto lam_ptr = [&](int pi, int which) { return lam[which] + a.lam_off[pi]; };
  std::vector<int> active;
  for (int lev = 0; lev < L; ++lev) {
    if (k % (1 << (L - 1 - lev))) continue;
    for (size_t pi = 0; pi < hg.P.size(); ++pi)
      if (hg.P[pi].level == lev) active.push_back((int)pi);
  }
  cudaError_t e = cudaSuccess;
  // lambda_old of patches with boundary-class nodes is accumulated and needs
  // clearing; the others are written entry by entry by their stream-collide
  // adjoint (k_adj_sc_st)
  for (int pi : active)
    if (!e && hg.P[pi].n_bc > 0)
      e = cudaMemsetAsync(lam_ptr(pi, 1 - lcur[pi]), 0, 27 * (size_t)hg.P[pi].plane * rb, g->stream);
  if (e) return cuda_check(g, e, "adjoint zero");
  for (int q = 0; q < 2 && !e; ++q)
    if (!g->adj_side[q]) e = side_stream(&g->adj_side[q]);
  if (!e && !g->adj_fork) e = cudaEventCreateWithFlags(&g->adj_fork, cudaEventDisableTiming);
  if (!e && !g->adj_sc) e = cudaEventCreateWithFlags(&g->adj_sc, cudaEventDisableTiming);
  if (!e && !g->adj_cf) e = cudaEventCreateWithFlags(&g->adj_cf, cudaEventDisableTiming);
  for (int q = 0; q < 2 && !e; ++q)
    if (!g->adj_join[q]) e = cudaEventCreateWithFlags(&g->adj_join[q], cudaEventDisableTiming);
  // side stream 0 carries the levels >= 1 from instant to instant and is not
  // joined into the bound stream at the end of an instant (the walk joins it
  // at its end), so that level 0's adjoint of the next coarse step runs beside
  // the level-1 work of an instant that steps level 1 alone; side stream 1
  // (the explode chain reads the children's lambda) waits for it
  if (!e && !g->adj_s0) e = cudaEventCreateWithFlags(&g->adj_s0, cudaEventDisableTiming);
  if (!e) e = cudaEventRecord(g->adj_fork, g->stream);
  for (int q = 0; q < 2 && !e; ++q) e = cudaStreamWaitEvent(g->adj_side[q], g->adj_fork, 0);
  if (!e) e = cudaEventRecord(g->adj_s0, g->adj_side[0]);
  if (!e) e = cudaStreamWaitEvent(g->adj_side[1], g->adj_s0, 0);
  if (e) return cuda_check(g, e, "adjoint streams");
  cudaStream_t sc = g->adj_side[0], sx = g->adj_side[1];
  // (1) the stream-collide adjoints, which write (or start) every lambda_old:
  // level 0 on the bound stream; the levels >= 1 on side stream 0, followed
  // there by (2) the coalesce adjoints, which add into the children's
  // lambda_old, so that level 0's runs beside both
  for (int pi : active) {
    HostPatch& p = hg.P[pi];
    const int lev = p.level;
    const int s = k / (1 << (L - 1 - lev));
    const int odd = (lev > 0 && (s % 2)) ? 1 : 0;
    if (!e)
      e = lbmk::launch_adj_sc(storage, view(g, p), state(pi), lam_ptr(pi, lcur[pi]), lam_ptr(pi, 1 - lcur[pi]),
                              p.beta, odd, lbgk, p.n_bc > 0, status_ptr(g), lev == 0 ? g->stream : sc);
  }
  if (!e) e = cudaEventRecord(g->adj_sc, g->stream);
  for (int pi : active) {
    HostPatch& p = hg.P[pi];
    const lbmk::PatchDev pv = view(g, p);
    for (int ci : p.kids) {
      HostPatch& c = hg.P[ci];
      if (!e)
        e = lbmk::launch_adj_coalesce(storage, view(g, c), state(ci), pv, lam_ptr(pi, lcur[pi]),
                                      lam_ptr(ci, 1 - lcur[ci]), at<uint32_t>(g, c.off_cf_parent),
                                      at<uint32_t>(g, c.off_cf_child), (int64_t)c.cf_parent.size(),
                                      2.0 * c.beta / p.beta, p.beta, lbgk, status_ptr(g), sc);
    }
  }
  if (!e) e = cudaEventRecord(g->adj_cf, sc);
  // (3) per child stepped with its parent: the explode chain -- the explode
  // adjoint on the reconstruction values the recompute recorded, the point
  // passes transposed (last first) -- beside (1) and (2), then the sample
  // adjoint, which adds into both levels' lambda_old after (1) and (2): each
  // entry takes its additions in a fixed order
  bool waited = false;
  for (int pi : active) {
    HostPatch& p = hg.P[pi];
    const int lev = p.level;
    const int s = k / (1 << (L - 1 - lev));
    if (!(lev > 0 && (s % 2) == 0)) continue;
    const lbmk::PatchDev pv = view(g, p);
    HostPatch& q = hg.P[p.parent];
    const int qi = p.parent;
    const lbmk::PatchDev qv = view(g, q);
    uint8_t* sbar = ws + a.sbar_off[pi];
    const int64_t ns = (int64_t)p.smp_node.size(), ld = (int64_t)p.n_points();
    // the reconstruction values of this explode, recorded by the recompute
    const uint8_t* val = step + a.smp_rec_off[pi][k];
    uint8_t* tbar = ws + a.tbar_off[pi];
    const int64_t nt = (int64_t)p.ex_node.size(), n1 = p.n_pt[0], n2 = p.n_pt[1];
    const uint32_t* uptr = at<uint32_t>(g, p.off_use_ptr);
    const uint32_t* uent = at<uint32_t>(g, p.off_use_ent);
    if (!e)
      e = lbmk::launch_adj_explode(storage, pv, lam_ptr(pi, lcur[pi]), at<uint32_t>(g, p.off_ex_node),
                                   at<uint32_t>(g, p.off_ex_src), (int64_t)p.ex_one, nt, val, tbar, ld, p.beta, lbgk,
                                   sx);
    // the point columns, last stage first, each from its consumers
    if (!e) e = lbmk::launch_adj_gather(storage, uptr, uent, ns + n1, ns + n1 + n2, sbar, ld, tbar, nt, sx);
    if (!e) e = lbmk::launch_adj_gather(storage, uptr, uent, ns, ns + n1, sbar, ld, tbar, nt, sx);
    if (!e) e = lbmk::launch_adj_gather(storage, uptr, uent, 0, ns, sbar, ld, tbar, nt, sx);
    if (!e && !waited) {
      e = cudaStreamWaitEvent(sx, g->adj_sc, 0);
      if (!e) e = cudaStreamWaitEvent(sx, g->adj_cf, 0);
      waited = true;
    }
    if (!e)
      e = lbmk::launch_adj_samples(storage, qv, state(qi), lam_ptr(qi, 1 - lcur[qi]), pv, state(pi),
                                   lam_ptr(pi, 1 - lcur[pi]), at<uint32_t>(g, p.off_smp_node),
                                   at<uint8_t>(g, p.off_smp_kind), ns, sbar, ld, q.beta / (2.0 * p.beta),
                                   status_ptr(g), sx);
  }
  // join side stream 1 back into the bound stream (side stream 0 at the end of the walk)
  {
    cudaError_t e2 = cudaEventRecord(g->adj_join[1], g->adj_side[1]);
    if (!e2) e2 = cudaStreamWaitEvent(g->stream, g->adj_join[1], 0);
    if (!e) e = e2;
  }
  if (e) return cuda_check(g, e, "adjoint instant");
  for (int pi : active) lcur[pi] ^= 1;
  return LBM_OK;
}

// Reverse walk of a segment of K coarse steps from their records: every
// instant's adjoint, last coarse step and top instant first; the pre-states
// come from the records, so nothing is replayed and the grid's state buffers
// are not touched.  Side stream 0 is joined into the bound stream at the end.
lbm_status adjoint_walk(lbm_grid* g, int K, uint8_t* lam[2], std::vector<int>& lcur, const AdjLayout& a, uint8_t* ws) {
  const int KI = 1 << (g->hg.nlev - 1);
  for (int s = K - 1; s >= 0; --s) {
    uint8_t* step = ws + a.snap_off + (size_t)s * a.step_bytes;
    for (int k = KI; k >= 1; --k)
      if (lbm_status st = adjoint_instant(g, k, lam, lcur, a, ws, step)) return st;
  }
  cudaError_t e = cudaEventRecord(g->adj_join[0], g->adj_side[0]);
  if (!e) e = cudaStreamWaitEvent(g->stream, g->adj_join[0], 0);
  return cuda_check(g, e, "adjoint walk join");
}

constexpr size_t kMaxAdjGraphs = 64;

// Captures n recording steps of the recompute as one graph; the host-side
// buffer indices are put back afterwards (capture launches nothing).
lbm_status capture_recording(lbm_grid* g, const AdjLayout& a, unsigned long long* slot, const std::vector<uint8_t>& key,
                             int n, cudaGraphExec_t* out) {
  if (!g->cap_stream) {
    if (cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking))
      return cuda_check(g, e, "capture stream");
  }
  cudaStream_t keep = g->stream;
  g->stream = g->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed);
  lbm_status st = LBM_OK;
  for (int j = 0; j < n && !e && !st; ++j) st = recording_step(g, a, slot);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = e ? cudaSuccess : cudaStreamEndCapture(g->cap_stream, &graph);
  g->stream = keep;
  for (size_t i = 0; i < g->hg.P.size(); ++i) g->hg.P[i].cur = key[i];
  if (e) return cuda_check(g, e, "cudaStreamBeginCapture");
  if (st || e2) {
    if (graph) cudaGraphDestroy(graph);
    return st ? st : cuda_check(g, e2, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(out, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  return cuda_check(g, e, "cudaGraphInstantiate");
}

// Captures the reverse walk; the host-side lambda indices advance as in the
// direct walk (the caller launches the graph).
lbm_status capture_walk(lbm_grid* g, int K, uint8_t* lam[2], std::vector<int>& lcur, const AdjLayout& a, uint8_t* ws,
                        cudaGraphExec_t* out) {
  if (!g->cap_stream) {
    if (cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking))
      return cuda_check(g, e, "capture stream");
  }
  cudaStream_t keep = g->stream;
  g->stream = g->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed);
  lbm_status st = e ? LBM_OK : adjoint_walk(g, K, lam, lcur, a, ws);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = e ? cudaSuccess : cudaStreamEndCapture(g->cap_stream, &graph);
  g->stream = keep;
  if (e) return cuda_check(g, e, "cudaStreamBeginCapture");
  if (st || e2) {
    if (graph) cudaGraphDestroy(graph);
    return st ? st : cuda_check(g, e2, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(out, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  return cuda_check(g, e, "cudaGraphInstantiate");
}

}  // namespace

lbm_status lbm_adjoint_workspace_bytes(lbm_grid_t g, int32_t K, size_t* lambda_bytes, size_t* workspace_bytes) {
  if (!g || K < 1) return LBM_ERR_ARG;
  if (lbm_status s = adjoint_supported(g)) return s;
  AdjLayout a = adjoint_layout(g, K);
  if (lambda_bytes) *lambda_bytes = a.lam_bytes;
  if (workspace_bytes) *workspace_bytes = a.total;
  return LBM_OK;
}

lbm_status lbm_adjoint_seed(lbm_grid_t g, void* lambda, void* workspace, double* ke_out) {
  if (lbm_status s = check_bound(g)) return s;
  if (lbm_status s = adjoint_supported(g)) return s;
  if (!lambda || !workspace) return fail(g, LBM_ERR_ARG, "null lambda or workspace");
  AdjLayout a = adjoint_layout(g, 1);
  double* partial = reinterpret_cast<double*>(static_cast<uint8_t*>(workspace) + a.partial_off);
  cudaError_t e = cudaSuccess;
  for (size_t pi = 0; pi < g->hg.P.size() && !e; ++pi) {
    HostPatch& p = g->hg.P[pi];
    e = lbmk::launch_adj_seed(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur],
                              static_cast<uint8_t*>(lambda) + a.lam_off[pi], 1.0 / (double)(1LL << (3 * p.level)),
                              p.level > 0 ? 1 : 0, partial + kDiagBlocks * pi, kDiagBlocks, g->stream);
  }
  double* dke = partial + kDiagBlocks * g->hg.P.size();
  if (!e) e = lbmk::launch_sum_partials(partial, kDiagBlocks * (int)g->hg.P.size(), dke, g->stream);
  double ke = 0;
  if (!e) e = cudaMemcpyAsync(&ke, dke, sizeof ke, cudaMemcpyDeviceToHost, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_check(g, e, "lbm_adjoint_seed");
  if (ke_out) *ke_out = ke;
  return LBM_OK;
}

lbm_status lbm_adjoint_step(lbm_grid_t g, const void* ckpt, int32_t K, void* lambda_inout, void* workspace,
                            size_t ws_bytes) {
  if (lbm_status s = check_bound(g)) return s;
  if (lbm_status s = adjoint_supported(g)) return s;
  if (!ckpt || !lambda_inout || !workspace || K < 1) return fail(g, LBM_ERR_ARG, "bad adjoint arguments");
  AdjLayout a = adjoint_layout(g, K);
  if (ws_bytes < a.total) return fail(g, LBM_ERR_OOM, "adjoint workspace smaller than lbm_adjoint_workspace_bytes");
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  uint8_t* lam[2] = {static_cast<uint8_t*>(lambda_inout), ws + a.second_off};
  std::vector<int> lcur(g->hg.P.size(), 0);
  cudaError_t e = copy_state(g, const_cast<uint8_t*>(static_cast<const uint8_t*>(ckpt)), false);
  if (e) return cuda_check(g, e, "adjoint restore");
  // recompute the segment, recording each coarse step (outer and inner
  // snapshots); the record's address is a device word the steps advance, so
  // the segment's recording steps replay as one CUDA graph
  auto* slot = reinterpret_cast<unsigned long long*>(ws + a.slot_off);
  e = lbmk::launch_word(slot, (unsigned long long)(uintptr_t)(ws + a.snap_off - a.step_bytes), 0, g->stream);
  if (e) return cuda_check(g, e, "adjoint record");
  int s0 = 0;
  if (!g->graphs || g->timing || !g->rec_warm) {
    // the first recording step runs directly, so that capture finds every
    // kernel loaded (every step, without graphs or under per-launch timing)
    const int n = (!g->graphs || g->timing) ? K : 1;
    for (; s0 < n; ++s0)
      if (lbm_status st = recording_step(g, a, slot)) return st;
    g->rec_warm = true;
  }
  if (s0 < K) {
    // the segment's remaining steps replay as one graph
    const int n = K - s0;
    const std::vector<uint8_t> key = cur_key(g);
    cudaGraphExec_t exec = nullptr;
    for (auto& x : g->rcache)
      if (x.cur == key && x.slot == slot && x.step_bytes == a.step_bytes && x.n == n) exec = x.exec;
    if (!exec) {
      if (g->rcache.size() >= kMaxStepGraphs) {
        for (auto& x : g->rcache) cudaGraphExecDestroy(x.exec);
        g->rcache.clear();
      }
      if (lbm_status st = capture_recording(g, a, slot, key, n, &exec)) return st;
      g->rcache.push_back({key, slot, a.step_bytes, n, exec});
    }
    if (cudaError_t e2 = cudaGraphLaunch(exec, g->stream)) return cuda_check(g, e2, "cudaGraphLaunch");
    const int L = g->hg.nlev, KI = 1 << (L - 1);
    for (int j = 0; j < n; ++j)
      for (auto& p : g->hg.P)
        if ((KI >> (L - 1 - p.level)) & 1) p.cur ^= 1;
  }
  if (cudaError_t e2 = last_values(g, a, slot)) return cuda_check(g, e2, "adjoint record");
  if (!g->graphs || g->timing || !g->adj_swept) {
    // the first walk runs directly, so that capture finds every kernel loaded
    if (lbm_status st = adjoint_walk(g, K, lam, lcur, a, ws)) return st;
    g->adj_swept = true;
  } else {
    std::vector<uint8_t> lkey(lcur.begin(), lcur.end());
    const lbm_grid::AdjGraph* hit = nullptr;
    for (auto& x : g->acache)
      if (x.lcur == lkey && x.K == K && x.lam == lam[0] && x.ws == ws) hit = &x;
    if (!hit) {
      if (g->acache.size() >= kMaxAdjGraphs) {
        for (auto& x : g->acache) cudaGraphExecDestroy(x.exec);
        g->acache.clear();
      }
      lbm_grid::AdjGraph ag{lkey, {}, K, lam[0], ws, nullptr};
      if (lbm_status st = capture_walk(g, K, lam, lcur, a, ws, &ag.exec)) return st;
      ag.lcur_after.assign(lcur.begin(), lcur.end());
      g->acache.push_back(ag);
      hit = &g->acache.back();
    }
    if (cudaError_t e2 = cudaGraphLaunch(hit->exec, g->stream)) return cuda_check(g, e2, "cudaGraphLaunch");
    for (size_t i = 0; i < g->hg.P.size(); ++i) lcur[i] = hit->lcur_after[i];
  }
  // lambda back into the caller's buffer; grid state back at the segment start
  for (size_t pi = 0; pi < g->hg.P.size() && !e; ++pi)
    if (lcur[pi] == 1)
      e = cudaMemcpyAsync(lam[0] + a.lam_off[pi], lam[1] + a.lam_off[pi], 27 * (size_t)g->hg.P[pi].plane * g->hg.real_bytes,
                          cudaMemcpyDeviceToDevice, g->stream);
  if (!e) e = copy_state(g, ws + a.snap_off, false);
  return cuda_check(g, e, "lbm_adjoint_step");
}

lbm_status lbm_adjoint_grad_u0(lbm_grid_t g, const void* lambda, int32_t patch, void* grad_u) {
  if (lbm_status s = check_patch(g, patch)) return s;
  if (lbm_status s = check_bound(g)) return s;
  if (lbm_status s = adjoint_supported(g)) return s;
  if (!lambda || !grad_u) return fail(g, LBM_ERR_ARG, "null lambda or gradient");
  AdjLayout a = adjoint_layout(g, 1);
  HostPatch& p = g->hg.P[patch];
  return cuda_check(g,
                    lbmk::launch_adj_grad_u0(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur],
                                             static_cast<const uint8_t*>(lambda) + a.lam_off[patch],
                                             static_cast<double*>(grad_u), g->stream),
                    "lbm_adjoint_grad_u0");
}

// ---------------------------------------------------------------------------
// Allocation-free diagnostics.  Its partial sums live in this file-scope
// device array instead of the grid's bound buffer.  Host code must not pass
// the array's name to a kernel (on the host it is only a stand-in symbol);
// the device address is looked up once per device with cudaGetSymbolAddress.
namespace {
constexpr int kNoAllocMaxPatches = 16;
constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_scratch[8 * kDiagBlocks * kNoAllocMaxPatches + 8];
std::atomic<double*> g_noalloc_ptr[kMaxDevices];
std::mutex g_noalloc_lookup;

// Makes a device current for the lifetime of the guard and restores the
// caller's current device afterwards.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (!err && prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Device address of the scratch array on device dev (current), looked up once
// per device under a lock and published atomically.
cudaError_t noalloc_scratch(int dev, double** out) {
  double* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_noalloc_lookup);
    p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
    if (!p) {
      void* ptr = nullptr;
      if (cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) return e;
      p = static_cast<double*>(ptr);
      g_noalloc_ptr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return cudaSuccess;
}
}  // namespace

lbm_status lbm_diagnostics_noalloc(lbm_grid_t g, double out[8]) {
  if (lbm_status s = check_bound(g)) return s;
  if (!out) return fail(g, LBM_ERR_ARG, "null output");
  if ((int)g->hg.P.size() > kNoAllocMaxPatches)
    return fail(g, LBM_ERR_ARG,
                "lbm_diagnostics_noalloc handles at most " + std::to_string(kNoAllocMaxPatches) +
                    " patches; this grid has " + std::to_string(g->hg.P.size()));
  // the grid's device (that of its bound buffer), current for this call
  const int dev = g->device;
  if (dev < 0 || dev >= kMaxDevices) return fail(g, LBM_ERR_ARG, "device index beyond the supported range");
  DeviceGuard guard(dev);
  if (guard.err) return cuda_check(g, guard.err, "cudaSetDevice");
  double* partial = nullptr;
  if (cudaError_t e = noalloc_scratch(dev, &partial)) return cuda_check(g, e, "cudaGetSymbolAddress");
  double* dout = partial + 8 * kDiagBlocks * kNoAllocMaxPatches;
  // every partial slot and the 8 outputs are written before they are read in
  // this call, so nothing needs clearing between calls
  int nb = 0;
  cudaError_t e = cudaSuccess;
  for (auto& p : g->hg.P) {
    if (!e)
      e = lbmk::launch_diag(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur],
                            1.0 / (double)(1LL << (3 * p.level)), level_force(g, p.level), partial + 8 * nb,
                            kDiagBlocks, g->stream);
    nb += kDiagBlocks;
  }
  if (!e) e = lbmk::launch_diag_final(partial, nb, dout, g->stream);
  double host[8];
  int status = 0;
  if (!e) e = cudaMemcpyAsync(host, dout, sizeof host, cudaMemcpyDeviceToHost, g->stream);
  if (!e) e = cudaMemcpyAsync(&status, status_ptr(g), sizeof status, cudaMemcpyDeviceToHost, g->stream);
  if (!e) e = cudaStreamSynchronize(g->stream);
  if (e) return cuda_check(g, e, "lbm_diagnostics_noalloc");
  return diag_result(g, host, status, out);
}

lbm_status lbm_force(lbm_grid_t g, const double* accel0, double* drag_out) {
  if (!g) return LBM_ERR_ARG;
  if (accel0) {
    for (int a = 0; a < 3; ++a) g->accel[a] = accel0[a];
    g->drop_graphs();  // the force is baked into the captured launches
  }
  if (!drag_out) return LBM_OK;
  if (lbm_status s = check_bound(g)) return s;
  double* partial = at<double>(g, g->off_partial);
  int nb = 0;
  cudaError_t e = cudaSuccess;
  for (auto& p : g->hg.P) {
    if (p.drag_node.empty()) continue;
    if (!e)
      e = lbmk::launch_drag(g->hg.desc.storage, view(g, p), g->base + p.off_f[p.cur], at<uint32_t>(g, p.off_drag_node),
                            at<uint32_t>(g, p.off_drag_mask), (int64_t)p.drag_node.size(),
                            1.0 / (double)(1LL << (2 * p.level)), partial + 3 * nb, kDiagBlocks, g->stream);
    nb += kDiagBlocks;
  }
  double host[3] = {0, 0, 0};
  if (nb > 0) {
    double* dout = at<double>(g, g->off_diag_out);
    if (!e) e = lbmk::launch_drag_final(partial, nb, dout, g->stream);
    if (!e) e = cudaMemcpyAsync(host, dout, sizeof host, cudaMemcpyDeviceToHost, g->stream);
    if (!e) e = cudaStreamSynchronize(g->stream);
    if (e) return cuda_check(g, e, "lbm_force drag");
  }
  for (int a = 0; a < 3; ++a) drag_out[a] = host[a];
  return LBM_OK;
}

lbm_status lbm_checkpoint_bytes(lbm_grid_t g, size_t* bytes) {
  if (!g || !bytes) return LBM_ERR_ARG;
  size_t b = 0;
  for (auto& p : g->hg.P) b += 27 * (size_t)p.plane * g->hg.pop_bytes * (g->hg.thermal ? 2 : 1);
  *bytes = b;
  return LBM_OK;
}

lbm_status lbm_checkpoint(lbm_grid_t g, void* dev, int32_t save) {
  if (lbm_status s = check_bound(g)) return s;
  if (!dev) return fail(g, LBM_ERR_ARG, "null checkpoint buffer");
  uint8_t* d = static_cast<uint8_t*>(dev);
  cudaError_t e = cudaSuccess;
  for (auto& p : g->hg.P) {
    const size_t n = 27 * (size_t)p.plane * g->hg.pop_bytes;
    for (int set = 0; set < (g->hg.thermal ? 2 : 1); ++set) {
      const size_t* off = set ? p.off_g : p.off_f;
      if (save) {
        if (!e) e = cudaMemcpyAsync(d, g->base + off[p.cur], n, cudaMemcpyDeviceToDevice, g->stream);
      } else {
        if (!e) e = cudaMemcpyAsync(g->base + off[p.cur], d, n, cudaMemcpyDeviceToDevice, g->stream);
        if (!e) e = cudaMemcpyAsync(g->base + off[1 - p.cur], d, n, cudaMemcpyDeviceToDevice, g->stream);
      }
      d += n;
    }
  }
  return cuda_check(g, e, "lbm_checkpoint");
}

lbm_status lbm_collide_nodes(const void* f_in, void* f_out, void* gamma_out, int64_t n, double beta,
                             const double du[3], int32_t lbgk, int32_t dtype, void* cuda_stream) {
  if (!f_in || !f_out || n < 0 || (dtype != 0 && dtype != 1)) return LBM_ERR_ARG;
  lbmk::Force F{};
  if (du)
    for (int a = 0; a < 3; ++a) F.du[a] = du[a];
  cudaError_t e = lbmk::launch_collide_nodes(f_in, f_out, gamma_out, n, beta, F, lbgk, dtype,
                                             static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_timing(lbm_grid_t g, int32_t enable) {
  if (!g) return LBM_ERR_ARG;
  if (enable) {
    g->recs.clear();
    g->pool_used = 0;
  }
  g->timing = enable != 0;
  return LBM_OK;
}

lbm_status lbm_timing_report(lbm_grid_t g, int32_t max_rows, int32_t* n_rows, int32_t* kind, int32_t* level,
                             int64_t* launches, double* ms, double* nodes) {
  if (!g || !n_rows) return LBM_ERR_ARG;
  if (cudaError_t e = cudaStreamSynchronize(g->stream)) return cuda_check(g, e, "lbm_timing_report");
  struct Row {
    int kind, level;
    int64_t n;
    double ms, nodes;
  };
  std::vector<Row> rows;
  for (auto& r : g->recs) {
    float t = 0;
    if (cudaError_t e = cudaEventElapsedTime(&t, r.e0, r.e1)) return cuda_check(g, e, "cudaEventElapsedTime");
    Row* row = nullptr;
    for (auto& x : rows)
      if (x.kind == r.kind && x.level == r.level) row = &x;
    if (!row) {
      rows.push_back(Row{r.kind, r.level, 0, 0.0, 0.0});
      row = &rows.back();
    }
    row->n += 1;
    row->ms += t;
    row->nodes += r.nodes;
  }
  *n_rows = (int32_t)rows.size();
  for (int32_t k = 0; k < (int32_t)rows.size() && k < max_rows; ++k) {
    if (kind) kind[k] = rows[k].kind;
    if (level) level[k] = rows[k].level;
    if (launches) launches[k] = rows[k].n;
    if (ms) ms[k] = rows[k].ms;
    if (nodes) nodes[k] = rows[k].nodes;
  }
  return LBM_OK;
}

const char* lbm_last_error(lbm_grid_t g) { return g ? g->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
