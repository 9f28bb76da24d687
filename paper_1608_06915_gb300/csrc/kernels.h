// Kernel launchers (host side).  Every launcher enqueues on the given stream
// and returns the launch status; storage selects the instantiation:
//   LBM_FP64 -> double/double, LBM_FP32 -> float/float,
//   LBM_FP16_SHIFT -> __half/float, LBM_BF16_SHIFT -> __nv_bfloat16/float.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

struct PatchDev;

struct Force {
  double du[3];  // velocity increment per step of this level (exact difference method)
  bool on() const { return du[0] != 0.0 || du[1] != 0.0 || du[2] != 0.0; }
  // compile-time force mask of the hot kernels: 0 none, 1 x only, 4 z only, 7 any
  int mask() const {
    const int m = (du[0] != 0.0) | ((du[1] != 0.0) << 1) | ((du[2] != 0.0) << 2);
    return (m == 0 || m == 1 || m == 4) ? m : 7;
  }
};

// Thermal parameters of one level: wall temperatures minus T0 per wall face,
// g*lambda / 2^level, T_ref - T0, beta, beta1, LBGK mirror flag.
struct ThermalLevel {
  double twd[7];  // wall temperature - T0 per wall face; [6]: isothermal solid surfaces
  double glam, tref_d, beta, beta1;
  int lbgk;
  int pr_gt1;     // Pr > 1 rows of Table I
  int solid_iso;  // solid surfaces held at twd[6] (else adiabatic)
  int wait_sleeps;  // bound of the TMA pass's waits for a loaded stage (lbm_wait_limit)
};

cudaError_t launch_th_tiles(int storage, const PatchDev& p, const void* fin, const void* gin, void* fout, void* gout,
                            const uint32_t* tiles, int64_t ntiles, int ntx, const ThermalLevel& L, int odd,
                            int* status, cudaStream_t st);
// Thermal TMA tile pass of one patch; maps = {f load, f store, f wrap, g load,
// g store, g wrap} descriptors (thermal_tma.cu).  Variant 0 stores f and g
// from registers directly to fout and gout (3 CTAs per SM); variant 1 stores
// them through a shared-memory stage with TMA (2 CTAs per SM).
int th_tma_variants();
cudaError_t launch_th_tma(int storage, int variant, const void* const maps[6], const PatchDev& p, const void* fin,
                          void* fout, void* gout, const unsigned long long* tiles, int64_t ntiles,
                          const ThermalLevel& L, int* status, cudaStream_t st);
cudaError_t launch_th_nodes(int storage, const PatchDev& p, const void* fin, const void* gin, void* fout, void* gout,
                            const uint32_t* nodes, int64_t n, const ThermalLevel& L, int* status, cudaStream_t st);
cudaError_t launch_th_coalesce(int storage, const PatchDev& child, const void* fin_c, const void* gin_c,
                               const PatchDev& parent, void* fo_p, void* go_p, const uint32_t* cf_parent,
                               const uint32_t* cf_child, int64_t n, double ff, double fg, const ThermalLevel& Lc,
                               const ThermalLevel& Lp, int* status, cudaStream_t st);
cudaError_t launch_th_samples(int storage, const PatchDev& parent, const void* fin_p, const void* gin_p,
                              const PatchDev& child, const void* fin_c, const void* gin_c, const uint32_t* smp_node,
                              const uint8_t* smp_kind, int64_t ns, void* smp_val, int64_t ld, double ff, double fg,
                              const ThermalLevel& Lp, const ThermalLevel& Lc, int* status, cudaStream_t st);
cudaError_t launch_th_explode(int storage, const PatchDev& child, void* fo_c, void* go_c, const uint32_t* ex_node,
                              const uint32_t* ex_src, int64_t n_one, int64_t n, const void* val, int64_t ld,
                              const ThermalLevel& Lc, cudaStream_t st);
cudaError_t launch_th_init(int storage, const PatchDev& p, void* f0, void* f1, void* g0, void* g1, const void* rho,
                           const void* u, const void* T, int dtype, const double u_in[3], cudaStream_t st);
cudaError_t launch_th_moments(int storage, const PatchDev& p, const void* fin, const void* gin, void* rho, void* u,
                              void* T, void* gamma, int dtype, const ThermalLevel& L, cudaStream_t st);

// Discrete adjoint kernels (adjoint.cu), FP32/FP64 storage, isothermal.
// with_bc: the patch has boundary-class nodes (their node-by-node kernel runs
// too, and both add into lambda_old, which must be cleared first); without
// them one kernel writes every entry of lambda_old with plain stores
cudaError_t launch_adj_sc(int storage, const PatchDev& p, const void* fin, const void* lam_new, void* lam_old,
                          double beta, int odd, int lbgk, bool with_bc, int* status, cudaStream_t st);
cudaError_t launch_adj_coalesce(int storage, const PatchDev& child, const void* fin_c, const PatchDev& parent,
                                const void* lam_new_p, void* lam_old_c, const uint32_t* cf_parent,
                                const uint32_t* cf_child, int64_t n, double r, double beta_p, int lbgk, int* status,
                                cudaStream_t st);
// vbar [31][ld]: adjoint of the point-space values (accumulated with atomics)
// the explode adjoint writes, per target k, the adjoint of its 31
// interpolated values to tbar[c][k] (c < 31, n targets)
cudaError_t launch_adj_explode(int storage, const PatchDev& child, const void* lam_new_c, const uint32_t* ex_node,
                               const uint32_t* ex_src, int64_t n_one, int64_t n, const void* val, void* tbar,
                               int64_t ld, double beta_c, int lbgk, cudaStream_t st);
// transpose of the interpolation in gather form: vbar[c][j] for columns j in
// [j0, j1) = sum over the consumers of column j (use_ptr, use_ent) of their
// weight times tbar[c][target] or vbar[c][point]; the consumers of a stage
// must be done first (stage 2, then stage 1, then the samples)
cudaError_t launch_adj_gather(int storage, const uint32_t* use_ptr, const uint32_t* use_ent, int64_t j0, int64_t j1,
                              void* vbar, int64_t ld, const void* tbar, int64_t nt, cudaStream_t st);
cudaError_t launch_adj_samples(int storage, const PatchDev& parent, const void* fin_p, void* lam_p,
                               const PatchDev& child, const void* fin_c, void* lam_c, const uint32_t* smp_node,
                               const uint8_t* smp_kind, int64_t ns, const void* sbar, int64_t ld, double rescale_p,
                               int* status, cudaStream_t st);
cudaError_t launch_adj_seed(int storage, const PatchDev& p, const void* fin, void* lam, double vol_weight,
                            int child_level, double* partial, int blocks, cudaStream_t st);
cudaError_t launch_sum_partials(const double* partial, int n, double* out, cudaStream_t st);
cudaError_t launch_adj_grad_u0(int storage, const PatchDev& p, const void* fin, const void* lam, double* grad,
                               cudaStream_t st);

// Bulk tiles through TMA (tmap_in / tmap_out / tmap_wrap: CUtensorMaps, 128
// bytes, of the source buffer with the load box, of the destination buffer with
// the store box, and of the source buffer with the wrap box; tiles:
// x-tile | y << 16 | z << 32) and mixed tiles node by node (tile id
// = (z * ny + y) * ntx + tx); a tile is 128 nodes along x, or 64 for the
// 64-node tile variant (its load descriptor and tile list then hold halves).
// One patch of a batched TMA tile pass.
struct TmaLaunchPatch {
  const void* tmap_in;    // load descriptor of the current buffer
  const void* tmap_out;   // store descriptor of the next buffer
  const void* tmap_wrap;  // 16-byte wrap descriptor of the current buffer
  PatchDev p;
  const void* fin;        // current buffer (the fixed inlet nodes are copied from it)
  const unsigned long long* tiles;
  int64_t ntiles;
  double beta;
  Force F;
};
// TMA tile pass over up to 8 patches in one persistent launch; variant picks
// the load-stage / occupancy configuration (0 .. sc_tma_variants() - 1).
// wait_sleeps: bound of the consumers' waits for a loaded stage (0.5 us
// suspensions; about a second by default, set from lbm_wait_limit).
cudaError_t launch_sc_tma(int storage, const TmaLaunchPatch* ps, int n, int variant, int lbgk, int wait_sleeps,
                          int* status, cudaStream_t st);
int sc_tma_variants(int storage);
// nodes per tile of a variant: 128, or 64 (tmap_in of kind 3, the half-tile list)
int sc_tma_tile_nodes(int storage, int variant);
// node-by-node recomputation of listed nodes (after the TMA tile pass)
cudaError_t launch_sc_nodes(int storage, const PatchDev& p, const void* fin, void* fout, const uint32_t* nodes,
                            int64_t n, double beta, const Force& F, int lbgk, int* status, cudaStream_t st);
cudaError_t launch_sc_tiles(int storage, const PatchDev& p, const void* fin, void* fout, const uint32_t* tiles,
                            int64_t ntiles, int ntx, double beta, const Force& F, int odd, int lbgk, int* status,
                            cudaStream_t st);
// kind 0: load box (128-node tile row + halos), 1: store box (one warp's 32 nodes),
// 2: 16-byte wrap box, 3: load box of a 64-node tile row + halos
cudaError_t make_tensor_map(int storage, void* out128, const void* base, const PatchDev& p, int kind);

cudaError_t launch_coalesce(int storage, const PatchDev& child, const void* fin_child, const PatchDev& parent,
                            void* fout_parent, const uint32_t* cf_parent, const uint32_t* cf_child, int64_t n,
                            double rescale, double beta_parent, const Force& Fp, int lbgk, int* status,
                            cudaStream_t st);

cudaError_t launch_samples(int storage, const PatchDev& parent, const void* fin_parent, const PatchDev& child,
                           const void* fin_child, const uint32_t* smp_node, const uint8_t* smp_kind, int64_t ns,
                           void* smp_val, int64_t ld, double rescale_parent, int* status, cudaStream_t st);

// Point space of the reconstruction: values [ncomp][ld] (compute type),
// samples in columns [0, ns), intermediate points after them.
// Intermediate points q < n: column out0 + q from the 4 columns pt_src[4q ..].
cudaError_t launch_points(int storage, int ncomp, const uint32_t* pt_src, int64_t n, void* val, int64_t ld,
                          int64_t out0, cudaStream_t st);
// Targets [0, n_one) read the column ex_src[4k], the others interpolate ex_src[4k .. 4k + 3].
cudaError_t launch_explode(int storage, const PatchDev& child, void* fout_child, const uint32_t* ex_node,
                           const uint32_t* ex_src, int64_t n_one, int64_t n, const void* val, int64_t ld,
                           double beta_child, const Force& Fc, int lbgk, cudaStream_t st);

cudaError_t launch_init(int storage, const PatchDev& p, void* f0, void* f1, const void* rho, const void* u,
                        int dtype, const double u_in[3], cudaStream_t st);

cudaError_t launch_moments(int storage, const PatchDev& p, const void* fin, void* rho, void* u, void* gamma,
                           int dtype, double beta, const Force& F, int lbgk, cudaStream_t st);

// gset = 1: the thermal g set, stored as the deviation from W_i c_i^2 (else from W_i)
cudaError_t launch_copy_pop(int storage, const PatchDev& p, void* fstore, void* dense, int dtype, int to_dense,
                            int gset, cudaStream_t st);

// FP64 partial sums of one patch into partial[blocks][8]; see lbm_diagnostics.
// Device-to-device copies of up to kCopySegs segments in one launch (the
// copy engines are slower than the SMs for state-sized copies).
// With rel set, dst[j] holds offsets from the address stored at *rel (a
// device word), so that a captured graph can copy to a moving destination.
constexpr int kCopySegs = 16;
struct CopySegs {
  void* dst[kCopySegs];
  const void* src[kCopySegs];
  size_t bytes[kCopySegs];
  int n;
  // destinations relative to *rel when set; with done set, the last block to
  // finish adds `advance` to *rel (every block has read it by then) and
  // clears *done, which must be 0 at launch
  unsigned long long* rel;
  unsigned long long advance;
  unsigned* done;
};
cudaError_t launch_copy(const CopySegs& segs, cudaStream_t st);
// *word = value (set, which also clears the 32-bit count that follows the
// word) or *word += value (advance), one thread
cudaError_t launch_word(unsigned long long* word, unsigned long long value, int advance, cudaStream_t st);

// Source patches of a state transfer (regridding): views, current f buffers,
// levels and betas, and the order in which a destination level tries them.
constexpr int kTransferMax = 16;
struct TransferSrc {
  PatchDev p[kTransferMax];
  const void* f[kTransferMax];
  int level[kTransferMax];
  double beta[kTransferMax];
  int order[kTransferMax];
  int n_src;
  int n[3];
  int periodic[3];
};
cudaError_t launch_transfer(int storage, const PatchDev& p, void* f0, void* f1, int level, double beta,
                            const double u_in[3], const TransferSrc& T, unsigned long long* missing,
                            cudaStream_t st);
cudaError_t launch_gamma_blocks(int storage, const PatchDev& p, const void* fin, double beta, int lbgk, int B,
                                float* out, int* status, cudaStream_t st);
cudaError_t launch_diag(int storage, const PatchDev& p, const void* fin, double vol_weight, const Force& F,
                        double* partial, int blocks, cudaStream_t st);
cudaError_t launch_diag_final(const double* partial, int total_blocks, double* out8, cudaStream_t st);
// clears the given bits of the device status word (one atomic)
cudaError_t launch_status_clear(int* status, int bits, cudaStream_t st);
// momentum-exchange force: per-block FP64 sums [blocks][3] of c_j (f'_j + f_{-j}) * scale over the links, the
// returning f_{-j} = f'_j at a half-way wall and interpolated along the link where p carries wall fractions
cudaError_t launch_drag(int storage, const PatchDev& p, const void* fin, const uint32_t* node, const uint32_t* mask,
                        int64_t n, double scale, double* partial, int blocks, cudaStream_t st);
cudaError_t launch_drag_final(const double* partial, int total_blocks, double* out3, cudaStream_t st);

cudaError_t launch_collide_nodes(const void* fin, void* fout, void* gamma, int64_t n, double beta, const Force& F,
                                 int lbgk, int dtype, cudaStream_t st);

}  // namespace lbmk
