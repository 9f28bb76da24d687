/*
 * lbm.h -- C ABI of liblbm.so: grid-refined entropic lattice Boltzmann
 * (D3Q27 KBC) on one GPU.
 *
 * The method is that of Dorschner, Frapolli, Chikatamarla & Karlin, "Grid
 * refinement for entropic lattice Boltzmann models" (arXiv:1608.06915):
 *   - per level, the lattice Boltzmann equation with the KBC mirror state and
 *     entropic stabiliser gamma (Sec. II.A, Eqs. f_equations, feq_iso,
 *     popSplit, f_mirr, gamma_min_approx);
 *   - the two-population thermal model, Pr <= 1 and Pr > 1 (Sec. II.B);
 *   - multi-domain refinement with r = 2: twin-node non-equilibrium
 *     rescaling (Sec. III.A, Eq. f_neq_rescaling_iso and the thermal g
 *     rule), centred four-point Lagrange reconstruction (Sec. III.B,
 *     Eq. interp) and the five-step algorithm without time interpolation
 *     (Sec. III.C), with the fine level taking two steps per parent step;
 *   - a body force by the exact difference method, du_f = du_c / r (Sec. III.A);
 *   - around the method: the momentum-exchange drag, a discrete adjoint of the
 *     refined step, the refinement indicator |gamma - 2| the paper proposes
 *     (Sec. IV and its conclusion) and a state transfer onto a new layout.
 *
 * Conventions
 *   Velocities: i = (cx+1) + 3(cy+1) + 9(cz+1); rest i = 13; opposite 26 - i.
 *   Units: everything in the descriptor is in coarse (level-0) lattice units.
 *   Level l has spacing 2^-l; its integer node coordinates are 2^l times the
 *   coarse coordinates.
 *   Layout: a patch is one refinement box of one level; its nodes live in a
 *   storage box (the bounding box of its nodes, lbm_patch_info).  Arrays that
 *   cross this ABI are dense over the storage box, x fastest: [z][y][x] for
 *   scalars, [27][z][y][x] for populations and [3][z][y][x] for vectors.
 *   Memory: the library allocates no device memory.  lbm_grid_bytes reports
 *   the size of the one device buffer a grid needs (populations, node tables,
 *   interface tables and workspace); the caller allocates it and hands it to
 *   lbm_grid_bind, and frees it after lbm_grid_destroy.  All other pointers
 *   marked "device" are caller-owned device memory; "host" pointers are
 *   caller-owned host memory that the call only reads during the call.
 *   Streams: every call that launches work enqueues it on the stream given
 *   to lbm_grid_bind and returns without waiting, unless it says otherwise.
 *   Errors: every call returns an lbm_status; nothing aborts.  A failed call
 *   leaves a message retrievable with lbm_last_error.
 */
#ifndef LBM_H_
#define LBM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_grid* lbm_grid_t;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,      /* bad argument (null pointer, out-of-range index, size) */
  LBM_ERR_LAYOUT = -2,   /* refinement layout violates the nesting rules */
  LBM_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  LBM_ERR_OOM = -4,      /* bound buffer smaller than lbm_grid_bytes */
  LBM_ERR_UNSTABLE = -5, /* non-finite or non-positive density detected */
  LBM_ERR_TIMEOUT = -6,  /* a bounded device-side wait expired */
  LBM_ERR_STATE = -7     /* call not valid in the grid's current state */
} lbm_status;

typedef enum {
  LBM_FP64 = 0,       /* populations stored and collided in double */
  LBM_FP32 = 1,       /* stored and collided in float */
  LBM_FP16_SHIFT = 2, /* stored as half of f_i - W_i*rho0 (rho0 = 1), collided in float */
  LBM_BF16_SHIFT = 3  /* stored as bfloat16 of f_i - W_i*rho0, collided in float */
} lbm_storage;

typedef enum { LBM_ISO_KBC = 0, LBM_THERMAL_KBC = 1 } lbm_model;

/* One refinement box: level >= 1, closed box [lo, hi] in coarse node
 * coordinates.  A box of level l must lie inside a box of level l-1 (or the
 * domain for l = 1), at least 4 level-(l-1) nodes inside its interface faces
 * and at least 8 level-(l-1) spacings wide across each interface axis.  A box
 * covering all coarse nodes of a periodic axis spans it (no interface there);
 * a face on a wall is a wall face (no interface there). */
typedef struct {
  int32_t level;
  int32_t lo[3], hi[3];
} lbm_box;

typedef struct {
  int32_t n[3];             /* coarse node counts */
  uint32_t periodic;        /* bit a: axis a periodic */
  uint32_t walls;           /* bit 2a: half-way bounce-back wall below node 0 of axis a,
                               bit 2a+1: above the last node (isothermal for g) */
  int32_t inflow_axis;      /* -1: none; else equilibrium inlet at the min face of this
                               axis (level 0) and zero-gradient outlet at the max face */
  double u_in[3];           /* inlet velocity (inlet density 1) */
  const lbm_box* boxes;     /* host; copied by lbm_grid_create */
  int32_t n_boxes;
  const uint8_t* solid;     /* host, nullable: solid mask on level solid_level, [z][y][x]
                               over solid_dims starting at solid_lo (that level's
                               coordinates); copied by lbm_grid_create */
  int32_t solid_level;
  int32_t solid_lo[3];
  int32_t solid_dims[3];
  double nu0;               /* coarse kinematic viscosity (beta_0 from Eq. visc) */
  double accel0[3];         /* body acceleration, coarse units (isothermal model) */
  lbm_model model;
  double pr, t0, glambda, t_ref; /* thermal: Prandtl (> 0; Table I's Pr > 1 rows above 1),
                                   T0 (1/3), g*lambda, Boussinesq T_ref */
  double wall_T[6];         /* thermal wall temperatures per wall face (bit order of walls) */
  lbm_storage storage;
  int32_t mirror_lbgk;      /* 1: LBGK mirror state (gamma fixed at 2) */
  double solid_T;           /* thermal: temperature of solid surfaces when solid_isothermal */
  int32_t solid_isothermal; /* thermal: 1 = solid surfaces held at solid_T (anti-bounce-back
                               of g, as at the plates; the heated sphere of Sec. IV),
                               0 = adiabatic solids (bounce-back of g) */
  /* Curved solid surface (the sphere of Sec. IV; the paper's own wall
   * condition is Grad's, whose definition it cites elsewhere): with
   * shape_kind 0 the solid mask's links reflect half-way (a staircase);
   * otherwise the analytic surface -- 1 sphere (centre shape_c, radius
   * shape_r), 2 cylinder along axis shape_axis, 3 plane normal to shape_axis
   * through shape_c; coarse units -- gives, on every link from a fluid node to
   * a solid node of solid_level, the fraction q of the link at which the wall
   * lies, and the returning populations are interpolated linearly along the
   * link (Bouzidi, Firdaouss & Lallemand 2001: f; the same construction on
   * the anti-bounce-back of g at an isothermal surface).  shape_solid_inside:
   * the solid is inside the sphere or cylinder (on the lower side of the
   * plane), else outside.  A link the surface does not cross in (0, 1]
   * reflects half-way. */
  int32_t shape_kind;
  double shape_c[3];
  double shape_r;
  int32_t shape_axis;
  int32_t shape_solid_inside;
} lbm_desc;

/* Builds the level/patch layout, node classes and interface tables
 * (Sec. III, Fig. 1 layout) and validates the nesting rules.
 * desc: host, read during the call.  out: receives the handle.
 * Returns LBM_ERR_LAYOUT (with a message) for invalid layouts. */
lbm_status lbm_grid_create(const lbm_desc* desc, lbm_grid_t* out);

/* Size in bytes of the device buffer the grid needs. */
lbm_status lbm_grid_bytes(lbm_grid_t g, size_t* device_bytes);

/* Binds caller-owned device memory (at least lbm_grid_bytes, 256-byte
 * aligned) and a CUDA stream (cudaStream_t, may be 0) to the grid and uploads
 * the node and interface tables.  Synchronises that stream before returning. */
lbm_status lbm_grid_bind(lbm_grid_t g, void* dev_ptr, size_t bytes, void* cuda_stream);

/* Releases the host-side descriptor and tables; does not free bound memory. */
lbm_status lbm_grid_destroy(lbm_grid_t g);

/* Number of patches (index 0 is level 0) and number of levels. */
lbm_status lbm_num_patches(lbm_grid_t g, int32_t* n_patches, int32_t* n_levels);

/* Patch metadata: level, parent patch (-1 for level 0), storage-box origin
 * (level coordinates) and extents, and the relaxation parameters beta, beta1
 * of its level (Sec. III.A: beta_f = 1/(1 + r(1/beta_c - 1))). */
lbm_status lbm_patch_info(lbm_grid_t g, int32_t patch, int32_t* level, int32_t* parent, int64_t org[3],
                          int64_t dim[3], double* beta, double* beta1);

/* Refinement indicator (Sec. IV, channel: the stabiliser gamma of Eq.
 * gamma_min_approx tends to its LBGK value 2 where the flow is resolved, so
 * its deviation measures under-resolution; the conclusion proposes it as the
 * criterion of adaptive refinement).  For each block of block^3 nodes of the
 * patch's storage box, out receives the largest |gamma - 2| over the block's
 * bulk and boundary-class nodes (0 without such nodes), gamma of the state
 * the next lbm_step collides there: the pull of the stored f.  Interface
 * nodes, whose next state comes from the coupling, are left out.  out: caller-owned device float [nbz][nby][nbx], nb_a =
 * ceil(dim_a / block) with dim from lbm_patch_info; zeroed, then filled,
 * asynchronously on the bound stream.  LBM_ERR_ARG for a bad patch, block < 1
 * or null out; LBM_ERR_STATE if unbound. */
lbm_status lbm_gamma_blocks(lbm_grid_t g, int32_t patch, int32_t block, float* out);

/* State transfer onto another layout (regridding), for adaptive refinement,
 * which the paper leaves to future work.  Every node of dst takes the state of
 * the src level nearest its own that holds it (own level, then finer ones,
 * then coarser ones): the coinciding node, or a trilinear interpolation of rho,
 * u and f - f^eq over the source cell around it.  The stored f - f^eq is
 * rescaled between levels by (1 - 2 beta_t)/(1 - 2 beta_s) beta_s/(r beta_t),
 * r = dx_s / dx_t: the ratio of Eq. f_neq_rescaling_iso for the pre-collision
 * part, with each level's post-collision factor.  Solid nodes take the rest
 * state and inlet nodes the inflow equilibrium.  Both grids bound, isothermal,
 * same storage, extents and periodicity; at most 16 source patches (else
 * LBM_ERR_ARG).  Waits for src's stream, runs on dst's and synchronises it.
 * missing (nullable) receives the number of fluid nodes no source level holds;
 * they take the rest state. */
lbm_status lbm_transfer(lbm_grid_t dst, lbm_grid_t src, int64_t* missing);

/* Node classes over the storage box, host output [z][y][x]: 0 no node (hole
 * or outside), 1 fluid, 2 solid. */
lbm_status lbm_patch_mask(lbm_grid_t g, int32_t patch, uint8_t* host_out);

/* Node updates per coarse step, sum over levels of fluid nodes * 2^level
 * (the fine-node-equivalent count behind the MLUPS metric). */
lbm_status lbm_node_updates(lbm_grid_t g, double* per_coarse_step);

/* f = f^eq(rho, u) (Eq. feq_iso) on every fluid node of a patch, and for the
 * thermal model g = g^eq(rho, u, T) (Table I, Eq. grad_general).  Inlet nodes
 * take f^eq(1, u_in).  rho: device [z][y][x]; u: device [3][z][y][x];
 * T: device [z][y][x] or NULL (T0).  dtype: 0 float, 1 double. */
lbm_status lbm_init_equilibrium(lbm_grid_t g, int32_t patch, const void* rho, const void* u, const void* T,
                                int32_t dtype);

/* Advances n_coarse_steps coarse steps: one coarse step runs the algorithm of
 * Sec. III.C recursively, level l taking 2^l steps.  Asynchronous with respect
 * to the host and ordered on the bound stream: work forked onto the library's
 * internal streams inside an instant is joined back into the bound stream
 * before the instant ends.  LBM_ERR_ARG for a negative count, LBM_ERR_STATE for
 * an unbound grid, LBM_ERR_CUDA for a launch failure. */
lbm_status lbm_step(lbm_grid_t g, int64_t n_coarse_steps);

/* Autotuner of the instant schedule.  Isothermal model: a variant is a TMA
 * kernel (load stages in shared memory x CTAs per SM the register allocation
 * aims for; for FP32 arithmetic also the node-pair kernels on packed FP32x2
 * instructions; last, the tile shape: 64-node tiles instead of 128, for rows
 * narrower than a 128-node tile) and a schedule of the reconstruction samples
 * (after the TMA pass, or beside it on the coupling streams): variant v =
 * kernel + n_kernels * schedule, 10 variants (6 for FP64 storage), all with
 * identical results.
 * Thermal model: 2 variants of its TMA pass (f and g stored from registers
 * straight to memory, or through a shared-memory stage by TMA), identical
 * results.  This times `trials` coarse steps of each variant
 * the way lbm_step runs them (graph replays unless lbm_graphs is off), CUDA
 * events around them, then the two fastest again over 3 * trials steps each,
 * and keeps the faster of those.  The state advances by
 * 1 + n_variants * (2 + trials) + 2 * (2 + 3 * trials) coarse steps (one
 * variant: 1 + 2 + trials): one untimed step first, and per timing two
 * untimed steps that capture the variant's step graphs before the trials.
 * chosen (nullable) gets the variant kept, ms_per_step[0 .. min(n,
 * max_variants)) (nullable) the measured time per coarse step of each (the
 * longer timing for the two fastest), n_variants (nullable) their number.
 * Synchronises the bound stream; drops captured step graphs.  Without a call
 * the grid uses variant 0.  The paper has no counterpart. */
lbm_status lbm_autotune(lbm_grid_t g, int32_t trials, int32_t* chosen, float* ms_per_step, int32_t max_variants,
                        int32_t* n_variants);

/* Selects a variant of lbm_autotune directly (0 .. n_variants - 1);
 * LBM_ERR_ARG out of range. */
lbm_status lbm_set_variant(lbm_grid_t g, int32_t variant);

/* Bound of the waits of the TMA stream-collide passes (isothermal and
 * thermal) for a loaded stage, in suspensions of at most 0.5 us each: default
 * 2^21 (about a second); 0 tests once without waiting.  A wait that runs out
 * sets bit 1 of the device status word, and its warps skip the rest of their
 * tiles after waiting (with the full bound) for the copies they may have in
 * flight, so the nodes of those tiles keep stale values; lbm_diagnostics then
 * returns LBM_ERR_TIMEOUT.  Only the consumers' waits take this bound; the
 * waits that drain copies keep the full one.  Not part of the method: this is
 * failure detection, and a small bound exists to test it.  Drops the captured
 * step graphs.  LBM_ERR_ARG for a null grid or a negative bound. */
lbm_status lbm_wait_limit(lbm_grid_t g, int32_t sleeps);

/* lbm_step replays each coarse step as a CUDA graph, one per buffer parity of
 * level 0, captured on a private stream the first time that parity comes up
 * (the first step after lbm_grid_bind launches directly).  Replays use the
 * bound stream.  Binding again or changing the force drops the graphs; steps
 * taken while lbm_timing is on launch directly.  enable = 0 launches every
 * kernel directly.  Default: on.  Returns LBM_ERR_ARG for a null grid. */
lbm_status lbm_graphs(lbm_grid_t g, int32_t enable);

/* Macroscopic fields of a patch's current populations: rho, u = j/rho + du/2
 * (du of the level's body force, Sec. III.A), T (thermal, else T0) and the
 * stabiliser gamma that Eq. gamma_min_approx gives for the stored state (for
 * a post-collision state, which lbm_step stores, that is 2 up to rounding;
 * lbm_gamma_blocks gives the stabiliser of the next collision instead).
 * All device outputs, nullable, layouts as above; dtype 0 float, 1 double. */
lbm_status lbm_moments(lbm_grid_t g, int32_t patch, void* rho, void* u, void* T, void* gamma, int32_t dtype);

/* Copies a patch's current populations (which = 0: f, 1: g) to/from a device
 * array [27][z][y][x], unshifted, dtype 0 float, 1 double. */
lbm_status lbm_get_populations(lbm_grid_t g, int32_t patch, int32_t which, void* dst, int32_t dtype);
lbm_status lbm_set_populations(lbm_grid_t g, int32_t patch, int32_t which, const void* src, int32_t dtype);

/* Sets the body acceleration (coarse units) when accel0 is non-NULL and, when
 * drag_out is non-NULL, returns the drag F_d of Sec. IV A 2 (flow past a
 * sphere) as the FP64 momentum-exchange force of half-way bounce-back on the
 * solid nodes: every link from a fluid node x to a solid neighbour x + c_j
 * hands the solid 2 c_j f'_j(x), evaluated on the current post-collision
 * state (what the next substep streams), scaled by 4^-level (a level-l node
 * holds 8^-l of a coarse volume, a substep lasts 2^-l of a coarse step) and
 * summed over levels: drag_out[3], coarse units.  Zeros for grids without
 * solid nodes.  Synchronises the bound stream when drag_out is set; needs a
 * bound grid (LBM_ERR_STATE otherwise).  Changing the force drops the
 * captured step graphs. */
lbm_status lbm_force(lbm_grid_t g, const double* accel0, double* drag_out);

/* Same results as lbm_diagnostics, for callers that must not allocate device
 * memory themselves -- for example code that runs while another component
 * owns the whole device memory budget, or a host process that hands the
 * library only the buffers it already holds.  lbm_diagnostics keeps its
 * partial sums in the grid's bound buffer; this variant keeps them in a
 * fixed array inside the library (about 300 KB, held on every GPU that loads
 * the library until the process exits), so it allocates nothing, directly or
 * through any library.  The paper has no counterpart: this is plumbing.
 * Limits and rules:
 *   - at most 16 patches per grid; larger grids get LBM_ERR_ARG and a message;
 *   - it runs on the device of the grid's bound buffer, made current for the
 *     call (the caller's current device is restored afterwards);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *     With CUDA's lazy module loading (the default), that first lookup may be
 *     where the driver loads the library's module, and with it the array,
 *     onto the device: device memory can change on the first call only, and
 *     later calls leave it unchanged;
 *   - every call uses the same array: calls that overlap on the GPU (two
 *     streams, or two grids at once) race and can return wrong sums.  Calls
 *     that follow one another are fine: each call writes every slot it reads.
 * Synchronises the bound stream, like lbm_diagnostics. */
lbm_status lbm_diagnostics_noalloc(lbm_grid_t g, double out[8]);

/* FP64 diagnostics over owned fluid nodes (parent nodes that are not twin
 * nodes of a child, child nodes of depth >= 1), volume-weighted 8^-level:
 * out = {mass, jx, jy, jz, kinetic energy 1/2 rho |u|^2, fluid node count,
 * min rho, device status word}.  Synchronises the stream.  The status word's
 * bit 0 flags a pull source that resolved to no node (never on a validated
 * layout), bit 1 an expired bounded wait (lbm_wait_limit).  Returns
 * LBM_ERR_TIMEOUT when bit 1 is set, and clears that bit, so the next call
 * reports only new expiries; otherwise LBM_ERR_UNSTABLE when a density is
 * non-finite or non-positive; out is filled in every case. */
lbm_status lbm_diagnostics(lbm_grid_t g, double out[8]);

/* Bytes of one checkpoint (all patches' current f and g populations). */
lbm_status lbm_checkpoint_bytes(lbm_grid_t g, size_t* bytes);

/* save = 1: copies the current state to dev_dst; save = 0: restores it.
 * dev: caller-owned device buffer of lbm_checkpoint_bytes. */
lbm_status lbm_checkpoint(lbm_grid_t g, void* dev, int32_t save);

/* One KBC collision (Eqs. f_equations, f_mirr, gamma_min_approx, plus the
 * exact-difference-method force du) of n independent nodes: f_in, f_out
 * device [27][n]; gamma_out device [n] or NULL; dtype 0 float, 1 double.
 * The same device code the step runs; used to test the collision alone. */
lbm_status lbm_collide_nodes(const void* f_in, void* f_out, void* gamma_out, int64_t n, double beta,
                             const double du[3], int32_t lbgk, int32_t dtype, void* cuda_stream);

/* Discrete adjoint of lbm_step (not in the paper; the reverse of its algorithm)
 * for isothermal layouts that are periodic -- no walls, solids, inflow or body
 * force -- with FP32 or FP64 storage.  Adjoint populations lambda use the
 * packed layout of all patches in order, each [27][z][y][x_padded] over the
 * storage box with the padded row length the library uses, in the compute
 * precision (float for FP32, double for FP64); they are device buffers the
 * caller owns.
 *
 * lbm_adjoint_workspace_bytes: sizes of lambda and of the workspace needed by
 * segments of K coarse steps (one state snapshot per step, a second lambda
 * buffer, reconstruction-sample adjoints).
 *
 * lbm_adjoint_seed: objective J = kinetic energy 1/2 sum rho |u|^2 8^-level of
 * the current state over owned nodes (a parent owns its nodes outside every
 * child's [a+1, b-1] box, a child its nodes two or more child spacings inside
 * its interface faces), returned in *ke_out (FP64, synchronises), and
 * lambda = dJ/df.
 *
 * lbm_adjoint_step: ckpt holds the state at the segment start (the layout of
 * lbm_checkpoint).  On entry lambda_inout is dJ/d(state after K coarse steps);
 * the call recomputes the K steps from ckpt (one snapshot each), runs their
 * adjoints in reverse and leaves dJ/d(state at the segment start) in
 * lambda_inout and the grid state at the segment start.
 *
 * lbm_adjoint_grad_u0: for a state f = f^eq(rho, u0) (Eq. feq_iso) -- the
 * initial state -- writes dJ/du0 of one patch, device double [3][z][y][x]. */
lbm_status lbm_adjoint_workspace_bytes(lbm_grid_t g, int32_t K, size_t* lambda_bytes, size_t* workspace_bytes);
lbm_status lbm_adjoint_seed(lbm_grid_t g, void* lambda, void* workspace, double* ke_out);
lbm_status lbm_adjoint_step(lbm_grid_t g, const void* ckpt, int32_t K, void* lambda_inout, void* workspace,
                            size_t ws_bytes);
lbm_status lbm_adjoint_grad_u0(lbm_grid_t g, const void* lambda, int32_t patch, void* grad_u);

/* Kernel timing for measurement: enable = 1 makes lbm_step bracket every
 * kernel it launches with CUDA events on the bound stream (and clears earlier
 * records); 0 stops recording.  Not part of the method. */
lbm_status lbm_timing(lbm_grid_t g, int32_t enable);

/* Synchronises the bound stream and reports, per kernel class, the number of
 * launches recorded, their summed device time (ms) and the fluid nodes they
 * wrote.  kind: 0 stream_collide, 1 coalesce, 2 samples, 3 explode; level:
 * the level of the patch written.  Host outputs of length max_rows;
 * *n_rows receives the number of classes. */
lbm_status lbm_timing_report(lbm_grid_t g, int32_t max_rows, int32_t* n_rows, int32_t* kind, int32_t* level,
                             int64_t* launches, double* ms, double* nodes);

const char* lbm_last_error(lbm_grid_t g); /* NULL g: last error of lbm_grid_create */

#ifdef __cplusplus
}
#endif
#endif /* LBM_H_ */
