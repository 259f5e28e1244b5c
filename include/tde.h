/*
 * tde.h -- C ABI of libtde.so, the GB300 (sm_103a) implementation of the
 * per-MeshBlock finite-volume hydro stage of "An End-to-End Numerical Framework
 * for Tidal Disruption Events with AthenaK" (arxiv 2609.37859).
 *
 * Conventions for every entry point:
 *  - Return value: a tde_status code.  No C++ exception, abort or device trap
 *    crosses this boundary; tde_last_error() gives a one-line message for the
 *    last failing call on a context.
 *  - "device" pointers are CUDA global-memory pointers on the context's device
 *    (e.g. from torch tensors); "host" pointers are ordinary CPU memory.
 *  - The library never frees memory it did not allocate.  Objects it creates
 *    (context, EOS, mesh, including their device workspaces) are released by the
 *    matching *_destroy / tde_finalize call.
 *  - Work is enqueued asynchronously on the context's CUDA stream.  Calls that
 *    return host data (tde_counts_read, tde_mesh_info) synchronise that stream.
 *    Every launch sequence of tde_hydro_stage / tde_step / tde_dual_energy_sync
 *    is free of host synchronisation and may be captured in a CUDA graph.
 *
 * State layout.  A MeshBlock is a box of nx*ny*nz interior cells padded with
 * ng ghost cells on both sides of every active direction (a direction whose
 * global extent is one cell is inactive: no ghosts, no flux).  A state is one
 * device array of nvar * ntot doubles,
 *     U[v * ntot + off_b + (k * py + j) * px + i],
 * v = 0..nvar-1 the conserved variables (rho, m_x, m_y, m_z, E_tot[, U_aux])
 * (Eq. remap-state-vector), off_b the first padded cell of block b (blocks in
 * the order given to tde_mesh_create), (px, py, pz) the padded block size and
 * (i, j, k) padded indices; interior cells start at ng.
 */
#ifndef TDE_H
#define TDE_H
#include <stddef.h>
#include <stdint.h>
#if defined(__GNUC__)
#define TDE_API __attribute__((visibility("default")))
#else
#define TDE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TDE_OK = 0,
  TDE_EINVAL = 1,    /* invalid argument (null pointer, bad size, inconsistent layout) */
  TDE_ENOMEM = 2,    /* device or host allocation failed */
  TDE_ECUDA = 3,     /* a CUDA runtime call failed (message in tde_last_error) */
  TDE_ERANGE = 4,    /* table input out of range (only where the call says so) */
  TDE_ENUMERIC = 5,  /* non-finite or non-positive density after floors */
  TDE_ETIMEOUT = 6   /* a bounded device wait expired */
} tde_status;

enum { TDE_EOS_IDEAL = 0, TDE_EOS_TABLE = 1 };
enum { TDE_RECON_PLM = 0, TDE_RECON_PPM = 1 };
enum { TDE_BC_OUTFLOW = 0, TDE_BC_PERIODIC = 1 };
enum { TDE_INVERT_BISECT = 0, TDE_INVERT_SURROGATE = 1, TDE_INVERT_BISECT_PLAIN = 2 };

typedef struct tde_ctx tde_ctx;
typedef struct tde_eos tde_eos;
typedef struct tde_mesh tde_mesh;

/* Scheme and physics parameters (Table 1 of the paper lists the production
 * values: RK2, PLM, CFL, floors, eta_1 = 1e-3, eta_2 = 1e-4). */
typedef struct {
  int eos;              /* TDE_EOS_IDEAL or TDE_EOS_TABLE (Sec. 4) */
  int recon;            /* TDE_RECON_PLM (ng >= 2) or TDE_RECON_PPM (ng >= 3) */
  int dual;             /* 1: evolve the auxiliary internal energy U_aux (Sec. 6) */
  double gamma;         /* ideal-gas adiabatic index (TDE_EOS_IDEAL) */
  double eta1, eta2;    /* Eq. dual-primitive-switch and Eq. dual-sync thresholds */
  double rho_floor, p_floor, u_floor;  /* floors; u_floor = internal energy density of the floor state */
  double unit_rho, unit_e;             /* code -> cgs factors applied before table lookups */
  int eos_mode;         /* TDE_EOS_TABLE: how the cons -> prim closure inverts the table,
                           TDE_INVERT_BISECT (default), TDE_INVERT_BISECT_PLAIN or
                           TDE_INVERT_SURROGATE (needs a trained network on the tde_eos when a
                           stage runs; the learned guess runs as separate launches over the
                           stage's cells).  All three give identical results. */
  int riemann;          /* TDE_RIEMANN_HLLC (default) or TDE_RIEMANN_HLLE (the solver of the
                           paper's production runs, Table 1) */
} tde_params;

enum { TDE_RIEMANN_HLLC = 0, TDE_RIEMANN_HLLE = 1 };

/* Softened point-mass potential on the trajectory
 * r_bh(t) = x0 + v0 (t - t0) + a0 (t - t0)^2 / 2 (Eq. bh-softened-gravity, Sec. 3.1),
 * and the moving frame: with frame_on, the uniform inertial acceleration -afr
 * acts on the gas (Eq. frame-momentum: -rho afr on the momentum, -(rho v).afr on
 * the energy, from each stage's input state); in the frame that follows the
 * star the point mass then moves with acceleration a0 = -afr (Sec. 3.1). */
typedef struct {
  int on;               /* gravity source terms on */
  int excise;           /* one-way sink of radius r_exc */
  double GM, r_soft, r_exc;
  double t0, x0[3], v0[3], a0[3];
  int frame_on;         /* inertial source of the accelerating frame on */
  double afr[3];        /* frame acceleration A_fr, held over the step */
} tde_bh_state;

/* One MeshBlock: index of its first interior cell on its level's grid, its
 * size, and its refinement level (static refinement, Sec. 7.1: a level-L block
 * has cells of width dx / 2^L in every active direction and counts cells on the
 * level-L grid of N[a] 2^L cells). */
typedef struct {
  int i0, j0, k0, nx, ny, nz;
  int level;            /* 0 = the grid's own cells */
} tde_block_desc;

/* The level-0 global grid covered by the MeshBlocks. */
typedef struct {
  int N[3];             /* level-0 cells per direction (1 = inactive direction) */
  double xmin[3];       /* lower domain corner */
  double dx[3];         /* level-0 cell widths */
  int bc[3];            /* TDE_BC_OUTFLOW / TDE_BC_PERIODIC per direction */
  int ng;               /* ghost width */
} tde_grid_desc;

/* Device-side event counters (cumulative until reset). */
typedef struct {
  uint64_t rho_floor, p_floor, u_floor, table_clamp, excised, dual_aux_used, synced, nonfinite;
  uint64_t surrogate_accepted;   /* table inversions settled by the learned guess's Newton step */
} tde_counts;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
TDE_API int tde_init(tde_ctx **out, int device, void *cuda_stream);
TDE_API int tde_set_stream(tde_ctx *ctx, void *cuda_stream);
/* One-line description of the last error on this context ("" if none). */
TDE_API const char *tde_last_error(const tde_ctx *ctx);
TDE_API int tde_finalize(tde_ctx *ctx);

/* ---- equation of state (Sec. 4.2) --------------------------------------- */

/* Load a tabulated EOS sampled on a uniform grid in (log10 rho, log10 T)
 * (Eq. eos-table-range: the paper's table is 640 x 640 on ln rho, ln T; any
 * n_rho, n_T >= 2 is accepted).  Host arrays [n_rho][n_T] (T fastest) of
 * log10 e_th (erg/g), log10 P (dyn/cm^2) and log10 c_s^2 (cm^2/s^2) are COPIED
 * to the device; the caller keeps ownership.  The runtime map (rho, U_EOS) ->
 * (T, P, c_s) interpolates bilinearly in the table (Sec. 4.2, last paragraph).
 * TDE_EINVAL if a log10 e column is not strictly increasing in T (the
 * inversion needs it) or a value is not finite. */
TDE_API int tde_eos_load_table(tde_ctx *ctx, int n_rho, int n_T, double log10_rho_min,
                       double log10_rho_max, double log10_T_min, double log10_T_max,
                       const double *log10_e, const double *log10_P, const double *log10_cs2,
                       tde_eos **out);
TDE_API int tde_eos_destroy(tde_eos *eos);

/* Invert n cells (rho, e) -> (T, P, cs2), all cgs, device arrays of n doubles.
 * mode TDE_INVERT_BISECT: binary search of the interpolated log10 e column,
 * carried out in FP32 on a rounded copy of the table and confirmed by the FP64
 * bracket of the cell (FP64 bisection where FP32 cannot decide);
 * TDE_INVERT_BISECT_PLAIN: the same search entirely in FP64 (the plain form of
 * Sec. 4.2's runtime map).  Both give identical results.  T, P or cs2 may be NULL.  Inputs outside the table are clamped to its edge and
 * counted (counts may be NULL; reading it synchronises the stream). */
TDE_API int tde_eos_invert(tde_eos *eos, int mode, int64_t n, const double *rho, const double *e,
                   double *T, double *P, double *cs2, tde_counts *counts);
/* ---- learned EOS guess (a project addition; the paper has none) -------------
 * A 2 -> 64 -> 64 -> 2 SiLU network maps normalised (log10 rho, z) to
 * normalised (log10 T, log10 P), where z = (log10 e - g_lo) / (g_hi - g_lo) is
 * the position of log10 e inside the table's interpolated log10 e column at
 * that density (0 at T_min, 1 at T_max); normalisation x_n = (x - c) / s with
 * c, s the centre and half-width of the log10 rho, z (0.5, 0.5), log10 T and
 * log10 P ranges (tde_eos_surrogate_norm).  Parameters, 4482 floats:
 *   W1[64][2], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
 * TDE_INVERT_SURROGATE uses the network (BF16 weights; the 64 x 64 layer on the
 * tensor cores, FP32 accumulation) to guess log10 T, takes one FP64 Newton step
 * on the interpolated log10 e column (linear inside a cell) from the guess's
 * cell, and accepts the cell the step lands in iff the table brackets the root
 * there -- then the result equals bisection's exactly.  The cells it does not
 * settle are gathered (warp-aggregated queue) and inverted by bisection in a
 * second launch.  The results of all modes are identical; only the work
 * differs. */
typedef struct {
  double loss_first, loss_last;   /* mean-squared error of the first and last batch */
  int epochs, samples, batches;
  double ms;                      /* device time of the training */
} tde_train_report;

/* Draw n_samples points (log10 rho, log10 T) uniformly over the table with a
 * counter-based generator seeded by seed, map them through the table to inputs
 * (log10 rho, log10 e) and targets (log10 T, log10 P), and train with Adam
 * (learning rate lr with cosine decay, batch size batch) for the given epochs,
 * from a seeded initialisation if the network has no weights yet.  rep may be
 * NULL.  Synchronises the stream. */
TDE_API int tde_eos_surrogate_train(tde_eos *eos, uint64_t seed, int n_samples, int epochs, int batch,
                                    double lr, tde_train_report *rep);
/* Forget the weights: the next tde_eos_surrogate_train starts from its seeded
 * initialisation. */
TDE_API int tde_eos_surrogate_reset(tde_eos *eos);
/* FP32 master weights in / out (host, n = 4482). */
TDE_API int tde_eos_surrogate_set_weights(tde_eos *eos, const float *w, size_t n);
TDE_API int tde_eos_surrogate_get_weights(tde_eos *eos, float *w, size_t n);
/* Loss L = (1/n) sum (y - target)^2 and its gradient (device: x, target [n][2],
 * grad [4482], loss [1]) with the BF16-rounded weights, FP32 arithmetic: the
 * training kernels' own forward and backward pass. */
TDE_API int tde_eos_surrogate_grad(tde_eos *eos, int64_t n, const float *x, const float *target,
                                   float *grad, float *loss);
/* Network outputs y [n][2] for inputs x [n][2] (device, normalised) through the
 * tensor-core inference kernel. */
TDE_API int tde_eos_surrogate_forward(tde_eos *eos, int64_t n, const float *x, float *y);
/* The eight normalisation constants (c, s for log10 rho, e, T, P), host. */
TDE_API int tde_eos_surrogate_norm(const tde_eos *eos, double *out8);

/* Forward evaluation at (rho, T), cgs, device arrays; outputs may be NULL. */
TDE_API int tde_eos_eval_rhoT(tde_eos *eos, int64_t n, const double *rho, const double *T, double *P,
                      double *e, double *cs2);

/* ---- mesh (MeshBlocks with ghost zones: Sec. 2, Sec. 3.2) ---------------- */

/* Build a mesh of nblocks MeshBlocks (host array) covering `grid` exactly once,
 * with the ghost map (periodic wrap / zero-gradient outflow; see tde_ghost_fill
 * for refined meshes).  eos may be NULL for TDE_EOS_IDEAL.  TDE_EINVAL for
 * overlaps, gaps, ng below the reconstruction's stencil (PLM 2, PPM 3), more
 * than 2^31 padded cells, a block edge above 32 cells, and on refined meshes
 * (some level > 0): levels above 8, blocks of level >= 1 whose first index or
 * size is not a multiple of 4 in an active direction, neighbours (face, edge or
 * corner, periodic images included) more than one level apart, or a ghost
 * stencil reaching a cell two levels coarser. */
TDE_API int tde_mesh_create(tde_ctx *ctx, int nblocks, const tde_block_desc *blocks,
                    const tde_grid_desc *grid, const tde_params *params, tde_eos *eos,
                    tde_mesh **out);
TDE_API int tde_mesh_destroy(tde_mesh *mesh);
/* ntot (padded cells of all blocks), nvar, and optionally the nblocks + 1 block
 * offsets (host array; may be NULL). */
TDE_API int tde_mesh_info(const tde_mesh *mesh, int64_t *ntot, int *nvar, int64_t *block_offsets);
/* Replace the scheme parameters (same eos kind and dual flag). */
TDE_API int tde_mesh_set_params(tde_mesh *mesh, const tde_params *params);

/* Bind the caller-owned device states: U (the evolved state) and U1 (the
 * intermediate Runge-Kutta state), nvar * ntot doubles each. */
TDE_API int tde_mesh_bind_state(tde_mesh *mesh, double *U, double *U1);

/* Primitive fields W (device, 5 * ntot: rho, vx, vy, vz, P) -> conserved state U
 * on the interior cells (U_aux = the thermal energy density).  The tabulated
 * EOS finds T from (rho, P) by bisection of the interpolated pressure. */
TDE_API int tde_prim_to_cons(tde_mesh *mesh, const double *W, double *U);

/* Fill the ghost cells of the first nvar fields of a state (a1) from the
 * neighbours' interior cells after the boundary map: a cell of the same level
 * is copied; a region covered by finer cells is their volume average
 * (restriction, conserved variables); a cell inside a coarser block is
 * prolonged: the parent plus, per active direction, a quarter of the minmod of
 * the parent's one-sided differences to its neighbours (each a copied or
 * restricted coarse value), signed toward the child's half. */
TDE_API int tde_ghost_fill(tde_mesh *mesh, double *state, int nvar);

/* One stage of the SSP-RK2 update (a1-a6 of the hydro stage) on nblk blocks:
 *   stage 0:  U1 = U + dt L(U)
 *   stage 1:  U  = (U_start + U1 + dt L(U1)) / 2   (U holds U_start on entry)
 * L is the finite-volume operator of Eqs. frame-momentum and frame-energy with
 * PLM/PPM reconstruction, the HLLC solver, the dual-energy flux and compression
 * (Eqs. dual-flux .. dual-tabulated-compression) and the point-mass source
 * (Eqs. lat-grav-momentum, lat-grav-energy) at the stage time (t_n, then
 * t_n + dt).  Ghost cells of the stage input are refreshed inside the call.
 * block_ids: device int32[nblk], or NULL for all blocks in order (nblk ignored).
 * dt_block, t_block: device double arrays indexed by block id (per-block step
 * and step start time, as LAT needs).  bh: host struct, may be NULL (no gravity). */
TDE_API int tde_hydro_stage(tde_mesh *mesh, int stage, int nblk, const int32_t *block_ids,
                    const double *dt_block, const double *t_block, const tde_bh_state *bh);
/* (On a refined mesh a single stage cannot apply the coarse-fine flux
 * correction, which spans both stages: TDE_EINVAL; use tde_step or LAT windows.) */

/* Per-block CFL step (a7, Sec. 7.1 "local CFL limit from hydrodynamic and source
 * terms"): dt_b = cfl * min over interior cells outside the excision sphere of
 * min_d dx_d / (|v_d| + c_s) and sqrt(dx_min / |g_bh|).  t_block (device, may be
 * NULL = 0) gives the BH time per block.  dt_block: device out [nblocks];
 * dt_min: device out [1] (may be NULL), the minimum over blocks (Eq. lat-base-dt). */
TDE_API int tde_compute_dt(tde_mesh *mesh, double cfl, const double *t_block, const tde_bh_state *bh,
                   double *dt_block, double *dt_min);

/* Excision reset (a8, Sec. 3.1): interior cells with |r - r_bh(t_end_b)| < r_exc
 * of the listed blocks become rho_floor, zero momentum, U = u_floor. */
TDE_API int tde_excise(tde_mesh *mesh, int nblk, const int32_t *block_ids, const double *t_end_block,
               const tde_bh_state *bh);

/* Dual-energy resynchronisation (a8, Eq. dual-sync): refreshes the E ghosts of
 * U, then U_aux <- U_cons where U_cons > 0 and U_cons > eta2 * max of E_tot
 * over the 3x3x3 neighbourhood.  eta2 < 0 uses the mesh parameter. */
TDE_API int tde_dual_energy_sync(tde_mesh *mesh, int nblk, const int32_t *block_ids, double eta2);

/* The mesh keeps its simulation time t in device memory (0 after creation).
 * tde_step advances it by the step's dt without a host round trip. */
TDE_API int tde_mesh_set_time(tde_mesh *mesh, double t);
TDE_API int tde_mesh_get_time(tde_mesh *mesh, double *t);   /* synchronises the stream */

/* One synchronised SSP-RK2 step of every block from the mesh time t: dt from the
 * CFL condition if cfl > 0 (else dt_fixed), stage 0, stage 1, excision (at
 * t + dt), resync if dual energy is on; then t += dt.  The step's dt is also
 * written to dt_out (device double, may be NULL).  On a refined mesh the step
 * is a LAT window with every factor 1 (the coarse-fine flux correction of
 * Eq. lat-flux-impulse at its end), and it leaves those factors assigned. */
TDE_API int tde_step(tde_mesh *mesh, double cfl, double dt_fixed, const tde_bh_state *bh, double *dt_out);

/* ---- localized adaptive time stepping (Sec. 7 of the paper) -------------- */

/* Per-block factors for the next window (Eq. lat-base-dt, Eq. lat-factor): the
 * CFL step of every block from U at the mesh time (as tde_compute_dt), dt0 =
 * min, f_b = 2^min(n_lat, floor(log2(dt_b / dt0))), top bins holding fewer than
 * merge_frac * nblocks blocks merged into the next smaller bin, then factors
 * lowered until blocks sharing a face, edge or corner differ by at most 2x.
 * Outputs (host, each may be NULL): factors[nblocks], f_max, dt0.  Synchronises
 * the stream (the schedule is built on the host).  TDE_ETIMEOUT if the bounded
 * limiting passes did not converge. */
TDE_API int tde_lat_assign(tde_mesh *mesh, int n_lat, double merge_frac, double cfl,
                           const tde_bh_state *bh, int32_t *factors, int *f_max, double *dt0);
/* Impose factors (host, powers of two) and dt0 instead of tde_lat_assign. */
TDE_API int tde_lat_set_factors(tde_mesh *mesh, const int32_t *factors, double dt0);
/* One LAT window of f_max * dt0 from the mesh time (Sec. 7.1): at each fine
 * sub-step tau the blocks of every factor f dividing tau advance one RK2 step of
 * f dt0 in one batched launch sequence per level, slow levels first; ghost
 * cells from a neighbour on another schedule are its frozen state (faster
 * neighbour) or a linear interpolation in time between its stored endpoint
 * states (slower neighbour); when a block completes, its faces shared with
 * faster neighbours take the neighbours' time-integrated fluxes
 * (Eq. lat-flux-impulse) with the gravitational work correction of
 * Eq. lat-grav-reflux, then excision and resync run for it.  All factors 1 is
 * the synchronised step.  use_graph = 1 captures the window's launches in a CUDA
 * graph on first use and replays it while factors, bh, states and parameters are
 * unchanged.  *block_updates (host, may be NULL) = MeshBlock steps taken. */
TDE_API int tde_lat_window(tde_mesh *mesh, const tde_bh_state *bh, int use_graph,
                           int64_t *block_updates);

/* How tde_lat_window runs one level sub-step (Sec. 7.1; the same results bit for
 * bit in both modes).  TDE_LAT_SEQUENCE (the default): a sequence of batched
 * launches over the level's blocks (save the start states; per RK stage the
 * conserved ghosts from other schedules, the conversion to primitives, the
 * primitive ghosts from the same schedule, the x, y, z sweeps).
 * TDE_LAT_PERSISTENT: the same phases inside one cooperative launch whose CTAs
 * stay resident and meet at grid barriers in device memory; a barrier wait is
 * limited to one second of the global timer, after which the launch ends and
 * tde_mesh_check reports TDE_ETIMEOUT.  It applies to 3-D meshes without
 * refined-mesh ghost operations whose closure is not the learned guess; other
 * meshes keep the sequence.  *active (host, may be NULL) = 1 if the mesh's
 * current scheme takes the persistent form.  A captured window is discarded on
 * a change of mode.  TDE_EINVAL for an unknown mode. */
enum { TDE_LAT_SEQUENCE = 0, TDE_LAT_PERSISTENT = 1 };
TDE_API int tde_mesh_set_lat_mode(tde_mesh *mesh, int mode, int *active);

/* Copy the cumulative device counters to *out (synchronises the stream) and
 * optionally reset them. */
TDE_API int tde_counts_read(tde_mesh *mesh, tde_counts *out, int reset);

/* Health of the asynchronous work so far (synchronises the stream; changes no
 * state but the expiry flag).  tde_mesh_check: TDE_ENUMERIC if a kernel counted a
 * non-finite value or a non-positive density after the floors since the counters
 * were last reset, else the result of tde_eos_check on the mesh's EOS.
 * tde_eos_check: TDE_ETIMEOUT if a bounded device wait of the learned-guess
 * inference expired since the last check (the cells of its tiles then took the
 * bisection fallback, so the results stand), clearing the flag; else TDE_OK.
 * tde_last_error() names the count or the wait. */
TDE_API int tde_mesh_check(tde_mesh *mesh);
TDE_API int tde_eos_check(tde_eos *eos);
/* Failure-detection test hook: with on != 0 the learned-guess inference issues
 * no tensor-core work, so that its bounded wait for the results expires and
 * takes the timeout path (about two seconds per launch: one-second limits on the
 * wait for the results and on the wait for work in flight); results stay those
 * of bisection.  on = 0 restores normal operation. */
TDE_API int tde_eos_inject_wait_expiry(tde_eos *eos, int on);
/* Failure-detection test hook of the mesh: with on != 0 the sweeps arm their
 * TMA completion barrier but issue no copy, so every sweep tile's bounded wait
 * (one second of the global timer, then one more for copies in flight) expires:
 * the tile is skipped, the state it would have written is left as it was (so
 * the step's result is not the method's), and tde_mesh_check reports
 * TDE_ETIMEOUT once.  on = 0 restores normal operation.  TDE_EINVAL for a mesh
 * whose sweeps stage without TMA (a padded block row that is not a whole number
 * of 16-byte units). */
TDE_API int tde_mesh_inject_wait_expiry(tde_mesh *mesh, int on);
/* Failure-detection test hook of the persistent level launch: with on != 0 its
 * CTA 0 does not arrive at the first grid barrier, so every CTA's bounded wait
 * there expires after one second and the launch ends without doing the level's
 * work; tde_mesh_check then reports TDE_ETIMEOUT once.  on = 0 restores normal
 * operation.  Discards a captured window. */
TDE_API int tde_mesh_inject_barrier_drop(tde_mesh *mesh, int on);

/* ---- allocation-free variant ---------------------------------------------- */

/* A tabulated EOS held in device arrays that the caller owns (same layout and
 * meaning as the host arrays of tde_eos_load_table).  The call checks that the
 * three pointers are non-null, n_rho, n_T >= 2 and both ranges increase
 * (TDE_EINVAL otherwise); the table's values are not validated. */
typedef struct {
  int n_rho, n_T;
  double log10_rho_min, log10_rho_max, log10_T_min, log10_T_max;
  const double *log10_e, *log10_P, *log10_cs2;   /* device, [n_rho][n_T] */
} tde_table_view;

/* The per-MeshBlock CFL step of tde_compute_dt, for callers that may not
 * allocate device memory: programs whose device memory is owned by another
 * allocator (a framework that reserves the whole device in its own pool at
 * start-up) or loops that forbid allocation after initialisation.  Such callers
 * cannot create a tde_mesh, so this call takes the block list (host), the grid
 * and scheme (host), the state U (device, the layout of tde.h for these blocks)
 * and, for TDE_EOS_TABLE, a table view; it writes dt_block (device, nblocks)
 * and/or dt_min (device, 1).  The paper has no counterpart: this is a library
 * service.  It calls no cudaMalloc, cudaFree or other allocating routine; its
 * scratch (block list copy, offsets, per-block minima) is one fixed device
 * array of about 176 KB that every GPU loading the library holds until exit,
 * beside a constant 4.6 KB array of the log10 / exp10 tables that the mesh's
 * EOS lookups use, so dt equals tde_compute_dt's bit for bit.
 * Limit: 1 <= nblocks <= 4096, else TDE_EINVAL; each block is checked as by
 * tde_mesh_create (edges of 1..32 cells, one cell across an inactive direction,
 * inside its level's grid).  The first call on a device looks up the arrays'
 * device addresses and copies the tables into the second (a synchronous copy).
 * All calls share the scratch array: calls whose
 * GPU work overlaps race.  The block list is read from host memory during the
 * call.  Uses ctx's stream; asynchronous. */
TDE_API int tde_compute_dt_noalloc(tde_ctx *ctx, int nblocks, const tde_block_desc *blocks,
                                   const tde_grid_desc *grid, const tde_params *params,
                                   const tde_table_view *table, const double *U, double cfl,
                                   const double *t_block, const tde_bh_state *bh,
                                   double *dt_block, double *dt_min);

/* ---- measurement ---------------------------------------------------------- */

/* Kernel classes counted and (optionally) timed by the context. */
enum {
  TDE_K_C2P = 0,      /* conserved -> primitive (+ CFL minimum) */
  TDE_K_DT = 1,       /* per-block dt finalisation */
  TDE_K_GHOST = 2,    /* ghost-layer gather */
  TDE_K_SWEEP_X = 3,  /* reconstruction + HLLC + divergence along x */
  TDE_K_SWEEP_Y = 4,
  TDE_K_SWEEP_Z = 5,  /* ... along z, with the final update of the stage */
  TDE_K_SYNC = 6,     /* dual-energy resync */
  TDE_K_EXCISE = 7,
  TDE_K_SCALAR = 8,   /* device scalar bookkeeping (time, dt) */
  TDE_K_P2C = 9,      /* primitive -> conserved */
  TDE_K_EOS = 10,     /* batch EOS inversion / evaluation */
  TDE_K_PROBE = 11,   /* peak-rate probe */
  TDE_K_LATGRAPH = 12, /* replayed LAT window graphs (launches counted per kernel inside) */
  TDE_K_GRAV = 13,    /* self-gravity multigrid */
  TDE_K_REMAP = 14,   /* domain remap (the staging pass counts as scalar) */
  TDE_K_LATLEVEL = 15, /* persistent LAT level sub-steps */
  TDE_K_NKIND = 16
};

/* Every kernel the context launches is counted per class.  With timing on, a
 * CUDA event pair on the context's stream brackets each launch and
 * tde_profile_read() accumulates the elapsed times.  enable: 1 on, 0 off;
 * both reset the counters. */
TDE_API int tde_profile(tde_ctx *ctx, int enable);
/* Per-class launch counts and summed device milliseconds since the last reset
 * (arrays of TDE_K_NKIND entries, either may be NULL).  Synchronises the stream. */
TDE_API int tde_profile_read(tde_ctx *ctx, uint64_t *launches, double *ms);

/* The table-driven log10 and exp10 that the EOS kernels use (device arrays of
 * n doubles; either output may be NULL), for checking them against the CUDA
 * math library.  Uses eos's tables; asynchronous. */
TDE_API int tde_math_selftest(tde_eos *eos, int64_t n, const double *x, double *log10_out,
                              double *exp10_out);

/* ---- sweep tile shapes and their autotuner (a9) -----------------------------
 * A sweep CTA works on a tile of pencils of one block along the sweep direction.
 * Shapes (index: lanes per tile, threads per CTA): 0: 8 x 288 (default), 1: 16 x
 * 288, 2: 4 x 160; a shape whose tile needs more than 226 KB of shared memory for
 * the mesh's block size is not available.  Results do not depend on the shape
 * (every face and cell is computed by the same operations); only the time does.
 *
 * tde_mesh_autotune times every available shape per active direction over all
 * blocks of the bound state (reps timed launches after one warm-up, CUDA events)
 * and keeps the fastest; bh (may be NULL) is the point mass the timing includes.
 * It reads the state and writes only scratch memory: state, counters and time are
 * unchanged.  tiles (may be NULL) receives the chosen shape per direction x, y, z;
 * ms (may be NULL) receives [3][3] mean launch times (-1 where a shape was not
 * run).  Synchronises the stream.  tde_mesh_set_tiles forces shapes (TDE_EINVAL
 * for an unknown or too large shape); tde_mesh_get_tiles reads them. */
TDE_API int tde_mesh_autotune(tde_mesh *mesh, const tde_bh_state *bh, int reps, int32_t *tiles,
                              float *ms);
TDE_API int tde_mesh_set_tiles(tde_mesh *mesh, const int32_t *tiles);
TDE_API int tde_mesh_get_tiles(const tde_mesh *mesh, int32_t *tiles);

/* ---- moving frame (Sec. 3.1) ---------------------------------------------
 * tde_frame_acceleration: Eq. frame-acceleration at the mesh time, the
 * mass-weighted acceleration -grad Phi_bh of the point mass bh over the interior
 * gas with rho > rho_min outside the excision sphere (bh->excise); A[3] and the
 * gas mass it averaged over (mass = 0: A = 0).  Deterministic (fixed-order
 * reduction).  Synchronises the stream.
 * tde_mesh_boost: Galilean boost of Eq. galilean-boost by V[3] of the interior
 * cells with rho > rho_min: (rho v)' = rho (v + V), E' = E + rho v.V + rho |V|^2/2;
 * floor-density cells and U_aux are left as they are.  Asynchronous. */
TDE_API int tde_frame_acceleration(tde_mesh *mesh, const tde_bh_state *bh, double rho_min,
                                   double *A, double *mass);
TDE_API int tde_mesh_boost(tde_mesh *mesh, const double *V, double rho_min);

/* ---- self-gravity (Sec. 3.2) -----------------------------------------------
 * Geometric multigrid for A_h phi = S_h, A_h = -lap_h (seven-point, weights
 * (dx/dy)^2 and (dx/dz)^2, Eq. selfgrav-poisson), S_h = -4 pi G rho_sg with
 * rho_sg = rho where rho > rho_min (floor gas excluded), on the mesh's uniform
 * grid (each active N a power of two).  Boundaries: TDE_GRAV_PERIODIC (every
 * active direction of the mesh periodic; the mean of S removed in two passes)
 * or TDE_GRAV_ISOLATED (the paper's multipole boundary conditions: phi on every
 * boundary face is the exterior multipole expansion of S to order lmax <= 4
 * about its S-weighted centroid, a Dirichlet condition at the face on every
 * level).  V-cycles of npre / npost red-black Gauss-Seidel sweeps with
 * over-relaxation omega (the paper: 2, 2, 1.15), a full-approximation coarse
 * correction, tricubic prolongation, post-smoothing on every level and one
 * extra fine sweep, until the rms defect (Eq. selfgrav-defect) is below tol or
 * max_cycles are done.  The start: fmg = 1 full multigrid (the paper's start for
 * a first or remapped solve: the source on every level, the coarsest solved,
 * then per finer level the prolonged solution and one V-cycle), else warm = 1
 * the previous potential, else zero. */
enum { TDE_GRAV_PERIODIC = 0, TDE_GRAV_ISOLATED = 1 };
typedef struct {
  double G;            /* gravitational constant in code units (1 / (4 pi) for Table 1's) */
  double rho_min;      /* density above which gas is a source */
  double tol;          /* rms defect to reach */
  int max_cycles, npre, npost;
  double omega;        /* over-relaxation of the Gauss-Seidel sweeps */
  int warm;            /* start from the previous potential */
  int boundary;        /* TDE_GRAV_PERIODIC or TDE_GRAV_ISOLATED */
  int lmax;            /* isolated: multipole order 0..4 */
  int fmg;             /* start with full multigrid */
} tde_grav_params;
/* Solve for phi_sg from the bound state's density; the potential is kept by the
 * mesh (also in the MeshBlock layout, ghosts included: periodic images, or
 * beyond an isolated boundary the expansion at the ghost centre).  cycles and
 * defect (may be NULL) receive the V-cycles run after the start and the final
 * rms defect.  TDE_EINVAL for an active size that is not a power of two, a
 * periodic solve on a mesh with a non-periodic active direction, lmax outside
 * 0..4 or a refined mesh.  Synchronises. */
TDE_API int tde_gravity_solve(tde_mesh *mesh, const tde_grav_params *params, int *cycles,
                              double *defect);
/* on = 1: the hydro stage adds the kept phi_sg (frozen between solves) to the
 * point mass's potential in its gravity sources (Eqs. lat-grav-momentum,
 * lat-grav-energy, and the refluxing of Eq. lat-grav-reflux). */
TDE_API int tde_gravity_enable(tde_mesh *mesh, int on);
/* The potential on the global grid, [Nz][Ny][Nx] doubles into device memory
 * phi (TDE_EINVAL before the first solve).  Asynchronous. */
TDE_API int tde_gravity_phi(tde_mesh *mesh, double *phi);

/* ---- domain remap (Sec. 5.2) ---------------------------------------------
 * Eqs. remap-state-vector and remap-cell-average: every interior cell of dst
 * becomes the mean of 2^(active directions of dst) midpoint samples (two per
 * active direction, at the centres of the cell's halves), each a trilinear
 * interpolation of src's cell-centred rho, m and thermal energy density U (src's
 * U_aux if it evolves one, else E - |m|^2 / (2 rho)); dst's E is rebuilt as
 * U + |m|^2 / (2 rho) (TDE_REMAP_THERMAL, the paper's form) or E itself is
 * interpolated (TDE_REMAP_TOTAL, the form it compares against); a dual dst gets
 * U_aux = U.  A dst cell coincident with a src cell (same width, centre within
 * 1e-9 cells) is copied, so a remap onto the same grid is the identity.
 * Samples outside src's domain in a non-periodic direction count as the floor
 * state at rest (rho_floor, zero momentum, thermal energy density u_floor);
 * lookups past src's last cells follow its boundary map (periodic wrap, outflow
 * copy of the edge cell).
 * Usrc: device, src's nvar * ntot layout (ghost cells not read); Udst: device,
 * dst's layout, interior cells written (fill its ghosts with tde_ghost_fill);
 * distinct buffers.  Both meshes on one context.  The excision reset of the new
 * domain is the caller's (tde_excise).  TDE_EINVAL on a bad mode, NULL or shared
 * buffers, or meshes of different contexts.  Asynchronous on the context's
 * stream. */
enum { TDE_REMAP_THERMAL = 0, TDE_REMAP_TOTAL = 1 };
TDE_API int tde_mesh_remap(tde_mesh *dst, double *Udst, const tde_mesh *src, const double *Usrc, int mode,
                           double rho_floor, double u_floor);

/* The reciprocal and square-root building blocks of the hydro kernels, on n
 * device doubles: TDE_MATH_RCP out = 1/x (refined hardware seed, within one
 * ulp), TDE_MATH_SQRT_RATIO out = sqrt(x / y) (within about two ulps; x y and
 * x / y normal), TDE_MATH_RCP_SEED and TDE_MATH_RSQRT_SEED the raw hardware
 * approximations of 1/x and 1/sqrt(x) that the two refine, TDE_MATH_RSQRT
 * out = 1/sqrt(x) (refined seed, within about two ulps; the point-mass
 * potential), TDE_MATH_INSIDE out = 1 if sqrt(x) < y else 0 (the excision test,
 * decided as with the correctly rounded square root, x >= 0).  y is read only by
 * TDE_MATH_SQRT_RATIO and TDE_MATH_INSIDE.  TDE_EINVAL for an unknown op or null
 * arrays with n > 0; asynchronous on the context's stream. */
enum {
  TDE_MATH_RCP = 0,
  TDE_MATH_SQRT_RATIO = 1,
  TDE_MATH_RCP_SEED = 2,
  TDE_MATH_RSQRT_SEED = 3,
  TDE_MATH_RSQRT = 4,
  TDE_MATH_INSIDE = 5
};
TDE_API int tde_math_probe(tde_ctx *ctx, int op, int64_t n, const double *x, const double *y,
                           double *out);

/* The Riemann solvers of the sweeps (a5, Sec. 2.1) on n face-state pairs, for a
 * unit check against an independent implementation: solver TDE_RIEMANN_HLLC or
 * TDE_RIEMANN_HLLE across a face normal to direction d (0, 1, 2).  wl, wr: device
 * arrays [n][8] of the left and right face states (rho, vx, vy, vz, P, Gamma_e,
 * Gamma_1, U_aux); with eos_table = 0 the two Gammas are ignored and gamma is
 * used, with dual = 0 U_aux is ignored.  F: device [n][6], the mass, momentum (x, y,
 * z), energy and U_aux fluxes (U_aux flux 0 unless dual); vf: device [n], the face
 * velocity of Eq. dual-face-velocity (0 unless dual).  TDE_EINVAL for a bad solver,
 * direction or gamma, or null arrays with n > 0; asynchronous on the context's stream. */
TDE_API int tde_riemann_probe(tde_ctx *ctx, int solver, int d, int eos_table, int dual, double gamma,
                              int64_t n, const double *wl, const double *wr, double *F, double *vf);

/* Measured FP64 fused multiply-add throughput of the device (FLOP/s, an FMA
 * counted as 2), from a kernel of independent FMA chains on every SM.  The
 * hydro stage is bound by this rate on sm_103a.  Synchronises the stream. */
TDE_API int tde_probe_fp64(tde_ctx *ctx, double *flops);

#ifdef __cplusplus
}
#endif
#endif
