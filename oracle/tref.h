/*
 * tref.h -- the ORACLE: a plain, slow, serial-per-block CPU reference of the
 * per-MeshBlock finite-volume hydro stage of "An End-to-End Numerical
 * Framework for Tidal Disruption Events with AthenaK" (arxiv 2609.37859).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library (include/tde.h) and the CUDA library
 * never calls it.
 *
 * Everything is IEEE double precision, compiled with -ffp-contract=off so that
 * every operation is rounded exactly as written.  Each function names the
 * passage of the paper it follows; where the paper is silent the reading that
 * is implemented is stated at the function.
 *
 * Parity status: every function in this file is pinned by a CPU test
 * (tests/test_oracle_*.py) against something other than itself (a closed
 * form, an exact Riemann solution, an invariant or brute force), except the
 * PPM reconstruction, whose absolute accuracy is pinned only by its measured
 * convergence order and by conservation.
 *
 * State layout (all hydro calls):  a mesh is a set of MeshBlocks, each a box of
 * nx*ny*nz interior cells padded by ng ghost cells on each side of every
 * active direction (a direction whose global extent is 1 cell is inactive and
 * carries no ghosts and no flux).  A state is one double array
 *     U[v * ntot + off_b + (k * Py + j) * Px + i]
 * with v the conserved variable (rho, m_x, m_y, m_z, E_tot[, U_aux]), ntot the
 * total number of padded cells of all blocks, off_b the first padded cell of
 * block b and (i, j, k) padded indices (interior cells start at ng).
 */
#ifndef TREF_H
#define TREF_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { TREF_EOS_IDEAL = 0, TREF_EOS_TABLE = 1 };
enum { TREF_PLM = 0, TREF_PPM = 1 };
enum { TREF_OUTFLOW = 0, TREF_PERIODIC = 1 };
enum { TREF_RHO = 0, TREF_MX = 1, TREF_MY = 2, TREF_MZ = 3, TREF_EN = 4, TREF_AUX = 5 };

/* Tabulated EOS on a uniform (log10 rho, log10 T) grid (Sec. 4.2).  Arrays are
 * [n_rho][n_T], T fastest, in cgs.  The oracle does not own them. */
typedef struct {
  int n_rho, n_T;
  double lrho_min, lrho_max, lT_min, lT_max;
  const double *log10_e, *log10_P, *log10_cs2;
} tref_table;

/* Physics and scheme parameters (Table 1 lists the production values). */
typedef struct {
  int eos;              /* TREF_EOS_IDEAL or TREF_EOS_TABLE */
  int recon;            /* TREF_PLM or TREF_PPM */
  int dual;             /* dual-energy auxiliary variable on (1) / off (0), Sec. 6 */
  double gamma;         /* ideal-gas adiabatic index */
  double eta1, eta2;    /* dual-energy switch and resync thresholds, Eqs. dual-primitive-switch, dual-sync */
  double rho_floor, p_floor, u_floor;   /* floors (Table 1); u_floor = internal energy density of the floor state */
  double unit_rho, unit_e;              /* code -> cgs factors used for table lookups */
  int bh_on, excision_on;               /* softened moving point mass, one-way sink (Sec. 3.1) */
  double GM, r_soft, r_exc;
  double bh_t0, bh_x0[3], bh_v0[3], bh_a0[3];   /* r_bh(t) = x0 + v0 (t-t0) + a0 (t-t0)^2 / 2 */
  int riemann;                          /* TREF_HLLC (0) or TREF_HLLE (1, the solver of Table 1) */
  int frame_on;                         /* moving frame: inertial source -rho A_fr (Eq. frame-momentum) */
  double afr[3];                        /* the frame acceleration A_fr held over the step */
} tref_params;

enum { TREF_HLLC = 0, TREF_HLLE = 1 };

/* Mesh: a global grid covered by MeshBlocks, optionally with static refinement.
 * A block of level L has cells of width dx / 2^L in every active direction and
 * its indices count level-L cells (the level-L grid has N[a] 2^L cells in an
 * active direction).  Refined meshes (some level > 0) must be 2:1 balanced
 * across faces, edges and corners, and every block of level >= 1 must have its
 * first index and its size multiples of 4 in the active directions (so that
 * the children of a coarser cell, and their children, lie in one block). */
typedef struct {
  int nb;               /* number of MeshBlocks */
  const int *blocks;    /* nb * 6 ints: i0, j0, k0, nx, ny, nz (first interior cell on the block's level grid, size) */
  int N[3];             /* level-0 cells per direction */
  double xmin[3];       /* lower domain corner */
  double dx[3];         /* level-0 cell widths */
  int bc[3];            /* TREF_OUTFLOW or TREF_PERIODIC per direction */
  int ng;               /* ghost width (2 for PLM, 3 for PPM) */
  const int *levels;    /* nb refinement levels, or NULL (all 0) */
} tref_mesh_desc;

/* Event counters (floors applied, table clamps, excised cells). */
typedef struct {
  int64_t rho_floor, p_floor, u_floor, table_clamp, excised, dual_aux_used, synced;
} tref_counts;

typedef struct tref_mesh tref_mesh;

/* ---- EOS (oracle/tref_eos.c) ---------------------------------------------- */

/* Saha H/He mixture with radiation at (rho, T) in cgs.  out[0..8] =
 * P, e (specific internal energy incl. ionisation and radiation), n_e, x_H+,
 * y_He+, y_He2+, mu, P_gas, n_nuc. */
void tref_saha_state(double rho, double T, double X, double Y, double *out);
/* Pure-hydrogen Saha ionised fraction from the closed-form quadratic (pin). */
double tref_saha_pure_h_xe(double rho, double T);
/* Fill the table: log10 e, log10 P, log10 cs^2 and Gamma_1 on the grid. */
void tref_eos_build(int n_rho, int n_T, double lrho_min, double lrho_max, double lT_min,
                    double lT_max, double X, double Y, double *log10_e, double *log10_P,
                    double *log10_cs2, double *gamma1);
/* Bilinear evaluation at (rho, T) (cgs): out P, e, cs2. */
void tref_eos_eval_rhoT(const tref_table *t, double rho, double T, double *P, double *e, double *cs2);
void tref_eos_eval_rhoT_n(const tref_table *t, int64_t n, const double *rho, const double *T, double *P,
                          double *e, double *cs2);
/* Inversion (rho, e) -> (T, P, cs2), cgs.  Returns 1 if clamped to the table edge. */
int tref_eos_invert(const tref_table *t, double rho, double e, double *T, double *P, double *cs2,
                    double *e_used);
/* Inversion from a guessed log10 T: one Newton step in the guessed cell of the
 * interpolated log10 e column, accepted iff the root lies in that cell (then the
 * result equals tref_eos_invert's exactly), else tref_eos_invert.  Returns 1 if
 * accepted. */
int tref_eos_invert_guess(const tref_table *t, double rho, double e, double log10_T_guess,
                          double *T, double *P, double *cs2);
/* Inversion (rho, P) -> T on the pressure column (initial data only). */
double tref_eos_T_from_P(const tref_table *t, double rho, double P);

/* ---- mesh and hydro (oracle/tref_hydro.c) ---------------------------------- */

tref_mesh *tref_mesh_new(const tref_mesh_desc *d, const tref_params *p, const tref_table *t);
void tref_mesh_free(tref_mesh *m);
int64_t tref_mesh_ntot(const tref_mesh *m);            /* padded cells of all blocks */
int64_t tref_mesh_block_offset(const tref_mesh *m, int b);
int tref_nvar(const tref_mesh *m);
int tref_num_threads(void);   /* OpenMP threads of the block loops */
void tref_set_num_threads(int n);
void tref_set_params(tref_mesh *m, const tref_params *p);

/* a1: fill the ghost cells of the listed blocks (all blocks if ids == NULL) from
 * the neighbours' interior cells after the boundary map (periodic wrap or
 * zero-gradient outflow): a cell of the same level is copied, a region covered
 * by finer cells is their volume average (restriction), a cell inside a coarser
 * block is prolonged from the coarser level (the parent plus minmod-limited
 * slopes toward its neighbours, each itself a level value). */
void tref_ghost_fill(const tref_mesh *m, double *U, int nvar, int nact, const int *ids);
/* a1 under LAT: mode[o] of the source block o selects the ghost value:
 * 0 copy from Udst, 1 copy from Ucur, 2 Uold + s_block[o] (Ucur - Uold). */
void tref_ghost_fill_modes(const tref_mesh *m, double *Udst, const double *Ucur, const double *Uold,
                           const int *mode, const double *s_block, int nact, const int *ids);
/* size (doubles) of one block's flux register: 6 sides x nvar x face cells */
int64_t tref_freg_block_size(const tref_mesh *m, int b);

/* a2 + a3: conserved -> primitive for one cell.  w[0..7] = rho, vx, vy, vz, P,
 * Gamma_e (= 1 + P/U), Gamma_1 (= rho cs^2 / P), U_aux. */
void tref_cons_to_prim(const tref_mesh *m, const double *u, double *w, tref_counts *c);

/* One Runge-Kutta stage (a2-a6) on the listed blocks.  stage 0:
 * Uout = U0 + dt L(U0); stage 1: Uout = (U0 + Uin + dt L(Uin)) / 2.  Uin must
 * have filled ghosts.  dt_b[], t_b[] are indexed by block id (t_b = time at the
 * start of the block's step).  If flux_reg != NULL the face fluxes of block
 * boundary faces are accumulated into it (LAT refluxing, a9). */
void tref_stage(const tref_mesh *m, int stage, int nact, const int *ids, const double *U0,
                const double *Uin, double *Uout, const double *dt_b, const double *t_b,
                double *flux_reg, tref_counts *c);
/* a8: excision reset of the listed blocks at time t_b[b] (+ dt_b[b]). */
void tref_excise(const tref_mesh *m, double *U, int nact, const int *ids, const double *t_end_b,
                 tref_counts *c);
/* a8: dual-energy resync (Eq. dual-sync) of the listed blocks; E ghosts must be filled. */
void tref_dual_sync(const tref_mesh *m, double *U, int nact, const int *ids, tref_counts *c);
/* a7: per-block CFL time step from state U at time t_b[b] (no ghosts needed). */
void tref_cfl_dt(const tref_mesh *m, const double *U, double cfl, const double *t_b, double *dt_b,
                 tref_counts *c);
/* Full synchronised RK2 step of every block with one dt (ghost fill, two
 * stages, excision, ghost fill, resync).  Uscr is a second state buffer. */
void tref_step(const tref_mesh *m, double *U, double *Uscr, double dt, double t, tref_counts *c);
/* Primitive (rho, vx, vy, vz, P) per interior cell -> conserved state, U_aux = U. */
void tref_prim_to_cons(const tref_mesh *m, const double *W, double *U);
/* a5 on n face-state pairs: HLLC (solver 0) or HLLE (1) across a face normal to
 * direction d; wl, wr [n][8] = (rho, vx, vy, vz, P, Gamma_e, Gamma_1, U_aux) (an
 * ideal gas has Gamma_e = Gamma_1 = gamma); F [n][6] = mass, momentum, energy and
 * U_aux fluxes (the last 0 unless dual), vf [n] = face velocity. */
void tref_riemann(int solver, int d, int dual, int64_t n, const double *wl, const double *wr, double *F,
                  double *vf);
/* Softened point-mass potential at position x (Eq. bh-softened-gravity). */
double tref_phi_bh(const tref_params *p, const double *x, double t);

/* ---- localized adaptive time stepping (oracle/tref_lat.c) ------------------ */

/* Eq. lat-base-dt, Eq. lat-factor, sparse-bin merging and neighbour limiting.
 * Returns f_max; *dt0 = min_b dt_b. */
int tref_lat_factors(const tref_mesh *m, const double *dt_b, int n_lat, double merge_frac,
                     int32_t *f_b, double *dt0);
/* One LAT window of f_max * dt0 from the synchronised state U at time t (Sec. 7.1).
 * Returns f_max; *block_updates = MeshBlock RK2 steps taken. */
int tref_lat_window(const tref_mesh *m, double *U, const int32_t *f_b, double dt0, double t,
                    tref_counts *c, int64_t *block_updates);

/* ---- learned EOS guess: MLP 2 -> 64 -> 64 -> 2 with SiLU (oracle/tref_mlp.c) */

enum { TREF_MLP_H = 64, TREF_MLP_NPARAM = 2 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2 };
/* y = MLP(x) for n inputs x[n][2] -> y[n][2]. */
void tref_mlp_forward(const double *params, int64_t n, const double *x, double *y);
/* Mean-squared-error loss over n samples and its gradient w.r.t. params. */
double tref_mlp_loss_grad(const double *params, int64_t n, const double *x, const double *target,
                          double *grad);

/* Frame acceleration of Eq. frame-acceleration at time t: the mass-weighted
 * point-mass acceleration g = -grad Phi_bh of the interior gas with rho > rho_min
 * outside the excision sphere; A[3], and the mass it averaged over (0: A = 0). */
void tref_frame_acceleration(const tref_mesh *m, const double *U, double t, double rho_min,
                             double *A, double *mass);
/* Galilean boost of Eq. galilean-boost by V[3] of the interior cells with
 * rho > rho_min (floor-density gas is left as it is). */
void tref_boost(const tref_mesh *m, double *U, const double *V, double rho_min);

/* Self-gravity multigrid (tref_grav.c): solve A_h phi = S_h, A_h = -lap_h with
 * anisotropic weights, on a periodic nx x ny x nz grid (each a power of two) of
 * cell widths dx[3]; src, phi [nz][ny][nx]; phi is the start and the result.
 * V-cycles (npre, npost red-black sweeps, over-relaxation omega) until the rms
 * defect is below tol or max_cycles; returns the cycles, *defect the final rms. */
int tref_mg_solve(int nx, int ny, int nz, const double *dx, const double *src, double *phi,
                  int max_cycles, double tol, int npre, int npost, double omega, double *defect);
double tref_mg_defect_rms(int nx, int ny, int nz, const double *dx, const double *src, const double *phi);
/* Prolongation of the V-cycle on its own (tricubic, cell centred): the coarse
 * field e (nc cells) onto the fine grid (nf, each direction equal to or twice
 * nc); iso = 1 mirrors e about zero beyond the faces, iso = 0 wraps. */
void tref_mg_prolong(const int *nf, const int *nc, int iso, const double *e, double *out);
/* The same on a periodic (isolated = 0) or isolated grid (lower corner xmin):
 * isolated boundary values from the multipole expansion of the source to order
 * lmax (<= 8) about centre (NULL: the source-weighted centroid); fmg = 1 starts
 * with full multigrid instead of phi.  *defect_start (may be NULL) = the rms
 * defect before the V-cycles; phiq[q] = the expansion at the nq points xq[3q..]
 * (isolated only). */
int tref_mg_solve_bc(int nx, int ny, int nz, const double *dx, const double *xmin, int isolated, int lmax,
                     const double *centre, int fmg, const double *src, double *phi, int max_cycles,
                     double tol, int npre, int npost, double omega, double *defect, double *defect_start,
                     int nq, const double *xq, double *phiq);

/* Self-gravity potential of the hydro sources, in the mesh's padded layout
 * (ghosts included; the caller keeps the array), NULL to switch it off.  It is
 * added to the point mass's potential in the stage and in the refluxing. */
void tref_set_phi_sg(tref_mesh *m, const double *phi_padded);
const double *tref_phi_sg(const tref_mesh *m);

const tref_mesh_desc *tref_mesh_get_desc(const tref_mesh *m);
/* padded index of the interior cell at global cell (i, j, k) */
int64_t tref_cell_index(const tref_mesh *m, int i, int j, int k);

/* Conserved-variable remap (Sec. 5.2) of src's state Usrc onto dst's state Udst
 * (interior cells): midpoint-quadrature averages of trilinear interpolants,
 * energy carried as thermal energy (mode TREF_REMAP_THERMAL) or as total energy
 * (TREF_REMAP_TOTAL); coincident cells copied; samples outside the source
 * domain take the floor state (rho_floor, at rest, internal energy u_floor). */
enum { TREF_REMAP_THERMAL = 0, TREF_REMAP_TOTAL = 1 };
void tref_remap(const tref_mesh *dst, double *Udst, const tref_mesh *src, const double *Usrc, int mode,
                double rho_floor, double u_floor);

#ifdef __cplusplus
}
#endif
#endif
