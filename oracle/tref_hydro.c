/*
 * tref_hydro.c -- ORACLE (test infrastructure only): MeshBlocks, ghost zones and
 * one Runge-Kutta stage of the finite-volume hydro update, written as plainly as
 * possible: every padded cell is converted to primitives, every face of every
 * direction is reconstructed and solved, then every interior cell is updated.
 *
 * What the paper fixes and what is read into it (the reading is stated where
 * the paper is silent):
 *  - Equations: Eqs. frame-momentum and frame-energy with Phi = Phi_bh only and
 *    no frame acceleration (the BH frame of the fallback stage, Sec. 2).
 *  - Time integration: "RK2" (Table 1), read as SSP-RK2 (Heun):
 *      U1 = U0 + dt L(U0),  U2 = (U0 + U1 + dt L(U1)) / 2.
 *  - Reconstruction: "PLM" (Table 1), read as primitive-variable PLM with the
 *    van Leer limiter delta = 2 dl dr / (dl + dr) if dl dr > 0 else 0, faces at
 *    q +- delta/2.  PPM: 4th-order interface value (7/12, -1/12), clipped to the
 *    two adjacent cell values, then the Colella-Woodward (1984) monotonicity
 *    constraints; no characteristic projection, no flattening.
 *    Reconstructed variables: rho, v, P, Gamma_e = 1 + P/U, Gamma_1 and the
 *    auxiliary internal energy density U_aux itself (face U = P/(Gamma_e - 1),
 *    cs^2 = Gamma_1 P / rho; no EOS call at faces).
 *  - Riemann solver: HLLC (Toro, Spruce & Speares) with Davis wave speeds
 *    S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R).
 *  - Dual energy (Sec. 6.2): switch Eq. dual-primitive-switch, auxiliary flux
 *    Eq. dual-flux and face velocity Eq. dual-face-velocity with the upwind
 *    reconstructed face state chosen by the sign of F_rho (zero if F_rho = 0);
 *    compression Eq. dual-divv with the analytic exponential for an ideal gas
 *    and Eq. dual-tabulated-compression for the table, using the stage's
 *    updated density, Delta t_l = dt (stage 1) and dt/2 (stage 2); resync
 *    Eq. dual-sync over the 3x3x3 neighbourhood, once per full step.
 *  - Gravity (Sec. 3.3): momentum source Eq. lat-grav-momentum, energy source
 *    Eq. lat-grav-energy with the Godunov mass fluxes, in every active
 *    direction; Phi = Eq. bh-softened-gravity at the stage time
 *    (t_n for stage 1, t_n + dt for stage 2) on the BH trajectory
 *    x0 + v0 (t - t0) + a0 (t - t0)^2 / 2.  A ghost cell takes the position of
 *    its periodic image (its own position across an outflow boundary).
 *  - Excision (Sec. 3.1): a cell is inside iff |r - r_bh| < r_exc at its centre.
 *    At a face between an outside and an inside cell the flux is kept only if
 *    its mass flux points into the excised cell, otherwise it is zeroed.  After
 *    each full step the inside cells are reset to rho_floor, zero momentum and
 *    internal energy density u_floor.
 *  - Floors (Table 1): rho < rho_floor and P < p_floor are raised at the
 *    conversion to primitives; after each stage rho and U_aux are raised to
 *    rho_floor and u_floor.
 *  - CFL (Sec. 7.1): dt_b = C min over interior non-excised cells of
 *    min_d dx_d / (|v_d| + c_s) and sqrt(dx_min / |g_bh|).
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "tref.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct tref_mesh {
  tref_mesh_desc d;
  int *blocks;
  tref_params p;
  tref_table t;
  int has_table;
  int active[3];
  int nvar;
  int64_t ntot;
  int64_t *off;
  int *pd;      /* nb * 3 padded sizes */
  int *lev;     /* refinement level per block */
  int lmax;     /* finest level */
  int NF[3];    /* cells per direction of the finest level's grid */
  int *owner;   /* finest-level cell -> block */
  const double *phi_sg;   /* self-gravity potential, padded layout (caller's), or NULL */
};

/* cells per direction of the level-L grid */
static int n_at(const tref_mesh *m, int a, int L) { return m->active[a] ? m->d.N[a] << L : 1; }

/* cell width of block b along a */
static double bdx(const tref_mesh *m, int b, int a) {
  return m->active[a] ? ldexp(m->d.dx[a], -m->lev[b]) : m->d.dx[a];
}

/* the block owning the level-L cell g (inside the level-L grid) */
static int owner_at(const tref_mesh *m, int L, const int *g) {
  int f[3];
  for (int a = 0; a < 3; ++a) f[a] = m->active[a] ? g[a] << (m->lmax - L) : 0;
  return m->owner[((int64_t)f[2] * m->NF[1] + f[1]) * m->NF[0] + f[0]];
}

/* boundary map of a level-L index: periodic wrap, outflow clamp to the edge cell.
 * Returns 0 if some direction was clamped. */
static int bmap(const tref_mesh *m, int L, int *g) {
  int in = 1;
  for (int a = 0; a < 3; ++a) {
    const int N = n_at(m, a, L);
    if (g[a] < 0 || g[a] >= N) {
      if (m->d.bc[a] == TREF_PERIODIC) g[a] = ((g[a] % N) + N) % N;
      else { g[a] = g[a] < 0 ? 0 : N - 1; in = 0; }
    }
  }
  return in;
}

/* ---------------------------------------------------------------- mesh --- */

tref_mesh *tref_mesh_new(const tref_mesh_desc *d, const tref_params *p, const tref_table *t) {
  tref_mesh *m = (tref_mesh *)calloc(1, sizeof(tref_mesh));
  m->d = *d;
  m->blocks = (int *)malloc(sizeof(int) * 6 * d->nb);
  memcpy(m->blocks, d->blocks, sizeof(int) * 6 * d->nb);
  m->d.blocks = m->blocks;
  m->p = *p;
  if (t) { m->t = *t; m->has_table = 1; }
  for (int a = 0; a < 3; ++a) m->active[a] = d->N[a] > 1;
  m->nvar = p->dual ? 6 : 5;
  m->off = (int64_t *)malloc(sizeof(int64_t) * (d->nb + 1));
  m->pd = (int *)malloc(sizeof(int) * 3 * d->nb);
  int64_t o = 0;
  for (int b = 0; b < d->nb; ++b) {
    m->off[b] = o;
    int64_t c = 1;
    for (int a = 0; a < 3; ++a) {
      m->pd[3 * b + a] = m->blocks[6 * b + 3 + a] + (m->active[a] ? 2 * d->ng : 0);
      c *= m->pd[3 * b + a];
    }
    o += c;
  }
  m->off[d->nb] = o;
  m->ntot = o;
  m->lev = (int *)calloc(d->nb, sizeof(int));
  m->lmax = 0;
  for (int b = 0; b < d->nb; ++b) {
    m->lev[b] = d->levels ? d->levels[b] : 0;
    if (m->lev[b] < 0 || m->lev[b] > 8) { tref_mesh_free(m); return NULL; }
    if (m->lev[b] > m->lmax) m->lmax = m->lev[b];
  }
  m->d.levels = m->lev;
  for (int a = 0; a < 3; ++a) m->NF[a] = n_at(m, a, m->lmax);
  int64_t ng = (int64_t)m->NF[0] * m->NF[1] * m->NF[2];
  m->owner = (int *)malloc(sizeof(int) * ng);
  for (int64_t c = 0; c < ng; ++c) m->owner[c] = -1;
  for (int b = 0; b < d->nb; ++b) {
    const int *B = m->blocks + 6 * b;
    const int L = m->lev[b];
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      if (B[a] < 0 || B[3 + a] < 1 || B[a] + B[3 + a] > n_at(m, a, L)) { tref_mesh_free(m); return NULL; }
      if (L > 0 && m->active[a] && ((B[a] & 3) || (B[3 + a] & 3))) { tref_mesh_free(m); return NULL; }
      const int s = m->active[a] ? m->lmax - L : 0;
      lo[a] = B[a] << s;
      hi[a] = (B[a] + B[3 + a]) << s;
    }
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int64_t c = ((int64_t)k * m->NF[1] + j) * m->NF[0] + i;
          if (m->owner[c] != -1) { tref_mesh_free(m); return NULL; }
          m->owner[c] = b;
        }
  }
  for (int64_t c = 0; c < ng; ++c)
    if (m->owner[c] < 0) { tref_mesh_free(m); return NULL; }
  /* 2:1 balance across faces, edges and corners */
  if (m->lmax > 0)
    for (int b = 0; b < d->nb; ++b) {
      const int *B = m->blocks + 6 * b;
      const int L = m->lev[b];
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = m->active[a] ? B[a] - 1 : 0;
        hi[a] = m->active[a] ? B[a] + B[3 + a] : 0;
      }
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            int g[3] = {i, j, k};
            if (!bmap(m, L, g)) continue;
            const int s = m->lmax - L;
            for (int fk = 0; fk < (m->active[2] ? 1 << s : 1); ++fk)
              for (int fj = 0; fj < (m->active[1] ? 1 << s : 1); ++fj)
                for (int fi = 0; fi < (m->active[0] ? 1 << s : 1); ++fi) {
                  int f[3] = {m->active[0] ? (g[0] << s) + fi : 0, m->active[1] ? (g[1] << s) + fj : 0,
                              m->active[2] ? (g[2] << s) + fk : 0};
                  int o = m->owner[((int64_t)f[2] * m->NF[1] + f[1]) * m->NF[0] + f[0]];
                  if (abs(m->lev[o] - L) > 1) { tref_mesh_free(m); return NULL; }
                }
          }
    }
  return m;
}

void tref_mesh_free(tref_mesh *m) {
  if (!m) return;
  free(m->blocks); free(m->off); free(m->pd); free(m->lev); free(m->owner); free(m);
}
int64_t tref_mesh_ntot(const tref_mesh *m) { return m->ntot; }
int64_t tref_mesh_block_offset(const tref_mesh *m, int b) { return m->off[b]; }
int tref_nvar(const tref_mesh *m) { return m->nvar; }

void tref_set_phi_sg(tref_mesh *m, const double *phi_padded) { m->phi_sg = phi_padded; }
const double *tref_phi_sg(const tref_mesh *m) { return m->phi_sg; }

/* Threads the OpenMP loops over blocks use (1 without OpenMP). */
int tref_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
/* Threads of the block loops from now on (n >= 1; no effect without OpenMP). */
void tref_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
void tref_set_params(tref_mesh *m, const tref_params *p) { m->p = *p; }

static int gofs(const tref_mesh *m, int a) { return m->active[a] ? m->d.ng : 0; }

static int64_t cidx(const tref_mesh *m, int b, int i, int j, int k) {
  const int *P = m->pd + 3 * b;
  return m->off[b] + ((int64_t)k * P[1] + j) * P[0] + i;
}

const tref_mesh_desc *tref_mesh_get_desc(const tref_mesh *m) { return &m->d; }
/* padded index (within all blocks) of the interior cell at global cell (i, j, k) */
int64_t tref_cell_index(const tref_mesh *m, int i, int j, int k) {
  const int g0[3] = {i, j, k};
  const int b = owner_at(m, 0, g0);
  const int *B = m->blocks + 6 * b;
  const int *P = m->pd + 3 * b;
  return m->off[b] + ((int64_t)(k - B[2] + gofs(m, 2)) * P[1] + (j - B[1] + gofs(m, 1))) * P[0] +
         (i - B[0] + gofs(m, 0));
}

static int is_interior(const tref_mesh *m, int b, int i, int j, int k) {
  const int *B = m->blocks + 6 * b;
  int gx = gofs(m, 0), gy = gofs(m, 1), gz = gofs(m, 2);
  return i >= gx && i < gx + B[3] && j >= gy && j < gy + B[4] && k >= gz && k < gz + B[5];
}

/* Where a ghost fill reads a source block's cells: mode == NULL, or mode[o] == 0:
 * from Udst; 1: from Ucur; 2: Uold + s[o] (Ucur - Uold). */
typedef struct {
  const double *Udst, *Ucur, *Uold;
  const int *mode;
  const double *s;
} src_ctx;

static double fetch(const tref_mesh *m, const src_ctx *sc, int o, int64_t l, int v) {
  const int64_t i = v * m->ntot + l;
  if (!sc->mode || sc->mode[o] == 0) return sc->Udst[i];
  if (sc->mode[o] == 1) return sc->Ucur[i];
  return sc->Uold[i] + sc->s[o] * (sc->Ucur[i] - sc->Uold[i]);
}

static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* The value (first nvar variables) of the level-L cell g after the boundary map:
 * a cell of a level-L block is read; a region covered by finer blocks is the
 * mean of its 2^d children's level values (restriction); a cell inside a
 * coarser block is prolonged: the parent's level value plus, per active
 * direction, a quarter of the minmod of the parent's one-sided differences to
 * its two neighbours (level values too), toward the child's side. */
static void level_value(const tref_mesh *m, const src_ctx *sc, int nvar, int L, const int *gin, double *out) {
  int g[3] = {gin[0], gin[1], gin[2]};
  bmap(m, L, g);
  const int o = owner_at(m, L, g);
  const int Lo = m->lev[o];
  if (Lo == L) {
    const int *O = m->blocks + 6 * o;
    const int64_t l = cidx(m, o, g[0] - O[0] + gofs(m, 0), g[1] - O[1] + gofs(m, 1), g[2] - O[2] + gofs(m, 2));
    for (int v = 0; v < nvar; ++v) out[v] = fetch(m, sc, o, l, v);
    return;
  }
  if (Lo > L) {
    double acc[6] = {0, 0, 0, 0, 0, 0}, ch[6];
    int nch = 0;
    for (int dk = 0; dk < (m->active[2] ? 2 : 1); ++dk)
      for (int dj = 0; dj < (m->active[1] ? 2 : 1); ++dj)
        for (int di = 0; di < (m->active[0] ? 2 : 1); ++di) {
          const int c[3] = {m->active[0] ? 2 * g[0] + di : 0, m->active[1] ? 2 * g[1] + dj : 0,
                            m->active[2] ? 2 * g[2] + dk : 0};
          level_value(m, sc, nvar, L + 1, c, ch);
          for (int v = 0; v < nvar; ++v) acc[v] += ch[v];
          ++nch;
        }
    for (int v = 0; v < nvar; ++v) out[v] = acc[v] / nch;
    return;
  }
  int p[3];
  for (int a = 0; a < 3; ++a) p[a] = m->active[a] ? g[a] >> 1 : 0;
  double c0[6], cp[6], cm[6];
  level_value(m, sc, nvar, L - 1, p, c0);
  for (int v = 0; v < nvar; ++v) out[v] = c0[v];
  for (int a = 0; a < 3; ++a) {
    if (!m->active[a]) continue;
    int q[3] = {p[0], p[1], p[2]};
    q[a] = p[a] + 1;
    level_value(m, sc, nvar, L - 1, q, cp);
    q[a] = p[a] - 1;
    level_value(m, sc, nvar, L - 1, q, cm);
    const double side = (g[a] & 1) ? 0.25 : -0.25;
    for (int v = 0; v < nvar; ++v) out[v] += side * minmod(cp[v] - c0[v], c0[v] - cm[v]);
  }
}

static void fill_ghosts(const tref_mesh *m, double *Udst, const src_ctx *sc, int nvar, int b) {
  const int *B = m->blocks + 6 * b;
  const int *P = m->pd + 3 * b;
  double val[6];
  for (int k = 0; k < P[2]; ++k)
    for (int j = 0; j < P[1]; ++j)
      for (int i = 0; i < P[0]; ++i) {
        if (is_interior(m, b, i, j, k)) continue;
        const int g[3] = {B[0] + i - gofs(m, 0), B[1] + j - gofs(m, 1), B[2] + k - gofs(m, 2)};
        level_value(m, sc, nvar, m->lev[b], g, val);
        const int64_t dst = cidx(m, b, i, j, k);
        for (int v = 0; v < nvar; ++v) Udst[v * m->ntot + dst] = val[v];
      }
}

void tref_ghost_fill(const tref_mesh *m, double *U, int nvar, int nact, const int *ids) {
  int n = ids ? nact : m->d.nb;
  const src_ctx sc = {U, NULL, NULL, NULL, NULL};
  for (int q = 0; q < n; ++q) fill_ghosts(m, U, &sc, nvar, ids ? ids[q] : q);
}

/* LAT ghost fill (Sec. 7.1, ghost states of neighbours on another schedule):
 * mode[o] = 0 copy from Udst (neighbour on the same schedule), 1 copy from
 * Ucur (faster neighbour, frozen at the current fine time), 2 linear
 * interpolation Uold + s (Ucur - Uold) with s = s_block[o] (slower neighbour).
 * At coarse-fine interfaces every cell entering a restriction or a prolongation
 * is first taken at the stage time this way (Sec. 7.1: the histories are
 * restricted, interpolated in time, then prolonged; restriction and the linear
 * time interpolation commute). */
void tref_ghost_fill_modes(const tref_mesh *m, double *Udst, const double *Ucur, const double *Uold,
                           const int *mode, const double *s_block, int nact, const int *ids) {
  const src_ctx sc = {Udst, Ucur, Uold, mode, s_block};
  for (int q = 0; q < nact; ++q) fill_ghosts(m, Udst, &sc, m->nvar, ids[q]);
}

/* -------------------------------------------------------------- physics --- */

static void bh_pos(const tref_params *p, double t, double *r) {
  double s = t - p->bh_t0;
  for (int a = 0; a < 3; ++a) r[a] = p->bh_x0[a] + p->bh_v0[a] * s + 0.5 * p->bh_a0[a] * s * s;
}

double tref_phi_bh(const tref_params *p, const double *x, double t) {
  double r[3];
  bh_pos(p, t, r);
  double dx = x[0] - r[0], dy = x[1] - r[1], dz = x[2] - r[2];
  return -p->GM / sqrt(dx * dx + dy * dy + dz * dz + p->r_soft * p->r_soft);
}

/* centre of padded cell (i,j,k) of block b, periodic images wrapped */
static void cell_pos(const tref_mesh *m, int b, int i, int j, int k, double *x) {
  const int *B = m->blocks + 6 * b;
  int g[3] = {B[0] + i - gofs(m, 0), B[1] + j - gofs(m, 1), B[2] + k - gofs(m, 2)};
  for (int a = 0; a < 3; ++a) {
    int N = n_at(m, a, m->lev[b]);
    if (m->d.bc[a] == TREF_PERIODIC) g[a] = ((g[a] % N) + N) % N;
    x[a] = m->d.xmin[a] + (g[a] + 0.5) * bdx(m, b, a);
  }
}

static int excised_at(const tref_params *p, const double *x, double t) {
  double r[3];
  bh_pos(p, t, r);
  double dx = x[0] - r[0], dy = x[1] - r[1], dz = x[2] - r[2];
  return sqrt(dx * dx + dy * dy + dz * dz) < p->r_exc;
}

/* EOS closure (a3): internal energy density U at density rho -> P, cs^2, and the
 * internal energy actually represented (differs from U only when clamped). */
static void eos_closure(const tref_mesh *m, double rho, double U, double *P, double *cs2,
                        double *U_used, tref_counts *c) {
  const tref_params *p = &m->p;
  if (p->eos == TREF_EOS_IDEAL) {
    *P = (p->gamma - 1.0) * U;
    *cs2 = p->gamma * (*P) / rho;
    *U_used = U;
    return;
  }
  double T, Pc, c2c, eu;
  int cl = tref_eos_invert(&m->t, rho * p->unit_rho, (U / rho) * p->unit_e, &T, &Pc, &c2c, &eu);
  if (cl && c) c->table_clamp++;
  *P = Pc / (p->unit_rho * p->unit_e);
  *cs2 = c2c / p->unit_e;
  *U_used = cl ? rho * (eu / p->unit_e) : U;
}

/* Eq. dual-econs */
static double u_conservative(double rho, const double *u) {
  double ir = 1.0 / rho;
  double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  return u[4] - 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz);
}

static void c2p(const tref_mesh *m, const double *u, double *w, tref_counts *c) {
  const tref_params *p = &m->p;
  double rho = u[0];
  if (rho < p->rho_floor) { rho = p->rho_floor; if (c) c->rho_floor++; }
  double ir = 1.0 / rho;
  double Ucons = u_conservative(rho, u);
  double Ueos = Ucons;
  if (p->dual) {   /* Eq. dual-primitive-switch */
    if (!(Ucons > 0.0 && Ucons > p->eta1 * u[4])) { Ueos = u[5]; if (c) c->dual_aux_used++; }
  }
  double P, cs2, Uu;
  eos_closure(m, rho, Ueos, &P, &cs2, &Uu, c);
  if (P < p->p_floor) { P = p->p_floor; if (c) c->p_floor++; }
  w[0] = rho;
  w[1] = u[1] * ir;
  w[2] = u[2] * ir;
  w[3] = u[3] * ir;
  w[4] = P;
  if (p->eos == TREF_EOS_IDEAL) { w[5] = p->gamma; w[6] = p->gamma; }
  else { w[5] = 1.0 + P / Uu; w[6] = rho * cs2 / P; }
  w[7] = p->dual ? u[5] : 0.0;
}

void tref_cons_to_prim(const tref_mesh *m, const double *u, double *w, tref_counts *c) { c2p(m, u, w, c); }

/* ------------------------------------------------------- reconstruction --- */

/* PLM, van Leer limiter: values at the left and right faces of the centre cell */
static void plm(double qm, double q0, double qp, double *left, double *right) {
  double dl = q0 - qm, dr = qp - q0;
  double delta = (dl * dr > 0.0) ? 2.0 * dl * dr / (dl + dr) : 0.0;
  *left = q0 - 0.5 * delta;
  *right = q0 + 0.5 * delta;
}

/* PPM interface value between q0 and q1 */
static double ppm_iface(double qm1, double q0, double q1, double q2) {
  double a = (7.0 / 12.0) * (q0 + q1) - (1.0 / 12.0) * (qm1 + q2);
  double lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
  if (a < lo) a = lo;
  if (a > hi) a = hi;
  return a;
}

static void ppm(double qm2, double qm1, double q0, double qp1, double qp2, double *left, double *right) {
  double aL = ppm_iface(qm2, qm1, q0, qp1);
  double aR = ppm_iface(qm1, q0, qp1, qp2);
  if ((aR - q0) * (q0 - aL) <= 0.0) {
    aL = q0;
    aR = q0;
  } else {
    double da = aR - aL;
    double q6 = 6.0 * (q0 - 0.5 * (aL + aR));
    if (da * q6 > da * da) aL = 3.0 * q0 - 2.0 * aR;
    else if (-(da * da) > da * q6) aR = 3.0 * q0 - 2.0 * aL;
  }
  *left = aL;
  *right = aR;
}

/* ------------------------------------------------------------------ HLLC --- */

/* physical flux of state w (8 primitives) along direction d; 5 components */
static void phys_flux(const double *w, int d, double E, double *F) {
  double rho = w[0], un = w[1 + d], P = w[4];
  F[0] = rho * un;
  F[1] = rho * un * w[1];
  F[2] = rho * un * w[2];
  F[3] = rho * un * w[3];
  F[1 + d] += P;
  F[4] = (E + P) * un;
}

static double total_energy(const double *w) {
  double U = w[4] / (w[5] - 1.0);
  return U + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

/* HLLC flux F[0..5] (rho, m_x, m_y, m_z, E, U_aux) and face velocity *vf */
static void hllc(const double *wl, const double *wr, int d, int dual, double *F, double *vf) {
  double rl = wl[0], ul = wl[1 + d], pl = wl[4];
  double rr = wr[0], ur = wr[1 + d], pr = wr[4];
  double cl = sqrt(wl[6] * pl / rl), cr = sqrt(wr[6] * pr / rr);
  double El = total_energy(wl), Er = total_energy(wr);
  double SL = fmin(ul - cl, ur - cr);
  double SR = fmax(ul + cl, ur + cr);
  if (SL >= 0.0) {
    phys_flux(wl, d, El, F);
  } else if (SR <= 0.0) {
    phys_flux(wr, d, Er, F);
  } else {
    double SM = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
                (rl * (SL - ul) - rr * (SR - ur));
    const double *w = SM >= 0.0 ? wl : wr;
    double S = SM >= 0.0 ? SL : SR;
    double E = SM >= 0.0 ? El : Er;
    double rho = w[0], un = w[1 + d], P = w[4];
    double Fk[5];
    phys_flux(w, d, E, Fk);
    double fac = rho * (S - un) / (S - SM);
    double Us[5], Uk[5];
    Us[0] = fac;
    Us[1] = fac * w[1];
    Us[2] = fac * w[2];
    Us[3] = fac * w[3];
    Us[1 + d] = fac * SM;
    Us[4] = fac * (E / rho + (SM - un) * (SM + P / (rho * (S - un))));
    Uk[0] = rho;
    Uk[1] = rho * w[1];
    Uk[2] = rho * w[2];
    Uk[3] = rho * w[3];
    Uk[4] = E;
    for (int q = 0; q < 5; ++q) F[q] = Fk[q] + S * (Us[q] - Uk[q]);
  }
  F[5] = 0.0;
  *vf = 0.0;
  if (dual) {   /* Eqs. dual-flux, dual-face-velocity */
    if (F[0] > 0.0) { F[5] = F[0] * (wl[7] / wl[0]); *vf = F[0] / wl[0]; }
    else if (F[0] < 0.0) { F[5] = F[0] * (wr[7] / wr[0]); *vf = F[0] / wr[0]; }
  }
}

/* HLLE flux (Harten, Lax and van Leer with Einfeldt's two-wave form; the
 * production solver of Table 1): with b- = min(S_L, 0) and b+ = max(S_R, 0) from
 * the same Davis wave-speed bounds as hllc,
 *   F = (b+ F_L - b- F_R + b+ b- (U_R - U_L)) / (b+ - b-);
 * the auxiliary-energy flux and face velocity follow the sign of the mass flux
 * as for hllc.  b+ = b- only when both states have zero speed and sound speed,
 * where both physical fluxes vanish. */
static void hlle(const double *wl, const double *wr, int d, int dual, double *F, double *vf) {
  double rl = wl[0], ul = wl[1 + d], pl = wl[4];
  double rr = wr[0], ur = wr[1 + d], pr = wr[4];
  double cl = sqrt(wl[6] * pl / rl), cr = sqrt(wr[6] * pr / rr);
  double El = total_energy(wl), Er = total_energy(wr);
  double bm = fmin(fmin(ul - cl, ur - cr), 0.0);
  double bp = fmax(fmax(ul + cl, ur + cr), 0.0);
  double FL[5], FR[5];
  phys_flux(wl, d, El, FL);
  phys_flux(wr, d, Er, FR);
  double UL[5] = {rl, rl * wl[1], rl * wl[2], rl * wl[3], El};
  double UR[5] = {rr, rr * wr[1], rr * wr[2], rr * wr[3], Er};
  for (int q = 0; q < 5; ++q)
    F[q] = bp > bm ? (bp * FL[q] - bm * FR[q] + bp * bm * (UR[q] - UL[q])) / (bp - bm) : FL[q];
  F[5] = 0.0;
  *vf = 0.0;
  if (dual) {   /* Eqs. dual-flux, dual-face-velocity */
    if (F[0] > 0.0) { F[5] = F[0] * (wl[7] / wl[0]); *vf = F[0] / wl[0]; }
    else if (F[0] < 0.0) { F[5] = F[0] * (wr[7] / wr[0]); *vf = F[0] / wr[0]; }
  }
}

/* The Riemann solvers on n face-state pairs (a unit check of a5): wl, wr are
 * [n][8] primitives (rho, vx, vy, vz, P, Gamma_e, Gamma_1, U_aux), F [n][6], vf [n]. */
void tref_riemann(int solver, int d, int dual, int64_t n, const double *wl, const double *wr, double *F,
                  double *vf) {
  for (int64_t q = 0; q < n; ++q) {
    if (solver == TREF_HLLE) hlle(wl + 8 * q, wr + 8 * q, d, dual, F + 6 * q, vf + q);
    else hllc(wl + 8 * q, wr + 8 * q, d, dual, F + 6 * q, vf + q);
  }
}

/* -------------------------------------------------------------- stage ----- */

/* flux-register layout of one block: sides x-, x+, y-, y+, z-, z+; each
 * nvar * (transverse interior cells) doubles; returns the block's size */
static int64_t freg_side_offset(const tref_mesh *m, int b, int side, int *n1) {
  const int *B = m->blocks + 6 * b;
  int64_t o = 0;
  for (int s = 0; s < 6; ++s) {
    int a = s / 2;
    int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    int64_t n = (int64_t)B[3 + t1] * B[3 + t2];
    if (s == side) { if (n1) *n1 = B[3 + t1]; return o; }
    o += n * m->nvar;
  }
  return o;
}

int64_t tref_freg_block_size(const tref_mesh *m, int b) { return freg_side_offset(m, b, 6, NULL); }

static void stage_block(const tref_mesh *m, int stage, int b, const double *U0, const double *Uin,
                        double *Uout, double dt, double t0, double *freg, tref_counts *c) {
  const tref_params *p = &m->p;
  const int *B = m->blocks + 6 * b;
  const int *P = m->pd + 3 * b;
  const int64_t npc = (int64_t)P[0] * P[1] * P[2];
  const int nvar = m->nvar;
  const int64_t nt = m->ntot;
  const double tst = stage == 0 ? t0 : t0 + dt;
  const int g[3] = {gofs(m, 0), gofs(m, 1), gofs(m, 2)};
  const int64_t st[3] = {1, P[0], (int64_t)P[0] * P[1]};
  const double dxb[3] = {bdx(m, b, 0), bdx(m, b, 1), bdx(m, b, 2)};   /* the block level's widths */

  /* a2 + a3 on every padded cell */
  double *W = (double *)malloc(sizeof(double) * 8 * npc);
  double *phi = (double *)calloc(npc, sizeof(double));
  char *exc = (char *)calloc(npc, 1);
  for (int k = 0; k < P[2]; ++k)
    for (int j = 0; j < P[1]; ++j)
      for (int i = 0; i < P[0]; ++i) {
        int64_t l = ((int64_t)k * P[1] + j) * P[0] + i;
        double u[6], w[8];
        for (int v = 0; v < nvar; ++v) u[v] = Uin[v * nt + m->off[b] + l];
        c2p(m, u, w, is_interior(m, b, i, j, k) ? c : NULL);
        for (int v = 0; v < 8; ++v) W[v * npc + l] = w[v];
        if (p->bh_on || p->excision_on) {
          double x[3];
          cell_pos(m, b, i, j, k, x);
          if (p->bh_on) phi[l] = tref_phi_bh(p, x, tst);
          if (p->excision_on) exc[l] = (char)excised_at(p, x, tst);
        }
        if (m->phi_sg) phi[l] += m->phi_sg[m->off[b] + l];   /* Eq. potential-decomposition */
      }

  /* a4 + a5: fluxes on every face of every active direction */
  double *F[3] = {NULL, NULL, NULL};
  int nf[3][3];
  for (int a = 0; a < 3; ++a) {
    if (!m->active[a]) continue;
    for (int e = 0; e < 3; ++e) nf[a][e] = B[3 + e] + (e == a ? 1 : 0);
    int64_t nfa = (int64_t)nf[a][0] * nf[a][1] * nf[a][2];
    F[a] = (double *)malloc(sizeof(double) * 7 * nfa);
    for (int fk = 0; fk < nf[a][2]; ++fk)
      for (int fj = 0; fj < nf[a][1]; ++fj)
        for (int fi = 0; fi < nf[a][0]; ++fi) {
          /* face lies on the low side of cell R = (fi, fj, fk) + g */
          int64_t lr = ((int64_t)(fk + g[2]) * P[1] + (fj + g[1])) * P[0] + (fi + g[0]);
          int64_t ll = lr - st[a];
          double wl[8], wr[8];
          for (int v = 0; v < 8; ++v) {
            const double *q = W + v * npc;
            double lft, rgt;
            if (p->recon == TREF_PLM) {
              plm(q[ll - st[a]], q[ll], q[ll + st[a]], &lft, &wl[v]);
              plm(q[lr - st[a]], q[lr], q[lr + st[a]], &wr[v], &rgt);
            } else {
              ppm(q[ll - 2 * st[a]], q[ll - st[a]], q[ll], q[ll + st[a]], q[ll + 2 * st[a]], &lft, &wl[v]);
              ppm(q[lr - 2 * st[a]], q[lr - st[a]], q[lr], q[lr + st[a]], q[lr + 2 * st[a]], &wr[v], &rgt);
            }
          }
          double Fl[6], vf;
          if (p->riemann == TREF_HLLE) hlle(wl, wr, a, p->dual, Fl, &vf);
          else hllc(wl, wr, a, p->dual, Fl, &vf);
          if (p->excision_on && exc[ll] != exc[lr]) {
            /* one-way sink: keep only mass flowing into the excised cell */
            int into = exc[lr] ? (Fl[0] > 0.0) : (Fl[0] < 0.0);
            if (!into) { for (int q = 0; q < 6; ++q) Fl[q] = 0.0; vf = 0.0; }
          }
          int64_t fidx = ((int64_t)fk * nf[a][1] + fj) * nf[a][0] + fi;
          int64_t nfa2 = nfa;
          for (int q = 0; q < 6; ++q) F[a][q * nfa2 + fidx] = Fl[q];
          F[a][6 * nfa2 + fidx] = vf;
        }
  }

  /* a6: divergence, gravity sources, RK combination, compression, floors */
  for (int k = 0; k < B[5]; ++k)
    for (int j = 0; j < B[4]; ++j)
      for (int i = 0; i < B[3]; ++i) {
        int64_t l = ((int64_t)(k + g[2]) * P[1] + (j + g[1])) * P[0] + (i + g[0]);
        int64_t gl = m->off[b] + l;
        double L[6] = {0, 0, 0, 0, 0, 0};
        double divv = 0.0;
        for (int a = 0; a < 3; ++a) {
          if (!m->active[a]) continue;
          int ci[3] = {i, j, k};
          int64_t nfa = (int64_t)nf[a][0] * nf[a][1] * nf[a][2];
          int64_t flo = ((int64_t)ci[2] * nf[a][1] + ci[1]) * nf[a][0] + ci[0];
          ci[a] += 1;
          int64_t fhi = ((int64_t)ci[2] * nf[a][1] + ci[1]) * nf[a][0] + ci[0];
          for (int q = 0; q < nvar; ++q) L[q] -= (F[a][q * nfa + fhi] - F[a][q * nfa + flo]) / dxb[a];
          divv += (F[a][6 * nfa + fhi] - F[a][6 * nfa + flo]) / dxb[a];
          if (p->bh_on || m->phi_sg) {
            double ph = phi[l + st[a]], p0 = phi[l], pl = phi[l - st[a]];
            L[1 + a] -= W[l] * (ph - pl) / (2.0 * dxb[a]);
            L[4] -= (F[a][fhi] * (ph - p0) + F[a][flo] * (p0 - pl)) / (2.0 * dxb[a]);
          }
        }
        if (p->frame_on) {
          /* inertial force of the accelerating frame (Eq. frame-momentum) and its
           * work, from the stage's input state at the cell centre */
          const double rho_in = Uin[gl];
          for (int a = 0; a < 3; ++a) L[1 + a] -= rho_in * p->afr[a];
          L[4] -= Uin[1 * nt + gl] * p->afr[0] + Uin[2 * nt + gl] * p->afr[1] + Uin[3 * nt + gl] * p->afr[2];
        }
        double un[6];
        for (int q = 0; q < nvar; ++q) {
          if (stage == 0) un[q] = U0[q * nt + gl] + dt * L[q];
          else un[q] = 0.5 * (U0[q * nt + gl] + (Uin[q * nt + gl] + dt * L[q]));
        }
        if (un[0] < p->rho_floor) { un[0] = p->rho_floor; if (c) c->rho_floor++; }
        if (p->dual) {
          double dtl = stage == 0 ? dt : 0.5 * dt;
          if (p->eos == TREF_EOS_IDEAL) {
            un[5] = un[5] * exp(-(p->gamma - 1.0) * divv * dtl);
          } else {
            double Pa, c2a, Uu;
            eos_closure(m, un[0], un[5], &Pa, &c2a, &Uu, c);
            un[5] = un[5] - Pa * divv * dtl;
          }
          if (un[5] < p->u_floor) { un[5] = p->u_floor; if (c) c->u_floor++; }
        }
        for (int q = 0; q < nvar; ++q) Uout[q * nt + gl] = un[q];
      }

  /* a9: time-integrated fluxes of the block's boundary faces (weights 1/2, 1/2) */
  if (freg) {
    double *R = freg;
    for (int a = 0; a < 3; ++a) {
      if (!m->active[a]) continue;
      int64_t nfa = (int64_t)nf[a][0] * nf[a][1] * nf[a][2];
      for (int side = 0; side < 2; ++side) {
        int n1;
        int64_t so = freg_side_offset(m, b, 2 * a + side, &n1);
        int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        for (int c2 = 0; c2 < B[3 + t2]; ++c2)
          for (int c1 = 0; c1 < B[3 + t1]; ++c1) {
            int ci[3];
            ci[a] = side ? B[3 + a] : 0;
            ci[t1] = c1;
            ci[t2] = c2;
            int64_t fidx = ((int64_t)ci[2] * nf[a][1] + ci[1]) * nf[a][0] + ci[0];
            int64_t ncell = (int64_t)B[3 + t1] * B[3 + t2];
            for (int q = 0; q < nvar; ++q)
              R[so + q * ncell + (int64_t)c2 * n1 + c1] += 0.5 * dt * F[a][q * nfa + fidx];
          }
      }
    }
  }
  for (int a = 0; a < 3; ++a) free(F[a]);
  free(W); free(phi); free(exc);
}

static void add_counts(tref_counts *dst, const tref_counts *s) {
  dst->rho_floor += s->rho_floor; dst->p_floor += s->p_floor; dst->u_floor += s->u_floor;
  dst->table_clamp += s->table_clamp; dst->excised += s->excised;
  dst->dual_aux_used += s->dual_aux_used; dst->synced += s->synced;
}

void tref_stage(const tref_mesh *m, int stage, int nact, const int *ids, const double *U0,
                const double *Uin, double *Uout, const double *dt_b, const double *t_b,
                double *flux_reg, tref_counts *c) {
  int n = ids ? nact : m->d.nb;
  /* flux-register base offset per block */
  int64_t *fo = NULL;
  if (flux_reg) {
    fo = (int64_t *)malloc(sizeof(int64_t) * (m->d.nb + 1));
    fo[0] = 0;
    for (int b = 0; b < m->d.nb; ++b) fo[b + 1] = fo[b] + tref_freg_block_size(m, b);
  }
#pragma omp parallel
  {
    tref_counts lc;
    memset(&lc, 0, sizeof lc);
#pragma omp for schedule(dynamic)
    for (int q = 0; q < n; ++q) {
      int b = ids ? ids[q] : q;
      stage_block(m, stage, b, U0, Uin, Uout, dt_b[b], t_b[b], flux_reg ? flux_reg + fo[b] : NULL, &lc);
    }
    if (c) {
#pragma omp critical
      add_counts(c, &lc);
    }
  }
  free(fo);
}

void tref_excise(const tref_mesh *m, double *U, int nact, const int *ids, const double *t_end_b,
                 tref_counts *c) {
  const tref_params *p = &m->p;
  if (!p->excision_on) return;
  int n = ids ? nact : m->d.nb;
  for (int q = 0; q < n; ++q) {
    int b = ids ? ids[q] : q;
    const int *B = m->blocks + 6 * b;
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          int ii = i + gofs(m, 0), jj = j + gofs(m, 1), kk = k + gofs(m, 2);
          double x[3];
          cell_pos(m, b, ii, jj, kk, x);
          if (!excised_at(p, x, t_end_b[b])) continue;
          int64_t l = cidx(m, b, ii, jj, kk);
          U[0 * m->ntot + l] = p->rho_floor;
          U[1 * m->ntot + l] = 0.0;
          U[2 * m->ntot + l] = 0.0;
          U[3 * m->ntot + l] = 0.0;
          U[4 * m->ntot + l] = p->u_floor;
          if (p->dual) U[5 * m->ntot + l] = p->u_floor;
          if (c) c->excised++;
        }
  }
}

void tref_dual_sync(const tref_mesh *m, double *U, int nact, const int *ids, tref_counts *c) {
  const tref_params *p = &m->p;
  if (!p->dual) return;
  int n = ids ? nact : m->d.nb;
  for (int q = 0; q < n; ++q) {
    int b = ids ? ids[q] : q;
    const int *B = m->blocks + 6 * b;
    const int *P = m->pd + 3 * b;
    int64_t st[3] = {1, P[0], (int64_t)P[0] * P[1]};
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          int64_t l = cidx(m, b, i + gofs(m, 0), j + gofs(m, 1), k + gofs(m, 2));
          double emax = -HUGE_VAL;
          for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
              for (int di = -1; di <= 1; ++di) {
                if ((di && !m->active[0]) || (dj && !m->active[1]) || (dk && !m->active[2])) continue;
                double e = U[4 * m->ntot + l + di * st[0] + dj * st[1] + dk * st[2]];
                if (e > emax) emax = e;
              }
          double u[6];
          for (int v = 0; v < 6; ++v) u[v] = U[v * m->ntot + l];
          double rho = u[0] < p->rho_floor ? p->rho_floor : u[0];
          double Uc = u_conservative(rho, u);
          if (Uc > 0.0 && Uc > p->eta2 * emax) {
            U[5 * m->ntot + l] = Uc;
            if (c) c->synced++;
          }
        }
  }
}

void tref_cfl_dt(const tref_mesh *m, const double *U, double cfl, const double *t_b, double *dt_b,
                 tref_counts *c) {
  const tref_params *p = &m->p;
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < m->d.nb; ++b) {
    const int *B = m->blocks + 6 * b;
    double dxmin = HUGE_VAL;
    for (int a = 0; a < 3; ++a)
      if (m->active[a] && bdx(m, b, a) < dxmin) dxmin = bdx(m, b, a);
    double best = HUGE_VAL;
    tref_counts lc;
    memset(&lc, 0, sizeof lc);
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          int ii = i + gofs(m, 0), jj = j + gofs(m, 1), kk = k + gofs(m, 2);
          double x[3];
          cell_pos(m, b, ii, jj, kk, x);
          double tb = t_b ? t_b[b] : 0.0;
          if (p->excision_on && excised_at(p, x, tb)) continue;
          int64_t l = cidx(m, b, ii, jj, kk);
          double u[6], w[8];
          for (int v = 0; v < m->nvar; ++v) u[v] = U[v * m->ntot + l];
          c2p(m, u, w, &lc);
          double cs = sqrt(w[6] * w[4] / w[0]);
          for (int a = 0; a < 3; ++a) {
            if (!m->active[a]) continue;
            double s = bdx(m, b, a) / (fabs(w[1 + a]) + cs);
            if (s < best) best = s;
          }
          if (p->bh_on) {
            double r[3];
            bh_pos(p, tb, r);
            double ddx = x[0] - r[0], ddy = x[1] - r[1], ddz = x[2] - r[2];
            double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            double s2 = r2 + p->r_soft * p->r_soft;
            double gmag = p->GM * sqrt(r2) / (s2 * sqrt(s2));
            if (gmag > 0.0) {
              double s = sqrt(dxmin / gmag);
              if (s < best) best = s;
            }
          }
        }
    dt_b[b] = cfl * best;
    if (c) {
#pragma omp critical
      add_counts(c, &lc);
    }
  }
}

void tref_step(const tref_mesh *m, double *U, double *Uscr, double dt, double t, tref_counts *c) {
  int nb = m->d.nb;
  if (m->lmax > 0) {
    /* refined mesh: the coarse-fine flux correction needs the flux registers;
     * one LAT window with every factor 1 is exactly the synchronised step */
    int32_t *ones = (int32_t *)malloc(sizeof(int32_t) * nb);
    for (int b = 0; b < nb; ++b) ones[b] = 1;
    tref_lat_window(m, U, ones, dt, t, c, NULL);
    free(ones);
    return;
  }
  double *dtb = (double *)malloc(sizeof(double) * nb);
  double *tb = (double *)malloc(sizeof(double) * nb);
  double *te = (double *)malloc(sizeof(double) * nb);
  for (int b = 0; b < nb; ++b) { dtb[b] = dt; tb[b] = t; te[b] = t + dt; }
  tref_ghost_fill(m, U, m->nvar, 0, NULL);
  tref_stage(m, 0, 0, NULL, U, U, Uscr, dtb, tb, NULL, c);
  tref_ghost_fill(m, Uscr, m->nvar, 0, NULL);
  tref_stage(m, 1, 0, NULL, U, Uscr, U, dtb, tb, NULL, c);
  tref_excise(m, U, 0, NULL, te, c);
  if (m->p.dual) {
    tref_ghost_fill(m, U, m->nvar, 0, NULL);
    tref_dual_sync(m, U, 0, NULL, c);
  }
  free(dtb); free(tb); free(te);
}

void tref_prim_to_cons(const tref_mesh *m, const double *W, double *U) {
  /* W holds 5 fields (rho, vx, vy, vz, P) in the same padded layout as U */
  const tref_params *p = &m->p;
  const int64_t nt = m->ntot;
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < m->d.nb; ++b) {
    const int *B = m->blocks + 6 * b;
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          int64_t l = cidx(m, b, i + gofs(m, 0), j + gofs(m, 1), k + gofs(m, 2));
          double rho = W[l], vx = W[nt + l], vy = W[2 * nt + l], vz = W[3 * nt + l], P = W[4 * nt + l];
          double Uint;
          if (p->eos == TREF_EOS_IDEAL) {
            Uint = P / (p->gamma - 1.0);
          } else {
            double T = tref_eos_T_from_P(&m->t, rho * p->unit_rho, P * p->unit_rho * p->unit_e);
            double Pc, ec, cc;
            tref_eos_eval_rhoT(&m->t, rho * p->unit_rho, T, &Pc, &ec, &cc);
            Uint = rho * (ec / p->unit_e);
          }
          U[l] = rho;
          U[nt + l] = rho * vx;
          U[2 * nt + l] = rho * vy;
          U[3 * nt + l] = rho * vz;
          U[4 * nt + l] = Uint + 0.5 * rho * (vx * vx + vy * vy + vz * vz);
          if (p->dual) U[5 * nt + l] = Uint;
        }
  }
}

/* read-only view of the mesh internals for the LAT oracle (tref_lat.c) */
typedef struct {
  int nb, N[3], bc[3], ng, active[3], nvar;
  const int *blocks;
  const int *pd;
  const int64_t *off;
  const int *owner;
  double dx[3];
  const tref_params *p;
  int64_t ntot;
  const int *lev;
  int lmax, NF[3];
} tref_mesh_view;

void tref_mesh_get_view(const tref_mesh *m, tref_mesh_view *v) {
  v->nb = m->d.nb;
  v->lev = m->lev;
  v->lmax = m->lmax;
  for (int a = 0; a < 3; ++a) v->NF[a] = m->NF[a];
  for (int a = 0; a < 3; ++a) {
    v->N[a] = m->d.N[a];
    v->bc[a] = m->d.bc[a];
    v->active[a] = m->active[a];
    v->dx[a] = m->d.dx[a];
  }
  v->ng = m->d.ng;
  v->nvar = m->nvar;
  v->blocks = m->blocks;
  v->pd = m->pd;
  v->off = m->off;
  v->owner = m->owner;
  v->p = &m->p;
  v->ntot = m->ntot;
}

void tref_cell_pos(const tref_mesh *m, int b, int i, int j, int k, double *x) { cell_pos(m, b, i, j, k, x); }

/* ---------------------------------------------------------- moving frame --- */

void tref_frame_acceleration(const tref_mesh *m, const double *U, double t, double rho_min,
                             double *A, double *mass) {
  const tref_params *p = &m->p;
  const int64_t nt = m->ntot;
  double rb[3];
  bh_pos(p, t, rb);
  double s0 = 0.0, s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < m->d.nb; ++b) {
    const int *B = m->blocks + 6 * b;
    const int *P = m->pd + 3 * b;
    /* a level-L cell holds 2^-(L d) level-0 cell volumes (d active directions) */
    const double vw = ldexp(1.0, -m->lev[b] * (m->active[0] + m->active[1] + m->active[2]));
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          const int ci = i + gofs(m, 0), cj = j + gofs(m, 1), ck = k + gofs(m, 2);
          const double rho = U[m->off[b] + ((int64_t)ck * P[1] + cj) * P[0] + ci];
          if (!(rho > rho_min)) continue;
          double x[3];
          cell_pos(m, b, ci, cj, ck, x);
          if (p->excision_on && excised_at(p, x, t)) continue;
          const double d[3] = {x[0] - rb[0], x[1] - rb[1], x[2] - rb[2]};
          const double q2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + p->r_soft * p->r_soft;
          const double gfac = -p->GM / (q2 * sqrt(q2));   /* g = -grad Phi_bh = -GM d / q^3 */
          const double rw = rho * vw;   /* mass in level-0 cell volumes */
          for (int a = 0; a < 3; ++a) s[a] += rw * gfac * d[a];
          s0 += rw;
        }
  }
  (void)nt;
  for (int a = 0; a < 3; ++a) A[a] = s0 > 0.0 ? s[a] / s0 : 0.0;
  *mass = s0 * m->d.dx[0] * m->d.dx[1] * m->d.dx[2];
}

void tref_boost(const tref_mesh *m, double *U, const double *V, double rho_min) {
  const int64_t nt = m->ntot;
  for (int b = 0; b < m->d.nb; ++b) {
    const int *B = m->blocks + 6 * b;
    const int *P = m->pd + 3 * b;
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          const int64_t l = m->off[b] + ((int64_t)(k + gofs(m, 2)) * P[1] + (j + gofs(m, 1))) * P[0] +
                            (i + gofs(m, 0));
          const double rho = U[l];
          if (!(rho > rho_min)) continue;
          const double mv = U[nt + l] * V[0] + U[2 * nt + l] * V[1] + U[3 * nt + l] * V[2];
          const double v2 = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
          U[4 * nt + l] += mv + 0.5 * rho * v2;          /* E' = E + rho v.V + rho |V|^2 / 2 */
          for (int a = 0; a < 3; ++a) U[(1 + a) * nt + l] += rho * V[a];   /* (rho v)' = rho (v + V) */
        }
  }
}

