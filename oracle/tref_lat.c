/*
 * tref_lat.c -- ORACLE (test infrastructure only): localized adaptive time
 * stepping (LAT), Sec. 7.1-7.2 of the paper.
 *
 * Factor assignment (Eq. lat-base-dt, Eq. lat-factor):
 *   dt0 = min_b dt_b;  f_b = 2^min(N_LAT, floor(log2(dt_b / dt0)));
 *   sparse top bins (fewer than merge_frac * nb blocks) are merged into the next
 *   smaller bin, repeatedly; then factors are lowered until every pair of blocks
 *   sharing a face, edge or corner differs by at most a factor of two.
 *
 * Window (Sec. 7.1): f_max = max f_b; the fine sub-steps tau = 0 .. f_max - 1 each
 * advance the active set {b : tau mod f_b = 0} by one RK2 step of f_b dt0,
 * level by level from the largest factor down (reading: slow blocks first).
 * Ghost states of a neighbour on another schedule (reading):
 *   - same factor: its state at the same stage;
 *   - faster neighbour: frozen at tau (its state before it advances), both stages;
 *   - slower neighbour: linear interpolation between its stored start-of-step
 *     state and its end-of-step state at the stage time.
 * Flux correction (Eq. lat-flux-impulse, reading of the garbled sentence): every
 * block accumulates the time integral dt (F^1 + F^2)/2 of its boundary fluxes per
 * face cell.  When a block completes a step, each of its boundary cells that
 * faces a faster neighbour is corrected by the difference between the
 * neighbour's accumulated impulse and its own, both over the completed step; the
 * gravitational work of the mass-impulse mismatch is corrected with
 * Eq. lat-grav-reflux (Phi at the completion time).  Then the block's excision
 * reset and dual-energy resync run.  With every f_b = 1 this is exactly the
 * synchronised step sequence of tref_step.
 */
#include "tref.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* internal access to the mesh (defined in tref_hydro.c) */
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
void tref_mesh_get_view(const tref_mesh *m, tref_mesh_view *v);
void tref_cell_pos(const tref_mesh *m, int b, int i, int j, int k, double *x);

static int gofs(const tref_mesh_view *v, int a) { return v->active[a] ? v->ng : 0; }

static int n_at(const tref_mesh_view *v, int a, int L) { return v->active[a] ? v->N[a] << L : 1; }

static double bdx(const tref_mesh_view *v, int b, int a) {
  return v->active[a] ? ldexp(v->dx[a], -v->lev[b]) : v->dx[a];
}

/* owner of the finest-level cell f */
static int owner_f(const tref_mesh_view *v, const int *f) {
  return v->owner[((int64_t)f[2] * v->NF[1] + f[1]) * v->NF[0] + f[0]];
}

/* boundary map of a level-L index (periodic wrap, outflow clamp); 0 if clamped */
static int bmap(const tref_mesh_view *v, int L, int *g) {
  int in = 1;
  for (int a = 0; a < 3; ++a) {
    const int N = n_at(v, a, L);
    if (g[a] < 0 || g[a] >= N) {
      if (v->bc[a] == TREF_PERIODIC) g[a] = ((g[a] % N) + N) % N;
      else { g[a] = g[a] < 0 ? 0 : N - 1; in = 0; }
    }
  }
  return in;
}

/* block adjacency: every block sharing a face, edge or corner with b (the
 * blocks covering its one-cell shell, on every level; across an outflow
 * boundary the shell maps onto the edge cells) */
static void neighbours(const tref_mesh_view *v, int b, int *nbr, int *nn) {
  const int *B = v->blocks + 6 * b;
  const int L = v->lev[b], sft = v->lmax - L;
  *nn = 0;
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = v->active[a] ? -1 : 0;
    hi[a] = v->active[a] ? B[3 + a] : B[3 + a] - 1;
  }
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int g[3] = {B[0] + i, B[1] + j, B[2] + k};
        bmap(v, L, g);
        for (int fk = 0; fk < (v->active[2] ? 1 << sft : 1); ++fk)
          for (int fj = 0; fj < (v->active[1] ? 1 << sft : 1); ++fj)
            for (int fi = 0; fi < (v->active[0] ? 1 << sft : 1); ++fi) {
              const int f[3] = {v->active[0] ? (g[0] << sft) + fi : 0, v->active[1] ? (g[1] << sft) + fj : 0,
                                v->active[2] ? (g[2] << sft) + fk : 0};
              const int o = owner_f(v, f);
              if (o == b) continue;
              int seen = 0;
              for (int q = 0; q < *nn; ++q)
                if (nbr[q] == o) seen = 1;
              if (!seen) nbr[(*nn)++] = o;
            }
      }
}

int tref_lat_factors(const tref_mesh *m, const double *dt_b, int n_lat, double merge_frac,
                     int32_t *f_b, double *dt0_out) {
  tref_mesh_view v;
  tref_mesh_get_view(m, &v);
  const int nb = v.nb;
  double dt0 = HUGE_VAL;
  for (int b = 0; b < nb; ++b)
    if (dt_b[b] < dt0) dt0 = dt_b[b];
  /* Eq. lat-factor: floor(log2(x)) taken exactly as the binary exponent */
  for (int b = 0; b < nb; ++b) {
    int e;
    frexp(dt_b[b] / dt0, &e);   /* x = m 2^e, m in [0.5, 1): floor(log2 x) = e - 1 */
    int k = e - 1;
    if (k > n_lat) k = n_lat;
    if (k < 0) k = 0;
    f_b[b] = 1 << k;
  }
  /* merge sparse top bins into the next smaller one */
  for (;;) {
    int fmax = 1, cnt = 0;
    for (int b = 0; b < nb; ++b)
      if (f_b[b] > fmax) fmax = f_b[b];
    if (fmax == 1) break;
    for (int b = 0; b < nb; ++b)
      if (f_b[b] == fmax) ++cnt;
    if (cnt >= merge_frac * nb) break;
    for (int b = 0; b < nb; ++b)
      if (f_b[b] == fmax) f_b[b] = fmax / 2;
  }
  /* neighbour limiting, by lowering factors until it holds: f_b <= 2 f_o over
   * face/edge/corner neighbours o, and f_fine <= f_coarse across coarse-fine
   * interfaces (with the first rule, f_fine <= f_coarse <= 2 f_fine) */
  int *nbr = (int *)malloc(sizeof(int) * nb);
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int b = 0; b < nb; ++b) {
      int nn;
      neighbours(&v, b, nbr, &nn);
      for (int q = 0; q < nn; ++q) {
        const int o = nbr[q];
        if (f_b[b] > 2 * f_b[o]) { f_b[b] = 2 * f_b[o]; changed = 1; }
        if (v.lev[b] > v.lev[o] && f_b[b] > f_b[o]) { f_b[b] = f_b[o]; changed = 1; }
      }
    }
  }
  free(nbr);
  int fmax = 1;
  for (int b = 0; b < nb; ++b)
    if (f_b[b] > fmax) fmax = f_b[b];
  if (dt0_out) *dt0_out = dt0;
  return fmax;
}

/* flux-register base offsets per block */
static int64_t *freg_offsets(const tref_mesh *m, int nb) {
  int64_t *fo = (int64_t *)malloc(sizeof(int64_t) * (nb + 1));
  fo[0] = 0;
  for (int b = 0; b < nb; ++b) fo[b + 1] = fo[b] + tref_freg_block_size(m, b);
  return fo;
}

/* offset (within a block's register) of side s, transverse cell (c1, c2) */
static int64_t side_index(const tref_mesh_view *v, int b, int side, int c1, int c2, int q) {
  const int *B = v->blocks + 6 * b;
  int64_t o = 0;
  for (int s = 0; s < side; ++s) {
    int a = s / 2;
    int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    o += (int64_t)B[3 + t1] * B[3 + t2] * v->nvar;
  }
  int a = side / 2;
  int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
  int64_t ncell = (int64_t)B[3 + t1] * B[3 + t2];
  return o + q * ncell + (int64_t)c2 * B[3 + t1] + c1;
}

/* Eq. lat-grav-reflux: the gravitational work of a mass-impulse mismatch dIrho
 * (local minus accepted) through the face between padded cell pos of block b and
 * its neighbour across side (a, sigma), with Phi at time t */
static double grav_reflux(const tref_mesh *m, const tref_mesh_view *v, int b, const int *pos, int a, int side,
                          double dIrho, double t) {
  const tref_params *p = v->p;
  const double *psg = tref_phi_sg(m);
  if (!p->bh_on && !psg) return 0.0;
  const int *P = v->pd + 3 * b;
  double xi[3], xn[3];
  tref_cell_pos(m, b, pos[0], pos[1], pos[2], xi);
  int pn[3] = {pos[0], pos[1], pos[2]};
  pn[a] += side ? 1 : -1;
  tref_cell_pos(m, b, pn[0], pn[1], pn[2], xn);
  double phi_i = p->bh_on ? tref_phi_bh(p, xi, t) : 0.0;
  double phi_n = p->bh_on ? tref_phi_bh(p, xn, t) : 0.0;
  if (psg) {   /* the frozen self-gravity potential */
    phi_i += psg[v->off[b] + ((int64_t)pos[2] * P[1] + pos[1]) * P[0] + pos[0]];
    phi_n += psg[v->off[b] + ((int64_t)pn[2] * P[1] + pn[1]) * P[0] + pn[0]];
  }
  const double sigma = side ? 1.0 : -1.0;
  return sigma / (2.0 * bdx(v, b, a)) * dIrho * (phi_n - phi_i);
}

/* Refluxing of the listed completing blocks at time t (see the file comment).
 * Across a coarse-fine face the fine side's impulses are the accepted ones: a
 * completing coarse block replaces its own impulse on each face cell by the mean
 * of the 2^(d-1) fine impulses behind it (their area-weighted flux), and a fine
 * block keeps its impulses for the coarse side (f_fine <= f_coarse, so the
 * coarse block completes at a phase where every fine neighbour completes too). */
static void reflux(const tref_mesh *m, const tref_mesh_view *v, double *U, double *R,
                   const int64_t *fo, const int32_t *f_b, int ncomp, const int *comp, double t) {
  for (int qb = 0; qb < ncomp; ++qb) {
    int b = comp[qb];
    const int *B = v->blocks + 6 * b;
    const int *P = v->pd + 3 * b;
    const int L = v->lev[b];
    for (int a = 0; a < 3; ++a) {
      if (!v->active[a]) continue;
      int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
      const double dxa = bdx(v, b, a);
      for (int side = 0; side < 2; ++side) {
        int s = 2 * a + side;
        double sigma = side ? 1.0 : -1.0;   /* outward orientation of the face */
        int os = 2 * a + (1 - side);
        for (int c2 = 0; c2 < B[3 + t2]; ++c2)
          for (int c1 = 0; c1 < B[3 + t1]; ++c1) {
            int ci[3];
            ci[a] = side ? B[3 + a] - 1 : 0;
            ci[t1] = c1;
            ci[t2] = c2;
            /* level-L cell across the face */
            int g[3] = {B[0] + ci[0], B[1] + ci[1], B[2] + ci[2]};
            g[a] += side ? 1 : -1;
            const int N = n_at(v, a, L);
            if (g[a] < 0 || g[a] >= N) {
              if (v->bc[a] != TREF_PERIODIC) continue;
              g[a] = ((g[a] % N) + N) % N;
            }
            const int sft = v->lmax - L;
            const int f[3] = {v->active[0] ? g[0] << sft : 0, v->active[1] ? g[1] << sft : 0,
                              v->active[2] ? g[2] << sft : 0};
            const int o = owner_f(v, f);
            const int pos[3] = {ci[0] + gofs(v, 0), ci[1] + gofs(v, 1), ci[2] + gofs(v, 2)};
            const int64_t l = v->off[b] + ((int64_t)pos[2] * P[1] + pos[1]) * P[0] + pos[0];
            double dI[6];
            if (v->lev[o] == L) {
              const int *O = v->blocks + 6 * o;
              int oc[3] = {g[0] - O[0], g[1] - O[1], g[2] - O[2]};
              if (f_b[o] < f_b[b]) {
                for (int q = 0; q < v->nvar; ++q) {
                  double Io = R[fo[o] + side_index(v, o, os, oc[t1], oc[t2], q)];
                  double Is = R[fo[b] + side_index(v, b, s, c1, c2, q)];
                  dI[q] = Io - Is;   /* accepted minus local impulse */
                }
                U[4 * v->ntot + l] += grav_reflux(m, v, b, pos, a, side, -dI[0], t);
                for (int q = 0; q < v->nvar; ++q) U[q * v->ntot + l] += -sigma * dI[q] / dxa;
                for (int q = 0; q < v->nvar; ++q)
                  R[fo[o] + side_index(v, o, os, oc[t1], oc[t2], q)] = 0.0;
              }
              if (f_b[o] <= f_b[b])
                for (int q = 0; q < v->nvar; ++q) R[fo[b] + side_index(v, b, s, c1, c2, q)] = 0.0;
            } else if (v->lev[o] == L + 1) {
              /* the fine face cells behind this coarse face cell, on level L + 1 */
              double acc[6] = {0, 0, 0, 0, 0, 0};
              int nf = 0;
              for (int e2 = 0; e2 < (v->active[t2] ? 2 : 1); ++e2)
                for (int e1 = 0; e1 < (v->active[t1] ? 2 : 1); ++e1) {
                  int h[3];
                  h[a] = side ? 2 * g[a] : 2 * g[a] + 1;
                  h[t1] = v->active[t1] ? 2 * g[t1] + e1 : 0;
                  h[t2] = v->active[t2] ? 2 * g[t2] + e2 : 0;
                  const int sf = v->lmax - L - 1;
                  const int ff[3] = {v->active[0] ? h[0] << sf : 0, v->active[1] ? h[1] << sf : 0,
                                     v->active[2] ? h[2] << sf : 0};
                  const int o2 = owner_f(v, ff);
                  const int *O = v->blocks + 6 * o2;
                  const int lc1 = h[t1] - O[t1], lc2 = h[t2] - O[t2];
                  for (int q = 0; q < v->nvar; ++q) {
                    int64_t r = fo[o2] + side_index(v, o2, os, lc1, lc2, q);
                    acc[q] += R[r];
                    R[r] = 0.0;
                  }
                  ++nf;
                }
              for (int q = 0; q < v->nvar; ++q) dI[q] = acc[q] / nf - R[fo[b] + side_index(v, b, s, c1, c2, q)];
              U[4 * v->ntot + l] += grav_reflux(m, v, b, pos, a, side, -dI[0], t);
              for (int q = 0; q < v->nvar; ++q) U[q * v->ntot + l] += -sigma * dI[q] / dxa;
              for (int q = 0; q < v->nvar; ++q) R[fo[b] + side_index(v, b, s, c1, c2, q)] = 0.0;
            }
            /* a coarser neighbour (level L - 1) reads this block's impulses */
          }
      }
    }
  }
}

int tref_lat_window(const tref_mesh *m, double *U, const int32_t *f_b, double dt0, double t,
                    tref_counts *c, int64_t *block_updates) {
  tref_mesh_view v;
  tref_mesh_get_view(m, &v);
  const int nb = v.nb, nvar = v.nvar;
  const int64_t nt = v.ntot;
  int fmax = 1;
  for (int b = 0; b < nb; ++b)
    if (f_b[b] > fmax) fmax = f_b[b];
  double *Uold = (double *)malloc(sizeof(double) * nvar * nt);
  double *U1 = (double *)calloc((size_t)nvar * nt, sizeof(double));
  memcpy(Uold, U, sizeof(double) * nvar * nt);
  int64_t *fo = freg_offsets(m, nb);
  double *R = (double *)calloc(fo[nb], sizeof(double));
  double *dtb = (double *)malloc(sizeof(double) * nb);
  double *tb = (double *)malloc(sizeof(double) * nb);
  double *te = (double *)malloc(sizeof(double) * nb);
  double *sb = (double *)malloc(sizeof(double) * nb);
  int *mode = (int *)malloc(sizeof(int) * nb);
  int *ids = (int *)malloc(sizeof(int) * nb);
  for (int b = 0; b < nb; ++b) dtb[b] = f_b[b] * dt0;
  int64_t updates = 0;
  for (int tau = 0; tau <= fmax; ++tau) {
    if (tau > 0) {   /* completion phase of the blocks whose step ends now */
      int n = 0;
      for (int b = 0; b < nb; ++b)
        if (tau % f_b[b] == 0) ids[n++] = b;
      double tc = t + tau * dt0;
      reflux(m, &v, U, R, fo, f_b, n, ids, tc);
      for (int b = 0; b < nb; ++b) te[b] = tc;
      tref_excise(m, U, n, ids, te, c);
      if (m && v.p->dual) {
        tref_ghost_fill(m, U, nvar, n, ids);
        tref_dual_sync(m, U, n, ids, c);
      }
    }
    if (tau == fmax) break;
    for (int f = fmax; f >= 1; f /= 2) {
      if (tau % f) continue;
      int n = 0;
      for (int b = 0; b < nb; ++b)
        if (f_b[b] == f) ids[n++] = b;
      if (!n) continue;
      for (int q = 0; q < n; ++q) {
        int b = ids[q];
        int64_t o0 = v.off[b], o1 = v.off[b + 1];
        for (int var = 0; var < nvar; ++var)
          memcpy(Uold + var * nt + o0, U + var * nt + o0, sizeof(double) * (o1 - o0));
        tb[b] = t + tau * dt0;
      }
      for (int stage = 0; stage < 2; ++stage) {
        for (int o = 0; o < nb; ++o) {
          if (f_b[o] == f) { mode[o] = 0; sb[o] = 0.0; }
          else if (f_b[o] < f) { mode[o] = 1; sb[o] = 0.0; }
          else { mode[o] = 2; sb[o] = (double)(tau % f_b[o] + stage * f) / (double)f_b[o]; }
        }
        double *Udst = stage == 0 ? U : U1;
        tref_ghost_fill_modes(m, Udst, U, Uold, mode, sb, n, ids);
        if (stage == 0) tref_stage(m, 0, n, ids, U, U, U1, dtb, tb, R, c);
        else tref_stage(m, 1, n, ids, U, U1, U, dtb, tb, R, c);
      }
      updates += n;
    }
  }
  if (block_updates) *block_updates = updates;
  free(Uold); free(U1); free(fo); free(R); free(dtb); free(tb); free(te); free(sb);
  free(mode); free(ids);
  return fmax;
}
