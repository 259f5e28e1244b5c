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
} tref_mesh_view;
void tref_mesh_get_view(const tref_mesh *m, tref_mesh_view *v);
void tref_cell_pos(const tref_mesh *m, int b, int i, int j, int k, double *x);

static int gofs(const tref_mesh_view *v, int a) { return v->active[a] ? v->ng : 0; }

/* block adjacency: every block whose interior supplies a ghost cell of b */
static void neighbours(const tref_mesh_view *v, int b, int *nbr, int *nn) {
  const int *B = v->blocks + 6 * b;
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
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
          if (g[a] < 0 || g[a] >= v->N[a]) {
            inside = 0;
            if (v->bc[a] == TREF_PERIODIC) g[a] = ((g[a] % v->N[a]) + v->N[a]) % v->N[a];
            else g[a] = g[a] < 0 ? 0 : v->N[a] - 1;
          }
        }
        (void)inside;
        int o = v->owner[((int64_t)g[2] * v->N[1] + g[1]) * v->N[0] + g[0]];
        if (o == b) continue;
        int seen = 0;
        for (int q = 0; q < *nn; ++q)
          if (nbr[q] == o) seen = 1;
        if (!seen) nbr[(*nn)++] = o;
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
  /* neighbour limiting: f_b <= 2 min over face/edge/corner neighbours */
  int *nbr = (int *)malloc(sizeof(int) * 27 * 64);
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int b = 0; b < nb; ++b) {
      int nn;
      neighbours(&v, b, nbr, &nn);
      for (int q = 0; q < nn; ++q)
        if (f_b[b] > 2 * f_b[nbr[q]]) { f_b[b] = 2 * f_b[nbr[q]]; changed = 1; }
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

/* refluxing of the listed completing blocks at time t (see the file comment) */
static void reflux(const tref_mesh *m, const tref_mesh_view *v, double *U, double *R,
                   const int64_t *fo, const int32_t *f_b, int ncomp, const int *comp, double t) {
  const tref_params *p = v->p;
  for (int qb = 0; qb < ncomp; ++qb) {
    int b = comp[qb];
    const int *B = v->blocks + 6 * b;
    const int *P = v->pd + 3 * b;
    for (int a = 0; a < 3; ++a) {
      if (!v->active[a]) continue;
      int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
      for (int side = 0; side < 2; ++side) {
        int s = 2 * a + side;
        double sigma = side ? 1.0 : -1.0;   /* outward orientation of the face */
        for (int c2 = 0; c2 < B[3 + t2]; ++c2)
          for (int c1 = 0; c1 < B[3 + t1]; ++c1) {
            int ci[3];
            ci[a] = side ? B[3 + a] - 1 : 0;
            ci[t1] = c1;
            ci[t2] = c2;
            /* neighbour cell across the face */
            int g[3] = {B[0] + ci[0], B[1] + ci[1], B[2] + ci[2]};
            g[a] += side ? 1 : -1;
            if (g[a] < 0 || g[a] >= v->N[a]) {
              if (v->bc[a] != TREF_PERIODIC) continue;
              g[a] = ((g[a] % v->N[a]) + v->N[a]) % v->N[a];
            }
            int o = v->owner[((int64_t)g[2] * v->N[1] + g[1]) * v->N[0] + g[0]];
            const int *O = v->blocks + 6 * o;
            int oc[3] = {g[0] - O[0], g[1] - O[1], g[2] - O[2]};
            int os = 2 * a + (1 - side);
            if (f_b[o] < f_b[b]) {
              int64_t l = v->off[b] + ((int64_t)(ci[2] + gofs(v, 2)) * P[1] + (ci[1] + gofs(v, 1))) * P[0] +
                          (ci[0] + gofs(v, 0));
              double dI[6];
              for (int q = 0; q < v->nvar; ++q) {
                double Io = R[fo[o] + side_index(v, o, os, oc[t1], oc[t2], q)];
                double Is = R[fo[b] + side_index(v, b, s, c1, c2, q)];
                dI[q] = Io - Is;   /* accepted minus local impulse */
              }
              const double *psg = tref_phi_sg(m);
              if (p->bh_on || psg) {
                double xi[3], xn[3];
                int pos[3] = {ci[0] + gofs(v, 0), ci[1] + gofs(v, 1), ci[2] + gofs(v, 2)};
                tref_cell_pos(m, b, pos[0], pos[1], pos[2], xi);
                int pn[3] = {pos[0], pos[1], pos[2]};
                pn[a] += side ? 1 : -1;
                tref_cell_pos(m, b, pn[0], pn[1], pn[2], xn);
                double phi_i = p->bh_on ? tref_phi_bh(p, xi, t) : 0.0;
                double phi_n = p->bh_on ? tref_phi_bh(p, xn, t) : 0.0;
                if (psg) {   /* the frozen self-gravity potential */
                  phi_i += psg[l];
                  phi_n += psg[v->off[b] + ((int64_t)pn[2] * P[1] + pn[1]) * P[0] + pn[0]];
                }
                /* Eq. lat-grav-reflux with dI_rho = local - accepted = -dI[0] */
                U[4 * v->ntot + l] += sigma / (2.0 * v->dx[a]) * (-dI[0]) * (phi_n - phi_i);
              }
              for (int q = 0; q < v->nvar; ++q) U[q * v->ntot + l] += -sigma * dI[q] / v->dx[a];
              for (int q = 0; q < v->nvar; ++q)
                R[fo[o] + side_index(v, o, os, oc[t1], oc[t2], q)] = 0.0;
            }
            if (f_b[o] <= f_b[b])
              for (int q = 0; q < v->nvar; ++q) R[fo[b] + side_index(v, b, s, c1, c2, q)] = 0.0;
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
