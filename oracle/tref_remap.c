/* tref_remap.c -- oracle of the conserved-variable remap (Sec. 5.2, Eqs.
 * remap-state-vector and remap-cell-average): each target cell is the average of
 * N_qd = 2^(active directions) midpoint samples (two per active direction, at
 * the centres of the cell's halves), each a trilinear interpolation of the
 * source's cell-centred values.  The energy is carried as thermal energy: rho,
 * m and U (the auxiliary energy where the source evolves it, else
 * E - |m|^2 / (2 rho)) are interpolated and the target's total energy rebuilt
 * as U + |m|^2 / (2 rho).  mode TREF_REMAP_TOTAL interpolates E instead (the
 * form the paper compares against).  A target cell coincident with a source
 * cell is copied.  Samples outside the source domain take the floor state.
 *
 * Test infrastructure (tests/test_oracle_remap.py pins it; the GPU remap is
 * checked against it); nothing in the product links it. */
#include <math.h>
#include <stdlib.h>

#include "tref.h"

/* cell-centred value of variable q at global cell (i, j, k) of the source;
 * indices beyond the domain follow the boundary condition (periodic wrap or
 * outflow copy of the edge cell) */
static double src_val(const tref_mesh *m, const double *U, int q, int i, int j, int k, int *ok) {
  int g[3] = {i, j, k};
  const tref_mesh_desc *d = tref_mesh_get_desc(m);
  for (int a = 0; a < 3; ++a) {
    const int N = d->N[a];
    if (g[a] < 0 || g[a] >= N) {
      if (d->bc[a] == TREF_PERIODIC) g[a] = ((g[a] % N) + N) % N;
      else g[a] = g[a] < 0 ? 0 : N - 1;
    }
  }
  *ok = 1;
  return U[(int64_t)q * tref_mesh_ntot(m) + tref_cell_index(m, g[0], g[1], g[2])];
}

/* thermal energy density of a source cell */
static double src_thermal(const tref_mesh *m, const double *U, int dual, int i, int j, int k) {
  int ok;
  if (dual) return src_val(m, U, TREF_AUX, i, j, k, &ok);
  const double r = src_val(m, U, 0, i, j, k, &ok);
  const double mx = src_val(m, U, 1, i, j, k, &ok), my = src_val(m, U, 2, i, j, k, &ok),
               mz = src_val(m, U, 3, i, j, k, &ok);
  return src_val(m, U, 4, i, j, k, &ok) - 0.5 * (mx * mx + my * my + mz * mz) / r;
}

void tref_remap(const tref_mesh *dst, double *Udst, const tref_mesh *src, const double *Usrc, int mode,
                double rho_floor, double u_floor) {
  const tref_mesh_desc *D = tref_mesh_get_desc(dst), *S = tref_mesh_get_desc(src);
  const int dual_s = tref_nvar(src) == 6, dual_d = tref_nvar(dst) == 6;
  const int64_t ntd = tref_mesh_ntot(dst);
  int act[3];
  for (int a = 0; a < 3; ++a) act[a] = D->N[a] > 1;
  for (int b = 0; b < D->nb; ++b) {
    const int *B = D->blocks + 6 * b;
    for (int k = 0; k < B[5]; ++k)
      for (int j = 0; j < B[4]; ++j)
        for (int i = 0; i < B[3]; ++i) {
          const int gi[3] = {B[0] + i, B[1] + j, B[2] + k};
          double xc[3];
          for (int a = 0; a < 3; ++a) xc[a] = D->xmin[a] + (gi[a] + 0.5) * D->dx[a];
          const int64_t l = tref_cell_index(dst, gi[0], gi[1], gi[2]);
          /* a coincident source cell: copied */
          int coinc = 1, sc[3];
          for (int a = 0; a < 3; ++a) {
            const double s = (xc[a] - S->xmin[a]) / S->dx[a] - 0.5;
            sc[a] = (int)floor(s + 0.5);
            if (fabs(D->dx[a] - S->dx[a]) > 1e-12 * S->dx[a] || fabs(s - sc[a]) > 1e-9 || sc[a] < 0 ||
                sc[a] >= S->N[a])
              coinc = 0;
          }
          if (coinc) {
            int ok;
            for (int q = 0; q < 5; ++q) Udst[q * ntd + l] = src_val(src, Usrc, q, sc[0], sc[1], sc[2], &ok);
            if (dual_d) Udst[5 * ntd + l] = src_thermal(src, Usrc, dual_s, sc[0], sc[1], sc[2]);
            continue;
          }
          /* midpoint samples: two per active direction */
          double acc[5] = {0, 0, 0, 0, 0};
          int ns = 0;
          for (int c = 0; c < (act[2] ? 2 : 1); ++c)
            for (int bb = 0; bb < (act[1] ? 2 : 1); ++bb)
              for (int aa = 0; aa < (act[0] ? 2 : 1); ++aa) {
                const int sub[3] = {aa, bb, c};
                double r[3];
                int inside = 1;
                for (int a = 0; a < 3; ++a) {
                  r[a] = act[a] ? xc[a] + (sub[a] ? 0.25 : -0.25) * D->dx[a] : xc[a];
                  const double lo = S->xmin[a], hi = S->xmin[a] + S->N[a] * S->dx[a];
                  if (S->N[a] > 1 && (r[a] < lo || r[a] > hi) && S->bc[a] != TREF_PERIODIC) inside = 0;
                }
                ++ns;
                if (!inside) {   /* floor state at rest */
                  acc[0] += rho_floor;
                  acc[4] += u_floor;
                  continue;
                }
                /* trilinear interpolation of rho, m, and U (or E) at r */
                int i0[3];
                double t[3];
                for (int a = 0; a < 3; ++a) {
                  if (S->N[a] == 1) { i0[a] = 0; t[a] = 0.0; continue; }
                  const double s = (r[a] - S->xmin[a]) / S->dx[a] - 0.5;
                  i0[a] = (int)floor(s);
                  t[a] = s - i0[a];
                }
                for (int cz = 0; cz < 2; ++cz)
                  for (int by = 0; by < 2; ++by)
                    for (int ax = 0; ax < 2; ++ax) {
                      const double w = (ax ? t[0] : 1.0 - t[0]) * (by ? t[1] : 1.0 - t[1]) * (cz ? t[2] : 1.0 - t[2]);
                      if (w == 0.0) continue;
                      const int ci = i0[0] + ax, cj = i0[1] + by, ck = i0[2] + cz;
                      int ok;
                      for (int q = 0; q < 4; ++q) acc[q] += w * src_val(src, Usrc, q, ci, cj, ck, &ok);
                      acc[4] += w * (mode == TREF_REMAP_TOTAL ? src_val(src, Usrc, 4, ci, cj, ck, &ok)
                                                              : src_thermal(src, Usrc, dual_s, ci, cj, ck));
                    }
              }
          for (int q = 0; q < 5; ++q) acc[q] /= ns;
          const double ke = 0.5 * (acc[1] * acc[1] + acc[2] * acc[2] + acc[3] * acc[3]) / acc[0];
          Udst[l] = acc[0];
          for (int q = 1; q < 4; ++q) Udst[q * ntd + l] = acc[q];
          if (mode == TREF_REMAP_TOTAL) {
            Udst[4 * ntd + l] = acc[4];
            if (dual_d) Udst[5 * ntd + l] = acc[4] - ke;
          } else {
            Udst[4 * ntd + l] = acc[4] + ke;
            if (dual_d) Udst[5 * ntd + l] = acc[4];
          }
        }
  }
}
