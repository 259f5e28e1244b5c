/* tref_grav.c -- oracle of the self-gravity solver (Sec. 3.2): a geometric
 * multigrid for A_h phi = S_h with A_h = -lap_h (the seven-point operator with
 * the anisotropic weights w_y = (dx/dy)^2, w_z = (dx/dz)^2, Eq. selfgrav-poisson)
 * and S_h = -4 pi G rho_sg, on a uniform periodic grid.
 *
 * Test infrastructure: the GPU implementation is checked against this file and
 * the file against closed forms (tests/test_oracle_grav.py); nothing in the
 * product links it.
 *
 * V-cycle, in the order the paper gives: red-black Gauss-Seidel pre-smoothing
 * with over-relaxation omega; defect d_h = S_h - A_h phi_h (Eq. selfgrav-defect);
 * restriction of phi and d by volume averages over the child cells;
 * full-approximation coarse equation A_H phi_H = R d_h + A_H R phi_h; the
 * coarse correction phi_H - R phi_h prolonged (trilinear, cell centred) and
 * added; post-smoothing on every level; one extra sweep on the finest level at
 * the end of the cycle.  Each direction is halved while it has more than one
 * cell, down to a single cell, where the periodic correction is zero.  The mean
 * of the source is removed in two passes. */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tref.h"

typedef struct {
  int n[3];
  double dx[3];
  double *phi, *src, *tmp;
} level_t;

static int64_t idx3(const level_t *L, int i, int j, int k) {
  i = (i % L->n[0] + L->n[0]) % L->n[0];
  j = (j % L->n[1] + L->n[1]) % L->n[1];
  k = (k % L->n[2] + L->n[2]) % L->n[2];
  return ((int64_t)k * L->n[1] + j) * L->n[0] + i;
}

/* weights of the seven-point operator relative to x: (dx/da)^2, 0 for a
 * direction with one cell (its neighbours are the cell itself) */
static void weights(const level_t *L, double w[3]) {
  for (int a = 0; a < 3; ++a) w[a] = L->n[a] > 1 ? (L->dx[0] / L->dx[a]) * (L->dx[0] / L->dx[a]) : 0.0;
}

/* (A phi)_i = -(1/dx^2) sum_a w_a (phi_{i+a} + phi_{i-a} - 2 phi_i) */
static double apply_A(const level_t *L, const double *phi, int i, int j, int k) {
  double w[3];
  weights(L, w);
  const double c = phi[idx3(L, i, j, k)];
  double s = 0.0;
  s += w[0] * (phi[idx3(L, i + 1, j, k)] + phi[idx3(L, i - 1, j, k)] - 2.0 * c);
  s += w[1] * (phi[idx3(L, i, j + 1, k)] + phi[idx3(L, i, j - 1, k)] - 2.0 * c);
  s += w[2] * (phi[idx3(L, i, j, k + 1)] + phi[idx3(L, i, j, k - 1)] - 2.0 * c);
  return -s / (L->dx[0] * L->dx[0]);
}

/* one red-black Gauss-Seidel sweep: colour 0 ((i + j + k) even), then colour 1 */
static void smooth(level_t *L, double omega) {
  double w[3];
  weights(L, w);
  const double diag = 2.0 * (w[0] + w[1] + w[2]);
  if (diag == 0.0) return;   /* a single cell */
  const double h2 = L->dx[0] * L->dx[0];
  for (int colour = 0; colour < 2; ++colour)
    for (int k = 0; k < L->n[2]; ++k)
      for (int j = 0; j < L->n[1]; ++j)
        for (int i = 0; i < L->n[0]; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          const int64_t c = idx3(L, i, j, k);
          double nb = w[0] * (L->phi[idx3(L, i + 1, j, k)] + L->phi[idx3(L, i - 1, j, k)]) +
                      w[1] * (L->phi[idx3(L, i, j + 1, k)] + L->phi[idx3(L, i, j - 1, k)]) +
                      w[2] * (L->phi[idx3(L, i, j, k + 1)] + L->phi[idx3(L, i, j, k - 1)]);
          const double gs = (h2 * L->src[c] + nb) / diag;
          L->phi[c] = (1.0 - omega) * L->phi[c] + omega * gs;
        }
}

static int64_t ncell(const level_t *L) { return (int64_t)L->n[0] * L->n[1] * L->n[2]; }

/* volume average of the children of coarse cell (I, J, K) in field f of level Lf */
static double restrict_cell(const level_t *Lf, const level_t *Lc, const double *f, int I, int J, int K) {
  const int r[3] = {Lf->n[0] / Lc->n[0], Lf->n[1] / Lc->n[1], Lf->n[2] / Lc->n[2]};
  double s = 0.0;
  for (int c = 0; c < r[2]; ++c)
    for (int b = 0; b < r[1]; ++b)
      for (int a = 0; a < r[0]; ++a) s += f[idx3(Lf, r[0] * I + a, r[1] * J + b, r[2] * K + c)];
  return s / (r[0] * r[1] * r[2]);
}

/* trilinear prolongation (cell centred) of the coarse field e at fine cell (i, j, k):
 * per halved direction weights 3/4 on the parent and 1/4 on its neighbour towards
 * the fine cell */
static double prolong_cell(const level_t *Lf, const level_t *Lc, const double *e, int i, int j, int k) {
  const int f[3] = {i, j, k};
  int p[3], q[3];
  double wp[3];
  for (int a = 0; a < 3; ++a) {
    const int r = Lf->n[a] / Lc->n[a];
    if (r == 1) { p[a] = f[a]; q[a] = f[a]; wp[a] = 1.0; continue; }
    p[a] = f[a] / 2;
    q[a] = (f[a] & 1) ? p[a] + 1 : p[a] - 1;
    wp[a] = 0.75;
  }
  double s = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const double wa = a ? 1.0 - wp[0] : wp[0];
        const double wb = b ? 1.0 - wp[1] : wp[1];
        const double wc = c ? 1.0 - wp[2] : wp[2];
        if (wa == 0.0 || wb == 0.0 || wc == 0.0) continue;
        s += wa * wb * wc * e[idx3(Lc, a ? q[0] : p[0], b ? q[1] : p[1], c ? q[2] : p[2])];
      }
  return s;
}

static void vcycle(level_t *Ls, int l, int nl, int npre, int npost, double omega) {
  level_t *L = &Ls[l];
  if (l == nl - 1) return;   /* a single cell: the periodic correction is zero */
  level_t *C = &Ls[l + 1];
  for (int s = 0; s < npre; ++s) smooth(L, omega);
  /* defect on the fine level */
  for (int k = 0; k < L->n[2]; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i)
        L->tmp[idx3(L, i, j, k)] = L->src[idx3(L, i, j, k)] - apply_A(L, L->phi, i, j, k);
  /* coarse phi = R phi, coarse source = R d + A_H R phi; keep R phi in C->tmp */
  for (int K = 0; K < C->n[2]; ++K)
    for (int J = 0; J < C->n[1]; ++J)
      for (int I = 0; I < C->n[0]; ++I) {
        const int64_t c = idx3(C, I, J, K);
        C->phi[c] = restrict_cell(L, C, L->phi, I, J, K);
        C->tmp[c] = C->phi[c];
      }
  for (int K = 0; K < C->n[2]; ++K)
    for (int J = 0; J < C->n[1]; ++J)
      for (int I = 0; I < C->n[0]; ++I)
        C->src[idx3(C, I, J, K)] = restrict_cell(L, C, L->tmp, I, J, K) + apply_A(C, C->phi, I, J, K);
  double *rphi = (double *)malloc(sizeof(double) * ncell(C));
  memcpy(rphi, C->tmp, sizeof(double) * ncell(C));
  vcycle(Ls, l + 1, nl, npre, npost, omega);
  for (int64_t q = 0; q < ncell(C); ++q) C->tmp[q] = C->phi[q] - rphi[q];
  free(rphi);
  for (int k = 0; k < L->n[2]; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) L->phi[idx3(L, i, j, k)] += prolong_cell(L, C, C->tmp, i, j, k);
  for (int s = 0; s < npost; ++s) smooth(L, omega);
}

double tref_mg_defect_rms(int nx, int ny, int nz, const double *dx, const double *src, const double *phi) {
  level_t L = {{nx, ny, nz}, {dx[0], dx[1], dx[2]}, (double *)phi, (double *)src, NULL};
  double s = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double d = src[idx3(&L, i, j, k)] - apply_A(&L, phi, i, j, k);
        s += d * d;
      }
  return sqrt(s / ((double)nx * ny * nz));
}

int tref_mg_solve(int nx, int ny, int nz, const double *dx, const double *src_in, double *phi,
                  int max_cycles, double tol, int npre, int npost, double omega, double *defect) {
  /* levels: halve every direction with more than one cell (each must be a power of two) */
  level_t Ls[64];
  int nl = 0;
  int n[3] = {nx, ny, nz};
  double h[3] = {dx[0], dx[1], dx[2]};
  for (;;) {
    level_t *L = &Ls[nl++];
    for (int a = 0; a < 3; ++a) { L->n[a] = n[a]; L->dx[a] = h[a]; }
    const int64_t nc = (int64_t)n[0] * n[1] * n[2];
    L->phi = nl == 1 ? phi : (double *)calloc(nc, sizeof(double));
    L->src = (double *)calloc(nc, sizeof(double));
    L->tmp = (double *)calloc(nc, sizeof(double));
    if (n[0] == 1 && n[1] == 1 && n[2] == 1) break;
    for (int a = 0; a < 3; ++a)
      if (n[a] > 1) { n[a] /= 2; h[a] *= 2.0; }
  }
  /* source without its mean, removed in two passes (one pass leaves a rounding
   * residual in the operator's null space) */
  const int64_t nc0 = (int64_t)nx * ny * nz;
  memcpy(Ls[0].src, src_in, sizeof(double) * nc0);
  for (int pass = 0; pass < 2; ++pass) {
    double m = 0.0;
    for (int64_t q = 0; q < nc0; ++q) m += Ls[0].src[q];
    m /= (double)nc0;
    for (int64_t q = 0; q < nc0; ++q) Ls[0].src[q] -= m;
  }
  int cycles = 0;
  double d = tref_mg_defect_rms(nx, ny, nz, dx, Ls[0].src, phi);
  while (cycles < max_cycles && !(d < tol)) {
    vcycle(Ls, 0, nl, npre, npost, omega);
    smooth(&Ls[0], omega);   /* the extra sweep on the finest level */
    ++cycles;
    d = tref_mg_defect_rms(nx, ny, nz, dx, Ls[0].src, phi);
  }
  for (int l = 0; l < nl; ++l) {
    if (l > 0) free(Ls[l].phi);
    free(Ls[l].src);
    free(Ls[l].tmp);
  }
  if (defect) *defect = d;
  return cycles;
}
