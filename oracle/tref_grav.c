/* tref_grav.c -- oracle of the self-gravity solver (Sec. 3.2): a geometric
 * multigrid for A_h phi = S_h with A_h = -lap_h (the seven-point operator with
 * the anisotropic weights w_y = (dx/dy)^2, w_z = (dx/dz)^2, Eq. selfgrav-poisson)
 * and S_h = -4 pi G rho_sg, on a uniform grid that is periodic or isolated.
 *
 * Test infrastructure: the GPU implementation is checked against this file and
 * the file against closed forms (tests/test_oracle_grav.py); nothing in the
 * product links it.
 *
 * V-cycle, in the order the paper gives: red-black Gauss-Seidel pre-smoothing
 * with over-relaxation omega; defect d_h = S_h - A_h phi_h (Eq. selfgrav-defect);
 * restriction of phi and d by volume averages over the child cells;
 * full-approximation coarse equation A_H phi_H = R d_h + A_H R phi_h; the
 * coarse correction phi_H - R phi_h prolonged (tricubic: per halved direction
 * the cubic through the four coarse cell centres nearest the fine cell's) and
 * added; post-smoothing on every level; one extra sweep on the finest level at
 * the end of the cycle.  Each direction is halved while it has more than one
 * cell, down to a single cell.
 *
 * Periodic: the mean of the source is removed in two passes; the single-cell
 * level's correction is zero.
 *
 * Isolated ("multipole boundary conditions", Sec. 3.2): phi on every boundary
 * face is the exterior multipole expansion of the source up to order l_max
 * about a centre c (a Dirichlet condition at the face: the cell beyond it is
 * 2 phi_face - phi_inside),
 *   phi(x) = sum_{l<=l_max} sum_{m<=l} r^-(l+1) P_l^m(cos t) (A_lm cos m p + B_lm sin m p),
 *   (A_lm, B_lm) = (2 - delta_m0) (l-m)!/(l+m)! / (4 pi) sum_cells S dV r'^l P_l^m(cos t') (cos m p', sin m p'),
 * (r, t, p) the spherical coordinates of x - c: the addition theorem of the
 * Legendre polynomials applied to phi = (1/4 pi) int S / |x - x'| dV', which is
 * -G int rho / |x - x'| for S = -4 pi G rho.  Every level takes its face values
 * from the same expansion; a coarse-grid correction vanishes on the faces; the
 * Gauss-Seidel update is implicit in the mirror cells; the single-cell level is
 * solved exactly.
 *
 * Full multigrid (the start of a first or remapped solve): the source restricted
 * to every level, the coarsest level solved, then on each finer level the
 * prolonged solution of the level below followed by one V-cycle on that level. */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "tref.h"

enum { MP_LMAX = 8 };

typedef struct {
  int iso;                 /* 0: periodic, 1: isolated */
  int act[3];              /* direction active on the finest level */
  double x0[3];            /* lower corner of the domain */
  int lmax;                /* multipole order */
  double c[3];             /* expansion centre */
  double A[MP_LMAX + 1][MP_LMAX + 1], B[MP_LMAX + 1][MP_LMAX + 1];
} bc_t;

typedef struct {
  int n[3];
  double dx[3];
  double *phi, *src, *tmp;
  const bc_t *bc;
} level_t;

/* associated Legendre functions P_l^m(x), 0 <= m <= l <= lmax (no Condon-Shortley
 * phase: it cancels in the products of the expansion) */
static void legendre(int lmax, double x, double P[MP_LMAX + 1][MP_LMAX + 1]) {
  const double s = sqrt(fmax(0.0, 1.0 - x * x));
  double pmm = 1.0;
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) pmm *= (2.0 * m - 1.0) * s;
    P[m][m] = pmm;
    if (m + 1 <= lmax) P[m + 1][m] = x * (2.0 * m + 1.0) * pmm;
    for (int l = m + 2; l <= lmax; ++l)
      P[l][m] = ((2.0 * l - 1.0) * x * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
  }
}

static void spherical(const bc_t *bc, const double *x, double *r, double *ct, double *ph) {
  const double d[3] = {x[0] - bc->c[0], x[1] - bc->c[1], x[2] - bc->c[2]};
  *r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  *ct = *r > 0.0 ? d[2] / *r : 1.0;
  *ph = atan2(d[1], d[0]);
}

/* the exterior expansion at x */
static double multipole(const bc_t *bc, const double *x) {
  double r, ct, ph, P[MP_LMAX + 1][MP_LMAX + 1];
  spherical(bc, x, &r, &ct, &ph);
  legendre(bc->lmax, ct, P);
  double s = 0.0;
  for (int l = 0; l <= bc->lmax; ++l) {
    double t = 0.0;
    for (int m = 0; m <= l; ++m) t += P[l][m] * (bc->A[l][m] * cos(m * ph) + bc->B[l][m] * sin(m * ph));
    s += t / pow(r, l + 1);
  }
  return s;
}

/* the moments of the finest level's source (cell volume dV) */
static void moments(bc_t *bc, const level_t *L) {
  double P[MP_LMAX + 1][MP_LMAX + 1], fact[2 * MP_LMAX + 2];
  fact[0] = 1.0;
  for (int q = 1; q < 2 * MP_LMAX + 2; ++q) fact[q] = fact[q - 1] * q;
  memset(bc->A, 0, sizeof bc->A);
  memset(bc->B, 0, sizeof bc->B);
  const double dV = L->dx[0] * L->dx[1] * L->dx[2];
  for (int k = 0; k < L->n[2]; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        const double S = L->src[((int64_t)k * L->n[1] + j) * L->n[0] + i];
        if (S == 0.0) continue;
        const double x[3] = {bc->x0[0] + (i + 0.5) * L->dx[0], bc->x0[1] + (j + 0.5) * L->dx[1],
                             bc->x0[2] + (k + 0.5) * L->dx[2]};
        double r, ct, ph;
        spherical(bc, x, &r, &ct, &ph);
        legendre(bc->lmax, ct, P);
        for (int l = 0; l <= bc->lmax; ++l) {
          const double rl = pow(r, l);
          for (int m = 0; m <= l; ++m) {
            bc->A[l][m] += S * dV * rl * P[l][m] * cos(m * ph);
            bc->B[l][m] += S * dV * rl * P[l][m] * sin(m * ph);
          }
        }
      }
  for (int l = 0; l <= bc->lmax; ++l)
    for (int m = 0; m <= l; ++m) {
      const double f = (m ? 2.0 : 1.0) * fact[l - m] / fact[l + m] / (4.0 * 3.14159265358979323846);
      bc->A[l][m] *= f;
      bc->B[l][m] *= f;
    }
}

static int64_t idx3(const level_t *L, int i, int j, int k) {
  i = (i % L->n[0] + L->n[0]) % L->n[0];
  j = (j % L->n[1] + L->n[1]) % L->n[1];
  k = (k % L->n[2] + L->n[2]) % L->n[2];
  return ((int64_t)k * L->n[1] + j) * L->n[0] + i;
}

/* field f at cell (i, j, k) of level L: periodic images; isolated, a cell
 * outside the grid mirrors the one inside across the boundary face, so that the
 * face value is the multipole expansion there (bval: 2 phi_face - f_inside) or
 * zero (a correction: -f_inside); corners mirror once per direction */
static double at(const level_t *L, const double *f, int i, int j, int k, int bval) {
  if (L->bc->iso) {
    int c[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
      if (c[a] >= 0 && c[a] < L->n[a]) continue;
      const int s = c[a] < 0 ? -1 : 1;
      c[a] = c[a] < 0 ? -1 - c[a] : 2 * L->n[a] - 1 - c[a];
      double g = 0.0;
      if (bval) {
        /* the mirror point on the face (a cell and its image are equally far
         * from the face, at any distance) */
        double x[3];
        for (int b = 0; b < 3; ++b) x[b] = L->bc->x0[b] + (c[b] + 0.5) * L->dx[b];
        x[a] = L->bc->x0[a] + (s < 0 ? 0.0 : L->n[a] * L->dx[a]);
        g = 2.0 * multipole(L->bc, x);
      }
      return g - at(L, f, c[0], c[1], c[2], bval);
    }
  }
  return f[idx3(L, i, j, k)];
}

/* weights of the seven-point operator relative to x: (dx/da)^2; periodic: 0 for
 * a direction with one cell (its neighbours are the cell itself); isolated: 0
 * only for a direction inactive on the finest level */
static void weights(const level_t *L, double w[3]) {
  for (int a = 0; a < 3; ++a) {
    const int on = L->bc->iso ? L->bc->act[a] : L->n[a] > 1;
    w[a] = on ? (L->dx[0] / L->dx[a]) * (L->dx[0] / L->dx[a]) : 0.0;
  }
}

/* (A phi)_i = -(1/dx^2) sum_a w_a (phi_{i+a} + phi_{i-a} - 2 phi_i) */
static double apply_A(const level_t *L, const double *phi, int i, int j, int k) {
  double w[3];
  weights(L, w);
  const double c = phi[idx3(L, i, j, k)];
  double s = 0.0;
  s += w[0] * (at(L, phi, i + 1, j, k, 1) + at(L, phi, i - 1, j, k, 1) - 2.0 * c);
  s += w[1] * (at(L, phi, i, j + 1, k, 1) + at(L, phi, i, j - 1, k, 1) - 2.0 * c);
  s += w[2] * (at(L, phi, i, j, k + 1, 1) + at(L, phi, i, j, k - 1, 1) - 2.0 * c);
  return -s / (L->dx[0] * L->dx[0]);
}

/* the Gauss-Seidel value of cell (i, j, k): the operator's equation solved for
 * the cell, whose mirror images across isolated boundaries (2 phi_face - phi)
 * move to the diagonal */
static double gs_value(const level_t *L, const double *w, double diag, int i, int j, int k) {
  const int64_t c = idx3(L, i, j, k);
  if (!L->bc->iso) {
    const double nb = w[0] * (at(L, L->phi, i + 1, j, k, 1) + at(L, L->phi, i - 1, j, k, 1)) +
                      w[1] * (at(L, L->phi, i, j + 1, k, 1) + at(L, L->phi, i, j - 1, k, 1)) +
                      w[2] * (at(L, L->phi, i, j, k + 1, 1) + at(L, L->phi, i, j, k - 1, 1));
    return (L->dx[0] * L->dx[0] * L->src[c] + nb) / diag;
  }
  const int g[3] = {i, j, k};
  double nb = 0.0, dg = diag;
  for (int a = 0; a < 3; ++a) {
    if (w[a] == 0.0) continue;
    for (int s = -1; s <= 1; s += 2) {
      int q[3] = {i, j, k};
      q[a] += s;
      if (q[a] >= 0 && q[a] < L->n[a]) {
        nb += w[a] * L->phi[idx3(L, q[0], q[1], q[2])];
      } else {
        double x[3];
        for (int b = 0; b < 3; ++b) x[b] = L->bc->x0[b] + (g[b] + 0.5) * L->dx[b];
        x[a] += 0.5 * s * L->dx[a];
        nb += w[a] * 2.0 * multipole(L->bc, x);
        dg += w[a];
      }
    }
  }
  return (L->dx[0] * L->dx[0] * L->src[c] + nb) / dg;
}

/* one red-black Gauss-Seidel sweep: colour 0 ((i + j + k) even), then colour 1 */
static void smooth(level_t *L, double omega) {
  double w[3];
  weights(L, w);
  const double diag = 2.0 * (w[0] + w[1] + w[2]);
  if (diag == 0.0) return;   /* a single periodic cell */
  for (int colour = 0; colour < 2; ++colour)
    for (int k = 0; k < L->n[2]; ++k)
      for (int j = 0; j < L->n[1]; ++j)
        for (int i = 0; i < L->n[0]; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          const int64_t c = idx3(L, i, j, k);
          const double gs = gs_value(L, w, diag, i, j, k);
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

/* tricubic prolongation (cell centred) of the coarse field e at fine cell
 * (i, j, k): along each halved direction the cubic through the four coarse
 * centres nearest the fine centre, which lies a quarter of a coarse cell from
 * its parent's centre p.  Lagrange weights at -1/4 on the nodes p-2, p-1, p,
 * p+1 (fine cell on the parent's low side): -5/128, 35/128, 105/128, -7/128;
 * at +1/4 on p-1, p, p+1, p+2: -7/128, 105/128, 35/128, -5/128.  The weights
 * of the three directions multiply.  Beyond an isolated boundary e is its
 * mirror image (bval: about the face value, else about 0). */
static void cubic_taps(int f, int halved, int *first, double w[4], int *ntap) {
  if (!halved) { *first = f; w[0] = 1.0; *ntap = 1; return; }
  const int p = f / 2;
  *ntap = 4;
  if (f & 1) {
    *first = p - 1;
    w[0] = -7.0 / 128.0; w[1] = 105.0 / 128.0; w[2] = 35.0 / 128.0; w[3] = -5.0 / 128.0;
  } else {
    *first = p - 2;
    w[0] = -5.0 / 128.0; w[1] = 35.0 / 128.0; w[2] = 105.0 / 128.0; w[3] = -7.0 / 128.0;
  }
}

static double prolong_cell(const level_t *Lf, const level_t *Lc, const double *e, int i, int j, int k, int bval) {
  const int f[3] = {i, j, k};
  int first[3], nt[3];
  double w[3][4];
  for (int a = 0; a < 3; ++a) cubic_taps(f[a], Lf->n[a] != Lc->n[a], &first[a], w[a], &nt[a]);
  double s = 0.0;
  for (int c = 0; c < nt[2]; ++c)
    for (int b = 0; b < nt[1]; ++b)
      for (int a = 0; a < nt[0]; ++a)
        s += w[0][a] * w[1][b] * w[2][c] * at(Lc, e, first[0] + a, first[1] + b, first[2] + c, bval);
  return s;
}

/* test access: prolong the coarse field e (nc) onto the fine grid (nf, each
 * direction equal or doubled), periodic (iso = 0) or with isolated zero-value
 * faces (iso = 1, the correction's boundary) */
void tref_mg_prolong(const int *nf, const int *nc, int iso, const double *e, double *out) {
  bc_t bc;
  memset(&bc, 0, sizeof bc);
  bc.iso = iso;
  level_t F = {{nf[0], nf[1], nf[2]}, {1.0, 1.0, 1.0}, NULL, NULL, NULL, &bc};
  level_t C = {{nc[0], nc[1], nc[2]}, {1.0, 1.0, 1.0}, NULL, NULL, NULL, &bc};
  for (int k = 0; k < nf[2]; ++k)
    for (int j = 0; j < nf[1]; ++j)
      for (int i = 0; i < nf[0]; ++i) out[idx3(&F, i, j, k)] = prolong_cell(&F, &C, e, i, j, k, 0);
}

static void vcycle(level_t *Ls, int l, int nl, int npre, int npost, double omega) {
  level_t *L = &Ls[l];
  if (l == nl - 1) {
    /* a single cell: periodic, the correction is zero; isolated, solved exactly */
    if (L->bc->iso) {
      double w[3];
      weights(L, w);
      const double diag = 2.0 * (w[0] + w[1] + w[2]);
      if (diag > 0.0) L->phi[0] = gs_value(L, w, diag, 0, 0, 0);
    }
    return;
  }
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
      for (int i = 0; i < L->n[0]; ++i) L->phi[idx3(L, i, j, k)] += prolong_cell(L, C, C->tmp, i, j, k, 0);
  for (int s = 0; s < npost; ++s) smooth(L, omega);
}

static double defect_rms(const level_t *L) {
  double s = 0.0;
  for (int k = 0; k < L->n[2]; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        const double d = L->src[idx3(L, i, j, k)] - apply_A(L, L->phi, i, j, k);
        s += d * d;
      }
  return sqrt(s / (double)ncell(L));
}

double tref_mg_defect_rms(int nx, int ny, int nz, const double *dx, const double *src, const double *phi) {
  bc_t bc;
  memset(&bc, 0, sizeof bc);
  level_t L = {{nx, ny, nz}, {dx[0], dx[1], dx[2]}, (double *)phi, (double *)src, NULL, &bc};
  return defect_rms(&L);
}

int tref_mg_solve_bc(int nx, int ny, int nz, const double *dx, const double *xmin, int isolated, int lmax,
                     const double *centre, int fmg, const double *src_in, double *phi, int max_cycles,
                     double tol, int npre, int npost, double omega, double *defect, double *defect_start,
                     int nq, const double *xq, double *phiq) {
  bc_t bc;
  memset(&bc, 0, sizeof bc);
  bc.iso = isolated;
  bc.lmax = lmax < 0 ? 0 : (lmax > MP_LMAX ? MP_LMAX : lmax);
  const int n0[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    bc.act[a] = n0[a] > 1;
    bc.x0[a] = xmin ? xmin[a] : 0.0;
  }
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
    L->bc = &bc;
    if (n[0] == 1 && n[1] == 1 && n[2] == 1) break;
    for (int a = 0; a < 3; ++a)
      if (n[a] > 1) { n[a] /= 2; h[a] *= 2.0; }
  }
  const int64_t nc0 = (int64_t)nx * ny * nz;
  memcpy(Ls[0].src, src_in, sizeof(double) * nc0);
  if (!isolated) {
    /* source without its mean, removed in two passes (one pass leaves a rounding
     * residual in the operator's null space) */
    for (int pass = 0; pass < 2; ++pass) {
      double m = 0.0;
      for (int64_t q = 0; q < nc0; ++q) m += Ls[0].src[q];
      m /= (double)nc0;
      for (int64_t q = 0; q < nc0; ++q) Ls[0].src[q] -= m;
    }
  } else {
    /* expansion centre: given, else the source-weighted centroid (the domain
     * centre for a source summing to zero) */
    double sw = 0.0, sx[3] = {0, 0, 0};
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          const double S = Ls[0].src[((int64_t)k * ny + j) * nx + i];
          const int g[3] = {i, j, k};
          sw += S;
          for (int a = 0; a < 3; ++a) sx[a] += S * (bc.x0[a] + (g[a] + 0.5) * dx[a]);
        }
    for (int a = 0; a < 3; ++a)
      bc.c[a] = centre ? centre[a] : (sw != 0.0 ? sx[a] / sw : bc.x0[a] + 0.5 * n0[a] * dx[a]);
    moments(&bc, &Ls[0]);
  }
  if (fmg) {
    /* the source on every level, the coarsest solved, then prolongation and one
     * V-cycle per finer level */
    for (int l = 1; l < nl; ++l)
      for (int K = 0; K < Ls[l].n[2]; ++K)
        for (int J = 0; J < Ls[l].n[1]; ++J)
          for (int I = 0; I < Ls[l].n[0]; ++I)
            Ls[l].src[idx3(&Ls[l], I, J, K)] = restrict_cell(&Ls[l - 1], &Ls[l], Ls[l - 1].src, I, J, K);
    memset(Ls[nl - 1].phi, 0, sizeof(double) * ncell(&Ls[nl - 1]));
    vcycle(Ls, nl - 1, nl, npre, npost, omega);
    for (int l = nl - 2; l >= 0; --l) {
      level_t *L = &Ls[l];
      /* (the V-cycle overwrites the sources of the levels below with its
       * full-approximation sources; this level's own is still the restriction) */
      for (int k = 0; k < L->n[2]; ++k)
        for (int j = 0; j < L->n[1]; ++j)
          for (int i = 0; i < L->n[0]; ++i)
            L->phi[idx3(L, i, j, k)] = prolong_cell(L, &Ls[l + 1], Ls[l + 1].phi, i, j, k, 1);
      vcycle(Ls, l, nl, npre, npost, omega);
      if (l == 0) smooth(L, omega);   /* the extra sweep on the finest level */
    }
  }
  int cycles = 0;
  double d = defect_rms(&Ls[0]);
  if (defect_start) *defect_start = d;
  while (cycles < max_cycles && !(d < tol)) {
    vcycle(Ls, 0, nl, npre, npost, omega);
    smooth(&Ls[0], omega);   /* the extra sweep on the finest level */
    ++cycles;
    d = defect_rms(&Ls[0]);
  }
  for (int q = 0; q < nq; ++q) phiq[q] = isolated ? multipole(&bc, xq + 3 * q) : 0.0;
  for (int l = 0; l < nl; ++l) {
    if (l > 0) free(Ls[l].phi);
    free(Ls[l].src);
    free(Ls[l].tmp);
  }
  if (defect) *defect = d;
  return cycles;
}

int tref_mg_solve(int nx, int ny, int nz, const double *dx, const double *src_in, double *phi,
                  int max_cycles, double tol, int npre, int npost, double omega, double *defect) {
  return tref_mg_solve_bc(nx, ny, nz, dx, NULL, 0, 0, NULL, 0, src_in, phi, max_cycles, tol, npre, npost, omega,
                          defect, NULL, 0, NULL, NULL);
}
