/*
 * tref_eos.c -- ORACLE (test infrastructure only): the tabulated H/He equation
 * of state.
 *
 * Sec. 4.2 of the paper builds a (ln rho, ln T) table of ln P, ln e_th, ln cs^2,
 * Gamma_1, ... for X = 0.7, Y = 0.3 and, at run time, maps (rho, U_EOS) to the
 * thermodynamic state by interpolation inside the table.  The paper's own table
 * (Tomida/Chabrier/HELM) is not available; this file generates a table from
 * Saha ionisation equilibrium of H, H+, He, He+, He2+ and free electrons, with
 * photon radiation added as in Eq. eos-radiation (P_rad = a T^4 / 3,
 * e_rad = a T^4 / rho).  Molecules and non-ideal terms are absent.
 *
 * Readings:
 *  - Saha ratios n_{i+1} n_e / n_i = G (2 pi m_e k T / h^2)^{3/2} exp(-chi / kT)
 *    with G = 2 g_{i+1} / g_i = 1 (H), 4 (He -> He+), 1 (He+ -> He2+).
 *  - Charge neutrality is solved by bisection in ln n_e.
 *  - Gamma_1 = chi_rho + chi_T^2 P / (rho T c_v) with centred differences of
 *    step 1e-4 in ln rho and ln T; cs^2 = Gamma_1 P / rho (Eq. eos-adiabatic-derivatives).
 *  - Interpolation is bilinear in (log10 rho, log10 T) of log10 e, log10 P and
 *    log10 cs^2.  Inversion keeps the density weight w fixed, so that along T
 *    the interpolated log10 e is a piecewise-linear strictly increasing function
 *    g(j + t); the cell j with g_j <= y < g_{j+1} is found and t solved exactly.
 *    Out-of-range input is clamped to the table edge and reported.
 */
#include "tref.h"
#include <math.h>

/* CODATA 2018 (cgs) */
static const double K_B = 1.380649e-16;          /* erg / K */
static const double H_PL = 6.62607015e-27;       /* erg s */
static const double M_E = 9.1093837015e-28;      /* g */
static const double M_U = 1.66053906660e-24;     /* g */
static const double EV = 1.602176634e-12;        /* erg */
static const double A_RAD = 7.565733250e-15;     /* erg cm^-3 K^-4, 4 sigma_SB / c */
static const double PI = 3.14159265358979323846;
/* standard atomic weights */
static const double A_H = 1.00794, A_HE = 4.002602;
/* ionisation potentials (eV) */
static const double CHI_H = 13.598434, CHI_HE1 = 24.587389, CHI_HE2 = 54.417765;

/* Saha ratio S = G lambda^-3 exp(-chi / kT) in cm^-3. */
static double saha_ratio(double G, double chi_ev, double T) {
  double kT = K_B * T;
  double lam = pow(2.0 * PI * M_E * kT / (H_PL * H_PL), 1.5);
  return G * lam * exp(-chi_ev * EV / kT);
}

/* He+ and He2+ fractions for electron density ne: the three stages stand in the
 * ratios 1 : S1/ne : S1 S2 / ne^2, normalised in logarithms so that no
 * intermediate overflows or underflows to 0/0. */
static void he_fractions(double S1, double S2, double ne, double *y1, double *y2) {
  double l1 = log(S1) - log(ne);
  double l2 = l1 + log(S2) - log(ne);
  double lm = 0.0;
  if (l1 > lm) lm = l1;
  if (l2 > lm) lm = l2;
  double e0 = exp(-lm), e1 = exp(l1 - lm), e2 = exp(l2 - lm);
  double s = e0 + e1 + e2;
  *y1 = e1 / s;
  *y2 = e2 / s;
}

void tref_saha_state(double rho, double T, double X, double Y, double *out) {
  double nH = X * rho / (A_H * M_U);
  double nHe = Y * rho / (A_HE * M_U);
  double SH = saha_ratio(1.0, CHI_H, T);
  double S1 = saha_ratio(4.0, CHI_HE1, T);
  double S2 = saha_ratio(1.0, CHI_HE2, T);
  /* f(ne) = supplied electrons - ne, strictly decreasing in ne */
  double lo = log(1e-300), hi = log(nH + 2.0 * nHe);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double ne = exp(mid);
    double xH = SH / (SH + ne), y1, y2;
    he_fractions(S1, S2, ne, &y1, &y2);
    double f = nH * xH + nHe * (y1 + 2.0 * y2) - ne;
    if (f > 0.0) lo = mid; else hi = mid;
  }
  double ne = exp(0.5 * (lo + hi));
  double xH = SH / (SH + ne), y1, y2;
  he_fractions(S1, S2, ne, &y1, &y2);
  double nnuc = nH + nHe;
  double kT = K_B * T;
  double Pgas = (nnuc + ne) * kT;
  double Prad = A_RAD * T * T * T * T / 3.0;
  double eion = nH * xH * CHI_H * EV + nHe * (y1 * CHI_HE1 + y2 * (CHI_HE1 + CHI_HE2)) * EV;
  double uden = 1.5 * (nnuc + ne) * kT + eion + A_RAD * T * T * T * T;
  out[0] = Pgas + Prad;
  out[1] = uden / rho;
  out[2] = ne;
  out[3] = xH;
  out[4] = y1;
  out[5] = y2;
  out[6] = rho / ((nnuc + ne) * M_U);
  out[7] = Pgas;
  out[8] = nnuc;
}

/* Pure hydrogen: ne^2 = S (nH - ne)  ->  ne = (-S + sqrt(S^2 + 4 S nH)) / 2. */
double tref_saha_pure_h_xe(double rho, double T) {
  double nH = rho / (A_H * M_U);
  double S = saha_ratio(1.0, CHI_H, T);
  double ne = 0.5 * (-S + sqrt(S * S + 4.0 * S * nH));
  return ne / nH;
}

void tref_eos_build(int n_rho, int n_T, double lrho_min, double lrho_max, double lT_min,
                    double lT_max, double X, double Y, double *log10_e, double *log10_P,
                    double *log10_cs2, double *gamma1) {
  const double h = 1e-4;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n_rho; ++i) {
    double lr = lrho_min + (lrho_max - lrho_min) * i / (n_rho - 1);
    double rho = pow(10.0, lr);
    for (int j = 0; j < n_T; ++j) {
      double lt = lT_min + (lT_max - lT_min) * j / (n_T - 1);
      double T = pow(10.0, lt);
      double s0[9], rp[9], rm[9], tp[9], tm[9];
      tref_saha_state(rho, T, X, Y, s0);
      tref_saha_state(rho * exp(h), T, X, Y, rp);
      tref_saha_state(rho * exp(-h), T, X, Y, rm);
      tref_saha_state(rho, T * exp(h), X, Y, tp);
      tref_saha_state(rho, T * exp(-h), X, Y, tm);
      double chi_rho = (log(rp[0]) - log(rm[0])) / (2.0 * h);
      double chi_T = (log(tp[0]) - log(tm[0])) / (2.0 * h);
      double cv = (tp[1] - tm[1]) / (T * exp(h) - T * exp(-h));
      double P = s0[0];
      double g1 = chi_rho + chi_T * chi_T * P / (rho * T * cv);
      log10_e[i * n_T + j] = log10(s0[1]);
      log10_P[i * n_T + j] = log10(P);
      log10_cs2[i * n_T + j] = log10(g1 * P / rho);
      if (gamma1) gamma1[i * n_T + j] = g1;
    }
  }
}

/* density cell and weight; returns 1 if rho lies outside the table */
static int rho_cell(const tref_table *t, double rho, int *i, double *w) {
  double d = (t->lrho_max - t->lrho_min) / (t->n_rho - 1);
  double x = (log10(rho) - t->lrho_min) / d;
  int clamped = 0;
  if (!(x >= 0.0)) { x = 0.0; clamped = 1; }
  if (x > (double)(t->n_rho - 1)) { x = (double)(t->n_rho - 1); clamped = 1; }
  int ii = (int)floor(x);
  if (ii > t->n_rho - 2) ii = t->n_rho - 2;
  *i = ii;
  *w = x - ii;
  return clamped;
}

static double bilin(const double *f, int nT, int i, double w, int j, double s) {
  return (1.0 - w) * ((1.0 - s) * f[i * nT + j] + s * f[i * nT + j + 1]) +
         w * ((1.0 - s) * f[(i + 1) * nT + j] + s * f[(i + 1) * nT + j + 1]);
}

void tref_eos_eval_rhoT(const tref_table *t, double rho, double T, double *P, double *e, double *cs2) {
  int i; double w;
  rho_cell(t, rho, &i, &w);
  double d = (t->lT_max - t->lT_min) / (t->n_T - 1);
  double y = (log10(T) - t->lT_min) / d;
  if (!(y >= 0.0)) y = 0.0;
  if (y > (double)(t->n_T - 1)) y = (double)(t->n_T - 1);
  int j = (int)floor(y);
  if (j > t->n_T - 2) j = t->n_T - 2;
  double s = y - j;
  *P = pow(10.0, bilin(t->log10_P, t->n_T, i, w, j, s));
  *e = pow(10.0, bilin(t->log10_e, t->n_T, i, w, j, s));
  *cs2 = pow(10.0, bilin(t->log10_cs2, t->n_T, i, w, j, s));
}

/* tref_eos_eval_rhoT on n cells (arrays; outputs may be NULL), OpenMP over cells. */
void tref_eos_eval_rhoT_n(const tref_table *t, int64_t n, const double *rho, const double *T, double *P,
                          double *e, double *cs2) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < n; ++q) {
    double p, en, c2;
    tref_eos_eval_rhoT(t, rho[q], T[q], &p, &en, &c2);
    if (P) P[q] = p;
    if (e) e[q] = en;
    if (cs2) cs2[q] = c2;
  }
}

int tref_eos_invert(const tref_table *t, double rho, double e, double *T, double *P, double *cs2,
                    double *e_used) {
  int i; double w;
  int clamped = rho_cell(t, rho, &i, &w);
  const int nT = t->n_T;
  const double *le = t->log10_e;
  int j;
  double s;
  double glo = (1.0 - w) * le[i * nT] + w * le[(i + 1) * nT];
  double ghi = (1.0 - w) * le[i * nT + nT - 1] + w * le[(i + 1) * nT + nT - 1];
  double y = (e > 0.0) ? log10(e) : -HUGE_VAL;
  if (!(y > glo)) {           /* below the coldest column entry (or e <= 0) */
    j = 0; s = 0.0; clamped = 1;
  } else if (y >= ghi) {      /* above the hottest entry */
    j = nT - 2; s = 1.0; clamped = 1;
  } else {
    /* plain scan for the cell with g_j <= y < g_{j+1} */
    j = 0;
    for (int jj = 0; jj < nT - 1; ++jj) {
      double g = (1.0 - w) * le[i * nT + jj + 1] + w * le[(i + 1) * nT + jj + 1];
      if (g <= y) j = jj + 1; else break;
    }
    double g0 = (1.0 - w) * le[i * nT + j] + w * le[(i + 1) * nT + j];
    double g1 = (1.0 - w) * le[i * nT + j + 1] + w * le[(i + 1) * nT + j + 1];
    s = (y - g0) / (g1 - g0);
  }
  double d = (t->lT_max - t->lT_min) / (nT - 1);
  *T = pow(10.0, t->lT_min + (j + s) * d);
  *P = pow(10.0, bilin(t->log10_P, nT, i, w, j, s));
  *cs2 = pow(10.0, bilin(t->log10_cs2, nT, i, w, j, s));
  if (e_used) *e_used = clamped ? pow(10.0, bilin(le, nT, i, w, j, s)) : e;
  return clamped;
}

double tref_eos_T_from_P(const tref_table *t, double rho, double P) {
  /* bisection on T of the bilinear pressure (initial data only) */
  double lo = t->lT_min, hi = t->lT_max;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double Pm, em, cm;
    tref_eos_eval_rhoT(t, rho, pow(10.0, mid), &Pm, &em, &cm);
    if (Pm < P) lo = mid; else hi = mid;
  }
  return pow(10.0, 0.5 * (lo + hi));
}

/* Learned-guess inversion (the project's addition to the runtime map of
 * Sec. 4.2): the guessed log10 T is placed in its temperature cell j (clamped
 * to the table) of the interpolated log10 e column g at the density weight of
 * rho.  g is linear inside a cell, so one Newton step from the guess lands on
 * x = j + t, t = (y - g_j) / (g_{j+1} - g_j).  If g_j <= y < g_{j+1} that is the
 * root; otherwise x lies in cell j' = floor(x), and if the column brackets y
 * there the root is taken in j'.  Either way the cell is the unique one that
 * bisection finds and the state is evaluated with the same formulas as
 * tref_eos_invert, so the result is the bisection result itself.  Otherwise (a
 * step that misses, a clamped input) the plain inversion is used.  Returns 1 if
 * the guess was accepted. */
static double column(const tref_table *t, int i, double w, int j) {
  const int nT = t->n_T;
  return (1.0 - w) * t->log10_e[i * nT + j] + w * t->log10_e[(i + 1) * nT + j];
}

int tref_eos_invert_guess(const tref_table *t, double rho, double e, double log10_T_guess,
                          double *T, double *P, double *cs2) {
  int i; double w;
  int clamped = rho_cell(t, rho, &i, &w);
  const int nT = t->n_T;
  double glo = column(t, i, w, 0), ghi = column(t, i, w, nT - 1);
  double y = (e > 0.0) ? log10(e) : -HUGE_VAL;
  double d = (t->lT_max - t->lT_min) / (nT - 1);
  int accepted = 0;
  if (!clamped && y > glo && y < ghi) {
    double xj = (log10_T_guess - t->lT_min) / d;
    if (!(xj >= 0.0)) xj = 0.0;
    if (xj > (double)(nT - 2)) xj = (double)(nT - 2);
    int j = (int)floor(xj);
    double g0 = column(t, i, w, j), g1 = column(t, i, w, j + 1);
    int in = g0 <= y && y < g1;
    if (!in) {
      double x = j + (y - g0) / (g1 - g0);   /* the Newton result */
      if (x >= 0.0 && x < (double)(nT - 1) && (int)floor(x) != j) {
        j = (int)floor(x);
        g0 = column(t, i, w, j);
        g1 = column(t, i, w, j + 1);
        in = g0 <= y && y < g1;
      }
    }
    if (in) {
      double s = (y - g0) / (g1 - g0);
      *T = pow(10.0, t->lT_min + (j + s) * d);
      *P = pow(10.0, bilin(t->log10_P, nT, i, w, j, s));
      *cs2 = pow(10.0, bilin(t->log10_cs2, nT, i, w, j, s));
      accepted = 1;
    }
  }
  if (!accepted) {
    double eu;
    tref_eos_invert(t, rho, e, T, P, cs2, &eu);
  }
  return accepted;
}
