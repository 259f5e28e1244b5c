// tde_device.cuh -- device-side building blocks of the hydro stage: the
// tabulated-EOS inversion, conserved -> primitive recovery with the dual-energy
// switch, PLM / PPM face reconstruction and the HLLC Riemann solver.
//
// Every routine is a per-cell or per-face function in registers; the kernels in
// tde_hydro.cu stage the data through shared memory and call them.  The FP64
// pipe is the limiting resource of this path on sm_103a (FP64 FMA issues at
// about 1/55 of the FP32 rate), so the routines avoid divisions where an algebraically
// equal form with fewer of them exists, and never branch on the Riemann wave
// pattern (a warp that diverged would pay for every branch).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tde {

enum { EOS_IDEAL = 0, EOS_TABLE = 1 };
enum { PLM = 0, PPM = 1 };

// Tabulated EOS on a uniform (log10 rho, log10 T) grid, [n_rho][n_T], cgs.
struct DTable {
  int nr, nt;
  double lr0, inv_dlr, lt0, dlt;
  const double *__restrict__ le;   // log10 e
  const double *__restrict__ lp;   // log10 P
  const double *__restrict__ lc;   // log10 cs^2
};

struct Counters {
  unsigned long long rho_floor, p_floor, u_floor, table_clamp, excised, dual_aux_used, synced,
      nonfinite, surrogate_accepted;
};

// Scheme, physics and geometry constants, passed by value to every kernel.
struct Phys {
  int eos, recon, dual, nvar, nwv;
  double gamma, gm1, inv_gm1, eta1, eta2;
  double rho_floor, p_floor, u_floor;
  double unit_rho, unit_e, inv_unit_p, inv_unit_e;
  DTable tab;
  int N[3], bc[3], active[3], g[3], ng;
  double xmin[3], dx[3], idx[3], dxmin;
};

struct BH {
  int on, excise;
  double GM, rs2, rexc, t0, x0[3], v0[3], a0[3];
};

// padded geometry of one MeshBlock
struct DevBlock {
  int i0, j0, k0, n[3], p[3], pad;
  long long off;
};

__device__ __forceinline__ void count(unsigned long long *c) {
  if (c) atomicAdd(c, 1ull);
}

// 1/d by Newton-Raphson (x <- x (2 - d x), written as two FMAs per step) from
// the hardware's approximate double reciprocal; two steps take the seed's
// ~2^-23 relative error below the FP64 rounding, so the result is within about
// one ulp of 1/d.  For normal d whose reciprocal is normal (every use below:
// sums of same-signed slopes, wave-speed differences, densities).
__device__ __forceinline__ double rcp_nr(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// ---------------------------------------------------------------- EOS ----

// Density cell i and weight w of log10 rho (clamped to the table).
__device__ __forceinline__ bool rho_cell(const DTable &t, double rho, int &i, double &w) {
  double x = (log10(rho) - t.lr0) * t.inv_dlr;
  bool cl = false;
  if (!(x >= 0.0)) { x = 0.0; cl = true; }
  if (x > (double)(t.nr - 1)) { x = (double)(t.nr - 1); cl = true; }
  int ii = (int)floor(x);
  if (ii > t.nr - 2) ii = t.nr - 2;
  i = ii;
  w = x - ii;
  return cl;
}

__device__ __forceinline__ double bilin(const double *__restrict__ f, int nt, int i, double w, int j,
                                        double s) {
  const double *a = f + (size_t)i * nt + j;
  const double *b = a + nt;
  double lo = (1.0 - s) * __ldg(a) + s * __ldg(a + 1);
  double hi = (1.0 - s) * __ldg(b) + s * __ldg(b + 1);
  return (1.0 - w) * lo + w * hi;
}

// (rho, e) -> P, cs2 (cgs) by binary search of the interpolated log10 e column
// at fixed density weight, then an exact linear solve inside the cell
// (Sec. 4.2, runtime map).  Returns true if the input was clamped to the table
// edge; then *e_used is the table's e at the clamped point.  WANT_CS2 = false
// computes P only (cs2, T and e_used are left untouched).
template <bool WANT_CS2 = true>
__device__ __forceinline__ bool eos_invert(const DTable &t, double rho, double e, double &P,
                                           double &cs2, double &e_used, double *T = nullptr) {
  int i;
  double w;
  bool cl = rho_cell(t, rho, i, w);
  const int nt = t.nt;
  const double *__restrict__ a = t.le + (size_t)i * nt;
  const double *__restrict__ b = a + nt;
  const double w1 = 1.0 - w;
  double glo = w1 * __ldg(a) + w * __ldg(b);
  double ghi = w1 * __ldg(a + nt - 1) + w * __ldg(b + nt - 1);
  double y = e > 0.0 ? log10(e) : -INFINITY;
  int j;
  double s;
  if (!(y > glo)) {
    j = 0; s = 0.0; cl = true;
  } else if (y >= ghi) {
    j = nt - 2; s = 1.0; cl = true;
  } else {
    int lo = 0, hi = nt - 1;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      double g = w1 * __ldg(a + mid) + w * __ldg(b + mid);
      if (g <= y) lo = mid; else hi = mid;
    }
    j = lo;
    double g0 = w1 * __ldg(a + j) + w * __ldg(b + j);
    double g1 = w1 * __ldg(a + j + 1) + w * __ldg(b + j + 1);
    s = (y - g0) / (g1 - g0);
  }
  P = exp10(bilin(t.lp, nt, i, w, j, s));
  if (WANT_CS2) {
    cs2 = exp10(bilin(t.lc, nt, i, w, j, s));
    if (T) *T = exp10(t.lt0 + (j + s) * t.dlt);
    e_used = cl ? exp10(bilin(t.le, nt, i, w, j, s)) : e;
  }
  return cl;
}

// EOS closure in code units: internal energy density U at density rho ->
// P, cs^2 and the internal energy the table actually represents.
template <int EOSK>
__device__ __forceinline__ void eos_closure(const Phys &p, double rho, double U, double &P,
                                            double &cs2, double &Uu, Counters *cnt) {
  if (EOSK == EOS_IDEAL) {
    P = p.gm1 * U;
    cs2 = p.gamma * P / rho;
    Uu = U;
  } else {
    double Pc, c2c, eu;
    bool cl = eos_invert(p.tab, rho * p.unit_rho, (U / rho) * p.unit_e, Pc, c2c, eu);
    if (cl && cnt) count(&cnt->table_clamp);
    P = Pc * p.inv_unit_p;
    cs2 = c2c * p.inv_unit_e;
    Uu = cl ? rho * (eu * p.inv_unit_e) : U;
  }
}

// Pressure of internal energy density U at density rho (code units), table EOS
// (the compression source of Eq. dual-tabulated-compression needs P only).
__device__ __forceinline__ double table_pressure(const Phys &p, double rho, double U,
                                                 Counters *cnt) {
  double Pc, c2c, eu;
  bool cl = eos_invert<false>(p.tab, rho * p.unit_rho, (U / rho) * p.unit_e, Pc, c2c, eu);
  if (cl && cnt) count(&cnt->table_clamp);
  return Pc * p.inv_unit_p;
}

// Conserved (rho, m, E[, U_aux]) -> primitives w = (rho, vx, vy, vz, P
// [, Gamma_e, Gamma_1][, U_aux]) with the dual-energy switch of
// Eq. dual-primitive-switch and the density / pressure floors.
template <int EOSK, int DUAL>
__device__ __forceinline__ void cons_to_prim(const Phys &p, const double *u, double *w,
                                             Counters *cnt) {
  double rho = u[0];
  if (rho < p.rho_floor) { rho = p.rho_floor; if (cnt) count(&cnt->rho_floor); }
  double ir = 1.0 / rho;
  double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  double Uc = u[4] - 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz);   // Eq. dual-econs
  double Ue = Uc;
  if (DUAL) {
    if (!(Uc > 0.0 && Uc > p.eta1 * u[4])) { Ue = u[5]; if (cnt) count(&cnt->dual_aux_used); }
  }
  double P, cs2, Uu;
  eos_closure<EOSK>(p, rho, Ue, P, cs2, Uu, cnt);
  if (P < p.p_floor) { P = p.p_floor; if (cnt) count(&cnt->p_floor); }
  w[0] = rho; w[1] = vx; w[2] = vy; w[3] = vz; w[4] = P;
  if (EOSK == EOS_TABLE) {
    w[5] = 1.0 + P / Uu;          // Gamma_e
    w[6] = rho * cs2 / P;         // Gamma_1
    if (DUAL) w[7] = u[5];
  } else {
    if (DUAL) w[5] = u[5];
  }
}

// ------------------------------------------------------- reconstruction ----

// PLM, van Leer limiter: half-slope h = dl dr / (dl + dr) if dl dr > 0; faces q -+ h
__device__ __forceinline__ void plm(double qm, double q0, double qp, double &left, double &right) {
  double dl = q0 - qm, dr = qp - q0;
  double pr = dl * dr;
  double h = (pr > 0.0) ? pr * rcp_nr(dl + dr) : 0.0;
  left = q0 - h;
  right = q0 + h;
}

// PPM: 4th-order interface value between q0 and q1, clipped to [q0, q1]
__device__ __forceinline__ double ppm_iface(double qm1, double q0, double q1, double q2) {
  double a = (7.0 / 12.0) * (q0 + q1) - (1.0 / 12.0) * (qm1 + q2);
  double lo = fmin(q0, q1), hi = fmax(q0, q1);
  return fmin(fmax(a, lo), hi);
}

// Colella-Woodward (1984) monotonicity constraints on the parabola (aL, q0, aR)
__device__ __forceinline__ void ppm_limit(double q0, double &aL, double &aR) {
  if ((aR - q0) * (q0 - aL) <= 0.0) {
    aL = q0;
    aR = q0;
  } else {
    double da = aR - aL;
    double q6 = 6.0 * (q0 - 0.5 * (aL + aR));
    if (da * q6 > da * da) aL = 3.0 * q0 - 2.0 * aR;
    else if (-(da * da) > da * q6) aR = 3.0 * q0 - 2.0 * aL;
  }
}

// ------------------------------------------------------------------ HLLC ----

// Face state: rho, v[3], P, Gamma_e (or gamma), Gamma_1 (or gamma), U_aux.
struct FState {
  double r, v[3], P, ge, g1, A;
};

// HLLC flux across a face normal to direction D (Toro, Spruce & Speares) with
// Davis wave-speed estimates; F[0..4] = mass, momentum, energy; F[5] = U_aux
// flux (Eq. dual-flux); vf = face velocity (Eq. dual-face-velocity).  The wave
// pattern is selected without branching on it.
template <int D, int EOSK, int DUAL>
__device__ __forceinline__ void hllc(const Phys &p, const FState &L, const FState &R, double *F,
                                     double &vf) {
  const int t1 = D == 0 ? 1 : 0, t2 = D == 2 ? 1 : 2;
  double ul = L.v[D], ur = R.v[D];
  double cl = sqrt(L.g1 * L.P / L.r), cr = sqrt(R.g1 * R.P / R.r);
  double Ul = EOSK == EOS_IDEAL ? L.P * p.inv_gm1 : L.P / (L.ge - 1.0);
  double Ur = EOSK == EOS_IDEAL ? R.P * p.inv_gm1 : R.P / (R.ge - 1.0);
  double El = Ul + 0.5 * L.r * (L.v[0] * L.v[0] + L.v[1] * L.v[1] + L.v[2] * L.v[2]);
  double Er = Ur + 0.5 * R.r * (R.v[0] * R.v[0] + R.v[1] * R.v[1] + R.v[2] * R.v[2]);
  double SL = fmin(ul - cl, ur - cr);
  double SR = fmax(ul + cl, ur + cr);
  double al = L.r * (SL - ul), ar = R.r * (SR - ur);
  double SM = (R.P - L.P + al * ul - ar * ur) * rcp_nr(al - ar);
  bool supL = SL >= 0.0, supR = SR <= 0.0;
  bool useL = supL || (!supR && SM >= 0.0);
  // chosen side K
  double r = useL ? L.r : R.r, un = useL ? ul : ur, P = useL ? L.P : R.P, E = useL ? El : Er;
  double vt1 = useL ? L.v[t1] : R.v[t1], vt2 = useL ? L.v[t2] : R.v[t2];
  double S = useL ? SL : SR;
  double Seff = (supL || supR) ? 0.0 : S;
  double den = S - SM;
  if (den == 0.0) den = 1.0;   // only reachable when Seff == 0
  double rS = r * (S - un);
  double inv = rcp_nr(den);
  double fac = rS * inv;
  double mflux = r * un;
  // U*_K - U_K and F_K in the (normal, t1, t2) frame
  double d0 = fac - r;
  double dn = fac * SM - mflux;
  double d1 = (fac - r) * vt1;
  double d2 = (fac - r) * vt2;
  double Es = (E * (S - un) + (SM - un) * (rS * SM + P)) * inv;
  double dE = Es - E;
  F[0] = mflux + Seff * d0;
  double Fn = mflux * un + P + Seff * dn;
  double F1 = mflux * vt1 + Seff * d1;
  double F2 = mflux * vt2 + Seff * d2;
  F[1 + D] = Fn;
  F[1 + t1] = F1;
  F[1 + t2] = F2;
  F[4] = (E + P) * un + Seff * dE;
  if (DUAL) {
    double f = F[0];
    bool up = f > 0.0;
    double ru = up ? L.r : R.r, Au = up ? L.A : R.A;
    double iru = rcp_nr(ru);
    F[5] = f != 0.0 ? f * (Au * iru) : 0.0;
    vf = f != 0.0 ? f * iru : 0.0;
  } else {
    F[5] = 0.0;
    vf = 0.0;
  }
}

}  // namespace tde
