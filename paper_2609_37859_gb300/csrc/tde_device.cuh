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
enum { RIEMANN_HLLC = 0, RIEMANN_HLLE = 1 };

// ------------------------------------- comparisons on the integer pipe ----
//
// A double's bit pattern, read as a signed 64-bit integer, orders positive
// values like the values themselves; flipping the magnitude bits of negative
// patterns extends that to a total order (-0 just below +0).  Comparisons,
// minima and maxima written this way run on the integer ALUs, which sit idle
// while the FP64 pipe (where DSETP and DMNMX would issue) bounds the path.
// For NaN operands they are not the IEEE predicates; the kernels count
// non-finite states rather than rely on comparisons with NaN.

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// order key: key(a) < key(b) iff a < b for non-NaN a, b (except -0 < +0)
__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// the same with -0 and +0 equal (the IEEE order of non-NaN values)
__device__ __forceinline__ long long dkey0(double x) {
  const long long k = dkey(x);
  return k < 0 ? k + 1 : k;
}
__device__ __forceinline__ bool dgt0(double x) { return dbits(x) > 0; }          // x > 0
__device__ __forceinline__ bool dge0(double x) { return dkey(x) >= -1; }         // x >= 0 (incl. -0)
__device__ __forceinline__ bool dle0(double x) { return dkey(x) <= 0; }          // x <= 0 (incl. +0)
__device__ __forceinline__ bool dzero(double x) { return (dbits(x) << 1) == 0; }  // x == +-0
__device__ __forceinline__ bool dlt(double a, double b) { return dkey(a) < dkey(b); }
__device__ __forceinline__ bool dle(double a, double b) { return dkey(a) <= dkey(b); }
__device__ __forceinline__ double dmin(double a, double b) { return dkey(a) <= dkey(b) ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return dkey(a) >= dkey(b) ? a : b; }
__device__ __forceinline__ bool dfinite(double x) { return ((dbits(x) >> 52) & 0x7ff) != 0x7ff; }
// the double value of a small integer |k| < 2^51, by one FP64 add
__device__ __forceinline__ double dint(long long k) {
  return __longlong_as_double(0x4338000000000000LL + k) - 6755399441055744.0;
}
// x truncated to FP32 on the integer pipe (a guide value: normal x with
// 2^-126 <= |x| < 2^128, or zero)
__device__ __forceinline__ float d2f_guide(double x) {
  const long long b = dbits(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return 0.0f;
  const unsigned u = (unsigned)((b >> 32) & 0x80000000u) | ((unsigned)e << 23) |
                     (unsigned)((b >> 29) & 0x7fffff);
  return __uint_as_float(u);
}

// ------------------------------------------------ log10 / exp10 (FP64) ----
//
// Table-driven logarithm and exponential after P. T. P. Tang (ACM TOMS 15, 1989:
// exp; ACM TOMS 16, 1990: log), written for this library: an exact argument
// reduction onto one of 128 table points, a short polynomial of the small
// remainder, and a split (Cody-Waite) constant so that the reduction adds no
// rounding.  Fewer FP64 instructions than the general-purpose routines; within
// a few units in the last place (checked against CUDA's log10 / exp10 by
// tde_math_selftest).  Arguments outside the normal range go to the library.

struct MathTables {
  double logF[182];    // ln(j/128), j = 90 .. 181 (the reduced argument's table points)
  double invF[182];    // 128 / j
  double F[182];       // j / 128
  double exp2j[128];   // 2^(j/128)
};

__device__ __forceinline__ double fast_log10(const MathTables *__restrict__ mt, double x) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7ff);
  if (ex == 0 || ex == 0x7ff || bits < 0) return log10(x);
  // x = 2^k m with m in [sqrt(1/2), sqrt(2)) (no cancellation near x = 1), and
  // m = F (1 + r) with F = j/128 the nearest table point, m - F exact
  const long long mant = bits & 0x000fffffffffffffLL;
  const bool upper = mant >= 0x6a09e667f3bcdLL;            // m0 = 1 + mant 2^-52 >= sqrt(2)
  const int k = upper ? ex - 1022 : ex - 1023;
  const double m = __longlong_as_double(mant | (upper ? 0x3fe0000000000000LL : 0x3ff0000000000000LL));
  const int j = upper ? 64 + (int)((mant + (1LL << 45)) >> 46) : 128 + (int)((mant + (1LL << 44)) >> 45);
  const double F = __ldg(&mt->F[j]);
  const double r = __dmul_rn(__dsub_rn(m, F), __ldg(&mt->invF[j]));    // |r| <= 2^-7.5
  // ln(1 + r) = r - r^2/2 + ... + r^7/7 (the next term, r^8/8, is below 2^-55.5
  // relative to the result for |r| <= 2^-7.5)
  double q = 1.0 / 7.0;
  q = __fma_rn(q, r, -1.0 / 6.0);
  q = __fma_rn(q, r, 1.0 / 5.0);
  q = __fma_rn(q, r, -1.0 / 4.0);
  q = __fma_rn(q, r, 1.0 / 3.0);
  q = __fma_rn(q, r, -0.5);
  const double lp = __fma_rn(__dmul_rn(q, r), r, r);
  const double kd = dint(k);
  const double ln2_hi = 0.6931471803691238;   // 32 significant bits: k * ln2_hi is exact
  const double ln2_lo = 1.9082149292705877e-10;
  const double hi = __fma_rn(kd, ln2_hi, __ldg(&mt->logF[j]));
  const double lo = __fma_rn(kd, ln2_lo, lp);
  return __dmul_rn(__dadd_rn(hi, lo), 0.4342944819032518);   // log10(e)
}

__device__ __forceinline__ double fast_exp10(const MathTables *__restrict__ mt, double x) {
  if (!((dbits(x) & 0x7fffffffffffffffLL) < dbits(300.0))) return exp10(x);   // |x| < 300
  // 10^x = 2^(n/128) 10^r with n = round(128 x log2 10), r = x - n log10(2)/128;
  // adding 1.5 2^52 rounds to an integer in the low mantissa bits
  const double big = __fma_rn(x, 425.20679614558236, 6755399441055744.0);   // 128 log2(10)
  const double n = __dsub_rn(big, 6755399441055744.0);
  const double c_hi = 0.002351796840230236;   // log10(2)/128, 32 significant bits
  const double c_lo = 8.946172576579561e-13;
  const double r = __fma_rn(-n, c_lo, __fma_rn(-n, c_hi, x));   // |r| <= log10(2)/256
  const double u = __dmul_rn(r, 2.302585092994046);             // ln 10
  // e^u - 1 = u + u^2/2 + ... + u^5/120, |u| <= 2.7e-3 (the next term, u^6/720,
  // is below 2^-60 relative to the result)
  double q = 1.0 / 120.0;
  q = __fma_rn(q, u, 1.0 / 24.0);
  q = __fma_rn(q, u, 1.0 / 6.0);
  q = __fma_rn(q, u, 0.5);
  const double eu = __fma_rn(__dmul_rn(q, u), u, u);
  const int ni = (int)dbits(big);   // n, from the low bits
  const int jj = ni & 127, kk = ni >> 7;
  const double tj = __ldg(&mt->exp2j[jj]);
  const double v = __fma_rn(tj, eu, tj);   // 2^(jj/128) e^u
  return __longlong_as_double(__double_as_longlong(v) + ((long long)kk << 52));
}

// Tabulated EOS on a uniform (log10 rho, log10 T) grid, [n_rho][n_T], cgs.
struct DTable {
  int nr, nt;
  double lr0, inv_dlr, lt0, dlt;
  double xr_max;                   // nr - 1 (the largest density coordinate)
  const double *__restrict__ le;   // log10 e
  const double *__restrict__ lp;   // log10 P
  const double *__restrict__ lc;   // log10 cs^2
  const float *__restrict__ le32;  // log10 e rounded to FP32 (guides the search)
  const MathTables *__restrict__ mt;   // tables of fast_log10 / fast_exp10 (or null)
};

__device__ __forceinline__ double tlog10(const DTable &t, double x) {
  return t.mt ? fast_log10(t.mt, x) : log10(x);
}
__device__ __forceinline__ double texp10(const DTable &t, double x) {
  return t.mt ? fast_exp10(t.mt, x) : exp10(x);
}

struct Counters {
  unsigned long long rho_floor, p_floor, u_floor, table_clamp, excised, dual_aux_used, synced,
      nonfinite, surrogate_accepted;
};

// Scheme, physics and geometry constants, passed by value to every kernel.
struct Phys {
  int eos, recon, dual, nvar, nwv;
  int eos_mode;   // TDE_INVERT_*: how the table is inverted (the results are identical)
  int riemann;    // RIEMANN_HLLC or RIEMANN_HLLE
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
  int frame;          // inertial source of the accelerating frame
  double afr[3];
};

// padded geometry of one MeshBlock; origin (i0, j0, k0) on its level's grid
struct DevBlock {
  int i0, j0, k0, n[3], p[3], level;
  long long off;
};

// 2^e for |e| < 1000, exact (built from the exponent field)
__host__ __device__ __forceinline__ double exp2i(int e) {
  unsigned long long b = (unsigned long long)(1023 + e) << 52;
  double r;
  memcpy(&r, &b, 8);
  return r;
}

// x 2^e for a normal x whose result is normal: an integer add on the exponent
// field (exact, and no FP64 instruction)
__device__ __forceinline__ double scale2i(double x, int e) {
  return __longlong_as_double(__double_as_longlong(x) + ((long long)e << 52));
}

// cell width, its reciprocal and the grid size along a on block B's level
// (refinement halves the cells of the active directions only)
__device__ __forceinline__ double block_dx(const Phys &p, const DevBlock &B, int a) {
  return p.active[a] ? scale2i(p.dx[a], -B.level) : p.dx[a];
}
__device__ __forceinline__ double block_idx(const Phys &p, const DevBlock &B, int a) {
  return p.active[a] ? scale2i(p.idx[a], B.level) : p.idx[a];
}
__device__ __forceinline__ int level_n(const Phys &p, int a, int L) {
  return p.active[a] ? p.N[a] << L : 1;
}

__device__ __forceinline__ void count(unsigned long long *c) {
  if (c) atomicAdd(c, 1ull);
}

// Hardware seeds: approximate double reciprocal and reciprocal square root
// (relative error about 2^-20, under 2^-19, over the normal range, measured by
// tde_math_probe; flush-to-zero).
__device__ __forceinline__ double rcp_seed(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  return r;
}
__device__ __forceinline__ double rsqrt_seed(double d) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  return r;
}

// 1/d from the seed r: with e = 1 - d r, 1/d = r / (1 - e) = r (1 + e + e^2 +
// e^3 + ...); keeping the terms through e^2 (two FMAs after the residual)
// leaves a truncation error ~e^3 < 2^-59, far below the FP64 rounding, so the
// result is within one ulp of 1/d.  For normal d whose reciprocal is normal
// (every use below: sums of same-signed slopes, wave-speed differences,
// densities, Gamma_e - 1).
__device__ __forceinline__ double rcp_nr(double d) {
  const double r = rcp_seed(d);
  const double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// sqrt(a / b) for a, b > 0 as a / sqrt(a b): y = seed of 1/sqrt(t), t = a b,
// e = 1 - t y^2, 1/sqrt(t) = y (1 - e)^(-1/2) = y (1 + e/2 + 3 e^2/8 + ...);
// the truncation error ~(5/16) e^3 is below 2^-61, and the roundings of t, y^2
// and the final product keep the result within about two ulps of the correctly
// rounded sqrt(a / b).  Replaces a division and a square root (the wave-speed
// estimates of the Riemann solver and of the time-step condition).  Where a b
// leaves the range in which the seed and y^2 are normal (floor states of
// 1e-300 give a b ~ 1e-600) the IEEE form is used instead.
__device__ __forceinline__ double sqrt_ratio(double a, double b) {
  const double t = a * b;
  if ((unsigned long long)(((dbits(t) >> 52) & 0x7ff) - 2) >= 0x7fcull) return sqrt(a / b);
  const double y = rsqrt_seed(t);
  const double e = fma(-t, y * y, 1.0);
  const double y1 = fma(y, e * fma(e, 0.375, 0.5), y);
  return a * y1;
}

// 1/sqrt(t) for t > 0: the hardware seed refined to second order as in
// sqrt_ratio, within about two ulps; the IEEE form outside the seed's normal range
__device__ __forceinline__ double rsqrt_nr(double t) {
  if ((unsigned long long)(((dbits(t) >> 52) & 0x7ff) - 2) >= 0x7fcull) return 1.0 / sqrt(t);
  const double y = rsqrt_seed(t);
  const double e = fma(-t, y * y, 1.0);
  return fma(y, e * fma(e, 0.375, 0.5), y);
}

// sqrt(r2) < r for r2 >= 0, decided as with the correctly rounded square root:
// away from the boundary the comparison of r2 with r^2 (1 -+ 2^-40) gives the
// same answer (the roundings of r^2 and of the square root are below 2^-51
// relative), and only within that band is the square root taken.  A negative
// or NaN r gives false, as the comparison does.
// The thresholds depend on r alone, so a kernel that tests many cells against one
// sphere forms them once (sphere_of) and tests with inside_sphere; inside_radius
// does both.
struct Sphere {
  double r, lo, hi;   // radius; r^2 (1 - 2^-40), r^2 (1 + 2^-40)
  int mode;           // 0: the band test; 1: r^2 near the subnormals (root test); 2: never inside
};
__device__ __forceinline__ Sphere sphere_of(double r) {
  Sphere s;
  s.r = r;
  const double r2b = r * r;
  s.lo = r2b * (1.0 - 0x1p-40);
  s.hi = r2b * (1.0 + 0x1p-40);
  s.mode = (unsigned long long)dbits(r) > 0x7ff0000000000000ull ? 2 : (((dbits(r2b) >> 52) & 0x7ff) < 64 ? 1 : 0);
  return s;
}
__device__ __forceinline__ bool inside_sphere(double r2, const Sphere &s) {
  if (s.mode == 2) return false;
  if (s.mode == 1) return dlt(sqrt(r2), s.r);   // r^2 near the subnormals
  if (dlt(r2, s.lo)) return true;
  if (dlt(s.hi, r2)) return false;
  return dlt(sqrt(r2), s.r);
}
__device__ __forceinline__ bool inside_radius(double r2, double r) { return inside_sphere(r2, sphere_of(r)); }

// Squared distance of a cell centre from the point mass, in one fixed order of
// roundings for every kernel (a cell's potential and excision flag then agree
// wherever they are evaluated); d0 enters last, so the two transverse terms of
// an x pencil can be summed once per pencil.
__device__ __forceinline__ double bh_r2_yz(double d1, double d2) { return fma(d1, d1, d2 * d2); }
__device__ __forceinline__ double bh_r2(double d0, double d1, double d2) { return fma(d0, d0, bh_r2_yz(d1, d2)); }

// The square of the point mass's time-step limit (the CFL condition with the
// point mass, Sec. 7.1): dt_g^2 = dx / |g| with |g| = GM r / (r^2 + r_s^2)^(3/2),
// written as (dx / GM) s2^2 / (sqrt(s2) r) with s2 = r^2 + r_s^2 from refined
// reciprocals (a few ulps); infinity where there is no limit (GM <= 0, r = 0).
// Its square root is taken once per block, after the minimum (the square root
// is monotonic, so the minimum of the roots is the root of the minimum).
// dxg = bh_dxg(dx, GM), the per-block factor dx / GM (infinite without a limit).
__device__ __forceinline__ double bh_dxg(double dx, double GM) {
  return dgt0(GM) ? dx * rcp_nr(GM) : INFINITY;
}
__device__ __forceinline__ double bh_dt2(double dxg, double r2, double rs2) {
  if (!dgt0(r2)) return INFINITY;
  const double s2 = r2 + rs2;
  return dxg * (s2 * s2) * (rsqrt_nr(s2) * rsqrt_nr(r2));
}

// ---------------------------------------------------------------- EOS ----

// floor(x) for 0 <= x < 2^31 (also -0) from the bit fields, on the integer pipe
__device__ __forceinline__ int ifloor_nonneg(double x) {
  const long long b = dbits(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < 0) return 0;
  return (int)(((b & 0xfffffffffffffLL) | 0x10000000000000LL) >> (52 - e));
}

// Density cell i and weight w of log10 rho (clamped to the table).
__device__ __forceinline__ bool rho_cell(const DTable &t, double rho, int &i, double &w) {
  double x = (tlog10(t, rho) - t.lr0) * t.inv_dlr;
  bool cl = false;
  if (!dge0(x) || (dbits(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) { x = 0.0; cl = true; }  // < 0, NaN
  if (dlt(t.xr_max, x)) { x = t.xr_max; cl = true; }
  // i = floor(x) and w = x - i from the bit fields (0 <= x <= nr - 1 < 2^31); the
  // same values as the FP64 floor and subtraction, without the FP64 pipe
  const long long b = dbits(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  int ii;
  if (e < 0) {
    ii = 0;
    w = x;
  } else {
    const long long m = (b & 0xfffffffffffffLL) | 0x10000000000000LL;
    ii = (int)(m >> (52 - e));
    w = __longlong_as_double(0x3ff0000000000000LL | ((m << e) & 0xfffffffffffffLL)) - 1.0;
  }
  if (ii > t.nr - 2) { ii = t.nr - 2; w = 1.0; }   // x = nr - 1 exactly
  i = ii;
  return cl;
}

// Interpolation formulas are written with explicit rounding so that every kernel
// computes the same bits for the same cell (the surrogate's accepted path must
// equal the bisection path exactly, whatever the compiler fuses around it).
__device__ __forceinline__ double lerp_rn(double w, double a, double b) {
  return __fma_rn(w, b, __dmul_rn(__dsub_rn(1.0, w), a));
}

__device__ __forceinline__ double bilin(const double *__restrict__ f, int nt, int i, double w, int j,
                                        double s) {
  const double *a = f + (size_t)i * nt + j;
  const double *b = a + nt;
  const double lo = lerp_rn(s, __ldg(a), __ldg(a + 1));
  const double hi = lerp_rn(s, __ldg(b), __ldg(b + 1));
  return lerp_rn(w, lo, hi);
}

// Exact linear solve inside temperature cell j of the interpolated column: the
// fraction s of the cell at which it reaches y (g0 <= y < g1), and log10 T
// there.  Shared by every inversion so that all of them compute the same bits.
__device__ __forceinline__ double cell_solve(double y, double g0, double g1) {
  return __dmul_rn(__dsub_rn(y, g0), rcp_nr(__dsub_rn(g1, g0)));
}
__device__ __forceinline__ double cell_log10T(const DTable &t, int j, double s) {
  return __fma_rn(__dadd_rn(dint(j), s), t.dlt, t.lt0);
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
  double glo = lerp_rn(w, __ldg(a), __ldg(b));
  double ghi = lerp_rn(w, __ldg(a + nt - 1), __ldg(b + nt - 1));
  double y = dgt0(e) ? tlog10(t, e) : -INFINITY;
  int j;
  double s;
  if (!dlt(glo, y)) {
    j = 0; s = 0.0; cl = true;
  } else if (dle(ghi, y)) {
    j = nt - 2; s = 1.0; cl = true;
  } else {
    // search in FP32 (FP64 issues 55x slower on this part), then confirm the cell
    // with the FP64 bracket the linear solve needs anyway; the cell with
    // g_j <= y < g_{j+1} is unique, so a confirmed FP32 answer equals the FP64
    // bisection's, and an unconfirmed one (y within FP32 rounding of a node)
    // falls back to it
    int lo = 0, hi = nt - 1;
    if (t.le32) {   // tables without the FP32 copy (caller-owned views) skip this
      const float *__restrict__ a32 = t.le32 + (size_t)i * nt;
      const float *__restrict__ b32 = a32 + nt;
      const float w32 = d2f_guide(w), y32 = d2f_guide(y);
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        const float a0 = __ldg(a32 + mid);
        const float g = fmaf(w32, __ldg(b32 + mid) - a0, a0);
        if (g <= y32) lo = mid; else hi = mid;
      }
    }
    j = lo;
    double g0 = lerp_rn(w, __ldg(a + j), __ldg(b + j));
    double g1 = lerp_rn(w, __ldg(a + j + 1), __ldg(b + j + 1));
    if (!(dle(g0, y) && dlt(y, g1))) {
      lo = 0;
      hi = nt - 1;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        const double g = lerp_rn(w, __ldg(a + mid), __ldg(b + mid));
        if (dle(g, y)) lo = mid; else hi = mid;
      }
      j = lo;
      g0 = lerp_rn(w, __ldg(a + j), __ldg(b + j));
      g1 = lerp_rn(w, __ldg(a + j + 1), __ldg(b + j + 1));
    }
    s = cell_solve(y, g0, g1);
  }
  P = texp10(t, bilin(t.lp, nt, i, w, j, s));
  if (WANT_CS2) {
    cs2 = texp10(t, bilin(t.lc, nt, i, w, j, s));
    if (T) *T = texp10(t, cell_log10T(t, j, s));
    e_used = cl ? texp10(t, bilin(t.le, nt, i, w, j, s)) : e;
  }
  return cl;
}

// The table's inputs (cgs density and specific internal energy) of a cell with
// density rho and internal energy density U in code units.
__device__ __forceinline__ void eos_inputs(const Phys &p, double rho, double U, double &rho_c,
                                           double &e_c) {
  rho_c = rho * p.unit_rho;
  e_c = (U * rcp_nr(rho)) * p.unit_e;
}

// Table results of a cell computed by a separate pass (the learned-guess
// inversion runs as its own launches): P, cs2 in cgs and eu = the clamped
// table energy, or 0 where the input was inside the table.
struct EOSBuf {
  const double *P, *cs2, *eu;
};

// EOS closure in code units: internal energy density U at density rho ->
// P, cs^2 and the internal energy the table actually represents.  EOSB: take
// the table results of the cell at index flat from eb instead of inverting.
template <int EOSK, int EOSB = 0>
__device__ __forceinline__ void eos_closure(const Phys &p, double rho, double U, double &P,
                                            double &cs2, double &Uu, Counters *cnt,
                                            const EOSBuf *eb = nullptr, long long flat = 0) {
  if (EOSK == EOS_IDEAL) {
    P = p.gm1 * U;
    cs2 = p.gamma * P / rho;
    Uu = U;
  } else {
    double Pc, c2c, eu;
    bool cl;
    if (EOSB) {
      Pc = eb->P[flat];
      c2c = eb->cs2[flat];
      eu = eb->eu[flat];
      cl = dgt0(eu);
    } else {
      double rc, ec;
      eos_inputs(p, rho, U, rc, ec);
      cl = eos_invert(p.tab, rc, ec, Pc, c2c, eu);
    }
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
  bool cl = eos_invert<false>(p.tab, rho * p.unit_rho, (U * rcp_nr(rho)) * p.unit_e, Pc, c2c, eu);
  if (cl && cnt) count(&cnt->table_clamp);
  return Pc * p.inv_unit_p;
}

// Density (floored), velocities and the internal energy density the EOS gets
// (Eq. dual-econs with the dual-energy switch of Eq. dual-primitive-switch).
template <int DUAL>
__device__ __forceinline__ void c2p_energy(const Phys &p, const double *u, double &rho, double &vx,
                                           double &vy, double &vz, double &Ue, Counters *cnt) {
  rho = u[0];
  if (dlt(rho, p.rho_floor)) { rho = p.rho_floor; if (cnt) count(&cnt->rho_floor); }
  double ir = rcp_nr(rho);
  vx = u[1] * ir; vy = u[2] * ir; vz = u[3] * ir;
  double Uc = u[4] - 0.5 * (u[1] * vx + u[2] * vy + u[3] * vz);   // Eq. dual-econs
  Ue = Uc;
  if (DUAL) {
    if (!(dgt0(Uc) && dlt(p.eta1 * u[4], Uc))) { Ue = u[5]; if (cnt) count(&cnt->dual_aux_used); }
  }
}

// Conserved (rho, m, E[, U_aux]) -> primitives w = (rho, vx, vy, vz, P
// [, Gamma_e, Gamma_1][, U_aux]) with the dual-energy switch of
// Eq. dual-primitive-switch and the density / pressure floors.
template <int EOSK, int DUAL, int EOSB = 0>
__device__ __forceinline__ void cons_to_prim(const Phys &p, const double *u, double *w,
                                             Counters *cnt, const EOSBuf *eb = nullptr,
                                             long long flat = 0) {
  double rho, vx, vy, vz, Ue;
  c2p_energy<DUAL>(p, u, rho, vx, vy, vz, Ue, cnt);
  double P, cs2, Uu;
  eos_closure<EOSK, EOSB>(p, rho, Ue, P, cs2, Uu, cnt, eb, flat);
  if (dlt(P, p.p_floor)) { P = p.p_floor; if (cnt) count(&cnt->p_floor); }
  w[0] = rho; w[1] = vx; w[2] = vy; w[3] = vz; w[4] = P;
  if (EOSK == EOS_TABLE) {
    w[5] = 1.0 + P * rcp_nr(Uu);         // Gamma_e
    w[6] = rho * cs2 * rcp_nr(P);        // Gamma_1
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
  double h = dgt0(pr) ? pr * rcp_nr(dl + dr) : 0.0;
  left = q0 - h;
  right = q0 + h;
}

// PPM: 4th-order interface value between q0 and q1, clipped to [q0, q1]
__device__ __forceinline__ double ppm_iface(double qm1, double q0, double q1, double q2) {
  double a = (7.0 / 12.0) * (q0 + q1) - (1.0 / 12.0) * (qm1 + q2);
  double lo = dmin(q0, q1), hi = dmax(q0, q1);
  return dmin(dmax(a, lo), hi);
}

// Colella-Woodward (1984) monotonicity constraints on the parabola (aL, q0, aR).
// The textbook tests (aR - q0)(q0 - aL) <= 0, da^2 < da q6 and da q6 < -da^2
// (da = aR - aL, q6 = 6 (q0 - (aL + aR) / 2)) are taken in equivalent forms that
// need no FP64 product: q0 not strictly between aL and aR; aL on the far side of
// 3 q0 - 2 aR; aR on the far side of 3 q0 - 2 aL ("far" along the sign of da,
// by which the textbook inequalities divide).  The comparisons run on the
// integer pipe; the forms agree with the products except within rounding of a
// tie, where both branches give the same interface value up to rounding (at the
// tie of the second test 3 q0 - 2 aR equals aL), and for products that
// underflow.  Three FP64 operations per variable and cell instead of about ten.
__device__ __forceinline__ void ppm_limit(double q0, double &aL, double &aR) {
  const long long kL = dkey0(aL), kR = dkey0(aR), kq = dkey0(q0);
  const bool up = kL < kR;
  if (up ? !(kL < kq && kq < kR) : !(kR < kq && kq < kL)) {
    aL = q0;
    aR = q0;
    return;
  }
  const double t3 = 3.0 * q0;
  const double nL = fma(-2.0, aR, t3), nR = fma(-2.0, aL, t3);
  const long long knL = dkey0(nL), knR = dkey0(nR);
  if (up ? kL < knL : knL < kL) aL = nL;
  else if (up ? knR < kR : kR < knR) aR = nR;
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
  double cl = sqrt_ratio(L.g1 * L.P, L.r), cr = sqrt_ratio(R.g1 * R.P, R.r);
  double SL = dmin(ul - cl, ur - cr);
  double SR = dmax(ul + cl, ur + cr);
  double al = L.r * (SL - ul), ar = R.r * (SR - ur);
  double SM = (R.P - L.P + al * ul - ar * ur) * rcp_nr(al - ar);
  bool supL = dge0(SL), supR = dle0(SR);
  bool useL = supL || (!supR && dge0(SM));
  // chosen side K; its total energy only (the other side's enters no flux)
  double r = useL ? L.r : R.r, un = useL ? ul : ur, P = useL ? L.P : R.P;
  const double vK0 = useL ? L.v[0] : R.v[0], vK1 = useL ? L.v[1] : R.v[1], vK2 = useL ? L.v[2] : R.v[2];
  const double UK = EOSK == EOS_IDEAL ? P * p.inv_gm1 : P * rcp_nr((useL ? L.ge : R.ge) - 1.0);
  double E = UK + 0.5 * r * (vK0 * vK0 + vK1 * vK1 + vK2 * vK2);
  double vt1 = useL ? L.v[t1] : R.v[t1], vt2 = useL ? L.v[t2] : R.v[t2];
  double S = useL ? SL : SR;
  double Seff = (supL || supR) ? 0.0 : S;
  double den = S - SM;
  if (dzero(den)) den = 1.0;   // only reachable when Seff == 0
  double rS = useL ? al : ar;   // r (S - u) of side K: the same product as al / ar
  double inv = rcp_nr(den);
  double fac = rS * inv;
  double mflux = r * un;
  // U*_K - U_K and F_K in the (normal, t1, t2) frame
  double d0 = fac - r;
  double dn = fac * SM - mflux;
  double d1 = (fac - r) * vt1;
  double d2 = (fac - r) * vt2;
  // E*_K - E_K = [E (S - u) + (SM - u)(rS SM + P)] / (S - SM) - E
  //            = (SM - u)(E + P + rS SM) / (S - SM): no cancellation, two fewer FP64 ops
  const double EP = E + P;
  double dE = (SM - un) * fma(rS, SM, EP) * inv;
  F[0] = mflux + Seff * d0;
  double Fn = mflux * un + P + Seff * dn;
  double F1 = mflux * vt1 + Seff * d1;
  double F2 = mflux * vt2 + Seff * d2;
  F[1 + D] = Fn;
  F[1 + t1] = F1;
  F[1 + t2] = F2;
  F[4] = EP * un + Seff * dE;
  if (DUAL) {
    double f = F[0];
    bool up = dgt0(f);
    double ru = up ? L.r : R.r, Au = up ? L.A : R.A;
    double iru = rcp_nr(ru);
    F[5] = !dzero(f) ? f * (Au * iru) : 0.0;
    vf = !dzero(f) ? f * iru : 0.0;
  } else {
    F[5] = 0.0;
    vf = 0.0;
  }
}

// HLLE flux across a face normal to direction D (Harten, Lax and van Leer with
// Einfeldt's two-wave form; the production solver of Table 1) with the same
// Davis wave-speed bounds as hllc: b- = min(S_L, 0), b+ = max(S_R, 0),
// F = (b+ F_L - b- F_R + b+ b- (U_R - U_L)) / (b+ - b-); F[5] and vf follow the
// sign of the mass flux as for hllc.
template <int D, int EOSK, int DUAL>
__device__ __forceinline__ void hlle(const Phys &p, const FState &L, const FState &R, double *F,
                                     double &vf) {
  double ul = L.v[D], ur = R.v[D];
  double cl = sqrt_ratio(L.g1 * L.P, L.r), cr = sqrt_ratio(R.g1 * R.P, R.r);
  double Ul = EOSK == EOS_IDEAL ? L.P * p.inv_gm1 : L.P * rcp_nr(L.ge - 1.0);
  double Ur = EOSK == EOS_IDEAL ? R.P * p.inv_gm1 : R.P * rcp_nr(R.ge - 1.0);
  double El = Ul + 0.5 * L.r * (L.v[0] * L.v[0] + L.v[1] * L.v[1] + L.v[2] * L.v[2]);
  double Er = Ur + 0.5 * R.r * (R.v[0] * R.v[0] + R.v[1] * R.v[1] + R.v[2] * R.v[2]);
  const double bm = dmin(dmin(ul - cl, ur - cr), 0.0);
  const double bp = dmax(dmax(ul + cl, ur + cr), 0.0);
  double den = bp - bm;
  if (dzero(den)) den = 1.0;   // both fluxes vanish there
  const double inv = rcp_nr(den), bpm = bp * bm;
  const double ml = L.r * ul, mr = R.r * ur;
  // mass, momentum (x, y, z), energy: physical fluxes and conserved states
  F[0] = (bp * ml - bm * mr + bpm * (R.r - L.r)) * inv;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double fl = ml * L.v[q] + (q == D ? L.P : 0.0);
    const double fr = mr * R.v[q] + (q == D ? R.P : 0.0);
    F[1 + q] = (bp * fl - bm * fr + bpm * (R.r * R.v[q] - L.r * L.v[q])) * inv;
  }
  F[4] = (bp * ((El + L.P) * ul) - bm * ((Er + R.P) * ur) + bpm * (Er - El)) * inv;
  if (DUAL) {
    double f = F[0];
    bool up = dgt0(f);
    double ru = up ? L.r : R.r, Au = up ? L.A : R.A;
    double iru = rcp_nr(ru);
    F[5] = !dzero(f) ? f * (Au * iru) : 0.0;
    vf = !dzero(f) ? f * iru : 0.0;
  } else {
    F[5] = 0.0;
    vf = 0.0;
  }
}

}  // namespace tde
