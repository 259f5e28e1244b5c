// tde_grav.cu -- self-gravity (Sec. 3.2): a geometric multigrid for
// A_h phi = S_h, A_h = -lap_h (seven-point, anisotropic weights
// w_y = (dx/dy)^2, w_z = (dx/dz)^2), S_h = -4 pi G rho_sg (Eq. selfgrav-poisson),
// on the mesh's uniform grid, periodic or isolated, and the coupling of the
// potential to the hydro sources (the sweeps add the stored phi_sg to the point
// mass's potential in Eqs. lat-grav-momentum and lat-grav-energy).
//
// V-cycle: red-black Gauss-Seidel with over-relaxation, defect and volume-average
// restriction fused in one pass, full-approximation coarse equation, tricubic
// prolongation of the coarse correction, post-smoothing on every level, one
// extra fine sweep per cycle; each direction halved while it has more than one
// cell.  The levels are global arrays (x fastest); the MeshBlock layout is
// gathered into level 0 and the potential scattered back (ghosts included).
//
// Isolated boundaries (the paper's multipole boundary conditions): phi on every
// boundary face is the exterior multipole expansion of the source to order
// l_max <= 4 about its source-weighted centroid, a Dirichlet condition at the
// face (the cell beyond it is 2 phi_face - phi_inside; a coarse correction's is
// -e_inside); the Gauss-Seidel update is implicit in those mirror cells and the
// single-cell level is solved exactly.  The expansion uses the regular solid
// harmonics R_l^m = r^l P_l^m(cos t) e^(i m p), built by their polynomial
// recurrences in (x, y, z) (no trigonometry): the moments are sums of
// S dV R_l^m(x'), the potential sum_lm Re(conj-free) (A R_re + B R_im) / r^(2l+1).
//
// Full multigrid start: the source restricted to every level, the coarsest
// solved, then per finer level the prolonged solution and one V-cycle.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "tde_internal.h"

namespace tde {

namespace {

constexpr int GT = 256;
constexpr int MP_LMAX = 4;                                       // largest expansion order
constexpr int MP_NC = (MP_LMAX + 1) * (MP_LMAX + 2) / 2;        // (l, m) pairs, m <= l

struct Lev {
  int n[3];
  double dx[3];
  double *phi, *src, *tmp;
  // seven-point operator, per level: (A phi)_c = aw . (2 phi_c - phi_{c+a} - phi_{c-a});
  // Gauss-Seidel value = cs src + cw . (phi_{c+a} + phi_{c-a}) (cw = w_a / diag,
  // cs = dx^2 / diag); zero weights in directions with one cell (periodic) or
  // inactive on the finest level (isolated)
  double aw[3], cw[3], cs;
  int iso;                  // isolated boundaries
  int act[3];               // weight along a nonzero (an integer test: an FP64
                            // comparison would take the FP64 pipe)
  double x0[3];             // lower domain corner
  const double *gf[6];      // isolated: phi on the boundary faces x-, x+, y-, y+, z-, z+
};

// the expansion: order, centre, coefficients (A_lm, B_lm) at 2 (l (l + 1) / 2 + m)
struct MP {
  int lmax;
  const double *cc;         // [0..2] centre, then the coefficients
};

// 32-bit index arithmetic throughout (levels have < 2^31 cells; 64-bit integer
// division would issue on the FP64 pipe)
__device__ __forceinline__ unsigned wrap_idx(const Lev &L, int i, int j, int k) {
  i = i < 0 ? i + L.n[0] : (i >= L.n[0] ? i - L.n[0] : i);
  j = j < 0 ? j + L.n[1] : (j >= L.n[1] ? j - L.n[1] : j);
  k = k < 0 ? k + L.n[2] : (k >= L.n[2] ? k - L.n[2] : k);
  return ((unsigned)k * L.n[1] + j) * L.n[0] + i;
}

__device__ __forceinline__ unsigned lin(const Lev &L, int i, int j, int k) {
  return ((unsigned)k * L.n[1] + j) * L.n[0] + i;
}

__device__ __forceinline__ void decompose(const Lev &L, unsigned c, int &i, int &j, int &k) {
  const unsigned r = c / (unsigned)L.n[0];
  i = (int)(c - r * L.n[0]);
  k = (int)(r / (unsigned)L.n[1]);
  j = (int)(r - (unsigned)k * L.n[1]);
}

// isolated: phi on the boundary face (a, side) of boundary cell c
__device__ __forceinline__ double face_phi(const Lev &L, int a, int side, const int c[3]) {
  const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
  return L.gf[2 * a + side][(unsigned)c[t2] * L.n[t1] + c[t1]];
}

// the regular solid harmonics R_l^m(d) (re, im) for l <= lmax, at 2 (l (l+1)/2 + m)
__device__ __forceinline__ void solid_harmonics(int lmax, const double d[3], double *R) {
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double mre = 1.0, mim = 0.0;   // (2m - 1)!! (x + i y)^m
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) {
      const double f = 2.0 * m - 1.0;
      const double re = f * (mre * d[0] - mim * d[1]), im = f * (mre * d[1] + mim * d[0]);
      mre = re;
      mim = im;
    }
    int q = m * (m + 1) / 2 + m;
    R[2 * q] = mre;
    R[2 * q + 1] = mim;
    if (m + 1 <= lmax) {
      q = (m + 1) * (m + 2) / 2 + m;
      R[2 * q] = (2.0 * m + 1.0) * d[2] * mre;
      R[2 * q + 1] = (2.0 * m + 1.0) * d[2] * mim;
    }
    for (int l = m + 2; l <= lmax; ++l) {
      const int q0 = l * (l + 1) / 2 + m, q1 = (l - 1) * l / 2 + m, q2 = (l - 2) * (l - 1) / 2 + m;
      const double a = (2.0 * l - 1.0) * d[2], b = (l + m - 1.0) * r2, inv = 1.0 / (l - m);
      R[2 * q0] = (a * R[2 * q1] - b * R[2 * q2]) * inv;
      R[2 * q0 + 1] = (a * R[2 * q1 + 1] - b * R[2 * q2 + 1]) * inv;
    }
  }
}

// the exterior expansion at x
__device__ double mp_eval(const MP &mp, const double x[3]) {
  const double d[3] = {x[0] - mp.cc[0], x[1] - mp.cc[1], x[2] - mp.cc[2]};
  double R[2 * MP_NC];
  solid_harmonics(mp.lmax, d, R);
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double ir = 1.0 / sqrt(r2), ir2 = 1.0 / r2;
  double s = 0.0, rp = ir;   // r^-(2l+1)
  for (int l = 0; l <= mp.lmax; ++l) {
    double t = 0.0;
    for (int m = 0; m <= l; ++m) {
      const int q = l * (l + 1) / 2 + m;
      t += mp.cc[3 + 2 * q] * R[2 * q] + mp.cc[3 + 2 * q + 1] * R[2 * q + 1];
    }
    s += t * rp;
    rp *= ir2;
  }
  return s;
}

// isolated: a cell with a neighbour beyond a boundary face
__device__ __forceinline__ bool on_boundary(const Lev &L, int i, int j, int k) {
  return (L.act[0] && (i == 0 || i == L.n[0] - 1)) || (L.act[1] && (j == 0 || j == L.n[1] - 1)) ||
         (L.act[2] && (k == 0 || k == L.n[2] - 1));
}

// the cell of thread e: x fastest; on an isolated grid of at least three cells
// along x the cells at the two x faces come after all others, so that warps of
// inner cells do not diverge into the boundary path (y and z boundary cells
// fill whole rows)
__device__ __forceinline__ void cell_of(const Lev &L, unsigned e, int &i, int &j, int &k) {
  if (!L.iso || L.n[0] < 3) {
    decompose(L, e, i, j, k);
    return;
  }
  const unsigned nin = (unsigned)L.n[0] - 2, nrow = (unsigned)L.n[1] * L.n[2];
  unsigned row;
  if (e < nrow * nin) {
    row = e / nin;
    i = 1 + (int)(e - row * nin);
  } else {
    const unsigned r = e - nrow * nin;
    row = r >> 1;
    i = (r & 1) ? L.n[0] - 1 : 0;
  }
  k = (int)(row / (unsigned)L.n[1]);
  j = (int)(row - (unsigned)k * L.n[1]);
}

// isolated boundary cell: its six neighbours, one beyond a face replaced by twice
// the face value (its mirror image is 2 phi_face - phi_c, whose -phi_c part the
// caller moves to the centre); out[a] = faces crossed along a.  Unrolled selects:
// only boundary cells come here, so computing both sides costs little.
struct Nb6 {
  double m[3], p[3];
  double out[3];
};
__device__ __forceinline__ Nb6 nbrs_iso(const Lev &L, const double *phi, int i, int j, int k, unsigned l) {
  Nb6 r;
  const unsigned sy = (unsigned)L.n[0], sz = (unsigned)L.n[0] * L.n[1];
  const bool xl = i > 0, xh = i < L.n[0] - 1, yl = j > 0, yh = j < L.n[1] - 1, zl = k > 0, zh = k < L.n[2] - 1;
  // (a direction inactive on the finest grid has no faces and weight 0: nothing read)
  const bool ax = L.act[0], ay = L.act[1], az = L.act[2];
  const unsigned fx = (unsigned)k * L.n[1] + j, fy = (unsigned)k * L.n[0] + i, fz = (unsigned)j * L.n[0] + i;
  r.m[0] = !ax ? 0.0 : (xl ? phi[l - 1] : 2.0 * L.gf[0][fx]);
  r.p[0] = !ax ? 0.0 : (xh ? phi[l + 1] : 2.0 * L.gf[1][fx]);
  r.m[1] = !ay ? 0.0 : (yl ? phi[l - sy] : 2.0 * L.gf[2][fy]);
  r.p[1] = !ay ? 0.0 : (yh ? phi[l + sy] : 2.0 * L.gf[3][fy]);
  r.m[2] = !az ? 0.0 : (zl ? phi[l - sz] : 2.0 * L.gf[4][fz]);
  r.p[2] = !az ? 0.0 : (zh ? phi[l + sz] : 2.0 * L.gf[5][fz]);
  r.out[0] = (xl ? 0.0 : 1.0) + (xh ? 0.0 : 1.0);
  r.out[1] = (yl ? 0.0 : 1.0) + (yh ? 0.0 : 1.0);
  r.out[2] = (zl ? 0.0 : 1.0) + (zh ? 0.0 : 1.0);
  return r;
}

__device__ __forceinline__ double apply_A(const Lev &L, const double *phi, int i, int j, int k) {
  if (L.iso && on_boundary(L, i, j, k)) {
    const unsigned l = lin(L, i, j, k);
    const double pc = phi[l];
    const Nb6 q = nbrs_iso(L, phi, i, j, k, l);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) s = fma(L.aw[a], (2.0 + q.out[a]) * pc - q.m[a] - q.p[a], s);
    return s;
  }
  // (periodic, or an isolated grid's inner cell, whose wrapped neighbours are its own)
  const double c2 = 2.0 * phi[wrap_idx(L, i, j, k)];
  double s = L.aw[0] * (c2 - phi[wrap_idx(L, i + 1, j, k)] - phi[wrap_idx(L, i - 1, j, k)]);
  s = fma(L.aw[1], c2 - phi[wrap_idx(L, i, j + 1, k)] - phi[wrap_idx(L, i, j - 1, k)], s);
  s = fma(L.aw[2], c2 - phi[wrap_idx(L, i, j, k + 1)] - phi[wrap_idx(L, i, j, k - 1)], s);
  return s;
}

// isolated Gauss-Seidel value of a boundary cell: the mirror cells' -phi_c parts
// move to the diagonal (w_a / diag per face crossed)
__device__ __forceinline__ double gs_iso(const Lev &L, int i, int j, int k) {
  const unsigned l = lin(L, i, j, k);
  const Nb6 q = nbrs_iso(L, L.phi, i, j, k, l);
  double nb = 0.0, dg = 1.0;   // in units of the inner cells' diagonal
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nb = fma(L.cw[a], q.m[a] + q.p[a], nb);
    dg = fma(L.cw[a], q.out[a], dg);
  }
  return fma(L.cs, L.src[l], nb) / dg;
}

// level-0 source from the MeshBlock density: S = -4 pi G rho where rho > rho_min
__global__ void __launch_bounds__(GT) k_mg_gather(Phys p, const DevBlock *__restrict__ blocks,
                                                  const double *__restrict__ U, Lev L, double fourpiG,
                                                  double rho_min) {
  const int b = blockIdx.y;
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  for (int e = blockIdx.x * GT + threadIdx.x; e < nint; e += gridDim.x * GT) {
    const int i = e % B.n[0], r = e / B.n[0];
    const int j = r % B.n[1], k = r / B.n[1];
    const double rho = U[B.off + ((long long)(k + p.g[2]) * B.p[1] + (j + p.g[1])) * B.p[0] + (i + p.g[0])];
    L.src[((long long)(B.k0 + k) * L.n[1] + (B.j0 + j)) * L.n[0] + (B.i0 + i)] =
        rho > rho_min ? -fourpiG * rho : 0.0;
  }
}

// partial sums (one per CTA) of f, or of the squared defect if sq
__global__ void __launch_bounds__(GT) k_mg_partial(Lev L, int sq, double *part) {
  __shared__ double red[GT / 32];
  double s = 0.0;
  if (sq) {
    const unsigned n = (unsigned)L.n[0] * L.n[1] * L.n[2];
    for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
      int i, j, k;
      cell_of(L, c, i, j, k);
      const double d = L.src[lin(L, i, j, k)] - apply_A(L, L.phi, i, j, k);
      s += d * d;
    }
  } else {
    const unsigned n = (unsigned)L.n[0] * L.n[1] * L.n[2];
    for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) s += L.src[c];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < GT / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// the partial sums in a fixed order: out = sum / n (a mean) or sqrt(sum / n)
__global__ void __launch_bounds__(GT) k_mg_final(const double *__restrict__ part, int np, double n,
                                                 int root, double *out) {
  __shared__ double red[GT];
  double s = 0.0;
  for (int q = threadIdx.x; q < np; q += GT) s += part[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = GT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = root ? sqrt(red[0] / n) : red[0] / n;
}

__global__ void __launch_bounds__(GT) k_mg_sub_mean(Lev L, const double *__restrict__ mean) {
  const unsigned n = (unsigned)L.n[0] * L.n[1] * L.n[2];
  const double m = *mean;
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) L.src[c] -= m;
}

// one colour of a red-black Gauss-Seidel sweep (colour = parity of i + j + k):
// phi <- phi + omega (GS value - phi)
__global__ void __launch_bounds__(GT) k_mg_smooth(Lev L, int colour, double omega) {
  const unsigned hx = (unsigned)(L.n[0] + 1) / 2;   // cells of one colour per row (n[0] even, or 1)
  const unsigned nrow = (unsigned)L.n[1] * L.n[2];
  // isolated, at least four cells along x: each row's one x-face cell of this
  // colour comes after all inner ones (no warp mixes the two paths)
  const bool split = L.iso && L.n[0] >= 4;
  for (unsigned e = blockIdx.x * GT + threadIdx.x; e < nrow * hx; e += gridDim.x * GT) {
    unsigned row;
    int i, j, k;
    if (split) {
      const unsigned nin = hx - 1;
      if (e < nrow * nin) {
        row = e / nin;
        k = (int)(row / (unsigned)L.n[1]);
        j = (int)(row - (unsigned)k * L.n[1]);
        const int par = (j + k + colour) & 1;
        i = 2 * (int)(e - row * nin) + 2 - par;
      } else {
        row = e - nrow * nin;
        k = (int)(row / (unsigned)L.n[1]);
        j = (int)(row - (unsigned)k * L.n[1]);
        i = ((j + k + colour) & 1) ? L.n[0] - 1 : 0;
      }
    } else {
      row = e / hx;
      k = (int)(row / (unsigned)L.n[1]);
      j = (int)(row - (unsigned)k * L.n[1]);
      if (L.n[0] > 1) {
        i = 2 * (int)(e - row * hx) + ((j + k + colour) & 1);
      } else {
        if (((j + k) & 1) != colour) continue;
        i = 0;
      }
    }
    const unsigned c = row * L.n[0] + i;
    double gs;
    if (L.iso && on_boundary(L, i, j, k)) {
      gs = gs_iso(L, i, j, k);
    } else {
      double nb = L.cw[0] * (L.phi[wrap_idx(L, i + 1, j, k)] + L.phi[wrap_idx(L, i - 1, j, k)]);
      nb = fma(L.cw[1], L.phi[wrap_idx(L, i, j + 1, k)] + L.phi[wrap_idx(L, i, j - 1, k)], nb);
      nb = fma(L.cw[2], L.phi[wrap_idx(L, i, j, k + 1)] + L.phi[wrap_idx(L, i, j, k - 1)], nb);
      gs = fma(L.cs, L.src[c], nb);
    }
    const double p0 = L.phi[c];
    L.phi[c] = fma(omega, gs - p0, p0);
  }
}

// coarse cell: phi_C = R phi_f (also kept in C.tmp), R d_f (defect of the fine
// level averaged over the children) into C.src
__global__ void __launch_bounds__(GT) k_mg_restrict(Lev F, Lev C, double inv) {
  const int r0 = F.n[0] / C.n[0], r1 = F.n[1] / C.n[1], r2 = F.n[2] / C.n[2];
  const unsigned n = (unsigned)C.n[0] * C.n[1] * C.n[2];
  for (unsigned e = blockIdx.x * GT + threadIdx.x; e < n; e += gridDim.x * GT) {
    int I, J, K;
    cell_of(C, e, I, J, K);
    const unsigned c = lin(C, I, J, K);
    double sp = 0.0, sd = 0.0;
    for (int cz = 0; cz < r2; ++cz)
      for (int by = 0; by < r1; ++by)
        for (int ax = 0; ax < r0; ++ax) {
          const int i = r0 * I + ax, j = r1 * J + by, k = r2 * K + cz;
          const unsigned f = ((unsigned)k * F.n[1] + j) * F.n[0] + i;
          sp += F.phi[f];
          sd += F.src[f] - apply_A(F, F.phi, i, j, k);
        }
    C.phi[c] = sp * inv;
    C.tmp[c] = sp * inv;
    C.src[c] = sd * inv;
  }
}

// coarse source of the full-approximation equation: S_C = R d_f + A_C (R phi_f)
__global__ void __launch_bounds__(GT) k_mg_fas(Lev C) {
  const unsigned n = (unsigned)C.n[0] * C.n[1] * C.n[2];
  for (unsigned e = blockIdx.x * GT + threadIdx.x; e < n; e += gridDim.x * GT) {
    int I, J, K;
    cell_of(C, e, I, J, K);
    C.src[lin(C, I, J, K)] += apply_A(C, C.tmp, I, J, K);
  }
}

// the coarse correction phi_C - R phi_f, formed once per coarse cell (into tmp)
__global__ void __launch_bounds__(GT) k_mg_corr(Lev C) {
  const unsigned n = (unsigned)C.n[0] * C.n[1] * C.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) C.tmp[c] = C.phi[c] - C.tmp[c];
}

// Tricubic prolongation (cell centred): along a halved direction the cubic
// through the four coarse centres nearest the fine centre, which lies a quarter
// of a coarse cell from its parent's centre p: Lagrange weights -5, 35, 105, -7
// (/128) on p-2 .. p+1 for a fine cell on the parent's low side, -7, 105, 35,
// -5 on p-1 .. p+2 on its high side; one tap (weight 1) along a kept
// direction; the weights of the three directions multiply.
__device__ __forceinline__ int cubic_taps(int f, bool halved, double w[4]) {
  if (!halved) {
    w[0] = 1.0;
    return f;
  }
  const int p = f >> 1;
  if (f & 1) {
    w[0] = -7.0 / 128.0; w[1] = 105.0 / 128.0; w[2] = 35.0 / 128.0; w[3] = -5.0 / 128.0;
    return p - 1;
  }
  w[0] = -5.0 / 128.0; w[1] = 35.0 / 128.0; w[2] = 105.0 / 128.0; w[3] = -7.0 / 128.0;
  return p - 2;
}

// index u of a direction with n cells mapped into the grid: periodic wrap, or
// (isolated) repeated mirror images about the faces, each flipping the sign
__device__ __forceinline__ int fold_idx(int u, int n, bool iso, double &sg) {
  if (!iso) {
    u %= n;
    return u < 0 ? u + n : u;
  }
  for (int r = 0; r < 4 && (u < 0 || u >= n); ++r) {   // |u| < n + 3: a few mirrors at most
    u = u < 0 ? -1 - u : 2 * n - 1 - u;
    sg = -sg;
  }
  return u;
}

// fine phi += P e, e = phi_C - R phi_f (in C.tmp), tricubic; beyond an isolated
// face the correction is the odd mirror image (it vanishes on the faces)
__global__ void __launch_bounds__(GT) k_mg_prolong(Lev F, Lev C) {
  const unsigned n = (unsigned)F.n[0] * F.n[1] * F.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int f[3];
    decompose(F, c, f[0], f[1], f[2]);
    double w[3][4];
    int first[3], nt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const bool h = F.n[a] != C.n[a];
      first[a] = cubic_taps(f[a], h, w[a]);
      nt[a] = h ? 4 : 1;
    }
    double s = 0.0;
    for (int cz = 0; cz < nt[2]; ++cz) {
      double sz = 1.0;
      const int uz = fold_idx(first[2] + cz, C.n[2], C.iso, sz);
      for (int by = 0; by < nt[1]; ++by) {
        double sy = sz;
        const int uy = fold_idx(first[1] + by, C.n[1], C.iso, sy);
        const double wyz = w[1][by] * w[2][cz];
        for (int ax = 0; ax < nt[0]; ++ax) {
          double sx = sy;
          const int ux = fold_idx(first[0] + ax, C.n[0], C.iso, sx);
          s = fma(w[0][ax] * wyz, sx * C.tmp[lin(C, ux, uy, uz)], s);
        }
      }
    }
    F.phi[c] += s;
  }
}

// The same prolongation for levels halved in every direction with edges that are
// multiples of 8: a CTA takes an 8^3 tile of fine cells, stages the 8^3 coarse
// cells its stencils reach (two beyond the tile's parents on each side; wrapped,
// or mirrored with a sign flip beyond an isolated face) and applies the 4-tap
// weights one direction at a time (x, then y, then z): 12 FMAs per fine cell
// instead of 64, the same weights summed in another order.
constexpr int PT = 8;   // fine tile edge
__device__ double full_value(const Lev &C, const MP &mp, int u0, int u1, int u2);
// FULL = 0: the V-cycle's correction (C.tmp, odd mirror images, added to F.phi);
// FULL = 1: the full-multigrid start's solution (C.phi with its boundary values,
// written to F.phi)
template <int FULL>
__global__ void __launch_bounds__(GT) k_mg_prolong_tiled(Lev F, Lev C, MP mp) {
  __shared__ double sc[PT][PT][PT];    // coarse [k][j][i]
  __shared__ double t1[PT][PT][PT];    // x done: [kc][jc][i]
  __shared__ double t2[PT][PT][PT];    // x, y done: [kc][j][i]
  const int ntx = F.n[0] / PT, nty = F.n[1] / PT;
  const int tx = blockIdx.x % ntx, r = blockIdx.x / ntx;
  const int ty = r % nty, tz = r / nty;
  const int c0[3] = {tx * (PT / 2) - 2, ty * (PT / 2) - 2, tz * (PT / 2) - 2};
  for (int e = threadIdx.x; e < PT * PT * PT; e += GT) {
    const int i = e % PT, j = (e / PT) % PT, k = e / (PT * PT);
    if (FULL) {
      sc[k][j][i] = full_value(C, mp, c0[0] + i, c0[1] + j, c0[2] + k);
    } else {
      double sg = 1.0;
      const int ux = fold_idx(c0[0] + i, C.n[0], C.iso, sg);
      const int uy = fold_idx(c0[1] + j, C.n[1], C.iso, sg);
      const int uz = fold_idx(c0[2] + k, C.n[2], C.iso, sg);
      sc[k][j][i] = sg * C.tmp[lin(C, ux, uy, uz)];
    }
  }
  __syncthreads();
  // tap window of fine index f (tile-local): starts at f/2 (low side) or f/2 + 1
  for (int e = threadIdx.x; e < PT * PT * PT; e += GT) {
    const int i = e % PT, jc = (e / PT) % PT, kc = e / (PT * PT);
    double w[4];
    const int a0 = (i >> 1) + (i & 1);
    cubic_taps(i, true, w);
    double v = w[0] * sc[kc][jc][a0];
    v = fma(w[1], sc[kc][jc][a0 + 1], v);
    v = fma(w[2], sc[kc][jc][a0 + 2], v);
    t1[kc][jc][i] = fma(w[3], sc[kc][jc][a0 + 3], v);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < PT * PT * PT; e += GT) {
    const int i = e % PT, j = (e / PT) % PT, kc = e / (PT * PT);
    double w[4];
    const int b0 = (j >> 1) + (j & 1);
    cubic_taps(j, true, w);
    double v = w[0] * t1[kc][b0][i];
    v = fma(w[1], t1[kc][b0 + 1][i], v);
    v = fma(w[2], t1[kc][b0 + 2][i], v);
    t2[kc][j][i] = fma(w[3], t1[kc][b0 + 3][i], v);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < PT * PT * PT; e += GT) {
    const int i = e % PT, j = (e / PT) % PT, k = e / (PT * PT);
    double w[4];
    const int z0 = (k >> 1) + (k & 1);
    cubic_taps(k, true, w);
    double v = w[0] * t2[z0][j][i];
    v = fma(w[1], t2[z0 + 1][j][i], v);
    v = fma(w[2], t2[z0 + 2][j][i], v);
    v = fma(w[3], t2[z0 + 3][j][i], v);
    const unsigned c = lin(F, tx * PT + i, ty * PT + j, tz * PT + k);
    if (FULL) F.phi[c] = v;
    else F.phi[c] += v;
  }
}

// the tiled form applies to levels halved in every direction, edges multiples of 8
__host__ __forceinline__ bool prolong_tiles(const Lev &F, const Lev &C) {
  bool ok = true;
  for (int a = 0; a < 3; ++a) ok = ok && F.n[a] == 2 * C.n[a] && F.n[a] % PT == 0;
  return ok;
}
__host__ __forceinline__ unsigned prolong_tile_count(const Lev &F) {
  return (unsigned)((F.n[0] / PT) * (F.n[1] / PT) * (F.n[2] / PT));
}

// the potential into the MeshBlock layout, every padded cell (ghosts by the
// periodic image of their global position)
__global__ void __launch_bounds__(GT) k_mg_scatter(Phys p, const DevBlock *__restrict__ blocks, Lev L,
                                                   MP mp, double *phi_pad) {
  const int b = blockIdx.y;
  const DevBlock B = blocks[b];
  const int npad = B.p[0] * B.p[1] * B.p[2];
  for (int e = blockIdx.x * GT + threadIdx.x; e < npad; e += gridDim.x * GT) {
    const int i = e % B.p[0], r = e / B.p[0];
    const int j = r % B.p[1], k = r / B.p[1];
    const int g[3] = {B.i0 + i - p.g[0], B.j0 + j - p.g[1], B.k0 + k - p.g[2]};
    // (isolated: the ghost cells beyond the boundary are k_mg_scatter_out's)
    if (L.iso && (g[0] < 0 || g[1] < 0 || g[2] < 0 || g[0] >= L.n[0] || g[1] >= L.n[1] || g[2] >= L.n[2])) continue;
    phi_pad[B.off + e] = L.phi[wrap_idx(L, g[0], g[1], g[2])];
  }
}

// isolated: the ghost cells beyond the boundary (a list built once per mesh)
// take the expansion at their centres
__global__ void __launch_bounds__(GT) k_mg_scatter_out(const long long *__restrict__ flat,
                                                       const int *__restrict__ gidx, int n, Lev L, MP mp,
                                                       double *phi_pad) {
  for (int e = blockIdx.x * GT + threadIdx.x; e < n; e += gridDim.x * GT) {
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = L.x0[a] + (gidx[3 * e + a] + 0.5) * L.dx[a];
    phi_pad[flat[e]] = mp_eval(mp, x);
  }
}

// full multigrid: the source of coarse cell (volume average of the children)
__global__ void __launch_bounds__(GT) k_mg_restrict_src(Lev F, Lev C, double inv) {
  const int r0 = F.n[0] / C.n[0], r1 = F.n[1] / C.n[1], r2 = F.n[2] / C.n[2];
  const unsigned n = (unsigned)C.n[0] * C.n[1] * C.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int I, J, K;
    decompose(C, c, I, J, K);
    double sd = 0.0;
    for (int cz = 0; cz < r2; ++cz)
      for (int by = 0; by < r1; ++by)
        for (int ax = 0; ax < r0; ++ax) sd += F.src[lin(F, r0 * I + ax, r1 * J + by, r2 * K + cz)];
    C.src[c] = sd * inv;
  }
}

// the solution's value at coarse cell u, beyond isolated faces by repeated
// mirror images (2 phi_face - phi_inside per face crossed, the face value at
// the point of the face between the cell and its image; where the image is
// outside the grid in another direction the expansion gives it directly)
__device__ double full_value(const Lev &C, const MP &mp, int u0, int u1, int u2) {
  int u[3] = {u0, u1, u2};
  if (!C.iso) {
    double one = 1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] = fold_idx(u[a], C.n[a], false, one);
    return C.phi[lin(C, u[0], u[1], u[2])];
  }
  double acc = 0.0, sg = 1.0;
  for (int a = 0; a < 3; ++a) {
    for (int r = 0; r < 4 && (u[a] < 0 || u[a] >= C.n[a]); ++r) {
      const int side = u[a] < 0 ? 0 : 1;
      u[a] = u[a] < 0 ? -1 - u[a] : 2 * C.n[a] - 1 - u[a];
      bool in = true;
      for (int b = 0; b < 3; ++b)
        if (u[b] < 0 || u[b] >= C.n[b]) in = false;
      double g;
      if (in) {
        g = face_phi(C, a, side, u);
      } else {
        double x[3];
        for (int b = 0; b < 3; ++b) x[b] = C.x0[b] + (u[b] + 0.5) * C.dx[b];
        x[a] = C.x0[a] + (side ? C.n[a] * C.dx[a] : 0.0);
        g = mp_eval(mp, x);
      }
      acc = fma(sg, 2.0 * g, acc);
      sg = -sg;
    }
  }
  return fma(sg, C.phi[lin(C, u[0], u[1], u[2])], acc);
}

// full multigrid: F.phi = P phi_C (the solution itself, tricubic)
__global__ void __launch_bounds__(GT) k_mg_prolong_full(Lev F, Lev C, MP mp) {
  const unsigned n = (unsigned)F.n[0] * F.n[1] * F.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int f[3];
    decompose(F, c, f[0], f[1], f[2]);
    double w[3][4];
    int first[3], nt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const bool h = F.n[a] != C.n[a];
      first[a] = cubic_taps(f[a], h, w[a]);
      nt[a] = h ? 4 : 1;
    }
    double s = 0.0;
    for (int cz = 0; cz < nt[2]; ++cz)
      for (int by = 0; by < nt[1]; ++by)
        for (int ax = 0; ax < nt[0]; ++ax)
          s = fma(w[0][ax] * w[1][by] * w[2][cz], full_value(C, mp, first[0] + ax, first[1] + by, first[2] + cz), s);
    F.phi[c] = s;
  }
}

// isolated single-cell level: its equation solved exactly
__global__ void k_mg_exact1(Lev L) {
  if (threadIdx.x == 0 && blockIdx.x == 0) L.phi[0] = gs_iso(L, 0, 0, 0);
}

// partial sums per CTA of (S, S x, S y, S z) over level 0 (the centroid)
__global__ void __launch_bounds__(GT) k_mp_centroid(Lev L, double *part) {
  __shared__ double red[4][GT / 32];
  const unsigned n = (unsigned)L.n[0] * L.n[1] * L.n[2];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int i, j, k;
    decompose(L, c, i, j, k);
    const double S = L.src[c];
    s[0] += S;
    s[1] += S * (L.x0[0] + (i + 0.5) * L.dx[0]);
    s[2] += S * (L.x0[1] + (j + 0.5) * L.dx[1]);
    s[3] += S * (L.x0[2] + (k + 0.5) * L.dx[2]);
  }
  for (int q = 0; q < 4; ++q) {
    double v = s[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < GT / 32; ++w) t += red[threadIdx.x][w];
    part[4 * blockIdx.x + threadIdx.x] = t;
  }
}

// the centroid from the partial sums (a fixed-order tree over GT threads; the
// domain centre for a source summing to zero)
__global__ void __launch_bounds__(GT) k_mp_centre(const double *__restrict__ part, int np, Lev L, double *cc) {
  __shared__ double red[4][GT];
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < np; b += GT)
    for (int q = 0; q < 4; ++q) t[q] += part[4 * b + q];
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = t[q];
  __syncthreads();
  for (int h = GT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    const int a = threadIdx.x;
    cc[a] = red[0][0] != 0.0 ? red[1 + a][0] / red[0][0] : L.x0[a] + 0.5 * L.n[a] * L.dx[a];
  }
}

// partial moments per CTA: sum S dV R_l^m(x - c), 2 MP_NC values
template <int LM>
__global__ void __launch_bounds__(GT) k_mp_moments(Lev L, const double *__restrict__ cc, double *part) {
  constexpr int NC = (LM + 1) * (LM + 2) / 2;
  __shared__ double red[2 * NC][GT / 32];
  const unsigned n = (unsigned)L.n[0] * L.n[1] * L.n[2];
  const double dV = L.dx[0] * L.dx[1] * L.dx[2];
  double acc[2 * NC];
#pragma unroll
  for (int q = 0; q < 2 * NC; ++q) acc[q] = 0.0;
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    const double S = L.src[c];
    if (S == 0.0) continue;
    int i, j, k;
    decompose(L, c, i, j, k);
    const double d[3] = {L.x0[0] + (i + 0.5) * L.dx[0] - cc[0], L.x0[1] + (j + 0.5) * L.dx[1] - cc[1],
                         L.x0[2] + (k + 0.5) * L.dx[2] - cc[2]};
    double R[2 * MP_NC];
    solid_harmonics(LM, d, R);
    const double w = S * dV;
#pragma unroll
    for (int q = 0; q < 2 * NC; ++q) acc[q] = fma(w, R[q], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < 2 * NC; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 2 * NC; q += GT) {
    double t = 0.0;
    for (int w = 0; w < GT / 32; ++w) t += red[q][w];
    part[2 * MP_NC * blockIdx.x + q] = t;
  }
}

// coefficients (A_lm, B_lm) = (2 - delta_m0) (l-m)! / (l+m)! / (4 pi) x the
// moments; one CTA per coefficient, a fixed-order tree over the partial sums
__global__ void __launch_bounds__(GT) k_mp_coef(const double *__restrict__ part, int np, int lmax, double *cc) {
  __shared__ double red[GT];
  const int q = blockIdx.x;
  double t = 0.0;
  for (int b = threadIdx.x; b < np; b += GT) t += part[2 * MP_NC * b + q];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int h = GT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int pair = q >> 1;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= pair) ++l;
    const int m = pair - l * (l + 1) / 2;
    double f = (m ? 2.0 : 1.0) / (4.0 * M_PI);
    for (int v = l - m + 1; v <= l + m; ++v) f /= v;   // (l-m)! / (l+m)!
    cc[3 + q] = l <= lmax ? red[0] * f : 0.0;
  }
}

// phi on the boundary faces of every level
struct FaceJob {
  Lev L;
  int start[7];   // entries of the faces x-, x+, ..., z+ of this level
};
__global__ void __launch_bounds__(GT) k_mp_faces(FaceJob job, MP mp, double *out) {
  const Lev &L = job.L;
  for (int e = blockIdx.x * GT + threadIdx.x; e < job.start[6]; e += gridDim.x * GT) {
    int f = 0;
    while (e >= job.start[f + 1]) ++f;
    const int a = f >> 1, side = f & 1;
    const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    const int r = e - job.start[f];
    int c[3];
    c[t1] = r % L.n[t1];
    c[t2] = r / L.n[t1];
    c[a] = side ? L.n[a] - 1 : 0;
    double x[3];
    for (int b = 0; b < 3; ++b) x[b] = L.x0[b] + (c[b] + 0.5) * L.dx[b];
    x[a] += (side ? 0.5 : -0.5) * L.dx[a];
    out[e] = mp_eval(mp, x);
  }
}

unsigned grid_for(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + GT - 1) / GT, 152LL * 8));
}

}  // namespace

// ------------------------------------------------------------- host side ----

struct GravState {
  long long launches = 0;   // kernels launched since the last count (for the profile)
  cudaGraphExec_t cycle = nullptr;   // one V-cycle + the extra sweep + the defect norm
  int cycle_launches = 0;
  double cycle_key[5] = {0, 0, 0, 0, 0};  // npre, npost, omega, 1, boundary the graph was captured with
  int nl = 0;
  int iso = -1;             // boundary kind the level weights were set for
  Lev lev[40];
  double *part = nullptr, *scal = nullptr;   // partial sums; [0] mean, [1] defect
  int npart = 0;
  double *faces = nullptr;  // isolated: phi on the boundary faces of every level
  int face_start[40][7];
  double *mp = nullptr;     // centre (3) + coefficients (2 MP_NC)
  double *mpart = nullptr;  // partial moments, 2 MP_NC per CTA
  long long *out_flat = nullptr;   // isolated: MeshBlock ghost cells beyond the boundary
  int *out_g = nullptr;            // their global indices (3 per cell)
  int nout = -1;                   // -1: list not built
};

static void grav_free(GravState *g) {
  if (!g) return;
  if (g->cycle) cudaGraphExecDestroy(g->cycle);
  for (int l = 0; l < g->nl; ++l) {
    cudaFree(g->lev[l].phi);
    cudaFree(g->lev[l].src);
    cudaFree(g->lev[l].tmp);
  }
  cudaFree(g->part);
  cudaFree(g->scal);
  cudaFree(g->faces);
  cudaFree(g->mp);
  cudaFree(g->mpart);
  cudaFree(g->out_flat);
  cudaFree(g->out_g);
  delete g;
}

void gravity_release(tde_mesh *m) {
  grav_free(reinterpret_cast<GravState *>(m->grav));
  m->grav = nullptr;
  cudaFree(m->d_phi_sg);
  m->d_phi_sg = nullptr;
}

// the operator's weights of every level for the boundary kind
static void set_weights(GravState *g, const Phys &p, int iso) {
  for (int l = 0; l < g->nl; ++l) {
    Lev &L = g->lev[l];
    const double *h = L.dx;
    double w[3], wsum = 0.0;
    for (int a = 0; a < 3; ++a) {
      const bool on = iso ? p.N[a] > 1 : L.n[a] > 1;
      w[a] = on ? (h[0] / h[a]) * (h[0] / h[a]) : 0.0;
      wsum += w[a];
    }
    const double diag = 2.0 * wsum;
    for (int a = 0; a < 3; ++a) {
      L.aw[a] = w[a] / (h[0] * h[0]);
      L.cw[a] = diag > 0.0 ? w[a] / diag : 0.0;
    }
    L.cs = diag > 0.0 ? h[0] * h[0] / diag : 0.0;
    for (int a = 0; a < 3; ++a) L.act[a] = w[a] != 0.0;
    L.iso = iso;
    for (int f = 0; f < 6; ++f) L.gf[f] = iso ? g->faces + g->face_start[l][f] : nullptr;
  }
  g->iso = iso;
}

static cudaError_t grav_init(tde_mesh *m) {
  if (m->grav) return cudaSuccess;
  GravState *g = new GravState;
  int n[3] = {m->phys.N[0], m->phys.N[1], m->phys.N[2]};
  double h[3] = {m->phys.dx[0], m->phys.dx[1], m->phys.dx[2]};
  cudaError_t err = cudaSuccess;
  int nface = 0;
  for (;;) {
    Lev &L = g->lev[g->nl];
    for (int a = 0; a < 3; ++a) { L.n[a] = n[a]; L.dx[a] = h[a]; L.x0[a] = m->phys.xmin[a]; }
    int *fs = g->face_start[g->nl];
    fs[0] = nface;
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1, t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
      nface += m->phys.N[a] > 1 ? n[t1] * n[t2] : 0;
      fs[f + 1] = nface;
    }
    ++g->nl;
    const size_t nc = (size_t)n[0] * n[1] * n[2];
    L.phi = L.src = L.tmp = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&L.phi, sizeof(double) * nc);
    if (err == cudaSuccess) err = cudaMalloc(&L.src, sizeof(double) * nc);
    if (err == cudaSuccess) err = cudaMalloc(&L.tmp, sizeof(double) * nc);
    if (err == cudaSuccess) err = cudaMemset(L.phi, 0, sizeof(double) * nc);
    if (n[0] == 1 && n[1] == 1 && n[2] == 1) break;
    for (int a = 0; a < 3; ++a)
      if (n[a] > 1) { n[a] /= 2; h[a] *= 2.0; }
  }
  g->npart = (int)grid_for((long long)m->phys.N[0] * m->phys.N[1] * m->phys.N[2]);
  if (err == cudaSuccess) err = cudaMalloc(&g->part, sizeof(double) * 4 * g->npart);
  if (err == cudaSuccess) err = cudaMalloc(&g->scal, sizeof(double) * 2);
  if (err == cudaSuccess) err = cudaMalloc(&g->faces, sizeof(double) * std::max(nface, 1));
  if (err == cudaSuccess) err = cudaMalloc(&g->mp, sizeof(double) * (3 + 2 * MP_NC));
  if (err == cudaSuccess) err = cudaMalloc(&g->mpart, sizeof(double) * 2 * MP_NC * g->npart);
  if (err == cudaSuccess && !m->d_phi_sg) err = cudaMalloc(&m->d_phi_sg, sizeof(double) * m->ntot);
  if (err == cudaSuccess) err = cudaMemset(m->d_phi_sg, 0, sizeof(double) * m->ntot);
  if (err == cudaSuccess) err = cudaMemset(g->mp, 0, sizeof(double) * (3 + 2 * MP_NC));
  if (err != cudaSuccess) {
    grav_free(g);
    return err;
  }
  m->grav = g;
  return cudaSuccess;
}

static cudaError_t reduce(GravState *g, const Lev &L, int sq, double *out, cudaStream_t s) {
  const long long n = (long long)L.n[0] * L.n[1] * L.n[2];
  const unsigned gr = std::min<unsigned>(grid_for(n), (unsigned)g->npart);
  k_mg_partial<<<gr, GT, 0, s>>>(L, sq, g->part);
  k_mg_final<<<1, GT, 0, s>>>(g->part, (int)gr, (double)n, sq, out);
  g->launches += 2;
  return cudaGetLastError();
}

static void smooth(GravState *g, const Lev &L, double omega, cudaStream_t s) {
  if (L.n[0] * L.n[1] * L.n[2] == 1) return;
  const long long half = (long long)L.n[1] * L.n[2] * ((L.n[0] + 1) / 2);
  for (int colour = 0; colour < 2; ++colour) k_mg_smooth<<<grid_for(half), GT, 0, s>>>(L, colour, omega);
  g->launches += 2;
}

static void vcycle(GravState *g, int l, const tde_grav_params &gp, cudaStream_t s) {
  if (l == g->nl - 1) {
    // a single cell: periodic, the correction is zero; isolated, solved exactly
    if (g->iso) {
      k_mg_exact1<<<1, 32, 0, s>>>(g->lev[l]);
      g->launches += 1;
    }
    return;
  }
  const Lev &F = g->lev[l], &C = g->lev[l + 1];
  for (int q = 0; q < gp.npre; ++q) smooth(g, F, gp.omega, s);
  const long long nc = (long long)C.n[0] * C.n[1] * C.n[2];
  const double inv = (double)nc / ((double)F.n[0] * F.n[1] * F.n[2]);   // 1 / children per cell
  k_mg_restrict<<<grid_for(nc), GT, 0, s>>>(F, C, inv);
  k_mg_fas<<<grid_for(nc), GT, 0, s>>>(C);
  vcycle(g, l + 1, gp, s);
  k_mg_corr<<<grid_for(nc), GT, 0, s>>>(C);
  if (prolong_tiles(F, C))
    k_mg_prolong_tiled<0><<<prolong_tile_count(F), GT, 0, s>>>(F, C, MP{0, nullptr});
  else
    k_mg_prolong<<<grid_for((long long)F.n[0] * F.n[1] * F.n[2]), GT, 0, s>>>(F, C);
  g->launches += 4;
  for (int q = 0; q < gp.npost; ++q) smooth(g, F, gp.omega, s);
}

// isolated: the centroid, the moments, and phi on every level's boundary faces
static void multipole_setup(GravState *g, int lmax, cudaStream_t s) {
  const Lev &L0 = g->lev[0];
  const long long n0 = (long long)L0.n[0] * L0.n[1] * L0.n[2];
  const unsigned gr = std::min<unsigned>(grid_for(n0), (unsigned)g->npart);
  k_mp_centroid<<<gr, GT, 0, s>>>(L0, g->part);
  k_mp_centre<<<1, GT, 0, s>>>(g->part, (int)gr, L0, g->mp);
  switch (lmax) {
    case 0: k_mp_moments<0><<<gr, GT, 0, s>>>(L0, g->mp, g->mpart); break;
    case 1: k_mp_moments<1><<<gr, GT, 0, s>>>(L0, g->mp, g->mpart); break;
    case 2: k_mp_moments<2><<<gr, GT, 0, s>>>(L0, g->mp, g->mpart); break;
    case 3: k_mp_moments<3><<<gr, GT, 0, s>>>(L0, g->mp, g->mpart); break;
    default: k_mp_moments<4><<<gr, GT, 0, s>>>(L0, g->mp, g->mpart); break;
  }
  k_mp_coef<<<2 * MP_NC, GT, 0, s>>>(g->mpart, (int)gr, lmax, g->mp);
  const MP mp{lmax, g->mp};
  for (int l = 0; l < g->nl; ++l) {
    FaceJob job;
    job.L = g->lev[l];
    for (int f = 0; f < 7; ++f) job.start[f] = g->face_start[l][f] - g->face_start[l][0];
    if (job.start[6] == 0) continue;
    k_mp_faces<<<grid_for(job.start[6]), GT, 0, s>>>(job, mp, g->faces + g->face_start[l][0]);
    g->launches += 1;
  }
  g->launches += 4;
}

// full multigrid: the source on every level, the coarsest solved, then per finer
// level the prolonged solution and one V-cycle (the extra sweep on the finest)
static void full_multigrid(GravState *g, const tde_grav_params &gp, int lmax, cudaStream_t s) {
  for (int l = 1; l < g->nl; ++l) {
    const Lev &F = g->lev[l - 1], &C = g->lev[l];
    const long long nc = (long long)C.n[0] * C.n[1] * C.n[2];
    k_mg_restrict_src<<<grid_for(nc), GT, 0, s>>>(F, C, (double)nc / ((double)F.n[0] * F.n[1] * F.n[2]));
    g->launches += 1;
  }
  cudaMemsetAsync(g->lev[g->nl - 1].phi, 0, sizeof(double), s);
  vcycle(g, g->nl - 1, gp, s);
  const MP mp{lmax, g->mp};
  for (int l = g->nl - 2; l >= 0; --l) {
    const Lev &F = g->lev[l];
    if (prolong_tiles(F, g->lev[l + 1]))
      k_mg_prolong_tiled<1><<<prolong_tile_count(F), GT, 0, s>>>(F, g->lev[l + 1], mp);
    else
      k_mg_prolong_full<<<grid_for((long long)F.n[0] * F.n[1] * F.n[2]), GT, 0, s>>>(F, g->lev[l + 1], mp);
    g->launches += 1;
    vcycle(g, l, gp, s);
    if (l == 0) smooth(g, F, gp.omega, s);
  }
}

cudaError_t gravity_solve(tde_mesh *m, const tde_grav_params &gp, int *cycles, double *defect) {
  tde_ctx *c = m->ctx;
  cudaStream_t s = c->stream;
  cudaError_t err = grav_init(m);
  if (err != cudaSuccess) return err;
  GravState *g = reinterpret_cast<GravState *>(m->grav);
  const int iso = gp.boundary == TDE_GRAV_ISOLATED ? 1 : 0;
  if (g->iso != iso) set_weights(g, m->phys, iso);
  Lev &L0 = g->lev[0];
  const long long n0 = (long long)L0.n[0] * L0.n[1] * L0.n[2];
  {
    ProfScope ps(c, TDE_K_GRAV, false);
    dim3 grid((unsigned)std::min<int64_t>((m->max_interior + GT - 1) / GT, 64), (unsigned)m->nb);
    k_mg_gather<<<grid, GT, 0, s>>>(m->phys, m->d_blocks, m->U, L0, 4.0 * M_PI * gp.G, gp.rho_min);
    if (!gp.warm || gp.fmg) cudaMemsetAsync(L0.phi, 0, sizeof(double) * n0, s);
    if (iso) {
      multipole_setup(g, gp.lmax, s);
    } else {
      for (int pass = 0; pass < 2; ++pass) {   // the source's mean, removed in two passes
        reduce(g, L0, 0, g->scal, s);
        k_mg_sub_mean<<<grid_for(n0), GT, 0, s>>>(L0, g->scal);
      }
      g->launches += 2;
    }
    if (gp.fmg) full_multigrid(g, gp, gp.lmax, s);
  }
  int ncyc = 0;
  double d = 0.0;
  {
    ProfScope ps(c, TDE_K_GRAV, false);
    reduce(g, L0, 1, g->scal + 1, s);
  }
  // one cycle (V-cycle, the extra fine sweep, the defect norm) as a CUDA graph:
  // about a hundred small launches on the coarse levels replayed as one
  const double key[5] = {(double)gp.npre, (double)gp.npost, gp.omega, 1.0, (double)iso};
  if (g->cycle && memcmp(key, g->cycle_key, sizeof key) != 0) {
    cudaGraphExecDestroy(g->cycle);
    g->cycle = nullptr;
  }
  if (!g->cycle && gp.max_cycles > 0) {
    // captured on the mesh's private stream (the context's stream may be the
    // legacy default stream, which cannot be captured), after the work queued so far
    if (!m->cap_stream) {
      err = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
      if (err != cudaSuccess) return err;
    }
    err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    const long long before = g->launches;
    cudaStream_t cs = m->cap_stream;
    cudaGraph_t graph = nullptr;
    err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      vcycle(g, 0, gp, cs);
      smooth(g, L0, gp.omega, cs);   // the extra sweep on the finest level
      reduce(g, L0, 1, g->scal + 1, cs);
      err = cudaStreamEndCapture(cs, &graph);
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&g->cycle, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
      g->cycle = nullptr;
      return err;
    }
    g->cycle_launches = (int)(g->launches - before);
    g->launches = before;
    memcpy(g->cycle_key, key, sizeof key);
  }
  for (;;) {
    err = cudaMemcpyAsync(&d, g->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    if (d < gp.tol || ncyc >= gp.max_cycles) break;
    ProfScope ps(c, TDE_K_GRAV, false);
    err = cudaGraphLaunch(g->cycle, s);
    if (err != cudaSuccess) return err;
    g->launches += g->cycle_launches;
    ++ncyc;
  }
  if (iso && g->nout < 0) {
    // the MeshBlock ghost cells beyond the boundary, once per mesh
    std::vector<long long> fl;
    std::vector<int> gi;
    const Phys &p = m->phys;
    for (int b = 0; b < m->nb; ++b) {
      const DevBlock &B = m->hblocks[b];
      for (int k = 0; k < B.p[2]; ++k)
        for (int j = 0; j < B.p[1]; ++j)
          for (int i = 0; i < B.p[0]; ++i) {
            const int gg[3] = {B.i0 + i - p.g[0], B.j0 + j - p.g[1], B.k0 + k - p.g[2]};
            bool out = false;
            for (int a = 0; a < 3; ++a)
              if (gg[a] < 0 || gg[a] >= p.N[a]) out = true;
            if (!out) continue;
            fl.push_back(B.off + ((long long)k * B.p[1] + j) * B.p[0] + i);
            gi.insert(gi.end(), gg, gg + 3);
          }
    }
    g->nout = (int)fl.size();
    if (g->nout > 0) {
      err = cudaMalloc(&g->out_flat, sizeof(long long) * fl.size());
      if (err == cudaSuccess) err = cudaMalloc(&g->out_g, sizeof(int) * gi.size());
      if (err == cudaSuccess)
        err = cudaMemcpy(g->out_flat, fl.data(), sizeof(long long) * fl.size(), cudaMemcpyHostToDevice);
      if (err == cudaSuccess) err = cudaMemcpy(g->out_g, gi.data(), sizeof(int) * gi.size(), cudaMemcpyHostToDevice);
      if (err != cudaSuccess) return err;
    }
  }
  {
    ProfScope ps(c, TDE_K_GRAV, false);
    dim3 grid((unsigned)std::min<int64_t>((m->max_interior + GT - 1) / GT, 64), (unsigned)m->nb);
    const MP mp{gp.lmax, g->mp};
    k_mg_scatter<<<grid, GT, 0, s>>>(m->phys, m->d_blocks, L0, mp, m->d_phi_sg);
    if (iso && g->nout > 0) {
      k_mg_scatter_out<<<grid_for(g->nout), GT, 0, s>>>(g->out_flat, g->out_g, g->nout, L0, mp, m->d_phi_sg);
      g->launches += 1;
    }
  }
  g->launches += 2;   // gather and scatter (the rest count at launch)
  c->launches[TDE_K_GRAV] += g->launches;
  g->launches = 0;
  if (cycles) *cycles = ncyc;
  if (defect) *defect = d;
  return cudaGetLastError();
}

cudaError_t gravity_copy_phi(tde_mesh *m, double *dst) {
  GravState *g = reinterpret_cast<GravState *>(m->grav);
  if (!g) return cudaErrorInvalidValue;
  const Lev &L0 = g->lev[0];
  return cudaMemcpyAsync(dst, L0.phi, sizeof(double) * L0.n[0] * L0.n[1] * L0.n[2],
                         cudaMemcpyDeviceToDevice, m->ctx->stream);
}

}  // namespace tde
