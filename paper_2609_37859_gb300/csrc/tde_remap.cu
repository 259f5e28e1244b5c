// tde_remap.cu -- conserved-variable remap between two meshes (Sec. 5.2,
// Eqs. remap-state-vector and remap-cell-average): every interior cell of the
// target mesh becomes the mean of N_qd = 2^(active directions) midpoint samples
// (the centres of the cell's halves in each active direction), each a trilinear
// interpolation of the source's cell-centred rho, m and thermal energy density
// (the auxiliary energy where the source evolves it, else E - |m|^2 / (2 rho));
// the target's total energy is rebuilt as U + |m|^2 / (2 rho), so the kinetic
// energy of velocity structure the target cannot hold is dropped, not heated.
// REMAP_TOTAL interpolates E instead.  A target cell that coincides with a
// source cell is copied (a remap onto the same grid is the identity).  Samples
// outside a non-periodic source domain take the floor state at rest; lookups
// beyond the source's edge follow its boundary map (periodic wrap, outflow copy).
//
// Three launches: the source's interior is staged into a ghost-free global
// array (the carried energy formed once per source cell), the per-direction
// sample weights are tabulated per target index, then one thread per target
// cell (the target's MeshBlocks on grid.y) applies the sample average as a
// separable stencil of at most 4 x 4 x 4 staged cells.  Coincident cells are
// copied from the source's own layout through its owner lattice.  32-bit index
// division only (a 64-bit integer division would issue on the FP64 pipe).
#include <math.h>

#include <algorithm>

#include "tde_internal.h"

namespace tde {

namespace {

constexpr int RT = 128;

struct RemapSrc {
  int N[3], bc[3], g[3], unit[3], cn[3];
  double xmin[3], dx[3], idx[3], hi[3];
  const DevBlock *blocks;
  const int32_t *owner;
  const double *U;
  long long ntot;
  int dual;
};

struct RemapDst {
  int g[3], active[3], N[3];
  int coinc;          // same cell widths and aligned centres: src index = dst index + shift
  int shift[3];
  double xmin[3], dx[3];
  const DevBlock *blocks;
  double *U;
  long long ntot;
  int dual, mode;
  double rho_floor, u_floor;
};

// global source index along one direction after the boundary map
__device__ __forceinline__ int src_wrap(int c, int N, int bc) {
  if ((unsigned)c < (unsigned)N) return c;
  if (bc == TDE_BC_PERIODIC) {
    const int r = c % N;
    return r < 0 ? r + N : r;
  }
  return c < 0 ? 0 : N - 1;
}

// padded index of global source cell (i, j, k) after the boundary map
__device__ __forceinline__ long long src_cell(const RemapSrc &s, int i, int j, int k) {
  i = src_wrap(i, s.N[0], s.bc[0]);
  j = src_wrap(j, s.N[1], s.bc[1]);
  k = src_wrap(k, s.N[2], s.bc[2]);
  const int o = s.owner[((unsigned)(k / s.unit[2]) * (unsigned)s.cn[1] + (unsigned)(j / s.unit[1])) *
                            (unsigned)s.cn[0] +
                        (unsigned)(i / s.unit[0])];
  const DevBlock &B = s.blocks[o];
  return B.off + ((long long)(k - B.k0 + s.g[2]) * B.p[1] + (j - B.j0 + s.g[1])) * B.p[0] +
         (i - B.i0 + s.g[0]);
}

// thermal energy density of the source cell at padded index l
__device__ __forceinline__ double src_thermal(const RemapSrc &s, long long l) {
  const double *U = s.U;
  if (s.dual) return U[5 * s.ntot + l];
  const double r = U[l], mx = U[s.ntot + l], my = U[2 * s.ntot + l], mz = U[3 * s.ntot + l];
  return U[4 * s.ntot + l] - 0.5 * (mx * mx + my * my + mz * mz) * rcp_nr(r);
}

// Stage: the source's interior cells into a ghost-free global array [5][Nz][Ny][Nx]
// of rho, m and the carried energy (thermal energy density, or E in the total
// form); the thermal energy is formed once per source cell here.
__global__ void __launch_bounds__(RT) k_remap_stage(RemapSrc s, int mode, double *__restrict__ G) {
  const DevBlock B = s.blocks[blockIdx.y];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  const long long nc = (long long)s.N[0] * s.N[1] * s.N[2];
  for (int e = blockIdx.x * RT + threadIdx.x; e < nint; e += gridDim.x * RT) {
    const int i = e % B.n[0], q = e / B.n[0];
    const int j = q % B.n[1], k = q / B.n[1];
    const long long l = B.off + ((long long)(k + s.g[2]) * B.p[1] + (j + s.g[1])) * B.p[0] + (i + s.g[0]);
    const long long c = ((long long)(B.k0 + k) * s.N[1] + (B.j0 + j)) * s.N[0] + (B.i0 + i);
#pragma unroll
    for (int v = 0; v < 4; ++v) G[v * nc + c] = s.U[v * s.ntot + l];
    G[4 * nc + c] = mode == TDE_REMAP_TOTAL ? s.U[4 * s.ntot + l] : src_thermal(s, l);
  }
}

// The sample average of Eq. remap-cell-average is separable: the N_qd samples
// are the product of one or two samples per direction, a sample lies outside the
// source domain when one of its coordinates does, and its trilinear weight is a
// product over directions.  So the target value is
//   sum_{x,y,z} wx wy wz G[z][y][x] + (1 - fx fy fz) floor,
// with, per direction, the averaged weights of the inside samples on at most
// four consecutive source indices, and fa the fraction of inside samples.
struct __align__(16) Axis {
  long long off[4];   // source index (after the boundary map) x the direction's stride
  double w[4];
  int n;              // entries used
  double f;           // fraction of samples inside the source
};

// one sample at coordinate r along direction a: inside the source?  If so its
// lower source index i0 and the fraction t toward i0 + 1
__device__ __forceinline__ bool axis_sample(const RemapSrc &s, int a, double r, int &i0, double &t) {
  if (s.N[a] > 1 && s.bc[a] != TDE_BC_PERIODIC && (r < s.xmin[a] || r > s.hi[a])) return false;
  if (s.N[a] == 1) {
    i0 = 0;
    t = 0.0;
    return true;
  }
  const double sa = (r - s.xmin[a]) * s.idx[a] - 0.5;
  const double fl = floor(sa);
  i0 = (int)fl;
  t = sa - fl;
  return true;
}

__device__ __forceinline__ void axis_weights(const RemapSrc &s, int a, bool active, double xc, double dx,
                                             long long stride, Axis &A) {
  int raw[4] = {0, 0, 0, 0};
  double w[4] = {0.0, 0.0, 0.0, 0.0};
  int n = 0;
  if (!active) {
    int i0;
    double t;
    A.f = axis_sample(s, a, xc, i0, t) ? 1.0 : 0.0;
    if (A.f > 0.0) {
      raw[0] = i0, raw[1] = i0 + 1, w[0] = 1.0 - t, w[1] = t, n = 2;
    }
  } else {
    int ia, ib;
    double ta, tb;
    const bool ina = axis_sample(s, a, xc - 0.25 * dx, ia, ta);
    const bool inb = axis_sample(s, a, xc + 0.25 * dx, ib, tb);
    A.f = 0.5 * ((ina ? 1 : 0) + (inb ? 1 : 0));
    if (ina && inb) {   // ib >= ia: the samples are in increasing order
      if (ib == ia) {
        raw[0] = ia, raw[1] = ia + 1, n = 2;
        w[0] = 0.5 * (1.0 - ta) + 0.5 * (1.0 - tb);
        w[1] = 0.5 * ta + 0.5 * tb;
      } else if (ib == ia + 1) {
        raw[0] = ia, raw[1] = ia + 1, raw[2] = ia + 2, n = 3;
        w[0] = 0.5 * (1.0 - ta);
        w[1] = 0.5 * ta + 0.5 * (1.0 - tb);
        w[2] = 0.5 * tb;
      } else {
        raw[0] = ia, raw[1] = ia + 1, raw[2] = ib, raw[3] = ib + 1, n = 4;
        w[0] = 0.5 * (1.0 - ta), w[1] = 0.5 * ta, w[2] = 0.5 * (1.0 - tb), w[3] = 0.5 * tb;
      }
    } else if (ina || inb) {
      const int i0 = ina ? ia : ib;
      const double t = ina ? ta : tb;
      raw[0] = i0, raw[1] = i0 + 1, w[0] = 0.5 * (1.0 - t), w[1] = 0.5 * t, n = 2;
    }
  }
  // drop a trailing zero weight (a sample on a source centre)
  if (n == 2 && w[1] == 0.0) n = 1;
  else if (n == 3 && w[2] == 0.0) n = 2;
  else if (n == 4 && w[3] == 0.0) n = 3;
  A.n = n;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    A.off[e] = e < n ? (long long)src_wrap(raw[e], s.N[a], s.bc[a]) * stride : 0;
    A.w[e] = e < n ? w[e] : 0.0;
  }
}

// The weights along direction a depend only on the target cell's index along a:
// one table entry per target index of each direction (tab[a] has N[a] entries).
__global__ void __launch_bounds__(RT) k_remap_axes(RemapDst d, RemapSrc s, Axis *__restrict__ tab) {
  const int t = blockIdx.x * RT + threadIdx.x;
  const int n01 = d.N[0] + d.N[1];
  if (t >= n01 + d.N[2]) return;
  const int a = t < d.N[0] ? 0 : (t < n01 ? 1 : 2);
  const int g = t - (a == 0 ? 0 : (a == 1 ? d.N[0] : n01));
  const long long stride = a == 0 ? 1 : (a == 1 ? (long long)s.N[0] : (long long)s.N[0] * s.N[1]);
  Axis A;
  axis_weights(s, a, d.active[a] != 0, d.xmin[a] + (g + 0.5) * d.dx[a], d.dx[a], stride, A);
  tab[t] = A;
}

__global__ void __launch_bounds__(RT) k_remap(RemapDst d, RemapSrc s, const double *__restrict__ G,
                                              const Axis *__restrict__ tab) {
  const DevBlock B = d.blocks[blockIdx.y];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  const long long nc = (long long)s.N[0] * s.N[1] * s.N[2];
  for (int e = blockIdx.x * RT + threadIdx.x; e < nint; e += gridDim.x * RT) {
    const int i = e % B.n[0], q = e / B.n[0];
    const int j = q % B.n[1], k = q / B.n[1];
    const int gi = B.i0 + i, gj = B.j0 + j, gk = B.k0 + k;
    const long long l =
        B.off + ((long long)(k + d.g[2]) * B.p[1] + (j + d.g[1])) * B.p[0] + (i + d.g[0]);
    if (d.coinc) {   // a coincident source cell is copied
      const int si = gi + d.shift[0], sj = gj + d.shift[1], sk = gk + d.shift[2];
      if ((unsigned)si < (unsigned)s.N[0] && (unsigned)sj < (unsigned)s.N[1] && (unsigned)sk < (unsigned)s.N[2]) {
        const long long c = src_cell(s, si, sj, sk);
#pragma unroll
        for (int v = 0; v < 5; ++v) d.U[v * d.ntot + l] = s.U[v * s.ntot + c];
        if (d.dual) d.U[5 * d.ntot + l] = src_thermal(s, c);
        continue;
      }
    }
    const Axis &X = tab[gi], &Y = tab[d.N[0] + gj], &Z = tab[d.N[0] + d.N[1] + gk];
    const int nx = X.n, ny = Y.n, nz = Z.n;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int cz = 0; cz < 4; ++cz) {
      if (cz >= nz) break;
#pragma unroll
      for (int cy = 0; cy < 4; ++cy) {
        if (cy >= ny) break;
        const double wyz = Z.w[cz] * Y.w[cy];
        const double *row = G + Z.off[cz] + Y.off[cy];
#pragma unroll
        for (int cx = 0; cx < 4; ++cx) {
          if (cx >= nx) break;
          const double w = X.w[cx] * wyz;
          const double *p = row + X.off[cx];
#pragma unroll
          for (int v = 0; v < 5; ++v) acc[v] = fma(w, __ldg(p + v * nc), acc[v]);
        }
      }
    }
    const double ffl = 1.0 - X.f * Y.f * Z.f;   // the floor samples' share
    if (dgt0(ffl)) {
      acc[0] = fma(ffl, d.rho_floor, acc[0]);
      acc[4] = fma(ffl, d.u_floor, acc[4]);
    }
    const double ke = 0.5 * (acc[1] * acc[1] + acc[2] * acc[2] + acc[3] * acc[3]) * rcp_nr(acc[0]);
    d.U[l] = acc[0];
#pragma unroll
    for (int v = 1; v < 4; ++v) d.U[v * d.ntot + l] = acc[v];
    if (d.mode == TDE_REMAP_TOTAL) {
      d.U[4 * d.ntot + l] = acc[4];
      if (d.dual) d.U[5 * d.ntot + l] = acc[4] - ke;
    } else {
      d.U[4 * d.ntot + l] = acc[4] + ke;
      if (d.dual) d.U[5 * d.ntot + l] = acc[4];
    }
  }
}

}  // namespace

cudaError_t launch_remap(tde_mesh *dst, double *Udst, const tde_mesh *src, const double *Usrc, int mode,
                         double rho_floor, double u_floor) {
  RemapSrc s{};
  RemapDst d{};
  const Phys &S = src->phys, &D = dst->phys;
  for (int a = 0; a < 3; ++a) {
    s.N[a] = S.N[a];
    s.bc[a] = S.bc[a];
    s.g[a] = S.g[a];
    s.unit[a] = src->unit[a];
    s.cn[a] = src->cn[a];
    s.xmin[a] = S.xmin[a];
    s.dx[a] = S.dx[a];
    s.idx[a] = 1.0 / S.dx[a];
    s.hi[a] = S.xmin[a] + S.N[a] * S.dx[a];
    d.g[a] = D.g[a];
    d.N[a] = D.N[a];
    d.active[a] = D.N[a] > 1;
    d.xmin[a] = D.xmin[a];
    d.dx[a] = D.dx[a];
  }
  s.blocks = src->d_blocks;
  s.owner = src->d_owner;
  s.U = Usrc;
  s.ntot = (long long)src->ntot;
  s.dual = S.dual;
  d.blocks = dst->d_blocks;
  d.U = Udst;
  d.ntot = (long long)dst->ntot;
  d.dual = D.dual;
  d.mode = mode;
  d.rho_floor = rho_floor;
  d.u_floor = u_floor;
  // coincidence (a dst cell centred on a src cell of the same widths, within
  // 1e-9 cells) holds for every cell or none: same widths and aligned origins
  d.coinc = 1;
  for (int a = 0; a < 3; ++a) {
    const double sh = (D.xmin[a] - S.xmin[a]) / S.dx[a];
    const double r = floor(sh + 0.5);
    d.shift[a] = (int)r;
    if (fabs(D.dx[a] - S.dx[a]) > 1e-12 * S.dx[a] || fabs(sh - r) > 1e-9) d.coinc = 0;
  }
  cudaStream_t st = dst->ctx->stream;
  const long long nc = (long long)S.N[0] * S.N[1] * S.N[2];
  const int ntab = D.N[0] + D.N[1] + D.N[2];
  const size_t gbytes = (sizeof(double) * 5 * nc + 255) / 256 * 256;
  double *G = nullptr;
  cudaError_t err = cudaMallocAsync((void **)&G, gbytes + sizeof(Axis) * ntab, st);
  if (err != cudaSuccess) return err;
  Axis *tab = (Axis *)((char *)G + gbytes);
  {
    ProfScope _ps(dst->ctx, TDE_K_SCALAR);
    const dim3 grid((unsigned)std::min<int64_t>((src->max_interior + RT - 1) / RT, 64), (unsigned)src->nb);
    k_remap_stage<<<grid, RT, 0, st>>>(s, mode, G);
  }
  {
    ProfScope _ps(dst->ctx, TDE_K_SCALAR);
    k_remap_axes<<<(ntab + RT - 1) / RT, RT, 0, st>>>(d, s, tab);
  }
  {
    ProfScope _ps(dst->ctx, TDE_K_REMAP);
    const dim3 grid((unsigned)std::min<int64_t>((dst->max_interior + RT - 1) / RT, 64), (unsigned)dst->nb);
    k_remap<<<grid, RT, 0, st>>>(d, s, G, tab);
  }
  err = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(G, st);
  return err != cudaSuccess ? err : e2;
}

}  // namespace tde
