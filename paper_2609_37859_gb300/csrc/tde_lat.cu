// tde_lat.cu -- localized adaptive time stepping (Sec. 7 of the paper) on the GPU.
//
//  * k_lat_factors: one CTA computes dt0 = min_b dt_b (Eq. lat-base-dt), the
//    power-of-two factors of Eq. lat-factor (exact floor(log2) via ilogb),
//    merges sparse top bins and limits neighbouring factors to a ratio of two
//    and, across coarse-fine interfaces, f_fine <= f_coarse by Jacobi passes
//    (the greatest fixed point, the same as any pass order);
//    the pass count is bounded and an overrun is reported in a status word.
//  * A window of f_max * dt0 advances, at each fine sub-step tau, every level
//    f with tau mod f = 0 as ONE batched launch sequence over that level's block
//    list (slow levels first).  The blocks sorted by factor make every level a
//    contiguous segment and the set of blocks completing at tau a prefix.
//  * k_ghost_lat fills conserved ghost cells per source block: faster -> frozen
//    current state, slower -> linear interpolation in time between the stored
//    start-of-step state and the end state; those cells (and the refined-mesh
//    ghosts of k_ghost_amr) are then converted to primitives from a per-level
//    list built on the device (k_glist_*), while ghost cells whose source block
//    is on the same schedule take that block's primitives (k_ghost_w_lat).
//  * The sweeps add dt (F^1 + F^2)/2 of every boundary face to per-face-cell
//    registers; k_reflux corrects the slower side of every mixed face at its
//    completion (Eq. lat-flux-impulse, Eq. lat-grav-reflux), one CTA per block,
//    faces in a fixed order so that shared corner cells are updated
//    deterministically.
//  * The whole window can be captured once in a CUDA graph and replayed while
//    the factors, the point-mass state and the parameters stay the same.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>

#include "tde_internal.h"

namespace tde {

cudaError_t launch_c2p(tde_mesh *m, const double *Uin, int nblk, const int32_t *ids, bool want_dt,
                       const BH &bh, TimeArgs ta);
cudaError_t launch_dt_finalize(tde_mesh *m, double cfl, double *dt_block, double *dt_min);
cudaError_t launch_excise(tde_mesh *m, double *U, int nblk, const int32_t *ids, const BH &bh,
                          TimeArgs ta);
cudaError_t launch_sync(tde_mesh *m, double *U, int nblk, const int32_t *ids, double eta2);

constexpr int LNT = 256;

__global__ void __launch_bounds__(1024) k_lat_factors(int nb, const double *__restrict__ dt, int n_lat,
                                                      double merge_frac,
                                                      const int32_t *__restrict__ nbr_start,
                                                      const int32_t *__restrict__ nbr,
                                                      const DevBlock *__restrict__ blocks, int32_t *f,
                                                      int32_t *f2, double *scal, int *flag) {
  __shared__ double sd[32];
  __shared__ int si[32], sc[32];
  __shared__ double s_dt0;
  __shared__ int s_fmax, s_cnt, s_changed;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  double m = INFINITY;
  for (int b = tid; b < nb; b += blockDim.x) m = fmin(m, dt[b]);
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) sd[wid] = m;
  __syncthreads();
  if (tid == 0) {
    double v = INFINITY;
    for (int w = 0; w < nw; ++w) v = fmin(v, sd[w]);
    s_dt0 = v;
  }
  __syncthreads();
  const double dt0 = s_dt0;
  for (int b = tid; b < nb; b += blockDim.x) {
    int k = ilogb(dt[b] / dt0);
    if (k > n_lat) k = n_lat;
    if (k < 0) k = 0;
    f[b] = 1 << k;
  }
  __syncthreads();
  // merge sparse top bins
  for (int it = 0; it <= n_lat; ++it) {
    int fm = 1;
    for (int b = tid; b < nb; b += blockDim.x) fm = max(fm, f[b]);
    for (int o = 16; o > 0; o >>= 1) fm = max(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if (lane == 0) si[wid] = fm;
    __syncthreads();
    if (tid == 0) {
      int v = 1;
      for (int w = 0; w < nw; ++w) v = max(v, si[w]);
      s_fmax = v;
    }
    __syncthreads();
    const int top = s_fmax;
    int c = 0;
    for (int b = tid; b < nb; b += blockDim.x) c += f[b] == top;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) sc[wid] = c;
    __syncthreads();
    if (tid == 0) {
      int v = 0;
      for (int w = 0; w < nw; ++w) v += sc[w];
      s_cnt = v;
    }
    __syncthreads();
    if (top == 1 || s_cnt >= merge_frac * nb) break;
    for (int b = tid; b < nb; b += blockDim.x)
      if (f[b] == top) f[b] = top / 2;
    __syncthreads();
  }
  // neighbour limiting, Jacobi passes into f2
  const long long max_pass = (long long)nb * (n_lat + 1) + 2;
  bool converged = false;
  for (long long pass = 0; pass < max_pass; ++pass) {
    if (tid == 0) s_changed = 0;
    __syncthreads();
    for (int b = tid; b < nb; b += blockDim.x) {
      int v = f[b], lim = v;
      const int Lb = blocks[b].level;
      // f_b <= 2 f_o; across a coarse-fine interface also f_fine <= f_coarse
      for (int q = nbr_start[b]; q < nbr_start[b + 1]; ++q) {
        const int o = nbr[q];
        lim = min(lim, (Lb > blocks[o].level ? 1 : 2) * f[o]);
      }
      f2[b] = lim;
      if (lim < v) s_changed = 1;
    }
    __syncthreads();
    for (int b = tid; b < nb; b += blockDim.x) f[b] = f2[b];
    __syncthreads();
    if (!s_changed) { converged = true; break; }
    __syncthreads();
  }
  if (tid == 0) {
    scal[3] = dt0;
    *flag = converged ? 0 : 1;
  }
}

// dt_b = f_b dt0 for the window
__global__ void k_lat_prepare(int nb, const int32_t *__restrict__ f, double *dtb,
                              const double *__restrict__ scal) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
    dtb[b] = f[b] * scal[3];
}

// step start time of the listed blocks: t_window + tau dt0
__global__ void k_lat_time(const int32_t *__restrict__ ids, int n, int tau, double *tstart,
                           const double *__restrict__ scal) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    tstart[ids[q]] = scal[0] + tau * scal[3];
}

// window end: t += f_max dt0
__global__ void k_lat_advance(double *scal, int fmax) {
  scal[1] = fmax * scal[3];
  scal[0] += scal[1];
}

// copy the listed blocks (all padded cells, all fields) src -> dst
__global__ void __launch_bounds__(LNT) k_copy_blocks(const DevBlock *__restrict__ blocks,
                                                     const int32_t *__restrict__ ids,
                                                     const double *__restrict__ src, double *dst,
                                                     int nvar, long long ntot) {
  const DevBlock B = blocks[ids[blockIdx.y]];
  const long long n = (long long)B.p[0] * B.p[1] * B.p[2];
  for (long long e = blockIdx.x * (long long)LNT + threadIdx.x; e < n; e += (long long)gridDim.x * LNT)
    for (int v = 0; v < nvar; ++v) dst[v * ntot + B.off + e] = src[v * ntot + B.off + e];
}

__global__ void __launch_bounds__(LNT) k_ghost_lat(const int32_t *__restrict__ map,
                                                   const int32_t *__restrict__ gstart,
                                                   const int32_t *__restrict__ gend,
                                                   const int32_t *__restrict__ gsrcb,
                                                   const int32_t *__restrict__ ids,
                                                   const int32_t *__restrict__ f, int flevel,
                                                   int tau, int stage, double *Udst,
                                                   const double *__restrict__ Ucur,
                                                   const double *__restrict__ Uold, int nvar,
                                                   long long ntot) {
  const int b = ids[blockIdx.y];
  const int s0 = gstart[b], s1 = gend[b];   // the ghost cells the sweeps read
  for (int e = s0 + blockIdx.x * LNT + threadIdx.x; e < s1; e += gridDim.x * LNT) {
    const int2 mp = reinterpret_cast<const int2 *>(map)[e];
    const int fn = f[gsrcb[e]];
    if (fn == flevel) {
      // same schedule: the primitives are copied instead (k_ghost_w_lat), and
      // nothing after reads a conserved ghost value
    } else if (fn < flevel) {
      // every field loaded before any is stored (sources are interior cells,
      // destinations ghost cells), so the loads overlap in flight
      double t[6];
#pragma unroll
      for (int v = 0; v < 6; ++v)
        if (v < nvar) t[v] = Ucur[v * ntot + mp.y];
#pragma unroll
      for (int v = 0; v < 6; ++v)
        if (v < nvar) Udst[v * ntot + mp.x] = t[v];
    } else {
      const double s = (double)(tau % fn + stage * flevel) / (double)fn;
      double t[6];
#pragma unroll
      for (int v = 0; v < 6; ++v)
        if (v < nvar) {
          const double a = Uold[v * ntot + mp.y];
          t[v] = a + s * (Ucur[v * ntot + mp.y] - a);
        }
#pragma unroll
      for (int v = 0; v < 6; ++v)
        if (v < nvar) Udst[v * ntot + mp.x] = t[v];
    }
  }
}

// ---- refined-mesh ghost ops (restriction, prolongation; Sec. 7.1) ----------

struct AmrSrc {
  const double *Udst, *Ucur, *Uold;
  const int32_t *f;   // NULL: every source cell from Udst
  int flevel, tau, stage;
  long long ntot;
};

// the value of padded cell l (variable offset included) of block o at the stage
// time: same level -> Udst, faster -> Ucur, slower -> interpolation in time
__device__ __forceinline__ double amr_fetch(const AmrSrc &S, int o, long long l) {
  if (!S.f) return S.Udst[l];
  const int fn = S.f[o];
  if (fn == S.flevel) return S.Udst[l];
  if (fn < S.flevel) return S.Ucur[l];
  const double sv = (double)(S.tau % fn + S.stage * S.flevel) / (double)fn;
  const double a = S.Uold[l];
  return a + sv * (S.Ucur[l] - a);
}

// mean of the (2^depth)^d cells of a coarse value (depth <= 2), the children
// summed in (z, y, x) order and each level averaged in turn
__device__ double amr_cv(const AmrSrc &S, const Phys &p, const DevBlock *__restrict__ blocks, const AmrCV &cv,
                         long long voff) {
  if (cv.depth == 0) return amr_fetch(S, cv.blk, voff + cv.base);
  const DevBlock O = blocks[cv.blk];
  const long long sx = p.active[0] ? 1 : 0, sy = p.active[1] ? O.p[0] : 0,
                  sz = p.active[2] ? (long long)O.p[0] * O.p[1] : 0;
  const int nx = p.active[0] ? 2 : 1, ny = p.active[1] ? 2 : 1, nz = p.active[2] ? 2 : 1;
  const int nch = nx * ny * nz;
  double acc = 0.0;
  for (int dk = 0; dk < nz; ++dk)
    for (int dj = 0; dj < ny; ++dj)
      for (int di = 0; di < nx; ++di) {
        if (cv.depth == 1) {
          acc += amr_fetch(S, cv.blk, voff + cv.base + dk * sz + dj * sy + di * sx);
        } else {
          const long long c0 = cv.base + 2 * (dk * sz + dj * sy + di * sx);
          double in = 0.0;
          for (int ek = 0; ek < nz; ++ek)
            for (int ej = 0; ej < ny; ++ej)
              for (int ei = 0; ei < nx; ++ei) in += amr_fetch(S, cv.blk, voff + c0 + ek * sz + ej * sy + ei * sx);
          acc += in / nch;
        }
      }
  return acc / nch;
}

__device__ __forceinline__ double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

__global__ void __launch_bounds__(LNT) k_ghost_amr(const AmrOp *__restrict__ ops, const int32_t *__restrict__ start,
                                                   const int32_t *__restrict__ ids, const DevBlock *__restrict__ blocks,
                                                   Phys p, AmrSrc S, double *Udst, int nvar) {
  const int b = ids[blockIdx.y];
  const int s0 = start[b], s1 = start[b + 1];
  for (int e = s0 + blockIdx.x * LNT + threadIdx.x; e < s1; e += gridDim.x * LNT) {
    const AmrOp op = ops[e];
    for (int v = 0; v < nvar; ++v) {
      const long long voff = v * S.ntot;
      const double c0 = amr_cv(S, p, blocks, op.cv[0], voff);
      double out = c0;
      if (op.kind >= 0)
        for (int a = 0; a < 3; ++a) {
          if (!p.active[a]) continue;
          const double cp = amr_cv(S, p, blocks, op.cv[1 + 2 * a], voff);
          const double cm = amr_cv(S, p, blocks, op.cv[2 + 2 * a], voff);
          out += ((op.kind >> a) & 1 ? 0.25 : -0.25) * minmod(cp - c0, c0 - cm);
        }
      Udst[voff + op.dst] = out;
    }
  }
}

// ghost cells whose source block is on the same schedule: the primitives of the
// source interior cell, converted in the same launch sequence (the conversion
// is a function of the cell's conserved values alone, so the copy equals the
// conversion of the copied conserved values bit for bit)
__global__ void __launch_bounds__(LNT) k_ghost_w_lat(const int32_t *__restrict__ map,
                                                     const int32_t *__restrict__ gstart,
                                                     const int32_t *__restrict__ gend,
                                                     const int32_t *__restrict__ gsrcb,
                                                     const int32_t *__restrict__ ids,
                                                     const int32_t *__restrict__ f, int flevel, double *W,
                                                     int nwv, long long ntot) {
  const int b = ids[blockIdx.y];
  const int s0 = gstart[b], s1 = gend[b];
  for (int e = s0 + blockIdx.x * LNT + threadIdx.x; e < s1; e += gridDim.x * LNT) {
    if (f[gsrcb[e]] != flevel) continue;
    const int2 mp = reinterpret_cast<const int2 *>(map)[e];
    double t[8];
#pragma unroll
    for (int v = 0; v < 8; ++v)
      if (v < nwv) t[v] = W[v * ntot + mp.y];
#pragma unroll
    for (int v = 0; v < 8; ++v)
      if (v < nwv) W[v * ntot + mp.x] = t[v];
  }
}

__device__ __forceinline__ void lat_cell_centre(const Phys &p, const DevBlock &B, const int c[3],
                                                double x[3]) {
  const int o[3] = {B.i0, B.j0, B.k0};
  for (int a = 0; a < 3; ++a) {
    int g = o[a] + c[a] - p.g[a];
    if (p.bc[a] == 1) {
      const int N = level_n(p, a, B.level);
      g %= N;
      if (g < 0) g += N;
    }
    x[a] = p.xmin[a] + (g + 0.5) * block_dx(p, B, a);
  }
}

__device__ __forceinline__ long long side_offset(const DevBlock &B, int side, int nvar) {
  long long so = 0;
  for (int s = 0; s < side; ++s) {
    const int aa = s >> 1;
    const int u1 = aa == 0 ? 1 : 0, u2 = aa == 2 ? 1 : 2;
    so += (long long)B.n[u1] * B.n[u2] * nvar;
  }
  return so;
}

// owner block of every cell of the finest level's grid, stored per unit cube
struct OwnerLattice {
  const int32_t *owner;
  int unit[3], cn[3];
  int lmax;
};

// the block owning the level-L cell g (inside the level-L grid)
__device__ __forceinline__ int owner_at(const OwnerLattice &ol, const Phys &p, int L, const int g[3]) {
  int f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) f[a] = p.active[a] ? (g[a] << (ol.lmax - L)) / ol.unit[a] : 0;
  return ol.owner[((long long)f[2] * ol.cn[1] + f[1]) * ol.cn[0] + f[0]];
}

__global__ void __launch_bounds__(LNT) k_reflux(Phys p, BH bh, OwnerLattice ol,
                                                const DevBlock *__restrict__ blocks,
                                                const int32_t *__restrict__ ids,
                                                const int32_t *__restrict__ f, double *U,
                                                long long ntot, double *R,
                                                const long long *__restrict__ fo, int nvar,
                                                const double *__restrict__ scal, int tau, const double *__restrict__ phi_sg) {
  const int b = ids[blockIdx.x];
  const DevBlock B = blocks[b];
  const int fb = f[b];
  const double t = scal[0] + tau * scal[3];
  double rb[3] = {0, 0, 0};
  if (bh.on) {
    const double s = t - bh.t0;
    for (int a = 0; a < 3; ++a) rb[a] = bh.x0[a] + bh.v0[a] * s + 0.5 * bh.a0[a] * s * s;
  }
  const int org[3] = {B.i0, B.j0, B.k0};
  for (int a = 0; a < 3; ++a) {
    if (!p.active[a]) continue;
    const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    for (int side = 0; side < 2; ++side) {
      const int s = 2 * a + side;
      const double sigma = side ? 1.0 : -1.0;
      const int ncell = B.n[t1] * B.n[t2];
      const long long sos = fo[b] + side_offset(B, s, nvar);
      for (int e = threadIdx.x; e < ncell; e += blockDim.x) {
        const int c1 = e % B.n[t1], c2 = e / B.n[t1];
        int ci[3];
        ci[a] = side ? B.n[a] - 1 : 0;
        ci[t1] = c1;
        ci[t2] = c2;
        int g[3] = {org[0] + ci[0], org[1] + ci[1], org[2] + ci[2]};
        g[a] += side ? 1 : -1;
        const int NL = level_n(p, a, B.level);
        if (g[a] < 0 || g[a] >= NL) {
          if (p.bc[a] != 1) continue;
          g[a] = ((g[a] % NL) + NL) % NL;
        }
        const int o = owner_at(ol, p, B.level, g);
        const DevBlock O = blocks[o];
        const int os = 2 * a + (1 - side);
        const long long cs = (long long)c2 * B.n[t1] + c1;
        const int pos[3] = {ci[0] + p.g[0], ci[1] + p.g[1], ci[2] + p.g[2]};
        const long long l = B.off + ((long long)pos[2] * B.p[1] + pos[1]) * B.p[0] + pos[0];
        double dI[6];
        bool correct = false;
        if (O.level == B.level) {
          const int oc[3] = {g[0] - O.i0, g[1] - O.j0, g[2] - O.k0};
          const long long soo = fo[o] + side_offset(O, os, nvar);
          const long long ncell_o = (long long)O.n[t1] * O.n[t2];
          const long long co = (long long)oc[t2] * O.n[t1] + oc[t1];
          if (f[o] < fb) {
            for (int q = 0; q < nvar; ++q) dI[q] = R[soo + q * ncell_o + co] - R[sos + q * ncell + cs];
            for (int q = 0; q < nvar; ++q) R[soo + q * ncell_o + co] = 0.0;
            correct = true;
          }
          if (f[o] <= fb && !correct)
            for (int q = 0; q < nvar; ++q) R[sos + q * ncell + cs] = 0.0;
        } else if (O.level == B.level + 1) {
          // the fine face cells behind this coarse face cell: their impulses are
          // the accepted ones, averaged over the coarse face
          double acc[6] = {0, 0, 0, 0, 0, 0};
          int nf = 0;
          for (int e2 = 0; e2 < (p.active[t2] ? 2 : 1); ++e2)
            for (int e1 = 0; e1 < (p.active[t1] ? 2 : 1); ++e1) {
              int h[3];
              h[a] = side ? 2 * g[a] : 2 * g[a] + 1;
              h[t1] = p.active[t1] ? 2 * g[t1] + e1 : 0;
              h[t2] = p.active[t2] ? 2 * g[t2] + e2 : 0;
              const int o2 = owner_at(ol, p, B.level + 1, h);
              const DevBlock F = blocks[o2];
              const int hc[3] = {h[0] - F.i0, h[1] - F.j0, h[2] - F.k0};
              const long long sof = fo[o2] + side_offset(F, os, nvar);
              const long long ncell_f = (long long)F.n[t1] * F.n[t2];
              const long long cf = (long long)hc[t2] * F.n[t1] + hc[t1];
              for (int q = 0; q < nvar; ++q) {
                acc[q] += R[sof + q * ncell_f + cf];
                R[sof + q * ncell_f + cf] = 0.0;
              }
              ++nf;
            }
          for (int q = 0; q < nvar; ++q) dI[q] = acc[q] / nf - R[sos + q * ncell + cs];
          correct = true;
        }
        // a coarser neighbour (level - 1) reads this block's impulses: kept
        if (correct) {
          const double dxa = block_dx(p, B, a);
          if (bh.on || phi_sg) {
            int pn[3] = {pos[0], pos[1], pos[2]};
            pn[a] += side ? 1 : -1;
            double phi_i = 0.0, phi_n = 0.0;
            if (bh.on) {
              double xi[3], xn[3];
              lat_cell_centre(p, B, pos, xi);
              lat_cell_centre(p, B, pn, xn);
              const double di0 = xi[0] - rb[0], di1 = xi[1] - rb[1], di2 = xi[2] - rb[2];
              const double dn0 = xn[0] - rb[0], dn1 = xn[1] - rb[1], dn2 = xn[2] - rb[2];
              phi_i = -bh.GM / sqrt(di0 * di0 + di1 * di1 + di2 * di2 + bh.rs2);
              phi_n = -bh.GM / sqrt(dn0 * dn0 + dn1 * dn1 + dn2 * dn2 + bh.rs2);
            }
            if (phi_sg) {   // the frozen self-gravity potential, ghosts included
              phi_i += phi_sg[l];
              phi_n += phi_sg[B.off + ((long long)pn[2] * B.p[1] + pn[1]) * B.p[0] + pn[0]];
            }
            U[4 * ntot + l] += sigma / (2.0 * dxa) * (-dI[0]) * (phi_n - phi_i);
          }
          for (int q = 0; q < nvar; ++q) U[q * ntot + l] += -sigma * dI[q] / dxa;
          for (int q = 0; q < nvar; ++q) R[sos + q * ncell + cs] = 0.0;
        }
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_ghost_amr(tde_mesh *m, double *Udst, const double *Ucur, const double *Uold, int nvar,
                             int nblk, const int32_t *ids, const int32_t *f, int flevel, int tau, int stage) {
  if (!m->d_amr || nblk <= 0) return cudaSuccess;
  ProfScope ps(m->ctx, TDE_K_GHOST);
  const AmrSrc S{Udst, Ucur, Uold, f, flevel, tau, stage, (long long)m->ntot};
  const unsigned gx = (unsigned)std::max(1, std::min((m->max_amr + LNT - 1) / LNT, 64));
  k_ghost_amr<<<dim3(gx, (unsigned)nblk), LNT, 0, m->ctx->stream>>>(m->d_amr, m->d_amr_start, ids, m->d_blocks,
                                                                   m->phys, S, Udst, nvar);
  return cudaGetLastError();
}

// ---- per level, the ghost cells a window converts (not copies) -------------
// Built on the device whenever the factors change: for the q-th block of the
// factor-sorted order, its copy entries whose source block is on another
// schedule, in map order, then its refined-mesh ops.  Blocks in sorted order
// make every level a contiguous segment of the list.
constexpr int GLT = 256;

__global__ void __launch_bounds__(GLT) k_glist_count(const int32_t *__restrict__ sorted,
                                                     const int32_t *__restrict__ f,
                                                     const int32_t *__restrict__ gstart,
                                                     const int32_t *__restrict__ gend,
                                                     const int32_t *__restrict__ gsrcb,
                                                     const int32_t *__restrict__ amr_start,
                                                     int32_t *__restrict__ cnt) {
  __shared__ int ws[GLT / 32];
  const int b = sorted[blockIdx.x], fb = f[b];
  int n = 0;
  for (int e = gstart[b] + threadIdx.x; e < gend[b]; e += GLT) n += f[gsrcb[e]] != fb;
  n = __reduce_add_sync(0xffffffffu, n);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = amr_start ? amr_start[b + 1] - amr_start[b] : 0;
    for (int w = 0; w < GLT / 32; ++w) t += ws[w];
    cnt[blockIdx.x] = t;
  }
}

// exclusive scan of the nb counts in place: cnt[q] -> start of block q, cnt[nb] = total
__global__ void __launch_bounds__(1024) k_glist_scan(int32_t *cnt, int nb) {
  __shared__ int ws[32];
  const int per = (nb + 1023) / 1024, q0 = threadIdx.x * per, q1 = min(nb, q0 + per);
  int s = 0;
  for (int q = q0; q < q1; ++q) s += cnt[q];
  // inclusive scan of the thread sums: within warps, then over warp totals
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int v = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    ws[lane] = v;
  }
  __syncthreads();
  int run = x - s + (w ? ws[w - 1] : 0);
  for (int q = q0; q < q1; ++q) {
    const int c = cnt[q];
    cnt[q] = run;
    run += c;
  }
  if (threadIdx.x == 1023) cnt[nb] = ws[31];
}

__global__ void __launch_bounds__(GLT) k_glist_fill(const int32_t *__restrict__ sorted,
                                                    const int32_t *__restrict__ f,
                                                    const int32_t *__restrict__ gstart,
                                                    const int32_t *__restrict__ gend,
                                                    const int32_t *__restrict__ gsrcb,
                                                    const int32_t *__restrict__ map,
                                                    const AmrOp *__restrict__ amr,
                                                    const int32_t *__restrict__ amr_start,
                                                    const int32_t *__restrict__ start,
                                                    int32_t *__restrict__ out) {
  __shared__ int ws[GLT / 32];
  const int b = sorted[blockIdx.x], fb = f[b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s1 = gend[b];   // the ghost cells the sweeps read
  int base = start[blockIdx.x];
  // ordered compaction, GLT entries per pass (the pass count is uniform over the CTA)
  for (int e0 = gstart[b]; e0 < s1; e0 += GLT) {
    const int e = e0 + threadIdx.x;
    const bool take = e < s1 && f[gsrcb[e]] != fb;
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (lane == 0) ws[w] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
    for (int k = 0; k < GLT / 32; ++k) {
      before += k < w ? ws[k] : 0;
      tot += ws[k];
    }
    if (take) out[base + before + __popc(bal & ((1u << lane) - 1u))] = map[2 * e];
    base += tot;
    __syncthreads();
  }
  if (amr_start)
    for (int e = amr_start[b] + threadIdx.x; e < amr_start[b + 1]; e += GLT)
      out[base + e - amr_start[b]] = amr[e].dst;
}

// Enqueues the list build on the mesh's stream; starts[q] (q = 0..nb) are the
// list offsets of the sorted blocks, read back by the caller after a sync.
cudaError_t launch_glist(tde_mesh *m, int32_t *starts) {
  const int nb = m->nb;
  cudaStream_t s = m->ctx->stream;
  ProfScope ps(m->ctx, TDE_K_SCALAR);
  k_glist_count<<<nb, GLT, 0, s>>>(m->d_sorted, m->d_f, m->d_gstart, m->d_gend, m->d_gsrcb, m->d_amr_start, starts);
  k_glist_scan<<<1, 1024, 0, s>>>(starts, nb);
  k_glist_fill<<<nb, GLT, 0, s>>>(m->d_sorted, m->d_f, m->d_gstart, m->d_gend, m->d_gsrcb, m->d_ghost, m->d_amr,
                                  m->d_amr_start, starts, m->d_lat_glist);
  return cudaGetLastError();
}

// A captured LAT window is stale once the mesh's launch configuration changes.
void invalidate_graph(tde_mesh *m) {
  if (m->lat_graph) {
    cudaGraphExecDestroy(m->lat_graph);
    m->lat_graph = nullptr;
  }
}

}  // namespace tde

using namespace tde;

namespace {

int lat_fail(tde_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

#define LCK(ctx, call)                                                       \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) {                                                 \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(_e);       \
      return TDE_ECUDA;                                                      \
    }                                                                        \
  } while (0)


// level lists from the factors (sorted on the host, the ghost-conversion list built
// on the device); allocates the LAT buffers once
int lat_build(tde_mesh *m) {
  tde_ctx *c = m->ctx;
  const int nb = m->nb;
  for (int b = 0; b < nb; ++b) {
    const int f = m->h_f[b];
    if (f < 1 || (f & (f - 1))) return lat_fail(c, TDE_EINVAL, "LAT: factors must be powers of two >= 1");
  }
  m->h_sorted.resize(nb);
  std::iota(m->h_sorted.begin(), m->h_sorted.end(), 0);
  std::stable_sort(m->h_sorted.begin(), m->h_sorted.end(),
                   [&](int a, int b) { return m->h_f[a] < m->h_f[b]; });
  const std::vector<int> old_levels = m->h_levels, old_start = m->h_level_start;
  m->h_levels.clear();
  m->h_level_start.clear();
  for (int q = 0; q < nb; ++q) {
    const int f = m->h_f[m->h_sorted[q]];
    if (m->h_levels.empty() || m->h_levels.back() != f) {
      m->h_levels.push_back(f);
      m->h_level_start.push_back(q);
    }
  }
  m->h_level_start.push_back(nb);
  m->lat_fmax = m->h_levels.back();
  const int nvar = m->phys.nvar;
  std::vector<long long> fo(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const DevBlock &B = m->hblocks[b];
    long long sz = 0;
    for (int s = 0; s < 6; ++s) {
      const int aa = s >> 1;
      const int u1 = aa == 0 ? 1 : 0, u2 = aa == 2 ? 1 : 2;
      sz += (long long)B.n[u1] * B.n[u2] * nvar;
    }
    fo[b + 1] = fo[b] + sz;
  }
  if (!m->d_Uold) LCK(c, cudaMalloc(&m->d_Uold, sizeof(double) * nvar * m->ntot));
  if (!m->d_freg) {
    LCK(c, cudaMalloc(&m->d_freg, sizeof(double) * fo[nb]));
    LCK(c, cudaMalloc(&m->d_fo, sizeof(long long) * (nb + 1)));
    LCK(c, cudaMemcpy(m->d_fo, fo.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice));
    m->freg_size = fo[nb];
  }
  if (!m->d_sorted) LCK(c, cudaMalloc(&m->d_sorted, sizeof(int32_t) * nb));
  if (!m->d_lat_bar) LCK(c, cudaMalloc(&m->d_lat_bar, LAT_BAR_WORDS * sizeof(unsigned)));
  if (!m->d_lat_pre) LCK(c, cudaMalloc(&m->d_lat_pre, 2 * sizeof(int32_t) * (nb + 1)));
  {
    // the persistent level kernel's work items: chunks of interior cells and of
    // ghost-map entries, counted per block in factor order (lat_pre is read by
    // the kernels when they run, so it is written before this call returns)
    m->h_lat_pre.assign(2 * (size_t)(nb + 1), 0);
    const int T = LAT_LEVEL_THREADS;
    for (int q = 0; q < nb; ++q) {
      const DevBlock &B = m->hblocks[m->h_sorted[q]];
      const int b = m->h_sorted[q];
      m->h_lat_pre[q + 1] = m->h_lat_pre[q] + (B.n[0] * B.n[1] * B.n[2] + T - 1) / T;
      m->h_lat_pre[nb + 1 + q + 1] = m->h_lat_pre[nb + 1 + q] + (m->h_gend[b] - m->h_gstart[b] + T - 1) / T;
    }
    LCK(c, cudaMemcpyAsync(m->d_lat_pre, m->h_lat_pre.data(), sizeof(int32_t) * m->h_lat_pre.size(),
                           cudaMemcpyHostToDevice, c->stream));
  }
  if (!m->d_lat_gstart) LCK(c, cudaMalloc(&m->d_lat_gstart, sizeof(int32_t) * (nb + 1)));
  if (!m->d_lat_glist)
    LCK(c, cudaMalloc(&m->d_lat_glist, sizeof(int32_t) * std::max<int64_t>(m->n_gcopy + m->n_amr, 1)));
  LCK(c, cudaMemcpyAsync(m->d_sorted, m->h_sorted.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice,
                         c->stream));
  LCK(c, cudaMemcpyAsync(m->d_f, m->h_f.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, c->stream));
  // per level, the ghost cells whose primitives are converted: copies from a
  // block on another schedule (time-interpolated or frozen) and the refined-mesh
  // ops; the others take their source's primitives
  std::vector<int32_t> starts(nb + 1);
  LCK(c, launch_glist(m, m->d_lat_gstart));
  LCK(c, cudaMemcpyAsync(starts.data(), m->d_lat_gstart, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost,
                         c->stream));
  LCK(c, cudaStreamSynchronize(c->stream));
  const std::vector<int32_t> old_goff = m->h_lat_glist_off;
  m->h_lat_glist_off.resize(m->h_levels.size() + 1);
  for (size_t L = 0; L <= m->h_levels.size(); ++L) m->h_lat_glist_off[L] = starts[m->h_level_start[L]];
  m->lat_ready = true;
  // a captured window reads the block lists, factors and dt0 from device memory
  // when it is replayed; it stays valid while the levels and their sizes do
  if (m->h_levels != old_levels || m->h_level_start != old_start || m->h_lat_glist_off != old_goff)
    invalidate_graph(m);
  return TDE_OK;
}

int ensure_factor_buffers(tde_mesh *m) {
  tde_ctx *c = m->ctx;
  if (!m->d_f) LCK(c, cudaMalloc(&m->d_f, sizeof(int32_t) * m->nb));
  if (!m->d_f2) LCK(c, cudaMalloc(&m->d_f2, sizeof(int32_t) * m->nb));
  if (!m->d_flag) LCK(c, cudaMalloc(&m->d_flag, sizeof(int)));
  return TDE_OK;
}

// enqueue one window on the context's stream
int lat_enqueue_window(tde_mesh *m, const BH &bh) {
  tde_ctx *c = m->ctx;
  const Phys &p = m->phys;
  const int nb = m->nb, nvar = p.nvar;
  cudaStream_t s = c->stream;
  {
    ProfScope ps(c, TDE_K_SCALAR);
    k_lat_prepare<<<(nb + 255) / 256, 256, 0, s>>>(nb, m->d_f, m->d_dtb, m->d_scal);
  }
  LCK(c, cudaMemsetAsync(m->d_freg, 0, sizeof(double) * m->freg_size, s));
  TimeArgs ta{m->d_dtb, 1, m->d_tstart, 1};
  OwnerLattice ol{m->d_owner, {m->unit[0], m->unit[1], m->unit[2]}, {m->cn[0], m->cn[1], m->cn[2]}, m->lmax};
  const int fmax = m->lat_fmax;
  const unsigned gx_ghost = (unsigned)std::max(1, std::min((m->max_ghosts + 255) / 256, 64));
  const unsigned gx_copy = 64;
  const bool persistent = m->lat_mode == TDE_LAT_PERSISTENT && lat_level_eligible(m);
  for (int tau = 0; tau <= fmax; ++tau) {
    if (tau > 0) {
      const int p2 = tau & -tau;   // completing: every level f <= largest power of two dividing tau
      int ncomp = 0;
      for (size_t L = 0; L < m->h_levels.size(); ++L)
        if (m->h_levels[L] <= p2) ncomp = m->h_level_start[L + 1];
      if (ncomp > 0) {
        {
          ProfScope ps(c, TDE_K_SCALAR);
          k_reflux<<<ncomp, LNT, 0, s>>>(p, bh, ol, m->d_blocks, m->d_sorted, m->d_f, m->U, (long long)m->ntot,
                                         m->d_freg, m->d_fo, nvar, m->d_scal, tau,
                                         m->grav_on ? m->d_phi_sg : nullptr);
        }
        LCK(c, cudaGetLastError());
        if (bh.excise) LCK(c, launch_excise(m, m->U, ncomp, m->d_sorted, bh, ta));
        if (p.dual) LCK(c, launch_sync(m, m->U, ncomp, m->d_sorted, p.eta2));
      }
    }
    if (tau == fmax) break;
    for (int L = (int)m->h_levels.size() - 1; L >= 0; --L) {
      const int f = m->h_levels[L];
      if (tau % f) continue;
      const int32_t *ids = m->d_sorted + m->h_level_start[L];
      const int n = m->h_level_start[L + 1] - m->h_level_start[L];
      if (persistent) {
        ProfScope ps(c, TDE_K_LATLEVEL);
        LCK(c, launch_lat_level(m, bh, ids, n, f, tau, m->d_lat_glist + m->h_lat_glist_off[L],
                                m->h_lat_glist_off[L + 1] - m->h_lat_glist_off[L]));
        continue;
      }
      {
        ProfScope ps(c, TDE_K_SCALAR);
        k_copy_blocks<<<dim3(gx_copy, n), LNT, 0, s>>>(m->d_blocks, ids, m->U, m->d_Uold, nvar,
                                                       (long long)m->ntot);
        k_lat_time<<<(n + 255) / 256, 256, 0, s>>>(ids, n, tau, m->d_tstart, m->d_scal);
      }
      for (int stage = 0; stage < 2; ++stage) {
        double *Udst = stage ? m->U1 : m->U;
        {
          ProfScope ps(c, TDE_K_GHOST);
          k_ghost_lat<<<dim3(gx_ghost, n), LNT, 0, s>>>(m->d_ghost, m->d_gstart, m->d_gend, m->d_gsrcb, ids, m->d_f, f, tau,
                                                        stage, Udst, m->U, m->d_Uold, nvar, (long long)m->ntot);
        }
        LCK(c, cudaGetLastError());
        LCK(c, launch_ghost_amr(m, Udst, m->U, m->d_Uold, nvar, n, ids, m->d_f, f, tau, stage));
        // primitives: the interiors, the converted ghost cells, then the copies
        LCK(c, launch_c2p(m, Udst, n, ids, false, bh, ta));
        LCK(c, launch_c2p_list(m, Udst, m->d_lat_glist + m->h_lat_glist_off[L],
                               m->h_lat_glist_off[L + 1] - m->h_lat_glist_off[L]));
        {
          ProfScope ps(c, TDE_K_GHOST);
          k_ghost_w_lat<<<dim3(gx_ghost, n), LNT, 0, s>>>(m->d_ghost, m->d_gstart, m->d_gend, m->d_gsrcb, ids, m->d_f, f,
                                                          m->d_W, p.nwv, (long long)m->ntot);
        }
        LCK(c, cudaGetLastError());
        LCK(c, launch_sweeps(m, stage, m->U, Udst, stage ? m->U : m->U1, n, ids, bh, ta, m->d_freg));
      }
    }
  }
  {
    ProfScope ps(c, TDE_K_SCALAR);
    k_lat_advance<<<1, 1, 0, s>>>(m->d_scal, fmax);
  }
  LCK(c, cudaGetLastError());
  return TDE_OK;
}

}  // namespace

int tde::lat_step_all_ones(tde_mesh *m, const BH &bh) {
  tde_ctx *c = m->ctx;
  int r = ensure_factor_buffers(m);
  if (r) return r;
  bool ones = m->lat_ready && (int)m->h_f.size() == m->nb;
  for (int b = 0; ones && b < m->nb; ++b) ones = m->h_f[b] == 1;
  if (!ones) {
    m->h_f.assign(m->nb, 1);
    r = lat_build(m);
    if (r) return r;
  }
  // dt0 = the step's dt, already on the device
  LCK(c, cudaMemcpyAsync(m->d_scal + 3, m->d_scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return lat_enqueue_window(m, bh);
}

extern "C" int tde_lat_assign(tde_mesh *m, int n_lat, double merge_frac, double cfl,
                              const tde_bh_state *bhs, int32_t *factors, int *f_max, double *dt0) {
  if (!m) return TDE_EINVAL;
  tde_ctx *c = m->ctx;
  if (!m->U || n_lat < 0 || n_lat > 20 || !(cfl > 0.0) || merge_frac < 0.0)
    return lat_fail(c, TDE_EINVAL, "tde_lat_assign: arguments");
  if (!closure_ready(m)) return lat_fail(c, TDE_EINVAL, "tde_lat_assign: surrogate closure without a trained network");
  int r = ensure_factor_buffers(m);
  if (r) return r;
  BH bh{};
  if (bhs) {
    bh.on = bhs->on; bh.excise = bhs->excise; bh.GM = bhs->GM; bh.rs2 = bhs->r_soft * bhs->r_soft;
    bh.rexc = bhs->r_exc; bh.t0 = bhs->t0;
    bh.frame = bhs->frame_on;
    for (int a = 0; a < 3; ++a) { bh.x0[a] = bhs->x0[a]; bh.v0[a] = bhs->v0[a]; bh.a0[a] = bhs->a0[a]; bh.afr[a] = bhs->afr[a]; }
  }
  TimeArgs ta{nullptr, 0, m->d_scal, 0};
  LCK(c, launch_c2p(m, m->U, m->nb, m->d_allids, true, bh, ta));
  LCK(c, launch_dt_finalize(m, cfl, m->d_dtb, nullptr));
  {
    ProfScope ps(c, TDE_K_DT);
    k_lat_factors<<<1, 1024, 0, c->stream>>>(m->nb, m->d_dtb, n_lat, merge_frac, m->d_nbr_start, m->d_nbr,
                                              m->d_blocks, m->d_f, m->d_f2, m->d_scal, m->d_flag);
  }
  LCK(c, cudaGetLastError());
  m->h_f.resize(m->nb);
  int flag = 0;
  LCK(c, cudaMemcpyAsync(m->h_f.data(), m->d_f, sizeof(int32_t) * m->nb, cudaMemcpyDeviceToHost, c->stream));
  LCK(c, cudaMemcpyAsync(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  LCK(c, cudaMemcpyAsync(&m->lat_dt0, m->d_scal + 3, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LCK(c, cudaStreamSynchronize(c->stream));
  if (flag) return lat_fail(c, TDE_ETIMEOUT, "tde_lat_assign: neighbour limiting did not converge");
  r = lat_build(m);
  if (r) return r;
  if (factors) memcpy(factors, m->h_f.data(), sizeof(int32_t) * m->nb);
  if (f_max) *f_max = m->lat_fmax;
  if (dt0) *dt0 = m->lat_dt0;
  return TDE_OK;
}

extern "C" int tde_lat_set_factors(tde_mesh *m, const int32_t *factors, double dt0) {
  if (!m || !factors || !(dt0 > 0.0)) return m ? lat_fail(m->ctx, TDE_EINVAL, "tde_lat_set_factors: arguments") : TDE_EINVAL;
  for (int b = 0; b < m->nb; ++b)   // reject before touching the current assignment
    if (factors[b] < 1 || (factors[b] & (factors[b] - 1)))
      return lat_fail(m->ctx, TDE_EINVAL, "tde_lat_set_factors: factors must be powers of two >= 1");
  int r = ensure_factor_buffers(m);
  if (r) return r;
  m->h_f.assign(factors, factors + m->nb);
  m->lat_dt0 = dt0;
  LCK(m->ctx, cudaMemcpyAsync(m->d_scal + 3, &m->lat_dt0, sizeof(double), cudaMemcpyHostToDevice, m->ctx->stream));
  return lat_build(m);
}

extern "C" int tde_lat_window(tde_mesh *m, const tde_bh_state *bhs, int use_graph,
                              int64_t *block_updates) {
  if (!m) return TDE_EINVAL;
  tde_ctx *c = m->ctx;
  if (!m->U || !m->U1) return lat_fail(c, TDE_EINVAL, "tde_lat_window: no bound state");
  if (!closure_ready(m)) return lat_fail(c, TDE_EINVAL, "tde_lat_window: surrogate closure without a trained network");
  if (!m->lat_ready) return lat_fail(c, TDE_EINVAL, "tde_lat_window: no factors (tde_lat_assign)");
  BH bh{};
  if (bhs) {
    bh.on = bhs->on; bh.excise = bhs->excise; bh.GM = bhs->GM; bh.rs2 = bhs->r_soft * bhs->r_soft;
    bh.rexc = bhs->r_exc; bh.t0 = bhs->t0;
    bh.frame = bhs->frame_on;
    for (int a = 0; a < 3; ++a) { bh.x0[a] = bhs->x0[a]; bh.v0[a] = bhs->v0[a]; bh.a0[a] = bhs->a0[a]; bh.afr[a] = bhs->afr[a]; }
  }
  int64_t upd = 0;
  for (size_t L = 0; L < m->h_levels.size(); ++L)
    upd += (int64_t)(m->lat_fmax / m->h_levels[L]) * (m->h_level_start[L + 1] - m->h_level_start[L]);
  if (block_updates) *block_updates = upd;
  if (!use_graph) return lat_enqueue_window(m, bh);
  if (m->lat_graph && (memcmp(&m->lat_graph_bh, &bh, sizeof bh) != 0 || m->lat_graph_U != m->U ||
                       m->lat_graph_U1 != m->U1))
    invalidate_graph(m);
  if (!m->lat_graph) {
    if (!m->cap_stream) LCK(c, cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    // the capture runs on a private stream ordered after the context's stream
    cudaEvent_t ev;
    LCK(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    LCK(c, cudaEventRecord(ev, c->stream));
    LCK(c, cudaStreamWaitEvent(m->cap_stream, ev, 0));
    LCK(c, cudaStreamSynchronize(m->cap_stream));
    cudaEventDestroy(ev);
    cudaStream_t keep = c->stream;
    const bool keep_prof = c->prof;
    uint64_t before[TDE_K_NKIND];
    memcpy(before, c->launches, sizeof before);
    c->stream = m->cap_stream;
    c->prof = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
    int r = e == cudaSuccess ? lat_enqueue_window(m, bh) : TDE_ECUDA;
    cudaError_t e2 = cudaStreamEndCapture(m->cap_stream, &g);
    c->stream = keep;
    c->prof = keep_prof;
    uint64_t per = 0;
    for (int k = 0; k < TDE_K_NKIND; ++k) {
      per += c->launches[k] - before[k];
      c->launches[k] = before[k];
    }
    m->lat_graph_launches = per;
    if (r || e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (!r) c->err = "tde_lat_window: graph capture failed";
      return r ? r : TDE_ECUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&m->lat_graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
      m->lat_graph = nullptr;
      c->err = std::string("tde_lat_window: cudaGraphInstantiate: ") + cudaGetErrorString(e3);
      return TDE_ECUDA;
    }
    m->lat_graph_bh = bh;
    m->lat_graph_U = m->U;
    m->lat_graph_U1 = m->U1;
  }
  {
    ProfScope ps(c, TDE_K_LATGRAPH);
    LCK(c, cudaGraphLaunch(m->lat_graph, c->stream));
  }
  c->launches[TDE_K_LATGRAPH] += m->lat_graph_launches - 1;
  return TDE_OK;
}
