// tde_hydro.cu -- the kernels of the per-MeshBlock hydro stage on sm_103a.
//
// One Runge-Kutta stage is four kinds of launches on the context's stream:
//   k_c2p     conserved -> primitive (+ EOS, + optional per-block CFL minimum)
//             on the interior cells only;
//   k_ghost   the ghost layer of the primitives (the face ghosts, the only ones
//             the sweeps read), gathered from the neighbours'
//             interiors through a precomputed (dst, src) map (a1) -- the
//             primitive recovery is pointwise, so copying primitives equals
//             converting copied conserved variables and saves the EOS work of
//             every ghost cell;
//   k_sweep   one launch per active direction: a CTA stages a tile of pencils
//             (with ghosts) in shared memory, reconstructs every cell's two face
//             states once, solves every face once (HLLC or HLLE), and accumulates the
//             flux divergence, the gravity sources and div v; the last active
//             direction also finishes the update (RK combination, dual-energy
//             compression, floors) and writes the output state.
// The FP64 pipe bounds this path on GB300, so no FP64 result is ever computed
// twice: a slope per cell and direction, a flux per face, an EOS inversion per
// interior cell.
#include <math.h>

#include <algorithm>

#include "tde_internal.h"
#include "tde_sweep.cuh"

namespace tde {

constexpr int NT = 256;   // threads per CTA

// minima of a and b over the CTA (valid in thread 0) for values >= 0 (time
// steps and their squares; NaN only if all are): the bit patterns of such
// doubles order like the values, so the minima run on the integer pipe
__device__ __forceinline__ unsigned long long umin64(unsigned long long x, unsigned long long y) {
  return x < y ? x : y;
}
__device__ __forceinline__ void block_min2(double &a, double &b) {
  __shared__ unsigned long long red[2][NT / 32];
  unsigned long long ka = (unsigned long long)dbits(a), kb = (unsigned long long)dbits(b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ka = umin64(ka, __shfl_xor_sync(0xffffffffu, ka, o));
    kb = umin64(kb, __shfl_xor_sync(0xffffffffu, kb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ka;
    red[1][threadIdx.x >> 5] = kb;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const unsigned long long inf = (unsigned long long)dbits(INFINITY);
    ka = threadIdx.x < NT / 32 ? red[0][threadIdx.x] : inf;
    kb = threadIdx.x < NT / 32 ? red[1][threadIdx.x] : inf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ka = umin64(ka, __shfl_xor_sync(0xffffffffu, ka, o));
      kb = umin64(kb, __shfl_xor_sync(0xffffffffu, kb, o));
    }
  }
  a = __longlong_as_double((long long)ka);
  b = __longlong_as_double((long long)kb);
}

// Squared distance from rb to the box of block B's interior cell centres: a
// lower bound of every interior cell's bh_r2 up to rounding (warp-collective;
// every lane of the calling warp gets it).  Interior centres never wrap, so no
// periodic image enters.
__device__ __forceinline__ double block_box_d2(const Phys &p, const DevBlock &B, const double rb[3]) {
  const int l = threadIdx.x & 31, a = l < 3 ? l : 0;
  const double lo = cell_coord(p, B, a, p.g[a]), hi = cell_coord(p, B, a, p.g[a] + B.n[a] - 1);
  const double ra = a == 0 ? rb[0] : (a == 1 ? rb[1] : rb[2]);
  const double da = dlt(ra, lo) ? lo - ra : (dlt(hi, ra) ? ra - hi : 0.0);
  const double q = l < 3 ? da * da : 0.0;
  return __shfl_sync(0xffffffffu, q, 0) + __shfl_sync(0xffffffffu, q, 1) + __shfl_sync(0xffffffffu, q, 2);
}

// The point mass's position at time t, the block factor dx / GM of its
// time-step limit and the squared distance to the block's box of interior cell
// centres, evaluated by one warp for the CTA.
__device__ __forceinline__ void cta_bh_info(const BH &bh, double t, double dx, const Phys &p, const DevBlock &B,
                                            double rb[3], double &dxg, double &d2box) {
  __shared__ double s_rb[5];
  if (threadIdx.x < 32) {
    double r[3];
    bh_pos(bh, t, r);
    const double d2 = block_box_d2(p, B, r);
    if (threadIdx.x < 3) s_rb[threadIdx.x] = r[threadIdx.x];
    if (threadIdx.x == 3) s_rb[3] = bh_dxg(dx, bh.GM);
    if (threadIdx.x == 4) s_rb[4] = d2;
  }
  __syncthreads();
  rb[0] = s_rb[0];
  rb[1] = s_rb[1];
  rb[2] = s_rb[2];
  dxg = s_rb[3];
  d2box = s_rb[4];
}

template <int EOSK, int DUAL, int EOSB = 0>
__global__ void __launch_bounds__(NT) k_c2p(Phys p, BH bh, TimeArgs ta,
                                            const DevBlock *__restrict__ blocks,
                                            const int32_t *__restrict__ ids,
                                            const double *__restrict__ U, double *__restrict__ W,
                                            long long ntot, Counters *cnt, int want_dt,
                                            unsigned long long *dtbits, EOSBuf eb) {
  const int b = ids[blockIdx.y];
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  const int e = blockIdx.x * NT + threadIdx.x;
  if (blockIdx.x * NT >= nint) return;   // whole CTA past this block (uniform)
  double best = INFINITY, best_g2 = INFINITY;   // the hydro limit; the point mass's, squared
  double rb[3], dxg = INFINITY, d2box = 0.0;
  const bool near = want_dt && (bh.on || bh.excise);   // uniform over the CTA
  if (near) cta_bh_info(bh, ta_t(ta, b), scale2i(p.dxmin, -B.level), p, B, rb, dxg, d2box);
  // some interior cell may lie within r_exc (else the per-cell test is false for
  // all: a margin of 2^-20 on r_exc^2 is far above the roundings of the box and
  // of the cells' r^2)
  const bool exc_box = bh.excise && !dlt(bh.rexc * bh.rexc * (1.0 + 0x1p-20), d2box);
  const int i = e % B.n[0], r = e / B.n[0];
  const int c[3] = {i + p.g[0], r % B.n[1] + p.g[1], r / B.n[1] + p.g[2]};
  bool skip = e >= nint;   // no CFL contribution (past the block, or excised)
  double r2 = -1.0;        // the cell's squared distance, once computed
  if (e < nint) {
    const long long flat = B.off + ((long long)c[2] * B.p[1] + c[1]) * B.p[0] + c[0];
    double u[6], w[8];
#pragma unroll
    for (int v = 0; v < 5 + DUAL; ++v) u[v] = U[v * ntot + flat];
    cons_to_prim<EOSK, DUAL, EOSB>(p, u, w, cnt, &eb, flat);
    constexpr int NWV = (EOSK == EOS_TABLE ? 7 : 5) + DUAL;
#pragma unroll
    for (int v = 0; v < NWV; ++v) W[v * ntot + flat] = w[v];
    if (want_dt) {
      if (exc_box) {
        double x[3];
        cell_centre(p, B, c, x);
        r2 = bh_r2(x[0] - rb[0], x[1] - rb[1], x[2] - rb[2]);
        skip = inside_radius(r2, bh.rexc);
      }
      if (!skip) {
        const double g1 = EOSK == EOS_TABLE ? w[6] : p.gamma;
        const double cs = sqrt_ratio(g1 * w[4], w[0]);
        // min_d dx_d / (|v_d| + cs) as the reciprocal of the largest signal rate
        double rate = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          if (p.active[a]) rate = dmax(rate, (fabs(w[1 + a]) + cs) * block_idx(p, B, a));
        best = dmin(best, rcp_nr(rate));
      }
    }
  }
  if (want_dt) {
    if (bh.on) {
      // The point mass's limit dt_g^2 grows with r beyond r_s / sqrt(2), so over a
      // box at least that far its value at the box is a lower bound (less a
      // margin of 2^-20 for the roundings); where that bound exceeds this CTA's
      // hydro minimum squared (with the same margin) the point mass cannot set
      // the CTA's minimum and is not evaluated per cell.  The result is the
      // same as evaluating it everywhere.
      __shared__ int s_grav;
      double bmin = best, none = INFINITY;
      block_min2(bmin, none);
      if (threadIdx.x == 0) {
        const double lb = dlt(0.5 * bh.rs2, d2box) ? bh_dt2(dxg, d2box, bh.rs2) * (1.0 - 0x1p-20) : 0.0;
        s_grav = !dle(bmin * bmin * (1.0 + 0x1p-20), lb);
      }
      __syncthreads();
      if (s_grav && !skip) {
        if (r2 < 0.0) {
          double x[3];
          cell_centre(p, B, c, x);
          r2 = bh_r2(x[0] - rb[0], x[1] - rb[1], x[2] - rb[2]);
        }
        best_g2 = bh_dt2(dxg, r2, bh.rs2);
      }
    }
    block_min2(best, best_g2);
    if (threadIdx.x == 0) {
      best = dmin(best, sqrt(best_g2));
      atomicMin(dtbits + b, (unsigned long long)__double_as_longlong(best));
    }
  }
}


// every padded cell of the listed blocks (used when only a subset of blocks
// advances, so the ghost layer cannot be copied from freshly converted
// neighbours); events are counted on interior cells only
template <int EOSK, int DUAL, int EOSB = 0>
__global__ void __launch_bounds__(NT) k_c2p_padded(Phys p, const DevBlock *__restrict__ blocks,
                                                   const int32_t *__restrict__ ids,
                                                   const double *__restrict__ U,
                                                   double *__restrict__ W, long long ntot,
                                                   Counters *cnt, EOSBuf eb) {
  const int b = ids[blockIdx.y];
  const DevBlock B = blocks[b];
  const int npad = B.p[0] * B.p[1] * B.p[2];
  for (int e = blockIdx.x * NT + threadIdx.x; e < npad; e += gridDim.x * NT) {
    const int i = e % B.p[0], r = e / B.p[0];
    const int j = r % B.p[1], k = r / B.p[1];
    const bool interior = i >= p.g[0] && i < p.g[0] + B.n[0] && j >= p.g[1] &&
                          j < p.g[1] + B.n[1] && k >= p.g[2] && k < p.g[2] + B.n[2];
    const long long flat = B.off + e;
    double u[6], w[8];
#pragma unroll
    for (int v = 0; v < 5 + DUAL; ++v) u[v] = U[v * ntot + flat];
    cons_to_prim<EOSK, DUAL, EOSB>(p, u, w, interior ? cnt : nullptr, &eb, flat);
    constexpr int NWV = (EOSK == EOS_TABLE ? 7 : 5) + DUAL;
#pragma unroll
    for (int v = 0; v < NWV; ++v) W[v * ntot + flat] = w[v];
  }
}

// primitives of listed cells (LAT ghost cells whose conserved values were
// interpolated in time, restricted or prolonged; nothing counted: ghost cells)
template <int EOSK, int DUAL, int EOSB = 0>
__global__ void __launch_bounds__(NT) k_c2p_list(Phys p, const int32_t *__restrict__ list, int n,
                                                 const double *__restrict__ U, double *__restrict__ W,
                                                 long long ntot, EOSBuf eb) {
  for (int e = blockIdx.x * NT + threadIdx.x; e < n; e += gridDim.x * NT) {
    const long long flat = list[e];
    double u[6], w[8];
#pragma unroll
    for (int v = 0; v < 5 + DUAL; ++v) u[v] = U[v * ntot + flat];
    cons_to_prim<EOSK, DUAL, EOSB>(p, u, w, nullptr, &eb, flat);
    constexpr int NWV = (EOSK == EOS_TABLE ? 7 : 5) + DUAL;
#pragma unroll
    for (int v = 0; v < NWV; ++v) W[v * ntot + flat] = w[v];
  }
}

// The table inputs (cgs rho, e) of the interior (PADDED = 0) or all padded
// (PADDED = 1) cells of the listed blocks, by the same expressions as the
// closure inside k_c2p, for the learned-guess inversion's launches; nothing is
// counted here (k_c2p counts when it takes the results).
template <int DUAL, int PADDED>
__global__ void __launch_bounds__(NT) k_c2p_eosin(Phys p, const DevBlock *__restrict__ blocks,
                                                  const int32_t *__restrict__ ids,
                                                  const double *__restrict__ U, double *rho_in,
                                                  double *e_in, long long ntot) {
  const int b = ids[blockIdx.y];
  const DevBlock B = blocks[b];
  const int n = PADDED ? B.p[0] * B.p[1] * B.p[2] : B.n[0] * B.n[1] * B.n[2];
  for (int e = blockIdx.x * NT + threadIdx.x; e < n; e += gridDim.x * NT) {
    long long flat;
    if (PADDED) {
      flat = B.off + e;
    } else {
      const int i = e % B.n[0], r = e / B.n[0];
      const int j = r % B.n[1], k = r / B.n[1];
      flat = B.off + ((long long)(k + p.g[2]) * B.p[1] + (j + p.g[1])) * B.p[0] + (i + p.g[0]);
    }
    double u[6];
#pragma unroll
    for (int v = 0; v < 5 + DUAL; ++v) u[v] = U[v * ntot + flat];
    double rho, vx, vy, vz, Ue;
    c2p_energy<DUAL>(p, u, rho, vx, vy, vz, Ue, nullptr);
    double rc, ec;
    eos_inputs(p, rho, Ue, rc, ec);
    rho_in[flat] = rc;
    e_in[flat] = ec;
  }
}

// table inputs of listed cells (the learned-guess closure over a cell list)
template <int DUAL>
__global__ void __launch_bounds__(NT) k_c2p_eosin_list(Phys p, const int32_t *__restrict__ list, int n,
                                                       const double *__restrict__ U, double *rho_in,
                                                       double *e_in, long long ntot) {
  for (int e = blockIdx.x * NT + threadIdx.x; e < n; e += gridDim.x * NT) {
    const long long flat = list[e];
    double u[6];
#pragma unroll
    for (int v = 0; v < 5 + DUAL; ++v) u[v] = U[v * ntot + flat];
    double rho, vx, vy, vz, Ue;
    c2p_energy<DUAL>(p, u, rho, vx, vy, vz, Ue, nullptr);
    double rc, ec;
    eos_inputs(p, rho, Ue, rc, ec);
    rho_in[flat] = rc;
    e_in[flat] = ec;
  }
}

// per-block dt = cfl * minimum; global minimum; re-arm the per-block minima
__global__ void __launch_bounds__(1024) k_dt_finalize(int nb, double cfl,
                                                      unsigned long long *dtbits,
                                                      double *dt_block, double *dt_min,
                                                      double *scal) {
  __shared__ double red[32];
  double m = INFINITY;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double v = cfl * __longlong_as_double((long long)dtbits[b]);
    if (dt_block) dt_block[b] = v;
    m = fmin(m, v);
    dtbits[b] = (unsigned long long)__double_as_longlong(INFINITY);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      if (dt_min) *dt_min = m;
      if (scal) { scal[1] = m; scal[2] = m; }
    }
  }
}

// ---------------------------------------------------------- k_ghost ----

// nf <= GHOST_NF_MAX fields per cell; every field of a cell is loaded before any
// is stored (the sources are interior cells, the destinations ghost cells, so
// they never overlap), which lets the loads of a cell overlap in flight
constexpr int GHOST_NF_MAX = 8;
__global__ void __launch_bounds__(NT) k_ghost(const int32_t *__restrict__ map,
                                              const int32_t *__restrict__ gstart,
                                              const int32_t *__restrict__ gend,
                                              const int32_t *__restrict__ ids, double *f, int nf,
                                              long long ntot) {
  const int b = ids[blockIdx.y];
  const int s0 = gstart[b], s1 = gend ? gend[b] : gstart[b + 1];
  for (int e = s0 + blockIdx.x * NT + threadIdx.x; e < s1; e += gridDim.x * NT) {
    const int2 m = reinterpret_cast<const int2 *>(map)[e];
    double t[GHOST_NF_MAX];
#pragma unroll
    for (int v = 0; v < GHOST_NF_MAX; ++v)
      if (v < nf) t[v] = f[v * ntot + m.y];
#pragma unroll
    for (int v = 0; v < GHOST_NF_MAX; ++v)
      if (v < nf) f[v * ntot + m.x] = t[v];
  }
}

// ---------------------------------------------------- excision, resync ----

// Excision reset of the interior cells within r_exc of the point mass.  A CTA
// covers a slice of one block; one warp first tests the block's box of cell
// centres against the sphere (with a margin of 2^-20 on r_exc^2, far above the
// roundings of the centres and of r^2), and a block entirely outside it is
// skipped, so the per-cell test (which decides as before) runs only near the
// point mass.
__global__ void __launch_bounds__(NT) k_excise(Phys p, BH bh, TimeArgs ta,
                                               const DevBlock *__restrict__ blocks,
                                               const int32_t *__restrict__ ids, double *U,
                                               long long ntot, Counters *cnt) {
  __shared__ int s_far;
  __shared__ double s_rb[3];
  const int b = ids[blockIdx.y];
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  if ((int)blockIdx.x * NT >= nint) return;   // uniform over the CTA
  if (threadIdx.x < 32) {
    double rb[3];
    bh_pos(bh, ta_t(ta, b) + ta_dt(ta, b), rb);
    const double d2 = block_box_d2(p, B, rb);
    if (threadIdx.x == 0) {
      // (interior cell centres never wrap, so no periodic image enters either test)
      s_far = dlt(bh.rexc * bh.rexc * (1.0 + 0x1p-20), d2);
      s_rb[0] = rb[0];
      s_rb[1] = rb[1];
      s_rb[2] = rb[2];
    }
  }
  __syncthreads();
  if (s_far) return;
  const double rb[3] = {s_rb[0], s_rb[1], s_rb[2]};
  for (int e = blockIdx.x * NT + threadIdx.x; e < nint; e += gridDim.x * NT) {
    const int i = e % B.n[0], r = e / B.n[0];
    const int c[3] = {i + p.g[0], r % B.n[1] + p.g[1], r / B.n[1] + p.g[2]};
    double x[3];
    cell_centre(p, B, c, x);
    if (!inside_radius(bh_r2(x[0] - rb[0], x[1] - rb[1], x[2] - rb[2]), bh.rexc)) continue;
    const long long flat = B.off + ((long long)c[2] * B.p[1] + c[1]) * B.p[0] + c[0];
    U[flat] = p.rho_floor;
    U[ntot + flat] = 0.0;
    U[2 * ntot + flat] = 0.0;
    U[3 * ntot + flat] = 0.0;
    U[4 * ntot + flat] = p.u_floor;
    if (p.dual) U[5 * ntot + flat] = p.u_floor;
    count(&cnt->excised);
  }
}

__global__ void __launch_bounds__(NT) k_sync(Phys p, const DevBlock *__restrict__ blocks,
                                             const int32_t *__restrict__ ids, double *U,
                                             long long ntot, double eta2, Counters *cnt) {
  const int b = ids[blockIdx.y];
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  const int e = blockIdx.x * NT + threadIdx.x;
  if (e >= nint) return;
  const int i = e % B.n[0], r = e / B.n[0];
  const int c[3] = {i + p.g[0], r % B.n[1] + p.g[1], r / B.n[1] + p.g[2]};
  const long long sy = B.p[0], sz = (long long)B.p[0] * B.p[1];
  const long long flat = B.off + c[2] * sz + c[1] * sy + c[0];
  const double *E = U + 4 * ntot;
  const int ax = p.active[0], ay = p.active[1], az = p.active[2];
  // the neighbourhood maximum on the integer pipe: order keys of the bit
  // patterns (the key map is its own inverse), 27 FP64 max operations saved
  long long kmax = dkey(-INFINITY);
  for (int dk = -az; dk <= az; ++dk)
    for (int dj = -ay; dj <= ay; ++dj)
      for (int di = -ax; di <= ax; ++di) {
        const long long k = dkey(E[flat + dk * sz + dj * sy + di]);
        kmax = k > kmax ? k : kmax;
      }
  const double emax = __longlong_as_double(kmax ^ ((kmax >> 63) & 0x7fffffffffffffffLL));
  const double u0 = U[flat], u1 = U[ntot + flat], u2 = U[2 * ntot + flat], u3 = U[3 * ntot + flat];
  const double rho = dlt(u0, p.rho_floor) ? p.rho_floor : u0;
  const double ir = rcp_nr(rho);
  const double Uc = E[flat] - 0.5 * (u1 * (u1 * ir) + u2 * (u2 * ir) + u3 * (u3 * ir));
  if (dgt0(Uc) && dlt(eta2 * emax, Uc)) {
    U[5 * ntot + flat] = Uc;
    count(&cnt->synced);
  }
}

// ------------------------------------------------------ prim -> cons ----

// log10 T at which the interpolated log10 P at density cell (i, w) equals lp
__device__ double table_lT_from_lP(const DTable &t, int i, double w, double lp) {
  double lo = 0.0, hi = (double)(t.nt - 1);   // in units of table cells
  for (int it = 0; it < 100; ++it) {
    const double mid = 0.5 * (lo + hi);
    int j = (int)floor(mid);
    if (j > t.nt - 2) j = t.nt - 2;
    if (bilin(t.lp, t.nt, i, w, j, mid - j) < lp) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

__global__ void __launch_bounds__(NT) k_prim2cons(Phys p, const DevBlock *__restrict__ blocks,
                                                  const double *__restrict__ W, double *U,
                                                  long long ntot, int nb) {
  const int b = blockIdx.y;
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  for (int e = blockIdx.x * NT + threadIdx.x; e < nint; e += gridDim.x * NT) {
    const int i = e % B.n[0], r = e / B.n[0];
    const int c[3] = {i + p.g[0], r % B.n[1] + p.g[1], r / B.n[1] + p.g[2]};
    const long long flat = B.off + ((long long)c[2] * B.p[1] + c[1]) * B.p[0] + c[0];
    const double rho = W[flat], vx = W[ntot + flat], vy = W[2 * ntot + flat];
    const double vz = W[3 * ntot + flat], P = W[4 * ntot + flat];
    double Uint;
    if (p.eos == EOS_IDEAL) {
      Uint = P * p.inv_gm1;
    } else {
      int ti;
      double tw;
      rho_cell(p.tab, rho * p.unit_rho, ti, tw);
      const double y = table_lT_from_lP(p.tab, ti, tw, log10(P * p.unit_rho * p.unit_e));
      int j = (int)floor(y);
      if (j > p.tab.nt - 2) j = p.tab.nt - 2;
      const double ec = exp10(bilin(p.tab.le, p.tab.nt, ti, tw, j, y - j));
      Uint = rho * (ec * p.inv_unit_e);
    }
    U[flat] = rho;
    U[ntot + flat] = rho * vx;
    U[2 * ntot + flat] = rho * vy;
    U[3 * ntot + flat] = rho * vz;
    U[4 * ntot + flat] = Uint + 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    if (p.dual) U[5 * ntot + flat] = Uint;
  }
}

// ------------------------------------------------------------- scalars ----

__global__ void k_advance_time(double *scal) { scal[0] += scal[1]; }
__global__ void k_set_dt(double *scal, double dt) { scal[1] = dt; scal[2] = dt; }

// ---------------------------------------------------------- EOS batch ----

__global__ void __launch_bounds__(NT) k_eos_invert(DTable t, long long n, const double *__restrict__ rho,
                                                   const double *__restrict__ en, double *T,
                                                   double *P, double *cs2, Counters *cnt) {
  for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) {
    double Pv, cv, eu, Tv;
    bool cl = eos_invert(t, rho[e], en[e], Pv, cv, eu, &Tv);
    if (cl) count(&cnt->table_clamp);
    if (T) T[e] = Tv;
    if (P) P[e] = Pv;
    if (cs2) cs2[e] = cv;
  }
}

__global__ void __launch_bounds__(NT) k_eos_eval(DTable t, long long n, const double *__restrict__ rho,
                                                 const double *__restrict__ T, double *P,
                                                 double *en, double *cs2) {
  for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) {
    int i;
    double w;
    rho_cell(t, rho[e], i, w);
    double y = (log10(T[e]) - t.lt0) / t.dlt;
    if (!(y >= 0.0)) y = 0.0;
    if (y > (double)(t.nt - 1)) y = (double)(t.nt - 1);
    int j = (int)floor(y);
    if (j > t.nt - 2) j = t.nt - 2;
    const double s = y - j;
    if (P) P[e] = exp10(bilin(t.lp, t.nt, i, w, j, s));
    if (en) en[e] = exp10(bilin(t.le, t.nt, i, w, j, s));
    if (cs2) cs2[e] = exp10(bilin(t.lc, t.nt, i, w, j, s));
  }
}

// ------------------------------------------------------- moving frame ----

// Partial sums of Eq. frame-acceleration: rho g (3) and rho over the interior
// cells with rho > rho_min outside the excision sphere, one slot per CTA.
__global__ void __launch_bounds__(NT) k_frame_partial(Phys p, BH bh, const double *__restrict__ tnow,
                                                      const DevBlock *__restrict__ blocks,
                                                      const double *__restrict__ U, double rho_min,
                                                      double *part) {
  __shared__ double red[4][NT / 32];
  const int b = blockIdx.y;
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  double rb[3];
  bh_pos(bh, *tnow, rb);
  // a level-L cell holds 2^-(L d) level-0 cell volumes (d active directions)
  const double vw = exp2i(-B.level * (p.active[0] + p.active[1] + p.active[2]));
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = blockIdx.x * NT + threadIdx.x; e < nint; e += gridDim.x * NT) {
    const int i = e % B.n[0], r = e / B.n[0];
    const int c[3] = {i + p.g[0], r % B.n[1] + p.g[1], r / B.n[1] + p.g[2]};
    const double rho = U[B.off + ((long long)c[2] * B.p[1] + c[1]) * B.p[0] + c[0]];
    if (!(rho > rho_min)) continue;
    double x[3];
    cell_centre(p, B, c, x);
    const double d0 = x[0] - rb[0], d1 = x[1] - rb[1], d2 = x[2] - rb[2];
    const double r2 = bh_r2(d0, d1, d2);
    if (bh.excise && inside_radius(r2, bh.rexc)) continue;
    const double q2 = r2 + bh.rs2;
    const double gfac = -bh.GM / (q2 * sqrt(q2));   // g = -grad Phi_bh = -GM d / q^3
    const double rw = rho * vw;   // mass in level-0 cell volumes
    s[0] += rw * gfac * d0;
    s[1] += rw * gfac * d1;
    s[2] += rw * gfac * d2;
    s[3] += rw;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += red[threadIdx.x][w];
    part[((long long)b * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = v;
  }
}

// The partial sums in a fixed order (deterministic): out = (A_fr[3], mass).
__global__ void __launch_bounds__(NT) k_frame_final(const double *__restrict__ part, int nparts,
                                                    double dV, double *out) {
  __shared__ double red[4][NT];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = threadIdx.x; q < nparts; q += NT)
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] += part[(long long)q * 4 + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int h = NT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = red[3][0];
    for (int k = 0; k < 3; ++k) out[k] = m > 0.0 ? red[k][0] / m : 0.0;
    out[3] = m * dV;
  }
}

// Galilean boost of Eq. galilean-boost of the interior cells with rho > rho_min.
__global__ void __launch_bounds__(NT) k_boost(Phys p, const DevBlock *__restrict__ blocks, double *U,
                                              long long ntot, double V0, double V1, double V2,
                                              double rho_min) {
  const int b = blockIdx.y;
  const DevBlock B = blocks[b];
  const int nint = B.n[0] * B.n[1] * B.n[2];
  for (int e = blockIdx.x * NT + threadIdx.x; e < nint; e += gridDim.x * NT) {
    const int i = e % B.n[0], r = e / B.n[0];
    const long long l = B.off + ((long long)(r / B.n[1] + p.g[2]) * B.p[1] + (r % B.n[1] + p.g[1])) * B.p[0] +
                        (i + p.g[0]);
    const double rho = U[l];
    if (!(rho > rho_min)) continue;
    const double mv = U[ntot + l] * V0 + U[2 * ntot + l] * V1 + U[3 * ntot + l] * V2;
    const double v2 = V0 * V0 + V1 * V1 + V2 * V2;
    U[4 * ntot + l] += mv + 0.5 * rho * v2;
    U[ntot + l] += rho * V0;
    U[2 * ntot + l] += rho * V1;
    U[3 * ntot + l] += rho * V2;
  }
}

// ============================================================ launchers ====

static int n_sm() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

static bool surrogate_closure(const tde_mesh *m) {
  return m->phys.eos == EOS_TABLE && m->phys.eos_mode == TDE_INVERT_SURROGATE;
}

// The learned-guess inversion of the listed blocks' cells (interior or all
// padded): table inputs -> guess, Newton, queued bisection -> m->sb (P, cs2, eu).
static cudaError_t surrogate_table_pass(tde_mesh *m, const double *Uin, int nblk, const int32_t *ids,
                                        bool padded, dim3 grid) {
  const Phys &p = m->phys;
  cudaStream_t s = m->ctx->stream;
  if (!m->sb.rho || !m->eos || !m->eos->has_net) return cudaErrorInvalidValue;
  const long long nt = (long long)m->ntot;
  if (padded) {
    if (p.dual) k_c2p_eosin<1, 1><<<grid, NT, 0, s>>>(p, m->d_blocks, ids, Uin, m->sb.rho, m->sb.e, nt);
    else k_c2p_eosin<0, 1><<<grid, NT, 0, s>>>(p, m->d_blocks, ids, Uin, m->sb.rho, m->sb.e, nt);
  } else {
    if (p.dual) k_c2p_eosin<1, 0><<<grid, NT, 0, s>>>(p, m->d_blocks, ids, Uin, m->sb.rho, m->sb.e, nt);
    else k_c2p_eosin<0, 0><<<grid, NT, 0, s>>>(p, m->d_blocks, ids, Uin, m->sb.rho, m->sb.e, nt);
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  m->ctx->launches[TDE_K_C2P] += 3;   // table inputs, guess + Newton, bisection of the misses
  CellMap cm{m->d_blocks, ids, nblk, padded ? 1 : 0, {p.g[0], p.g[1], p.g[2]}};
  int64_t nmax = 0;
  for (const DevBlock &B : m->hblocks)
    nmax = std::max<int64_t>(nmax, padded ? (int64_t)B.p[0] * B.p[1] * B.p[2]
                                          : (int64_t)B.n[0] * B.n[1] * B.n[2]);
  return launch_eos_surrogate_cells(m->eos, cm, nmax, m->sb, m->d_cnt, s);
}

cudaError_t launch_c2p(tde_mesh *m, const double *Uin, int nblk, const int32_t *ids, bool want_dt,
                       const BH &bh, TimeArgs ta) {
  ProfScope _ps(m->ctx, TDE_K_C2P);
  dim3 grid((unsigned)((m->max_interior + NT - 1) / NT), (unsigned)nblk);
  const Phys &p = m->phys;
  EOSBuf eb{m->sb.P, m->sb.cs2, m->sb.eu};
  if (surrogate_closure(m)) {
    cudaError_t err = surrogate_table_pass(m, Uin, nblk, ids, false, grid);
    if (err != cudaSuccess) return err;
  }
#define C2P_ARGS p, bh, ta, m->d_blocks, ids, Uin, m->d_W, (long long)m->ntot, m->d_cnt, \
                 (int)want_dt, m->d_dtbits, eb
  if (p.eos == EOS_IDEAL) {
    if (p.dual) k_c2p<EOS_IDEAL, 1><<<grid, NT, 0, m->ctx->stream>>>(C2P_ARGS);
    else k_c2p<EOS_IDEAL, 0><<<grid, NT, 0, m->ctx->stream>>>(C2P_ARGS);
  } else if (surrogate_closure(m)) {
    if (p.dual) k_c2p<EOS_TABLE, 1, 1><<<grid, NT, 0, m->ctx->stream>>>(C2P_ARGS);
    else k_c2p<EOS_TABLE, 0, 1><<<grid, NT, 0, m->ctx->stream>>>(C2P_ARGS);
  } else {
    if (p.dual) k_c2p<EOS_TABLE, 1><<<grid, NT, 0, m->ctx->stream>>>(C2P_ARGS);
    else k_c2p<EOS_TABLE, 0><<<grid, NT, 0, m->ctx->stream>>>(C2P_ARGS);
  }
#undef C2P_ARGS
  return cudaGetLastError();
}

cudaError_t launch_c2p_padded(tde_mesh *m, const double *Uin, int nblk, const int32_t *ids) {
  ProfScope _ps(m->ctx, TDE_K_C2P);
  int64_t npad = 0;
  for (const DevBlock &B : m->hblocks) npad = std::max<int64_t>(npad, (int64_t)B.p[0] * B.p[1] * B.p[2]);
  dim3 grid((unsigned)std::min<int64_t>((npad + NT - 1) / NT, 256), (unsigned)nblk);
  const Phys &p = m->phys;
  EOSBuf eb{m->sb.P, m->sb.cs2, m->sb.eu};
  if (surrogate_closure(m)) {
    cudaError_t err = surrogate_table_pass(m, Uin, nblk, ids, true, grid);
    if (err != cudaSuccess) return err;
  }
#define C2PP_ARGS p, m->d_blocks, ids, Uin, m->d_W, (long long)m->ntot, m->d_cnt, eb
  if (p.eos == EOS_IDEAL) {
    if (p.dual) k_c2p_padded<EOS_IDEAL, 1><<<grid, NT, 0, m->ctx->stream>>>(C2PP_ARGS);
    else k_c2p_padded<EOS_IDEAL, 0><<<grid, NT, 0, m->ctx->stream>>>(C2PP_ARGS);
  } else if (surrogate_closure(m)) {
    if (p.dual) k_c2p_padded<EOS_TABLE, 1, 1><<<grid, NT, 0, m->ctx->stream>>>(C2PP_ARGS);
    else k_c2p_padded<EOS_TABLE, 0, 1><<<grid, NT, 0, m->ctx->stream>>>(C2PP_ARGS);
  } else {
    if (p.dual) k_c2p_padded<EOS_TABLE, 1><<<grid, NT, 0, m->ctx->stream>>>(C2PP_ARGS);
    else k_c2p_padded<EOS_TABLE, 0><<<grid, NT, 0, m->ctx->stream>>>(C2PP_ARGS);
  }
#undef C2PP_ARGS
  return cudaGetLastError();
}

cudaError_t launch_c2p_list(tde_mesh *m, const double *Uin, const int32_t *list, int n) {
  if (n <= 0) return cudaSuccess;
  ProfScope _ps(m->ctx, TDE_K_C2P);
  const Phys &p = m->phys;
  cudaStream_t s = m->ctx->stream;
  const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)n + NT - 1) / NT, 8LL * n_sm());
  EOSBuf eb{m->sb.P, m->sb.cs2, m->sb.eu};
  if (surrogate_closure(m)) {
    if (!m->sb.rho || !m->eos || !m->eos->has_net) return cudaErrorInvalidValue;
    if (p.dual) k_c2p_eosin_list<1><<<grid, NT, 0, s>>>(p, list, n, Uin, m->sb.rho, m->sb.e, (long long)m->ntot);
    else k_c2p_eosin_list<0><<<grid, NT, 0, s>>>(p, list, n, Uin, m->sb.rho, m->sb.e, (long long)m->ntot);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    m->ctx->launches[TDE_K_C2P] += 3;   // table inputs, guess + Newton, bisection of the misses
    CellMap cm{};
    cm.nblk = 1;
    cm.list = list;
    err = launch_eos_surrogate_cells(m->eos, cm, n, m->sb, m->d_cnt, s);
    if (err != cudaSuccess) return err;
  }
#define C2PL_ARGS p, list, n, Uin, m->d_W, (long long)m->ntot, eb
  if (p.eos == EOS_IDEAL) {
    if (p.dual) k_c2p_list<EOS_IDEAL, 1><<<grid, NT, 0, s>>>(C2PL_ARGS);
    else k_c2p_list<EOS_IDEAL, 0><<<grid, NT, 0, s>>>(C2PL_ARGS);
  } else if (surrogate_closure(m)) {
    if (p.dual) k_c2p_list<EOS_TABLE, 1, 1><<<grid, NT, 0, s>>>(C2PL_ARGS);
    else k_c2p_list<EOS_TABLE, 0, 1><<<grid, NT, 0, s>>>(C2PL_ARGS);
  } else {
    if (p.dual) k_c2p_list<EOS_TABLE, 1><<<grid, NT, 0, s>>>(C2PL_ARGS);
    else k_c2p_list<EOS_TABLE, 0><<<grid, NT, 0, s>>>(C2PL_ARGS);
  }
#undef C2PL_ARGS
  return cudaGetLastError();
}

cudaError_t launch_dt_finalize(tde_mesh *m, double cfl, double *dt_block, double *dt_min) {
  ProfScope _ps(m->ctx, TDE_K_DT);
  k_dt_finalize<<<1, 1024, 0, m->ctx->stream>>>(m->nb, cfl, m->d_dtbits, dt_block, dt_min,
                                                m->d_scal);
  return cudaGetLastError();
}

cudaError_t launch_ghost(tde_mesh *m, double *field, int nf, int nblk, const int32_t *ids, bool sweep_only) {
  if (m->max_ghosts == 0) return cudaSuccess;
  if (nf < 1 || nf > GHOST_NF_MAX) return cudaErrorInvalidValue;
  ProfScope _ps(m->ctx, TDE_K_GHOST);
  unsigned gx = (unsigned)min((m->max_ghosts + NT - 1) / NT, 64);
  k_ghost<<<dim3(gx, (unsigned)nblk), NT, 0, m->ctx->stream>>>(m->d_ghost, m->d_gstart,
                                                                 sweep_only ? m->d_gend : nullptr, ids, field,
                                                                 nf, (long long)m->ntot);
  return cudaGetLastError();
}

// lanes per staged row of a y or z sweep tile and the column of lane 0: a TMA
// row starts on a 16-byte boundary, so with an odd ghost width the row starts
// one cell early and carries two extra columns
static void sweep_lane_layout(const Phys &p, int D, int M, int &LS, int &XO) {
  XO = D == 0 ? 0 : (p.g[0] & 1);
  LS = D == 0 ? M : M + 2 * XO;
}

// The sweeps' TMA tensor maps: for every tile shape, direction and block, a
// 4-D view (x, y, z, field) of the block's primitives in W whose box is one
// tile's staging area (D = 0: PD x M lanes x 1 x NV; D = 1: LS x PD x 1 x NV;
// D = 2: LS x 1 x PD x NV), copied in place by one cp.async.bulk.tensor.
// Requires every padded x row to be a whole number of 16-byte units (even
// padded widths; then every block offset and plane is one too); otherwise,
// or if the driver entry point is unavailable, no maps are built and the
// sweeps stage by a copy loop (same values).  Returns a CUDA error only for a
// failed allocation or copy.
cudaError_t build_sweep_tmaps(tde_mesh *m) {
  const Phys &p = m->phys;
  m->d_tmaps = nullptr;
  if (m->ntot & 1) return cudaSuccess;
  for (int b = 0; b < m->nb; ++b)
    if (m->hblocks[b].p[0] & 1) return cudaSuccess;
  for (int D = 0; D < 3; ++D)
    if (p.active[D] && ((m->nmax[D] + 2 * p.g[D]) & 1)) return cudaSuccess;
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return cudaSuccess;
  }
  auto encode = reinterpret_cast<CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill)>(fn);
  const int nb = m->nb, NV = p.nwv;
  std::vector<CUtensorMap> maps((size_t)N_TILE_SHAPES * 3 * nb);
  memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  for (int shape = 0; shape < N_TILE_SHAPES; ++shape)
    for (int D = 0; D < 3; ++D) {
      if (!p.active[D]) continue;
      const int M = kTileShapes[shape].M, PD = m->nmax[D] + 2 * p.g[D];
      int LS, XO;
      sweep_lane_layout(p, D, M, LS, XO);
      const cuuint32_t box[4] = {(cuuint32_t)(D == 0 ? PD : LS), (cuuint32_t)(D == 0 ? M : (D == 1 ? PD : 1)),
                                 (cuuint32_t)(D == 2 ? PD : 1), (cuuint32_t)NV};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      for (int b = 0; b < nb; ++b) {
        const DevBlock &B = m->hblocks[b];
        const cuuint64_t dims[4] = {(cuuint64_t)B.p[0], (cuuint64_t)B.p[1], (cuuint64_t)B.p[2], (cuuint64_t)NV};
        const cuuint64_t strides[3] = {(cuuint64_t)B.p[0] * 8, (cuuint64_t)B.p[0] * B.p[1] * 8,
                                       (cuuint64_t)m->ntot * 8};
        CUtensorMap &t = maps[((size_t)shape * 3 + D) * nb + b];
        if (encode(&t, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void *)(m->d_W + B.off), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
          return cudaSuccess;   // this layout stays on the copy loop
      }
    }
  CUtensorMap *d = nullptr;
  cudaError_t err = cudaMalloc(&d, sizeof(CUtensorMap) * maps.size());
  if (err == cudaSuccess) err = cudaMemcpy(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(d);
    return err;
  }
  m->d_tmaps = d;
  return cudaSuccess;
}

// shared memory of one sweep CTA (doubles, then the excision bytes): the
// staging / flux union, the face values, the PPM interface scratch, the
// potential and the density of the tile's cells
static size_t sweep_smem(const Phys &p, int D, int PD, int NF, int M) {
  const int NV = p.nwv;
  int LS, XO;
  sweep_lane_layout(p, D, M, LS, XO);
  size_t nd = (size_t)sweep_union_len(D, NV, PD, NF, M, LS) + 2 * (size_t)NV * NF * M +
              (p.recon == PPM ? 4 * (size_t)(NF + 1) * M : 0) + 2 * (size_t)NF * M;
  // then the excision flags (NF M bytes, rounded up to doubles) and the TMA barrier
  return (nd + ((size_t)NF * M + 7) / 8 + 1) * sizeof(double);
}

size_t sweep_smem_for(const tde_mesh *m, int D, int shape) {
  const int PD = m->nmax[D] + 2 * m->phys.g[D], NF = m->nmax[D] + 2;
  return sweep_smem(m->phys, D, PD, NF, kTileShapes[shape].M);
}

size_t sweep_smem_max(const tde_mesh *m) {
  size_t best = 0;
  for (int D = 0; D < 3; ++D) best = std::max(best, sweep_smem_for(m, D, m->tile[D]));
  return best;
}

static cudaError_t sweep_launch_by_shape(int shape, const SweepArgs &a, int D, bool last, dim3 grid,
                                         size_t smem, cudaStream_t s) {
  switch (shape) {
    case 1: return sweep_launch_m16(a, D, last, grid, smem, s);
    case 2: return sweep_launch_m4(a, D, last, grid, smem, s);
    default: return sweep_launch_m8(a, D, last, grid, smem, s);
  }
}

static SweepArgs sweep_args(tde_mesh *m, int stage, const double *U0, const double *Uin,
                            double *Uout, const int32_t *ids, const BH &bh, TimeArgs ta,
                            double *freg) {
  SweepArgs a;
  a.p = m->phys;
  a.bh = bh;
  a.ta = ta;
  a.blocks = m->d_blocks;
  a.ids = ids;
  a.W = m->d_W;
  a.dU = m->d_dU;
  a.U0 = U0;
  a.Uin = Uin;
  a.Uout = Uout;
  a.ntot = (long long)m->ntot;
  a.cnt = m->d_cnt;
  a.stage = stage;
  a.freg = freg;
  a.fo = m->d_fo;
  a.nvar = m->phys.nvar;
  a.phi_sg = m->grav_on ? m->d_phi_sg : nullptr;
  a.tmap = nullptr;
  a.status = m->d_status;
  a.skip_tma = m->inject_tma_skip;
  a.phic = m->d_phic;
  a.exc_c = m->d_excc;
  return a;
}

// the direction's part of a sweep's arguments (tile shape `shape`)
static void sweep_dir_fill(const tde_mesh *m, SweepArgs &a, int D, int shape, bool first) {
  const Phys &p = m->phys;
  a.first = first;
  a.PD = m->nmax[D] + 2 * p.g[D];
  a.NF = m->nmax[D] + 2;
  sweep_lane_layout(p, D, kTileShapes[shape].M, a.LS, a.XO);
  a.tmap = m->d_tmaps ? m->d_tmaps + ((size_t)shape * 3 + D) * m->nb : nullptr;
}

SweepArgs sweep_args_dir(tde_mesh *m, int stage, int D, int shape, bool first, const double *U0,
                         const double *Uin, double *Uout, const int32_t *ids, const BH &bh, TimeArgs ta,
                         double *freg) {
  SweepArgs a = sweep_args(m, stage, U0, Uin, Uout, ids, bh, ta, freg);
  sweep_dir_fill(m, a, D, shape, first);
  return a;
}

// One direction's sweep over nblk blocks with tile shape `shape`.
static cudaError_t sweep_dir(tde_mesh *m, SweepArgs &a, int D, int shape, bool first, bool last,
                             int nblk) {
  const Phys &p = m->phys;
  const int M = kTileShapes[shape].M;
  const int LA = D == 0 ? 1 : 0, OA = D == 2 ? 1 : 2;
  sweep_dir_fill(m, a, D, shape, first);
  const size_t smem = sweep_smem(p, D, a.PD, a.NF, M);
  dim3 grid((unsigned)(((m->nmax[LA] + M - 1) / M) * m->nmax[OA]), (unsigned)nblk);
  return sweep_launch_by_shape(shape, a, D, last, grid, smem, m->ctx->stream);
}

static void active_range(const Phys &p, int &firstD, int &lastD) {
  firstD = lastD = -1;
  for (int D = 0; D < 3; ++D)
    if (p.active[D]) { lastD = D; if (firstD < 0) firstD = D; }
}

cudaError_t launch_sweeps(tde_mesh *m, int stage, const double *U0, const double *Uin,
                          double *Uout, int nblk, const int32_t *ids, const BH &bh, TimeArgs ta,
                          double *freg) {
  int firstD, lastD;
  active_range(m->phys, firstD, lastD);
  if (lastD < 0) return cudaErrorInvalidValue;
  SweepArgs a = sweep_args(m, stage, U0, Uin, Uout, ids, bh, ta, freg);
  for (int D = 0; D < 3; ++D) {
    if (!m->phys.active[D]) continue;
    ProfScope _ps(m->ctx, TDE_K_SWEEP_X + D);
    cudaError_t err = sweep_dir(m, a, D, m->tile[D], D == firstD, D == lastD, nblk);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Time every tile shape that fits in shared memory on each active direction
// (one warm-up and `reps` timed launches over all blocks, CUDA events on the
// context's stream) and keep the fastest.  The sweeps read the bound state and
// the primitives computed from it here, and write only scratch arrays: the
// state, the counters and the workspaces the next step reads are untouched.
cudaError_t autotune_sweeps(tde_mesh *m, const BH &bh, int reps, float ms_out[3][N_TILE_SHAPES]) {
  tde_ctx *c = m->ctx;
  cudaStream_t s = c->stream;
  int firstD, lastD;
  active_range(m->phys, firstD, lastD);
  if (lastD < 0) return cudaErrorInvalidValue;
  const size_t nt = (size_t)m->ntot;
  double *dU = nullptr, *Uo = nullptr, *zero = nullptr;
  Counters *cnt_save = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&dU, sizeof(double) * nt * (m->phys.nvar + 1));
  if (err == cudaSuccess) err = cudaMalloc(&Uo, sizeof(double) * nt * m->phys.nvar);
  if (err == cudaSuccess) err = cudaMalloc(&zero, sizeof(double));
  if (err == cudaSuccess) err = cudaMalloc(&cnt_save, sizeof(Counters));
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaMemsetAsync(dU, 0, sizeof(double) * nt * (m->phys.nvar + 1), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(zero, 0, sizeof(double), s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(cnt_save, m->d_cnt, sizeof(Counters), cudaMemcpyDeviceToDevice, s);
  TimeArgs ta{zero, 0, m->d_scal, 0};
  if (err == cudaSuccess) err = launch_c2p(m, m->U, m->nb, m->d_allids, false, bh, ta);
  if (err == cudaSuccess) err = launch_ghost(m, m->d_W, m->phys.nwv, m->nb, m->d_allids, true);
  for (int D = 0; D < 3 && err == cudaSuccess; ++D) {
    for (int t = 0; t < N_TILE_SHAPES; ++t) ms_out[D][t] = -1.f;
    if (!m->phys.active[D]) continue;
    for (int t = 0; t < N_TILE_SHAPES && err == cudaSuccess; ++t) {
      if (sweep_smem_for(m, D, t) > SWEEP_SMEM_LIMIT) continue;
      SweepArgs a = sweep_args(m, 0, m->U, m->U, Uo, m->d_allids, bh, ta, nullptr);
      a.dU = dU;
      a.cnt = nullptr;
      err = sweep_dir(m, a, D, t, D == firstD, D == lastD, m->nb);
      if (err == cudaSuccess) err = cudaEventRecord(e0, s);
      for (int r = 0; r < reps && err == cudaSuccess; ++r)
        err = sweep_dir(m, a, D, t, D == firstD, D == lastD, m->nb);
      if (err == cudaSuccess) err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      ms_out[D][t] = ms / (float)std::max(reps, 1);
    }
    int best = m->tile[D];
    for (int t = 0; t < N_TILE_SHAPES; ++t)
      if (ms_out[D][t] >= 0.f && (ms_out[D][best] < 0.f || ms_out[D][t] < ms_out[D][best])) best = t;
    m->tile[D] = best;
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(m->d_cnt, cnt_save, sizeof(Counters), cudaMemcpyDeviceToDevice, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(dU);
  cudaFree(Uo);
  cudaFree(zero);
  cudaFree(cnt_save);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return err;
}

cudaError_t launch_excise(tde_mesh *m, double *U, int nblk, const int32_t *ids, const BH &bh,
                          TimeArgs ta) {
  ProfScope _ps(m->ctx, TDE_K_EXCISE);
  dim3 grid((unsigned)std::min<int64_t>((m->max_interior + NT - 1) / NT, 8), (unsigned)nblk);
  k_excise<<<grid, NT, 0, m->ctx->stream>>>(m->phys, bh, ta, m->d_blocks, ids, U,
                                             (long long)m->ntot, m->d_cnt);
  return cudaGetLastError();
}

cudaError_t launch_sync(tde_mesh *m, double *U, int nblk, const int32_t *ids, double eta2) {
  cudaError_t err = launch_ghost(m, U + 4 * m->ntot, 1, nblk, ids);
  if (err != cudaSuccess) return err;
  err = launch_ghost_amr(m, U + 4 * m->ntot, nullptr, nullptr, 1, nblk, ids, nullptr, 0, 0, 0);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)((m->max_interior + NT - 1) / NT), (unsigned)nblk);
  ProfScope _ps(m->ctx, TDE_K_SYNC);
  k_sync<<<grid, NT, 0, m->ctx->stream>>>(m->phys, m->d_blocks, ids, U, (long long)m->ntot, eta2,
                                           m->d_cnt);
  return cudaGetLastError();
}

cudaError_t launch_prim2cons(tde_mesh *m, const double *W, double *U) {
  ProfScope _ps(m->ctx, TDE_K_P2C);
  dim3 grid((unsigned)min((m->max_interior + NT - 1) / NT, (int64_t)1024), (unsigned)m->nb);
  k_prim2cons<<<grid, NT, 0, m->ctx->stream>>>(m->phys, m->d_blocks, W, U, (long long)m->ntot, m->nb);
  return cudaGetLastError();
}

cudaError_t launch_advance_time(tde_mesh *m) {
  ProfScope _ps(m->ctx, TDE_K_SCALAR);
  k_advance_time<<<1, 1, 0, m->ctx->stream>>>(m->d_scal);
  return cudaGetLastError();
}

cudaError_t launch_set_dt(tde_mesh *m, double dt) {
  ProfScope _ps(m->ctx, TDE_K_SCALAR);
  k_set_dt<<<1, 1, 0, m->ctx->stream>>>(m->d_scal, dt);
  return cudaGetLastError();
}

cudaError_t launch_eos_invert(tde_eos *e, int64_t n, const double *rho, const double *en,
                              double *T, double *P, double *cs2, cudaStream_t s, bool plain) {
  ProfScope _ps(e->ctx, TDE_K_EOS);
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + NT - 1) / NT;
  unsigned g = (unsigned)(blocks < 8LL * n_sm() ? blocks : 8LL * n_sm());
  DTable t = e->tab;
  if (plain) t.le32 = nullptr;   // no FP32 guide: every bisection step in FP64
  k_eos_invert<<<g, NT, 0, s>>>(t, (long long)n, rho, en, T, P, cs2, e->d_cnt);
  return cudaGetLastError();
}

cudaError_t launch_eos_eval(tde_eos *e, int64_t n, const double *rho, const double *T, double *P,
                            double *en, double *cs2, cudaStream_t s) {
  ProfScope _ps(e->ctx, TDE_K_EOS);
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + NT - 1) / NT;
  unsigned g = (unsigned)(blocks < 8LL * n_sm() ? blocks : 8LL * n_sm());
  k_eos_eval<<<g, NT, 0, s>>>(e->tab, (long long)n, rho, T, P, en, cs2);
  return cudaGetLastError();
}

cudaError_t launch_frame_acceleration(tde_mesh *m, const BH &bh, double rho_min, double *out4) {
  ProfScope _ps(m->ctx, TDE_K_SCALAR);
  const int gx = (int)std::min<int64_t>((m->max_interior + NT - 1) / NT, 64);
  const size_t need = (size_t)m->nb * gx * 4;
  if (m->frame_part_cap < need) {
    cudaFree(m->d_frame_part);
    m->d_frame_part = nullptr;
    m->frame_part_cap = 0;
    cudaError_t err = cudaMalloc(&m->d_frame_part, sizeof(double) * need);
    if (err != cudaSuccess) return err;
    m->frame_part_cap = need;
  }
  k_frame_partial<<<dim3((unsigned)gx, (unsigned)m->nb), NT, 0, m->ctx->stream>>>(
      m->phys, bh, m->d_scal, m->d_blocks, m->U, rho_min, m->d_frame_part);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const double dV = m->phys.dx[0] * m->phys.dx[1] * m->phys.dx[2];
  k_frame_final<<<1, NT, 0, m->ctx->stream>>>(m->d_frame_part, m->nb * gx, dV, out4);
  return cudaGetLastError();
}

cudaError_t launch_boost(tde_mesh *m, const double *V, double rho_min) {
  ProfScope _ps(m->ctx, TDE_K_SCALAR);
  dim3 grid((unsigned)std::min<int64_t>((m->max_interior + NT - 1) / NT, 64), (unsigned)m->nb);
  k_boost<<<grid, NT, 0, m->ctx->stream>>>(m->phys, m->d_blocks, m->U, (long long)m->ntot, V[0], V[1],
                                           V[2], rho_min);
  return cudaGetLastError();
}

}  // namespace tde
