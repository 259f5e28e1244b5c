// tde_sweep.cuh -- the per-direction sweep kernel of the hydro stage
// (reconstruction, HLLC, flux divergence, sources, and on the last direction
// the stage update), templated on the tile shape, and the device helpers it
// shares with the other hydro kernels.
#pragma once
#include <math.h>

#include <cuda.h>

#include "tde_internal.h"

namespace tde {

__device__ __forceinline__ double ta_t(const TimeArgs &ta, int b) {
  return ta.t ? ta.t[ta.t_pb ? b : 0] : 0.0;
}
__device__ __forceinline__ double ta_dt(const TimeArgs &ta, int b) {
  return ta.dt ? ta.dt[ta.dt_pb ? b : 0] : 0.0;
}

__device__ __forceinline__ void bh_pos(const BH &bh, double t, double r[3]) {
  double s = t - bh.t0;
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = bh.x0[a] + bh.v0[a] * s + 0.5 * bh.a0[a] * s * s;
}

// coordinate along direction a of padded cell index c of block B; periodic
// directions wrap to the image
__device__ __forceinline__ double cell_coord(const Phys &p, const DevBlock &B, int a, int c) {
  const int o = a == 0 ? B.i0 : (a == 1 ? B.j0 : B.k0);
  int g = o + c - p.g[a];
  if (p.bc[a] == 1) {
    const int N = level_n(p, a, B.level);
    g %= N;
    if (g < 0) g += N;
  }
  return p.xmin[a] + (g + 0.5) * block_dx(p, B, a);
}

// centre of padded cell c[] of block B
__device__ __forceinline__ void cell_centre(const Phys &p, const DevBlock &B, const int c[3],
                                            double x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = cell_coord(p, B, a, c[a]);
}

// ---------------------------------------------------------- k_sweep ----

struct SweepArgs {
  Phys p;
  BH bh;
  TimeArgs ta;
  const DevBlock *blocks;
  const int32_t *ids;
  const double *W;
  double *dU;
  const double *U0;
  const double *Uin;
  double *Uout;
  long long ntot;
  Counters *cnt;
  int stage, first, PD, NF;
  double *freg;              // flux impulse registers (LAT) or null
  const double *phi_sg;      // self-gravity potential (MeshBlock layout) or null
  const long long *fo;       // register offset per block
  int nvar;
  // TMA staging of phase A: the tensor maps of this direction and tile shape,
  // one per block (null: staged by a copy loop); LS = lanes per staged row of
  // y and z tiles, XO = staged column of lane 0 (LS = M + 2 and XO = 1 when the
  // ghost width is odd: a TMA row must start on a 16-byte boundary)
  const CUtensorMap *tmap;
  int LS, XO;
  int *status;               // set to 1 if a bounded wait for the TMA expired
  int skip_tma;              // failure-detection test: issue no copy, so the wait expires
  // the potential and excision flag of every interior cell at the stage time,
  // written by the stage's first sweep and read by the others (null: each
  // sweep computes them)
  double *phic;
  unsigned char *exc_c;
};

// A sweep tile is M pencils (lanes) of one block along D; its CTA has NTS
// threads.  NTS >= (n + 3) M for pencils of n cells makes every phase (the n + 3
// PPM interfaces, n + 2 cells, n + 1 faces, n cells) a single pass, so no warp
// waits at a barrier for another warp's second pass; for n = 32 and M = 8 that
// is 280 threads, and 288 (nine whole warps) costs no more warps or registers.  The shapes offered (tile_shapes)
// are chosen per direction by tde_mesh_autotune; every shape computes the same
// operations on the same data, so results do not depend on the choice.
template <int D>
struct SweepGeo {
  static constexpr int LA = D == 0 ? 1 : 0;   // lane axis (transverse, one thread column per lane)
  static constexpr int OA = D == 2 ? 1 : 2;   // other transverse axis (one CTA per index)
};

// Bounded wait on an mbarrier phase: at most one second of the global
// nanosecond timer (try_wait may suspend the thread, so the limit is on time).
__device__ __forceinline__ bool sweep_wait(uint32_t mbar, uint32_t parity) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

// Shared memory of a sweep tile, in doubles (then the excision bytes):
// the staged primitives, later reused for the fluxes; the face values; the
// PPM interface scratch; the potential and the density of the tile's cells.
__host__ __device__ __forceinline__ int sweep_stage_len(int D, int NV, int PD, int M, int LS) {
  return D == 0 ? NV * PD * M : NV * PD * LS;
}
__host__ __device__ __forceinline__ int sweep_union_len(int D, int NV, int PD, int NF, int M, int LS) {
  const int st = sweep_stage_len(D, NV, PD, M, LS), fl = 7 * (NF - 1) * M;
  return st > fl ? st : fl;
}

// the TMA completion barrier of a sweep CTA: 8-byte aligned after the excision
// flags (the last part of the tile's shared memory)
template <int D, int RECON, int NV, int M>
__device__ __forceinline__ unsigned long long *sweep_mbar(double *sm, int PD, int NF, int LS) {
  double *Rh = sm + sweep_union_len(D, NV, PD, NF, M, LS) + 2 * NV * NF * M +
               (RECON == PPM ? 4 * (NF + 1) * M : 0) + NF * M;
  return reinterpret_cast<unsigned long long *>(Rh + NF * M + (NF * M + 7) / 8);
}

// initialise a CTA's TMA barrier (thread 0; the caller synchronises before use)
__device__ __forceinline__ void sweep_mbar_init(unsigned long long *mbar) {
  const uint32_t ma = (uint32_t)__cvta_generic_to_shared(mbar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ma), "r"(1));
  asm volatile("fence.mbarrier_init.release.cluster;");
  asm volatile("fence.proxy.async.shared::cta;");
}

// One sweep tile: tile `tile` of block ids[qb].  The TMA barrier (at `mbar`,
// initialised) completes once per staged tile with the parity `parity`, which
// the caller flips after every tile that returns staged = true.  Returns false
// if the bounded wait for the staging copy expired (the tile is skipped and the
// status word set).
template <int D, int RECON, int EOSK, int DUAL, int LAST, int M, int NTS>
__device__ __forceinline__ bool sweep_tile(const SweepArgs &a, int qb, int tile, double *sm,
                                           unsigned long long *mbar, uint32_t parity, bool &staged) {
  constexpr int LA = SweepGeo<D>::LA, OA = SweepGeo<D>::OA;
  constexpr int NV = (EOSK == EOS_TABLE ? 7 : 5) + DUAL;   // reconstructed primitives
  constexpr int NVAR = 5 + DUAL;                            // conserved variables
  const Phys &p = a.p;
  const int b = a.ids[qb];
  const DevBlock B = a.blocks[b];
  const int nd = B.n[D], nl = B.n[LA], no = B.n[OA];
  const int nlc = (nl + M - 1) / M;
  staged = false;
  if (tile >= nlc * no) return true;   // uniform over the CTA
  const int l0 = (tile % nlc) * M, o = tile / nlc;
  const int nlane = min(M, nl - l0);
  const int g = p.g[D], pd = B.p[D];
  const long long st[3] = {1, B.p[0], (long long)B.p[0] * B.p[1]};
  const long long sD = st[D], sL = st[LA];
  const long long base = B.off + (long long)(p.g[LA] + l0) * sL + (long long)(p.g[OA] + o) * st[OA];
  const int PD = a.PD, NF = a.NF, NFF = a.NF - 1;
  const int LS = D == 0 ? M : a.LS, XO = D == 0 ? 0 : a.XO;
  const long long ntot = a.ntot;

  // staged primitives (D = 0: [NV][M][PD], pencil contiguous as in global
  // memory; D = 1, 2: [NV][PD][LS], lanes contiguous), reused for the fluxes
  // [7][NFF][M] once the face values exist
  double *Wt = sm;
  double *Fl = sm;
  double *FMs = sm + sweep_union_len(D, NV, PD, NF, M, LS);   // [NV][NF][M]  low face of cells g-1 .. g+nd
  double *FPs = FMs + NV * NF * M;       // [NV][NF][M]  high face
  double *If = FPs + NV * NF * M;        // PPM: [4][NF + 1][M] interface values
  double *Ph = If + (RECON == PPM ? 4 * (NF + 1) * M : 0);   // [NF][M] potential of cells g-1 .. g+nd
  double *Rh = Ph + NF * M;              // [NF][M] density of the same cells (gravity source)
  unsigned char *Ex = reinterpret_cast<unsigned char *>(Rh + NF * M);   // [NF][M] excised

  auto sw = [&](int v, int pos, int lane) {
    return D == 0 ? (v * M + lane) * PD + pos : (v * PD + pos) * LS + lane + XO;
  };
  auto sf = [&](int v, int c, int lane) {
    return D == 0 ? (v * M + lane) * NF + c : (v * NF + c) * M + lane;
  };
  auto sfl = [&](int q, int f, int lane) {
    return D == 0 ? (q * M + lane) * NFF + f : (q * NFF + f) * M + lane;
  };
  auto split = [&](int e, int len, int &c, int &lane) {
    if (D == 0) { lane = e / len; c = e - lane * len; }
    else { c = e / M; lane = e - c * M; }
  };

  // ---- A: stage the tile's primitives (all pencil cells incl. ghosts): one
  // TMA tensor copy of the tile's box (out-of-block parts of the box are
  // zero-filled and never read), or a copy loop
  const uint32_t mbar_addr = (uint32_t)__cvta_generic_to_shared(mbar);
  if (a.tmap) {
    staged = true;
    if (threadIdx.x == 0) {
      // earlier tiles' generic reads of the staging area before the async write
      asm volatile("fence.proxy.async.shared::cta;");
      const uint32_t bytes = (uint32_t)sweep_stage_len(D, NV, PD, M, LS) * 8u;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_addr), "r"(bytes)
                   : "memory");
      int c0, c1, c2;
      if (D == 0) { c0 = 0; c1 = p.g[1] + l0; c2 = p.g[2] + o; }
      else if (D == 1) { c0 = p.g[0] + l0 - XO; c1 = 0; c2 = p.g[2] + o; }
      else { c0 = p.g[0] + l0 - XO; c1 = p.g[1] + o; c2 = 0; }
      const unsigned long long tm = reinterpret_cast<unsigned long long>(a.tmap + b);
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Wt);
      if (!a.skip_tma)
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
            ::"r"(dst), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(0), "r"(mbar_addr)
            : "memory");
    }
  } else {
    const int per = pd * M;
    for (int e = threadIdx.x; e < NV * per; e += NTS) {
      const int v = e / per;
      int pos, lane;
      split(e - v * per, pd, pos, lane);
      if (lane < nlane) Wt[sw(v, pos, lane)] = a.W[v * ntot + base + pos * sD + lane * sL];
    }
  }
  const bool grav = a.bh.on || a.phi_sg, exc = a.bh.excise;
  if (grav || exc) {
    // one warp evaluates the point mass's position at the stage time and, for
    // an x pencil, the transverse part of each lane's squared distance (the
    // FP64 pipe charges a warp instruction whatever its active lanes)
    __shared__ double s_rb[3], s_yz[M];
    __shared__ Sphere s_exc;   // the excision sphere's thresholds
    if (threadIdx.x < 32) {
      const double ts = ta_t(a.ta, b) + (a.stage ? ta_dt(a.ta, b) : 0.0);
      double rb[3];
      bh_pos(a.bh, ts, rb);
      if (threadIdx.x < 3) s_rb[threadIdx.x] = rb[threadIdx.x];
      if (threadIdx.x == 0 && exc) s_exc = sphere_of(a.bh.rexc);
      if (D == 0 && threadIdx.x < M)
        s_yz[threadIdx.x] = bh_r2_yz(cell_coord(p, B, 1, p.g[1] + l0 + threadIdx.x) - rb[1],
                                     cell_coord(p, B, 2, p.g[2] + o) - rb[2]);
    }
    __syncthreads();
    const double rb0 = s_rb[0], rb1 = s_rb[1], rb2 = s_rb[2];
    const bool cached = a.phic != nullptr;
    for (int e = threadIdx.x; e < (nd + 2) * M; e += NTS) {
      int c, lane;
      split(e, nd + 2, c, lane);
      if (lane >= nlane) continue;
      const int idx = D == 0 ? lane * NF + c : c * M + lane;
      const bool inner = c > 0 && c <= nd;
      const long long cflat = base + (long long)(g - 1 + c) * sD + lane * sL;
      if (cached && inner && !a.first) {   // interior cell: the first sweep's value
        if (grav) Ph[idx] = a.phic[cflat];
        if (exc) Ex[idx] = a.exc_c[cflat];
        continue;
      }
      double r2;
      if (D == 0) {
        const double d0 = cell_coord(p, B, 0, g - 1 + c) - rb0;
        r2 = fma(d0, d0, s_yz[lane]);   // = bh_r2
      } else {
        int cc[3];
        cc[D] = g - 1 + c;
        cc[LA] = p.g[LA] + l0 + lane;
        cc[OA] = p.g[OA] + o;
        double x[3];
        cell_centre(p, B, cc, x);
        r2 = bh_r2(x[0] - rb0, x[1] - rb1, x[2] - rb2);
      }
      if (grav) {
        double ph = a.bh.on ? -a.bh.GM * rsqrt_nr(r2 + a.bh.rs2) : 0.0;
        if (a.phi_sg) ph += a.phi_sg[cflat];   // Phi_bh + Phi_sg
        Ph[idx] = ph;
        if (cached && inner) a.phic[cflat] = ph;
      }
      if (exc) {
        const unsigned char x = inside_sphere(r2, s_exc) ? 1 : 0;
        Ex[idx] = x;
        if (cached && inner) a.exc_c[cflat] = x;
      }
    }
  }
  __syncthreads();
  if (a.tmap) {
    // every thread waits for the copy (bounded); if it did not complete, the
    // tile is skipped, the status word set, and thread 0 waits once more
    // (bounded) so that no copy is in flight when the CTA goes on or exits
    const bool ok = sweep_wait(mbar_addr, parity);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(a.status, 1);
        sweep_wait(mbar_addr, parity);
      }
      return false;
    }
  }

  // ---- B: face values of every cell adjacent to a face of the tile; the
  // density of those cells kept for the gravity source (the staged primitives
  // become the flux area after this phase)
  if (grav) {
    for (int e = threadIdx.x; e < (nd + 2) * M; e += NTS) {
      int c, lane;
      split(e, nd + 2, c, lane);
      if (lane >= nlane) continue;
      Rh[D == 0 ? lane * NF + c : c * M + lane] = Wt[sw(0, g - 1 + c, lane)];
    }
  }
  if (RECON == PLM) {
    for (int e = threadIdx.x; e < (nd + 2) * M; e += NTS) {
      int c, lane;
      split(e, nd + 2, c, lane);
      if (lane >= nlane) continue;
      const int pos = g - 1 + c;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double lo, hi;
        plm(Wt[sw(v, pos - 1, lane)], Wt[sw(v, pos, lane)], Wt[sw(v, pos + 1, lane)], lo, hi);
        FMs[sf(v, c, lane)] = lo;
        FPs[sf(v, c, lane)] = hi;
      }
    }
    __syncthreads();
  } else {
    // PPM: the interpolated value of each of the nd + 3 interfaces once (a cell's
    // upper interface is its neighbour's lower one), four variables at a time,
    // then the monotonicity limits per cell
    const int NI = NF + 1, nfc = nd + 3;
    auto si = [&](int vv, int f, int lane) {
      return D == 0 ? (vv * M + lane) * NI + f : (vv * NI + f) * M + lane;
    };
#pragma unroll
    for (int h = 0; h < NV; h += 4) {
      for (int e = threadIdx.x; e < nfc * M; e += NTS) {
        int f, lane;
        split(e, nfc, f, lane);
        if (lane >= nlane) continue;
        const int p0 = g - 3 + f;   // interface f lies between cells p0 + 1 and p0 + 2
#pragma unroll
        for (int vv = 0; vv < 4; ++vv) {
          if (h + vv >= NV) break;
          const int v = h + vv;
          If[si(vv, f, lane)] = ppm_iface(Wt[sw(v, p0, lane)], Wt[sw(v, p0 + 1, lane)],
                                          Wt[sw(v, p0 + 2, lane)], Wt[sw(v, p0 + 3, lane)]);
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < (nd + 2) * M; e += NTS) {
        int c, lane;
        split(e, nd + 2, c, lane);
        if (lane >= nlane) continue;
        const int pos = g - 1 + c;
#pragma unroll
        for (int vv = 0; vv < 4; ++vv) {
          if (h + vv >= NV) break;
          const int v = h + vv;
          double lo = If[si(vv, c, lane)], hi = If[si(vv, c + 1, lane)];
          ppm_limit(Wt[sw(v, pos, lane)], lo, hi);
          FMs[sf(v, c, lane)] = lo;
          FPs[sf(v, c, lane)] = hi;
        }
      }
      __syncthreads();
    }
  }

  // ---- C: one HLLC solve per face
  for (int e = threadIdx.x; e < (nd + 1) * M; e += NTS) {
    int f, lane;
    split(e, nd + 1, f, lane);
    if (lane >= nlane) continue;
    FState L, R;
    L.r = FPs[sf(0, f, lane)];
    R.r = FMs[sf(0, f + 1, lane)];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      L.v[q] = FPs[sf(1 + q, f, lane)];
      R.v[q] = FMs[sf(1 + q, f + 1, lane)];
    }
    L.P = FPs[sf(4, f, lane)];
    R.P = FMs[sf(4, f + 1, lane)];
    if (EOSK == EOS_TABLE) {
      L.ge = FPs[sf(5, f, lane)]; R.ge = FMs[sf(5, f + 1, lane)];
      L.g1 = FPs[sf(6, f, lane)]; R.g1 = FMs[sf(6, f + 1, lane)];
    } else {
      L.ge = L.g1 = R.ge = R.g1 = p.gamma;
    }
    if (DUAL) {
      L.A = FPs[sf(NV - 1, f, lane)];
      R.A = FMs[sf(NV - 1, f + 1, lane)];
    } else {
      L.A = R.A = 0.0;
    }
    double F[6], vf;
    if (p.riemann == RIEMANN_HLLE) hlle<D, EOSK, DUAL>(p, L, R, F, vf);   // uniform branch
    else hllc<D, EOSK, DUAL>(p, L, R, F, vf);
    if (exc) {
      const int il = D == 0 ? lane * NF + f : f * M + lane;
      const int ir = D == 0 ? lane * NF + f + 1 : (f + 1) * M + lane;
      if (Ex[il] != Ex[ir]) {
        const bool into = Ex[ir] ? dgt0(F[0]) : !dge0(F[0]);
        if (!into) {
#pragma unroll
          for (int q = 0; q < 6; ++q) F[q] = 0.0;
          vf = 0.0;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NVAR; ++q) Fl[sfl(q, f, lane)] = F[q];
    if (DUAL) Fl[sfl(6, f, lane)] = vf;
    if (a.freg && (f == 0 || f == nd)) {
      // time integral dt (F^1 + F^2) / 2 of a boundary face (Eq. lat-flux-impulse);
      // register sides x-, x+, y-, y+, z-, z+, each [nvar][n_OA][n_LA]
      long long so = a.fo[b];
      const int side = 2 * D + (f == nd ? 1 : 0);
      for (int s = 0; s < side; ++s) {
        const int aa = s >> 1;
        const int u1 = aa == 0 ? 1 : 0, u2 = aa == 2 ? 1 : 2;
        so += (long long)B.n[u1] * B.n[u2] * a.nvar;
      }
      const long long ncell = (long long)nl * no;
      const long long cidx = (long long)o * nl + l0 + lane;
      const double w = 0.5 * ta_dt(a.ta, b);
#pragma unroll
      for (int q = 0; q < NVAR; ++q) a.freg[so + q * ncell + cidx] += w * F[q];
    }
  }
  __syncthreads();

  // ---- D: divergence, sources; the last direction completes the update
  // the level read where it is needed (keeps it out of the live registers)
  const double idx = scale2i(p.idx[D], __ldg(&a.blocks[b].level));
  const double hidx = 0.5 * idx;
  for (int e = threadIdx.x; e < nd * M; e += NTS) {
    int c, lane;
    split(e, nd, c, lane);
    if (lane >= nlane) continue;
    const long long flat = base + (long long)(g + c) * sD + lane * sL;
    double acc[NVAR], dv = 0.0;
#pragma unroll
    for (int q = 0; q < NVAR; ++q) acc[q] = a.first ? 0.0 : a.dU[q * ntot + flat];
    if (DUAL) dv = a.first ? 0.0 : a.dU[NVAR * ntot + flat];
#pragma unroll
    for (int q = 0; q < NVAR; ++q) acc[q] -= (Fl[sfl(q, c + 1, lane)] - Fl[sfl(q, c, lane)]) * idx;
    if (DUAL) dv += (Fl[sfl(6, c + 1, lane)] - Fl[sfl(6, c, lane)]) * idx;
    if (grav) {
      const int i0 = D == 0 ? lane * NF + c : c * M + lane;
      const int i1 = D == 0 ? i0 + 1 : i0 + M;
      const int i2 = D == 0 ? i0 + 2 : i0 + 2 * M;
      const double phm = Ph[i0], ph0 = Ph[i1], php = Ph[i2];
      const double rho = Rh[i1];
      acc[1 + D] -= rho * (php - phm) * hidx;
      acc[4] -= (Fl[sfl(0, c + 1, lane)] * (php - ph0) + Fl[sfl(0, c, lane)] * (ph0 - phm)) * hidx;
    }
    if (!LAST) {
#pragma unroll
      for (int q = 0; q < NVAR; ++q) a.dU[q * ntot + flat] = acc[q];
      if (DUAL) a.dU[NVAR * ntot + flat] = dv;
    } else {
      const double dt = ta_dt(a.ta, b);
      if (a.bh.frame) {
        // inertial force of the accelerating frame (Eq. frame-momentum) and its
        // work, from the stage's input state at the cell centre
        const double rin = a.Uin[flat];
        acc[1] -= rin * a.bh.afr[0];
        acc[2] -= rin * a.bh.afr[1];
        acc[3] -= rin * a.bh.afr[2];
        acc[4] -= a.Uin[ntot + flat] * a.bh.afr[0] + a.Uin[2 * ntot + flat] * a.bh.afr[1] +
                  a.Uin[3 * ntot + flat] * a.bh.afr[2];
      }
      double un[NVAR];
#pragma unroll
      for (int q = 0; q < NVAR; ++q) {
        const double u0 = a.U0[q * ntot + flat];
        un[q] = a.stage == 0 ? u0 + dt * acc[q] : 0.5 * (u0 + (a.Uin[q * ntot + flat] + dt * acc[q]));
      }
      if (dlt(un[0], p.rho_floor)) { un[0] = p.rho_floor; count(&a.cnt->rho_floor); }
      if (DUAL) {
        const double dtl = a.stage == 0 ? dt : 0.5 * dt;
        if (EOSK == EOS_IDEAL) {
          un[5] = un[5] * exp(-p.gm1 * dv * dtl);
        } else {
          const double Pa = table_pressure(p, un[0], un[5], a.cnt);
          un[5] = un[5] - Pa * dv * dtl;
        }
        if (dlt(un[5], p.u_floor)) { un[5] = p.u_floor; count(&a.cnt->u_floor); }
      }
      bool bad = !dgt0(un[0]);
#pragma unroll
      for (int q = 0; q < NVAR; ++q) {
        bad |= !dfinite(un[q]);
        a.Uout[q * ntot + flat] = un[q];
      }
      if (bad) count(&a.cnt->nonfinite);
    }
  }
  return true;
}

template <int D, int RECON, int EOSK, int DUAL, int LAST, int M, int NTS, int MINB>
__global__ void __launch_bounds__(NTS, MINB) k_sweep(const SweepArgs a) {
  constexpr int NV = (EOSK == EOS_TABLE ? 7 : 5) + DUAL;
  extern __shared__ __align__(128) double sm[];
  unsigned long long *mbar =
      sweep_mbar<D, RECON, NV, M>(sm, a.PD, a.NF, D == 0 ? M : a.LS);
  if (a.tmap && threadIdx.x == 0) sweep_mbar_init(mbar);   // the tile's __syncthreads orders it
  bool staged;
  sweep_tile<D, RECON, EOSK, DUAL, LAST, M, NTS>(a, blockIdx.y, blockIdx.x, sm, mbar, 0, staged);
}

// ============================================================ launchers ====

template <int D, int RECON, int EOSK, int DUAL, int M, int NTS, int MINB>
cudaError_t sweep_one(const SweepArgs &a, bool last, dim3 grid, size_t smem, cudaStream_t s) {
  // the dynamic shared-memory limit is a per-function attribute (set to this
  // launch's size on every launch: cheap, and correct on whichever device is
  // current; the kernel's static shared memory counts against the same 227 KB)
  auto k = last ? k_sweep<D, RECON, EOSK, DUAL, 1, M, NTS, MINB> : k_sweep<D, RECON, EOSK, DUAL, 0, M, NTS, MINB>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<grid, NTS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, int M, int NTS, int MINB>
cudaError_t sweep_dispatch(const SweepArgs &a, bool last, dim3 grid, size_t smem, cudaStream_t s) {
  const Phys &p = a.p;
  if (p.recon == PLM) {
    if (p.eos == EOS_IDEAL) {
      return p.dual ? sweep_one<D, PLM, EOS_IDEAL, 1, M, NTS, MINB>(a, last, grid, smem, s)
                    : sweep_one<D, PLM, EOS_IDEAL, 0, M, NTS, MINB>(a, last, grid, smem, s);
    }
    return p.dual ? sweep_one<D, PLM, EOS_TABLE, 1, M, NTS, MINB>(a, last, grid, smem, s)
                  : sweep_one<D, PLM, EOS_TABLE, 0, M, NTS, MINB>(a, last, grid, smem, s);
  }
  if (p.eos == EOS_IDEAL) {
    return p.dual ? sweep_one<D, PPM, EOS_IDEAL, 1, M, NTS, MINB>(a, last, grid, smem, s)
                  : sweep_one<D, PPM, EOS_IDEAL, 0, M, NTS, MINB>(a, last, grid, smem, s);
  }
  return p.dual ? sweep_one<D, PPM, EOS_TABLE, 1, M, NTS, MINB>(a, last, grid, smem, s)
                : sweep_one<D, PPM, EOS_TABLE, 0, M, NTS, MINB>(a, last, grid, smem, s);
}

// All directions and scheme variants of one tile shape (instantiated in its own
// translation unit, tde_sweep_m<M>.cu, so that the shapes compile in parallel).
template <int M, int NTS, int MINB>
cudaError_t sweep_launch_shape(const SweepArgs &a, int D, bool last, dim3 grid, size_t smem,
                               cudaStream_t s) {
  if (D == 0) return sweep_dispatch<0, M, NTS, MINB>(a, last, grid, smem, s);
  if (D == 1) return sweep_dispatch<1, M, NTS, MINB>(a, last, grid, smem, s);
  return sweep_dispatch<2, M, NTS, MINB>(a, last, grid, smem, s);
}

// The tile shapes offered to the autotuner: lanes per tile, CTA width, and the
// CTAs per SM the register budget is sized for.  Index 0 is the default.
struct TileShape {
  int M, NTS, MINB;
};
constexpr int N_TILE_SHAPES = N_SWEEP_SHAPES;
constexpr TileShape kTileShapes[N_TILE_SHAPES] = {{8, 288, 3}, {16, 288, 3}, {4, 160, 5}};

cudaError_t sweep_launch_m8(const SweepArgs &a, int D, bool last, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t sweep_launch_m16(const SweepArgs &a, int D, bool last, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t sweep_launch_m4(const SweepArgs &a, int D, bool last, dim3 grid, size_t smem, cudaStream_t s);

// A sweep's complete arguments for direction D and tile shape `shape` (the
// launchers' own arguments, for kernels that run sweep tiles themselves).
SweepArgs sweep_args_dir(tde_mesh *m, int stage, int D, int shape, bool first, const double *U0,
                         const double *Uin, double *Uout, const int32_t *ids, const BH &bh, TimeArgs ta,
                         double *freg);

}  // namespace tde
