// tde_lat_level.cu -- one LAT level sub-step (Sec. 7.1) as one persistent launch.
//
// The launch sequence of a level sub-step (tde_lat.cu: save the start states;
// per RK stage the conserved ghosts of neighbours on other schedules, the
// conversion to primitives of the interiors and of those ghosts, the primitive
// ghosts of neighbours on the same schedule, and the x, y and z sweeps) runs
// here inside one cooperative kernel whose CTAs stay resident and pass through
// the same phases, separated by grid barriers instead of launch boundaries.
// Each phase does the per-cell work of the corresponding kernel with the same
// device functions on the same data, so the results are the sequence's bit for
// bit; only the distribution of the work over CTAs differs (sweep tiles of the
// default 8-lane shape taken from a work counter per phase, cells and ghost-map
// entries in chunks of one CTA width strided over the CTAs).  The start states
// are saved for their interiors only (no ghost cell of them is read), in the
// first stage's ghost phase.
//
// A barrier is an arrival counter and a generation word in device memory,
// zeroed before each launch (with the work counters from which the CTAs take
// sweep tiles).  A CTA waiting at a barrier gives up after one
// second of the global timer, sets the mesh's status word (tde_mesh_check then
// reports TDE_ETIMEOUT) and leaves the kernel; every later barrier then expires
// for the other CTAs too, so a launch that lost a CTA ends within seconds.  A
// test hook makes CTA 0 skip its first arrival, so that the first wait expires.
//
// Scope: 3-D meshes without refined-mesh ghost operations whose closure is the
// ideal gas or the table inverted by bisection (plain or FP32-guided).  The
// learned-guess closure runs its tensor-core inference in kernels of its own,
// so its levels stay on the launch sequence.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "tde_internal.h"
#include "tde_sweep.cuh"

namespace tde {

namespace {

constexpr int LM = 8, LNTS = LAT_LEVEL_THREADS, LMINB = 3;   // the sweeps' default tile shape
static_assert(kTileShapes[0].M == LM && kTileShapes[0].NTS == LNTS && kTileShapes[0].MINB == LMINB,
              "the level kernel runs the default sweep tile shape");

struct LevelArgs {
  SweepArgs sw[2][3];        // per stage and direction
  const int32_t *ids;        // the level's blocks
  int n;
  const int32_t *f;          // factor of every block
  int flevel, tau;
  const DevBlock *blocks;
  double *U, *U1, *Uold, *W;
  long long ntot;
  const int32_t *gmap;       // ghost (dst, src) pairs
  const int32_t *gstart;     // each block's range of them
  const int32_t *gend;       // the end of its face entries (the ones the sweeps read)
  const int32_t *gsrcb;      // source block of each pair
  const int32_t *glist;      // the level's ghost cells that are converted
  int nglist;
  double *tstart;
  const double *scal;
  Counters *cnt;
  int *status;
  unsigned *bar;             // [0] arrivals, [1] generation, [2 + 3 stage + D] sweep tile counters
  int drop;                  // test hook: CTA 0 skips its first arrival
  const int32_t *pre_int;    // [n + 1] prefix sums of the blocks' interior chunks
  const int32_t *pre_gh;     // [n + 1] prefix sums of their ghost-map chunks
  int tiles[3];              // sweep tiles per block and direction
  size_t mbar_off;           // byte offset of the TMA barrier in shared memory
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number idx (0, 1, ... in program order; the generation word
// counts the completed ones) with a bounded wait.  Returns false (status set)
// if the wait expired.
__device__ __forceinline__ bool grid_barrier(const LevelArgs &a, unsigned idx, bool arrive) {
  __shared__ int s_ok;
  // generic-proxy writes of this phase (the primitives) before the sweeps'
  // tensor copies of other CTAs read them
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();   // this CTA's writes become visible before its arrival
    if (arrive && atomicAdd(&a.bar[0], 1u) == gridDim.x - 1) {
      // last arrival: reset the counter before releasing the others, who
      // cannot arrive at the next barrier before they see the new generation
      atomicExch(&a.bar[0], 0u);
      __threadfence();
      atomicAdd(&a.bar[1], 1u);
    }
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (ld_acquire(&a.bar[1]) <= idx) {
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > 1000000000ull) {
        ok = 0;
        atomicExch(a.status, 1);
        break;
      }
    }
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// one direction's sweep tiles of the level's blocks, taken one at a time from
// the phase's work counter (tile costs differ: empty tiles of smaller blocks,
// excised cells), the next tile's index fetched while the current one runs
template <int D, int RECON, int EOSK, int DUAL, int LAST>
__device__ __forceinline__ bool level_sweep(const SweepArgs &s, int n, int tpb, unsigned *ctr, double *sm,
                                            unsigned long long *mbar, uint32_t *s_par) {
  __shared__ unsigned s_item;
  const unsigned items = (unsigned)n * (unsigned)tpb;
  unsigned next = 0;
  if (threadIdx.x == 0) next = atomicAdd(ctr, 1u);
  for (;;) {
    __syncthreads();   // the previous tile is done with shared memory and s_item
    if (threadIdx.x == 0) s_item = next;
    __syncthreads();
    const unsigned k = s_item;
    if (k >= items) return true;
    // the TMA barrier's phase parity, kept in shared memory (thread 0 flips it
    // after the tile, past the tile's own barriers)
    const uint32_t parity = *s_par;
    if (threadIdx.x == 0) next = atomicAdd(ctr, 1u);
    bool staged;
    if (!sweep_tile<D, RECON, EOSK, DUAL, LAST, LM, LNTS>(s, (int)(k / tpb), (int)(k % tpb), sm, mbar, parity,
                                                          staged))
      return false;
    if (staged && threadIdx.x == 0) *s_par = parity ^ 1u;
  }
}

// The chunks (LNTS consecutive cells or ghost-map entries of one block) of a
// level's blocks, strided over the CTAs: pre[0 .. n] are their prefix sums over
// the level's blocks (offset by the earlier levels' chunks).  fn(q, c) runs
// chunk c of the level's q-th block; q only grows along a CTA's items, so it
// is found by walking forward.
template <typename Fn>
__device__ __forceinline__ void level_chunks(const int32_t *pre, int n, Fn fn) {
  const int base = pre[0], items = pre[n] - base;
  int q = 0;
  for (int k = blockIdx.x; k < items; k += gridDim.x) {
    while (pre[q + 1] <= base + k) ++q;
    fn(q, base + k - pre[q]);
  }
}

// interior cell e of block B: its flat index (-1 past the interior)
__device__ __forceinline__ long long interior_flat(const Phys &p, const DevBlock &B, int e) {
  if (e >= B.n[0] * B.n[1] * B.n[2]) return -1;
  const int i = e % B.n[0], r = e / B.n[0];
  const int j = r % B.n[1], k = r / B.n[1];
  return B.off + ((long long)(k + p.g[2]) * B.p[1] + (j + p.g[1])) * B.p[0] + (i + p.g[0]);
}

// One RK stage of the level (STAGE a template parameter, so that every access to
// the kernel's argument block has a constant offset).
template <int STAGE, int RECON, int EOSK, int DUAL>
__device__ __forceinline__ bool level_stage(const LevelArgs &a, double *sm, unsigned long long *mbar,
                                            uint32_t *s_par) {
  constexpr unsigned B0 = 6 * STAGE;   // this stage's first grid barrier
  constexpr int NVAR = 5 + DUAL;
  constexpr int NWV = (EOSK == EOS_TABLE ? 7 : 5) + DUAL;
  const long long ntot = a.ntot;
  const Phys &p = a.sw[STAGE][0].p;
  double *Udst = STAGE ? a.U1 : a.U;
  if (STAGE == 0) {
    // ---- the start states of the level's blocks (the endpoints of the time
    // interpolation read by faster neighbours later in the window; their
    // interiors only: no ghost cell of Uold is read) and the step start time
    level_chunks(a.pre_int, a.n, [&](int q, int c) {
      const long long flat = interior_flat(p, a.blocks[a.ids[q]], c * LNTS + threadIdx.x);
      if (flat < 0) return;
#pragma unroll
      for (int v = 0; v < NVAR; ++v) a.Uold[v * ntot + flat] = a.U[v * ntot + flat];
    });
    if (blockIdx.x == 0)
      for (int q = threadIdx.x; q < a.n; q += LNTS) a.tstart[a.ids[q]] = a.scal[0] + a.tau * a.scal[3];
  }
  // ---- conserved ghosts from neighbours on other schedules: a faster one's
  // current state, a slower one's state interpolated in time
  level_chunks(a.pre_gh, a.n, [&](int q, int c) {
    const int b = a.ids[q];
    const int e = a.gstart[b] + c * LNTS + threadIdx.x;
    if (e >= a.gend[b]) return;
    const int fn = a.f[a.gsrcb[e]];
    if (fn == a.flevel) return;   // same schedule: its primitives are copied below
    const int2 mp = reinterpret_cast<const int2 *>(a.gmap)[e];
    double t[NVAR];   // every field loaded before any is stored (no overlap)
    if (fn < a.flevel) {
#pragma unroll
      for (int v = 0; v < NVAR; ++v) t[v] = a.U[v * ntot + mp.y];
    } else {
      const double s = (double)(a.tau % fn + STAGE * a.flevel) / (double)fn;
#pragma unroll
      for (int v = 0; v < NVAR; ++v) {
        const double o = a.Uold[v * ntot + mp.y];
        t[v] = o + s * (a.U[v * ntot + mp.y] - o);
      }
    }
#pragma unroll
    for (int v = 0; v < NVAR; ++v) Udst[v * ntot + mp.x] = t[v];
  });
  if (!grid_barrier(a, B0, !(STAGE == 0 && a.drop && blockIdx.x == 0))) return false;
  // ---- primitives of the interiors (events counted) and of the converted
  // ghost cells (not counted)
  level_chunks(a.pre_int, a.n, [&](int q, int c) {
    const long long flat = interior_flat(p, a.blocks[a.ids[q]], c * LNTS + threadIdx.x);
    if (flat < 0) return;
    double u[6], w[8];
#pragma unroll
    for (int v = 0; v < NVAR; ++v) u[v] = Udst[v * ntot + flat];
    cons_to_prim<EOSK, DUAL>(p, u, w, a.cnt);
#pragma unroll
    for (int v = 0; v < NWV; ++v) a.W[v * ntot + flat] = w[v];
  });
  for (int e = blockIdx.x * LNTS + threadIdx.x; e < a.nglist; e += gridDim.x * LNTS) {
    const long long flat = a.glist[e];
    double u[6], w[8];
#pragma unroll
    for (int v = 0; v < NVAR; ++v) u[v] = Udst[v * ntot + flat];
    cons_to_prim<EOSK, DUAL>(p, u, w, nullptr);
#pragma unroll
    for (int v = 0; v < NWV; ++v) a.W[v * ntot + flat] = w[v];
  }
  if (!grid_barrier(a, B0 + 1, true)) return false;
  // ---- primitive ghosts of neighbours on the same schedule
  level_chunks(a.pre_gh, a.n, [&](int q, int c) {
    const int b = a.ids[q];
    const int e = a.gstart[b] + c * LNTS + threadIdx.x;
    if (e >= a.gend[b] || a.f[a.gsrcb[e]] != a.flevel) return;
    const int2 mp = reinterpret_cast<const int2 *>(a.gmap)[e];
    double t[NWV];
#pragma unroll
    for (int v = 0; v < NWV; ++v) t[v] = a.W[v * ntot + mp.y];
#pragma unroll
    for (int v = 0; v < NWV; ++v) a.W[v * ntot + mp.x] = t[v];
  });
  if (!grid_barrier(a, B0 + 2, true)) return false;
  // ---- the sweeps; z completes the stage
  unsigned *ctr = a.bar + 2 + 3 * STAGE;
  if (!level_sweep<0, RECON, EOSK, DUAL, 0>(a.sw[STAGE][0], a.n, a.tiles[0], ctr, sm, mbar, s_par)) return false;
  if (!grid_barrier(a, B0 + 3, true)) return false;
  if (!level_sweep<1, RECON, EOSK, DUAL, 0>(a.sw[STAGE][1], a.n, a.tiles[1], ctr + 1, sm, mbar, s_par))
    return false;
  if (!grid_barrier(a, B0 + 4, true)) return false;
  return level_sweep<2, RECON, EOSK, DUAL, 1>(a.sw[STAGE][2], a.n, a.tiles[2], ctr + 2, sm, mbar, s_par);
}

template <int RECON, int EOSK, int DUAL>
__global__ void __launch_bounds__(LNTS, LMINB) k_lat_level(const LevelArgs a) {
  extern __shared__ __align__(128) double sm[];
  unsigned long long *mbar = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(sm) + a.mbar_off);
  if (a.sw[0][0].tmap && threadIdx.x == 0) sweep_mbar_init(mbar);   // ordered by the first barrier
  __shared__ uint32_t s_par;
  if (threadIdx.x == 0) s_par = 0;   // ordered by the first barrier
  if (!level_stage<0, RECON, EOSK, DUAL>(a, sm, mbar, &s_par)) return;
  if (!grid_barrier(a, 5, true)) return;
  level_stage<1, RECON, EOSK, DUAL>(a, sm, mbar, &s_par);
}

template <int RECON, int EOSK, int DUAL>
cudaError_t launch_level_kernel(const LevelArgs &a, size_t smem, int max_items, cudaStream_t s, int device) {
  auto k = k_lat_level<RECON, EOSK, DUAL>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, sms = 0;
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, LNTS, smem);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // every CTA resident at once (the cooperative launch refuses a grid that is
  // not), and no more CTAs than the largest phase has work items
  const int grid = std::max(1, std::min(per_sm * sms, max_items));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(LNTS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace

bool lat_level_eligible(const tde_mesh *m) {
  const Phys &p = m->phys;
  return p.active[0] && p.active[1] && p.active[2] && m->n_amr == 0 &&
         !(p.eos == EOS_TABLE && p.eos_mode == TDE_INVERT_SURROGATE);
}

cudaError_t launch_lat_level(tde_mesh *m, const BH &bh, const int32_t *ids, int n, int flevel, int tau,
                             const int32_t *glist, int nglist) {
  const Phys &p = m->phys;
  cudaStream_t s = m->ctx->stream;
  LevelArgs a;
  memset(&a, 0, sizeof a);
  const TimeArgs ta{m->d_dtb, 1, m->d_tstart, 1};
  size_t smem = 0;
  for (int stage = 0; stage < 2; ++stage)
    for (int D = 0; D < 3; ++D)
      a.sw[stage][D] = sweep_args_dir(m, stage, D, 0, D == 0, m->U, stage ? m->U1 : m->U, stage ? m->U : m->U1,
                                      ids, bh, ta, m->d_freg);
  for (int D = 0; D < 3; ++D) smem = std::max(smem, sweep_smem_for(m, D, 0));
  a.mbar_off = (smem + 7) / 8 * 8;   // past every direction's layout
  smem = a.mbar_off + 8;
  a.ids = ids;
  a.n = n;
  a.f = m->d_f;
  a.flevel = flevel;
  a.tau = tau;
  a.blocks = m->d_blocks;
  a.U = m->U;
  a.U1 = m->U1;
  a.Uold = m->d_Uold;
  a.W = m->d_W;
  a.ntot = (long long)m->ntot;
  a.gmap = m->d_ghost;
  a.gstart = m->d_gstart;
  a.gend = m->d_gend;
  a.gsrcb = m->d_gsrcb;
  a.glist = glist;
  a.nglist = nglist;
  a.tstart = m->d_tstart;
  a.scal = m->d_scal;
  a.cnt = m->d_cnt;
  a.status = m->d_status;
  a.bar = m->d_lat_bar;
  a.drop = m->inject_level_drop;
  // the level's blocks start at sorted position q0; its chunk prefix sums there
  const int q0 = (int)(ids - m->d_sorted);
  a.pre_int = m->d_lat_pre + q0;
  a.pre_gh = m->d_lat_pre + (m->nb + 1) + q0;
  const int64_t nint = m->h_lat_pre[q0 + n] - m->h_lat_pre[q0];
  const int64_t ngh = m->h_lat_pre[m->nb + 1 + q0 + n] - m->h_lat_pre[m->nb + 1 + q0];
  int64_t items = std::max<int64_t>(std::max(nint, ngh), (nglist + LNTS - 1) / LNTS);
  for (int D = 0; D < 3; ++D) {
    const int LA = D == 0 ? 1 : 0, OA = D == 2 ? 1 : 2;
    a.tiles[D] = ((m->nmax[LA] + LM - 1) / LM) * m->nmax[OA];
    items = std::max<int64_t>(items, (int64_t)n * a.tiles[D]);
  }
  const int max_items = (int)std::min<int64_t>(items, 1 << 30);
  if ((int64_t)n * std::max(a.tiles[0], std::max(a.tiles[1], a.tiles[2])) >= (1LL << 31))
    return cudaErrorInvalidValue;   // tile indices are 32-bit
  cudaError_t err = cudaMemsetAsync(m->d_lat_bar, 0, LAT_BAR_WORDS * sizeof(unsigned), s);
  if (err != cudaSuccess) return err;
  const int dev = m->ctx->device;
  if (p.recon == PPM) {
    if (p.eos == EOS_IDEAL)
      return p.dual ? launch_level_kernel<PPM, EOS_IDEAL, 1>(a, smem, max_items, s, dev)
                    : launch_level_kernel<PPM, EOS_IDEAL, 0>(a, smem, max_items, s, dev);
    return p.dual ? launch_level_kernel<PPM, EOS_TABLE, 1>(a, smem, max_items, s, dev)
                  : launch_level_kernel<PPM, EOS_TABLE, 0>(a, smem, max_items, s, dev);
  }
  if (p.eos == EOS_IDEAL)
    return p.dual ? launch_level_kernel<PLM, EOS_IDEAL, 1>(a, smem, max_items, s, dev)
                  : launch_level_kernel<PLM, EOS_IDEAL, 0>(a, smem, max_items, s, dev);
  return p.dual ? launch_level_kernel<PLM, EOS_TABLE, 1>(a, smem, max_items, s, dev)
                : launch_level_kernel<PLM, EOS_TABLE, 0>(a, smem, max_items, s, dev);
}

}  // namespace tde
