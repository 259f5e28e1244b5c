// tde_noalloc.cu -- tde_compute_dt_noalloc: the per-MeshBlock CFL time step
// computed without allocating any device memory.
//
// Who needs it: programs whose device memory belongs to another allocator and
// that may not call cudaMalloc themselves -- for example a host application
// whose framework reserves the whole device in its own memory pool at start-up,
// or a real-time driver loop that forbids allocation after initialisation.
// Those callers cannot create a tde_mesh (which allocates its workspace), so
// this entry point takes the block list, the grid and the state directly and
// keeps all of its scratch -- a copy of the block list, the padded-block
// offsets and the per-block CFL minima -- in one fixed file-scope device array
// that exists in every process that loads the library.  A second, constant
// file-scope array holds the log10 / exp10 tables of the EOS lookups, so the
// results equal tde_compute_dt's bit for bit.
//
// The scratch array is shared by every call in the process: calls whose GPU
// work overlaps (on two streams, or from two threads) race on it and must be
// serialised by the caller.  Each call re-initialises the parts it reads.
#include <math.h>
#include <string.h>

#include "tde_internal.h"

namespace {

using namespace tde;

constexpr int NA_MAX_BLOCKS = 4096;   // largest block count one call accepts
constexpr int NA_NT = 256;

struct NAScratch {
  tde_block_desc blocks[NA_MAX_BLOCKS];      // copy of the caller's block list
  long long off[NA_MAX_BLOCKS + 1];          // first padded cell of each block
  unsigned long long minbits[NA_MAX_BLOCKS]; // per-block CFL minima (IEEE bits)
};

// The only scratch of this entry point (about 176 KB per device).
static __device__ __align__(256) NAScratch g_noalloc_scratch;
// Tables of the table-driven log10 / exp10 that the mesh path's EOS lookups use
// (4.6 KB, constant: written once per device at set-up, never by a kernel).
static __device__ __align__(256) MathTables g_noalloc_mt;

// device addresses of the two arrays, looked up once per device
NAScratch *g_scratch_ptr[64] = {};
const MathTables *g_mt_ptr[64] = {};

__device__ __forceinline__ void na_bh_pos(const BH &bh, double t, double r[3]) {
  const double s = t - bh.t0;
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = bh.x0[a] + bh.v0[a] * s + 0.5 * bh.a0[a] * s * s;
}

// padded sizes, offsets and the +inf initial minima of every block
__global__ void k_na_setup(NAScratch *S, int nb, Phys p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long o = 0;
    for (int b = 0; b < nb; ++b) {
      const tde_block_desc &d = S->blocks[b];
      S->off[b] = o;
      o += (long long)(d.nx + 2 * p.g[0]) * (d.ny + 2 * p.g[1]) * (d.nz + 2 * p.g[2]);
    }
    S->off[nb] = o;
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
    S->minbits[b] = (unsigned long long)__double_as_longlong(INFINITY);
}

// The CFL minimum of tde_compute_dt (k_c2p's want_dt path) with the same
// expressions, so that both entry points give the same bits.
template <int EOSK, int DUAL>
__global__ void __launch_bounds__(NA_NT) k_na_cfl(NAScratch *S, Phys p, BH bh,
                                                  const double *__restrict__ U, long long ntot,
                                                  const double *__restrict__ t_block) {
  const int b = blockIdx.y;
  const tde_block_desc d = S->blocks[b];
  const int n[3] = {d.nx, d.ny, d.nz};
  const int px = d.nx + 2 * p.g[0], py = d.ny + 2 * p.g[1];
  const int nint = n[0] * n[1] * n[2];
  if ((int)blockIdx.x * NA_NT >= nint) return;   // uniform over the CTA
  const int e = blockIdx.x * NA_NT + threadIdx.x;
  double best = INFINITY, best_g2 = INFINITY;   // the hydro limit; the point mass's, squared
  if (e < nint) {
    const int i = e % n[0], r = e / n[0];
    const int c[3] = {i + p.g[0], r % n[1] + p.g[1], r / n[1] + p.g[2]};
    const long long flat = S->off[b] + ((long long)c[2] * py + c[1]) * px + c[0];
    double u[6], w[8];
#pragma unroll
    for (int v = 0; v < 5 + DUAL; ++v) u[v] = U[v * ntot + flat];
    cons_to_prim<EOSK, DUAL>(p, u, w, nullptr);
    bool skip = false;
    double r2 = 0.0;
    if (bh.on || bh.excise) {
      const int o[3] = {d.i0, d.j0, d.k0};
      double x[3], rb[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int g = o[a] + c[a] - p.g[a];
        if (p.bc[a] == 1) {
          const int N = p.active[a] ? p.N[a] << d.level : 1;
          g %= N;
          if (g < 0) g += N;
        }
        x[a] = p.xmin[a] + (g + 0.5) * (p.active[a] ? scale2i(p.dx[a], -d.level) : p.dx[a]);
      }
      na_bh_pos(bh, t_block ? t_block[b] : 0.0, rb);
      r2 = bh_r2(x[0] - rb[0], x[1] - rb[1], x[2] - rb[2]);
      if (bh.excise && inside_radius(r2, bh.rexc)) skip = true;
    }
    if (!skip) {
      const double g1 = EOSK == EOS_TABLE ? w[6] : p.gamma;
      const double cs = sqrt_ratio(g1 * w[4], w[0]);
      // min_d dx_d / (|v_d| + cs) as the reciprocal of the largest signal rate
      double rate = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (p.active[a])
          rate = dmax(rate, (fabs(w[1 + a]) + cs) * scale2i(p.idx[a], d.level));
      best = dmin(best, rcp_nr(rate));
      if (bh.on) best_g2 = bh_dt2(bh_dxg(scale2i(p.dxmin, -d.level), bh.GM), r2, bh.rs2);
    }
  }
  __shared__ double red[2][NA_NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    best_g2 = fmin(best_g2, __shfl_xor_sync(0xffffffffu, best_g2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = best;
    red[1][threadIdx.x >> 5] = best_g2;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < NA_NT / 32 ? red[0][threadIdx.x] : INFINITY;
    best_g2 = threadIdx.x < NA_NT / 32 ? red[1][threadIdx.x] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
      best_g2 = fmin(best_g2, __shfl_xor_sync(0xffffffffu, best_g2, o));
    }
    if (threadIdx.x == 0) {
      best = dmin(best, sqrt(best_g2));
      atomicMin(S->minbits + b, (unsigned long long)__double_as_longlong(best));
    }
  }
}

__global__ void __launch_bounds__(1024) k_na_finalize(NAScratch *S, int nb, double cfl,
                                                      double *dt_block, double *dt_min) {
  __shared__ double red[32];
  double m = INFINITY;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double v = cfl * __longlong_as_double((long long)S->minbits[b]);
    if (dt_block) dt_block[b] = v;
    m = fmin(m, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0 && dt_min) *dt_min = m;
  }
}

int na_fail(tde_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

}  // namespace

extern "C" int tde_compute_dt_noalloc(tde_ctx *ctx, int nblocks, const tde_block_desc *blocks,
                                      const tde_grid_desc *grid, const tde_params *params,
                                      const tde_table_view *table, const double *U, double cfl,
                                      const double *t_block, const tde_bh_state *bhs,
                                      double *dt_block, double *dt_min) {
  if (!ctx) return TDE_EINVAL;
  if (!blocks || !grid || !params || !U || !(cfl > 0.0) || (!dt_block && !dt_min))
    return na_fail(ctx, TDE_EINVAL, "tde_compute_dt_noalloc: null argument or cfl <= 0");
  if (nblocks < 1 || nblocks > NA_MAX_BLOCKS)
    return na_fail(ctx, TDE_EINVAL,
                   "tde_compute_dt_noalloc: nblocks must be 1..4096 (size of its fixed scratch)");
  if (params->eos == TDE_EOS_TABLE && !table)
    return na_fail(ctx, TDE_EINVAL, "tde_compute_dt_noalloc: tabulated EOS without a table view");
  if (params->eos != TDE_EOS_IDEAL && params->eos != TDE_EOS_TABLE)
    return na_fail(ctx, TDE_EINVAL, "tde_compute_dt_noalloc: eos kind");
  if (params->eos == TDE_EOS_TABLE &&
      (!table->log10_e || !table->log10_P || !table->log10_cs2 || table->n_rho < 2 ||
       table->n_T < 2 || !(table->log10_rho_max > table->log10_rho_min) ||
       !(table->log10_T_max > table->log10_T_min)))
    return na_fail(ctx, TDE_EINVAL,
                   "tde_compute_dt_noalloc: table view needs three arrays, n_rho, n_T >= 2 and "
                   "increasing ranges");
  if (ctx->device < 0 || ctx->device >= 64) return na_fail(ctx, TDE_EINVAL, "tde_compute_dt_noalloc: device");
  if (grid->ng < 0 || grid->ng > 8 || grid->N[0] < 1 || grid->N[1] < 1 || grid->N[2] < 1)
    return na_fail(ctx, TDE_EINVAL, "tde_compute_dt_noalloc: grid (N >= 1, ghost width 0..8)");

  // one-time set-up per device (the first call on a device does it; that first
  // call should therefore come before any stream capture): the two arrays'
  // device addresses, and the log10 / exp10 tables copied into the second
  cudaError_t err = cudaSetDevice(ctx->device);
  if (err == cudaSuccess && !g_scratch_ptr[ctx->device]) {
    MathTables h;
    fill_math_tables(&h);
    void *ps = nullptr, *pm = nullptr;
    err = cudaMemcpyToSymbol(g_noalloc_mt, &h, sizeof h);
    if (err == cudaSuccess) err = cudaGetSymbolAddress(&pm, g_noalloc_mt);
    if (err == cudaSuccess) err = cudaGetSymbolAddress(&ps, g_noalloc_scratch);
    if (err == cudaSuccess) {
      g_mt_ptr[ctx->device] = static_cast<const MathTables *>(pm);
      g_scratch_ptr[ctx->device] = static_cast<NAScratch *>(ps);
    }
  }
  if (err != cudaSuccess) {
    ctx->err = std::string("tde_compute_dt_noalloc: ") + cudaGetErrorString(err);
    return TDE_ECUDA;
  }
  NAScratch *S = g_scratch_ptr[ctx->device];

  Phys p{};
  p.eos = params->eos;
  p.dual = params->dual ? 1 : 0;
  p.nvar = 5 + p.dual;
  p.gamma = params->gamma;
  p.gm1 = params->gamma - 1.0;
  p.eta1 = params->eta1;
  p.rho_floor = params->rho_floor;
  p.p_floor = params->p_floor;
  p.unit_rho = params->unit_rho;
  p.unit_e = params->unit_e;
  p.inv_unit_p = 1.0 / (params->unit_rho * params->unit_e);
  p.inv_unit_e = 1.0 / params->unit_e;
  if (p.eos == TDE_EOS_TABLE) {
    p.tab.nr = table->n_rho;
    p.tab.nt = table->n_T;
    p.tab.lr0 = table->log10_rho_min;
    p.tab.inv_dlr = (table->n_rho - 1) / (table->log10_rho_max - table->log10_rho_min);
    p.tab.xr_max = (double)(table->n_rho - 1);
    p.tab.lt0 = table->log10_T_min;
    p.tab.dlt = (table->log10_T_max - table->log10_T_min) / (table->n_T - 1);
    p.tab.le = table->log10_e;
    p.tab.lp = table->log10_P;
    p.tab.lc = table->log10_cs2;
    p.tab.mt = g_mt_ptr[ctx->device];
  }
  p.dxmin = INFINITY;
  for (int a = 0; a < 3; ++a) {
    const int act = grid->N[a] > 1;
    p.N[a] = grid->N[a];
    p.bc[a] = grid->bc[a];
    p.active[a] = act;
    p.g[a] = act ? grid->ng : 0;
    p.xmin[a] = grid->xmin[a];
    p.dx[a] = grid->dx[a];
    p.idx[a] = 1.0 / grid->dx[a];
    if (act && grid->dx[a] < p.dxmin) p.dxmin = grid->dx[a];
  }
  BH bh{};
  if (bhs) {
    bh.on = bhs->on;
    bh.excise = bhs->excise;
    bh.GM = bhs->GM;
    bh.rs2 = bhs->r_soft * bhs->r_soft;
    bh.rexc = bhs->r_exc;
    bh.t0 = bhs->t0;
    for (int a = 0; a < 3; ++a) {
      bh.x0[a] = bhs->x0[a];
      bh.v0[a] = bhs->v0[a];
      bh.a0[a] = bhs->a0[a];
    }
  }
  long long ntot = 0, max_int = 0;
  for (int b = 0; b < nblocks; ++b) {
    const tde_block_desc &d = blocks[b];
    if (d.level < 0 || d.level > 8) return na_fail(ctx, TDE_EINVAL, "tde_compute_dt_noalloc: level");
    // the checks of tde_mesh_create on one block: edges of 1..32 cells, one
    // cell across an inactive direction, the block inside its level's grid
    const int o[3] = {d.i0, d.j0, d.k0}, nn[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
      const int N = p.active[a] ? p.N[a] << d.level : 1;
      if (nn[a] < 1 || nn[a] > 32 || (!p.active[a] && nn[a] != 1) || o[a] < 0 || o[a] + nn[a] > N)
        return na_fail(ctx, TDE_EINVAL,
                       "tde_compute_dt_noalloc: block outside the grid or edge above 32 cells");
    }
    ntot += (long long)(d.nx + 2 * p.g[0]) * (d.ny + 2 * p.g[1]) * (d.nz + 2 * p.g[2]);
    const long long ni = (long long)d.nx * d.ny * d.nz;
    if (ni > max_int) max_int = ni;
  }

  cudaStream_t s = ctx->stream;
  err = cudaMemcpyAsync(S->blocks, blocks, sizeof(tde_block_desc) * nblocks, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) {
    ctx->err = std::string("tde_compute_dt_noalloc: ") + cudaGetErrorString(err);
    return TDE_ECUDA;
  }
  k_na_setup<<<(nblocks + 255) / 256, 256, 0, s>>>(S, nblocks, p);
  dim3 grid_c((unsigned)((max_int + NA_NT - 1) / NA_NT), (unsigned)nblocks);
  if (p.eos == TDE_EOS_IDEAL) {
    if (p.dual) k_na_cfl<EOS_IDEAL, 1><<<grid_c, NA_NT, 0, s>>>(S, p, bh, U, ntot, t_block);
    else k_na_cfl<EOS_IDEAL, 0><<<grid_c, NA_NT, 0, s>>>(S, p, bh, U, ntot, t_block);
  } else {
    if (p.dual) k_na_cfl<EOS_TABLE, 1><<<grid_c, NA_NT, 0, s>>>(S, p, bh, U, ntot, t_block);
    else k_na_cfl<EOS_TABLE, 0><<<grid_c, NA_NT, 0, s>>>(S, p, bh, U, ntot, t_block);
  }
  k_na_finalize<<<1, 1024, 0, s>>>(S, nblocks, cfl, dt_block, dt_min);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    ctx->err = std::string("tde_compute_dt_noalloc: ") + cudaGetErrorString(err);
    return TDE_ECUDA;
  }
  return TDE_OK;
}
