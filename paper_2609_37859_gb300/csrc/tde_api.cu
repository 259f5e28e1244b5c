// tde_api.cu -- the C ABI of libtde.so (declared in include/tde.h): object
// lifetimes, argument checking, the ghost map and the launch sequences of a
// stage and of a step.  No exception or abort leaves this file.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "tde_internal.h"

using namespace tde;

// tables of the table-driven log10 / exp10 (tde_device.cuh), computed in
// extended precision on the host
void tde::fill_math_tables(MathTables *h) {
  for (int j = 0; j < 182; ++j) {
    const long double F = j / 128.0L;
    h->logF[j] = j > 0 ? (double)logl(F) : 0.0;
    h->invF[j] = j > 0 ? (double)(1.0L / F) : 0.0;
    h->F[j] = j / 128.0;
  }
  for (int j = 0; j < 128; ++j) h->exp2j[j] = (double)exp2l(j / 128.0L);
}

namespace {

int fail(tde_ctx *c, int code, const char *msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(tde_ctx *c, cudaError_t e, const char *where) {
  if (c) {
    c->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return TDE_ECUDA;
}

#define CK(ctx, call)                                             \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return cuda_fail((ctx), _e, #call);    \
  } while (0)

BH make_bh(const tde_bh_state *s) {
  BH b{};
  if (!s) return b;
  b.on = s->on;
  b.excise = s->excise;
  b.GM = s->GM;
  b.rs2 = s->r_soft * s->r_soft;
  b.rexc = s->r_exc;
  b.t0 = s->t0;
  b.frame = s->frame_on;
  for (int a = 0; a < 3; ++a) {
    b.x0[a] = s->x0[a];
    b.v0[a] = s->v0[a];
    b.a0[a] = s->a0[a];
    b.afr[a] = s->afr[a];
  }
  return b;
}

bool fill_phys(tde_mesh *m, const tde_params *pr, tde_eos *eos) {
  Phys &p = m->phys;
  p.eos = pr->eos;
  p.recon = pr->recon;
  p.dual = pr->dual ? 1 : 0;
  p.nvar = 5 + p.dual;
  p.nwv = (p.eos == EOS_TABLE ? 7 : 5) + p.dual;
  p.gamma = pr->gamma;
  p.gm1 = pr->gamma - 1.0;
  p.inv_gm1 = 1.0 / (pr->gamma - 1.0);
  p.eta1 = pr->eta1;
  p.eta2 = pr->eta2;
  p.rho_floor = pr->rho_floor;
  p.p_floor = pr->p_floor;
  p.u_floor = pr->u_floor;
  p.unit_rho = pr->unit_rho;
  p.unit_e = pr->unit_e;
  p.inv_unit_p = 1.0 / (pr->unit_rho * pr->unit_e);
  p.inv_unit_e = 1.0 / pr->unit_e;
  p.eos_mode = pr->eos_mode;
  p.riemann = pr->riemann;
  if (p.riemann != TDE_RIEMANN_HLLC && p.riemann != TDE_RIEMANN_HLLE) return false;
  if (p.eos_mode < TDE_INVERT_BISECT || p.eos_mode > TDE_INVERT_BISECT_PLAIN) return false;
  if (p.eos == EOS_TABLE) {
    if (!eos) return false;
    p.tab = eos->tab;
    if (p.eos_mode == TDE_INVERT_BISECT_PLAIN) p.tab.le32 = nullptr;   // every step in FP64
  }
  return true;
}

}  // namespace

namespace tde {
// A mesh whose closure uses the learned guess needs a trained network.
bool closure_ready(const tde_mesh *m) {
  return !(m->phys.eos == EOS_TABLE && m->phys.eos_mode == TDE_INVERT_SURROGATE) ||
         (m->eos && m->eos->has_net && m->sb.rho);
}
}  // namespace tde

namespace {

// Buffers of the learned-guess closure (allocated when a mesh first selects it).
int ensure_surrogate_buffers(tde_mesh *m) {
  if (m->sb.rho || !(m->phys.eos == EOS_TABLE && m->phys.eos_mode == TDE_INVERT_SURROGATE)) return TDE_OK;
  const size_t nt = (size_t)m->ntot;
  cudaError_t err = cudaMalloc(&m->sb.rho, sizeof(double) * nt * 5);
  if (err == cudaSuccess) err = cudaMalloc(&m->sb.queue, sizeof(long long) * nt);
  if (err == cudaSuccess) err = cudaMalloc(&m->sb.qcount, sizeof(unsigned long long));
  if (err != cudaSuccess) return cuda_fail(m->ctx, err, "learned-guess closure buffers");
  m->sb.e = m->sb.rho + nt;
  m->sb.P = m->sb.rho + 2 * nt;
  m->sb.cs2 = m->sb.rho + 3 * nt;
  m->sb.eu = m->sb.rho + 4 * nt;
  return TDE_OK;
}

}  // namespace

// ======================================================== context ====

extern "C" int tde_init(tde_ctx **out, int device, void *cuda_stream) {
  if (!out) return TDE_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TDE_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return TDE_ECUDA;
  tde_ctx *c = new (std::nothrow) tde_ctx;
  if (!c) return TDE_ENOMEM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  *out = c;
  return TDE_OK;
}

extern "C" int tde_set_stream(tde_ctx *ctx, void *cuda_stream) {
  if (!ctx) return TDE_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return TDE_OK;
}

extern "C" const char *tde_last_error(const tde_ctx *ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int tde_finalize(tde_ctx *ctx) {
  if (!ctx) return TDE_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  for (auto &r : ctx->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
  return TDE_OK;
}

// ============================================================= EOS ====

extern "C" int tde_eos_load_table(tde_ctx *ctx, int n_rho, int n_T, double lr_min, double lr_max,
                                  double lT_min, double lT_max, const double *log10_e,
                                  const double *log10_P, const double *log10_cs2, tde_eos **out) {
  if (!ctx || !out) return TDE_EINVAL;
  *out = nullptr;
  if (n_rho < 2 || n_T < 2 || !log10_e || !log10_P || !log10_cs2)
    return fail(ctx, TDE_EINVAL, "tde_eos_load_table: table size or pointer");
  if (!(lr_max > lr_min) || !(lT_max > lT_min))
    return fail(ctx, TDE_EINVAL, "tde_eos_load_table: empty range");
  const size_t nn = (size_t)n_rho * n_T;
  for (size_t k = 0; k < nn; ++k)
    if (!isfinite(log10_e[k]) || !isfinite(log10_P[k]) || !isfinite(log10_cs2[k]))
      return fail(ctx, TDE_EINVAL, "tde_eos_load_table: non-finite entry");
  for (int i = 0; i < n_rho; ++i)
    for (int j = 0; j + 1 < n_T; ++j)
      if (!(log10_e[(size_t)i * n_T + j + 1] > log10_e[(size_t)i * n_T + j]))
        return fail(ctx, TDE_EINVAL, "tde_eos_load_table: log10 e column not increasing in T");
  tde_eos *e = new (std::nothrow) tde_eos;
  if (!e) return TDE_ENOMEM;
  e->ctx = ctx;
  cudaError_t err = cudaMalloc(&e->d_data, 3 * nn * sizeof(double) + nn * sizeof(float));
  if (err == cudaSuccess) err = cudaMalloc(&e->d_cnt, sizeof(Counters));
  if (err != cudaSuccess) {
    cudaFree(e->d_data);
    delete e;
    return cuda_fail(ctx, err, "tde_eos_load_table: cudaMalloc");
  }
  cudaMemcpy(e->d_data, log10_e, nn * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(e->d_data + nn, log10_P, nn * sizeof(double), cudaMemcpyHostToDevice);
  err = cudaMemcpy(e->d_data + 2 * nn, log10_cs2, nn * sizeof(double), cudaMemcpyHostToDevice);
  {
    std::vector<float> le32(nn);
    for (size_t k = 0; k < nn; ++k) le32[k] = (float)log10_e[k];
    if (err == cudaSuccess)
      err = cudaMemcpy(e->d_data + 3 * nn, le32.data(), nn * sizeof(float), cudaMemcpyHostToDevice);
  }
  cudaMemset(e->d_cnt, 0, sizeof(Counters));
  if (err != cudaSuccess) {
    cudaFree(e->d_data);
    cudaFree(e->d_cnt);
    delete e;
    return cuda_fail(ctx, err, "tde_eos_load_table: cudaMemcpy");
  }
  {   // normalisation of the learned guess: centre and half-width of each range
    double emin = log10_e[0], emax = log10_e[0], pmin = log10_P[0], pmax = log10_P[0];
    for (size_t k = 0; k < nn; ++k) {
      emin = std::min(emin, log10_e[k]);
      emax = std::max(emax, log10_e[k]);
      pmin = std::min(pmin, log10_P[k]);
      pmax = std::max(pmax, log10_P[k]);
    }
    // second network input: z = position of log10 e in its interpolated column, in [0, 1]
    const double nv[8] = {0.5 * (lr_min + lr_max), 0.5 * (lr_max - lr_min), 0.5, 0.5,
                          0.5 * (lT_min + lT_max), 0.5 * (lT_max - lT_min),
                          0.5 * (pmin + pmax),     0.5 * (pmax - pmin)};
    (void)emin;
    (void)emax;
    memcpy(e->norm, nv, sizeof nv);
  }
  DTable &t = e->tab;
  t.nr = n_rho;
  t.nt = n_T;
  t.lr0 = lr_min;
  t.inv_dlr = (n_rho - 1) / (lr_max - lr_min);
  t.xr_max = (double)(n_rho - 1);
  t.lt0 = lT_min;
  t.dlt = (lT_max - lT_min) / (n_T - 1);
  t.le = e->d_data;
  t.lp = e->d_data + nn;
  t.lc = e->d_data + 2 * nn;
  t.le32 = reinterpret_cast<const float *>(e->d_data + 3 * nn);
  {   // tables of the table-driven log10 / exp10, computed in extended precision
    MathTables h;
    fill_math_tables(&h);
    err = cudaMalloc(&e->d_mt, sizeof(MathTables));
    if (err == cudaSuccess) err = cudaMemcpy(e->d_mt, &h, sizeof h, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
      cudaFree(e->d_data);
      cudaFree(e->d_cnt);
      cudaFree(e->d_mt);
      delete e;
      return cuda_fail(ctx, err, "tde_eos_load_table: math tables");
    }
    t.mt = e->d_mt;
  }
  *out = e;
  return TDE_OK;
}

extern "C" int tde_eos_destroy(tde_eos *e) {
  if (!e) return TDE_EINVAL;
  cudaFree(e->d_mt);
  cudaFree(e->d_data);
  cudaFree(e->d_cnt);
  cudaFree(e->d_w);
  cudaFree(e->d_wb);
  cudaFree(e->d_status);
  cudaFree(e->d_queue);
  cudaFree(e->d_guess);
  cudaFree(e->d_qcount);
  delete e;
  return TDE_OK;
}

extern "C" int tde_eos_invert(tde_eos *e, int mode, int64_t n, const double *rho, const double *en,
                              double *T, double *P, double *cs2, tde_counts *counts) {
  if (!e) return TDE_EINVAL;
  tde_ctx *c = e->ctx;
  if (n < 0 || (n > 0 && (!rho || !en))) return fail(c, TDE_EINVAL, "tde_eos_invert: arguments");
  if (mode == TDE_INVERT_BISECT || mode == TDE_INVERT_BISECT_PLAIN) {
    CK(c, launch_eos_invert(e, n, rho, en, T, P, cs2, c->stream, mode == TDE_INVERT_BISECT_PLAIN));
  } else if (mode == TDE_INVERT_SURROGATE) {
    if (!e->has_net) return fail(c, TDE_EINVAL, "tde_eos_invert: no trained surrogate");
    CK(c, launch_eos_surrogate(e, n, rho, en, T, P, cs2, c->stream));
  } else {
    return fail(c, TDE_EINVAL, "tde_eos_invert: unknown mode");
  }
  if (counts) {
    Counters h;
    CK(c, cudaMemcpyAsync(&h, e->d_cnt, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    memcpy(counts, &h, sizeof h);
  }
  return TDE_OK;
}

extern "C" int tde_eos_eval_rhoT(tde_eos *e, int64_t n, const double *rho, const double *T,
                                 double *P, double *en, double *cs2) {
  if (!e) return TDE_EINVAL;
  tde_ctx *c = e->ctx;
  if (n < 0 || (n > 0 && (!rho || !T))) return fail(c, TDE_EINVAL, "tde_eos_eval_rhoT: arguments");
  CK(c, launch_eos_eval(e, n, rho, T, P, en, cs2, c->stream));
  return TDE_OK;
}

// ============================================================ mesh ====

static int gcd_int(int a, int b) {
  while (b) { int t = a % b; a = b; b = t; }
  return a < 0 ? -a : a;
}

extern "C" int tde_mesh_create(tde_ctx *ctx, int nblocks, const tde_block_desc *blocks,
                               const tde_grid_desc *grid, const tde_params *params, tde_eos *eos,
                               tde_mesh **out) {
  if (!ctx || !out) return TDE_EINVAL;
  *out = nullptr;
  if (nblocks <= 0 || !blocks || !grid || !params)
    return fail(ctx, TDE_EINVAL, "tde_mesh_create: null argument or no blocks");
  const int ng = grid->ng;
  int act[3];
  for (int a = 0; a < 3; ++a) {
    if (grid->N[a] < 1 || !(grid->dx[a] > 0.0)) return fail(ctx, TDE_EINVAL, "tde_mesh_create: grid");
    if (grid->bc[a] != TDE_BC_OUTFLOW && grid->bc[a] != TDE_BC_PERIODIC)
      return fail(ctx, TDE_EINVAL, "tde_mesh_create: boundary condition");
    act[a] = grid->N[a] > 1;
  }
  if (!act[0] && !act[1] && !act[2]) return fail(ctx, TDE_EINVAL, "tde_mesh_create: no active direction");
  if (params->recon != TDE_RECON_PLM && params->recon != TDE_RECON_PPM)
    return fail(ctx, TDE_EINVAL, "tde_mesh_create: reconstruction");
  if (ng < (params->recon == TDE_RECON_PPM ? 3 : 2) || ng > 4)
    return fail(ctx, TDE_EINVAL, "tde_mesh_create: ghost width below the reconstruction stencil");
  if (params->eos != TDE_EOS_IDEAL && params->eos != TDE_EOS_TABLE)
    return fail(ctx, TDE_EINVAL, "tde_mesh_create: eos kind");
  if (params->eos == TDE_EOS_TABLE && !eos) return fail(ctx, TDE_EINVAL, "tde_mesh_create: table EOS without a table");
  if (params->eos == TDE_EOS_IDEAL && !(params->gamma > 1.0)) return fail(ctx, TDE_EINVAL, "tde_mesh_create: gamma");
  if (!(params->unit_rho > 0.0) || !(params->unit_e > 0.0)) return fail(ctx, TDE_EINVAL, "tde_mesh_create: units");

  tde_mesh *m = new (std::nothrow) tde_mesh;
  if (!m) return TDE_ENOMEM;
  m->ctx = ctx;
  m->eos = eos;
  m->params = *params;
  m->grid = *grid;
  m->nb = nblocks;
  if (!fill_phys(m, params, eos)) { delete m; return fail(ctx, TDE_EINVAL, "tde_mesh_create: eos"); }
  Phys &p = m->phys;
  p.ng = ng;
  p.dxmin = INFINITY;
  for (int a = 0; a < 3; ++a) {
    p.N[a] = grid->N[a];
    p.bc[a] = grid->bc[a];
    p.active[a] = act[a];
    p.g[a] = act[a] ? ng : 0;
    p.xmin[a] = grid->xmin[a];
    p.dx[a] = grid->dx[a];
    p.idx[a] = 1.0 / grid->dx[a];
    if (act[a] && grid->dx[a] < p.dxmin) p.dxmin = grid->dx[a];
  }

  // block geometry, offsets, levels
  m->hblocks.resize(nblocks);
  m->hoff.resize(nblocks + 1);
  int lmax = 0;
  for (int b = 0; b < nblocks; ++b) {
    if (blocks[b].level < 0 || blocks[b].level > 8) {
      delete m;
      return fail(ctx, TDE_EINVAL, "tde_mesh_create: refinement level outside 0..8");
    }
    lmax = std::max(lmax, blocks[b].level);
  }
  m->lmax = lmax;
  auto n_at = [&](int a, int L) { return act[a] ? grid->N[a] << L : 1; };
  int unit[3] = {0, 0, 0};
  int64_t off = 0;
  for (int b = 0; b < nblocks; ++b) {
    const tde_block_desc &d = blocks[b];
    const int o[3] = {d.i0, d.j0, d.k0}, n[3] = {d.nx, d.ny, d.nz};
    DevBlock &B = m->hblocks[b];
    B.i0 = d.i0; B.j0 = d.j0; B.k0 = d.k0;
    B.level = d.level;
    int64_t cells = 1, inter = 1;
    for (int a = 0; a < 3; ++a) {
      if (n[a] < 1 || o[a] < 0 || o[a] + n[a] > n_at(a, d.level) || n[a] > 32 || (!act[a] && n[a] != 1)) {
        delete m;
        return fail(ctx, TDE_EINVAL, "tde_mesh_create: block outside the grid or edge above 32 cells");
      }
      if (d.level > 0 && act[a] && ((o[a] & 3) || (n[a] & 3))) {
        delete m;
        return fail(ctx, TDE_EINVAL, "tde_mesh_create: refined block not aligned to 4 cells");
      }
      B.n[a] = n[a];
      B.p[a] = n[a] + 2 * p.g[a];
      cells *= B.p[a];
      inter *= n[a];
      const int sh = act[a] ? lmax - d.level : 0;   // on the finest level's grid
      unit[a] = gcd_int(gcd_int(unit[a], o[a] << sh), n[a] << sh);
      m->nmax[a] = std::max(m->nmax[a], n[a]);
    }
    B.off = off;
    m->hoff[b] = off;
    off += cells;
    m->max_interior = std::max(m->max_interior, inter);
  }
  m->hoff[nblocks] = off;
  m->ntot = off;
  if (off >= (int64_t)INT32_MAX) { delete m; return fail(ctx, TDE_EINVAL, "tde_mesh_create: more than 2^31 padded cells"); }
  if (sweep_smem_max(m) > SWEEP_SMEM_LIMIT) { delete m; return fail(ctx, TDE_EINVAL, "tde_mesh_create: block too large for one sweep tile"); }

  // owner map of the finest level's grid, one entry per cube of unit cells that
  // every block edge lies on
  int cn[3], NF[3];
  for (int a = 0; a < 3; ++a) {
    NF[a] = n_at(a, lmax);
    unit[a] = gcd_int(unit[a], NF[a]);
    if (unit[a] <= 0) unit[a] = 1;
    cn[a] = NF[a] / unit[a];
  }
  const int64_t ncoarse = (int64_t)cn[0] * cn[1] * cn[2];
  std::vector<int32_t> owner(ncoarse, -1);
  int64_t covered = 0;
  for (int b = 0; b < nblocks; ++b) {
    const tde_block_desc &d = blocks[b];
    int lo[3], hi[3];
    const int o[3] = {d.i0, d.j0, d.k0}, n[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
      const int sh = act[a] ? lmax - d.level : 0;
      lo[a] = (o[a] << sh) / unit[a];
      hi[a] = ((o[a] + n[a]) << sh) / unit[a];
    }
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int32_t &w = owner[((int64_t)k * cn[1] + j) * cn[0] + i];
          if (w != -1) { delete m; return fail(ctx, TDE_EINVAL, "tde_mesh_create: overlapping blocks"); }
          w = b;
          ++covered;
        }
  }
  if (covered != ncoarse) { delete m; return fail(ctx, TDE_EINVAL, "tde_mesh_create: blocks do not cover the grid"); }

  // level-L index helpers: boundary map (periodic wrap, outflow clamp), owner
  auto bmap = [&](int L, int *g) {
    for (int a = 0; a < 3; ++a) {
      const int N = n_at(a, L);
      if (g[a] < 0 || g[a] >= N) {
        if (grid->bc[a] == TDE_BC_PERIODIC) g[a] = ((g[a] % N) + N) % N;
        else g[a] = g[a] < 0 ? 0 : N - 1;
      }
    }
  };
  auto owner_f = [&](const int *f) {
    return owner[((int64_t)(f[2] / unit[2]) * cn[1] + f[1] / unit[1]) * cn[0] + f[0] / unit[0]];
  };
  auto owner_at = [&](int L, const int *g) {
    int f[3];
    for (int a = 0; a < 3; ++a) f[a] = act[a] ? g[a] << (lmax - L) : 0;
    return owner_f(f);
  };
  auto padded = [&](int o, const int *c) {   // padded index of level cell c in block o
    const DevBlock &O = m->hblocks[o];
    return O.off + ((int64_t)(c[2] - O.k0 + p.g[2]) * O.p[1] + (c[1] - O.j0 + p.g[1])) * O.p[0] +
           (c[0] - O.i0 + p.g[0]);
  };
  // a coarse value of the level-L cell g: one cell of a level-L block, or the
  // mean of its children (one or two levels finer, inside one block)
  auto coarse_value = [&](int L, const int *gin, AmrCV &cv) {
    int g[3] = {gin[0], gin[1], gin[2]};
    bmap(L, g);
    const int o = owner_at(L, g);
    const int d = m->hblocks[o].level - L;
    if (d < 0 || d > 2) return false;
    int c[3], last[3];
    for (int a = 0; a < 3; ++a) {
      c[a] = act[a] ? g[a] << d : 0;
      last[a] = act[a] ? c[a] + (1 << d) - 1 : 0;
    }
    if (owner_at(L + d, last) != o) return false;
    cv.base = (int32_t)padded(o, c);
    cv.blk = o;
    cv.depth = d;
    return true;
  };

  // 2:1 balance (faces, edges, corners, periodic images) and the neighbour
  // lists of the factor limiting: every block covering a cell of the one-cell
  // shell, on the finest grid
  m->h_nbr_start.assign(nblocks + 1, 0);
  m->h_nbr.clear();
  for (int b = 0; b < nblocks; ++b) {
    const DevBlock &B = m->hblocks[b];
    const int o[3] = {B.i0, B.j0, B.k0};
    const int L = B.level;
    std::vector<int32_t> nbrs;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = act[a] ? -1 : 0;
      hi[a] = act[a] ? B.n[a] : 0;
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          const int c[3] = {i, j, k};
          bool shell = false;
          for (int a = 0; a < 3; ++a)
            if (act[a] && (c[a] < 0 || c[a] >= B.n[a])) shell = true;
          if (!shell) continue;
          int g[3] = {o[0] + i, o[1] + j, o[2] + k};
          bmap(L, g);
          const int sh = lmax - L;
          for (int fk = 0; fk < (act[2] ? 1 << sh : 1); ++fk)
            for (int fj = 0; fj < (act[1] ? 1 << sh : 1); ++fj)
              for (int fi = 0; fi < (act[0] ? 1 << sh : 1); ++fi) {
                const int f[3] = {act[0] ? (g[0] << sh) + fi : 0, act[1] ? (g[1] << sh) + fj : 0,
                                  act[2] ? (g[2] << sh) + fk : 0};
                const int ob = owner_f(f);
                if (std::abs(m->hblocks[ob].level - L) > 1) {
                  delete m;
                  return fail(ctx, TDE_EINVAL, "tde_mesh_create: neighbours more than one level apart");
                }
                if (ob != b && std::find(nbrs.begin(), nbrs.end(), ob) == nbrs.end()) nbrs.push_back(ob);
              }
        }
    m->h_nbr.insert(m->h_nbr.end(), nbrs.begin(), nbrs.end());
    m->h_nbr_start[b + 1] = (int32_t)m->h_nbr.size();
  }

  // ghost map: a ghost cell whose mapped cell lies in a block of its own level
  // is a copy (gmap, source block gsrcb); on a refined mesh the others are
  // restriction or prolongation ops
  std::vector<int32_t> gmap, gsrcb;
  std::vector<int32_t> gstart(nblocks + 1, 0), gend(nblocks, 0);
  std::vector<int32_t> fmap, omap, fsrc, osrc;   // one block's face and other copies
  std::vector<AmrOp> amr;
  std::vector<int32_t> amr_start(nblocks + 1, 0);
  for (int b = 0; b < nblocks; ++b) {
    const DevBlock &B = m->hblocks[b];
    const int o[3] = {B.i0, B.j0, B.k0};
    const int L = B.level;
    int cnt = 0, namr = 0;
    for (int k = 0; k < B.p[2]; ++k)
      for (int j = 0; j < B.p[1]; ++j)
        for (int i = 0; i < B.p[0]; ++i) {
          const int c[3] = {i, j, k};
          bool inside = true;
          for (int a = 0; a < 3; ++a)
            if (c[a] < p.g[a] || c[a] >= p.g[a] + B.n[a]) inside = false;
          if (inside) continue;
          int gg[3];
          for (int a = 0; a < 3; ++a) gg[a] = o[a] + c[a] - p.g[a];
          bmap(L, gg);
          const int ob = owner_at(L, gg);
          const int64_t dst = B.off + ((int64_t)k * B.p[1] + j) * B.p[0] + i;
          const int Lo = m->hblocks[ob].level;
          if (Lo == L) {
            // face ghosts (one direction outside the interior) first
            int nout = 0;
            for (int a = 0; a < 3; ++a)
              if (c[a] < p.g[a] || c[a] >= p.g[a] + B.n[a]) ++nout;
            std::vector<int32_t> &em = nout == 1 ? fmap : omap;
            em.push_back((int32_t)dst);
            em.push_back((int32_t)padded(ob, gg));
            (nout == 1 ? fsrc : osrc).push_back(ob);
            ++cnt;
            continue;
          }
          AmrOp op{};
          op.dst = (int32_t)dst;
          bool ok = true;
          if (Lo > L) {
            op.kind = -1;
            ok = coarse_value(L, gg, op.cv[0]);
          } else {
            int par[3];
            op.kind = 0;
            for (int a = 0; a < 3; ++a) {
              par[a] = act[a] ? gg[a] >> 1 : 0;
              if (act[a] && (gg[a] & 1)) op.kind |= 1 << a;
            }
            ok = Lo == L - 1 && coarse_value(L - 1, par, op.cv[0]);
            for (int a = 0; ok && a < 3; ++a) {
              if (!act[a]) continue;
              int q[3] = {par[0], par[1], par[2]};
              q[a] = par[a] + 1;
              ok = coarse_value(L - 1, q, op.cv[1 + 2 * a]);
              q[a] = par[a] - 1;
              if (ok) ok = coarse_value(L - 1, q, op.cv[2 + 2 * a]);
            }
          }
          if (!ok) {
            delete m;
            return fail(ctx, TDE_EINVAL, "tde_mesh_create: a ghost stencil reaches two levels coarser or finer");
          }
          amr.push_back(op);
          ++namr;
        }
    gstart[b + 1] = gstart[b] + cnt;
    gend[b] = gstart[b] + (int32_t)fsrc.size();
    gmap.insert(gmap.end(), fmap.begin(), fmap.end());
    gmap.insert(gmap.end(), omap.begin(), omap.end());
    gsrcb.insert(gsrcb.end(), fsrc.begin(), fsrc.end());
    gsrcb.insert(gsrcb.end(), osrc.begin(), osrc.end());
    fmap.clear(); omap.clear(); fsrc.clear(); osrc.clear();
    amr_start[b + 1] = amr_start[b] + namr;
    m->max_ghosts = std::max(m->max_ghosts, cnt);
    m->max_amr = std::max(m->max_amr, namr);
  }

  // device allocations
  std::vector<int32_t> allids(nblocks);
  std::iota(allids.begin(), allids.end(), 0);
  const size_t nt = (size_t)m->ntot;
  cudaError_t err = cudaSuccess;
  auto A = [&](void **ptr, size_t bytes) {
    if (err == cudaSuccess) err = cudaMalloc(ptr, bytes > 0 ? bytes : 8);
  };
  A((void **)&m->d_blocks, sizeof(DevBlock) * nblocks);
  A((void **)&m->d_ghost, sizeof(int32_t) * gmap.size());
  A((void **)&m->d_gstart, sizeof(int32_t) * (nblocks + 1));
  A((void **)&m->d_gend, sizeof(int32_t) * nblocks);
  A((void **)&m->d_allids, sizeof(int32_t) * nblocks);
  A((void **)&m->d_W, sizeof(double) * nt * p.nwv);
  A((void **)&m->d_dU, sizeof(double) * nt * (p.nvar + 1));
  A((void **)&m->d_scal, sizeof(double) * 4);
  A((void **)&m->d_dtb, sizeof(double) * nblocks);
  A((void **)&m->d_dtbits, sizeof(unsigned long long) * nblocks);
  A((void **)&m->d_cnt, sizeof(Counters));
  A((void **)&m->d_status, sizeof(int));
  A((void **)&m->d_phic, sizeof(double) * nt);
  A((void **)&m->d_excc, nt);
  A((void **)&m->d_gsrcb, sizeof(int32_t) * gsrcb.size());
  A((void **)&m->d_nbr_start, sizeof(int32_t) * (nblocks + 1));
  A((void **)&m->d_nbr, sizeof(int32_t) * m->h_nbr.size());
  A((void **)&m->d_owner, sizeof(int32_t) * owner.size());
  A((void **)&m->d_tstart, sizeof(double) * nblocks);
  if (!amr.empty()) {
    A((void **)&m->d_amr, sizeof(AmrOp) * amr.size());
    A((void **)&m->d_amr_start, sizeof(int32_t) * (nblocks + 1));
  }
  if (err != cudaSuccess) {
    tde_mesh_destroy(m);
    return cuda_fail(ctx, err, "tde_mesh_create: cudaMalloc");
  }
  std::vector<unsigned long long> inf_bits(nblocks);
  const double inf = INFINITY;
  unsigned long long ib;
  memcpy(&ib, &inf, 8);
  std::fill(inf_bits.begin(), inf_bits.end(), ib);
  const double zeros[4] = {0, 0, 0, 0};
  cudaMemcpy(m->d_blocks, m->hblocks.data(), sizeof(DevBlock) * nblocks, cudaMemcpyHostToDevice);
  if (!gmap.empty()) cudaMemcpy(m->d_ghost, gmap.data(), sizeof(int32_t) * gmap.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_gstart, gstart.data(), sizeof(int32_t) * (nblocks + 1), cudaMemcpyHostToDevice);
  m->h_gstart = gstart;
  if (!amr.empty())   // refined meshes: every entry
    for (int b = 0; b < nblocks; ++b) gend[b] = gstart[b + 1];
  m->h_gend = gend;
  cudaMemcpy(m->d_gend, gend.data(), sizeof(int32_t) * nblocks, cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_allids, allids.data(), sizeof(int32_t) * nblocks, cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_scal, zeros, sizeof zeros, cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_dtbits, inf_bits.data(), sizeof(unsigned long long) * nblocks, cudaMemcpyHostToDevice);
  if (!gsrcb.empty()) cudaMemcpy(m->d_gsrcb, gsrcb.data(), sizeof(int32_t) * gsrcb.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_nbr_start, m->h_nbr_start.data(), sizeof(int32_t) * (nblocks + 1), cudaMemcpyHostToDevice);
  if (!m->h_nbr.empty()) cudaMemcpy(m->d_nbr, m->h_nbr.data(), sizeof(int32_t) * m->h_nbr.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(m->d_owner, owner.data(), sizeof(int32_t) * owner.size(), cudaMemcpyHostToDevice);
  cudaMemset(m->d_tstart, 0, sizeof(double) * nblocks);
  if (!amr.empty()) {
    cudaMemcpy(m->d_amr, amr.data(), sizeof(AmrOp) * amr.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(m->d_amr_start, amr_start.data(), sizeof(int32_t) * (nblocks + 1), cudaMemcpyHostToDevice);
  }
  m->n_gcopy = (int64_t)gsrcb.size();
  m->n_amr = (int64_t)amr.size();
  for (int a = 0; a < 3; ++a) {
    m->unit[a] = unit[a];
    m->cn[a] = cn[a];
  }
  cudaMemset(m->d_dU, 0, sizeof(double) * nt * (p.nvar + 1));
  cudaMemset(m->d_W, 0, sizeof(double) * nt * p.nwv);
  err = cudaMemset(m->d_cnt, 0, sizeof(Counters));
  if (err == cudaSuccess) err = cudaMemset(m->d_status, 0, sizeof(int));
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = build_sweep_tmaps(m);
  if (err != cudaSuccess) {
    tde_mesh_destroy(m);
    return cuda_fail(ctx, err, "tde_mesh_create: upload");
  }
  if (ensure_surrogate_buffers(m) != TDE_OK) {
    tde_mesh_destroy(m);
    return TDE_ENOMEM;
  }
  *out = m;
  return TDE_OK;
}

extern "C" int tde_mesh_destroy(tde_mesh *m) {
  if (!m) return TDE_EINVAL;
  cudaFree(m->d_blocks);
  cudaFree(m->d_ghost);
  cudaFree(m->d_gstart);
  cudaFree(m->d_gend);
  cudaFree(m->d_allids);
  cudaFree(m->d_W);
  cudaFree(m->d_dU);
  cudaFree(m->d_scal);
  cudaFree(m->d_dtb);
  cudaFree(m->d_dtbits);
  cudaFree(m->d_cnt);
  cudaFree(m->d_status);
  cudaFree(m->d_phic);
  cudaFree(m->d_excc);
  cudaFree(m->d_tmaps);
  cudaFree(m->d_gsrcb);
  cudaFree(m->d_nbr_start);
  cudaFree(m->d_nbr);
  cudaFree(m->d_owner);
  cudaFree(m->d_tstart);
  cudaFree(m->d_amr);
  cudaFree(m->d_amr_start);
  cudaFree(m->d_lat_glist);
  cudaFree(m->d_lat_gstart);
  cudaFree(m->sb.rho);
  cudaFree(m->sb.lTg);
  cudaFree(m->sb.queue);
  cudaFree(m->sb.qcount);
  cudaFree(m->d_frame_part);
  cudaFree(m->d_frame_out);
  gravity_release(m);
  cudaFree(m->d_f);
  cudaFree(m->d_f2);
  cudaFree(m->d_sorted);
  cudaFree(m->d_lat_bar);
  cudaFree(m->d_lat_pre);
  cudaFree(m->d_Uold);
  cudaFree(m->d_freg);
  cudaFree(m->d_fo);
  cudaFree(m->d_flag);
  if (m->lat_graph) cudaGraphExecDestroy(m->lat_graph);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  delete m;
  return TDE_OK;
}

extern "C" int tde_mesh_info(const tde_mesh *m, int64_t *ntot, int *nvar, int64_t *offsets) {
  if (!m) return TDE_EINVAL;
  if (ntot) *ntot = m->ntot;
  if (nvar) *nvar = m->phys.nvar;
  if (offsets) memcpy(offsets, m->hoff.data(), sizeof(int64_t) * (m->nb + 1));
  return TDE_OK;
}

extern "C" int tde_mesh_set_params(tde_mesh *m, const tde_params *pr) {
  if (!m || !pr) return TDE_EINVAL;
  if (pr->eos != m->params.eos || (pr->dual ? 1 : 0) != m->phys.dual)
    return fail(m->ctx, TDE_EINVAL, "tde_mesh_set_params: eos kind or dual flag changed");
  if (pr->recon == TDE_RECON_PPM && m->phys.ng < 3) return fail(m->ctx, TDE_EINVAL, "tde_mesh_set_params: PPM needs ng >= 3");
  Phys keep = m->phys;
  if (!fill_phys(m, pr, m->eos)) { m->phys = keep; return TDE_EINVAL; }
  Phys &p = m->phys;
  for (int a = 0; a < 3; ++a) {
    p.N[a] = keep.N[a]; p.bc[a] = keep.bc[a]; p.active[a] = keep.active[a]; p.g[a] = keep.g[a];
    p.xmin[a] = keep.xmin[a]; p.dx[a] = keep.dx[a]; p.idx[a] = keep.idx[a];
  }
  p.ng = keep.ng;
  p.dxmin = keep.dxmin;
  m->params = *pr;
  int rb = ensure_surrogate_buffers(m);
  if (rb) return rb;
  if (m->lat_graph) {   // captured launches hold the old parameters
    cudaGraphExecDestroy(m->lat_graph);
    m->lat_graph = nullptr;
  }
  return TDE_OK;
}

extern "C" int tde_mesh_bind_state(tde_mesh *m, double *U, double *U1) {
  if (!m || !U || !U1 || U == U1) return m ? fail(m->ctx, TDE_EINVAL, "tde_mesh_bind_state: states") : TDE_EINVAL;
  m->U = U;
  m->U1 = U1;
  return TDE_OK;
}

extern "C" int tde_prim_to_cons(tde_mesh *m, const double *W, double *U) {
  if (!m || !W || !U) return TDE_EINVAL;
  CK(m->ctx, launch_prim2cons(m, W, U));
  return TDE_OK;
}

extern "C" int tde_ghost_fill(tde_mesh *m, double *state, int nvar) {
  if (!m || !state || nvar < 1 || nvar > 8) return TDE_EINVAL;
  CK(m->ctx, launch_ghost(m, state, nvar, m->nb, m->d_allids));
  CK(m->ctx, launch_ghost_amr(m, state, nullptr, nullptr, nvar, m->nb, m->d_allids, nullptr, 0, 0, 0));
  return TDE_OK;
}

extern "C" int tde_mesh_set_time(tde_mesh *m, double t) {
  if (!m) return TDE_EINVAL;
  CK(m->ctx, cudaMemcpyAsync(m->d_scal, &t, sizeof t, cudaMemcpyHostToDevice, m->ctx->stream));
  CK(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  return TDE_OK;
}

extern "C" int tde_mesh_get_time(tde_mesh *m, double *t) {
  if (!m || !t) return TDE_EINVAL;
  CK(m->ctx, cudaMemcpyAsync(t, m->d_scal, sizeof *t, cudaMemcpyDeviceToHost, m->ctx->stream));
  CK(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  return TDE_OK;
}

// ============================================================ stage ====

static int run_stage(tde_mesh *m, int stage, int nblk, const int32_t *ids, const BH &bh,
                     TimeArgs ta, bool prims_ready) {
  tde_ctx *c = m->ctx;
  const double *Uin = stage == 0 ? m->U : m->U1;
  double *Uout = stage == 0 ? m->U1 : m->U;
  const bool all = ids == m->d_allids;
  if (all) {
    // every block advances: primitives of the interiors, then a copy of the
    // neighbours' primitives into the ghost layer
    if (!prims_ready) CK(c, launch_c2p(m, Uin, nblk, ids, false, bh, ta));
    CK(c, launch_ghost(m, m->d_W, m->phys.nwv, nblk, ids, true));
  } else {
    // a subset advances: refresh the conserved ghosts of the listed blocks from
    // the stage input and convert every padded cell of those blocks
    CK(c, launch_ghost(m, const_cast<double *>(Uin), m->phys.nvar, nblk, ids));
    CK(c, launch_c2p_padded(m, Uin, nblk, ids));
  }
  CK(c, launch_sweeps(m, stage, m->U, Uin, Uout, nblk, ids, bh, ta));
  return TDE_OK;
}

extern "C" int tde_hydro_stage(tde_mesh *m, int stage, int nblk, const int32_t *ids,
                               const double *dt_block, const double *t_block,
                               const tde_bh_state *bh) {
  if (!m) return TDE_EINVAL;
  if (!m->U || !m->U1) return fail(m->ctx, TDE_EINVAL, "tde_hydro_stage: no bound state");
  if (!closure_ready(m)) return fail(m->ctx, TDE_EINVAL, "tde_hydro_stage: surrogate closure without a trained network");
  if ((stage != 0 && stage != 1) || !dt_block) return fail(m->ctx, TDE_EINVAL, "tde_hydro_stage: arguments");
  if (m->lmax > 0) return fail(m->ctx, TDE_EINVAL, "tde_hydro_stage: refined mesh (use tde_step or LAT windows)");
  if (!ids) { ids = m->d_allids; nblk = m->nb; }
  if (nblk <= 0 || nblk > m->nb) return fail(m->ctx, TDE_EINVAL, "tde_hydro_stage: block count");
  TimeArgs ta{dt_block, 1, t_block, 1};
  return run_stage(m, stage, nblk, ids, make_bh(bh), ta, false);
}

extern "C" int tde_compute_dt(tde_mesh *m, double cfl, const double *t_block,
                              const tde_bh_state *bh, double *dt_block, double *dt_min) {
  if (!m || !m->U || !(cfl > 0.0)) return m ? fail(m->ctx, TDE_EINVAL, "tde_compute_dt: arguments") : TDE_EINVAL;
  if (!closure_ready(m)) return fail(m->ctx, TDE_EINVAL, "tde_compute_dt: surrogate closure without a trained network");
  TimeArgs ta{nullptr, 0, t_block, 1};
  CK(m->ctx, launch_c2p(m, m->U, m->nb, m->d_allids, true, make_bh(bh), ta));
  CK(m->ctx, launch_dt_finalize(m, cfl, dt_block ? dt_block : m->d_dtb, dt_min));
  return TDE_OK;
}

extern "C" int tde_excise(tde_mesh *m, int nblk, const int32_t *ids, const double *t_end_block,
                          const tde_bh_state *bh) {
  if (!m || !m->U || !t_end_block) return TDE_EINVAL;
  if (!bh || !bh->excise) return TDE_OK;
  if (!ids) { ids = m->d_allids; nblk = m->nb; }
  TimeArgs ta{nullptr, 0, t_end_block, 1};
  CK(m->ctx, launch_excise(m, m->U, nblk, ids, make_bh(bh), ta));
  return TDE_OK;
}

extern "C" int tde_dual_energy_sync(tde_mesh *m, int nblk, const int32_t *ids, double eta2) {
  if (!m || !m->U) return TDE_EINVAL;
  if (!m->phys.dual) return TDE_OK;
  if (!ids) { ids = m->d_allids; nblk = m->nb; }
  CK(m->ctx, launch_sync(m, m->U, nblk, ids, eta2 < 0.0 ? m->phys.eta2 : eta2));
  return TDE_OK;
}

extern "C" int tde_step(tde_mesh *m, double cfl, double dt_fixed, const tde_bh_state *bhs,
                        double *dt_out) {
  if (!m) return TDE_EINVAL;
  if (!m->U || !m->U1) return fail(m->ctx, TDE_EINVAL, "tde_step: no bound state");
  if (!closure_ready(m)) return fail(m->ctx, TDE_EINVAL, "tde_step: surrogate closure without a trained network");
  if (!(cfl > 0.0) && !(dt_fixed > 0.0)) return fail(m->ctx, TDE_EINVAL, "tde_step: need cfl or dt");
  tde_ctx *c = m->ctx;
  const BH bh = make_bh(bhs);
  TimeArgs ta{m->d_scal + 1, 0, m->d_scal, 0};
  if (cfl > 0.0) {
    CK(c, launch_c2p(m, m->U, m->nb, m->d_allids, true, bh, ta));
    CK(c, launch_dt_finalize(m, cfl, m->d_dtb, nullptr));
  } else {
    CK(c, launch_set_dt(m, dt_fixed));
    if (m->lmax == 0) CK(c, launch_c2p(m, m->U, m->nb, m->d_allids, false, bh, ta));
  }
  if (m->lmax > 0) {
    // refined mesh: one LAT window with every factor 1 (dt0 = this step's dt)
    int r = lat_step_all_ones(m, bh);
    if (r) return r;
    if (dt_out) CK(c, cudaMemcpyAsync(dt_out, m->d_scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return TDE_OK;
  }
  int r = run_stage(m, 0, m->nb, m->d_allids, bh, ta, true);
  if (r) return r;
  r = run_stage(m, 1, m->nb, m->d_allids, bh, ta, false);
  if (r) return r;
  if (bh.excise) CK(c, launch_excise(m, m->U, m->nb, m->d_allids, bh, ta));
  if (m->phys.dual) CK(c, launch_sync(m, m->U, m->nb, m->d_allids, m->phys.eta2));
  if (dt_out) CK(c, cudaMemcpyAsync(dt_out, m->d_scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  CK(c, launch_advance_time(m));
  return TDE_OK;
}

extern "C" int tde_mesh_set_tiles(tde_mesh *m, const int32_t *tiles) {
  if (!m) return TDE_EINVAL;
  if (!tiles) return fail(m->ctx, TDE_EINVAL, "tde_mesh_set_tiles: null");
  for (int D = 0; D < 3; ++D)
    if (tiles[D] < 0 || tiles[D] >= N_SWEEP_SHAPES || sweep_smem_for(m, D, tiles[D]) > SWEEP_SMEM_LIMIT)
      return fail(m->ctx, TDE_EINVAL, "tde_mesh_set_tiles: unknown shape or tile too large");
  for (int D = 0; D < 3; ++D) m->tile[D] = tiles[D];
  invalidate_graph(m);
  return TDE_OK;
}

extern "C" int tde_mesh_get_tiles(const tde_mesh *m, int32_t *tiles) {
  if (!m || !tiles) return TDE_EINVAL;
  for (int D = 0; D < 3; ++D) tiles[D] = m->tile[D];
  return TDE_OK;
}

extern "C" int tde_mesh_autotune(tde_mesh *m, const tde_bh_state *bhs, int reps, int32_t *tiles,
                                 float *ms) {
  if (!m) return TDE_EINVAL;
  if (!m->U || !m->U1) return fail(m->ctx, TDE_EINVAL, "tde_mesh_autotune: no bound state");
  if (reps < 1) return fail(m->ctx, TDE_EINVAL, "tde_mesh_autotune: reps < 1");
  float t[3][N_SWEEP_SHAPES];
  CK(m->ctx, autotune_sweeps(m, make_bh(bhs), reps, t));
  invalidate_graph(m);
  if (tiles)
    for (int D = 0; D < 3; ++D) tiles[D] = m->tile[D];
  if (ms)
    for (int D = 0; D < 3; ++D)
      for (int k = 0; k < N_SWEEP_SHAPES; ++k) ms[D * N_SWEEP_SHAPES + k] = t[D][k];
  return TDE_OK;
}

extern "C" int tde_frame_acceleration(tde_mesh *m, const tde_bh_state *bh, double rho_min, double *A,
                                      double *mass) {
  if (!m) return TDE_EINVAL;
  if (!m->U || !bh || !A) return fail(m->ctx, TDE_EINVAL, "tde_frame_acceleration: arguments");
  if (!m->d_frame_out) CK(m->ctx, cudaMalloc(&m->d_frame_out, sizeof(double) * 4));
  CK(m->ctx, launch_frame_acceleration(m, make_bh(bh), rho_min, m->d_frame_out));
  double h[4];
  CK(m->ctx, cudaMemcpyAsync(h, m->d_frame_out, sizeof h, cudaMemcpyDeviceToHost, m->ctx->stream));
  CK(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  for (int k = 0; k < 3; ++k) A[k] = h[k];
  if (mass) *mass = h[3];
  return TDE_OK;
}

extern "C" int tde_mesh_boost(tde_mesh *m, const double *V, double rho_min) {
  if (!m) return TDE_EINVAL;
  if (!m->U || !V) return fail(m->ctx, TDE_EINVAL, "tde_mesh_boost: arguments");
  CK(m->ctx, launch_boost(m, V, rho_min));
  return TDE_OK;
}

static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

extern "C" int tde_gravity_solve(tde_mesh *m, const tde_grav_params *gp, int *cycles, double *defect) {
  if (!m) return TDE_EINVAL;
  if (!m->U || !gp || gp->max_cycles < 0 || gp->npre < 0 || gp->npost < 0 ||
      (gp->boundary != TDE_GRAV_PERIODIC && gp->boundary != TDE_GRAV_ISOLATED) ||
      (gp->boundary == TDE_GRAV_ISOLATED && (gp->lmax < 0 || gp->lmax > 4)))
    return fail(m->ctx, TDE_EINVAL, "tde_gravity_solve: arguments");
  for (int a = 0; a < 3; ++a)
    if (m->phys.N[a] > 1 && (!pow2(m->phys.N[a]) ||
                             (gp->boundary == TDE_GRAV_PERIODIC && m->phys.bc[a] != TDE_BC_PERIODIC)))
      return fail(m->ctx, TDE_EINVAL, "tde_gravity_solve: needs power-of-two directions (periodic ones for a periodic solve)");
  if (m->lmax > 0) return fail(m->ctx, TDE_EINVAL, "tde_gravity_solve: refined mesh");
  CK(m->ctx, gravity_solve(m, *gp, cycles, defect));
  invalidate_graph(m);
  return TDE_OK;
}

extern "C" int tde_gravity_enable(tde_mesh *m, int on) {
  if (!m) return TDE_EINVAL;
  if (on && !m->d_phi_sg) return fail(m->ctx, TDE_EINVAL, "tde_gravity_enable: no potential solved yet");
  m->grav_on = on ? 1 : 0;
  invalidate_graph(m);
  return TDE_OK;
}

extern "C" int tde_gravity_phi(tde_mesh *m, double *phi) {
  if (!m) return TDE_EINVAL;
  if (!phi || !m->grav) return fail(m->ctx, TDE_EINVAL, "tde_gravity_phi: no potential");
  CK(m->ctx, gravity_copy_phi(m, phi));
  return TDE_OK;
}

extern "C" int tde_mesh_remap(tde_mesh *dst, double *Udst, const tde_mesh *src, const double *Usrc, int mode,
                              double rho_floor, double u_floor) {
  if (!dst) return TDE_EINVAL;
  if (!src || !Udst || !Usrc || (const double *)Udst == Usrc ||
      (mode != TDE_REMAP_THERMAL && mode != TDE_REMAP_TOTAL))
    return fail(dst->ctx, TDE_EINVAL, "tde_mesh_remap: arguments");
  if (src->ctx != dst->ctx) return fail(dst->ctx, TDE_EINVAL, "tde_mesh_remap: meshes of different contexts");
  if (src->lmax > 0 || dst->lmax > 0) return fail(dst->ctx, TDE_EINVAL, "tde_mesh_remap: refined mesh");
  CK(dst->ctx, launch_remap(dst, Udst, src, Usrc, mode, rho_floor, u_floor));
  return TDE_OK;
}

extern "C" int tde_counts_read(tde_mesh *m, tde_counts *out, int reset) {
  if (!m || !out) return TDE_EINVAL;
  Counters h;
  CK(m->ctx, cudaMemcpyAsync(&h, m->d_cnt, sizeof h, cudaMemcpyDeviceToHost, m->ctx->stream));
  if (reset) CK(m->ctx, cudaMemsetAsync(m->d_cnt, 0, sizeof(Counters), m->ctx->stream));
  CK(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  static_assert(sizeof(Counters) == sizeof(tde_counts), "counter layout");
  memcpy(out, &h, sizeof h);
  return TDE_OK;
}

extern "C" int tde_mesh_check(tde_mesh *m) {
  if (!m) return TDE_EINVAL;
  Counters h;
  CK(m->ctx, cudaMemcpyAsync(&h, m->d_cnt, sizeof h, cudaMemcpyDeviceToHost, m->ctx->stream));
  CK(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  if (h.nonfinite) {
    char msg[160];
    snprintf(msg, sizeof msg, "tde_mesh_check: %llu non-finite or non-positive-density results",
             (unsigned long long)h.nonfinite);
    return fail(m->ctx, TDE_ENUMERIC, msg);
  }
  int st = 0;
  CK(m->ctx, cudaMemcpy(&st, m->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (st) {
    CK(m->ctx, cudaMemset(m->d_status, 0, sizeof st));
    return fail(m->ctx, TDE_ETIMEOUT, "tde_mesh_check: a bounded device wait of a mesh kernel expired");
  }
  return m->eos ? tde_eos_check(m->eos) : TDE_OK;
}

extern "C" int tde_mesh_inject_wait_expiry(tde_mesh *m, int on) {
  if (!m) return TDE_EINVAL;
  if (on && !m->d_tmaps)
    return fail(m->ctx, TDE_EINVAL, "tde_mesh_inject_wait_expiry: this mesh stages its sweeps without TMA");
  m->inject_tma_skip = on ? 1 : 0;
  if (m->lat_graph) {   // captured launches hold the old flag
    cudaGraphExecDestroy(m->lat_graph);
    m->lat_graph = nullptr;
  }
  return TDE_OK;
}

extern "C" int tde_mesh_set_lat_mode(tde_mesh *m, int mode, int *active) {
  if (!m) return TDE_EINVAL;
  if (mode != TDE_LAT_SEQUENCE && mode != TDE_LAT_PERSISTENT)
    return fail(m->ctx, TDE_EINVAL, "tde_mesh_set_lat_mode: unknown mode");
  if (mode != m->lat_mode) invalidate_graph(m);
  m->lat_mode = mode;
  if (active) *active = mode == TDE_LAT_PERSISTENT && lat_level_eligible(m) ? 1 : 0;
  return TDE_OK;
}

extern "C" int tde_mesh_inject_barrier_drop(tde_mesh *m, int on) {
  if (!m) return TDE_EINVAL;
  m->inject_level_drop = on ? 1 : 0;
  invalidate_graph(m);   // captured launches hold the old flag
  return TDE_OK;
}

// ====================================================== measurement ====

extern "C" int tde_profile(tde_ctx *ctx, int enable) {
  if (!ctx) return TDE_EINVAL;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto &r : ctx->pending) {
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->pending.clear();
  for (int k = 0; k < TDE_K_NKIND; ++k) {
    ctx->launches[k] = 0;
    ctx->ms[k] = 0.0;
  }
  ctx->prof = enable != 0;
  return TDE_OK;
}

extern "C" int tde_profile_read(tde_ctx *ctx, uint64_t *launches, double *ms) {
  if (!ctx) return TDE_EINVAL;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto &r : ctx->pending) {
    float t = 0.f;
    CK(ctx, cudaEventElapsedTime(&t, r.a, r.b));
    ctx->ms[r.kind] += t;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->pending.clear();
  for (int k = 0; k < TDE_K_NKIND; ++k) {
    if (launches) launches[k] = ctx->launches[k];
    if (ms) ms[k] = ctx->ms[k];
  }
  return TDE_OK;
}

namespace tde {
// 8 independent FMA chains per thread; the result is stored so nothing is elided
__global__ void __launch_bounds__(256) k_probe_fp64(double *out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
}  // namespace tde

extern "C" int tde_probe_fp64(tde_ctx *ctx, double *flops) {
  if (!ctx || !flops) return TDE_EINVAL;
  int sms = 0;
  CK(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int grid = sms * 8, iters = 4096;
  double *buf = nullptr;
  CK(ctx, cudaMalloc(&buf, sizeof(double) * grid * 256));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    ProfScope ps(ctx, TDE_K_PROBE);
    cudaEventRecord(e0, ctx->stream);
    k_probe_fp64<<<grid, 256, 0, ctx->stream>>>(buf, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err != cudaSuccess) {
      cudaFree(buf);
      return cuda_fail(ctx, err, "tde_probe_fp64");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  *flops = 2.0 * 8.0 * iters * (double)grid * 256 / (best * 1e-3);
  return TDE_OK;
}

namespace tde {
__global__ void k_math_selftest(const MathTables *mt, long long n, const double *x, double *lg,
                                double *ex) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (lg) lg[i] = fast_log10(mt, x[i]);
    if (ex) ex[i] = fast_exp10(mt, x[i]);
  }
}

__global__ void k_math_probe(int op, long long n, const double *x, const double *y, double *out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = x[i];
    double r;
    switch (op) {
      case TDE_MATH_RCP: r = rcp_nr(a); break;
      case TDE_MATH_SQRT_RATIO: r = sqrt_ratio(a, y[i]); break;
      case TDE_MATH_RCP_SEED: r = rcp_seed(a); break;
      case TDE_MATH_RSQRT: r = rsqrt_nr(a); break;
      case TDE_MATH_INSIDE: r = inside_radius(a, y[i]) ? 1.0 : 0.0; break;
      default: r = rsqrt_seed(a); break;
    }
    out[i] = r;
  }
}

template <int D, int EOSK, int DUAL, int SOLVER>
__global__ void k_riemann_probe(Phys p, long long n, const double *__restrict__ wl,
                                const double *__restrict__ wr, double *F, double *vf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double *a = wl + 8 * i, *b = wr + 8 * i;
    FState L, R;
    L.r = a[0]; R.r = b[0];
#pragma unroll
    for (int q = 0; q < 3; ++q) { L.v[q] = a[1 + q]; R.v[q] = b[1 + q]; }
    L.P = a[4]; R.P = b[4];
    // as the sweeps assemble the states
    if (EOSK == EOS_TABLE) {
      L.ge = a[5]; L.g1 = a[6]; R.ge = b[5]; R.g1 = b[6];
    } else {
      L.ge = L.g1 = R.ge = R.g1 = p.gamma;
    }
    L.A = DUAL ? a[7] : 0.0;
    R.A = DUAL ? b[7] : 0.0;
    double f[6], v;
    if (SOLVER == RIEMANN_HLLE) hlle<D, EOSK, DUAL>(p, L, R, f, v);
    else hllc<D, EOSK, DUAL>(p, L, R, f, v);
#pragma unroll
    for (int q = 0; q < 6; ++q) F[6 * i + q] = f[q];
    vf[i] = v;
  }
}

template <int D, int EOSK, int DUAL>
void riemann_probe_solver(int solver, const Phys &p, long long n, const double *wl, const double *wr,
                          double *F, double *vf, unsigned grid, cudaStream_t s) {
  if (solver == RIEMANN_HLLE) k_riemann_probe<D, EOSK, DUAL, RIEMANN_HLLE><<<grid, 256, 0, s>>>(p, n, wl, wr, F, vf);
  else k_riemann_probe<D, EOSK, DUAL, RIEMANN_HLLC><<<grid, 256, 0, s>>>(p, n, wl, wr, F, vf);
}

template <int D>
void riemann_probe_dir(int solver, int table, int dual, const Phys &p, long long n, const double *wl,
                       const double *wr, double *F, double *vf, unsigned grid, cudaStream_t s) {
  if (table) {
    if (dual) riemann_probe_solver<D, EOS_TABLE, 1>(solver, p, n, wl, wr, F, vf, grid, s);
    else riemann_probe_solver<D, EOS_TABLE, 0>(solver, p, n, wl, wr, F, vf, grid, s);
  } else {
    if (dual) riemann_probe_solver<D, EOS_IDEAL, 1>(solver, p, n, wl, wr, F, vf, grid, s);
    else riemann_probe_solver<D, EOS_IDEAL, 0>(solver, p, n, wl, wr, F, vf, grid, s);
  }
}
}  // namespace tde

extern "C" int tde_math_probe(tde_ctx *c, int op, int64_t n, const double *x, const double *y,
                              double *out) {
  if (!c) return TDE_EINVAL;
  if (op < TDE_MATH_RCP || op > TDE_MATH_INSIDE || n < 0 || (n > 0 && (!x || !out)) ||
      (n > 0 && (op == TDE_MATH_SQRT_RATIO || op == TDE_MATH_INSIDE) && !y))
    return fail(c, TDE_EINVAL, "tde_math_probe: arguments");
  if (n == 0) return TDE_OK;
  ProfScope ps(c, TDE_K_PROBE);
  k_math_probe<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, c->stream>>>(
      op, (long long)n, x, y, out);
  CK(c, cudaGetLastError());
  return TDE_OK;
}

extern "C" int tde_riemann_probe(tde_ctx *c, int solver, int d, int eos_table, int dual, double gamma,
                                 int64_t n, const double *wl, const double *wr, double *F, double *vf) {
  if (!c) return TDE_EINVAL;
  if ((solver != RIEMANN_HLLC && solver != RIEMANN_HLLE) || d < 0 || d > 2 || !(gamma > 1.0) || n < 0 ||
      (n > 0 && (!wl || !wr || !F || !vf)))
    return fail(c, TDE_EINVAL, "tde_riemann_probe: arguments");
  if (n == 0) return TDE_OK;
  Phys p{};
  p.gamma = gamma;
  p.gm1 = gamma - 1.0;
  p.inv_gm1 = 1.0 / (gamma - 1.0);
  p.riemann = solver;
  ProfScope ps(c, TDE_K_PROBE);
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  const int t = eos_table ? 1 : 0, du = dual ? 1 : 0;
  if (d == 0) riemann_probe_dir<0>(solver, t, du, p, (long long)n, wl, wr, F, vf, grid, c->stream);
  else if (d == 1) riemann_probe_dir<1>(solver, t, du, p, (long long)n, wl, wr, F, vf, grid, c->stream);
  else riemann_probe_dir<2>(solver, t, du, p, (long long)n, wl, wr, F, vf, grid, c->stream);
  CK(c, cudaGetLastError());
  return TDE_OK;
}

extern "C" int tde_math_selftest(tde_eos *e, int64_t n, const double *x, double *log10_out,
                                 double *exp10_out) {
  if (!e || n < 0 || (n > 0 && !x)) return TDE_EINVAL;
  if (n == 0) return TDE_OK;
  ProfScope ps(e->ctx, TDE_K_PROBE);
  k_math_selftest<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, e->ctx->stream>>>(
      e->d_mt, (long long)n, x, log10_out, exp10_out);
  CK(e->ctx, cudaGetLastError());
  return TDE_OK;
}
