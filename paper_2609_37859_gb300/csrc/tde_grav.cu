// tde_grav.cu -- self-gravity (Sec. 3.2): a geometric multigrid for
// A_h phi = S_h, A_h = -lap_h (seven-point, anisotropic weights
// w_y = (dx/dy)^2, w_z = (dx/dz)^2), S_h = -4 pi G rho_sg (Eq. selfgrav-poisson),
// on the mesh's uniform grid with periodic boundaries, and the coupling of the
// potential to the hydro sources (the sweeps add the stored phi_sg to the point
// mass's potential in Eqs. lat-grav-momentum and lat-grav-energy).
//
// V-cycle: red-black Gauss-Seidel with over-relaxation, defect and volume-average
// restriction fused in one pass, full-approximation coarse equation, trilinear
// prolongation of the coarse correction, post-smoothing on every level, one
// extra fine sweep per cycle; each direction halved while it has more than one
// cell.  The levels are global arrays (x fastest); the MeshBlock layout is
// gathered into level 0 and the potential scattered back (ghosts included).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "tde_internal.h"

namespace tde {

namespace {

constexpr int GT = 256;

struct Lev {
  int n[3];
  double dx[3];
  double *phi, *src, *tmp;
  // seven-point operator, per level: (A phi)_c = aw . (2 phi_c - phi_{c+a} - phi_{c-a});
  // Gauss-Seidel value = cs src + cw . (phi_{c+a} + phi_{c-a}) (cw = w_a / diag,
  // cs = dx^2 / diag); zero weights in directions with one cell
  double aw[3], cw[3], cs;
};

// 32-bit index arithmetic throughout (levels have < 2^31 cells; 64-bit integer
// division would issue on the FP64 pipe)
__device__ __forceinline__ unsigned wrap_idx(const Lev &L, int i, int j, int k) {
  i = i < 0 ? i + L.n[0] : (i >= L.n[0] ? i - L.n[0] : i);
  j = j < 0 ? j + L.n[1] : (j >= L.n[1] ? j - L.n[1] : j);
  k = k < 0 ? k + L.n[2] : (k >= L.n[2] ? k - L.n[2] : k);
  return ((unsigned)k * L.n[1] + j) * L.n[0] + i;
}

__device__ __forceinline__ void decompose(const Lev &L, unsigned c, int &i, int &j, int &k) {
  const unsigned r = c / (unsigned)L.n[0];
  i = (int)(c - r * L.n[0]);
  k = (int)(r / (unsigned)L.n[1]);
  j = (int)(r - (unsigned)k * L.n[1]);
}

__device__ __forceinline__ double apply_A(const Lev &L, const double *phi, int i, int j, int k) {
  const double c2 = 2.0 * phi[wrap_idx(L, i, j, k)];
  double s = L.aw[0] * (c2 - phi[wrap_idx(L, i + 1, j, k)] - phi[wrap_idx(L, i - 1, j, k)]);
  s = fma(L.aw[1], c2 - phi[wrap_idx(L, i, j + 1, k)] - phi[wrap_idx(L, i, j - 1, k)], s);
  s = fma(L.aw[2], c2 - phi[wrap_idx(L, i, j, k + 1)] - phi[wrap_idx(L, i, j, k - 1)], s);
  return s;
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
  const unsigned n = (unsigned)L.n[0] * L.n[1] * L.n[2];
  double s = 0.0;
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    if (sq) {
      int i, j, k;
      decompose(L, c, i, j, k);
      const double d = L.src[c] - apply_A(L, L.phi, i, j, k);
      s += d * d;
    } else {
      s += L.src[c];
    }
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
  for (unsigned e = blockIdx.x * GT + threadIdx.x; e < nrow * hx; e += gridDim.x * GT) {
    const unsigned row = e / hx;
    const int k = (int)(row / (unsigned)L.n[1]), j = (int)(row - (unsigned)k * L.n[1]);
    int i;
    if (L.n[0] > 1) {
      i = 2 * (int)(e - row * hx) + ((j + k + colour) & 1);
    } else {
      if (((j + k) & 1) != colour) continue;
      i = 0;
    }
    const unsigned c = row * L.n[0] + i;
    double nb = L.cw[0] * (L.phi[wrap_idx(L, i + 1, j, k)] + L.phi[wrap_idx(L, i - 1, j, k)]);
    nb = fma(L.cw[1], L.phi[wrap_idx(L, i, j + 1, k)] + L.phi[wrap_idx(L, i, j - 1, k)], nb);
    nb = fma(L.cw[2], L.phi[wrap_idx(L, i, j, k + 1)] + L.phi[wrap_idx(L, i, j, k - 1)], nb);
    const double gs = fma(L.cs, L.src[c], nb);
    const double p0 = L.phi[c];
    L.phi[c] = fma(omega, gs - p0, p0);
  }
}

// coarse cell: phi_C = R phi_f (also kept in C.tmp), R d_f (defect of the fine
// level averaged over the children) into C.src
__global__ void __launch_bounds__(GT) k_mg_restrict(Lev F, Lev C, double inv) {
  const int r0 = F.n[0] / C.n[0], r1 = F.n[1] / C.n[1], r2 = F.n[2] / C.n[2];
  const unsigned n = (unsigned)C.n[0] * C.n[1] * C.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int I, J, K;
    decompose(C, c, I, J, K);
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
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int I, J, K;
    decompose(C, c, I, J, K);
    C.src[c] += apply_A(C, C.tmp, I, J, K);
  }
}

// the coarse correction phi_C - R phi_f, formed once per coarse cell (into tmp)
__global__ void __launch_bounds__(GT) k_mg_corr(Lev C) {
  const unsigned n = (unsigned)C.n[0] * C.n[1] * C.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) C.tmp[c] = C.phi[c] - C.tmp[c];
}

// fine phi += P e, e = phi_C - R phi_f (in C.tmp), trilinear (cell centred):
// per halved direction 3/4 on the parent, 1/4 on its neighbour towards the fine cell
__global__ void __launch_bounds__(GT) k_mg_prolong(Lev F, Lev C) {
  const unsigned n = (unsigned)F.n[0] * F.n[1] * F.n[2];
  for (unsigned c = blockIdx.x * GT + threadIdx.x; c < n; c += gridDim.x * GT) {
    int f[3];
    decompose(F, c, f[0], f[1], f[2]);
    int p[3], q[3];
    bool h[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      h[a] = F.n[a] != C.n[a];
      p[a] = h[a] ? f[a] >> 1 : f[a];
      q[a] = h[a] ? ((f[a] & 1) ? p[a] + 1 : p[a] - 1) : p[a];
    }
    // the weight of coarse cell (ax, by, cz) is the product over halved directions
    // of 3/4 (parent) or 1/4 (neighbour): w = 3^(number of parents) / 4^(halved)
    const int nh = (int)h[0] + (int)h[1] + (int)h[2];
    const double scale = nh == 3 ? 1.0 / 64.0 : (nh == 2 ? 1.0 / 16.0 : (nh == 1 ? 0.25 : 1.0));
    double s = 0.0;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int by = 0; by < 2; ++by)
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          if ((ax && !h[0]) || (by && !h[1]) || (cz && !h[2])) continue;
          const int np = (h[0] && !ax) + (h[1] && !by) + (h[2] && !cz);
          const double w = np == 3 ? 27.0 : (np == 2 ? 9.0 : (np == 1 ? 3.0 : 1.0));
          s = fma(w, C.tmp[wrap_idx(C, ax ? q[0] : p[0], by ? q[1] : p[1], cz ? q[2] : p[2])], s);
        }
    F.phi[c] = fma(scale, s, F.phi[c]);
  }
}

// the potential into the MeshBlock layout, every padded cell (ghosts by the
// periodic image of their global position)
__global__ void __launch_bounds__(GT) k_mg_scatter(Phys p, const DevBlock *__restrict__ blocks, Lev L,
                                                   double *phi_pad) {
  const int b = blockIdx.y;
  const DevBlock B = blocks[b];
  const int npad = B.p[0] * B.p[1] * B.p[2];
  for (int e = blockIdx.x * GT + threadIdx.x; e < npad; e += gridDim.x * GT) {
    const int i = e % B.p[0], r = e / B.p[0];
    const int j = r % B.p[1], k = r / B.p[1];
    phi_pad[B.off + e] = L.phi[wrap_idx(L, B.i0 + i - p.g[0], B.j0 + j - p.g[1], B.k0 + k - p.g[2])];
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
  double cycle_key[4] = {0, 0, 0, 0};  // npre, npost, omega the graph was captured with
  int nl = 0;
  Lev lev[40];
  double *part = nullptr, *scal = nullptr;   // partial sums; [0] mean, [1] defect
  int npart = 0;
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
  delete g;
}

void gravity_release(tde_mesh *m) {
  grav_free(reinterpret_cast<GravState *>(m->grav));
  m->grav = nullptr;
  cudaFree(m->d_phi_sg);
  m->d_phi_sg = nullptr;
}

static cudaError_t grav_init(tde_mesh *m) {
  if (m->grav) return cudaSuccess;
  GravState *g = new GravState;
  int n[3] = {m->phys.N[0], m->phys.N[1], m->phys.N[2]};
  double h[3] = {m->phys.dx[0], m->phys.dx[1], m->phys.dx[2]};
  cudaError_t err = cudaSuccess;
  for (;;) {
    Lev &L = g->lev[g->nl++];
    for (int a = 0; a < 3; ++a) { L.n[a] = n[a]; L.dx[a] = h[a]; }
    double w[3], wsum = 0.0;
    for (int a = 0; a < 3; ++a) {
      w[a] = n[a] > 1 ? (h[0] / h[a]) * (h[0] / h[a]) : 0.0;
      wsum += w[a];
    }
    const double diag = 2.0 * wsum;
    for (int a = 0; a < 3; ++a) {
      L.aw[a] = w[a] / (h[0] * h[0]);
      L.cw[a] = diag > 0.0 ? w[a] / diag : 0.0;
    }
    L.cs = diag > 0.0 ? h[0] * h[0] / diag : 0.0;
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
  if (err == cudaSuccess) err = cudaMalloc(&g->part, sizeof(double) * g->npart);
  if (err == cudaSuccess) err = cudaMalloc(&g->scal, sizeof(double) * 2);
  if (err == cudaSuccess && !m->d_phi_sg) err = cudaMalloc(&m->d_phi_sg, sizeof(double) * m->ntot);
  if (err == cudaSuccess) err = cudaMemset(m->d_phi_sg, 0, sizeof(double) * m->ntot);
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
  if (l == g->nl - 1) return;   // a single cell: the periodic correction is zero
  const Lev &F = g->lev[l], &C = g->lev[l + 1];
  for (int q = 0; q < gp.npre; ++q) smooth(g, F, gp.omega, s);
  const long long nc = (long long)C.n[0] * C.n[1] * C.n[2];
  const double inv = (double)nc / ((double)F.n[0] * F.n[1] * F.n[2]);   // 1 / children per cell
  k_mg_restrict<<<grid_for(nc), GT, 0, s>>>(F, C, inv);
  k_mg_fas<<<grid_for(nc), GT, 0, s>>>(C);
  vcycle(g, l + 1, gp, s);
  k_mg_corr<<<grid_for(nc), GT, 0, s>>>(C);
  k_mg_prolong<<<grid_for((long long)F.n[0] * F.n[1] * F.n[2]), GT, 0, s>>>(F, C);
  g->launches += 4;
  for (int q = 0; q < gp.npost; ++q) smooth(g, F, gp.omega, s);
}

cudaError_t gravity_solve(tde_mesh *m, const tde_grav_params &gp, int *cycles, double *defect) {
  tde_ctx *c = m->ctx;
  cudaStream_t s = c->stream;
  cudaError_t err = grav_init(m);
  if (err != cudaSuccess) return err;
  GravState *g = reinterpret_cast<GravState *>(m->grav);
  Lev &L0 = g->lev[0];
  const long long n0 = (long long)L0.n[0] * L0.n[1] * L0.n[2];
  {
    ProfScope ps(c, TDE_K_GRAV, false);
    dim3 grid((unsigned)std::min<int64_t>((m->max_interior + GT - 1) / GT, 64), (unsigned)m->nb);
    k_mg_gather<<<grid, GT, 0, s>>>(m->phys, m->d_blocks, m->U, L0, 4.0 * M_PI * gp.G, gp.rho_min);
    if (!gp.warm) cudaMemsetAsync(L0.phi, 0, sizeof(double) * n0, s);
    for (int pass = 0; pass < 2; ++pass) {   // the source's mean, removed in two passes
      reduce(g, L0, 0, g->scal, s);
      k_mg_sub_mean<<<grid_for(n0), GT, 0, s>>>(L0, g->scal);
    }
  }
  int ncyc = 0;
  double d = 0.0;
  {
    ProfScope ps(c, TDE_K_GRAV, false);
    reduce(g, L0, 1, g->scal + 1, s);
  }
  // one cycle (V-cycle, the extra fine sweep, the defect norm) as a CUDA graph:
  // about a hundred small launches on the coarse levels replayed as one
  const double key[4] = {(double)gp.npre, (double)gp.npost, gp.omega, 1.0};
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
  {
    ProfScope ps(c, TDE_K_GRAV, false);
    dim3 grid((unsigned)std::min<int64_t>((m->max_interior + GT - 1) / GT, 64), (unsigned)m->nb);
    k_mg_scatter<<<grid, GT, 0, s>>>(m->phys, m->d_blocks, L0, m->d_phi_sg);
  }
  g->launches += 4;   // gather, scatter and the two mean subtractions (the rest count at launch)
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
