// tde_mlp.cu -- the learned EOS guess: a 2 -> 64 -> 64 -> 2 SiLU network that maps
// normalised (log10 rho, log10 e) to normalised (log10 T, log10 P).  The paper
// has no learned component; the network only chooses the temperature cell in
// which one FP64 Newton step on the interpolated log10 e column is taken, and
// table bisection stays both the fallback and the judge (Sec. 4.2 runtime map).
//
//  * Training: FP32 forward/backward kernels on BF16-rounded weights (the
//    weights inference uses), gradients reduced per CTA in shared memory, then
//    Adam on FP32 master weights.  Samples are drawn on the device from the
//    table itself with a counter-based generator (SplitMix64).
//  * Inference: per CTA tile of 128 cells, layer 1 and the SiLU in FP32 CUDA
//    cores, the 64 x 64 layer on the 5th-generation tensor cores
//    (tcgen05.mma kind::f16, BF16 operands from shared memory, FP32 accumulator
//    in tensor memory, read back with tcgen05.ld), layer 3 in FP32, then the
//    FP64 Newton step with the bisection fallback.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "tde_internal.h"

namespace tde {

constexpr int H = 64;
constexpr int NPARAM = 2 * H + H + H * H + H + 2 * H + 2;   // 4482
// parameter offsets (same layout as the oracle's)
constexpr int OW1 = 0, OB1 = 2 * H, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + 2 * H;

struct MLPNorm {
  float cr, sr, ce, se, cT, sT, cP, sP;   // x_norm = (x - c) / s
  float isr, ise;                         // 1 / sr, 1 / se
  float idlt;                             // 1 / (log10 T cell width)
};

__device__ __forceinline__ float silu_f(float a) { return a / (1.0f + __expf(-a)); }
// SiLU for inference with one MUFU operation: sigmoid(a) = (1 + tanh(a / 2)) / 2
__device__ __forceinline__ float silu_tanh(float a) {
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(0.5f * a));
  return a * fmaf(0.5f, th, 0.5f);
}
__device__ __forceinline__ float dsilu_f(float a) {
  const float s = 1.0f / (1.0f + __expf(-a));
  return s * (1.0f + a * (1.0f - s));
}

// ---------------------------------------------------------------- SplitMix64
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long ctr) {
  return (double)(splitmix64(seed ^ splitmix64(ctr)) >> 11) * (1.0 / 9007199254740992.0);
}

// training samples: (log rho, log T) uniform over the table -> inputs
// (log rho, log e) and targets (log T, log P), normalised
__global__ void k_mlp_samples(DTable t, MLPNorm nm, long long n, unsigned long long seed, float *x,
                              float *y) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
       s += (long long)gridDim.x * blockDim.x) {
    const double a = u01(seed, 2 * s), c = u01(seed, 2 * s + 1);
    const double xr = a * (t.nr - 1), yt = c * (t.nt - 1);
    int i = (int)floor(xr), j = (int)floor(yt);
    if (i > t.nr - 2) i = t.nr - 2;
    if (j > t.nt - 2) j = t.nt - 2;
    const double w = xr - i, u = yt - j;
    const double lr = t.lr0 + xr / t.inv_dlr;
    const double lT = t.lt0 + yt * t.dlt;
    const double le = bilin(t.le, t.nt, i, w, j, u);
    const double lp = bilin(t.lp, t.nt, i, w, j, u);
    // second input: position of log10 e inside the interpolated column at this density
    const double glo = (1.0 - w) * t.le[(size_t)i * t.nt] + w * t.le[(size_t)(i + 1) * t.nt];
    const double ghi = (1.0 - w) * t.le[(size_t)i * t.nt + t.nt - 1] + w * t.le[(size_t)(i + 1) * t.nt + t.nt - 1];
    x[2 * s] = (float)((lr - nm.cr) / nm.sr);
    x[2 * s + 1] = (float)(((le - glo) / (ghi - glo) - nm.ce) / nm.se);
    y[2 * s] = (float)((lT - nm.cT) / nm.sT);
    y[2 * s + 1] = (float)((lp - nm.cP) / nm.sP);
  }
}

// ------------------------------------------------------------------ training

constexpr int GT = 128;   // samples (threads) per CTA in the gradient kernel

// loss and gradient of L = (1/n) sum_s sum_o (y - target)^2 over samples
// [s0, s0 + count) with the BF16-rounded weights wb; gradient and loss are
// accumulated into g (NPARAM floats) and *loss.
__global__ void __launch_bounds__(GT) k_mlp_grad(const __nv_bfloat16 *__restrict__ wb,
                                                 const float *__restrict__ x,
                                                 const float *__restrict__ tg, long long s0,
                                                 long long count, float inv_n, float *g,
                                                 float *loss) {
  extern __shared__ float sh[];
  float *sw = sh;                       // NPARAM weights (as float)
  float *sh1 = sw + NPARAM;             // [GT][H + 1]
  float *sga2 = sh1 + GT * (H + 1);     // [GT][H + 1]
  float *sh2 = sga2 + GT * (H + 1);     // [GT][H + 1]
  float *sga1 = sh2 + GT * (H + 1);     // [GT][H + 1]
  float *sx = sga1 + GT * (H + 1);      // [GT][2]
  float *sgy = sx + 2 * GT;             // [GT][2]
  const int tid = threadIdx.x;
  for (int q = tid; q < NPARAM; q += GT) sw[q] = __bfloat162float(wb[q]);
  __syncthreads();
  const long long s = s0 + blockIdx.x * (long long)GT + tid;
  const bool live = s < s0 + count;
  float *ra1 = sga1 + tid * (H + 1), *ra2 = sga2 + tid * (H + 1);   // pre-activations, then grads
  float *rh1 = sh1 + tid * (H + 1), *rh2 = sh2 + tid * (H + 1);
  float xi0 = 0.f, xi1 = 0.f, t0 = 0.f, t1 = 0.f;
  if (live) {
    xi0 = x[2 * s]; xi1 = x[2 * s + 1];
    t0 = tg[2 * s]; t1 = tg[2 * s + 1];
  }
  for (int o = 0; o < H; ++o) {
    const float a1 = sw[OW1 + 2 * o] * xi0 + sw[OW1 + 2 * o + 1] * xi1 + sw[OB1 + o];
    ra1[o] = a1;
    rh1[o] = silu_f(a1);
  }
  for (int o = 0; o < H; ++o) {
    float acc = sw[OB2 + o];
#pragma unroll 16
    for (int i = 0; i < H; ++i) acc += sw[OW2 + o * H + i] * rh1[i];
    ra2[o] = acc;
    rh2[o] = silu_f(acc);
  }
  float y0 = sw[OB3], y1 = sw[OB3 + 1];
  for (int i = 0; i < H; ++i) {
    const float h = rh2[i];
    y0 += sw[OW3 + i] * h;
    y1 += sw[OW3 + H + i] * h;
  }
  const float r0 = live ? y0 - t0 : 0.f, r1 = live ? y1 - t1 : 0.f;
  const float gy0 = 2.f * r0 * inv_n, gy1 = 2.f * r1 * inv_n;
  sx[2 * tid] = xi0;
  sx[2 * tid + 1] = xi1;
  sgy[2 * tid] = gy0;
  sgy[2 * tid + 1] = gy1;
  float gh1[H];
#pragma unroll
  for (int i = 0; i < H; ++i) gh1[i] = 0.f;
  for (int o = 0; o < H; ++o) {
    const float gh2 = sw[OW3 + o] * gy0 + sw[OW3 + H + o] * gy1;
    const float ga2 = gh2 * dsilu_f(ra2[o]);
    ra2[o] = ga2;
#pragma unroll
    for (int i = 0; i < H; ++i) gh1[i] += sw[OW2 + o * H + i] * ga2;
  }
#pragma unroll
  for (int o = 0; o < H; ++o) ra1[o] = gh1[o] * dsilu_f(ra1[o]);
  // per-CTA loss
  float l = r0 * r0 + r1 * r1;
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((tid & 31) == 0) atomicAdd(loss, l * inv_n);
  __syncthreads();
  // reductions over the CTA's samples
  for (int q = tid; q < H * H; q += GT) {   // dW2[o][i] = sum_s ga2[s][o] h1[s][i]
    const int o = q / H, i = q % H;
    float acc = 0.f;
    for (int k = 0; k < GT; ++k) acc += sga2[k * (H + 1) + o] * sh1[k * (H + 1) + i];
    atomicAdd(g + OW2 + q, acc);
  }
  if (tid < H) {
    const int o = tid;
    float d1 = 0.f, w0 = 0.f, w1 = 0.f, d2 = 0.f, v0 = 0.f, v1 = 0.f;
    for (int k = 0; k < GT; ++k) {
      const float ga1 = sga1[k * (H + 1) + o];
      d1 += ga1;
      w0 += ga1 * sx[2 * k];
      w1 += ga1 * sx[2 * k + 1];
      d2 += sga2[k * (H + 1) + o];
      const float h2 = sh2[k * (H + 1) + o];
      v0 += sgy[2 * k] * h2;
      v1 += sgy[2 * k + 1] * h2;
    }
    atomicAdd(g + OB1 + o, d1);
    atomicAdd(g + OW1 + 2 * o, w0);
    atomicAdd(g + OW1 + 2 * o + 1, w1);
    atomicAdd(g + OB2 + o, d2);
    atomicAdd(g + OW3 + o, v0);
    atomicAdd(g + OW3 + H + o, v1);
  }
  if (tid == H) {
    float b0 = 0.f, b1 = 0.f;
    for (int k = 0; k < GT; ++k) { b0 += sgy[2 * k]; b1 += sgy[2 * k + 1]; }
    atomicAdd(g + OB3, b0);
    atomicAdd(g + OB3 + 1, b1);
  }
}

__global__ void k_adam(float *w, float *m, float *v, float *g, __nv_bfloat16 *wb, int n, float lr,
                       float b1, float b2, float eps, float bc1, float bc2) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float wq = w[q] - lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
    w[q] = wq;
    wb[q] = __float2bfloat16_rn(wq);
    g[q] = 0.f;
  }
}

__global__ void k_round_bf16(const float *w, __nv_bfloat16 *wb, int n) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    wb[q] = __float2bfloat16_rn(w[q]);
}

// ---------------------------------------------------------------- inference

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle ("interleaved"
// core matrices of 8 rows x 16 bytes), leading-dimension byte offset = distance
// between core matrices along K, stride byte offset = distance between 8-row
// groups, descriptor version 1 (bits 46-47).
__device__ __forceinline__ unsigned long long smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28
constexpr uint32_t IDESC_BF16_M128_N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                                         ((128u >> 4) << 24);

// byte offset of element (row r, k) of a [rows][64] BF16 tile in the core-matrix layout
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

constexpr int IT = 128;   // cells per tile = threads per CTA

// Wait until the mbarrier's phase of the given parity completes, for at most one
// second of the global nanosecond timer (try_wait may suspend the thread for a
// while, so the limit is on time, not on polls); false if it expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar_addr, uint32_t parity) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar_addr), "r"(parity));
    if (done) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
}

struct SurrogateArgs {
  DTable t;
  MLPNorm nm;
  const __nv_bfloat16 *wb;
  long long n;
  const double *rho, *e;
  double *T, *P, *cs2;
  float *yout;        // optional: raw network outputs [n][2] (normalised)
  const float *xin;   // optional: network inputs instead of (rho, e) [n][2]
  Counters *cnt;
  int *status;        // set to 1 if a bounded wait expired
  int skip_mma;       // failure-detection test: issue no MMA, so the wait expires
  float *lTg;         // optional: the guessed log10 T of each cell
  CellMap cm;         // which cells: plain arrays (cm.blocks null) or cells of blocks
  // the fused Newton step (k_eos_surrogate<1>): results of accepted cells, the
  // closure's clamped energy (eu, or null), the queue of cells left for
  // bisection and its length
  double *eu;
  long long *queue;
  unsigned long long *qcount;
};

// Cells of a cell map: block position bp's cell count, and the array index of
// its cell `local` (plain arrays: one "block" of n cells, index = local).
__device__ __forceinline__ long long cm_cells(const CellMap &cm, long long n, int bp) {
  if (!cm.blocks) return n;
  const DevBlock &B = cm.blocks[cm.ids[bp]];
  return cm.padded ? (long long)B.p[0] * B.p[1] * B.p[2] : (long long)B.n[0] * B.n[1] * B.n[2];
}
__device__ __forceinline__ long long cm_flat(const CellMap &cm, int bp, long long local) {
  if (!cm.blocks) return cm.list ? (long long)cm.list[local] : local;
  const DevBlock &B = cm.blocks[cm.ids[bp]];
  if (cm.padded) return B.off + local;
  // 32-bit division only (a block has < 2^31 cells; 64-bit division would
  // take the FP64 pipe)
  const unsigned l = (unsigned)local, nx = (unsigned)B.n[0], ny = (unsigned)B.n[1];
  const unsigned r = l / nx;
  const int i = (int)(l - r * nx), k = (int)(r / ny), j = (int)(r - (unsigned)k * ny);
  return B.off + ((long long)(k + cm.g[2]) * B.p[1] + (j + cm.g[1])) * B.p[0] + (i + cm.g[0]);
}

// Split a tile or chunk index of a cell map into (block position, first cell),
// per = tiles or chunks per block, size = cells per tile or chunk; 32-bit
// division (counts < 2^31), none for plain arrays.
__device__ __forceinline__ void cm_split(const CellMap &cm, long long t, long long per, int size, int &bp,
                                         long long &first) {
  if (!cm.blocks) {
    bp = 0;
    first = t * size;
    return;
  }
  const unsigned q = (unsigned)t / (unsigned)per;
  bp = (int)q;
  first = (long long)((unsigned)t - q * (unsigned)per) * size;
}

// One FP64 Newton step from the guessed log10 T, judged by the table bracket.
// The column g is linear inside a temperature cell, so the step from the
// guess's cell j lands on x = j + s with s the cell solve; if the root is in
// cell j that is the root itself, otherwise x lies in the cell j' the linear
// extension points to, and the root is taken there when j' brackets it.  An
// accepted cell is the one bisection finds (g_j <= y < g_{j+1} is unique) and the
// state is evaluated with the same formulas, so the result is the bisection
// result bit for bit.  Returns false for the cells left to bisection (clamped
// inputs, a step that misses).
__device__ __forceinline__ bool newton_cell(const DTable &t, double rho_c, double e, float lTg, float idlt,
                                            long long c, double *T, double *P, double *cs2, double *eu) {
  const int nt = t.nt;
  int i;
  double w;
  const bool cl = rho_cell(t, rho_c, i, w);
  // the decisions below compare on the integer pipe (dgt0, dle, dlt: the
  // same outcomes as the FP64 comparisons for every non-NaN value)
  const bool pos = dgt0(e);
  if (cl || !pos) return false;
  const double ly = tlog10(t, e);
  const double *__restrict__ ra = t.le + (size_t)i * nt;
  const double *__restrict__ rb = ra + nt;
  const float xg = (lTg - (float)t.lt0) * idlt;
  int j = (int)floorf(fminf(fmaxf(xg, 0.f), (float)(nt - 2)));
  j = min(max(j, 0), nt - 2);
  double g0 = lerp_rn(w, __ldg(ra + j), __ldg(rb + j));
  double g1 = lerp_rn(w, __ldg(ra + j + 1), __ldg(rb + j + 1));
  double sc = cell_solve(ly, g0, g1);
  bool in = dle(g0, ly) && dlt(ly, g1);
  if (!in) {
    const double xn = __dadd_rn(dint(j), sc);   // the Newton result, in cell units
    if (dge0(xn) && dlt(xn, dint(nt - 1))) {
      const int j2 = ifloor_nonneg(xn);
      if (j2 != j) {
        j = j2;
        g0 = lerp_rn(w, __ldg(ra + j), __ldg(rb + j));
        g1 = lerp_rn(w, __ldg(ra + j + 1), __ldg(rb + j + 1));
        in = dle(g0, ly) && dlt(ly, g1);
        if (in) sc = cell_solve(ly, g0, g1);
      }
    }
  }
  // at the coldest node bisection clamps (y <= g_0): leave that to it
  if (!(in && (j > 0 || dlt(g0, ly)))) return false;
  if (P) P[c] = texp10(t, bilin(t.lp, nt, i, w, j, sc));
  if (cs2) cs2[c] = texp10(t, bilin(t.lc, nt, i, w, j, sc));
  if (T) T[c] = texp10(t, cell_log10T(t, j, sc));
  if (eu) eu[c] = 0.0;   // inside the table
  return true;
}

// The learned guess.  NEWTON = 0: the network alone (raw outputs, the guess);
// NEWTON = 1: the guess goes straight into the FP64 Newton step in the same
// thread (newton_cell), accepted cells are written and the rest queued for
// k_eos_fallback (one atomic per tile reserves the tile's queue slots; the
// accepted count is added once per CTA).
template <int NEWTON>
__global__ void __launch_bounds__(IT, 8) k_eos_surrogate(SurrogateArgs a) {
  __shared__ __align__(1024) unsigned char sA[IT * H * 2];   // h1, BF16, core-matrix layout
  __shared__ __align__(1024) unsigned char sB[H * H * 2];    // W2, BF16, core-matrix layout
  __shared__ float sW1[2 * H], sb1[H], sb2[H], sW3[2 * H], sb3[2];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  __shared__ unsigned s_wc[IT / 32];
  __shared__ unsigned long long s_base;
  __shared__ unsigned s_acc;
  unsigned n_acc = 0;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sA_addr = (uint32_t)__cvta_generic_to_shared(sA);
  const uint32_t sB_addr = (uint32_t)__cvta_generic_to_shared(sB);
  const uint32_t mbar_addr = (uint32_t)__cvta_generic_to_shared(&mbar);
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(64));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int q = tid; q < H * H; q += IT) {
    const int o = q / H, i = q % H;
    *reinterpret_cast<__nv_bfloat16 *>(sB + core_off(o, i)) = a.wb[OW2 + q];
  }
  for (int q = tid; q < 2 * H; q += IT) {
    sW1[q] = __bfloat162float(a.wb[OW1 + q]);
    sW3[q] = __bfloat162float(a.wb[OW3 + q]);
  }
  if (tid < H) {
    sb1[tid] = __bfloat162float(a.wb[OB1 + tid]);
    sb2[tid] = __bfloat162float(a.wb[OB2 + tid]);
  }
  if (tid < 2) sb3[tid] = __bfloat162float(a.wb[OB3 + tid]);
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar_addr), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;
  uint32_t phase = 0;
  // tiles of IT cells, tpb per block (a.n = the largest block's cell count)
  const long long tpb = (a.n + IT - 1) / IT;
  const long long ntiles = tpb * (a.cm.blocks ? a.cm.nblk : 1);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int bp;
    long long first;
    cm_split(a.cm, tile, tpb, IT, bp, first);
    const long long ncell = cm_cells(a.cm, a.n, bp);
    if (first >= ncell) continue;   // the whole tile (uniform)
    const long long local = first + tid;
    const bool live = local < ncell;
    const long long c = live ? cm_flat(a.cm, bp, local) : 0;
    // after an expired wait (s_abort, uniform) the network is skipped: the
    // Newton kernel queues the remaining cells for bisection, the plain one stops
    float y0 = 0.f, y1 = 0.f;
    if (!s_abort) {
      // ---- inputs and layer 1, FP32 only: the network needs log10 rho and the
      // position z of log10 e in its column to FP32 accuracy (the FP64 work of
      // the inversion is newton_cell's)
      float x0 = 0.f, x1 = 0.f;
      if (live) {
        if (a.xin) {
          x0 = a.xin[2 * c];
          x1 = a.xin[2 * c + 1];
        } else {
          const DTable &t = a.t;
          const float lr = __log2f((float)a.rho[c]) * 0.30102999566f;
          const float ly = __log2f((float)a.e[c]) * 0.30102999566f;
          const float xr = fminf(fmaxf((lr - (float)t.lr0) * (float)t.inv_dlr, 0.f), (float)(t.nr - 1));
          const int ti = min((int)xr, t.nr - 2);
          const float w32 = xr - (float)ti;
          const float *__restrict__ ra = t.le32 + (size_t)ti * t.nt;
          const float *__restrict__ rb = ra + t.nt;
          const float glo = fmaf(w32, __ldg(rb) - __ldg(ra), __ldg(ra));
          const float ghi = fmaf(w32, __ldg(rb + t.nt - 1) - __ldg(ra + t.nt - 1), __ldg(ra + t.nt - 1));
          x0 = fminf(fmaxf((lr - a.nm.cr) * a.nm.isr, -2.f), 2.f);
          const float z = __fdividef(ly - glo, ghi - glo);
          x1 = (fminf(fmaxf(z, -1.f), 2.f) - a.nm.ce) * a.nm.ise;
        }
      }
#pragma unroll
      for (int k8 = 0; k8 < H / 8; ++k8) {
        __align__(16) __nv_bfloat16 hv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int o = 8 * k8 + u;
          hv[u] = __float2bfloat16_rn(silu_tanh(sW1[2 * o] * x0 + sW1[2 * o + 1] * x1 + sb1[o]));
        }
        *reinterpret_cast<uint4 *>(sA + core_off(tid, 8 * k8)) = *reinterpret_cast<uint4 *>(hv);
      }
      // make the generic-proxy shared stores visible to the tensor core
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      // ---- layer 2 on the tensor core: D[128 x 64] = h1[128 x 64] * W2^T
      if (tid == 0 && !a.skip_mma) {
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int ks = 0; ks < H / 16; ++ks) {
          const unsigned long long ad = smem_desc(sA_addr + ks * 256, 128, 1024);
          const unsigned long long bd = smem_desc(sB_addr + ks * 256, 128, 1024);
          const uint32_t acc = ks > 0 ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tbase),
              "l"(ad), "l"(bd), "r"(IDESC_BF16_M128_N64), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            mbar_addr));
      }
      // bounded wait for the MMAs (one second of the global timer at most)
      if (!mbar_wait_bounded(mbar_addr, phase)) s_abort = 1;
      phase ^= 1u;
      __syncthreads();
      if (!s_abort) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- read the accumulator row of this thread (warp w owns TMEM lanes
        // 32w..32w+31) in two halves of 32 columns, and apply layer 3 (FP32)
        y0 = sb3[0];
        y1 = sb3[1];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          uint32_t r[32];
          const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * hf);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
              "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int o = 32 * hf + q;
            const float h2 = silu_tanh(__uint_as_float(r[q]) + sb2[o]);
            y0 += sW3[o] * h2;
            y1 += sW3[H + o] * h2;
          }
        }
        if (live && a.yout) {
          a.yout[2 * c] = y0;
          a.yout[2 * c + 1] = y1;
        }
        if (live && a.lTg) a.lTg[c] = a.nm.cT + a.nm.sT * y0;
      }
      // every thread has its row in registers: the next tile may reuse sA and TMEM
      asm volatile("tcgen05.fence::before_thread_sync;");
    }
    const bool have = !s_abort;   // uniform: set before the last barrier
    if (!NEWTON && !have) break;
    if (NEWTON) {
      // the FP64 Newton step from this thread's guess; misses are queued
      const bool ok = live ? (have && newton_cell(a.t, a.rho[c], a.e[c], a.nm.cT + a.nm.sT * y0, a.nm.idlt, c,
                                                  a.T, a.P, a.cs2, a.eu))
                           : true;
      n_acc += (live && ok) ? 1u : 0u;
      const int lane = tid & 31;
      const unsigned rm = __ballot_sync(0xffffffffu, !ok);
      if (lane == 0) s_wc[warp] = __popc(rm);
      __syncthreads();
      if (tid == 0) {
        unsigned tot = 0;
        for (int q = 0; q < IT / 32; ++q) {
          const unsigned v = s_wc[q];
          s_wc[q] = tot;   // exclusive prefix over the warps
          tot += v;
        }
        s_base = tot ? atomicAdd(a.qcount, (unsigned long long)tot) : 0ull;
      }
      __syncthreads();
      if (!ok) a.queue[s_base + s_wc[warp] + __popc(rm & ((1u << lane) - 1u))] = c;
    }
    __syncthreads();
  }
  if (NEWTON) {   // accepted cells: one atomic per CTA
    for (int o = 16; o > 0; o >>= 1) n_acc += __shfl_xor_sync(0xffffffffu, n_acc, o);
    if (tid == 0) s_acc = 0;
    __syncthreads();
    if ((tid & 31) == 0) atomicAdd(&s_acc, n_acc);
    __syncthreads();
    if (tid == 0 && a.cnt && s_acc) atomicAdd(&a.cnt->surrogate_accepted, (unsigned long long)s_acc);
  }
  if (s_abort && tid == 0) atomicExch(a.status, 1);
  // wait (bounded) for any MMA still in flight before freeing tensor memory
  if (s_abort) mbar_wait_bounded(mbar_addr, phase ^ 1u);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(64));
}

// Table bisection for the cells the Newton step left (their indices in queue).
// With eu (the hydro closure's buffers) the clamped table energy is returned
// (0 inside the table) and the closure counts clamps; without, they are counted here.
__global__ void __launch_bounds__(256) k_eos_fallback(DTable t, const long long *__restrict__ queue,
                                                      const unsigned long long *__restrict__ qcount,
                                                      const double *__restrict__ rho,
                                                      const double *__restrict__ e, double *T, double *P,
                                                      double *cs2, double *eu, Counters *cnt) {
  const long long nq = (long long)*qcount;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = queue[q];
    double Pv, cv, euv, Tv;
    const bool cl = eos_invert(t, rho[c], e[c], Pv, cv, euv, &Tv);
    if (cl && !eu) count(&cnt->table_clamp);
    if (T) T[c] = Tv;
    if (P) P[c] = Pv;
    if (cs2) cs2[c] = cv;
    if (eu) eu[c] = cl ? euv : 0.0;
  }
}

}  // namespace tde

// ================================================================ host side

#include <random>

using namespace tde;

namespace {

int mlp_fail(tde_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

#define MCK(ctx, call)                                                   \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) {                                             \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(_e);   \
      return TDE_ECUDA;                                                  \
    }                                                                    \
  } while (0)

MLPNorm norm_of(const tde_eos *e) {
  MLPNorm n;
  n.cr = (float)e->norm[0]; n.sr = (float)e->norm[1];
  n.ce = (float)e->norm[2]; n.se = (float)e->norm[3];
  n.cT = (float)e->norm[4]; n.sT = (float)e->norm[5];
  n.cP = (float)e->norm[6]; n.sP = (float)e->norm[7];
  n.isr = (float)(1.0 / e->norm[1]);
  n.ise = (float)(1.0 / e->norm[3]);
  n.idlt = (float)(1.0 / e->tab.dlt);
  return n;
}

int ensure_net_buffers(tde_eos *e) {
  tde_ctx *c = e->ctx;
  if (!e->d_w) {
    MCK(c, cudaMalloc(&e->d_w, sizeof(float) * 4 * NPARAM));
    MCK(c, cudaMemset(e->d_w, 0, sizeof(float) * 4 * NPARAM));
  }
  if (!e->d_wb) MCK(c, cudaMalloc(&e->d_wb, sizeof(__nv_bfloat16) * NPARAM));
  if (!e->d_status) {
    MCK(c, cudaMalloc(&e->d_status, sizeof(int)));
    MCK(c, cudaMemset(e->d_status, 0, sizeof(int)));
  }
  return TDE_OK;
}

int upload_weights(tde_eos *e, const float *w) {
  tde_ctx *c = e->ctx;
  MCK(c, cudaMemcpyAsync(e->d_w, w, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, c->stream));
  MCK(c, cudaMemsetAsync(e->d_w + NPARAM, 0, sizeof(float) * 3 * NPARAM, c->stream));   // m, v, g
  k_round_bf16<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(e->d_w, (__nv_bfloat16 *)e->d_wb, NPARAM);
  MCK(c, cudaGetLastError());
  MCK(c, cudaStreamSynchronize(c->stream));
  e->has_net = true;
  return TDE_OK;
}

size_t grad_smem() { return sizeof(float) * (NPARAM + 4 * GT * (H + 1) + 4 * GT); }

cudaError_t launch_grad(tde_eos *e, const float *x, const float *tg, long long s0, long long count,
                        float inv_n, float *g, float *loss, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
    attr = true;
  }
  const unsigned grid = (unsigned)((count + GT - 1) / GT);
  k_mlp_grad<<<grid, GT, grad_smem(), s>>>((const __nv_bfloat16 *)e->d_wb, x, tg, s0, count, inv_n, g,
                                           loss);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_kernel(tde_eos *e, long long n, const double *rho, const double *en,
                                    double *T, double *P, double *cs2, const float *xin, float *yout,
                                    cudaStream_t s, float *lTg = nullptr, const CellMap *cm = nullptr) {
  SurrogateArgs a;
  a.t = e->tab;
  a.nm = norm_of(e);
  a.wb = (const __nv_bfloat16 *)e->d_wb;
  a.n = n;
  a.rho = rho;
  a.e = en;
  a.T = T;
  a.P = P;
  a.cs2 = cs2;
  a.yout = yout;
  a.xin = xin;
  a.cnt = e->d_cnt;
  a.status = e->d_status;
  a.skip_mma = e->inject_wait_expiry;
  a.lTg = lTg;
  a.cm = cm ? *cm : CellMap{};
  a.eu = nullptr;
  a.queue = nullptr;
  a.qcount = nullptr;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->ctx->device);
  // one wave of resident CTAs: registers (64 x 128 threads) and shared memory
  // (26 KB, largest carveout) admit 8 per SM, and 8 x 64 TMEM columns fill the
  // SM's 512 exactly
  cudaFuncSetAttribute(k_eos_surrogate<0>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  const int per_sm = 8;
  const long long tiles = (n + IT - 1) / IT * (a.cm.blocks ? a.cm.nblk : 1);
  const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)sms * per_sm);
  k_eos_surrogate<0><<<grid, IT, 0, s>>>(a);
  return cudaGetLastError();
}

// the network and the Newton step in one pass (k_eos_surrogate<1>): 8 CTAs per
// SM (64 registers, no spills), 8 x 64 TMEM columns fill the SM's 512
cudaError_t launch_surrogate_newton(tde_eos *e, const CellMap &cm, long long n, const double *rho,
                                    const double *en, double *T, double *P, double *cs2, double *eu,
                                    long long *queue, unsigned long long *qcount, Counters *cnt,
                                    cudaStream_t s) {
  SurrogateArgs a;
  a.t = e->tab;
  a.nm = norm_of(e);
  a.wb = (const __nv_bfloat16 *)e->d_wb;
  a.n = n;
  a.rho = rho;
  a.e = en;
  a.T = T;
  a.P = P;
  a.cs2 = cs2;
  a.yout = nullptr;
  a.xin = nullptr;
  a.cnt = cnt;
  a.status = e->d_status;
  a.skip_mma = e->inject_wait_expiry;
  a.lTg = nullptr;
  a.cm = cm;
  a.eu = eu;
  a.queue = queue;
  a.qcount = qcount;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->ctx->device);
  cudaFuncSetAttribute(k_eos_surrogate<1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  const int per_sm = 8;
  const long long tiles = (n + IT - 1) / IT * (cm.blocks ? cm.nblk : 1);
  const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)sms * per_sm);
  k_eos_surrogate<1><<<grid, IT, 0, s>>>(a);
  return cudaGetLastError();
}

// The learned-guess inversion of the cells of cm (n = largest block's cell
// count, or the array length): guess, FP64 Newton with queueing, bisection of
// the queue.  The same inputs give the bisection results bit for bit.
cudaError_t surrogate_run(tde_eos *e, const CellMap &cm, long long n, const double *rho,
                          const double *en, double *T, double *P, double *cs2, double *eu,
                          float *lTg, long long *queue, unsigned long long *qcount, Counters *cnt,
                          cudaStream_t s) {
  cudaError_t r = cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), s);
  if (r != cudaSuccess) return r;
  (void)lTg;
  r = launch_surrogate_newton(e, cm, n, rho, en, T, P, cs2, eu, queue, qcount, cnt, s);
  if (r != cudaSuccess) return r;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->ctx->device);
  const long long ncell = n * (cm.blocks ? cm.nblk : 1);
  const unsigned gf = (unsigned)std::min<long long>((ncell + 255) / 256, (long long)sms * 8);
  k_eos_fallback<<<gf, 256, 0, s>>>(e->tab, queue, qcount, rho, en, T, P, cs2, eu, cnt);
  return cudaGetLastError();
}

}  // namespace

namespace tde {
cudaError_t launch_eos_surrogate(tde_eos *e, int64_t n, const double *rho, const double *en,
                                 double *T, double *P, double *cs2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (e->queue_cap < n) {
    cudaFree(e->d_queue);
    cudaFree(e->d_guess);
    e->d_queue = nullptr;
    e->d_guess = nullptr;
    e->queue_cap = 0;
    cudaError_t r = cudaMalloc(&e->d_queue, sizeof(long long) * (size_t)n);
    if (r != cudaSuccess) return r;
    e->queue_cap = n;
  }
  if (!e->d_qcount) {
    cudaError_t r = cudaMalloc(&e->d_qcount, sizeof(unsigned long long));
    if (r != cudaSuccess) return r;
  }
  ProfScope ps(e->ctx, TDE_K_EOS);
  e->ctx->launches[TDE_K_EOS] += 1;   // the guess with its Newton step, then the bisection of the misses
  return surrogate_run(e, CellMap{}, n, rho, en, T, P, cs2, nullptr, nullptr, e->d_queue,
                       e->d_qcount, e->d_cnt, s);
}

cudaError_t launch_eos_surrogate_cells(tde_eos *e, const CellMap &cm, int64_t nmax,
                                       const SurrogateBuf &sb, Counters *cnt, cudaStream_t s) {
  if (nmax <= 0 || cm.nblk <= 0) return cudaSuccess;
  return surrogate_run(e, cm, nmax, sb.rho, sb.e, nullptr, sb.P, sb.cs2, sb.eu, nullptr, sb.queue,
                       sb.qcount, cnt, s);
}
}  // namespace tde

extern "C" int tde_eos_surrogate_set_weights(tde_eos *e, const float *w, size_t n) {
  if (!e) return TDE_EINVAL;
  if (!w || n != (size_t)NPARAM) return mlp_fail(e->ctx, TDE_EINVAL, "tde_eos_surrogate_set_weights: need 4482 floats");
  int r = ensure_net_buffers(e);
  if (r) return r;
  return upload_weights(e, w);
}

extern "C" int tde_eos_surrogate_get_weights(tde_eos *e, float *w, size_t n) {
  if (!e) return TDE_EINVAL;
  if (!w || n != (size_t)NPARAM || !e->has_net) return mlp_fail(e->ctx, TDE_EINVAL, "tde_eos_surrogate_get_weights: no weights or size");
  MCK(e->ctx, cudaMemcpyAsync(w, e->d_w, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, e->ctx->stream));
  MCK(e->ctx, cudaStreamSynchronize(e->ctx->stream));
  return TDE_OK;
}

extern "C" int tde_eos_surrogate_reset(tde_eos *e) {
  if (!e) return TDE_EINVAL;
  e->has_net = false;
  return TDE_OK;
}

extern "C" int tde_eos_inject_wait_expiry(tde_eos *e, int on) {
  if (!e) return TDE_EINVAL;
  e->inject_wait_expiry = on ? 1 : 0;
  return TDE_OK;
}

extern "C" int tde_eos_check(tde_eos *e) {
  if (!e) return TDE_EINVAL;
  tde_ctx *c = e->ctx;
  MCK(c, cudaStreamSynchronize(c->stream));
  if (!e->d_status) return TDE_OK;
  int st = 0;
  MCK(c, cudaMemcpy(&st, e->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (!st) return TDE_OK;
  MCK(c, cudaMemset(e->d_status, 0, sizeof(int)));
  return mlp_fail(c, TDE_ETIMEOUT,
                  "learned-guess inference: a bounded wait for the tensor-core results expired (the cells "
                  "took the bisection fallback)");
}

extern "C" int tde_eos_surrogate_norm(const tde_eos *e, double *out8) {
  if (!e || !out8) return TDE_EINVAL;
  memcpy(out8, e->norm, sizeof(e->norm));
  return TDE_OK;
}

extern "C" int tde_eos_surrogate_grad(tde_eos *e, int64_t n, const float *x, const float *target,
                                      float *grad, float *loss) {
  if (!e) return TDE_EINVAL;
  tde_ctx *c = e->ctx;
  if (n <= 0 || !x || !target || !grad || !loss || !e->has_net)
    return mlp_fail(c, TDE_EINVAL, "tde_eos_surrogate_grad: arguments or no weights");
  MCK(c, cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, c->stream));
  MCK(c, cudaMemsetAsync(loss, 0, sizeof(float), c->stream));
  ProfScope ps(c, TDE_K_EOS);
  MCK(c, launch_grad(e, x, target, 0, n, 1.0f / (float)n, grad, loss, c->stream));
  return TDE_OK;
}

extern "C" int tde_eos_surrogate_forward(tde_eos *e, int64_t n, const float *x, float *y) {
  if (!e) return TDE_EINVAL;
  tde_ctx *c = e->ctx;
  if (n <= 0 || !x || !y || !e->has_net) return mlp_fail(c, TDE_EINVAL, "tde_eos_surrogate_forward: arguments or no weights");
  ProfScope ps(c, TDE_K_EOS);
  MCK(c, launch_surrogate_kernel(e, n, nullptr, nullptr, nullptr, nullptr, nullptr, x, y, c->stream));
  return TDE_OK;
}

extern "C" int tde_eos_surrogate_train(tde_eos *e, uint64_t seed, int n_samples, int epochs, int batch,
                                       double lr, tde_train_report *rep) {
  if (!e) return TDE_EINVAL;
  tde_ctx *c = e->ctx;
  if (n_samples < GT || epochs < 1 || batch < GT || batch % GT || !(lr > 0.0))
    return mlp_fail(c, TDE_EINVAL, "tde_eos_surrogate_train: sizes (batch a multiple of 128)");
  int r = ensure_net_buffers(e);
  if (r) return r;
  if (!e->has_net) {   // seeded Glorot-normal initialisation, zero biases
    std::vector<float> w(NPARAM, 0.f);
    std::mt19937_64 rng(seed ^ 0x5eedull);
    auto fill = [&](int off, int fan_out, int fan_in) {
      std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (fan_in + fan_out)));
      for (int q = 0; q < fan_out * fan_in; ++q) w[off + q] = nd(rng);
    };
    fill(OW1, H, 2);
    fill(OW2, H, H);
    fill(OW3, 2, H);
    r = upload_weights(e, w.data());
    if (r) return r;
  }
  float *d_x = nullptr, *d_y = nullptr, *d_loss = nullptr;
  const int nb_per_epoch = n_samples / batch;
  const int nbt = nb_per_epoch * epochs;
  MCK(c, cudaMalloc(&d_x, sizeof(float) * 2 * n_samples));
  MCK(c, cudaMalloc(&d_y, sizeof(float) * 2 * n_samples));
  MCK(c, cudaMalloc(&d_loss, sizeof(float) * nbt));
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaMemsetAsync(d_loss, 0, sizeof(float) * nbt, s);
  k_mlp_samples<<<1024, 256, 0, s>>>(e->tab, norm_of(e), n_samples, seed, d_x, d_y);
  float *w = e->d_w, *m = w + NPARAM, *v = m + NPARAM, *g = v + NPARAM;
  const float b1 = 0.9f, b2 = 0.999f;
  int step = 0;
  cudaError_t err = cudaGetLastError();
  for (int ep = 0; ep < epochs && err == cudaSuccess; ++ep) {
    for (int bi = 0; bi < nb_per_epoch && err == cudaSuccess; ++bi, ++step) {
      err = launch_grad(e, d_x, d_y, (long long)bi * batch, batch, 1.0f / batch, g, d_loss + step, s);
      const double prog = (double)step / (double)nbt;
      const float lrs = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + cos(3.141592653589793 * prog))));
      const float bc1 = 1.f - powf(b1, (float)(step + 1)), bc2 = 1.f - powf(b2, (float)(step + 1));
      k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(w, m, v, g, (__nv_bfloat16 *)e->d_wb, NPARAM, lrs, b1, b2,
                                                   1e-8f, bc1, bc2);
      if (err == cudaSuccess) err = cudaGetLastError();
    }
  }
  cudaEventRecord(e1, s);
  std::vector<float> losses(nbt);
  if (err == cudaSuccess) err = cudaMemcpyAsync(losses.data(), d_loss, sizeof(float) * nbt, cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_x);
  cudaFree(d_y);
  cudaFree(d_loss);
  if (err != cudaSuccess) {
    c->err = std::string("tde_eos_surrogate_train: ") + cudaGetErrorString(err);
    return TDE_ECUDA;
  }
  c->launches[TDE_K_EOS] += 2 * (uint64_t)nbt + 1;
  if (rep) {
    rep->loss_first = losses.front();
    rep->loss_last = losses.back();
    rep->epochs = epochs;
    rep->samples = n_samples;
    rep->batches = nbt;
    rep->ms = ms;
  }
  return TDE_OK;
}
