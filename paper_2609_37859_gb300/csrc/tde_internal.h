// tde_internal.h -- host-side objects of libtde.so and the kernel launchers
// shared between the C-ABI layer (tde_api.cu) and the kernels (tde_hydro.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tde_device.cuh"
#include "../../include/tde.h"

struct tde_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // launch accounting (always) and event timing (when prof is set)
  bool prof = false;
  uint64_t launches[TDE_K_NKIND] = {};
  double ms[TDE_K_NKIND] = {};
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
};

namespace tde {
// fills the tables of fast_log10 / fast_exp10 (host, extended precision)
void fill_math_tables(MathTables *h);

// brackets one kernel launch: counts it and, when profiling, records events
struct ProfScope {
  tde_ctx *c;
  int kind;
  cudaEvent_t a = nullptr;
  // count = false: the caller counts the scope's launches itself
  ProfScope(tde_ctx *ctx, int k, bool count = true) : c(ctx), kind(k) {
    if (count) c->launches[k]++;
    if (c->prof) {
      a = take();
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = take();
      cudaEventRecord(b, c->stream);
      c->pending.push_back({kind, a, b});
    }
  }
  cudaEvent_t take() {
    if (!c->pool.empty()) {
      cudaEvent_t e = c->pool.back();
      c->pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};
}  // namespace tde

struct tde_eos {
  tde_ctx *ctx = nullptr;
  tde::DTable tab{};
  tde::MathTables *d_mt = nullptr;   // tables of the fast log10 / exp10
  double *d_data = nullptr;          // 3 * n_rho * n_T doubles
  tde::Counters *d_cnt = nullptr;
  // learned guess (tde_mlp.cu): normalisation of inputs and outputs
  // (c_rho, s_rho, c_e, s_e, c_T, s_T, c_P, s_P; x_norm = (x - c) / s)
  double norm[8] = {0, 1, 0, 1, 0, 1, 0, 1};
  bool has_net = false;
  float *d_w = nullptr;              // FP32 master weights, then Adam m, v and the gradient
  void *d_wb = nullptr;              // BF16 weights used by training forward and inference
  long long *d_queue = nullptr;      // cells the surrogate's Newton step left for bisection
  float *d_guess = nullptr;          // the network's log10 T guess per cell
  int64_t queue_cap = 0;
  unsigned long long *d_qcount = nullptr;
  int *d_status = nullptr;
  int inject_wait_expiry = 0;        // test hook: inference issues no tensor-core work
};

namespace tde {
// The cells a pass covers: the interior (padded = 0) or all padded cells
// (padded = 1) of the blocks ids[0 .. nblk); blocks == null means plain arrays.
// Refined-mesh ghost cells (tde_ghost_fill): a coarse value is the mean of
// (2^depth)^d cells of block blk starting at padded index base (depth 0: one
// cell); a ghost op writes, at padded index dst, either one coarse value
// (kind < 0: restriction) or a prolongation: cv[0] the parent, cv[1 + 2a] and
// cv[2 + 2a] its neighbours at +a and -a (active directions), bit a of kind set
// when the ghost cell is the parent's upper half along a.
struct AmrCV {
  int32_t base, blk, depth;
};
struct AmrOp {
  int32_t dst, kind;
  AmrCV cv[7];
};

struct CellMap {
  const DevBlock *blocks;
  const int32_t *ids;
  int nblk, padded;
  int g[3];
  const int32_t *list;   // blocks == NULL: the cells' flat indices (NULL: cells 0..n-1)
};
// Buffers of the learned-guess closure, each indexed like the state (ntot):
// table inputs, results (eu = clamped table energy or 0), guess and queue.
struct SurrogateBuf {
  double *rho = nullptr, *e = nullptr, *P = nullptr, *cs2 = nullptr, *eu = nullptr;
  float *lTg = nullptr;
  long long *queue = nullptr;
  unsigned long long *qcount = nullptr;
};
}  // namespace tde

struct tde_mesh {
  tde_ctx *ctx = nullptr;
  tde_eos *eos = nullptr;
  tde::Phys phys{};
  tde_params params{};
  tde_grid_desc grid{};
  int nb = 0;
  int nmax[3] = {0, 0, 0};           // largest interior block edge per direction
  int tile[3] = {0, 0, 0};           // sweep tile shape per direction (kTileShapes index)
  tde::SurrogateBuf sb;              // learned-guess closure buffers (eos_mode SURROGATE)
  double *d_frame_part = nullptr;    // partial sums of the frame acceleration
  size_t frame_part_cap = 0;
  double *d_frame_out = nullptr;     // (A_fr[3], mass)
  void *grav = nullptr;              // multigrid levels (tde_grav.cu)
  double *d_phi_sg = nullptr;        // self-gravity potential, MeshBlock layout
  int grav_on = 0;                   // the hydro sources add d_phi_sg
  int64_t ntot = 0;
  int64_t max_interior = 0;          // largest interior cell count of a block
  int max_ghosts = 0;                // largest ghost count of a block
  std::vector<tde::DevBlock> hblocks;
  std::vector<int64_t> hoff;
  tde::DevBlock *d_blocks = nullptr;
  // TMA tensor maps of the primitives W for the sweeps' staging, one per
  // (tile shape, direction, block) at [(shape * 3 + D) * nb + b]; null when
  // some block's rows are not 16-byte multiples (the sweeps then copy by loop)
  CUtensorMap *d_tmaps = nullptr;
  int *d_status = nullptr;           // 1 after a bounded device wait of a mesh kernel expired
  int inject_tma_skip = 0;           // test hook: the sweeps issue no TMA copy (their waits expire)
  double *d_phic = nullptr;          // potential of each interior cell at the stage time (sweep cache)
  unsigned char *d_excc = nullptr;   // excision flag of each interior cell (sweep cache)
  int32_t *d_ghost = nullptr;        // [n_ghost][2] (dst, src) flat padded indices
  int32_t *d_gstart = nullptr;       // [nb + 1]
  std::vector<int32_t> h_gstart;     // its host copy
  // [nb] end of each block's ghost entries that the sweeps read: the face ghosts
  // (one direction outside the interior), listed first in each block's range;
  // the sweeps never read an edge or corner ghost cell.  On a refined mesh every
  // entry (gend[b] = gstart[b + 1]).
  int32_t *d_gend = nullptr;
  std::vector<int32_t> h_gend;
  int32_t *d_allids = nullptr;       // 0..nb-1
  double *d_W = nullptr;             // primitives, nwv * ntot
  double *d_dU = nullptr;            // accumulated L(U) and div v, (nvar + 1) * ntot
  double *d_scal = nullptr;          // device scalars: [0] t, [1] dt, [2] dt_min
  double *d_dtb = nullptr;           // per-block dt [nb]
  unsigned long long *d_dtbits = nullptr;  // per-block CFL minima (bit patterns) [nb]
  tde::Counters *d_cnt = nullptr;
  double *U = nullptr, *U1 = nullptr;  // caller-owned states
  // neighbour lists (blocks supplying ghost cells) and the owner lattice
  std::vector<int32_t> h_nbr_start, h_nbr;
  int32_t *d_nbr_start = nullptr, *d_nbr = nullptr;
  int32_t *d_gsrcb = nullptr;          // source block of each ghost entry
  int unit[3] = {1, 1, 1}, cn[3] = {1, 1, 1};
  int64_t n_gcopy = 0, n_amr = 0;      // ghost copy entries, refined-mesh ghost ops
  // LAT: per level, the ghost cells whose primitives are converted (not copied)
  int32_t *d_lat_glist = nullptr;
  int32_t *d_lat_gstart = nullptr;        // list offset of each block in factor order [nb + 1]
  std::vector<int32_t> h_lat_glist_off;   // [levels + 1]
  int32_t *d_owner = nullptr;          // owner block per unit cube of the finest level's grid
  int lmax = 0;                        // finest refinement level
  tde::AmrOp *d_amr = nullptr;         // refined-mesh ghost ops, grouped by block
  int32_t *d_amr_start = nullptr;      // [nb + 1]
  int max_amr = 0;                     // most ops of one block
  // localized adaptive time stepping
  bool lat_ready = false;
  int lat_fmax = 1;
  double lat_dt0 = 0.0;
  std::vector<int32_t> h_f;            // factor per block
  std::vector<int32_t> h_sorted;       // block ids by ascending factor
  std::vector<int> h_levels;           // distinct factors, ascending
  std::vector<int> h_level_start;      // segment of each level in h_sorted
  int32_t *d_f = nullptr, *d_f2 = nullptr, *d_sorted = nullptr;
  double *d_Uold = nullptr;            // start-of-step states (LAT)
  double *d_freg = nullptr;            // flux impulse registers
  long long *d_fo = nullptr;           // register offset per block
  long long freg_size = 0;
  double *d_tstart = nullptr;          // per-block step start time
  int *d_flag = nullptr;               // device status word of the factor kernel
  int lat_mode = TDE_LAT_SEQUENCE;     // how a level sub-step is launched
  unsigned *d_lat_bar = nullptr;       // grid barrier words of the persistent level kernel
  // its work items in factor order: prefix sums of the interior and ghost-map
  // chunks (LAT_LEVEL_THREADS cells each) of the sorted blocks, [2][nb + 1]
  int32_t *d_lat_pre = nullptr;
  std::vector<int32_t> h_lat_pre;      // its host copy (the source of the upload)
  int inject_level_drop = 0;           // test hook: its CTA 0 skips the first arrival
  cudaGraphExec_t lat_graph = nullptr;
  tde::BH lat_graph_bh{};
  const double *lat_graph_U = nullptr, *lat_graph_U1 = nullptr;
  cudaStream_t cap_stream = nullptr;
  uint64_t lat_graph_launches = 0;
};

namespace tde {

// time / step-size source of a launch: per-block device array or one device scalar
struct TimeArgs {
  const double *dt;   // dt[b] if dt_pb else dt[0]
  int dt_pb;
  const double *t;    // t[b] if t_pb else t[0]; NULL = 0
  int t_pb;
};

cudaError_t launch_c2p(tde_mesh *m, const double *Uin, int nblk, const int32_t *ids, bool want_dt,
                       const BH &bh, TimeArgs ta);
cudaError_t launch_dt_finalize(tde_mesh *m, double cfl, double *dt_block, double *dt_min);
// every ghost cell of the listed blocks, or (sweep_only) the face ghosts the sweeps read
cudaError_t launch_ghost(tde_mesh *m, double *field, int nf, int nblk, const int32_t *ids,
                         bool sweep_only = false);
cudaError_t launch_sweeps(tde_mesh *m, int stage, const double *U0, const double *Uin,
                          double *Uout, int nblk, const int32_t *ids, const BH &bh, TimeArgs ta,
                          double *freg = nullptr);
cudaError_t launch_c2p_padded(tde_mesh *m, const double *Uin, int nblk, const int32_t *ids);
// primitives of n listed cells (flat indices, device), nothing counted
cudaError_t launch_c2p_list(tde_mesh *m, const double *Uin, const int32_t *list, int n);
size_t sweep_smem_max(const tde_mesh *m);
cudaError_t build_sweep_tmaps(tde_mesh *m);
size_t sweep_smem_for(const tde_mesh *m, int D, int shape);
constexpr int N_SWEEP_SHAPES = 3;
// the largest dynamic shared memory of a sweep tile: 227 KB less a reserve for
// the sweep kernels' static shared memory (a few hundred bytes)
constexpr size_t SWEEP_SMEM_LIMIT = 227 * 1024 - 1024;
cudaError_t autotune_sweeps(tde_mesh *m, const BH &bh, int reps, float ms_out[3][N_SWEEP_SHAPES]);
void invalidate_graph(tde_mesh *m);
// the persistent form of a LAT level sub-step (tde_lat_level.cu): whether the
// mesh's scheme admits it, and one level sub-step (tau, level factor flevel, the
// level's nglist converted ghost cells) as one launch
bool lat_level_eligible(const tde_mesh *m);
constexpr int LAT_BAR_WORDS = 8;   // barrier counter and generation, six sweep tile counters
constexpr int LAT_LEVEL_THREADS = 288;   // CTA width of the persistent level kernel
cudaError_t launch_lat_level(tde_mesh *m, const BH &bh, const int32_t *ids, int n, int flevel, int tau,
                             const int32_t *glist, int nglist);
cudaError_t launch_frame_acceleration(tde_mesh *m, const BH &bh, double rho_min, double *out4);
cudaError_t launch_boost(tde_mesh *m, const double *V, double rho_min);
cudaError_t gravity_solve(tde_mesh *m, const tde_grav_params &gp, int *cycles, double *defect);
cudaError_t gravity_copy_phi(tde_mesh *m, double *dst);
void gravity_release(tde_mesh *m);
// one window of every block with factor 1 and dt0 = the device scalar dt
// (the synchronised step of a refined mesh); advances the mesh time
int lat_step_all_ones(tde_mesh *m, const BH &bh);
// refined-mesh ghost ops of the listed blocks into Udst (nvar fields); f == NULL:
// every source from Udst, else the LAT modes of k_ghost_lat (level flevel, fine
// sub-step tau, stage)
cudaError_t launch_ghost_amr(tde_mesh *m, double *Udst, const double *Ucur, const double *Uold, int nvar,
                             int nblk, const int32_t *ids, const int32_t *f, int flevel, int tau, int stage);
cudaError_t launch_remap(tde_mesh *dst, double *Udst, const tde_mesh *src, const double *Usrc, int mode,
                         double rho_floor, double u_floor);
bool closure_ready(const tde_mesh *m);
cudaError_t launch_excise(tde_mesh *m, double *U, int nblk, const int32_t *ids, const BH &bh,
                          TimeArgs ta);
cudaError_t launch_sync(tde_mesh *m, double *U, int nblk, const int32_t *ids, double eta2);
cudaError_t launch_prim2cons(tde_mesh *m, const double *W, double *U);
cudaError_t launch_advance_time(tde_mesh *m);
cudaError_t launch_set_dt(tde_mesh *m, double dt);
cudaError_t launch_eos_invert(tde_eos *e, int64_t n, const double *rho, const double *en,
                              double *T, double *P, double *cs2, cudaStream_t s, bool plain = false);
cudaError_t launch_eos_surrogate(tde_eos *e, int64_t n, const double *rho, const double *en,
                                 double *T, double *P, double *cs2, cudaStream_t s);
cudaError_t launch_eos_surrogate_cells(tde_eos *e, const CellMap &cm, int64_t nmax,
                                       const SurrogateBuf &sb, Counters *cnt, cudaStream_t s);
cudaError_t launch_eos_eval(tde_eos *e, int64_t n, const double *rho, const double *T, double *P,
                            double *en, double *cs2, cudaStream_t s);

}  // namespace tde
