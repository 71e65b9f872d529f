// sx_api.cu -- the extern "C" boundary declared in include/simplexgb.h.
// Host code only marshals arguments, copies inputs and queues kernels; every
// step of the transport path runs in the kernels of sx_setup.cu / sx_step.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "simplexgb.h"
#include "sx_ckpt_io.h"
#include "sx_internal.cuh"

#include <nvtx3/nvToolsExt.h>

// A named NVTX range over a call of the C ABI: profilers (nsys, ncu --nvtx)
// see the library's calls around its kernels; without one attached a range
// costs nothing.
namespace {
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

struct sx_ctx {
  sx_config cfg;
  cudaStream_t stream = nullptr;
  std::vector<double> bins;
  sx::DevGrid g{};
  sx::Layout L{};
  double *bins_dev = nullptr;  // inside the workspace
  void *ws_base = nullptr;     // the caller's workspace of the loaded grid
  size_t ws_used = 0;          // bytes of it the grid uses
  bool loaded = false;
  int64_t step = 0;
  double emitted = 0.0;
  std::vector<int32_t> src_vertex;
  std::vector<double> src_rate;
  std::unordered_map<int32_t, int> src_slot;
  int32_t max_degree = 0;
  bool punit_set = false;  // FP32 photons are stored in units of g.punit photons
  bool has_ghosts = false;  // the grid is a shard of a larger one (vertices flagged SX_FLAG_GHOST)
  bool staging_ok = false;  // the load-time staging (flags, edge vectors) still holds the grid's
  bool profiling = false;
  // dynamic grid update
  bool marked = false;
  int64_t mark_step = -1;
  std::vector<int32_t> removed;
  double carry_abs = 0.0, carry_esc = 0.0, carry_fly = 0.0;  // budget of replaced grids
  bool fresh_update = false;  // no step since the last grid update
  // CUDA graph of kGraphSteps steps (rotation + step kernels), captured on the
  // context's stream for a given dt and source count and replayed by sx_step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0.0;
  int graph_nsrc = -1;
  double graph_punit = 0.0;
  int graph_steps = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  size_t events_used = 0;
  double kernel_ms = 0.0;
  int64_t kernel_launches = 0;
  std::string err;
  ~sx_ctx() {
    if (graph) cudaGraphExecDestroy(graph);
    for (auto &e : events) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  }
};

static thread_local std::string g_create_err;
static constexpr int kGraphSteps = sx::kRotAhead;  // one rotation launch per graph
static_assert(sx::kRotAhead == SX_STEP_BLOCK, "the step block of the header");
static_assert(int(sx::kTransportDct) == int(SX_TRANSPORT_DCT) &&
                  int(sx::kTransportBallistic) == int(SX_TRANSPORT_BALLISTIC) &&
                  int(sx::kTransportCombined) == int(SX_TRANSPORT_COMBINED),
              "transport values of the header");

static int fail(sx_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg; else g_create_err = msg;
  return code;
}

static int cuda_fail(sx_ctx *c, cudaError_t e, const char *what) {
  return fail(c, SX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SX_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// FP32 storage: fix the photon unit at the power of two just above the photons
// the sources emit in one step, so that packets stay near 1 and the scaling
// itself is exact.
static void ensure_punit(sx_ctx *c, double dt) {
  if (c->punit_set) return;
  double tot = 0.0;
  for (double r : c->src_rate) tot += r * dt;
  if (tot > 0.0) {
    int ex = 0;
    std::frexp(tot, &ex);
    c->g.punit = std::ldexp(1.0, ex);
    c->punit_set = true;
  }
}

struct sx_batch {
  int32_t max_grids = 0;
  int32_t device = 0;
  cudaStream_t stream = nullptr;
  sx::RotArgs *d_rot = nullptr;
  sx::StepArgs *d_args = nullptr;
  int64_t *d_prefix = nullptr;
  unsigned long long *d_queue = nullptr;
  std::vector<sx::RotArgs> h_rot;
  std::vector<sx::StepArgs> h_args;
  std::vector<int64_t> h_prefix;
  cudaEvent_t ev = nullptr;       // end of the last queued batch work
  cudaEvent_t ev_copy = nullptr;  // the argument tables of the last call reached the device
  bool copy_pending = false;
  std::string err;
  ~sx_batch() {
    if (ev) cudaEventDestroy(ev);
    if (ev_copy) cudaEventDestroy(ev_copy);
  }
};

// Grids of at least this many tiles (32 vertices each) in a batch step in
// launches of their own.
constexpr int64_t kBatchAloneTiles = 8192;

static size_t batch_bytes(int32_t max_grids) {
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  return up(sizeof(sx::RotArgs) * max_grids) + up(sizeof(sx::StepArgs) * max_grids) +
         up(sizeof(int64_t) * (max_grids + 1)) + up(sizeof(unsigned long long));
}

static int bfail(sx_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg; else g_create_err = msg;
  return code;
}

// Copy a grid to the device workspace and build its tables (used by the load
// and by the dynamic grid update).  Leaves the context's step and sources alone.
static int build_grid(sx_ctx *c, int64_t n, const double *pos, const int64_t *row_ptr,
                      const int32_t *col, const double *nH, const double *volume,
                      const uint8_t *flags, const double *y0, void *d_workspace,
                      int64_t workspace_bytes, sx::DevGrid &g, sx::Layout &L, double **bins_dev) {
  if (n < 1 || !pos || !row_ptr || !nH || !volume || !flags || !d_workspace)
    return fail(c, SX_EINVAL, "n < 1 or a required pointer is NULL");
  if (n >= (int64_t)1 << 31) return fail(c, SX_EINVAL, "n must be < 2^31");
  const int64_t nnz = row_ptr[n];
  if (!sx::row_ptr_nondecreasing(n, row_ptr))
    return fail(c, SX_EINVAL, "row_ptr must start at 0 and must not decrease");
  if (nnz > 0 && !col) return fail(c, SX_EINVAL, "col is NULL");
  if (nnz >= (int64_t)1 << 31) return fail(c, SX_EINVAL, "nnz must be < 2^31");
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
    return fail(c, SX_EINVAL, "workspace must be 256-byte aligned");
  const sx::Layout Lw = sx::make_layout(n, nnz, c->cfg.nbins, c->cfg.precision, c->cfg.transport);
  const int64_t need = (int64_t)(Lw.total + sizeof(double) * 3 * sx::kMaxBins + 256);
  if (workspace_bytes < need)
    return fail(c, SX_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  const cudaStream_t st = c->stream;
  L = Lw;
  g = sx::DevGrid{};
  sx::bind_layout(g, d_workspace, L);
  g.n = n;
  g.nnz = nnz;
  g.nbins = c->cfg.nbins;
  g.nbp = sx::bin_stride_packed(g.nbins);
  g.mw = g.nbins <= 32 ? 1 : (g.nbins <= 64 ? 2 : 4);
  g.precision = c->cfg.precision;
  g.chem_fp32 = c->cfg.precision == SX_FP32_TRANSPORT && c->cfg.chem_fp32 ? 1 : 0;
  g.diffuse = c->cfg.alpha_A > 0.0 ? 1 : 0;
  g.ground = g.diffuse ? (c->cfg.alpha_A - c->cfg.alpha_B) / c->cfg.alpha_A : 0.0;
  g.punit = 1.0;
  g.transport = c->cfg.transport;
  g.tau_switch = c->cfg.tau_switch;
  *bins_dev = reinterpret_cast<double *>(static_cast<char *>(d_workspace) + L.total);
  c->ws_base = d_workspace;
  c->ws_used = L.total + sizeof(double) * 3 * (size_t)c->cfg.nbins;
  char *base = static_cast<char *>(d_workspace);
  // zero the state that must start at zero
  SX_CUDA(c, cudaMemsetAsync(base + L.off_dif, 0, L.off_P0 - L.off_dif, st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_P0, 0, L.off_M0 - L.off_P0, st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_M0, 0, L.off_partials - L.off_M0, st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_partials, 0, L.off_tabs - L.off_partials, st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_diag, 0, sizeof(unsigned long long) * sx::kDiagCount, st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_steps, 0, sizeof(unsigned long long), st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_incoming, 0, sizeof(int), st));
  SX_CUDA(c, cudaMemsetAsync(base + L.off_src, 0, sizeof(double) * sx::kMaxSources, st));
  // inputs
  SX_CUDA(c, cudaMemcpyAsync(g.pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaMemcpyAsync(g.s_row_ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
  if (nnz) SX_CUDA(c, cudaMemcpyAsync(g.s_col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaMemcpyAsync(g.s_nH, nH, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaMemcpyAsync(g.s_vol, volume, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaMemcpyAsync(g.s_flags, flags, n, cudaMemcpyHostToDevice, st));
  if (y0) SX_CUDA(c, cudaMemcpyAsync(g.s_y0, y0, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaMemcpyAsync(*bins_dev, c->bins.data(), sizeof(double) * c->bins.size(),
                             cudaMemcpyHostToDevice, st));
  // tables
  SX_CUDA(c, sx::launch_setup(g, st));
  if (g.stb) {  // ballistic and combined transport: no packets yet, every vertex thin so far
    SX_CUDA(c, cudaMemsetAsync(base + L.off_B0, 0, L.off_stb - L.off_B0, st));
    SX_CUDA(c, sx::launch_ballistic_tables(g, st));
  }
  SX_CUDA(c, sx::launch_rotation(g, *bins_dev, c->cfg.seed, 1, 1, 1.0, st));
  // recombination at case A where the cells re-emit the ground-level photons
  // (diffuse radiation), else at case B (on the spot)
  SX_CUDA(c, sx::launch_kappa_and_consts(g, *bins_dev, c->cfg.sigma,
                                          c->cfg.alpha_A > 0.0 ? c->cfg.alpha_A : c->cfg.alpha_B,
                                          c->cfg.kappa, y0 ? g.s_y0 : nullptr, st));
  unsigned long long diag[sx::kDiagCount];
  SX_CUDA(c, cudaMemcpyAsync(diag, g.diag, sizeof(diag), cudaMemcpyDeviceToHost, st));
  SX_CUDA(c, cudaStreamSynchronize(st));
  const unsigned long long errb = diag[sx::kDiagError];
  c->max_degree = (int32_t)diag[sx::kDiagMaxDeg];
  if (errb) {
    std::string m = "malformed grid:";
    if (errb & sx::kErrColRange) m += " neighbour id out of range;";
    if (errb & sx::kErrSelfLoop) m += " self loop;";
    if (errb & sx::kErrUnsorted) m += " row not sorted strictly ascending;";
    if (errb & sx::kErrAsym) m += " CSR not symmetric;";
    if (errb & sx::kErrRowPtr) m += " row_ptr not monotone;";
    if (errb & sx::kErrDegree) m += " non-sink degree > " + std::to_string(SX_MAX_DEGREE) + ";";
    return fail(c, SX_EINVAL, m);
  }
  SX_CUDA(c, cudaMemsetAsync(g.diag, 0, sizeof(unsigned long long) * sx::kDiagCount, st));
  return SX_OK;
}

// The scale and carries that turn the tiles' sums into the reported budget.
static sx::BudgetScale budget_scale(const sx_ctx *c) {
  sx::BudgetScale sc;
  sc.emitted = c->emitted;
  sc.punit = c->g.punit;
  sc.carry_abs = c->carry_abs;
  sc.carry_esc = c->carry_esc;
  sc.carry_fly = c->carry_fly;
  sc.fly_mode = c->fresh_update ? 1 : (c->step > 0 ? 2 : 0);
  sc.diffuse = c->g.diffuse;
  return sc;
}

// Entry points that handle direction-conserving transport only.
static int dct_only(sx_ctx *c, const char *what) {
  if (c->cfg.transport != SX_TRANSPORT_DCT)
    return fail(c, SX_EINVAL, std::string(what) + " takes direction-conserving transport only");
  return SX_OK;
}

extern "C" {

void sx_config_default(sx_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->nbins = 42;
  cfg->precision = SX_FP32_TRANSPORT;
  cfg->seed = 0;
  cfg->sigma = 6.3e-18;
  cfg->alpha_B = 2.59e-13;
  cfg->kappa = 0.0;
  cfg->chem_frac = 0.5;
  cfg->chem_tol = 1e-5;
  cfg->chem_max_sub = 1000;
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->transport = SX_TRANSPORT_DCT;
  cfg->tau_switch = 1.0;
  cfg->chem_fp32 = 0;
  cfg->alpha_A = 0.0;
}

int sx_create(const sx_config *cfg, const double *bin_dirs, sx_ctx **out) {
  if (!out) return fail(nullptr, SX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, SX_EINVAL, "cfg is NULL");
  if (cfg->nbins < 1 || cfg->nbins > SX_MAX_BINS)
    return fail(nullptr, SX_EINVAL, "nbins must be in 1..128");
  std::vector<double> fib;
  if (!bin_dirs) {  // the Fibonacci lattice
    const int nb = cfg->nbins;
    fib.resize(3 * (size_t)nb);
    const double golden = M_PI * (3.0 - std::sqrt(5.0));
    for (int j = 0; j < nb; ++j) {
      const double z = 1.0 - (2.0 * j + 1.0) / nb;
      const double r = std::sqrt(std::max(0.0, 1.0 - z * z));
      const double phi = j * golden;
      double d[3] = {r * std::cos(phi), r * std::sin(phi), z};
      const double l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      for (int k = 0; k < 3; ++k) fib[3 * (size_t)j + k] = d[k] / l;
    }
    bin_dirs = fib.data();
  }
  if (cfg->precision != SX_FP64 && cfg->precision != SX_FP32_TRANSPORT)
    return fail(nullptr, SX_EINVAL, "precision must be SX_FP64 or SX_FP32_TRANSPORT");
  if (!(cfg->chem_frac > 0.0 && cfg->chem_frac <= 1.0))
    return fail(nullptr, SX_EINVAL, "chem_frac must be in (0, 1]");
  if (!(cfg->chem_tol >= 0.0) || cfg->chem_max_sub < 1)
    return fail(nullptr, SX_EINVAL, "chem_tol must be >= 0 and chem_max_sub >= 1");
  if (!(cfg->sigma >= 0.0) || !(cfg->alpha_B >= 0.0))
    return fail(nullptr, SX_EINVAL, "sigma and alpha_B must be >= 0");
  if (cfg->transport != SX_TRANSPORT_DCT && cfg->transport != SX_TRANSPORT_BALLISTIC &&
      cfg->transport != SX_TRANSPORT_COMBINED)
    return fail(nullptr, SX_EINVAL, "transport must be SX_TRANSPORT_DCT, _BALLISTIC or _COMBINED");
  if (std::isnan(cfg->tau_switch)) return fail(nullptr, SX_EINVAL, "tau_switch is NaN");
  if (cfg->chem_fp32 != 0 && cfg->chem_fp32 != 1) return fail(nullptr, SX_EINVAL, "chem_fp32 must be 0 or 1");
  if (!(cfg->alpha_A == 0.0 || (cfg->alpha_A >= cfg->alpha_B && std::isfinite(cfg->alpha_A))))
    return fail(nullptr, SX_EINVAL, "alpha_A must be 0 (on the spot) or a finite value >= alpha_B");
  for (int b = 0; b < cfg->nbins; ++b) {
    const double *d = bin_dirs + 3 * b;
    const double l2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(std::fabs(l2 - 1.0) < 1e-6)) return fail(nullptr, SX_EINVAL, "bin directions must be unit vectors");
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail(nullptr, SX_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (cfg->device < 0 || cfg->device >= ndev) return fail(nullptr, SX_EINVAL, "device ordinal out of range");
  sx_ctx *c = new sx_ctx();
  c->cfg = *cfg;
  c->stream = static_cast<cudaStream_t>(cfg->stream);
  c->bins.assign(bin_dirs, bin_dirs + 3 * cfg->nbins);
  *out = c;
  return SX_OK;
}

int sx_workspace_bytes(const sx_ctx *ctx, int64_t n, int64_t nnz, int64_t *bytes) {
  if (!ctx || !bytes || n < 1 || nnz < 0) return fail(const_cast<sx_ctx *>(ctx), SX_EINVAL, "bad arguments");
  const sx::Layout L = sx::make_layout(n, nnz, ctx->cfg.nbins, ctx->cfg.precision, ctx->cfg.transport);
  *bytes = (int64_t)(L.total + sizeof(double) * 3 * sx::kMaxBins + 256);
  return SX_OK;
}

int sx_load_grid(sx_ctx *c, int64_t n, const double *pos, const int64_t *row_ptr,
                 const int32_t *col, const double *nH, const double *volume, const uint8_t *flags,
                 const double *y0, void *d_workspace, int64_t workspace_bytes) {
  NvtxRange nvtx_range_("sx_load_grid");
  if (!c) return SX_EINVAL;
  c->loaded = false;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  int rc = build_grid(c, n, pos, row_ptr, col, nH, volume, flags, y0, d_workspace, workspace_bytes,
                      c->g, c->L, &c->bins_dev);
  if (rc) return rc;
  c->g.punit = 1.0;
  c->punit_set = c->cfg.precision == SX_FP64;
  c->step = 0;
  c->emitted = 0.0;
  c->carry_abs = c->carry_esc = c->carry_fly = 0.0;
  c->fresh_update = false;
  c->marked = false;
  c->src_vertex.clear();
  c->src_rate.clear();
  c->src_slot.clear();
  c->g.nsrc = 0;
  c->has_ghosts = false;
  for (int64_t i = 0; i < n; ++i) c->has_ghosts |= (flags[i] & SX_FLAG_GHOST) != 0;
  c->staging_ok = true;
  c->loaded = true;
  return SX_OK;
}

int sx_grid_update_mark(sx_ctx *c, double y_thresh, double min_spacing, int32_t *removed,
                        int64_t *n_removed) {
  NvtxRange nvtx_range_("sx_grid_update_mark");
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "the dynamic grid update")) return rc;
  if (c->cfg.alpha_A > 0.0)
    return fail(c, SX_EINVAL, "the dynamic grid update does not hand over diffuse photons (alpha_A > 0)");
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (c->has_ghosts) return fail(c, SX_EINVAL, "the dynamic grid update takes a whole grid, not a shard");
  if (!removed || !n_removed) return fail(c, SX_EINVAL, "NULL argument");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  sx::DevGrid &g = c->g;
  c->staging_ok = false;
  // load-time scratch regions are free after the load
  uint8_t *cand = g.s_flags;
  uint8_t *rem = reinterpret_cast<uint8_t *>(g.s_y0);
  int64_t *blk = reinterpret_cast<int64_t *>(g.s_nH);
  int64_t *total_d = reinterpret_cast<int64_t *>(g.s_vol);
  int32_t *ids = reinterpret_cast<int32_t *>(g.s_out);
  SX_CUDA(c, sx::launch_mark(g, y_thresh, min_spacing, cand, rem, blk, total_d, ids, c->stream));
  int64_t total = 0;
  SX_CUDA(c, cudaMemcpyAsync(&total, total_d, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  if (total)
    SX_CUDA(c, cudaMemcpyAsync(removed, ids, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, c->stream));
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  *n_removed = total;
  c->removed.assign(removed, removed + total);
  c->marked = true;
  c->mark_step = c->step;
  return SX_OK;
}

int sx_grid_update_apply(sx_ctx *c, int64_t n_new, const double *pos, const int64_t *row_ptr,
                         const int32_t *col, const double *nH, const double *volume,
                         const uint8_t *flags, const int32_t *old_of_new, void *d_workspace,
                         int64_t workspace_bytes) {
  NvtxRange nvtx_range_("sx_grid_update_apply");
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "the dynamic grid update")) return rc;
  if (c->cfg.alpha_A > 0.0)
    return fail(c, SX_EINVAL, "the dynamic grid update does not hand over diffuse photons (alpha_A > 0)");
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (!c->marked || c->mark_step != c->step)
    return fail(c, SX_ESTATE, "sx_grid_update_mark must come right before sx_grid_update_apply");
  if (!old_of_new) return fail(c, SX_EINVAL, "old_of_new is NULL");
  sx::DevGrid &go = c->g;
  if (n_new != go.n - (int64_t)c->removed.size())
    return fail(c, SX_EINVAL, "n_new must be n minus the marked vertices");
  std::vector<int32_t> new_of_old(go.n, -1);
  {
    std::vector<uint8_t> is_rem(go.n, 0);
    for (int32_t r : c->removed) is_rem[r] = 1;
    for (int64_t i = 0; i < n_new; ++i) {
      const int32_t o = old_of_new[i];
      if (o < 0 || o >= go.n || is_rem[o] || new_of_old[o] >= 0)
        return fail(c, SX_EINVAL, "old_of_new must list every surviving vertex once");
      new_of_old[o] = (int32_t)i;
    }
  }
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  const cudaStream_t st = c->stream;
  // photons in flight towards every old vertex, per bin, into the old grid's
  // free buffer; then the removed vertices hand theirs over
  const int last = (int)((c->step + 1) & 1), freeb = last ^ 1;
  const size_t tsz = c->cfg.precision == SX_FP64 ? sizeof(double) : sizeof(float);
  if (c->step > 0) {
    SX_CUDA(c, sx::launch_incoming_bins(go, last, go.P[freeb], st));
  } else {
    SX_CUDA(c, cudaMemsetAsync(go.P[freeb], 0, tsz * go.nbp * go.n, st));
  }
  SX_CUDA(c, sx::launch_hand_over(go, reinterpret_cast<uint8_t *>(go.s_y0),
                                  reinterpret_cast<int32_t *>(go.s_out), go.P[freeb], st));
  // budget so far
  double tmp[3] = {0, 0, 0};
  SX_CUDA(c, sx::launch_budget(go, budget_scale(c), st));
  SX_CUDA(c, cudaMemcpyAsync(tmp, go.budget_dev, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  SX_CUDA(c, cudaStreamSynchronize(st));
  // the new grid
  sx::DevGrid gn{};
  sx::Layout Ln{};
  double *bins_new = nullptr;
  int rc = build_grid(c, n_new, pos, row_ptr, col, nH, volume, flags, nullptr, d_workspace,
                      workspace_bytes, gn, Ln, &bins_new);
  if (rc) return rc;
  gn.punit = go.punit;
  gn.nbp = go.nbp;  // the row stride carries over (the new workspace has room for either)
  const int64_t s = c->step;
  const int prev_new = (int)((s & 1) ^ 1);
  int32_t *d_map = reinterpret_cast<int32_t *>(gn.s_out);
  SX_CUDA(c, cudaMemcpyAsync(d_map, old_of_new, sizeof(int32_t) * n_new, cudaMemcpyHostToDevice, st));
  SX_CUDA(c, sx::launch_carry(c->cfg.precision, n_new, gn.nbp, d_map, go.y, go.P[freeb], gn.y,
                              gn.P[prev_new], st));
  const unsigned long long sd = (unsigned long long)s;
  const int inc = s > 0 ? 1 : 0;
  SX_CUDA(c, cudaMemcpyAsync(gn.steps_done, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaMemcpyAsync(gn.incoming, &inc, sizeof(int), cudaMemcpyHostToDevice, st));
  // sources keep their slots at their new ids (a source is never removed)
  for (size_t k = 0; k < c->src_vertex.size(); ++k) {
    const int32_t nv = new_of_old[c->src_vertex[k]];
    const int32_t slot = (int32_t)k;
    SX_CUDA(c, cudaMemcpyAsync(reinterpret_cast<char *>(gn.vc + nv) + offsetof(sx::VConst, src), &slot,
                               sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SX_CUDA(c, cudaMemcpyAsync(gn.src_rate + k, &c->src_rate[k], sizeof(double), cudaMemcpyHostToDevice, st));
  }
  gn.nsrc = (int)c->src_vertex.size();
  // photons now in flight (the carried field)
  const int nblk = 128;
  double parts[nblk];
  SX_CUDA(c, sx::launch_sum_rows(c->cfg.precision, n_new, gn.nbins, gn.nbp, gn.P[prev_new],
                                 reinterpret_cast<double *>(gn.s_nH), nblk, st));
  SX_CUDA(c, cudaMemcpyAsync(parts, gn.s_nH, sizeof(parts), cudaMemcpyDeviceToHost, st));
  SX_CUDA(c, cudaStreamSynchronize(st));
  double fly = 0.0;
  for (int k = 0; k < nblk; ++k) fly += parts[k];
  std::unordered_map<int32_t, int> slots;
  for (size_t k = 0; k < c->src_vertex.size(); ++k) {
    c->src_vertex[k] = new_of_old[c->src_vertex[k]];
    slots[c->src_vertex[k]] = (int)k;
  }
  c->src_slot.swap(slots);
  c->carry_abs += tmp[0] * go.punit;
  c->carry_esc += tmp[1] * go.punit;
  c->carry_fly = fly * go.punit;
  c->fresh_update = true;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->g = gn;
  c->L = Ln;
  c->bins_dev = bins_new;
  c->marked = false;
  c->removed.clear();
  c->staging_ok = true;  // the new grid's flags and edge vectors
  return SX_OK;
}

int sx_add_source(sx_ctx *c, int32_t vertex, double rate) {
  if (!c) return SX_EINVAL;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (vertex < 0 || vertex >= c->g.n) return fail(c, SX_EINVAL, "source vertex out of range");
  if (!(rate >= 0.0) || !std::isfinite(rate)) return fail(c, SX_EINVAL, "rate must be finite and >= 0");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  auto it = c->src_slot.find(vertex);
  int slot;
  if (it != c->src_slot.end()) {
    slot = it->second;
    c->src_rate[slot] += rate;
  } else {
    if ((int)c->src_vertex.size() >= sx::kMaxSources) return fail(c, SX_EINVAL, "too many sources");
    slot = (int)c->src_vertex.size();
    c->src_vertex.push_back(vertex);
    c->src_rate.push_back(rate);
    c->src_slot[vertex] = slot;
    c->g.nsrc = (int)c->src_vertex.size();
    const int32_t s32 = slot;
    SX_CUDA(c, cudaMemcpyAsync(reinterpret_cast<char *>(c->g.vc + vertex) + offsetof(sx::VConst, src),
                               &s32, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  }
  SX_CUDA(c, cudaMemcpyAsync(c->g.src_rate + slot, &c->src_rate[slot], sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  return SX_OK;
}

}  // extern "C"

// Steps with direct launches, the rotation tables of up to kRotAhead steps
// at a time; with `budgets`, after every step the budget is reduced and copied
// to budgets[k] without waiting.
static int step_direct(sx_ctx *c, double dt, int32_t nsteps, sx_budget *budgets) {
  int32_t k_read = 0;  // budgets[k_read ..] are staged on the device, not yet read back
  auto read_back = [&](int32_t k_end) -> int {
    if (k_end > k_read)
      SX_CUDA(c, cudaMemcpyAsync(budgets + k_read, c->g.bhist, sizeof(sx_budget) * (size_t)(k_end - k_read),
                                 cudaMemcpyDeviceToHost, c->stream));
    k_read = k_end;
    return SX_OK;
  };
  static_assert(sizeof(sx_budget) == 4 * sizeof(double), "a staged budget is four doubles");
  for (int32_t k = 0; k < nsteps;) {
    const int m = std::min<int32_t>(nsteps - k, sx::kRotAhead);
    SX_CUDA(c, sx::launch_rotation(c->g, c->bins_dev, c->cfg.seed, m, 0, dt, c->stream));
    for (int j = 0; j < m; ++j, ++k) {
      if (c->profiling) {
        if (c->events_used == c->events.size()) {
          cudaEvent_t a, b;
          SX_CUDA(c, cudaEventCreate(&a));
          SX_CUDA(c, cudaEventCreate(&b));
          c->events.emplace_back(a, b);
        }
        SX_CUDA(c, cudaEventRecord(c->events[c->events_used].first, c->stream));
      }
      SX_CUDA(c, sx::launch_step(c->g, j, dt, c->cfg.chem_frac, c->cfg.chem_tol, c->cfg.chem_max_sub,
                                 c->stream));
      if (c->profiling) SX_CUDA(c, cudaEventRecord(c->events[c->events_used++].second, c->stream));
      for (size_t s = 0; s < c->src_rate.size(); ++s) c->emitted += c->src_rate[s] * dt;
      c->step++;
      if (budgets) {
        SX_CUDA(c, sx::launch_budget(c->g, budget_scale(c), c->stream, c->g.bhist + 4 * (k - k_read)));
        if (k + 1 - k_read == sx::kBudgetHist) {
          const int rc = read_back(k + 1);
          if (rc) return rc;
        }
      }
    }
  }
  if (budgets) return read_back(nsteps);
  return SX_OK;
}

extern "C" {

int sx_step(sx_ctx *c, double dt, int32_t nsteps) {
  NvtxRange nvtx_range_("sx_step");
  if (!c) return SX_EINVAL;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(c, SX_EINVAL, "dt must be > 0 and nsteps >= 0");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  ensure_punit(c, dt);
  if (nsteps > 0) c->fresh_update = false;
  int32_t k0 = 0;
  if (!c->profiling && c->stream != nullptr && nsteps >= kGraphSteps) {
    // replay a captured block of steps: identical launches, the step index
    // lives on the device
    if (!c->graph || c->graph_dt != dt || c->graph_nsrc != c->g.nsrc || c->graph_punit != c->g.punit) {
      if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
      }
      cudaGraph_t gr = nullptr;
      SX_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = cudaSuccess;
      ce = sx::launch_rotation(c->g, c->bins_dev, c->cfg.seed, kGraphSteps, 0, dt, c->stream);
      for (int k = 0; k < kGraphSteps && ce == cudaSuccess; ++k)
        ce = sx::launch_step(c->g, k, dt, c->cfg.chem_frac, c->cfg.chem_tol, c->cfg.chem_max_sub, c->stream);
      cudaError_t ee = cudaStreamEndCapture(c->stream, &gr);
      if (ce != cudaSuccess) return cuda_fail(c, ce, "graph capture");
      if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture");
      cudaError_t ie = cudaGraphInstantiate(&c->graph, gr, 0);
      cudaGraphDestroy(gr);
      if (ie != cudaSuccess) return cuda_fail(c, ie, "cudaGraphInstantiate");
      c->graph_dt = dt;
      c->graph_nsrc = c->g.nsrc;
      c->graph_punit = c->g.punit;
      c->graph_steps = kGraphSteps;
    }
    for (; k0 + c->graph_steps <= nsteps; k0 += c->graph_steps) {
      SX_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
      for (int k = 0; k < c->graph_steps; ++k)
        for (size_t s = 0; s < c->src_rate.size(); ++s) c->emitted += c->src_rate[s] * dt;
      c->step += c->graph_steps;
    }
  }
  // the rest: the tables of up to kRotAhead steps, then their step launches
  return step_direct(c, dt, nsteps - k0, nullptr);
}

int sx_step_budgets(sx_ctx *c, double dt, int32_t nsteps, sx_budget *budgets) {
  NvtxRange nvtx_range_("sx_step_budgets");
  if (!c) return SX_EINVAL;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(c, SX_EINVAL, "dt must be > 0 and nsteps >= 0");
  if (nsteps > 0 && !budgets) return fail(c, SX_EINVAL, "budgets is NULL");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  ensure_punit(c, dt);
  if (nsteps > 0) c->fresh_update = false;
  return step_direct(c, dt, nsteps, budgets);
}

int sx_sync(sx_ctx *c) {
  NvtxRange nvtx_range_("sx_sync");
  if (!c) return SX_EINVAL;
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  return SX_OK;
}

int sx_read_neutral_fraction(sx_ctx *c, double *y_out) {
  NvtxRange nvtx_range_("sx_read_neutral_fraction");
  if (!c || !y_out) return fail(c, SX_EINVAL, "NULL argument");
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  SX_CUDA(c, cudaMemcpyAsync(y_out, c->g.y, sizeof(double) * c->g.n, cudaMemcpyDeviceToHost, c->stream));
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  return SX_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints: the grid's tables and state as workspace regions, plus the
// host state, in one little-endian file.
// ---------------------------------------------------------------------------
namespace {
constexpr char kCkptMagic[8] = {'S', 'X', 'C', 'K', 'P', 'T', '0', '3'};

struct CkptHeader {
  char magic[8];
  int64_t n, nnz;
  int32_t nbins, precision;
  uint64_t seed;
  double sigma, alpha_B, kappa_cfg, chem_frac, chem_tol;
  int32_t chem_max_sub, nsrc;
  int64_t step;
  double emitted, punit;
  int32_t punit_set, fresh_update;
  double carry_abs, carry_esc, carry_fly;
  int32_t group, max_degree;
  uint64_t bytes_a, bytes_p, bytes_m, bytes_b, bytes_col;
  int32_t chem_fp32, has_ghosts;
  double alpha_A;
  int32_t nbp, reserved;  // the live row stride of the stored photons
};

using sx::File;  // checksummed writes (sx_ckpt_io.h)

// The workspace regions a checkpoint holds, for a grid of this layout whose
// next step is `step`: [offset, bytes] of the tables and y, the photons and
// masks that step reads, the partials/tables/sources/counters, the sender
// ids, kappa.
constexpr int kCkptRegions = 6;
struct CkptRegions {
  size_t off[kCkptRegions], bytes[kCkptRegions];
};
CkptRegions ckpt_regions(const sx::Layout &L, int64_t n, int64_t nnz, int nbins, int nbp,
                         int precision, int64_t step) {
  const int mw = nbins <= 32 ? 1 : (nbins <= 64 ? 2 : 4);
  const size_t tsz = precision == SX_FP64 ? sizeof(double) : sizeof(float);
  const int next = (int)((step & 1) ^ 1);  // the buffers the next step reads
  CkptRegions r;
  r.off[0] = L.off_pos;
  r.bytes[0] = L.off_P0 - L.off_pos;
  r.off[1] = next ? L.off_P1 : L.off_P0;
  r.bytes[1] = tsz * (size_t)nbp * (size_t)n;
  r.off[2] = next ? L.off_M1 : L.off_M0;
  r.bytes[2] = sizeof(uint32_t) * (size_t)mw * (size_t)nnz;
  r.off[3] = L.off_partials;
  r.bytes[3] = L.off_kpart - L.off_partials;
  r.off[4] = L.off_s_col;
  r.bytes[4] = sizeof(int32_t) * (size_t)nnz;
  r.off[5] = L.off_kappa;
  r.bytes[5] = sizeof(double);
  return r;
}
}  // namespace

int sx_checkpoint_info(const char *path, int64_t *n, int64_t *nnz) {
  if (!path || !n || !nnz) return SX_EINVAL;
  File f(path, "rb");
  CkptHeader h;
  if (!f.f || !f.read(&h, sizeof(h)) || std::memcmp(h.magic, kCkptMagic, 8) != 0) return SX_EINVAL;
  *n = h.n;
  *nnz = h.nnz;
  return SX_OK;
}

int sx_checkpoint_verify(const char *path) {
  if (!path) return SX_EINVAL;
  std::string why;
  if (!sx::verify_checkpoint_file(path, kCkptMagic, why)) {
    g_create_err = std::string(path) + ": " + why;
    return SX_EINVAL;
  }
  return SX_OK;
}

int sx_save(sx_ctx *c, const char *path) {
  NvtxRange nvtx_range_("sx_save");
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "a checkpoint")) return rc;
  if (!path) return fail(c, SX_EINVAL, "NULL path");
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (c->marked) return fail(c, SX_ESTATE, "a grid update is pending (mark without apply)");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  const sx::DevGrid &g = c->g;
  const CkptRegions r = ckpt_regions(c->L, g.n, g.nnz, g.nbins, g.nbp, c->cfg.precision, c->step);
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.n = g.n;
  h.nnz = g.nnz;
  h.nbins = c->cfg.nbins;
  h.precision = c->cfg.precision;
  h.seed = c->cfg.seed;
  h.sigma = c->cfg.sigma;
  h.alpha_B = c->cfg.alpha_B;
  h.kappa_cfg = c->cfg.kappa;
  h.chem_frac = c->cfg.chem_frac;
  h.chem_tol = c->cfg.chem_tol;
  h.chem_max_sub = c->cfg.chem_max_sub;
  h.nsrc = (int32_t)c->src_vertex.size();
  h.step = c->step;
  h.emitted = c->emitted;
  h.punit = g.punit;
  h.punit_set = c->punit_set ? 1 : 0;
  h.fresh_update = c->fresh_update ? 1 : 0;
  h.carry_abs = c->carry_abs;
  h.carry_esc = c->carry_esc;
  h.carry_fly = c->carry_fly;
  h.group = g.group;
  h.max_degree = c->max_degree;
  h.bytes_a = r.bytes[0];
  h.bytes_p = r.bytes[1];
  h.bytes_m = r.bytes[2];
  h.bytes_b = r.bytes[3];
  h.bytes_col = r.bytes[4];
  h.chem_fp32 = c->cfg.chem_fp32;
  h.alpha_A = c->cfg.alpha_A;
  h.has_ghosts = c->has_ghosts ? 1 : 0;
  h.nbp = g.nbp;
  // written to path.tmp, synced and renamed over path: a save that fails
  // part-way leaves the previous file at path as it was
  const std::string tmp = std::string(path) + ".tmp";
  std::vector<char> buf;
  File f(tmp.c_str(), "wb");
  if (!f.f) return fail(c, SX_EINVAL, "cannot open " + tmp + " for writing");
  bool ok = f.write(&h, sizeof(h)) && f.write(c->bins.data(), sizeof(double) * c->bins.size()) &&
            f.write(c->src_vertex.data(), sizeof(int32_t) * c->src_vertex.size()) &&
            f.write(c->src_rate.data(), sizeof(double) * c->src_rate.size());
  const char *base = static_cast<const char *>(c->ws_base);
  for (int k = 0; k < kCkptRegions && ok; ++k) {
    buf.resize(r.bytes[k]);
    cudaError_t e = cudaMemcpyAsync(buf.data(), base + r.off[k], r.bytes[k], cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      f.close();
      std::remove(tmp.c_str());
      return fail(c, SX_ECUDA, std::string("cuda: ") + cudaGetErrorString(e));
    }
    ok = f.write(buf.data(), r.bytes[k]);
  }
  ok = ok && sx::write_trailer(f);
  ok = f.close() && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(c, SX_EINVAL, std::string("write to ") + path + " failed");
  }
  return SX_OK;
}

int sx_restore(sx_ctx *c, const char *path, void *d_workspace, int64_t workspace_bytes) {
  NvtxRange nvtx_range_("sx_restore");
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "a checkpoint")) return rc;
  if (!path || !d_workspace) return fail(c, SX_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
    return fail(c, SX_EINVAL, "workspace not 256-byte aligned");
  // One handle for the check and the restore: the whole file is read
  // against its checksum before anything of it is used, then read again from
  // its start.  (A file replaced by a rename in between is not seen: the
  // handle keeps the file it opened.)
  File f(path, "rb");
  {
    std::string why;
    if (!sx::verify_checkpoint_stream(f, kCkptMagic, why))
      return fail(c, SX_EINVAL, std::string(path) + ": " + why);
  }
  CkptHeader h;
  if (fseeko(f.f, 0, SEEK_SET) != 0 || !f.read(&h, sizeof(h)) || std::memcmp(h.magic, kCkptMagic, 8) != 0)
    return fail(c, SX_EINVAL, std::string(path) + " is not a checkpoint");
  if (h.nbins != c->cfg.nbins || h.precision != c->cfg.precision)
    return fail(c, SX_EINVAL, "checkpoint bins or precision differ from the context's");
  // the bounds sx_load_grid applies (the checksum finds damage only: a
  // checkpoint is trusted input)
  if (h.n < 1 || h.n >= ((int64_t)1 << 31) || h.nnz < 0 || h.nnz >= ((int64_t)1 << 31) ||
      h.nsrc < 0 || h.nsrc > sx::kMaxSources || h.step < 0 || (h.group != 0 && h.group != 2 && h.group != 4) ||
      h.max_degree < 0 || h.max_degree > SX_MAX_DEGREE || !(h.punit > 0.0) || (h.chem_fp32 != 0 && h.chem_fp32 != 1) ||
      !(h.alpha_A == 0.0 || (h.alpha_A >= h.alpha_B && std::isfinite(h.alpha_A))) ||
      (h.nbp != sx::bin_stride_packed(h.nbins) && h.nbp != sx::bin_stride_aligned(h.nbins)))
    return fail(c, SX_EINVAL, "corrupt checkpoint header");
  std::vector<double> bins(3 * (size_t)h.nbins);
  std::vector<int32_t> srcv(h.nsrc);
  std::vector<double> srcr(h.nsrc);
  if (!f.read(bins.data(), sizeof(double) * bins.size()) ||
      !f.read(srcv.data(), sizeof(int32_t) * srcv.size()) ||
      !f.read(srcr.data(), sizeof(double) * srcr.size()))
    return fail(c, SX_EINVAL, "truncated checkpoint");
  if (bins != c->bins) return fail(c, SX_EINVAL, "checkpoint bin directions differ from the context's");
  const sx::Layout L = sx::make_layout(h.n, h.nnz, h.nbins, h.precision);
  const size_t need = L.total + sizeof(double) * 3 * sx::kMaxBins + 256;
  if (workspace_bytes < 0 || (size_t)workspace_bytes < need)
    return fail(c, SX_ENOMEM, "workspace too small for the checkpoint's grid");
  const CkptRegions r = ckpt_regions(L, h.n, h.nnz, h.nbins, h.nbp, h.precision, h.step);
  if (r.bytes[0] != h.bytes_a || r.bytes[1] != h.bytes_p || r.bytes[2] != h.bytes_m ||
      r.bytes[3] != h.bytes_b || r.bytes[4] != h.bytes_col)
    return fail(c, SX_EINVAL, "checkpoint written by an incompatible layout");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  const cudaStream_t st = c->stream;
  c->loaded = false;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  char *base = static_cast<char *>(d_workspace);
  // the buffers of the step that is not restored start clear
  SX_CUDA(c, cudaMemsetAsync(base + L.off_P0, 0, L.off_partials - L.off_P0, st));
  std::vector<char> buf;
  for (int k = 0; k < kCkptRegions; ++k) {
    buf.resize(r.bytes[k]);
    if (!f.read(buf.data(), r.bytes[k])) return fail(c, SX_EINVAL, "truncated checkpoint");
    SX_CUDA(c, cudaMemcpyAsync(base + r.off[k], buf.data(), r.bytes[k], cudaMemcpyHostToDevice, st));
    SX_CUDA(c, cudaStreamSynchronize(st));  // buf is reused
  }
  sx::DevGrid g{};
  sx::bind_layout(g, d_workspace, L);
  g.n = h.n;
  g.nnz = h.nnz;
  g.nbins = h.nbins;
  g.nbp = h.nbp;
  g.mw = h.nbins <= 32 ? 1 : (h.nbins <= 64 ? 2 : 4);
  g.precision = h.precision;
  g.chem_fp32 = h.precision == SX_FP32_TRANSPORT && h.chem_fp32 ? 1 : 0;
  g.diffuse = h.alpha_A > 0.0 ? 1 : 0;
  g.ground = g.diffuse ? (h.alpha_A - h.alpha_B) / h.alpha_A : 0.0;
  g.punit = h.punit;
  g.nsrc = h.nsrc;
  g.group = h.group;
  c->bins_dev = reinterpret_cast<double *>(base + L.total);
  SX_CUDA(c, cudaMemcpyAsync(c->bins_dev, c->bins.data(), sizeof(double) * c->bins.size(),
                             cudaMemcpyHostToDevice, st));
  SX_CUDA(c, cudaStreamSynchronize(st));
  c->g = g;
  c->L = L;
  c->ws_base = d_workspace;
  c->ws_used = L.total + sizeof(double) * 3 * (size_t)h.nbins;
  c->cfg.seed = h.seed;
  c->cfg.sigma = h.sigma;
  c->cfg.alpha_B = h.alpha_B;
  c->cfg.kappa = h.kappa_cfg;
  c->cfg.chem_frac = h.chem_frac;
  c->cfg.chem_tol = h.chem_tol;
  c->cfg.chem_max_sub = h.chem_max_sub;
  c->cfg.chem_fp32 = h.chem_fp32;
  c->cfg.alpha_A = h.alpha_A;
  c->has_ghosts = h.has_ghosts != 0;
  c->staging_ok = false;  // the load-time staging is not in a checkpoint
  c->step = h.step;
  c->emitted = h.emitted;
  c->punit_set = h.punit_set != 0;
  c->fresh_update = h.fresh_update != 0;
  c->carry_abs = h.carry_abs;
  c->carry_esc = h.carry_esc;
  c->carry_fly = h.carry_fly;
  c->max_degree = h.max_degree;
  c->marked = false;
  c->removed.clear();
  c->src_vertex = srcv;
  c->src_rate = srcr;
  c->src_slot.clear();
  for (int32_t k = 0; k < h.nsrc; ++k) c->src_slot[srcv[k]] = k;
  c->loaded = true;
  return SX_OK;
}

// ---------------------------------------------------------------------------
// Shards of one grid: kappa's sums and the halo exchange
// ---------------------------------------------------------------------------
int sx_kappa_sums(sx_ctx *c, double *num, double *den) {
  NvtxRange nvtx_range_("sx_kappa_sums");
  if (!c) return SX_EINVAL;
  if (!num || !den) return fail(c, SX_EINVAL, "NULL argument");
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (!c->staging_ok)
    return fail(c, SX_ESTATE, "the load-time tables are gone (after a restore or a grid update mark)");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  SX_CUDA(c, sx::launch_kappa_parts(c->g, c->bins_dev, c->stream));
  std::vector<double> part(2 * (size_t)c->g.nblocks_kappa);
  SX_CUDA(c, cudaMemcpyAsync(part.data(), c->g.kappa_part, sizeof(double) * part.size(),
                             cudaMemcpyDeviceToHost, c->stream));
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  double a = 0.0, b = 0.0;
  for (int64_t k = 0; k < c->g.nblocks_kappa; ++k) {  // ascending blocks
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  *num = a;
  *den = b;
  return SX_OK;
}

int sx_set_photon_unit(sx_ctx *c, double unit) {
  if (!c) return SX_EINVAL;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (c->step != 0) return fail(c, SX_ESTATE, "the photon unit is fixed once a step has run");
  int ex = 0;
  if (!(unit > 0.0) || !std::isfinite(unit) || std::frexp(unit, &ex) != 0.5)
    return fail(c, SX_EINVAL, "the photon unit must be a positive power of two");
  if (c->cfg.precision == SX_FP64) return SX_OK;  // FP64 stores photons as they are
  c->g.punit = unit;
  c->punit_set = true;
  return SX_OK;
}

int sx_halo_bytes(const sx_ctx *c, int64_t n_edges, int64_t n_rows, int64_t *bytes) {
  if (!c || !bytes || n_edges < 0 || n_rows < 0) return fail(const_cast<sx_ctx *>(c), SX_EINVAL, "bad arguments");
  const int nbp = c->loaded ? c->g.nbp : sx::bin_stride_packed(c->cfg.nbins);  // the live row stride
  const int mw = c->cfg.nbins <= 32 ? 1 : (c->cfg.nbins <= 64 ? 2 : 4);
  const size_t tsz = c->cfg.precision == SX_FP64 ? sizeof(double) : sizeof(float);
  *bytes = (int64_t)(sx::halo_rows_offset(n_edges, mw) + (size_t)n_rows * nbp * tsz);
  return SX_OK;
}

static int halo(sx_ctx *c, bool pack, int64_t n_edges, const int32_t *d_edge_idx, int64_t n_rows,
                const int32_t *d_row_idx, void *d_buf) {
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "the halo exchange")) return rc;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (c->step < 1) return fail(c, SX_ESTATE, "no step taken yet: nothing to exchange");
  if (n_edges < 0 || n_rows < 0 || n_edges >= ((int64_t)1 << 31) || n_rows >= ((int64_t)1 << 31))
    return fail(c, SX_EINVAL, "bad counts");
  if ((n_edges && !d_edge_idx) || (n_rows && !d_row_idx) || ((n_edges || n_rows) && !d_buf))
    return fail(c, SX_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(d_buf) % 16 != 0) return fail(c, SX_EINVAL, "buffer not 16-byte aligned");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  // the buffers the last step wrote, which the next step reads
  const int buf = (int)((c->step - 1) & 1);
  SX_CUDA(c, sx::launch_halo(c->g, buf, pack, n_edges, d_edge_idx, n_rows, d_row_idx, d_buf, c->stream));
  return SX_OK;
}

int sx_halo_pack(sx_ctx *c, int64_t n_edges, const int32_t *d_edge_idx, int64_t n_rows,
                 const int32_t *d_row_idx, void *d_buf) {
  NvtxRange nvtx_range_("sx_halo_pack");
  return halo(c, true, n_edges, d_edge_idx, n_rows, d_row_idx, d_buf);
}

int sx_halo_unpack(sx_ctx *c, int64_t n_edges, const int32_t *d_edge_idx, int64_t n_rows,
                   const int32_t *d_row_idx, const void *d_buf) {
  NvtxRange nvtx_range_("sx_halo_unpack");
  return halo(c, false, n_edges, d_edge_idx, n_rows, d_row_idx, const_cast<void *>(d_buf));
}

int sx_read_photons(sx_ctx *c, double *per_vertex, sx_budget *b) {
  NvtxRange nvtx_range_("sx_read_photons");
  if (!c) return SX_EINVAL;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  if (b) {  // the same device arithmetic as the reads of sx_step_budgets
    SX_CUDA(c, sx::launch_budget(c->g, budget_scale(c), c->stream));
    SX_CUDA(c, cudaMemcpyAsync(b, c->g.budget_dev + 4, sizeof(sx_budget), cudaMemcpyDeviceToHost, c->stream));
    SX_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (per_vertex) {
    if (c->fresh_update) {
      const int prev = (int)((c->step & 1) ^ 1);
      SX_CUDA(c, sx::launch_row_totals(c->cfg.precision, c->g.n, c->g.nbins, c->g.nbp, c->g.P[prev],
                                       c->g.s_out, c->stream));
      SX_CUDA(c, cudaMemcpyAsync(per_vertex, c->g.s_out, sizeof(double) * c->g.n, cudaMemcpyDeviceToHost, c->stream));
      SX_CUDA(c, cudaStreamSynchronize(c->stream));
      for (int64_t i = 0; i < c->g.n; ++i) per_vertex[i] *= c->g.punit;
    } else if (c->step == 0) {
      std::memset(per_vertex, 0, sizeof(double) * c->g.n);
    } else {
      SX_CUDA(c, sx::launch_inflight(c->g, c->step, c->stream));
      SX_CUDA(c, cudaMemcpyAsync(per_vertex, c->g.s_out, sizeof(double) * c->g.n, cudaMemcpyDeviceToHost, c->stream));
      SX_CUDA(c, cudaStreamSynchronize(c->stream));
      for (int64_t i = 0; i < c->g.n; ++i) per_vertex[i] *= c->g.punit;
    }
  }
  return SX_OK;
}

static int drain_events(sx_ctx *c) {
  if (!c->events_used) return SX_OK;
  SX_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t k = 0; k < c->events_used; ++k) {
    float ms = 0.f;
    SX_CUDA(c, cudaEventElapsedTime(&ms, c->events[k].first, c->events[k].second));
    c->kernel_ms += ms;
  }
  c->kernel_launches += (int64_t)c->events_used;
  c->events_used = 0;
  return SX_OK;
}

int sx_profile(sx_ctx *c, int enable) {
  if (!c) return SX_EINVAL;
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  int rc = drain_events(c);
  if (rc) return rc;
  c->profiling = enable != 0;
  if (c->profiling) {
    c->kernel_ms = 0.0;
    c->kernel_launches = 0;
  }
  return SX_OK;
}

int sx_set_variant(sx_ctx *c, int32_t variant) {
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "a launch variant")) return rc;
  if (variant != 2 && variant != 4) return fail(c, SX_EINVAL, "variant must be 2 or 4 vertices per warp");
  if (c->g.group != variant && c->graph) {  // a captured graph holds the old kernel
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->g.group = variant;
  return SX_OK;
}

int sx_get_variant(sx_ctx *c, int32_t *variant) {
  if (!c || !variant) return SX_EINVAL;
  *variant = c->g.group == 2 ? 2 : 4;
  return SX_OK;
}

// The stored photons' row stride: the buffer the next step reads is moved to
// the new stride (the other holds nothing the next step reads).
static int set_stride(sx_ctx *c, int stride) {
  if (stride == c->g.nbp) return SX_OK;
  const int live = (int)((c->step & 1) ^ 1);
  SX_CUDA(c, sx::launch_restride(c->g, live, stride, c->stream));
  c->g.nbp = stride;
  if (c->graph) {  // a captured graph holds the old stride
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return SX_OK;
}

int sx_set_bin_stride(sx_ctx *c, int32_t stride) {
  NvtxRange nvtx_range_("sx_set_bin_stride");
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "a launch variant")) return rc;
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (c->marked) return fail(c, SX_ESTATE, "a grid update is pending (mark without apply)");
  const int nb = c->cfg.nbins;
  if (stride != sx::bin_stride_packed(nb) && stride != sx::bin_stride_aligned(nb))
    return fail(c, SX_EINVAL, "stride must be nbins rounded up to 4 or to 8");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  return set_stride(c, stride);
}

int sx_get_bin_stride(sx_ctx *c, int32_t *stride) {
  if (!c || !stride) return SX_EINVAL;
  *stride = c->loaded ? c->g.nbp : sx::bin_stride_packed(c->cfg.nbins);
  return SX_OK;
}

int sx_autotune(sx_ctx *c, double dt, int32_t nsteps, void *scratch, size_t scratch_bytes,
                sx_tune_result *out) {
  NvtxRange nvtx_range_("sx_autotune");
  if (!c) return SX_EINVAL;
  if (int rc = dct_only(c, "the autotuner")) return rc;
  if (!out || !scratch) return fail(c, SX_EINVAL, "NULL argument");
  if (!c->loaded) return fail(c, SX_ESTATE, "no grid loaded");
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 1 || nsteps > 1000)
    return fail(c, SX_EINVAL, "dt must be > 0 and 1 <= nsteps <= 1000");
  if (scratch_bytes < c->ws_used) return fail(c, SX_EINVAL, "scratch smaller than the grid's workspace");
  if (reinterpret_cast<uintptr_t>(scratch) % 256 != 0) return fail(c, SX_EINVAL, "scratch not 256-byte aligned");
  SX_CUDA(c, cudaSetDevice(c->cfg.device));
  int rc = drain_events(c);
  if (rc) return rc;
  ensure_punit(c, dt);
  const cudaStream_t st = c->stream;
  const int32_t before = c->g.group == 2 ? 2 : 4;
  const int32_t stride0 = c->g.nbp;
  // the state: every device buffer of the grid, and the host counters
  SX_CUDA(c, cudaMemcpyAsync(scratch, c->ws_base, c->ws_used, cudaMemcpyDeviceToDevice, st));
  std::memset(out, 0, sizeof(*out));
  // candidates: vertices per warp (4, 2) x row stride (bins rounded up to 4
  // and to 8; one stride when they coincide)
  const int nb = c->cfg.nbins;
  const int32_t strides[2] = {sx::bin_stride_packed(nb), sx::bin_stride_aligned(nb)};
  const int nstrides = strides[0] == strides[1] ? 1 : 2;
  int32_t cand[SX_TUNE_MAX_CANDIDATES], cstride[SX_TUNE_MAX_CANDIDATES];
  int ncand = 0;
  for (int si = 0; si < nstrides; ++si)
    for (int32_t gq : {4, 2}) {
      cand[ncand] = gq;
      cstride[ncand++] = strides[si];
    }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SX_CUDA(c, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  double best = 0.0;
  int32_t pick = before, pick_stride = stride0;
  for (int i = 0; i < ncand && ce == cudaSuccess; ++i) {
    c->g.group = cand[i];
    // the candidate's stride, from the saved layout (stride0)
    if (cstride[i] != stride0) {
      ce = sx::launch_restride(c->g, (int)((c->step & 1) ^ 1), cstride[i], st);
      if (ce != cudaSuccess) break;
    }
    c->g.nbp = cstride[i];
    // one untimed step (first launch of the variant), then the timed ones
    for (int32_t k = 0; k <= nsteps && ce == cudaSuccess; ++k) {
      if (k == 1) ce = cudaEventRecord(e0, st);
      if (ce == cudaSuccess) ce = sx::launch_rotation(c->g, c->bins_dev, c->cfg.seed, 1, 0, dt, st);
      if (ce == cudaSuccess)
        ce = sx::launch_step(c->g, 0, dt, c->cfg.chem_frac, c->cfg.chem_tol, c->cfg.chem_max_sub, st);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess) {
      out->candidates[i] = cand[i];
      out->strides[i] = cstride[i];
      out->ms_per_step[i] = (double)ms / nsteps;
      out->ncandidates = i + 1;
      if (i == 0 || out->ms_per_step[i] < best) {
        best = out->ms_per_step[i];
        pick = cand[i];
        pick_stride = cstride[i];
      }
      ce = cudaMemcpyAsync(c->ws_base, scratch, c->ws_used, cudaMemcpyDeviceToDevice, st);
    }
    c->g.nbp = stride0;  // the restored layout
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->g.group = before;
  c->g.nbp = stride0;
  if (ce != cudaSuccess) {
    // put the state back in any case, then report
    cudaMemcpyAsync(c->ws_base, scratch, c->ws_used, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    return cuda_fail(c, ce, "sx_autotune");
  }
  out->variant = pick;
  out->stride = pick_stride;
  if (int rc = sx_set_variant(c, pick)) return rc;
  return set_stride(c, pick_stride);
}

int sx_get_info(sx_ctx *c, sx_info *info) {
  if (!c || !info) return SX_EINVAL;
  std::memset(info, 0, sizeof(*info));
  if (!c->loaded) return SX_OK;
  int rc = drain_events(c);
  if (rc) return rc;
  info->step_kernel_ms = c->kernel_ms;
  info->step_kernel_launches = c->kernel_launches;
  unsigned long long diag[sx::kDiagCount];
  double kappa = 0.0;
  if (cudaSetDevice(c->cfg.device) != cudaSuccess) return SX_ECUDA;
  if (cudaMemcpyAsync(diag, c->g.diag, sizeof(diag), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(&kappa, c->g.kappa_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return SX_ECUDA;
  info->n = c->g.n;
  info->nnz = c->g.nnz;
  info->step = c->step;
  int64_t wb = 0;
  sx_workspace_bytes(c, c->g.n, c->g.nnz, &wb);
  info->workspace_bytes = wb;
  info->kappa = kappa;
  info->subcycles = (int64_t)diag[sx::kDiagSubcycles];
  info->capped = (int64_t)diag[sx::kDiagCapped];
  info->index_errors = (int64_t)diag[sx::kDiagIndex];
  info->max_degree = c->max_degree;
  info->nsources = (int32_t)c->src_vertex.size();
  return SX_OK;
}

int sx_batch_workspace_bytes(int32_t max_grids, int64_t *bytes) {
  if (max_grids < 1 || !bytes) return bfail(nullptr, SX_EINVAL, "max_grids < 1 or bytes is NULL");
  *bytes = (int64_t)batch_bytes(max_grids);
  return SX_OK;
}

int sx_batch_create(int32_t max_grids, int32_t device, void *stream, void *d_workspace,
                    int64_t workspace_bytes, sx_batch **out) {
  if (!out) return bfail(nullptr, SX_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_grids < 1 || !d_workspace) return bfail(nullptr, SX_EINVAL, "max_grids < 1 or no workspace");
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
    return bfail(nullptr, SX_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < (int64_t)batch_bytes(max_grids)) return bfail(nullptr, SX_ENOMEM, "workspace too small");
  if (cudaSetDevice(device) != cudaSuccess) return bfail(nullptr, SX_ECUDA, "cudaSetDevice failed");
  sx_batch *b = new sx_batch();
  b->max_grids = max_grids;
  b->device = device;
  b->stream = static_cast<cudaStream_t>(stream);
  char *p = static_cast<char *>(d_workspace);
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  b->d_rot = reinterpret_cast<sx::RotArgs *>(p);
  p += up(sizeof(sx::RotArgs) * max_grids);
  b->d_args = reinterpret_cast<sx::StepArgs *>(p);
  p += up(sizeof(sx::StepArgs) * max_grids);
  b->d_prefix = reinterpret_cast<int64_t *>(p);
  p += up(sizeof(int64_t) * (max_grids + 1));
  b->d_queue = reinterpret_cast<unsigned long long *>(p);
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_copy, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return bfail(nullptr, SX_ECUDA, "cudaEventCreate failed");
  }
  *out = b;
  return SX_OK;
}

#define SX_BCUDA(b, call)                                                                    \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return bfail(b, SX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int sx_batch_step(sx_batch *b, sx_ctx *const *ctxs, int32_t n, const double *dt_s, int32_t nsteps) {
  NvtxRange nvtx_range_("sx_batch_step");
  if (!b) return SX_EINVAL;
  if (!ctxs || !dt_s || n < 1 || n > b->max_grids || nsteps < 0)
    return bfail(b, SX_EINVAL, "bad arguments");
  const sx_ctx *c0 = ctxs[0];
  for (int32_t i = 0; i < n; ++i) {
    const sx_ctx *c = ctxs[i];
    if (!c) return bfail(b, SX_EINVAL, "NULL context");
    if (!c->loaded) return bfail(b, SX_ESTATE, "context without grid");
    if (c->cfg.transport != SX_TRANSPORT_DCT)
      return bfail(b, SX_EINVAL, "a batch takes direction-conserving transport only");
    if (c->cfg.nbins != c0->cfg.nbins || c->cfg.precision != c0->cfg.precision ||
        c->cfg.device != b->device)
      return bfail(b, SX_EINVAL, "contexts differ in nbins, precision or device");
    if (!(dt_s[i] > 0.0) || !std::isfinite(dt_s[i])) return bfail(b, SX_EINVAL, "dt must be > 0");
  }
  if (nsteps == 0) return SX_OK;
  SX_BCUDA(b, cudaSetDevice(b->device));
  // the host tables are reused: the previous call's copies must have run
  if (b->copy_pending) SX_BCUDA(b, cudaEventSynchronize(b->ev_copy));
  b->h_rot.resize(n);
  b->h_args.resize(n);
  b->h_prefix.resize(n + 1);
  b->h_prefix[0] = 0;
  // Grids of many waves of tiles step in launches of their own (their
  // arguments in the launch's constant bank, no work queue); the others
  // share the persistent launch.
  std::vector<int32_t> alone;
  int32_t ns = 0;  // grids in the shared launch: h_args[0 .. ns-1]
  const sx_ctx *cs = nullptr;
  for (int32_t i = 0; i < n; ++i) {
    sx_ctx *c = ctxs[i];
    ensure_punit(c, dt_s[i]);
    b->h_rot[i] = sx::make_rot_args(c->g, c->bins_dev, c->cfg.seed, 0, dt_s[i]);
    if (c->g.nblocks >= kBatchAloneTiles) {
      alone.push_back(i);
    } else {
      if (!cs) cs = c;
      b->h_args[ns] = sx::make_step_args(c->g, dt_s[i], c->cfg.chem_frac, c->cfg.chem_tol, c->cfg.chem_max_sub);
      b->h_prefix[ns + 1] = b->h_prefix[ns] + c->g.nblocks;
      ++ns;
    }
    // the batch stream runs after the context's queued work
    SX_BCUDA(b, cudaEventRecord(b->ev, c->stream));
    SX_BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev, 0));
  }
  SX_BCUDA(b, cudaMemcpyAsync(b->d_rot, b->h_rot.data(), sizeof(sx::RotArgs) * n, cudaMemcpyHostToDevice, b->stream));
  if (ns > 0) {
    SX_BCUDA(b, cudaMemcpyAsync(b->d_args, b->h_args.data(), sizeof(sx::StepArgs) * ns, cudaMemcpyHostToDevice, b->stream));
    SX_BCUDA(b, cudaMemcpyAsync(b->d_prefix, b->h_prefix.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, b->stream));
  }
  SX_BCUDA(b, cudaEventRecord(b->ev_copy, b->stream));
  b->copy_pending = true;
  for (int32_t k = 0; k < nsteps;) {  // the tables of up to kRotAhead steps, then their steps
    const int m = std::min<int32_t>(nsteps - k, sx::kRotAhead);
    SX_BCUDA(b, sx::launch_rotation_batch(b->d_rot, n, m, b->stream));
    for (int j = 0; j < m; ++j, ++k) {
      if (ns > 0)
        SX_BCUDA(b, sx::launch_step_batch(cs->cfg.precision, cs->g.group, b->d_args, b->d_prefix, ns,
                                          b->h_prefix[ns], b->d_queue, cs->cfg.nbins, j, b->device,
                                          b->stream));
      for (const int32_t i : alone) {
        sx_ctx *c = ctxs[i];
        SX_BCUDA(b, sx::launch_step(c->g, j, dt_s[i], c->cfg.chem_frac, c->cfg.chem_tol, c->cfg.chem_max_sub,
                                    b->stream));
      }
    }
  }
  SX_BCUDA(b, cudaEventRecord(b->ev, b->stream));
  for (int32_t i = 0; i < n; ++i) {
    sx_ctx *c = ctxs[i];
    c->fresh_update = false;
    for (int32_t k = 0; k < nsteps; ++k)
      for (size_t s = 0; s < c->src_rate.size(); ++s) c->emitted += c->src_rate[s] * dt_s[i];
    c->step += nsteps;
    SX_BCUDA(b, cudaStreamWaitEvent(c->stream, b->ev, 0));
  }
  return SX_OK;
}

void sx_batch_destroy(sx_batch *b) { delete b; }

const char *sx_batch_last_error(const sx_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

void sx_destroy(sx_ctx *c) { delete c; }

const char *sx_last_error(const sx_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
