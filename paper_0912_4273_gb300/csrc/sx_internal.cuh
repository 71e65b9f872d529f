// sx_internal.cuh -- device data layout and shared device helpers of the
// SimpleX2 DCT library (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sx {

constexpr int kQ = 127;            // quantisation of unit vectors (int8)
constexpr int kMaxBins = 128;
constexpr int kMaxDeg = 64;        // largest non-sink degree the step kernel stages
// transports (the values of SX_TRANSPORT_*)
enum Transport { kTransportDct = 0, kTransportBallistic = 1, kTransportCombined = 2 };
constexpr int kBudgetBlocks = 256;  // most first-level CTAs of the budget sum
constexpr int kBudgetHist = 256;    // per-step budgets staged on the device before one read-back
constexpr int kTile = 32;          // vertices per CTA in the step kernel (one chemistry warp)
constexpr int kMaxSources = 4096;
// vertex flags: a sink absorbs everything into "escaped"; a ghost is a copy of
// a vertex that another shard of the grid steps (the halo exchange fills in
// what it sends), so it is neither stepped nor counted here
constexpr int kFlagSink = 1, kFlagGhost = 2;
constexpr uint32_t kRotTag = 0x53583252u;  // Philox counter word 3 of the rotation draws
constexpr int kRotMaxAttempts = 64;
// Step tables are made kRotAhead steps at a time (one rotation launch for up
// to kRotAhead step launches); the ring holds them, then the unrotated table.
constexpr int kRotAhead = 16;
constexpr int kTabUnrotated = kRotAhead;
constexpr int kTabCount = kRotAhead + 1;

// One directed Delaunay edge i -> col, stored in i's CSR row (16 bytes).
struct __align__(16) Edge {
  int32_t col;   // target vertex
  int32_t twin;  // index of the reverse edge col -> i in col's row
  char4 q;       // rint(127 * unit vector); w = 0
  uchar4 st;     // most-straightforward slots of this edge (x, y, z), count in w
};

// Per-vertex constants (32 bytes).
struct __align__(16) VConst {
  double invA;     // 1 / (hydrogen atoms n_H V); 0 for an empty cell
  double tau_max;  // optical depth of the neutral cell, n_H sigma kappa <L>
  double R0;       // alpha_B n_H
  int32_t flags;   // bit 0 sink
  int32_t src;     // source slot or -1
};

// Written by the rotation kernel for every step, read by every CTA of that
// step.
struct StepTables {
  float4 qb[kMaxBins];            // quantised rotated bins (x, y, z), as exact floats
  uint32_t qbq[kMaxBins];         // the same as signed bytes (x, y, z, 0), for byte dot products
  unsigned char fwd[kMaxBins];    // closest bin of this step's orientation for every bin of
                                  //   the previous one (identity when nothing is remapped)
  long long step;                 // the step these tables are for
  int32_t attempts;
  int32_t remap;                  // 0: step 0, no previous orientation
  int32_t incoming;               // 1: the stored photons of the previous buffer are this
                                  //    step's incoming photons (after a grid update)
};

// Arguments of the rotation kernel for one grid.  The step index lives on the
// device (*steps_done), so that launches of successive blocks of steps are
// identical and can be captured in a CUDA graph.
struct RotArgs {
  const double *bins;              // nbins x 3, unrotated
  uint64_t seed;
  unsigned long long *steps_done;  // read, then advanced by the steps made (unless unrotated)
  StepTables *tab;                 // the tables of the first step; the next ones follow
  int nbins;
  int unrotated;                   // 1: identity orientation (kappa), counter untouched
  int nsrc;
  const double *src_rate;
  double dt;
  double inv_punit;
  double *share;
  float *share_f;
  int *incoming;                   // one-shot flag handed to the step tables, then cleared
};

// Arguments of the step kernel for one grid (the batched kernel takes an array).
struct StepArgs {
  int64_t n;
  int nbins, nbp;
  double dt, inv_dt;
  double punit;      // photons per stored unit (a power of two; 1 in FP64 mode)
  double fc, tol;
  int max_sub;
  int chem_fp32;     // FP32 transport: 1 = subcycle rates in FP32, 0 = FP64 subcycles
  const int32_t *row_ptr;
  const Edge *edges;
  const VConst *vc;
  double *y;
  const int32_t *col;  // sender of every in-edge (the CSR neighbour array)
  void *P[2];        // stored photons, ping-pong by step parity
  uint32_t *M[2];    // per-edge bin masks, ping-pong by step parity
  const StepTables *tab;
  const double *src_share;
  const float *src_share_f;
  double *partials;
  unsigned long long *diag;
  // ballistic and combined transport (unused in direction-conserving transport)
  void *B[2];              // edge packets at the receivers' in-edges, ping-pong by step parity
  uint8_t *mode[2];        // 1 where the vertex sent ballistically, ping-pong by step parity
  const uint32_t *stb;     // ballistic straight set of every in-edge
  const uint16_t *bpos;    // per out-slot: start (low byte) and length of its in-edge list
  const uint8_t *binv;     // the in-edge lists, 3 bytes per edge of a row
  const double *src_rate;  // photons/s of each source slot
  double src_scale;        // dt / punit: a source's photons of the step in stored units
  int transport;
  double tau_switch;
  // diffuse recombination radiation (Sect. 2.2.1, 4.5)
  int diffuse;             // 1: the cells re-emit their ground-level recombination photons
  double ground;           // (alpha_A - alpha_B) / alpha_A: photons per recombination
  double *dif;             // n: photons (stored units) each vertex made in the last step
};

enum Diag { kDiagSubcycles = 0, kDiagCapped = 1, kDiagError = 2, kDiagMaxDeg = 3, kDiagIndex = 4,
            kDiagCount = 8 };

// Debug builds (-DSX_DEBUG) check the data-dependent indices of the step
// kernels: an index out of range is counted in diag[kDiagIndex] and its
// access skipped (never a trap).  Release builds do not evaluate the check.
#ifdef SX_DEBUG
__device__ __forceinline__ bool sx_index_ok(bool ok, unsigned long long *diag) {
  if (!ok) atomicAdd(&diag[kDiagIndex], 1ull);
  return ok;
}
#define SX_INDEX_OK(cond, diag) ::sx::sx_index_ok((cond), (diag))
#else
#define SX_INDEX_OK(cond, diag) true
#endif

// Error bits reported by the load kernels.
enum : unsigned long long {
  kErrColRange = 1ull, kErrSelfLoop = 2ull, kErrUnsorted = 4ull, kErrAsym = 8ull,
  kErrRowPtr = 16ull, kErrDegree = 32ull
};

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011)
// ----------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// rint(127 u) clamped to [-127, 127]; u is the IEEE result of the caller's ops.
__device__ __forceinline__ int quantise(double u) {
  double r = rint(__dmul_rn(127.0, u));
  r = fmin(fmax(r, -127.0), 127.0);
  return (int)r;
}

// ----------------------------------------------------------------------------
// Float-float accumulation: hi + lo carries ~48 bits with FP32 arithmetic only
// (Knuth two-sum).  Used for per-vertex and per-block photon sums in FP32 mode.
// ----------------------------------------------------------------------------
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, float b) {
  const float s = __fadd_rn(a.hi, b);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return FF{s, __fadd_rn(a.lo, err)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF r = ff_add(a, b.hi);
  r.lo = __fadd_rn(r.lo, b.lo);
  return r;
}
__device__ __forceinline__ FF ff_shfl_down(FF a, int d) {
  return FF{__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ FF ff_warp_sum(FF a) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) a = ff_add(a, ff_shfl_down(a, d));
  return a;  // lane 0
}
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }
// a * b for b >= 0, as float-float (the product of hi exactly by FMA)
__device__ __forceinline__ FF ff_mul(FF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return FF{p, __fmaf_rn(a.lo, b, e)};
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  return v;  // lane 0
}

// ----------------------------------------------------------------------------
// Asynchronous copies global -> shared (sm_80 and later): issued by a thread,
// completed by the same thread's wait; other lanes see the data after a
// warp barrier.  Addresses aligned to the copy size.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ----------------------------------------------------------------------------
// Host-side launch wrappers (defined in the .cu files)
// ----------------------------------------------------------------------------
struct DevGrid {
  int64_t n, nnz;
  int nbins, nbp, mw;   // bins, bins padded to 4, mask words per edge (1, 2 or 4)
  int precision;        // 0 FP64, 1 FP32 transport
  int chem_fp32;        // FP32 transport: subcycle rates in FP32 (1) or FP64 subcycles (0)
  double punit;         // photons per stored unit (power of two; stored = photons / punit)
  double *pos;          // n*3
  int32_t *row_ptr;     // n+1
  Edge *edges;          // nnz
  VConst *vc;           // n
  double *mean_len;     // n
  double *y;            // n
  double *dif;          // n: diffuse recombination photons made in the last step, stored units
  int diffuse;          // 1: diffuse recombination radiation on
  double ground;        // (alpha_A - alpha_B) / alpha_A
  void *P[2];           // n*nbp photons (T), ping-pong
  uint32_t *M[2];       // nnz*mw masks, ping-pong
  double *partials;     // nblocks*4: absorbed, escaped (acc), in flight (last), diffuse emitted (acc)
  int64_t nblocks;      // tiles of kTile vertices
  int group;            // step kernel variant: vertices per warp (2 or 4; 0 = 4)
  StepTables *tabs;     // [kTabCount]: the next steps' tables, then the unrotated one (kappa)
  unsigned long long *steps_done;  // device step counter (advanced by the rotation kernel)
  int *incoming;        // set by a grid update: the next step takes P[prev] as incoming photons
  double *src_rate;     // kMaxSources
  double *src_share;    // kMaxSources: photons per bin per step of each source, stored units
  float *src_share_f;   // the same in FP32
  int nsrc;
  unsigned long long *diag;  // kDiagCount
  double *kappa_part;   // nblocks_kappa*2
  int64_t nblocks_kappa;
  double *kappa_dev;    // 1
  double *budget_dev;   // 8: the sums, then the reported budget (k_budget)
  double *bsum;         // kBudgetBlocks*4: the first level of the budget sums
  double *bhist;        // kBudgetHist*4: reported budgets of recent steps, read back in one copy
  // load-time scratch
  int64_t *s_row_ptr;
  int32_t *s_col;       // nnz neighbour ids as loaded; kept: the step kernel reads the senders here
  double *s_nH, *s_vol, *s_y0;
  uint8_t *s_flags;
  float4 *s_ev;         // nnz: edge vector (x, y, z) and length (w), FP32
  double *s_out;        // n doubles for readouts
  // ballistic and combined transport (null in direction-conserving transport)
  int transport;        // Transport
  double tau_switch;    // combined: ballistic where y tau_max >= tau_switch
  void *B[2];           // nnz edge packets (T) at the receivers' in-edges, ping-pong
  uint8_t *mode[2];     // n: 1 where the vertex sent ballistically, ping-pong
  uint32_t *stb;        // nnz: ballistic straight set of each in-edge (3 slot bytes, count)
  uint16_t *bpos;       // nnz: per out-slot, where its in-edge list starts (low byte) and its length
  uint8_t *binv;        // 3 nnz: the in-edges whose set holds each out-slot, ascending
};

// Row strides (elements) of the stored photons: the bins rounded up to 4
// ("packed") or to 8 ("aligned": rows of 32 bytes in FP32, 64 in FP64).  A
// grid's workspace has room for the aligned stride; the live one is
// DevGrid::nbp, one of the two (a launch variant the autotuner picks).
__host__ __device__ inline int bin_stride_packed(int nbins) { return (nbins + 3) / 4 * 4; }
__host__ __device__ inline int bin_stride_aligned(int nbins) { return (nbins + 7) / 8 * 8; }

struct Layout {
  size_t off_pos, off_row_ptr, off_edges, off_vc, off_mean_len, off_y, off_dif, off_P0, off_P1, off_M0,
      off_M1, off_partials, off_tabs, off_src, off_share, off_share_f, off_steps, off_incoming, off_diag, off_kpart, off_kappa, off_budget, off_bsum, off_bhist,
      off_s_row_ptr, off_s_col, off_s_nH, off_s_vol, off_s_y0, off_s_flags, off_s_ev, off_s_out,
      off_B0, off_B1, off_mode0, off_mode1, off_stb, off_bpos, off_binv, total;
  int64_t nblocks, nblocks_kappa;
};

Layout make_layout(int64_t n, int64_t nnz, int nbins, int precision, int transport = 0);
void bind_layout(DevGrid &g, void *base, const Layout &L);

// Host check of a row_ptr in host memory (n + 1 entries): it starts at 0 and
// never decreases, so every row lies inside [0, row_ptr[n]).  The setup
// kernels index col and the edge tables by it before their own checks are
// read back, so it runs before any of them.
inline bool row_ptr_nondecreasing(int64_t n, const int64_t *row_ptr) {
  if (row_ptr[0] != 0) return false;
  for (int64_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return false;
  return true;
}

cudaError_t launch_setup(DevGrid &g, cudaStream_t st);
cudaError_t launch_kappa_and_consts(DevGrid &g, const double *bins_dev, double sigma,
                                    double alpha_B, double kappa_cfg, const double *y0_dev,
                                    cudaStream_t st);
// Tables of the next `count` (1..kRotAhead) steps into tabs[0..count-1], or
// the unrotated table (count 1).
cudaError_t launch_rotation(DevGrid &g, const double *bins_dev, uint64_t seed, int count,
                            int unrotated, double dt, cudaStream_t st);
// One step with the tables in tabs[slot].
cudaError_t launch_step(DevGrid &g, int slot, double dt, double chem_frac, double chem_tol,
                        int chem_max_sub, cudaStream_t st);
RotArgs make_rot_args(DevGrid &g, const double *bins_dev, uint64_t seed, int unrotated, double dt);
StepArgs make_step_args(DevGrid &g, double dt, double chem_frac, double chem_tol, int chem_max_sub);
// Batched: one rotation CTA per grid (tables of `count` steps), then one
// persistent launch per step over the tiles of all grids (work queue), with
// the tables in slot `slot` of each grid.  All grids share nbins and precision.
cudaError_t launch_rotation_batch(const RotArgs *d_rot, int ngrids, int count, cudaStream_t st);
// One step of ballistic transport alone (sx_ballistic.cu): ntiles CTAs of
// kTile vertices; precision 0 = FP64.
cudaError_t launch_step_ballistic(const StepArgs &a, int64_t ntiles, int precision, cudaStream_t st);
cudaError_t launch_step_batch(int precision, int group, const StepArgs *d_args, const int64_t *d_prefix,
                              int ngrids, int64_t total_tiles, unsigned long long *d_queue,
                              int nbins, int slot, int device, cudaStream_t st);
// The budget as reported: sums x punit plus the carries of earlier grids;
// the photons in flight are 0 before the first step (fly_mode 0), the carry
// right after a grid update (1), else the sum (2).
struct BudgetScale {
  double emitted, punit, carry_abs, carry_esc, carry_fly;
  int fly_mode;
  int diffuse;  // 1: add the diffuse photons the cells emitted (the tiles' fourth partial)
};
// The budget of the grid's tiles into g.budget_dev (and the reported four
// terms also into copy_to[0..3] when given).
cudaError_t launch_budget(DevGrid &g, const BudgetScale &sc, cudaStream_t st, double *copy_to = nullptr);
cudaError_t launch_kappa(DevGrid &g, const double *bins_dev, cudaStream_t st);
// dynamic grid update (sx_update.cu)
cudaError_t launch_mark(DevGrid &g, double y_thresh, double min_spacing, uint8_t *cand,
                        uint8_t *rem, int64_t *blk, int64_t *total, int32_t *out,
                        cudaStream_t st);
cudaError_t launch_incoming_bins(DevGrid &g, int last, void *I, cudaStream_t st);
cudaError_t launch_hand_over(DevGrid &g, const uint8_t *rem, int32_t *target, void *I,
                             cudaStream_t st);
cudaError_t launch_carry(int precision, int64_t n_new, int nbp, const int32_t *old_of_new,
                         const double *y_old, const void *I_old, double *y_new, void *I_new,
                         cudaStream_t st);
cudaError_t launch_row_totals(int precision, int64_t n, int nbins, int nbp, const void *I,
                              double *out, cudaStream_t st);
cudaError_t launch_sum_rows(int precision, int64_t n, int nbins, int nbp, const void *I,
                            double *part, int nblk, cudaStream_t st);
cudaError_t launch_inflight(DevGrid &g, int64_t step, cudaStream_t st);
// Move the stored photons of buffer `buf` from the row stride g.nbp to
// `stride`, through the other buffer (whose contents the next step does not
// read); g.nbp is left for the caller to set.
cudaError_t launch_restride(DevGrid &g, int buf, int stride, cudaStream_t st);
// ballistic straight sets of every in-edge (after the edge tables)
cudaError_t launch_ballistic_tables(DevGrid &g, cudaStream_t st);
// kappa's per-block sums (numerator, denominator) into g.kappa_part, from the
// unrotated table (the context's kappa is not touched)
cudaError_t launch_kappa_parts(DevGrid &g, const double *bins_dev, cudaStream_t st);
// halo exchange (sx_halo.cu): pack (or unpack) the masks at ne in-edge
// indices and the photon rows of nr vertices of buffer `buf` into (from) data
size_t halo_rows_offset(int64_t n_edges, int mw);
cudaError_t launch_halo(DevGrid &g, int buf, bool pack, int64_t ne, const int32_t *eidx, int64_t nr,
                        const int32_t *ridx, void *data, cudaStream_t st);

}  // namespace sx
