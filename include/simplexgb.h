/*
 * simplexgb.h -- C ABI of the GB300 (sm_103a) SimpleX2 direction-conserving
 * photon transport library.
 *
 * The library runs the data-parallel hot path of SimpleX2 (Paardekooper,
 * Kruip & Icke 2010): repeated radiative-transfer steps on a Delaunay graph in
 * which photons held in n global direction bins move one edge per step along
 * the most straightforward neighbours of the edge associated with their bin
 * (Sect. 2.2.3), are absorbed with optical depth n_HI sigma dL (Sect. 4.4,
 * Eq. optical_depth) and ionise hydrogen through the subcycled rate equation
 * (Sect. 4.5, Eqs. rate_eq_subcycle, phot_ion_rate_subcycle).
 *
 * Conventions shared by every call
 *   - Return value: SX_OK (0) or a negative SX_E* code; sx_last_error() gives
 *     a one-line reason.  A failed call leaves the context usable unless it
 *     returns SX_ECUDA (a CUDA error; the CUDA context may be lost).
 *   - Host pointers are read during the call (or, for sx_step, not at all);
 *     the library keeps no reference to them, except the budgets array of
 *     sx_step_budgets, which is written behind the queued steps and must stay
 *     valid until the stream has reached them.  Device memory is the caller's:
 *     the per-grid state lives in one device workspace the caller allocates
 *     (size from sx_workspace_bytes) and keeps alive until sx_destroy and
 *     until the work queued on the context's stream has run.
 *   - Vertex ids are the caller's order 0..n-1.  The CSR is symmetric, each
 *     row sorted strictly ascending, no self loops (a Delaunay graph).
 *   - Work is queued on the stream given in sx_config (NULL = the legacy
 *     default stream).  sx_step returns once its work is queued; the read
 *     calls synchronise the stream before returning.
 *   - A context is not thread-safe; distinct contexts on distinct streams may
 *     be driven from distinct threads.
 */
#ifndef SIMPLEXGB_H
#define SIMPLEXGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SX_OK = 0,
    SX_EINVAL = -1,   /* bad argument or malformed grid */
    SX_ENOMEM = -2,   /* workspace too small */
    SX_ECUDA = -3,    /* CUDA runtime error */
    SX_ESTATE = -4,   /* call out of order (e.g. step before load) */
    SX_ETIMEOUT = -5  /* a bounded device wait gave up */
};

enum {
    SX_FP64 = 0,           /* photons, transport and chemistry in FP64 */
    SX_FP32_TRANSPORT = 1  /* photons and transport in FP32: every bin's
                              packets are summed in a fixed order with a
                              compensated (Kahan-Babuska) addition; N_in and
                              the per-tile budget terms in float-float.  The
                              chemistry -- the neutral fraction y and the
                              recombination subcycling (Sect. 4.5) -- runs in
                              FP64 unless sx_config.chem_fp32 = 1, which
                              evaluates the subcycle rates, lengths and
                              exponentials in FP32 and keeps only y in FP64.
                              The budget's global reduction is FP64. */
};

/* Transport of the photons that a vertex passes on (Sect. 2.2):
     SX_TRANSPORT_DCT        direction conserving (Sect. 2.2.3): photons in n
                             global direction bins, rotated every step;
     SX_TRANSPORT_BALLISTIC  ballistic (Sect. 2.2.2): photons kept per
                             incoming edge and sent on, in 3 equal parts, to
                             the most straightforward neighbours with respect
                             to that edge (none beyond 90 degrees); a source
                             sends to all its neighbours;
     SX_TRANSPORT_COMBINED   combined (Sect. 2.2.4): a vertex is ballistic in a
                             step when its optical depth y tau_max (y its
                             neutral fraction at the start of the step) is at
                             least tau_switch, else direction conserving;
                             photons arriving at a direction-conserving vertex
                             along an edge go to the bin closest to the
                             direction they travelled, bins arriving at a
                             ballistic vertex along an edge are summed into
                             that edge.
   Ballistic and combined transport support sx_step, sx_step_budgets and the
   readouts; the dynamic grid update, checkpoints, batches and the autotuner
   take direction-conserving contexts only (SX_EINVAL otherwise). */
enum {
    SX_TRANSPORT_DCT = 0,
    SX_TRANSPORT_BALLISTIC = 1,
    SX_TRANSPORT_COMBINED = 2
};

#define SX_MAX_BINS 128
#define SX_MAX_DEGREE 64      /* per non-sink vertex */
#define SX_MAX_SOURCES 4096
#define SX_FLAG_SINK 1u
#define SX_FLAG_GHOST 2u      /* a copy of a vertex another shard steps (see the halo exchange) */

typedef struct sx_ctx sx_ctx;

typedef struct {
    int32_t nbins;          /* direction bins n, 1..SX_MAX_BINS (paper: 42 or 84) */
    int32_t precision;      /* SX_FP64 or SX_FP32_TRANSPORT */
    uint64_t seed;          /* random rotations: Philox4x32-10 key */
    double sigma;           /* photoionisation cross-section, cm^2 (6.3e-18 at 13.6 eV) */
    double alpha_B;         /* case-B recombination coefficient, cm^3/s (2.59e-13 at 1e4 K) */
    double kappa;           /* global path-length correction; <= 0: computed at load */
    double chem_frac;       /* subcycle length = chem_frac / (Gamma + R), 0 < f <= 1 */
    double chem_tol;        /* equilibrium when |dy| <= chem_tol * y after a subcycle */
    int32_t chem_max_sub;   /* subcycle cap per step (>= 1) */
    int32_t device;         /* CUDA device ordinal */
    void *stream;           /* cudaStream_t, or NULL */
    int32_t transport;      /* SX_TRANSPORT_DCT (default), _BALLISTIC or _COMBINED */
    double tau_switch;      /* combined: ballistic where y tau_max >= tau_switch (default 1,
                               Sect. 5.1.3) */
    int32_t chem_fp32;      /* SX_FP32_TRANSPORT only: 0 (default) = FP64 subcycles;
                               1 = subcycle rates in FP32, y in FP64 (faster, less exact);
                               ignored in SX_FP64.  Other values: SX_EINVAL */
    double alpha_A;         /* diffuse recombination radiation (Sect. 2.2.1, 4.5; the paper's
                               tests leave it out): 0 (default) = the on-the-spot
                               approximation, recombination at alpha_B; > 0 = the case-A
                               coefficient (cm^3/s, >= alpha_B; 4.18e-13 at 1e4 K):
                               recombination runs at alpha_A, and the fraction
                               (alpha_A - alpha_B) / alpha_A of a cell's recombinations in a
                               step (summed over its subcycles) become ionising photons that
                               the cell emits in the next step as a source does -- an equal
                               share in every bin of its incoming photons, after the sources'
                               (a ballistic vertex sends them with its own photons to all its
                               neighbours).  They count as emitted when they enter.  The
                               dynamic grid update refuses alpha_A > 0. */
} sx_config;

typedef struct {
    double emitted;     /* photons injected by the sources */
    double absorbed;    /* photons used by photoionisation */
    double escaped;     /* photons that reached a sink (or had no outgoing edge) */
    double in_flight;   /* photons travelling along edges after the last step */
} sx_budget;

typedef struct {
    int64_t n, nnz;          /* vertices, directed edges */
    int64_t step;            /* steps taken so far */
    int64_t workspace_bytes; /* bytes the grid uses */
    double kappa;            /* path-length correction in use */
    int64_t subcycles;       /* chemistry subcycles summed over vertices and steps */
    int64_t capped;          /* vertex-steps that hit chem_max_sub */
    int32_t max_degree;      /* largest non-sink degree */
    int32_t nsources;
    double step_kernel_ms;   /* summed duration of the timed step-kernel launches */
    int64_t step_kernel_launches;
    int64_t index_errors;    /* debug builds (SX_DEBUG): indices the step kernels found out of
                                range and skipped; always 0 in release builds, which do not check */
} sx_info;

/* Fill cfg with the Test-1 defaults of Sect. 5.1 (42 bins, FP32 transport
   with FP64 chemistry, sigma 6.3e-18, alpha_B 2.59e-13, chem_frac 0.5,
   chem_tol 1e-5, chem_max_sub 1000, seed 0, device 0, NULL stream). */
void sx_config_default(sx_config *cfg);

/* Create a context.  bin_dirs: nbins x 3 unit vectors (row-major, FP64) --
   the global direction bins of Sect. 2.2.3 before rotation.  They are copied.
   NULL: the library's Fibonacci lattice, z_j = 1 - (2j + 1)/n,
   phi_j = j pi (3 - sqrt 5), j = 0..n-1, in that order (the paper does not
   give its construction); pass the directions explicitly where results must
   match another program bit for bit (their cosines and sines come from the
   host's math library).  Errors: SX_EINVAL (nbins out of range, not unit
   vectors, bad precision or chemistry parameters), SX_ECUDA. */
int sx_create(const sx_config *cfg, const double *bin_dirs, sx_ctx **out);

/* Device workspace needed for a grid of n vertices and nnz directed edges. */
int sx_workspace_bytes(const sx_ctx *ctx, int64_t n, int64_t nnz, int64_t *bytes);

/* Load a grid (Sect. 2.1): copy it to the device and build the per-edge
   tables -- reverse edge, int8-quantised edge direction, the <= 3 most
   straightforward neighbours of every edge (Sect. 2.2.2, within 90 degrees)
   -- the global path correction kappa (Sect. 2.2.3) and the per-vertex
   constants A = n_H V, tau_max = n_H sigma kappa <L>, alpha_B n_H.
     pos     n x 3 FP64 positions (cm)
     row_ptr n + 1 int64 CSR offsets; col nnz int32 neighbour ids
     nH      n FP64 hydrogen densities (cm^-3); volume n FP64 cell volumes (cm^3)
     flags   n bytes, bit 0 = sink (absorbs everything into "escaped"), bit 1 = ghost
             (a shard's copy of another shard's vertex: SX_FLAG_GHOST below)
     y0      n FP64 initial neutral fractions, or NULL for 1 (neutral)
     d_workspace, workspace_bytes: caller-owned device memory, >= sx_workspace_bytes,
             256-byte aligned.
   Resets the step counter, the sources and the budget.  Errors: SX_EINVAL
   (row_ptr not starting at 0 or decreasing -- checked on the host before
   anything runs on the device --, asymmetric/unsorted CSR, id out of range,
   self loop, non-sink degree > SX_MAX_DEGREE, n or nnz >= 2^31), SX_ENOMEM
   (workspace too small), SX_ECUDA. */
int sx_load_grid(sx_ctx *ctx, int64_t n, const double *pos, const int64_t *row_ptr,
                 const int32_t *col, const double *nH, const double *volume,
                 const uint8_t *flags, const double *y0, void *d_workspace,
                 int64_t workspace_bytes);

/* Make vertex a source of photons_per_s ionising photons (Sect. 4.3); the
   photons of a step, photons_per_s * dt, enter the vertex in equal shares per
   bin.  Adding a source to a vertex twice adds the rates.  Errors: SX_EINVAL
   (vertex out of range, negative rate, too many sources), SX_ESTATE. */
int sx_add_source(sx_ctx *ctx, int32_t vertex, double photons_per_s);

/* Queue nsteps radiative-transfer steps of dt_s seconds each (Sect. 4.6):
   per step, rotate the bins at random (Philox4x32-10, counter = step), move
   packets in flight to the closest bin of the new orientation, inject the
   sources, update ionisation and absorb, route the transmitted photons one
   edge further.  The rotation tables of up to SX_STEP_BLOCK consecutive steps
   are made by one kernel launch, so nsteps steps take nsteps step launches
   and ceil(nsteps / SX_STEP_BLOCK) rotation launches.
   Errors: SX_EINVAL (dt <= 0, nsteps < 0), SX_ESTATE. */
#define SX_STEP_BLOCK 16
int sx_step(sx_ctx *ctx, double dt_s, int32_t nsteps);

/* sx_step with the photon budget read after every step: budgets[k] receives
   the budget (as sx_read_photons reports it) after the k-th of the nsteps
   steps.  Nothing waits: the reads are queued on the context's stream behind
   their steps (a reduction of the tiles' partial sums after every step into
   a device staging area; one device-to-host copy per 256 steps and one at
   the end of the call), and budgets holds them once sx_sync, or a call that
   returns results, has returned.  budgets must stay valid until then; in
   page-locked host memory the copies run asynchronously.  Steps are launched
   directly (not through the graph of sx_step).  Errors: as sx_step, and
   SX_EINVAL if budgets is NULL with nsteps > 0. */
int sx_step_budgets(sx_ctx *ctx, double dt_s, int32_t nsteps, sx_budget *budgets);

/* Wait for the context's queued work. */
int sx_sync(sx_ctx *ctx);

/* Neutral fraction y = 1 - x per vertex (caller order), n doubles. */
int sx_read_neutral_fraction(sx_ctx *ctx, double *y_out);

/* Photon budget (FP64) and, if per_vertex != NULL, the photons in flight
   towards every vertex (n doubles). */
int sx_read_photons(sx_ctx *ctx, double *per_vertex, sx_budget *budget);

/* Counters of the grid; synchronises the stream if kernel timing is on. */
int sx_get_info(sx_ctx *ctx, sx_info *info);

/* Host side of the dynamic grid update, Sect. 2.1.4: remove an independent set
   of vertices (no two adjacent) from a Delaunay tetrahedralisation by
   re-triangulating their cavities.  Each removed vertex's cavity (the union
   of its tetrahedra) is filled with the Delaunay tetrahedra of its neighbours
   that lie inside it, built by Bowyer-Watson insertion in host memory; the
   graph, the cell volumes (1/4 of the incident tetrahedra) and the
   tetrahedra are patched, and the survivors renumbered in their old order.
     pos n x 3, row_ptr n + 1 (int64), col nnz (ascending rows, symmetric),
     tets ntet x 4, volume n; removed nrem vertex ids.
   On success *out holds the new grid in arrays this call allocates (free them
   with sx_remesh_free).  A cavity whose new tetrahedra do not fill its
   volume (a vertex on the convex hull, a degenerate neighbourhood) returns
   SX_EINVAL with out->bad_vertex set: the caller rebuilds the grid instead.
   Errors: SX_EINVAL (bad arguments, a row_ptr that decreases, a col or tets
   entry outside [0, n), adjacent removed vertices: bad_vertex -1),
   SX_ENOMEM.  No device memory or GPU is used.  The call runs on up to 16
   host threads (fewer for small grids), joined before it returns; its
   result does not depend on their number. */
typedef struct {
    int64_t n, nnz, ntet;
    int64_t *row_ptr;     /* n + 1 */
    int32_t *col;         /* nnz */
    double *volume;       /* n */
    int32_t *tets;        /* ntet x 4 */
    int32_t *old_of_new;  /* n: the old id of each survivor */
    int32_t bad_vertex;   /* a removed vertex whose cavity could not be filled, or -1 */
} sx_remesh_result;
int sx_remesh_remove(int64_t n, const double *pos, const int64_t *row_ptr, const int32_t *col,
                     int64_t ntet, const int32_t *tets, const double *volume, int64_t nrem,
                     const int32_t *removed, sx_remesh_result *out);
void sx_remesh_free(sx_remesh_result *result);

/* Dynamic grid, Sect. 2.1.4: where the optical depth fell, vertices are removed
   down to a minimum resolution and the survivors are re-triangulated.
   sx_grid_update_mark lists the vertices to remove: not sinks, not sources,
   neutral fraction < y_thresh (the cell became transparent) and mean edge
   length < min_spacing_cm (finer than the minimum resolution), keeping only
   those whose such neighbours all have larger ids, so that no two removed
   vertices are adjacent.  removed: caller buffer of capacity n, filled in
   ascending order; *n_removed its length.  Errors: SX_EINVAL, SX_ESTATE. */
int sx_grid_update_mark(sx_ctx *ctx, double y_thresh, double min_spacing_cm, int32_t *removed,
                        int64_t *n_removed);

/* Replace the grid by the survivors of the last sx_grid_update_mark (which must
   come right before, without steps in between).  The caller re-triangulates
   the survivors and passes their grid as for sx_load_grid, with old_of_new[i]
   = the old id of new vertex i (n_new = n - n_removed entries, each survivor
   once).  Photons in flight towards a removed vertex go to its nearest
   surviving neighbour, same bin; neutral fractions, photons, sources, the
   step count and the photon budget carry over; kappa is recomputed unless
   fixed in sx_config.  d_workspace: a new caller-owned workspace for the new
   grid (the old one may be released after the call).  Errors: SX_EINVAL,
   SX_ENOMEM, SX_ESTATE, SX_ECUDA. */
int sx_grid_update_apply(sx_ctx *ctx, int64_t n_new, const double *pos, const int64_t *row_ptr,
                         const int32_t *col, const double *nH, const double *volume,
                         const uint8_t *flags, const int32_t *old_of_new, void *d_workspace,
                         int64_t workspace_bytes);

/* enable = 1: bracket every step-kernel launch with a CUDA event pair on the
   context's stream and accumulate the durations (reported by sx_get_info);
   enabling resets the sums.  enable = 0: stop timing. */
int sx_profile(sx_ctx *ctx, int enable);

/* ---------------------------------------------------------------------------
 * Checkpoints (a system facility, no counterpart in the paper).  A
 * checkpoint holds a loaded grid's tables and state -- positions, CSR,
 * per-edge and per-vertex tables, neutral fractions, the photons in flight
 * and their routing, budget, sources, step counters -- in one little-endian
 * file that ends with a checksum of all its other bytes; restoring it and
 * stepping on gives bit-identical results to stepping on from the save.
 * ------------------------------------------------------------------------- */

/* Write the context's grid and state to path (overwritten).  Waits for the
   stream.  Errors: SX_EINVAL (path not writable), SX_ESTATE (no grid, or a
   grid update marked but not applied), SX_ECUDA. */
int sx_save(sx_ctx *ctx, const char *path);

/* Vertex and directed-edge counts of the grid in a checkpoint, to size the
   workspace (sx_workspace_bytes).  Reads the header only.  Errors: SX_EINVAL
   (not a checkpoint). */
int sx_checkpoint_info(const char *path, int64_t *n, int64_t *nnz);

/* Read a checkpoint through and check it against its checksum (host only, no
   GPU).  SX_OK, or SX_EINVAL (not a checkpoint, no checksum, damaged or
   truncated) with the reason from sx_last_error(NULL). */
int sx_checkpoint_verify(const char *path);

/* Replace the context's grid and state by the checkpoint's, in the caller's
   workspace (>= sx_workspace_bytes for the checkpoint's n and nnz, 256-byte
   aligned).  The context must have the checkpoint's bins (directions) and
   precision; the run parameters (seed, sigma, alpha_B, kappa, chemistry)
   are the checkpoint's.  The whole file is first checked against its
   checksum (as sx_checkpoint_verify), so a damaged file is refused before
   the context is touched; the file is then read a second time to restore
   it.  A call that fails after those checks leaves the context without a
   grid (SX_ESTATE until the next load).  Errors: SX_EINVAL (not a
   checkpoint, damaged, other bins or precision, truncated file), SX_ENOMEM
   (workspace too small), SX_ECUDA. */
int sx_restore(sx_ctx *ctx, const char *path, void *d_workspace, int64_t workspace_bytes);

/* ---------------------------------------------------------------------------
 * Launch shape of the step kernel (a system choice, no counterpart in the
 * paper).  A step launch works on 32-vertex tiles; its variant is the number
 * of consecutive vertices one warp works on: 4 (8 warps per tile, the
 * default) or 2 (16 warps per tile).  Both compute the same step; sums whose
 * order follows the warps (N_in, the budget) can differ in the last bits, so
 * results are reproducible for a given variant.  A batch steps with the
 * variant of its first grid.  The stored photons' row stride (bin packing)
 * is the other launch choice: nbins rounded up to 4 ("packed", the default:
 * 44 for 42 bins) or to 8 ("aligned": 48, rows of 32-byte multiples in
 * FP32); it changes no result.  The workspace has room for either.
 * ------------------------------------------------------------------------- */
#define SX_TUNE_MAX_CANDIDATES 4

typedef struct sx_tune_result {
  int32_t variant;                        /* chosen: vertices per warp */
  int32_t ncandidates;                    /* variants tried (vertices per warp x stride) */
  int32_t candidates[SX_TUNE_MAX_CANDIDATES];  /* vertices per warp of each */
  double ms_per_step[SX_TUNE_MAX_CANDIDATES]; /* mean step time of each (rotation + step) */
  int32_t stride;                         /* chosen: row stride of the stored photons */
  int32_t strides[SX_TUNE_MAX_CANDIDATES];  /* row stride of each */
} sx_tune_result;

/* Set (2 or 4) or read the variant of a context.  Errors: SX_EINVAL. */
int sx_set_variant(sx_ctx *ctx, int32_t variant);
int sx_get_variant(sx_ctx *ctx, int32_t *variant);

/* Set or read the row stride of the stored photons: nbins rounded up to 4 or
   to 8.  Setting moves the photons the next step reads to the new stride (a
   queued copy on the context's stream); results are unchanged bit for bit.
   Errors: SX_EINVAL (another stride, not direction conserving), SX_ESTATE (no
   grid, or a grid update marked but not applied), SX_ECUDA. */
int sx_set_bin_stride(sx_ctx *ctx, int32_t stride);
int sx_get_bin_stride(sx_ctx *ctx, int32_t *stride);

/* Autotuner: times every variant (vertices per warp x row stride) for
   nsteps steps of size dt_s on the loaded grid, from its current state,
   and keeps the fastest.  The grid's state is
   saved in `scratch` (device memory owned by the caller, at least
   sx_workspace_bytes of the loaded grid, 256-byte aligned) and restored
   after every trial, so the call leaves the simulation exactly where it was
   (step count, budget, every device buffer).  Waits for the context's
   stream.  1 <= nsteps <= 1000.  Errors: SX_EINVAL (arguments, scratch too
   small), SX_ESTATE (no grid), SX_ECUDA. */
int sx_autotune(sx_ctx *ctx, double dt_s, int32_t nsteps, void *scratch, size_t scratch_bytes,
                sx_tune_result *out);

/* ---------------------------------------------------------------------------
 * Batched stepping of many grids (a system form of the method, not in the
 * paper): one rotation launch and one persistent step launch per step cover
 * every grid of the batch; the CTAs pull (grid, 32-vertex tile) items from a
 * work queue, so uneven grids share the GPU.  Each grid keeps its own state
 * and gets results identical to stepping it alone with sx_step.
 * ------------------------------------------------------------------------- */
typedef struct sx_batch sx_batch;

/* Device bytes the batch tables need for up to max_grids grids. */
int sx_batch_workspace_bytes(int32_t max_grids, int64_t *bytes);

/* Create a batch driver on a device and stream (NULL = legacy default
   stream).  d_workspace (caller-owned, 256-byte aligned, >=
   sx_batch_workspace_bytes) holds the per-grid argument tables.
   Errors: SX_EINVAL, SX_ENOMEM, SX_ECUDA. */
int sx_batch_create(int32_t max_grids, int32_t device, void *stream, void *d_workspace,
                    int64_t workspace_bytes, sx_batch **out);

/* Advance n loaded contexts by nsteps steps, context i with time step
   dt_s[i].  All contexts must share nbins, precision and device.  Work is
   queued on the batch stream after the contexts' pending work; the contexts'
   streams wait for it before their next call.  Per step, grids of fewer
   than 8192 tiles (262,144 vertices) share one persistent launch; each
   larger grid steps in a launch of its own, as sx_step would (results are
   the same either way).  Errors: SX_EINVAL (n out of
   1..max_grids, mixed nbins/precision/device, dt <= 0), SX_ESTATE (a context
   without grid), SX_ECUDA. */
int sx_batch_step(sx_batch *batch, sx_ctx *const *ctxs, int32_t n, const double *dt_s,
                  int32_t nsteps);

void sx_batch_destroy(sx_batch *batch);
const char *sx_batch_last_error(const sx_batch *batch);

/* ---------------------------------------------------------------------------
 * For callers that cannot allocate device memory.  (The paper has no
 * counterpart of this entry point: it is an interface of this library.)
 * ------------------------------------------------------------------------- */
#define SX_NOALLOC_MAX_VERTICES 16384
#define SX_NOALLOC_MAX_EDGES 262144

/* The path-length correction kappa of a grid -- the value sx_load_grid
   computes and sx_get_info reports -- for callers that cannot allocate
   device memory (code running while another allocator owns the device, or
   that must not call the allocator): it allocates nothing, and needs no
   workspace.  Host inputs as for sx_load_grid, bin_dirs as for sx_create.
   Its device scratch is one fixed array of about 10 MB that every GPU loading
   this library holds until exit, so n <= SX_NOALLOC_MAX_VERTICES and nnz <=
   SX_NOALLOC_MAX_EDGES (SX_EINVAL beyond).  The first call on a device looks
   up that array's address there; make it before any stream capture.  Calls
   share the array: the call waits for its stream before returning (also
   when it fails after queuing work), and calls whose GPU work overlaps would
   race (the calls of one process are serialised on the host).  `device` is
   current during the call; the caller's current device is current again when
   it returns.  Errors: SX_EINVAL, SX_ECUDA; reason from
   sx_kappa_noalloc_last_error(). */
int sx_kappa_noalloc(int64_t n, const double *pos, const int64_t *row_ptr, const int32_t *col,
                     const uint8_t *flags, int32_t nbins, const double *bin_dirs, int32_t device,
                     void *stream, double *kappa_out);
const char *sx_kappa_noalloc_last_error(void);

/* ---------------------------------------------------------------------------
 * One grid split into shards (the paper's domain decomposition for
 * distributed memory, Sect. 3.1-3.2: every vertex depends only on its
 * neighbours' photons of the previous step, so the subdomains exchange their
 * boundary once per step).  A shard is an ordinary grid whose vertices are a
 * range of the whole grid's vertices plus, flagged SX_FLAG_GHOST, their
 * neighbours owned by other shards; its CSR holds every local neighbour of
 * every local vertex (for a ghost: those of its neighbours that are local).
 * A ghost is not stepped, sends nothing and counts in no budget term, and is
 * not part of kappa; sources go on the owning shard only.  After every step
 * each shard packs, for each other shard, what that shard's gather will read
 * from this shard's vertices -- the routing masks at the receivers' in-edge
 * indices and the senders' transmitted photons -- and the other shard
 * unpacks them at its own indices (the ghosts' out-edges' masks and the
 * ghosts' photon rows) before its next step.  With the local vertices in
 * the whole grid's order (ghosts below, owned, ghosts above) every vertex
 * gathers in the same order as in the whole grid, so the neutral fractions
 * equal the whole grid's bit for bit; the budget, summed over the shards, to
 * its rounding.  Direction-conserving transport only (SX_EINVAL otherwise);
 * the dynamic grid update refuses a shard.
 * ------------------------------------------------------------------------- */

/* kappa's two sums (Sect. 2.2.3) over the loaded grid's interior, non-ghost
   vertices: progress along the unrotated bins and path length of their
   straight moves (each a mean over the straight set), summed per vertex in
   FP32 and across vertices in FP64.  kappa of the whole grid is the sum of
   the shards' num over the sum of their den; pass it as sx_config.kappa.
   Waits for the stream.  Errors: SX_ESTATE (no grid, or after sx_restore or
   sx_grid_update_mark, which reuse the load-time tables), SX_ECUDA. */
int sx_kappa_sums(sx_ctx *ctx, double *num, double *den);

/* SX_FP32_TRANSPORT stores photons in units of a power of two, by default
   the power of two just above the photons the sources emit in the first
   step (so that packets stay near 1 and the scaling is exact).  Shards of
   one grid exchange stored values, so they must share the unit: set it, on
   every shard, to the whole grid's (frexp of the sum over all its sources of
   rate x dt, as 2^exponent) after the load and before the first step.
   SX_FP64 ignores it.  Errors: SX_EINVAL (not a positive power of two),
   SX_ESTATE (no grid, or a step has run). */
int sx_set_photon_unit(sx_ctx *ctx, double unit);

/* Bytes of one halo buffer of n_edges masks and n_rows photon rows: the
   masks (the grid's mask words per edge: 1, 2 or 4 x 32 bits), then, at the
   next 16-byte boundary, the rows (nbins rounded up to 4 values of the
   photon type: FP64, or FP32 in SX_FP32_TRANSPORT). */
int sx_halo_bytes(const sx_ctx *ctx, int64_t n_edges, int64_t n_rows, int64_t *bytes);

/* Queue, on the context's stream, the gather of the buffers the last step
   wrote into d_buf (device memory, 16-byte aligned, >= sx_halo_bytes):
   mask k = the mask at in-edge index d_edge_idx[k] (0 <= k < n_edges), row
   k = the transmitted photons of vertex d_row_idx[k] (local ids; both index
   arrays in device memory, read when the work runs).  An index out of range
   is skipped and counted in sx_info.index_errors.  Errors: SX_EINVAL (counts,
   NULL pointers, alignment, not direction conserving), SX_ESTATE (no grid or
   no step taken), SX_ECUDA. */
int sx_halo_pack(sx_ctx *ctx, int64_t n_edges, const int32_t *d_edge_idx, int64_t n_rows,
                 const int32_t *d_row_idx, void *d_buf);

/* The inverse: queue the scatter of d_buf into the buffers the last step
   wrote, so that the next step's gather reads them (mask k to in-edge index
   d_edge_idx[k], row k to vertex d_row_idx[k]).  Same arguments and errors
   as sx_halo_pack; d_buf must stay valid until the work has run. */
int sx_halo_unpack(sx_ctx *ctx, int64_t n_edges, const int32_t *d_edge_idx, int64_t n_rows,
                   const int32_t *d_row_idx, const void *d_buf);

/* Release the context (not the caller's workspace).  It does not wait for
   the context's stream: free the workspace after sx_sync, or in stream order
   behind the queued work. */
void sx_destroy(sx_ctx *ctx);

/* Reason for the last failure of a call on ctx (or of sx_create if ctx is NULL). */
const char *sx_last_error(const sx_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SIMPLEXGB_H */
