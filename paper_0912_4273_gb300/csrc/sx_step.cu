// sx_step.cu -- per-step kernels of the SimpleX2 DCT sweep on sm_103a.
//
//  k_rotation   one CTA: random rotation of the direction bins (Philox4x32-10,
//               uniform quaternion), quantised rotated bins, and the map that
//               moves packets in flight to the closest bin of the new
//               orientation (Sect. 2.2.3).
//  k_step<T,MW,G> one launch per step, pull formulation.  A CTA owns a tile
//               of 32 consecutive vertices, a warp a group of G (4 or 2)
//               consecutive vertices whose edges are contiguous:
//     phase 1   lanes over the group's in-edges: gather the packets routed to
//               the group in the previous step (per-edge bin masks), each
//               moved to the closest bin of the new orientation and added in
//               a fixed order; add the sources (Sect. 4.3);
//     phase 2   lane per vertex: N_in and the subcycled photoionisation /
//               recombination (Sect. 4.5), transmitted fraction f;
//     phase 3   lanes over the group's occupied (vertex, bin) pairs: O = f I;
//               associate every bin holding photons with the edge of largest
//               quantised dot product; split O over the <= 3 most
//               straightforward neighbours of that edge (store O / |S| once,
//               one bin mask per outgoing edge); budget partials.
//  k_step_batch the same tiles for several independent grids in one
//               persistent launch (a shared work counter hands out tiles).
//  k_budget     deterministic reduction of the per-CTA budget partials.
//  k_inflight   photons in flight towards every vertex (readout).
#include <limits.h>

#include <algorithm>

#include "sx_internal.cuh"
#include "sx_step_common.cuh"  // chemistry, mask words, budget sums, packet rounds

#ifndef SX_COMBINED_MIN_BLOCKS
#define SX_COMBINED_MIN_BLOCKS 6  // resident CTAs per SM the combined kernel's registers aim for
#endif

namespace sx {

// ----------------------------------------------------------------------------
// Rotation of the bins for `step` (unrotated = identity, used for kappa).
// ----------------------------------------------------------------------------
__device__ void rotation_matrix(uint64_t seed, int64_t step, double R[9], int *attempts) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint64_t s = (uint64_t)step;
  for (int a = 0; a < kRotMaxAttempts; ++a) {
    uint32_t c[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)a, kRotTag};
    philox4x32_10(c, k0, k1);
    double v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __dmul_rn(__dadd_rn((double)(int32_t)c[i], 0.5), 0x1p-31);
    const double w = v[0], qx = v[1], qy = v[2], qz = v[3];
    const double ww = __dmul_rn(w, w), xx = __dmul_rn(qx, qx), yy = __dmul_rn(qy, qy),
                 zz = __dmul_rn(qz, qz);
    const double n2 = __dadd_rn(__dadd_rn(__dadd_rn(ww, xx), yy), zz);
    if (!(n2 <= 1.0)) continue;
    const double xy = __dmul_rn(qx, qy), xz = __dmul_rn(qx, qz), yz = __dmul_rn(qy, qz);
    const double wx = __dmul_rn(w, qx), wy = __dmul_rn(w, qy), wz = __dmul_rn(w, qz);
    R[0] = __ddiv_rn(__dsub_rn(__dsub_rn(__dadd_rn(ww, xx), yy), zz), n2);
    R[1] = __ddiv_rn(__dmul_rn(__dsub_rn(xy, wz), 2.0), n2);
    R[2] = __ddiv_rn(__dmul_rn(__dadd_rn(xz, wy), 2.0), n2);
    R[3] = __ddiv_rn(__dmul_rn(__dadd_rn(xy, wz), 2.0), n2);
    R[4] = __ddiv_rn(__dsub_rn(__dadd_rn(__dsub_rn(ww, xx), yy), zz), n2);
    R[5] = __ddiv_rn(__dmul_rn(__dsub_rn(yz, wx), 2.0), n2);
    R[6] = __ddiv_rn(__dmul_rn(__dsub_rn(xz, wy), 2.0), n2);
    R[7] = __ddiv_rn(__dmul_rn(__dadd_rn(yz, wx), 2.0), n2);
    R[8] = __ddiv_rn(__dadd_rn(__dsub_rn(__dsub_rn(ww, xx), yy), zz), n2);
    *attempts = a + 1;
    return;
  }
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  *attempts = kRotMaxAttempts;
}

__device__ void rotate_quantise(const double R[9], const double *d, int q[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double u = __dadd_rn(__dadd_rn(__dmul_rn(R[3 * r], d[0]), __dmul_rn(R[3 * r + 1], d[1])),
                               __dmul_rn(R[3 * r + 2], d[2]));
    q[r] = quantise(u);
  }
}

constexpr int kRotThreads = 256;

// Tables of `count` consecutive steps s0 .. s0+count-1 (s0 = the device step
// counter) in one CTA.  Row k of s_R / s_q holds the orientation of step
// s0-1+k and the bins quantised under it, so that row k is the previous
// orientation of the step in row k+1 (at step 0 row 0 repeats step 0, which
// remaps nothing).
__device__ void rotation_body(const RotArgs &r, int count) {
  __shared__ double s_R[kRotAhead + 1][9];
  __shared__ int s_att[kRotAhead + 1];
  __shared__ long long s_step0;
  __shared__ int s_inc;
  __shared__ int4 s_q[kRotAhead + 1][kMaxBins];
  const int t = threadIdx.x;
  const int nbins = r.nbins;
  if (t == 0) {
    long long s0 = 0;
    int inc = 0;
    if (!r.unrotated) {
      s0 = (long long)*r.steps_done;
      *r.steps_done = (unsigned long long)(s0 + count);
      if (r.incoming) {  // a grid update hands its photons to the first of these steps
        inc = *r.incoming;
        *r.incoming = 0;
      }
    }
    s_step0 = s0;
    s_inc = inc;
  }
  __syncthreads();
  const long long s0 = s_step0;
  if (t <= count) {  // one thread per orientation
    if (r.unrotated) {
      for (int i = 0; i < 9; ++i) s_R[t][i] = (i % 4 == 0) ? 1.0 : 0.0;
      s_att[t] = 0;
    } else {
      rotation_matrix(r.seed, (t == 0 && s0 == 0) ? 0 : s0 - 1 + t, s_R[t], &s_att[t]);
    }
  }
  // photons each source puts in every bin per step, in stored units:
  // ((rate dt) / n) / unit, the unit being a power of two
  for (int k = t; k < r.nsrc; k += blockDim.x) {
    r.share[k] = __dmul_rn(__ddiv_rn(__dmul_rn(r.src_rate[k], r.dt), (double)nbins), r.inv_punit);
    r.share_f[k] = (float)r.share[k];
  }
  __syncthreads();
  for (int i = t; i < (count + 1) * nbins; i += blockDim.x) {
    const int k = i / nbins, b = i - k * nbins;
    int q[3];
    rotate_quantise(s_R[k], r.bins + 3 * b, q);
    s_q[k][b] = make_int4(q[0], q[1], q[2], 0);
    if (k > 0) {
      StepTables *out = r.tab + (k - 1);
      out->qb[b] = make_float4((float)q[0], (float)q[1], (float)q[2], 0.f);
      out->qbq[b] = (uint32_t)(q[0] & 0xFF) | ((uint32_t)(q[1] & 0xFF) << 8) | ((uint32_t)(q[2] & 0xFF) << 16);
    }
  }
  __syncthreads();
  // for every step, the closest bin of its orientation to every bin of the
  // previous one (ties -> lowest index); packets of an old bin move there.
  // Nothing moves at step 0 or in the unrotated table.
  for (int i = t; i < count * kMaxBins; i += blockDim.x) {
    const int k = i / kMaxBins, b = i - k * kMaxBins;
    int best = b;
    if (!r.unrotated && s0 + k > 0 && b < nbins) {
      const int4 o = s_q[k][b];
      int bestd = 0;
      for (int b2 = 0; b2 < nbins; ++b2) {
        const int4 nq = s_q[k + 1][b2];
        const int d = nq.x * o.x + nq.y * o.y + nq.z * o.z;
        if (b2 == 0 || d > bestd) {
          best = b2;
          bestd = d;
        }
      }
    }
    r.tab[k].fwd[b] = (unsigned char)best;
  }
  if (t < count) {
    StepTables *out = r.tab + t;
    out->attempts = s_att[t + 1];
    out->step = s0 + t;
    out->remap = (!r.unrotated && s0 + t > 0) ? 1 : 0;
    out->incoming = t == 0 ? s_inc : 0;
  }
}

__global__ void __launch_bounds__(kRotThreads) k_rotation(const RotArgs r, int count) {
  rotation_body(r, count);
}

// one CTA per grid of a batch
__global__ void __launch_bounds__(kRotThreads) k_rotation_batch(const RotArgs *__restrict__ ra,
                                                                int count) {
  rotation_body(ra[blockIdx.x], count);
}

RotArgs make_rot_args(DevGrid &g, const double *bins_dev, uint64_t seed, int unrotated, double dt) {
  RotArgs r;
  r.bins = bins_dev;
  r.seed = seed;
  r.steps_done = g.steps_done;
  r.tab = g.tabs + (unrotated ? kTabUnrotated : 0);
  r.nbins = g.nbins;
  r.unrotated = unrotated;
  r.nsrc = unrotated ? 0 : g.nsrc;
  r.src_rate = g.src_rate;
  r.dt = dt;
  r.inv_punit = 1.0 / g.punit;
  r.share = g.src_share;
  r.share_f = g.src_share_f;
  r.incoming = unrotated ? nullptr : g.incoming;
  return r;
}

cudaError_t launch_rotation(DevGrid &g, const double *bins_dev, uint64_t seed, int count,
                            int unrotated, double dt, cudaStream_t st) {
  if (unrotated) count = 1;
  if (count < 1 || count > kRotAhead) return cudaErrorInvalidValue;
  k_rotation<<<1, kRotThreads, 0, st>>>(make_rot_args(g, bins_dev, seed, unrotated, dt), count);
  return cudaGetLastError();
}

cudaError_t launch_rotation_batch(const RotArgs *d_rot, int ngrids, int count, cudaStream_t st) {
  if (ngrids <= 0) return cudaSuccess;
  if (count < 1 || count > kRotAhead) return cudaErrorInvalidValue;
  k_rotation_batch<<<ngrids, kRotThreads, 0, st>>>(d_rot, count);
  return cudaGetLastError();
}

// One tile of kTile consecutive vertices; warp w owns the group of kGroup
// vertices kGroup w .. kGroup w + kGroup - 1 in phases 1 and 3, whose edges
// are one contiguous range of the CSR arrays.
//   phase 1  lanes over the group's in-edges: gather the packets routed to
//            the group last step (per-edge bin masks), each moved to the
//            closest bin of this step's orientation and added in a fixed
//            order; add the sources.
//   phase 2  lane per vertex: N_in, chemistry, transmitted fraction f.
//   phase 3  lanes over the group's (vertex, bin) pairs holding photons: the
//            edge closest to the bin, its straight set, O / |S|; then lanes
//            over the group's out-edges write the bin masks at the receivers'
//            in-edges.
// Only bins that hold photons are touched: a bin without photons sets no mask
// bit, so no reader looks at its stored value, and it is not written.
// With BAL (ballistic and combined transport) a vertex of the tile is thick
// (ballistic) or thin (direction conserving) in the step: a thick vertex keeps
// its photons per in-edge (the bins arriving along an edge summed into it)
// and sends each in-edge's photons to that edge's ballistic straight set; a
// thin vertex is handled as without BAL, and turns photons arriving along an
// edge from a thick sender into the bin closest to their direction.
template <typename T, int MW, int G, bool BAL = false>
__device__ __forceinline__ void step_tile(const StepArgs &a, const StepTables *__restrict__ tab, int64_t tile,
                                          bool reload, bool more) {
  constexpr int kGroup = G;
  constexpr int kWarps = Shape<G>::kWarps;
  constexpr int kThreads = Shape<G>::kThreads;
  constexpr int kGroupCap = Shape<G>::kCap;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s_I = reinterpret_cast<T *>(smem_raw);  // [kTile][tile_stride(nbins)]
  __shared__ uint32_t s_qbq[kMaxBins];
  __shared__ unsigned char s_fwd[kMaxBins];
  __shared__ T s_f[kTile];
  __shared__ uint32_t s_occ[kTile][MW];
  __shared__ int32_t s_R[kWarps][kGroup + 1];  // row pointers of each warp's group
  // the chemistry's inputs: per-vertex constants and y (copied in while
  // phase 1 runs)
  __shared__ __align__(16) VConst s_vc[kTile];
  __shared__ __align__(16) double s_y[kTile];

  __shared__ int s_incoming;
  __shared__ long long s_step;
  // diffuse radiation: the photons each tile vertex emits in this step (made
  // in the last one), for the budget
  __shared__ double s_D[kTile];
  // the tile's running budget terms (absorbed, escaped, -, diffuse emitted),
  // fetched in the prologue so that the end of the tile does not wait on them
  __shared__ __align__(16) double s_run[4];
  // each warp's sum of the photons its pairs let escape in phase 3, and the
  // chemistry lanes' absorbed, sink-bound and transmitted photons (kept here
  // through phase 3)
  __shared__ typename Bud<T>::type s_esc[kWarps];
  __shared__ typename Bud<T>::type s_bud[3][kTile];
  __shared__ typename Bud<T>::type s_sum[4];  // the tile's sums of s_bud and of s_D
  // BAL: thick vertices' photons per in-edge and their sources' photons of
  // the step, and every tile vertex's mode (one element each without BAL)
  // With 65 or more bins a thick vertex's packets per in-edge sit in its own
  // bin row, which it does not use (it keeps no bins); with fewer bins the
  // row is shorter than kMaxDeg and they get rows of their own.
  constexpr bool kEAlias = BAL && MW >= 3;
  __shared__ T s_E[(BAL && !kEAlias) ? kTile : 1][(BAL && !kEAlias) ? kMaxDeg : 1];
  __shared__ T s_S[BAL ? kTile : 1];
  __shared__ unsigned char s_thick[BAL ? kTile : 1];
  // Per-warp scratch: phase 1 (the packet list), then, after the barrier,
  // phase 3 (the group's staged out-edges and masks, its occupied bins).
  // phase 1 (FP32) keeps the compensation words of the group's rows there
  constexpr int kScr1 = sizeof(T) == 4 ? kGroup * (32 * MW + 1) * (int)sizeof(T) : 0;
  constexpr int kScr3 = kGroupCap * 12 + kGroupCap * MW * 4 + kGroup * 32 * MW * 2;
  constexpr int kScr = ((kScr1 > kScr3 ? kScr1 : kScr3) + 15) / 16 * 16;
  __shared__ __align__(16) unsigned char s_scr[kWarps][kScr];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the chemistry warp (lane per tile vertex)
  constexpr int cw = 0;
  static_assert(kTile == 32 && kWarps >= 4, "one chemistry warp of 32 lanes, among >= 4 warps");
  const int nbins = a.nbins, nbp = a.nbp, nbs = tile_stride(nbins);
  auto erow = [&](int v) -> T * {  // a thick vertex's packets per in-edge
    if constexpr (kEAlias) return s_I + (size_t)v * nbs; else return s_E[v];
  };
  const uint32_t lt_mask = (1u << lane) - 1u;
  if (reload) {  // this step's tables (a CTA keeps them from tile to tile of one grid)
    for (int b = tid; b < kMaxBins; b += kThreads) {
      s_qbq[b] = tab->qbq[b];
      s_fwd[b] = tab->fwd[b];
    }
    if (tid == 0) {
      s_step = tab->step;
      s_incoming = tab->incoming;
    }
  }
  const int64_t v0 = tile * kTile;

  if (warp == cw) {  // the chemistry warp fetches its vertices' constants and y
    const int64_t nv = min((int64_t)32, a.n - v0);
    for (int i = lane; i < 2 * nv; i += 32)
      cp_async16(reinterpret_cast<char *>(s_vc) + 16 * i, reinterpret_cast<const char *>(a.vc + v0) + 16 * i);
    if (lane < nv) cp_async8(s_y + lane, a.y + v0 + lane);
    if (lane == 0) cp_async16(s_run, a.partials + 4 * tile);
    if (lane == 1) cp_async16(s_run + 2, a.partials + 4 * tile + 2);
    cp_async_commit();
  }
  const int g0 = warp * kGroup;          // first tile vertex of the warp's group
  const int64_t vg = v0 + g0;            // its grid index
  T *grow = s_I + (size_t)g0 * nbs;      // the group's rows
  uint32_t(*gocc)[MW] = s_occ + g0;      // and occupancy
  // FP32: the rows' compensation words during phase 1 (bin_add), in the
  // warp's scratch; FP64 sums plainly and never touches them
  T *gcomp = reinterpret_cast<T *>(s_scr[warp]);
  // the group's rows (and FP32 compensation words), kGroup * nbs *
  // sizeof(T) bytes at an offset that is a multiple of the same, are
  // cleared with 16-byte stores when G sizeof(T) is a multiple of 16, else
  // 8-byte ones (G even)
  if constexpr (kGroup * sizeof(T) % 16 == 0) {
    for (int i = lane; i < kGroup * nbs * (int)sizeof(T) / 16; i += 32) {
      reinterpret_cast<uint4 *>(grow)[i] = make_uint4(0u, 0u, 0u, 0u);
      if constexpr (sizeof(T) == 4) reinterpret_cast<uint4 *>(gcomp)[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  } else {
    static_assert(kGroup * sizeof(T) % 8 == 0, "rows cleared in 8-byte words");
    for (int i = lane; i < kGroup * nbs * (int)sizeof(T) / 8; i += 32) {
      reinterpret_cast<uint2 *>(grow)[i] = make_uint2(0u, 0u);
      if constexpr (sizeof(T) == 4) reinterpret_cast<uint2 *>(gcomp)[i] = make_uint2(0u, 0u);
    }
  }
  if (lane < kGroup * MW) (&gocc[0][0])[lane] = 0u;
  if (lane <= kGroup) s_R[warp][lane] = a.row_ptr[vg + lane < a.n ? vg + lane : a.n];
  // Ballistic transport alone: every vertex but the sinks (and ghosts) is
  // thick in every step and writes every out-edge's packet, so an in-edge's
  // packet is always the sender's of the last step (0 from a sink, which
  // never writes), and no bin masks or sender modes are needed.
  const bool pure_bal = BAL && a.transport == kTransportBallistic;
  if constexpr (BAL) {  // the group's modes: thick where y tau_max reaches tau_switch
    if (lane < kGroup) {
      bool thick = false;
      if (vg + lane < a.n) {
        const VConst c = a.vc[vg + lane];
        thick = !(c.flags & (kFlagSink | kFlagGhost)) && (a.transport == kTransportBallistic ||
                                   __dmul_rn(a.y[vg + lane], c.tau_max) >= a.tau_switch);
      }
      s_thick[g0 + lane] = thick ? 1 : 0;
      s_S[g0 + lane] = T(0);
    }
  }
  if (reload) __syncthreads(); else __syncwarp();  // the rest of the prologue is the warp's own

  const int cur = (int)(s_step & 1);
  const T *__restrict__ Pp = static_cast<const T *>(a.P[cur ^ 1]);
  T *__restrict__ Pn = static_cast<T *>(a.P[cur]);
  const uint32_t *__restrict__ M_prev = a.M[cur ^ 1];
  uint32_t *__restrict__ M_next = a.M[cur];
  int32_t R[kGroup + 1];
#pragma unroll
  for (int g = 0; g <= kGroup; ++g) R[g] = s_R[warp][g];

  // ---------------- phase 1: gather, remap, sources ----------------
  {
    if (s_incoming) {
      // after a grid update the photons in flight arrive as a field in the
      // previous buffer (the masks are all clear: no gather this step)
      for (int g = 0; g < kGroup; ++g) {
        if (vg + g >= a.n) break;
        const T *__restrict__ Pin = Pp + (size_t)(vg + g) * nbp;
        for (int b0 = 0; b0 < nbins; b0 += 32) {
          const int b = b0 + lane;
          const T val = b < nbins ? Pin[b] : T(0);
          const bool on = val != T(0);
          add_round<T, MW>(grow, gcomp, nbs, gocc, on, on ? ((g << 7) | s_fwd[b]) : 0, val, lt_mask);
        }
      }
    }
    for (int32_t e0 = R[0]; e0 < R[kGroup]; e0 += 32) {
      // lane: in-edge e of group vertex g, its sender and the bins the
      // sender routed along it (written at this edge's index)
      const int32_t e = e0 + lane;
      int g = 0;
#pragma unroll
      for (int q = 1; q < kGroup; ++q) g += (e >= R[q]) ? 1 : 0;
      int32_t my_src = 0;
      uint32_t my_m[MW];
#pragma unroll
      for (int w = 0; w < MW; ++w) my_m[w] = 0u;
      T edge_val = T(0);  // BAL: a packet that a thick sender routed along this edge
      if (e < R[kGroup]) {
        if (!pure_bal) {
          my_src = a.col[e];
          if (!SX_INDEX_OK((unsigned)my_src < (unsigned)a.n, a.diag)) my_src = 0;
        }
        // phase 3 stages this edge's record as an out-edge: on its way to L1
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.edges + e));
        if constexpr (BAL) {
          if (pure_bal || a.mode[cur ^ 1][my_src]) edge_val = static_cast<const T *>(a.B[cur ^ 1])[e];
          else load_mask<MW>(M_prev, (int64_t)e, my_m);
        } else {
          load_mask<MW>(M_prev, (int64_t)e, my_m);
        }
      }
      if constexpr (BAL) {
        // A thick receiver keeps the edge's photons together: the bins its
        // thin sender routed along the edge, summed by the whole warp one
        // edge at a time (lanes over the bins, a fixed tree), then the edge
        // packet.
        const bool thick_recv = e < R[kGroup] && s_thick[g0 + g];
        uint32_t any_m = 0u;
#pragma unroll
        for (int w = 0; w < MW; ++w) any_m |= my_m[w];
        uint32_t todo = __ballot_sync(0xffffffffu, thick_recv && any_m != 0u);
        T binsum = T(0);
        while (todo) {
          const int l = __ffs(todo) - 1;
          todo &= todo - 1u;
          const int32_t sl = __shfl_sync(0xffffffffu, my_src, l);
          typename Bud<T>::type part{};
#pragma unroll
          for (int w = 0; w < MW; ++w) {
            const uint32_t ml = __shfl_sync(0xffffffffu, my_m[w], l);
            if ((ml >> lane) & 1u) {
              const T x = Pp[(size_t)sl * nbp + 32 * w + lane];
              if constexpr (sizeof(T) == 8) part = __dadd_rn(part, x); else part = ff_add(part, x);
            }
          }
          part = Bud<T>::warp_sum(part);  // lane 0
          T tot;
          if constexpr (sizeof(T) == 8) {
            tot = __shfl_sync(0xffffffffu, part, 0);
          } else {
            tot = __fadd_rn(__shfl_sync(0xffffffffu, part.hi, 0), __shfl_sync(0xffffffffu, part.lo, 0));
          }
          if (lane == l) binsum = tot;
        }
        if (thick_recv) {
          CSum<T> acc;
          acc.add(binsum);
          acc.add(edge_val);
          if (SX_INDEX_OK(e - R[g] < kMaxDeg, a.diag)) erow(g0 + g)[e - R[g]] = acc.value();
          edge_val = T(0);
#pragma unroll
          for (int w = 0; w < MW; ++w) my_m[w] = 0u;
        }
      }
      int cnt = 0;
#pragma unroll
      for (int w = 0; w < MW; ++w) cnt += __popc(my_m[w]);
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      // The packets of the chunk in (edge, bin) order: lane j takes packet
      // p + j, found without a list: its edge is the lowest lane whose
      // inclusive count exceeds p + j (binary search over the lanes), its
      // bin the r-th set bit of that edge's mask.
      for (int p = 0; p < total; p += 32) {
        const int j = p + lane;
        const bool on = j < total;
        int k = 0;
#pragma unroll
        for (int s2 = 16; s2 > 0; s2 >>= 1) {
          const int ik = __shfl_sync(0xffffffffu, incl, k + s2 - 1);
          if (ik <= j) k += s2;
        }
        k = min(k, 31);
        const int ek = __shfl_sync(0xffffffffu, incl - cnt, k);  // packets before edge k
        const int32_t src = __shfl_sync(0xffffffffu, my_src, k);
        const int gk = __shfl_sync(0xffffffffu, g, k);
        int r = j - ek;  // rank of the packet among edge k's bins
        // the word holding the r-th set bit and the rank within it, then the
        // bit by halving (a fixed cost, whatever the rank)
        uint32_t m = 0u;
        int base = 0, rr = 0;
#pragma unroll
        for (int w = 0; w < MW; ++w) {
          const uint32_t mk = __shfl_sync(0xffffffffu, my_m[w], k);
          const int c = __popc(mk);
          if (r >= 0 && r < c) {
            m = mk;
            base = 32 * w;
            rr = r;
          }
          r -= c;
        }
        int pos = 0, c = __popc(m & 0xFFFFu);
        if (rr >= c) { rr -= c; m >>= 16; pos += 16; }
        c = __popc(m & 0xFFu);
        if (rr >= c) { rr -= c; m >>= 8; pos += 8; }
        c = __popc(m & 0xFu);
        if (rr >= c) { rr -= c; m >>= 4; pos += 4; }
        c = __popc(m & 0x3u);
        if (rr >= c) { rr -= c; m >>= 2; pos += 2; }
        if (rr >= (int)(m & 1u)) pos += 1;
        const int bo = base + pos;
        int key = 0;
        T val = T(0);
        if (on && SX_INDEX_OK(bo < nbins, a.diag)) {
          val = Pp[(size_t)src * nbp + bo];
          key = (gk << 7) | s_fwd[bo];
        }
        add_round<T, MW>(grow, gcomp, nbs, gocc, on, key, val, lt_mask);
      }
      if constexpr (BAL) {
        // packets from thick senders at thin receivers: into the bin closest
        // to the direction they travelled (the edge to the sender reversed),
        // ties -> lowest bin
        const bool on = edge_val != T(0);
        uint32_t need = __ballot_sync(0xffffffffu, on);
        if (need) {
          int nq = 0;
          if (on) {
            const char4 q = a.edges[e].q;
            nq = (int)(unsigned char)(-q.x) | ((int)(unsigned char)(-q.y) << 8) |
                 ((int)(unsigned char)(-q.z) << 16);
          }
          // one packet at a time, lanes over the bins: key dot * 128 +
          // (127 - bin), largest for the largest dot and then the lowest bin
          int best = 0;
          while (need) {
            const int l = __ffs(need) - 1;
            need &= need - 1u;
            const int nql = __shfl_sync(0xffffffffu, nq, l);
            int bk = INT_MIN;
            for (int b = lane; b < nbins; b += 32) bk = max(bk, __dp4a((int)s_qbq[b], nql, 0) * 128 + (127 - b));
            bk = __reduce_max_sync(0xffffffffu, bk);
            if (lane == l) best = 127 - (bk & 127);
          }
          add_round<T, MW>(grow, gcomp, nbs, gocc, on, on ? ((g << 7) | best) : 0, edge_val, lt_mask);
        }
      }
    }
    // a source puts its share in every bin (BAL: a thick source keeps its
    // photons of the step apart)
    int vsrc = -1;
    if (lane < kGroup && vg + lane < a.n) vsrc = a.vc[vg + lane].src;
    uint32_t srcs = __ballot_sync(0xffffffffu, vsrc >= 0);
    while (srcs) {
      const int g = __ffs(srcs) - 1;
      srcs &= srcs - 1u;
      const int slot = __shfl_sync(0xffffffffu, vsrc, g);
      if constexpr (BAL) {
        if (s_thick[g0 + g]) {  // rate dt photons, in stored units
          if (lane == 0) s_S[g0 + g] = (T)__dmul_rn(a.src_rate[slot], a.src_scale);
          __syncwarp();
          continue;
        }
      }
      T share;
      if constexpr (sizeof(T) == 8) share = a.src_share[slot]; else share = a.src_share_f[slot];
      T *row = grow + (size_t)g * nbs;
      T *crow = gcomp + (size_t)g * nbs;
      for (int b = lane; b < nbins; b += 32) bin_add(row + b, crow + b, share);
      if (lane < MW) gocc[g][lane] = word_bins(nbins, lane);
      __syncwarp();
    }
    if (a.diffuse) {
      // diffuse radiation: the ground-level recombination photons each vertex
      // made in the last step enter now, after the sources' and as a
      // source's do: D / n in every bin (BAL, thick: with its own photons)
      double dv = 0.0;
      if (lane < kGroup && vg + lane < a.n) dv = a.dif[vg + lane];
      if (lane < kGroup) s_D[g0 + lane] = dv;
      uint32_t ds = __ballot_sync(0xffffffffu, dv > 0.0);
      while (ds) {
        const int g = __ffs(ds) - 1;
        ds &= ds - 1u;
        const double d = __shfl_sync(0xffffffffu, dv, g);
        if constexpr (BAL) {
          if (s_thick[g0 + g]) {
            if (lane == 0) s_S[g0 + g] += (T)d;
            __syncwarp();
            continue;
          }
        }
        const T share = (T)__ddiv_rn(d, (double)nbins);
        T *row = grow + (size_t)g * nbs;
        T *crow = gcomp + (size_t)g * nbs;
        for (int b = lane; b < nbins; b += 32) bin_add(row + b, crow + b, share);
        if (lane < MW) gocc[g][lane] = word_bins(nbins, lane);
        __syncwarp();
      }
    }
    if constexpr (sizeof(T) == 4) {  // fold the compensation words into the occupied bins
      __syncwarp();
      if (lane < kGroup * MW) {  // lane: mask word lane % MW of group vertex lane / MW
        const int g = lane / MW, w = lane % MW;
        uint32_t m = gocc[g][w];
        T *row = grow + (size_t)g * nbs + 32 * w;
        const T *crow = gcomp + (size_t)g * nbs + 32 * w;
        while (m) {
          const int i = __ffs(m) - 1;
          m &= m - 1u;
          const float c = crow[i];
          if (c != 0.f) row[i] = __fadd_rn(row[i], c);
        }
      }
    }
  }
  __syncthreads();

  // ---------------- phase 2: N_in and chemistry, lane per vertex ----------------
  // photons absorbed in the tile's cells and passed to sinks, in stored units
  // (FP64 sums, or float-float in FP32 mode)
  // and transmitted (N_in f: in flight, but for what phase 3 finds no edge for)
  double bud_abs = 0.0, bud_sink = 0.0, bud_tr = 0.0;
  FF bud_abs_ff{0.f, 0.f}, bud_sink_ff{0.f, 0.f}, bud_tr_ff{0.f, 0.f};
  unsigned diag_nsub = 0, diag_capped = 0;  // subcycle counters, summed after phase 3
  if (warp == cw) {
    cp_async_wait_all();
    __syncwarp();
    const int vl = lane;
    const int64_t v = v0 + vl;
    T f = T(0);
    int nsub = 0, capped = 0;
    if (v < a.n) {
      const VConst c = s_vc[vl];
      // N_in in stored units: the occupied bins of the vertex, ascending
      // (BAL, thick: its in-edges ascending, then its source's photons)
      const T *row = s_I + (size_t)vl * nbs;
      typename Bud<T>::type nin_acc{};
      bool thick_v = false;
      if constexpr (BAL) {
        thick_v = s_thick[vl] != 0;
        if (thick_v) {
          const int gw = vl / kGroup, gi = vl % kGroup;
          const int dg = s_R[gw][gi + 1] - s_R[gw][gi];
          for (int j = 0; j <= dg; ++j) {
            const T x = j < dg ? erow(vl)[j] : s_S[vl];
            if constexpr (sizeof(T) == 8) nin_acc = __dadd_rn(nin_acc, x);
            else nin_acc = ff_add(nin_acc, x);
          }
        }
      }
      if constexpr (BAL) {
        // a thick vertex without photons sends nothing: it passes on as a
        // thin one (its masks are empty) and skips the per-edge sends
        bool dark;
        if constexpr (sizeof(T) == 8) dark = nin_acc == 0.0; else dark = nin_acc.hi == 0.f;
        if (thick_v && dark && !pure_bal) s_thick[vl] = 0;
      }
#pragma unroll
      for (int w = 0; w < MW; ++w) {
        uint32_t m = thick_v ? 0u : s_occ[vl][w];
        while (m) {
          const int i = __ffs(m) - 1;
          m &= m - 1u;
          if constexpr (sizeof(T) == 8) nin_acc = __dadd_rn(nin_acc, row[32 * w + i]);
          else nin_acc = ff_add(nin_acc, row[32 * w + i]);
        }
      }
      if constexpr (sizeof(T) == 8)
        f = vertex_chem<T>(a, c, v, s_y[vl], nin_acc, a.diffuse ? s_D[vl] : 0.0, nsub, capped,
                           bud_abs, bud_sink, bud_tr);
      else
        f = vertex_chem<T>(a, c, v, s_y[vl], nin_acc, a.diffuse ? s_D[vl] : 0.0, nsub, capped,
                           bud_abs_ff, bud_sink_ff, bud_tr_ff);
    }
    s_f[vl] = f;
    diag_nsub = (unsigned)nsub;
    diag_capped = (unsigned)capped;
    if constexpr (sizeof(T) == 8) {
      s_bud[0][vl] = bud_abs;
      s_bud[1][vl] = bud_sink;
      s_bud[2][vl] = bud_tr;
    } else {
      s_bud[0][vl] = bud_abs_ff;
      s_bud[1][vl] = bud_sink_ff;
      s_bud[2][vl] = bud_tr_ff;
    }
  }
  __syncthreads();

  // ---------------- phase 3: transmit, associate, route ----------------
  Acc<T> esc;  // photons this lane's pairs let escape
  {
    uint32_t *s_q = reinterpret_cast<uint32_t *>(s_scr[warp]);                   // [kGroupCap] q bytes
    uint32_t *s_st = s_q + kGroupCap;                                             // [kGroupCap] straight sets
    int32_t *s_tw = reinterpret_cast<int32_t *>(s_st + kGroupCap);               // [kGroupCap] reverse edges
    uint32_t(*s_am)[MW] = reinterpret_cast<uint32_t(*)[MW]>(s_tw + kGroupCap);  // [kGroupCap][MW]
    uint16_t *s_pair = reinterpret_cast<uint16_t *>(s_am + kGroupCap);          // [kGroup * 32 * MW]
    int vflags = 1;  // lanes < kGroup: flags of group vertex `lane` (past the grid: a sink)
    if (lane < kGroup && vg + lane < a.n) vflags = s_vc[g0 + lane].flags;
    if (vflags & kFlagGhost) vflags |= kFlagSink;  // a ghost sends nothing (its owner does)
    if constexpr (BAL) {  // thick vertices send no bins either
      if (lane < kGroup && s_thick[g0 + lane]) vflags |= 1;
    }
    const uint32_t sinks = __ballot_sync(0xffffffffu, vflags & 1);
    // consecutive vertices ga .. gb - 1 whose out-edges fit in the staging area
    // (ballistic transport alone sends no bins: nothing to stage)
    for (int ga = pure_bal ? kGroup : 0; ga < kGroup;) {
      int gb = ga + 1;
      while (gb < kGroup && s_R[warp][gb + 1] - s_R[warp][ga] <= kGroupCap) ++gb;
      const int32_t EA = s_R[warp][ga], EB = s_R[warp][gb];
      for (int32_t e = EA + lane; e < EB; e += 32) {
        const int idx = e - EA;
        if (idx < kGroupCap) {
          const Edge E = a.edges[e];
          uint32_t qw, stw;
          memcpy(&qw, &E.q, 4);
          memcpy(&stw, &E.st, 4);
          s_q[idx] = qw;
          s_st[idx] = stw;
          s_tw[idx] = E.twin;
#pragma unroll
          for (int w = 0; w < MW; ++w) s_am[idx][w] = 0u;
        }
      }
      // the (vertex, bin) pairs holding photons, vertex-major, bins ascending
      // (sinks pass nothing on): lane c takes mask word c % MW of vertex
      // ga + c / MW, places its bits after those of the lower lanes
      int np;
      {
        const int nw = (gb - ga) * MW;
        uint32_t word = 0u;
        int gq = 0, wq = 0;
        if (lane < nw) {
          gq = ga + lane / MW;
          wq = lane % MW;
          if (!((sinks >> gq) & 1u)) word = gocc[gq][wq];
        }
        const int cnt = __popc(word);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += t;
        }
        np = __shfl_sync(0xffffffffu, incl, 31);
        int pos = incl - cnt;
        while (word) {
          const int i = __ffs(word) - 1;
          word &= word - 1u;
          s_pair[pos++] = (uint16_t)((gq << 7) | (32 * wq + i));
        }
      }
      __syncwarp();
      for (int j0 = 0; j0 < np; j0 += 32) {
        const int j = j0 + lane;
        if (j < np) {
          const int pk = s_pair[j];
          const int g = pk >> 7, b = pk & 127;
          const T O = grow[(size_t)g * nbs + b] * s_f[g0 + g];
          if (O != T(0)) {
            const int ka = s_R[warp][g] - EA;
            const int dg = s_R[warp][g + 1] - s_R[warp][g];
            if (dg == 0 || dg > kMaxDeg) {
              esc.add(O);  // a vertex without (usable) edges loses what it transmits
            } else {
              // key (q_e . q_b) * 64 + 2^22 + (63 - k): largest for the largest
              // dot and, among equal dots, the lowest slot
              const int qb = (int)s_qbq[b];
              const int *qk = reinterpret_cast<const int *>(s_q + ka);
              int key = INT_MIN, k = 0;
              for (; k + 4 <= dg; k += 4) {
                const int c = (1 << 22) + 63 - k;
                const int k0 = __dp4a(qk[k], qb, 0) * 64 + c;
                const int k1 = __dp4a(qk[k + 1], qb, 0) * 64 + (c - 1);
                const int k2 = __dp4a(qk[k + 2], qb, 0) * 64 + (c - 2);
                const int k3 = __dp4a(qk[k + 3], qb, 0) * 64 + (c - 3);
                key = max(key, max(max(k0, k1), max(k2, k3)));
              }
              for (; k < dg; ++k) key = max(key, __dp4a(qk[k], qb, 0) * 64 + ((1 << 22) + 63 - k));
              const int kst = 63 - (key & 63);
              const uint32_t stw = s_st[ka + kst];
              const int cnt = (int)(stw >> 24);
              if (cnt == 0) {
                esc.add(O);
              } else {
                T P;
                if constexpr (sizeof(T) == 8) {
                  P = O / (T)cnt;
                } else {
                  P = O * (cnt == 1 ? 1.f : (cnt == 2 ? 0.5f : (1.f / 3.f)));
                }
                Pn[(size_t)(vg + g) * nbp + b] = P;
                const uint32_t bit = 1u << (b & 31);
                for (int m = 0; m < cnt; ++m) {
                  const int sl = (int)((stw >> (8 * m)) & 0xFFu);
                  if (SX_INDEX_OK(sl < dg && ka + sl < kGroupCap, a.diag)) atomicOr(&s_am[ka + sl][b >> 5], bit);
                }
              }
            }
          }
        }
      }
      __syncwarp();
      for (int32_t e = EA + lane; e < EB; e += 32) {
        const int idx = e - EA;
        uint32_t m[MW];
#pragma unroll
        for (int w = 0; w < MW; ++w) m[w] = idx < kGroupCap ? s_am[idx][w] : 0u;
        const int32_t tw = idx < kGroupCap ? s_tw[idx] : a.edges[e].twin;
        if (SX_INDEX_OK((unsigned)tw < (unsigned)a.row_ptr[a.n], a.diag))
          store_mask<MW>(M_next, (int64_t)tw, m);  // at the receiver's in-edge index
      }
      __syncwarp();
      ga = gb;
    }
    if constexpr (BAL) {
      // thick vertices: the photons of in-edge j, O_j = f E_j, go in equal
      // parts w_j = O_j / |S_j| to j's ballistic straight set S_j.  Lanes
      // over the group's in-edges turn E_j into w_j in place; then lanes over
      // its out-edges sum, for out-slot k, the w_j of the in-edges whose set
      // holds k (j ascending), add the source's f S / degree and store the
      // sum at the receiver's in-edge.
      const int32_t EA = s_R[warp][0], EB = s_R[warp][kGroup];
      for (int32_t e = EA + lane; e < EB; e += 32) {
        int g = 0;
#pragma unroll
        for (int q = 1; q < kGroup; ++q) g += (e >= s_R[warp][q]) ? 1 : 0;
        if (s_thick[g0 + g]) {
          T &E = erow(g0 + g)[e - s_R[warp][g]];
          const T o = E * s_f[g0 + g];
          const int cnt = (int)(a.stb[e] >> 24);
          if (cnt == 0) {
            esc.add(o);  // no neighbour within 90 degrees: escaped
            E = T(0);
          } else {
            if constexpr (sizeof(T) == 8) E = o / (T)cnt;
            else E = o * (cnt == 1 ? 1.f : (cnt == 2 ? 0.5f : (1.f / 3.f)));
          }
        }
      }
      if (lane < kGroup && s_thick[g0 + lane] && s_S[g0 + lane] != T(0)) {
        const T os = s_S[g0 + lane] * s_f[g0 + lane];  // a source sends to all its neighbours
        if (s_R[warp][lane + 1] == s_R[warp][lane]) esc.add(os);  // ... if it has any
      }
      __syncwarp();
      T *__restrict__ Bn = static_cast<T *>(a.B[cur]);
      for (int32_t e = EA + lane; e < EB; e += 32) {
        int g = 0;
#pragma unroll
        for (int q = 1; q < kGroup; ++q) g += (e >= s_R[warp][q]) ? 1 : 0;
        if (s_thick[g0 + g]) {
          const int32_t r0 = s_R[warp][g];
          const int dg = s_R[warp][g + 1] - r0;
          const unsigned ent = a.bpos[e];
          const uint8_t *lst = a.binv + 3 * (int64_t)r0 + (ent & 0xFFu);
          const T *Eg = erow(g0 + g);
          CSum<T> acc;
          for (unsigned i = 0; i < (ent >> 8); ++i)
            if (SX_INDEX_OK(lst[i] < dg, a.diag)) acc.add(Eg[lst[i]]);
          const T S = s_S[g0 + g];
          if (S != T(0)) acc.add((S * s_f[g0 + g]) / (T)dg);
          const int32_t tw = a.edges[e].twin;
          if (SX_INDEX_OK((unsigned)tw < (unsigned)a.row_ptr[a.n], a.diag)) Bn[tw] = acc.value();
        }
      }
      // every vertex's mode of this step, for its receivers in the next
      if (!pure_bal && lane < kGroup && vg + lane < a.n) a.mode[cur][vg + lane] = s_thick[g0 + lane];
    }
  }
  if (warp == cw) {  // the chemistry lanes' subcycle counters
    unsigned ns = diag_nsub, nc = diag_capped;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      ns += __shfl_down_sync(0xffffffffu, ns, d);
      nc += __shfl_down_sync(0xffffffffu, nc, d);
    }
    if (lane == 0) {
      if (ns) atomicAdd(&a.diag[kDiagSubcycles], (unsigned long long)ns);
      if (nc) atomicAdd(&a.diag[kDiagCapped], (unsigned long long)nc);
    }
  }
  // ---------------- budget partials of the tile ----------------
  // The chemistry warp's lanes hold each tile vertex's absorbed, transmitted
  // and sink-bound photons; phase 3 adds the transmitted photons that found
  // no edge (rare) to "escaped" and takes them from "in flight".  Each sum
  // runs in a fixed order: lanes by a shuffle tree, warps ascending.
  {
    using B = Bud<T>;
    using BT = typename B::type;
    {  // this warp's escapes
      BT e = esc.v;
      bool nz;
      if constexpr (sizeof(T) == 8) nz = e != 0.0; else nz = e.hi != 0.f;
      if (__any_sync(0xffffffffu, nz)) e = B::warp_sum(e); else e = BT{};
      if (lane == 0) s_esc[warp] = e;
    }
    // the chemistry lanes' three terms summed by warps 1..3 at once, the
    // diffuse photons by warp 4 (warp 0 with 4 warps)
    constexpr int wd = kWarps > 4 ? 4 : 0;
    if (warp >= 1 && warp <= 3) {
      const BT t = B::warp_sum(s_bud[warp - 1][lane]);
      if (lane == 0) s_sum[warp - 1] = t;
    }
    if (warp == wd && a.diffuse) {
      BT t;
      if constexpr (sizeof(T) == 8) {
        t = B::warp_sum(v0 + lane < a.n ? s_D[lane] : 0.0);
      } else {  // the photons emitted, as double: hi + lo in float-float
        const double d = v0 + lane < a.n ? s_D[lane] : 0.0;
        const float hi = (float)d;
        t = B::warp_sum(FF{hi, (float)(d - (double)hi)});
      }
      if (lane == 0) s_sum[3] = t;
    }
    __syncthreads();
    if (warp == cw && lane == 0) {
      BT e3 = s_esc[0];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) e3 = B::add(e3, s_esc[w]);
      BT neg;
      if constexpr (sizeof(T) == 8) neg = -e3; else neg = FF{-e3.hi, -e3.lo};
      double *p = a.partials + 4 * tile;
      p[0] = s_run[0] + B::to_double(s_sum[0]);
      p[1] = s_run[1] + B::to_double(B::add(s_sum[1], e3));
      p[2] = B::to_double(B::add(s_sum[2], neg));  // in flight after this step
      if (a.diffuse) p[3] = s_run[3] + B::to_double(s_sum[3]);  // diffuse photons emitted
    }
  }
  if (more) __syncthreads();  // shared state is reused by the next tile of a persistent CTA
}

// One grid, one CTA per tile (the hardware hands tiles to SMs as they free up,
// which balances tiles of unequal cost).
template <typename T, int MW, int G>
__global__ void __launch_bounds__(Shape<G>::kThreads, Shape<G>::kMinBlocks) k_step(const StepArgs a) {
  step_tile<T, MW, G>(a, a.tab, blockIdx.x, true, false);
}

// Combined transport: the same tiles with thick vertices (4 vertices per
// warp), at 6 CTAs/SM and 40 registers (with 65 or more bins the thick
// vertices' in-edge packets share the bin rows, so 6 tiles fit in shared
// memory; the extra resident warps hide more of the dependent loads than
// 5 CTAs/SM at 48 registers do).
template <typename T, int MW>
__global__ void __launch_bounds__(Shape<4>::kThreads, SX_COMBINED_MIN_BLOCKS) k_step_bal(const StepArgs a) {
  step_tile<T, MW, 4, true>(a, a.tab, blockIdx.x, true, false);
}

// Persistent CTAs pull (grid, tile) work items of a batch of grids from a
// queue, `grab` (1..kBatchChunk) consecutive tiles at a time; a tile is one
// grid's 32 consecutive vertices.
constexpr int kBatchChunk = 8;
template <typename T, int MW, int G>
__global__ void __launch_bounds__(Shape<G>::kThreads, Shape<G>::kMinBlocks)
    k_step_batch(const StepArgs *__restrict__ args, const int64_t *__restrict__ prefix, int ngrids,
                 unsigned long long *__restrict__ queue, int slot, int grab) {
  __shared__ long long s_item;
  __shared__ StepArgs s_args;  // the current grid's arguments
  const int64_t total = prefix[ngrids];
  int cur_grid = -1;
  for (;;) {
    // several consecutive tiles per grab: one atomic on the shared counter
    // serves them all
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, (unsigned long long)grab);
    __syncthreads();
    const int64_t t0 = s_item;
    __syncthreads();
    if (t0 >= total) break;
    const int64_t t1 = t0 + grab < total ? t0 + grab : total;
    for (int64_t t = t0; t < t1; ++t) {
      int lo = 0, hi = ngrids - 1;  // the grid whose tile range holds t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
      }
      static_assert(sizeof(StepArgs) % 4 == 0, "StepArgs is copied in 4-byte words");
      if (lo != cur_grid) {  // every thread is past the last tile's use of s_args
        const uint32_t *src = reinterpret_cast<const uint32_t *>(args + lo);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_args);
        for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
      }
      step_tile<T, MW, G>(s_args, s_args.tab + slot, t - prefix[lo], lo != cur_grid, true);
      cur_grid = lo;
    }
  }
}

StepArgs make_step_args(DevGrid &g, double dt, double fc, double tol, int max_sub) {
  StepArgs a;
  a.n = g.n;
  a.nbins = g.nbins;
  a.nbp = g.nbp;
  a.dt = dt;
  a.inv_dt = 1.0 / dt;
  a.punit = g.punit;
  a.fc = fc;
  a.tol = tol;
  a.max_sub = max_sub;
  a.chem_fp32 = g.chem_fp32;
  a.row_ptr = g.row_ptr;
  a.edges = g.edges;
  a.vc = g.vc;
  a.y = g.y;
  a.P[0] = g.P[0];
  a.P[1] = g.P[1];
  a.col = g.s_col;
  a.M[0] = g.M[0];
  a.M[1] = g.M[1];
  a.tab = g.tabs;
  a.src_share = g.src_share;
  a.src_share_f = g.src_share_f;
  a.partials = g.partials;
  a.diag = g.diag;
  a.B[0] = g.B[0];
  a.B[1] = g.B[1];
  a.mode[0] = g.mode[0];
  a.mode[1] = g.mode[1];
  a.stb = g.stb;
  a.bpos = g.bpos;
  a.binv = g.binv;
  a.src_rate = g.src_rate;
  a.src_scale = dt / g.punit;
  a.transport = g.transport;
  a.tau_switch = g.tau_switch;
  a.diffuse = g.diffuse;
  a.ground = g.ground;
  a.dif = g.dif;
  return a;
}

template <typename T, int MW, int G>
static void configure_smem() {
  static const bool done = [] {  // once per instantiation (thread-safe initialisation)
    cudaFuncSetAttribute(k_step<T, MW, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_step_batch<T, MW, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    return true;
  }();
  (void)done;
}

// Mask words a step kernel works with for nbins bins.
static int compute_words(int nbins) { return nbins <= 32 ? 1 : nbins <= 64 ? 2 : nbins <= 96 ? 3 : 4; }

// Calls f.template run<T, MW, G>() for the instantiation that serves
// (precision, nbins, group); group is 2 or 4 vertices per warp (else 4).
template <typename F>
static cudaError_t dispatch_step(int precision, int nbins, int group, const F &f) {
  const int w = compute_words(nbins);
  const bool g2 = group == 2;
#define SX_DISPATCH_W(T)                                                                 \
  if (w == 1) return g2 ? f.template run<T, 1, 2>() : f.template run<T, 1, 4>();        \
  if (w == 2) return g2 ? f.template run<T, 2, 2>() : f.template run<T, 2, 4>();        \
  if (w == 3) return g2 ? f.template run<T, 3, 2>() : f.template run<T, 3, 4>();        \
  return g2 ? f.template run<T, 4, 2>() : f.template run<T, 4, 4>();
  if (precision == 0) {
    SX_DISPATCH_W(double)
  }
  SX_DISPATCH_W(float)
#undef SX_DISPATCH_W
}

struct StepLaunch {
  const StepArgs &a;
  int64_t ntiles;
  int nbins;
  cudaStream_t st;
  template <typename T, int MW, int G>
  cudaError_t run() const {
    const size_t smem = sizeof(T) * (size_t)kTile * tile_stride(nbins);
    configure_smem<T, MW, G>();
    k_step<T, MW, G><<<(unsigned)ntiles, Shape<G>::kThreads, smem, st>>>(a);
    return cudaGetLastError();
  }
};

struct BalLaunch {
  const StepArgs &a;
  int64_t ntiles;
  int nbins;
  cudaStream_t st;
  template <typename T, int MW>
  cudaError_t run() const {
    const size_t smem = sizeof(T) * (size_t)kTile * tile_stride(nbins);
    static const bool done = [] {
      cudaFuncSetAttribute(k_step_bal<T, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
      return true;
    }();
    (void)done;
    k_step_bal<T, MW><<<(unsigned)ntiles, Shape<4>::kThreads, smem, st>>>(a);
    return cudaGetLastError();
  }
};

static cudaError_t dispatch_bal(int precision, int nbins, const BalLaunch &f) {
  const int w = compute_words(nbins);
  if (precision == 0) {
    if (w == 1) return f.run<double, 1>();
    if (w == 2) return f.run<double, 2>();
    if (w == 3) return f.run<double, 3>();
    return f.run<double, 4>();
  }
  if (w == 1) return f.run<float, 1>();
  if (w == 2) return f.run<float, 2>();
  if (w == 3) return f.run<float, 3>();
  return f.run<float, 4>();
}

cudaError_t launch_step(DevGrid &g, int slot, double dt, double chem_frac, double chem_tol,
                        int chem_max_sub, cudaStream_t st) {
  if (g.nblocks <= 0) return cudaSuccess;
  if (slot < 0 || slot >= kRotAhead) return cudaErrorInvalidValue;
  StepArgs a = make_step_args(g, dt, chem_frac, chem_tol, chem_max_sub);
  a.tab = g.tabs + slot;
  if (g.transport == kTransportBallistic) return launch_step_ballistic(a, g.nblocks, g.precision, st);
  if (g.transport != kTransportDct) return dispatch_bal(g.precision, g.nbins, BalLaunch{a, g.nblocks, g.nbins, st});
  return dispatch_step(g.precision, g.nbins, g.group, StepLaunch{a, g.nblocks, g.nbins, st});
}

struct BatchLaunch {
  const StepArgs *d_args;
  const int64_t *d_prefix;
  int ngrids;
  int64_t total_tiles;
  unsigned long long *d_queue;
  int nbins, slot, device;
  cudaStream_t st;
  template <typename T, int MW, int G>
  cudaError_t run() const {
    configure_smem<T, MW, G>();
    int nsm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const size_t smem = sizeof(T) * (size_t)kTile * tile_stride(nbins);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batch<T, MW, G>, Shape<G>::kThreads,
                                                  smem);
    int64_t ctas = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (ctas > total_tiles) ctas = total_tiles;
    // tiles per grab: up to kBatchChunk while every CTA still gets about
    // eight grabs, so that a small batch does not end on a few CTAs' long
    // last grabs
    const int64_t per = ctas > 0 ? total_tiles / (ctas * 8) : 1;
    const int grab = per < 1 ? 1 : (per > kBatchChunk ? kBatchChunk : (int)per);
    cudaError_t e = cudaMemsetAsync(d_queue, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (ctas <= 0) return cudaSuccess;
    k_step_batch<T, MW, G><<<(unsigned)ctas, Shape<G>::kThreads, smem, st>>>(d_args, d_prefix, ngrids,
                                                                              d_queue, slot, grab);
    return cudaGetLastError();
  }
};

cudaError_t launch_step_batch(int precision, int group, const StepArgs *d_args, const int64_t *d_prefix,
                              int ngrids, int64_t total_tiles, unsigned long long *d_queue,
                              int nbins, int slot, int device, cudaStream_t st) {
  if (slot < 0 || slot >= kRotAhead) return cudaErrorInvalidValue;
  return dispatch_step(precision, nbins, group,
                       BatchLaunch{d_args, d_prefix, ngrids, total_tiles, d_queue, nbins, slot, device, st});
}

// ----------------------------------------------------------------------------
// Budget: sum of the per-CTA partials in a fixed order, in two levels (one
// CTA over every tile's partials took 51 us on C1's 35,746 tiles, as long as
// a tenth of a step): up to kBudgetBlocks CTAs each sum a fixed range of
// tiles, then one CTA sums their results; every sum is a fixed tree, so the
// result does not depend on the schedule.
// ----------------------------------------------------------------------------
// The four sums of a 256-thread CTA in a fixed tree: within each warp by
// shuffles, then the 8 warps' sums by warp 0; the result in thread 0.
__device__ __forceinline__ void budget_tree(double (*s)[8], double a[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], d);
  }
  if (lane == 0)
    for (int c = 0; c < 4; ++c) s[c][warp] = a[c];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      a[c] = lane < 8 ? s[c][lane] : 0.0;
#pragma unroll
      for (int d = 4; d > 0; d >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], d);
    }
  }
}

// CTA b: the partials of tiles [b per, min(nb, (b + 1) per)) into bsum[4 b ..].
__global__ void __launch_bounds__(256) k_budget_part(int64_t nb, int64_t per, const double *__restrict__ part,
                                                     double *__restrict__ bsum, int diffuse) {
  __shared__ double s[4][8];
  const int64_t lo = blockIdx.x * per, hi = lo + per < nb ? lo + per : nb;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    a[0] += part[4 * k];
    a[1] += part[4 * k + 1];
    a[2] += part[4 * k + 2];
    if (diffuse) a[3] += part[4 * k + 3];
  }
  budget_tree(s, a);
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; ++c) bsum[4 * blockIdx.x + c] = a[c];
}

// out[0..2]: the sums of the tiles' partials (absorbed, escaped, in flight,
// in stored units); out[4..7]: the budget as the C ABI reports it
// (emitted, absorbed, escaped, in flight in photons, carries included), also
// into copy_to[0..3] when given.
__global__ void __launch_bounds__(256) k_budget(int nblk, const double *__restrict__ bsum,
                                                double *__restrict__ out, double *__restrict__ copy_to,
                                                BudgetScale sc) {
  __shared__ double s[4][8];
  const int t = threadIdx.x;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  if (t < nblk)
    for (int c = 0; c < 4; ++c) a[c] = bsum[4 * t + c];
  budget_tree(s, a);
  if (t == 0) {
    out[0] = a[0];
    out[1] = a[1];
    out[2] = a[2];
    out[3] = a[3];
    // the sources' photons (host) and, with diffuse radiation, the photons
    // the recombining cells emitted
    double r[4];
    r[0] = sc.diffuse ? __dadd_rn(sc.emitted, __dmul_rn(a[3], sc.punit)) : sc.emitted;
    r[1] = __dadd_rn(__dmul_rn(a[0], sc.punit), sc.carry_abs);
    r[2] = __dadd_rn(__dmul_rn(a[1], sc.punit), sc.carry_esc);
    r[3] = sc.fly_mode == 2 ? __dmul_rn(a[2], sc.punit) : (sc.fly_mode == 1 ? sc.carry_fly : 0.0);
    for (int c = 0; c < 4; ++c) {
      out[4 + c] = r[c];
      if (copy_to) copy_to[c] = r[c];
    }
  }
}

cudaError_t launch_budget(DevGrid &g, const BudgetScale &sc, cudaStream_t st, double *copy_to) {
  const int64_t nb = g.nblocks > 0 ? g.nblocks : 0;
  int64_t nblk = (nb + 255) / 256;  // about 256 tiles per first-level CTA
  if (nblk > kBudgetBlocks) nblk = kBudgetBlocks;
  if (nblk < 1) nblk = 1;
  const int64_t per = (nb + nblk - 1) / nblk;
  k_budget_part<<<(unsigned)nblk, 256, 0, st>>>(nb, per, g.partials, g.bsum, sc.diffuse);
  k_budget<<<1, 256, 0, st>>>((int)nblk, g.bsum, g.budget_dev, copy_to, sc);
  return cudaGetLastError();
}

// Photons in flight towards every vertex after the last step (gather, FP64
// sum): the bins its in-edges' masks name, or (ballistic and combined
// transport) the edge packet where the sender was thick.
template <typename T, int MW>
__global__ void k_inflight(int64_t n, int nbins, int nbp, const int32_t *__restrict__ rp,
                           const Edge *__restrict__ edges, const T *__restrict__ P,
                           const uint32_t *__restrict__ M, const uint8_t *__restrict__ mode,
                           const T *__restrict__ B, double *__restrict__ out, bool all_ballistic) {
  const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  double s = 0.0;
  for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
    const Edge E = edges[e];
    if (all_ballistic || (mode && mode[E.col])) {
      if (lane == 0) s += (double)B[e];
      continue;
    }
    uint32_t m[MW];
    load_mask<MW>(M, e, m);
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      const int b = lane + 32 * w;
      if (b < nbins && ((m[w] >> lane) & 1u)) s += (double)P[(size_t)E.col * nbp + b];
    }
  }
  s = warp_sum_d(s);
  if (lane == 0) out[v] = s;
}

cudaError_t launch_inflight(DevGrid &g, int64_t step, cudaStream_t st) {
  // state after `step` steps lives in buffer (step - 1) & 1
  const int cur = (int)((step + 1) & 1);
  const unsigned blocks = (unsigned)((g.n * 32 + 255) / 256);
  const uint8_t *mode = g.mode[cur];  // null in direction-conserving transport
  const bool allb = g.transport == kTransportBallistic;
  if (g.precision == 0) {
    const double *P = static_cast<const double *>(g.P[cur]);
    const double *B = static_cast<const double *>(g.B[cur]);
    if (g.mw == 1) k_inflight<double, 1><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], mode, B, g.s_out, allb);
    else if (g.mw == 2) k_inflight<double, 2><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], mode, B, g.s_out, allb);
    else k_inflight<double, 4><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], mode, B, g.s_out, allb);
  } else {
    const float *P = static_cast<const float *>(g.P[cur]);
    const float *B = static_cast<const float *>(g.B[cur]);
    if (g.mw == 1) k_inflight<float, 1><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], mode, B, g.s_out, allb);
    else if (g.mw == 2) k_inflight<float, 2><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], mode, B, g.s_out, allb);
    else k_inflight<float, 4><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], mode, B, g.s_out, allb);
  }
  return cudaGetLastError();
}

}  // namespace sx
