// sx_ballistic.cu -- the step of ballistic transport alone (Sect. 2.2.2).
//
// Every vertex but the sinks (and ghosts) is thick in every step: the
// photons that reach it along in-edge j leave it, transmitted (O_j = f E_j),
// in equal parts w_j = O_j / |S_j| along the in-edge's straight set S_j (the
// <= 3 out-edges most aligned with its direction of travel); a source's
// photons of the step go in equal parts to all its neighbours.  No bins, no
// masks: the state is one packet per directed edge, B[e], at the receiver's
// in-edge index.  This is the same step as the ballistic tile of the
// combined kernel (sx_step.cu), with the bin phases left out:
//
//   prologue  the chemistry warp copies its 32 vertices' constants and y
//             with cp.async; each warp reads its group's row pointers and
//             flags.
//   phase A   lanes over each group's in-edges stage E_j = B_prev[e] in
//             shared memory (thick receivers only).
//   phase B   the chemistry warp, lane per vertex: N_in = sum of E_j in slot
//             order, then the source's (and the diffuse) photons of the
//             step; the cell's subcycles (vertex_chem); a sink sums its
//             in-edges' packets as it absorbs them.
//   phase C   lanes over each group's in-edges turn E_j into w_j (or an
//             escape when S_j is empty); lanes over its out-edges sum, for
//             out-slot k, the w_j of the in-edges whose set holds k, slot
//             order, plus the source's share, and store the sum at the
//             receiver's in-edge (B_next[twin]).
//   budget    as the combined kernel's tile: fixed-order sums of the
//             chemistry lanes' terms and the warps' escapes.
//
// Results are those of the combined kernel's ballistic tiles bit for bit in
// y and in every edge packet; a sink's absorbed photons are summed in edge
// order here (the combined kernel bins them first), so the budget agrees to
// rounding.
#include "sx_internal.cuh"
#include "sx_step_common.cuh"

#ifndef SX_BALLISTIC_GROUP
#define SX_BALLISTIC_GROUP 8  // vertices per warp: 4 warps per 32-vertex tile
#endif
#ifndef SX_BALLISTIC_WARPS_PER_SM
#define SX_BALLISTIC_WARPS_PER_SM 48  // resident warps per SM the registers are sized for
#endif

namespace sx {

template <int G>
struct BalShape {
  static constexpr int kGroup = G;            // vertices per warp
  static constexpr int kWarps = kTile / G;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kMinBlocks = SX_BALLISTIC_WARPS_PER_SM / kWarps;
  // staged in-edge packets per vertex: kMaxDeg slots, rows offset by 16
  // banks so that two consecutive vertices' first 16 slots do not collide
  static constexpr int kStride = kMaxDeg + 16;
};

template <typename T, int G>
__device__ __forceinline__ void ballistic_tile(const StepArgs &a, int64_t tile) {
  using S = BalShape<G>;
  constexpr int kGroup = S::kGroup, kWarps = S::kWarps;
  using BT = typename Bud<T>::type;
  __shared__ T s_E[kTile][S::kStride];
  __shared__ T s_f[kTile];
  __shared__ T s_S[kTile];
  __shared__ __align__(16) VConst s_vc[kTile];
  __shared__ __align__(16) double s_y[kTile];
  __shared__ double s_D[kTile];
  // the tile's running budget terms (absorbed, escaped, -, diffuse emitted),
  // fetched in the prologue so that the end of the tile does not wait on them
  __shared__ __align__(16) double s_run[4];
  __shared__ int32_t s_R[kWarps][kGroup + 1];
  __shared__ BT s_bud[3][kTile];
  __shared__ BT s_esc[kWarps];
  __shared__ BT s_sum[4];  // the tile's sums of s_bud and of s_D

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int cw = 0;  // the chemistry warp (lane per tile vertex)
  const int64_t v0 = tile * kTile;
  const int cur = (int)(a.tab->step & 1);
  if (warp == cw) {
    const int64_t nv = min((int64_t)32, a.n - v0);
    for (int i = lane; i < 2 * nv; i += 32)
      cp_async16(reinterpret_cast<char *>(s_vc) + 16 * i, reinterpret_cast<const char *>(a.vc + v0) + 16 * i);
    if (lane < nv) cp_async8(s_y + lane, a.y + v0 + lane);
    if (lane == 0) cp_async16(s_run, a.partials + 4 * tile);
    if (lane == 1) cp_async16(s_run + 2, a.partials + 4 * tile + 2);
    cp_async_commit();
  }
  const int g0 = warp * kGroup;
  const int64_t vg = v0 + g0;
  if (lane <= kGroup) s_R[warp][lane] = a.row_ptr[vg + lane < a.n ? vg + lane : a.n];
  // thick: neither sink nor ghost (past the grid: nothing)
  int vfl = kFlagGhost;
  if (lane < kGroup && vg + lane < a.n) vfl = a.vc[vg + lane].flags;
  const uint32_t thick = __ballot_sync(0xffffffffu, lane < kGroup && !(vfl & (kFlagSink | kFlagGhost)));
  __syncwarp();
  int32_t R[kGroup + 1];
#pragma unroll
  for (int g = 0; g <= kGroup; ++g) R[g] = s_R[warp][g];
  const T *__restrict__ Bp = static_cast<const T *>(a.B[cur ^ 1]);
  T *__restrict__ Bn = static_cast<T *>(a.B[cur]);

  // ---------------- phase A: the in-edges' packets ----------------
  for (int32_t e = R[0] + lane; e < R[kGroup]; e += 32) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < kGroup; ++q) g += (e >= R[q]) ? 1 : 0;
    if ((thick >> g) & 1u) {
      const T x = Bp[e];
      if (SX_INDEX_OK(e - R[g] < kMaxDeg, a.diag)) s_E[g0 + g][e - R[g]] = x;
      // phase C's tables of this edge, on their way to L1 while the
      // chemistry runs
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a.stb + e));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a.bpos + e));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a.edges + e));
    }
  }
  if (lane < kGroup && ((thick >> lane) & 1u))
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a.binv + 3 * (int64_t)s_R[warp][lane]));
  __syncthreads();

  // ---------------- phase B: N_in and chemistry, lane per vertex ----------------
  BT bud_abs{}, bud_sink{}, bud_tr{};
  unsigned diag_nsub = 0, diag_capped = 0;
  if (warp == cw) {
    cp_async_wait_all();
    __syncwarp();
    const int vl = lane;
    const int64_t v = v0 + vl;
    T f = T(0), src = T(0);
    double dv = 0.0;
    if (v < a.n) {
      const VConst c = s_vc[vl];
      const int gw = vl / kGroup, gi = vl % kGroup;
      const int32_t r0 = s_R[gw][gi], r1 = s_R[gw][gi + 1];
      if (a.diffuse) dv = a.dif[v];
      BT nin{};
      if (!(c.flags & (kFlagSink | kFlagGhost))) {
        // the source's photons of the step, then the diffuse photons the
        // cell made in the last one, as one packet of the vertex
        if (c.src >= 0) src = (T)__dmul_rn(a.src_rate[c.src], a.src_scale);
        if (dv > 0.0) src += (T)dv;
        const int dg = r1 - r0 < kMaxDeg ? r1 - r0 : kMaxDeg;
        for (int j = 0; j <= dg; ++j) {
          const T x = j < dg ? s_E[vl][j] : src;
          if constexpr (sizeof(T) == 8) nin = __dadd_rn(nin, x); else nin = ff_add(nin, x);
        }
      } else if (c.flags & kFlagSink) {
        // what reaches a sink, in edge order (and a source's photons there)
        for (int32_t e = r0; e < r1; ++e) {
          if constexpr (sizeof(T) == 8) nin = __dadd_rn(nin, Bp[e]); else nin = ff_add(nin, Bp[e]);
        }
        if (c.src >= 0) {
          const T x = (T)__dmul_rn(a.src_rate[c.src], a.src_scale);
          if constexpr (sizeof(T) == 8) nin = __dadd_rn(nin, x); else nin = ff_add(nin, x);
        }
      }
      int nsub = 0, capped = 0;
      f = vertex_chem<T>(a, c, v, s_y[vl], nin, dv, nsub, capped, bud_abs, bud_sink, bud_tr);
      diag_nsub = (unsigned)nsub;
      diag_capped = (unsigned)capped;
    }
    s_f[vl] = f;
    s_S[vl] = src;
    s_D[vl] = dv;
    s_bud[0][vl] = bud_abs;
    s_bud[1][vl] = bud_sink;
    s_bud[2][vl] = bud_tr;
  }
  __syncthreads();

  // ---------------- phase C: transmit and send ----------------
  Acc<T> esc;  // photons this lane lets escape
  for (int32_t e = R[0] + lane; e < R[kGroup]; e += 32) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < kGroup; ++q) g += (e >= R[q]) ? 1 : 0;
    if (((thick >> g) & 1u) && e - R[g] < kMaxDeg) {
      T &E = s_E[g0 + g][e - R[g]];
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
  if (lane < kGroup && ((thick >> lane) & 1u) && s_S[g0 + lane] != T(0)) {
    const T os = s_S[g0 + lane] * s_f[g0 + lane];  // a source sends to all its neighbours
    if (s_R[warp][lane + 1] == s_R[warp][lane]) esc.add(os);  // ... if it has any
  }
  __syncwarp();
  for (int32_t e = R[0] + lane; e < R[kGroup]; e += 32) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < kGroup; ++q) g += (e >= R[q]) ? 1 : 0;
    if ((thick >> g) & 1u) {
      const int32_t r0 = R[g];
      const int dg = R[g + 1] - r0;
      const unsigned ent = a.bpos[e];
      const uint8_t *lst = a.binv + 3 * (int64_t)r0 + (ent & 0xFFu);
      const T *Eg = s_E[g0 + g];
      CSum<T> acc;
      for (unsigned i = 0; i < (ent >> 8); ++i)
        if (SX_INDEX_OK(lst[i] < dg && lst[i] < kMaxDeg, a.diag)) acc.add(Eg[lst[i]]);
      const T Sv = s_S[g0 + g];
      if (Sv != T(0)) acc.add((Sv * s_f[g0 + g]) / (T)dg);
      const int32_t tw = a.edges[e].twin;
      if (SX_INDEX_OK((unsigned)tw < (unsigned)a.row_ptr[a.n], a.diag)) Bn[tw] = acc.value();
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
  // absorbed, passed to sinks plus escaped, in flight (transmitted minus the
  // escapes), and with diffuse radiation the photons the cells emitted; each
  // sum in a fixed order: lanes by a shuffle tree, warps ascending
  {
    using B = Bud<T>;
    BT e = esc.v;
    bool nz;
    if constexpr (sizeof(T) == 8) nz = e != 0.0; else nz = e.hi != 0.f;
    if (__any_sync(0xffffffffu, nz)) e = B::warp_sum(e); else e = BT{};
    if (lane == 0) s_esc[warp] = e;
    // the chemistry lanes' three terms summed by warps 1..3 at once (warp 0
    // when the tile has fewer warps), the diffuse photons by warp 4 (or 0)
    auto term_warp = [](int k) { return kWarps > 3 ? k + 1 : 0; };
    constexpr int wd = kWarps > 4 ? 4 : 0;
    for (int k = 0; k < 3; ++k) {
      if (warp == term_warp(k)) {
        const BT t = B::warp_sum(s_bud[k][lane]);
        if (lane == 0) s_sum[k] = t;
      }
    }
    if (warp == wd && a.diffuse) {
      const double d = v0 + lane < a.n ? s_D[lane] : 0.0;
      BT t;
      if constexpr (sizeof(T) == 8) {
        t = B::warp_sum(d);
      } else {  // the photons emitted, as double: hi + lo in float-float
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
}

template <typename T, int G>
__global__ void __launch_bounds__(BalShape<G>::kThreads, BalShape<G>::kMinBlocks)
    k_step_ballistic(const StepArgs a) {
  ballistic_tile<T, G>(a, blockIdx.x);
}

cudaError_t launch_step_ballistic(const StepArgs &a, int64_t ntiles, int precision, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  constexpr int G = SX_BALLISTIC_GROUP;
  if (precision == 0)
    k_step_ballistic<double, G><<<(unsigned)ntiles, BalShape<G>::kThreads, 0, st>>>(a);
  else
    k_step_ballistic<float, G><<<(unsigned)ntiles, BalShape<G>::kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sx
