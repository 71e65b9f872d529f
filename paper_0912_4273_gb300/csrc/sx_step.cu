// sx_step.cu -- per-step kernels of the SimpleX2 DCT sweep on sm_103a.
//
//  k_rotation   one CTA: random rotation of the direction bins (Philox4x32-10,
//               uniform quaternion), quantised rotated bins, and the map that
//               moves packets in flight to the closest bin of the new
//               orientation (Sect. 2.2.3).
//  k_step<T,MW> one launch per step, pull formulation.  A CTA owns a tile of
//               32 consecutive vertices:
//     phase 1   warp per vertex: gather the photons routed to it in the
//               previous step (reverse edges, per-edge bin masks, fixed order,
//               Kahan in FP32), move them to the new orientation, add the
//               sources (Sect. 4.3), sum N_in;
//     phase 2   lane per vertex: subcycled photoionisation / recombination in
//               FP64 (Sect. 4.5), transmitted fraction f;
//     phase 3   warp per vertex: O = f I; associate every bin with the edge of
//               largest quantised dot product; split O over the <= 3 most
//               straightforward neighbours of that edge (store O / |S| once
//               and one bin mask per outgoing edge); budget partials.
//  k_budget     deterministic reduction of the per-CTA budget partials.
//  k_inflight   photons in flight towards every vertex (readout).
#include <float.h>

#include "sx_internal.cuh"

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

__global__ void __launch_bounds__(128) k_rotation(int nbins, const double *__restrict__ bins,
                                                  uint64_t seed, int64_t step, int unrotated,
                                                  StepTables *__restrict__ out) {
  __shared__ double sR[9], sRp[9];
  __shared__ int s_att;
  __shared__ int s_qn[kMaxBins][3], s_qo[kMaxBins][3];
  __shared__ int s_map[kMaxBins];
  const int t = threadIdx.x;
  if (t == 0) {
    int att = 0, attp = 0;
    if (unrotated) {
      for (int i = 0; i < 9; ++i) sR[i] = sRp[i] = (i % 4 == 0) ? 1.0 : 0.0;
    } else {
      rotation_matrix(seed, step, sR, &att);
      if (step > 0) rotation_matrix(seed, step - 1, sRp, &attp);
      else
        for (int i = 0; i < 9; ++i) sRp[i] = sR[i];
    }
    s_att = att;
  }
  __syncthreads();
  for (int b = t; b < nbins; b += blockDim.x) {
    int q[3];
    rotate_quantise(sR, bins + 3 * b, q);
    s_qn[b][0] = q[0]; s_qn[b][1] = q[1]; s_qn[b][2] = q[2];
    out->qb[b] = make_float4((float)q[0], (float)q[1], (float)q[2], 0.f);
    rotate_quantise(sRp, bins + 3 * b, q);
    s_qo[b][0] = q[0]; s_qo[b][1] = q[1]; s_qo[b][2] = q[2];
  }
  __syncthreads();
  // closest new bin of every old bin (ties -> lowest index)
  for (int b = t; b < nbins; b += blockDim.x) {
    int best = 0, bestd = 0;
    for (int b2 = 0; b2 < nbins; ++b2) {
      const int d = s_qn[b2][0] * s_qo[b][0] + s_qn[b2][1] * s_qo[b][1] + s_qn[b2][2] * s_qo[b][2];
      if (b2 == 0 || d > bestd) {
        best = b2;
        bestd = d;
      }
    }
    s_map[b] = best;
  }
  __syncthreads();
  if (t == 0) {
    int o = 0;
    for (int b2 = 0; b2 < nbins; ++b2) {
      out->inv_off[b2] = o;
      for (int b = 0; b < nbins; ++b)
        if (s_map[b] == b2) out->inv_idx[o++] = b;
    }
    out->inv_off[nbins] = o;
    out->attempts = s_att;
    out->remap = (!unrotated && step > 0) ? 1 : 0;
  }
}

cudaError_t launch_rotation(DevGrid &g, const double *bins_dev, uint64_t seed, int64_t step,
                            int unrotated, cudaStream_t st) {
  k_rotation<<<1, 128, 0, st>>>(g.nbins, bins_dev, seed, step, unrotated,
                                g.tabs + (unrotated ? 1 : 0));
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Chemistry of one cell over one step; IEEE FP64 operations in the order of
// the rate-equation update (no contraction).  Returns the transmitted fraction.
// ----------------------------------------------------------------------------
__device__ double chem_cell(double &y_io, double N_in, double dt, double A, double tau_max,
                            double R0, double fc, double tol, int max_sub, int &nsub,
                            int &capped) {
  double y = y_io;
  const double F = __ddiv_rn(N_in, dt);
  double t_left = dt;
  double trans_int = 0.0;
  nsub = 0;
  capped = 0;
  while (t_left > 0.0) {
    const double tau = __dmul_rn(tau_max, y);
    const double tr = exp(-tau);
    const double ab = -expm1(-tau);
    const double ion = __ddiv_rn(__dmul_rn(F, ab), A);
    const double x = __dsub_rn(1.0, y);
    const double rec = __dmul_rn(__dmul_rn(R0, x), x);
    const double gam = (y > 0.0) ? __ddiv_rn(ion, y) : __ddiv_rn(__dmul_rn(F, tau_max), A);
    const double rate = __dadd_rn(gam, __dmul_rn(R0, x));
    double h = t_left;
    if (rate > 0.0) {
      const double hc = __ddiv_rn(fc, rate);
      if (hc < h) h = hc;
    }
    const double y_new = __dadd_rn(y, __dmul_rn(__dsub_rn(rec, ion), h));
    trans_int = __dadd_rn(trans_int, __dmul_rn(tr, h));
    t_left = (h == t_left) ? 0.0 : __dsub_rn(t_left, h);
    nsub++;
    const bool eq = fabs(__dsub_rn(y_new, y)) <= __dmul_rn(tol, y_new);
    y = y_new;
    if (t_left > 0.0 && (eq || nsub >= max_sub)) {
      if (!eq) capped = 1;
      trans_int = __dadd_rn(trans_int, __dmul_rn(tr, t_left));
      t_left = 0.0;
    }
  }
  y_io = y;
  return __ddiv_rn(trans_int, dt);
}

// ----------------------------------------------------------------------------
// Mask words of one edge.
// ----------------------------------------------------------------------------
template <int MW>
__device__ __forceinline__ void load_mask(const uint32_t *__restrict__ M, int64_t e, uint32_t m[MW]) {
  if constexpr (MW == 1) {
    m[0] = __ldg(M + e);
  } else if constexpr (MW == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(M) + e);
    m[0] = v.x; m[1] = v.y;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(M) + e);
    m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
  }
}
template <int MW>
__device__ __forceinline__ void store_mask(uint32_t *__restrict__ M, int64_t e, const uint32_t m[MW]) {
  if constexpr (MW == 1) {
    M[e] = m[0];
  } else if constexpr (MW == 2) {
    reinterpret_cast<uint2 *>(M)[e] = make_uint2(m[0], m[1]);
  } else {
    reinterpret_cast<uint4 *>(M)[e] = make_uint4(m[0], m[1], m[2], m[3]);
  }
}

template <typename T>
__device__ __forceinline__ void acc_add(T &acc, T &c, T x);
template <>
__device__ __forceinline__ void acc_add<double>(double &acc, double &, double x) {
  acc = __dadd_rn(acc, x);  // FP64: plain sum in the fixed edge order
}
template <>
__device__ __forceinline__ void acc_add<float>(float &acc, float &c, float x) {
  // Kahan-compensated FP32 sum
  const float yv = __fsub_rn(x, c);
  const float t = __fadd_rn(acc, yv);
  c = __fsub_rn(__fsub_rn(t, acc), yv);
  acc = t;
}

struct StepArgs {
  int64_t n;
  int nbins, nbp;
  double dt;
  double punit;      // photons per stored unit (a power of two; 1 in FP64 mode)
  double inv_punit;
  double fc, tol;
  int max_sub;
  const int32_t *__restrict__ row_ptr;
  const Edge *__restrict__ edges;
  const VConst *__restrict__ vc;
  double *__restrict__ y;
  const void *__restrict__ P_prev;
  void *__restrict__ P_next;
  const uint32_t *__restrict__ M_prev;
  uint32_t *__restrict__ M_next;
  const StepTables *__restrict__ tab;
  const double *__restrict__ src_rate;
  double *__restrict__ partials;
  unsigned long long *__restrict__ diag;
};

template <typename T, int MW>
__global__ void __launch_bounds__(kThreads) k_step(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s_I = reinterpret_cast<T *>(smem_raw);  // [kTile][nbp]
  __shared__ float4 s_qb[kMaxBins];
  __shared__ int32_t s_inv_off[kMaxBins + 1];
  __shared__ int32_t s_inv_idx[kMaxBins];
  __shared__ double s_Nin[kTile];
  __shared__ double s_f[kTile];
  __shared__ float4 s_eq[kWarps][kMaxDeg];
  __shared__ uint32_t s_am[kWarps][kMaxDeg][MW];
  __shared__ double s_bud[kWarps][3];
  __shared__ double s_sink_esc;
  __shared__ int s_remap;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nbins = a.nbins, nbp = a.nbp;
  for (int b = tid; b < nbins; b += kThreads) {
    s_qb[b] = a.tab->qb[b];
    s_inv_idx[b] = a.tab->inv_idx[b];
  }
  for (int b = tid; b <= nbins; b += kThreads) s_inv_off[b] = a.tab->inv_off[b];
  if (tid == 0) s_remap = a.tab->remap;
  __syncthreads();

  const int64_t v0 = (int64_t)blockIdx.x * kTile;
  const T *__restrict__ Pp = static_cast<const T *>(a.P_prev);
  T *__restrict__ Pn = static_cast<T *>(a.P_next);

  // ---------------- phase 1: gather, remap, sources, N_in ----------------
  for (int vl = warp; vl < kTile; vl += kWarps) {
    const int64_t v = v0 + vl;
    T *row = s_I + (size_t)vl * nbp;
    if (v >= a.n) {
      if (lane == 0) s_Nin[vl] = 0.0;
      continue;
    }
    T acc[MW], cmp[MW];
#pragma unroll
    for (int w = 0; w < MW; ++w) acc[w] = cmp[w] = T(0);
    const int32_t r0 = a.row_ptr[v], r1 = a.row_ptr[v + 1];
    for (int32_t e0 = r0; e0 < r1; e0 += 32) {
      // lane k fetches the reverse edge and source of in-edge e0 + k
      int32_t my_src = 0;
      uint32_t my_m[MW];
#pragma unroll
      for (int w = 0; w < MW; ++w) my_m[w] = 0u;
      if (e0 + lane < r1) {
        const Edge E = a.edges[e0 + lane];
        my_src = E.col;
        load_mask<MW>(a.M_prev, E.twin, my_m);
      }
      const int cnt = min(32, r1 - e0);
      for (int k = 0; k < cnt; ++k) {
        const int32_t src = __shfl_sync(0xffffffffu, my_src, k);
        const T *__restrict__ Ps = Pp + (size_t)src * nbp;
#pragma unroll
        for (int w = 0; w < MW; ++w) {
          const uint32_t mw = __shfl_sync(0xffffffffu, my_m[w], k);
          const int b = lane + 32 * w;
          if ((mw >> lane) & 1u) acc_add<T>(acc[w], cmp[w], Ps[b]);
        }
      }
    }
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      const int b = lane + 32 * w;
      if (b < nbp) row[b] = (b < nbins) ? acc[w] : T(0);
    }
    __syncwarp();
    // move packets to the closest bin of this step's orientation, add sources
    T nv[MW];
    const int src = a.vc[v].src;
    const double share =
        src >= 0 ? __dmul_rn(__ddiv_rn(__dmul_rn(a.src_rate[src], a.dt), (double)nbins), a.inv_punit)
                 : 0.0;
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      const int b = lane + 32 * w;
      T s = T(0);
      if (b < nbins) {
        if (s_remap) {
          for (int j = s_inv_off[b]; j < s_inv_off[b + 1]; ++j) s = s + row[s_inv_idx[j]];
        } else {
          s = row[b];
        }
        if (src >= 0) s = s + (T)share;
      }
      nv[w] = s;
    }
    __syncwarp();
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      const int b = lane + 32 * w;
      if (b < nbins) row[b] = nv[w];
    }
    __syncwarp();
    if constexpr (sizeof(T) == 8) {
      // FP64: sequential sum over bins, the order of the plain definition
      if (lane == 0) {
        double s = 0.0;
        for (int b = 0; b < nbins; ++b) s = __dadd_rn(s, (double)row[b]);
        s_Nin[vl] = s;
      }
    } else {
      FF s{0.f, 0.f};
#pragma unroll
      for (int w = 0; w < MW; ++w) s = ff_add(s, (float)nv[w]);
      s = ff_warp_sum(s);
      if (lane == 0) s_Nin[vl] = ff_to_double(s);
    }
  }
  __syncthreads();

  // ---------------- phase 2: chemistry, lane per vertex ----------------
  if (warp == 0) {
    const int64_t v = v0 + lane;
    double f = 0.0, sink_esc = 0.0;
    int nsub = 0, capped = 0;
    if (v < a.n) {
      const VConst c = a.vc[v];
      const double Nin = __dmul_rn(s_Nin[lane], a.punit);  // photons
      if (c.flags & 1) {
        sink_esc = s_Nin[lane];  // stored units, like every budget partial
      } else {
        double yv = a.y[v];
        f = chem_cell(yv, Nin, a.dt, c.A, c.tau_max, c.R0, a.fc, a.tol, a.max_sub, nsub, capped);
        a.y[v] = yv;
      }
    }
    s_f[lane] = f;
    sink_esc = warp_sum_d(sink_esc);
    unsigned ns = (unsigned)nsub, nc = (unsigned)capped;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      ns += __shfl_down_sync(0xffffffffu, ns, d);
      nc += __shfl_down_sync(0xffffffffu, nc, d);
    }
    if (lane == 0) {
      s_sink_esc = sink_esc;
      if (ns) atomicAdd(&a.diag[kDiagSubcycles], (unsigned long long)ns);
      if (nc) atomicAdd(&a.diag[kDiagCapped], (unsigned long long)nc);
    }
  }
  __syncthreads();

  // ---------------- phase 3: transmit, associate, route ----------------
  double w_abs = 0.0, w_esc = 0.0, w_fly = 0.0;  // lane 0 of each warp
  for (int vl = warp; vl < kTile; vl += kWarps) {
    const int64_t v = v0 + vl;
    if (v >= a.n) continue;
    const T *row = s_I + (size_t)vl * nbp;
    T *__restrict__ Pv = Pn + (size_t)v * nbp;
    const int32_t r0 = a.row_ptr[v], r1 = a.row_ptr[v + 1];
    const int deg = r1 - r0;
    const int flags = a.vc[v].flags;
    const double Nin = s_Nin[vl];
    if ((flags & 1) || deg == 0 || deg > kMaxDeg) {
      // sinks pass nothing on; a vertex without edges loses what it transmits
      double esc = 0.0;
      if (!(flags & 1)) {
        const T f = (T)s_f[vl];
        double o = 0.0;
        for (int b = lane; b < nbins; b += 32) o += (double)(row[b] * f);
        o = warp_sum_d(o);
        esc = o;
        if (lane == 0) w_abs += Nin - o;
      }
      if (lane == 0) w_esc += esc;
      for (int b = lane; b < nbp; b += 32) Pv[b] = T(0);
      for (int k = lane; k < deg; k += 32) {
        uint32_t z[MW];
#pragma unroll
        for (int w = 0; w < MW; ++w) z[w] = 0u;
        store_mask<MW>(a.M_next, (int64_t)r0 + k, z);
      }
      continue;
    }
    // stage the vertex's edges: q * 256 as exact floats, straight table in w
    for (int k = lane; k < deg; k += 32) {
      const Edge E = a.edges[r0 + k];
      uint32_t stw;
      memcpy(&stw, &E.st, 4);
      s_eq[warp][k] = make_float4((float)E.q.x * 256.f, (float)E.q.y * 256.f,
                                  (float)E.q.z * 256.f, __uint_as_float(stw));
#pragma unroll
      for (int w = 0; w < MW; ++w) s_am[warp][k][w] = 0u;
    }
    __syncwarp();
    const T f = (T)s_f[vl];
    double o_sum = 0.0, o_fly = 0.0, o_esc = 0.0;
    FF fo{0.f, 0.f}, ffly{0.f, 0.f}, fesc{0.f, 0.f};
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      const int b = lane + 32 * w;
      if (b < nbins) {
        const T O = row[b] * f;
        const float4 qb = s_qb[b];
        float best = -FLT_MAX;
        for (int k = 0; k < deg; ++k) {
          const float4 qe = s_eq[warp][k];
          // (q_e . q_b) * 256 + (255 - k): exact integer in FP32; the max
          // picks the largest dot and, among equal dots, the lowest slot
          const float d = fmaf(qe.x, qb.x, fmaf(qe.y, qb.y, fmaf(qe.z, qb.z, (float)(255 - k))));
          best = fmaxf(best, d);
        }
        const int kb = 255 - ((int)best & 255);
        const uint32_t stw = __float_as_uint(s_eq[warp][kb].w);
        const int cnt = (int)(stw >> 24);
        T P = T(0);
        if (cnt == 0) {
          if constexpr (sizeof(T) == 8) o_esc += (double)O; else fesc = ff_add(fesc, (float)O);
        } else {
          P = O / (T)cnt;
          if constexpr (sizeof(T) == 8) o_fly += (double)O; else ffly = ff_add(ffly, (float)O);
          for (int j = 0; j < cnt; ++j) {
            const int s = (int)((stw >> (8 * j)) & 0xFFu);
            atomicOr(&s_am[warp][s][w], 1u << lane);
          }
        }
        if constexpr (sizeof(T) == 8) o_sum += (double)O; else fo = ff_add(fo, (float)O);
        Pv[b] = P;
      } else if (b < nbp) {
        Pv[b] = T(0);
      }
    }
    __syncwarp();
    for (int k = lane; k < deg; k += 32) {
      uint32_t m[MW];
#pragma unroll
      for (int w = 0; w < MW; ++w) m[w] = s_am[warp][k][w];
      store_mask<MW>(a.M_next, (int64_t)r0 + k, m);
    }
    if constexpr (sizeof(T) == 8) {
      o_sum = warp_sum_d(o_sum);
      o_fly = warp_sum_d(o_fly);
      o_esc = warp_sum_d(o_esc);
    } else {
      o_sum = ff_to_double(ff_warp_sum(fo));
      o_fly = ff_to_double(ff_warp_sum(ffly));
      o_esc = ff_to_double(ff_warp_sum(fesc));
    }
    if (lane == 0) {
      w_abs += Nin - o_sum;
      w_fly += o_fly;
      w_esc += o_esc;
    }
    __syncwarp();
  }
  if (lane == 0) {
    s_bud[warp][0] = w_abs;
    s_bud[warp][1] = w_esc;
    s_bud[warp][2] = w_fly;
  }
  __syncthreads();
  if (tid == 0) {
    double ab = 0.0, es = s_sink_esc, fl = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      ab += s_bud[w][0];
      es += s_bud[w][1];
      fl += s_bud[w][2];
    }
    double *p = a.partials + 4 * (int64_t)blockIdx.x;
    p[0] += ab;
    p[1] += es;
    p[2] = fl;
  }
}

template <typename T, int MW>
static cudaError_t launch_step_t(DevGrid &g, int64_t step, double dt, double fc, double tol,
                                 int max_sub, cudaStream_t st) {
  StepArgs a;
  a.n = g.n;
  a.nbins = g.nbins;
  a.nbp = g.nbp;
  a.dt = dt;
  a.punit = g.punit;
  a.inv_punit = 1.0 / g.punit;
  a.fc = fc;
  a.tol = tol;
  a.max_sub = max_sub;
  a.row_ptr = g.row_ptr;
  a.edges = g.edges;
  a.vc = g.vc;
  a.y = g.y;
  const int cur = (int)(step & 1), prev = cur ^ 1;
  a.P_prev = g.P[prev];
  a.P_next = g.P[cur];
  a.M_prev = g.M[prev];
  a.M_next = g.M[cur];
  a.tab = g.tabs;
  a.src_rate = g.src_rate;
  a.partials = g.partials;
  a.diag = g.diag;
  const size_t smem = sizeof(T) * (size_t)kTile * g.nbp;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_step<T, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    configured = true;
  }
  k_step<T, MW><<<(unsigned)g.nblocks, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_step(DevGrid &g, int64_t step, double dt, double chem_frac, double chem_tol,
                        int chem_max_sub, cudaStream_t st) {
  if (g.precision == 0) {
    if (g.mw == 1) return launch_step_t<double, 1>(g, step, dt, chem_frac, chem_tol, chem_max_sub, st);
    if (g.mw == 2) return launch_step_t<double, 2>(g, step, dt, chem_frac, chem_tol, chem_max_sub, st);
    return launch_step_t<double, 4>(g, step, dt, chem_frac, chem_tol, chem_max_sub, st);
  }
  if (g.mw == 1) return launch_step_t<float, 1>(g, step, dt, chem_frac, chem_tol, chem_max_sub, st);
  if (g.mw == 2) return launch_step_t<float, 2>(g, step, dt, chem_frac, chem_tol, chem_max_sub, st);
  return launch_step_t<float, 4>(g, step, dt, chem_frac, chem_tol, chem_max_sub, st);
}

// ----------------------------------------------------------------------------
// Budget: sum of the per-CTA partials in a fixed order.
// ----------------------------------------------------------------------------
__global__ void k_budget(int64_t nb, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double s[3][256];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int64_t k = threadIdx.x; k < nb; k += blockDim.x) {
    a0 += part[4 * k];
    a1 += part[4 * k + 1];
    a2 += part[4 * k + 2];
  }
  s[0][threadIdx.x] = a0;
  s[1][threadIdx.x] = a1;
  s[2][threadIdx.x] = a2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s[0][0];
    out[1] = s[1][0];
    out[2] = s[2][0];
  }
}

cudaError_t launch_budget(DevGrid &g, cudaStream_t st) {
  k_budget<<<1, 256, 0, st>>>(g.nblocks, g.partials, g.budget_dev);
  return cudaGetLastError();
}

// Photons in flight towards every vertex after the last step (gather, FP64 sum).
template <typename T, int MW>
__global__ void k_inflight(int64_t n, int nbins, int nbp, const int32_t *__restrict__ rp,
                           const Edge *__restrict__ edges, const T *__restrict__ P,
                           const uint32_t *__restrict__ M, double *__restrict__ out) {
  const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  double s = 0.0;
  for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
    const Edge E = edges[e];
    uint32_t m[MW];
    load_mask<MW>(M, E.twin, m);
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
  if (g.precision == 0) {
    const double *P = static_cast<const double *>(g.P[cur]);
    if (g.mw == 1) k_inflight<double, 1><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], g.s_out);
    else if (g.mw == 2) k_inflight<double, 2><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], g.s_out);
    else k_inflight<double, 4><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], g.s_out);
  } else {
    const float *P = static_cast<const float *>(g.P[cur]);
    if (g.mw == 1) k_inflight<float, 1><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], g.s_out);
    else if (g.mw == 2) k_inflight<float, 2><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], g.s_out);
    else k_inflight<float, 4><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, P, g.M[cur], g.s_out);
  }
  return cudaGetLastError();
}

}  // namespace sx
