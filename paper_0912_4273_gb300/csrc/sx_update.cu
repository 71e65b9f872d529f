// sx_update.cu -- kernels of the dynamic grid update (Sect. 2.1.4): vertices
// where the optical depth fell are removed down to a minimum resolution; the
// photons arriving at a removed vertex move to its nearest surviving
// neighbour, and the state of the survivors carries over to their new
// (re-triangulated) grid.
//
//   k_mark_candidates  not a sink, not a source, y < y_thresh, mean edge
//                      length < min_spacing
//   k_mark_removed     a candidate whose candidate neighbours all have larger
//                      ids (an independent set, decided in one pass)
//   k_count / k_scan / k_scatter   deterministic stream compaction of the
//                      removed ids (block counts, one scan, ordered scatter)
//   k_incoming_bins    photons in flight towards every vertex, per bin
//   k_targets, k_hand_over         nearest surviving neighbour, hand-over in
//                      ascending id of the removed vertices
//   k_carry            neutral fraction and photons of the survivors into
//                      the new grid's state
//   k_sum_rows         deterministic FP64 sum of a photon field
#include <algorithm>

#include "sx_internal.cuh"

namespace sx {

__global__ void k_mark_candidates(int64_t n, const double *__restrict__ y,
                                  const double *__restrict__ mean_len,
                                  const VConst *__restrict__ vc, double y_thresh,
                                  double min_spacing, uint8_t *__restrict__ cand) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const VConst c = vc[i];
  cand[i] = !(c.flags & 1) && c.src < 0 && y[i] < y_thresh && mean_len[i] < min_spacing;
}

__global__ void k_mark_removed(int64_t n, const int32_t *__restrict__ rp, const Edge *__restrict__ edges,
                               const uint8_t *__restrict__ cand, uint8_t *__restrict__ rem) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint8_t r = cand[i];
  if (r)
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int32_t j = edges[e].col;
      if (cand[j] && j < (int32_t)i) {
        r = 0;
        break;
      }
    }
  rem[i] = r;
}

constexpr int kScanBlock = 1024;

__global__ void k_count(int64_t n, const uint8_t *__restrict__ flag, int64_t *__restrict__ blk) {
  __shared__ int s[kScanBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int v = (i < n) ? (int)flag[i] : 0;
  const int c = __popc(__ballot_sync(0xffffffffu, v != 0));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanBlock / 32; ++w) t += s[w];
    blk[blockIdx.x] = t;
  }
}

// exclusive scan of the block counts (one block, sequential over chunks)
__global__ void k_scan(int64_t nblk, int64_t *__restrict__ blk, int64_t *__restrict__ total) {
  if (threadIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t c = blk[b];
    blk[b] = run;
    run += c;
  }
  *total = run;
}

__global__ void k_scatter(int64_t n, const uint8_t *__restrict__ flag, const int64_t *__restrict__ blk,
                          int32_t *__restrict__ out) {
  __shared__ int s[kScanBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int v = (i < n) ? (int)flag[i] : 0;
  const uint32_t bal = __ballot_sync(0xffffffffu, v != 0);
  if (lane == 0) s[w] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < kScanBlock / 32; ++k) {
      const int c = s[k];
      s[k] = run;
      run += c;
    }
  }
  __syncthreads();
  if (v) out[blk[blockIdx.x] + s[w] + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
}

template <typename T>
__device__ __forceinline__ void sum_add(T &acc, T &c, T x);
template <>
__device__ __forceinline__ void sum_add<double>(double &acc, double &, double x) {
  acc = __dadd_rn(acc, x);
}
template <>
__device__ __forceinline__ void sum_add<float>(float &acc, float &c, float x) {
  const float yv = __fsub_rn(x, c);
  const float t = __fadd_rn(acc, yv);
  c = __fsub_rn(__fsub_rn(t, acc), yv);
  acc = t;
}

// I[v][b] = photons routed to v in the last step (in-edges in ascending
// source order), as the next step's gather would see them.  Warp per vertex.
template <typename T, int MW>
__global__ void k_incoming_bins(int64_t n, int nbins, int nbp, const int32_t *__restrict__ rp,
                                const Edge *__restrict__ edges, const T *__restrict__ P,
                                const uint32_t *__restrict__ M, T *__restrict__ I) {
  const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n) return;
  T acc[MW], cmp[MW];
#pragma unroll
  for (int w = 0; w < MW; ++w) acc[w] = cmp[w] = T(0);
  for (int32_t e = rp[v]; e < rp[v + 1]; ++e) {
    const Edge E = edges[e];
    uint32_t m[MW];
    if constexpr (MW == 1) {
      m[0] = M[e];
    } else if constexpr (MW == 2) {
      const uint2 q = reinterpret_cast<const uint2 *>(M)[e];
      m[0] = q.x; m[1] = q.y;
    } else {
      const uint4 q = reinterpret_cast<const uint4 *>(M)[e];
      m[0] = q.x; m[1] = q.y; m[2] = q.z; m[3] = q.w;
    }
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      const int b = lane + 32 * w;
      if (b < nbins && ((m[w] >> lane) & 1u)) sum_add<T>(acc[w], cmp[w], P[(size_t)E.col * nbp + b]);
    }
  }
#pragma unroll
  for (int w = 0; w < MW; ++w) {
    const int b = lane + 32 * w;
    if (b < nbp) I[(size_t)v * nbp + b] = (b < nbins) ? acc[w] : T(0);
  }
}

// nearest surviving neighbour of every removed vertex (ties -> lowest id)
__global__ void k_targets(int64_t n, const int32_t *__restrict__ rp, const Edge *__restrict__ edges,
                          const double *__restrict__ pos, const uint8_t *__restrict__ rem,
                          int32_t *__restrict__ target) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int32_t best = -1;
  if (rem[r]) {
    double bestd = 0.0;
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t j = edges[e].col;
      if (rem[j]) continue;
      const double dx = __dsub_rn(pos[3 * (int64_t)j], pos[3 * r]);
      const double dy = __dsub_rn(pos[3 * (int64_t)j + 1], pos[3 * r + 1]);
      const double dz = __dsub_rn(pos[3 * (int64_t)j + 2], pos[3 * r + 2]);
      const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      if (best < 0 || d2 < bestd || (d2 == bestd && j < best)) {
        best = j;
        bestd = d2;
      }
    }
  }
  target[r] = best;
}

// a surviving vertex takes the photons of the removed neighbours that chose
// it, in ascending id of the removed vertex.  Warp per vertex.
template <typename T>
__global__ void k_hand_over(int64_t n, int nbins, int nbp, const int32_t *__restrict__ rp,
                            const Edge *__restrict__ edges, const uint8_t *__restrict__ rem,
                            const int32_t *__restrict__ target, T *__restrict__ I) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n || rem[t]) return;
  for (int32_t e = rp[t]; e < rp[t + 1]; ++e) {
    const int32_t r = edges[e].col;
    if (!rem[r] || target[r] != (int32_t)t) continue;
    for (int b = lane; b < nbins; b += 32)
      I[(size_t)t * nbp + b] = I[(size_t)t * nbp + b] + I[(size_t)r * nbp + b];
  }
}

// y_new[i] = y_old[old_of_new[i]];  I_new[i][:] = I_old[old_of_new[i]][:]
template <typename T>
__global__ void k_carry(int64_t n_new, int nbp, const int32_t *__restrict__ old_of_new,
                        const double *__restrict__ y_old, const T *__restrict__ I_old,
                        double *__restrict__ y_new, T *__restrict__ I_new) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n_new) return;
  const int64_t o = old_of_new[i];
  if (lane == 0) y_new[i] = y_old[o];
  for (int b = lane; b < nbp; b += 32) I_new[(size_t)i * nbp + b] = I_old[(size_t)o * nbp + b];
}

// sum of a photon field (rows of nbp, first nbins used), FP64, fixed order
template <typename T>
__global__ void k_sum_rows(int64_t n, int nbins, int nbp, const T *__restrict__ I,
                           double *__restrict__ part) {
  __shared__ double s[256];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int b = 0; b < nbins; ++b) a += (double)I[(size_t)i * nbp + b];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// photons of a carried field per vertex (readout right after a grid update)
template <typename T>
__global__ void k_row_totals(int64_t n, int nbins, int nbp, const T *__restrict__ I,
                             double *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int b = 0; b < nbins; ++b) a += (double)I[(size_t)i * nbp + b];
  out[i] = a;
}

cudaError_t launch_row_totals(int precision, int64_t n, int nbins, int nbp, const void *I,
                              double *out, cudaStream_t st) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (precision == 0)
    k_row_totals<double><<<blocks, 256, 0, st>>>(n, nbins, nbp, static_cast<const double *>(I), out);
  else
    k_row_totals<float><<<blocks, 256, 0, st>>>(n, nbins, nbp, static_cast<const float *>(I), out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
cudaError_t launch_mark(DevGrid &g, double y_thresh, double min_spacing, uint8_t *cand,
                        uint8_t *rem, int64_t *blk, int64_t *total, int32_t *out,
                        cudaStream_t st) {
  const int T = 256;
  const unsigned nb = (unsigned)((g.n + T - 1) / T);
  k_mark_candidates<<<nb, T, 0, st>>>(g.n, g.y, g.mean_len, g.vc, y_thresh, min_spacing, cand);
  k_mark_removed<<<nb, T, 0, st>>>(g.n, g.row_ptr, g.edges, cand, rem);
  const int64_t nblk = (g.n + kScanBlock - 1) / kScanBlock;
  k_count<<<(unsigned)nblk, kScanBlock, 0, st>>>(g.n, rem, blk);
  k_scan<<<1, 32, 0, st>>>(nblk, blk, total);
  k_scatter<<<(unsigned)nblk, kScanBlock, 0, st>>>(g.n, rem, blk, out);
  return cudaGetLastError();
}

template <typename T, int MW>
static cudaError_t incoming_t(DevGrid &g, int last, T *I, cudaStream_t st) {
  const unsigned blocks = (unsigned)((g.n * 32 + 255) / 256);
  k_incoming_bins<T, MW><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges,
                                                  static_cast<const T *>(g.P[last]), g.M[last], I);
  return cudaGetLastError();
}

cudaError_t launch_incoming_bins(DevGrid &g, int last, void *I, cudaStream_t st) {
  if (g.precision == 0) {
    double *d = static_cast<double *>(I);
    if (g.mw == 1) return incoming_t<double, 1>(g, last, d, st);
    if (g.mw == 2) return incoming_t<double, 2>(g, last, d, st);
    return incoming_t<double, 4>(g, last, d, st);
  }
  float *f = static_cast<float *>(I);
  if (g.mw == 1) return incoming_t<float, 1>(g, last, f, st);
  if (g.mw == 2) return incoming_t<float, 2>(g, last, f, st);
  return incoming_t<float, 4>(g, last, f, st);
}

cudaError_t launch_hand_over(DevGrid &g, const uint8_t *rem, int32_t *target, void *I,
                             cudaStream_t st) {
  const int T = 256;
  k_targets<<<(unsigned)((g.n + T - 1) / T), T, 0, st>>>(g.n, g.row_ptr, g.edges, g.pos, rem, target);
  const unsigned blocks = (unsigned)((g.n * 32 + 255) / 256);
  if (g.precision == 0)
    k_hand_over<double><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, rem,
                                                target, static_cast<double *>(I));
  else
    k_hand_over<float><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, g.row_ptr, g.edges, rem, target,
                                               static_cast<float *>(I));
  return cudaGetLastError();
}

cudaError_t launch_carry(int precision, int64_t n_new, int nbp, const int32_t *old_of_new,
                         const double *y_old, const void *I_old, double *y_new, void *I_new,
                         cudaStream_t st) {
  const unsigned blocks = (unsigned)((n_new * 32 + 255) / 256);
  if (blocks == 0) return cudaSuccess;
  if (precision == 0)
    k_carry<double><<<blocks, 256, 0, st>>>(n_new, nbp, old_of_new, y_old,
                                            static_cast<const double *>(I_old), y_new,
                                            static_cast<double *>(I_new));
  else
    k_carry<float><<<blocks, 256, 0, st>>>(n_new, nbp, old_of_new, y_old,
                                           static_cast<const float *>(I_old), y_new,
                                           static_cast<float *>(I_new));
  return cudaGetLastError();
}

cudaError_t launch_sum_rows(int precision, int64_t n, int nbins, int nbp, const void *I,
                            double *part, int nblk, cudaStream_t st) {
  if (precision == 0)
    k_sum_rows<double><<<nblk, 256, 0, st>>>(n, nbins, nbp, static_cast<const double *>(I), part);
  else
    k_sum_rows<float><<<nblk, 256, 0, st>>>(n, nbins, nbp, static_cast<const float *>(I), part);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Row stride change of the stored photons (a launch variant): buffer `buf`
// at stride g.nbp is copied, bins 0..nbins-1 of every row, into the other
// buffer at the new stride, then back in one contiguous copy.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void k_restride(int64_t n, int nbins, int from, const T *__restrict__ src, int to,
                           T *__restrict__ dst) {
  const int64_t total = n * nbins;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = k / nbins;
    const int b = (int)(k - v * nbins);
    dst[v * to + b] = src[v * from + b];
  }
}

cudaError_t launch_restride(DevGrid &g, int buf, int stride, cudaStream_t st) {
  if (stride == g.nbp || g.n <= 0) return cudaSuccess;
  const int64_t total = g.n * g.nbins;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 4096);
  const size_t tsz = g.precision == 0 ? sizeof(double) : sizeof(float);
  void *live = g.P[buf], *tmp = g.P[buf ^ 1];
  if (g.precision == 0)
    k_restride<double><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, static_cast<const double *>(live),
                                               stride, static_cast<double *>(tmp));
  else
    k_restride<float><<<blocks, 256, 0, st>>>(g.n, g.nbins, g.nbp, static_cast<const float *>(live),
                                              stride, static_cast<float *>(tmp));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(live, tmp, tsz * (size_t)stride * (size_t)g.n, cudaMemcpyDeviceToDevice, st);
}

}  // namespace sx
