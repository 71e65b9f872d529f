// sx_setup.cu -- device layout of one grid and the load-time kernels:
// CSR checks, reverse edges, quantised edge directions, most-straightforward
// neighbour table (Sect. 2.2.2), path correction kappa (Sect. 2.2.3) and the
// per-vertex constants of the optical depth (Sect. 4.4, Eq. optical_depth).
#include <algorithm>

#include "sx_internal.cuh"

namespace sx {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout make_layout(int64_t n, int64_t nnz, int nbins, int precision, int transport) {
  Layout L{};
  const int nbp = bin_stride_aligned(nbins);  // room for either row stride (bin_stride_*)
  const int mw = nbins <= 32 ? 1 : (nbins <= 64 ? 2 : 4);
  const size_t tsz = precision == 0 ? sizeof(double) : sizeof(float);
  L.nblocks = (n + kTile - 1) / kTile;
  L.nblocks_kappa = (n + 255) / 256;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + std::max<size_t>(bytes, 1), 256);
    return at;
  };
  L.off_pos = take(sizeof(double) * 3 * n);
  L.off_row_ptr = take(sizeof(int32_t) * (n + 1));
  L.off_edges = take(sizeof(Edge) * nnz);
  L.off_vc = take(sizeof(VConst) * n);
  L.off_mean_len = take(sizeof(double) * n);
  L.off_y = take(sizeof(double) * n);
  L.off_dif = take(sizeof(double) * n);
  L.off_P0 = take(tsz * nbp * n);
  L.off_P1 = take(tsz * nbp * n);
  L.off_M0 = take(sizeof(uint32_t) * mw * nnz);
  L.off_M1 = take(sizeof(uint32_t) * mw * nnz);
  L.off_partials = take(sizeof(double) * 4 * L.nblocks);
  L.off_tabs = take(sizeof(StepTables) * kTabCount);
  L.off_src = take(sizeof(double) * kMaxSources);
  L.off_share = take(sizeof(double) * kMaxSources);
  L.off_share_f = take(sizeof(float) * kMaxSources);
  L.off_steps = take(sizeof(unsigned long long));
  L.off_incoming = take(sizeof(int));
  L.off_diag = take(sizeof(unsigned long long) * kDiagCount);
  L.off_kpart = take(sizeof(double) * 2 * L.nblocks_kappa);
  L.off_kappa = take(sizeof(double));
  L.off_budget = take(sizeof(double) * 8);
  L.off_bsum = take(sizeof(double) * 4 * kBudgetBlocks);
  L.off_bhist = take(sizeof(double) * 4 * kBudgetHist);
  L.off_s_row_ptr = take(sizeof(int64_t) * (n + 1));
  L.off_s_col = take(sizeof(int32_t) * nnz);
  L.off_s_nH = take(sizeof(double) * n);
  L.off_s_vol = take(sizeof(double) * n);
  L.off_s_y0 = take(sizeof(double) * n);
  L.off_s_flags = take(n);
  L.off_s_ev = take(sizeof(float4) * nnz);
  L.off_s_out = take(sizeof(double) * n);
  if (transport != 0) {  // ballistic and combined transport: edge packets, modes, straight sets
    L.off_B0 = take(tsz * nnz);
    L.off_B1 = take(tsz * nnz);
    L.off_mode0 = take(n);
    L.off_mode1 = take(n);
    L.off_stb = take(sizeof(uint32_t) * nnz);
    L.off_bpos = take(sizeof(uint16_t) * nnz);
    L.off_binv = take(3 * (size_t)nnz);
  }
  L.total = o;
  return L;
}

void bind_layout(DevGrid &g, void *base, const Layout &L) {
  char *b = static_cast<char *>(base);
  g.pos = reinterpret_cast<double *>(b + L.off_pos);
  g.row_ptr = reinterpret_cast<int32_t *>(b + L.off_row_ptr);
  g.edges = reinterpret_cast<Edge *>(b + L.off_edges);
  g.vc = reinterpret_cast<VConst *>(b + L.off_vc);
  g.mean_len = reinterpret_cast<double *>(b + L.off_mean_len);
  g.y = reinterpret_cast<double *>(b + L.off_y);
  g.dif = reinterpret_cast<double *>(b + L.off_dif);
  g.P[0] = b + L.off_P0;
  g.P[1] = b + L.off_P1;
  g.M[0] = reinterpret_cast<uint32_t *>(b + L.off_M0);
  g.M[1] = reinterpret_cast<uint32_t *>(b + L.off_M1);
  g.partials = reinterpret_cast<double *>(b + L.off_partials);
  g.nblocks = L.nblocks;
  g.tabs = reinterpret_cast<StepTables *>(b + L.off_tabs);
  g.src_rate = reinterpret_cast<double *>(b + L.off_src);
  g.src_share = reinterpret_cast<double *>(b + L.off_share);
  g.src_share_f = reinterpret_cast<float *>(b + L.off_share_f);
  g.steps_done = reinterpret_cast<unsigned long long *>(b + L.off_steps);
  g.incoming = reinterpret_cast<int *>(b + L.off_incoming);
  g.diag = reinterpret_cast<unsigned long long *>(b + L.off_diag);
  g.kappa_part = reinterpret_cast<double *>(b + L.off_kpart);
  g.nblocks_kappa = L.nblocks_kappa;
  g.kappa_dev = reinterpret_cast<double *>(b + L.off_kappa);
  g.budget_dev = reinterpret_cast<double *>(b + L.off_budget);
  g.bsum = reinterpret_cast<double *>(b + L.off_bsum);
  g.bhist = reinterpret_cast<double *>(b + L.off_bhist);
  g.s_row_ptr = reinterpret_cast<int64_t *>(b + L.off_s_row_ptr);
  g.s_col = reinterpret_cast<int32_t *>(b + L.off_s_col);
  g.s_nH = reinterpret_cast<double *>(b + L.off_s_nH);
  g.s_vol = reinterpret_cast<double *>(b + L.off_s_vol);
  g.s_y0 = reinterpret_cast<double *>(b + L.off_s_y0);
  g.s_flags = reinterpret_cast<uint8_t *>(b + L.off_s_flags);
  g.s_ev = reinterpret_cast<float4 *>(b + L.off_s_ev);
  g.s_out = reinterpret_cast<double *>(b + L.off_s_out);
  if (L.off_stb) {
    g.B[0] = b + L.off_B0;
    g.B[1] = b + L.off_B1;
    g.mode[0] = reinterpret_cast<uint8_t *>(b + L.off_mode0);
    g.mode[1] = reinterpret_cast<uint8_t *>(b + L.off_mode1);
    g.stb = reinterpret_cast<uint32_t *>(b + L.off_stb);
    g.bpos = reinterpret_cast<uint16_t *>(b + L.off_bpos);
    g.binv = reinterpret_cast<uint8_t *>(b + L.off_binv);
  } else {
    g.B[0] = g.B[1] = nullptr;
    g.mode[0] = g.mode[1] = nullptr;
    g.stb = nullptr;
    g.bpos = nullptr;
    g.binv = nullptr;
  }
}

// ----------------------------------------------------------------------------
// Ballistic straight sets (Sect. 2.2.2): photons that came in along the edge
// from neighbour j (travelling along -q_ij) go on to the <= 3 slots k with
// the largest positive quantised dot q_ik . (-q_ij), ties -> lowest slot.
// Packed as slot bytes (x, y, z) and the count in the top byte.  Rows longer
// than 255 slots (sinks', which never send) get no set.
// ----------------------------------------------------------------------------
//   The inverse: for out-slot k of vertex i, the in-edges j whose set holds k,
//   ascending, as bytes at binv[3 r0 + off] (r0 the row start, 3 bytes per
//   edge of the row) with bpos[r0 + k] = off | count << 8.
__global__ void k_ballistic_tables(int64_t n, const int32_t *__restrict__ rp, const Edge *__restrict__ edges,
                                   uint32_t *__restrict__ stb, uint16_t *__restrict__ bpos,
                                   uint8_t *__restrict__ binv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r0 = rp[i], r1 = rp[i + 1];
  for (int32_t e = r0; e < r1; ++e) {
    const char4 qe = edges[e].q;
    int best[3];
    int slot[3];
    int cnt = 0;
    if (r1 - r0 <= 255) {
      for (int32_t e2 = r0; e2 < r1; ++e2) {
        const char4 q2 = edges[e2].q;
        const int d = -((int)qe.x * q2.x + (int)qe.y * q2.y + (int)qe.z * q2.z);
        if (d <= 0) continue;
        int at = cnt;
        while (at > 0 && d > best[at - 1]) at--;
        if (at >= 3) continue;
        const int last = cnt < 3 ? cnt : 2;
        for (int m = last; m > at; --m) {
          best[m] = best[m - 1];
          slot[m] = slot[m - 1];
        }
        best[at] = d;
        slot[at] = (int)(e2 - r0);
        if (cnt < 3) cnt++;
      }
    }
    uint32_t w = (uint32_t)cnt << 24;
    for (int m = 0; m < 3; ++m) w |= (uint32_t)(m < cnt ? slot[m] : 0xFF) << (8 * m);
    stb[e] = w;
  }
  int off = 0;
  for (int32_t k = 0; k < r1 - r0; ++k) {
    int c = 0;
    if (r1 - r0 <= kMaxDeg) {  // 3 kMaxDeg < 256: the start fits its byte (longer rows are sinks')
      for (int32_t j = 0; j < r1 - r0; ++j) {
        const uint32_t w = stb[r0 + j];
        const int cnt = (int)(w >> 24);
        bool hit = false;
        for (int m = 0; m < cnt; ++m) hit |= (int)((w >> (8 * m)) & 0xFFu) == k;
        if (hit) binv[3 * (int64_t)r0 + off + c++] = (uint8_t)j;
      }
    }
    bpos[r0 + k] = (uint16_t)(off | (c << 8));
    off += c;
  }
}

cudaError_t launch_ballistic_tables(DevGrid &g, cudaStream_t st) {
  if (!g.stb || g.n <= 0) return cudaSuccess;
  k_ballistic_tables<<<(unsigned)((g.n + 255) / 256), 256, 0, st>>>(g.n, g.row_ptr, g.edges, g.stb,
                                                                     g.bpos, g.binv);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// CSR offsets: int64 -> int32, monotone, degree statistics.
// ----------------------------------------------------------------------------
__global__ void k_row_ptr(int64_t n, const int64_t *__restrict__ rp64, const uint8_t *__restrict__ flags,
                          int32_t *__restrict__ rp32, unsigned long long *__restrict__ diag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > n) return;
  const int64_t r = rp64[i];
  rp32[i] = (int32_t)r;
  if (i == n) return;
  const int64_t deg = rp64[i + 1] - r;
  if (deg < 0 || (i == 0 && r != 0)) atomicOr(&diag[kDiagError], kErrRowPtr);
  if (!(flags[i] & 1u) && deg > 0) atomicMax(&diag[kDiagMaxDeg], (unsigned long long)deg);
  if (!(flags[i] & 1u) && deg > kMaxDeg) atomicOr(&diag[kDiagError], kErrDegree);
}

// ----------------------------------------------------------------------------
// Per-vertex edge tables.  One thread per vertex.
//   twin: binary search of i in the sorted row of col
//   q: rint(127 * (p_k - p_i) / |p_k - p_i|) with IEEE FP64 operations in the
//      stated order (no contraction), so that both sides of a parity test
//      quantise to the same integers
//   st: the <= 3 slots k' with the largest positive q_k . q_k', ties -> lower k'
// ----------------------------------------------------------------------------
__global__ void k_edges(int64_t n, const double *__restrict__ pos, const int32_t *__restrict__ rp,
                        const int32_t *__restrict__ col, Edge *__restrict__ edges,
                        double *__restrict__ mean_len, float4 *__restrict__ ev,
                        unsigned long long *__restrict__ diag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r0 = rp[i], r1 = rp[i + 1];
  const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
  double sum = 0.0;
  unsigned long long err = 0;
  for (int32_t e = r0; e < r1; ++e) {
    const int32_t j = col[e];
    Edge E;
    E.col = j;
    E.twin = -1;
    E.q = make_char4(0, 0, 0, 0);
    E.st = make_uchar4(0xFF, 0xFF, 0xFF, 0);
    if (j < 0 || j >= n) {
      err |= kErrColRange;
      edges[e] = E;
      continue;
    }
    if (j == i) err |= kErrSelfLoop;
    if (e > r0 && col[e - 1] >= j) err |= kErrUnsorted;
    // reverse edge
    int32_t lo = rp[j], hi = rp[j + 1] - 1, tw = -1;
    while (lo <= hi) {
      const int32_t mid = (lo + hi) >> 1;
      const int32_t c = col[mid];
      if (c == (int32_t)i) {
        tw = mid;
        break;
      }
      if (c < (int32_t)i) lo = mid + 1; else hi = mid - 1;
    }
    if (tw < 0) err |= kErrAsym;
    E.twin = tw;
    const double dx = __dsub_rn(pos[3 * (int64_t)j], px);
    const double dy = __dsub_rn(pos[3 * (int64_t)j + 1], py);
    const double dz = __dsub_rn(pos[3 * (int64_t)j + 2], pz);
    const double len = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                            __dmul_rn(dz, dz)));
    E.q = make_char4((signed char)quantise(__ddiv_rn(dx, len)),
                     (signed char)quantise(__ddiv_rn(dy, len)),
                     (signed char)quantise(__ddiv_rn(dz, len)), 0);
    sum = __dadd_rn(sum, len);
    ev[e] = make_float4((float)dx, (float)dy, (float)dz, (float)len);
    edges[e] = E;
  }
  mean_len[i] = (r1 > r0) ? __ddiv_rn(sum, (double)(r1 - r0)) : 0.0;
  // most-straightforward table
  for (int32_t e = r0; e < r1; ++e) {
    const char4 qe = edges[e].q;
    int best[3];
    int slot[3];
    int cnt = 0;
    for (int32_t e2 = r0; e2 < r1; ++e2) {
      const char4 q2 = edges[e2].q;
      const int d = (int)qe.x * q2.x + (int)qe.y * q2.y + (int)qe.z * q2.z;
      if (d <= 0) continue;
      int at = cnt;
      while (at > 0 && d > best[at - 1]) at--;
      if (at >= 3) continue;
      const int last = cnt < 3 ? cnt : 2;
      for (int m = last; m > at; --m) {
        best[m] = best[m - 1];
        slot[m] = slot[m - 1];
      }
      best[at] = d;
      slot[at] = (int)(e2 - r0);
      if (cnt < 3) cnt++;
    }
    uchar4 st;
    st.x = cnt > 0 ? (unsigned char)slot[0] : 0xFF;
    st.y = cnt > 1 ? (unsigned char)slot[1] : 0xFF;
    st.z = cnt > 2 ? (unsigned char)slot[2] : 0xFF;
    st.w = (unsigned char)cnt;
    edges[e].st = st;
  }
  if (err) atomicOr(&diag[kDiagError], err);
}

// ----------------------------------------------------------------------------
// kappa: sum over interior vertices and unrotated bins of the progress of the
// straight moves along the bin, divided by their length (Sect. 2.2.3, global
// correction of the zig-zag path).  FP32 per vertex, FP64 across vertices.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_kappa(int64_t n, int nbins, const int32_t *__restrict__ rp,
                                               const Edge *__restrict__ edges,
                                               const float4 *__restrict__ ev,
                                               const uint8_t *__restrict__ flags,
                                               const StepTables *__restrict__ tab0,
                                               const double *__restrict__ bins,
                                               double *__restrict__ part) {
  __shared__ double s_num[256], s_den[256];
  __shared__ float s_d[kMaxBins][3];
  __shared__ float4 s_qb[kMaxBins];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    s_qb[b] = tab0->qb[b];
    s_d[b][0] = (float)bins[3 * b];
    s_d[b][1] = (float)bins[3 * b + 1];
    s_d[b][2] = (float)bins[3 * b + 2];
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (i < n && !(flags[i] & (kFlagSink | kFlagGhost))) {  // interior vertices this grid steps
    const int32_t r0 = rp[i], r1 = rp[i + 1];
    if (r1 > r0) {
      float fn = 0.f, fd = 0.f;
      for (int b = 0; b < nbins; ++b) {
        const float4 qb = s_qb[b];
        int bestk = 0;
        float bestd = -1e30f;
        for (int32_t e = r0; e < r1; ++e) {
          const char4 q = edges[e].q;
          const float d = (float)q.x * qb.x + (float)q.y * qb.y + (float)q.z * qb.z;  // exact ints
          if (d > bestd) {
            bestd = d;
            bestk = e - r0;
          }
        }
        const uchar4 st = edges[r0 + bestk].st;
        const int cnt = st.w;
        if (cnt == 0) continue;
        float prog = 0.f, path = 0.f;
        const unsigned char sl[3] = {st.x, st.y, st.z};
        for (int m = 0; m < cnt; ++m) {
          const float4 v = ev[r0 + sl[m]];
          prog += v.x * s_d[b][0] + v.y * s_d[b][1] + v.z * s_d[b][2];
          path += v.w;
        }
        fn += prog / cnt;
        fd += path / cnt;
      }
      num = fn;
      den = fd;
    }
  }
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_num[threadIdx.x] += s_num[threadIdx.x + s];
      s_den[threadIdx.x] += s_den[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s_num[0];
    part[2 * blockIdx.x + 1] = s_den[0];
  }
}

__global__ void k_kappa_final(int64_t nb, const double *__restrict__ part, double kappa_cfg,
                              double *__restrict__ kappa) {
  __shared__ double s_num[256], s_den[256];
  double a = 0.0, b = 0.0;
  for (int64_t k = threadIdx.x; k < nb; k += blockDim.x) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  s_num[threadIdx.x] = a;
  s_den[threadIdx.x] = b;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s_num[threadIdx.x] += s_num[threadIdx.x + s];
      s_den[threadIdx.x] += s_den[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (kappa_cfg > 0.0) *kappa = kappa_cfg;
    else *kappa = s_den[0] > 0.0 ? s_num[0] / s_den[0] : 1.0;
  }
}

// Per-vertex constants and the initial neutral fraction.
__global__ void k_vconst(int64_t n, const double *__restrict__ nH, const double *__restrict__ vol,
                         const uint8_t *__restrict__ flags, const double *__restrict__ y0,
                         const double *__restrict__ mean_len, const double *__restrict__ kappa,
                         double sigma, double alpha_B, VConst *__restrict__ vc,
                         double *__restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  VConst c;
  const double nh = nH[i];
  const double A = __dmul_rn(nh, vol[i]);
  c.invA = A > 0.0 ? __ddiv_rn(1.0, A) : 0.0;
  c.tau_max = __dmul_rn(__dmul_rn(nh, sigma), __dmul_rn(*kappa, mean_len[i]));
  c.R0 = __dmul_rn(alpha_B, nh);
  c.flags = flags[i];
  c.src = -1;
  vc[i] = c;
  y[i] = y0 ? y0[i] : 1.0;
}

cudaError_t launch_setup(DevGrid &g, cudaStream_t st) {
  const int64_t n = g.n;
  const int T = 256;
  k_row_ptr<<<(unsigned)((n + 1 + T - 1) / T), T, 0, st>>>(n, g.s_row_ptr, g.s_flags, g.row_ptr,
                                                          g.diag);
  k_edges<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(n, g.pos, g.row_ptr, g.s_col, g.edges,
                                                     g.mean_len, g.s_ev, g.diag);
  return cudaGetLastError();
}

cudaError_t launch_kappa_and_consts(DevGrid &g, const double *bins_dev, double sigma,
                                    double alpha_B, double kappa_cfg, const double *y0_dev,
                                    cudaStream_t st) {
  const int64_t n = g.n;
  const int T = 256;
  if (kappa_cfg <= 0.0) {
    k_kappa<<<(unsigned)g.nblocks_kappa, T, 0, st>>>(n, g.nbins, g.row_ptr, g.edges, g.s_ev,
                                                     g.s_flags, g.tabs + kTabUnrotated, bins_dev,
                                                     g.kappa_part);
    k_kappa_final<<<1, T, 0, st>>>(g.nblocks_kappa, g.kappa_part, kappa_cfg, g.kappa_dev);
  } else {
    k_kappa_final<<<1, T, 0, st>>>(0, g.kappa_part, kappa_cfg, g.kappa_dev);
  }
  k_vconst<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(n, g.s_nH, g.s_vol, g.s_flags, y0_dev,
                                                      g.mean_len, g.kappa_dev, sigma, alpha_B,
                                                      g.vc, g.y);
  return cudaGetLastError();
}

cudaError_t launch_kappa_parts(DevGrid &g, const double *bins_dev, cudaStream_t st) {
  const int T = 256;
  k_kappa<<<(unsigned)g.nblocks_kappa, T, 0, st>>>(g.n, g.nbins, g.row_ptr, g.edges, g.s_ev,
                                                   g.s_flags, g.tabs + kTabUnrotated, bins_dev, g.kappa_part);
  return cudaGetLastError();
}

// kappa alone (k_kappa + k_kappa_final on the unrotated tables in g.tabs[kTabUnrotated]).
cudaError_t launch_kappa(DevGrid &g, const double *bins_dev, cudaStream_t st) {
  const int T = 256;
  k_kappa<<<(unsigned)g.nblocks_kappa, T, 0, st>>>(g.n, g.nbins, g.row_ptr, g.edges, g.s_ev,
                                                   g.s_flags, g.tabs + kTabUnrotated, bins_dev, g.kappa_part);
  k_kappa_final<<<1, T, 0, st>>>(g.nblocks_kappa, g.kappa_part, 0.0, g.kappa_dev);
  return cudaGetLastError();
}

}  // namespace sx
