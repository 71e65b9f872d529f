// sx_halo.cu -- the halo exchange of a grid split over several shards
// (the paper's distributed-memory decomposition, Sect. 3.1-3.2).
//
// Each shard holds its own vertices and, as ghosts, the neighbours they have
// on other shards.  After a step the next step's gather at a vertex reads,
// for each in-edge, the routing mask its sender wrote and the sender's
// transmitted photons.  For an in-edge from a ghost those were made by the
// ghost's owner, so after every step the owner packs them (the masks at the
// receivers' in-edge indices, the senders' photon rows) and the receiving
// shard unpacks them into the same buffers at its own indices.
//
// Buffer layout (one pack): n_edges mask records of mw 32-bit words (mw = the
// grid's stored words per edge: 1, 2 or 4), then, at the next 16-byte
// boundary, n_rows photon rows of nbp values of the grid's photon type.
// Indices out of range are skipped and counted in diag[kDiagIndex].
#include "sx_internal.cuh"

namespace sx {

size_t halo_rows_offset(int64_t n_edges, int mw) {
  return ((size_t)n_edges * (size_t)mw * sizeof(uint32_t) + 15) / 16 * 16;
}

template <typename T>
__global__ void k_halo_pack(int64_t ne, const int32_t *__restrict__ eidx, int mw, int64_t nnz,
                            const uint32_t *__restrict__ M, int64_t nr, const int32_t *__restrict__ ridx,
                            int nbp, int64_t n, const T *__restrict__ P, uint32_t *__restrict__ out_m,
                            T *__restrict__ out_p, unsigned long long *__restrict__ diag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t k = t0; k < ne * mw; k += stride) {
    const int64_t j = k / mw;
    const int32_t e = eidx[j];
    if ((uint64_t)e < (uint64_t)nnz) out_m[k] = M[(int64_t)e * mw + (k - j * mw)];
    else if (k == j * mw) atomicAdd(&diag[kDiagIndex], 1ull);
  }
  for (int64_t k = t0; k < nr * nbp; k += stride) {
    const int64_t j = k / nbp;
    const int32_t r = ridx[j];
    if ((uint64_t)r < (uint64_t)n) out_p[k] = P[(int64_t)r * nbp + (k - j * nbp)];
    else if (k == j * nbp) atomicAdd(&diag[kDiagIndex], 1ull);
  }
}

template <typename T>
__global__ void k_halo_unpack(int64_t ne, const int32_t *__restrict__ eidx, int mw, int64_t nnz,
                              uint32_t *__restrict__ M, int64_t nr, const int32_t *__restrict__ ridx,
                              int nbp, int64_t n, T *__restrict__ P, const uint32_t *__restrict__ in_m,
                              const T *__restrict__ in_p, unsigned long long *__restrict__ diag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t k = t0; k < ne * mw; k += stride) {
    const int64_t j = k / mw;
    const int32_t e = eidx[j];
    if ((uint64_t)e < (uint64_t)nnz) M[(int64_t)e * mw + (k - j * mw)] = in_m[k];
    else if (k == j * mw) atomicAdd(&diag[kDiagIndex], 1ull);
  }
  for (int64_t k = t0; k < nr * nbp; k += stride) {
    const int64_t j = k / nbp;
    const int32_t r = ridx[j];
    if ((uint64_t)r < (uint64_t)n) P[(int64_t)r * nbp + (k - j * nbp)] = in_p[k];
    else if (k == j * nbp) atomicAdd(&diag[kDiagIndex], 1ull);
  }
}

cudaError_t launch_halo(DevGrid &g, int buf, bool pack, int64_t ne, const int32_t *eidx, int64_t nr,
                        const int32_t *ridx, void *data, cudaStream_t st) {
  const int64_t work = ne * g.mw > nr * g.nbp ? ne * g.mw : nr * g.nbp;
  if (work == 0) return cudaSuccess;
  const int T = 256;
  int64_t blocks = (work + T - 1) / T;
  if (blocks > 4096) blocks = 4096;
  uint32_t *m = static_cast<uint32_t *>(data);
  char *rows = static_cast<char *>(data) + halo_rows_offset(ne, g.mw);
  if (g.precision == 0) {
    double *p = reinterpret_cast<double *>(rows);
    if (pack)
      k_halo_pack<double><<<(unsigned)blocks, T, 0, st>>>(ne, eidx, g.mw, g.nnz, g.M[buf], nr, ridx, g.nbp, g.n,
                                                           static_cast<const double *>(g.P[buf]), m, p, g.diag);
    else
      k_halo_unpack<double><<<(unsigned)blocks, T, 0, st>>>(ne, eidx, g.mw, g.nnz, g.M[buf], nr, ridx, g.nbp, g.n,
                                                             static_cast<double *>(g.P[buf]), m, p, g.diag);
  } else {
    float *p = reinterpret_cast<float *>(rows);
    if (pack)
      k_halo_pack<float><<<(unsigned)blocks, T, 0, st>>>(ne, eidx, g.mw, g.nnz, g.M[buf], nr, ridx, g.nbp, g.n,
                                                          static_cast<const float *>(g.P[buf]), m, p, g.diag);
    else
      k_halo_unpack<float><<<(unsigned)blocks, T, 0, st>>>(ne, eidx, g.mw, g.nnz, g.M[buf], nr, ridx, g.nbp, g.n,
                                                            static_cast<float *>(g.P[buf]), m, p, g.diag);
  }
  return cudaGetLastError();
}

}  // namespace sx
