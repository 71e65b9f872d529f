// sx_noalloc.cu -- sx_kappa_noalloc: the path-length correction kappa of a
// grid for callers that cannot allocate device memory.
//
// Why it exists: every other entry point keeps its device state in a
// workspace that the caller allocates.  Some callers cannot allocate device
// memory at all -- for example code that runs while another allocator owns
// the whole device, or that must not touch the allocator at all at that
// point -- and so cannot provide one.  This entry point allocates nothing:
// its device scratch is one fixed-size array, declared below, that every GPU
// loading this library holds until the process exits.
//
// Contract
//   - limits: n <= SX_NOALLOC_MAX_VERTICES, nnz <= SX_NOALLOC_MAX_EDGES,
//     nbins <= SX_MAX_BINS; larger inputs are refused with SX_EINVAL.
//   - the first call on a device looks up the array's device address there
//     (cudaGetSymbolAddress, with that device current); make that first call
//     before any stream capture on the device.
//   - every call on a device shares the one array.  The call synchronises its
//     stream before it returns, so calls issued one after the other are
//     safe; calls whose GPU work overlaps (other threads or streams of the
//     same process) race on the array.  The calls of one process are
//     serialised on the host by a mutex.
//   - what must start at zero (the error and degree counters) is cleared on
//     every call; the rest of the array keeps the last call's contents.
//   - the call makes `device` current while it runs and the caller's current
//     device current again before it returns; a call that fails after it
//     queued work waits for its stream first, so that no work of it still
//     uses the array when the next call starts.
// The kernels are the ones sx_load_grid runs; only their buffers differ.
#include <cstring>
#include <mutex>
#include <string>

#include "simplexgb.h"
#include "sx_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int64_t kNv = SX_NOALLOC_MAX_VERTICES;
constexpr int64_t kNe = SX_NOALLOC_MAX_EDGES;
constexpr int64_t kKappaBlocks = (kNv + 255) / 256;

// byte offsets of the views carved out of the scratch array
constexpr size_t kOffPos = 0;
constexpr size_t kOffRp64 = kOffPos + up(sizeof(double) * 3 * kNv);
constexpr size_t kOffRp32 = kOffRp64 + up(sizeof(int64_t) * (kNv + 1));
constexpr size_t kOffCol = kOffRp32 + up(sizeof(int32_t) * (kNv + 1));
constexpr size_t kOffFlags = kOffCol + up(sizeof(int32_t) * kNe);
constexpr size_t kOffEdges = kOffFlags + up(kNv);
constexpr size_t kOffEv = kOffEdges + up(sizeof(sx::Edge) * kNe);
constexpr size_t kOffMeanLen = kOffEv + up(sizeof(float4) * kNe);
constexpr size_t kOffBins = kOffMeanLen + up(sizeof(double) * kNv);
constexpr size_t kOffTabs = kOffBins + up(sizeof(double) * 3 * sx::kMaxBins);
constexpr size_t kOffKpart = kOffTabs + up(sizeof(sx::StepTables) * sx::kTabCount);
constexpr size_t kOffKappa = kOffKpart + up(sizeof(double) * 2 * kKappaBlocks);
constexpr size_t kOffDiag = kOffKappa + up(sizeof(double));
constexpr size_t kOffSteps = kOffDiag + up(sizeof(unsigned long long) * sx::kDiagCount);
constexpr size_t kScratchBytes = kOffSteps + up(sizeof(unsigned long long));

}  // namespace

// The scratch of sx_kappa_noalloc (about 10 MB; see SX_NOALLOC_MAX_*).
static __device__ __align__(256) unsigned char sx_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void *g_base[64] = {nullptr};  // device address of the scratch, per device ordinal
thread_local std::string g_err;

int fail(int code, const std::string &m) {
  g_err = m;
  return code;
}

// Runs when the call returns (while the lock is still held): waits for the
// stream if the call queued work and failed, then makes the caller's device
// current again.
struct CallScope {
  int prev_device = -1;
  cudaStream_t st = nullptr;
  bool queued = false, ok = false;
  ~CallScope() {
    if (queued && !ok) cudaStreamSynchronize(st);  // best effort: the error is already reported
    if (prev_device >= 0) cudaSetDevice(prev_device);
  }
};

}  // namespace

extern "C" int sx_kappa_noalloc(int64_t n, const double *pos, const int64_t *row_ptr,
                                const int32_t *col, const uint8_t *flags, int32_t nbins,
                                const double *bin_dirs, int32_t device, void *stream,
                                double *kappa_out) {
  if (!pos || !row_ptr || !flags || !bin_dirs || !kappa_out) return fail(SX_EINVAL, "NULL argument");
  if (n < 1 || n > kNv) return fail(SX_EINVAL, "n must be in 1..SX_NOALLOC_MAX_VERTICES");
  const int64_t nnz = row_ptr[n];
  if (!sx::row_ptr_nondecreasing(n, row_ptr) || nnz > kNe)
    return fail(SX_EINVAL, "row_ptr must start at 0, must not decrease, and nnz <= SX_NOALLOC_MAX_EDGES");
  if (nnz > 0 && !col) return fail(SX_EINVAL, "col is NULL");
  if (nbins < 1 || nbins > SX_MAX_BINS) return fail(SX_EINVAL, "nbins must be in 1..SX_MAX_BINS");
  if (device < 0 || device >= 64) return fail(SX_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  CallScope scope;
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return fail(SX_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  scope.prev_device = prev;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(SX_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  if (!g_base[device]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, sx_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(SX_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_base[device] = p;
  }
  char *b = static_cast<char *>(g_base[device]);
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  scope.st = st;
  sx::DevGrid g{};
  g.n = n;
  g.nnz = nnz;
  g.nbins = nbins;
  g.nbp = (nbins + 3) / 4 * 4;
  g.punit = 1.0;
  g.pos = reinterpret_cast<double *>(b + kOffPos);
  g.s_row_ptr = reinterpret_cast<int64_t *>(b + kOffRp64);
  g.row_ptr = reinterpret_cast<int32_t *>(b + kOffRp32);
  g.s_col = reinterpret_cast<int32_t *>(b + kOffCol);
  g.s_flags = reinterpret_cast<uint8_t *>(b + kOffFlags);
  g.edges = reinterpret_cast<sx::Edge *>(b + kOffEdges);
  g.s_ev = reinterpret_cast<float4 *>(b + kOffEv);
  g.mean_len = reinterpret_cast<double *>(b + kOffMeanLen);
  g.tabs = reinterpret_cast<sx::StepTables *>(b + kOffTabs);
  g.kappa_part = reinterpret_cast<double *>(b + kOffKpart);
  g.nblocks_kappa = (n + 255) / 256;
  g.kappa_dev = reinterpret_cast<double *>(b + kOffKappa);
  g.diag = reinterpret_cast<unsigned long long *>(b + kOffDiag);
  g.steps_done = reinterpret_cast<unsigned long long *>(b + kOffSteps);
  double *bins_dev = reinterpret_cast<double *>(b + kOffBins);
#define NA_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(SX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  // what must start at zero: the error and degree counters
  scope.queued = true;
  NA_CUDA(cudaMemsetAsync(g.diag, 0, sizeof(unsigned long long) * sx::kDiagCount, st));
  NA_CUDA(cudaMemcpyAsync(g.pos, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(g.s_row_ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
  if (nnz) NA_CUDA(cudaMemcpyAsync(g.s_col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(g.s_flags, flags, n, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(bins_dev, bin_dirs, sizeof(double) * 3 * nbins, cudaMemcpyHostToDevice, st));
  NA_CUDA(sx::launch_setup(g, st));
  NA_CUDA(sx::launch_rotation(g, bins_dev, 0, 1, 1, 1.0, st));
  NA_CUDA(sx::launch_kappa(g, bins_dev, st));
  unsigned long long diag[sx::kDiagCount];
  double kappa = 0.0;
  NA_CUDA(cudaMemcpyAsync(diag, g.diag, sizeof(diag), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaMemcpyAsync(&kappa, g.kappa_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  scope.ok = true;  // nothing of the call is left on the stream
#undef NA_CUDA
  if (diag[sx::kDiagError])
    return fail(SX_EINVAL, "malformed grid (as sx_load_grid would refuse it)");
  *kappa_out = kappa;
  return SX_OK;
}

extern "C" const char *sx_kappa_noalloc_last_error(void) { return g_err.c_str(); }
