// Allocation-free compliance c_k = f_k^T u_k (topo_compliance_noalloc in include/topo.h).
//
// The paper has no counterpart: this is an interface variant of topo_compliance for callers that
// cannot allocate device memory at the point of the call.  Those are callers without a solver
// object (topo_compliance needs one, and creating one allocates the whole multigrid hierarchy,
// hundreds of MB on a 2048 x 1024 grid) and callers whose device memory a caching allocator
// has already reserved, where a fresh cudaMalloc can fail with out-of-memory and cudaFree
// synchronizes the whole device.
//
// The reduction is the one of topo_compliance (same kernel, same fixed grid of kRedBlocks
// blocks, so the same bits); only its scratch differs.  Instead of the solver's buffers it uses
// the file-scope device array below: kRedBlocks partial sums per right-hand side followed by
// one ticket counter per right-hand side, kMaxRhs right-hand sides at most (311,552 bytes).
// Its address on a device is looked up once, by the first call made with that device current
// (cudaGetSymbolAddress); that first call should therefore come before any stream capture.
// The address is kept for the life of the process; after a device reset (cudaDeviceReset) the
// module may load at another address, so the entry point must not be used on that device again.
// The ticket counters must start at zero: the array is zero when the module loads, and every
// reduction puts its counter back to zero when it finishes.  The partial sums need no start
// value.  Calls whose kernels overlap on one device (other streams, other host threads) share
// the array and race; the caller orders them.
#include <mutex>
#include <string>

#include "topo_internal.cuh"

using namespace topo;

namespace {

constexpr int kScratchPartials = kRedBlocks * kMaxRhs;      // doubles
constexpr int kScratchCounters = kMaxRhs;                   // unsigned ints
constexpr int kScratchDoubles = kScratchPartials + (kScratchCounters + 1) / 2;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up on the first call per device).
topo_status scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "topo_compliance_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("topo_compliance_noalloc: device ordinal " + std::to_string(dev) +
              " is beyond the " + std::to_string(kMaxDevices) + " devices it tracks");
    return TOPO_E_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_status(e, "topo_compliance_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TOPO_OK;
}

}  // namespace

extern "C" {

topo_status topo_compliance_noalloc(const double* f, const double* u, long long n, int nrhs,
                                    double* c, void* cuda_stream) {
  if (n < 0) {
    set_error("topo_compliance_noalloc: n = " + std::to_string(n) + " is negative");
    return TOPO_E_INVALID_ARG;
  }
  if (nrhs < 1 || nrhs > kMaxRhs) {
    set_error("topo_compliance_noalloc: nrhs = " + std::to_string(nrhs) +
              " is outside 1.." + std::to_string(kMaxRhs) +
              " (the static scratch holds the partial sums of at most " +
              std::to_string(kMaxRhs) + " right-hand sides)");
    return TOPO_E_INVALID_ARG;
  }
  if (!c || (n > 0 && (!f || !u))) {
    set_error("topo_compliance_noalloc: null argument");
    return TOPO_E_INVALID_ARG;
  }
  double* scratch = nullptr;
  topo_status st = scratch_for_current_device(&scratch);
  if (st != TOPO_OK) return st;
  double* partials = scratch;
  unsigned* counters = reinterpret_cast<unsigned*>(scratch + kScratchPartials);
  cudaError_t e = launch_dot(n, nrhs, f, u, partials, counters, c,
                             static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_status(e, "topo_compliance_noalloc");
  return TOPO_OK;
}

}  // extern "C"
