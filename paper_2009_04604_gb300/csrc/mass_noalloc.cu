// mass_noalloc.cu -- lbm_mass_noalloc: the total-mass reduction without any
// device allocation.
//
// lbm_mass() keeps its per-block partial sums in scratch memory that the handle
// allocates on first use. cudaMalloc and cudaFree can synchronise the whole device.
// Some callers cannot allocate:
//   - monitoring code inside a step loop that must not stall on the allocator;
//   - code in a process where another allocator (a framework's caching pool, for
//     example) has already claimed the device memory, so cudaMalloc fails.
// For them this entry point keeps the partials in a file-scope static device
// array of fixed size. The array exists on every GPU that loads the library,
// from load until the process exits. The caller passes the handle (the state to
// reduce) and a device buffer for the result.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm.h"
#include "launch.hpp"
#include "sim.hpp"

namespace {

// One FP64 partial sum per block of the mass reduction: 1 MiB per device.
constexpr long long kMaxPartials = LBM_NOALLOC_MAX_PARTIALS;
static __device__ __align__(256) double g_partials[kMaxPartials];

// Device address of g_partials for each device, looked up once per device. In
// host code the name g_partials is only a host-side stand-in for the symbol;
// passing it to a kernel would hand the kernel the wrong memory.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_addr[kMaxDevices] = {nullptr};

int partials_address(lbm_sim *h, double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbm_fail(h, LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return lbm_fail(h, LBM_ERR_ARG, "device index beyond 63");
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess)
      return lbm_fail(h, LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<double *>(p);
  }
  *out = g_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_mass_noalloc(lbm_handle h, double *mass_dev) {
  if (!h || !mass_dev) return lbm_fail(h, LBM_ERR_ARG, "null argument");
  if (!h->geom_ok || !h->state_ok) return lbm_fail(h, LBM_ERR_STATE, "no state yet");
  const lbm::Launch l = h->aux_shape();
  const long long nblk = (long long)l.grid.x * l.grid.y * l.grid.z;
  if (nblk > kMaxPartials)
    return lbm_fail(h, LBM_ERR_ARG,
                    "lattice too large for lbm_mass_noalloc: it needs " + std::to_string(nblk) +
                        " partial sums and the static array holds " + std::to_string(kMaxPartials) +
                        " (about 33.5 million padded nodes); use lbm_mass");
  double *partials = nullptr;
  int rc = partials_address(h, &partials);
  if (rc) return rc;
  // Every partial the final sum reads is written first by its block in this call,
  // so nothing needs clearing. Calls that overlap on the GPU share g_partials and race.
  cudaError_t e = lbm::launch_read(h->lattice, h->dtype, h->view(), h->f[h->cur], nullptr, nullptr,
                                   nullptr, partials, l);
  if (e == cudaSuccess) e = lbm::launch_reduce_final(partials, nblk, 1, mass_dev, h->stream);
  if (e != cudaSuccess) return lbm_fail(h, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}
