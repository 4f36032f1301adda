// Scalar flux readout that allocates nothing.
//
// dd_dlra_scalar_flux keeps its per-subdomain scratch (the vectors S <V, 1>) in
// memory the solver allocated at create time.  This variant keeps that scratch in
// a file-scope device array instead, so the call itself needs no allocation from
// anyone: for callers that read the density while they must not allocate, for
// example inside a region they are capturing into their own CUDA graph, or under a
// memory policy that forbids device allocation after start-up.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ddlra.h"
#include "dd_internal.cuh"
#include "dd_launch.h"

// Scratch of the allocation-free readout: one vector of r_cap doubles per
// subdomain.  Every GPU that loads the library holds this array until the
// process exits.
#define DD_FLUX_SCRATCH_DOUBLES 16384
static __device__ __align__(256) double g_flux_scratch[DD_FLUX_SCRATCH_DOUBLES];

namespace {

const int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices];   // device address of g_flux_scratch per device, or null

}  // namespace

namespace dd {
// defined in dd_api.cu
dd_status noalloc_flux_impl(dd_dlra_t h, double* scratch, int scratch_doubles, double* out);
dd_status set_error(dd_status s, const char* msg);
}  // namespace dd

extern "C" dd_status dd_dlra_scalar_flux_noalloc(dd_dlra_t h, double* out) {
  if (!h || !out) return dd::set_error(DD_ERR_ARG, "null argument");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return dd::set_error(DD_ERR_CUDA, "cudaGetDevice failed");
  double* addr = nullptr;
  {
    // once per device, with that device current: the host-side name of the array is
    // only a stand-in, the kernels need its device address
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_flux_scratch);
      if (e != cudaSuccess)
        return dd::set_error(DD_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") +
                                           cudaGetErrorString(e)).c_str());
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    addr = g_scratch_addr[dev];
  }
  return dd::noalloc_flux_impl(h, addr, DD_FLUX_SCRATCH_DOUBLES, out);
}
