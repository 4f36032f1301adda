// Scalar flux readout that allocates nothing.
//
// dd_dlra_scalar_flux keeps its per-subdomain scratch (the vectors S <V, 1>) in
// memory the solver allocated at create time.  This variant keeps that scratch in
// a file-scope device array instead, so the call itself needs no allocation from
// anyone: for callers that read the density at a moment when they must not
// allocate device memory, for example under a memory policy that allows device
// allocation only at start-up, or inside a region whose allocator is not to be
// touched.
#include <cuda_runtime.h>

#include <string>

#include "../../include/ddlra.h"
#include "dd_internal.cuh"
#include "dd_launch.h"

// Scratch of the allocation-free readout: one vector of r_cap doubles per
// subdomain.  Every GPU that loads the library holds this array until the
// process exits.
#define DD_FLUX_SCRATCH_DOUBLES 16384
static __device__ __align__(256) double g_flux_scratch[DD_FLUX_SCRATCH_DOUBLES];

namespace dd {

// defined in dd_api.cu
dd_status noalloc_flux_impl(dd_dlra_t h, int scratch_doubles, double* out);
dd_status set_error(dd_status s, const char* msg);

// Device address of the scratch array in the current context.  In host code the
// array's name is only a stand-in; kernels need this address.  Called once per solver
// at create time, with the solver's device current, so the address belongs to the same
// context as the solver's own memory and lives exactly as long.
cudaError_t noalloc_scratch_address(double** addr) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_flux_scratch);
  *addr = e == cudaSuccess ? static_cast<double*>(p) : nullptr;
  return e;
}

}  // namespace dd

extern "C" dd_status dd_dlra_scalar_flux_noalloc(dd_dlra_t h, double* out) {
  if (!h || !out) return dd::set_error(DD_ERR_ARG, "null argument");
  return dd::noalloc_flux_impl(h, DD_FLUX_SCRATCH_DOUBLES, out);
}
