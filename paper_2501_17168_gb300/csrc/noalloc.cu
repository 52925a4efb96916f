// noalloc.cu -- tgp_fitness_mse_noalloc: the fitness call for callers that
// cannot allocate device memory.  Its scratch is a fixed array in the
// library's device memory instead of a caller workspace; everything else is
// tgp_fitness_mse unchanged.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/tgp.h"

namespace {

// The scratch.  Every GPU that loads the library holds one copy until the
// process exits.  Host code must not use its name as a device address: the
// device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_ws[TGP_NOALLOC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (with that device current) and cached.
tgp_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TGP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) return TGP_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TGP_OK;
}

}  // namespace

extern "C" tgp_status tgp_fitness_mse_noalloc(const tgp_population* pop, const tgp_data* data,
                                              const float* y, int32_t n_outputs, double* mse,
                                              int32_t* tree_status, void* stream) {
  if (!pop || !data) return TGP_ERR_INVALID_ARG;
  // the device comes first, so that a CUDA failure is reported as such and
  // not as the invalid-argument answer of the size query
  void* ws = nullptr;
  const tgp_status s = scratch_address(&ws);
  if (s != TGP_OK) return s;
  const size_t need = tgp_workspace_size(pop, data, n_outputs, nullptr);
  if (need == 0) return TGP_ERR_INVALID_ARG;
  if (need > (size_t)TGP_NOALLOC_WS_BYTES) return TGP_ERR_WORKSPACE;
  return tgp_fitness_mse(pop, data, y, n_outputs, mse, tree_status, ws,
                         (size_t)TGP_NOALLOC_WS_BYTES, stream);
}

extern "C" tgp_status tgp_check_device_error_noalloc(void* stream) {
  void* ws = nullptr;
  const tgp_status s = scratch_address(&ws);
  if (s != TGP_OK) return s;
  return tgp_check_device_error(ws, (size_t)TGP_NOALLOC_WS_BYTES, stream);
}
