// Forward render whose scratch space is a fixed array inside the library, for
// callers that cannot allocate device memory when they render.
//
// Who needs this: code that runs where another component owns the device's
// memory and forbids allocation after start-up (plugin hosts, services with
// a fixed memory footprint), and code that must not make the implicit
// device-wide synchronisation cudaFree can cause.  Such a caller cannot
// allocate the workspace pulsar_render_fwd expects, so this entry point uses
// a file-scope device array instead and allocates nothing itself.
//
// Set-up: the array's device address is looked up with cudaGetSymbolAddress
// on every call, in the context current at the call (the lookup is cheap once
// the module is loaded), so a device reset or a new context never leaves a
// stale address behind.  In host code the array's name is only a host-side
// stand-in, so the kernels are always given the looked-up address.
#include "pulsar_internal.cuh"

namespace pulsar {
namespace {

static __device__ __align__(256) unsigned char g_static_ws[PULSAR_STATIC_WORKSPACE_BYTES];

// Device address of g_static_ws in the current context.
cudaError_t static_ws_address(void** out) { return cudaGetSymbolAddress(out, g_static_ws); }

}  // namespace
}  // namespace pulsar

using namespace pulsar;

extern "C" pulsar_status pulsar_render_fwd_static(const pulsar_params* params,
                                                  const pulsar_scene* scene, float* image,
                                                  float* log_norm, void* stream) {
  // the same validation, in the same order, as pulsar_render_fwd
  const pulsar_status valid = validate_params(params);
  if (valid != PULSAR_OK) return valid;
  const size_t need = pulsar_workspace_size(params);
  if (need > (size_t)PULSAR_STATIC_WORKSPACE_BYTES) return PULSAR_ERR_CAPACITY;
  if (!scene || !image || !log_norm) return PULSAR_ERR_INVALID_ARG;
  void* ws = nullptr;
  if (static_ws_address(&ws) != cudaSuccess) return PULSAR_ERR_CUDA;
  // Everything the three stages read is written earlier in the same call
  // (the set-up kernel resets the counters and flags, binning clears the
  // tile ranges and merge counters), so the previous call's contents do not
  // need clearing.
  pulsar_status st = pulsar_project(params, scene, ws, PULSAR_STATIC_WORKSPACE_BYTES, stream);
  if (st == PULSAR_OK) st = pulsar_bin(params, ws, PULSAR_STATIC_WORKSPACE_BYTES, stream);
  if (st == PULSAR_OK)
    st = pulsar_render_fwd(params, scene, ws, PULSAR_STATIC_WORKSPACE_BYTES, image, log_norm,
                           nullptr, nullptr, nullptr, stream);
  return st;
}

extern "C" pulsar_status pulsar_static_read_status(int64_t* pairs_needed, void* stream) {
  void* ws = nullptr;
  if (static_ws_address(&ws) != cudaSuccess) return PULSAR_ERR_CUDA;
  return pulsar_read_status(ws, PULSAR_STATIC_WORKSPACE_BYTES, pairs_needed, stream);
}
