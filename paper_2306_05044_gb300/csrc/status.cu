// Status strings, the ABI version and host-side fault injection of libvndf.
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "vndf.h"

extern "C" int vndf_abi_version(void) { return 3; }

extern "C" const char* vndf_status_string(int status) {
  switch (status) {
    case VNDF_OK: return "ok";
    case VNDF_ERR_NULL: return "a required pointer is NULL";
    case VNDF_ERR_SIZE: return "a size is negative or above its limit";
    case VNDF_ERR_ALIGN: return "a pointer is not aligned to its element size";
    case VNDF_ERR_METHOD: return "unknown sampling method";
    case VNDF_ERR_WORKSPACE: return "workspace missing or too small";
    case VNDF_ERR_CUDA: return "a CUDA runtime call or kernel launch failed";
    case VNDF_ERR_ARG: return "optional arguments given in an invalid combination";
    default: return "unknown status";
  }
}

#include <cuda_runtime.h>

// 1 when the current device can dereference p (device memory, managed memory,
// or host memory that is page-locked and mapped into the device's address
// space), 0 when it cannot, VNDF_ERR_CUDA when the query itself fails.
extern "C" int vndf_pointer_device_accessible(const void* p) {
  if (p == nullptr) return 0;
  cudaPointerAttributes attr;
  const cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unregistered pointer
    return e == cudaErrorInvalidValue ? 0 : VNDF_ERR_CUDA;
  }
  switch (attr.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return 1;
    case cudaMemoryTypeHost:
      return attr.devicePointer == p ? 1 : 0;
    default:
      return 0;
  }
}

namespace vndf {

// VNDF_FAULT = "<kind>[@<entry point>]" (see common.cuh).  Read on every call,
// so a test can set and clear it between calls; an unset variable costs one
// getenv per call, far below the cost of a launch.
int injected_fault(const char* entry, bool takes_workspace) {
  const char* spec = std::getenv("VNDF_FAULT");
  if (spec == nullptr || *spec == '\0') return VNDF_OK;
  const char* at = std::strchr(spec, '@');
  const size_t kind_len = at ? size_t(at - spec) : std::strlen(spec);
  if (at && std::strcmp(at + 1, entry) != 0) return VNDF_OK;
  auto is = [&](const char* k) { return kind_len == std::strlen(k) && std::strncmp(spec, k, kind_len) == 0; };
  if (is("launch")) return VNDF_ERR_CUDA;
  if (is("align")) return VNDF_ERR_ALIGN;
  if (is("workspace")) return takes_workspace ? VNDF_ERR_WORKSPACE : VNDF_OK;
  return VNDF_OK;
}

}  // namespace vndf
