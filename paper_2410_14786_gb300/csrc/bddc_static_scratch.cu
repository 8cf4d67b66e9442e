// bddc_apply_static_scratch: the preconditioner apply with its temporaries in
// memory that the library reserves when it is loaded, instead of in the
// handle's workspace. The paper has no counterpart; this is a service for
// callers that must not allocate device memory (see include/bddc.h).
//
// The temporaries of one apply (compact interior, interface and coarse
// vectors) live in the file-scope array `g_apply_scratch`. Host code cannot
// use the array's name as a device address (in host code the name refers to
// a host-side stand-in), so the device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, on the first call on
// that device, and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/bddc.h"
#include "internal.hpp"
#include "kernels.cuh"

// 1 Mi doubles = 8 MiB on every device that loads the library.
constexpr long long kScratchDoubles = 1LL << 20;
static __device__ __align__(256) double g_apply_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_apply_scratch on `device` (current), looked up once.
cudaError_t scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

long long round_up(long long n) { return (n + 31) / 32 * 32; }   // 256-byte slices

}  // namespace

extern "C" int bddc_apply_static_scratch(bddc_handle_t h, const double* r, double* z, int32_t nrhs,
                                         void* stream) {
  if (!h) return bddc::set_last_error(BDDC_ERR_INVALID_ARG, "null handle");
  if (nrhs < 1 || nrhs > h->nrhs_max || !r || !z || r == z)
    return bddc::set_last_error(BDDC_ERR_INVALID_ARG, "bad nrhs or vector pointers");
  if (h->coarse_cg)
    return bddc::set_last_error(BDDC_ERR_INVALID_ARG,
                                "bddc_apply_static_scratch: the coarse CG mode is not supported; use bddc_apply");
  if (h->sparse_local)
    return bddc::set_last_error(BDDC_ERR_INVALID_ARG,
                                "bddc_apply_static_scratch: the sparse local solver is not supported; use bddc_apply");
  // slices: rI, tI, bI (interior), yG, zG, eG (interface copies), g (local
  // constraints), rc, uc (coarse), then the coarse solve's own temporaries,
  // each nrhs columns wide
  const long long R = nrhs;
  const long long nI = round_up(h->nI_tot * R), nG = round_up(h->nG_tot * R);
  const long long nC = round_up(h->nC_tot * R), nc = round_up(h->n_c * R);
  // coarse temporaries: the panel products (dense mode) or r' and y
  // (sparse mode)
  const long long ncoarse = h->coarse_dense ? round_up((long long)h->n_cpanels * h->n_c * R) : 2 * nc;
  const long long need = 3 * nI + 3 * nG + nC + 2 * nc + ncoarse;
  if (need > kScratchDoubles)
    return bddc::set_last_error(BDDC_ERR_INVALID_ARG,
                                "bddc_apply_static_scratch: this problem needs " + std::to_string(need) +
                                    " doubles of temporaries, more than the " + std::to_string(kScratchDoubles) +
                                    " reserved; use bddc_apply");
  bddc::DeviceGuard device_guard(h->device);   // the caller's current device is restored on return
  if (!device_guard.ok) return bddc::set_last_error(BDDC_ERR_CUDA, "could not make the handle's device current");
  double* base = nullptr;
  cudaError_t ae = scratch_address(h->device, &base);
  if (ae != cudaSuccess)
    return bddc::set_last_error(BDDC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ae));
  // this call's work vectors: slices of the static array (the handle itself
  // is not modified)
  bddc::ApplyWork W;
  double* p = base;
  W.rI = p; p += nI;
  W.tI = p; p += nI;
  W.bI = p; p += nI;
  W.yG = p; p += nG;
  W.zG = p; p += nG;
  W.eG = p; p += nG;
  W.g = p; p += nC;
  W.rc = p; p += nc;
  W.uc = p; p += nc;
  if (h->coarse_dense) {
    W.cpart = p;
  } else {
    W.cr = p; p += nc;
    W.cy = p;
  }
  cudaError_t e = bddc::launch_apply(h, r, z, nrhs, static_cast<cudaStream_t>(stream), nullptr, &W);
  if (e != cudaSuccess) return bddc::set_last_error(BDDC_ERR_CUDA, cudaGetErrorString(e));
  return BDDC_OK;
}
