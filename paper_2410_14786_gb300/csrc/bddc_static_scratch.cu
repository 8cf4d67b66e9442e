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
  // slices: rI, tI, bI (interior), yG, zG, eG (interface copies), g, ucl
  // (local constraints), rc, uc (coarse), then the coarse solve's own
  // temporaries, each nrhs columns wide
  const long long R = nrhs;
  const long long nI = round_up(h->nI_tot * R), nG = round_up(h->nG_tot * R);
  const long long nC = round_up(h->nC_tot * R), nc = round_up(h->n_c * R);
  // coarse temporaries: the panel products (dense mode) or r' and y
  // (sparse mode)
  const long long ncoarse = h->coarse_dense ? round_up((long long)h->n_cpanels * h->n_c * R) : 2 * nc;
  const long long need = 3 * nI + 3 * nG + 2 * nC + 2 * nc + ncoarse;
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
  // Point the handle's workspace at the static array for this one call.
  // Calls on a handle are not re-entrant, and the launches below capture
  // the pointer values when they are enqueued, so the handle's own
  // workspace pointers are restored right after.
  double* saved[13] = {h->w_rI, h->w_tI, h->w_bI, h->w_yG, h->w_zG, h->w_eG,
                       h->w_g,  h->w_ucl, h->w_rc, h->w_uc, h->w_cr, h->w_cy, h->w_cpart};
  double* p = base;
  h->w_rI = p; p += nI;
  h->w_tI = p; p += nI;
  h->w_bI = p; p += nI;
  h->w_yG = p; p += nG;
  h->w_zG = p; p += nG;
  h->w_eG = p; p += nG;
  h->w_g = p; p += nC;
  h->w_ucl = p; p += nC;
  h->w_rc = p; p += nc;
  h->w_uc = p; p += nc;
  if (h->coarse_dense) {
    h->w_cpart = p;
  } else {
    h->w_cr = p; p += nc;
    h->w_cy = p;
  }
  cudaError_t e = bddc::launch_apply(h, r, z, nrhs, static_cast<cudaStream_t>(stream));
  h->w_rI = saved[0]; h->w_tI = saved[1]; h->w_bI = saved[2]; h->w_yG = saved[3]; h->w_zG = saved[4];
  h->w_eG = saved[5]; h->w_g = saved[6]; h->w_ucl = saved[7]; h->w_rc = saved[8]; h->w_uc = saved[9];
  h->w_cr = saved[10]; h->w_cy = saved[11]; h->w_cpart = saved[12];
  if (e != cudaSuccess) return bddc::set_last_error(BDDC_ERR_CUDA, cudaGetErrorString(e));
  return BDDC_OK;
}
