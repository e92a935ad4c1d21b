// fc2d_coeffs_static: the 2D DFT of fc2d_coeffs for callers that cannot allocate
// device memory.
//
// fc2d_coeffs keeps its row-pass intermediate in plan workspace and grows that
// workspace with cudaMalloc on the first call of a new size.  Some callers may not
// allocate at that point, for example a host that owns every byte of device memory
// through its own allocator, or a real-time loop that cannot take the implicit device
// synchronisation of cudaMalloc/cudaFree.  This entry point calls no allocator.  Its
// scratch is a fixed array in device global memory (kStaticScratchBytes, 64 MiB),
// which every GPU that loads the library holds until the process exits.
//
// In host code `g_scratch` names a host-side stand-in, not a device address.  The
// device address is fetched once per device with cudaGetSymbolAddress, with that
// device current, on the first call of the entry point on that device.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "fc2d_kernels.cuh"
#include "plan_internal.h"

namespace fc2d {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on `device` (which must be current).
static fc2d_status scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices)
    return set_error(FC2D_ERR_UNSUPPORTED, "fc2d_coeffs_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr)
      return set_error(FC2D_ERR_CUDA, std::string("fc2d_coeffs_static: cudaGetSymbolAddress: ") +
                                          cudaGetErrorString(e));
    g_scratch_addr[device] = ptr;
  }
  *out = g_scratch_addr[device];
  return FC2D_OK;
}

}  // namespace fc2d

using namespace fc2d;

extern "C" fc2d_status fc2d_coeffs_static(fc2d_plan_t p, int n_f, const void* ext,
                                          void* fhat, void* stream) {
  fc2d_status st = check_nf(p, n_f);
  if (st) return st;
  if (!ext || !fhat) return set_error(FC2D_ERR_ARG, "fc2d_coeffs_static: null argument");
  const bool f64 = p->prm.precision == FC2D_FP64;
  const size_t pitch = row_pitch(p);
  const size_t need = (size_t)n_f * p->grid.ny * pitch * 2 * (f64 ? 8 : 4);
  if (need > kStaticScratchBytes)
    return set_error(FC2D_ERR_ARG,
                     "fc2d_coeffs_static: n_f * ny * (nx/2+1 rounded up to 16) complex values need " +
                         std::to_string(need) + " bytes, above the fixed scratch of " +
                         std::to_string(kStaticScratchBytes) + " bytes");
  cudaError_t e = cudaSetDevice(p->device);
  if (e != cudaSuccess) return cuda_check(e, "fc2d_coeffs_static: cudaSetDevice");
  void* scratch = nullptr;
  st = scratch_address(p->device, &scratch);
  if (st) return st;
  // The row pass writes every intermediate element the column pass reads, so nothing
  // needs clearing between calls.  The argument blocks are the plan's own, as in
  // fc2d_coeffs.
  const FftArgs fa = fft_args(p);
  const RowArgs ra = row_args(p);
  cudaStream_t s = (cudaStream_t)stream;
  launch_fft_rows(fa, ra, n_f, f64, 0, ext, nullptr, nullptr, scratch, s);
  launch_fft_cols(fa, n_f, f64, scratch, fhat, s);
  return cuda_check(cudaGetLastError(), "fc2d_coeffs_static launch");
}
