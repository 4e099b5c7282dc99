// noalloc.cu -- fio_apply_noalloc: the forward apply on a fixed device scratch
// array instead of the plan's workspace, for callers that must not allocate
// device memory while they run (see include/fio.h).
//
// The scratch is one file-scope __device__ array.  Host code cannot use the
// array's name as a device address (on the host it is only a stand-in), so
// every call asks the runtime for the array's address on the current device.
// The query allocates nothing, and it stays right after a device reset or a
// new context, where the module (and so the array) is loaded again.
#include <cuda_runtime.h>

#include <string>

#include "fio_internal.h"

namespace {

constexpr size_t kScratchBytes = FIO_NOALLOC_SCRATCH_BYTES;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.
cudaError_t scratch_address(void **addr) {
  return cudaGetSymbolAddress(addr, g_noalloc_scratch);
}

}  // namespace

extern "C" fio_status fio_apply_noalloc(fio_plan p, const void *f, void *out, int batch,
                                        void *stream) {
  if (!p || !p->d_alpha) {
    fio::set_error("fio_apply_noalloc: invalid plan handle");
    return FIO_EINVAL;
  }
  if (!f || !out || f == out || batch < 1) {
    fio::set_error("fio_apply_noalloc: null/aliased pointers or batch < 1");
    return FIO_EINVAL;
  }
  const size_t cs = p->precision == FIO_FP64 ? 16 : 8;
  const size_t grid_bytes = (size_t)p->grid_units * batch * cs;
  const size_t fhat_bytes = (size_t)p->N * p->N * batch * cs;
  if (grid_bytes + fhat_bytes > kScratchBytes) {
    fio::set_error("fio_apply_noalloc: this plan and batch need " +
                   std::to_string(grid_bytes + fhat_bytes) + " bytes of scratch, more than the " +
                   std::to_string(kScratchBytes) +
                   " bytes of FIO_NOALLOC_SCRATCH_BYTES; use fio_apply or a smaller batch");
    return FIO_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev != p->device || dev < 0) {
    fio::set_error("fio_apply_noalloc: the plan's device must be the current device");
    return e != cudaSuccess ? FIO_ECUDA : FIO_EINVAL;
  }
  void *base = nullptr;
  e = scratch_address(&base);
  if (e != cudaSuccess) {
    fio::set_error(std::string("fio_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return FIO_ECUDA;
  }
  // grids first (their offsets keep 16-byte alignment), then the spectrum
  void *grid_ws = base;
  void *fhat_ws = static_cast<unsigned char *>(base) + grid_bytes;
  e = fio::launch_apply_ws(p, f, out, batch, (cudaStream_t)stream, grid_ws, fhat_ws, false);
  if (e != cudaSuccess) {
    fio::set_error(std::string("fio_apply_noalloc: ") + cudaGetErrorString(e));
    return FIO_ECUDA;
  }
  return FIO_OK;
}
