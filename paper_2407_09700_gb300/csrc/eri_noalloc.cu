// eri_jk_noalloc: the J/K build of eri_jk for callers that must not allocate device memory
// during the call, with the class kernels' team scratch taken from a fixed static array.
//
// Why: the plan's scratch buffer is shared with eri_jk_grad and eri_shell_quartet, which
// may regrow it with cudaMalloc / cudaFree after a device-wide synchronisation.  Code
// running under an allocator or a memory budget that owns the device's memory, or inside
// a host callback, cannot let a library call cudaMalloc / cudaFree.  This entry point calls
// neither, nor any allocating library routine.
//
// The scratch lives in g_noalloc_scratch below: ERI_NOALLOC_SCRATCH_BYTES (32 MiB) of
// device memory that every GPU loading this library holds until the process exits.  Host
// code cannot use the array's name as a device address (on the host it is only a
// stand-in), so the address is looked up once per device with cudaGetSymbolAddress and
// cached (for the life of the process: it is not looked up again after a device reset).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/eri.h"
#include "eri_internal.h"

#define ERI_NOALLOC_SCRATCH_DOUBLES (4u << 20)
#define ERI_NOALLOC_SCRATCH_BYTES (ERI_NOALLOC_SCRATCH_DOUBLES * sizeof(double))

static __device__ __align__(256) double g_noalloc_scratch[ERI_NOALLOC_SCRATCH_DOUBLES];

extern "C" eri_status eri_internal_fail(eri_status s, const char* msg);
extern "C" eri_status eri_internal_jk_fixed_scratch(eri_plan* p, const double* D, int nD, double* J, double* K,
                                                    int flags, void* cuda_stream, double* scratch,
                                                    size_t scratch_doubles);

namespace {
std::mutex g_mu;
double* g_addr[64] = {nullptr};
}  // namespace

extern "C" eri_status eri_jk_noalloc(eri_plan* plan, const double* D, int nD, double* J, double* K, int flags,
                                     void* cuda_stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return eri_internal_fail(ERI_ERR_NO_DEVICE, "eri_jk_noalloc: no usable current CUDA device");
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      // once per device, with that device current: the device address of the static array
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return eri_internal_fail(ERI_ERR_CUDA, "eri_jk_noalloc: cudaGetSymbolAddress of the static scratch failed");
      }
      g_addr[dev] = (double*)ptr;
    }
    scratch = g_addr[dev];
  }
  return eri_internal_jk_fixed_scratch(plan, D, nD, J, K, flags, cuda_stream, scratch, ERI_NOALLOC_SCRATCH_DOUBLES);
}
