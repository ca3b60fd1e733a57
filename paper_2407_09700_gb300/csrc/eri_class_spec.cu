// The class kernel of eri_class_kernel.cuh compiled for single classes: the FP64 team
// kernels (8 lanes per quartet, both Eq. 1 assembly paths) of the s/p/d classes that take the
// most time in the 6-31G(d)-like builds, (dp|ds), (dp|dp), (dd|ds), (dd|dp) and (dp|pp).
// With the class fixed at compile time the root count N (Sec. 2, Eq. 3), the recurrence
// bounds and the table sizes are constants, so the 2D recurrences unroll and the
// shared-memory offsets fold.  Every other class, team size and precision runs the generic
// instantiations of eri_kernels.cu.  (dp|dp) also has a variant whose teams stage their
// primitive-pair records into shared memory by bulk copy, chosen by the tuning override.
#include "eri_class_kernel.cuh"

#define SPEC_CLASSES(X) X(2120) X(2121) X(2220) X(2221) X(2111)

extern "C" int erik_upload_cart_tables_spec(void) { return (int)upload_cart_table(); }

// 1 when a kernel compiled for class (la lb | lc ld) exists for this team size (FP64).
extern "C" int erik_class_spec_available(int ts, int la, int lb, int lc, int ld) {
  if (ts != 8) return 0;
  const int cls = 1000 * la + 100 * lb + 10 * lc + ld;
#define SPEC_HAS(C) \
  if (cls == C) return 1;
  SPEC_CLASSES(SPEC_HAS)
#undef SPEC_HAS
  return 0;
}

extern "C" int erik_launch_class_spec(int ts, int xy, const KernelArgs* a, int grid, int smem_bytes, void* stream,
                                      int* rc) {
  if (ts != 8) return 0;
  const int cls = 1000 * a->c.la + 100 * a->c.lb + 10 * a->c.lc + a->c.ld;
  cudaStream_t s = (cudaStream_t)stream;
  // (dp|dp) with its pair records staged into shared memory by bulk copies (tuning override)
  if (a->c.stage && cls == 2121) {
    if (xy)
      eri_class_kernel<8, double, true, 2121, true><<<grid, TPB, smem_bytes, s>>>(*a);
    else
      eri_class_kernel<8, double, false, 2121, true><<<grid, TPB, smem_bytes, s>>>(*a);
    *rc = (int)cudaGetLastError();
    return 1;
  }
#define SPEC_LAUNCH(C)                                                                  \
  if (cls == C) {                                                                       \
    if (xy)                                                                             \
      eri_class_kernel<8, double, true, C><<<grid, TPB, smem_bytes, s>>>(*a);           \
    else                                                                                \
      eri_class_kernel<8, double, false, C><<<grid, TPB, smem_bytes, s>>>(*a);          \
    *rc = (int)cudaGetLastError();                                                      \
    return 1;                                                                           \
  }
  SPEC_CLASSES(SPEC_LAUNCH)
#undef SPEC_LAUNCH
  return 0;
}

// The same dynamic shared-memory limit as the generic kernels, set once per kernel.
extern "C" int erik_class_spec_prepare(void) {
#define SPEC_ATTR(C)                                                                                        \
  {                                                                                                         \
    cudaError_t e = cudaFuncSetAttribute((const void*)eri_class_kernel<8, double, true, C>,                \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);          \
    if (e == cudaSuccess)                                                                                   \
      e = cudaFuncSetAttribute((const void*)eri_class_kernel<8, double, false, C>,                          \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);                    \
    if (e != cudaSuccess) return (int)e;                                                                    \
  }
  SPEC_CLASSES(SPEC_ATTR)
#undef SPEC_ATTR
  cudaError_t e = cudaFuncSetAttribute((const void*)eri_class_kernel<8, double, true, 2121, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)eri_class_kernel<8, double, false, 2121, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return (int)e;
}
