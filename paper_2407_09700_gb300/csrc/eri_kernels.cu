// Rys-quadrature ERI class kernels and helpers for the integral-direct J/K build
// (arXiv 2407.09700, Secs. 2-3), written for sm_103a.
//
// One launch per angular-momentum class (la lb | lc ld).  A "team" of TS threads
// owns one contracted shell quartet at a time (TS = 1, 2, 4, 8 or 32, or 128: the whole
// block, for the classes with 2048 or more [e0|f0] values); a warp holds 32/TS teams and
// all control flow is warp-uniform (block-uniform for TS = 128), so the FP64 pipe never
// runs a warp instruction for a team that has left the loop.  A quartet whose class has
// too few quartets to fill the GPU may run as several tasks over ranges of its primitive
// quartets (KernelArgs::qsplit), each digesting its partial sums.  Per quartet:
//   1. loop over primitive quartets in batches of bp:
//      a. scalars of each primitive quartet (Gaussian product, T = rho |PQ|^2);
//      b. for each (primitive, root): Rys root u and weight w from the generated
//         table, then the 2D integrals I_x, I_y, I_z by the recurrences for
//         I(n, m), n <= la+lb, m <= lc+ld (bra on centre A, ket on centre C),
//         with w * Theta folded into I_z(0,0);
//      c. each lane accumulates its slots of the contracted [e0|f0] by Eq. 1
//         (sum over roots of I_x I_y I_z) and Eq. 5 (sum over primitives) in
//         registers;
//   2. the transfer (horizontal) relations (a, b+1_i| = (a+1_i, b| + (A-B)_i (a, b|
//      on the bra and the same with C-D on the ket turn [e0|f0] into (ab|cd);
//   3. digestion into J~ and K~ with the six updates of Alg. 2 and the
//      permutation weights of the unique quartet, by FP64 atomicAdd.
// The Rys roots, weights and recurrences are FP64 throughout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "eri_internal.h"

#include "eri_class_kernel.cuh"

// Stable compaction of a class's task space into the FP64 list (front of tlist, ascending
// task order) and, in the mixed mode, the FP32 list (back of tlist, read back-to-front in
// ascending task order).  Three steps: per-tile counts, an exclusive scan over tiles,
// ordered writes.  Keeping the order keeps neighbouring tasks on the same bra pair and on
// ket pairs of equal contraction depth, so a warp's primitive loops stay uniform.
#define CTILE 1024
__device__ __forceinline__ int task_category(const KernelArgs& a, long long task, int mixed) {
  if (task >= a.ntask) return 0;
  int ib, ik;
  decode_task(a, task, ib, ik);
  return quartet_category(a, a.pairs + ib, a.pairs + ik, mixed != 0);
}

// Block-wide counts of categories 1 and 2 over one tile (256 threads x 4 tasks).
__global__ void compact_count_kernel(const KernelArgs a, int mixed, unsigned* tilecnt) {
  __shared__ unsigned s1[8], s2[8];
  const long long t0 = (long long)blockIdx.x * CTILE;
  unsigned c1 = 0, c2 = 0;
  for (int k = 0; k < CTILE / 256; ++k) {
    const int cat = task_category(a, t0 + k * 256 + threadIdx.x, mixed);
    c1 += cat == 1;
    c2 += cat == 2;
  }
  for (int off = 16; off > 0; off >>= 1) {
    c1 += __shfl_xor_sync(0xffffffffu, c1, off);
    c2 += __shfl_xor_sync(0xffffffffu, c2, off);
  }
  if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = c1; s2[threadIdx.x >> 5] = c2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t1 = 0, t2 = 0;
    for (int w = 0; w < 8; ++w) { t1 += s1[w]; t2 += s2[w]; }
    tilecnt[2 * blockIdx.x] = t1;
    tilecnt[2 * blockIdx.x + 1] = t2;
  }
}

// Exclusive scan of the tile counts (one block); totals to counts[0..1].
__global__ void compact_scan_kernel(unsigned* tilecnt, long long ntiles, unsigned long long* counts) {
  __shared__ unsigned long long w1[32], w2[32];
  __shared__ unsigned long long carry1, carry2;
  if (threadIdx.x == 0) { carry1 = 0; carry2 = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (long long base = 0; base < ntiles; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    unsigned long long v1 = (i < ntiles) ? tilecnt[2 * i] : 0, v2 = (i < ntiles) ? tilecnt[2 * i + 1] : 0;
    unsigned long long x1 = v1, x2 = v2;
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y1 = __shfl_up_sync(0xffffffffu, x1, off);
      const unsigned long long y2 = __shfl_up_sync(0xffffffffu, x2, off);
      if (lane >= off) { x1 += y1; x2 += y2; }
    }
    if (lane == 31) { w1[wid] = x1; w2[wid] = x2; }
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x >> 5;
      unsigned long long z1 = (lane < nw) ? w1[lane] : 0, z2 = (lane < nw) ? w2[lane] : 0;
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y1 = __shfl_up_sync(0xffffffffu, z1, off);
        const unsigned long long y2 = __shfl_up_sync(0xffffffffu, z2, off);
        if (lane >= off) { z1 += y1; z2 += y2; }
      }
      if (lane < nw) { w1[lane] = z1; w2[lane] = z2; }
    }
    __syncthreads();
    const unsigned long long pre1 = carry1 + (wid ? w1[wid - 1] : 0) + x1 - v1;
    const unsigned long long pre2 = carry2 + (wid ? w2[wid - 1] : 0) + x2 - v2;
    __syncthreads();
    if (i < ntiles) { tilecnt[2 * i] = (unsigned)pre1; tilecnt[2 * i + 1] = (unsigned)pre2; }
    if (threadIdx.x == blockDim.x - 1) { carry1 = pre1 + v1; carry2 = pre2 + v2; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { counts[0] = carry1; counts[1] = carry2; }
}

// Ordered writes: each tile recomputes its categories and writes at its scanned offset.
__global__ void compact_write_kernel(const KernelArgs a, int mixed, const unsigned* tileoff, unsigned* tlist,
                                     unsigned long long cap) {
  __shared__ unsigned s1[8], s2[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long t0 = (long long)blockIdx.x * CTILE;
  unsigned base1 = tileoff[2 * blockIdx.x], base2 = tileoff[2 * blockIdx.x + 1];
  for (int k = 0; k < CTILE / 256; ++k) {
    const long long task = t0 + k * 256 + threadIdx.x;
    const int cat = task_category(a, task, mixed);
    const unsigned m1 = __ballot_sync(0xffffffffu, cat == 1), m2 = __ballot_sync(0xffffffffu, cat == 2);
    if (lane == 0) { s1[wid] = __popc(m1); s2[wid] = __popc(m2); }
    __syncthreads();
    unsigned p1 = base1, p2 = base2, tot1 = 0, tot2 = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < wid) { p1 += s1[w]; p2 += s2[w]; }
      tot1 += s1[w];
      tot2 += s2[w];
    }
    const unsigned below = (1u << lane) - 1u;
    if (cat == 1) tlist[p1 + __popc(m1 & below)] = (unsigned)task;
    if (cat == 2) tlist[cap - 1 - (p2 + __popc(m2 & below))] = (unsigned)task;
    base1 += tot1;
    base2 += tot2;
    __syncthreads();
  }
}

// Batched variant: reserve this job's place in a class's merged lists, then write
// entries job << 32 | task (FP64 list from the front, FP32 list from the back).
__global__ void compact_reserve_kernel(const unsigned long long* counts, unsigned long long* cursor,
                                       unsigned long long* base) {
  if (threadIdx.x == 0) {
    base[0] = atomicAdd(cursor + 0, counts[0]);
    base[1] = atomicAdd(cursor + 1, counts[1]);
  }
}

__global__ void compact_write_batched_kernel(const KernelArgs a, int mixed, const unsigned* tileoff,
                                             unsigned long long* blist, unsigned long long cap,
                                             unsigned long long job, const unsigned long long* base) {
  __shared__ unsigned s1[8], s2[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long t0 = (long long)blockIdx.x * CTILE;
  unsigned long long base1 = base[0] + tileoff[2 * blockIdx.x], base2 = base[1] + tileoff[2 * blockIdx.x + 1];
  for (int k = 0; k < CTILE / 256; ++k) {
    const long long task = t0 + k * 256 + threadIdx.x;
    const int cat = task_category(a, task, mixed);
    const unsigned m1 = __ballot_sync(0xffffffffu, cat == 1), m2 = __ballot_sync(0xffffffffu, cat == 2);
    if (lane == 0) { s1[wid] = __popc(m1); s2[wid] = __popc(m2); }
    __syncthreads();
    unsigned long long p1 = base1, p2 = base2;
    unsigned tot1 = 0, tot2 = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < wid) { p1 += s1[w]; p2 += s2[w]; }
      tot1 += s1[w];
      tot2 += s2[w];
    }
    const unsigned below = (1u << lane) - 1u;
    const unsigned long long e = (job << 32) | (unsigned long long)(unsigned)task;
    if (cat == 1) blist[p1 + __popc(m1 & below)] = e;
    if (cat == 2) blist[cap - 1 - (p2 + __popc(m2 & below))] = e;
    base1 += tot1;
    base2 += tot2;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ helper kernels
// Dmax[I][J] = max over densities and a in I, b in J of |D_ab| (Eq. 9's block maxima).
__global__ void dmax_kernel(const double* __restrict__ D, int nD, int nbf, int nsh,
                            const int* __restrict__ bf0, const int* __restrict__ nfun, double* Dmax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nsh * nsh) return;
  const int I = (int)(t / nsh), Jsh = (int)(t % nsh);
  double m = 0.0;
  for (int x = 0; x < nD; ++x)
    for (int a = 0; a < nfun[I]; ++a)
      for (int b = 0; b < nfun[Jsh]; ++b)
        m = fmax(m, fabs(D[(size_t)x * nbf * nbf + (size_t)(bf0[I] + a) * nbf + bf0[Jsh] + b]));
  Dmax[t] = m;
}

// out[0] = max over densities of |D_ij - D_ji|, out[1] = max |D_ij|, as the bit patterns of
// non-negative doubles (which order like unsigned integers, so atomicMax applies).
__global__ void symcheck_kernel(const double* __restrict__ D, int nD, int nbf, unsigned long long* out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)nbf * nbf;
  double asym = 0.0, mx = 0.0;
  if (t < per * nD) {
    const int x = (int)(t / per);
    const long long r = t % per;
    const int i = (int)(r / nbf), j = (int)(r % nbf);
    const double* Dx = D + (size_t)x * per;
    const double a = Dx[(size_t)i * nbf + j];
    mx = fabs(a);
    if (j > i) asym = fabs(a - Dx[(size_t)j * nbf + i]);
    if (!(mx <= 1.7e308)) { mx = __longlong_as_double(0x7ff0000000000000LL); asym = mx; }  // NaN / inf
  }
  for (int off = 16; off > 0; off >>= 1) {
    asym = fmax(asym, __shfl_xor_sync(0xffffffffu, asym, off));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 0, (unsigned long long)__double_as_longlong(asym));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(mx));
  }
}

// M <- M + M^T in place for every density (J = J~ + J~^T, K = K~ + K~^T).
__global__ void symmetrize_kernel(double* M, int nD, int nbf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)nbf * nbf;
  if (t >= per * nD) return;
  const int x = (int)(t / per);
  const long long r = t % per;
  const int i = (int)(r / nbf), j = (int)(r % nbf);
  double* Mx = M + (size_t)x * per;
  if (i < j) {
    const double v = Mx[(size_t)i * nbf + j] + Mx[(size_t)j * nbf + i];
    Mx[(size_t)i * nbf + j] = v;
    Mx[(size_t)j * nbf + i] = v;
  } else if (i == j) {
    Mx[(size_t)i * nbf + i] *= 2.0;
  }
}

__global__ void rys_test_kernel(int N, int n, const double* T, double* u, double* w, const double* coef,
                                const double* au, const double* aw, int tcut) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int ti;
  double x, invT, rsqT;
  rys_locate(T[t], tcut, ti, x, invT, rsqT);
  for (int r = 0; r < N; ++r) rys_root(coef, au, aw, N, ti, x, invT, rsqT, r, u[t * N + r], w[t * N + r]);
}

template <typename Tp>
__global__ void fma_probe_kernel(Tp* out, int iters, Tp a, Tp b) {
  Tp x0 = threadIdx.x * (Tp)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  Tp x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// ------------------------------------------------------------------ host launchers
extern "C" int erik_upload_cart_tables(void) { return (int)upload_cart_table(); }

static const void* class_kernel_ptr(int ts, int fp32, int xy) {
  if (fp32) {
    switch (ts * 2 + (xy ? 1 : 0)) {
      case 2: return (const void*)eri_class_kernel<1, float, false>;
      case 4: return (const void*)eri_class_kernel<2, float, false>;
      case 8: return (const void*)eri_class_kernel<4, float, false>;
      case 16: return (const void*)eri_class_kernel<8, float, false>;
      case 64: return (const void*)eri_class_kernel<32, float, false>;
      case 256: return (const void*)eri_class_kernel<128, float, false>;
    }
  } else {
    switch (ts * 2 + (xy ? 1 : 0)) {
      case 2: return (const void*)eri_class_kernel<1, double, false>;
      case 4: return (const void*)eri_class_kernel<2, double, false>;
      case 5: return (const void*)eri_class_kernel<2, double, true>;
      case 8: return (const void*)eri_class_kernel<4, double, false>;
      case 9: return (const void*)eri_class_kernel<4, double, true>;
      case 16: return (const void*)eri_class_kernel<8, double, false>;
      case 17: return (const void*)eri_class_kernel<8, double, true>;
      case 64: return (const void*)eri_class_kernel<32, double, false>;
      case 65: return (const void*)eri_class_kernel<32, double, true>;
      case 256: return (const void*)eri_class_kernel<128, double, false>;
      case 257: return (const void*)eri_class_kernel<128, double, true>;
    }
  }
  return nullptr;
}

extern "C" int erik_blocks_per_sm(int ts, int fp32, int xy, int smem_bytes, int* out) {
  const void* k = class_kernel_ptr(ts, fp32, xy);
  if (!k) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, TPB, smem_bytes);
}

// FP64 launches of classes with c.xy take the shared products instantiation; FP32 launches
// always run lane programs.
extern "C" int erik_launch_class(int ts, int fp32, const KernelArgs* a, int grid, int smem_bytes, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const bool xy = a->c.xy != 0 && !fp32;
  if (xy && ts == 1) return (int)cudaErrorInvalidValue;
  // a kernel compiled for this class, team size and assembly path, where one exists
  int rc = 0;
  if (!fp32 && erik_launch_class_spec(ts, xy ? 1 : 0, a, grid, smem_bytes, stream, &rc)) return rc;
#define CLASS_LAUNCH(T, R)                                                                     \
  if (xy)                                                                                      \
    eri_class_kernel<T, R, (T > 1 && sizeof(R) == 8)><<<grid, TPB, smem_bytes, s>>>(*a);      \
  else                                                                                         \
    eri_class_kernel<T, R, false><<<grid, TPB, smem_bytes, s>>>(*a);
  if (fp32) {
    switch (ts) {
      case 1: CLASS_LAUNCH(1, float) break;
      case 2: CLASS_LAUNCH(2, float) break;
      case 4: CLASS_LAUNCH(4, float) break;
      case 8: CLASS_LAUNCH(8, float) break;
      case 32: CLASS_LAUNCH(32, float) break;
      case 128: CLASS_LAUNCH(128, float) break;
      default: return (int)cudaErrorInvalidValue;
    }
  } else {
    switch (ts) {
      case 1: CLASS_LAUNCH(1, double) break;
      case 2: CLASS_LAUNCH(2, double) break;
      case 4: CLASS_LAUNCH(4, double) break;
      case 8: CLASS_LAUNCH(8, double) break;
      case 32: CLASS_LAUNCH(32, double) break;
      case 128: CLASS_LAUNCH(128, double) break;
      default: return (int)cudaErrorInvalidValue;
    }
  }
#undef CLASS_LAUNCH
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_compact(const KernelArgs* a, unsigned* tlist, unsigned long long cap,
                                   unsigned long long* counts, unsigned* tiles, int mixed, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const long long ntiles = (a->ntask + CTILE - 1) / CTILE;
  if (ntiles == 0) return (int)cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st);
  compact_count_kernel<<<(unsigned)ntiles, 256, 0, st>>>(*a, mixed, tiles);
  compact_scan_kernel<<<1, 1024, 0, st>>>(tiles, ntiles, counts);
  compact_write_kernel<<<(unsigned)ntiles, 256, 0, st>>>(*a, mixed, tiles, tlist, cap);
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_compact_batched(const KernelArgs* a, unsigned long long* blist, unsigned long long cap,
                                           unsigned long long* counts, unsigned* tiles, unsigned long long* cursor,
                                           unsigned long long* base, unsigned long long job, int mixed, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const long long ntiles = (a->ntask + CTILE - 1) / CTILE;
  if (ntiles == 0) return (int)cudaSuccess;
  compact_count_kernel<<<(unsigned)ntiles, 256, 0, st>>>(*a, mixed, tiles);
  compact_scan_kernel<<<1, 1024, 0, st>>>(tiles, ntiles, counts);
  compact_reserve_kernel<<<1, 32, 0, st>>>(counts, cursor, base);
  compact_write_batched_kernel<<<(unsigned)ntiles, 256, 0, st>>>(*a, mixed, tiles, blist, cap, job, base);
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_dmax(const double* D, int nD, int nbf, int nsh, const int* sh_bf0, const int* sh_n,
                                double* Dmax, void* stream) {
  const long long n = (long long)nsh * nsh;
  const int grid = (int)((n + 255) / 256);
  dmax_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(D, nD, nbf, nsh, sh_bf0, sh_n, Dmax);
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_symcheck(const double* D, int nD, int nbf, unsigned long long* out, void* stream) {
  const long long n = (long long)nbf * nbf * nD;
  const int grid = (int)((n + 255) / 256);
  symcheck_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(D, nD, nbf, out);
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_symmetrize(double* M, int nD, int nbf, void* stream) {
  const long long n = (long long)nbf * nbf * nD;
  const int grid = (int)((n + 255) / 256);
  symmetrize_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(M, nD, nbf);
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_rys(int N, int n, const double* T, double* u, double* w, const double* coef,
                               const double* au, const double* aw, int tcut, void* stream) {
  rys_test_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(N, n, T, u, w, coef, au, aw, tcut);
  return (int)cudaGetLastError();
}

extern "C" int erik_probe_fma(double* fp64_tflops, double* fp32_tflops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8, threads = 256;
  void* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  const int it64 = 2000, it32 = 40000;
  for (int w = 0; w < 2; ++w) fma_probe_kernel<double><<<blocks, threads>>>((double*)out, it64 / 4, 0.999, 1e-4);
  cudaEventRecord(e0);
  fma_probe_kernel<double><<<blocks, threads>>>((double*)out, it64, 0.999, 1e-4);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp64_tflops = 2.0 * 64.0 * it64 * (double)blocks * threads / (ms * 1e-3) / 1e12;
  for (int w = 0; w < 2; ++w) fma_probe_kernel<float><<<blocks, threads>>>((float*)out, it32 / 4, 0.999f, 1e-4f);
  cudaEventRecord(e0);
  fma_probe_kernel<float><<<blocks, threads>>>((float*)out, it32, 0.999f, 1e-4f);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *fp32_tflops = 2.0 * 64.0 * it32 * (double)blocks * threads / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return (int)cudaGetLastError();
}
