// Compile-time specialised Rys kernels for the low angular-momentum classes whose
// contracted [e0|f0] block fits a lane's registers (up to 54 values in FP64, 96 in the
// FP32 path of the mixed mode); each runs with one lane per shell quartet.  Following
// Sec. 3's design for small root counts (Alg. 2: unrolled recurrences, intermediates in
// registers, contraction before digestion), every loop here has compile-time bounds: the
// 2D tables I_x, I_y, I_z of one root and the contracted accumulators live in registers
// and the Eq. 1 index map is folded into the code.  Task fetching, screening, the
// transfer relations and the digestion are the shared device functions of eri_device.cuh.
#include <type_traits>

#include "eri_device.cuh"

namespace {

template <int I, int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor<I + 1, N>(f);
  }
}

__host__ __device__ constexpr int cb(int l) { return l * (l + 1) * (l + 2) / 6; }
__host__ __device__ constexpr int cart_l(int g) {
  int l = 0;
  while (cb(l + 1) <= g) ++l;
  return l;
}
// exponent of axis ax (0 = x, 1 = y, 2 = z) of the Cartesian function with global index g
__host__ __device__ constexpr int cart_e(int g, int ax) {
  const int l = cart_l(g);
  const int pos = g - cb(l);
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= pos) ++r;
  const int lz = pos - r * (r + 1) / 2;
  return ax == 0 ? l - r : (ax == 1 ? r - lz : lz);
}

template <int LA, int LB, int LC, int LD>
struct Small {
  static constexpr int LE = LA + LB, LF = LC + LD, L1 = LF + 1, NI = (LE + 1) * L1;
  static constexpr int N = (LA + LB + LC + LD) / 2 + 1;
  static constexpr int EB = cb(LA), FB = cb(LC);
  static constexpr int NE = cb(LE + 1) - EB, NF = cb(LF + 1) - FB, NOUT = NE * NF;
  // offset into the 2D table of axis ax for output o = ie * NF + jf
  __host__ __device__ static constexpr int idx(int o, int ax) {
    return cart_e(EB + o / NF, ax) * L1 + cart_e(FB + o % NF, ax);
  }
};

template <int LA, int LB, int LC, int LD, typename R>
__global__ void __launch_bounds__(TPB, (Small<LA, LB, LC, LD>::NOUT > 32 ? 2 : 3)) eri_small_kernel(const KernelArgs a) {
  using S = Small<LA, LB, LC, LD>;
  typedef typename PairOf<R>::type PP;
  constexpr int LE = S::LE, LF = S::LF, L1 = S::L1, NI = S::NI, N = S::N, NOUT = S::NOUT;
  const int lane = threadIdx.x & 31;
  const long long gteam = (long long)blockIdx.x * TPB + threadIdx.x;
  const ClassDesc& c = a.c;
  // contracted [e0|f0] and the transfer relations are FP64 in both paths (see eri_kernels.cu)
  double* scr = a.scratch + gteam * c.scratch_per_team;
  double* E0 = scr;
  double* bufA = scr + c.nout;
  double* bufB = bufA + c.hrr_doubles;
  const bool listed = a.tlist != nullptr || a.jobs != nullptr;
  const int qs = (a.mode == KMODE_JK && a.qsplit > 1) ? a.qsplit : 1;   // tasks per quartet (primitive ranges)
  const long long ntask = (listed ? (long long)*a.tcount : a.ntask) * qs;
  unsigned long long cnt_q = 0, cnt_p = 0;

  while (true) {
    unsigned long long tbase = 0;
    if (lane == 0) tbase = atomicAdd(a.counter, 32ULL);
    tbase = __shfl_sync(0xffffffffu, tbase, 0);
    if (tbase >= (unsigned long long)ntask) break;
    const long long slot = (long long)tbase + lane;
    bool active = slot < ntask;
    const long long task = slot / qs;
    const int ch = (int)(slot - task * qs);
    int ib = 0, ik = 0;
    TaskCtx tc = single_ctx(a);
    if (active) resolve_task(a, task, listed, tc, ib, ik);
    const PP* prims_r = reinterpret_cast<const PP*>(sizeof(R) == 8 ? (const void*)tc.prims : (const void*)tc.primsf);
    const ShellPair* bra = tc.pairs + ib;
    const ShellPair* ket = tc.pairs + ik;
    if (active && !listed) {
      const int cat = quartet_category(a, bra, ket, a.prec_sel != 0);
      active = cat != 0 && (a.prec_sel == 0 || cat == a.prec_sel);
    }
    const int npb = active ? bra->nprim : 0;
    const int npk = active ? ket->nprim : 0;
    // primitive quartets [qlo, qlo + nq) of this task (the last range counts the quartet)
    const int nqf = npb * npk;
    const int qlo = (qs > 1) ? (int)((long long)ch * nqf / qs) : 0;
    const int nq = (qs > 1) ? (int)((long long)(ch + 1) * nqf / qs) - qlo : nqf;
    if (nq == 0) active = false;
    const int maxq = warp_max(nq);
    if (active) { cnt_q += (ch == qs - 1) ? 1 : 0; cnt_p += (unsigned long long)nq; }
    double AB[3], CD[3];
    if (active) {
      AB[0] = bra->AB[0]; AB[1] = bra->AB[1]; AB[2] = bra->AB[2];
      CD[0] = ket->AB[0]; CD[1] = ket->AB[1]; CD[2] = ket->AB[2];
    }
    const int boff = active ? bra->prim_off : 0, koff = active ? ket->prim_off : 0;

    R acc[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; ++o) acc[o] = R(0);

    for (int q = 0; q < maxq; ++q) {
      if (q < nq) {
        const int ixp = boff + (qlo + q) / npk, iyp = koff + (qlo + q) % npk;
        const PrimPair* xd = tc.prims + ixp;
        const PrimPair* yd = tc.prims + iyp;
        // T and the Rys-table lookup in FP64
        const double s = xd->zeta + yd->zeta;
        const double rd = rsqrt(s);
        const double PQ0 = xd->P[0] - yd->P[0], PQ1 = xd->P[1] - yd->P[1], PQ2 = xd->P[2] - yd->P[2];
        const double T = xd->zeta * yd->zeta * (rd * rd) * fma(PQ0, PQ0, fma(PQ1, PQ1, PQ2 * PQ2));
        int ti;
        double xx, invT, rsqT;
        rys_locate(T, a.rys_tcut_d, ti, xx, invT, rsqT);
        // Gaussian-product scalars in the recurrence type
        const PP* x = (sizeof(R) == 8) ? reinterpret_cast<const PP*>(xd) : prims_r + ixp;
        const PP* y = (sizeof(R) == 8) ? reinterpret_cast<const PP*>(yd) : prims_r + iyp;
        const R zeta = x->zeta, eta = y->zeta;
        // P - Q and 1/sqrt(zeta + eta) from their FP64 values: P - Q formed in FP32 from rounded
        // centres would carry an absolute error of ~|P| 6e-8 bohr
        const R r = (R)rd, P0 = (R)PQ0, P1 = (R)PQ1, P2 = (R)PQ2;
        const R inv_s = r * r;
        const R rz = eta * inv_s, re = zeta * inv_s;
        const R hs = R(0.5) * inv_s;
        const R hz = x->hz, he = y->hz;
        const R hzrz = hz * rz, here = he * re;
        const R theta = x->E * y->E * r;
        const R PA0 = x->PA[0], PA1 = x->PA[1], PA2 = x->PA[2];
        const R QC0 = y->PA[0], QC1 = y->PA[1], QC2 = y->PA[2];
        const R aP0 = rz * P0, aP1 = rz * P1, aP2 = rz * P2;
        const R bP0 = re * P0, bP1 = re * P1, bP2 = re * P2;
#pragma unroll
        for (int n = 0; n < N; ++n) {
          double ud, wd;
          rys_root(a.rys_coef, a.rys_au, a.rys_aw, N, ti, xx, invT, rsqT, n, ud, wd);
          const R u = (R)ud, w = (R)wd;
          const R B00 = u * hs;
          const R B10 = fma(-u, hzrz, hz);
          const R B01 = fma(-u, here, he);
          const R wt = w * theta;
          const R C[3] = {fma(-u, aP0, PA0), fma(-u, aP1, PA1), fma(-u, aP2, PA2)};
          const R Cp[3] = {fma(u, bP0, QC0), fma(u, bP1, QC1), fma(u, bP2, QC2)};
          R g[3][NI];
          g[0][0] = R(1);
          g[1][0] = R(1);
          g[2][0] = wt;
          if constexpr (LE >= 1) {
            g[0][L1] = C[0];
            g[1][L1] = C[1];
            g[2][L1] = C[2] * wt;
          }
#pragma unroll
          for (int n2 = 1; n2 < LE; ++n2) {
            const R nb10 = R(n2) * B10;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
              g[ax][(n2 + 1) * L1] = fma(C[ax], g[ax][n2 * L1], nb10 * g[ax][(n2 - 1) * L1]);
          }
#pragma unroll
          for (int n2 = 0; n2 <= LE; ++n2) {
            const R nb00 = R(n2) * B00;
#pragma unroll
            for (int m = 0; m < LF; ++m) {
              const R mb01 = R(m) * B01;
#pragma unroll
              for (int ax = 0; ax < 3; ++ax) {
                const int e = n2 * L1 + m;
                R v = Cp[ax] * g[ax][e];
                if (n2 > 0) v = fma(nb00, g[ax][e - L1], v);
                if (m > 0) v = fma(mb01, g[ax][e - 1], v);
                g[ax][e + 1] = v;
              }
            }
          }
          // Eq. 1 products, accumulated over roots and primitives (Eq. 5)
          sfor<0, NOUT>([&](auto oc) {
            constexpr int o = decltype(oc)::value;
            constexpr int i0 = S::idx(o, 0), i1 = S::idx(o, 1), i2 = S::idx(o, 2);
            acc[o] = fma(g[0][i0] * g[1][i1], g[2][i2], acc[o]);
          });
        }
      }
    }
    if (active) {
#pragma unroll
      for (int o = 0; o < NOUT; ++o) E0[o] = (double)acc[o];
    }
    __syncwarp();
    finish_quartet<1, double>(a, tc, c, E0, bufA, bufB, 0, active, AB, CD, bra, ket, ib, ik, task);
    __syncwarp();
  }
  for (int off = 16; off > 0; off >>= 1) {
    cnt_q += __shfl_xor_sync(0xffffffffu, cnt_q, off);
    cnt_p += __shfl_xor_sync(0xffffffffu, cnt_p, off);
  }
  if (lane == 0 && a.stats) {
    atomicAdd(a.stats + 0, cnt_q);
    atomicAdd(a.stats + 1, cnt_p);
  }
}

// (la lb | lc ld) of the specialised classes and their kernels
#define SMALL_CLASSES(X)                                                                       \
  X(0, 0, 0, 0) X(1, 0, 0, 0) X(1, 1, 0, 0) X(2, 0, 0, 0) X(2, 1, 0, 0) X(2, 2, 0, 0)           \
  X(3, 0, 0, 0) X(3, 1, 0, 0) X(4, 0, 0, 0) X(1, 0, 1, 0) X(1, 1, 1, 0) X(2, 0, 1, 0) X(3, 0, 1, 0)      \
  X(2, 1, 1, 0) X(2, 0, 2, 0) X(2, 0, 1, 1)

// classes whose accumulators fit a lane's registers only in FP32: specialised for the FP32
// path of the mixed mode, team kernels for FP64
#define SMALL_CLASSES_F32(X) X(1, 1, 1, 1) X(2, 1, 2, 0) X(2, 2, 1, 0)

const void* small_ptr(int la, int lb, int lc, int ld, int fp32) {
#define SMALL_CASE(A, B, C, D)                                                   \
  if (la == A && lb == B && lc == C && ld == D)                                  \
    return fp32 ? (const void*)eri_small_kernel<A, B, C, D, float>               \
                : (const void*)eri_small_kernel<A, B, C, D, double>;
  SMALL_CLASSES(SMALL_CASE)
#undef SMALL_CASE
#define SMALL_CASE_F32(A, B, C, D)                                               \
  if (fp32 && la == A && lb == B && lc == C && ld == D) return (const void*)eri_small_kernel<A, B, C, D, float>;
  SMALL_CLASSES_F32(SMALL_CASE_F32)
#undef SMALL_CASE_F32
  return nullptr;
}

}  // namespace

extern "C" int erik_upload_cart_tables_small(void) { return (int)upload_cart_table(); }

// 1 if (la lb | lc ld) has a specialised kernel for this precision (fp32 = 1: FP32 path).
extern "C" int erik_small_available(int la, int lb, int lc, int ld, int fp32) {
  return small_ptr(la, lb, lc, ld, fp32) != nullptr;
}

extern "C" int erik_small_blocks_per_sm(int la, int lb, int lc, int ld, int fp32, int* out) {
  const void* k = small_ptr(la, lb, lc, ld, fp32);
  if (!k) return (int)cudaErrorInvalidValue;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, TPB, 0);
}

extern "C" int erik_launch_small(int la, int lb, int lc, int ld, int fp32, const KernelArgs* a, int grid, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
#define SMALL_LAUNCH(A, B, C, D)                                                              \
  if (la == A && lb == B && lc == C && ld == D) {                                             \
    if (fp32)                                                                                 \
      eri_small_kernel<A, B, C, D, float><<<grid, TPB, 0, s>>>(*a);                           \
    else                                                                                      \
      eri_small_kernel<A, B, C, D, double><<<grid, TPB, 0, s>>>(*a);                          \
    return (int)cudaGetLastError();                                                           \
  }
  SMALL_CLASSES(SMALL_LAUNCH)
#undef SMALL_LAUNCH
#define SMALL_LAUNCH_F32(A, B, C, D)                                                          \
  if (fp32 && la == A && lb == B && lc == C && ld == D) {                                     \
    eri_small_kernel<A, B, C, D, float><<<grid, TPB, 0, s>>>(*a);                             \
    return (int)cudaGetLastError();                                                           \
  }
  SMALL_CLASSES_F32(SMALL_LAUNCH_F32)
#undef SMALL_LAUNCH_F32
  return (int)cudaErrorInvalidValue;
}
