// Device code shared by the class kernels (eri_kernels.cu) and the compile-time
// specialised small-class kernels (eri_small.cu).  Each translation unit gets its own
// copy of the constant Cartesian table and uploads it at device set-up.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eri_internal.h"
#include "rys_table.h"

#define TPB 128        // threads per block of the class kernels
#define GSLOTS 32      // accumulator slots per lane

// lx, ly, lz, l by global Cartesian index.  Global memory read through the read-only
// path (L1-resident, 880 bytes): lanes of a team read different entries, which constant
// memory would serialise.
static __device__ uchar4 c_cart[ERI_MAXCART];
__device__ __forceinline__ uchar4 cart_of(int g) { return __ldg(c_cart + g); }

// Copy the table to this translation unit's c_cart (x-descending order, l = 0..9).
static inline cudaError_t upload_cart_table() {
  uchar4 h[ERI_MAXCART];
  int g = 0;
  for (int l = 0; l <= ERI_CART_LMAX; ++l)
    for (int lx = l; lx >= 0; --lx)
      for (int ly = l - lx; ly >= 0; --ly)
        h[g++] = make_uchar4((unsigned char)lx, (unsigned char)ly, (unsigned char)(l - lx - ly), (unsigned char)l);
  return cudaMemcpyToSymbol(c_cart, h, sizeof(h));
}

__device__ __forceinline__ int cart_below(int l) { return l * (l + 1) * (l + 2) / 6; }
__device__ __forceinline__ int cart_pos(int ly, int lz) { int r = ly + lz; return r * (r + 1) / 2 + lz; }
__device__ __forceinline__ int cart_index(int lx, int ly, int lz) {
  return cart_below(lx + ly + lz) + cart_pos(ly, lz);
}

// ------------------------------------------------------------------ shared-memory accessor
// A team's shared region: element e lives at base[e * es].  TS = 1 interleaves the
// 128 private regions of a block (es = 128) so that a warp reading the same entry
// hits 32 consecutive words; larger teams use contiguous regions (es = 1).
template <typename T>
struct Smem {
  T* base;
  int es;
  __device__ __forceinline__ T& operator[](int e) const { return base[e * es]; }
};

// ------------------------------------------------------------------ Rys roots and weights
// Degree-RYS_DEG polynomial, highest power first, by Horner's rule.
__device__ __forceinline__ double horner_rys(const double* __restrict__ c, double x) {
  double a = __ldg(c);
#pragma unroll
  for (int k = 1; k <= RYS_DEG; ++k) a = fma(a, x, __ldg(c + k));
  return a;
}

// floor(T) for 0 <= T < 2^30 using integer operations only (no FP64-pipe conversion)
__device__ __forceinline__ int floor_nonneg(double T) {
  const long long b = __double_as_longlong(T);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < 0) return 0;
  const long long m = (b & 0xfffffffffffffLL) | 0x10000000000000LL;
  return (int)(m >> (52 - e));
}

// Prepare the table lookup for one T: ti >= 0 selects interval ti (of width 1/RYS_SUB),
// else the large-T limit.
__device__ __forceinline__ void rys_locate(double T, double tcut, int& ti, double& x, double& invT, double& rsqT) {
  if (T < tcut) {
    ti = floor_nonneg((double)RYS_SUB * T);
    x = fma(2.0 * RYS_SUB, T, -(double)(2 * ti + 1));
    invT = 0.0;
    rsqT = 0.0;
  } else {
    ti = -1;
    x = 0.0;
    invT = 1.0 / T;
    rsqT = rsqrt(T);
  }
}

__device__ __forceinline__ void rys_root(const double* __restrict__ coef, const double* __restrict__ au,
                                         const double* __restrict__ aw, int N, int ti, double x,
                                         double invT, double rsqT, int n, double& u, double& w) {
  if (ti >= 0) {
    const double* c = coef + ((size_t)ti * N + n) * (2 * (RYS_DEG + 1));
    u = horner_rys(c, x);
    w = horner_rys(c + RYS_DEG + 1, x);
  } else {
    u = __ldg(au + n) * invT;
    w = __ldg(aw + n) * rsqT;
  }
}

// ------------------------------------------------------------------ 2D recurrences
// I(n, m) for n <= Le, m <= Lf at g[o + n*(Lf+1) + m], for the x, y and z tables at once
// (Sec. 2's RRs in the Rys-Dupuis-King form):
//   I(n+1, 0) = C00 I(n, 0) + n B10 I(n-1, 0)
//   I(n, m+1) = C00' I(n, m) + n B00 I(n-1, m) + m B01 I(n, m-1)
// I_x(0,0) = I_y(0,0) = 1 and I_z(0,0) = w Theta.  The running multiples n B10, n B00 and
// m B01 are shared by the three axes.
template <typename R>
__device__ __forceinline__ void rys_2d3(const Smem<R>& g, const int o[3], int Le, int Lf, R I0z, const R C[3],
                                        const R Cp[3], R B00, R B10, R B01) {
  const int L1 = Lf + 1;
  g[o[0]] = R(1);
  g[o[1]] = R(1);
  g[o[2]] = I0z;
  if (Le >= 1) {
    g[o[0] + L1] = C[0];
    g[o[1] + L1] = C[1];
    g[o[2] + L1] = C[2] * I0z;
  }
  R nb10 = B10;
  for (int n = 1; n < Le; ++n) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      g[o[a] + (n + 1) * L1] = fma(C[a], g[o[a] + n * L1], nb10 * g[o[a] + (n - 1) * L1]);
    nb10 += B10;
  }
  if (Lf == 0) return;
  // row n = 0
  g[o[0] + 1] = Cp[0];
  g[o[1] + 1] = Cp[1];
  g[o[2] + 1] = Cp[2] * I0z;
  R mb01 = B01;
  for (int m = 1; m < Lf; ++m) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g[o[a] + m + 1] = fma(Cp[a], g[o[a] + m], mb01 * g[o[a] + m - 1]);
    mb01 += B01;
  }
  // rows n >= 1
  R nb00 = B00;
  for (int n = 1; n <= Le; ++n) {
    const int r = n * L1;
#pragma unroll
    for (int a = 0; a < 3; ++a) g[o[a] + r + 1] = fma(Cp[a], g[o[a] + r], nb00 * g[o[a] + r - L1]);
    R mb = B01;
    for (int m = 1; m < Lf; ++m) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int e = o[a] + r + m;
        g[e + 1] = fma(Cp[a], g[e], fma(nb00, g[e - L1], mb * g[e - 1]));
      }
      mb += B01;
    }
    nb00 += B00;
  }
}

// The same recurrences for one axis: I(n, m) at g[o + n*(Lf+1) + m] from I(0,0) = I00
// (1 for x and y, w Theta for z).  Used when the (primitive, root) items of a batch are
// too few to fill a team, so the three axes run on separate lanes.
template <typename R>
__device__ __forceinline__ void rys_2d1(const Smem<R>& g, int o, int Le, int Lf, R I00, R C, R Cp, R B00, R B10,
                                        R B01) {
  const int L1 = Lf + 1;
  g[o] = I00;
  if (Le >= 1) g[o + L1] = C * I00;
  R nb10 = B10;
  for (int n = 1; n < Le; ++n) {
    g[o + (n + 1) * L1] = fma(C, g[o + n * L1], nb10 * g[o + (n - 1) * L1]);
    nb10 += B10;
  }
  if (Lf == 0) return;
  g[o + 1] = Cp * I00;
  R mb01 = B01;
  for (int m = 1; m < Lf; ++m) {
    g[o + m + 1] = fma(Cp, g[o + m], mb01 * g[o + m - 1]);
    mb01 += B01;
  }
  R nb00 = B00;
  for (int n = 1; n <= Le; ++n) {
    const int r = o + n * L1;
    g[r + 1] = fma(Cp, g[r], nb00 * g[r - L1]);
    R mb = B01;
    for (int m = 1; m < Lf; ++m) {
      g[r + m + 1] = fma(Cp, g[r + m], fma(nb00, g[r + m - L1], mb * g[r + m - 1]));
      mb += B01;
    }
    nb00 += B00;
  }
}

// ------------------------------------------------------------------ transfer (horizontal) relations
// Input element (e, v) at X[e*xe + v*xv] for la <= |e| <= la+lb (e relative to cart_below(la)).
// Output contiguous [a][b][v] with |a| = la, |b| = lb; returns the output pointer (X when lb = 0).
// Team-cooperative; every thread of the team must call it (it contains team barriers:
// __syncwarp, or __syncthreads for a block-wide team, BLK).
template <typename R, bool BLK = false>
__device__ const R* hrr_team(int la, int lb, const double* AB, int nv, const R* X, int xe, int xv, R* bufA,
                             R* bufB, int tl, int TS, bool active) {
  const R ABr[3] = {(R)AB[0], (R)AB[1], (R)AB[2]};
  const R* cur = X;
  int cse = xe, csb = 0, csv = xv;
  const int base = cart_below(la);
  for (int k = 1; k <= lb; ++k) {
    R* nxt = (cur == bufA) ? bufB : bufA;
    const int na = cart_below(la + lb - k + 1) - base;
    const int nb = (k + 1) * (k + 2) / 2;
    // output row r = (ia, ib) of the level: its two input rows (a + 1_i, b - 1_i) and
    // (a, b - 1_i) and the axis i that b was built along
    auto row = [&](int r, const R*& hi, const R*& lo, R& f) {
      const int ia = r / nb, ib = r - (r / nb) * nb;
      const uchar4 av = cart_of(base + ia);
      const uchar4 bv = cart_of(cart_below(k) + ib);
      const int i = bv.x ? 0 : (bv.y ? 1 : 2);
      int bm[3] = {bv.x, bv.y, bv.z};
      bm[i] -= 1;
      const int ibm = cart_pos(bm[1], bm[2]);
      int ap[3] = {av.x, av.y, av.z};
      ap[i] += 1;
      const int iap = cart_index(ap[0], ap[1], ap[2]) - base;
      hi = cur + iap * cse + ibm * csb;
      lo = cur + ia * cse + ibm * csb;
      f = (i == 0) ? ABr[0] : (i == 1 ? ABr[1] : ABr[2]);
    };
    if (active && !BLK) {
      // warp teams: one output per lane at a time (measured faster for them, and for the
      // gradient's many small blocks, than the forms below)
      for (int t = tl; t < na * nb * nv; t += TS) {
        const int v = t % nv;
        const int r = t / nv;
        const int ib = r % nb;
        const int ia = r / nb;
        const uchar4 av = cart_of(base + ia);
        const uchar4 bv = cart_of(cart_below(k) + ib);
        const int i = bv.x ? 0 : (bv.y ? 1 : 2);
        int bm[3] = {bv.x, bv.y, bv.z};
        bm[i] -= 1;
        const int ibm = cart_pos(bm[1], bm[2]);
        int ap[3] = {av.x, av.y, av.z};
        ap[i] += 1;
        const int iap = cart_index(ap[0], ap[1], ap[2]) - base;
        const R hi = cur[iap * cse + ibm * csb + v * csv];
        const R lo = cur[ia * cse + ibm * csb + v * csv];
        nxt[(ia * nb + ib) * nv + v] = fma(ABr[i], lo, hi);
      }
    } else if (active) {
      const int nr = na * nb;
      if (nv >= TS) {
        // block teams, long rows: rows in groups of four, the team's lanes along v; the
        // index arithmetic runs once per row, consecutive lanes touch consecutive outputs,
        // and the eight loads of a group are in flight together (the transfer phase of a
        // block team reads L2 / DRAM-resident scratch: 12-atom s..g build 1067 -> 1035 ms)
        int r = 0;
        for (; r + 4 <= nr; r += 4) {
          const R *h0, *l0, *h1, *l1, *h2, *l2, *h3, *l3;
          R f0, f1, f2, f3;
          row(r, h0, l0, f0);
          row(r + 1, h1, l1, f1);
          row(r + 2, h2, l2, f2);
          row(r + 3, h3, l3, f3);
          R* o = nxt + r * nv;
          for (int v = tl; v < nv; v += TS) {
            const int vo = v * csv;
            const R a0 = h0[vo], b0 = l0[vo], a1 = h1[vo], b1 = l1[vo];
            const R a2 = h2[vo], b2 = l2[vo], a3 = h3[vo], b3 = l3[vo];
            o[v] = fma(f0, b0, a0);
            o[nv + v] = fma(f1, b1, a1);
            o[2 * nv + v] = fma(f2, b2, a2);
            o[3 * nv + v] = fma(f3, b3, a3);
          }
        }
        for (; r < nr; ++r) {
          const R *h0, *l0;
          R f0;
          row(r, h0, l0, f0);
          R* o = nxt + r * nv;
          for (int v = tl; v < nv; v += TS) o[v] = fma(f0, l0[v * csv], h0[v * csv]);
        }
      } else {
        // short rows: the outputs in order over all lanes, four per lane at a time (the
        // loads of the four before their stores)
        const int nt = nr * nv;
        for (int t0 = tl; t0 < nt; t0 += 4 * TS) {
          R hv[4], lv[4], fv[4];
          int dst[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * TS;
            dst[u] = t < nt ? t : -1;
            const int tt = t < nt ? t : 0;
            const int r = tt / nv, v = tt - (tt / nv) * nv;
            const R *h0, *l0;
            row(r, h0, l0, fv[u]);
            hv[u] = h0[v * csv];
            lv[u] = l0[v * csv];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (dst[u] >= 0) nxt[dst[u]] = fma(fv[u], lv[u], hv[u]);
        }
      }
    }
    if (BLK) __syncthreads();
    else __syncwarp();
    cur = nxt;
    cse = nb * nv;
    csb = nv;
    csv = 1;
  }
  return cur;
}

// Shared-memory doubles a block team needs for one transfer sequence (la, lb) through
// hrr_seq_block with W vectors per slice (0 when lb = 0).
__host__ __device__ inline int hrr_seq_rows(int la, int lb, int k) {
  const int a0 = la * (la + 1) * (la + 2) / 6;
  const int L = la + lb - k + 1;
  return (L * (L + 1) * (L + 2) / 6 - a0) * ((k + 1) * (k + 2) / 2);
}
__host__ __device__ inline int hrr_seq_block_doubles(int la, int lb, int W) {
  if (lb == 0) return 0;
  int p = 0, q = 0, info = 0;
  for (int k = 1; k <= lb; ++k) {
    const int r = hrr_seq_rows(la, lb, k);
    info += r;
    if (k & 1) p = p > r ? p : r;
    else q = q > r ? q : r;
  }
  return hrr_seq_rows(la, lb, 0) * W + (p + q) * W + (info + 1) / 2;
}

// One transfer sequence (a, b+1| = (a+1, b| + (A-B)(a, b| for a block-wide team (TS = TPB
// threads, __syncthreads barriers), on nv independent vectors taken W at a time through
// shared memory: a slice's input rows are staged once, every level of the sequence is
// built in shared memory (rows [row][w]), and only the last level goes back to scratch.
// Input element (e, v) at X[e*xe + v*xv] (e relative to cart_below(la), la <= |e| <=
// la + lb); output row ab = (a, b) of vector v at Out[v*ov + ab*oab].  lb >= 1.  sh holds
// hrr_seq_block_doubles(la, lb, W) doubles.  Every thread of the block calls it.
template <int TS>
__device__ void hrr_seq_block(int la, int lb, const double* ABv, int nv, const double* X, int xe, int xv, double* Out,
                              int ov, int oab, double* sh, int W, int tl, bool active) {
  const int n0 = hrr_seq_rows(la, lb, 0);
  int P = 0, Q = 0, ninfo = 0;
  for (int k = 1; k <= lb; ++k) {
    const int r = hrr_seq_rows(la, lb, k);
    ninfo += r;
    if (k & 1) P = max(P, r);
    else Q = max(Q, r);
  }
  double* b0 = sh;                       // [n0][W]
  double* bP = b0 + n0 * W;              // odd levels
  double* bQ = bP + P * W;               // even levels
  int* info = reinterpret_cast<int*>(bQ + Q * W);
  // row table of every level: input rows (a + 1_i, b - 1_i), (a, b - 1_i) and the axis i
  const int base = cart_below(la);
  {
    int off = 0;
    for (int k = 1; k <= lb; ++k) {
      const int nb = (k + 1) * (k + 2) / 2, nbp = k * (k + 1) / 2;
      const int nr = hrr_seq_rows(la, lb, k);
      for (int r = tl; r < nr; r += TS) {
        const int ia = r / nb, ib = r - (r / nb) * nb;
        const uchar4 av = cart_of(base + ia);
        const uchar4 bv = cart_of(cart_below(k) + ib);
        const int i = bv.x ? 0 : (bv.y ? 1 : 2);
        int bm[3] = {bv.x, bv.y, bv.z};
        bm[i] -= 1;
        const int ibm = cart_pos(bm[1], bm[2]);
        int ap[3] = {av.x, av.y, av.z};
        ap[i] += 1;
        const int iap = cart_index(ap[0], ap[1], ap[2]) - base;
        info[off + r] = ((iap * nbp + ibm) << 16) | ((ia * nbp + ibm) << 2) | i;
      }
      off += nr;
    }
  }
  __syncthreads();
  const int rpl = TS / W, w = tl % W, r0 = tl / W;   // lanes: W vectors x rpl rows
  const int nlast = hrr_seq_rows(la, lb, lb);
  for (int v0 = 0; v0 < nv; v0 += W) {
    const int wv = min(W, nv - v0);
    // stage the slice's input rows (the loop order follows the unit stride of X)
    if (active) {
      if (xv == 1) {
        for (int t = tl; t < n0 * W; t += TS) {
          const int e = t / W, ww = t - (t / W) * W;
          if (ww < wv) b0[t] = X[e * xe + v0 + ww];
        }
      } else {
        for (int t = tl; t < n0 * W; t += TS) {
          const int ww = t / n0, e = t - (t / n0) * n0;
          if (ww < wv) b0[e * W + ww] = X[e * xe + (v0 + ww) * xv];
        }
      }
    }
    __syncthreads();
    const double* cur = b0;
    int off = 0;
    for (int k = 1; k <= lb; ++k) {
      double* nxt = (k & 1) ? bP : bQ;
      const int nr = hrr_seq_rows(la, lb, k);
      if (active && r0 < rpl && w < wv) {
        for (int r = r0; r < nr; r += rpl) {
          const int in = info[off + r];
          const int i = in & 3;
          const double f = (i == 0) ? ABv[0] : (i == 1 ? ABv[1] : ABv[2]);
          nxt[r * W + w] = fma(f, cur[((in >> 2) & 0x3fff) * W + w], cur[(in >> 16) * W + w]);
        }
      }
      __syncthreads();
      cur = nxt;
      off += nr;
    }
    // the last level of the slice back to scratch
    if (active) {
      if (ov == 1) {
        for (int t = tl; t < nlast * W; t += TS) {
          const int r = t / W, ww = t - (t / W) * W;
          if (ww < wv) Out[(v0 + ww) + r * oab] = cur[t];
        }
      } else {
        for (int t = tl; t < nlast * W; t += TS) {
          const int ww = t / nlast, r = t - (t / nlast) * nlast;
          if (ww < wv) Out[(v0 + ww) * ov + r * oab] = cur[r * W + ww];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ bulk copies into shared memory
// One-dimensional cp.async.bulk (no tensor map, no multicast) from this GPU's global memory
// into the executing block's shared memory, completed on an mbarrier.  Source, destination
// and size must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic-proxy accesses of shared memory before later bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  (void)state;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Wait for phase `parity` of the barrier to complete, for at most ~1 s of SM clock; false if
// the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(0xffffffffu, v); }

// Team of TS lanes: TS <= 32 lanes share a warp (32 / TS teams per warp); TS = TPB is the
// whole block (one team per block, several warps).  team_sync orders the team's shared and
// scratch accesses; every thread of the team must call it.
template <int TS>
__device__ __forceinline__ void team_sync() {
  if (TS > 32) __syncthreads();
  else __syncwarp();
}
// Maximum of m over the TS lanes of a team (every thread of the team calls it).
template <int TS>
__device__ __forceinline__ double team_max(double m) {
  if (TS <= 1) return m;
  constexpr int W = TS < 32 ? TS : 32;
  for (int off = W / 2; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if constexpr (TS > 32) {
    __shared__ double wmax[TS / 32];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    m = wmax[0];
    for (int w = 1; w < TS / 32; ++w) m = fmax(m, wmax[w]);
  }
  return m;
}

// ------------------------------------------------------------------ task decoding and screening
// Task t of a class enumerates (bra pair, ket pair): rectangular bra x ket, or the
// triangle ket <= bra when both come from the same pair type.
__device__ __forceinline__ void decode_task_in(long long task, bool tri, int bra0, int ket0, int nket, int& ib,
                                               int& ik) {
  if (tri) {
    long long i = (long long)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > task) --i;
    while ((i + 1) * (i + 2) / 2 <= task) ++i;
    ib = bra0 + (int)i;
    ik = ket0 + (int)(task - i * (i + 1) / 2);
  } else {
    ib = bra0 + (int)(task / nket);
    ik = ket0 + (int)(task % nket);
  }
}

__device__ __forceinline__ void decode_task(const KernelArgs& a, long long task, int& ib, int& ik) {
  decode_task_in(task, a.tri != 0, a.bra0, a.ket0, a.nket, ib, ik);
}

// What one task reads and writes: the launch's single job, or one job of a batched launch.
struct TaskCtx {
  const ShellPair* pairs;
  const PrimPair* prims;
  const PrimPairF* primsf;
  const double* D;
  double* J;
  double* K;
  int nbf, nD, want;
};

__device__ __forceinline__ TaskCtx single_ctx(const KernelArgs& a) {
  TaskCtx c;
  c.pairs = a.pairs;
  c.prims = a.prims;
  c.primsf = a.primsf;
  c.D = a.D;
  c.J = a.J;
  c.K = a.K;
  c.nbf = a.nbf;
  c.nD = a.nD;
  c.want = a.want;
  return c;
}

// Resolve list position `task` of a JK launch into (bra pair, ket pair) and its job context.
__device__ __forceinline__ void resolve_task(const KernelArgs& a, long long task, bool listed, TaskCtx& ctx, int& ib,
                                             int& ik) {
  if (a.jobs != nullptr) {
    const unsigned long long e =
        a.from_back ? a.blist[a.list_cap - 1 - (unsigned long long)task] : a.blist[task];
    const JobDesc& jd = a.jobs[e >> 32];
    ctx.pairs = jd.pairs;
    ctx.prims = jd.prims;
    ctx.primsf = jd.primsf;
    ctx.D = jd.D;
    ctx.J = jd.J;
    ctx.K = jd.K;
    ctx.nbf = jd.nbf;
    ctx.nD = jd.nD;
    ctx.want = jd.want;
    decode_task_in((long long)(e & 0xffffffffULL), a.X == a.Y, jd.type_off[a.X], jd.type_off[a.Y],
                   jd.type_cnt[a.Y], ib, ik);
  } else if (listed) {
    const unsigned t = a.from_back ? a.tlist[a.list_cap - 1 - (unsigned long long)task] : a.tlist[task];
    decode_task(a, (long long)t, ib, ik);
  } else {
    decode_task(a, task, ib, ik);
  }
}

// Screening and precision of one unique quartet.  0: dropped, Q_ij Q_kl max|D| < tau with
// max|D| over the six cross blocks (Eqs. 7-9); 1: FP64; 2: FP32 recurrences (mixed mode
// only).  The mixed mode bounds what the FP32 stage produces, the contracted [e0|f0] before
// the FP64 transfer relations: |[e0|f0]| <= sqrt([e0|e0] [f0|f0]) (Cauchy-Schwarz), and the
// transfer relations multiply an [e0| error by at most (1 + max_x |A-B|_x)^lb, so the split
// compares Qe_ij Qe_kl max|D| (>= the Eq. 7-9 bound; equal to it when lb = ld = 0) with
// mixed_thr.
__device__ __forceinline__ int quartet_category(const KernelArgs& a, const ShellPair* bra, const ShellPair* ket,
                                                bool mixed) {
  const int P = bra->sh0, Qs = bra->sh1, Rr = ket->sh0, S = ket->sh1;
  const double* Dm = a.Dmax;
  const int n = a.nsh;
  const double dm = fmax(fmax(Dm[P * n + Qs], Dm[Rr * n + S]),
                         fmax(fmax(Dm[P * n + Rr], Dm[P * n + S]), fmax(Dm[Qs * n + Rr], Dm[Qs * n + S])));
  if (!(bra->Q * ket->Q * dm >= a.tau)) return 0;
  if (!mixed) return 1;
  return ((double)bra->Qe * (double)ket->Qe * dm > a.mixed_thr) ? 1 : 2;
}

// Per-primitive-quartet scalars in shared memory: NPD doubles (root lookup, FP64 always)
// followed by NPR values of the recurrence type R.
#define NPD 4
#define NPR 18

template <typename R> struct PairOf;
template <> struct PairOf<double> { typedef PrimPair type; };
template <> struct PairOf<float> { typedef PrimPairF type; };


// Digestion of one contracted quartet (ab|cd) from shared memory (team kernels): the team
// copies G = (ab|cd) (rows ldg = ncd | 1 apart) and the six density blocks D_ab, D_cd, D_ac,
// D_bd, D_ad, D_bc of each density into its shared region, then every output element of
// J~ and K~ is a dot product over shared data followed by one atomic.  The sums run in the
// same order as in the global-memory form below, so both give the same bits.  Every lane
// of the team calls it (team synchronisations inside).
template <int TS>
__device__ __forceinline__ void digest_shared(const TaskCtx& tc, const ClassDesc& c, const double* G, int sab, int scd,
                                              double* sh, int tl, bool active, double w, int p0, int q0b, int r0,
                                              int s0) {
  const int na = c.na, nb = c.nb, nc = c.nc, nd = c.nd, nab = na * nb, ncd = nc * nd;
  const int ldg = ncd | 1;
  double* Gs = sh;
  double* Dab = Gs + nab * ldg;
  double* Dcd = Dab + nab;
  double* Dac = Dcd + ncd;
  double* Dbd = Dac + na * nc;
  double* Dad = Dbd + nb * nd;
  double* Dbc = Dad + na * nd;
  const int nbf = tc.nbf;
  if (active)
    for (int t = tl; t < nab * ncd; t += TS) {
      const int ab = t / ncd, cd = t - (t / ncd) * ncd;
      Gs[ab * ldg + cd] = G[ab * sab + cd * scd];
    }
  const int nDw = warp_max(active ? tc.nD : 0);
  for (int xd = 0; xd < nDw; ++xd) {
    const bool on = active && xd < tc.nD;
    const double* Dx = tc.D + (size_t)xd * nbf * nbf;
    if (on) {
      for (int t = tl; t < nab; t += TS) Dab[t] = __ldg(Dx + (size_t)(p0 + t / nb) * nbf + q0b + t % nb);
      for (int t = tl; t < ncd; t += TS) Dcd[t] = __ldg(Dx + (size_t)(r0 + t / nd) * nbf + s0 + t % nd);
      for (int t = tl; t < na * nc; t += TS) Dac[t] = __ldg(Dx + (size_t)(p0 + t / nc) * nbf + r0 + t % nc);
      for (int t = tl; t < nb * nd; t += TS) Dbd[t] = __ldg(Dx + (size_t)(q0b + t / nd) * nbf + s0 + t % nd);
      for (int t = tl; t < na * nd; t += TS) Dad[t] = __ldg(Dx + (size_t)(p0 + t / nd) * nbf + s0 + t % nd);
      for (int t = tl; t < nb * nc; t += TS) Dbc[t] = __ldg(Dx + (size_t)(q0b + t / nc) * nbf + r0 + t % nc);
    }
    team_sync<TS>();
    if (on) {
      if (tc.want & 1) {
        double* Jx = tc.J + (size_t)xd * nbf * nbf;
        for (int t = tl; t < nab; t += TS) {
          double s = 0.0;
#pragma unroll 4
          for (int cd = 0; cd < ncd; ++cd) s = fma(Gs[t * ldg + cd], Dcd[cd], s);
          atomicAdd(Jx + (size_t)(p0 + t / nb) * nbf + q0b + t % nb, 2.0 * w * s);
        }
        for (int t = tl; t < ncd; t += TS) {
          double s = 0.0;
#pragma unroll 4
          for (int ab = 0; ab < nab; ++ab) s = fma(Gs[ab * ldg + t], Dab[ab], s);
          atomicAdd(Jx + (size_t)(r0 + t / nd) * nbf + s0 + t % nd, 2.0 * w * s);
        }
      }
      if (tc.want & 2) {
        double* Kx = tc.K + (size_t)xd * nbf * nbf;
        for (int t = tl; t < na * nc; t += TS) {          // K_ac += w sum_bd g D_bd
          const int ia = t / nc, ic = t - (t / nc) * nc;
          double s = 0.0;
          for (int ibb = 0; ibb < nb; ++ibb)
            for (int id = 0; id < nd; ++id) s = fma(Gs[(ia * nb + ibb) * ldg + ic * nd + id], Dbd[ibb * nd + id], s);
          atomicAdd(Kx + (size_t)(p0 + ia) * nbf + r0 + ic, w * s);
        }
        for (int t = tl; t < nb * nd; t += TS) {          // K_bd += w sum_ac g D_ac
          const int ibb = t / nd, id = t - (t / nd) * nd;
          double s = 0.0;
          for (int ia = 0; ia < na; ++ia)
            for (int ic = 0; ic < nc; ++ic) s = fma(Gs[(ia * nb + ibb) * ldg + ic * nd + id], Dac[ia * nc + ic], s);
          atomicAdd(Kx + (size_t)(q0b + ibb) * nbf + s0 + id, w * s);
        }
        for (int t = tl; t < na * nd; t += TS) {          // K_ad += w sum_bc g D_bc
          const int ia = t / nd, id = t - (t / nd) * nd;
          double s = 0.0;
          for (int ibb = 0; ibb < nb; ++ibb)
            for (int ic = 0; ic < nc; ++ic) s = fma(Gs[(ia * nb + ibb) * ldg + ic * nd + id], Dbc[ibb * nc + ic], s);
          atomicAdd(Kx + (size_t)(p0 + ia) * nbf + s0 + id, w * s);
        }
        for (int t = tl; t < nb * nc; t += TS) {          // K_bc += w sum_ad g D_ad
          const int ibb = t / nc, ic = t - (t / nc) * nc;
          double s = 0.0;
          for (int ia = 0; ia < na; ++ia)
            for (int id = 0; id < nd; ++id) s = fma(Gs[(ia * nb + ibb) * ldg + ic * nd + id], Dad[ia * nd + id], s);
          atomicAdd(Kx + (size_t)(q0b + ibb) * nbf + r0 + ic, w * s);
        }
      }
    }
    team_sync<TS>();
  }
}

// Shared-memory doubles digest_shared needs for a class (G with odd rows + six D blocks).
__host__ __device__ inline int digest_shared_doubles(int na, int nb, int nc, int nd) {
  return na * nb * ((nc * nd) | 1) + na * nb + nc * nd + na * nc + nb * nd + na * nd + nb * nc;
}

// Transfer relations on the contracted [e0|f0] in E0, then digestion into J~ / K~ (KMODE_JK),
// the block (KMODE_BLOCK) or the diagonal maximum (KMODE_SCHWARZ).  Team-cooperative;
// every thread of the team calls it.  Team kernels pass their shared region sh of sh_cap
// doubles (free once the quartet's assembly is done): digestion then runs from shared
// memory when G and the density blocks fit (digest_shared).
template <int TS, typename R>
__device__ __forceinline__ void finish_quartet(const KernelArgs& a, const TaskCtx& tc, const ClassDesc& c, R* E0,
                                               R* bufA, R* bufB, int tl, bool active, const double* AB,
                                               const double* CD, const ShellPair* bra, const ShellPair* ket, int ib,
                                               int ik, long long task, double* sh = nullptr, int sh_cap = 0) {
  if (a.mode == KMODE_SCHWARZ) {  // [e0|e0] of the diagonal quartet (ne = nf), before the transfer
    double m = 0.0;
    if (active)
      for (int e = tl; e < c.ne; e += TS) m = fmax(m, fabs((double)E0[e * c.nf + e]));
    m = team_max<TS>(m);
    if (active && tl == 0) a.qout[a.ntask + task] = m;
  }
  // ---- 2. transfer relations: bra on e (vector over f), then ket on f (vector over ab)
  const int nab = c.na * c.nb, ncd = c.nc * c.nd;
  const R* G;
  int sab, scd;            // (ab|cd) = G[ab*sab + cd*scd]
  bool done = false;
  if constexpr (TS > 32 && sizeof(R) == 8) {
    // block teams: both sequences through the team's shared region in slices (only E0, the
    // bra result Y = (ab|f0] and G touch scratch); W vectors per slice as the region allows
    auto width = [&](int la_, int lb_, int nv) {
      const int fixed = 2 * hrr_seq_block_doubles(la_, lb_, 1) - hrr_seq_block_doubles(la_, lb_, 2);
      const int per = hrr_seq_block_doubles(la_, lb_, 2) - hrr_seq_block_doubles(la_, lb_, 1);
      return per > 0 ? min(min(nv, TS), (sh_cap - fixed) / per) : TS;
    };
    const int Wb = c.lb > 0 ? width(c.la, c.lb, c.nf) : TS;
    const int Wk = c.ld > 0 ? width(c.lc, c.ld, nab) : TS;
    if (sh != nullptr && Wb >= 1 && Wk >= 1) {
      const double* Yp = E0;
      if (c.lb > 0) {
        hrr_seq_block<TS>(c.la, c.lb, AB, c.nf, E0, c.nf, 1, bufA, 1, c.nf, sh, Wb, tl, active);
        Yp = bufA;
      }
      if (c.ld > 0) {
        hrr_seq_block<TS>(c.lc, c.ld, CD, nab, Yp, 1, c.nf, bufB, ncd, 1, sh, Wk, tl, active);
        G = bufB;
        sab = ncd;
        scd = 1;
      } else {
        G = Yp;
        sab = c.nf;
        scd = 1;
      }
      done = true;
    }
  }
  if (!done) {
    const R* Y = hrr_team<R, (TS > 32)>(c.la, c.lb, AB, c.nf, E0, c.nf, 1, bufA, bufB, tl, TS, active);
    G = hrr_team<R, (TS > 32)>(c.lc, c.ld, CD, nab, Y, 1, c.nf, bufA, bufB, tl, TS, active);
    sab = (c.ld > 0) ? 1 : c.nf;
    scd = (c.ld > 0) ? nab : 1;
  }

  // ---- 3. digestion (FP64) / output
  if (TS > 1 && sizeof(R) == 8 && a.mode == KMODE_JK && sh != nullptr &&
      digest_shared_doubles(c.na, c.nb, c.nc, c.nd) <= sh_cap) {
    double w = 1.0;
    if (active) {
      if (bra->sh0 == bra->sh1) w *= 0.5;
      if (ket->sh0 == ket->sh1) w *= 0.5;
      if (ib == ik) w *= 0.5;
    }
    digest_shared<TS>(tc, c, reinterpret_cast<const double*>(G), sab, scd, sh, tl, active, w,
                      active ? bra->bf0 : 0, active ? bra->bf1 : 0, active ? ket->bf0 : 0, active ? ket->bf1 : 0);
  } else if (a.mode == KMODE_JK) {
    if (active) {
      double w = 1.0;
      if (bra->sh0 == bra->sh1) w *= 0.5;
      if (ket->sh0 == ket->sh1) w *= 0.5;
      if (ib == ik) w *= 0.5;
      const int p0 = bra->bf0, q0b = bra->bf1, r0 = ket->bf0, s0 = ket->bf1;
      const int na = c.na, nb = c.nb, nc = c.nc, nd = c.nd;
      const int nbf = tc.nbf;
      for (int xd = 0; xd < tc.nD; ++xd) {
        const double* Dx = tc.D + (size_t)xd * nbf * nbf;
        if (tc.want & 1) {
          double* Jx = tc.J + (size_t)xd * nbf * nbf;
          for (int t = tl; t < nab; t += TS) {
            const int ia = t / nb, ibb = t - (t / nb) * nb;
            double s = 0.0;
            for (int cd = 0; cd < ncd; ++cd) {
              const int ic = cd / nd, id = cd - (cd / nd) * nd;
              s = fma((double)G[t * sab + cd * scd], __ldg(Dx + (size_t)(r0 + ic) * nbf + s0 + id), s);
            }
            atomicAdd(Jx + (size_t)(p0 + ia) * nbf + q0b + ibb, 2.0 * w * s);
          }
          for (int t = tl; t < ncd; t += TS) {
            const int ic = t / nd, id = t - (t / nd) * nd;
            double s = 0.0;
            for (int ab = 0; ab < nab; ++ab) {
              const int ia = ab / nb, ibb = ab - (ab / nb) * nb;
              s = fma((double)G[ab * sab + t * scd], __ldg(Dx + (size_t)(p0 + ia) * nbf + q0b + ibb), s);
            }
            atomicAdd(Jx + (size_t)(r0 + ic) * nbf + s0 + id, 2.0 * w * s);
          }
        }
        if (tc.want & 2) {
          double* Kx = tc.K + (size_t)xd * nbf * nbf;
          // K_ac += w sum_bd g D_bd
          for (int t = tl; t < na * nc; t += TS) {
            const int ia = t / nc, ic = t - (t / nc) * nc;
            double s = 0.0;
            for (int ibb = 0; ibb < nb; ++ibb)
              for (int id = 0; id < nd; ++id)
                s = fma((double)G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                        __ldg(Dx + (size_t)(q0b + ibb) * nbf + s0 + id), s);
            atomicAdd(Kx + (size_t)(p0 + ia) * nbf + r0 + ic, w * s);
          }
          // K_bd += w sum_ac g D_ac
          for (int t = tl; t < nb * nd; t += TS) {
            const int ibb = t / nd, id = t - (t / nd) * nd;
            double s = 0.0;
            for (int ia = 0; ia < na; ++ia)
              for (int ic = 0; ic < nc; ++ic)
                s = fma((double)G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                        __ldg(Dx + (size_t)(p0 + ia) * nbf + r0 + ic), s);
            atomicAdd(Kx + (size_t)(q0b + ibb) * nbf + s0 + id, w * s);
          }
          // K_ad += w sum_bc g D_bc
          for (int t = tl; t < na * nd; t += TS) {
            const int ia = t / nd, id = t - (t / nd) * nd;
            double s = 0.0;
            for (int ibb = 0; ibb < nb; ++ibb)
              for (int ic = 0; ic < nc; ++ic)
                s = fma((double)G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                        __ldg(Dx + (size_t)(q0b + ibb) * nbf + r0 + ic), s);
            atomicAdd(Kx + (size_t)(p0 + ia) * nbf + s0 + id, w * s);
          }
          // K_bc += w sum_ad g D_ad
          for (int t = tl; t < nb * nc; t += TS) {
            const int ibb = t / nc, ic = t - (t / nc) * nc;
            double s = 0.0;
            for (int ia = 0; ia < na; ++ia)
              for (int id = 0; id < nd; ++id)
                s = fma((double)G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                        __ldg(Dx + (size_t)(p0 + ia) * nbf + s0 + id), s);
            atomicAdd(Kx + (size_t)(q0b + ibb) * nbf + r0 + ic, w * s);
          }
        }
      }
    }
  } else if (a.mode == KMODE_BLOCK) {
    if (active) {
      double* out = a.blockout + a.blockoff[task];
      for (int t = tl; t < nab * ncd; t += TS) {
        const int ab = t / ncd, cd = t - (t / ncd) * ncd;
        out[t] = (double)G[ab * sab + cd * scd];
      }
    }
  } else {  // KMODE_SCHWARZ: bra and ket are the same pair; max_{a,b} |(ab|ab)|, max_e |[e0|e0]|
    double m = 0.0;
    if (active)
      for (int t = tl; t < nab; t += TS) m = fmax(m, fabs((double)G[t * sab + t * scd]));
    m = team_max<TS>(m);
    if (active && tl == 0) a.qout[task] = m;
  }
}
