// Rys-quadrature ERI class kernels and helpers for the integral-direct J/K build
// (arXiv 2407.09700, Secs. 2-3), written for sm_103a.
//
// One launch per angular-momentum class (la lb | lc ld).  A "team" of TS threads
// owns one contracted shell quartet at a time (TS = 1, 8 or 32); a warp holds
// 32/TS teams and all control flow is warp-uniform, so the FP64 pipe never runs a
// warp instruction for a team that has left the loop.  Per quartet:
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

#define TPB 128        // threads per block of the class kernels
#define GSLOTS 32      // accumulator slots per lane
#define NPS 24         // shared doubles of per-primitive-quartet scalars

__constant__ unsigned char c_cart[ERI_MAXCART][4];   // lx, ly, lz, l by global Cartesian index

__device__ __forceinline__ int cart_below(int l) { return l * (l + 1) * (l + 2) / 6; }
__device__ __forceinline__ int cart_pos(int ly, int lz) { int r = ly + lz; return r * (r + 1) / 2 + lz; }
__device__ __forceinline__ int cart_index(int lx, int ly, int lz) {
  return cart_below(lx + ly + lz) + cart_pos(ly, lz);
}

// ------------------------------------------------------------------ shared-memory accessor
// A team's shared region: element e lives at base[e * es].  TS = 1 interleaves the
// 128 private regions of a block (es = 128) so that a warp reading the same entry
// hits 32 consecutive words; larger teams use contiguous regions (es = 1).
struct Smem {
  double* base;
  int es;
  __device__ __forceinline__ double& operator[](int e) const { return base[e * es]; }
};

// ------------------------------------------------------------------ Rys roots and weights
__device__ __forceinline__ double horner12(const double* __restrict__ c, double x) {
  double a = __ldg(c);
#pragma unroll
  for (int k = 1; k <= 11; ++k) a = fma(a, x, __ldg(c + k));
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

// Prepare the table lookup for one T: ti >= 0 selects interval ti, else the large-T limit.
__device__ __forceinline__ void rys_locate(double T, double tcut, int& ti, double& x, double& invT, double& rsqT) {
  if (T < tcut) {
    ti = floor_nonneg(T);
    x = fma(2.0, T, -(double)(2 * ti + 1));
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
    const double* c = coef + ((size_t)ti * N + n) * 24;
    u = horner12(c, x);
    w = horner12(c + 12, x);
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
__device__ __forceinline__ void rys_2d3(const Smem& g, const int o[3], int Le, int Lf, double I0z,
                                        const double C[3], const double Cp[3], double B00, double B10,
                                        double B01) {
  const int L1 = Lf + 1;
  g[o[0]] = 1.0;
  g[o[1]] = 1.0;
  g[o[2]] = I0z;
  if (Le >= 1) {
    g[o[0] + L1] = C[0];
    g[o[1] + L1] = C[1];
    g[o[2] + L1] = C[2] * I0z;
  }
  double nb10 = B10;
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
  double mb01 = B01;
  for (int m = 1; m < Lf; ++m) {
#pragma unroll
    for (int a = 0; a < 3; ++a) g[o[a] + m + 1] = fma(Cp[a], g[o[a] + m], mb01 * g[o[a] + m - 1]);
    mb01 += B01;
  }
  // rows n >= 1
  double nb00 = B00;
  for (int n = 1; n <= Le; ++n) {
    const int r = n * L1;
#pragma unroll
    for (int a = 0; a < 3; ++a) g[o[a] + r + 1] = fma(Cp[a], g[o[a] + r], nb00 * g[o[a] + r - L1]);
    double mb = B01;
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

// ------------------------------------------------------------------ transfer (horizontal) relations
// Input element (e, v) at X[e*xe + v*xv] for la <= |e| <= la+lb (e relative to cart_below(la)).
// Output contiguous [a][b][v] with |a| = la, |b| = lb; returns the output pointer (X when lb = 0).
// Team-cooperative; every lane of the warp must call it (it contains __syncwarp).
__device__ const double* hrr_team(int la, int lb, const double* AB, int nv, const double* X, int xe,
                                  int xv, double* bufA, double* bufB, int tl, int TS, bool active) {
  const double* cur = X;
  int cse = xe, csb = 0, csv = xv;
  const int base = cart_below(la);
  for (int k = 1; k <= lb; ++k) {
    double* nxt = (cur == bufA) ? bufB : bufA;
    const int na = cart_below(la + lb - k + 1) - base;
    const int nb = (k + 1) * (k + 2) / 2;
    const int total = na * nb * nv;
    if (active) {
      for (int t = tl; t < total; t += TS) {
        const int v = t % nv;
        const int r = t / nv;
        const int ib = r % nb;
        const int ia = r / nb;
        const unsigned char* av = c_cart[base + ia];
        const unsigned char* bv = c_cart[cart_below(k) + ib];
        const int i = bv[0] ? 0 : (bv[1] ? 1 : 2);
        int bm[3] = {bv[0], bv[1], bv[2]};
        bm[i] -= 1;
        const int ibm = cart_pos(bm[1], bm[2]);
        int ap[3] = {av[0], av[1], av[2]};
        ap[i] += 1;
        const int iap = cart_index(ap[0], ap[1], ap[2]) - base;
        const double hi = cur[iap * cse + ibm * csb + v * csv];
        const double lo = cur[ia * cse + ibm * csb + v * csv];
        nxt[(ia * nb + ib) * nv + v] = fma(AB[i], lo, hi);
      }
    }
    __syncwarp();
    cur = nxt;
    cse = nb * nv;
    csb = nv;
    csv = 1;
  }
  return cur;
}

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(0xffffffffu, v); }

// ------------------------------------------------------------------ the class kernel
template <int TS>
__global__ void __launch_bounds__(TPB) eri_class_kernel(const KernelArgs a) {
  extern __shared__ double smem[];
  constexpr int TEAMS_PER_WARP = 32 / TS;
  const int lane = threadIdx.x & 31;
  const int tl = lane % TS;                          // lane within team
  const int team_in_block = threadIdx.x / TS;
  const long long gteam = (long long)blockIdx.x * (TPB / TS) + team_in_block;
  const ClassDesc& c = a.c;
  const int N = c.nroots, nI = c.nI, Le = c.Le, Lf = c.Lf;
  const int bp = c.bp;

  Smem sm;
  if (TS == 1) {
    sm.base = smem + threadIdx.x;
    sm.es = TPB;
  } else {
    sm.base = smem + (size_t)team_in_block * c.team_doubles;
    sm.es = 1;
  }
  double* scr = a.scratch + gteam * c.scratch_per_team;
  double* E0 = scr;                                  // [ne][nf] contracted [e0|f0]
  double* bufA = scr + c.nout;
  double* bufB = bufA + c.hrr_doubles;

  // layout of the shared team region
  const int S_PRIM = 0;                              // [bp][NPS]
  const int S_2D = bp * NPS;                         // [bp][3][N][nI]

  unsigned long long cnt_q = 0, cnt_p = 0;

  while (true) {
    // ---- fetch TEAMS_PER_WARP tasks per warp
    unsigned long long tbase = 0;
    if (lane == 0) tbase = atomicAdd(a.counter, (unsigned long long)TEAMS_PER_WARP);
    tbase = __shfl_sync(0xffffffffu, tbase, 0);
    if (tbase >= (unsigned long long)a.ntask) break;
    const long long task = (long long)tbase + lane / TS;
    bool active = task < a.ntask;

    // ---- decode the task into (bra pair, ket pair)
    int ib = 0, ik = 0;
    if (active) {
      if (a.mode != KMODE_JK) {
        ib = a.tasklist[2 * task];
        ik = a.tasklist[2 * task + 1];
      } else if (a.tri) {
        long long i = (long long)((sqrt(8.0 * (double)task + 1.0) - 1.0) * 0.5);
        while (i * (i + 1) / 2 > task) --i;
        while ((i + 1) * (i + 2) / 2 <= task) ++i;
        ib = a.bra0 + (int)i;
        ik = a.ket0 + (int)(task - i * (i + 1) / 2);
      } else {
        ib = a.bra0 + (int)(task / a.nket);
        ik = a.ket0 + (int)(task % a.nket);
      }
    }
    const ShellPair* bra = a.pairs + ib;
    const ShellPair* ket = a.pairs + ik;
    // ---- screening (Eqs. 7-9): Q_ij Q_kl max|D| over the six cross blocks >= tau
    if (active && a.mode == KMODE_JK) {
      const int P = bra->sh0, Qs = bra->sh1, R = ket->sh0, S = ket->sh1;
      const double* Dm = a.Dmax;
      const int n = a.nsh;
      double dm = fmax(fmax(Dm[P * n + Qs], Dm[R * n + S]),
                       fmax(fmax(Dm[P * n + R], Dm[P * n + S]), fmax(Dm[Qs * n + R], Dm[Qs * n + S])));
      active = bra->Q * ket->Q * dm >= a.tau;
    }
    const int npb = active ? bra->nprim : 0;
    const int npk = active ? ket->nprim : 0;
    const int nq = npb * npk;
    const int maxq = warp_max(nq);
    if (tl == 0 && active) { cnt_q += 1; cnt_p += (unsigned long long)nq; }

    double AB[3], CD[3];
    if (active) {
      AB[0] = bra->AB[0]; AB[1] = bra->AB[1]; AB[2] = bra->AB[2];
      CD[0] = ket->AB[0]; CD[1] = ket->AB[1]; CD[2] = ket->AB[2];
    }
    const PrimPair* pb = a.prims + (active ? bra->prim_off : 0);
    const PrimPair* pk = a.prims + (active ? ket->prim_off : 0);

    for (int pass = 0; pass < c.npass; ++pass) {
      // ---- my output slots for this pass
      const int o0 = pass * TS * GSLOTS;
      uint32_t pkd[GSLOTS];
      double acc[GSLOTS];
#pragma unroll
      for (int k = 0; k < GSLOTS; ++k) {
        const int o = o0 + k * TS + tl;
        pkd[k] = (o < c.nout) ? __ldg(c.outidx + o) : 0u;
        acc[k] = 0.0;
      }
      const int kcnt = min(GSLOTS, (c.nout - o0 + TS - 1) / TS);   // uniform

      for (int q0 = 0; q0 < maxq; q0 += bp) {
        const int nbt = min(bp, nq - q0);            // this team's primitives in the batch (may be <= 0)
        // ---- a. primitive-quartet scalars
        for (int j = tl; j < bp; j += TS) {
          if (j < nbt) {
            const int q = q0 + j;
            const PrimPair* x = pb + q / npk;
            const PrimPair* y = pk + q % npk;
            const double zeta = x->zeta, eta = y->zeta;
            const double s = zeta + eta;
            const double r = rsqrt(s);
            const double inv_s = r * r;
            const double PQ0 = x->P[0] - y->P[0], PQ1 = x->P[1] - y->P[1], PQ2 = x->P[2] - y->P[2];
            const double rz = eta * inv_s, re = zeta * inv_s;
            const double T = zeta * rz * fma(PQ0, PQ0, fma(PQ1, PQ1, PQ2 * PQ2));
            int ti;
            double xx, invT, rsqT;
            rys_locate(T, a.rys_tcut_d, ti, xx, invT, rsqT);
            const double hz = x->hz, he = y->hz;
            const int o = S_PRIM + j * NPS;
            sm[o + 0] = x->PA[0]; sm[o + 1] = x->PA[1]; sm[o + 2] = x->PA[2];
            sm[o + 3] = y->PA[0]; sm[o + 4] = y->PA[1]; sm[o + 5] = y->PA[2];
            sm[o + 6] = rz * PQ0; sm[o + 7] = rz * PQ1; sm[o + 8] = rz * PQ2;
            sm[o + 9] = re * PQ0; sm[o + 10] = re * PQ1; sm[o + 11] = re * PQ2;
            sm[o + 12] = 0.5 * inv_s;
            sm[o + 13] = hz;
            sm[o + 14] = he;
            sm[o + 15] = hz * rz;
            sm[o + 16] = he * re;
            sm[o + 17] = x->E * y->E * r;           // Theta with contraction coefficients
            sm[o + 18] = xx;
            sm[o + 19] = invT;
            sm[o + 20] = rsqT;
            sm[o + 21] = __longlong_as_double((long long)ti);
          }
        }
        __syncwarp();
        // ---- b. roots, weights and 2D integrals per (primitive, root)
        for (int tk = tl; tk < bp * N; tk += TS) {
          const int j = tk / N, n = tk - (tk / N) * N;
          if (j < nbt) {
            const int o = S_PRIM + j * NPS;
            double u, w;
            rys_root(a.rys_coef, a.rys_au, a.rys_aw, N, (int)__double_as_longlong(sm[o + 21]), sm[o + 18],
                     sm[o + 19], sm[o + 20], n, u, w);
            const double B00 = u * sm[o + 12];
            const double B10 = fma(-u, sm[o + 15], sm[o + 13]);
            const double B01 = fma(-u, sm[o + 16], sm[o + 14]);
            const double wt = w * sm[o + 17];
            const double C[3] = {fma(-u, sm[o + 6], sm[o + 0]), fma(-u, sm[o + 7], sm[o + 1]),
                                 fma(-u, sm[o + 8], sm[o + 2])};
            const double Cp[3] = {fma(u, sm[o + 9], sm[o + 3]), fma(u, sm[o + 10], sm[o + 4]),
                                  fma(u, sm[o + 11], sm[o + 5])};
            const int g0 = S_2D + ((j * 3 + 0) * N + n) * nI;
            const int og[3] = {g0, g0 + N * nI, g0 + 2 * N * nI};
            rys_2d3(sm, og, Le, Lf, wt, C, Cp, B00, B10, B01);
          }
        }
        __syncwarp();
        // ---- c. assembly of [e0|f0] (Eq. 1) and contraction (Eq. 5) in registers
        for (int j = 0; j < bp; ++j) {
          if (j < nbt) {
            for (int n = 0; n < N; ++n) {
              const int gx = S_2D + ((j * 3 + 0) * N + n) * nI;
              const int gy = gx + N * nI;
              const int gz = gy + N * nI;
#pragma unroll
              for (int k = 0; k < GSLOTS; ++k) {
                if (k < kcnt) {
                  const uint32_t p = pkd[k];
                  const double v = sm[gx + (int)(p & 0xffu)] * sm[gy + (int)((p >> 8) & 0xffu)];
                  acc[k] = fma(v, sm[gz + (int)((p >> 16) & 0xffu)], acc[k]);
                }
              }
            }
          }
        }
        __syncwarp();
      }
      // ---- contracted values of this pass -> team scratch
      if (active) {
#pragma unroll
        for (int k = 0; k < GSLOTS; ++k) {
          const int o = o0 + k * TS + tl;
          if (k < kcnt && o < c.nout) E0[o] = acc[k];
        }
      }
    }
    __syncwarp();

    // ---- 2. transfer relations: bra on e (vector over f), then ket on f (vector over ab)
    const int nab = c.na * c.nb, ncd = c.nc * c.nd;
    const double* Y = hrr_team(c.la, c.lb, AB, c.nf, E0, c.nf, 1, bufA, bufB, tl, TS, active);
    const double* G = hrr_team(c.lc, c.ld, CD, nab, Y, 1, c.nf, bufA, bufB, tl, TS, active);
    // (ab|cd) = G[ab*sab + cd*scd]
    const int sab = (c.ld > 0) ? 1 : c.nf;
    const int scd = (c.ld > 0) ? nab : 1;

    // ---- 3. digestion / output
    if (a.mode == KMODE_JK) {
      if (active) {
        double w = 1.0;
        if (bra->sh0 == bra->sh1) w *= 0.5;
        if (ket->sh0 == ket->sh1) w *= 0.5;
        if (ib == ik) w *= 0.5;
        const int p0 = bra->bf0, q0b = bra->bf1, r0 = ket->bf0, s0 = ket->bf1;
        const int na = c.na, nb = c.nb, nc = c.nc, nd = c.nd;
        const int nbf = a.nbf;
        for (int xd = 0; xd < a.nD; ++xd) {
          const double* Dx = a.D + (size_t)xd * nbf * nbf;
          if (a.want & 1) {
            double* Jx = a.J + (size_t)xd * nbf * nbf;
            for (int t = tl; t < nab; t += TS) {
              const int ia = t / nb, ibb = t - (t / nb) * nb;
              double s = 0.0;
              for (int cd = 0; cd < ncd; ++cd) {
                const int ic = cd / nd, id = cd - (cd / nd) * nd;
                s = fma(G[t * sab + cd * scd], __ldg(Dx + (size_t)(r0 + ic) * nbf + s0 + id), s);
              }
              atomicAdd(Jx + (size_t)(p0 + ia) * nbf + q0b + ibb, 2.0 * w * s);
            }
            for (int t = tl; t < ncd; t += TS) {
              const int ic = t / nd, id = t - (t / nd) * nd;
              double s = 0.0;
              for (int ab = 0; ab < nab; ++ab) {
                const int ia = ab / nb, ibb = ab - (ab / nb) * nb;
                s = fma(G[ab * sab + t * scd], __ldg(Dx + (size_t)(p0 + ia) * nbf + q0b + ibb), s);
              }
              atomicAdd(Jx + (size_t)(r0 + ic) * nbf + s0 + id, 2.0 * w * s);
            }
          }
          if (a.want & 2) {
            double* Kx = a.K + (size_t)xd * nbf * nbf;
            // K_ac += w sum_bd g D_bd
            for (int t = tl; t < na * nc; t += TS) {
              const int ia = t / nc, ic = t - (t / nc) * nc;
              double s = 0.0;
              for (int ibb = 0; ibb < nb; ++ibb)
                for (int id = 0; id < nd; ++id)
                  s = fma(G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                          __ldg(Dx + (size_t)(q0b + ibb) * nbf + s0 + id), s);
              atomicAdd(Kx + (size_t)(p0 + ia) * nbf + r0 + ic, w * s);
            }
            // K_bd += w sum_ac g D_ac
            for (int t = tl; t < nb * nd; t += TS) {
              const int ibb = t / nd, id = t - (t / nd) * nd;
              double s = 0.0;
              for (int ia = 0; ia < na; ++ia)
                for (int ic = 0; ic < nc; ++ic)
                  s = fma(G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                          __ldg(Dx + (size_t)(p0 + ia) * nbf + r0 + ic), s);
              atomicAdd(Kx + (size_t)(q0b + ibb) * nbf + s0 + id, w * s);
            }
            // K_ad += w sum_bc g D_bc
            for (int t = tl; t < na * nd; t += TS) {
              const int ia = t / nd, id = t - (t / nd) * nd;
              double s = 0.0;
              for (int ibb = 0; ibb < nb; ++ibb)
                for (int ic = 0; ic < nc; ++ic)
                  s = fma(G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
                          __ldg(Dx + (size_t)(q0b + ibb) * nbf + r0 + ic), s);
              atomicAdd(Kx + (size_t)(p0 + ia) * nbf + s0 + id, w * s);
            }
            // K_bc += w sum_ad g D_ad
            for (int t = tl; t < nb * nc; t += TS) {
              const int ibb = t / nc, ic = t - (t / nc) * nc;
              double s = 0.0;
              for (int ia = 0; ia < na; ++ia)
                for (int id = 0; id < nd; ++id)
                  s = fma(G[(ia * nb + ibb) * sab + (ic * nd + id) * scd],
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
          out[t] = G[ab * sab + cd * scd];
        }
      }
    } else {  // KMODE_SCHWARZ: bra and ket are the same pair; max_{a,b} |(ab|ab)|
      double m = 0.0;
      if (active)
        for (int t = tl; t < nab; t += TS) m = fmax(m, fabs(G[t * sab + t * scd]));
      if (TS > 1) {
        for (int off = TS / 2; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
      }
      if (active && tl == 0) a.qout[task] = m;
    }
    __syncwarp();
  }
  // ---- counters: one atomic pair per warp
  for (int off = 16; off > 0; off >>= 1) {
    cnt_q += __shfl_xor_sync(0xffffffffu, cnt_q, off);
    cnt_p += __shfl_xor_sync(0xffffffffu, cnt_p, off);
  }
  if (lane == 0 && a.stats) {
    atomicAdd(a.stats + 0, cnt_q);
    atomicAdd(a.stats + 1, cnt_p);
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
extern "C" int erik_upload_cart_tables(void) {
  unsigned char h[ERI_MAXCART][4];
  int g = 0;
  for (int l = 0; l <= 8; ++l)
    for (int lx = l; lx >= 0; --lx)
      for (int ly = l - lx; ly >= 0; --ly) {
        h[g][0] = (unsigned char)lx;
        h[g][1] = (unsigned char)ly;
        h[g][2] = (unsigned char)(l - lx - ly);
        h[g][3] = (unsigned char)l;
        ++g;
      }
  return (int)cudaMemcpyToSymbol(c_cart, h, sizeof(h));
}

extern "C" int erik_team_config(int ts, int* threads_per_block, int* max_g) {
  *threads_per_block = TPB;
  *max_g = GSLOTS;
  return (ts == 1 || ts == 8 || ts == 32) ? 0 : 1;
}

static const void* class_kernel_ptr(int ts) {
  switch (ts) {
    case 1: return (const void*)eri_class_kernel<1>;
    case 8: return (const void*)eri_class_kernel<8>;
    case 32: return (const void*)eri_class_kernel<32>;
  }
  return nullptr;
}

extern "C" int erik_blocks_per_sm(int ts, int smem_bytes, int* out) {
  const void* k = class_kernel_ptr(ts);
  if (!k) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, TPB, smem_bytes);
}

extern "C" int erik_launch_class(int ts, const KernelArgs* a, int grid, int smem_bytes, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (ts) {
    case 1: eri_class_kernel<1><<<grid, TPB, smem_bytes, s>>>(*a); break;
    case 8: eri_class_kernel<8><<<grid, TPB, smem_bytes, s>>>(*a); break;
    case 32: eri_class_kernel<32><<<grid, TPB, smem_bytes, s>>>(*a); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

extern "C" int erik_launch_dmax(const double* D, int nD, int nbf, int nsh, const int* sh_bf0, const int* sh_n,
                                double* Dmax, void* stream) {
  const long long n = (long long)nsh * nsh;
  const int grid = (int)((n + 255) / 256);
  dmax_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(D, nD, nbf, nsh, sh_bf0, sh_n, Dmax);
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
