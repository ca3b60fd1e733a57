// Two-electron energy-gradient class kernels (arXiv 2407.09700, Sec. 4, Eqs. 10-14,
// Alg. 4), written for sm_103a.
//
// With a fixed symmetric density D, E_J = 1/2 sum_abcd (ab|cd) D_ab D_cd and
// E_K = -1/4 sum_abcd (ab|cd) D_ac D_bd.  Their nuclear gradients are double contractions
// of the ERI derivatives with density products, accumulated directly (the derivative Fock
// matrices are never formed).  One launch per angular-momentum class runs over the unique
// shell quartets of the J/K build (8-fold symmetry, the same screening); a team of TS lanes
// owns one quartet at a time:
//   1. primitive loop: Rys roots for L+1, 2D tables one order higher on the bra
//      (Le+1) and on the ket (Lf+1), and four contracted sets of [e0|f0] (Eq. 1 products,
//      Eq. 5 contraction): unweighted, and weighted per primitive quartet by 2 alpha,
//      2 beta, 2 gamma (exponents of the primitives on centres A, B, C), the weights folded
//      into three scaled copies of the I_z table so that the sets share their I_x I_y
//      products (lane programs).  This is Eq. 10's linear map on the 2D integrals,
//      d/dA_x = 2 alpha (+1_x) - a_x (-1_x), applied after contraction;
//   2. the six shifted blocks (a+-1 b|cd), (a b+-1|cd), (ab|c+-1 d) by the transfer
//      relations, so d(ab|cd)/dA_x = (a+1_x b|cd)_{2 alpha} - a_x (a-1_x b|cd) and likewise
//      for B and C; the derivative on D follows from translational invariance;
//   3. each block is contracted with Gamma_J = 4 w D_ab D_cd and
//      Gamma_K = -w (D_ac D_bd + D_ad D_bc), w the permutation weight of the unique quartet
//      (8 w ordered quartets share it); the 18 per-lane sums (J, K x centres A, B, C x xyz)
//      are reduced over the team and 24 values (with D = -(A + B + C)) go to the gradient
//      by FP64 atomics, once per quartet (Alg. 4's accumulate-then-add).
// Everything runs in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "eri_internal.h"

#include "eri_device.cuh"

#define GNPR 21   // NPR recurrence scalars, then 2 alpha, 2 beta, 2 gamma

__device__ __forceinline__ int ncart_d(int l) { return (l + 1) * (l + 2) / 2; }

// Contract one shifted block G with Gamma_J / Gamma_K.  pos = 0, 1, 2 names the shifted
// index (a, b or c), lsh its angular momentum; plus: the l+1 block (coefficient 1 on
// Gamma at index - 1_x), else the l-1 block (coefficient -(v_x + 1) on Gamma at index + 1_x).
// Element (i0, i1, i2, i3) of G sits at G[(i0 m1 + i1) sab + (i2 m3 + i3) scd].
template <int TS>
__device__ __forceinline__ void contract_shift(const double* G, int sab, int scd, int pos, int lsh, bool plus,
                                               const int n[4], const double* GJ, const double* GK, int tl,
                                               bool active, double gj[3], double gk[3]) {
  if (!active) return;
  int m[4] = {n[0], n[1], n[2], n[3]};
  m[pos] = ncart_d(lsh);
  const int total = m[0] * m[1] * m[2] * m[3];
  const int base = cart_below(lsh);
  for (int t = tl; t < total; t += TS) {
    int r = t;
    const int i3 = r % m[3];
    r /= m[3];
    const int i2 = r % m[2];
    r /= m[2];
    const int i1 = r % m[1];
    const int i0 = r / m[1];
    const double v = G[(i0 * m[1] + i1) * sab + (i2 * m[3] + i3) * scd];
    const int is = (pos == 0) ? i0 : (pos == 1 ? i1 : i2);
    const uchar4 cv = cart_of(base + is);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      int q[3] = {cv.x, cv.y, cv.z};
      double coef;
      if (plus) {
        if (q[x] == 0) continue;
        q[x] -= 1;
        coef = 1.0;
      } else {
        coef = -(double)(q[x] + 1);
        q[x] += 1;
      }
      const int ip = cart_pos(q[1], q[2]);
      const int j0 = (pos == 0) ? ip : i0;
      const int j1 = (pos == 1) ? ip : i1;
      const int j2 = (pos == 2) ? ip : i2;
      const int gi = ((j0 * n[1] + j1) * n[2] + j2) * n[3] + i3;
      const double cvv = coef * v;
      gj[x] = fma(cvv, GJ[gi], gj[x]);
      gk[x] = fma(cvv, GK[gi], gk[x]);
    }
  }
}

// Transfer relations for one shifted block: bra (la_, lb_) on the set S (row stride snf),
// starting at row eo and column fo, vectorised over the nv columns of the ket shell lc_;
// then ket (lc_, ld_).  Returns the block with its (ab, cd) strides.  Team-cooperative.
// Block teams (TS > 32) run both sequences through their shared region sh (sh_cap doubles,
// free once the assembly is done) in slices, as the J/K kernel does.
template <int TS>
__device__ __forceinline__ const double* shifted_block(const double* S, int snf, int eo, int fo, int la_, int lb_,
                                                       int lc_, int ld_, const double* AB, const double* CD,
                                                       double* bufA, double* bufB, int tl, bool active, int& sab,
                                                       int& scd, double* sh, int sh_cap) {
  const int nv = cart_below(lc_ + ld_ + 1) - cart_below(lc_);
  const double* X = S + (size_t)eo * snf + fo;
  if constexpr (TS > 32) {
    auto width = [&](int l0, int l1, int n) {
      const int fixed = 2 * hrr_seq_block_doubles(l0, l1, 1) - hrr_seq_block_doubles(l0, l1, 2);
      const int per = hrr_seq_block_doubles(l0, l1, 2) - hrr_seq_block_doubles(l0, l1, 1);
      return per > 0 ? min(min(n, TS), (sh_cap - fixed) / per) : TS;
    };
    const int nab = ncart_d(la_) * ncart_d(lb_);
    const int Wb = lb_ > 0 ? width(la_, lb_, nv) : TS;
    const int Wk = ld_ > 0 ? width(lc_, ld_, nab) : TS;
    if (sh != nullptr && Wb >= 1 && Wk >= 1) {
      const double* Y = X;
      int sab1 = snf;
      if (lb_ > 0) {       // (ab|f] at bufA[ab * nv + f]
        hrr_seq_block<TS>(la_, lb_, AB, nv, X, snf, 1, bufA, 1, nv, sh, Wb, tl, active);
        Y = bufA;
        sab1 = nv;
      }
      if (ld_ == 0) {
        sab = sab1;
        scd = 1;
        return Y;
      }
      // (ab|cd) at bufB[cd * nab + ab]
      hrr_seq_block<TS>(lc_, ld_, CD, nab, Y, 1, sab1, bufB, 1, nab, sh, Wk, tl, active);
      sab = 1;
      scd = nab;
      return bufB;
    }
  }
  const double* Y = hrr_team<double, (TS > 32)>(la_, lb_, AB, nv, X, snf, 1, bufA, bufB, tl, TS, active);
  const int sab1 = (lb_ > 0) ? nv : snf;
  const int nab = ncart_d(la_) * ncart_d(lb_);
  const double* G = hrr_team<double, (TS > 32)>(lc_, ld_, CD, nab, Y, 1, sab1, bufA, bufB, tl, TS, active);
  if (ld_ > 0) {
    sab = 1;
    scd = nab;
  } else {
    sab = sab1;
    scd = 1;
  }
  return G;
}

template <int TS>
__global__ void __launch_bounds__(TPB, (TS == 1 ? 3 : 2)) eri_grad_kernel(const GradArgs ga) {
  extern __shared__ double smem[];
  const KernelArgs& a = ga.k;
  const GradDesc& g = ga.g;
  // TS = TPB: one team per block (team barriers are __syncthreads), as in the J/K kernel
  constexpr bool BLK = TS > 32;
  static_assert(!BLK || TS == TPB, "a team is a warp's part or the whole block");
  constexpr int TEAMS_PER_WARP = BLK ? 1 : 32 / TS;
  const int lane = threadIdx.x & 31;
  const int tl = BLK ? (int)threadIdx.x : lane % TS;
  const int team_in_block = threadIdx.x / TS;
  const long long gteam = (long long)blockIdx.x * (TPB / TS) + team_in_block;
  const int N = g.nroots, nI = g.nI, Le2 = g.Le2, Lf2 = g.Lf2;
  const int bp = g.bp;

  // team region: [bp][NPD] doubles, then [bp][GNPR], then [bp][6][N][nI]: I_x, I_y and
  // I_z scaled by 1, 2 alpha, 2 beta, 2 gamma
  Smem<double> sd, sr;
  if (TS == 1) {
    sd.base = smem + threadIdx.x;
    sd.es = TPB;
    sr.base = smem + (size_t)TPB * bp * NPD + threadIdx.x;
    sr.es = TPB;
  } else {
    sd.base = smem + (size_t)team_in_block * g.team_doubles;
    sd.es = 1;
    sr.base = sd.base + bp * NPD;
    sr.es = 1;
  }
  const int S_2D = bp * GNPR;
  double* scr = a.scratch + gteam * g.scratch_per_team;
  const int nabcd = g.na * g.nb * g.nc * g.nd;
  double* GJ = scr + g.gam_off;
  double* GK = GJ + nabcd;
  double* bufA = scr + g.hrr_off;
  double* bufB = bufA + g.hrr_doubles;
  double* part = scr + g.part_off;     // slot-ordered partial sums between batches (several passes)
  const int nbase[4] = {g.na, g.nb, g.nc, g.nd};

  unsigned long long cnt_q = 0, cnt_p = 0;
  const long long ntask = (long long)*a.tcount;

  while (true) {
    unsigned long long tbase = 0;
    if constexpr (BLK) {
      __shared__ unsigned long long s_tbase;
      if (threadIdx.x == 0) s_tbase = atomicAdd(a.counter, 1ull);
      __syncthreads();
      tbase = s_tbase;
      __syncthreads();
    } else {
      if (lane == 0) tbase = atomicAdd(a.counter, (unsigned long long)TEAMS_PER_WARP);
      tbase = __shfl_sync(0xffffffffu, tbase, 0);
    }
    if (tbase >= (unsigned long long)ntask) break;
    const long long task = (long long)tbase + (BLK ? 0 : lane / TS);
    const bool active = task < ntask;

    int ib = 0, ik = 0;
    if (active) decode_task(a, (long long)a.tlist[task], ib, ik);
    const ShellPair* bra = a.pairs + ib;
    const ShellPair* ket = a.pairs + ik;
    const int npb = active ? bra->nprim : 0;
    const int npk = active ? ket->nprim : 0;
    const int nq = npb * npk;
    const int maxq = warp_max(nq);
    if (tl == 0 && active) {
      cnt_q += 1;
      cnt_p += (unsigned long long)nq;
    }
    double AB[3] = {0.0, 0.0, 0.0}, CD[3] = {0.0, 0.0, 0.0};
    if (active) {
      AB[0] = bra->AB[0]; AB[1] = bra->AB[1]; AB[2] = bra->AB[2];
      CD[0] = ket->AB[0]; CD[1] = ket->AB[1]; CD[2] = ket->AB[2];
    }
    const int boff = active ? bra->prim_off : 0, koff = active ? ket->prim_off : 0;

    // ---- 1. the four contracted sets, in passes of TS * GSLOTS values.  With several passes
    //      the batches of primitive quartets run outside the passes: the roots and 2D tables
    //      of a batch are evaluated once and each pass carries its partial sums in the team's
    //      scratch from batch to batch (as in the J/K class kernel).
    int o0 = 0, kcnt = 0;
    uint32_t pkd[GSLOTS];
    double acc[GSLOTS];
    uint32_t gm = 0u;
    auto slot_valid = [&](int k) -> bool {
      const int o = o0 + k * TS + tl;
      if (!(k < kcnt && o < g.nslot)) return false;
      const uint32_t p = (TS == 1) ? __ldg(g.outidx + o0 + k) : pkd[k];
      return !(p >> 31);
    };
    auto begin_pass = [&](int pass, bool from_part) {
      o0 = pass * TS * GSLOTS;
      kcnt = min(GSLOTS, (g.nslot - o0 + TS - 1) / TS);
#pragma unroll
      for (int k = 0; k < GSLOTS; ++k) {
        const int o = o0 + k * TS + tl;
        if (TS > 1) pkd[k] = (o < g.nslot) ? __ldg(g.outidx + o) : (1u << 31);
        acc[k] = 0.0;
      }
      if (from_part && active) {
#pragma unroll
        for (int k = 0; k < GSLOTS; ++k) {
          const int o = o0 + k * TS + tl;
          if (k < kcnt && o < g.nslot) acc[k] = part[o];
        }
      }
      gm = __ldg(g.gmask + pass);
    };
    auto end_pass = [&](bool last) {
      if (active) {
        if (last) {
#pragma unroll
          for (int k = 0; k < GSLOTS; ++k)
            if (slot_valid(k)) scr[__ldg(g.dst + o0 + k * TS + tl)] = acc[k];
        } else {
#pragma unroll
          for (int k = 0; k < GSLOTS; ++k) {
            const int o = o0 + k * TS + tl;
            if (k < kcnt && o < g.nslot) part[o] = acc[k];
          }
        }
      }
    };
    auto batch_tables = [&](int q0, int nbt) {
      // a. primitive-quartet scalars
      for (int j = tl; j < bp; j += TS) {
        if (j < nbt) {
          const int q = q0 + j;
          const PrimPair* x = a.prims + boff + q / npk;
          const PrimPair* y = a.prims + koff + q % npk;
          const double zeta = x->zeta, eta = y->zeta;
          const double rd = rsqrt(zeta + eta);
          const double PQ0 = x->P[0] - y->P[0], PQ1 = x->P[1] - y->P[1], PQ2 = x->P[2] - y->P[2];
          const double inv_s = rd * rd;
          const double T = zeta * eta * inv_s * fma(PQ0, PQ0, fma(PQ1, PQ1, PQ2 * PQ2));
          int ti;
          double xx, invT, rsqT;
          rys_locate(T, a.rys_tcut_d, ti, xx, invT, rsqT);
          const int od = j * NPD;
          sd[od + 0] = xx;
          sd[od + 1] = invT;
          sd[od + 2] = rsqT;
          sd[od + 3] = __longlong_as_double((long long)ti);
          const double rz = eta * inv_s, re = zeta * inv_s;
          const int o = j * GNPR;
          sr[o + 0] = x->PA[0]; sr[o + 1] = x->PA[1]; sr[o + 2] = x->PA[2];
          sr[o + 3] = y->PA[0]; sr[o + 4] = y->PA[1]; sr[o + 5] = y->PA[2];
          sr[o + 6] = rz * PQ0; sr[o + 7] = rz * PQ1; sr[o + 8] = rz * PQ2;
          sr[o + 9] = re * PQ0; sr[o + 10] = re * PQ1; sr[o + 11] = re * PQ2;
          sr[o + 12] = 0.5 * inv_s;
          sr[o + 13] = x->hz * rz;
          sr[o + 14] = y->hz * re;
          sr[o + 15] = x->E * y->E * rd;
          sr[o + 16] = x->hz;
          sr[o + 17] = y->hz;
          sr[o + 18] = 2.0 * x->alpha;
          sr[o + 19] = 2.0 * (zeta - x->alpha);
          sr[o + 20] = 2.0 * y->alpha;
        }
      }
      team_sync<TS>();
      // b. roots, weights and the 2D tables per (primitive, root), or per (primitive, root,
      //    axis) when that fills more of the team's lanes
      if (TS > 1 && g.split3) {
        for (int tk = tl; tk < bp * N * 3; tk += TS) {
          const int jn = tk / 3, ax = tk - jn * 3;
          const int j = jn / N, n = jn - (jn / N) * N;
          if (j < nbt) {
            const int od = j * NPD, o = j * GNPR;
            double u, w;
            rys_root(a.rys_coef, a.rys_au, a.rys_aw, N, (int)__double_as_longlong(sd[od + 3]), sd[od + 0],
                     sd[od + 1], sd[od + 2], n, u, w);
            const double B00 = u * sr[o + 12];
            const double B10 = fma(-u, sr[o + 13], sr[o + 16]);
            const double B01 = fma(-u, sr[o + 14], sr[o + 17]);
            const double Cax = fma(-u, sr[o + 6 + ax], sr[o + 0 + ax]);
            const double Cpx = fma(u, sr[o + 9 + ax], sr[o + 3 + ax]);
            const double I00 = (ax == 2) ? w * sr[o + 15] : 1.0;
            const int gt = S_2D + ((j * 6 + ax) * N + n) * nI;
            rys_2d1<double>(sr, gt, Le2, Lf2, I00, Cax, Cpx, B00, B10, B01);
            if (ax == 2) {
              const double w1 = sr[o + 18], w2 = sr[o + 19], w3 = sr[o + 20];
              for (int i = 0; i < nI; ++i) {
                const double z = sr[gt + i];
                sr[gt + N * nI + i] = w1 * z;
                sr[gt + 2 * N * nI + i] = w2 * z;
                sr[gt + 3 * N * nI + i] = w3 * z;
              }
            }
          }
        }
      } else {
        for (int tk = tl; tk < bp * N; tk += TS) {
          const int j = tk / N, n = tk - (tk / N) * N;
          if (j < nbt) {
            const int od = j * NPD, o = j * GNPR;
            double u, w;
            rys_root(a.rys_coef, a.rys_au, a.rys_aw, N, (int)__double_as_longlong(sd[od + 3]), sd[od + 0],
                     sd[od + 1], sd[od + 2], n, u, w);
            const double B00 = u * sr[o + 12];
            const double B10 = fma(-u, sr[o + 13], sr[o + 16]);
            const double B01 = fma(-u, sr[o + 14], sr[o + 17]);
            const double wt = w * sr[o + 15];
            const double C[3] = {fma(-u, sr[o + 6], sr[o + 0]), fma(-u, sr[o + 7], sr[o + 1]),
                                 fma(-u, sr[o + 8], sr[o + 2])};
            const double Cp[3] = {fma(u, sr[o + 9], sr[o + 3]), fma(u, sr[o + 10], sr[o + 4]),
                                  fma(u, sr[o + 11], sr[o + 5])};
            const int g0 = S_2D + ((j * 6 + 0) * N + n) * nI;
            const int og[3] = {g0, g0 + N * nI, g0 + 2 * N * nI};
            rys_2d3<double>(sr, og, Le2, Lf2, wt, C, Cp, B00, B10, B01);
            // the I_z table scaled by the primitive weights 2 alpha, 2 beta, 2 gamma
            const double w1 = sr[o + 18], w2 = sr[o + 19], w3 = sr[o + 20];
            for (int i = 0; i < nI; ++i) {
              const double z = sr[og[2] + i];
              sr[og[2] + N * nI + i] = w1 * z;
              sr[og[2] + 2 * N * nI + i] = w2 * z;
              sr[og[2] + 3 * N * nI + i] = w3 * z;
            }
          }
        }
      }
      team_sync<TS>();
    };
    auto assemble = [&](int nbt) {
      // c. assembly and contraction in registers by lane programs: a slot that starts a
      //    group forms the group's I_x I_y product, each value adds product x weighted I_z
      for (int j = 0; j < bp; ++j) {
        if (j < nbt) {
          for (int n = 0; n < N; ++n) {
            const int gx = S_2D + ((j * 6 + 0) * N + n) * nI;
            const int gy = gx + N * nI;
            const int gz = gy + N * nI;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < GSLOTS; ++k) {
              if (k < kcnt) {
                const uint32_t p = (TS == 1) ? __ldg(g.outidx + o0 + k) : pkd[k];
                if ((gm >> k) & 1u) v = sr[gx + (int)(p & 0xffu)] * sr[gy + (int)((p >> 8) & 0xffu)];
                acc[k] = fma(v, sr[gz + (int)((p >> 16) & 0xfffu)], acc[k]);
              }
            }
          }
        }
      }
      team_sync<TS>();
    };
    const int nbatch = (maxq + bp - 1) / bp;        // uniform
    if (g.npass > 1) {
      for (int bi = 0; bi < nbatch; ++bi) {
        const int q0 = bi * bp, nbt = min(bp, nq - q0);
        batch_tables(q0, nbt);
        for (int pass = 0; pass < g.npass; ++pass) {
          begin_pass(pass, bi > 0);
          assemble(nbt);
          end_pass(bi == nbatch - 1);
        }
      }
    } else {
      begin_pass(0, false);
      for (int bi = 0; bi < nbatch; ++bi) {
        const int q0 = bi * bp, nbt = min(bp, nq - q0);
        batch_tables(q0, nbt);
        assemble(nbt);
      }
      end_pass(true);
    }
    team_sync<TS>();

    // ---- Gamma_J, Gamma_K of this quartet
    if (active) {
      double w = 1.0;
      if (bra->sh0 == bra->sh1) w *= 0.5;
      if (ket->sh0 == ket->sh1) w *= 0.5;
      if (ib == ik) w *= 0.5;
      const int nbf = a.nbf;
      const double* D = a.D;
      const int p0 = bra->bf0, q0b = bra->bf1, r0 = ket->bf0, s0 = ket->bf1;
      for (int t = tl; t < nabcd; t += TS) {
        int r = t;
        const int id = r % g.nd;
        r /= g.nd;
        const int ic = r % g.nc;
        r /= g.nc;
        const int ibb = r % g.nb;
        const int ia = r / g.nb;
        const size_t A_ = p0 + ia, B_ = q0b + ibb, C_ = r0 + ic, D_ = s0 + id;
        const double dab = __ldg(D + A_ * nbf + B_), dcd = __ldg(D + C_ * nbf + D_);
        const double dac = __ldg(D + A_ * nbf + C_), dbd = __ldg(D + B_ * nbf + D_);
        const double dad = __ldg(D + A_ * nbf + D_), dbc = __ldg(D + B_ * nbf + C_);
        GJ[t] = 4.0 * w * dab * dcd;
        GK[t] = -w * fma(dac, dbd, dad * dbc);
      }
    }
    team_sync<TS>();

    // ---- 2-3. the six shifted blocks, contracted with Gamma
    double jA[3] = {0, 0, 0}, jB[3] = {0, 0, 0}, jC[3] = {0, 0, 0};
    double kA[3] = {0, 0, 0}, kB[3] = {0, 0, 0}, kC[3] = {0, 0, 0};
    const int la = g.la, lb = g.lb, lc = g.lc, ld = g.ld;
    const double* S0 = scr + g.s_off[0];
    const int e0row = cart_below(la) - cart_below(g.s_elo[0]);       // row of e = la in set 0
    const int f0col = cart_below(lc) - cart_below(g.s_flo[0]);       // column of f = lc in set 0
    int sab, scd;
    const double* G;
    // A+ : (a+1 b|cd) from the 2 alpha set
    G = shifted_block<TS>(scr + g.s_off[1], g.s_nf[1], 0, 0, la + 1, lb, lc, ld, AB, CD, bufA, bufB, tl, active,
                          sab, scd, TS > 1 ? sd.base : nullptr, g.team_doubles);
    contract_shift<TS>(G, sab, scd, 0, la + 1, true, nbase, GJ, GK, tl, active, jA, kA);
    team_sync<TS>();
    if (la > 0) {  // A- : (a-1 b|cd) from the unweighted set
      G = shifted_block<TS>(S0, g.s_nf[0], 0, f0col, la - 1, lb, lc, ld, AB, CD, bufA, bufB, tl, active, sab, scd,
                            TS > 1 ? sd.base : nullptr, g.team_doubles);
      contract_shift<TS>(G, sab, scd, 0, la - 1, false, nbase, GJ, GK, tl, active, jA, kA);
      team_sync<TS>();
    }
    // B+ : (a b+1|cd) from the 2 beta set
    G = shifted_block<TS>(scr + g.s_off[2], g.s_nf[2], 0, 0, la, lb + 1, lc, ld, AB, CD, bufA, bufB, tl, active,
                          sab, scd, TS > 1 ? sd.base : nullptr, g.team_doubles);
    contract_shift<TS>(G, sab, scd, 1, lb + 1, true, nbase, GJ, GK, tl, active, jB, kB);
    team_sync<TS>();
    if (lb > 0) {  // B- : (a b-1|cd)
      G = shifted_block<TS>(S0, g.s_nf[0], e0row, f0col, la, lb - 1, lc, ld, AB, CD, bufA, bufB, tl, active, sab,
                            scd, TS > 1 ? sd.base : nullptr, g.team_doubles);
      contract_shift<TS>(G, sab, scd, 1, lb - 1, false, nbase, GJ, GK, tl, active, jB, kB);
      team_sync<TS>();
    }
    // C+ : (ab|c+1 d) from the 2 gamma set
    G = shifted_block<TS>(scr + g.s_off[3], g.s_nf[3], 0, 0, la, lb, lc + 1, ld, AB, CD, bufA, bufB, tl, active,
                          sab, scd, TS > 1 ? sd.base : nullptr, g.team_doubles);
    contract_shift<TS>(G, sab, scd, 2, lc + 1, true, nbase, GJ, GK, tl, active, jC, kC);
    team_sync<TS>();
    if (lc > 0) {  // C- : (ab|c-1 d)
      G = shifted_block<TS>(S0, g.s_nf[0], e0row, 0, la, lb, lc - 1, ld, AB, CD, bufA, bufB, tl, active, sab, scd,
                            TS > 1 ? sd.base : nullptr, g.team_doubles);
      contract_shift<TS>(G, sab, scd, 2, lc - 1, false, nbase, GJ, GK, tl, active, jC, kC);
      team_sync<TS>();
    }

    // ---- team reduction and the once-per-quartet atomics
    if (TS > 1) {
      constexpr int W = TS < 32 ? TS : 32;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        for (int off = W / 2; off > 0; off >>= 1) {
          jA[x] += __shfl_xor_sync(0xffffffffu, jA[x], off);
          jB[x] += __shfl_xor_sync(0xffffffffu, jB[x], off);
          jC[x] += __shfl_xor_sync(0xffffffffu, jC[x], off);
          kA[x] += __shfl_xor_sync(0xffffffffu, kA[x], off);
          kB[x] += __shfl_xor_sync(0xffffffffu, kB[x], off);
          kC[x] += __shfl_xor_sync(0xffffffffu, kC[x], off);
        }
      }
    }
    if constexpr (BLK) {       // the block's warps: partial sums through shared memory
      __shared__ double red[TS / 32][18];
      if (lane == 0)
        for (int x = 0; x < 3; ++x) {
          red[threadIdx.x >> 5][x] = jA[x];
          red[threadIdx.x >> 5][3 + x] = jB[x];
          red[threadIdx.x >> 5][6 + x] = jC[x];
          red[threadIdx.x >> 5][9 + x] = kA[x];
          red[threadIdx.x >> 5][12 + x] = kB[x];
          red[threadIdx.x >> 5][15 + x] = kC[x];
        }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int w = 1; w < TS / 32; ++w)
          for (int x = 0; x < 3; ++x) {
            jA[x] += red[w][x];
            jB[x] += red[w][3 + x];
            jC[x] += red[w][6 + x];
            kA[x] += red[w][9 + x];
            kB[x] += red[w][12 + x];
            kC[x] += red[w][15 + x];
          }
    }
    if (active && tl == 0) {
      const int atA = __ldg(ga.sh_atom + bra->sh0), atB = __ldg(ga.sh_atom + bra->sh1);
      const int atC = __ldg(ga.sh_atom + ket->sh0), atD = __ldg(ga.sh_atom + ket->sh1);
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        atomicAdd(ga.gJ + 3 * atA + x, jA[x]);
        atomicAdd(ga.gJ + 3 * atB + x, jB[x]);
        atomicAdd(ga.gJ + 3 * atC + x, jC[x]);
        atomicAdd(ga.gJ + 3 * atD + x, -(jA[x] + jB[x] + jC[x]));
        atomicAdd(ga.gK + 3 * atA + x, kA[x]);
        atomicAdd(ga.gK + 3 * atB + x, kB[x]);
        atomicAdd(ga.gK + 3 * atC + x, kC[x]);
        atomicAdd(ga.gK + 3 * atD + x, -(kA[x] + kB[x] + kC[x]));
      }
    }
    team_sync<TS>();
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

// ------------------------------------------------------------------ host launchers
extern "C" int erik_upload_cart_tables_grad(void) { return (int)upload_cart_table(); }

static const void* grad_kernel_ptr(int ts) {
  switch (ts) {
    case 1: return (const void*)eri_grad_kernel<1>;
    case 8: return (const void*)eri_grad_kernel<8>;
    case 32: return (const void*)eri_grad_kernel<32>;
    case 128: return (const void*)eri_grad_kernel<128>;
  }
  return nullptr;
}

extern "C" int erik_grad_blocks_per_sm(int ts, int smem_bytes, int* out) {
  const void* k = grad_kernel_ptr(ts);
  if (!k) return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, TPB, smem_bytes);
}

extern "C" int erik_launch_grad(int ts, const GradArgs* a, int grid, int smem_bytes, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (ts) {
    case 1: eri_grad_kernel<1><<<grid, TPB, smem_bytes, s>>>(*a); break;
    case 8: eri_grad_kernel<8><<<grid, TPB, smem_bytes, s>>>(*a); break;
    case 32: eri_grad_kernel<32><<<grid, TPB, smem_bytes, s>>>(*a); break;
    case 128: eri_grad_kernel<128><<<grid, TPB, smem_bytes, s>>>(*a); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}
