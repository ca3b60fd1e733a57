// The Rys-quadrature class kernel of the J/K build (arXiv 2407.09700, Secs. 2-3), shared by
// the generic instantiations (eri_kernels.cu) and the ones compiled for a single class
// (eri_class_spec.cu).  See eri_kernels.cu for the per-quartet steps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eri_internal.h"

#include "eri_device.cuh"

#define XQ 12      // product indices a lane keeps in registers (products path)

// ------------------------------------------------------------------ the class kernel
// R = double: the FP64 path.  R = float: the FP32 path of the mixed mode (Sec. 2's
// recurrences, Eq. 1's products and the Eq. 5 contraction in FP32; T and the Rys roots /
// weights in FP64, rounded at the recurrence input; the transfer relations, digestion and
// the J / K accumulation in FP64).
// CLS < 0: one kernel for every class, with the class's root count, recurrence sizes and
// tables read from the ClassDesc at run time.  CLS = 1000 la + 100 lb + 10 lc + ld: the same
// kernel compiled for that one class (eri_class_spec.cu), so the root count N, the recurrence
// bounds Le, Lf and the table sizes are compile-time constants (the recurrence loops unroll
// and the shared-memory offsets fold); the slot tables are still read per pass.
//
// STAGE (FP64 team kernels compiled for one class): each team's bra and ket PrimPair records
// (at most STAGE_REC together) are copied into shared memory by two bulk copies completed on
// the team's mbarrier, and the primitive-quartet scalars read them there; larger pairs read
// global memory.  A wait that gives up (after ~1 s) sets *a.err and ends the warp's work.
#define STAGE_REC 20
template <int TS, typename R, bool XY, int CLS = -1, bool STAGE = false>
__global__ void __launch_bounds__(TPB, (TS == 1 ? 3 : ((sizeof(R) == 4 && !XY) ? 3 : 2))) eri_class_kernel(const KernelArgs a) {
  static_assert(!STAGE || (TS > 1 && sizeof(R) == 8), "staging is for FP64 team kernels");
  extern __shared__ double smem[];
  typedef typename PairOf<R>::type PP;
  // TS = TPB: one team per block (its warps share the quartet, the batch tables and the
  // scratch; team barriers are __syncthreads)
  constexpr bool BLK = TS > 32;
  static_assert(!BLK || TS == TPB, "a team is a warp's part or the whole block");
  constexpr int TEAMS_PER_WARP = BLK ? 1 : 32 / TS;
  const int lane = threadIdx.x & 31;
  const int tl = BLK ? (int)threadIdx.x : lane % TS;  // lane within team
  const int team_in_block = threadIdx.x / TS;
  const long long gteam = (long long)blockIdx.x * (TPB / TS) + team_in_block;
  const ClassDesc& c = a.c;
  constexpr bool SPEC = CLS >= 0;
  constexpr int SLe = SPEC ? CLS / 1000 + (CLS / 100) % 10 : 0, SLf = SPEC ? (CLS / 10) % 10 + CLS % 10 : 0;
  constexpr int SN = (SLe + SLf) / 2 + 1, SnI = (SLe + 1) * (SLf + 1);
  constexpr int SnIs = TS > 1 ? (SnI | 1) : SnI;
  const int N = SPEC ? SN : c.nroots, nIs = SPEC ? SnIs : c.nIs, Le = SPEC ? SLe : c.Le, Lf = SPEC ? SLf : c.Lf;
  const int bp = XY ? c.bp_xy : c.bp;
  const int npass = XY ? c.xy_npass : c.npass;
  const int nslot = XY ? c.nout : c.nslot;
  const uint32_t* outidx = XY ? c.xy_outidx : c.outidx;
  const uint32_t* dsttab = XY ? c.xy_dst : c.dst;

  // team region: [bp][NPD] doubles, then [bp][NPR] R, then [bp][3][N] tables of nI R, nIs apart
  Smem<double> sd;
  Smem<R> sr;
  if (TS == 1) {
    sd.base = smem + threadIdx.x;
    sd.es = TPB;
    sr.base = reinterpret_cast<R*>(smem + (size_t)TPB * bp * NPD) + threadIdx.x;
    sr.es = TPB;
  } else {
    sd.base = smem + (size_t)team_in_block * (XY ? c.team_doubles_xy : (sizeof(R) == 8 ? c.team_doubles : c.team_doubles_f32));
    sd.es = 1;
    sr.base = reinterpret_cast<R*>(sd.base + bp * NPD);
    sr.es = 1;
  }
  // staging area after the block's team regions: per team STAGE_REC records, then the
  // teams' mbarriers (16-byte aligned throughout)
  PrimPair* stage = nullptr;
  unsigned long long* mbar = nullptr;
  unsigned stage_phase = 0;
  if (STAGE) {
    const size_t team_bytes = sizeof(double) * (size_t)(XY ? c.team_doubles_xy : c.team_doubles);
    char* base = reinterpret_cast<char*>(smem) + (((size_t)(TPB / TS) * team_bytes + 15) & ~(size_t)15);
    stage = reinterpret_cast<PrimPair*>(base) + (size_t)team_in_block * STAGE_REC;
    mbar = reinterpret_cast<unsigned long long*>(base + (size_t)(TPB / TS) * STAGE_REC * sizeof(PrimPair)) +
           team_in_block;
    if (tl == 0) mbar_init(mbar, 1);
    __syncwarp();
  }
  const int S_2D = bp * NPR;                         // R offset of the 2D tables
  R* xyb = XY ? &sr[S_2D + bp * 3 * N * nIs] : nullptr;   // product buffers (xy classes)
  // contracted [e0|f0] and the transfer relations are FP64 in both paths: the FP32 path
  // hands its contracted values over before the transfer, whose cancellations grow with |A-B|
  double* scr = a.scratch + gteam * c.scratch_per_team;
  double* E0 = scr;                                  // [ne][nf] contracted [e0|f0]
  double* bufA = scr + c.nout;
  double* bufB = bufA + c.hrr_doubles;
  double* part = scr + c.part_off;                   // slot-ordered partial sums (several passes)

  unsigned long long cnt_q = 0, cnt_p = 0;

  const bool listed = (a.mode == KMODE_JK) && (a.tlist != nullptr || a.jobs != nullptr);
  const int qs = (a.mode == KMODE_JK && a.qsplit > 1) ? a.qsplit : 1;   // tasks per quartet
  const long long ntask = (listed ? (long long)*a.tcount : a.ntask) * qs;

  while (true) {
    // ---- fetch TEAMS_PER_WARP tasks per warp (one per block for a block-wide team)
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
    const long long slot = (long long)tbase + (BLK ? 0 : lane / TS);
    bool active = slot < ntask;
    const long long task = slot / qs;                // the quartet; ch: its primitive range
    const int ch = (int)(slot - task * qs);

    // ---- decode the task into (bra pair, ket pair)
    int ib = 0, ik = 0;
    TaskCtx tc = single_ctx(a);
    if (active) {
      if (a.mode != KMODE_JK) {
        ib = a.tasklist[2 * task];
        ik = a.tasklist[2 * task + 1];
      } else {
        resolve_task(a, task, listed, tc, ib, ik);
      }
    }
    const PP* prims_r = reinterpret_cast<const PP*>(sizeof(R) == 8 ? (const void*)tc.prims : (const void*)tc.primsf);
    const ShellPair* bra = tc.pairs + ib;
    const ShellPair* ket = tc.pairs + ik;
    // ---- screening (Eqs. 7-9) and, in the mixed mode, the precision split
    //      (quartet_category).  Listed tasks were screened by the compaction.
    if (active && a.mode == KMODE_JK && !listed) {
      const int cat = quartet_category(a, bra, ket, a.prec_sel != 0);
      active = cat != 0 && (a.prec_sel == 0 || cat == a.prec_sel);
    }
    const int npb = active ? bra->nprim : 0;
    const int npk = active ? ket->nprim : 0;
    // this task's primitive quartets [qlo, qlo + nq) of the quartet's npb * npk (the last
    // range is never empty, so it counts the quartet)
    const int nqf = npb * npk;
    const int qlo = (qs > 1) ? (int)((long long)ch * nqf / qs) : 0;
    const int nq = (qs > 1) ? (int)((long long)(ch + 1) * nqf / qs) - qlo : nqf;
    if (nq == 0) active = false;
    const int maxq = warp_max(nq);
    if (tl == 0 && active) { cnt_q += (ch == qs - 1) ? 1 : 0; cnt_p += (unsigned long long)nq; }

    double AB[3], CD[3];
    if (active) {
      AB[0] = bra->AB[0]; AB[1] = bra->AB[1]; AB[2] = bra->AB[2];
      CD[0] = ket->AB[0]; CD[1] = ket->AB[1]; CD[2] = ket->AB[2];
    }
    const int boff = active ? bra->prim_off : 0, koff = active ? ket->prim_off : 0;
    // the team's primitive pairs into shared memory (STAGE), when they fit
    bool staged = false;
    if (STAGE) {
      staged = active && npb + npk <= STAGE_REC;
      if (staged && tl == 0) {
        fence_proxy_async_smem();        // the team's earlier reads of the area come first
        mbar_arrive_expect_tx(mbar, (unsigned)((npb + npk) * sizeof(PrimPair)));
        bulk_copy_g2s(stage, tc.prims + boff, (unsigned)(npb * sizeof(PrimPair)), mbar);
        bulk_copy_g2s(stage + npb, tc.prims + koff, (unsigned)(npk * sizeof(PrimPair)), mbar);
      }
      bool ok = true;
      if (staged) {
        ok = mbar_wait_bounded(mbar, stage_phase);
        stage_phase ^= 1u;
      }
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0 && a.err) atomicOr(a.err, 1u);
        // let every copy this warp issued land before leaving (bounded as well)
        if (staged && !ok) mbar_wait_bounded(mbar, stage_phase ^ 1u);
        break;
      }
    }

    // Per pass: this lane's output slots (pkd), accumulators, group-start bits and (xy classes)
    // the pass's products.  Loop order: passes outside primitive batches (one pass, or the
    // FP32 path), or, for FP64 classes with several passes, batches outside passes, so that
    // the roots and 2D tables of a batch are evaluated once for all passes and each pass
    // carries its partial sums in the team's E0 scratch from batch to batch.
    int o0 = 0, kcnt = 0, ncp = 0;
    uint32_t pkd[GSLOTS];
    R acc[GSLOTS];
    uint32_t gm = 0u;
    const uint32_t* xyt = nullptr;
    uint32_t xq[XY ? XQ : 1];
    auto slot_valid = [&](int k) -> bool {
      const int o = o0 + k * TS + tl;
      if (!(k < kcnt && o < nslot)) return false;
      const uint32_t p = (TS == 1) ? __ldg(outidx + o0 + k) : pkd[k];
      return XY || !(p >> 31);
    };
    auto begin_pass = [&](int pass, bool from_part) {
      o0 = pass * TS * GSLOTS;
      kcnt = min(GSLOTS, (nslot - o0 + TS - 1) / TS);     // uniform
#pragma unroll
      for (int k = 0; k < GSLOTS; ++k) {
        const int o = o0 + k * TS + tl;
        // TS = 1: every lane has the same slots, so the index is re-read (broadcast) instead
        if (TS > 1) pkd[k] = (o < nslot) ? __ldg(outidx + o) : (1u << 31);
        acc[k] = R(0);
      }
      if (from_part && active) {
#pragma unroll
        for (int k = 0; k < GSLOTS; ++k) {
          const int o = o0 + k * TS + tl;
          if (k < kcnt && o < nslot) acc[k] = (R)part[o];
        }
      }
      gm = XY ? 0u : __ldg(c.gmask + pass);           // group starts (uniform)
      if (XY) {
        xyt = c.xytab + __ldg(c.passinfo + 2 * pass);
        ncp = (int)__ldg(c.passinfo + 2 * pass + 1);
#pragma unroll
        for (int i = 0; i < XQ; ++i) {
          const int t = tl + i * TS;
          xq[i] = (t < ncp) ? __ldg(xyt + t) : 0u;
        }
      }
    };
    // ---- contracted values of this pass -> team scratch: [e][f] order after the last batch,
    //      else the partial sums in slot order (consecutive lanes, consecutive addresses)
    auto end_pass = [&](bool last) {
      if (active) {
        if (last) {
#pragma unroll
          for (int k = 0; k < GSLOTS; ++k)
            if (slot_valid(k)) E0[(int)__ldg(dsttab + o0 + k * TS + tl)] = (double)acc[k];
        } else {
#pragma unroll
          for (int k = 0; k < GSLOTS; ++k) {
            const int o = o0 + k * TS + tl;
            if (k < kcnt && o < nslot) part[o] = (double)acc[k];
          }
        }
      }
    };
    // ---- a. and b. of one batch of primitive quartets (every lane of the warp calls it)
    auto batch_tables = [&](int q0, int nbt) {
      // ---- a. primitive-quartet scalars: T and the table lookup in FP64, the rest in R
      for (int j = tl; j < bp; j += TS) {
        if (j < nbt) {
          const int q = qlo + q0 + j;
          const int ixp = boff + q / npk, iyp = koff + q % npk;
          const PrimPair* xd = (STAGE && staged) ? stage + q / npk : tc.prims + ixp;
          const PrimPair* yd = (STAGE && staged) ? stage + npb + q % npk : tc.prims + iyp;
          const double s = xd->zeta + yd->zeta;
          const double rd = rsqrt(s);
          const double PQ0 = xd->P[0] - yd->P[0], PQ1 = xd->P[1] - yd->P[1], PQ2 = xd->P[2] - yd->P[2];
          const double T = xd->zeta * yd->zeta * (rd * rd) * fma(PQ0, PQ0, fma(PQ1, PQ1, PQ2 * PQ2));
          int ti;
          double xx, invT, rsqT;
          rys_locate(T, a.rys_tcut_d, ti, xx, invT, rsqT);
          const int od = j * NPD;
          sd[od + 0] = xx;
          sd[od + 1] = invT;
          sd[od + 2] = rsqT;
          sd[od + 3] = __longlong_as_double((long long)ti);
          const PP* x = (sizeof(R) == 8) ? reinterpret_cast<const PP*>(xd) : prims_r + ixp;
          const PP* y = (sizeof(R) == 8) ? reinterpret_cast<const PP*>(yd) : prims_r + iyp;
          const R zeta = x->zeta, eta = y->zeta;
          // P - Q and 1/sqrt(zeta + eta) from their FP64 values (P - Q formed in FP32 from
          // rounded centres would carry an absolute error of ~|P| 6e-8 bohr)
          const R r = (R)rd, P0 = (R)PQ0, P1 = (R)PQ1, P2 = (R)PQ2;
          const R inv_s = r * r;
          const R rz = eta * inv_s, re = zeta * inv_s;
          const R hz = x->hz, he = y->hz;
          const int o = j * NPR;
          sr[o + 0] = x->PA[0]; sr[o + 1] = x->PA[1]; sr[o + 2] = x->PA[2];
          sr[o + 3] = y->PA[0]; sr[o + 4] = y->PA[1]; sr[o + 5] = y->PA[2];
          sr[o + 6] = rz * P0; sr[o + 7] = rz * P1; sr[o + 8] = rz * P2;
          sr[o + 9] = re * P0; sr[o + 10] = re * P1; sr[o + 11] = re * P2;
          sr[o + 12] = R(0.5) * inv_s;
          sr[o + 13] = hz * rz;
          sr[o + 14] = he * re;
          sr[o + 15] = x->E * y->E * r;             // Theta with contraction coefficients
          sr[o + 16] = hz;
          sr[o + 17] = he;
        }
      }
      team_sync<TS>();
      // ---- b. roots, weights (FP64) and 2D integrals (R) per (primitive, root), or per
      //      (primitive, root, axis) when that fills more of the team's lanes
      if (TS > 1 && (XY ? c.split3_xy : c.split3)) {
        for (int tk = tl; tk < bp * N * 3; tk += TS) {
          const int jn = tk / 3, ax = tk - jn * 3;
          const int j = jn / N, n = jn - (jn / N) * N;
          if (j < nbt) {
            const int od = j * NPD, o = j * NPR;
            double ud, wd;
            rys_root(a.rys_coef, a.rys_au, a.rys_aw, N, (int)__double_as_longlong(sd[od + 3]), sd[od + 0],
                     sd[od + 1], sd[od + 2], n, ud, wd);
            const R u = (R)ud;
            const R B00 = u * sr[o + 12];
            const R B10 = fma(-u, sr[o + 13], sr[o + 16]);
            const R B01 = fma(-u, sr[o + 14], sr[o + 17]);
            const R Cax = fma(-u, sr[o + 6 + ax], sr[o + 0 + ax]);
            const R Cpx = fma(u, sr[o + 9 + ax], sr[o + 3 + ax]);
            const R I00 = (ax == 2) ? (R)wd * sr[o + 15] : R(1);
            rys_2d1<R>(sr, S_2D + ((j * 3 + ax) * N + n) * nIs, Le, Lf, I00, Cax, Cpx, B00, B10, B01);
          }
        }
      } else {
        for (int tk = tl; tk < bp * N; tk += TS) {
          const int j = tk / N, n = tk - (tk / N) * N;
          if (j < nbt) {
            const int od = j * NPD, o = j * NPR;
            double ud, wd;
            rys_root(a.rys_coef, a.rys_au, a.rys_aw, N, (int)__double_as_longlong(sd[od + 3]), sd[od + 0],
                     sd[od + 1], sd[od + 2], n, ud, wd);
            const R u = (R)ud, w = (R)wd;
            const R B00 = u * sr[o + 12];
            const R B10 = fma(-u, sr[o + 13], sr[o + 16]);
            const R B01 = fma(-u, sr[o + 14], sr[o + 17]);
            const R wt = w * sr[o + 15];
            const R C[3] = {fma(-u, sr[o + 6], sr[o + 0]), fma(-u, sr[o + 7], sr[o + 1]),
                            fma(-u, sr[o + 8], sr[o + 2])};
            const R Cp[3] = {fma(u, sr[o + 9], sr[o + 3]), fma(u, sr[o + 10], sr[o + 4]),
                             fma(u, sr[o + 11], sr[o + 5])};
            const int g0 = S_2D + ((j * 3 + 0) * N + n) * nIs;
            const int og[3] = {g0, g0 + N * nIs, g0 + 2 * N * nIs};
            rys_2d3<R>(sr, og, Le, Lf, wt, C, Cp, B00, B10, B01);
          }
        }
      }
      team_sync<TS>();
    };
    // ---- c. of one batch for the current pass
    auto assemble = [&](int nbt) {
      if (XY) {
        // products path: per (primitive, root) step the team forms this pass's distinct
        // I_x I_y products once, then each value is one FMA with I_z.  Software-pipelined
        // over steps: the products of step s+1 (buffer (s+1)&1) are formed while the FMAs
        // of step s read buffer s&1, with one warp synchronisation per step.  Steps of a
        // team past its primitive count compute on stale (in-bounds) table entries and
        // leave the accumulators unchanged.
        const int nsteps = warp_max(nbt) * N;
        auto form = [&](int st) {
          const int jj = st / N, nn = st - (st / N) * N;
          const int gx = S_2D + ((jj * 3 + 0) * N + nn) * nIs;
          const int gy = gx + N * nIs;
          R* buf = xyb + (st & 1) * c.xymax;
#pragma unroll
          for (int i = 0; i < XQ; ++i) {
            const int t = tl + i * TS;
            if (t < ncp) buf[t] = sr[gx + (int)(xq[i] & 0xffu)] * sr[gy + (int)((xq[i] >> 8) & 0xffu)];
          }
          for (int t = tl + XQ * TS; t < ncp; t += TS) {
            const uint32_t q = __ldg(xyt + t);
            buf[t] = sr[gx + (int)(q & 0xffu)] * sr[gy + (int)((q >> 8) & 0xffu)];
          }
        };
        if (nsteps > 0) form(0);
        team_sync<TS>();
        for (int st = 0; st < nsteps; ++st) {
          if (st + 1 < nsteps) form(st + 1);
          const int jj = st / N, nn = st - (st / N) * N;
          const bool jv = jj < nbt;
          const int gz = S_2D + ((jj * 3 + 2) * N + nn) * nIs;
          const R* buf = xyb + (st & 1) * c.xymax;
#pragma unroll
          for (int k = 0; k < GSLOTS; ++k) {
            if (k < kcnt) {
              const uint32_t p = pkd[k];
              const R v = fma(buf[(int)(p & 0xffffu)], sr[gz + (int)((p >> 16) & 0xffu)], acc[k]);
              acc[k] = jv ? v : acc[k];
            }
          }
          team_sync<TS>();
        }
      } else {
        // lane programs: a slot that starts a group forms the group's I_x I_y product, the
        // rest of the group reuses it; the start bits are the same for every lane
        for (int j = 0; j < bp; ++j) {
          if (j < nbt) {
            for (int n = 0; n < N; ++n) {
              const int gx = S_2D + ((j * 3 + 0) * N + n) * nIs;
              const int gy = gx + N * nIs;
              const int gz = gy + N * nIs;
              R v = R(0);
#pragma unroll
              for (int k = 0; k < GSLOTS; ++k) {
                if (k < kcnt) {
                  const uint32_t p = (TS == 1) ? __ldg(outidx + o0 + k) : pkd[k];
                  if ((gm >> k) & 1u) v = sr[gx + (int)(p & 0xffu)] * sr[gy + (int)((p >> 8) & 0xffu)];
                  acc[k] = fma(v, sr[gz + (int)((p >> 16) & 0xffu)], acc[k]);
                }
              }
            }
          }
        }
      }
      team_sync<TS>();
    };
    const int nbatch = (maxq + bp - 1) / bp;        // uniform
    if (sizeof(R) == 8 && npass > 1) {
      for (int bi = 0; bi < nbatch; ++bi) {
        const int q0 = bi * bp, nbt = min(bp, nq - q0);
        batch_tables(q0, nbt);
        for (int pass = 0; pass < npass; ++pass) {
          begin_pass(pass, bi > 0);
          assemble(nbt);
          end_pass(bi == nbatch - 1);
        }
      }
    } else {
      for (int pass = 0; pass < npass; ++pass) {
        begin_pass(pass, false);
        for (int bi = 0; bi < nbatch; ++bi) {
          const int q0 = bi * bp, nbt = min(bp, nq - q0);   // this team's primitives in the batch (may be <= 0)
          batch_tables(q0, nbt);
          assemble(nbt);
        }
        end_pass(true);
      }
    }
    team_sync<TS>();

    // the team's shared region is free here: team kernels digest from it
    finish_quartet<TS, double>(a, tc, c, E0, bufA, bufB, tl, active, AB, CD, bra, ket, ib, ik, task,
                               TS > 1 ? sd.base : nullptr,
                               XY ? c.team_doubles_xy : (sizeof(R) == 8 ? c.team_doubles : c.team_doubles_f32));
    team_sync<TS>();
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

