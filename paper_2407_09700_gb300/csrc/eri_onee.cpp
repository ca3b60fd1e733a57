// One-electron integrals for the RHF driver: overlap S, kinetic T and nuclear
// attraction V over the same contracted Cartesian shells as the ERIs.  The paper
// evaluates these on the CPU (Sec. 4); so does this file (host C++, OpenMP).
//
//   S, T: Obara-Saika recursions on the 1D overlaps of the Gaussian product,
//         S_x(i, j+1) = PB_x S_x(i, j) + (i S_x(i-1, j) + j S_x(i, j-1)) / (2 zeta),
//         T_x(i, j) = beta (2j+1) S_x(i, j) - 2 beta^2 S_x(i, j+2) - j(j-1)/2 S_x(i, j-2);
//   V:    Obara-Saika vertical recursion on [e|A(0)|0]^(m) for every point charge,
//         then the transfer relation (a, b+1_i) = (a+1_i, b) + (A-B)_i (a, b).
//         The Boys values F_m(T) come from the Rys rule of Eq. 1: with N roots,
//         F_m(T) = sum_n w_n u_n^m exactly for m < 2N (the rule's moment property).
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/eri.h"
#include "eri_internal.h"
#include "rys_table.h"

namespace {

inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
inline int cart_below(int l) { return l * (l + 1) * (l + 2) / 6; }
inline int cart_index(int lx, int ly, int lz) {
  const int l = lx + ly + lz, r = ly + lz;
  return cart_below(l) + r * (r + 1) / 2 + lz;
}
inline void cart_lmn(int l, int pos, int v[3]) {
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= pos) ++r;
  const int lz = pos - r * (r + 1) / 2;
  v[0] = l - r;
  v[1] = r - lz;
  v[2] = lz;
}

// Host evaluation of the Rys table: N roots u and weights w at T.
void rys_host(int N, double T, double* u, double* w) {
  if (T < (double)RYS_TCUT[N]) {
    const int ti = (int)(RYS_SUB * T);
    const double x = 2.0 * (RYS_SUB * T - ti) - 1.0;
    const double* c = RYS_COEF + RYS_COEF_OFFSET[N] + (size_t)ti * N * 2 * (RYS_DEG + 1);
    for (int n = 0; n < N; ++n) {
      const double* cu = c + n * 2 * (RYS_DEG + 1);
      const double* cw = cu + RYS_DEG + 1;
      double a = cu[0], b = cw[0];
      for (int k = 1; k <= RYS_DEG; ++k) {
        a = a * x + cu[k];
        b = b * x + cw[k];
      }
      u[n] = a;
      w[n] = b;
    }
  } else {
    const int o = RYS_ASYM_OFFSET[N];
    for (int n = 0; n < N; ++n) {
      u[n] = RYS_ASYM_U[o + n] / T;
      w[n] = RYS_ASYM_W[o + n] / std::sqrt(T);
    }
  }
}

// F_m(T), m = 0..mmax, from the moments of the Rys rule with N = mmax/2 + 1 roots.
void boys_from_rys(int mmax, double T, double* F) {
  const int N = mmax / 2 + 1;
  double u[RYS_NMAX], w[RYS_NMAX];
  rys_host(N, T, u, w);
  for (int m = 0; m <= mmax; ++m) F[m] = 0.0;
  for (int n = 0; n < N; ++n) {
    double p = w[n];
    for (int m = 0; m <= mmax; ++m) {
      F[m] += p;
      p *= u[n];
    }
  }
}

// 1D overlaps S(i, j), i <= imax, j <= jmax (unnormalised, without the Gaussian prefactor).
void overlap_1d(double PA, double PB, double zeta, int imax, int jmax, double* S, int ld) {
  const double h = 0.5 / zeta;
  S[0] = std::sqrt(M_PI / zeta);
  for (int i = 0; i <= imax; ++i) {
    if (i > 0) {
      S[i * ld] = PA * S[(i - 1) * ld] + (i > 1 ? (i - 1) * h * S[(i - 2) * ld] : 0.0);
    }
    for (int j = 0; j < jmax; ++j) {
      double v = PB * S[i * ld + j];
      if (i > 0) v += i * h * S[(i - 1) * ld + j];
      if (j > 0) v += j * h * S[i * ld + j - 1];
      S[i * ld + j + 1] = v;
    }
  }
}

struct Basis1e {
  int nshell, nbf;
  std::vector<int> l, atom, nprim, off, bf0;
  std::vector<double> exps, coefs, coords;
};

}  // namespace

extern "C" void eri_host_normalise(int nshell, const int* l, const int* nprim, const int* off, const double* exps,
                                   const double* raw, double* out);

extern "C" eri_status eri_internal_fail(eri_status s, const char* msg);

extern "C" eri_status eri_one_electron(const eri_basis* basis, int ncharge, const double* charge_xyz,
                                       const double* charges, double* S, double* T, double* V) {
  if (!basis || !basis->coords || !basis->shell_l || !basis->shell_atom || !basis->shell_nprim ||
      !basis->shell_off || !basis->exps || !basis->coefs || basis->nshell < 1 || basis->natm < 1)
    return eri_internal_fail(ERI_ERR_ARG, "eri_one_electron: incomplete basis");
  if (ncharge < 0 || (ncharge > 0 && (!charge_xyz || !charges)))
    return eri_internal_fail(ERI_ERR_ARG, "eri_one_electron: bad charges");
  Basis1e b;
  b.nshell = basis->nshell;
  int nprim_total = 0;
  for (int s = 0; s < b.nshell; ++s) {
    const int l = basis->shell_l[s];
    if (l < 0 || l > ERI_LMAX) return eri_internal_fail(ERI_ERR_UNSUPPORTED_L, "eri_one_electron: l outside 0..4");
    if (basis->shell_nprim[s] < 1 || basis->shell_off[s] < 0 || basis->shell_atom[s] < 0 ||
        basis->shell_atom[s] >= basis->natm)
      return eri_internal_fail(ERI_ERR_BASIS, "eri_one_electron: malformed shell");
    nprim_total = std::max(nprim_total, basis->shell_off[s] + basis->shell_nprim[s]);
  }
  for (int p = 0; p < nprim_total; ++p)
    if (!(basis->exps[p] > 0) || !std::isfinite(basis->exps[p]))
      return eri_internal_fail(ERI_ERR_BASIS, "eri_one_electron: exponent must be finite and > 0");
  b.l.assign(basis->shell_l, basis->shell_l + b.nshell);
  b.atom.assign(basis->shell_atom, basis->shell_atom + b.nshell);
  b.nprim.assign(basis->shell_nprim, basis->shell_nprim + b.nshell);
  b.off.assign(basis->shell_off, basis->shell_off + b.nshell);
  b.exps.assign(basis->exps, basis->exps + nprim_total);
  b.coefs.assign(basis->coefs, basis->coefs + nprim_total);
  b.coords.assign(basis->coords, basis->coords + 3 * basis->natm);
  if (basis->normalise)
    eri_host_normalise(b.nshell, b.l.data(), b.nprim.data(), b.off.data(), b.exps.data(), basis->coefs,
                       b.coefs.data());
  b.bf0.resize(b.nshell);
  b.nbf = 0;
  for (int s = 0; s < b.nshell; ++s) {
    b.bf0[s] = b.nbf;
    b.nbf += ncart(b.l[s]);
  }
  const int nbf = b.nbf;
  if (S) memset(S, 0, sizeof(double) * nbf * nbf);
  if (T) memset(T, 0, sizeof(double) * nbf * nbf);
  if (V) memset(V, 0, sizeof(double) * nbf * nbf);

#pragma omp parallel for schedule(dynamic)
  for (int I = 0; I < b.nshell; ++I) {
    std::vector<double> Sx(12 * 12), Sy(12 * 12), Sz(12 * 12), Vt, Ve, F(12);
    for (int Jsh = 0; Jsh <= I; ++Jsh) {
      const int la = b.l[I], lb = b.l[Jsh], na = ncart(la), nb = ncart(lb);
      const double* A = &b.coords[3 * b.atom[I]];
      const double* B = &b.coords[3 * b.atom[Jsh]];
      double AB[3], AB2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        AB[x] = A[x] - B[x];
        AB2 += AB[x] * AB[x];
      }
      std::vector<double> blkS(na * nb, 0.0), blkT(na * nb, 0.0), blkV(na * nb, 0.0);
      const int Le = la + lb, ne_all = cart_below(Le + 1);
      Ve.assign((size_t)ne_all, 0.0);                     // contracted [e|V|0] of this shell pair
      for (int p = 0; p < b.nprim[I]; ++p)
        for (int q = 0; q < b.nprim[Jsh]; ++q) {
          const double al = b.exps[b.off[I] + p], be = b.exps[b.off[Jsh] + q];
          const double cc = b.coefs[b.off[I] + p] * b.coefs[b.off[Jsh] + q];
          const double zeta = al + be;
          const double K = std::exp(-al * be / zeta * AB2);
          double P[3], PA[3], PB[3];
          for (int x = 0; x < 3; ++x) {
            P[x] = (al * A[x] + be * B[x]) / zeta;
            PA[x] = P[x] - A[x];
            PB[x] = P[x] - B[x];
          }
          // ---- S and T from 1D overlaps with j up to lb + 2
          const int ld = lb + 3;
          overlap_1d(PA[0], PB[0], zeta, la, lb + 2, Sx.data(), ld);
          overlap_1d(PA[1], PB[1], zeta, la, lb + 2, Sy.data(), ld);
          overlap_1d(PA[2], PB[2], zeta, la, lb + 2, Sz.data(), ld);
          const double* S1[3] = {Sx.data(), Sy.data(), Sz.data()};
          for (int ia = 0; ia < na; ++ia) {
            int av[3];
            cart_lmn(la, ia, av);
            for (int jb = 0; jb < nb; ++jb) {
              int bv[3];
              cart_lmn(lb, jb, bv);
              double s[3], t[3];
              for (int x = 0; x < 3; ++x) {
                const int i = av[x], j = bv[x];
                s[x] = S1[x][i * ld + j];
                t[x] = be * (2 * j + 1) * S1[x][i * ld + j] - 2.0 * be * be * S1[x][i * ld + j + 2];
                if (j >= 2) t[x] -= 0.5 * j * (j - 1) * S1[x][i * ld + j - 2];
              }
              blkS[ia * nb + jb] += cc * K * s[0] * s[1] * s[2];
              blkT[ia * nb + jb] += cc * K * (t[0] * s[1] * s[2] + s[0] * t[1] * s[2] + s[0] * s[1] * t[2]);
            }
          }
          // ---- V: OS vertical recursion on [e|C|0]^(m), |e| <= Le, per charge
          if (V && ncharge > 0) {
            const int nm = Le + 1;
            Vt.assign((size_t)ne_all * nm, 0.0);
            for (int ic = 0; ic < ncharge; ++ic) {
              const double* Cc = charge_xyz + 3 * ic;
              double PC[3], PC2 = 0.0;
              for (int x = 0; x < 3; ++x) {
                PC[x] = P[x] - Cc[x];
                PC2 += PC[x] * PC[x];
              }
              boys_from_rys(Le, zeta * PC2, F.data());
              const double pre = -charges[ic] * 2.0 * M_PI / zeta * K;
              for (int m = 0; m <= Le; ++m) Vt[m] = pre * F[m];
              const double h = 0.5 / zeta;
              for (int le = 1; le <= Le; ++le)
                for (int pe = 0; pe < ncart(le); ++pe) {
                  int e[3];
                  cart_lmn(le, pe, e);
                  const int i = e[0] ? 0 : (e[1] ? 1 : 2);
                  int em[3] = {e[0], e[1], e[2]};
                  em[i] -= 1;
                  const int ie = cart_index(e[0], e[1], e[2]), iem = cart_index(em[0], em[1], em[2]);
                  const int n = em[i];
                  int iemm = -1;
                  if (n > 0) {
                    int emm[3] = {em[0], em[1], em[2]};
                    emm[i] -= 1;
                    iemm = cart_index(emm[0], emm[1], emm[2]);
                  }
                  for (int m = 0; m <= Le - le; ++m) {
                    double v = PA[i] * Vt[iem * nm + m] - PC[i] * Vt[iem * nm + m + 1];
                    if (n > 0) v += n * h * (Vt[iemm * nm + m] - Vt[iemm * nm + m + 1]);
                    Vt[ie * nm + m] = v;
                  }
                }
              for (int e = 0; e < ne_all; ++e) Ve[e] += cc * Vt[e * nm];
            }
          }
        }
      // ---- transfer (a, b+1_i) = (a+1_i, b) + AB_i (a, b) on the contracted [e|V|0]
      if (V && ncharge > 0) {
        std::vector<double> cur(Ve.begin() + cart_below(la), Ve.end());   // |e| in [la, Le]
        int cur_nb = 1;
        for (int k = 1; k <= lb; ++k) {
          const int base = cart_below(la);
          const int na_k = cart_below(la + lb - k + 1) - base;
          const int nbk = ncart(k), nbm = ncart(k - 1);
          std::vector<double> nxt((size_t)na_k * nbk);
          for (int ia = 0; ia < na_k; ++ia) {
            const int g = base + ia;
            int lg = 0;
            while (cart_below(lg + 1) <= g) ++lg;
            int av[3];
            cart_lmn(lg, g - cart_below(lg), av);
            for (int pb = 0; pb < nbk; ++pb) {
              int bv[3];
              cart_lmn(k, pb, bv);
              const int i = bv[0] ? 0 : (bv[1] ? 1 : 2);
              int bm[3] = {bv[0], bv[1], bv[2]};
              bm[i] -= 1;
              const int pbm = cart_index(bm[0], bm[1], bm[2]) - cart_below(k - 1);
              int ap[3] = {av[0], av[1], av[2]};
              ap[i] += 1;
              const int iap = cart_index(ap[0], ap[1], ap[2]) - base;
              nxt[(size_t)ia * nbk + pb] = cur[(size_t)iap * nbm + pbm] + AB[i] * cur[(size_t)ia * nbm + pbm];
            }
          }
          cur.swap(nxt);
          cur_nb = nbk;
        }
        for (int ia = 0; ia < na; ++ia)
          for (int jb = 0; jb < nb; ++jb) blkV[ia * nb + jb] = cur[(size_t)ia * cur_nb + jb];
      }
      const int a0 = b.bf0[I], b0 = b.bf0[Jsh];
      for (int ia = 0; ia < na; ++ia)
        for (int jb = 0; jb < nb; ++jb) {
          const size_t u = (size_t)(a0 + ia) * nbf + b0 + jb, v = (size_t)(b0 + jb) * nbf + a0 + ia;
          if (S) S[u] = S[v] = blkS[ia * nb + jb];
          if (T) T[u] = T[v] = blkT[ia * nb + jb];
          if (V) V[u] = V[v] = blkV[ia * nb + jb];
        }
    }
  }
  return ERI_OK;
}
