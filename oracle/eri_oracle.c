/*
 * CPU oracle for the integral-direct J/K build of arXiv 2407.09700 (GPU4PySCF).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA library.
 *
 * What it computes, in plain FP64:
 *   - contracted Cartesian ERIs (ij|kl) over the Gaussians of Eq. 2 and the
 *     contractions of Eqs. 4-5 (Sec. 2), by a different algorithm from the
 *     paper's Rys quadrature (Eq. 1): Obara-Saika vertical recursion on
 *     [e0|f0]^(m) followed by Head-Gordon-Pople horizontal recursion
 *     (Obara & Saika, JCP 84, 3963 (1986); Head-Gordon & Pople, JCP 89, 5777
 *     (1988)), with its own Boys function;
 *   - Coulomb J_ij = sum_kl (ij|kl) D_kl and exchange K_ik = sum_jl (ij|kl) D_jl
 *     by their definitions: every ordered shell quartet of a unique quartet's
 *     orbit under the 8-fold permutation symmetry (Sec. 3) is expanded
 *     explicitly, with no weight factors;
 *   - the Cauchy-Schwarz factor of Eq. 7 and the screening predicate built from
 *     Eqs. 7-9 (Sec. 3): a unique quartet is kept when Q_ij > tau, Q_kl > tau
 *     and Q_ij * Q_kl * max|D| over the six cross blocks >= tau.
 *
 * Conventions the paper leaves open (the same readings as the library's):
 *   - primitive radial norm (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!), then the
 *     contracted shell rescaled so its x^l component has unit self-overlap;
 *   - Cartesian order x-descending: for lx = l..0, for ly = l-lx..0;
 *   - atomic units (Bohr).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 5   /* l <= 4 shells and their l+1 derivative companions */
#define ORC_MMAX (4 * ORC_LMAX + 1)

/* ------------------------------------------------------------------ operation counter
 * Floating-point operations this oracle performs, by phase, on the calling thread: every
 * add, subtract, multiply and divide of the source counts 1, each exp / sqrt / erf / pow
 * call counts 1, negations and integer index arithmetic count 0.  The counts are added once per loop iteration from the statement counts
 * written beside each loop (integer additions only, so the oracle's own speed is not
 * affected).  oracle_class_ops reads them for one synthetic quartet of a class. */
enum { OPS_PRIM = 0, OPS_BOYS, OPS_VRR, OPS_CONTRACT, OPS_HRR, OPS_DIGEST, OPS_N };
static _Thread_local long long g_ops[OPS_N];
#define COUNT_OPS(phase, n) (g_ops[phase] += (long long)(n))

/* ------------------------------------------------------------------ Cartesian indexing */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }
/* number of Cartesian triples with total angular momentum below l */
static int cart_below(int l) { return l * (l + 1) * (l + 2) / 6; }
/* position of (lx,ly,lz) inside its shell, x-descending order */
static int cart_pos(int ly, int lz) { int r = ly + lz; return r * (r + 1) / 2 + lz; }
static int cart_index(int lx, int ly, int lz) { return cart_below(lx + ly + lz) + cart_pos(ly, lz); }
static void cart_lmn(int l, int pos, int v[3]) {
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= pos) ++r;
  int lz = pos - r * (r + 1) / 2;
  v[0] = l - r; v[1] = r - lz; v[2] = lz;
}

/* ------------------------------------------------------------------ Boys function */

/* F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt for m = 0..mmax.
 * T < 35: the everywhere-convergent positive series
 *   F_M(T) = exp(-T) sum_k (2T)^k / ((2M+1)(2M+3)...(2M+2k+1))
 * for the top order, then the stable downward recursion
 *   F_{m-1} = (2T F_m + exp(-T)) / (2m-1).
 * T >= 35: F_0 = (1/2) sqrt(pi/T) erf(sqrt T) and the upward recursion
 *   F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), stable while T is large. */
void oracle_boys(int mmax, double T, double* F) {
  double eT = exp(-T);
  COUNT_OPS(OPS_BOYS, 1);                                   /* exp */
  if (T < 35.0) {
    double term = 1.0 / (2 * mmax + 1), sum = term;
    COUNT_OPS(OPS_BOYS, 1);
    for (int k = 1; k < 100000; ++k) {
      term *= 2.0 * T / (2 * mmax + 2 * k + 1);
      sum += term;
      COUNT_OPS(OPS_BOYS, 5);                               /* 2T, /, *=, +=, 1e-18 sum */
      if (term < 1e-18 * sum) break;
    }
    F[mmax] = eT * sum;
    COUNT_OPS(OPS_BOYS, 1);
    for (int m = mmax; m > 0; --m) F[m - 1] = (2.0 * T * F[m] + eT) / (2 * m - 1);
    COUNT_OPS(OPS_BOYS, 4 * mmax);
  } else {
    F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
    COUNT_OPS(OPS_BOYS, 6);                                 /* pi/T, sqrt, sqrt, erf, two * */
    for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - eT) / (2.0 * T);
    COUNT_OPS(OPS_BOYS, 4 * mmax);
  }
}

/* ------------------------------------------------------------------ basis */

typedef struct {
  int natm;
  const double* coords;   /* natm*3, Bohr */
  int nshell;
  const int* atom;
  const int* l;
  const int* nprim;
  const int* off;
  const double* exps;
  const double* coefs;    /* normalised (oracle_normalise) */
} obasis;

static double dfact(int n) { double r = 1.0; for (int k = n; k > 1; k -= 2) r *= k; return r; }

/* Normalise raw contraction coefficients (convention in the header). */
void oracle_normalise(int nshell, const int* l, const int* nprim, const int* off,
                      const double* exps, const double* raw, double* out) {
  for (int s = 0; s < nshell; ++s) {
    int L = l[s], K = nprim[s], o = off[s];
    double df = dfact(2 * L - 1);
    for (int p = 0; p < K; ++p) {
      double a = exps[o + p];
      out[o + p] = raw[o + p] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * L) / sqrt(df);
    }
    /* self-overlap of the x^L component: int x^(2L) exp(-s r^2) = (2L-1)!!/(2s)^L (pi/s)^(3/2) */
    double S = 0.0;
    for (int p = 0; p < K; ++p)
      for (int q = 0; q < K; ++q) {
        double s2 = exps[o + p] + exps[o + q];
        S += out[o + p] * out[o + q] * df / pow(2.0 * s2, L) * pow(M_PI / s2, 1.5);
      }
    double f = 1.0 / sqrt(S);
    for (int p = 0; p < K; ++p) out[o + p] *= f;
  }
}

/* ------------------------------------------------------------------ OS vertical recursion */

/* Primitive [e|f]^(m) for all |e| <= Le, |f| <= Lf, m <= Le+Lf-|e|-|f|.
 * V is laid out [e][f][m] with e, f global Cartesian indices and m stride Lt+1. */
static void os_vrr(int Le, int Lf, double a, const double A[3], double b, const double B[3],
                   double c, const double C[3], double d, const double D[3], double* V) {
  int Lt = Le + Lf, nm = Lt + 1;
  int ne = cart_below(Le + 1), nf = cart_below(Lf + 1);
  double zeta = a + b, eta = c + d, s = zeta + eta, rho = zeta * eta / s;
  double P[3], Q[3], W[3], PA[3], WP[3], QC[3], WQ[3], AB2 = 0, CD2 = 0, PQ2 = 0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (a * A[i] + b * B[i]) / zeta;
    Q[i] = (c * C[i] + d * D[i]) / eta;
    W[i] = (zeta * P[i] + eta * Q[i]) / s;
    PA[i] = P[i] - A[i]; WP[i] = W[i] - P[i];
    QC[i] = Q[i] - C[i]; WQ[i] = W[i] - Q[i];
    AB2 += (A[i] - B[i]) * (A[i] - B[i]);
    CD2 += (C[i] - D[i]) * (C[i] - D[i]);
    PQ2 += (P[i] - Q[i]) * (P[i] - Q[i]);
  }
  double T = rho * PQ2;
  double theta = 2.0 * pow(M_PI, 2.5) / (zeta * eta * sqrt(s)) *
                 exp(-a * b / zeta * AB2) * exp(-c * d / eta * CD2);
  /* zeta, eta, s, rho (2); per axis P, Q, W (4 each), PA WP QC WQ, AB2 CD2 PQ2 (two
   * subtractions, a multiply and an add each); T; theta: pow, *, sqrt, two *, /, two exp with
   * 4 operations each, two * */
  COUNT_OPS(OPS_PRIM, 5 + 3 * (12 + 4 + 12) + 1 + 16);
  double F[ORC_MMAX + 1];
  oracle_boys(Lt, T, F);
#define VV(e, f, m) V[((size_t)(e) * nf + (f)) * nm + (m)]
  for (int m = 0; m <= Lt; ++m) VV(0, 0, m) = theta * F[m];
  COUNT_OPS(OPS_VRR, Lt + 1);
  /* bra: [e+1_i|0]^(m) = PA_i [e|0]^(m) + WP_i [e|0]^(m+1)
                          + e_i/(2 zeta) ([e-1_i|0]^(m) - rho/zeta [e-1_i|0]^(m+1)) */
  for (int le = 1; le <= Le; ++le)
    for (int pe = 0; pe < ncart(le); ++pe) {
      int e[3]; cart_lmn(le, pe, e);
      int i = e[0] ? 0 : (e[1] ? 1 : 2);
      int em[3] = {e[0], e[1], e[2]}; em[i] -= 1;
      int ie = cart_index(e[0], e[1], e[2]), iem = cart_index(em[0], em[1], em[2]);
      int n = em[i];
      int iemm = -1;
      if (n > 0) { int emm[3] = {em[0], em[1], em[2]}; emm[i] -= 1; iemm = cart_index(emm[0], emm[1], emm[2]); }
      for (int m = 0; m <= Lt - le; ++m) {
        double v = PA[i] * VV(iem, 0, m) + WP[i] * VV(iem, 0, m + 1);
        if (n > 0) v += n / (2.0 * zeta) * (VV(iemm, 0, m) - rho / zeta * VV(iemm, 0, m + 1));
        VV(ie, 0, m) = v;
      }
      COUNT_OPS(OPS_VRR, (long long)(Lt - le + 1) * (n > 0 ? 3 + 7 : 3));
    }
  /* ket: [e|f+1_i]^(m) = QC_i [e|f]^(m) + WQ_i [e|f]^(m+1)
                          + f_i/(2 eta) ([e|f-1_i]^(m) - rho/eta [e|f-1_i]^(m+1))
                          + e_i/(2(zeta+eta)) [e-1_i|f]^(m+1) */
  for (int lf = 1; lf <= Lf; ++lf)
    for (int pf = 0; pf < ncart(lf); ++pf) {
      int f[3]; cart_lmn(lf, pf, f);
      int i = f[0] ? 0 : (f[1] ? 1 : 2);
      int fm[3] = {f[0], f[1], f[2]}; fm[i] -= 1;
      int jf = cart_index(f[0], f[1], f[2]), jfm = cart_index(fm[0], fm[1], fm[2]);
      int n = fm[i];
      int jfmm = -1;
      if (n > 0) { int fmm[3] = {fm[0], fm[1], fm[2]}; fmm[i] -= 1; jfmm = cart_index(fmm[0], fmm[1], fmm[2]); }
      for (int le = 0; le <= Le; ++le)
        for (int pe = 0; pe < ncart(le); ++pe) {
          int e[3]; cart_lmn(le, pe, e);
          int ie = cart_index(e[0], e[1], e[2]);
          int iem = -1;
          if (e[i] > 0) { int em[3] = {e[0], e[1], e[2]}; em[i] -= 1; iem = cart_index(em[0], em[1], em[2]); }
          for (int m = 0; m <= Lt - le - lf; ++m) {
            double v = QC[i] * VV(ie, jfm, m) + WQ[i] * VV(ie, jfm, m + 1);
            if (n > 0) v += n / (2.0 * eta) * (VV(ie, jfmm, m) - rho / eta * VV(ie, jfmm, m + 1));
            if (e[i] > 0) v += e[i] / (2.0 * s) * VV(iem, jfm, m + 1);
            VV(ie, jf, m) = v;
          }
          if (Lt - le - lf >= 0)
            COUNT_OPS(OPS_VRR, (long long)(Lt - le - lf + 1) * (3 + (n > 0 ? 7 : 0) + (e[i] > 0 ? 4 : 0)));
        }
    }
#undef VV
}

/* ------------------------------------------------------------------ HGP horizontal recursion */

/* (a, b+1_i| = (a+1_i, b| + (A-B)_i (a, b|.
 * X: [e][v], e over |e| in [la, la+lb] indexed cart_index(e) - cart_below(la), v < nv.
 * Y: [a][b][v] with |a| = la, |b| = lb, positions inside the shells. */
static void hgp_hrr(int la, int lb, const double AB[3], int nv, const double* X, double* Y) {
  int base = cart_below(la);
  int n0 = cart_below(la + lb + 1) - base;
  double* cur = (double*)malloc(sizeof(double) * (size_t)n0 * nv);
  memcpy(cur, X, sizeof(double) * (size_t)n0 * nv);
  int cur_nb = 1;                  /* b shells so far: |b| = k */
  for (int k = 1; k <= lb; ++k) {
    int na = cart_below(la + lb - k + 1) - base;      /* |a| in [la, la+lb-k] */
    int na_prev = cart_below(la + lb - k + 2) - base;
    int nb = ncart(k), nbm = ncart(k - 1);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)na * nb * nv);
    for (int ia = 0; ia < na; ++ia) {
      int g = ia + base, la_ = 0;
      while (cart_below(la_ + 1) <= g) ++la_;
      int av[3]; cart_lmn(la_, g - cart_below(la_), av);
      for (int pb = 0; pb < nb; ++pb) {
        int bv[3]; cart_lmn(k, pb, bv);
        int i = bv[0] ? 0 : (bv[1] ? 1 : 2);
        int bm[3] = {bv[0], bv[1], bv[2]}; bm[i] -= 1;
        int pbm = cart_pos(bm[1], bm[2]);
        int ap[3] = {av[0], av[1], av[2]}; ap[i] += 1;
        int iap = cart_index(ap[0], ap[1], ap[2]) - base;
        const double* x1 = cur + ((size_t)iap * nbm + pbm) * nv;
        const double* x0 = cur + ((size_t)ia * nbm + pbm) * nv;
        double* y = nxt + ((size_t)ia * nb + pb) * nv;
        for (int v = 0; v < nv; ++v) y[v] = x1[v] + AB[i] * x0[v];
        COUNT_OPS(OPS_HRR, 2LL * nv);
      }
    }
    (void)na_prev;
    free(cur);
    cur = nxt;
    cur_nb = nb;
  }
  /* keep |a| = la only (the first ncart(la) rows) */
  memcpy(Y, cur, sizeof(double) * (size_t)ncart(la) * cur_nb * nv);
  free(cur);
}

/* ------------------------------------------------------------------ contracted shell quartet */

/* out[a][b][c][d], row-major over the Cartesian components of shells I, J, K, L. */
void oracle_shell_quartet(const obasis* bs, int I, int J, int K, int L, double* out) {
  int la = bs->l[I], lb = bs->l[J], lc = bs->l[K], ld = bs->l[L];
  int Le = la + lb, Lf = lc + ld;
  const double* A = bs->coords + 3 * bs->atom[I];
  const double* B = bs->coords + 3 * bs->atom[J];
  const double* C = bs->coords + 3 * bs->atom[K];
  const double* D = bs->coords + 3 * bs->atom[L];
  int ne_all = cart_below(Le + 1), nf_all = cart_below(Lf + 1);
  int e0 = cart_below(la), ne = ne_all - e0;       /* |e| in [la, Le] */
  int f0 = cart_below(lc), nf = nf_all - f0;       /* |f| in [lc, Lf] */
  size_t vsz = (size_t)ne_all * nf_all * (Le + Lf + 1);
  double* V = (double*)malloc(sizeof(double) * vsz);
  double* E = (double*)calloc((size_t)ne * nf, sizeof(double));   /* contracted [e0|f0] */
  const int *np = bs->nprim, *of = bs->off;
  for (int p = 0; p < np[I]; ++p)
    for (int q = 0; q < np[J]; ++q)
      for (int r = 0; r < np[K]; ++r)
        for (int s = 0; s < np[L]; ++s) {
          double ca = bs->coefs[of[I] + p] * bs->coefs[of[J] + q] * bs->coefs[of[K] + r] * bs->coefs[of[L] + s];
          os_vrr(Le, Lf, bs->exps[of[I] + p], A, bs->exps[of[J] + q], B, bs->exps[of[K] + r], C,
                 bs->exps[of[L] + s], D, V);
          int nm = Le + Lf + 1;
          for (int ie = 0; ie < ne; ++ie)
            for (int jf = 0; jf < nf; ++jf)
              E[(size_t)ie * nf + jf] += ca * V[((size_t)(ie + e0) * nf_all + (jf + f0)) * nm];
          COUNT_OPS(OPS_CONTRACT, 3 + 2LL * ne * nf);
        }
  free(V);
  int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
  double CD[3] = {C[0] - D[0], C[1] - D[1], C[2] - D[2]};
  /* bra HRR with the ket index f as the vector: (e0|f0) -> (ab|f0) */
  double* Y = (double*)malloc(sizeof(double) * (size_t)na * nb * nf);
  hgp_hrr(la, lb, AB, nf, E, Y);
  free(E);
  /* transpose to [f][ab] and run the ket HRR: (ab|f0) -> (ab|cd) */
  double* Yt = (double*)malloc(sizeof(double) * (size_t)nf * na * nb);
  for (int ab = 0; ab < na * nb; ++ab)
    for (int jf = 0; jf < nf; ++jf) Yt[(size_t)jf * na * nb + ab] = Y[(size_t)ab * nf + jf];
  free(Y);
  double* Z = (double*)malloc(sizeof(double) * (size_t)nc * nd * na * nb);
  hgp_hrr(lc, ld, CD, na * nb, Yt, Z);
  free(Yt);
  for (int ab = 0; ab < na * nb; ++ab)
    for (int cd = 0; cd < nc * nd; ++cd) out[(size_t)ab * nc * nd + cd] = Z[(size_t)cd * na * nb + ab];
  free(Z);
}

/* ------------------------------------------------------------------ Schwarz factors, Eq. 7 */

static int max_block(const obasis* bs) {
  int m = 0;
  for (int s = 0; s < bs->nshell; ++s) if (ncart(bs->l[s]) > m) m = ncart(bs->l[s]);
  return m;
}

/* Q[I*nsh+J] = sqrt(max_{a in I, b in J} |(ab|ab)|) */
void oracle_schwarz(const obasis* bs, double* Q) {
  int nsh = bs->nshell, mb = max_block(bs);
#pragma omp parallel
  {
    double* g = (double*)malloc(sizeof(double) * (size_t)mb * mb * mb * mb);
#pragma omp for schedule(dynamic)
    for (int I = 0; I < nsh; ++I)
      for (int J = 0; J <= I; ++J) {
        oracle_shell_quartet(bs, I, J, I, J, g);
        int na = ncart(bs->l[I]), nb = ncart(bs->l[J]);
        double mx = 0.0;
        for (int a = 0; a < na; ++a)
          for (int b = 0; b < nb; ++b) {
            double v = fabs(g[(((size_t)a * nb + b) * na + a) * nb + b]);
            if (v > mx) mx = v;
          }
        Q[I * nsh + J] = Q[J * nsh + I] = sqrt(mx);
      }
    free(g);
  }
}

/* ------------------------------------------------------------------ J/K by definition */

static void first_bf(const obasis* bs, int* f0) {
  int acc = 0;
  for (int s = 0; s < bs->nshell; ++s) { f0[s] = acc; acc += ncart(bs->l[s]); }
}

/* Dmax[I*nsh+J] = max over densities and a in I, b in J of |D_ab| (Eq. 9's block maxima) */
static void block_dmax(const obasis* bs, int nD, int nbf, const double* Dm, const int* f0, double* Dmax) {
  int nsh = bs->nshell;
  for (int I = 0; I < nsh; ++I)
    for (int J = 0; J < nsh; ++J) {
      double mx = 0.0;
      for (int x = 0; x < nD; ++x)
        for (int a = 0; a < ncart(bs->l[I]); ++a)
          for (int b = 0; b < ncart(bs->l[J]); ++b) {
            double v = fabs(Dm[(size_t)x * nbf * nbf + (size_t)(f0[I] + a) * nbf + f0[J] + b]);
            if (v > mx) mx = v;
          }
      Dmax[I * nsh + J] = mx;
    }
}

static double max6(const double* Dmax, int nsh, int I, int J, int K, int L) {
  double v[6] = {Dmax[I * nsh + J], Dmax[K * nsh + L], Dmax[I * nsh + K],
                 Dmax[I * nsh + L], Dmax[J * nsh + K], Dmax[J * nsh + L]};
  double m = 0.0;
  for (int i = 0; i < 6; ++i) if (v[i] > m) m = v[i];
  return m;
}

/* the screening predicate of one unique quartet (it is invariant under the 8 permutations) */
static int keep_quartet(const double* Q, const double* Dmax, int nsh, double tau, int I, int J, int K, int L) {
  double qij = Q[I * nsh + J], qkl = Q[K * nsh + L];
  if (!(qij > tau) || !(qkl > tau)) return 0;
  return qij * qkl * max6(Dmax, nsh, I, J, K, L) >= tau;
}

/* Accumulate one ordered shell quartet block g(I J|K L) into J and K by the definitions
 * J_ij += (ij|kl) D_kl and K_ik += (ij|kl) D_jl, for every density. */
static void digest_block(const obasis* bs, const int* f0, int nbf, int nD, const double* Dm,
                         double* Jm, double* Km, const int sh[4], const double* g, const int perm[4]) {
  /* g is stored for the shell order (s0 s1|s2 s3) = sh; perm gives the ordered quartet as
   * positions into sh: the ordered quartet is (sh[perm0] sh[perm1] | sh[perm2] sh[perm3]). */
  int n[4];
  for (int t = 0; t < 4; ++t) n[t] = ncart(bs->l[sh[t]]);
  int idx[4];
  for (idx[0] = 0; idx[0] < n[0]; ++idx[0])
    for (idx[1] = 0; idx[1] < n[1]; ++idx[1])
      for (idx[2] = 0; idx[2] < n[2]; ++idx[2])
        for (idx[3] = 0; idx[3] < n[3]; ++idx[3]) {
          double v = g[(((size_t)idx[0] * n[1] + idx[1]) * n[2] + idx[2]) * n[3] + idx[3]];
          int i = f0[sh[perm[0]]] + idx[perm[0]];
          int j = f0[sh[perm[1]]] + idx[perm[1]];
          int k = f0[sh[perm[2]]] + idx[perm[2]];
          int l = f0[sh[perm[3]]] + idx[perm[3]];
          for (int x = 0; x < nD; ++x) {
            const double* Dx = Dm + (size_t)x * nbf * nbf;
            Jm[(size_t)x * nbf * nbf + (size_t)i * nbf + j] += v * Dx[(size_t)k * nbf + l];
            Km[(size_t)x * nbf * nbf + (size_t)i * nbf + k] += v * Dx[(size_t)j * nbf + l];
          }
        }
  COUNT_OPS(OPS_DIGEST, 4LL * nD * n[0] * n[1] * n[2] * n[3]);
}

int oracle_nbf(const obasis* bs) {
  int n = 0;
  for (int s = 0; s < bs->nshell; ++s) n += ncart(bs->l[s]);
  return n;
}

/* The 8 index permutations of (ij|kl) that leave the integral unchanged. */
static const int PERMS[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                                {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};

/* Evaluate one unique shell quartet (I >= J, K >= L, pair IJ >= pair KL) and add every
 * distinct ordered shell quartet of its orbit to J and K by the definitions. */
static void unique_quartet_jk(const obasis* bs, const int* f0, int nbf, int nD, const double* Dm,
                              double* Jl, double* Kl, double* g, int I, int J, int K, int L) {
  int sh[4] = {I, J, K, L};
  oracle_shell_quartet(bs, I, J, K, L, g);
  int seen[8][4], nseen = 0;
  for (int t = 0; t < 8; ++t) {
    int o[4] = {sh[PERMS[t][0]], sh[PERMS[t][1]], sh[PERMS[t][2]], sh[PERMS[t][3]]};
    int dup = 0;
    for (int u = 0; u < nseen; ++u)
      if (seen[u][0] == o[0] && seen[u][1] == o[1] && seen[u][2] == o[2] && seen[u][3] == o[3]) dup = 1;
    if (dup) continue;
    memcpy(seen[nseen++], o, sizeof(o));
    digest_block(bs, f0, nbf, nD, Dm, Jl, Kl, sh, g, PERMS[t]);
  }
}

static void pair_of(long long p, int* I, int* J) {
  long long i = (long long)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > p) --i;
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  *I = (int)i;
  *J = (int)(p - i * (i + 1) / 2);
}

/* J/K over the unique quartets listed in qidx (all of them when qidx is NULL and nq < 0).
 * A unique quartet's linear index u enumerates pairs of shell pairs p >= q with
 * u = p (p + 1) / 2 + q and p = I (I + 1) / 2 + J (I >= J).  screen: 0 = none,
 * 1 = the predicate.  Returns the number of quartets evaluated. */
static long long jk_core(const obasis* bs, int nD, const double* Dm, double* Jout, double* Kout,
                         double tau, int screen, const long long* qidx, long long nq) {
  int nsh = bs->nshell, nbf = oracle_nbf(bs), mb = max_block(bs);
  int* f0 = (int*)malloc(sizeof(int) * nsh);
  first_bf(bs, f0);
  double* Q = (double*)malloc(sizeof(double) * nsh * nsh);
  double* Dmax = (double*)malloc(sizeof(double) * nsh * nsh);
  if (screen) { oracle_schwarz(bs, Q); block_dmax(bs, nD, nbf, Dm, f0, Dmax); }
  size_t mat = (size_t)nD * nbf * nbf;
  memset(Jout, 0, sizeof(double) * mat);
  memset(Kout, 0, sizeof(double) * mat);
  long long npair = (long long)nsh * (nsh + 1) / 2;
  long long total = qidx ? nq : npair * (npair + 1) / 2;
  long long count = 0;
#pragma omp parallel reduction(+ : count)
  {
    double* Jl = (double*)calloc(mat, sizeof(double));
    double* Kl = (double*)calloc(mat, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * (size_t)mb * mb * mb * mb);
#pragma omp for schedule(dynamic, 16)
    for (long long t = 0; t < total; ++t) {
      long long u = qidx ? qidx[t] : t;
      int I, J, K, L;
      long long p, q;
      {
        long long i = (long long)((sqrt(8.0 * (double)u + 1.0) - 1.0) * 0.5);
        while (i * (i + 1) / 2 > u) --i;
        while ((i + 1) * (i + 2) / 2 <= u) ++i;
        p = i;
        q = u - i * (i + 1) / 2;
      }
      pair_of(p, &I, &J);
      pair_of(q, &K, &L);
      if (screen && !keep_quartet(Q, Dmax, nsh, tau, I, J, K, L)) continue;
      ++count;
      unique_quartet_jk(bs, f0, nbf, nD, Dm, Jl, Kl, g, I, J, K, L);
    }
#pragma omp critical
    {
      for (size_t t = 0; t < mat; ++t) { Jout[t] += Jl[t]; Kout[t] += Kl[t]; }
    }
    free(Jl); free(Kl); free(g);
  }
  free(f0); free(Q); free(Dmax);
  return count;
}

/* Full J/K.  screen: 0 = every unique quartet, 1 = the screening predicate.
 * Returns the number of unique shell quartets evaluated. */
long long oracle_jk(const obasis* bs, int nD, const double* Dm, double* Jout, double* Kout,
                    double tau, int screen) {
  return jk_core(bs, nD, Dm, Jout, Kout, tau, screen, NULL, -1);
}

/* Partial J/K over a list of unique-quartet indices (see jk_core); used to time the
 * oracle on a bounded random sample of a large build. */
long long oracle_jk_sample(const obasis* bs, int nD, const double* Dm, double* Jout, double* Kout,
                           double tau, int screen, const long long* qidx, long long nq) {
  return jk_core(bs, nD, Dm, Jout, Kout, tau, screen, qidx, nq);
}

/* Sampled blocks for large inputs, straight from the definitions with no symmetry:
 *   Jblk[s] = sum over all ordered (K,L) of (I_s J_s|K L) D_KL   (n_I x n_J per density)
 *   Kblk[s] = sum over all ordered (J,L) of (I_s J|K_s L) D_JL   (n_I x n_K per density)
 * pairs[2s], pairs[2s+1] give (I_s, J_s) for J and (I_s, K_s) for K.  Output block s starts
 * at s * nD * mb * mb, laid out [density][row][col] with row stride equal to the block width.
 * screen = 1 applies the same unique-quartet predicate as oracle_jk. */
void oracle_jk_blocks(const obasis* bs, int nD, const double* Dm, int nsample, const int* pairs,
                      double* Jblk, double* Kblk, double tau, int screen) {
  int nsh = bs->nshell, nbf = oracle_nbf(bs), mb = max_block(bs);
  int* f0 = (int*)malloc(sizeof(int) * nsh);
  first_bf(bs, f0);
  double* Q = (double*)malloc(sizeof(double) * nsh * nsh);
  double* Dmax = (double*)malloc(sizeof(double) * nsh * nsh);
  if (screen) { oracle_schwarz(bs, Q); block_dmax(bs, nD, nbf, Dm, f0, Dmax); }
  size_t bsz = (size_t)nD * mb * mb;
  memset(Jblk, 0, sizeof(double) * bsz * nsample);
  memset(Kblk, 0, sizeof(double) * bsz * nsample);
#pragma omp parallel
  {
    double* g = (double*)malloc(sizeof(double) * (size_t)mb * mb * mb * mb);
#pragma omp for schedule(dynamic) collapse(2)
    for (int s = 0; s < nsample; ++s)
      for (int X = 0; X < nsh; ++X) {
        int I = pairs[2 * s], S2 = pairs[2 * s + 1];
        int nI = ncart(bs->l[I]), n2 = ncart(bs->l[S2]);
        for (int Y = 0; Y < nsh; ++Y) {
          /* J: (I S2 | X Y) D_XY */
          if (!screen || keep_quartet(Q, Dmax, nsh, tau, I, S2, X, Y)) {
            oracle_shell_quartet(bs, I, S2, X, Y, g);
            int nx = ncart(bs->l[X]), ny = ncart(bs->l[Y]);
            for (int x = 0; x < nD; ++x) {
              const double* Dx = Dm + (size_t)x * nbf * nbf;
              double* out = Jblk + s * bsz + (size_t)x * mb * mb;
              for (int a = 0; a < nI; ++a)
                for (int b = 0; b < n2; ++b) {
                  double acc = 0.0;
                  for (int c = 0; c < nx; ++c)
                    for (int d = 0; d < ny; ++d)
                      acc += g[(((size_t)a * n2 + b) * nx + c) * ny + d] * Dx[(size_t)(f0[X] + c) * nbf + f0[Y] + d];
#pragma omp atomic
                  out[a * n2 + b] += acc;
                }
            }
          }
          /* K: (I X | S2 Y) D_XY */
          if (!screen || keep_quartet(Q, Dmax, nsh, tau, I, X, S2, Y)) {
            oracle_shell_quartet(bs, I, X, S2, Y, g);
            int nx = ncart(bs->l[X]), ny = ncart(bs->l[Y]);
            for (int x = 0; x < nD; ++x) {
              const double* Dx = Dm + (size_t)x * nbf * nbf;
              double* out = Kblk + s * bsz + (size_t)x * mb * mb;
              for (int a = 0; a < nI; ++a)
                for (int c = 0; c < n2; ++c) {
                  double acc = 0.0;
                  for (int b = 0; b < nx; ++b)
                    for (int d = 0; d < ny; ++d)
                      acc += g[(((size_t)a * nx + b) * n2 + c) * ny + d] * Dx[(size_t)(f0[X] + b) * nbf + f0[Y] + d];
#pragma omp atomic
                  out[a * n2 + c] += acc;
                }
            }
          }
        }
      }
    free(g);
  }
  free(f0); free(Q); free(Dmax);
}

/* Number of unique shell quartets passing the predicate (0 = no screening). */
long long oracle_count_quartets(const obasis* bs, int nD, const double* Dm, double tau, int screen) {
  int nsh = bs->nshell, nbf = oracle_nbf(bs);
  int* f0 = (int*)malloc(sizeof(int) * nsh);
  first_bf(bs, f0);
  double* Q = (double*)malloc(sizeof(double) * nsh * nsh);
  double* Dmax = (double*)malloc(sizeof(double) * nsh * nsh);
  if (screen) { oracle_schwarz(bs, Q); block_dmax(bs, nD, nbf, Dm, f0, Dmax); }
  long long count = 0;
  int npair = nsh * (nsh + 1) / 2;
  for (int p = 0; p < npair; ++p) {
    int I = 0;
    while ((I + 1) * (I + 2) / 2 <= p) ++I;
    int J = p - I * (I + 1) / 2;
    for (int q = 0; q <= p; ++q) {
      int K = 0;
      while ((K + 1) * (K + 2) / 2 <= q) ++K;
      int L = q - K * (K + 1) / 2;
      if (!screen || keep_quartet(Q, Dmax, nsh, tau, I, J, K, L)) ++count;
    }
  }
  free(f0); free(Q); free(Dmax);
  return count;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ operation counts
 * Operations of this oracle for one unique shell quartet (I J | K L) of bs whose eight
 * ordered quartets are all distinct: the contracted quartet and the digestion of its orbit
 * into J and K for nD densities.  out[OPS_N]: set-up, Boys, VRR, contraction, HRR,
 * digestion.  Runs on the calling thread. */
void oracle_quartet_ops(const obasis* bs, int I, int J, int K, int L, int nD, double* out) {
  int sh[4] = {I, J, K, L}, n[4], nbf = oracle_nbf(bs);
  size_t nabcd = 1;
  for (int t = 0; t < 4; ++t) { n[t] = ncart(bs->l[sh[t]]); nabcd *= (size_t)n[t]; }
  int* f0 = (int*)malloc(sizeof(int) * bs->nshell);
  first_bf(bs, f0);
  double* g = (double*)malloc(sizeof(double) * nabcd);
  double* Dm = (double*)calloc((size_t)nD * nbf * nbf, sizeof(double));
  double* Jm = (double*)calloc((size_t)nD * nbf * nbf, sizeof(double));
  double* Km = (double*)calloc((size_t)nD * nbf * nbf, sizeof(double));
  memset(g_ops, 0, sizeof(g_ops));
  oracle_shell_quartet(bs, I, J, K, L, g);
  for (int t = 0; t < 8; ++t) digest_block(bs, f0, nbf, nD, Dm, Jm, Km, sh, g, PERMS[t]);
  for (int k = 0; k < OPS_N; ++k) out[k] = (double)g_ops[k];
  free(f0); free(g); free(Dm); free(Jm); free(Km);
}

/* Operations per class (la lb | lc ld): ops = prim * sum(per_prim) + sum(per_quartet) for a
 * quartet with prim primitive quartets.  per_prim[OPS_N] holds the set-up, Boys, VRR and
 * contraction of one primitive quartet, per_quartet[OPS_N] the HRR and the digestion of nD
 * densities (other entries 0).  Counted on one synthetic quartet with one primitive per shell
 * (centres (0,0,0), (0,0,1.1), (0.9,0,0), (0.8,1.2,0.3) bohr, exponents 0.9, 0.6, 0.7, 0.5).
 * Every phase but the Boys function is independent of the geometry and the exponents; the
 * Boys series is counted at this geometry's T (about 0.3). */
void oracle_class_ops(int la, int lb, int lc, int ld, int nD, double* per_prim, double* per_quartet) {
  const double xyz[12] = {0.0, 0.0, 0.0, 0.0, 0.0, 1.1, 0.9, 0.0, 0.0, 0.8, 1.2, 0.3};
  const int atom[4] = {0, 1, 2, 3}, l[4] = {la, lb, lc, ld}, nprim[4] = {1, 1, 1, 1}, off[4] = {0, 1, 2, 3};
  const double exps[4] = {0.9, 0.6, 0.7, 0.5}, coefs[4] = {1.0, 1.0, 1.0, 1.0};
  obasis bs = {4, xyz, 4, atom, l, nprim, off, exps, coefs};
  double ops[OPS_N];
  oracle_quartet_ops(&bs, 0, 1, 2, 3, nD, ops);
  for (int k = 0; k < OPS_N; ++k) {
    const int per_q = (k == OPS_HRR || k == OPS_DIGEST);
    per_prim[k] = per_q ? 0.0 : ops[k];
    per_quartet[k] = per_q ? ops[k] : 0.0;
  }
}
