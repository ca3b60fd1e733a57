// Internal data layout shared by the host planner and the CUDA kernels.
// Plain structs only (no CUDA types) so both g++ and nvcc can include it.
#pragma once
#include <stdint.h>

#define ERI_LMAX 4
#define ERI_NPAIRTYPE 15          // canonical pair types (l0 >= l1), l <= 4
#define ERI_CART_LMAX 9           // Cartesian tables cover l <= 9 (gradient transfer of (gg| reaches 9)
#define ERI_MAXCART 220           // Cartesian triples with l <= 9

// One primitive pair (Gaussian product of Eq. 2's primitives on the pair's two
// centres A, B).  80 bytes, 16-byte aligned.
struct PrimPair {
  double zeta;     // alpha + beta
  double P[3];     // (alpha A + beta B) / zeta
  double PA[3];    // P - A
  double E;        // sqrt(2) pi^(5/4) / zeta * exp(-alpha beta |A-B|^2 / zeta) * c_alpha c_beta
  double hz;       // 1 / (2 zeta)
  double alpha;    // exponent of the primitive on A (the gradient kernels weight by 2 alpha, 2 beta)
};

// FP32 shadow of PrimPair for the FP32 path of the mixed mode (P - Q comes from the FP64
// centres, so P itself is not shadowed).  32 bytes.
struct PrimPairF {
  float zeta;
  float PA[3];
  float E;
  float hz;
  float pad[2];
};

// One shell pair in canonical orientation (l of sh0 >= l of sh1).  64 bytes.
struct ShellPair {
  int sh0, sh1;    // shell indices
  int bf0, bf1;    // first basis function of each shell
  int prim_off;    // first PrimPair
  int nprim;       // K_sh0 * K_sh1
  int ptype;       // l0 * (l0 + 1) / 2 + l1
  float Qe;        // Cauchy-Schwarz factor of the pair's [e0| intermediates weighted by the
                   // transfer coefficients, sqrt(max_e [e0|e0]) (1 + max_x |A-B|_x)^l1 >= Q: the
                   // mixed mode's precision split uses Qe_ij Qe_kl max|D| (see quartet_category)
  double AB[3];    // A - B (A = centre of sh0)
  double Q;        // Cauchy-Schwarz factor of Eq. 7
};

// Static description of one angular-momentum class (la lb | lc ld).
struct ClassDesc {
  int la, lb, lc, ld;
  int nroots;            // floor((la+lb+lc+ld)/2) + 1
  int Le, Lf;            // la + lb, lc + ld
  int nI;                // (Le+1)(Lf+1) 2D-integral entries per axis and root
  int nIs;               // shared-memory stride of one such table: nI, odd in team kernels
  int ne, nf;            // Cartesian e with la <= |e| <= Le, f with lc <= |f| <= Lf
  int nout;              // ne * nf contracted [e0|f0] values
  int na, nb, nc, nd;    // shell sizes
  int e_base, f_base;    // global Cartesian index of the first e / f
  int npass;             // output chunks of TS*G values
  int bp;                // primitive quartets per batch (team kernels)
  int team_doubles;      // shared-memory doubles per team (FP64 recurrences)
  int team_doubles_f32;  // shared-memory doubles per team (FP32 recurrences)
  int hrr_doubles;       // size of one HRR ping-pong buffer (doubles)
  long long scratch_per_team;  // global scratch doubles per team
  long long part_off;    // FP64 classes with several passes: offset of the slot-ordered partial sums
                         // carried between primitive batches (0 when a class has one pass)
  int split3, split3_xy; // 1: the root phase runs (primitive, root, axis) items (batch bp / bp_xy)
  // Assembly of Eq. 1 by lane programs (every FP32 launch; FP64 launches with xy = 0): the
  // values sharing an I_x I_y product form groups; every lane of a team runs the same
  // sequence of group sizes, so slot k of a pass starts a group (one multiply) for all lanes
  // or for none: bit k of gmask[pass].  Slot tables: outidx = ix | iy << 8 | iz << 16 |
  // unused << 31 with E0 position dst; nslot = lanes x slots per lane (>= nout; padding
  // slots are computed and dropped); xysum = products formed per (primitive, root).
  int nslot, xysum;
  const uint32_t* outidx;
  const uint32_t* dst;
  const uint32_t* gmask;       // [npass]
  // Shared products path (FP64 launches with xy = 1): values ordered by their product; per
  // pass the team forms the pass's products once per (primitive, root) in shared memory
  // and every value is one FMA with I_z.  Own pass count, batch and team region.
  int xy;
  int xy_npass, bp_xy, team_doubles_xy;
  int xymax;                   // most products in one pass
  int xysum_xy;                // products formed per (primitive, root) over all passes
  const uint32_t* xy_outidx;   // [nout] product index within the pass | iz << 16
  const uint32_t* xy_dst;      // [nout] E0 position
  const uint32_t* xytab;       // [products] ix | iy << 8
  const uint32_t* passinfo;    // [xy_npass][2] first product, products in the pass
  int ncomb;                   // distinct products of the class
  int stage;                   // 1: stage each team's bra / ket PrimPair records into shared memory
                               // by bulk copy (tuning override; kernels compiled for the class only)
  // offsets of the tables in the class's block of the device table (host bookkeeping)
  int dst_off, gmask_off, xy_outidx_off, xy_dst_off, xytab_off, pass_off;
};

enum { KMODE_JK = 0, KMODE_BLOCK = 1, KMODE_SCHWARZ = 2 };

// One job of a batched J/K launch: everything the class kernel reads or writes that
// belongs to one plan and one density set.
struct JobDesc {
  const struct ShellPair* pairs;
  const struct PrimPair* prims;
  const struct PrimPairF* primsf;
  const double* D;
  double* J;
  double* K;
  int nbf, nD, want, pad;
  int type_off[ERI_NPAIRTYPE];
  int type_cnt[ERI_NPAIRTYPE];
};

struct KernelArgs {
  ClassDesc c;
  const ShellPair* pairs;
  const PrimPair* prims;
  const PrimPairF* primsf;     // FP32 shadow (FP32 kernels)
  // task space: bra pairs [bra0, bra0+nbra), ket pairs [ket0, ket0+nket); tri = same range, ket <= bra
  int bra0, nbra, ket0, nket, tri;
  long long ntask;
  // screening (KMODE_JK)
  const double* Dmax;    // [nsh][nsh]
  int nsh;
  double tau;
  int prec_sel;          // 0: every kept quartet; 1: the FP64 quartets of the mixed split only; 2: its FP32
                         // quartets only (quartet_category)
  double mixed_thr;
  // compacted task lists (KMODE_JK): when tlist is set, the tasks are tlist[0 .. *tcount) or,
  // with from_back, tlist[cap-1-t] for t < *tcount; they already passed the screen
  const unsigned* tlist;
  const unsigned long long* tcount;
  unsigned long long list_cap;
  int from_back;
  // batched launches (several jobs, one class): entries job << 32 | task of that job,
  // blist[0 .. *tcount) or from the back as above; X, Y = the class's pair types
  const JobDesc* jobs;
  const unsigned long long* blist;
  int X, Y;
  // densities and outputs (KMODE_JK): row-major [nD][nbf][nbf]
  const double* D;
  double* J;
  double* K;
  int nD, nbf, want;
  // KMODE_BLOCK / KMODE_SCHWARZ: explicit tasks (bra, ket) and outputs
  int mode;
  const int* tasklist;   // [2*ntask]
  double* blockout;      // KMODE_BLOCK: per task nabcd values, [cd][ab] layout as stored
  const long long* blockoff;
  double* qout;          // KMODE_SCHWARZ: per task max_{a,b} |(ab|ab)| at [task] and
                         // max_e |[e0|e0]| (before the transfer relations) at [ntask + task]
  // scheduling, scratch, counters
  unsigned long long* counter;
  double* scratch;
  // KMODE_JK: each listed quartet runs as qsplit tasks over consecutive ranges of its
  // primitive quartets (0 or 1: one task per quartet); the transfer relations and the
  // digestion are linear, so every range digests its partial [e0|f0] on its own
  int qsplit;
  unsigned long long* stats;   // [0] quartets computed, [1] primitive quartets
  unsigned* err;               // set to 1 when a bounded device wait gave up (staged kernels)
  // Rys table for this class's root count
  const double* rys_coef;      // block of this N
  const double* rys_au;
  const double* rys_aw;
  int rys_tcut;
  double rys_tcut_d;           // the same cutoff as a double
};

// One angular-momentum class of the two-electron energy gradient (Sec. 4, Eqs. 11-14).
// The 2D tables run to Le2 = la+lb+1, Lf2 = lc+ld+1 with nroots = floor((L+1)/2) + 1.
// Four contracted sets of [e0|f0] are assembled, concatenated in this order, each stored
// [e][f] row-major with e, f relative to the set's first Cartesian:
//   set 0  weight 1      e in [max(la-1,0), Le],  f in [max(lc-1,0), Lf]
//   set 1  weight 2 alpha e in [la+1, Le+1],      f in [lc, Lf]
//   set 2  weight 2 beta  e in [la, Le+1],        f in [lc, Lf]
//   set 3  weight 2 gamma e in [la, Le],          f in [lc+1, Lf+1]
// (alpha, beta, gamma: exponents of the primitives on centres A, B, C).  Each primitive
// quartet keeps four I_z tables scaled by the four weights, so every value of every set is
// one FMA with a shared I_x I_y product (lane programs, as for the J/K classes): slot words
// ix | iy << 8 | (k N nI + iz) << 16 | unused << 31, E0 positions dst, group starts gmask.
struct GradDesc {
  int la, lb, lc, ld;
  int na, nb, nc, nd;
  int nroots, Le2, Lf2, nI;
  int s_elo[4], s_ne[4], s_flo[4], s_nf[4];   // first l and Cartesian count of e / f per set
  int s_off[4];                               // offset of each set in the team scratch
  int nout;                                   // total assembled values (sum of the four sets)
  int nslot;                                  // lane-program slots (>= nout)
  int npass, bp, team_doubles;
  int split3;                                 // 1: root phase over (primitive, root, axis) items
  int gam_off;                                // Gamma_J, Gamma_K: 2 * na nb nc nd doubles
  int hrr_off, hrr_doubles;                   // two HRR ping-pong buffers
  long long scratch_per_team;
  long long part_off;                         // slot-ordered partial sums between batches (npass > 1)
  const uint32_t* outidx;                     // [nslot] slot words
  const uint32_t* dst;                        // [nslot] position in the concatenated sets
  const uint32_t* gmask;                      // [npass] group starts
  int dst_off, gmask_off;                     // table offsets (host)
};

struct GradArgs {
  KernelArgs k;          // task space, pair data, compacted list, Rys table of nroots
  GradDesc g;
  const int* sh_atom;    // [nshell] atom of each shell
  double* gJ;            // [natm][3] += d E_J / d R
  double* gK;            // [natm][3] += d E_K / d R
};

// Host-side launchers implemented in eri_kernels.cu.  All return a cudaError_t as int.
#ifdef __cplusplus
extern "C" {
#endif
int erik_upload_cart_tables(void);
int erik_blocks_per_sm(int ts, int fp32, int xy, int smem_bytes, int* out);
int erik_launch_class(int ts, int fp32, const struct KernelArgs* a, int grid, int smem_bytes, void* stream);
// FP64 class kernels compiled for one class (eri_class_spec.cu): launches and returns 1 (launch
// status in *rc) when one matches the class, team size and assembly path, else returns 0
int erik_launch_class_spec(int ts, int xy, const struct KernelArgs* a, int grid, int smem_bytes, void* stream, int* rc);
int erik_class_spec_prepare(void);
int erik_class_spec_available(int ts, int la, int lb, int lc, int ld);
int erik_upload_cart_tables_spec(void);
int erik_launch_compact(const struct KernelArgs* a, unsigned* tlist, unsigned long long cap,
                        unsigned long long* counts, unsigned* tiles, int mixed, void* stream);
int erik_launch_compact_batched(const struct KernelArgs* a, unsigned long long* blist, unsigned long long cap,
                                unsigned long long* counts, unsigned* tiles, unsigned long long* cursor,
                                unsigned long long* base, unsigned long long job, int mixed, void* stream);
int erik_launch_dmax(const double* D, int nD, int nbf, int nsh, const int* sh_bf0, const int* sh_n,
                     double* Dmax, void* stream);
int erik_launch_symmetrize(double* M, int nD, int nbf, void* stream);
int erik_launch_symcheck(const double* D, int nD, int nbf, unsigned long long* out, void* stream);
int erik_launch_rys(int N, int n, const double* T, double* u, double* w, const double* coef,
                    const double* au, const double* aw, int tcut, void* stream);
int erik_probe_fma(double* fp64_tflops, double* fp32_tflops);
// compile-time specialised kernels of the small classes (eri_small.cu)
int erik_upload_cart_tables_small(void);
int erik_small_available(int la, int lb, int lc, int ld, int fp32);
int erik_small_blocks_per_sm(int la, int lb, int lc, int ld, int fp32, int* out);
int erik_launch_small(int la, int lb, int lc, int ld, int fp32, const struct KernelArgs* a, int grid, void* stream);
// energy-gradient class kernels (eri_grad.cu)
int erik_upload_cart_tables_grad(void);
int erik_grad_blocks_per_sm(int ts, int smem_bytes, int* out);
int erik_launch_grad(int ts, const struct GradArgs* a, int grid, int smem_bytes, void* stream);
#ifdef __cplusplus
}
#endif
