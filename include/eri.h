/*
 * liberi: integral-direct Coulomb / exchange (J/K) builds over contracted
 * Cartesian Gaussian shells up to g, evaluated by Rys quadrature on one
 * NVIDIA GB300 (sm_103a).  Method: arXiv 2407.09700 (GPU4PySCF), Secs. 2-3.
 *
 * All entry points are plain C.  Status codes are returned, nothing aborts and
 * no exception crosses the boundary; on failure eri_last_error() gives a
 * message (thread-local, valid until the next call on the same thread).
 *
 * Conventions shared by every entry point:
 *   - atomic units (Bohr); coordinates row-major [natm][3];
 *   - Cartesian components of a shell in x-descending order
 *     (for lx = l..0, for ly = l-lx..0: xx, xy, xz, yy, yz, zz for d);
 *   - basis functions numbered shell by shell in the order given;
 *   - contraction coefficients, when normalise = 1, get the radial primitive
 *     norm (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!) and the contracted shell is
 *     rescaled so its x^l component has unit self-overlap (Eqs. 2, 4-5, Sec. 2;
 *     the paper leaves the convention open);
 *   - matrices are row-major [nD][nbf][nbf] FP64.
 */
#ifndef ERI_H
#define ERI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ERI_OK = 0,
  ERI_ERR_ARG = 1,            /* bad argument (null pointer, size, index, option) */
  ERI_ERR_BASIS = 2,          /* malformed basis: nprim < 1, non-finite or non-positive exponent, bad atom index */
  ERI_ERR_OOM = 3,            /* device or host allocation failed; the plan is left unchanged */
  ERI_ERR_CUDA = 4,           /* a CUDA runtime call failed; message in eri_last_error() */
  ERI_ERR_NO_DEVICE = 5,      /* no CUDA device is visible */
  ERI_ERR_TIMEOUT = 6,        /* a bounded device wait gave up (eri_flop_stats reports it) */
  ERI_ERR_UNSUPPORTED_L = 7   /* angular momentum above g (l > 4); Sec. 3 stops at g */
} eri_status;

enum { ERI_FP64 = 0, ERI_MIXED = 1 };
enum { ERI_WANT_J = 1, ERI_WANT_K = 2 };

typedef struct eri_plan eri_plan;

/* Basis set: all arrays on the host, read during eri_plan_create only. */
typedef struct {
  int natm;
  const double* coords;      /* [natm][3], Bohr */
  int nshell;
  const int* shell_atom;     /* [nshell] atom of each shell */
  const int* shell_l;        /* [nshell] angular momentum, 0..4 */
  const int* shell_nprim;    /* [nshell] contraction depth K >= 1 */
  const int* shell_off;      /* [nshell] first primitive of the shell in exps / coefs */
  const double* exps;        /* primitive exponents, > 0 */
  const double* coefs;       /* contraction coefficients (raw if normalise = 1) */
  int normalise;             /* 1: apply the normalisation above; 0: use coefs as given */
} eri_basis;

typedef struct {
  double screen_thresh;      /* tau of Eqs. 6-9 (Sec. 3); shell pairs with Q <= tau are dropped */
  int precision;             /* ERI_FP64 (all FP64) or ERI_MIXED */
  double mixed_thresh;       /* ERI_MIXED: a quartet whose bound Qe_ij Qe_kl max|D| is <= this runs its
                                recurrences, Eq. 1 products and contraction in FP32 (Qe: the
                                transfer-aware Schwarz factor of eri_schwarz_transfer, >= the Q of
                                Eq. 7, so every quartet above the Eqs. 7-9 bound stays FP64); Rys
                                roots/weights, T, P - Q, the transfer relations, digestion and J/K
                                accumulation stay FP64 */
  int max_nd;                /* largest nD an eri_jk call may pass (>= 1) */
  int mixed_min_tasks;       /* ERI_MIXED: a class gets its FP32 launch only when its task space (unique
                                quartets of its pair types before screening) has at least this many
                                quartets; smaller classes run every quartet in FP64, where a second
                                launch would cost more than the FP32 arithmetic saves.  0: every class. */
  int check_symmetric;       /* 1: eri_jk and eri_jk_host first verify that every D is symmetric
                                (max|D_ij - D_ji| <= 1e-12 max|D|, see eri_check_density) and return
                                ERI_ERR_ARG otherwise; eri_jk then synchronises its stream.  0: not
                                checked.  The 8-fold symmetry of Sec. 3 needs a symmetric D. */
} eri_opts;

/* Counters of the last eri_jk call on the plan (filled after that call's stream completes). */
typedef struct {
  long long quartets_candidate;   /* unique shell quartets formed from the kept shell pairs */
  long long quartets_computed;    /* unique shell quartets that passed the screening test */
  long long prim_quartets;        /* primitive quartets evaluated */
  long long quartets_fp32;        /* of quartets_computed, those run in FP32 (ERI_MIXED) */
  double model_flops;             /* FP64+FP32 arithmetic of the Rys kernels, counted per class */
  int npairs_total;               /* shell pairs i >= j */
  int npairs_kept;                /* shell pairs with Q > tau */
  int nclasses_launched;          /* class kernel launches (two per class in ERI_MIXED) */
  double model_flops_fp32;        /* the FP32 part of model_flops (ERI_MIXED) */
  int device_status;              /* 0, or 1 once a kernel of the plan gave up a bounded wait (the
                                     bulk-copy staging of the tuning override); then
                                     eri_flop_stats returns ERI_ERR_TIMEOUT and results since
                                     are incomplete */
} eri_stats;

/*
 * Symmetry check of nD densities [nD][nbf][nbf] in HOST memory: ERI_OK when max over the
 * densities of |D_ij - D_ji| <= 1e-12 max|D| and every element is finite, ERI_ERR_ARG
 * otherwise (message in eri_last_error).  Needs no GPU.  The J/K build's digestion
 * (Alg. 2's six updates with the weights of the 8-fold symmetry, Sec. 3) is correct only for
 * symmetric D.
 */
eri_status eri_check_density(const double* D, int nD, int nbf);

/*
 * Create a plan: validates and normalises the basis, forms every shell pair
 * (i >= j) with its primitive-pair data (Gaussian product theorem, Eq. 2),
 * computes the Cauchy-Schwarz factors Q_ij = max |(ab|ab)|^(1/2) of Eq. 7 on
 * the GPU, keeps pairs with Q > tau and groups them by angular-momentum class
 * (Alg. 1 of Sec. 3).  Synchronous.  The plan owns all its device memory, including
 * eri_jk's scratch, task lists and tile counts, which are sized here from the plan so that
 * eri_jk itself allocates nothing.  cuda_stream: a cudaStream_t or NULL for the default stream.
 * Errors: ERI_ERR_ARG (null pointers, tau < 0, max_nd < 1, check_symmetric not 0 / 1), ERI_ERR_BASIS,
 * ERI_ERR_UNSUPPORTED_L, ERI_ERR_NO_DEVICE, ERI_ERR_OOM, ERI_ERR_CUDA.
 */
eri_status eri_plan_create(const eri_basis* basis, const eri_opts* opts, void* cuda_stream,
                           eri_plan** out);

/* Free a plan and its device memory (synchronises the device first).  NULL is accepted. */
eri_status eri_plan_destroy(eri_plan* plan);

/* Number of Cartesian basis functions, or -1 for a NULL plan. */
int eri_plan_nbf(const eri_plan* plan);

/*
 * Coulomb and exchange matrices (Sec. 3, Algs. 1-3):
 *   J_ij = sum_kl (ij|kl) D_kl,   K_ik = sum_jl (ij|kl) D_jl,
 * for nD symmetric densities, using the 8-fold permutation symmetry of (ij|kl)
 * and the screening of Eqs. 7-9: a unique shell quartet is evaluated when
 * Q_ij * Q_kl * max|D| over its six cross blocks >= tau.
 * D, J, K: DEVICE pointers, contiguous [nD][nbf][nbf] FP64, 1 <= nD <= max_nd.
 * D must be symmetric (checked only when the plan's check_symmetric is 1: ERI_ERR_ARG).
 * J and K are overwritten, never accumulated.  flags: ERI_WANT_J | ERI_WANT_K (an unwanted
 * output may be NULL and is not touched).  Asynchronous on cuda_stream (unless
 * check_symmetric); allocates no device memory (the plan's buffers were sized at
 * creation); the plan's scratch is reused by every call, so calls on one plan must not
 * overlap on the GPU.
 */
eri_status eri_jk(eri_plan* plan, const double* D, int nD, double* J, double* K, int flags,
                  void* cuda_stream);

/*
 * eri_jk for callers that cannot allocate device memory during the call.  The
 * paper has no counterpart; this is a library convenience.  A plan owns scratch
 * sized for eri_jk, but eri_jk_grad and eri_shell_quartet may regrow it with
 * cudaMalloc / cudaFree (after synchronising the device); code running under an
 * allocator or a memory budget that owns all device memory, or in a host
 * callback, must not let a library call those at all.  This call allocates
 * nothing and calls no cudaMalloc / cudaFree or allocating library routine,
 * and it leaves the plan's own scratch untouched: the class kernels' scratch is a file-scope
 * static device array of 32 MiB (ERI_NOALLOC_SCRATCH_BYTES) that every GPU
 * loading the library holds until the process exits.  Arguments, layout and
 * results are those of eri_jk (D, J, K device pointers; J and K overwritten).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array, and nothing in it needs to start
 * at zero (each value is written before it is read in the same call); calls
 * that overlap on the GPU, on any plan, race on it.  A class launch uses as
 * many blocks as the array can hold; a class whose single block needs more
 * scratch than the array is rejected with ERI_ERR_ARG before any launch.
 * The plan must belong to the current device (ERI_ERR_ARG otherwise).  The
 * cached address does not survive cudaDeviceReset (or the end of the primary
 * context): after one, the process must not call this entry point on that device.
 * A call leaves no per-launch records (eri_launch_records then reports none).
 */
eri_status eri_jk_noalloc(eri_plan* plan, const double* D, int nD, double* J, double* K, int flags,
                          void* cuda_stream);

/*
 * Same as eri_jk, with D, J and K in HOST memory: copies D to the device,
 * builds J/K and copies them back.  Synchronous.
 */
eri_status eri_jk_host(eri_plan* plan, const double* D, int nD, double* J, double* K, int flags,
                       void* cuda_stream);

/*
 * Nuclear gradients of the Coulomb and exchange energies for one fixed density
 * (Sec. 4, Eqs. 10-14, Alg. 4):
 *   E_J = 1/2 sum_abcd (ab|cd) D_ab D_cd,   E_K = -1/4 sum_abcd (ab|cd) D_ac D_bd,
 * so that for a closed-shell density E_J + E_K is the two-electron energy
 * 1/2 tr(D J) - 1/4 tr(D K).  gJ[A][x] = dE_J/dR_Ax and gK[A][x] = dE_K/dR_Ax with D
 * held fixed (the ERI-derivative part of the RHF gradient).  The ERI derivatives are
 * contracted with the density products inside the kernels; no derivative Fock matrix
 * is formed.  Unique shell quartets with the plan's screening as in eri_jk (a quartet is
 * evaluated when Q_ij * Q_kl * max|D| over its six cross blocks >= tau).  FP64 for every
 * plan precision.
 * D: DEVICE pointer, [nbf][nbf] FP64, symmetric (not checked).  gJ, gK: DEVICE
 * pointers, [natm][3] FP64 each, overwritten.  Asynchronous on cuda_stream; shares the
 * plan's scratch with eri_jk (calls on one plan must not overlap on the GPU).
 * Errors: ERI_ERR_ARG (NULL pointers), ERI_ERR_OOM, ERI_ERR_CUDA.
 */
eri_status eri_jk_grad(eri_plan* plan, const double* D, double* gJ, double* gK, void* cuda_stream);

/* Shell quartets and primitive quartets evaluated by the last eri_jk_grad call
 * (synchronises that call's stream). */
eri_status eri_grad_stats(eri_plan* plan, long long* quartets, long long* prim_quartets);

/*
 * One contracted shell quartet (ij|kl) by Rys quadrature (Eq. 1 contracted by
 * Eq. 5), no screening: writes n_i*n_j*n_k*n_l FP64 values in (i,j,k,l)
 * row-major Cartesian order to out (HOST memory).  Synchronous.
 * Errors: ERI_ERR_ARG for a shell index outside [0, nshell).
 */
eri_status eri_shell_quartet(eri_plan* plan, int i, int j, int k, int l, double* out);

/* Schwarz factors of Eq. 7 for every shell pair: Q[i*nshell+j] (HOST, symmetric). */
eri_status eri_schwarz(const eri_plan* plan, double* Q);

/*
 * Transfer-aware factors of the mixed mode's precision split, for every shell pair:
 * Qe[i*nshell+j] (HOST, symmetric) = sqrt(max_e [e0|e0]) (1 + max_x |A-B|_x)^lb, the
 * Cauchy-Schwarz factor of the pair's contracted [e0| intermediates (|e| from la to la+lb,
 * centre A of the shell with the larger l, before the transfer relations of Sec. 2) times
 * the largest sum of absolute transfer coefficients, rounded up to FP32; Qe >= Q, equal to
 * it (up to that rounding) when lb = 0.  The paper has no mixed precision; this is the
 * library's reading of the Schwarz x density bound for the values that the FP32 stage
 * computes.  A quartet of an ERI_MIXED plan runs in FP32 when it passes the screen and
 * Qe_ij Qe_kl max|D| (six cross blocks) <= mixed_thresh.  Filled for every plan.
 */
eri_status eri_schwarz_transfer(const eri_plan* plan, double* Qe);

/*
 * Rys roots and weights on the device, for testing the quadrature of Eq. 1:
 * for each T[t] (t < n, T >= 0) writes u[t*N+r] = t_r^2 (ascending) and
 * w[t*N+r], with sum_r w = F_0(T).  1 <= N <= 9.  Host arrays.  Synchronous.
 */
eri_status eri_rys_roots(int N, int n, const double* T, double* u, double* w);

/* Per-launch record of the last eri_jk call when profiling is on. */
typedef struct {
  int la, lb, lc, ld;             /* class of the launch */
  int team_size;                  /* threads per shell quartet (1, 2, 4, 8, 32 or 128) */
  int grid;                       /* blocks launched */
  float ms;                       /* CUDA-event time of the launch on the call's stream */
  long long quartets;             /* shell quartets evaluated (after screening) */
  long long prim_quartets;        /* primitive quartets evaluated */
  double model_flops;             /* arithmetic of the launch by the kernel's operation count (FP64 + FP32) */
  double model_flops_fp32;        /* its FP32 part */
  int fp32;                       /* 1 for the FP32 path of ERI_MIXED */
  int specialised;                /* 1 for a compile-time specialised small-class kernel */
  int shared_products;            /* 1 when the launch formed each I_x I_y product once per team in
                                     shared memory; 0 for lane programs (products reused within a
                                     lane) */
  int compiled_class;             /* 1 when the team kernel was compiled for this one class (its root
                                     count and recurrence sizes constants) */
  int quartet_split;              /* tasks per shell quartet: > 1 when the class had too few quartets
                                     to fill the GPU and each ran as that many ranges of its
                                     primitive quartets, each digesting its partial sums */
  int listed;                     /* 1 when the kept quartets were compacted into a task list before
                                     the launch; 0 when the kernel screened the class's candidates */
} eri_launch_record;

/* Turn per-launch CUDA-event timing of later eri_jk calls on (1) or off (0). */
eri_status eri_set_profiling(eri_plan* plan, int enable);

/* Records of the last eri_jk call (synchronises its stream): writes up to cap records to
 * out (HOST) and the number available to *n.  Requires profiling to have been on. */
eri_status eri_launch_records(eri_plan* plan, eri_launch_record* out, int cap, int* n);

/*
 * Batched J/K over several jobs (the serving pattern): every job is (plan, D, J, K,
 * flags) exactly as for eri_jk, and the result of each job is that of eri_jk on it
 * alone (up to the order of FP64 atomic additions).  For every angular-momentum
 * class present in any job, the jobs' screened quartets are compacted into one merged
 * task list whose entries carry the job index, and the class runs as ONE kernel launch
 * per precision over all jobs.  Plans may mix ERI_FP64 and ERI_MIXED; all must belong to
 * the device current when the batch was created.  D, J, K: device pointers per job.
 * The batch object owns the merged lists and scratch (grown on demand); calls on one
 * batch must not overlap on the GPU.  Asynchronous on cuda_stream.
 */
typedef struct eri_batch eri_batch;
eri_status eri_batch_create(eri_batch** out);
eri_status eri_batch_destroy(eri_batch* batch);
eri_status eri_jk_batch(eri_batch* batch, int njobs, eri_plan* const* plans, const double* const* D,
                        const int* nD, double* const* J, double* const* K, const int* flags,
                        void* cuda_stream);
/* Quartets evaluated by the last eri_jk_batch call (and how many in FP32), class launches. */
eri_status eri_batch_stats(eri_batch* batch, long long* quartets, long long* quartets_fp32,
                           int* launches);

/*
 * One-electron integrals for the RHF driver (the paper evaluates them on the CPU,
 * Sec. 4): overlap S_ab, kinetic T_ab = -1/2 <a|nabla^2|b> and nuclear attraction
 * V_ab = -sum_C Z_C <a| 1/|r - R_C| |b> over ncharge point charges (charge_xyz
 * [ncharge][3] Bohr, charges [ncharge]).  Same shells, normalisation and Cartesian
 * order as the ERIs.  HOST arrays; S, T, V are [nbf][nbf] row-major, symmetric; any of
 * them may be NULL.  Needs no GPU.  Errors: ERI_ERR_ARG, ERI_ERR_BASIS,
 * ERI_ERR_UNSUPPORTED_L.
 */
eri_status eri_one_electron(const eri_basis* basis, int ncharge, const double* charge_xyz,
                            const double* charges, double* S, double* T, double* V);

/*
 * Host self-check of the per-class assembly tables, needs no GPU: for every J/K class and
 * every gradient class, each [e0|f0] value is assembled by exactly one slot, each slot's
 * 2D-table offsets belong to its value, slots that reuse an I_x I_y product share it with
 * the slot that formed it, and the team regions fit in shared memory.  Writes the number
 * of classes checked and of violations found (0 expected).  Honours ERI_CLASS_CONFIG.
 */
eri_status eri_check_class_tables(int* nclasses, int* problems);

/* Counters of the last eri_jk call (synchronises that call's stream). */
eri_status eri_flop_stats(eri_plan* plan, eri_stats* out);

/* Measured FP64 and FP32 FMA-pipe throughput of device 0 (TFLOP/s), by a timed
 * register-resident FMA loop; the denominators of the fraction-of-peak figures. */
eri_status eri_probe_fma_peak(double* fp64_tflops, double* fp32_tflops);

/* Message of the last failure on this thread ("" if none). */
const char* eri_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ERI_H */
