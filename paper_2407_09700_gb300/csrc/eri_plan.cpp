// Host planner and C-ABI of liberi (see include/eri.h).
//
// Plan creation follows Alg. 1 of Sec. 3: shells are paired (i >= j), each pair
// gets its primitive-pair data (Gaussian product theorem applied to the
// primitives of Eq. 2), Cauchy-Schwarz factors Q_ij (Eq. 7) are computed on the
// GPU from the diagonal quartets (ij|ij), pairs with Q <= tau are dropped and
// the rest are grouped by angular-momentum type (l0 >= l1) and sorted by
// contraction depth.  eri_jk then forms the density block maxima (Eq. 9),
// launches one class kernel per pair of pair types and symmetrises J and K.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/eri.h"
#include "eri_internal.h"
#include "rys_table.h"

namespace {

thread_local std::string g_err;

eri_status fail(eri_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t _e = (cudaError_t)(expr);                                                   \
    if (_e != cudaSuccess) {                                                                \
      if (_e == cudaErrorMemoryAllocation)                                                  \
        return fail(ERI_ERR_OOM, "%s: %s", #expr, cudaGetErrorString(_e));                  \
      return fail(ERI_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                  __LINE__);                                                                \
    }                                                                                       \
  } while (0)

inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
inline int cart_below(int l) { return l * (l + 1) * (l + 2) / 6; }
inline int ptype_of(int l0, int l1) { return l0 * (l0 + 1) / 2 + l1; }
inline void ptype_ls(int t, int* l0, int* l1) {
  int a = 0;
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  *l0 = a;
  *l1 = t - a * (a + 1) / 2;
}

// Cartesian triples in x-descending order, l = 0..9 (host copy of the device table).
struct CartTab {
  int lx[ERI_MAXCART], ly[ERI_MAXCART], lz[ERI_MAXCART];
  CartTab() {
    int g = 0;
    for (int l = 0; l <= ERI_CART_LMAX; ++l)
      for (int x = l; x >= 0; --x)
        for (int y = l - x; y >= 0; --y) {
          lx[g] = x;
          ly[g] = y;
          lz[g] = l - x - y;
          ++g;
        }
  }
};
const CartTab& cart() {
  static CartTab t;
  return t;
}

// ---------------------------------------------------------------- per-device shared state
struct DeviceState {
  bool ready = false;
  double* rys_coef = nullptr;
  double* rys_au = nullptr;
  double* rys_aw = nullptr;
  uint32_t* outidx = nullptr;        // all 225 class index tables
  ClassDesc classes[ERI_NPAIRTYPE][ERI_NPAIRTYPE];
  int ts[ERI_NPAIRTYPE][ERI_NPAIRTYPE];
  uint32_t* grad_outidx = nullptr;   // all gradient class index tables
  GradDesc gclasses[ERI_NPAIRTYPE][ERI_NPAIRTYPE];
  int gts[ERI_NPAIRTYPE][ERI_NPAIRTYPE];
  int sms = 0;
};
std::mutex g_dev_mu;
DeviceState g_dev[64];

int choose_ts(int nout) {
  if (nout <= 32) return 1;
  if (nout <= 8 * 32) return 8;
  return 32;
}

// Block-wide teams (128 lanes, the whole block on one quartet) for the classes with at
// least block_team_min_out() contracted [e0|f0] values: at 32 lanes such a class needs
// several output passes, a batch holds one or two primitive quartets, and every batch
// reloads and restores all partial sums from the team's scratch, while 8 teams per SM hold
// ~1 GB of scratch (far beyond L2).  One team per block with the block's shared memory
// (two blocks per SM) holds ~6 primitive quartets per batch and a quarter of the scratch.
// Measured on the 12-atom s..g build: 1248 ms with 32-lane teams, 1067 ms with block teams
// (lane programs) at two blocks per SM, 1918 ms at one block per SM (four warps do not keep
// the FP64 pipe busy through the team barriers and the transfer phase); block teams from
// 1024 values: 1088 ms.
// ERI_BLOCK_TEAM="min_values budget_doubles" overrides both (tuning on new hardware).
struct BlockTeam { int min_out = 2048, budget = 12000; };
const BlockTeam& block_team() {
  static BlockTeam bt;
  static bool read = false;
  if (!read) {
    read = true;
    if (const char* env = std::getenv("ERI_BLOCK_TEAM")) {
      int m = 0, b = 0;
      if (sscanf(env, "%d %d", &m, &b) == 2 && m > 0 && b >= 1024 && b <= 25000) {
        bt.min_out = m;
        bt.budget = b;
      }
    }
  }
  return bt;
}

// Shared-memory doubles per team for the batch tables: about 98 KB per 128-thread block,
// so two blocks fit on an SM (block-wide teams: the block_team() budget).
int team_budget(int ts) {
  return ts == 2 ? 192 : ts == 4 ? 384 : ts == 8 ? 768 : ts == 128 ? block_team().budget : 3072;
}

// Shared-memory stride between the team regions of a block.  With TS lanes per team, the
// 32 / TS teams of a warp read the same table entries at the same time; a stride of TS
// doubles modulo 16 (FP64 tables) or of TS/2 doubles modulo 16 (FP32 tables, TS floats
// modulo 32) puts the teams of a half-warp on disjoint windows of TS banks (pairs of banks
// for doubles), so their reads of a slot's entries do not collide as long as a team's own
// entries lie in distinct bank windows.
int team_stride(int doubles, int ts, bool f32) {
  if (ts <= 1 || ts >= 16) return doubles;
  const int r = f32 ? ts / 2 : ts;
  return doubles + ((r - doubles % 16) % 16 + 16) % 16;
}

// Per-class overrides of the team size, the products path and the staging of pair records:
// "la lb lc ld ts xy [stage]" entries separated by ';' in ERI_CLASS_CONFIG (xy -1 = automatic;
// stage 1 = bulk-copy staging, where a kernel compiled for the class has it), read once per
// process.  For tuning the choices on new hardware.
struct ClassTune { int ts = -1, xy = -1, stage = 0; };
ClassTune class_tune(int la, int lb, int lc, int ld) {
  static std::vector<std::vector<int>> table;
  static bool read = false;
  if (!read) {
    read = true;
    if (const char* env = std::getenv("ERI_CLASS_CONFIG")) {
      std::string str(env);
      size_t pos = 0;
      while (pos < str.size()) {
        size_t end = str.find(';', pos);
        if (end == std::string::npos) end = str.size();
        std::vector<int> v(7, -1);
        v[6] = 0;
        if (sscanf(str.substr(pos, end - pos).c_str(), "%d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                   &v[6]) >= 5)
          table.push_back(v);
        pos = end + 1;
      }
    }
  }
  ClassTune t;
  // team sizes and assembly paths measured fastest on GB300 for the s/p/d classes of
  // contracted 6-31G(d)-like shells (per-class CUDA-event times of the FP64 build, 1/2/4/8/32
  // lanes compared, 1 = the specialised one-lane kernel; products path -1 = the automatic
  // rule, 0 = lane programs: (dd|dp) 981 -> 878 ms on the 30-atom build)
  static const int measured[][6] = {{2, 1, 1, 0, 1, -1}, {2, 0, 1, 1, 1, -1}, {2, 0, 2, 0, 1, -1},
                                    {2, 2, 1, 0, 4, -1}, {1, 1, 1, 1, 4, -1}, {2, 2, 2, 1, 8, 0}};
  for (const auto& m : measured)
    if (m[0] == la && m[1] == lb && m[2] == lc && m[3] == ld) {
      t.ts = m[4];
      t.xy = m[5];
    }
  for (const auto& v : table)
    if (v[0] == la && v[1] == lb && v[2] == lc && v[3] == ld) {
      if (v[4] == 1 || v[4] == 2 || v[4] == 4 || v[4] == 8 || v[4] == 32 || v[4] == 128) t.ts = v[4];
      t.xy = v[5];
      t.stage = v[6] == 1 ? 1 : 0;
    }
  return t;
}

// Lane programs: values with equal key (their I_x I_y product) form groups; groups are
// split until every group size occurs a multiple of T times (a leftover group of size
// s > 1 becomes s-1 and 1; a leftover of single values is padded) and dealt out so that
// each lane of a T-lane team gets one group of each program entry.  Out: slot_val[o] =
// value index or -1 (padding) for slot o = (k / 32) * 32 T + (k % 32) * T + lane of the
// lane's k-th slot; gm[pass] bit k % 32 set where slot k starts a group (every pass starts
// one); *slots_per_lane.
void lane_programs(const std::vector<int>& key, int T, std::vector<int>* slot_val, std::vector<uint32_t>* gm,
                   int* slots_per_lane) {
  std::vector<std::pair<int, int>> kv;
  for (int v = 0; v < (int)key.size(); ++v) kv.push_back({key[v], v});
  std::stable_sort(kv.begin(), kv.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
    return x.first < y.first;
  });
  std::vector<std::vector<int>> groups;
  for (size_t i = 0; i < kv.size(); ++i) {
    if (i == 0 || kv[i].first != kv[i - 1].first) groups.emplace_back();
    groups.back().push_back(kv[i].second);
  }
  int smax = 1;
  for (const auto& g : groups) smax = std::max(smax, (int)g.size());
  std::vector<std::vector<std::vector<int>>> bys(smax + 1);
  for (auto& g : groups) bys[g.size()].push_back(g);
  std::vector<std::vector<std::vector<int>>> lane(T);
  std::vector<int> prog;
  for (int sz = smax; sz >= 1; --sz) {
    auto& L = bys[sz];
    const int q = (int)L.size() / T, r = (int)L.size() % T;
    for (int t = 0; t < q; ++t) {
      prog.push_back(sz);
      for (int ln = 0; ln < T; ++ln) lane[ln].push_back(L[t * T + ln]);
    }
    if (r) {
      if (sz > 1) {
        for (int t = q * T; t < (int)L.size(); ++t) {
          std::vector<int> head(L[t].begin(), L[t].end() - 1), tail(1, L[t].back());
          bys[sz - 1].push_back(head);
          bys[1].push_back(tail);
        }
      } else {
        prog.push_back(1);
        for (int ln = 0; ln < T; ++ln) lane[ln].push_back(ln < r ? L[q * T + ln] : std::vector<int>(1, -1));
      }
    }
  }
  int Ls = 0;
  for (int sz : prog) Ls += sz;
  const int npass = (Ls + 31) / 32;
  slot_val->assign((size_t)npass * 32 * T, -1);
  slot_val->resize((size_t)Ls * T);
  gm->assign(npass, 0u);
  int k = 0;
  for (int sz : prog) {
    (*gm)[k / 32] |= 1u << (k % 32);
    k += sz;
  }
  for (int p = 0; p < npass; ++p) (*gm)[p] |= 1u;
  for (int ln = 0; ln < T; ++ln) {
    int kk = 0;
    for (const auto& g : lane[ln])
      for (size_t m = 0; m < g.size(); ++m, ++kk) (*slot_val)[(kk / 32) * 32 * T + (kk % 32) * T + ln] = g[m];
  }
  *slots_per_lane = Ls;
}

// Root phase of a batch: items (primitive, root) each evaluate the root polynomials and the
// three axes' recurrences, or (split) items (primitive, root, axis) each evaluate the root
// and one axis.  Split when it needs fewer lane iterations x item cost: it fills teams whose
// bp N items leave lanes idle (high angular momentum, one primitive per batch).
int choose_split3(int T, int bp, int N, int nI, int extra_z) {
  if (T == 1) return 0;
  const double root = 2.0 * RYS_DEG + 12.0, axis = 2.5 * nI;
  const double whole = (double)((bp * N + T - 1) / T) * (root + 3 * axis + extra_z);
  const double split = (double)((3 * bp * N + T - 1) / T) * (root + axis + extra_z);
  return split < 0.9 * whole ? 1 : 0;
}

// Fill the static part of a class descriptor (no device pointers).  idx receives the
// class's u32 tables: lane-program outidx [nslot], dst [nslot], gmask [npass], then (xy
// classes) the shared-products tables xy_outidx [nout], xy_dst [nout], xytab [ncomb],
// passinfo [xy_npass][2].
void make_class(int la, int lb, int lc, int ld, ClassDesc* c, int* ts, std::vector<uint32_t>* idx) {
  memset(c, 0, sizeof(*c));
  c->la = la; c->lb = lb; c->lc = lc; c->ld = ld;
  c->nroots = (la + lb + lc + ld) / 2 + 1;
  c->Le = la + lb;
  c->Lf = lc + ld;
  c->nI = (c->Le + 1) * (c->Lf + 1);
  c->e_base = cart_below(la);
  c->f_base = cart_below(lc);
  c->ne = cart_below(c->Le + 1) - c->e_base;
  c->nf = cart_below(c->Lf + 1) - c->f_base;
  c->nout = c->ne * c->nf;
  c->na = ncart(la); c->nb = ncart(lb); c->nc = ncart(lc); c->nd = ncart(ld);
  const CartTab& ct = cart();
  idx->clear();
  const int L1 = c->Lf + 1;
  const ClassTune tune = class_tune(la, lb, lc, ld);
  *ts = tune.ts > 0 ? tune.ts : (c->nout >= block_team().min_out ? 128 : choose_ts(c->nout));
  c->stage = (tune.stage && *ts == 8 && la == 2 && lb == 1 && lc == 2 && ld == 1) ? 1 : 0;
  const int T = *ts;
  const int per_pass = T * 32;

  // distinct (e_x, e_y) over the e range and (f_x, f_y) over the f range
  std::vector<int> eid(c->ne), fid(c->nf);
  std::vector<int> erep, frep;
  {
    std::vector<int> seen((c->Le + 1) * (c->Le + 1), -1);
    for (int ie = 0; ie < c->ne; ++ie) {
      const int e = c->e_base + ie, key = ct.lx[e] * (c->Le + 1) + ct.ly[e];
      if (seen[key] < 0) { seen[key] = (int)erep.size(); erep.push_back(e); }
      eid[ie] = seen[key];
    }
  }
  {
    std::vector<int> seen((c->Lf + 1) * (c->Lf + 1), -1);
    for (int jf = 0; jf < c->nf; ++jf) {
      const int f = c->f_base + jf, key = ct.lx[f] * (c->Lf + 1) + ct.ly[f];
      if (seen[key] < 0) { seen[key] = (int)frep.size(); frep.push_back(f); }
      fid[jf] = seen[key];
    }
  }
  const int nec = (int)erep.size(), nfc = (int)frep.size();
  c->ncomb = nec * nfc;
  auto slot_word = [&](int ie, int jf) {
    const int e = c->e_base + ie, f = c->f_base + jf;
    return (uint32_t)(ct.lx[e] * L1 + ct.lx[f]) | ((uint32_t)(ct.ly[e] * L1 + ct.ly[f]) << 8) |
           ((uint32_t)(ct.lz[e] * L1 + ct.lz[f]) << 16);
  };

  // ---- lane programs (products reused within a lane's group)
  {
    std::vector<int> key(c->nout);
    for (int ie = 0; ie < c->ne; ++ie)
      for (int jf = 0; jf < c->nf; ++jf) key[ie * c->nf + jf] = eid[ie] * nfc + fid[jf];
    std::vector<int> sv;
    std::vector<uint32_t> gm;
    int Ls = 0;
    lane_programs(key, T, &sv, &gm, &Ls);
    c->nslot = Ls * T;
    c->npass = (int)gm.size();
    std::vector<uint32_t> outi(c->nslot, 1u << 31), dst(c->nslot, 0);
    int xys = 0;
    for (int o = 0; o < c->nslot; ++o) {
      if (sv[o] < 0) continue;
      outi[o] = slot_word(sv[o] / c->nf, sv[o] % c->nf);
      dst[o] = (uint32_t)sv[o];
      const int k = (o / (32 * T)) * 32 + (o % (32 * T)) / T;
      if ((gm[k / 32] >> (k % 32)) & 1u) ++xys;
    }
    c->xysum = xys;
    idx->insert(idx->end(), outi.begin(), outi.end());
    c->dst_off = (int)idx->size();
    idx->insert(idx->end(), dst.begin(), dst.end());
    c->gmask_off = (int)idx->size();
    idx->insert(idx->end(), gm.begin(), gm.end());
  }
  // per primitive quartet: 4 doubles (table lookup) + 18 recurrence-type scalars + three 2D tables
  // the tables of one (primitive, root, axis) lie nIs apart, odd in team kernels: the lanes
  // of a team building different tables then write distinct banks
  c->nIs = (T > 1) ? (c->nI | 1) : c->nI;
  const int per_prim = 4 + 18 + 3 * c->nroots * c->nIs;
  c->bp = (T == 1) ? 1 : std::max(1, std::min(32, team_budget(T) / per_prim));
  c->team_doubles = team_stride(c->bp * per_prim, T, false);
  c->team_doubles_f32 = team_stride(c->bp * 4 + (c->bp * (18 + 3 * c->nroots * c->nIs) + 1) / 2, T, true);
  c->split3 = choose_split3(T, c->bp, c->nroots, c->nI, 0);

  // ---- shared products path (FP64 launches of the classes where it measured faster):
  // values ordered by their product; per pass the first product and the count.
  // Lane programs share a product only within one lane's group and need no
  // synchronisation; the shared path forms each product once per team in shared memory at
  // the cost of a warp synchronisation and a shared-memory round trip per (primitive, root)
  // step and a smaller batch.  Measured on GB300 the shared path wins for FP64 when a lane
  // accumulates at least 20 values per pass, its products save at least a fifth of the
  // multiplies, and the smaller batch costs no more root-phase lane iterations per primitive
  // quartet (ceil(bp N / TS) / bp) than the larger one; for FP32 it never did.
  if (T > 1) {
    struct O { int comb, ie, jf; };
    std::vector<O> ord;
    for (int ie = 0; ie < c->ne; ++ie)
      for (int jf = 0; jf < c->nf; ++jf) ord.push_back({eid[ie] * nfc + fid[jf], ie, jf});
    std::stable_sort(ord.begin(), ord.end(), [](const O& x, const O& y) { return x.comb < y.comb; });
    const int xnp = (c->nout + per_pass - 1) / per_pass;
    std::vector<uint32_t> pinfo(2 * xnp);
    int xymax = 0, xysum = 0;
    for (int p = 0; p < xnp; ++p) {
      const int o0 = p * per_pass, o1 = std::min(c->nout, o0 + per_pass) - 1;
      pinfo[2 * p] = (uint32_t)ord[o0].comb;
      pinfo[2 * p + 1] = (uint32_t)(ord[o1].comb - ord[o0].comb + 1);
      xymax = std::max(xymax, (int)pinfo[2 * p + 1]);
      xysum += (int)pinfo[2 * p + 1];
    }
    const int kcnt = std::min(32, (c->nout + T - 1) / T);
    const int bp_on = std::max(1, std::min(32, (team_budget(T) - 2 * xymax) / per_prim));
    auto iters = [&](int bp) { return (double)((bp * c->nroots + T - 1) / T) / bp; };
    const bool fills = iters(bp_on) <= 1.1 * iters(c->bp);
    // block-wide teams run lane programs: the shared products' barrier per (primitive, root)
    // step stalls four warps at once (12-atom s..g build: 1067 ms with lane programs for
    // every block-team class, 1153 ms with the rule below, 1255 ms with shared products)
    c->xy = (T <= 32 && kcnt >= 20 && 5 * xysum <= 4 * c->nout && fills) ? 1 : 0;
    if (tune.xy >= 0) c->xy = tune.xy ? 1 : 0;
    if (c->xy) {
      c->xy_npass = xnp;
      c->xymax = xymax;
      c->xysum_xy = xysum;
      c->bp_xy = bp_on;
      c->split3_xy = choose_split3(T, bp_on, c->nroots, c->nI, 0);
      c->team_doubles_xy = team_stride(bp_on * per_prim + 2 * xymax, T, false);
      std::vector<uint32_t> outi(c->nout), dst(c->nout);
      for (int p = 0; p < xnp; ++p) {
        const int o0 = p * per_pass, o1 = std::min(c->nout, o0 + per_pass) - 1;
        for (int o = o0; o <= o1; ++o) {
          const uint32_t iz = slot_word(ord[o].ie, ord[o].jf) & 0xff0000u;
          outi[o] = (uint32_t)(ord[o].comb - (int)pinfo[2 * p]) | iz;
          dst[o] = (uint32_t)(ord[o].ie * c->nf + ord[o].jf);
        }
      }
      c->xy_outidx_off = (int)idx->size();
      idx->insert(idx->end(), outi.begin(), outi.end());
      c->xy_dst_off = (int)idx->size();
      idx->insert(idx->end(), dst.begin(), dst.end());
      c->xytab_off = (int)idx->size();
      for (int a2 = 0; a2 < nec; ++a2)
        for (int b2 = 0; b2 < nfc; ++b2) idx->push_back(slot_word(erep[a2] - c->e_base, frep[b2] - c->f_base) & 0xffffu);
      c->pass_off = (int)idx->size();
      idx->insert(idx->end(), pinfo.begin(), pinfo.end());
    }
  }
  // HRR ping-pong size: max level size of the bra (vector nf) and ket (vector nab) passes
  long long m = 1;
  for (int k = 1; k <= lb; ++k) {
    long long na = cart_below(la + lb - k + 1) - cart_below(la);
    m = std::max(m, na * ncart(k) * c->nf);
  }
  for (int k = 1; k <= ld; ++k) {
    long long nc = cart_below(lc + ld - k + 1) - cart_below(lc);
    m = std::max(m, nc * ncart(k) * (long long)(c->na * c->nb));
  }
  c->hrr_doubles = (int)((m + 1) & ~1LL);
  c->scratch_per_team = ((long long)c->nout + 1) / 2 * 2 + 2LL * c->hrr_doubles;
  // FP64 classes with several output passes carry each pass's partial sums from batch to
  // batch in slot order (a warp's loads and stores of them are contiguous)
  const bool multi = c->npass > 1 || (c->xy && c->xy_npass > 1);
  c->part_off = multi ? c->scratch_per_team : 0;
  if (multi) c->scratch_per_team += ((long long)std::max(c->nslot, c->nout) + 1) / 2 * 2;
}

// Fill the static part of a gradient class descriptor (Sec. 4): the four contracted sets,
// their 2D-table offsets tagged with the set, team sizes and the scratch layout.
void make_grad_class(int la, int lb, int lc, int ld, GradDesc* g, int* ts, std::vector<uint32_t>* idx) {
  memset(g, 0, sizeof(*g));
  g->la = la; g->lb = lb; g->lc = lc; g->ld = ld;
  g->na = ncart(la); g->nb = ncart(lb); g->nc = ncart(lc); g->nd = ncart(ld);
  const int Le = la + lb, Lf = lc + ld;
  g->nroots = (Le + Lf + 1) / 2 + 1;
  g->Le2 = Le + 1;
  g->Lf2 = Lf + 1;
  g->nI = (g->Le2 + 1) * (g->Lf2 + 1);
  const int elo[4] = {std::max(la - 1, 0), la + 1, la, la}, ehi[4] = {Le, Le + 1, Le + 1, Le};
  const int flo[4] = {std::max(lc - 1, 0), lc, lc, lc + 1}, fhi[4] = {Lf, Lf, Lf, Lf + 1};
  const CartTab& ct = cart();
  const int L1 = g->Lf2 + 1;
  const int NnI = g->nroots * g->nI;
  idx->clear();
  // values of the four sets (set k, e, f) at S position s_off[k] + ie * s_nf[k] + jf; their
  // I_x I_y key and their I_z offset within the four weighted z tables of a primitive quartet
  std::vector<int> key;
  std::vector<uint32_t> word;
  int off = 0;
  for (int k = 0; k < 4; ++k) {
    g->s_elo[k] = elo[k];
    g->s_flo[k] = flo[k];
    g->s_ne[k] = cart_below(ehi[k] + 1) - cart_below(elo[k]);
    g->s_nf[k] = cart_below(fhi[k] + 1) - cart_below(flo[k]);
    g->s_off[k] = off;
    for (int ie = 0; ie < g->s_ne[k]; ++ie)
      for (int jf = 0; jf < g->s_nf[k]; ++jf) {
        const int e = cart_below(elo[k]) + ie, f = cart_below(flo[k]) + jf;
        const uint32_t ix = ct.lx[e] * L1 + ct.lx[f];
        const uint32_t iy = ct.ly[e] * L1 + ct.ly[f];
        const uint32_t iz = (uint32_t)(k * NnI) + ct.lz[e] * L1 + ct.lz[f];
        key.push_back((int)(ix | (iy << 8)));
        word.push_back(ix | (iy << 8) | (iz << 16));
      }
    off += g->s_ne[k] * g->s_nf[k];
  }
  g->nout = off;
  // block-wide teams for the large classes, as in the J/K build
  *ts = g->nout >= block_team().min_out ? 128 : choose_ts(g->nout);
  std::vector<int> sv;
  std::vector<uint32_t> gm;
  int Ls = 0;
  lane_programs(key, *ts, &sv, &gm, &Ls);
  g->nslot = Ls * *ts;
  g->npass = (int)gm.size();
  std::vector<uint32_t> dst(g->nslot, 0);
  for (int o = 0; o < g->nslot; ++o) {
    idx->push_back(sv[o] < 0 ? (1u << 31) : word[sv[o]]);
    if (sv[o] >= 0) dst[o] = (uint32_t)sv[o];
  }
  g->dst_off = (int)idx->size();
  idx->insert(idx->end(), dst.begin(), dst.end());
  g->gmask_off = (int)idx->size();
  idx->insert(idx->end(), gm.begin(), gm.end());
  // per primitive quartet: 4 doubles (table lookup) + 21 scalars + the I_x, I_y tables and
  // four weighted I_z tables (weights 1, 2 alpha, 2 beta, 2 gamma)
  const int per_prim = 4 + 21 + 6 * NnI;
  if (*ts == 1) {
    g->bp = 1;
  } else {
    g->bp = std::max(1, std::min(32, team_budget(*ts) / per_prim));
  }
  g->team_doubles = team_stride(g->bp * per_prim, *ts, false);
  g->split3 = choose_split3(*ts, g->bp, g->nroots, g->nI, 3 * g->nI);
  const int nabcd = g->na * g->nb * g->nc * g->nd;
  g->gam_off = (off + 1) & ~1;
  g->hrr_off = g->gam_off + ((2 * nabcd + 1) & ~1);
  // largest level of the six transfer sequences: bra (la', lb') over the ket shell's
  // columns, then ket (lc', ld') over the bra block
  long long m = 1;
  auto seq = [&](int a_, int b_, int c_, int d_) {
    const long long nv = cart_below(c_ + d_ + 1) - cart_below(c_);
    for (int k = 1; k <= b_; ++k) m = std::max(m, (long long)(cart_below(a_ + b_ - k + 1) - cart_below(a_)) * ncart(k) * nv);
    const long long nab = (long long)ncart(a_) * ncart(b_);
    for (int k = 1; k <= d_; ++k) m = std::max(m, (long long)(cart_below(c_ + d_ - k + 1) - cart_below(c_)) * ncart(k) * nab);
  };
  seq(la + 1, lb, lc, ld);
  if (la > 0) seq(la - 1, lb, lc, ld);
  seq(la, lb + 1, lc, ld);
  if (lb > 0) seq(la, lb - 1, lc, ld);
  seq(la, lb, lc + 1, ld);
  if (lc > 0) seq(la, lb, lc - 1, ld);
  g->hrr_doubles = (int)((m + 1) & ~1LL);
  g->scratch_per_team = (long long)g->hrr_off + 2LL * g->hrr_doubles;
  g->part_off = g->npass > 1 ? g->scratch_per_team : 0;
  if (g->npass > 1) g->scratch_per_team += ((long long)g->nslot + 1) / 2 * 2;
  g->outidx = nullptr;
}

eri_status device_init(int dev, DeviceState** out) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev < 0 || dev >= 64) return fail(ERI_ERR_ARG, "device index %d out of range", dev);
  DeviceState& s = g_dev[dev];
  if (!s.ready) {
    CUDA_TRY(erik_upload_cart_tables());
    CUDA_TRY(erik_upload_cart_tables_small());
    CUDA_TRY(erik_upload_cart_tables_grad());
    CUDA_TRY(erik_upload_cart_tables_spec());
    CUDA_TRY(erik_class_spec_prepare());
    size_t ncoef = (size_t)RYS_NCOEF, nas = (size_t)RYS_ASYM_OFFSET[RYS_NMAX] + RYS_NMAX;
    CUDA_TRY(cudaMalloc(&s.rys_coef, sizeof(double) * ncoef));
    CUDA_TRY(cudaMalloc(&s.rys_au, sizeof(double) * nas));
    CUDA_TRY(cudaMalloc(&s.rys_aw, sizeof(double) * nas));
    CUDA_TRY(cudaMemcpy(s.rys_coef, RYS_COEF, sizeof(double) * ncoef, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(s.rys_au, RYS_ASYM_U, sizeof(double) * nas, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(s.rys_aw, RYS_ASYM_W, sizeof(double) * nas, cudaMemcpyHostToDevice));
    std::vector<uint32_t> all, one;
    size_t offs[ERI_NPAIRTYPE][ERI_NPAIRTYPE];
    for (int X = 0; X < ERI_NPAIRTYPE; ++X)
      for (int Y = 0; Y < ERI_NPAIRTYPE; ++Y) {
        int la, lb, lc, ld;
        ptype_ls(X, &la, &lb);
        ptype_ls(Y, &lc, &ld);
        make_class(la, lb, lc, ld, &s.classes[X][Y], &s.ts[X][Y], &one);
        offs[X][Y] = all.size();
        all.insert(all.end(), one.begin(), one.end());
      }
    CUDA_TRY(cudaMalloc(&s.outidx, sizeof(uint32_t) * all.size()));
    CUDA_TRY(cudaMemcpy(s.outidx, all.data(), sizeof(uint32_t) * all.size(), cudaMemcpyHostToDevice));
    for (int X = 0; X < ERI_NPAIRTYPE; ++X)
      for (int Y = 0; Y < ERI_NPAIRTYPE; ++Y) {
        ClassDesc& cd = s.classes[X][Y];
        const uint32_t* base = s.outidx + offs[X][Y];
        cd.outidx = base;
        cd.dst = base + cd.dst_off;
        cd.gmask = base + cd.gmask_off;
        if (cd.xy) {
          cd.xy_outidx = base + cd.xy_outidx_off;
          cd.xy_dst = base + cd.xy_dst_off;
          cd.xytab = base + cd.xytab_off;
          cd.passinfo = base + cd.pass_off;
        }
      }
    all.clear();
    for (int X = 0; X < ERI_NPAIRTYPE; ++X)
      for (int Y = 0; Y < ERI_NPAIRTYPE; ++Y) {
        int la, lb, lc, ld;
        ptype_ls(X, &la, &lb);
        ptype_ls(Y, &lc, &ld);
        make_grad_class(la, lb, lc, ld, &s.gclasses[X][Y], &s.gts[X][Y], &one);
        offs[X][Y] = all.size();
        all.insert(all.end(), one.begin(), one.end());
      }
    CUDA_TRY(cudaMalloc(&s.grad_outidx, sizeof(uint32_t) * all.size()));
    CUDA_TRY(cudaMemcpy(s.grad_outidx, all.data(), sizeof(uint32_t) * all.size(), cudaMemcpyHostToDevice));
    for (int X = 0; X < ERI_NPAIRTYPE; ++X)
      for (int Y = 0; Y < ERI_NPAIRTYPE; ++Y) {
        GradDesc& gd = s.gclasses[X][Y];
        gd.outidx = s.grad_outidx + offs[X][Y];
        gd.dst = gd.outidx + gd.dst_off;
        gd.gmask = gd.outidx + gd.gmask_off;
      }
    CUDA_TRY(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev));
    s.ready = true;
  }
  *out = &s;
  return ERI_OK;
}

// Operation count of the class kernel's algorithm (an FMA counts as 2), mirroring
// eri_kernels.cu, split by pipe: per primitive quartet the Gaussian-product scalars and T,
// per root the two degree-11 Horner sums (FP64 always) and the recurrence coefficients,
// the three 2D tables and the Eq. 1 products (a multiply and an FMA per [e0|f0] value and
// root); per contracted quartet the transfer relations and the six digestion updates (both
// FP64 always).  fp32 = 1 counts the FP32 path of the mixed mode.
void class_model_flops2(const ClassDesc& c, int nD, int want, int fp32, double* prim64, double* prim32,
                        double* quart64, double* quart32) {
  const int N = c.nroots, Le = c.Le, Lf = c.Lf;
  const double t_setup = 1 + 4 + 3 + 8 + 3;            // s, rsqrt, PQ, T, table lookup (FP64)
  const double r_setup = 1 + 2 + 6 + 1 + 2 + 2;        // r^2, rz, re, scaled PQ, hs, hz*rz, he*re, Theta
  const double horner = 2.0 * 2.0 * RYS_DEG;             // two Horner sums of RYS_DEG FMAs
  const double coef = 1 + 2 + 2 + 1 + 6 + 6;
  double mult = 0.0, vrr = 0.0;                        // running multiples; three axes
  if (Le >= 1) vrr += 1;                               // z: C00 * I0z
  vrr += 3 * 3.0 * std::max(0, Le - 1);                // fma(C, I, nb10 * I)
  mult += std::max(0, Le - 1);
  if (Lf >= 1) {
    vrr += 1;                                          // z: C00' * I0z
    vrr += 3 * 3.0 * (Lf - 1);                         // row 0
    mult += Lf - 1;
    vrr += Le * (3 * 3.0 + 3 * 5.0 * (Lf - 1));        // rows 1..Le
    mult += Le * (Lf - 1) + Le;
  }
  // Eq. 1 products: one multiply per shared I_x I_y product formed and an FMA per value
  const double asm_ops = (double)((!fp32 && c.xy) ? c.xysum_xy : c.xysum) + 2.0 * c.nout;
  const double rec = N * (coef + mult + vrr) + N * asm_ops;
  double hrr = 0.0;
  for (int k = 1; k <= c.lb; ++k)
    hrr += 2.0 * (cart_below(c.la + c.lb - k + 1) - cart_below(c.la)) * ncart(k) * c.nf;
  for (int k = 1; k <= c.ld; ++k)
    hrr += 2.0 * (cart_below(c.lc + c.ld - k + 1) - cart_below(c.lc)) * ncart(k) * c.na * c.nb;
  const double nabcd = (double)c.na * c.nb * c.nc * c.nd;
  const double dig = 2.0 * nabcd * nD * (((want & 1) ? 2 : 0) + ((want & 2) ? 4 : 0));
  if (fp32) {
    *prim64 = t_setup + N * horner;
    *prim32 = r_setup + 4 + rec;                       // + FP32 rsqrt and PQ
    *quart64 = hrr + dig;
    *quart32 = 0.0;
  } else {
    *prim64 = t_setup + r_setup + N * horner + rec;
    *prim32 = 0.0;
    *quart64 = hrr + dig;
    *quart32 = 0.0;
  }
}

void normalise(int nshell, const int* l, const int* nprim, const int* off, const double* exps,
               const double* raw, std::vector<double>& out) {
  for (int s = 0; s < nshell; ++s) {
    const int L = l[s], K = nprim[s], o = off[s];
    double df = 1.0;
    for (int k = 2 * L - 1; k > 1; k -= 2) df *= k;
    for (int p = 0; p < K; ++p) {
      const double a = exps[o + p];
      out[o + p] = raw[o + p] * std::pow(2.0 * a / M_PI, 0.75) * std::pow(4.0 * a, 0.5 * L) / std::sqrt(df);
    }
    double S = 0.0;
    for (int p = 0; p < K; ++p)
      for (int q = 0; q < K; ++q) {
        const double s2 = exps[o + p] + exps[o + q];
        S += out[o + p] * out[o + q] * df / std::pow(2.0 * s2, L) * std::pow(M_PI / s2, 1.5);
      }
    const double f = 1.0 / std::sqrt(S);
    for (int p = 0; p < K; ++p) out[o + p] *= f;
  }
}

}  // namespace

// ---------------------------------------------------------------- the plan
struct eri_plan {
  int device = 0;
  DeviceState* dev = nullptr;
  eri_opts opts{};
  int natm = 0, nshell = 0, nbf = 0;
  std::vector<double> coords;
  std::vector<int> sh_l, sh_atom, sh_nprim, sh_off, sh_bf0;
  std::vector<double> exps, coefs;
  // all pairs (i >= j) in canonical orientation, grouped by type then depth
  std::vector<ShellPair> pairs_all;
  std::vector<int> pair_index;       // [i*nshell + j] -> index into pairs_all (both orders)
  std::vector<PrimPair> prims;
  int type_off_all[ERI_NPAIRTYPE] = {0}, type_cnt_all[ERI_NPAIRTYPE] = {0};
  // kept pairs (Q > tau)
  int type_off[ERI_NPAIRTYPE] = {0}, type_cnt[ERI_NPAIRTYPE] = {0};
  int type_maxprim[ERI_NPAIRTYPE] = {0};   // most primitive pairs of a kept pair, per type
  int npairs_kept = 0;
  std::vector<double> Q;             // [nshell*nshell]
  std::vector<double> Qe;            // [nshell*nshell] transfer-aware factors of the mixed split
  // device buffers
  ShellPair* d_pairs_all = nullptr;
  ShellPair* d_pairs = nullptr;
  PrimPair* d_prims = nullptr;
  PrimPairF* d_primsf = nullptr;
  int* d_sh_bf0 = nullptr;
  int* d_sh_n = nullptr;
  int* d_sh_atom = nullptr;
  double* d_Dmax = nullptr;
  unsigned long long* d_counters = nullptr;   // one per class launch
  unsigned long long* d_stats = nullptr;      // [2][256][2]: FP64 launches, then FP32 launches
  double* d_scratch = nullptr;
  size_t scratch_doubles = 0;
  int* d_tasks = nullptr;
  size_t tasks_cap = 0;
  double* d_out = nullptr;
  size_t out_cap = 0;
  long long* d_off = nullptr;
  size_t off_cap = 0;
  double* d_host_io = nullptr;                // D, J, K staging for eri_jk_host
  unsigned* d_tlist = nullptr;                // compacted task lists (largest class)
  size_t tlist_cap = 0;
  unsigned long long* d_tcount = nullptr;     // [256][2] FP64 / FP32 list lengths
  unsigned* d_tiles = nullptr;                // per-tile counts / offsets of the compaction
  unsigned long long* d_gstats = nullptr;     // [2] quartets / primitive quartets of eri_jk_grad
  unsigned long long* d_symchk = nullptr;     // [2] max|D_ij - D_ji|, max|D| (check_symmetric)
  unsigned* d_err = nullptr;                  // set by a kernel whose bounded device wait gave up
  cudaStream_t grad_stream = nullptr;
  // second stream of eri_jk: classes alternate between the caller's stream and this one,
  // each with its own half of the task lists, tile counts and scratch
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t tiles_cap = 0;
  size_t host_io_cap = 0;
  cudaStream_t last_stream = nullptr;
  // last eri_jk bookkeeping
  long long last_candidates = 0;
  int last_nclasses = 0, last_nD = 1, last_want = 3;
  // optional per-launch timing
  bool profiling = false;
  std::vector<cudaEvent_t> events;            // 2 per launch
  std::vector<int> last_launch_xy;            // X*15+Y per launch
  std::vector<int> last_launch_ts, last_launch_grid, last_launch_fp32, last_launch_small;
  std::vector<int> last_launch_qsplit, last_launch_listed;
};

namespace {

eri_status ensure_scratch(eri_plan* p, size_t doubles) {
  if (doubles <= p->scratch_doubles) return ERI_OK;
  if (p->d_scratch) {
    CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(p->d_scratch);
    p->d_scratch = nullptr;
    p->scratch_doubles = 0;
  }
  CUDA_TRY(cudaMalloc(&p->d_scratch, sizeof(double) * doubles));
  p->scratch_doubles = doubles;
  return ERI_OK;
}

template <typename T>
eri_status ensure_buf(T** ptr, size_t* cap, size_t n) {
  if (n <= *cap) return ERI_OK;
  if (*ptr) {
    CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
  }
  CUDA_TRY(cudaMalloc(ptr, sizeof(T) * n));
  *cap = n;
  return ERI_OK;
}

// Grid and dynamic shared memory for one class launch.
eri_status launch_shape(eri_plan* p, int X, int Y, int fp32, long long nteams_needed, int* grid, int* smem,
                        int* ts_out) {
  const ClassDesc& c = p->dev->classes[X][Y];
  const int ts = p->dev->ts[X][Y];
  const int teams_per_block = 128 / ts;
  *smem = (int)(sizeof(double) * (size_t)(fp32 ? c.team_doubles_f32 : (c.xy ? c.team_doubles_xy : c.team_doubles)) *
                teams_per_block);
  // staged FP64 launches: per team STAGE_REC 80-byte pair records and an mbarrier, 16-aligned
  if (c.stage && !fp32) *smem = ((*smem + 15) & ~15) + teams_per_block * (20 * (int)sizeof(PrimPair) + 8);
  if (*smem > 200 * 1024) return fail(ERI_ERR_ARG, "class (%d%d|%d%d) needs %d bytes of shared memory", c.la, c.lb, c.lc, c.ld, *smem);
  int bps = 0;
  CUDA_TRY(erik_blocks_per_sm(ts, fp32, (c.xy && !fp32) ? 1 : 0, *smem, &bps));
  if (bps < 1) bps = 1;
  long long full = (long long)p->dev->sms * bps;
  long long need = (nteams_needed + teams_per_block - 1) / teams_per_block;
  *grid = (int)std::max(1LL, std::min(full, need));
  *ts_out = ts;
  return ERI_OK;
}

KernelArgs base_args(eri_plan* p, int X, int Y) {
  KernelArgs a;
  memset(&a, 0, sizeof(a));
  a.c = p->dev->classes[X][Y];
  a.prims = p->d_prims;
  a.primsf = p->d_primsf;
  a.nsh = p->nshell;
  a.nbf = p->nbf;
  const int N = a.c.nroots;
  a.rys_coef = p->dev->rys_coef + RYS_COEF_OFFSET[N];
  a.rys_au = p->dev->rys_au + RYS_ASYM_OFFSET[N];
  a.rys_aw = p->dev->rys_aw + RYS_ASYM_OFFSET[N];
  a.rys_tcut = RYS_TCUT[N];
  a.rys_tcut_d = (double)RYS_TCUT[N];
  a.err = p->d_err;
  return a;
}

// Run explicit (bra, ket) tasks of one class in KMODE_BLOCK or KMODE_SCHWARZ on the all-pairs array.
eri_status run_explicit(eri_plan* p, int X, int Y, int mode, const std::vector<int>& tasks,
                        const std::vector<long long>& offs, size_t out_doubles, cudaStream_t st) {
  const long long nt = (long long)tasks.size() / 2;
  if (nt == 0) return ERI_OK;
  eri_status s;
  if ((s = ensure_buf(&p->d_tasks, &p->tasks_cap, tasks.size())) != ERI_OK) return s;
  if ((s = ensure_buf(&p->d_out, &p->out_cap, std::max<size_t>(out_doubles, 1))) != ERI_OK) return s;
  if (mode == KMODE_BLOCK && (s = ensure_buf(&p->d_off, &p->off_cap, offs.size())) != ERI_OK) return s;
  int grid, smem, ts;
  if ((s = launch_shape(p, X, Y, 0, nt, &grid, &smem, &ts)) != ERI_OK) return s;
  const ClassDesc& c = p->dev->classes[X][Y];
  size_t need = (size_t)grid * (size_t)(128 / ts) * (size_t)c.scratch_per_team;
  if ((s = ensure_scratch(p, need)) != ERI_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(p->d_tasks, tasks.data(), sizeof(int) * tasks.size(), cudaMemcpyHostToDevice, st));
  if (mode == KMODE_BLOCK)
    CUDA_TRY(cudaMemcpyAsync(p->d_off, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned long long), st));
  KernelArgs a = base_args(p, X, Y);
  a.pairs = p->d_pairs_all;
  a.ntask = nt;
  a.mode = mode;
  a.tasklist = p->d_tasks;
  a.blockout = p->d_out;
  a.blockoff = p->d_off;
  a.qout = p->d_out;
  a.counter = p->d_counters;
  a.scratch = p->d_scratch;
  a.stats = nullptr;
  CUDA_TRY(erik_launch_class(ts, 0, &a, grid, smem, st));
  return ERI_OK;
}

eri_status validate_basis(const eri_basis* b) {
  if (!b) return fail(ERI_ERR_ARG, "basis is NULL");
  if (b->natm < 1 || !b->coords) return fail(ERI_ERR_ARG, "natm must be >= 1 with coords");
  if (b->nshell < 1 || !b->shell_atom || !b->shell_l || !b->shell_nprim || !b->shell_off || !b->exps ||
      !b->coefs)
    return fail(ERI_ERR_ARG, "nshell must be >= 1 and every shell array non-NULL");
  for (int i = 0; i < 3 * b->natm; ++i)
    if (!std::isfinite(b->coords[i])) return fail(ERI_ERR_BASIS, "coordinate %d is not finite", i);
  for (int s = 0; s < b->nshell; ++s) {
    if (b->shell_l[s] < 0) return fail(ERI_ERR_BASIS, "shell %d has l < 0", s);
    if (b->shell_l[s] > ERI_LMAX) return fail(ERI_ERR_UNSUPPORTED_L, "shell %d has l = %d > 4", s, b->shell_l[s]);
    if (b->shell_nprim[s] < 1) return fail(ERI_ERR_BASIS, "shell %d has nprim < 1", s);
    if (b->shell_off[s] < 0) return fail(ERI_ERR_BASIS, "shell %d has a negative offset", s);
    if (b->shell_atom[s] < 0 || b->shell_atom[s] >= b->natm) return fail(ERI_ERR_BASIS, "shell %d has a bad atom index", s);
    for (int p = 0; p < b->shell_nprim[s]; ++p) {
      const double e = b->exps[b->shell_off[s] + p], c = b->coefs[b->shell_off[s] + p];
      if (!std::isfinite(e) || !(e > 0)) return fail(ERI_ERR_BASIS, "shell %d primitive %d: exponent must be finite and > 0", s, p);
      if (!std::isfinite(c)) return fail(ERI_ERR_BASIS, "shell %d primitive %d: coefficient is not finite", s, p);
    }
  }
  return ERI_OK;
}


// ---------------------------------------------------------------- J/K launch machinery
struct Launch {
  int X, Y, fp32, grid, smem, ts;
  long long nt;
  int small;             // 1: compile-time specialised kernel (eri_small.cu)
  int split;             // 1: the class runs an FP64 and an FP32 launch (mixed mode)
  int qsplit;            // tasks per quartet (ranges of its primitive quartets), 1 = none
};

// Classes with at most this many candidate quartets screen in the kernel instead of being
// compacted first (three launches saved per class on small molecules).
constexpr long long kListMinTasks = 8192;
// Tasks per quartet for a class launch whose candidate quartets cannot fill the grid's
// teams: a team works through its quartet's primitive quartets one after another, and an
// FP64 warp instruction occupies a sub-partition's FP64 unit for 64 cycles on GB300, so a
// handful of deep quartets (81 primitive quartets for three-term shells) leaves the launch
// waiting on a few teams.  Split each quartet into ranges of its primitive quartets, as many
// as the idle teams allow (at most one per primitive quartet, at most 64), each range
// digesting its partial [e0|f0] (the transfer relations and digestion are linear).
// teams: the teams a full grid holds; minq: the fewest primitive quartets worth a task (a
// batch of the team kernel).
int choose_qsplit(long long nt, long long teams, int maxq, int minq) {
  if (nt <= 0 || maxq <= minq || nt * 2 > teams) return 1;
  const long long q = (teams + nt - 1) / nt;
  return (int)std::max(1LL, std::min<long long>({q, (long long)(maxq / std::max(1, minq)), 64LL}));
}

eri_status check_jk_args(eri_plan* p, const double* D, int nD, double* J, double* K, int flags) {
  if (!p) return fail(ERI_ERR_ARG, "plan is NULL");
  if (!D) return fail(ERI_ERR_ARG, "D is NULL");
  if (nD < 1 || nD > p->opts.max_nd) return fail(ERI_ERR_ARG, "nD = %d outside [1, %d]", nD, p->opts.max_nd);
  const int want = flags & 3;
  if (want == 0) return fail(ERI_ERR_ARG, "flags request neither J nor K");
  if ((want & 1) && !J) return fail(ERI_ERR_ARG, "J requested but NULL");
  if ((want & 2) && !K) return fail(ERI_ERR_ARG, "K requested but NULL");
  return ERI_OK;
}

// In the mixed mode, whether class (X|Y) gets an FP32 launch: its task space must reach the
// plan's mixed_min_tasks (a second launch for a handful of quartets costs more than the FP32
// arithmetic saves); otherwise every quartet of the class runs in FP64.
bool fp32_pays(const eri_plan* p, int X, int Y, long long nt) {
  (void)X;
  (void)Y;
  return nt >= (long long)p->opts.mixed_min_tasks;
}

// One launch per class (pair-type pair X >= Y); in the mixed mode one FP64 and one FP32
// launch per class.  Grids are capped so that grid * teams * scratch <= max_scratch when
// max_scratch > 0.
eri_status plan_launches(eri_plan* p, size_t max_scratch, std::vector<Launch>* out) {
  out->clear();
  const int nprec = (p->opts.precision == ERI_MIXED) ? 2 : 1;
  for (int X = 0; X < ERI_NPAIRTYPE; ++X) {
    if (!p->type_cnt[X]) continue;
    for (int Y = 0; Y <= X; ++Y) {
      if (!p->type_cnt[Y]) continue;
      const long long nx = p->type_cnt[X], ny = p->type_cnt[Y];
      const long long nt = (X == Y) ? nx * (nx + 1) / 2 : nx * ny;
      const int np = (nprec == 2 && fp32_pays(p, X, Y, nt)) ? 2 : 1;
      for (int fp32 = 0; fp32 < np; ++fp32) {
        Launch l{X, Y, fp32, 0, 0, 0, nt, 0, np == 2 ? 1 : 0, 1};
        const ClassDesc& cd = p->dev->classes[X][Y];
        // a full grid first: the teams it holds decide the split, the split the grid
        eri_status s = launch_shape(p, X, Y, fp32, 1LL << 40, &l.grid, &l.smem, &l.ts);
        if (s != ERI_OK) return s;
        const int maxq = p->type_maxprim[X] * p->type_maxprim[Y];
        l.qsplit = choose_qsplit(nt, (long long)l.grid * (128 / l.ts), maxq,
                                 fp32 ? cd.bp : (cd.xy ? cd.bp_xy : cd.bp));
        s = launch_shape(p, X, Y, fp32, nt * l.qsplit, &l.grid, &l.smem, &l.ts);
        if (s != ERI_OK) return s;
        // specialised one-lane kernel: FP64 when the class runs with one lane per quartet,
        // FP32 whenever one exists (its accumulators fit a lane in FP32)
        if ((fp32 || l.ts == 1) && erik_small_available(cd.la, cd.lb, cd.lc, cd.ld, fp32)) {
          l.ts = 1;
          int bps = 0;
          CUDA_TRY(erik_small_blocks_per_sm(cd.la, cd.lb, cd.lc, cd.ld, fp32, &bps));
          if (bps < 1) bps = 1;
          const long long full = (long long)p->dev->sms * bps;
          l.qsplit = choose_qsplit(nt, full * 128, maxq, 2);
          const long long need = (nt * l.qsplit + 127) / 128;
          l.grid = (int)std::max(1LL, std::min(full, need));
          l.smem = 0;
          l.small = 1;
        }
        if (max_scratch > 0) {
          const ClassDesc& c = p->dev->classes[X][Y];
          const size_t per_block = (size_t)(128 / l.ts) * (size_t)c.scratch_per_team;
          if (per_block > max_scratch)
            return fail(ERI_ERR_ARG,
                        "class (%d%d|%d%d) needs %zu bytes of scratch for one block, more than the %zu-byte "
                        "static scratch of eri_jk_noalloc",
                        c.la, c.lb, c.lc, c.ld, per_block * sizeof(double), max_scratch * sizeof(double));
          l.grid = (int)std::min<size_t>((size_t)l.grid, max_scratch / per_block);
        }
        out->push_back(l);
      }
    }
  }
  return ERI_OK;
}

// Density maxima, every class launch, symmetrisation.  Records launches for the profiler
// when record is set.  Allocates nothing except profiling events when record is set.
// With two streams (nstreams = 2) the class launches alternate between st and the plan's
// side stream, so one class's launch fills the SMs that the previous class's tail leaves
// idle; stream s uses task list d_tlist + s * list_half, tile counts d_tiles + s *
// tiles_half and scratch + s * scratch_half.  Per-launch profiling forces one stream so
// that each launch's events time it alone.
eri_status run_jk(eri_plan* p, const std::vector<Launch>& launches, const double* D, int nD, double* J, double* K,
                  int want, cudaStream_t st, double* scratch, bool record, bool use_lists, int nstreams = 1,
                  size_t list_half = 0, size_t tiles_half = 0, size_t scratch_half = 0) {
  const size_t mat = (size_t)nD * p->nbf * p->nbf;
  if (want & 1) CUDA_TRY(cudaMemsetAsync(J, 0, sizeof(double) * mat, st));
  if (want & 2) CUDA_TRY(cudaMemsetAsync(K, 0, sizeof(double) * mat, st));
  CUDA_TRY(erik_launch_dmax(D, nD, p->nbf, p->nshell, p->d_sh_bf0, p->d_sh_n, p->d_Dmax, st));
  CUDA_TRY(cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned long long) * 256, st));
  CUDA_TRY(cudaMemsetAsync(p->d_stats, 0, sizeof(unsigned long long) * 4 * 256, st));
  if (use_lists) CUDA_TRY(cudaMemsetAsync(p->d_tcount, 0, sizeof(unsigned long long) * 2 * 256, st));
  const bool prof = record && p->profiling;
  if (prof) nstreams = 1;
  cudaStream_t ss[2] = {st, st};
  if (nstreams == 2) {
    if (!p->side) {
      CUDA_TRY(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    }
    ss[1] = p->side;
  }
  if (prof) {
    while (p->events.size() < 2 * launches.size()) {
      cudaEvent_t e;
      CUDA_TRY(cudaEventCreate(&e));
      p->events.push_back(e);
    }
  }
  // an unrecorded call (eri_jk_noalloc) leaves no records, so eri_launch_records never mixes
  // an earlier call's launches with this call's counters
  p->last_launch_xy.clear();
  p->last_launch_ts.clear();
  p->last_launch_grid.clear();
  p->last_launch_fp32.clear();
  p->last_launch_small.clear();
  p->last_launch_qsplit.clear();
  p->last_launch_listed.clear();
  if (nstreams == 2) {
    CUDA_TRY(cudaEventRecord(p->ev_fork, st));
    CUDA_TRY(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  }
  const size_t list_cap = nstreams == 2 ? list_half : p->tlist_cap;
  long long cand = 0;
  int li = 0, ci = -1;
  const bool mixed = p->opts.precision == ERI_MIXED;
  for (const Launch& l : launches) {
    const bool listed = use_lists && l.nt > kListMinTasks && (unsigned long long)l.nt <= 0xffffffffULL &&
                        (size_t)l.nt <= list_cap;
    const int sidx = (nstreams == 2) ? ((ci + (l.fp32 ? 0 : 1)) & 1) : 0;
    const cudaStream_t sl = ss[sidx];
    unsigned* tlist_l = p->d_tlist + (size_t)sidx * list_half;
    unsigned* tiles_l = p->d_tiles + (size_t)sidx * tiles_half;
    KernelArgs a = base_args(p, l.X, l.Y);
    a.pairs = p->d_pairs;
    a.bra0 = p->type_off[l.X];
    a.nbra = p->type_cnt[l.X];
    a.ket0 = p->type_off[l.Y];
    a.nket = p->type_cnt[l.Y];
    a.tri = (l.X == l.Y);
    a.ntask = l.nt;
    a.Dmax = p->d_Dmax;
    a.tau = p->opts.screen_thresh;
    a.prec_sel = l.split ? (l.fp32 ? 2 : 1) : 0;
    a.mixed_thr = p->opts.mixed_thresh;
    a.D = D;
    a.J = J;
    a.K = K;
    a.nD = nD;
    a.want = want;
    a.mode = KMODE_JK;
    a.counter = p->d_counters + li;
    a.scratch = scratch + (size_t)sidx * scratch_half;
    a.qsplit = l.qsplit;
    a.stats = p->d_stats + 2 * (256 * l.fp32 + l.X * ERI_NPAIRTYPE + l.Y);
    if (!l.fp32) ++ci;
    if (listed) {
      unsigned long long* cnt = p->d_tcount + 2 * ci;
      if (!l.fp32)
        CUDA_TRY(erik_launch_compact(&a, tlist_l, (unsigned long long)l.nt, cnt, tiles_l, l.split, sl));
      a.tlist = tlist_l;
      a.list_cap = (unsigned long long)l.nt;
      a.from_back = l.fp32;
      a.tcount = cnt + l.fp32;
    }
    if (prof) CUDA_TRY(cudaEventRecord(p->events[2 * li], sl));
    if (l.small)
      CUDA_TRY(erik_launch_small(a.c.la, a.c.lb, a.c.lc, a.c.ld, l.fp32, &a, l.grid, sl));
    else
      CUDA_TRY(erik_launch_class(l.ts, l.fp32, &a, l.grid, l.smem, sl));
    if (prof) CUDA_TRY(cudaEventRecord(p->events[2 * li + 1], sl));
    if (record) {
      p->last_launch_xy.push_back(l.X * ERI_NPAIRTYPE + l.Y);
      p->last_launch_ts.push_back(l.ts);
      p->last_launch_grid.push_back(l.grid);
      p->last_launch_fp32.push_back(l.fp32);
      p->last_launch_small.push_back(l.small);
      p->last_launch_qsplit.push_back(l.qsplit);
      p->last_launch_listed.push_back(listed ? 1 : 0);
    }
    if (!l.fp32) cand += l.nt;
    ++li;
  }
  if (nstreams == 2) {
    CUDA_TRY(cudaEventRecord(p->ev_join, p->side));
    CUDA_TRY(cudaStreamWaitEvent(st, p->ev_join, 0));
  }
  if (want & 1) CUDA_TRY(erik_launch_symmetrize(J, nD, p->nbf, st));
  if (want & 2) CUDA_TRY(erik_launch_symmetrize(K, nD, p->nbf, st));
  p->last_stream = st;
  p->last_candidates = cand;
  p->last_nclasses = (int)launches.size();
  p->last_nD = nD;
  p->last_want = want;
  return ERI_OK;
}

// eri_jk's launches and the sizes of its buffers: scratch per stream (need doubles), task
// list per stream (maxnt) and tile counts per stream (tiles).  Everything depends on the
// plan alone, so the buffers are allocated once, at plan creation, and no eri_jk call
// allocates (ensure_* find them large enough).  The side stream and its events too.
eri_status size_jk_buffers(eri_plan* p, std::vector<Launch>* launches, size_t* need_out, size_t* maxnt_out,
                           size_t* tiles_out) {
  eri_status s;
  if ((s = plan_launches(p, 0, launches)) != ERI_OK) return s;
  size_t need = 0;
  for (const Launch& l : *launches)
    need = std::max(need, (size_t)l.grid * (size_t)(128 / l.ts) * (size_t)p->dev->classes[l.X][l.Y].scratch_per_team);
  need = (need + 31) & ~(size_t)31;
  size_t maxnt = 1;
  for (const Launch& l : *launches)
    if ((unsigned long long)l.nt <= 0xffffffffULL) maxnt = std::max(maxnt, (size_t)l.nt);
  maxnt = (maxnt + 31) & ~(size_t)31;
  const size_t tiles = 2 * ((maxnt + 1023) / 1024 + 1);
  // two streams, each with its own half of scratch, task lists and tile counts
  if ((s = ensure_scratch(p, 2 * need)) != ERI_OK) return s;
  if ((s = ensure_buf(&p->d_tlist, &p->tlist_cap, 2 * maxnt)) != ERI_OK) return s;
  if ((s = ensure_buf(&p->d_tiles, &p->tiles_cap, 2 * tiles)) != ERI_OK) return s;
  if (!p->side) {
    CUDA_TRY(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  }
  *need_out = need;
  *maxnt_out = maxnt;
  *tiles_out = tiles;
  return ERI_OK;
}

// Symmetry of the densities on the device (the plan's check_symmetric option): max|D_ij - D_ji|
// against 1e-12 max|D|; synchronises the stream.  The plan's d_symchk holds the two maxima.
eri_status check_density_device(eri_plan* p, const double* D, int nD, cudaStream_t st) {
  unsigned long long h[2] = {0, 0};
  CUDA_TRY(cudaMemsetAsync(p->d_symchk, 0, sizeof(h), st));
  CUDA_TRY(erik_launch_symcheck(D, nD, p->nbf, p->d_symchk, st));
  CUDA_TRY(cudaMemcpyAsync(h, p->d_symchk, sizeof(h), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  double asym, mx;
  memcpy(&asym, &h[0], sizeof(double));
  memcpy(&mx, &h[1], sizeof(double));
  if (!(asym <= 1e-12 * mx))
    return fail(ERI_ERR_ARG, "D is not symmetric: max|D_ij - D_ji| = %.3e, max|D| = %.3e", asym, mx);
  return ERI_OK;
}
}  // namespace

// ================================================================= C-ABI
extern "C" {

const char* eri_last_error(void) { return g_err.c_str(); }

int eri_plan_nbf(const eri_plan* p) { return p ? p->nbf : -1; }

eri_status eri_plan_destroy(eri_plan* p) {
  if (!p) return ERI_OK;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  void* bufs[] = {p->d_pairs_all, p->d_pairs, p->d_prims, p->d_primsf, p->d_sh_bf0, p->d_sh_n, p->d_sh_atom, p->d_Dmax, p->d_counters,
                  p->d_stats, p->d_scratch, p->d_tasks, p->d_out, p->d_off, p->d_host_io, p->d_tlist,
                  p->d_tcount, p->d_tiles, p->d_gstats, p->d_symchk, p->d_err};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
  return ERI_OK;
}

eri_status eri_plan_create(const eri_basis* basis, const eri_opts* opts, void* cuda_stream, eri_plan** out) {
  g_err.clear();
  if (!out) return fail(ERI_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!opts) return fail(ERI_ERR_ARG, "opts is NULL");
  if (!(opts->screen_thresh >= 0) || !std::isfinite(opts->screen_thresh))
    return fail(ERI_ERR_ARG, "screen_thresh must be finite and >= 0");
  if (opts->max_nd < 1) return fail(ERI_ERR_ARG, "max_nd must be >= 1");
  if (opts->precision != ERI_FP64 && opts->precision != ERI_MIXED) return fail(ERI_ERR_ARG, "unknown precision mode");
  if (opts->check_symmetric != 0 && opts->check_symmetric != 1) return fail(ERI_ERR_ARG, "check_symmetric must be 0 or 1");
  if (opts->mixed_min_tasks < 0) return fail(ERI_ERR_ARG, "mixed_min_tasks must be >= 0");
  eri_status s = validate_basis(basis);
  if (s != ERI_OK) return s;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(ERI_ERR_NO_DEVICE, "no CUDA device is visible");
  }
  eri_plan* p = new (std::nothrow) eri_plan();
  if (!p) return fail(ERI_ERR_OOM, "host allocation failed");
  cudaGetDevice(&p->device);
  if ((s = device_init(p->device, &p->dev)) != ERI_OK) { delete p; return s; }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  p->opts = *opts;
  p->natm = basis->natm;
  p->nshell = basis->nshell;
  p->coords.assign(basis->coords, basis->coords + 3 * basis->natm);
  p->sh_l.assign(basis->shell_l, basis->shell_l + p->nshell);
  p->sh_atom.assign(basis->shell_atom, basis->shell_atom + p->nshell);
  p->sh_nprim.assign(basis->shell_nprim, basis->shell_nprim + p->nshell);
  p->sh_off.assign(basis->shell_off, basis->shell_off + p->nshell);
  int nprim_total = 0;
  for (int i = 0; i < p->nshell; ++i) nprim_total = std::max(nprim_total, p->sh_off[i] + p->sh_nprim[i]);
  p->exps.assign(basis->exps, basis->exps + nprim_total);
  p->coefs.assign(basis->coefs, basis->coefs + nprim_total);
  if (basis->normalise) normalise(p->nshell, p->sh_l.data(), p->sh_nprim.data(), p->sh_off.data(), p->exps.data(), basis->coefs, p->coefs);
  p->sh_bf0.resize(p->nshell);
  std::vector<int> sh_n(p->nshell);
  for (int i = 0; i < p->nshell; ++i) {
    p->sh_bf0[i] = p->nbf;
    sh_n[i] = ncart(p->sh_l[i]);
    p->nbf += sh_n[i];
  }

  // ---- shell pairs (i >= j) in canonical orientation, grouped by type and depth.
  // A primitive pair whose Gaussian-product factor exp(-ab/(a+b) |A-B|^2) is below 1e-30
  // (exponent argument above PRIM_PAIR_CUT) is dropped: with contraction coefficients and
  // polynomial factors each below ~1e4 its contribution to any integral stays under 1e-22,
  // far below FP64 resolution of the retained terms.  Each shell pair keeps at least its
  // primitive pair of largest factor.
  const double PRIM_PAIR_CUT = 69.0;
  struct Tmp { int t, np, i, j; std::vector<int> keep; };
  std::vector<Tmp> tmp;
  for (int i = 0; i < p->nshell; ++i)
    for (int j = 0; j <= i; ++j) {
      int a = i, b = j;
      if (p->sh_l[b] > p->sh_l[a]) std::swap(a, b);
      const double* A = &p->coords[3 * p->sh_atom[a]];
      const double* B = &p->coords[3 * p->sh_atom[b]];
      double AB2 = 0.0;
      for (int x = 0; x < 3; ++x) AB2 += (A[x] - B[x]) * (A[x] - B[x]);
      Tmp t{ptype_of(p->sh_l[a], p->sh_l[b]), 0, a, b, {}};
      int best = 0;
      double best_arg = 1e300;
      for (int u = 0; u < p->sh_nprim[a]; ++u)
        for (int v = 0; v < p->sh_nprim[b]; ++v) {
          const double al = p->exps[p->sh_off[a] + u], be = p->exps[p->sh_off[b] + v];
          const double arg = al * be / (al + be) * AB2;
          const int code = u * p->sh_nprim[b] + v;
          if (arg <= PRIM_PAIR_CUT) t.keep.push_back(code);
          if (arg < best_arg) { best_arg = arg; best = code; }
        }
      if (t.keep.empty()) t.keep.push_back(best);
      t.np = (int)t.keep.size();
      tmp.push_back(std::move(t));
    }
  std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp& x, const Tmp& y) {
    return x.t != y.t ? x.t < y.t : x.np > y.np;
  });
  const double pref = std::sqrt(2.0) * std::pow(M_PI, 1.25);
  p->pair_index.assign((size_t)p->nshell * p->nshell, -1);
  for (size_t k = 0; k < tmp.size(); ++k) {
    const Tmp& t = tmp[k];
    ShellPair sp;
    memset(&sp, 0, sizeof(sp));
    sp.sh0 = t.i;
    sp.sh1 = t.j;
    sp.bf0 = p->sh_bf0[t.i];
    sp.bf1 = p->sh_bf0[t.j];
    sp.prim_off = (int)p->prims.size();
    sp.nprim = t.np;
    sp.ptype = t.t;
    sp.Qe = 0.f;
    const double* A = &p->coords[3 * p->sh_atom[t.i]];
    const double* B = &p->coords[3 * p->sh_atom[t.j]];
    double AB2 = 0.0;
    for (int x = 0; x < 3; ++x) {
      sp.AB[x] = A[x] - B[x];
      AB2 += sp.AB[x] * sp.AB[x];
    }
    for (int code : t.keep) {
      const int u = code / p->sh_nprim[t.j], v = code % p->sh_nprim[t.j];
      const double al = p->exps[p->sh_off[t.i] + u], be = p->exps[p->sh_off[t.j] + v];
      const double ca = p->coefs[p->sh_off[t.i] + u], cb = p->coefs[p->sh_off[t.j] + v];
      PrimPair pp;
      pp.zeta = al + be;
      for (int x = 0; x < 3; ++x) {
        pp.P[x] = (al * A[x] + be * B[x]) / pp.zeta;
        pp.PA[x] = pp.P[x] - A[x];
      }
      pp.E = pref / pp.zeta * std::exp(-al * be / pp.zeta * AB2) * ca * cb;
      pp.hz = 0.5 / pp.zeta;
      pp.alpha = al;
      p->prims.push_back(pp);
    }
    p->pairs_all.push_back(sp);
    p->pair_index[(size_t)t.i * p->nshell + t.j] = (int)k;
    p->pair_index[(size_t)t.j * p->nshell + t.i] = (int)k;
    p->type_cnt_all[t.t]++;
  }
  for (int t = 1; t < ERI_NPAIRTYPE; ++t) p->type_off_all[t] = p->type_off_all[t - 1] + p->type_cnt_all[t - 1];

  auto cleanup = [&](eri_status e) { eri_plan_destroy(p); return e; };
  const size_t npair = p->pairs_all.size();
  if (cudaMalloc(&p->d_pairs_all, sizeof(ShellPair) * npair) != cudaSuccess ||
      cudaMalloc(&p->d_pairs, sizeof(ShellPair) * npair) != cudaSuccess ||
      cudaMalloc(&p->d_prims, sizeof(PrimPair) * p->prims.size()) != cudaSuccess ||
      cudaMalloc(&p->d_primsf, sizeof(PrimPairF) * p->prims.size()) != cudaSuccess ||
      cudaMalloc(&p->d_sh_bf0, sizeof(int) * p->nshell) != cudaSuccess ||
      cudaMalloc(&p->d_sh_n, sizeof(int) * p->nshell) != cudaSuccess ||
      cudaMalloc(&p->d_sh_atom, sizeof(int) * p->nshell) != cudaSuccess ||
      cudaMalloc(&p->d_Dmax, sizeof(double) * p->nshell * p->nshell) != cudaSuccess ||
      cudaMalloc(&p->d_counters, sizeof(unsigned long long) * 256) != cudaSuccess ||
      cudaMalloc(&p->d_stats, sizeof(unsigned long long) * 4 * 256) != cudaSuccess ||
      cudaMalloc(&p->d_tcount, sizeof(unsigned long long) * 2 * 256) != cudaSuccess ||
      cudaMalloc(&p->d_symchk, sizeof(unsigned long long) * 2) != cudaSuccess ||
      cudaMalloc(&p->d_err, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(fail(ERI_ERR_OOM, "device allocation failed in eri_plan_create"));
  }
#define PLAN_TRY(expr)                                        \
  do {                                                        \
    cudaError_t _e = (cudaError_t)(expr);                     \
    if (_e != cudaSuccess)                                    \
      return cleanup(fail(ERI_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e))); \
  } while (0)
  PLAN_TRY(cudaMemcpyAsync(p->d_pairs_all, p->pairs_all.data(), sizeof(ShellPair) * npair, cudaMemcpyHostToDevice, st));
  PLAN_TRY(cudaMemcpyAsync(p->d_prims, p->prims.data(), sizeof(PrimPair) * p->prims.size(), cudaMemcpyHostToDevice, st));
  std::vector<PrimPairF> primsf(p->prims.size());
  for (size_t k = 0; k < p->prims.size(); ++k) {
    const PrimPair& x = p->prims[k];
    PrimPairF& f = primsf[k];
    f.zeta = (float)x.zeta;
    for (int c = 0; c < 3; ++c) f.PA[c] = (float)x.PA[c];
    f.E = (float)x.E;
    f.hz = (float)x.hz;
    f.pad[0] = f.pad[1] = 0.f;
  }
  PLAN_TRY(cudaMemcpyAsync(p->d_primsf, primsf.data(), sizeof(PrimPairF) * primsf.size(), cudaMemcpyHostToDevice, st));
  PLAN_TRY(cudaMemcpyAsync(p->d_sh_bf0, p->sh_bf0.data(), sizeof(int) * p->nshell, cudaMemcpyHostToDevice, st));
  PLAN_TRY(cudaMemcpyAsync(p->d_sh_n, sh_n.data(), sizeof(int) * p->nshell, cudaMemcpyHostToDevice, st));
  PLAN_TRY(cudaMemcpyAsync(p->d_sh_atom, p->sh_atom.data(), sizeof(int) * p->nshell, cudaMemcpyHostToDevice, st));
  PLAN_TRY(cudaMemsetAsync(p->d_stats, 0, sizeof(unsigned long long) * 4 * 256, st));
  PLAN_TRY(cudaMemsetAsync(p->d_err, 0, sizeof(unsigned), st));

  // ---- Schwarz factors (Eq. 7) from the diagonal quartets (ij|ij), one class (X|X) at a time;
  // the same launches give max_e [e0|e0] before the transfer relations, for the mixed mode's
  // transfer-aware factor Qe = sqrt(max_e [e0|e0]) (1 + max_x |A-B|_x)^l1
  p->Q.assign((size_t)p->nshell * p->nshell, 0.0);
  p->Qe.assign((size_t)p->nshell * p->nshell, 0.0);
  std::vector<double> qmax(npair, 0.0), emax(npair, 0.0), qbuf;
  for (int X = 0; X < ERI_NPAIRTYPE; ++X) {
    const int n = p->type_cnt_all[X];
    if (n == 0) continue;
    std::vector<int> tasks(2 * n);
    for (int k = 0; k < n; ++k) tasks[2 * k] = tasks[2 * k + 1] = p->type_off_all[X] + k;
    if ((s = run_explicit(p, X, X, KMODE_SCHWARZ, tasks, {}, 2 * (size_t)n, st)) != ERI_OK) return cleanup(s);
    qbuf.resize(2 * (size_t)n);
    PLAN_TRY(cudaMemcpyAsync(qbuf.data(), p->d_out, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st));
    PLAN_TRY(cudaStreamSynchronize(st));
    std::copy(qbuf.begin(), qbuf.begin() + n, qmax.begin() + p->type_off_all[X]);
    std::copy(qbuf.begin() + n, qbuf.end(), emax.begin() + p->type_off_all[X]);
  }
  for (size_t k = 0; k < npair; ++k) {
    ShellPair& sp = p->pairs_all[k];
    sp.Q = std::sqrt(qmax[k]);
    const double ab = std::max(std::fabs(sp.AB[0]), std::max(std::fabs(sp.AB[1]), std::fabs(sp.AB[2])));
    const double qe = std::sqrt(emax[k]) * std::pow(1.0 + ab, p->sh_l[sp.sh1]);
    // rounded up so that the FP32 factor never falls below the FP64 one
    sp.Qe = std::nextafter((float)std::max(qe, sp.Q), std::numeric_limits<float>::infinity());
    p->Q[(size_t)sp.sh0 * p->nshell + sp.sh1] = sp.Q;
    p->Q[(size_t)sp.sh1 * p->nshell + sp.sh0] = sp.Q;
    p->Qe[(size_t)sp.sh0 * p->nshell + sp.sh1] = (double)sp.Qe;
    p->Qe[(size_t)sp.sh1 * p->nshell + sp.sh0] = (double)sp.Qe;
  }
  PLAN_TRY(cudaMemcpyAsync(p->d_pairs_all, p->pairs_all.data(), sizeof(ShellPair) * npair, cudaMemcpyHostToDevice, st));

  // ---- kept pairs: Q > tau, still grouped by type and sorted by depth
  std::vector<ShellPair> kept;
  for (int X = 0; X < ERI_NPAIRTYPE; ++X) {
    p->type_off[X] = (int)kept.size();
    for (int k = 0; k < p->type_cnt_all[X]; ++k) {
      const ShellPair& sp = p->pairs_all[p->type_off_all[X] + k];
      if (sp.Q > p->opts.screen_thresh) {
        kept.push_back(sp);
        p->type_maxprim[X] = std::max(p->type_maxprim[X], sp.nprim);
      }
    }
    p->type_cnt[X] = (int)kept.size() - p->type_off[X];
  }
  p->npairs_kept = (int)kept.size();
  if (!kept.empty())
    PLAN_TRY(cudaMemcpyAsync(p->d_pairs, kept.data(), sizeof(ShellPair) * kept.size(), cudaMemcpyHostToDevice, st));
  PLAN_TRY(cudaStreamSynchronize(st));
#undef PLAN_TRY
  {
    // eri_jk's scratch, task lists and tile counts, sized now from the plan alone
    std::vector<Launch> launches;
    size_t need, maxnt, tiles;
    if ((s = size_jk_buffers(p, &launches, &need, &maxnt, &tiles)) != ERI_OK) return cleanup(s);
  }
  *out = p;
  return ERI_OK;
}

eri_status eri_jk(eri_plan* p, const double* D, int nD, double* J, double* K, int flags, void* cuda_stream) {
  g_err.clear();
  eri_status s = check_jk_args(p, D, nD, J, K, flags);
  if (s != ERI_OK) return s;
  std::vector<Launch> launches;
  size_t need, maxnt, tiles;
  if ((s = size_jk_buffers(p, &launches, &need, &maxnt, &tiles)) != ERI_OK) return s;
  if (p->opts.check_symmetric && (s = check_density_device(p, D, nD, (cudaStream_t)cuda_stream)) != ERI_OK) return s;
  return run_jk(p, launches, D, nD, J, K, flags & 3, (cudaStream_t)cuda_stream, p->d_scratch, true, true, 2, maxnt,
                tiles, need);
}

eri_status eri_jk_grad(eri_plan* p, const double* D, double* gJ, double* gK, void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(ERI_ERR_ARG, "plan is NULL");
  if (!D || !gJ || !gK) return fail(ERI_ERR_ARG, "D, gJ and gK must be non-NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  struct GL { int X, Y, ts, grid, smem; long long nt; };
  std::vector<GL> ls;
  size_t need = 0, maxnt = 1;
  for (int X = 0; X < ERI_NPAIRTYPE; ++X) {
    if (!p->type_cnt[X]) continue;
    for (int Y = 0; Y <= X; ++Y) {
      if (!p->type_cnt[Y]) continue;
      const long long nx = p->type_cnt[X], ny = p->type_cnt[Y];
      const long long nt = (X == Y) ? nx * (nx + 1) / 2 : nx * ny;
      if ((unsigned long long)nt > 0xffffffffULL) return fail(ERI_ERR_ARG, "class task space above 2^32");
      const GradDesc& g = p->dev->gclasses[X][Y];
      GL l{X, Y, p->dev->gts[X][Y], 0, 0, nt};
      const int tpb = 128 / l.ts;
      l.smem = (int)(sizeof(double) * (size_t)g.team_doubles * tpb);
      if (l.smem > 200 * 1024)
        return fail(ERI_ERR_ARG, "gradient class (%d%d|%d%d) needs %d bytes of shared memory", g.la, g.lb, g.lc, g.ld, l.smem);
      int bps = 0;
      CUDA_TRY(erik_grad_blocks_per_sm(l.ts, l.smem, &bps));
      if (bps < 1) bps = 1;
      l.grid = (int)std::max(1LL, std::min((long long)p->dev->sms * bps, (nt + tpb - 1) / tpb));
      need = std::max(need, (size_t)l.grid * tpb * (size_t)g.scratch_per_team);
      maxnt = std::max(maxnt, (size_t)nt);
      ls.push_back(l);
    }
  }
  eri_status s;
  // two streams, as in eri_jk: each with its own half of scratch, task lists and tile counts
  need = (need + 31) & ~(size_t)31;
  maxnt = (maxnt + 31) & ~(size_t)31;
  const size_t tiles = 2 * ((maxnt + 1023) / 1024 + 1);
  if ((s = ensure_scratch(p, 2 * need)) != ERI_OK) return s;
  if ((s = ensure_buf(&p->d_tlist, &p->tlist_cap, 2 * maxnt)) != ERI_OK) return s;
  if ((s = ensure_buf(&p->d_tiles, &p->tiles_cap, 2 * tiles)) != ERI_OK) return s;
  if (!p->d_gstats) CUDA_TRY(cudaMalloc(&p->d_gstats, sizeof(unsigned long long) * 2));
  if (!p->side) {
    CUDA_TRY(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  }
  const cudaStream_t ss[2] = {st, p->side};
  CUDA_TRY(cudaMemsetAsync(gJ, 0, sizeof(double) * 3 * p->natm, st));
  CUDA_TRY(cudaMemsetAsync(gK, 0, sizeof(double) * 3 * p->natm, st));
  CUDA_TRY(cudaMemsetAsync(p->d_gstats, 0, sizeof(unsigned long long) * 2, st));
  CUDA_TRY(erik_launch_dmax(D, 1, p->nbf, p->nshell, p->d_sh_bf0, p->d_sh_n, p->d_Dmax, st));
  CUDA_TRY(cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned long long) * 256, st));
  CUDA_TRY(cudaMemsetAsync(p->d_tcount, 0, sizeof(unsigned long long) * 2 * 256, st));
  CUDA_TRY(cudaEventRecord(p->ev_fork, st));
  CUDA_TRY(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  int li = 0;
  for (const GL& l : ls) {
    const GradDesc& g = p->dev->gclasses[l.X][l.Y];
    const int sidx = li & 1;
    const cudaStream_t sl = ss[sidx];
    unsigned* tlist_l = p->d_tlist + (size_t)sidx * maxnt;
    unsigned* tiles_l = p->d_tiles + (size_t)sidx * tiles;
    KernelArgs a = base_args(p, l.X, l.Y);
    const int N = g.nroots;
    a.rys_coef = p->dev->rys_coef + RYS_COEF_OFFSET[N];
    a.rys_au = p->dev->rys_au + RYS_ASYM_OFFSET[N];
    a.rys_aw = p->dev->rys_aw + RYS_ASYM_OFFSET[N];
    a.rys_tcut = RYS_TCUT[N];
    a.rys_tcut_d = (double)RYS_TCUT[N];
    a.pairs = p->d_pairs;
    a.bra0 = p->type_off[l.X];
    a.nbra = p->type_cnt[l.X];
    a.ket0 = p->type_off[l.Y];
    a.nket = p->type_cnt[l.Y];
    a.tri = (l.X == l.Y);
    a.ntask = l.nt;
    a.Dmax = p->d_Dmax;
    a.tau = p->opts.screen_thresh;
    a.prec_sel = 0;
    a.D = D;
    a.nD = 1;
    a.want = 3;
    a.mode = KMODE_JK;
    a.counter = p->d_counters + li;
    a.scratch = p->d_scratch + (size_t)sidx * need;
    a.stats = p->d_gstats;
    unsigned long long* cnt = p->d_tcount + 2 * li;
    CUDA_TRY(erik_launch_compact(&a, tlist_l, (unsigned long long)l.nt, cnt, tiles_l, 0, sl));
    a.tlist = tlist_l;
    a.list_cap = (unsigned long long)l.nt;
    a.from_back = 0;
    a.tcount = cnt;
    GradArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.k = a;
    ga.g = g;
    ga.sh_atom = p->d_sh_atom;
    ga.gJ = gJ;
    ga.gK = gK;
    CUDA_TRY(erik_launch_grad(l.ts, &ga, l.grid, l.smem, sl));
    ++li;
  }
  CUDA_TRY(cudaEventRecord(p->ev_join, p->side));
  CUDA_TRY(cudaStreamWaitEvent(st, p->ev_join, 0));
  p->grad_stream = st;
  return ERI_OK;
}

eri_status eri_grad_stats(eri_plan* p, long long* quartets, long long* prim_quartets) {
  g_err.clear();
  if (!p || !quartets || !prim_quartets) return fail(ERI_ERR_ARG, "NULL argument");
  unsigned long long h[2] = {0, 0};
  if (p->d_gstats) {
    CUDA_TRY(cudaStreamSynchronize(p->grad_stream));
    CUDA_TRY(cudaMemcpy(h, p->d_gstats, sizeof(h), cudaMemcpyDeviceToHost));
  }
  *quartets = (long long)h[0];
  *prim_quartets = (long long)h[1];
  return ERI_OK;
}

eri_status eri_jk_host(eri_plan* p, const double* D, int nD, double* J, double* K, int flags, void* cuda_stream) {
  g_err.clear();
  if (!p) return fail(ERI_ERR_ARG, "plan is NULL");
  if (!D) return fail(ERI_ERR_ARG, "D is NULL");
  if (nD < 1 || nD > p->opts.max_nd) return fail(ERI_ERR_ARG, "nD = %d outside [1, %d]", nD, p->opts.max_nd);
  const int want = flags & 3;
  if (want == 0) return fail(ERI_ERR_ARG, "flags request neither J nor K");
  if ((want & 1) && !J) return fail(ERI_ERR_ARG, "J requested but NULL");
  if ((want & 2) && !K) return fail(ERI_ERR_ARG, "K requested but NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t mat = (size_t)nD * p->nbf * p->nbf;
  eri_status s;
  if (p->opts.check_symmetric && (s = eri_check_density(D, nD, p->nbf)) != ERI_OK) return s;
  if ((s = ensure_buf(&p->d_host_io, &p->host_io_cap, 3 * mat)) != ERI_OK) return s;
  double* dD = p->d_host_io;
  double* dJ = dD + mat;
  double* dK = dJ + mat;
  CUDA_TRY(cudaMemcpyAsync(dD, D, sizeof(double) * mat, cudaMemcpyHostToDevice, st));
  if ((s = eri_jk(p, dD, nD, dJ, dK, want, st)) != ERI_OK) return s;
  if (want & 1) CUDA_TRY(cudaMemcpyAsync(J, dJ, sizeof(double) * mat, cudaMemcpyDeviceToHost, st));
  if (want & 2) CUDA_TRY(cudaMemcpyAsync(K, dK, sizeof(double) * mat, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return ERI_OK;
}

eri_status eri_shell_quartet(eri_plan* p, int i, int j, int k, int l, double* out) {
  g_err.clear();
  if (!p || !out) return fail(ERI_ERR_ARG, "plan or out is NULL");
  const int ns = p->nshell;
  if (i < 0 || j < 0 || k < 0 || l < 0 || i >= ns || j >= ns || k >= ns || l >= ns)
    return fail(ERI_ERR_ARG, "shell index outside [0, %d)", ns);
  const int pb = p->pair_index[(size_t)i * ns + j], pk = p->pair_index[(size_t)k * ns + l];
  const ShellPair& B = p->pairs_all[pb];
  const ShellPair& Kt = p->pairs_all[pk];
  const int X = B.ptype, Y = Kt.ptype;
  const ClassDesc& c = p->dev->classes[X][Y];
  const size_t nblk = (size_t)c.na * c.nb * c.nc * c.nd;
  std::vector<int> tasks = {pb, pk};
  std::vector<long long> offs = {0};
  cudaStream_t st = nullptr;
  eri_status s = run_explicit(p, X, Y, KMODE_BLOCK, tasks, offs, nblk, st);
  if (s != ERI_OK) return s;
  std::vector<double> blk(nblk);
  CUDA_TRY(cudaMemcpyAsync(blk.data(), p->d_out, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  // canonical block [a(sh0 of bra)][b(sh1)][c(sh0 of ket)][d(sh1)] -> requested (i j | k l)
  const bool sw_b = (B.sh0 != i);
  const bool sw_k = (Kt.sh0 != k);
  const int ni = ncart(p->sh_l[i]), nj = ncart(p->sh_l[j]), nk = ncart(p->sh_l[k]), nl = ncart(p->sh_l[l]);
  for (int x = 0; x < ni; ++x)
    for (int y = 0; y < nj; ++y)
      for (int z = 0; z < nk; ++z)
        for (int w = 0; w < nl; ++w) {
          const int a = sw_b ? y : x, b = sw_b ? x : y;
          const int cc = sw_k ? w : z, d = sw_k ? z : w;
          out[(((size_t)x * nj + y) * nk + z) * nl + w] = blk[(((size_t)a * c.nb + b) * c.nc + cc) * c.nd + d];
        }
  return ERI_OK;
}

eri_status eri_schwarz(const eri_plan* p, double* Q) {
  g_err.clear();
  if (!p || !Q) return fail(ERI_ERR_ARG, "plan or Q is NULL");
  memcpy(Q, p->Q.data(), sizeof(double) * p->Q.size());
  return ERI_OK;
}

eri_status eri_schwarz_transfer(const eri_plan* p, double* Qe) {
  g_err.clear();
  if (!p || !Qe) return fail(ERI_ERR_ARG, "plan or Qe is NULL");
  memcpy(Qe, p->Qe.data(), sizeof(double) * p->Qe.size());
  return ERI_OK;
}

eri_status eri_rys_roots(int N, int n, const double* T, double* u, double* w) {
  g_err.clear();
  if (N < 1 || N > RYS_NMAX) return fail(ERI_ERR_ARG, "N = %d outside [1, 9]", N);
  if (n < 0 || (n > 0 && (!T || !u || !w))) return fail(ERI_ERR_ARG, "bad sizes or NULL arrays");
  for (int t = 0; t < n; ++t)
    if (!(T[t] >= 0) || !std::isfinite(T[t])) return fail(ERI_ERR_ARG, "T[%d] must be finite and >= 0", t);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(ERI_ERR_NO_DEVICE, "no CUDA device is visible");
  }
  if (n == 0) return ERI_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  DeviceState* ds = nullptr;
  eri_status s = device_init(dev, &ds);
  if (s != ERI_OK) return s;
  double *dT = nullptr, *du = nullptr, *dw = nullptr;
  CUDA_TRY(cudaMalloc(&dT, sizeof(double) * n));
  if (cudaMalloc(&du, sizeof(double) * n * N) != cudaSuccess || cudaMalloc(&dw, sizeof(double) * n * N) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dT); cudaFree(du); cudaFree(dw);
    return fail(ERI_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpy(dT, T, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = (cudaError_t)erik_launch_rys(N, n, dT, du, dw, ds->rys_coef + RYS_COEF_OFFSET[N], ds->rys_au + RYS_ASYM_OFFSET[N],
                                     ds->rys_aw + RYS_ASYM_OFFSET[N], RYS_TCUT[N], nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(u, du, sizeof(double) * n * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(w, dw, sizeof(double) * n * N, cudaMemcpyDeviceToHost);
  cudaFree(dT); cudaFree(du); cudaFree(dw);
  if (e != cudaSuccess) return fail(ERI_ERR_CUDA, "eri_rys_roots: %s", cudaGetErrorString(e));
  return ERI_OK;
}

eri_status eri_flop_stats(eri_plan* p, eri_stats* out) {
  g_err.clear();
  if (!p || !out) return fail(ERI_ERR_ARG, "plan or out is NULL");
  CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  std::vector<unsigned long long> st(4 * 256);
  CUDA_TRY(cudaMemcpy(st.data(), p->d_stats, sizeof(unsigned long long) * 4 * 256, cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->quartets_candidate = p->last_candidates;
  for (int f = 0; f < 2; ++f)
    for (int X = 0; X < ERI_NPAIRTYPE; ++X)
      for (int Y = 0; Y < ERI_NPAIRTYPE; ++Y) {
        const size_t k = 2 * (256 * f + X * ERI_NPAIRTYPE + Y);
        const unsigned long long q = st[k], pq = st[k + 1];
        out->quartets_computed += (long long)q;
        out->prim_quartets += (long long)pq;
        if (f) out->quartets_fp32 += (long long)q;
        double a64, a32, q64, q32;
        class_model_flops2(p->dev->classes[X][Y], p->last_nD, p->last_want, f, &a64, &a32, &q64, &q32);
        out->model_flops += (a64 + a32) * (double)pq + (q64 + q32) * (double)q;
        out->model_flops_fp32 += a32 * (double)pq + q32 * (double)q;
      }
  out->npairs_total = (int)p->pairs_all.size();
  out->npairs_kept = p->npairs_kept;
  out->nclasses_launched = p->last_nclasses;
  unsigned err = 0;
  CUDA_TRY(cudaMemcpy(&err, p->d_err, sizeof(err), cudaMemcpyDeviceToHost));
  out->device_status = (int)err;
  if (err) return fail(ERI_ERR_TIMEOUT, "a bounded device wait of the plan's kernels gave up");
  return ERI_OK;
}

eri_status eri_check_density(const double* D, int nD, int nbf) {
  g_err.clear();
  if (!D || nD < 1 || nbf < 1) return fail(ERI_ERR_ARG, "D is NULL or nD, nbf < 1");
  double asym = 0.0, mx = 0.0;
  for (int x = 0; x < nD; ++x) {
    const double* Dx = D + (size_t)x * nbf * nbf;
    for (int i = 0; i < nbf; ++i)
      for (int j = 0; j < nbf; ++j) {
        const double a = Dx[(size_t)i * nbf + j];
        if (!std::isfinite(a)) return fail(ERI_ERR_ARG, "D has a non-finite element");
        mx = std::max(mx, std::fabs(a));
        if (j > i) asym = std::max(asym, std::fabs(a - Dx[(size_t)j * nbf + i]));
      }
  }
  if (!(asym <= 1e-12 * mx))
    return fail(ERI_ERR_ARG, "D is not symmetric: max|D_ij - D_ji| = %.3e, max|D| = %.3e", asym, mx);
  return ERI_OK;
}

eri_status eri_set_profiling(eri_plan* p, int enable) {
  g_err.clear();
  if (!p) return fail(ERI_ERR_ARG, "plan is NULL");
  p->profiling = enable != 0;
  return ERI_OK;
}

eri_status eri_launch_records(eri_plan* p, eri_launch_record* out, int cap, int* n) {
  g_err.clear();
  if (!p || !n || (cap > 0 && !out)) return fail(ERI_ERR_ARG, "NULL argument");
  if (!p->profiling) return fail(ERI_ERR_ARG, "profiling is off for this plan");
  CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  const int nl = (int)p->last_launch_xy.size();
  *n = nl;
  if (nl == 0) return ERI_OK;
  std::vector<unsigned long long> st(4 * 256);
  CUDA_TRY(cudaMemcpy(st.data(), p->d_stats, sizeof(unsigned long long) * 4 * 256, cudaMemcpyDeviceToHost));
  for (int i = 0; i < nl && i < cap; ++i) {
    const int xy = p->last_launch_xy[i];
    const int f = p->last_launch_fp32[i];
    const ClassDesc& c = p->dev->classes[xy / ERI_NPAIRTYPE][xy % ERI_NPAIRTYPE];
    eri_launch_record& r = out[i];
    r.la = c.la; r.lb = c.lb; r.lc = c.lc; r.ld = c.ld;
    r.team_size = p->last_launch_ts[i];
    r.grid = p->last_launch_grid[i];
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, p->events[2 * i], p->events[2 * i + 1]));
    r.ms = ms;
    r.quartets = (long long)st[2 * (256 * f + xy)];
    r.prim_quartets = (long long)st[2 * (256 * f + xy) + 1];
    double a64, a32, q64, q32;
    class_model_flops2(c, p->last_nD, p->last_want, f, &a64, &a32, &q64, &q32);
    r.model_flops = (a64 + a32) * (double)r.prim_quartets + (q64 + q32) * (double)r.quartets;
    r.model_flops_fp32 = a32 * (double)r.prim_quartets + q32 * (double)r.quartets;
    r.fp32 = f;
    r.specialised = p->last_launch_small[i];
    r.shared_products = (!f && !r.specialised && c.xy) ? 1 : 0;
    r.compiled_class = (!f && !r.specialised && erik_class_spec_available(r.team_size, c.la, c.lb, c.lc, c.ld)) ? 1 : 0;
    r.quartet_split = p->last_launch_qsplit[i];
    r.listed = p->last_launch_listed[i];
  }
  return ERI_OK;
}

// Host self-check of the per-class tables (no GPU needed): every [e0|f0] value of every
// J/K and gradient class appears exactly once among the slots, each slot's 2D-table
// offsets belong to its value, a slot that does not start a group shares its group's
// I_x I_y offsets, every pass starts a group, offsets stay inside the tables and the team
// regions fit in shared memory.
eri_status eri_check_class_tables(int* nclasses, int* problems) {
  g_err.clear();
  if (!nclasses || !problems) return fail(ERI_ERR_ARG, "NULL output");
  const CartTab& ct = cart();
  int bad = 0, n = 0;
  auto check_lp = [&](const uint32_t* outi, const uint32_t* dst, const uint32_t* gm, int T, int nslot, int nval,
                      auto&& expect) {
    const int Ls = nslot / T;
    if (Ls * T != nslot) ++bad;
    std::vector<int> seen(nval, 0);
    for (int p = 0; p < (Ls + 31) / 32; ++p)
      if (!(gm[p] & 1u)) ++bad;
    for (int ln = 0; ln < T; ++ln) {
      uint32_t cur = 0xffffffffu;
      for (int k = 0; k < Ls; ++k) {
        const int o = (k / 32) * T * 32 + (k % 32) * T + ln;
        const uint32_t q = outi[o];
        if ((gm[k / 32] >> (k % 32)) & 1u) cur = q & 0xffffu;
        if (q >> 31) continue;
        if ((q & 0xffffu) != cur) ++bad;
        if ((int)dst[o] < 0 || (int)dst[o] >= nval) { ++bad; continue; }
        if (seen[dst[o]]++) ++bad;
        if (!expect((int)dst[o], q)) ++bad;
      }
    }
    for (int v = 0; v < nval; ++v)
      if (seen[v] != 1) ++bad;
  };
  for (int X = 0; X < ERI_NPAIRTYPE; ++X)
    for (int Y = 0; Y < ERI_NPAIRTYPE; ++Y) {
      int la, lb, lc, ld, ts;
      ptype_ls(X, &la, &lb);
      ptype_ls(Y, &lc, &ld);
      {
        ClassDesc c;
        std::vector<uint32_t> idx;
        make_class(la, lb, lc, ld, &c, &ts, &idx);
        ++n;
        const int L1 = c.Lf + 1;
        auto word = [&](int v) {
          const int e = c.e_base + v / c.nf, f = c.f_base + v % c.nf;
          return (uint32_t)(ct.lx[e] * L1 + ct.lx[f]) | ((uint32_t)(ct.ly[e] * L1 + ct.ly[f]) << 8) |
                 ((uint32_t)(ct.lz[e] * L1 + ct.lz[f]) << 16);
        };
        check_lp(idx.data(), idx.data() + c.dst_off, idx.data() + c.gmask_off, ts, c.nslot, c.nout,
                 [&](int v, uint32_t q) { return (q & 0xffffffu) == word(v); });
        const int tpb = 128 / ts;
        if (ts > 1 && (8L * c.team_doubles * tpb > 200 * 1024 || 8L * c.team_doubles_f32 * tpb > 200 * 1024)) ++bad;
        if (c.xy) {
          if (8L * c.team_doubles_xy * tpb > 200 * 1024) ++bad;
          const uint32_t* xo = idx.data() + c.xy_outidx_off;
          const uint32_t* xd = idx.data() + c.xy_dst_off;
          const uint32_t* xt = idx.data() + c.xytab_off;
          const uint32_t* pi = idx.data() + c.pass_off;
          std::vector<int> seen(c.nout, 0);
          for (int o = 0; o < c.nout; ++o) {
            const int p = o / (32 * ts);
            const uint32_t q = xo[o] & 0xffffu;
            if (q >= pi[2 * p + 1] || (int)pi[2 * p + 1] > c.xymax) { ++bad; continue; }
            const uint32_t w = word((int)xd[o]);
            if (((xt[pi[2 * p] + q]) & 0xffffu) != (w & 0xffffu) || (xo[o] & 0xff0000u) != (w & 0xff0000u)) ++bad;
            if (seen[xd[o]]++) ++bad;
          }
        }
      }
      {
        GradDesc g;
        std::vector<uint32_t> idx;
        make_grad_class(la, lb, lc, ld, &g, &ts, &idx);
        ++n;
        const int L1 = g.Lf2 + 1, NnI = g.nroots * g.nI;
        auto expect = [&](int v, uint32_t q) {
          int set = 0;
          while (set < 3 && v >= g.s_off[set + 1]) ++set;
          const int r = v - g.s_off[set], ie = r / g.s_nf[set], jf = r % g.s_nf[set];
          const int e = cart_below(g.s_elo[set]) + ie, f = cart_below(g.s_flo[set]) + jf;
          return (q & 0xffu) == (uint32_t)(ct.lx[e] * L1 + ct.lx[f]) &&
                 ((q >> 8) & 0xffu) == (uint32_t)(ct.ly[e] * L1 + ct.ly[f]) &&
                 ((q >> 16) & 0xfffu) == (uint32_t)(set * NnI + ct.lz[e] * L1 + ct.lz[f]);
        };
        check_lp(idx.data(), idx.data() + g.dst_off, idx.data() + g.gmask_off, ts, g.nslot, g.nout, expect);
        if (ts > 1 && 8L * g.team_doubles * (128 / ts) > 200 * 1024) ++bad;
      }
    }
  *nclasses = n;
  *problems = bad;
  return ERI_OK;
}

eri_status eri_probe_fma_peak(double* fp64_tflops, double* fp32_tflops) {
  g_err.clear();
  if (!fp64_tflops || !fp32_tflops) return fail(ERI_ERR_ARG, "NULL output");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(ERI_ERR_NO_DEVICE, "no CUDA device is visible");
  }
  CUDA_TRY(erik_probe_fma(fp64_tflops, fp32_tflops));
  return ERI_OK;
}

}  // extern "C"

// ================================================================= internal hooks for other translation units
extern "C" __attribute__((visibility("hidden"))) void eri_host_normalise(int nshell, const int* l, const int* nprim,
                                                                          const int* off, const double* exps,
                                                                          const double* raw, double* out) {
  int n = 0;
  for (int s = 0; s < nshell; ++s) n = std::max(n, off[s] + nprim[s]);
  std::vector<double> tmp(raw, raw + n);
  normalise(nshell, l, nprim, off, exps, raw, tmp);
  std::copy(tmp.begin(), tmp.end(), out);
}

// Record a failure for eri_last_error() from another translation unit.
extern "C" __attribute__((visibility("hidden"))) eri_status eri_internal_fail(eri_status s, const char* msg) {
  return fail(s, "%s", msg);
}

// The J/K build of eri_jk with caller-provided team scratch of a fixed size: nothing is
// allocated.  Each class launch uses as many blocks as its scratch need allows (at most the
// occupancy-limited grid); a class whose single block needs more than scratch_doubles is
// rejected with ERI_ERR_ARG before anything is launched.
extern "C" __attribute__((visibility("hidden"))) eri_status eri_internal_jk_fixed_scratch(
    eri_plan* p, const double* D, int nD, double* J, double* K, int flags, void* cuda_stream, double* scratch,
    size_t scratch_doubles) {
  g_err.clear();
  eri_status s = check_jk_args(p, D, nD, J, K, flags);
  if (s != ERI_OK) return s;
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != p->device) return fail(ERI_ERR_ARG, "the plan belongs to device %d but device %d is current", p->device, cur);
  std::vector<Launch> launches;
  if ((s = plan_launches(p, scratch_doubles, &launches)) != ERI_OK) return s;
  return run_jk(p, launches, D, nD, J, K, flags & 3, (cudaStream_t)cuda_stream, scratch, false, false);
}

// ================================================================= batched J/K across plans
struct eri_batch {
  int device = 0;
  JobDesc* d_jobs = nullptr;
  size_t jobs_cap = 0;
  unsigned long long* d_blist = nullptr;
  size_t blist_cap = 0;
  unsigned* d_tiles = nullptr;
  size_t tiles_cap = 0;
  unsigned long long* d_small = nullptr;     // per stream: counts[2], base[2]
  unsigned long long* d_cursor = nullptr;    // [256][2]
  unsigned long long* d_counter = nullptr;   // [512]
  unsigned long long* d_stats = nullptr;     // [2][256][2]
  double* d_scratch = nullptr;
  size_t scratch_doubles = 0;
  cudaStream_t last_stream = nullptr;
  long long last_quartets = 0;
  int last_launches = 0;
  // second stream: classes alternate between the caller's stream and this one, each with
  // its own half of the merged lists, tile counts, small counters and scratch
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_done = nullptr;             // end of the last call on its stream
  bool called = false;
};

namespace {
// Grow a batch buffer without synchronising the host or the device: the old buffer is freed
// and the new one allocated in stream order on the call's stream, after the previous call's
// work (ev_done); capacities grow by half again so that a growing job mix regrows rarely.
template <typename T>
eri_status ensure_batch_buf(eri_batch* b, T** ptr, size_t* cap, size_t n, cudaStream_t st) {
  if (n <= *cap) return ERI_OK;
  if (b->called) CUDA_TRY(cudaStreamWaitEvent(st, b->ev_done, 0));
  if (*ptr) {
    CUDA_TRY(cudaFreeAsync(*ptr, st));
    *ptr = nullptr;
    *cap = 0;
  }
  const size_t grow = std::max(n, n + n / 2);
  cudaError_t e = cudaMallocAsync((void**)ptr, sizeof(T) * grow, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(ERI_ERR_OOM, "stream-ordered allocation of %zu bytes failed", sizeof(T) * grow);
  }
  *cap = grow;
  return ERI_OK;
}
}  // namespace

extern "C" {

eri_status eri_batch_create(eri_batch** out) {
  g_err.clear();
  if (!out) return fail(ERI_ERR_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(ERI_ERR_NO_DEVICE, "no CUDA device is visible");
  }
  eri_batch* b = new (std::nothrow) eri_batch();
  if (!b) return fail(ERI_ERR_OOM, "host allocation failed");
  cudaGetDevice(&b->device);
  if (cudaMalloc(&b->d_small, sizeof(unsigned long long) * 8) != cudaSuccess ||
      cudaMalloc(&b->d_cursor, sizeof(unsigned long long) * 2 * 256) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(unsigned long long) * 512) != cudaSuccess ||
      cudaMalloc(&b->d_stats, sizeof(unsigned long long) * 4 * 256) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_small); cudaFree(b->d_cursor); cudaFree(b->d_counter); cudaFree(b->d_stats);
    delete b;
    return fail(ERI_ERR_OOM, "device allocation failed in eri_batch_create");
  }
  *out = b;
  return ERI_OK;
}

eri_status eri_batch_destroy(eri_batch* b) {
  if (!b) return ERI_OK;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  void* bufs[] = {b->d_jobs, b->d_blist, b->d_tiles, b->d_small, b->d_cursor, b->d_counter, b->d_stats, b->d_scratch};
  for (void* x : bufs)
    if (x) cudaFree(x);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  delete b;
  return ERI_OK;
}

eri_status eri_jk_batch(eri_batch* b, int njobs, eri_plan* const* plans, const double* const* D, const int* nD,
                        double* const* J, double* const* K, const int* flags, void* cuda_stream) {
  g_err.clear();
  if (!b || njobs < 1 || !plans || !D || !nD || !J || !K || !flags) return fail(ERI_ERR_ARG, "NULL argument or njobs < 1");
  if (njobs > (1 << 24)) return fail(ERI_ERR_ARG, "too many jobs");
  eri_status s;
  for (int j = 0; j < njobs; ++j) {
    if ((s = check_jk_args(plans[j], D[j], nD[j], J[j], K[j], flags[j])) != ERI_OK) return s;
    if (plans[j]->device != b->device) return fail(ERI_ERR_ARG, "job %d's plan is on another device", j);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  eri_plan* p0 = plans[0];
  // ---- job descriptors
  std::vector<JobDesc> jobs(njobs);
  for (int j = 0; j < njobs; ++j) {
    eri_plan* p = plans[j];
    JobDesc& jd = jobs[j];
    memset(&jd, 0, sizeof(jd));
    jd.pairs = p->d_pairs;
    jd.prims = p->d_prims;
    jd.primsf = p->d_primsf;
    jd.D = D[j];
    jd.J = J[j];
    jd.K = K[j];
    jd.nbf = p->nbf;
    jd.nD = nD[j];
    jd.want = flags[j] & 3;
    for (int t = 0; t < ERI_NPAIRTYPE; ++t) {
      jd.type_off[t] = p->type_off[t];
      jd.type_cnt[t] = p->type_cnt[t];
    }
  }
  if (!b->side) {
    CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming));
  }
  // the previous call's kernels may still read the job table and lists: this call's writes
  // to them are ordered after that call's end
  if (b->called) CUDA_TRY(cudaStreamWaitEvent(st, b->ev_done, 0));
  if ((s = ensure_batch_buf(b, &b->d_jobs, &b->jobs_cap, (size_t)njobs, st)) != ERI_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(b->d_jobs, jobs.data(), sizeof(JobDesc) * njobs, cudaMemcpyHostToDevice, st));
  // ---- classes present in any job, their merged capacities and launch shapes
  struct BL { int X, Y; long long total; long long maxnt; int any_fp32, maxq; };
  std::vector<BL> cls;
  for (int X = 0; X < ERI_NPAIRTYPE; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      long long tot = 0, mx = 0;
      int any32 = 0, maxq = 1;
      for (int j = 0; j < njobs; ++j) {
        const long long nx = plans[j]->type_cnt[X], ny = plans[j]->type_cnt[Y];
        if (!nx || !ny) continue;
        maxq = std::max(maxq, plans[j]->type_maxprim[X] * plans[j]->type_maxprim[Y]);
        const long long nt = (X == Y) ? nx * (nx + 1) / 2 : nx * ny;
        if ((unsigned long long)nt > 0xffffffffULL) return fail(ERI_ERR_ARG, "job %d has more than 2^32 tasks in a class", j);
        tot += nt;
        mx = std::max(mx, nt);
        if (plans[j]->opts.precision == ERI_MIXED && fp32_pays(plans[j], X, Y, nt)) any32 = 1;
      }
      if (tot) cls.push_back({X, Y, tot, mx, any32, maxq});
    }
  size_t cap = 1, tcap = 2, need = 0;
  struct LL { int X, Y, fp32, grid, smem, ts, small; long long total; int qsplit; };
  std::vector<LL> launches;
  for (const BL& c : cls) {
    cap = std::max(cap, (size_t)c.total);
    tcap = std::max(tcap, (size_t)(2 * ((c.maxnt + 1023) / 1024 + 1)));
    for (int fp32 = 0; fp32 < (c.any_fp32 ? 2 : 1); ++fp32) {
      LL l{c.X, c.Y, fp32, 0, 0, 0, 0, c.total, 1};
      const ClassDesc& cd = p0->dev->classes[c.X][c.Y];
      // as in eri_jk: a class whose merged quartets cannot fill the grid splits them into
      // ranges of primitive quartets (a full grid decides the split, the split the grid)
      if ((s = launch_shape(p0, c.X, c.Y, fp32, 1LL << 40, &l.grid, &l.smem, &l.ts)) != ERI_OK) return s;
      l.qsplit = choose_qsplit(c.total, (long long)l.grid * (128 / l.ts), c.maxq,
                               fp32 ? cd.bp : (cd.xy ? cd.bp_xy : cd.bp));
      if ((s = launch_shape(p0, c.X, c.Y, fp32, c.total * l.qsplit, &l.grid, &l.smem, &l.ts)) != ERI_OK) return s;
      if ((fp32 || l.ts == 1) && erik_small_available(cd.la, cd.lb, cd.lc, cd.ld, fp32)) {
        l.ts = 1;
        int bps = 0;
        CUDA_TRY(erik_small_blocks_per_sm(cd.la, cd.lb, cd.lc, cd.ld, fp32, &bps));
        const long long full = (long long)p0->dev->sms * std::max(bps, 1);
        l.qsplit = choose_qsplit(c.total, full * 128, c.maxq, 2);
        l.grid = (int)std::max(1LL, std::min(full, (c.total * l.qsplit + 127) / 128));
        l.smem = 0;
        l.small = 1;
      }
      need = std::max(need, (size_t)l.grid * (size_t)(128 / l.ts) * (size_t)cd.scratch_per_team);
      launches.push_back(l);
    }
  }
  cap = (cap + 31) & ~(size_t)31;
  tcap = (tcap + 31) & ~(size_t)31;
  need = (need + 31) & ~(size_t)31;
  // per-stream halves sized from the largest request seen; when they grow they are
  // reallocated with stream-ordered frees and allocations (no host or device synchronisation)
  if (cap > b->blist_cap / 2 && (s = ensure_batch_buf(b, &b->d_blist, &b->blist_cap, 2 * cap, st)) != ERI_OK) return s;
  if (tcap > b->tiles_cap / 2 && (s = ensure_batch_buf(b, &b->d_tiles, &b->tiles_cap, 2 * tcap, st)) != ERI_OK) return s;
  if (need > b->scratch_doubles / 2 &&
      (s = ensure_batch_buf(b, &b->d_scratch, &b->scratch_doubles, 2 * need, st)) != ERI_OK)
    return s;
  cap = b->blist_cap / 2;
  tcap = b->tiles_cap / 2;
  need = b->scratch_doubles / 2;
  const cudaStream_t ss[2] = {st, b->side};
  // ---- per job: zero outputs, density block maxima
  for (int j = 0; j < njobs; ++j) {
    eri_plan* p = plans[j];
    const size_t mat = (size_t)nD[j] * p->nbf * p->nbf;
    if (flags[j] & 1) CUDA_TRY(cudaMemsetAsync(J[j], 0, sizeof(double) * mat, st));
    if (flags[j] & 2) CUDA_TRY(cudaMemsetAsync(K[j], 0, sizeof(double) * mat, st));
    CUDA_TRY(erik_launch_dmax(D[j], nD[j], p->nbf, p->nshell, p->d_sh_bf0, p->d_sh_n, p->d_Dmax, st));
  }
  CUDA_TRY(cudaMemsetAsync(b->d_cursor, 0, sizeof(unsigned long long) * 2 * 256, st));
  CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long) * 512, st));
  CUDA_TRY(cudaMemsetAsync(b->d_stats, 0, sizeof(unsigned long long) * 4 * 256, st));
  CUDA_TRY(cudaEventRecord(b->ev_fork, st));
  CUDA_TRY(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
  // ---- per class (alternating streams): merged compaction over jobs, then one launch per
  //      precision
  int li = 0;
  for (size_t ci = 0; ci < cls.size(); ++ci) {
    const BL& c = cls[ci];
    const int sidx = (int)(ci & 1);
    const cudaStream_t sl = ss[sidx];
    unsigned long long* blist_l = b->d_blist + (size_t)sidx * cap;
    unsigned* tiles_l = b->d_tiles + (size_t)sidx * tcap;
    unsigned long long* small_l = b->d_small + 4 * sidx;
    unsigned long long* cursor = b->d_cursor + 2 * ci;
    for (int j = 0; j < njobs; ++j) {
      eri_plan* p = plans[j];
      const long long nx = p->type_cnt[c.X], ny = p->type_cnt[c.Y];
      if (!nx || !ny) continue;
      KernelArgs a = base_args(p, c.X, c.Y);
      a.pairs = p->d_pairs;
      a.bra0 = p->type_off[c.X];
      a.nbra = (int)nx;
      a.ket0 = p->type_off[c.Y];
      a.nket = (int)ny;
      a.tri = (c.X == c.Y);
      a.ntask = (c.X == c.Y) ? nx * (nx + 1) / 2 : nx * ny;
      a.Dmax = p->d_Dmax;
      a.nsh = p->nshell;
      a.tau = p->opts.screen_thresh;
      a.mixed_thr = p->opts.mixed_thresh;
      const bool split = p->opts.precision == ERI_MIXED && fp32_pays(p, c.X, c.Y, a.ntask);
      CUDA_TRY(erik_launch_compact_batched(&a, blist_l, (unsigned long long)c.total, small_l, tiles_l, cursor,
                                           small_l + 2, (unsigned long long)j, split ? 1 : 0, sl));
    }
    for (const LL& l : launches) {
      if (l.X != c.X || l.Y != c.Y) continue;
      KernelArgs a = base_args(p0, c.X, c.Y);
      a.mode = KMODE_JK;
      a.jobs = b->d_jobs;
      a.blist = blist_l;
      a.list_cap = (unsigned long long)c.total;
      a.from_back = l.fp32;
      a.tcount = cursor + l.fp32;
      a.X = c.X;
      a.Y = c.Y;
      a.counter = b->d_counter + li;
      a.scratch = b->d_scratch + (size_t)sidx * need;
      a.qsplit = l.qsplit;
      a.stats = b->d_stats + 2 * (256 * l.fp32 + c.X * ERI_NPAIRTYPE + c.Y);
      if (l.small)
        CUDA_TRY(erik_launch_small(a.c.la, a.c.lb, a.c.lc, a.c.ld, l.fp32, &a, l.grid, sl));
      else
        CUDA_TRY(erik_launch_class(l.ts, l.fp32, &a, l.grid, l.smem, sl));
      ++li;
    }
  }
  CUDA_TRY(cudaEventRecord(b->ev_join, b->side));
  CUDA_TRY(cudaStreamWaitEvent(st, b->ev_join, 0));
  for (int j = 0; j < njobs; ++j) {
    if (flags[j] & 1) CUDA_TRY(erik_launch_symmetrize(J[j], nD[j], plans[j]->nbf, st));
    if (flags[j] & 2) CUDA_TRY(erik_launch_symmetrize(K[j], nD[j], plans[j]->nbf, st));
  }
  CUDA_TRY(cudaEventRecord(b->ev_done, st));
  b->called = true;
  b->last_stream = st;
  b->last_launches = li;
  return ERI_OK;
}

eri_status eri_batch_stats(eri_batch* b, long long* quartets, long long* quartets_fp32, int* launches) {
  g_err.clear();
  if (!b) return fail(ERI_ERR_ARG, "batch is NULL");
  CUDA_TRY(cudaStreamSynchronize(b->last_stream));
  std::vector<unsigned long long> st(4 * 256);
  CUDA_TRY(cudaMemcpy(st.data(), b->d_stats, sizeof(unsigned long long) * 4 * 256, cudaMemcpyDeviceToHost));
  long long q = 0, q32 = 0;
  for (int f = 0; f < 2; ++f)
    for (int k = 0; k < 256; ++k) {
      q += (long long)st[2 * (256 * f + k)];
      if (f) q32 += (long long)st[2 * (256 * f + k)];
    }
  if (quartets) *quartets = q;
  if (quartets_fp32) *quartets_fp32 = q32;
  if (launches) *launches = b->last_launches;
  return ERI_OK;
}

}  // extern "C"
