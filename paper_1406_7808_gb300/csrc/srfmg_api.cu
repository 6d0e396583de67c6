// Host side of the solver: configuration checks, the level / segment plan,
// device workspace, the launch sequence of FMG and SR-FMG, the float64
// defect-correction loop of the mixed-precision mode, and the C ABI declared
// in include/srfmg.h.
//
// Launch sequence of one FMG / SR-FMG solve (Sec. 3 and Sec. 4 of the paper):
//   f hierarchy      f_{k-1} = 8-child average of f_k, every level
//   FMG              coarsest exact solve, then per global level: prolongation,
//                    S^alpha, one FAS V-cycle (Fig. "Full multigrid")
//   SR stages k=1..K per stage, on all segments at once: prolongation onto
//                    Omega^C u Omega^GSR, S^alpha, the down-leg of FASMGVSR
//                    (S^nu1, residual + restriction onto Omega^F, modified tau
//                    right-hand side), the transition-level right-hand side,
//                    the global V-cycle, then the up-leg (corrections onto
//                    Omega^C u Omega^GSR and S^nu2) (Figs. "FMG segmental
//                    refinement", "FAS V-cycle segmental refinement")
//   output           genuine cells of the finest level into u
// Mixed precision (SR_MIXED): that solve runs in float32 storage and
// arithmetic (coarse right-hand sides and the coarsest solve in float64
// arithmetic) inside n_outer passes of float64 defect correction:
//   pass 1: u = S32(f);  pass p > 1: d = f - A u (float64), u += S32(d).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "srfmg.h"
#include "srfmg_internal.cuh"

using namespace srfmg;

namespace {

// ---------------------------------------------------------------------------
// plan

// geometry of one level: its boxes on the host and the device
struct Geom {
  int n = 0;                     // cells per unit length
  int nd[3] = {0, 0, 0};         // cells per dimension of the whole level grid
  int nbox = 0;
  long long slot = 0;            // elements per box (SR levels)
  std::vector<BoxDesc> hboxes;
  BoxDesc* dboxes = nullptr;     // device copy of hboxes
  BoxDesc* dglobal = nullptr;    // device descriptor of the whole level, unpadded
  LevelView view{};
  // totals over the boxes, for the algorithmic work counts of the profiler
  double tot_cells = 0, tot_prolong = 0, tot_restrict = 0, tot_genuine = 0;
};

// a level's arrays in storage type T
template <typename T>
struct Level : Geom {
  T *u = nullptr, *t = nullptr, *rhs = nullptr, *r = nullptr, *rho = nullptr, *d = nullptr,
    *f = nullptr;
};

template <typename T>
struct Hier {
  std::vector<Level<T>> glev;  // global levels, glev[G-1] is level 0
  std::vector<Level<T>> slev;  // SR levels, slev[k], k = 1..K
  // The finest level's boxes cut to what its genuine cells still depend on
  // in the last operations of the solve (final correction and the degree-2
  // post-smoother of the last stage): trim_r has the genuine region grown by
  // one as compute region and grown by two as prolongation range, trim_u the
  // genuine region as compute region (clipped to the full regions).
  Geom trim_r, trim_u;
  // The coarser SR levels j < K cut the same way for the last stage's
  // up-leg, from the cells U_j that the trimmed correction of level j + 1
  // reads: ctrim_u[j] has U_j inside the compute region as compute region
  // (the post-smoother's update) and U_j as prolongation range (the cells
  // of w - t formed); ctrim_r[j] has U_j grown by one as compute region (the
  // residual) and by two as prolongation range (the correction onto level j).
  // Box i of every one of these views is segment i, as on every SR level.
  // Invariant: after a solve with trimming, slev[j].u and slev[j].r of the
  // levels j < K hold the final values only on ctrim_u[j] (and slev[K] on
  // trim_u); elsewhere they are stale.  Every solve (and every pass of the
  // mixed mode) rebuilds the SR levels from the FMG prolongation before it
  // reads them, so nothing reads the stale cells.
  std::vector<Geom> ctrim_r, ctrim_u;
};

// kernel kinds for the per-kernel profile: float64 storage and arithmetic;
// "_f32": float32 storage and arithmetic; "_mixed": float32 storage, float64
// arithmetic
enum Kind {
  kChebResidual, kCheb2Update, kChebStep, kResidRestrict, kCoarseRhs, kTransitionRhs,
  kProlongSet, kProlongAdd, kCoarseSolve, kRestrictF, kGather, kApply,
  kChebResidualF32, kCheb2UpdateF32, kChebStepF32, kResidRestrictF32, kCoarseRhsMixed,
  kTransitionRhsMixed, kProlongSetF32, kProlongAddF32, kCoarseSolveMixed, kRestrictFF32,
  kGatherMixed, kDefect, kAccumulate, kDiff, kDiffF32, kResidNorm, kShellCopy, kShellCopyF32,
  kLegDownF32, kLegUpF32, kVcyclePersistent, kKinds
};
const char* const kKindName[kKinds] = {
  "cheb_residual", "cheb2_update", "cheb_step", "resid_restrict", "coarse_rhs",
  "transition_rhs", "prolong", "prolong_correct", "coarse_solve", "restrict_f",
  "gather_genuine", "apply",
  "cheb_residual_f32", "cheb2_update_f32", "cheb_step_f32", "resid_restrict_f32",
  "coarse_rhs_mixed", "transition_rhs_mixed", "prolong_f32", "prolong_correct_f32",
  "coarse_solve_mixed", "restrict_f_f32", "gather_genuine_mixed", "defect", "accumulate",
  "correction", "correction_f32", "resid_norm", "shell_copy", "shell_copy_f32",
  "leg_down_f32", "leg_up_f32", "vcycle_persistent"};

// kind of a kernel for storage type T: float64 kinds shift to their float32
// counterparts (same order)
template <typename T>
int kind_of(int k64) {
  if (k64 == kDiff) return sizeof(T) == 8 ? kDiff : kDiffF32;
  if (k64 == kShellCopy) return sizeof(T) == 8 ? kShellCopy : kShellCopyF32;
  return sizeof(T) == 8 ? k64 : k64 + kChebResidualF32;
}

struct ProfRec {
  int kind;
  double ops, bytes;
  cudaEvent_t e0, e1;
};

struct Profile {
  bool on = false;
  std::vector<cudaEvent_t> pool;  // free events
  std::vector<ProfRec> recs;      // recorded, not yet read
  long long launches[kKinds] = {};
  double ms[kKinds] = {}, ops[kKinds] = {}, bytes[kKinds] = {};
};

}  // namespace

// Chebyshev coefficients (declared in srfmg_internal.cuh)
Cheb srfmg::chebyshev(int nu, double lo_frac, double hi_frac, double lmax) {
  Cheb c;
  c.nu = nu;
  const double lo = lmax * lo_frac, hi = lmax * hi_frac;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  // three-term recurrence: d_0 = r_0/theta, d_m = rho_m rho_{m-1} d_{m-1} + (2 rho_m/delta) r_m
  double rho_old = delta / theta;
  for (int m = 0; m < nu; ++m) {
    if (m == 0) {
      c.alpha.push_back(0.0);
      c.beta.push_back(1.0 / theta);
    } else {
      const double rho = 1.0 / (2.0 * theta / delta - rho_old);
      c.alpha.push_back(rho * rho_old);
      c.beta.push_back(2.0 * rho / delta);
      rho_old = rho;
    }
  }
  if (nu == 2) {
    // x2 = x0 + c1 r0 + c2 B r0 with B r0 = D^-1 A r0 = r0 - W r0, W the
    // neighbour part (7-point: the sum of the 6 neighbours of r0 over 6)
    const double r0 = delta / theta;
    const double r1 = 1.0 / (2.0 * theta / delta - r0);
    const double c1 = (1.0 + r1 * r0) / theta + 2.0 * r1 / delta;
    const double c2 = -2.0 * r1 / (delta * theta);
    c.a = c1 + c2;
    c.b = -c2 / 6.0;
    c.c2 = c2;
  }
  return c;
}

// Allocation bookkeeping of the whole library (every handle): device
// allocations made, bytes currently held, and the failure-injection
// countdown of sr_debug_fail_alloc (0: off; n > 0: the n-th allocation from
// now fails as if cudaMalloc had run out of memory).
std::atomic<long long> g_allocs{0}, g_live_bytes{0}, g_fail_countdown{0};

bool injected_failure() {
  long long c = g_fail_countdown.load();
  while (c > 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}

// Every device allocation of a handle goes through here; h->allocs owns it
// (freed by free_all).
struct sr_fmg_s {
  sr_fmg_config cfg{};
  int device = 0;
  bool mixed = false;              // SR_MIXED: float32 inner solver
  int K = 0;                       // SR levels
  int G = 0;                       // global levels
  Hier<double> h64;                // levels of the float64 solver
  Hier<float> h32;                 // levels of the float32 inner solver
  float* defect = nullptr;         // SR_MIXED: float32 defect, n^3
  double* minv = nullptr;          // dense inverse of the coarsest operator (small grids)
  double* sep = nullptr;           // separable coarsest solve: bases and 1/lambda
  double *sep_g = nullptr, *sep_q = nullptr;  // its float64 scratch
  unsigned int* status = nullptr;  // device status bits
  Cheb pre, post, fmg;
  int len[3] = {1, 1, 1};          // domain lengths
  bool op27 = false;               // 27-point operator (float64 only)
  W27 w27{6.0, 1.0, 0.0, 0.0};     // operator weights (7-point: w0 = 6, w1 = 1)
  double lmax = 2.0;               // lambda_max(D^-1 A)
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;  // size of each entry of allocs
  double* hbuf_f = nullptr;        // device staging for sr_fmg_solve_host
  double* hbuf_u = nullptr;
  unsigned long long* norms = nullptr;  // sr_fmg_vsolve: ||f||, ||f - A u|| as double bits
  // graph mode: a captured graph (a batch of this one handle) per (f, u)
  // pair, the most recent few pairs
  struct GraphEntry {
    const double* f;
    double* u;
    sr_fmg_batch_t b;
  };
  std::vector<GraphEntry> graphs;
  // pipelined host solves: two slots of device staging, copy streams and
  // the events that order copies, solves and reuse of a slot
  double *pf[2] = {nullptr, nullptr}, *pu[2] = {nullptr, nullptr};
  cudaStream_t cin = nullptr, cout = nullptr, last = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_solved[2] = {}, ev_out[2] = {};
  int pslot = 0;
  bool pused[2] = {false, false};
  int launches = 0;                // kernel launches queued by the last solve
  bool trim = true;                // last-stage trimming (sr_debug_last_stage_trim)
  bool sharded = false;            // the handle owns a range of the segments only
  // segment-resident legs of the float32 SR levels j < K (segment_leg.cu):
  // cluster size, planes per CTA and shared memory per level; C = 0: the
  // level runs the separate kernels
  struct Leg {
    int C = 0, max_planes = 0;
    size_t smem = 0;
  };
  std::vector<Leg> legs;
  bool legs_on = false;            // sr_debug_segment_legs (measured slower: off)
  int zchunk = kDefaultZChunk, cpt = kDefaultCellsPerThread;  // launch shape
  // the global V-cycle as one persistent launch (persistent.cu) from the
  // first global level of at most kPersistentCells cells down
  bool persistent = false;         // usable: float64, 7-point, degree-2 smoothers
  bool persistent_on = true;       // sr_debug_persistent_vcycle
  int vc_blocks = 0;               // blocks of the cooperative launch
  unsigned* vbar = nullptr;        // its grid barrier
  long long generation = 0;        // bumped when the launch sequence changes
  int force_timeout = 0;           // sr_debug_force_wait_timeout
  Profile prof;

  Hier<double>& hier(double*) { return h64; }
  Hier<float>& hier(float*) { return h32; }
};

namespace {

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return SR_ERR_CUDA;    \
  } while (0)

cudaEvent_t take_event(Profile& p) {
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Every kernel launch of a solve goes through here: it counts the launch and,
// when profiling, brackets it with events and records the algorithmic
// floating-point operations and bytes of the launch (units x per-unit counts).
template <class F>
int launch(sr_fmg_s* h, int kind, double units, double ops_per_unit, double bytes_per_unit,
           cudaStream_t s, F&& fn) {
  ++h->launches;
  ProfRec rec{kind, units * ops_per_unit, units * bytes_per_unit, nullptr, nullptr};
  if (h->prof.on) {
    rec.e0 = take_event(h->prof);
    rec.e1 = take_event(h->prof);
    if (rec.e0) cudaEventRecord(rec.e0, s);
  }
  const cudaError_t e = fn();
  if (h->prof.on) {
    if (rec.e1) cudaEventRecord(rec.e1, s);
    if (rec.e0 && rec.e1) h->prof.recs.push_back(rec);
  }
  return e == cudaSuccess ? SR_OK : SR_ERR_CUDA;
}

#define LAUNCH(h, kind, units, ops, bytes, s, call)                                  \
  do {                                                                             \
    int rc_ = launch((h), (kind), (units), (ops), (bytes), (s), [&] { return (call); }); \
    if (rc_) return rc_;                                                           \
  } while (0)

int halvings_to_coarsest(int n, int nc) {
  int m = 0;
  while (nc ? n > nc : n > 3) {
    if (n % 2) return -1;
    n /= 2;
    ++m;
  }
  if (nc) return n == nc ? m : -1;
  return n >= 2 ? m : -1;
}

void schedule(const sr_fmg_config& c, int* J) {
  for (int k = 1; k <= c.K; ++k) {
    if (c.mbs) {  // maximum buffer schedule, Sec. 5.2.1
      J[k - 1] = c.A << (k - 1);
    } else if (c.use_J) {
      J[k - 1] = c.J[k - 1];
    } else {
      const int v = c.A + c.B * (c.K - k);  // Eq. (eq:nb)
      J[k - 1] = 2 * (v / 2);
    }
  }
}

// weights of the configured operator; SR_ERR_INVALID if the stencil is not
// 7, or a 27-point one consistent with -Delta and positive definite.  The
// operator's symbol on the sine mode with c_d = cos(theta_d) is
// w0 - 2 w1 sum c_d - 4 w2 sum c_d c_e - 8 w3 c_0 c_1 c_2, multilinear in c,
// so its extremes over [-1, 1]^3 lie at the corners.
int op_weights(const sr_fmg_config* c, W27* w, double* lmax) {
  if (c->stencil == 0 || c->stencil == 7) {
    *w = W27{6.0, 1.0, 0.0, 0.0};
    *lmax = kLambdaMax7;
    return SR_OK;
  }
  if (c->stencil != 27) return SR_ERR_INVALID;
  const double w1 = c->w[0], w2 = c->w[1], w3 = c->w[2];
  if (!(std::fabs(w1 + 4.0 * w2 + 4.0 * w3 - 1.0) <= 1e-12)) return SR_ERR_INVALID;
  const double w0 = 6.0 * w1 + 12.0 * w2 + 8.0 * w3;
  if (!(w0 > 0.0)) return SR_ERR_INVALID;
  double top = 0.0;
  for (int v = 0; v < 8; ++v) {
    const double x = (v & 1) ? 1.0 : -1.0, y = (v & 2) ? 1.0 : -1.0, z = (v & 4) ? 1.0 : -1.0;
    const double sym = w0 - 2.0 * w1 * (x + y + z) - 4.0 * w2 * (x * y + x * z + y * z) -
                       8.0 * w3 * x * y * z;
    if (v != 7 && !(sym > 0.0)) return SR_ERR_INVALID;
    if (sym > top) top = sym;
  }
  *w = W27{w0, w1, w2, w3};
  *lmax = top / w0;
  return SR_OK;
}

int lengths_of(const sr_fmg_config* c, int len[3]) {
  for (int d = 0; d < 3; ++d) {
    len[d] = c->len[d] ? c->len[d] : 1;
    if (len[d] < 1 || len[d] > 64) return SR_ERR_INVALID;
  }
  return SR_OK;
}

// how the coarsest grid of nd cells is solved exactly (see build_coarse)
enum CoarsePlan { kCoarseDense = 0, kCoarseSeparable = 1, kCoarseUnsupported = -1 };

CoarsePlan coarse_plan(const int nd[3]) {
  const long long m = (long long)nd[0] * nd[1] * nd[2];
  const bool narrow = nd[0] <= 32 && nd[1] <= 32 && nd[2] <= 32;
  if (m <= 512) return kCoarseDense;
  if (narrow) return kCoarseSeparable;
  return m <= 4096 ? kCoarseDense : kCoarseUnsupported;
}

int check_config(const sr_fmg_config* c) {
  if (!c) return SR_ERR_INVALID;
  if (c->precision != SR_FP64 && c->precision != SR_MIXED) return SR_ERR_INVALID;
  int len[3];
  W27 w;
  double lmax;
  if (lengths_of(c, len) || op_weights(c, &w, &lmax)) return SR_ERR_INVALID;
  if (c->stencil == 27 && c->precision != SR_FP64) return SR_ERR_INVALID;
  {
    // the kernels index the cells of a box (up to the whole finest grid)
    // with 32-bit integers
    const long long cells = (long long)c->n * c->n * c->n * len[0] * len[1] * len[2];
    if (c->n > 0 && cells >= (1LL << 31)) return SR_ERR_UNSUPPORTED_SIZE;
  }
  if (c->precision == SR_MIXED && (c->n_outer < 0 || c->n_outer > 16)) return SR_ERR_INVALID;
  if (c->alpha < 0 || c->nu1 < 0 || c->nu2 < 0 || c->alpha > 16 || c->nu1 > 16 || c->nu2 > 16)
    return SR_ERR_INVALID;
  if (!(c->cheb_lo > 0.0 && c->cheb_hi > c->cheb_lo && c->cheb_hi < 4.0)) return SR_ERR_INVALID;
  if (c->n_coarse < 0 || c->n_coarse > 16 || c->n_coarse == 1) return SR_ERR_UNSUPPORTED_SIZE;
  if (c->n < 2 || c->n > 2048) return SR_ERR_UNSUPPORTED_SIZE;
  const int halvings = halvings_to_coarsest(c->n, c->n_coarse);
  if (halvings < 0) return SR_ERR_UNSUPPORTED_SIZE;
  {
    const int ncs = c->n >> halvings, nd[3] = {ncs * len[0], ncs * len[1], ncs * len[2]};
    if (coarse_plan(nd) == kCoarseUnsupported) return SR_ERR_UNSUPPORTED_SIZE;
  }
  if (c->seg < 0 || c->K < 0 || c->K > SR_FMG_MAXK) return SR_ERR_INVALID;
  if (c->seg == 0 || c->K == 0) return (c->seg_count || c->seg_first) ? SR_ERR_INVALID : SR_OK;
  if (c->mbs && (c->A < 0 || c->A % 2 || c->A > 4096 >> c->K)) return SR_ERR_INVALID;
  if (c->n % c->seg) return SR_ERR_INVALID;
  if (c->seg % (1 << c->K)) return SR_ERR_INVALID;
  if (halvings_to_coarsest(c->n >> c->K, c->n_coarse) < 0) return SR_ERR_UNSUPPORTED_SIZE;
  const long long nseg1 = c->n / c->seg;
  const long long nsegs = nseg1 * nseg1 * nseg1 * len[0] * len[1] * len[2];
  if (nsegs > 65535) return SR_ERR_UNSUPPORTED_SIZE;
  if (c->seg_count < 0 || c->seg_first < 0) return SR_ERR_INVALID;
  if (c->seg_count > 0 &&
      ((long long)c->seg_first + c->seg_count > nsegs || c->precision != SR_FP64))
    return SR_ERR_INVALID;
  int J[SR_FMG_MAXK];
  schedule(*c, J);
  for (int k = 1; k <= c->K; ++k) {
    if (J[k - 1] < 0 || J[k - 1] % 2) return SR_ERR_INVALID;
    if (k >= 2 && 2 * J[k - 2] < J[k - 1]) return SR_ERR_INVALID;
  }
  return SR_OK;
}

template <typename T>
int dalloc(sr_fmg_s* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return SR_OK;
  void* q = nullptr;
  ++g_allocs;
  if (injected_failure()) return SR_ERR_OOM;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return SR_ERR_OOM;
  }
  h->allocs.push_back(q);
  h->alloc_bytes.push_back(count * sizeof(T));
  g_live_bytes += (long long)(count * sizeof(T));
  h->bytes += count * sizeof(T);
  if (cudaMemset(q, 0, count * sizeof(T)) != cudaSuccess) return SR_ERR_CUDA;
  *p = static_cast<T*>(q);
  return SR_OK;
}

// With F(1, 2, ...) in float64 and the 7-point operator, the FMG degree-1
// step S^alpha is followed by the V-cycle's degree-2 pre-smoother on the same
// level and f; the step also forms that smoother's first residual
// D^-1 (f - A u_new) = (1 - beta) r + (beta/6) (sum of the neighbours of r)
// into the level's d, and the pre-smoother starts from it.
template <typename T>
bool fused_fmg_step(const sr_fmg_s* h) {
  return !h->op27 && h->fmg.nu == 1 && h->fmg.alpha[0] == 0.0 && h->pre.nu == 2;
}

BoxDesc whole_box(const int nd[3]) {
  BoxDesc b;
  std::memset(&b, 0, sizeof(b));
  for (int d = 0; d < 3; ++d) {
    b.lo[d] = 0; b.hi[d] = nd[d];
    b.plo[d] = 0; b.phi[d] = nd[d];
    b.rlo[d] = 0; b.rhi[d] = nd[d] / 2;
    b.glo[d] = 0; b.ghi[d] = nd[d];
  }
  b.ox = b.oy = b.oz = 0;
  b.sy = nd[0];
  b.sz = (long long)nd[0] * nd[1];
  b.base = 0;
  return b;
}

void set_dims(Geom& L, int n, const int len[3]) {
  L.n = n;
  for (int d = 0; d < 3; ++d) L.nd[d] = n * len[d];
}

long long cells_of(const Geom& L) { return (long long)L.nd[0] * L.nd[1] * L.nd[2]; }
Dims dims_of(const Geom& L) { return Dims{L.nd[0], L.nd[1], L.nd[2]}; }

long long prod(const int lo[3], const int hi[3]) {
  return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
}

int finish_level(sr_fmg_s* h, Geom& L) {
  L.nbox = (int)L.hboxes.size();
  int rc = dalloc(h, &L.dboxes, L.hboxes.size());
  if (rc) return rc;
  CK(cudaMemcpy(L.dboxes, L.hboxes.data(), sizeof(BoxDesc) * L.hboxes.size(),
                cudaMemcpyHostToDevice));
  BoxDesc g = whole_box(L.nd);
  rc = dalloc(h, &L.dglobal, 1);
  if (rc) return rc;
  CK(cudaMemcpy(L.dglobal, &g, sizeof(BoxDesc), cudaMemcpyHostToDevice));
  LevelView v{};
  v.zchunk = kDefaultZChunk;
  v.cpt = kDefaultCellsPerThread;
  v.boxes = L.dboxes;
  v.nbox = L.nbox;
  v.n = L.n;
  v.nx = L.nd[0];
  v.ny = L.nd[1];
  v.nz = L.nd[2];
  v.shell = !L.hboxes.empty() && L.hboxes[0].ox < L.hboxes[0].lo[0];
  for (const BoxDesc& b : L.hboxes) {
    const int slo[3] = {b.ox, b.oy, b.oz};
    int shi[3];
    const bool shell = b.ox < b.lo[0];
    for (int d = 0; d < 3; ++d) shi[d] = shell ? b.hi[d] + 1 : b.hi[d];
    auto mx = [](int& m, long long x) { if (x > m) m = (int)x; };
    mx(v.max_cells, prod(b.lo, b.hi));
    mx(v.max_stored, prod(slo, shi));
    mx(v.max_prolong, prod(b.plo, b.phi));
    mx(v.max_restrict, prod(b.rlo, b.rhi));
    mx(v.max_genuine, prod(b.glo, b.ghi));
    mx(v.max_ex, b.hi[0] - b.lo[0]);
    mx(v.max_ey, b.hi[1] - b.lo[1]);
    mx(v.max_ez, b.hi[2] - b.lo[2]);
    L.tot_cells += (double)prod(b.lo, b.hi);
    L.tot_prolong += (double)prod(b.plo, b.phi);
    L.tot_restrict += (double)prod(b.rlo, b.rhi);
    L.tot_genuine += (double)prod(b.glo, b.ghi);
  }
  L.view = v;
  return SR_OK;
}

// Exact coarsest solves.  On each axis of N cells the factors
// sin(k pi (i + 1/2) / N), k = 1..N, are orthogonal with squared norms N/2
// (k < N) and N (k = N); the operator's eigenvalue on their product is
// n^2 (w0 - 2 w1 sum c_d - 4 w2 sum c_d c_e - 8 w3 c_0 c_1 c_2),
// c_d = cos(k_d pi / N_d) (7-point: w = (6, 1, 0, 0)).  Small grids use the
// dense inverse built from that eigen-decomposition (one launch); larger
// ones, with at most 32 cells per axis, apply it as separable transforms
// (three launches, about 2 (nx + ny + nz) operations per cell instead of
// nx ny nz).
// orthonormal sine basis of an axis of N cells, row k - 1 = mode k, and the
// mode cosines cos(k pi / N)
void sine_basis(int N, std::vector<double>& phi, std::vector<double>& cs) {
  const double pi = 3.14159265358979323846;
  phi.assign((size_t)N * N, 0.0);
  cs.assign(N, 0.0);
  for (int k = 1; k <= N; ++k) {
    const double norm = std::sqrt((k < N) ? 2.0 / N : 1.0 / N);
    for (int i = 0; i < N; ++i) phi[(size_t)(k - 1) * N + i] = norm * std::sin(pi * k * (i + 0.5) / N);
    cs[k - 1] = std::cos(pi * k / N);
  }
}

double symbol_eig(const W27& w, double n2, double x, double y, double z) {
  return n2 * (w.w0 - 2.0 * w.w1 * (x + y + z) - 4.0 * w.w2 * (x * y + x * z + y * z) -
               8.0 * w.w3 * x * y * z);
}

std::vector<double> coarsest_inverse(const int nd[3], int n, const W27& w) {
  const int m = nd[0] * nd[1] * nd[2];
  std::vector<double> phi[3], cs[3];
  for (int d = 0; d < 3; ++d) sine_basis(nd[d], phi[d], cs[d]);
  const double n2 = (double)n * n;
  std::vector<double> minv((size_t)m * m, 0.0), v(m);
  for (int k3 = 0; k3 < nd[2]; ++k3)
    for (int k2 = 0; k2 < nd[1]; ++k2)
      for (int k1 = 0; k1 < nd[0]; ++k1) {
        const double il = 1.0 / symbol_eig(w, n2, cs[0][k1], cs[1][k2], cs[2][k3]);
        for (int zz = 0; zz < nd[2]; ++zz)
          for (int yy = 0; yy < nd[1]; ++yy)
            for (int xx = 0; xx < nd[0]; ++xx)
              v[((size_t)zz * nd[1] + yy) * nd[0] + xx] =
                  phi[0][(size_t)k1 * nd[0] + xx] * phi[1][(size_t)k2 * nd[1] + yy] *
                  phi[2][(size_t)k3 * nd[2] + zz];
        for (int p = 0; p < m; ++p) {
          const double wv = il * v[p];
          double* row = &minv[(size_t)p * m];
          for (int q = 0; q < m; ++q) row[q] += wv * v[q];
        }
      }
  return minv;
}

// [Px | Py | Pz | 1/lambda] for the separable solve
std::vector<double> coarsest_separable(const int nd[3], int n, const W27& w) {
  std::vector<double> phi[3], cs[3], out;
  for (int d = 0; d < 3; ++d) {
    sine_basis(nd[d], phi[d], cs[d]);
    out.insert(out.end(), phi[d].begin(), phi[d].end());
  }
  const double n2 = (double)n * n;
  for (int k3 = 0; k3 < nd[2]; ++k3)
    for (int k2 = 0; k2 < nd[1]; ++k2)
      for (int k1 = 0; k1 < nd[0]; ++k1)
        out.push_back(1.0 / symbol_eig(w, n2, cs[0][k1], cs[1][k2], cs[2][k3]));
  return out;
}

struct CoarseOp {
  double* minv = nullptr;
  double *sep = nullptr, *g = nullptr, *q = nullptr;
};

// device data of the exact solve on a coarsest grid of nd cells (allocated
// through h, freed with it)
int build_coarse(sr_fmg_s* h, const int nd[3], int n, const W27& w, CoarseOp* op) {
  const CoarsePlan plan = coarse_plan(nd);
  if (plan == kCoarseUnsupported) return SR_ERR_UNSUPPORTED_SIZE;
  const std::vector<double> data = plan == kCoarseDense ? coarsest_inverse(nd, n, w)
                                                        : coarsest_separable(nd, n, w);
  double* dev = nullptr;
  int rc = dalloc(h, &dev, data.size());
  if (rc) return rc;
  CK(cudaMemcpy(dev, data.data(), data.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (plan == kCoarseDense) {
    op->minv = dev;
    return SR_OK;
  }
  op->sep = dev;
  const size_t m = (size_t)nd[0] * nd[1] * nd[2];
  if ((rc = dalloc(h, &op->g, m))) return rc;
  return dalloc(h, &op->q, m);
}

// global levels of ntop down to the coarsest grid; with top_user the finest
// level's u is the caller's array (no allocation); the finest level never
// allocates f, t, rhs or rho (it reads f from the caller or the defect)
template <typename T>
int build_global_levels(sr_fmg_s* h, Hier<T>& H, int ntop, bool top_user) {
  const int m = halvings_to_coarsest(ntop, h->cfg.n_coarse);
  h->G = m + 1;
  H.glev.resize(h->G);
  const bool need_d =
      h->cfg.alpha > 2 || h->cfg.nu1 > 2 || h->cfg.nu2 > 2 || fused_fmg_step<T>(h);
  const bool sr = h->K > 0;
  for (int g = 0; g < h->G; ++g) {
    Level<T>& L = H.glev[g];
    set_dims(L, ntop >> (h->G - 1 - g), h->len);
    L.hboxes.assign(1, whole_box(L.nd));
    if (g == 0) for (int d = 0; d < 3; ++d) { L.hboxes[0].rlo[d] = 0; L.hboxes[0].rhi[d] = 0; }
    int rc = finish_level(h, L);
    if (rc) return rc;
    const size_t cells = (size_t)cells_of(L);
    const bool finest = (g == h->G - 1) && !sr;
    if ((rc = dalloc(h, &L.r, cells))) return rc;
    if (need_d && (rc = dalloc(h, &L.d, cells))) return rc;
    if (!(finest && top_user) && (rc = dalloc(h, &L.u, cells))) return rc;
    if (finest) continue;
    if ((rc = dalloc(h, &L.t, cells))) return rc;
    if ((rc = dalloc(h, &L.rhs, cells))) return rc;
    if ((rc = dalloc(h, &L.rho, cells))) return rc;
    if ((rc = dalloc(h, &L.f, cells))) return rc;
  }
  if (!h->minv && !h->sep) {
    CoarseOp op;
    int rc = build_coarse(h, H.glev[0].nd, H.glev[0].n, h->w27, &op);
    if (rc) return rc;
    h->minv = op.minv;
    h->sep = op.sep;
    h->sep_g = op.g;
    h->sep_q = op.q;
  }
  return SR_OK;
}

template <typename T>
int build_sr_levels(sr_fmg_s* h, Hier<T>& H) {
  const sr_fmg_config& c = h->cfg;
  const int K = h->K;
  int J[SR_FMG_MAXK];
  schedule(c, J);
  int nsd[3];
  for (int d = 0; d < 3; ++d) nsd[d] = c.n * h->len[d] / c.seg;  // segments per dimension
  // the segments this handle owns: [seg_lo, seg_hi) in x-fastest order
  const int seg_lo = c.seg_count > 0 ? c.seg_first : 0;
  const int seg_hi = c.seg_count > 0 ? c.seg_first + c.seg_count : nsd[0] * nsd[1] * nsd[2];
  const bool need_d = c.alpha > 2 || c.nu1 > 2 || c.nu2 > 2 || fused_fmg_step<T>(h);
  H.slev.resize(K + 1);
  for (int k = 1; k <= K; ++k) {
    Level<T>& L = H.slev[k];
    set_dims(L, c.n >> (K - k), h->len);
    const int sk = c.seg >> (K - k);
    const int s0 = c.seg >> K;
    std::vector<BoxDesc> boxes;
    long long slot = 0;
    int index = -1;  // segment number, x fastest over the segment grid
    for (int pz = 0; pz < nsd[2]; ++pz)
      for (int py = 0; py < nsd[1]; ++py)
        for (int px = 0; px < nsd[0]; ++px) {
          ++index;
          if (index < seg_lo || index >= seg_hi) continue;  // another handle's segment
          const int q[3] = {px, py, pz};
          BoxDesc b;
          std::memset(&b, 0, sizeof(b));
          for (int d = 0; d < 3; ++d) {
            b.glo[d] = q[d] * sk;
            b.ghi[d] = (q[d] + 1) * sk;
            const int nd = L.nd[d];
            b.lo[d] = b.glo[d] - J[k - 1] < 0 ? 0 : b.glo[d] - J[k - 1];
            b.hi[d] = b.ghi[d] + J[k - 1] > nd ? nd : b.ghi[d] + J[k - 1];
            b.plo[d] = b.lo[d] > 0 ? b.lo[d] - 1 : 0;
            b.phi[d] = b.hi[d] < nd ? b.hi[d] + 1 : nd;
            if (k > 1) {  // Omega^F on level k-1: the cells under the compute region
              b.rlo[d] = b.lo[d] / 2;
              b.rhi[d] = b.hi[d] / 2;
            } else {      // transition: this segment's genuine level-0 cells
              b.rlo[d] = q[d] * s0;
              b.rhi[d] = (q[d] + 1) * s0;
            }
          }
          b.ox = b.lo[0] - 1;
          b.oy = b.lo[1] - 1;
          b.oz = b.lo[2] - 1;
          const int e0 = b.hi[0] - b.lo[0] + 2, e1 = b.hi[1] - b.lo[1] + 2,
                    e2 = b.hi[2] - b.lo[2] + 2;
          b.sy = e0;
          b.sz = (long long)e0 * e1;
          const long long size = (long long)e0 * e1 * e2;
          if (size > slot) slot = size;
          boxes.push_back(b);
        }
    for (size_t i = 0; i < boxes.size(); ++i) boxes[i].base = (long long)i * slot;
    L.slot = slot;
    L.hboxes = boxes;
    int rc = finish_level(h, L);
    if (rc) return rc;
    if (k == K) {
      H.trim_r.n = H.trim_u.n = L.n;
      for (int d = 0; d < 3; ++d) H.trim_r.nd[d] = H.trim_u.nd[d] = L.nd[d];
      H.trim_r.hboxes = H.trim_u.hboxes = boxes;
      for (size_t i = 0; i < boxes.size(); ++i) {
        BoxDesc& r = H.trim_r.hboxes[i];
        BoxDesc& u = H.trim_u.hboxes[i];
        for (int d = 0; d < 3; ++d) {
          r.lo[d] = std::max(r.lo[d], r.glo[d] - 1);
          r.hi[d] = std::min(r.hi[d], r.ghi[d] + 1);
          r.plo[d] = std::max(r.plo[d], r.glo[d] - 2);
          r.phi[d] = std::min(r.phi[d], r.ghi[d] + 2);
          u.lo[d] = u.glo[d];
          u.hi[d] = u.ghi[d];
        }
      }
      if ((rc = finish_level(h, H.trim_r))) return rc;
      if ((rc = finish_level(h, H.trim_u))) return rc;
    }
    const size_t elems = (size_t)slot * boxes.size();
    if ((rc = dalloc(h, &L.u, elems))) return rc;
    if ((rc = dalloc(h, &L.r, elems))) return rc;
    if (need_d && (rc = dalloc(h, &L.d, elems))) return rc;
    if (k < K) {
      if ((rc = dalloc(h, &L.t, elems))) return rc;
      if ((rc = dalloc(h, &L.rhs, elems))) return rc;
      if ((rc = dalloc(h, &L.rho, elems))) return rc;
      if ((rc = dalloc(h, &L.f, (size_t)cells_of(L)))) return rc;
    }
  }
  // the coarse levels' last-stage regions, from the finest level's trim down
  H.ctrim_r.assign(K + 1, Geom{});
  H.ctrim_u.assign(K + 1, Geom{});
  auto floor_half = [](int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); };
  for (int j = K - 1; j >= 1; --j) {
    const Level<T>& L = H.slev[j];
    const Geom& F = (j + 1 == K) ? H.trim_r : H.ctrim_r[j + 1];
    Geom& R = H.ctrim_r[j];
    Geom& U = H.ctrim_u[j];
    R.n = U.n = L.n;
    for (int d = 0; d < 3; ++d) R.nd[d] = U.nd[d] = L.nd[d];
    R.hboxes = U.hboxes = L.hboxes;
    // box i of both levels must be the same segment: the fine box's genuine
    // region is the coarse one's doubled
    if (F.hboxes.size() != L.hboxes.size()) return SR_ERR_INVALID;
    for (size_t i = 0; i < L.hboxes.size(); ++i)
      for (int d = 0; d < 3; ++d)
        if (F.hboxes[i].glo[d] != 2 * L.hboxes[i].glo[d] ||
            F.hboxes[i].ghi[d] != 2 * L.hboxes[i].ghi[d])
          return SR_ERR_INVALID;
    for (size_t i = 0; i < L.hboxes.size(); ++i) {
      const BoxDesc& c = L.hboxes[i];
      const BoxDesc& f = F.hboxes[i];
      BoxDesc& r = R.hboxes[i];
      BoxDesc& u = U.hboxes[i];
      for (int d = 0; d < 3; ++d) {
        // the prolongation of fine cells [a, b) reads coarse cells
        // floor((a - 1) / 2) .. floor(b / 2), inside the domain and the
        // coarse box's stored cells
        int ulo = floor_half(f.plo[d] - 1), uhi = floor_half(f.phi[d]) + 1;
        ulo = std::max(ulo, std::max(c.lo[d] - 1, 0));
        uhi = std::min(uhi, std::min(c.hi[d] + 1, L.nd[d]));
        u.lo[d] = std::max(c.lo[d], ulo);
        u.hi[d] = std::min(c.hi[d], uhi);
        u.plo[d] = ulo;
        u.phi[d] = uhi;
        r.lo[d] = std::max(c.lo[d], ulo - 1);
        r.hi[d] = std::min(c.hi[d], uhi + 1);
        r.plo[d] = std::max(c.plo[d], ulo - 2);
        r.phi[d] = std::min(c.phi[d], uhi + 2);
      }
    }
    int rc = finish_level(h, R);
    if (rc) return rc;
    if ((rc = finish_level(h, U))) return rc;
  }
  return SR_OK;
}

// The persistent global V-cycle (persistent.cu): float64, 7-point,
// degree-2 smoothers; one block per SM.  One block of 256 threads per SM
// measured faster than two (each grid barrier waits on half as many
// arrivals; the per-pass work is HBM- or FP64-bound either way) and than a
// half or a quarter of the SMs (too few warps to cover the finest level).
int plan_persistent(sr_fmg_s* h) {
  h->persistent = false;
  if (h->mixed || h->op27 || h->pre.nu != 2 || h->post.nu != 2 || h->G < 2) return SR_OK;
  if ((int)h->h64.glev.size() > kVcycleMaxLevels) return SR_OK;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    return SR_OK;
  }
  const int per_sm = std::min(vcycle_max_blocks_per_sm(), 1);
  if (per_sm < 1 || sms < 1) return SR_OK;
  int rc = dalloc(h, &h->vbar, 2);
  if (rc) return rc;
  h->vc_blocks = sms * per_sm;
  h->persistent = true;
  return SR_OK;
}

// Segment-resident legs for the float32 SR levels j = 1 .. K-1 (the
// levels below a stage's top): a level qualifies when its boxes' stored
// planes can be split over a cluster of at most 16 CTAs whose shared memory
// holds two arrays of a slab, when every box row and plane keeps the
// 16-byte alignment of the bulk copies, and the operator, smoothers and
// precision are those the fused legs implement (7-point, degree-2 pre- and
// post-smoother, float32).
int plan_legs(sr_fmg_s* h) {
  h->legs.assign(h->K + 1, sr_fmg_s::Leg{});
  if (!h->mixed || h->op27 || h->pre.nu != 2 || h->post.nu != 2 || h->K < 2) return SR_OK;
  constexpr size_t kMaxSmem = 232448 - 1024;  // dynamic shared memory per CTA on sm_103a
  if (leg_prepare(kMaxSmem) != cudaSuccess) {
    cudaGetLastError();
    return SR_OK;  // no fused legs on this device
  }
  for (int j = 1; j < h->K; ++j) {
    const Level<float>& L = h->h32.slev[j];
    int e0 = 0, e1 = 0, e2 = 0;
    bool aligned = L.slot % 4 == 0 && L.nbox <= 65535;
    for (const BoxDesc& b : L.hboxes) {
      const int a0 = b.hi[0] - b.lo[0] + 2, a1 = b.hi[1] - b.lo[1] + 2, a2 = b.hi[2] - b.lo[2] + 2;
      aligned = aligned && (a0 * a1) % 4 == 0 && b.base % 4 == 0;
      e0 = std::max(e0, a0);
      e1 = std::max(e1, a1);
      e2 = std::max(e2, a2);
    }
    if (!aligned) continue;
    sr_fmg_s::Leg best;
    for (size_t cap : {(size_t)113 * 1024, kMaxSmem}) {  // two CTAs per SM if possible
      for (int C = 1; C <= 16 && !best.C; C *= 2) {
        const int planes = (e2 + C - 1) / C;
        const size_t smem = leg_smem_bytes(e0, e1, planes);
        if (planes < 1 || smem > cap || leg_max_clusters(C, smem) < 1) continue;
        best.C = C;
        best.max_planes = planes;
        best.smem = smem;
      }
      if (best.C) break;
    }
    h->legs[j] = best;
  }
  return SR_OK;
}

// ---------------------------------------------------------------------------
// launch sequence, for storage type T

template <typename T>
FieldT<T> view_global(const Geom& L, const T* p) { return FieldT<T>{p, L.dglobal, 1}; }
template <typename T>
FieldT<T> view_boxes(const Geom& L, const T* p) { return FieldT<T>{p, L.dboxes, 0}; }

// algorithmic per-cell counts (floating-point operations; bytes with each
// array element read or written once) of each kernel
// The operator-dependent launches: the 7-point kernels, or the 27-point ones
// (float64 only) when the handle's stencil is 27.
template <typename T>
cudaError_t op_cheb_residual(const sr_fmg_s* h, const LevelView& L, const T* u, T* r,
                             FieldT<T> f, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (h->op27) return launch27_cheb_residual(L, u, r, f, h->w27, s);
  }
  return launch_cheb_residual<T>(L, u, r, f, s);
}
template <typename T>
cudaError_t op_cheb2_update(const sr_fmg_s* h, const LevelView& L, T* u, const T* r,
                            const Cheb& c, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (h->op27) return launch27_cheb2_update(L, u, r, c.a, c.c2, h->w27, s);
  }
  return launch_cheb2_update<T>(L, u, r, c.a, c.b, s);
}
template <typename T>
cudaError_t op_coarse_rhs(const sr_fmg_s* h, const LevelView& C, const LevelView& F, const T* u,
                          const T* rho, T* rhs, T* t, T* r, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (h->op27) return launch27_coarse_rhs(C, F, u, rho, rhs, t, r, h->w27, s);
  }
  return launch_coarse_rhs<T>(C, F, u, rho, rhs, t, r, s);
}
template <typename T>
cudaError_t op_transition_rhs(const sr_fmg_s* h, const LevelView& C, const T* t, const T* rho,
                              T* u, T* rhs, T* r, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (h->op27) return launch27_transition_rhs(C, t, rho, u, rhs, r, h->w27, s);
  }
  return launch_transition_rhs<T>(C, t, rho, u, rhs, r, s);
}

// algorithmic floating-point operations per unit of the operator kernels
// (7-point / 27-point): smoother passes per cell, residual + restriction per
// coarse cell, coarse right-hand side per cell
double ops_smooth(const sr_fmg_s* h) { return h->op27 ? 15 : 7; }
double ops_rhs(const sr_fmg_s* h) { return h->op27 ? 15 : 7; }

// uhat, rho on the coarse cells of F's restriction region from the fine u
// and right-hand side f: one fused 7-point pass (the residual of the 8
// children summed through the faces of the 2x2x2 block), or for the
// 27-point operator the residual into F's smoother scratch r (column form)
// followed by the restriction of u and r
template <typename T>
int resid_restrict(sr_fmg_s* h, const Level<T>& F, const T* u, FieldT<T> f, const Level<T>& C,
                   T* uhat, T* rho, cudaStream_t s) {
  const double w = sizeof(T);
  if constexpr (sizeof(T) == 8) {
    if (h->op27) {
      LAUNCH(h, kResidRestrict, F.tot_cells, 16, 3 * w, s,
             launch27_residual_zm(F.view, u, f, F.r, h->w27, s));
      LAUNCH(h, kResidRestrict, F.tot_restrict, 16, 18 * w, s,
             launch27_restrict_pair(F.view, u, F.r, C.view, uhat, rho, s));
      return SR_OK;
    }
  }
  LAUNCH(h, kind_of<T>(kResidRestrict), F.tot_restrict, 42, 18 * w, s,
         launch_resid_restrict<T>(F.view, u, f, C.view, uhat, rho, s));
  return SR_OK;
}

// After restriction the coarse smoother's first residual D^-1 (rhs - A u) is
// D^-1 rho inside the restriction region and 0 elsewhere (rhs = rho + A u,
// or A u, with the same u), so the float64 solve writes it with the coarse
// right-hand side instead of forming rhs - A u again.  The float32 inner
// solver of the mixed mode keeps the literal pass: its rhs is rounded to
// float32, and the later residuals see that rounding.
template <typename T>
constexpr bool kFirstResidual = sizeof(T) == 8;

// r_first: the first residual D^-1 (f - A u) is already formed there (L.r,
// written with the level's coarse right-hand side, or L.d, written by the
// fused FMG step), so the first residual pass is skipped; r_first == L.d only
// with c.nu == 2
template <typename T>
int smooth(sr_fmg_s* h, const Level<T>& L, const Cheb& c, T* u, FieldT<T> f, cudaStream_t s,
           const T* r_first = nullptr) {
  if (c.nu == 0) return SR_OK;
  const double cells = L.tot_cells;
  const double w = sizeof(T);
  if (c.nu == 2) {
    if (!r_first)
      LAUNCH(h, kind_of<T>(kChebResidual), cells, ops_smooth(h), 3 * w, s,
             op_cheb_residual<T>(h, L.view, u, L.r, f, s));
    LAUNCH(h, kind_of<T>(kCheb2Update), cells, ops_smooth(h), 3 * w, s,
           op_cheb2_update<T>(h, L.view, u, r_first ? r_first : L.r, c, s));
    return SR_OK;
  }
  for (int m = 0; m < c.nu; ++m) {
    if (!(r_first && m == 0))
      LAUNCH(h, kind_of<T>(kChebResidual), cells, ops_smooth(h), 3 * w, s,
             op_cheb_residual<T>(h, L.view, u, L.r, f, s));
    const int write_d = (c.nu > 1 && m < c.nu - 1) ? 1 : 0;
    const bool with_d = write_d || c.alpha[m] != 0.0;
    LAUNCH(h, kind_of<T>(kChebStep), cells, with_d ? 3 : 2, (with_d ? 5 : 3) * w, s,
           launch_cheb_step<T>(L.view, u, L.d, L.r, c.alpha[m], c.beta[m], write_d, s));
  }
  return SR_OK;
}

// S^alpha on level L before the FMG V-cycle from it; returns (in *r_first)
// the pre-smoother's first residual when the fused step formed it
template <typename T>
int fmg_step(sr_fmg_s* h, const Level<T>& L, T* u, FieldT<T> f, cudaStream_t s,
             const T** r_first) {
  *r_first = nullptr;
  if (!fused_fmg_step<T>(h)) return smooth(h, L, h->fmg, u, f, s);
  const double cells = L.tot_cells;
  const double w = sizeof(T);
  LAUNCH(h, kind_of<T>(kChebResidual), cells, ops_smooth(h), 3 * w, s,
         op_cheb_residual<T>(h, L.view, u, L.r, f, s));
  LAUNCH(h, kind_of<T>(kChebStep), cells, 8, 4 * w, s,
         launch_cheb1_next<T>(L.view, u, L.r, L.d, h->fmg.beta[0], s));
  *r_first = L.d;
  return SR_OK;
}

// exact solve on the coarsest global level L: u = A^-1 f (dense inverse or
// separable transforms, whichever the handle built)
template <typename T>
int coarse_solve(sr_fmg_s* h, const Level<T>& L, FieldT<T> f, T* u, cudaStream_t s) {
  const double m = L.tot_cells;
  if (h->minv) {
    LAUNCH(h, kind_of<T>(kCoarseSolve), m * m, 1, 8, s,
           launch_coarse_solve<T>(L.view, h->minv, f, u, s));
    return SR_OK;
  }
  const double ops = 2.0 * (L.nd[0] + L.nd[1] + L.nd[2]) + 1.0;
  LAUNCH(h, kind_of<T>(kCoarseSolve), m, ops, 40.0 + 2.0 * sizeof(T), s,
         launch_coarse_solve_sep<T>(L.view, h->sep, h->sep_g, h->sep_q, f, u, s));
  h->launches += 2;  // three kernels
  return SR_OK;
}

// The persistent cycle takes over from the first global level of at most
// this many cells (its cooperative launch keeps two blocks per SM: enough for
// these small levels, fewer warps than the separate kernels give a large one).
constexpr long long kPersistentCells = 64LL * 64 * 64;

// FASMGV from global level g down (g >= 1) in one persistent launch
int persistent_vcycle(sr_fmg_s* h, Hier<double>& H, int g, double* u, const double* f,
                      const double* r_first, cudaStream_t s) {
  VcycleArgs a{};
  a.top = g;
  for (int j = 0; j <= g; ++j) {
    Level<double>& L = H.glev[j];
    VcycleLevel& v = a.lev[j];
    const double n2 = (double)L.n * L.n;
    v.view = L.view;
    v.u = (j == g) ? u : L.u;
    v.r = L.r;
    v.t = L.t;
    v.rhs = L.rhs;
    v.rho = L.rho;
    v.f = (j == g) ? f : L.rhs;
    // the constants the separate kernels' launchers pass
    v.cf = 1.0 / (6.0 * n2);
    v.cS = -3.0 * n2 / 8.0;
    v.cO = n2 / 8.0;
    v.c6 = 6.0 * n2;
    v.cn = -n2;
    v.cr = 1.0 / (6.0 * n2);
  }
  a.r_first = r_first;
  a.minv = h->minv;
  a.sep = h->sep;
  a.sep_g = h->sep_g;
  a.sep_q = h->sep_q;
  {
    const Geom& c = H.glev[0];
    int W = 1;
    while (W < std::max(c.nd[0], std::max(c.nd[1], c.nd[2]))) W *= 2;
    a.sep_w = W;
  }
  a.pre_a = h->pre.a;
  a.pre_b = h->pre.b;
  a.post_a = h->post.a;
  a.post_b = h->post.b;
  a.sixth = 1.0 / 6.0;
  a.eighth = 0.125;
  a.three = 3.0;
  a.w64 = 1.0 / 64.0;
  a.mone = -1.0;
  a.one = 1.0;
  a.zero = 0.0;
  a.bar = h->vbar;
  a.status = h->status;
  a.force_timeout = h->force_timeout;
  CK(cudaMemsetAsync(h->vbar, 0, sizeof(unsigned), s));
  // algorithmic counts per cell of the top level: about 45 operations and
  // 200 bytes per cell of each level with the coarser ones adding 1/8 each
  const double cells = H.glev[g].tot_cells;
  LAUNCH(h, kVcyclePersistent, cells, 45.0 * 8 / 7, 200.0 * 8 / 7, s,
         launch_vcycle(a, h->vc_blocks, s));
  return SR_OK;
}

// FASMGV on global level g (Fig. "FAS multigrid V-cycle"); u is the level's
// u (or the caller's u on the finest plain FP64 level).
template <typename T>
int vcycle_global(sr_fmg_s* h, Hier<T>& H, int g, T* u, FieldT<T> rhs, cudaStream_t s,
                  const T* r_first = nullptr) {
  Level<T>& L = H.glev[g];
  const double w = sizeof(T);
  if (g == 0) return coarse_solve<T>(h, L, rhs, u, s);
  if constexpr (sizeof(T) == 8) {
    if (h->persistent && h->persistent_on && cells_of(L) <= kPersistentCells)
      return persistent_vcycle(h, H, g, u, rhs.p, r_first, s);
  }
  Level<T>& C = H.glev[g - 1];
  int rc = smooth(h, L, h->pre, u, rhs, s, r_first);
  if (rc) return rc;
  rc = resid_restrict<T>(h, L, u, rhs, C, C.u, C.rho, s);
  if (rc) return rc;
  // the coarse level's first residual comes with its right-hand side in
  // float64 (the coarsest level is solved directly and needs none)
  const bool cr = kFirstResidual<T> && g - 1 >= 1;
  LAUNCH(h, kind_of<T>(kCoarseRhs), C.tot_cells, ops_rhs(h) + (cr ? 1 : 0), (cr ? 5 : 4) * w, s,
         op_coarse_rhs<T>(h, C.view, L.view, C.u, C.rho, C.rhs, C.t, cr ? C.r : nullptr, s));
  rc = vcycle_global(h, H, g - 1, C.u, view_global<T>(C, C.rhs), s, cr ? C.r : nullptr);
  if (rc) return rc;
  LAUNCH(h, kind_of<T>(kDiff), C.tot_cells, 1, 3 * w, s,
         launch_diff<T>(C.view, C.u, C.t, C.rho, s));
  LAUNCH(h, kind_of<T>(kProlongAdd), L.tot_prolong, 3.75, 2.125 * w, s,
         launch_prolong<T>(C.view, C.rho, L.view, u, 1, s));
  return smooth(h, L, h->post, u, rhs, s);
}

// FMG over the global levels (Fig. "Full multigrid"); ftop / utop are the
// finest global level's f and u when there are no SR levels
template <typename T>
int run_fmg_global(sr_fmg_s* h, Hier<T>& H, const T* ftop, T* utop, cudaStream_t s) {
  const int top = h->G - 1;
  const bool plain = h->K == 0;
  auto fg = [&](int g) -> const T* { return (g == top && plain) ? ftop : H.glev[g].f; };
  auto ug = [&](int g) -> T* { return (g == top && plain) ? utop : H.glev[g].u; };
  {
    const int rc = coarse_solve<T>(h, H.glev[0], view_global<T>(H.glev[0], fg(0)), ug(0), s);
    if (rc) return rc;
  }
  const double w = sizeof(T);
  for (int g = 1; g <= top; ++g) {
    Level<T>& L = H.glev[g];
    LAUNCH(h, kind_of<T>(kProlongSet), L.tot_prolong, 3.75, 1.125 * w, s,
           launch_prolong<T>(H.glev[g - 1].view, ug(g - 1), L.view, ug(g), 0, s));
    FieldT<T> f = view_global<T>(L, fg(g));
    const T* r_first = nullptr;
    int rc = fmg_step(h, L, ug(g), f, s, &r_first);
    if (rc) return rc;
    rc = vcycle_global(h, H, g, ug(g), f, s, r_first);
    if (rc) return rc;
  }
  return SR_OK;
}

// f_{k-1} = average of f_k down all levels, from the finest f (n^3)
template <typename T>
int f_hierarchy(sr_fmg_s* h, Hier<T>& H, const T* f, int check, cudaStream_t s) {
  const T* src = f;
  Dims dsrc{h->cfg.n * h->len[0], h->cfg.n * h->len[1], h->cfg.n * h->len[2]};
  const double w = sizeof(T);
  for (int k = h->K - 1; k >= 1; --k) {
    const double cells = (double)cells_of(H.slev[k]);
    LAUNCH(h, kind_of<T>(kRestrictF), cells, 8, 9 * w, s,
           launch_restrict_global<T>(dsrc, src, H.slev[k].f, check, h->status, s));
    check = 0;
    src = H.slev[k].f;
    dsrc = dims_of(H.slev[k]);
  }
  for (int g = h->G - (h->K ? 1 : 2); g >= 0; --g) {
    const double cells = (double)cells_of(H.glev[g]);
    LAUNCH(h, kind_of<T>(kRestrictF), cells, 8, 9 * w, s,
           launch_restrict_global<T>(dsrc, src, H.glev[g].f, check, h->status, s));
    check = 0;
    src = H.glev[g].f;
    dsrc = dims_of(H.glev[g]);
  }
  return SR_OK;
}

// level j (below stage k's top) runs as a segment-resident leg in this solve
template <typename T>
bool leg_on(const sr_fmg_s* h, int j, int k) {
  if constexpr (sizeof(T) == 4) {
    return h->legs_on && j >= 1 && j < k && j < (int)h->legs.size() && h->legs[j].C > 0;
  }
  return false;
}

// algorithmic counts of a leg per compute cell: floating-point operations
// (smoother 14, restriction 42 per coarse cell / prolongation about 3.75,
// correction 1) and bytes (down: u read and written, rhs, the coarse uhat
// and rho; up: u read and written, rhs, t, e, the coarse e)
constexpr double kLegDownOps = 14.0 + 42.0 / 8, kLegDownBytes = 12.0 + 1.0;
constexpr double kLegUpOps = 14.0 + 3.75 + 1.0, kLegUpBytes = 20.0 + 0.5;

// SR stage k, first half: the FMG prolongation onto level k and S^alpha,
// then the down-leg of FASMGVSR(k) to the transition level, where every
// segment owner-writes its genuine level-0 cells of \hat I u_1 (into t_0) and
// of the restricted residual (rho_0)
template <typename T>
int sr_stage_down(sr_fmg_s* h, Hier<T>& H, const T* f, int k, cudaStream_t s) {
  const int K = h->K;
  Level<T>& L0 = H.glev[h->G - 1];
  const double w = sizeof(T);
  auto fview = [&](int j) -> FieldT<T> {
    return view_global<T>(H.slev[j], j == K ? f : H.slev[j].f);
  };
  Level<T>& Lk = H.slev[k];
  // u_k <- Pi u_{k-1} on Omega^C_k u Omega^GSR_k, then S^alpha on Omega^C_k
  const T* r_first = nullptr;
  {
    const Level<T>& C = (k == 1) ? L0 : H.slev[k - 1];
    LAUNCH(h, kind_of<T>(kProlongSet), Lk.tot_prolong, 3.75, 1.125 * w, s,
           launch_prolong<T>(C.view, C.u, Lk.view, Lk.u, 0, s));
    int rc = fmg_step(h, Lk, Lk.u, fview(k), s, &r_first);
    if (rc) return rc;
  }
  // FASMGVSR(k): down-leg
  for (int j = k; j >= 1; --j) {
    Level<T>& Lj = H.slev[j];
    Level<T>& C = (j > 1) ? H.slev[j - 1] : L0;
    T* uhat = (j > 1) ? C.u : L0.t;  // the transition level owner-writes into t_0
    bool leg = false;
    if constexpr (sizeof(T) == 4) leg = leg_on<T>(h, j, k);
    if (leg) {
      // the pre-smoother and the restriction of level j in one cluster launch
      // per segment box (float32 only)
      if constexpr (sizeof(T) == 4) {
        const sr_fmg_s::Leg& g = h->legs[j];
        LAUNCH(h, kLegDownF32, Lj.tot_cells, kLegDownOps, kLegDownBytes, s,
               launch_leg_down(Lj.view, C.view, Lj.u, Lj.rhs, uhat, C.rho, h->pre.a, h->pre.b,
                               g.C, g.max_planes, g.smem, h->status, h->force_timeout, s));
      }
    } else {
      const FieldT<T> rhs = (j == k) ? fview(k) : view_boxes<T>(Lj, Lj.rhs);
      // at the stage's top level the first residual may come from the fused
      // FMG step; below it, with the level's right-hand side (float64)
      const T* rf = (j == k) ? r_first : (kFirstResidual<T> ? Lj.r : nullptr);
      int rc = smooth(h, Lj, h->pre, Lj.u, rhs, s, rf);
      if (rc) return rc;
      rc = resid_restrict<T>(h, Lj, Lj.u, rhs, C, uhat, C.rho, s);
      if (rc) return rc;
    }
    if (j > 1) {
      const bool cr = kFirstResidual<T>;
      LAUNCH(h, kind_of<T>(kCoarseRhs), C.tot_cells, ops_rhs(h) + (cr ? 1 : 0), (cr ? 5 : 4) * w,
             s,
             op_coarse_rhs<T>(h, C.view, Lj.view, C.u, C.rho, C.rhs, C.t, cr ? C.r : nullptr, s));
      LAUNCH(h, kind_of<T>(kShellCopy), C.tot_cells / 4, 0, 2 * w, s,
             launch_shell_copy<T>(C.view, C.u, C.t, s));
    }
  }
  return SR_OK;
}

// SR stage k, second half (t_0 and rho_0 complete on the whole transition
// level): u_0 <- t_0, r_0 = rho_0 + L_0 u_0, the global FASMGV, then the
// up-leg (corrections onto Omega^C u Omega^GSR and S^nu2) back to level k
template <typename T>
int sr_stage_up(sr_fmg_s* h, Hier<T>& H, const T* f, int k, cudaStream_t s) {
  const int K = h->K;
  Level<T>& L0 = H.glev[h->G - 1];
  const double w = sizeof(T);
  auto fview = [&](int j) -> FieldT<T> {
    return view_global<T>(H.slev[j], j == K ? f : H.slev[j].f);
  };
  // level 0 is solved directly and needs no residual
  const bool cr = kFirstResidual<T> && h->G - 1 >= 1;
  LAUNCH(h, kind_of<T>(kTransitionRhs), L0.tot_cells, ops_rhs(h) + (cr ? 1 : 0), (cr ? 5 : 4) * w,
         s, op_transition_rhs<T>(h, L0.view, L0.t, L0.rho, L0.u, L0.rhs, cr ? L0.r : nullptr, s));
  int rc = vcycle_global(h, H, h->G - 1, L0.u, view_global<T>(L0, L0.rhs), s, cr ? L0.r : nullptr);
  if (rc) return rc;
  // up-leg
  for (int j = 1; j <= k; ++j) {
    Level<T>& Lj = H.slev[j];
    const Level<T>& C = (j == 1) ? L0 : H.slev[j - 1];
    if constexpr (sizeof(T) == 4) {
      // level j-1's leg has formed e_{j-1} = w - t already
      const bool have_e = j > 1 && leg_on<T>(h, j - 1, k);
      if (leg_on<T>(h, j, k)) {
        if (!have_e)
          LAUNCH(h, kind_of<T>(kDiff), C.tot_cells, 1, 3 * w, s,
                 launch_diff<T>(C.view, C.u, C.t, C.rho, s));
        // correction, post-smoother and level j's own w - t in one cluster
        // launch per segment box
        const sr_fmg_s::Leg& g = h->legs[j];
        LAUNCH(h, kLegUpF32, Lj.tot_cells, kLegUpOps, kLegUpBytes, s,
               launch_leg_up(Lj.view, C.view, Lj.u, Lj.t, Lj.rhs, C.rho, Lj.rho, h->post.a,
                             h->post.b, g.C, g.max_planes, g.smem, h->status, h->force_timeout,
                             s));
        continue;
      }
      if (have_e) {
        // the correction onto level j (a separate-kernel level) from the
        // leg's e_{j-1}
        const FieldT<T> rhs = (j == k) ? fview(k) : view_boxes<T>(Lj, Lj.rhs);
        const bool last = k == K && h->post.nu == 2 && h->trim;
        if (last) {
          const Geom& TR = (j == K) ? H.trim_r : H.ctrim_r[j];
          const Geom& TU = (j == K) ? H.trim_u : H.ctrim_u[j];
          LAUNCH(h, kind_of<T>(kProlongAdd), TR.tot_prolong, 3.75, 2.125 * w, s,
                 launch_prolong<T>(C.view, C.rho, TR.view, Lj.u, 1, s));
          LAUNCH(h, kind_of<T>(kChebResidual), TR.tot_cells, ops_smooth(h), 3 * w, s,
                 op_cheb_residual<T>(h, TR.view, Lj.u, Lj.r, rhs, s));
          LAUNCH(h, kind_of<T>(kCheb2Update), TU.tot_cells, ops_smooth(h), 3 * w, s,
                 op_cheb2_update<T>(h, TU.view, Lj.u, Lj.r, h->post, s));
          continue;
        }
        LAUNCH(h, kind_of<T>(kProlongAdd), Lj.tot_prolong, 3.75, 2.125 * w, s,
               launch_prolong<T>(C.view, C.rho, Lj.view, Lj.u, 1, s));
        rc = smooth(h, Lj, h->post, Lj.u, rhs, s);
        if (rc) return rc;
        continue;
      }
    }
    // The solve's last operations: only the finest level's genuine cells
    // are returned.  After its correction they depend on u within two
    // cells and on r within one cell of them; the correction reads the
    // level below on the cells U its prolongation touches, which depend
    // on that level's u and r within two and one cells of U, and so on
    // down the SR levels.  In the last stage the correction, the residual
    // and the update of every SR level therefore run on those regions only
    // (every value they keep is computed exactly as on the full box).
    const bool last = k == K && h->post.nu == 2 && h->trim;
    if (last && j >= 2) {
      const Geom& D = H.ctrim_u[j - 1];
      LAUNCH(h, kind_of<T>(kDiff), D.tot_prolong, 1, 3 * w, s,
             launch_diff<T>(D.view, C.u, C.t, C.rho, s, 1));
    } else {
      LAUNCH(h, kind_of<T>(kDiff), C.tot_cells, 1, 3 * w, s,
             launch_diff<T>(C.view, C.u, C.t, C.rho, s));
    }
    const FieldT<T> rhs = (j == k) ? fview(k) : view_boxes<T>(Lj, Lj.rhs);
    if (last) {
      const Geom& TR = (j == K) ? H.trim_r : H.ctrim_r[j];
      const Geom& TU = (j == K) ? H.trim_u : H.ctrim_u[j];
      LAUNCH(h, kind_of<T>(kProlongAdd), TR.tot_prolong, 3.75, 2.125 * w, s,
             launch_prolong<T>(C.view, C.rho, TR.view, Lj.u, 1, s));
      LAUNCH(h, kind_of<T>(kChebResidual), TR.tot_cells, ops_smooth(h), 3 * w, s,
             op_cheb_residual<T>(h, TR.view, Lj.u, Lj.r, rhs, s));
      LAUNCH(h, kind_of<T>(kCheb2Update), TU.tot_cells, ops_smooth(h), 3 * w, s,
             op_cheb2_update<T>(h, TU.view, Lj.u, Lj.r, h->post, s));
      continue;
    }
    LAUNCH(h, kind_of<T>(kProlongAdd), Lj.tot_prolong, 3.75, 2.125 * w, s,
           launch_prolong<T>(C.view, C.rho, Lj.view, Lj.u, 1, s));
    rc = smooth(h, Lj, h->post, Lj.u, rhs, s);
    if (rc) return rc;
  }
  return SR_OK;
}

// genuine finest cells of the handle's segments into u (add == 0) or added
// to it (add == 1)
template <typename T>
int sr_gather(sr_fmg_s* h, Hier<T>& H, double* u, int add, cudaStream_t s) {
  const double w = sizeof(T);
  const int K = h->K;
  LAUNCH(h, kind_of<T>(kGather), H.slev[K].tot_genuine, add ? 1 : 0, w + (add ? 16 : 8), s,
         launch_gather_genuine<T>(H.slev[K].view, H.slev[K].u, u, add, s));
  return SR_OK;
}

// the SR stages k = 1..K after the global FMG; the genuine finest cells go to
// u (add == 0) or are added to it (add == 1)
template <typename T>
int run_sr(sr_fmg_s* h, Hier<T>& H, const T* f, double* u, int add, cudaStream_t s) {
  for (int k = 1; k <= h->K; ++k) {
    int rc = sr_stage_down<T>(h, H, f, k, s);
    if (!rc) rc = sr_stage_up<T>(h, H, f, k, s);
    if (rc) return rc;
  }
  return sr_gather<T>(h, H, u, add, s);
}

// one FMG / SR-FMG solve of A x = f in storage type T.  With T = double and
// no SR levels the solve works in the caller's out directly; otherwise the
// result goes to out (add == 1: out += x).
template <typename T>
int solve_once(sr_fmg_s* h, const T* f, double* out, int add, int check, cudaStream_t s) {
  Hier<T>& H = h->hier((T*)nullptr);
  int rc = f_hierarchy<T>(h, H, f, check, s);
  if (rc) return rc;
  const bool user_top = (sizeof(T) == 8) && h->K == 0;
  T* utop = user_top ? reinterpret_cast<T*>(out) : H.glev[h->G - 1].u;
  rc = run_fmg_global<T>(h, H, f, utop, s);
  if (rc) return rc;
  if (h->K) return run_sr<T>(h, H, f, out, add, s);
  if (!user_top) {
    const long long cells = cells_of(H.glev[h->G - 1]);
    LAUNCH(h, kAccumulate, (double)cells, add ? 1 : 0, add ? 20 : 12, s,
           launch_accumulate(cells, reinterpret_cast<const float*>(utop), out, add, s));
  }
  return SR_OK;
}

int enqueue_solve(sr_fmg_s* h, const double* f, double* u, cudaStream_t s) {
  if (h->sharded) return SR_ERR_INVALID;  // a segment range solves stage by stage
  h->launches = 0;
  if (!h->mixed) return solve_once<double>(h, f, u, 0, 1, s);
  // float64 defect correction around the float32 solve
  const int n = h->cfg.n;
  const Dims g{n * h->len[0], n * h->len[1], n * h->len[2]};
  const double cells = (double)g.x * g.y * g.z;
  const int passes = h->cfg.n_outer > 0 ? h->cfg.n_outer : 2;
  for (int p = 1; p <= passes; ++p) {
    LAUNCH(h, kDefect, cells, p == 1 ? 0 : 7, p == 1 ? 12 : 20, s,
           launch_defect(g, n, f, p == 1 ? nullptr : u, h->defect, h->status, s));
    int rc = solve_once<float>(h, h->defect, u, p > 1 ? 1 : 0, 0, s);
    if (rc) return rc;
  }
  return SR_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool dev_ok_any(const void* p) { return p && is_device_ptr(p); }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void free_all(sr_fmg_s* h) {
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    cudaFree(h->allocs[i]);
    g_live_bytes -= (long long)h->alloc_bytes[i];
  }
  h->allocs.clear();
  h->alloc_bytes.clear();
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  for (ProfRec& r : h->prof.recs) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  h->prof.pool.clear();
  h->prof.recs.clear();
}

// fold recorded launches into the per-kind totals (after the stream is idle)
int collect_profile(sr_fmg_s* h) {
  for (ProfRec& r : h->prof.recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return SR_ERR_CUDA;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return SR_ERR_CUDA;
    h->prof.launches[r.kind] += 1;
    h->prof.ms[r.kind] += ms;
    h->prof.ops[r.kind] += r.ops;
    h->prof.bytes[r.kind] += r.bytes;
    h->prof.pool.push_back(r.e0);
    h->prof.pool.push_back(r.e1);
  }
  h->prof.recs.clear();
  return SR_OK;
}

}  // namespace

// the solve queued kernel by kernel, or (graph mode, profiler off) as the
// handle's captured graph
static int queue_solve(sr_fmg_s* h, const double* f, double* u, cudaStream_t s) {
  if (!h->cfg.graph || h->prof.on) return enqueue_solve(h, f, u, s);
  constexpr size_t kGraphs = 4;
  for (const sr_fmg_s::GraphEntry& g : h->graphs)
    if (g.f == f && g.u == u) return sr_fmg_batch_solve_async(g.b, &f, &u, s);
  if (h->graphs.size() >= kGraphs) {  // the oldest pair's graph goes (freed once idle)
    sr_fmg_batch_destroy(h->graphs.front().b);
    h->graphs.erase(h->graphs.begin());
  }
  sr_fmg_batch_t b = nullptr;
  int rc = sr_fmg_batch_create(&b, &h, 1);
  if (rc) return rc;
  h->graphs.push_back({f, u, b});
  return sr_fmg_batch_solve_async(b, &f, &u, s);
}

// release the pipelined-host-solve resources
void free_pipeline(sr_fmg_s* h) {
  if (h->cin) cudaStreamDestroy(h->cin);
  if (h->cout) cudaStreamDestroy(h->cout);
  for (int k = 0; k < 2; ++k) {
    if (h->ev_in[k]) cudaEventDestroy(h->ev_in[k]);
    if (h->ev_solved[k]) cudaEventDestroy(h->ev_solved[k]);
    if (h->ev_out[k]) cudaEventDestroy(h->ev_out[k]);
  }
}

int srfmg::enqueue_solve_unchecked(sr_fmg_s* h, const double* f, double* u, cudaStream_t s) {
  DeviceGuard g(h->device);
  return enqueue_solve(h, f, u, s);
}

long long srfmg::handle_generation(const sr_fmg_s* h) { return h->generation; }

// the handle's launch sequence changes: its captured graphs go, and batches
// holding it re-capture theirs
static void sequence_changed(sr_fmg_s* h) {
  for (const sr_fmg_s::GraphEntry& e : h->graphs) sr_fmg_batch_destroy(e.b);
  h->graphs.clear();
  ++h->generation;
}

template <typename T>
static void set_shape(Hier<T>& H, int zchunk, int cpt) {
  auto apply = [&](Geom& g) {
    g.view.zchunk = zchunk;
    g.view.cpt = cpt;
  };
  for (Geom& g : H.glev) apply(g);
  for (Geom& g : H.slev) apply(g);
  apply(H.trim_r);
  apply(H.trim_u);
  for (Geom& g : H.ctrim_r) apply(g);
  for (Geom& g : H.ctrim_u) apply(g);
}


long long srfmg::handle_cells(const sr_fmg_s* h) {
  return (long long)h->cfg.n * h->cfg.n * h->cfg.n * h->len[0] * h->len[1] * h->len[2];
}

extern "C" {

void sr_fmg_default_config(sr_fmg_config* cfg, int n) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n = n;
  cfg->n_coarse = 0;
  cfg->seg = 0;
  cfg->K = 0;
  cfg->A = 8;
  cfg->B = 0;
  cfg->use_J = 0;
  cfg->alpha = 1;
  cfg->nu1 = 2;
  cfg->nu2 = 2;
  cfg->cheb_lo = 1.0 / 6.0;
  cfg->cheb_hi = 1.0;
  cfg->precision = SR_FP64;
  cfg->n_outer = 2;
}

int sr_fmg_create(sr_fmg_t* out, const sr_fmg_config* cfg) {
  if (!out) return SR_ERR_INVALID;
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return SR_ERR_NO_DEVICE;
  }
  sr_fmg_s* h = new (std::nothrow) sr_fmg_s();
  if (!h) return SR_ERR_OOM;
  h->cfg = *cfg;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return SR_ERR_CUDA;
  }
  h->mixed = cfg->precision == SR_MIXED;
  h->K = (cfg->seg > 0) ? cfg->K : 0;
  h->sharded = cfg->seg_count > 0;
  lengths_of(cfg, h->len);
  op_weights(cfg, &h->w27, &h->lmax);
  h->op27 = cfg->stencil == 27;
  h->pre = chebyshev(cfg->nu1, cfg->cheb_lo, cfg->cheb_hi, h->lmax);
  h->post = chebyshev(cfg->nu2, cfg->cheb_lo, cfg->cheb_hi, h->lmax);
  h->fmg = chebyshev(cfg->alpha, cfg->cheb_lo, cfg->cheb_hi, h->lmax);
  rc = dalloc(h, &h->status, 1);
  if (!h->mixed) {
    if (!rc) rc = build_global_levels<double>(h, h->h64, cfg->n >> h->K, h->K == 0);
    if (!rc && h->K) rc = build_sr_levels<double>(h, h->h64);
    if (!rc) rc = plan_persistent(h);
  } else {
    const size_t cells = (size_t)srfmg::handle_cells(h);
    if (!rc) rc = dalloc(h, &h->defect, cells);
    if (!rc) rc = build_global_levels<float>(h, h->h32, cfg->n >> h->K, false);
    if (!rc && h->K) rc = build_sr_levels<float>(h, h->h32);
    if (!rc && h->K) rc = plan_legs(h);
  }
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return SR_OK;
}

int sr_fmg_destroy(sr_fmg_t h) {
  if (!h) return SR_OK;
  DeviceGuard g(h->device);
  for (const sr_fmg_s::GraphEntry& e : h->graphs) sr_fmg_batch_destroy(e.b);
  free_pipeline(h);
  free_all(h);
  delete h;
  return SR_OK;
}

int sr_fmg_workspace_bytes(sr_fmg_t h, size_t* bytes) {
  if (!h || !bytes) return SR_ERR_INVALID;
  *bytes = h->bytes;
  return SR_OK;
}

int sr_fmg_solve_async(sr_fmg_t h, const double* f_dev, double* u_dev, void* stream) {
  if (!h || !f_dev || !u_dev) return SR_ERR_INVALID;
  const char* fa = (const char*)f_dev;
  const char* ua = (const char*)u_dev;
  const size_t bytes = (size_t)srfmg::handle_cells(h) * sizeof(double);
  if (fa < ua + bytes && ua < fa + bytes) return SR_ERR_INVALID;
  if (!is_device_ptr(f_dev) || !is_device_ptr(u_dev)) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  return queue_solve(h, f_dev, u_dev, (cudaStream_t)stream);
}

int sr_fmg_check(sr_fmg_t h, void* stream) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned int st = 0;
  CK(cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  // the status accumulates over the solves since the previous check
  CK(cudaMemset(h->status, 0, sizeof(st)));
  if (st & 1u) return SR_ERR_NONFINITE;
  if (st & 2u) return SR_ERR_TIMEOUT;
  return SR_OK;
}

int sr_fmg_solve_host_async(sr_fmg_t h, const double* f_host, double* u_host, void* stream) {
  if (!h || !f_host || !u_host) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  const size_t cells = (size_t)srfmg::handle_cells(h);
  const size_t bytes = cells * sizeof(double);
  if (!h->cin) {
    // staging slots (a retry after a failed allocation keeps what it got)
    int rc = SR_OK;
    for (int k = 0; k < 2 && !rc; ++k) {
      if (!h->pf[k]) rc = dalloc(h, &h->pf[k], cells);
      if (!rc && !h->pu[k]) rc = dalloc(h, &h->pu[k], cells);
    }
    if (rc) return rc;
    CK(cudaStreamCreateWithFlags(&h->cin, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&h->cout, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CK(cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->ev_solved[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming));
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int k = h->pslot;
  h->pslot ^= 1;
  // copy in on its own stream once the solve that last read this slot is done
  if (h->pused[k]) CK(cudaStreamWaitEvent(h->cin, h->ev_solved[k], 0));
  CK(cudaMemcpyAsync(h->pf[k], f_host, bytes, cudaMemcpyHostToDevice, h->cin));
  CK(cudaEventRecord(h->ev_in[k], h->cin));
  // solve on the caller's stream once the copy is in and the slot's previous
  // result has been copied out
  CK(cudaStreamWaitEvent(s, h->ev_in[k], 0));
  if (h->pused[k]) CK(cudaStreamWaitEvent(s, h->ev_out[k], 0));
  int rc = queue_solve(h, h->pf[k], h->pu[k], s);
  if (rc) return rc;
  CK(cudaEventRecord(h->ev_solved[k], s));
  // copy out on its own stream
  CK(cudaStreamWaitEvent(h->cout, h->ev_solved[k], 0));
  CK(cudaMemcpyAsync(u_host, h->pu[k], bytes, cudaMemcpyDeviceToHost, h->cout));
  CK(cudaEventRecord(h->ev_out[k], h->cout));
  h->pused[k] = true;
  h->last = s;
  return SR_OK;
}

int sr_fmg_check_host(sr_fmg_t h) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  if (h->cout) CK(cudaStreamSynchronize(h->cout));
  return sr_fmg_check(h, h->last);
}

int sr_fmg_solve(sr_fmg_t h, const double* f_dev, double* u_dev, void* stream) {
  int rc = sr_fmg_solve_async(h, f_dev, u_dev, stream);
  if (rc) return rc;
  return sr_fmg_check(h, stream);
}

int sr_fmg_solve_host(sr_fmg_t h, const double* f_host, double* u_host, void* stream) {
  if (!h || !f_host || !u_host) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  const size_t cells = (size_t)srfmg::handle_cells(h);
  const size_t bytes = cells * sizeof(double);
  {
    int rc = h->hbuf_f ? SR_OK : dalloc(h, &h->hbuf_f, cells);
    if (!rc && !h->hbuf_u) rc = dalloc(h, &h->hbuf_u, cells);
    if (rc) return rc;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->hbuf_f, f_host, bytes, cudaMemcpyHostToDevice, s));
  int rc = queue_solve(h, h->hbuf_f, h->hbuf_u, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(u_host, h->hbuf_u, bytes, cudaMemcpyDeviceToHost, s));
  return sr_fmg_check(h, stream);
}

int sr_fmg_vsolve(sr_fmg_t h, const double* f_dev, double* u_dev, double rtol, int max_cycles,
                  int* cycles, double* rel_resid, void* stream) {
  if (!h || !f_dev || !u_dev || !cycles || !rel_resid) return SR_ERR_INVALID;
  if (h->K || h->mixed || !(rtol >= 0.0) || max_cycles < 0) return SR_ERR_INVALID;
  const int n = h->cfg.n;
  const size_t bytes = (size_t)srfmg::handle_cells(h) * sizeof(double);
  const char* fa = (const char*)f_dev;
  const char* ua = (const char*)u_dev;
  if (fa < ua + bytes && ua < fa + bytes) return SR_ERR_INVALID;
  if (!is_device_ptr(f_dev) || !is_device_ptr(u_dev)) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  if (!h->norms) {
    int rc = dalloc(h, &h->norms, 2);
    if (rc) return rc;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int top = h->G - 1;
  Hier<double>& H = h->h64;
  const double cells = (double)cells_of(H.glev[top]);
  *cycles = 0;
  h->launches = 0;
  // one norm into slot k (u == nullptr: ||f||), read back on the host
  auto norm = [&](const double* u, int k, double* out) -> int {
    CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned int), s));
    CK(cudaMemsetAsync(h->norms + k, 0, sizeof(unsigned long long), s));
    if (h->op27) {
      LAUNCH(h, kResidNorm, cells, u ? ops_rhs(h) : 0, u ? 16 : 8, s,
             launch27_resid_norm(H.glev[top].view, f_dev, u, h->norms + k, h->status, h->w27,
                                 s));
    } else {
      LAUNCH(h, kResidNorm, cells, u ? 7 : 0, u ? 16 : 8, s,
             launch_resid_norm(dims_of(H.glev[top]), n, f_dev, u, h->norms + k, h->status, s));
    }
    unsigned long long bits = 0;
    unsigned int st = 0;
    CK(cudaMemcpyAsync(&bits, h->norms + k, sizeof(bits), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st & 1u) return SR_ERR_NONFINITE;
    std::memcpy(out, &bits, sizeof(*out));
    return SR_OK;
  };
  double fnorm = 0.0, r = 0.0;
  int rc = norm(nullptr, 0, &fnorm);
  if (rc) return rc;
  if ((rc = norm(u_dev, 1, &r))) return rc;
  const FieldT<double> fv = view_global<double>(H.glev[top], f_dev);
  for (;;) {
    const double q = fnorm > 0.0 ? r / fnorm : (r > 0.0 ? HUGE_VAL : 0.0);
    *rel_resid = q;
    if (q <= rtol || *cycles >= max_cycles) break;
    if ((rc = vcycle_global<double>(h, H, top, u_dev, fv, s))) return rc;
    ++*cycles;
    if ((rc = norm(u_dev, 1, &r))) return rc;
  }
  return SR_OK;
}

int sr_fmg_stage_down(sr_fmg_t h, const double* f_dev, int k, void* stream) {
  if (!h || !f_dev || h->mixed || h->K == 0 || k < 1 || k > h->K) return SR_ERR_INVALID;
  if (!is_device_ptr(f_dev)) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  Hier<double>& H = h->h64;
  if (k == 1) {  // the f hierarchy and the global FMG up to the transition level
    h->launches = 0;
    int rc = f_hierarchy<double>(h, H, f_dev, 1, s);
    if (!rc) rc = run_fmg_global<double>(h, H, f_dev, nullptr, s);
    if (rc) return rc;
  }
  // the exchange arrays hold this handle's genuine cells only: clear them
  const Level<double>& L0 = H.glev[h->G - 1];
  const size_t bytes = (size_t)cells_of(L0) * sizeof(double);
  CK(cudaMemsetAsync(L0.t, 0, bytes, s));
  CK(cudaMemsetAsync(L0.rho, 0, bytes, s));
  return sr_stage_down<double>(h, H, f_dev, k, s);
}

int sr_fmg_stage_buffers(sr_fmg_t h, double** uhat0, double** rho0, size_t* count) {
  if (!h || !uhat0 || !rho0 || !count || h->mixed || h->K == 0) return SR_ERR_INVALID;
  const Level<double>& L0 = h->h64.glev[h->G - 1];
  *uhat0 = L0.t;
  *rho0 = L0.rho;
  *count = (size_t)cells_of(L0);
  return SR_OK;
}

int sr_fmg_stage_up(sr_fmg_t h, const double* f_dev, int k, double* u_dev, void* stream) {
  if (!h || !f_dev || h->mixed || h->K == 0 || k < 1 || k > h->K) return SR_ERR_INVALID;
  if (k == h->K && (!u_dev || !is_device_ptr(u_dev))) return SR_ERR_INVALID;
  if (!is_device_ptr(f_dev)) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = sr_stage_up<double>(h, h->h64, f_dev, k, s);
  if (!rc && k == h->K) rc = sr_gather<double>(h, h->h64, u_dev, 0, s);
  return rc;
}

int sr_fmg_launches_per_solve(sr_fmg_t h, int* launches) {
  if (!h || !launches) return SR_ERR_INVALID;
  *launches = h->launches;
  return SR_OK;
}

int sr_fmg_profile(sr_fmg_t h, int enable) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return SR_ERR_CUDA;
  int rc = collect_profile(h);
  if (rc) return rc;
  if (enable) {
    for (int k = 0; k < kKinds; ++k) {
      h->prof.launches[k] = 0;
      h->prof.ms[k] = h->prof.ops[k] = h->prof.bytes[k] = 0.0;
    }
  }
  h->prof.on = enable != 0;
  return SR_OK;
}

int sr_fmg_profile_kinds(void) { return kKinds; }

int sr_fmg_profile_read(sr_fmg_t h, int kind, const char** name, long long* launches,
                        double* ms, double* ops, double* bytes) {
  if (!h || kind < 0 || kind >= kKinds) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  int rc = collect_profile(h);
  if (rc) return rc;
  if (name) *name = kKindName[kind];
  if (launches) *launches = h->prof.launches[kind];
  if (ms) *ms = h->prof.ms[kind];
  if (ops) *ops = h->prof.ops[kind];
  if (bytes) *bytes = h->prof.bytes[kind];
  return SR_OK;
}

int sr_debug_fail_alloc(int nth) {
  if (nth < 0) return SR_ERR_INVALID;
  g_fail_countdown.store(nth);
  return SR_OK;
}

long long sr_debug_alloc_count(void) { return g_allocs.load(); }

int sr_debug_narrow(const double* in, float* out, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!dev_ok_any(in) || !dev_ok_any(out)))) return SR_ERR_INVALID;
  if (n == 0) return SR_OK;
  CK(launch_narrow(in, out, n, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SR_OK;
}

int sr_fmg_set_launch_shape(sr_fmg_t h, int zchunk, int cells_per_thread) {
  if (!h || zchunk < 1 || zchunk > 256 || cells_per_thread < 1 || cells_per_thread > 16)
    return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  h->zchunk = zchunk;
  h->cpt = cells_per_thread;
  set_shape(h->h64, zchunk, cells_per_thread);
  set_shape(h->h32, zchunk, cells_per_thread);
  sequence_changed(h);
  return SR_OK;
}

int sr_fmg_launch_shape(sr_fmg_t h, int* zchunk, int* cells_per_thread) {
  if (!h || !zchunk || !cells_per_thread) return SR_ERR_INVALID;
  *zchunk = h->zchunk;
  *cells_per_thread = h->cpt;
  return SR_OK;
}

int sr_debug_segment_legs(sr_fmg_t h, int enable, int* levels) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  sequence_changed(h);
  h->legs_on = enable != 0;
  if (levels) {
    *levels = 0;
    for (size_t j = 1; j < h->legs.size(); ++j)
      if (h->legs[j].C > 0) *levels |= 1 << j;
  }
  return SR_OK;
}

int sr_debug_persistent_vcycle(sr_fmg_t h, int enable, int* available) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  sequence_changed(h);
  h->persistent_on = enable != 0;
  if (available) *available = h->persistent ? 1 : 0;
  return SR_OK;
}

int sr_debug_force_wait_timeout(sr_fmg_t h, int enable) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  sequence_changed(h);
  h->force_timeout = enable != 0;
  return SR_OK;
}

int sr_debug_last_stage_trim(sr_fmg_t h, int enable) {
  if (!h) return SR_ERR_INVALID;
  DeviceGuard g(h->device);
  sequence_changed(h);
  h->trim = enable != 0;
  return SR_OK;
}

long long sr_debug_live_bytes(void) { return g_live_bytes.load(); }

const char* sr_fmg_status_string(int status) {
  switch (status) {
    case SR_OK: return "ok";
    case SR_ERR_INVALID: return "invalid argument or configuration";
    case SR_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case SR_ERR_OOM: return "out of memory";
    case SR_ERR_CUDA: return "CUDA error";
    case SR_ERR_TIMEOUT: return "device wait timed out";
    case SR_ERR_NONFINITE: return "right-hand side is not finite";
    case SR_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------
// single components on whole grids (float64)

namespace {

struct TmpLevel {
  sr_fmg_s h;
  Level<double> L;
  ~TmpLevel() { free_all(&h); }
};

// a handle shell carrying cfg's domain and operator, and one whole level of
// n cells per unit length
int tmp_level(TmpLevel& T, const sr_fmg_config& c, int n) {
  if (lengths_of(&c, T.h.len) || op_weights(&c, &T.h.w27, &T.h.lmax)) return SR_ERR_INVALID;
  T.h.op27 = c.stencil == 27;
  set_dims(T.L, n, T.h.len);
  T.L.hboxes.assign(1, whole_box(T.L.nd));
  return finish_level(&T.h, T.L);
}

bool dev_ok(const void* p) { return p && is_device_ptr(p); }

sr_fmg_config cube7(int n) {
  sr_fmg_config c;
  sr_fmg_default_config(&c, n);
  return c;
}

}  // namespace

int sr_op_apply_ex(const sr_fmg_config* cfg, const double* u, double* out, void* stream) {
  if (!cfg || cfg->n < 1 || !dev_ok(u) || !dev_ok(out)) return SR_ERR_INVALID;
  TmpLevel T;
  int rc = tmp_level(T, *cfg, cfg->n);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CK(T.h.op27 ? launch27_apply(T.L.view, u, out, T.h.w27, s)
              : launch_apply<double>(T.L.view, u, out, s));
  CK(cudaStreamSynchronize(s));
  return SR_OK;
}

int sr_op_residual_ex(const sr_fmg_config* cfg, const double* f, const double* u, double* r,
                      void* stream) {
  if (!cfg || cfg->n < 1 || !dev_ok(f) || !dev_ok(u) || !dev_ok(r)) return SR_ERR_INVALID;
  TmpLevel T;
  int rc = tmp_level(T, *cfg, cfg->n);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const FieldT<double> fv = view_global<double>(T.L, f);
  CK(T.h.op27 ? launch27_residual(T.L.view, u, fv, r, T.h.w27, s)
              : launch_residual<double>(T.L.view, u, fv, r, s));
  CK(cudaStreamSynchronize(s));
  return SR_OK;
}

int sr_op_smooth_ex(const sr_fmg_config* cfg, int nu, const double* f, double* u, void* stream) {
  if (!cfg || cfg->n < 1 || nu < 0 || nu > 16 || !dev_ok(f) || !dev_ok(u)) return SR_ERR_INVALID;
  if (!(cfg->cheb_lo > 0.0 && cfg->cheb_hi > cfg->cheb_lo)) return SR_ERR_INVALID;
  TmpLevel T;
  int rc = tmp_level(T, *cfg, cfg->n);
  const size_t cells = (size_t)cells_of(T.L);
  if (!rc) rc = dalloc(&T.h, &T.L.r, cells);
  if (!rc) rc = dalloc(&T.h, &T.L.d, cells);
  if (rc) return rc;
  Cheb c = chebyshev(nu, cfg->cheb_lo, cfg->cheb_hi, T.h.lmax);
  rc = smooth<double>(&T.h, T.L, c, u, view_global<double>(T.L, f), (cudaStream_t)stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SR_OK;
}

int sr_op_restrict_ex(const sr_fmg_config* cfg, const double* a, double* ac, void* stream) {
  if (!cfg || cfg->n < 2 || cfg->n % 2 || !dev_ok(a) || !dev_ok(ac)) return SR_ERR_INVALID;
  TmpLevel T;
  int rc = tmp_level(T, *cfg, cfg->n);
  if (!rc) rc = dalloc(&T.h, &T.h.status, 1);
  if (rc) return rc;
  CK(launch_restrict_global<double>(dims_of(T.L), a, ac, 0, T.h.status, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SR_OK;
}

int sr_op_prolong_ex(const sr_fmg_config* cfg, const double* ac, double* af, void* stream) {
  if (!cfg || cfg->n < 1 || !dev_ok(ac) || !dev_ok(af)) return SR_ERR_INVALID;
  TmpLevel C, F;
  int rc = tmp_level(C, *cfg, cfg->n);
  if (!rc) rc = tmp_level(F, *cfg, 2 * cfg->n);
  if (rc) return rc;
  CK(launch_prolong<double>(C.L.view, ac, F.L.view, af, 0, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return SR_OK;
}

int sr_op_coarse_solve_ex(const sr_fmg_config* cfg, const double* f, double* u, void* stream) {
  if (!cfg || cfg->n < 1 || !dev_ok(f) || !dev_ok(u)) return SR_ERR_INVALID;
  TmpLevel T;
  int rc = tmp_level(T, *cfg, cfg->n);
  if (rc) return rc;
  CoarseOp op;
  if ((rc = build_coarse(&T.h, T.L.nd, T.L.n, T.h.w27, &op))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const FieldT<double> fv = view_global<double>(T.L, f);
  CK(op.minv ? launch_coarse_solve<double>(T.L.view, op.minv, fv, u, s)
             : launch_coarse_solve_sep<double>(T.L.view, op.sep, op.g, op.q, fv, u, s));
  CK(cudaStreamSynchronize(s));
  return SR_OK;
}

int sr_op_apply(int n, const double* u, double* out, void* stream) {
  const sr_fmg_config c = cube7(n);
  return sr_op_apply_ex(&c, u, out, stream);
}

int sr_op_residual(int n, const double* f, const double* u, double* r, void* stream) {
  const sr_fmg_config c = cube7(n);
  return sr_op_residual_ex(&c, f, u, r, stream);
}

int sr_op_smooth(int n, int nu, double cheb_lo, double cheb_hi, const double* f, double* u,
                 void* stream) {
  sr_fmg_config c = cube7(n);
  c.cheb_lo = cheb_lo;
  c.cheb_hi = cheb_hi;
  return sr_op_smooth_ex(&c, nu, f, u, stream);
}

int sr_op_restrict(int n, const double* a, double* ac, void* stream) {
  const sr_fmg_config c = cube7(n);
  return sr_op_restrict_ex(&c, a, ac, stream);
}

int sr_op_prolong(int nc, const double* ac, double* af, void* stream) {
  const sr_fmg_config c = cube7(nc);
  return sr_op_prolong_ex(&c, ac, af, stream);
}

int sr_op_coarse_solve(int n, const double* f, double* u, void* stream) {
  if (n > 32) return SR_ERR_INVALID;
  const sr_fmg_config c = cube7(n);
  return sr_op_coarse_solve_ex(&c, f, u, stream);
}

int sr_op_vcycle(const sr_fmg_config* cfg, const double* f, double* u, void* stream) {
  if (!cfg || !dev_ok(f) || !dev_ok(u)) return SR_ERR_INVALID;
  sr_fmg_config c = *cfg;
  c.seg = 0;
  c.K = 0;
  c.precision = SR_FP64;
  sr_fmg_t h = nullptr;
  int rc = sr_fmg_create(&h, &c);
  if (rc) return rc;
  const int top = h->G - 1;
  rc = vcycle_global<double>(h, h->h64, top, u, view_global<double>(h->h64.glev[top], f),
                             (cudaStream_t)stream);
  if (!rc && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = SR_ERR_CUDA;
  sr_fmg_destroy(h);
  return rc;
}

}  // extern "C"
