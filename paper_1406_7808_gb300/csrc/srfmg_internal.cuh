// Internal definitions shared by the solver's translation units: the box
// descriptors that describe where each level lives in device memory, and the
// launchers of the kernels (kernels.cu), instantiated for float64 (the FP64
// solver) and float32 (the inner solver of the mixed-precision mode).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

struct sr_fmg_s;  // solver handle (srfmg_api.cu)

namespace srfmg {

// One box of cells of a level grid.  A global level is a single box covering
// [0, n)^3 stored without a ghost shell; an SR level has one box per segment,
// stored with a one-cell ghost shell that holds the frozen SR ghost values.
// Element (x, y, z) of a box lives at
//   base + (z - oz) * sz + (y - oy) * sy + (x - ox)
// in every array of its level (offsets in elements, whatever the type).
struct BoxDesc {
  int lo[3], hi[3];    // compute region Omega^C
  int rlo[3], rhi[3];  // restriction target on the next coarser level
  int plo[3], phi[3];  // prolongation range Omega^C u Omega^GSR
  int glo[3], ghi[3];  // genuine region on this level
  int ox, oy, oz;      // storage origin (lo - 1 with a shell, 0 without)
  int sy;              // row stride
  long long sz;        // plane stride
  long long base;      // offset of the box's storage in the level arrays
};

// Cells per dimension of a whole level grid.
struct Dims {
  int x, y, z;
};

// A level as the kernels see it.  The domain is [0, l0] x [0, l1] x [0, l2]
// (unit cube by default) with n cells per unit length (h = 1/n); the level
// grid has nx x ny x nz = n l0 x n l1 x n l2 cells.
struct LevelView {
  const BoxDesc* boxes;  // device array, nbox entries
  int nbox;
  int n;                 // cells per unit length of the level grid
  int nx, ny, nz;        // cells per dimension of the level grid
  int max_cells;         // largest compute-region cell count over the boxes
  int max_stored;        // largest stored-region (compute plus shell) cell count
  int max_prolong;       // largest prolongation-range cell count
  int max_restrict;      // largest restriction-target cell count
  int max_genuine;       // largest genuine-region cell count
  int max_ex, max_ey, max_ez;  // largest compute-region extents
  int shell;             // 1: the boxes are stored with a one-cell shell (SR levels)
  // launch shape (results do not depend on it): cells in z a thread of a
  // z-column kernel walks, and cells a thread of a per-cell kernel takes
  int zchunk;            // default kDefaultZChunk
  int cpt;               // default kDefaultCellsPerThread
};

constexpr int kDefaultZChunk = 16, kDefaultCellsPerThread = 2;

// A field read with a possibly different layout than the level's boxes (the
// caller's global f on the finest SR level): single != 0 means every box
// reads through boxes[0].
template <typename T>
struct FieldT {
  const T* p;
  const BoxDesc* boxes;
  int single;
};
using FieldView = FieldT<double>;

// ---- launches.  Every kernel of the library is launched with programmatic
// stream serialization (Programmatic Dependent Launch): its grid may be
// scheduled while the kernel before it on the stream drains, and each of its
// blocks first waits, in grid_dep_wait, until that kernel has completed and
// its writes are visible.  As every block of every kernel waits before any
// other work (or early return), completion stays ordered along the stream.
// Launched without the attribute (or after a copy or an event) the wait
// returns at once.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// (x, y, z) of flat index i of an nx x ny x nz grid, C order.  Grids of
// fewer than 2^32 cells (up to 1625^3) take 32-bit divisions, several times
// cheaper than the 64-bit ones the integer pipe emulates.
__device__ __forceinline__ void split3(long long i, int nx, int ny, int& x, int& y, int& z) {
  if (i <= 0xffffffffLL) {
    const unsigned ui = (unsigned)i, t = ui / (unsigned)nx;
    x = (int)(ui - t * (unsigned)nx);
    y = (int)(t % (unsigned)ny);
    z = (int)(t / (unsigned)ny);
  } else {
    const long long t = i / nx;
    x = (int)(i - t * nx);
    y = (int)(t % ny);
    z = (int)(t / ny);
  }
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// return the launch status from the enclosing launcher on failure
#define SRFMG_LAUNCH(call)                         \
  do {                                             \
    const cudaError_t launch_status_ = (call);     \
    if (launch_status_ != cudaSuccess) return launch_status_; \
  } while (0)

enum Region { kCompute = 0, kProlong = 1, kRestrict = 2, kGenuine = 3 };

// lambda_max(D^-1 A) of the 7-point operator (D = 6 n^2): the DST mode with
// every wavenumber N has eigenvalue 12 n^2, i.e. 2 after D^-1
constexpr double kLambdaMax7 = 2.0;

// Chebyshev smoother S^nu on D^-1 A over [lo_frac, hi_frac] * lmax (Sec. 5.1):
// the three-term recurrence d_m = alpha_m d_{m-1} + beta_m r_m, u += d_m,
// and for nu = 2 the equivalent polynomial x2 = x0 + c1 r0 + c2 (D^-1 A) r0,
// stored as a = c1 + c2 and b = -c2 / 6 (7-point: (D^-1 A) r = r - S(r) / 6,
// S the neighbour sum) and c2 (srfmg_api.cu)
struct Cheb {
  int nu = 0;
  double a = 0, b = 0, c2 = 0;      // degree-2 polynomial form
  std::vector<double> alpha, beta;  // recurrence steps
};
Cheb chebyshev(int nu, double lo_frac, double hi_frac, double lmax);

// ---- launchers; all enqueue on stream and return the launch status.  T is
// ---- the storage and arithmetic type, except where noted.

// r = D^-1 (f - A u) on the compute region, D = 6 n^2.
template <typename T>
cudaError_t launch_cheb_residual(const LevelView& L, const T* u, T* r, FieldT<T> f,
                                 cudaStream_t s);
// Chebyshev degree 2 finish: u += a r + b * (sum of the 6 neighbours of r),
// neighbours outside the domain mirrored with a sign flip, ghosts inside the
// domain read as stored (zero for the residual array).
template <typename T>
cudaError_t launch_cheb2_update(const LevelView& L, T* u, const T* r, double a, double b,
                                cudaStream_t s);
// One step of the Chebyshev recurrence: d = alpha d + beta r, u += d
// (d untouched and unused when write_d == 0 and alpha == 0).
// A degree-1 step u += beta r that also forms the residual the next
// smoothing of the level starts from, r2 = D^-1 (f - A u_new) =
// (1 - beta) r + (beta / 6) (sum of the neighbours of r) (7-point operator;
// r2 must not alias r).
template <typename T>
cudaError_t launch_cheb1_next(const LevelView& L, T* u, const T* r, T* r2, double beta,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_cheb_step(const LevelView& L, T* u, T* d, const T* r, double alpha,
                             double beta, int write_d, cudaStream_t s);
// out = A u on the compute region.
template <typename T>
cudaError_t launch_apply(const LevelView& L, const T* u, T* out, cudaStream_t s);
// r = f - A u on the compute region.
template <typename T>
cudaError_t launch_residual(const LevelView& L, const T* u, FieldT<T> f, T* r, cudaStream_t s);
// For every coarse cell of the fine boxes' restriction region:
// uhat = average of the 8 children of u, rho = average of the 8 children of
// (f - A u).  uhat_dst and rho_dst are arrays of the coarse level.
template <typename T>
cudaError_t launch_resid_restrict(const LevelView& F, const T* u, FieldT<T> f,
                                  const LevelView& C, T* uhat_dst, T* rho_dst, cudaStream_t s);
// Coarse right-hand side of the FAS cycle (Eq. eq:cresid2 and its SR form):
// rhs = rho + A u inside the fine boxes' restriction region, rhs = A u on the
// rest of the compute region; t = u on the compute region.  Arithmetic in
// float64 whatever T.  With r (may be null), also the coarse smoother's first
// residual D^-1 (rhs - A u) as it stands, which is D^-1 rho inside the
// restriction region and 0 on the rest of the compute region.
template <typename T>
cudaError_t launch_coarse_rhs(const LevelView& C, const LevelView& F, const T* u, const T* rho,
                              T* rhs, T* t, T* r, cudaStream_t s);
// t = u on the shell cells of the boxes that lie inside the domain (levels
// stored with a shell; with launch_coarse_rhs, t = u on the whole box).
template <typename T>
cudaError_t launch_shell_copy(const LevelView& C, const T* u, T* t, cudaStream_t s);
// Transition level: u = t (the owner-written restricted solution) and
// rhs = rho + A t on the whole (global) level; float64 arithmetic.  With r
// (may be null), also the smoother's first residual D^-1 rho.
template <typename T>
cudaError_t launch_transition_rhs(const LevelView& C, const T* t, const T* rho, T* u, T* rhs,
                                  T* r, cudaStream_t s);
// Prolongation onto the fine boxes' prolongation range:
// add == 0: uf = P uc;  add == 1: uf += P uc.
template <typename T>
cudaError_t launch_prolong(const LevelView& C, const T* uc, const LevelView& F, T* uf, int add,
                           cudaStream_t s);
// e = u - t on the stored cells of every box that lie inside the domain (the
// coarse-grid correction w - t of the FAS V-cycle); prolong_range != 0: on
// each box's prolongation range [plo, phi) instead (the trimmed views of the
// last stage carry the needed cells there).
template <typename T>
cudaError_t launch_diff(const LevelView& C, const T* u, const T* t, T* e, cudaStream_t s,
                        int prolong_range = 0);
// Coarsest grid: u = Minv f, Minv the dense float64 inverse (m x m,
// m = nx ny nz); float64 arithmetic.
template <typename T>
cudaError_t launch_coarse_solve(const LevelView& L, const double* minv, FieldT<T> f, T* u,
                                cudaStream_t s);
// Coarsest grid by the separable sine transform, u = P^T (Lambda^-1 (P f)),
// every axis at most 32 cells; sep = [Px | Py | Pz | 1/lambda] (per-axis
// orthonormal bases P_d[k][i], k, i < N_d, then nx ny nz inverse
// eigenvalues indexed (kz ny + ky) nx + kx); g, q: float64 scratch of
// nx ny nz values.  Three launches; float64 arithmetic.
template <typename T>
cudaError_t launch_coarse_solve_sep(const LevelView& L, const double* sep, double* g, double* q,
                                    FieldT<T> f, T* u, cudaStream_t s);
// f_c = 8-child average of f_f on whole global levels (fd: the fine grid's
// cells per dimension); sets *status |= 1 if an input value is not finite
// (check != 0).
template <typename T>
cudaError_t launch_restrict_global(Dims fd, const T* ff, T* fc, int check, unsigned int* status,
                                   cudaStream_t s);
// Genuine cells of every box of L into the global float64 array out:
// out = u (add == 0) or out += u (add == 1).
template <typename T>
cudaError_t launch_gather_genuine(const LevelView& L, const T* u, double* out, int add,
                                  cudaStream_t s);

// ---- float64 defect correction around the float32 inner solver

// d = float(f - A u) on the whole grid g with n cells per unit length
// (float64 arithmetic, unpadded arrays); with u == nullptr, d = float(f).
// Sets *status |= 1 if f holds a value that is not finite.
cudaError_t launch_defect(Dims g, int n, const double* f, const double* u, float* d,
                          unsigned int* status, cudaStream_t s);
// *norm = max over the cells of grid g of |f - A u| (float64; |f| when u is
// null), stored as the bit pattern of the double; *norm must be 0 on entry.
// Sets *status |= 1 if a value is not finite.
cudaError_t launch_resid_norm(Dims g, int n, const double* f, const double* u,
                              unsigned long long* norm, unsigned int* status, cudaStream_t s);
// out[i] = in[i] rounded to float by the solver's integer-pipe conversion
// (the one its float64-arithmetic kernels store float32 results with).
cudaError_t launch_narrow(const double* in, float* out, long long n, cudaStream_t s);
// u = e (add == 0) or u += e (add == 1) on `cells` cells, e float32.
cudaError_t launch_accumulate(long long cells, const float* e, double* u, int add,
                              cudaStream_t s);

// ---- the 27-point operator (kernels27.cu; float64 only)
// A u = n^2 (w0 u - w1 sum_faces - w2 sum_edges - w3 sum_corners)
struct W27 {
  double w0, w1, w2, w3;
};

// r = D^-1 (f - A u), D = w0 n^2, on the compute region.
cudaError_t launch27_cheb_residual(const LevelView& L, const double* u, double* r,
                                   FieldT<double> f, W27 w, cudaStream_t s);
// u += a r - c2 W r with W r = (w1 sf + w2 se + w3 sc)(r) / w0 (the degree-2
// Chebyshev polynomial; r's shell inside the domain reads as zero).
cudaError_t launch27_cheb2_update(const LevelView& L, double* u, const double* r, double a,
                                  double c2, W27 w, cudaStream_t s);
cudaError_t launch27_apply(const LevelView& L, const double* u, double* out, W27 w,
                           cudaStream_t s);
cudaError_t launch27_residual(const LevelView& L, const double* u, FieldT<double> f, double* r,
                              W27 w, cudaStream_t s);
// r = f - A u on the compute region (column form; r's shell is not written)
cudaError_t launch27_residual_zm(const LevelView& L, const double* u, FieldT<double> f,
                                 double* r, W27 w, cudaStream_t s);
// uhat = average of the 8 children of u, rho = average of the 8 children of r
// on the fine boxes' restriction region
cudaError_t launch27_restrict_pair(const LevelView& F, const double* u, const double* r,
                                   const LevelView& C, double* uhat_dst, double* rho_dst,
                                   cudaStream_t s);
// (r: as launch_coarse_rhs and launch_transition_rhs, D = w0 n^2)
cudaError_t launch27_coarse_rhs(const LevelView& C, const LevelView& F, const double* u,
                                const double* rho, double* rhs, double* t, double* r, W27 w,
                                cudaStream_t s);
cudaError_t launch27_transition_rhs(const LevelView& C, const double* t, const double* rho,
                                    double* u, double* rhs, double* r, W27 w, cudaStream_t s);
// max |f - A u| (|f| without u) over the whole unpadded level L (one box)
cudaError_t launch27_resid_norm(const LevelView& L, const double* f, const double* u,
                                unsigned long long* norm, unsigned int* status, W27 w,
                                cudaStream_t s);

// ---- segment-resident legs of the float32 SR V-cycle (segment_leg.cu): one
// thread-block cluster of C CTAs per segment box of level L, the box's
// stored planes split into z-slabs of at most max_planes planes whose u and
// smoother residual are held in shared memory (smem bytes, leg_smem_bytes).
// down: the degree-2 pre-smoother (a, b) with the level's right-hand side
// rhs, then residual + restriction into uhat_dst / rho_dst of Cv.
cudaError_t launch_leg_down(const LevelView& L, const LevelView& Cv, float* u, const float* rhs,
                            float* uhat_dst, float* rho_dst, double a, double b, int C,
                            int max_planes, size_t smem, unsigned* status, int force_timeout,
                            cudaStream_t s);
// up: u += P ec (ec on Cv), the degree-2 post-smoother (a, b), e_out = u - t.
cudaError_t launch_leg_up(const LevelView& L, const LevelView& Cv, float* u, const float* t,
                          const float* rhs, const float* ec, float* e_out, double a, double b,
                          int C, int max_planes, size_t smem, unsigned* status,
                          int force_timeout, cudaStream_t s);
size_t leg_smem_bytes(int e0, int e1, int planes);
// clusters of C CTAs with smem bytes each that fit on the device at once
int leg_max_clusters(int C, size_t smem);
// allow smem bytes of dynamic shared memory for the leg kernels
cudaError_t leg_prepare(size_t smem);

// ---- the global V-cycle in one persistent cooperative launch (persistent.cu;
// float64, 7-point, degree-2 smoothers).  Levels 0 (coarsest) .. top.
constexpr int kVcycleThreads = 256;
constexpr int kVcycleMaxLevels = 12;
struct VcycleLevel {
  LevelView view;        // one whole global level
  double* u;             // the level's solution (the caller's at the top)
  double *r, *t, *rhs, *rho;
  const double* f;       // right-hand side: the caller's at the top, rhs below
  double cf;             // 1 / (6 n^2)                 (smoother residual)
  double cS, cO;         // -3 n^2 / 8, n^2 / 8          (residual + restriction)
  double c6, cn, cr;     // 6 n^2, -n^2, 1 / (6 n^2)     (coarse right-hand side)
};
struct VcycleArgs {
  VcycleLevel lev[kVcycleMaxLevels];
  int top;
  const double* r_first;  // the top level's first residual, or null
  const double* minv;     // dense coarsest inverse, or null for the separable solve
  const double* sep;
  double *sep_g, *sep_q;
  int sep_w;
  double pre_a, pre_b, post_a, post_b;
  double sixth, eighth, three, w64, mone, one, zero;
  unsigned* bar;          // grid barrier: arrivals (zero at launch), generation
  unsigned* status;
  int force_timeout;
};
cudaError_t launch_vcycle(const VcycleArgs& a, int blocks, cudaStream_t s);
int vcycle_max_blocks_per_sm();

// Queue one solve of handle h on stream without validating the pointers
// (the batch path validates them before stream capture); srfmg_api.cu.
int enqueue_solve_unchecked(::sr_fmg_s* h, const double* f, double* u, cudaStream_t s);
// cells of the handle's fine grid
long long handle_cells(const ::sr_fmg_s* h);
// changes whenever the handle's launch sequence changes (launch shape,
// debug modes): a batch re-captures its graph when it does
long long handle_generation(const ::sr_fmg_s* h);

}  // namespace srfmg
