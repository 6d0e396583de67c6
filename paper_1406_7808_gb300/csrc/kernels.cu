// Kernels of the FMG / SR-FMG solver (sm_103a), templated on the storage
// type: float64 for the FP64 solver, float32 for the inner solver of the
// mixed-precision mode (whose coarse right-hand sides, coarsest solve and
// outer defect stay in float64 arithmetic).
//
// Every kernel runs over the boxes of one level: blockIdx.y selects the box
// (one per segment on an SR level, a single box on a global level) and the
// threads of blockIdx.x stride over the cells of the kernel's region in x-
// fastest order.  On GB300 the float64 pipe (two lanes per clock per SM) is
// the binding resource for these stencils, far below what HBM can feed, so
// the kernels are written to spend as little float64 pipe time per cell as
// the arithmetic allows:
//   - ghost cells outside the domain are never stored: a neighbour outside
//     the domain is replaced by minus the mirror cell on the fly (Sec. 3.3),
//     with the sign flip done on the integer pipe;
//   - every float64 operation is a fused multiply-add whose constant operands
//     are kernel parameters (adds as fma(a, one, b), scalings as
//     fma(a, c, zero)): on sm_103a that form issues faster than DADD, DMUL or
//     an FMA with an immediate operand (0.63 against 0.53 T lane-op/s);
//   - the degree-2 Chebyshev smoother is evaluated as x2 = x0 + a r0 + b S(r0)
//     (two stencil passes, 14 operations per cell) instead of the three-term
//     recurrence (19);
//   - the residual of the 8 children of a coarse cell is summed through the
//     24 faces of the 2x2x2 block (41 operations per coarse cell instead of 72);
//   - trilinear interpolation walks fine z-columns and forms each coarse
//     plane's bilinear (x, y) value once per column, so a fine cell costs
//     about 3.5 operations for the correction instead of 16.
#include "srfmg_device.cuh"
#include "srfmg_internal.cuh"

namespace srfmg {
namespace {

constexpr int kThreads = 256;

using namespace dev;

// ---------------------------------------------------------------------------

// The two smoother passes, r = D^-1 (f - A u) = f h^2/6 - u + (sum of
// neighbours)/6 and u += a r + b (sum of the neighbours of r), in column
// (z-marching) form: the threads of a block take consecutive cells of the
// box's flattened (x, y) plane (so warps stay full whatever the box width),
// and each thread walks a chunk of L.zchunk cells in z, carrying the
// z-neighbours in registers.  blockIdx.x enumerates (plane block, z chunk).
constexpr int kZThreads = 256;

struct ZTiles {
  int nplane, nzc;  // plane blocks, z chunks
  int zc;           // cells per z chunk
};

__device__ __forceinline__ bool ztile(const BoxDesc& B, ZTiles t, int& x, int& y, int& z0,
                                      int& z1) {
  const int tz = blockIdx.x / t.nplane, pb = blockIdx.x - tz * t.nplane;
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1];
  const int i = pb * kZThreads + threadIdx.x;
  const int iy = i / ex;
  x = B.lo[0] + (i - iy * ex);
  y = B.lo[1] + iy;
  z0 = B.lo[2] + tz * t.zc;
  z1 = min(z0 + t.zc, B.hi[2]);
  return iy < ey && z0 < z1;
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) k_cheb_residual_zm(LevelView L,
                                                               const T* __restrict__ u,
                                                               T* __restrict__ r, FieldT<T> f,
                                                               T cf, T sixth, ZTiles tiles) {
  grid_dep_wait();
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
  }
  __syncthreads();
  int x, y, z0, z1;
  if (!ztile(B, tiles, x, y, z0, z1)) return;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const long long sy = B.sy, sz = B.sz, fsz = FB.sz;
  long long c = at(B, x, y, z0);
  long long fc = at(FB, x, y, z0);
  T uc = u[c];
  T um = (z0 > 0) ? u[c - sz] : negx(uc);
  for (int z = z0; z < z1; ++z) {
    const T m = negx(uc);
    const T up = (z < nz - 1) ? u[c + sz] : m;
    T v[6];
    v[0] = (x > 0) ? u[c - 1] : m;
    v[1] = (x < nx - 1) ? u[c + 1] : m;
    v[2] = (y > 0) ? u[c - sy] : m;
    v[3] = (y < ny - 1) ? u[c + sy] : m;
    v[4] = um;
    v[5] = up;
    const T fv = f.p[fc];
    r[c] = fma6(sixth, v, fma(fv, cf, m));
    um = uc;
    uc = up;
    c += sz;
    fc += fsz;
  }
}

template <typename T>
__global__ void __launch_bounds__(kZThreads) k_cheb2_update_zm(LevelView L, T* __restrict__ u,
                                                              const T* __restrict__ r, T a, T b,
                                                              ZTiles tiles) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  int x, y, z0, z1;
  if (!ztile(B, tiles, x, y, z0, z1)) return;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const long long sy = B.sy, sz = B.sz;
  long long c = at(B, x, y, z0);
  T rc = r[c];
  T rm = (z0 > 0) ? r[c - sz] : negx(rc);
  // the two streams read from DRAM (r one plane up, u) are loaded one step
  // ahead; the planes loaded stay within the column's chunk and the stored
  // region (4 % faster; the same prefetch in the residual pass was slower)
  T rpr = (z0 < nz - 1) ? r[c + sz] : rc;
  T uv = u[c];
  for (int z = z0; z < z1; ++z) {
    const T rpn = (z + 2 < nz && z + 2 <= z1) ? r[c + 2 * sz] : rc;
    const T uvn = (z + 1 < z1) ? u[c + sz] : uv;
    const T m = negx(rc);
    const T rp = (z < nz - 1) ? rpr : m;
    T v[6];
    v[0] = (x > 0) ? r[c - 1] : m;
    v[1] = (x < nx - 1) ? r[c + 1] : m;
    v[2] = (y > 0) ? r[c - sy] : m;
    v[3] = (y < ny - 1) ? r[c + sy] : m;
    v[4] = rm;
    v[5] = rp;
    u[c] = fma6(b, v, fma(a, rc, uv));
    rm = rc;
    rc = rp;
    rpr = rpn;
    uv = uvn;
    c += sz;
  }
}

// Column form of k_cheb1_next (float32, HBM bound): u += beta r and
// r2 = (1 - beta) r + (beta / 6) (sum of the neighbours of r).
template <typename T>
__global__ void __launch_bounds__(kZThreads) k_cheb1_next_zm(LevelView L, T* __restrict__ u,
                                                            const T* __restrict__ r,
                                                            T* __restrict__ r2, T beta, T keep,
                                                            T b6, ZTiles tiles) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  int x, y, z0, z1;
  if (!ztile(B, tiles, x, y, z0, z1)) return;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const long long sy = B.sy, sz = B.sz;
  long long c = at(B, x, y, z0);
  T rc = r[c];
  T rm = (z0 > 0) ? r[c - sz] : negx(rc);
  for (int z = z0; z < z1; ++z) {
    const T m = negx(rc);
    const T rp = (z < nz - 1) ? r[c + sz] : m;
    T v[6];
    v[0] = (x > 0) ? r[c - 1] : m;
    v[1] = (x < nx - 1) ? r[c + 1] : m;
    v[2] = (y > 0) ? r[c - sy] : m;
    v[3] = (y < ny - 1) ? r[c + sy] : m;
    v[4] = rm;
    v[5] = rp;
    u[c] = fma(beta, rc, u[c]);
    r2[c] = fma6(b6, v, keep * rc);
    rm = rc;
    rc = rp;
    c += sz;
  }
}

// Per-cell form of the two smoother passes (one thread per cell, x-fastest
// over the box's compute region), used for float64: there the float64 pipe
// binds and fully packed warps matter more than the index arithmetic the
// column form saves.
// r = D^-1 (f - A u) = f h^2/6 - u + (sum of neighbours)/6
template <typename T>
__global__ void __launch_bounds__(kThreads, 7) k_cheb_residual(LevelView L, const T* __restrict__ u,
                                                            T* __restrict__ r, FieldT<T> f,
                                                            T cf, T sixth) {
  grid_dep_wait();
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;

  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const T uc = u[c];
    T v[6];
    neighbours<T>(u, c, B, L, q.x, q.y, q.z, uc, v);
    const T fv = f.p[at(FB, q.x, q.y, q.z)];
    r[c] = fma6(sixth, v, fma(fv, cf, negx(uc)));
  }
}

// u += a r + b (sum of the neighbours of r)
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_cheb2_update(LevelView L, T* __restrict__ u,
                                                           const T* __restrict__ r, T a, T b) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;

  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const T rc = r[c];
    T v[6];
    neighbours<T>(r, c, B, L, q.x, q.y, q.z, rc, v);
    u[c] = fma6(b, v, fma(a, rc, u[c]));
  }
}

// A degree-1 smoothing step followed by the residual the next smoothing of
// the same level and f starts from: u += beta r and
// r2 = D^-1 (f - A (u + beta r)) = r - beta D^-1 A r
//    = (1 - beta) r + (beta / 6) (sum of the neighbours of r),
// neighbours as in k_cheb2_update (mirrored with a sign flip outside the
// domain, stored ghosts, which are zero in a residual array, inside it).
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_cheb1_next(LevelView L, T* __restrict__ u,
                                                         const T* __restrict__ r,
                                                         T* __restrict__ r2, T beta, T keep,
                                                         T b6) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;

  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const T rc = r[c];
    T v[6];
    neighbours<T>(r, c, B, L, q.x, q.y, q.z, rc, v);
    u[c] = fma(beta, rc, u[c]);
    r2[c] = fma6(b6, v, keep * rc);
  }
}

// residual == 0: out = A u = n^2 (6 u - sum);  residual == 1: out = f - A u
template <typename T>
__global__ void __launch_bounds__(kThreads) k_apply(LevelView L, const T* __restrict__ u,
                                                    T* __restrict__ out, FieldT<T> f,
                                                    int residual, T c6, T cn, Fk<T> k) {
  grid_dep_wait();
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = residual ? (f.single ? f.boxes[0] : f.boxes[blockIdx.y]) : B;
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;

  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const T uc = u[c];
    T v[6];
    neighbours<T>(u, c, B, L, q.x, q.y, q.z, uc, v);
    // apply: c6 = 6 n^2, cn = -n^2; residual: c6 = -6 n^2, cn = n^2
    const T base = residual ? f.p[at(FB, q.x, q.y, q.z)] : k.zero;
    out[c] = fma6(cn, v, fma(c6, uc, base));
  }
}

// Residual of the 8 children of each coarse cell, restricted, and the
// restricted solution.  With S the sum of the children, the children's
// operator values add up to n^2 (3 S - O), O the sum of the 24 neighbours
// across the outer faces of the 2x2x2 block (each inner face cancels), so
//   rho = (sum of f)/8 - (3 n^2/8) S + (n^2/8) O,   uhat = S/8.
template <typename T>
__global__ void __launch_bounds__(kThreads, 5) k_resid_restrict(LevelView F, const T* __restrict__ u,
                                                             FieldT<T> f, LevelView C,
                                                             T* __restrict__ uhat_dst,
                                                             T* __restrict__ rho_dst, T cS, T cO,
                                                             T eighth, Fk<T> k) {
  grid_dep_wait();
  __shared__ BoxDesc B, FB, CB;
  if (threadIdx.x == 0) {
    B = F.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
    CB = (C.nbox == 1) ? C.boxes[0] : C.boxes[blockIdx.y];
  }
  __syncthreads();
  int lo[3], hi[3];
  region_of(B, kRestrict, lo, hi);
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int ncell = ex * ey * ez;

  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, lo, ex, ey);
    const int x0 = 2 * q.x, y0 = 2 * q.y, z0 = 2 * q.z;
    const long long c0 = at(B, x0, y0, z0);
    const long long sy = B.sy, sz = B.sz;
    T v[2][2][2];
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) v[cz][cy][cx] = u[c0 + cz * sz + cy * sy + cx];
    T fs;
    {
      const long long f0 = at(FB, x0, y0, z0);
      const long long fy = FB.sy, fz = FB.sz;
      fs = fma(f.p[f0], k.one, f.p[f0 + 1]);
      fs = fma(f.p[f0 + fy], k.one, fs);
      fs = fma(f.p[f0 + fy + 1], k.one, fs);
      fs = fma(f.p[f0 + fz], k.one, fs);
      fs = fma(f.p[f0 + fz + 1], k.one, fs);
      fs = fma(f.p[f0 + fz + fy], k.one, fs);
      fs = fma(f.p[f0 + fz + fy + 1], k.one, fs);
    }
    T S = fma(v[0][0][0], k.one, v[0][0][1]);
    S = fma(v[0][1][0], k.one, S);
    S = fma(v[0][1][1], k.one, S);
    S = fma(v[1][0][0], k.one, S);
    S = fma(v[1][0][1], k.one, S);
    S = fma(v[1][1][0], k.one, S);
    S = fma(v[1][1][1], k.one, S);
    // the 24 outer neighbours, mirrored with a sign flip outside the domain
    const bool xl = x0 > 0, xr = x0 + 2 < F.nx, yl = y0 > 0, yr = y0 + 2 < F.ny, zl = z0 > 0,
               zr = z0 + 2 < F.nz;
    T O = k.zero;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        const long long row = c0 + cz * sz + cy * sy;
        O = fma(xl ? u[row - 1] : negx(v[cz][cy][0]), k.one, O);
        O = fma(xr ? u[row + 2] : negx(v[cz][cy][1]), k.one, O);
      }
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const long long col = c0 + cz * sz + cx;
        O = fma(yl ? u[col - sy] : negx(v[cz][0][cx]), k.one, O);
        O = fma(yr ? u[col + 2 * sy] : negx(v[cz][1][cx]), k.one, O);
      }
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const long long pil = c0 + cy * sy + cx;
        O = fma(zl ? u[pil - sz] : negx(v[0][cy][cx]), k.one, O);
        O = fma(zr ? u[pil + 2 * sz] : negx(v[1][cy][cx]), k.one, O);
      }
    const long long cc = at(CB, q.x, q.y, q.z);
    rho_dst[cc] = fma(cS, S, fma(cO, O, fma(fs, eighth, k.zero)));
    uhat_dst[cc] = fma(S, eighth, k.zero);
  }
}

// rhs = rho + A u inside the restriction region of the matching fine box,
// A u elsewhere in the compute region (float64 arithmetic); t = u on the
// whole stored box; with r, the smoother's first residual D^-1 (rhs - A u),
// which is D^-1 rho and 0 respectively (cr = D^-1)
template <typename T>
__global__ void __launch_bounds__(kThreads, 8) k_coarse_rhs(LevelView C, LevelView F,
                                                         const T* __restrict__ u,
                                                         const T* __restrict__ rho,
                                                         T* __restrict__ rhs, T* __restrict__ t,
                                                         T* __restrict__ r, double c6, double cn,
                                                         double cr, Fk<double> k) {
  grid_dep_wait();
  __shared__ BoxDesc B, FBx;
  if (threadIdx.x == 0) {
    B = C.boxes[blockIdx.y];
    FBx = (F.nbox == 1) ? F.boxes[0] : F.boxes[blockIdx.y];
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const T uc = u[c];
    t[c] = uc;
    const bool inF = q.x >= FBx.rlo[0] && q.x < FBx.rhi[0] && q.y >= FBx.rlo[1] &&
                     q.y < FBx.rhi[1] && q.z >= FBx.rlo[2] && q.z < FBx.rhi[2];
    double v[6];
    neighbours<double>(u, c, B, C, q.x, q.y, q.z, uc, v);
    const double rh = inF ? widen(rho[c]) : k.zero;
    rhs[c] = stored<T>(fma6(cn, v, fma(c6, widen(uc), rh)));
    if (r) r[c] = stored<T>(cr * rh);
  }
}

// u = t, rhs = rho + A t on the whole (global) transition level (float64
// arithmetic); with r, the smoother's first residual D^-1 rho (cr = D^-1)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_transition_rhs(LevelView C,
                                                             const T* __restrict__ t,
                                                             const T* __restrict__ rho,
                                                             T* __restrict__ u,
                                                             T* __restrict__ rhs,
                                                             T* __restrict__ r, double c6,
                                                             double cn, double cr) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = C.boxes[0];
  __syncthreads();

  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const T tc = t[c];
    double v[6];
    neighbours<double>(t, c, B, C, q.x, q.y, q.z, tc, v);
    u[c] = tc;
    const double rh = widen(rho[c]);
    rhs[c] = stored<T>(fma6(cn, v, fma(c6, widen(tc), rh)));
    if (r) r[c] = stored<T>(cr * rh);
  }
}

// One warp per row of the dense inverse (float64 arithmetic).
template <typename T>
__global__ void k_coarse_solve(LevelView L, const double* __restrict__ minv, FieldT<T> f,
                               T* __restrict__ u, Fk<double> k) {
  grid_dep_wait();
  const BoxDesc B = L.boxes[0];
  const BoxDesc FB = f.boxes[0];
  const int nx = L.nx, ny = L.ny, m = nx * ny * L.nz;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  double s = k.zero;
  for (int j = lane; j < m; j += 32) {
    const int x = j % nx, y = (j / nx) % ny, z = j / (nx * ny);
    s = fma(minv[(long long)warp * m + j], widen(f.p[at(FB, x, y, z)]), s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fma(__shfl_xor_sync(0xffffffffu, s, o), k.one, s);
  if (lane == 0) {
    const int x = warp % nx, y = (warp / nx) % ny, z = warp / (nx * ny);
    u[at(B, x, y, z)] = stored<T>(s);
  }
}

// Coarsest grid by the separable sine transform: the operator is diagonal
// in the products of the per-axis bases P_d[k][i] = c_k sin(pi (k + 1)(i + 1/2) / N_d)
// (rows orthonormal), so u = P^T (Lambda^-1 (P f)) with P = Px (x) Py (x) Pz.
// Three passes, each a set of independent tasks of W lanes (W a power of two
// covering every axis, 32 / W tasks per warp; lane l holds index l of its
// line and the sums run over the line through shuffles within the task):
//   fwd_xy  task (z, ky):   t[x] = sum_y Py[ky][y] f[z][y][x],  g[z][ky][kx] = sum_x Px[kx][x] t[x]
//   z       task (ky, kx):  h[kz] = sum_z Pz[kz][z] g[z][ky][kx] / lambda,  q[z][ky][kx] = sum_kz Pz[kz][z] h[kz]
//   inv_xy  task (z, y):    t[kx] = sum_ky Py[ky][y] q[z][ky][kx],  u[z][y][x] = sum_kx Px[kx][x] t[kx]
// sep holds Px (nx^2), Py (ny^2), Pz (nz^2) and 1/lambda (indexed
// (kz ny + ky) nx + kx); g and q are float64 scratch of nx ny nz values.
struct SepTask {
  int lane, task;  // lane within the task, task index (may be past the last task)
};

__device__ __forceinline__ SepTask sep_task(int W) {
  const int gl = blockIdx.x * blockDim.x + threadIdx.x;
  return SepTask{gl & (W - 1), gl / W};
}

template <typename T>
__global__ void __launch_bounds__(64) k_sep_fwd_xy(LevelView L, FieldT<T> f,
                                                   const double* __restrict__ sep,
                                                   double* __restrict__ g, int W, Fk<double> k) {
  grid_dep_wait();
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const SepTask q = sep_task(W);
  const bool live = q.task < nz * ny;
  const int z = live ? q.task / ny : 0, ky = live ? q.task - (q.task / ny) * ny : 0;
  const BoxDesc FB = f.boxes[0];
  const double* Px = sep;
  const double* Py = sep + nx * nx;
  double t = k.zero;
  if (live && q.lane < nx)
    for (int y = 0; y < ny; ++y) t = fma(Py[ky * ny + y], widen(f.p[at(FB, q.lane, y, z)]), t);
  double o = k.zero;
  for (int x = 0; x < nx; ++x) {
    const double tx = __shfl_sync(0xffffffffu, t, x, W);
    if (q.lane < nx) o = fma(Px[q.lane * nx + x], tx, o);
  }
  if (live && q.lane < nx) g[((long long)z * ny + ky) * nx + q.lane] = o;
}

__global__ void __launch_bounds__(64) k_sep_z(int nx, int ny, int nz,
                                              const double* __restrict__ sep,
                                              const double* __restrict__ g,
                                              double* __restrict__ qo, int W, Fk<double> k) {
  grid_dep_wait();
  const SepTask q = sep_task(W);
  const bool live = q.task < ny * nx;
  const int ky = live ? q.task / nx : 0, kx = live ? q.task - (q.task / nx) * nx : 0;
  const double* Pz = sep + nx * nx + ny * ny;
  const double* il = Pz + nz * nz;
  const long long pl = (long long)ny * nx;
  const bool on = live && q.lane < nz;
  const double v = on ? g[q.lane * pl + (long long)ky * nx + kx] : k.zero;
  double h = k.zero;
  for (int z = 0; z < nz; ++z) {
    const double vz = __shfl_sync(0xffffffffu, v, z, W);
    if (q.lane < nz) h = fma(Pz[q.lane * nz + z], vz, h);
  }
  if (on) h = fma(h, il[q.lane * pl + (long long)ky * nx + kx], k.zero);
  double o = k.zero;
  for (int kz = 0; kz < nz; ++kz) {
    const double hz = __shfl_sync(0xffffffffu, h, kz, W);
    if (q.lane < nz) o = fma(Pz[kz * nz + q.lane], hz, o);
  }
  if (on) qo[q.lane * pl + (long long)ky * nx + kx] = o;
}

template <typename T>
__global__ void __launch_bounds__(64) k_sep_inv_xy(LevelView L, const double* __restrict__ sep,
                                                   const double* __restrict__ qi,
                                                   T* __restrict__ u, int W, Fk<double> k) {
  grid_dep_wait();
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const SepTask q = sep_task(W);
  const bool live = q.task < nz * ny;
  const int z = live ? q.task / ny : 0, y = live ? q.task - (q.task / ny) * ny : 0;
  const BoxDesc B = L.boxes[0];
  const double* Px = sep;
  const double* Py = sep + nx * nx;
  double t = k.zero;
  if (live && q.lane < nx)
    for (int ky = 0; ky < ny; ++ky)
      t = fma(Py[ky * ny + y], qi[((long long)z * ny + ky) * nx + q.lane], t);
  double o = k.zero;
  for (int kx = 0; kx < nx; ++kx) {
    const double tk = __shfl_sync(0xffffffffu, t, kx, W);
    if (q.lane < nx) o = fma(Px[kx * nx + q.lane], tk, o);
  }
  if (live && q.lane < nx) u[at(B, q.lane, y, z)] = stored<T>(o);
}

__device__ __forceinline__ bool not_finite(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
}
__device__ __forceinline__ bool not_finite(float v) {
  return ((__float_as_uint(v) >> 23) & 0xff) == 0xff;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_restrict_global(Dims fd, const T* __restrict__ ff,
                                                              T* __restrict__ fc, int check,
                                                              unsigned int* status, T eighth,
                                                              Fk<T> k) {
  grid_dep_wait();
  const int cx = fd.x / 2, cy = fd.y / 2, cz = fd.z / 2;
  const long long ncell = (long long)cx * cy * cz;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    split3(i, cx, cy, x, y, z);
    const long long py = fd.x, pz = (long long)fd.x * fd.y;
    const long long f0 = (2 * z) * pz + (2 * y) * py + 2 * x;
    const T a[8] = {ff[f0], ff[f0 + 1], ff[f0 + py], ff[f0 + py + 1],
                    ff[f0 + pz], ff[f0 + pz + 1], ff[f0 + pz + py], ff[f0 + pz + py + 1]};
    T s = k.zero;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (check) bad |= not_finite(a[j]);
      s = fma(a[j], eighth, s);
    }
    fc[i] = s;
  }
  if (check && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

// d = float(f - A u) with float64 arithmetic, or d = float(f) without u;
// 8 blocks per SM (32 registers: 2.49 -> 2.43 ms per 512^3 mixed solve
// against 6)
__global__ void __launch_bounds__(kThreads, 8) k_defect(Dims g, const double* __restrict__ f,
                                                        const double* __restrict__ u,
                                                        float* __restrict__ d,
                                                        unsigned int* status, double c6,
                                                        double cn) {
  grid_dep_wait();
  // 32-bit cell indices (grids hold fewer than 2^31 cells): fewer registers
  // and index instructions than the 64-bit loop, more resident warps to
  // cover the neighbour loads of this float64-pipe-bound pass
  const unsigned nx = (unsigned)g.x, ny = (unsigned)g.y;
  const unsigned ncell = nx * ny * (unsigned)g.z;
  const unsigned sy = nx, sz = nx * ny;
  bool bad = false;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const double fv = f[i];
    bad |= not_finite(fv);
    if (!u) {
      d[i] = narrow(fv);
      continue;
    }
    const unsigned t = i / nx;
    const unsigned x = i - t * nx, y = t % ny, z = t / ny;
    const double uc = u[i];
    const double m = negx(uc);
    double v[6];
    v[0] = (x > 0) ? u[i - 1] : m;
    v[1] = (x < nx - 1) ? u[i + 1] : m;
    v[2] = (y > 0) ? u[i - sy] : m;
    v[3] = (y < ny - 1) ? u[i + sy] : m;
    v[4] = (z > 0) ? u[i - sz] : m;
    v[5] = (z < (unsigned)g.z - 1) ? u[i + sz] : m;
    d[i] = narrow(fma6(cn, v, fma(c6, uc, fv)));
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

// *norm = max over the cells of the grid of |f - A u| (float64; |f| without u), as
// the bit pattern of a non-negative double (which orders like the unsigned
// integer); sets *status |= 1 if a value is not finite.  *norm must hold 0
// on entry.
__global__ void __launch_bounds__(kThreads) k_resid_norm(Dims g, const double* __restrict__ f,
                                                         const double* __restrict__ u,
                                                         unsigned long long* norm,
                                                         unsigned int* status, double c6,
                                                         double cn) {
  grid_dep_wait();
  const long long ncell = (long long)g.x * g.y * g.z;
  const long long sy = g.x, sz = (long long)g.x * g.y;
  unsigned long long m = 0;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    double r = f[i];
    if (u) {
      int x, y, z;
      split3(i, g.x, g.y, x, y, z);
      const double uc = u[i];
      const double mu = negx(uc);
      double v[6];
      v[0] = (x > 0) ? u[i - 1] : mu;
      v[1] = (x < g.x - 1) ? u[i + 1] : mu;
      v[2] = (y > 0) ? u[i - sy] : mu;
      v[3] = (y < g.y - 1) ? u[i + sy] : mu;
      v[4] = (z > 0) ? u[i - sz] : mu;
      v[5] = (z < g.z - 1) ? u[i + sz] : mu;
      r = fma6(cn, v, fma(c6, uc, r));
    }
    bad |= not_finite(r);
    // |r| by clearing the sign bit on the integer pipe
    const unsigned long long a = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, o);
    m = w > m ? w : m;
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(status, 1u);
    atomicMax(norm, m);
  }
}

__global__ void __launch_bounds__(kThreads) k_accumulate(long long cells, const float* __restrict__ e,
                                                         double* __restrict__ u, int add,
                                                         Fk<double> k) {
  grid_dep_wait();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cells;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = widen(e[i]);
    u[i] = add ? fma(v, k.one, u[i]) : v;
  }
}

// ---------------------------------------------------------------------------
// The transfer and pointwise passes walk z-columns: a thread owns an (x, y)
// of the region and zc cells in z, which keeps many independent loads
// in flight per thread (these passes are memory- or latency-bound in both
// precisions) and amortises the index arithmetic.

// region [lo, hi) of box B as z-columns: thread -> (x, y) of the flattened
// region plane, blockIdx.x -> (plane block, z chunk)
__device__ __forceinline__ bool zcolumn(const int lo[3], const int hi[3], int nplane, int zc,
                                        int& x, int& y, int& z0, int& z1) {
  const int tz = blockIdx.x / nplane, pb = blockIdx.x - tz * nplane;
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1];
  if (ex <= 0 || ey <= 0) return false;
  const int i = pb * kZThreads + threadIdx.x;
  const int iy = i / ex;
  x = lo[0] + (i - iy * ex);
  y = lo[1] + iy;
  z0 = lo[2] + tz * zc;
  z1 = min(z0 + zc, hi[2]);
  return iy < ey && z0 < z1;
}

// trilinear prolongation in fine z-columns: a thread owns a fine (x, y) of
// the box's prolongation range and walks F.zchunk fine cells in z.  Its two
// coarse columns per dimension are the fine cell's own coarse cell and the
// neighbour on its side (mirrored with a sign flip outside the domain); for
// every coarse plane it meets it forms the bilinear (x, y) value once
// (4 reads, 3 FMA, weights 3/4 and 1/4 as 3 a + b), and a fine cell combines
// the plane of its own coarse cell with the one on its side (1 FMA) and is
// scaled by 1/64 into uf (uf = P uc, or uf += P uc).
// kMode: 0 sets uf, 1 adds to it, 2 adds if add != 0 (one kernel for both,
// the float64 form: splitting it costs the set mode 1 %).  Register bound:
// 6 blocks per SM in float64, 8 in float32 (32 registers, no spills; the
// float32 passes ran 14-16 % faster than at 6)
template <typename T, int kMode>
__global__ void __launch_bounds__(kZThreads, sizeof(T) == 4 ? 8 : 6)
    k_prolong_zcol(LevelView C, const T* __restrict__ uc, LevelView F, T* __restrict__ uf,
                   int add, T three, T w64, int nplane, Fk<T> k) {
  constexpr bool kAdd = kMode == 1;
  grid_dep_wait();
  __shared__ BoxDesc B, CB;
  if (threadIdx.x == 0) {
    B = F.boxes[blockIdx.y];
    CB = (C.nbox == 1) ? C.boxes[0] : C.boxes[blockIdx.y];
  }
  __syncthreads();
  int lo[3], hi[3];
  region_of(B, kProlong, lo, hi);
  int x, y, z0, z1;
  if (!zcolumn(lo, hi, nplane, F.zchunk, x, y, z0, z1)) return;
  // coarse columns and their offsets within the coarse box
  const int X0 = x >> 1, Y0 = y >> 1;
  int Xo = (x & 1) ? X0 + 1 : X0 - 1, Yo = (y & 1) ? Y0 + 1 : Y0 - 1;
  const bool fx = Xo < 0 || Xo >= C.nx, fy = Yo < 0 || Yo >= C.ny;
  const long long dx = fx ? 0 : Xo - X0, dy = fy ? 0 : (long long)(Yo - Y0) * CB.sy;
  // bilinear value of coarse plane Z (mirrored plane outside the domain)
  auto plane = [&](int Z) -> T {
    const bool fz = Z < 0 || Z >= C.nz;
    const int Zi = fz ? (Z < 0 ? 0 : C.nz - 1) : Z;
    const long long b0 = at(CB, X0, Y0, Zi);
    const T a = fma(three, uc[b0], neg_if(uc[b0 + dx], fx));
    const T b = fma(three, neg_if(uc[b0 + dy], fy), neg_if(uc[b0 + dy + dx], fx ^ fy));
    return neg_if(fma(three, a, b), fz);
  };
  // walk the coarse planes Z of the chunk: the even fine cell 2Z combines
  // plane Z with Z-1, the odd one 2Z+1 with Z+1; every plane is formed once,
  // and only planes some cell of the chunk needs are read
  const int Zlo = z0 >> 1, Zhi = (z1 - 1) >> 1;
  T pm = (z0 & 1) ? k.zero : plane(Zlo - 1);
  T pc = plane(Zlo);
  const long long sz = B.sz;
  long long o = at(B, x, y, 2 * Zlo);
  if constexpr (kAdd && sizeof(T) == 4) {
    // float32 correction: the fine values (the stream from DRAM) are loaded
    // one coarse step ahead, from the planes of this thread's own chunk
    // (2.16 -> 1.87 ms per 512^3 mixed solve; the float64 kernel and the
    // FMG prolongation, which reads no fine values, keep the plain loop)
    T oe = (2 * Zlo >= z0) ? uf[o] : k.zero;
    T oo = (2 * Zlo + 1 < z1) ? uf[o + sz] : k.zero;
#pragma unroll 2
    for (int Zc = Zlo; Zc <= Zhi; ++Zc, o += 2 * sz) {
      const int fe = 2 * Zc, fo = fe + 1;
      const bool we = fe >= z0, wo = fo < z1;
      const bool next = Zc + 1 <= Zhi;
      const T ne = next ? uf[o + 2 * sz] : k.zero;
      const T no = (next && fo + 2 < z1) ? uf[o + 3 * sz] : k.zero;
      const T pp = wo ? plane(Zc + 1) : k.zero;
      if (we) uf[o] = fma(w64, fma(three, pc, pm), oe);
      if (wo) uf[o + sz] = fma(w64, fma(three, pc, pp), oo);
      pm = pc;
      pc = pp;
      oe = ne;
      oo = no;
    }
  } else {
#pragma unroll 2
    for (int Zc = Zlo; Zc <= Zhi; ++Zc, o += 2 * sz) {
      const int fe = 2 * Zc, fo = fe + 1;
      const bool we = fe >= z0, wo = fo < z1;
      const T pp = wo ? plane(Zc + 1) : k.zero;
      const bool addv = kMode == 2 ? add != 0 : kAdd;
      const T oe = (addv && we) ? uf[o] : k.zero;
      const T oo = (addv && wo) ? uf[o + sz] : k.zero;
      if (we) uf[o] = fma(w64, fma(three, pc, pm), oe);
      if (wo) uf[o + sz] = fma(w64, fma(three, pc, pp), oo);
      pm = pc;
      pc = pp;
    }
  }
}

// Column form of k_resid_restrict (float32, where the pass streams): a thread
// owns a coarse (X, Y) of the restriction region and walks zc coarse cells
// in z (a quarter of the handle's z-chunk: more blocks, as the kernel holds
// few warps per SM; 6 blocks per SM).  The 2x2 inner values of the fine plane below a coarse cell
// are the upper children of the previous one, and those of the plane above
// are the next cell's lower children, so each is loaded once (32 loads per
// coarse cell instead of 40).  Every sum takes the per-cell kernel's terms
// in its order (bit-identical results).
template <typename T>
__global__ void __launch_bounds__(kZThreads, 6)
    k_resid_restrict_zm(LevelView F, const T* __restrict__ u, FieldT<T> f, LevelView C,
                        T* __restrict__ uhat_dst, T* __restrict__ rho_dst, T cS, T cO, T eighth,
                        Fk<T> k, int nplane, int zc) {
  grid_dep_wait();
  __shared__ BoxDesc B, FB, CB;
  if (threadIdx.x == 0) {
    B = F.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
    CB = (C.nbox == 1) ? C.boxes[0] : C.boxes[blockIdx.y];
  }
  __syncthreads();
  int lo[3], hi[3];
  region_of(B, kRestrict, lo, hi);
  int X, Y, Z0, Z1;
  if (!zcolumn(lo, hi, nplane, zc, X, Y, Z0, Z1)) return;
  const int x0 = 2 * X, y0 = 2 * Y;
  const long long sy = B.sy, sz = B.sz, fy = FB.sy, fz = FB.sz;
  const bool xl = x0 > 0, xr = x0 + 2 < F.nx, yl = y0 > 0, yr = y0 + 2 < F.ny;
  long long c0 = at(B, x0, y0, 2 * Z0);
  long long f0 = at(FB, x0, y0, 2 * Z0);
  long long cc = at(CB, X, Y, Z0);
  T below[2][2], cur[2][2];
  bool zl = 2 * Z0 > 0;
  if (zl) {
    below[0][0] = u[c0 - sz];
    below[0][1] = u[c0 - sz + 1];
    below[1][0] = u[c0 - sz + sy];
    below[1][1] = u[c0 - sz + sy + 1];
  }
  cur[0][0] = u[c0];
  cur[0][1] = u[c0 + 1];
  cur[1][0] = u[c0 + sy];
  cur[1][1] = u[c0 + sy + 1];
  for (int Z = Z0; Z < Z1; ++Z) {
    const int z0 = 2 * Z;
    T v[2][2][2];
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        v[0][cy][cx] = cur[cy][cx];
        v[1][cy][cx] = u[c0 + sz + cy * sy + cx];
      }
    const bool zr = z0 + 2 < F.nz;
    T above[2][2];
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) above[cy][cx] = zr ? u[c0 + 2 * sz + cy * sy + cx] : k.zero;
    T fs = fma(f.p[f0], k.one, f.p[f0 + 1]);
    fs = fma(f.p[f0 + fy], k.one, fs);
    fs = fma(f.p[f0 + fy + 1], k.one, fs);
    fs = fma(f.p[f0 + fz], k.one, fs);
    fs = fma(f.p[f0 + fz + 1], k.one, fs);
    fs = fma(f.p[f0 + fz + fy], k.one, fs);
    fs = fma(f.p[f0 + fz + fy + 1], k.one, fs);
    T S = fma(v[0][0][0], k.one, v[0][0][1]);
    S = fma(v[0][1][0], k.one, S);
    S = fma(v[0][1][1], k.one, S);
    S = fma(v[1][0][0], k.one, S);
    S = fma(v[1][0][1], k.one, S);
    S = fma(v[1][1][0], k.one, S);
    S = fma(v[1][1][1], k.one, S);
    T O = k.zero;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        const long long row = c0 + cz * sz + cy * sy;
        O = fma(xl ? u[row - 1] : negx(v[cz][cy][0]), k.one, O);
        O = fma(xr ? u[row + 2] : negx(v[cz][cy][1]), k.one, O);
      }
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const long long col = c0 + cz * sz + cx;
        O = fma(yl ? u[col - sy] : negx(v[cz][0][cx]), k.one, O);
        O = fma(yr ? u[col + 2 * sy] : negx(v[cz][1][cx]), k.one, O);
      }
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        O = fma(zl ? below[cy][cx] : negx(v[0][cy][cx]), k.one, O);
        O = fma(zr ? above[cy][cx] : negx(v[1][cy][cx]), k.one, O);
      }
    rho_dst[cc] = fma(cS, S, fma(cO, O, fma(fs, eighth, k.zero)));
    uhat_dst[cc] = fma(S, eighth, k.zero);
    // the next coarse cell: its plane below is this cell's upper children,
    // its lower children the plane above (loaded when it lies in the domain,
    // which it does whenever there is a next cell)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        below[cy][cx] = v[1][cy][cx];
        cur[cy][cx] = above[cy][cx];
      }
    zl = true;
    c0 += 2 * sz;
    f0 += 2 * fz;
    cc += CB.sz;
  }
}

// d = alpha d + beta r (alpha == 0: d = beta r); u += d (the Chebyshev
// recurrence step for degrees other than 2), over the compute region
template <typename T>
__global__ void __launch_bounds__(kZThreads, 8) k_cheb_step_zm(LevelView L, T* __restrict__ u,
                                                            T* __restrict__ d,
                                                            const T* __restrict__ r, T alpha,
                                                            T beta, int write_d, int nplane,
                                                            Fk<T> k) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  int x, y, z0, z1;
  if (!zcolumn(B.lo, B.hi, nplane, L.zchunk, x, y, z0, z1)) return;
  const bool use_d = alpha != T(0);
  long long c = at(B, x, y, z0);
#pragma unroll 4
  for (int z = z0; z < z1; ++z, c += B.sz) {
    T dn = fma(beta, r[c], k.zero);
    if (use_d) dn = fma(alpha, d[c], dn);
    if (write_d) d[c] = dn;
    u[c] = fma(dn, k.one, u[c]);
  }
}

// e = u - t on every stored cell of the box inside the domain (compute
// cells and frozen SR ghosts): the coarse-grid correction w - t of the FAS
// V-cycle, ready for prolongation
template <typename T>
__global__ void __launch_bounds__(kZThreads, 8) k_diff_zm(LevelView C, const T* __restrict__ u,
                                                       const T* __restrict__ t,
                                                       T* __restrict__ e, int nplane, T mone,
                                                       int prolong_range) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = C.boxes[blockIdx.y];
  __syncthreads();
  const int nd[3] = {C.nx, C.ny, C.nz};
  const bool shell = B.ox < B.lo[0];
  int lo[3], hi[3];
  if (prolong_range) {
    region_of(B, kProlong, lo, hi);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = shell ? max(B.lo[d] - 1, 0) : B.lo[d];
      hi[d] = shell ? min(B.hi[d] + 1, nd[d]) : B.hi[d];
    }
  }
  int x, y, z0, z1;
  if (!zcolumn(lo, hi, nplane, C.zchunk, x, y, z0, z1)) return;
  long long c = at(B, x, y, z0);
#pragma unroll 4
  for (int z = z0; z < z1; ++z, c += B.sz) e[c] = fma(t[c], mone, u[c]);
}

// t = u on the shell cells of every box that lie inside the domain (the
// compute cells get t from k_coarse_rhs), in z-columns of the stored region:
// a column on the ring of the stored plane copies its whole chunk, any other
// column only the chunk's cells below or above the compute region
template <typename T>
__global__ void __launch_bounds__(kZThreads) k_shell_copy(LevelView C, const T* __restrict__ u,
                                                          T* __restrict__ t, int nplane) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = C.boxes[blockIdx.y];
  __syncthreads();
  const int nd[3] = {C.nx, C.ny, C.nz};
  int lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = max(B.lo[d] - 1, 0);
    hi[d] = min(B.hi[d] + 1, nd[d]);
  }
  int x, y, z0, z1;
  if (!zcolumn(lo, hi, nplane, C.zchunk, x, y, z0, z1)) return;
  const bool ring = x < B.lo[0] || x >= B.hi[0] || y < B.lo[1] || y >= B.hi[1];
  if (!ring) {  // only the cells outside the compute region in z
    if (z0 >= B.lo[2]) z0 = max(z0, B.hi[2]);
    if (z1 <= B.hi[2]) z1 = min(z1, B.lo[2]);
  }
  for (int z = z0; z < z1; ++z) {
    if (!ring && z >= B.lo[2] && z < B.hi[2]) continue;
    const long long c = at(B, x, y, z);
    t[c] = u[c];
  }
}

// genuine cells of the box into the global float64 array (out = u or
// out += u), in z-columns
template <typename T>
__global__ void __launch_bounds__(kZThreads) k_gather_zm(LevelView L, const T* __restrict__ u,
                                                         double* __restrict__ out, int add,
                                                         int nplane, Fk<double> k) {
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  int x, y, z0, z1;
  if (!zcolumn(B.glo, B.ghi, nplane, L.zchunk, x, y, z0, z1)) return;
  const long long pz = (long long)L.nx * L.ny;
  long long c = at(B, x, y, z0);
  long long o = (long long)z0 * pz + (long long)y * L.nx + x;
#pragma unroll 4
  for (int z = z0; z < z1; ++z, c += B.sz, o += pz) {
    const double v = widen(u[c]);
    out[o] = add ? fma(v, k.one, out[o]) : v;
  }
}

__global__ void __launch_bounds__(kThreads) k_narrow(const double* __restrict__ in,
                                                      float* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = narrow(in[i]);
}

// per-cell kernels: blocks of kThreads per box, each thread taking L.cpt
// cells of the grid-stride loop (two by default: amortises the box
// descriptor fetch and the block barrier, measured 1-8 % faster than one)
dim3 grid_for(const LevelView& L, int cells) {
  const int per = kThreads * L.cpt;
  int bx = (cells + per - 1) / per;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)L.nbox, 1);
}

unsigned flat_blocks(long long cells) {
  long long blocks = (cells + kThreads - 1) / kThreads;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

double sq(int n) { return (double)n * (double)n; }

}  // namespace

ZTiles ztiles(const LevelView& L) {
  const int plane = L.max_ex * L.max_ey;  // bounds every box's (x, y) plane
  return ZTiles{(plane + kZThreads - 1) / kZThreads, (L.max_ez + L.zchunk - 1) / L.zchunk,
                L.zchunk};
}

dim3 zgrid(const LevelView& L, ZTiles t) {
  return dim3((unsigned)(t.nplane * t.nzc), (unsigned)L.nbox, 1);
}

// z-column tiling of a region no larger than the compute region grown by
// one cell on every side (the stored region)
ZTiles ztiles_stored(const LevelView& L) {
  const int plane = (L.max_ex + 2) * (L.max_ey + 2);
  return ZTiles{(plane + kZThreads - 1) / kZThreads, (L.max_ez + 2 + L.zchunk - 1) / L.zchunk,
                L.zchunk};
}

// float64: per-cell form; float32: column form
template <typename T>
cudaError_t launch_cheb_residual(const LevelView& L, const T* u, T* r, FieldT<T> f,
                                 cudaStream_t s) {
  const T cf = T(1.0 / (6.0 * sq(L.n)));
  if (sizeof(T) == 8) {
    SRFMG_LAUNCH(pdl_launch(k_cheb_residual<T>, grid_for(L, L.max_cells), kThreads, 0, s, L, u, r,
                            f, cf, T(1.0 / 6.0)));
  } else {
    const ZTiles t = ztiles(L);
    SRFMG_LAUNCH(pdl_launch(k_cheb_residual_zm<T>, zgrid(L, t), kZThreads, 0, s, L, u, r, f, cf,
                            T(1.0 / 6.0), t));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb2_update(const LevelView& L, T* u, const T* r, double a, double b,
                                cudaStream_t s) {
  if (sizeof(T) == 8) {
    SRFMG_LAUNCH(pdl_launch(k_cheb2_update<T>, grid_for(L, L.max_cells), kThreads, 0, s, L, u, r,
                            T(a), T(b)));
  } else {
    const ZTiles t = ztiles(L);
    SRFMG_LAUNCH(pdl_launch(k_cheb2_update_zm<T>, zgrid(L, t), kZThreads, 0, s, L, u, r, T(a),
                            T(b), t));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb1_next(const LevelView& L, T* u, const T* r, T* r2, double beta,
                              cudaStream_t s) {
  // float64: per-cell form (float64 pipe bound); float32: column form
  if (sizeof(T) == 8) {
    SRFMG_LAUNCH(pdl_launch(k_cheb1_next<T>, grid_for(L, L.max_cells), kThreads, 0, s, L, u, r,
                            r2, T(beta), T(1.0 - beta), T(beta / 6.0)));
  } else {
    const ZTiles t = ztiles(L);
    SRFMG_LAUNCH(pdl_launch(k_cheb1_next_zm<T>, zgrid(L, t), kZThreads, 0, s, L, u, r, r2,
                            T(beta), T(1.0 - beta), T(beta / 6.0), t));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb_step(const LevelView& L, T* u, T* d, const T* r, double alpha,
                             double beta, int write_d, cudaStream_t s) {
  const ZTiles t = ztiles(L);
  SRFMG_LAUNCH(pdl_launch(k_cheb_step_zm<T>, zgrid(L, t), kZThreads, 0, s, L, u, d, r, T(alpha),
                          T(beta), write_d, t.nplane, fk<T>()));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const LevelView& L, const T* u, T* out, cudaStream_t s) {
  FieldT<T> none{nullptr, L.boxes, 0};
  SRFMG_LAUNCH(pdl_launch(k_apply<T>, grid_for(L, L.max_cells), kThreads, 0, s, L, u, out, none, 0,
                          T(6.0 * sq(L.n)), T(-sq(L.n)), fk<T>()));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const LevelView& L, const T* u, FieldT<T> f, T* r, cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k_apply<T>, grid_for(L, L.max_cells), kThreads, 0, s, L, u, r, f, 1,
                          T(-6.0 * sq(L.n)), T(sq(L.n)), fk<T>()));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid_restrict(const LevelView& F, const T* u, FieldT<T> f,
                                  const LevelView& C, T* uhat_dst, T* rho_dst, cudaStream_t s) {
  const double n2 = sq(F.n);
  if constexpr (sizeof(T) == 4) {
    // coarse z-columns over the restriction region, which lies within half
    // the compute region in each dimension
    const int rx = (F.max_ex + 1) / 2, ry = (F.max_ey + 1) / 2, rz = (F.max_ez + 1) / 2;
    const int nplane = (rx * ry + kZThreads - 1) / kZThreads;
    const int zc = F.zchunk / 4 > 1 ? F.zchunk / 4 : 1;
    const dim3 grid((unsigned)(nplane * ((rz + zc - 1) / zc)), (unsigned)F.nbox, 1);
    SRFMG_LAUNCH(pdl_launch(k_resid_restrict_zm<T>, grid, kZThreads, 0, s, F, u, f, C, uhat_dst,
                            rho_dst, T(-3.0 * n2 / 8.0), T(n2 / 8.0), T(0.125), fk<T>(), nplane,
                            zc));
  } else {
    SRFMG_LAUNCH(pdl_launch(k_resid_restrict<T>, grid_for(F, F.max_restrict), kThreads, 0, s, F,
                            u, f, C, uhat_dst, rho_dst, T(-3.0 * n2 / 8.0), T(n2 / 8.0),
                            T(0.125), fk<T>()));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_rhs(const LevelView& C, const LevelView& F, const T* u, const T* rho,
                              T* rhs, T* t, T* r, cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k_coarse_rhs<T>, grid_for(C, C.max_cells), kThreads, 0, s, C, F, u, rho,
                          rhs, t, r, 6.0 * sq(C.n), -sq(C.n), 1.0 / (6.0 * sq(C.n)), fk<double>()));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_shell_copy(const LevelView& C, const T* u, T* t, cudaStream_t s) {
  const ZTiles z = ztiles_stored(C);
  SRFMG_LAUNCH(pdl_launch(k_shell_copy<T>, zgrid(C, z), kZThreads, 0, s, C, u, t, z.nplane));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transition_rhs(const LevelView& C, const T* t, const T* rho, T* u, T* rhs,
                                  T* r, cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k_transition_rhs<T>, grid_for(C, C.max_cells), kThreads, 0, s, C, t, rho,
                          u, rhs, r, 6.0 * sq(C.n), -sq(C.n), 1.0 / (6.0 * sq(C.n))));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const LevelView& C, const T* uc, const LevelView& F, T* uf, int add,
                           cudaStream_t s) {
  // float32: columns twice the handle's z-chunk (each coarse plane's bilinear
  // values then serve more fine cells; 1.50 -> 1.33 ms and 2.28 -> 2.16 ms for
  // the FMG and correction prolongations of a 512^3 mixed solve, while the
  // float64 kernel and the smoother passes are fastest at the chunk itself)
  LevelView Fz = F;
  if (sizeof(T) == 4) Fz.zchunk = 2 * F.zchunk;
  const ZTiles z = ztiles_stored(Fz);  // the prolongation range lies in the stored region
  if constexpr (sizeof(T) == 8) {
    SRFMG_LAUNCH(pdl_launch(k_prolong_zcol<T, 2>, zgrid(Fz, z), kZThreads, 0, s, C, uc, Fz, uf,
                            add, T(3.0), T(1.0 / 64.0), z.nplane, fk<T>()));
  } else if (add) {
    SRFMG_LAUNCH(pdl_launch(k_prolong_zcol<T, 1>, zgrid(Fz, z), kZThreads, 0, s, C, uc, Fz, uf,
                            add, T(3.0), T(1.0 / 64.0), z.nplane, fk<T>()));
  } else {
    SRFMG_LAUNCH(pdl_launch(k_prolong_zcol<T, 0>, zgrid(Fz, z), kZThreads, 0, s, C, uc, Fz, uf,
                            add, T(3.0), T(1.0 / 64.0), z.nplane, fk<T>()));
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diff(const LevelView& C, const T* u, const T* t, T* e, cudaStream_t s,
                        int prolong_range) {
  const ZTiles z = ztiles_stored(C);
  SRFMG_LAUNCH(pdl_launch(k_diff_zm<T>, zgrid(C, z), kZThreads, 0, s, C, u, t, e, z.nplane,
                          T(-1.0), prolong_range));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(const LevelView& L, const double* minv, FieldT<T> f, T* u,
                                cudaStream_t s) {
  const int m = L.nx * L.ny * L.nz;
  const int warps_per_block = 8;
  const int blocks = (m + warps_per_block - 1) / warps_per_block;
  SRFMG_LAUNCH(pdl_launch(k_coarse_solve<T>, blocks, warps_per_block * 32, 0, s, L, minv, f, u,
                          fk<double>()));
  return cudaGetLastError();
}

int sep_lanes(const LevelView& L) {
  const int m = max(L.nx, max(L.ny, L.nz));
  int W = 1;
  while (W < m) W *= 2;
  return W;
}

unsigned sep_blocks(int tasks, int W) {
  const long long threads = (long long)tasks * W;
  return (unsigned)((threads + 63) / 64);
}

template <typename T>
cudaError_t launch_coarse_solve_sep(const LevelView& L, const double* sep, double* g, double* q,
                                    FieldT<T> f, T* u, cudaStream_t s) {
  const int W = sep_lanes(L);
  if (W > 32) return cudaErrorInvalidValue;
  SRFMG_LAUNCH(pdl_launch(k_sep_fwd_xy<T>, sep_blocks(L.nz * L.ny, W), 64, 0, s, L, f, sep, g, W,
                          fk<double>()));
  SRFMG_LAUNCH(pdl_launch(k_sep_z, sep_blocks(L.ny * L.nx, W), 64, 0, s, L.nx, L.ny, L.nz, sep,
                          (const double*)g, q, W, fk<double>()));
  SRFMG_LAUNCH(pdl_launch(k_sep_inv_xy<T>, sep_blocks(L.nz * L.ny, W), 64, 0, s, L, sep,
                          (const double*)q, u, W, fk<double>()));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict_global(Dims fd, const T* ff, T* fc, int check, unsigned int* status,
                                   cudaStream_t s) {
  const long long cells = (long long)(fd.x / 2) * (fd.y / 2) * (fd.z / 2);
  SRFMG_LAUNCH(pdl_launch(k_restrict_global<T>, flat_blocks(cells), kThreads, 0, s, fd, ff, fc,
                          check, status, T(0.125), fk<T>()));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_genuine(const LevelView& L, const T* u, double* out, int add,
                                  cudaStream_t s) {
  const ZTiles z = ztiles(L);  // the genuine region lies inside the compute region
  SRFMG_LAUNCH(pdl_launch(k_gather_zm<T>, zgrid(L, z), kZThreads, 0, s, L, u, out, add, z.nplane,
                          fk<double>()));
  return cudaGetLastError();
}

cudaError_t launch_defect(Dims g, int n, const double* f, const double* u, float* d,
                          unsigned int* status, cudaStream_t s) {
  const long long cells = (long long)g.x * g.y * g.z;
  SRFMG_LAUNCH(pdl_launch(k_defect, flat_blocks(cells), kThreads, 0, s, g, f, u, d, status,
                          -6.0 * sq(n), sq(n)));
  return cudaGetLastError();
}

cudaError_t launch_resid_norm(Dims g, int n, const double* f, const double* u,
                              unsigned long long* norm, unsigned int* status, cudaStream_t s) {
  const long long cells = (long long)g.x * g.y * g.z;
  SRFMG_LAUNCH(pdl_launch(k_resid_norm, flat_blocks(cells), kThreads, 0, s, g, f, u, norm, status,
                          -6.0 * sq(n), sq(n)));
  return cudaGetLastError();
}

cudaError_t launch_accumulate(long long cells, const float* e, double* u, int add,
                              cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k_accumulate, flat_blocks(cells), kThreads, 0, s, cells, e, u, add,
                          fk<double>()));
  return cudaGetLastError();
}

cudaError_t launch_narrow(const double* in, float* out, long long n, cudaStream_t s) {
  k_narrow<<<flat_blocks(n), kThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

#define SRFMG_INSTANTIATE(T)                                                                   \
  template cudaError_t launch_cheb_residual<T>(const LevelView&, const T*, T*, FieldT<T>,      \
                                               cudaStream_t);                                  \
  template cudaError_t launch_cheb2_update<T>(const LevelView&, T*, const T*, double, double,  \
                                              cudaStream_t);                                   \
  template cudaError_t launch_cheb1_next<T>(const LevelView&, T*, const T*, T*, double,        \
                                            cudaStream_t);                                     \
  template cudaError_t launch_cheb_step<T>(const LevelView&, T*, T*, const T*, double, double, \
                                           int, cudaStream_t);                                 \
  template cudaError_t launch_apply<T>(const LevelView&, const T*, T*, cudaStream_t);          \
  template cudaError_t launch_residual<T>(const LevelView&, const T*, FieldT<T>, T*,           \
                                          cudaStream_t);                                       \
  template cudaError_t launch_resid_restrict<T>(const LevelView&, const T*, FieldT<T>,         \
                                                const LevelView&, T*, T*, cudaStream_t);       \
  template cudaError_t launch_coarse_rhs<T>(const LevelView&, const LevelView&, const T*,      \
                                            const T*, T*, T*, T*, cudaStream_t);               \
  template cudaError_t launch_shell_copy<T>(const LevelView&, const T*, T*, cudaStream_t);     \
  template cudaError_t launch_transition_rhs<T>(const LevelView&, const T*, const T*, T*, T*,  \
                                                T*, cudaStream_t);                             \
  template cudaError_t launch_prolong<T>(const LevelView&, const T*, const LevelView&, T*, int, \
                                         cudaStream_t);                                        \
  template cudaError_t launch_diff<T>(const LevelView&, const T*, const T*, T*, cudaStream_t,   \
                                      int);                                                    \
  template cudaError_t launch_coarse_solve<T>(const LevelView&, const double*, FieldT<T>, T*,  \
                                              cudaStream_t);                                   \
  template cudaError_t launch_coarse_solve_sep<T>(const LevelView&, const double*, double*,    \
                                                  double*, FieldT<T>, T*, cudaStream_t);       \
  template cudaError_t launch_restrict_global<T>(Dims, const T*, T*, int, unsigned int*,       \
                                                 cudaStream_t);                                \
  template cudaError_t launch_gather_genuine<T>(const LevelView&, const T*, double*, int,      \
                                                cudaStream_t);

SRFMG_INSTANTIATE(double)
SRFMG_INSTANTIATE(float)

}  // namespace srfmg
