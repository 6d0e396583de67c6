// FP64 kernels of the FMG / SR-FMG solver (sm_103a).
//
// Every kernel runs over the boxes of one level: blockIdx.y selects the box
// (one per segment on an SR level, a single box on a global level) and the
// threads of blockIdx.x stride over the cells of the kernel's region in x-
// fastest order.  On GB300 the float64 pipe (two lanes per clock per SM) is
// the binding resource for these stencils, far below what HBM can feed, so
// the kernels are written to spend as few float64 instructions per cell as
// the arithmetic allows:
//   - ghost cells outside the domain are never stored: a neighbour outside
//     the domain is replaced by minus the mirror cell on the fly (Sec. 3.3),
//     with the sign flip done on the integer pipe;
//   - the degree-2 Chebyshev smoother is evaluated as x2 = x0 + a r0 + b S(r0)
//     (two stencil passes, 14 float64 operations per cell) instead of the
//     three-term recurrence (19);
//   - the residual of the 8 children of a coarse cell is summed through the
//     24 faces of the 2x2x2 block (41 operations per coarse cell instead of 72).
#include "srfmg_internal.cuh"

namespace srfmg {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ long long at(const BoxDesc& b, int x, int y, int z) {
  return b.base + (long long)(z - b.oz) * b.sz + (long long)(y - b.oy) * b.sy + (x - b.ox);
}

// -v, by flipping the sign bit on the integer pipe
__device__ __forceinline__ double negd(double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
}

// v or -v, selected on the integer pipe
__device__ __forceinline__ double neg_if(double v, bool flip) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)flip << 63));
}

__device__ __forceinline__ void region_of(const BoxDesc& b, int which, int lo[3], int hi[3]) {
  const int* l = b.lo;
  const int* h = b.hi;
  if (which == kProlong) { l = b.plo; h = b.phi; }
  if (which == kRestrict) { l = b.rlo; h = b.rhi; }
  if (which == kGenuine) { l = b.glo; h = b.ghi; }
#pragma unroll
  for (int d = 0; d < 3; ++d) { lo[d] = l[d]; hi[d] = h[d]; }
}

// Sum of the six neighbours of stored cell c at (x, y, z); a neighbour outside
// [0, n) is minus the centre value (mirror through u = 0 on the face).
__device__ __forceinline__ double neighbour_sum(const double* __restrict__ a, long long c,
                                                const BoxDesc& b, int n, int x, int y, int z,
                                                double centre) {
  const double m = negd(centre);
  const double xm = (x > 0) ? a[c - 1] : m;
  const double xp = (x < n - 1) ? a[c + 1] : m;
  const double ym = (y > 0) ? a[c - b.sy] : m;
  const double yp = (y < n - 1) ? a[c + b.sy] : m;
  const double zm = (z > 0) ? a[c - b.sz] : m;
  const double zp = (z < n - 1) ? a[c + b.sz] : m;
  return ((xm + xp) + (ym + yp)) + (zm + zp);
}

struct Cell {
  int x, y, z;
};

__device__ __forceinline__ Cell cell_of(int i, const int lo[3], int ex, int ey) {
  Cell c;
  c.x = lo[0] + i % ex;
  const int t = i / ex;
  c.y = lo[1] + t % ey;
  c.z = lo[2] + t / ey;
  return c;
}

// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads) k_cheb_residual(LevelView L,
                                                            const double* __restrict__ u,
                                                            double* __restrict__ r, FieldView f,
                                                            double cf) {
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  const int n = L.n;
  constexpr double sixth = 1.0 / 6.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double uc = u[c];
    const double s = neighbour_sum(u, c, B, n, q.x, q.y, q.z, uc);
    const double fv = f.p[at(FB, q.x, q.y, q.z)];
    // D^-1 (f - A u) = f h^2/6 - u + s/6
    r[c] = fma(s, sixth, fma(fv, cf, negd(uc)));
  }
}

__global__ void __launch_bounds__(kThreads) k_cheb2_update(LevelView L, double* __restrict__ u,
                                                           const double* __restrict__ r,
                                                           double a, double b) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  const int n = L.n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double rc = r[c];
    const double s = neighbour_sum(r, c, B, n, q.x, q.y, q.z, rc);
    u[c] = fma(b, s, fma(a, rc, u[c]));
  }
}

__global__ void __launch_bounds__(kThreads) k_cheb_step(LevelView L, double* __restrict__ u,
                                                        double* __restrict__ d,
                                                        const double* __restrict__ r,
                                                        double alpha, double beta, int write_d) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double dn = (alpha != 0.0) ? fma(alpha, d[c], beta * r[c]) : beta * r[c];
    if (write_d) d[c] = dn;
    u[c] += dn;
  }
}

__global__ void __launch_bounds__(kThreads) k_apply(LevelView L, const double* __restrict__ u,
                                                    double* __restrict__ out, FieldView f,
                                                    int residual) {
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = residual ? (f.single ? f.boxes[0] : f.boxes[blockIdx.y]) : B;
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  const int n = L.n;
  const double ih2 = (double)n * (double)n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double uc = u[c];
    const double s = neighbour_sum(u, c, B, n, q.x, q.y, q.z, uc);
    const double au = fma(6.0, uc, negd(s));
    out[c] = residual ? fma(-ih2, au, f.p[at(FB, q.x, q.y, q.z)]) : ih2 * au;
  }
}

// Residual of the 8 children of each coarse cell, restricted, and the
// restricted solution.  With S the sum of the children, the children's
// operator values add up to n^2 (3 S - O), O the sum of the 24 neighbours
// across the outer faces of the 2x2x2 block (each inner face cancels).
__global__ void __launch_bounds__(kThreads) k_resid_restrict(LevelView F,
                                                             const double* __restrict__ u,
                                                             FieldView f, LevelView C,
                                                             double* __restrict__ uhat_dst,
                                                             double* __restrict__ rho_dst) {
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
  const int n = F.n;
  const double ih2 = (double)n * (double)n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, lo, ex, ey);
    const int x0 = 2 * q.x, y0 = 2 * q.y, z0 = 2 * q.z;
    const long long c0 = at(B, x0, y0, z0);
    const long long sy = B.sy, sz = B.sz;
    double v[2][2][2];
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) v[cz][cy][cx] = u[c0 + cz * sz + cy * sy + cx];
    double fs = 0.0;
    {
      const long long f0 = at(FB, x0, y0, z0);
      const long long fy = FB.sy, fz = FB.sz;
      fs = ((f.p[f0] + f.p[f0 + 1]) + (f.p[f0 + fy] + f.p[f0 + fy + 1])) +
           ((f.p[f0 + fz] + f.p[f0 + fz + 1]) + (f.p[f0 + fz + fy] + f.p[f0 + fz + fy + 1]));
    }
    const double S = ((v[0][0][0] + v[0][0][1]) + (v[0][1][0] + v[0][1][1])) +
                     ((v[1][0][0] + v[1][0][1]) + (v[1][1][0] + v[1][1][1]));
    // the 24 outer neighbours, mirrored with a sign flip outside the domain
    const bool xl = x0 > 0, xr = x0 + 2 < n, yl = y0 > 0, yr = y0 + 2 < n, zl = z0 > 0,
               zr = z0 + 2 < n;
    double O = 0.0;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        const long long row = c0 + cz * sz + cy * sy;
        const double a = xl ? u[row - 1] : negd(v[cz][cy][0]);
        const double b = xr ? u[row + 2] : negd(v[cz][cy][1]);
        O += a + b;
      }
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const long long col = c0 + cz * sz + cx;
        const double a = yl ? u[col - sy] : negd(v[cz][0][cx]);
        const double b = yr ? u[col + 2 * sy] : negd(v[cz][1][cx]);
        O += a + b;
      }
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const long long pil = c0 + cy * sy + cx;
        const double a = zl ? u[pil - sz] : negd(v[0][cy][cx]);
        const double b = zr ? u[pil + 2 * sz] : negd(v[1][cy][cx]);
        O += a + b;
      }
    const long long cc = at(CB, q.x, q.y, q.z);
    const double au = fma(3.0, S, negd(O));  // h^2 * sum of the children's A u
    rho_dst[cc] = 0.125 * fma(-ih2, au, fs);
    uhat_dst[cc] = 0.125 * S;
  }
}

__global__ void __launch_bounds__(kThreads) k_coarse_rhs(LevelView C, LevelView F,
                                                         const double* __restrict__ u,
                                                         const double* __restrict__ rho,
                                                         double* __restrict__ rhs,
                                                         double* __restrict__ t) {
  __shared__ BoxDesc B, FBx;
  if (threadIdx.x == 0) {
    B = C.boxes[blockIdx.y];
    FBx = (F.nbox == 1) ? F.boxes[0] : F.boxes[blockIdx.y];
  }
  __syncthreads();
  const int n = C.n;
  const double ih2 = (double)n * (double)n;
  const bool shell = B.ox < B.lo[0];
  int lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = shell ? B.lo[d] - 1 : B.lo[d];
    hi[d] = shell ? B.hi[d] + 1 : B.hi[d];
  }
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, lo, ex, ey);
    const bool inside_domain = q.x >= 0 && q.x < n && q.y >= 0 && q.y < n && q.z >= 0 && q.z < n;
    if (!inside_domain) continue;
    const long long c = at(B, q.x, q.y, q.z);
    const double uc = u[c];
    t[c] = uc;
    const bool compute = q.x >= B.lo[0] && q.x < B.hi[0] && q.y >= B.lo[1] && q.y < B.hi[1] &&
                         q.z >= B.lo[2] && q.z < B.hi[2];
    if (!compute) continue;
    const bool inF = q.x >= FBx.rlo[0] && q.x < FBx.rhi[0] && q.y >= FBx.rlo[1] &&
                     q.y < FBx.rhi[1] && q.z >= FBx.rlo[2] && q.z < FBx.rhi[2];
    const double s = neighbour_sum(u, c, B, n, q.x, q.y, q.z, uc);
    const double au = fma(6.0, uc, negd(s));
    rhs[c] = inF ? fma(ih2, au, rho[c]) : ih2 * au;
  }
}

__global__ void __launch_bounds__(kThreads) k_transition_rhs(LevelView C,
                                                             const double* __restrict__ t,
                                                             const double* __restrict__ rho,
                                                             double* __restrict__ u,
                                                             double* __restrict__ rhs) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = C.boxes[0];
  __syncthreads();
  const int n = C.n;
  const double ih2 = (double)n * (double)n;
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double tc = t[c];
    const double s = neighbour_sum(t, c, B, n, q.x, q.y, q.z, tc);
    u[c] = tc;
    rhs[c] = fma(ih2, fma(6.0, tc, negd(s)), rho[c]);
  }
}

// coarse value for trilinear interpolation: mirrored with a sign flip outside
// the domain; with tc != nullptr the value is uc - tc.
__device__ __forceinline__ double coarse_value(const double* __restrict__ uc,
                                               const double* __restrict__ tc,
                                               const BoxDesc& C, int nc, int x, int y, int z) {
  bool flip = false;
  if (x < 0) { x = 0; flip = !flip; } else if (x >= nc) { x = nc - 1; flip = !flip; }
  if (y < 0) { y = 0; flip = !flip; } else if (y >= nc) { y = nc - 1; flip = !flip; }
  if (z < 0) { z = 0; flip = !flip; } else if (z >= nc) { z = nc - 1; flip = !flip; }
  const long long i = at(C, x, y, z);
  const double v = tc ? uc[i] - tc[i] : uc[i];
  return neg_if(v, flip);
}

// Trilinear prolongation in factored form: with 1D weights 3/4 (own coarse
// cell) and 1/4 (neighbour), the fine value is (1/64) * the x, y, z passes of
// 3 a + b.
__global__ void __launch_bounds__(kThreads) k_prolong(LevelView C, const double* __restrict__ uc,
                                                      const double* __restrict__ tc, LevelView F,
                                                      double* __restrict__ uf, int add) {
  __shared__ BoxDesc B, CB;
  if (threadIdx.x == 0) {
    B = F.boxes[blockIdx.y];
    CB = (C.nbox == 1) ? C.boxes[0] : C.boxes[blockIdx.y];
  }
  __syncthreads();
  int lo[3], hi[3];
  region_of(B, kProlong, lo, hi);
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int ncell = ex * ey * ez;
  const int nc = C.n;
  const double* tcp = add ? tc : nullptr;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, lo, ex, ey);
    const int cx = q.x >> 1, cy = q.y >> 1, cz = q.z >> 1;
    const int nx = (q.x & 1) ? cx + 1 : cx - 1;
    const int ny = (q.y & 1) ? cy + 1 : cy - 1;
    const int nz = (q.z & 1) ? cz + 1 : cz - 1;
    const int xs[2] = {cx, nx}, ys[2] = {cy, ny}, zs[2] = {cz, nz};
    double pz[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      double py[2];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const double v0 = coarse_value(uc, tcp, CB, nc, xs[0], ys[b], zs[a]);
        const double v1 = coarse_value(uc, tcp, CB, nc, xs[1], ys[b], zs[a]);
        py[b] = fma(3.0, v0, v1);
      }
      pz[a] = fma(3.0, py[0], py[1]);
    }
    const double e = fma(3.0, pz[0], pz[1]);
    const long long c = at(B, q.x, q.y, q.z);
    constexpr double w = 1.0 / 64.0;
    if (add)
      uf[c] = fma(w, e, uf[c]);
    else
      uf[c] = w * e;
  }
}

// One warp per row of the dense inverse.
__global__ void k_coarse_solve(LevelView L, const double* __restrict__ minv, FieldView f,
                               double* __restrict__ u) {
  const BoxDesc B = L.boxes[0];
  const BoxDesc FB = f.boxes[0];
  const int n = L.n, m = n * n * n;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  double s = 0.0;
  for (int j = lane; j < m; j += 32) {
    const int x = j % n, y = (j / n) % n, z = j / (n * n);
    s = fma(minv[(long long)warp * m + j], f.p[at(FB, x, y, z)], s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const int x = warp % n, y = (warp / n) % n, z = warp / (n * n);
    u[at(B, x, y, z)] = s;
  }
}

__device__ __forceinline__ bool not_finite(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
}

__global__ void __launch_bounds__(kThreads) k_restrict_global(int nf, const double* __restrict__ ff,
                                                              double* __restrict__ fc, int check,
                                                              unsigned int* status) {
  const int nc = nf / 2;
  const long long ncell = (long long)nc * nc * nc;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nc);
    const long long t = i / nc;
    const int y = (int)(t % nc), z = (int)(t / nc);
    const long long f0 = ((long long)(2 * z) * nf + 2 * y) * nf + 2 * x;
    const long long py = nf, pz = (long long)nf * nf;
    const double a0 = ff[f0], a1 = ff[f0 + 1], a2 = ff[f0 + py], a3 = ff[f0 + py + 1];
    const double a4 = ff[f0 + pz], a5 = ff[f0 + pz + 1], a6 = ff[f0 + pz + py],
                 a7 = ff[f0 + pz + py + 1];
    if (check)
      bad |= not_finite(a0) | not_finite(a1) | not_finite(a2) | not_finite(a3) | not_finite(a4) |
             not_finite(a5) | not_finite(a6) | not_finite(a7);
    fc[i] = 0.125 * (((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7)));
  }
  if (check && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1u);
}

__global__ void __launch_bounds__(kThreads) k_gather_genuine(LevelView L,
                                                             const double* __restrict__ u,
                                                             double* __restrict__ out) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  int lo[3], hi[3];
  region_of(B, kGenuine, lo, hi);
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int ncell = ex * ey * ez;
  const long long n = L.n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell q = cell_of(i, lo, ex, ey);
    out[(q.z * n + q.y) * n + q.x] = u[at(B, q.x, q.y, q.z)];
  }
}

dim3 grid_for(const LevelView& L, int cells) {
  int bx = (cells + kThreads - 1) / kThreads;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)L.nbox, 1);
}

}  // namespace

cudaError_t launch_cheb_residual(const LevelView& L, const double* u, double* r, FieldView f,
                                 cudaStream_t s) {
  const double cf = 1.0 / (6.0 * (double)L.n * (double)L.n);
  k_cheb_residual<<<grid_for(L, L.max_cells), kThreads, 0, s>>>(L, u, r, f, cf);
  return cudaGetLastError();
}

cudaError_t launch_cheb2_update(const LevelView& L, double* u, const double* r, double a, double b,
                                cudaStream_t s) {
  k_cheb2_update<<<grid_for(L, L.max_cells), kThreads, 0, s>>>(L, u, r, a, b);
  return cudaGetLastError();
}

cudaError_t launch_cheb_step(const LevelView& L, double* u, double* d, const double* r,
                             double alpha, double beta, int write_d, cudaStream_t s) {
  k_cheb_step<<<grid_for(L, L.max_cells), kThreads, 0, s>>>(L, u, d, r, alpha, beta, write_d);
  return cudaGetLastError();
}

cudaError_t launch_apply(const LevelView& L, const double* u, double* out, cudaStream_t s) {
  FieldView none{nullptr, L.boxes, 0};
  k_apply<<<grid_for(L, L.max_cells), kThreads, 0, s>>>(L, u, out, none, 0);
  return cudaGetLastError();
}

cudaError_t launch_residual(const LevelView& L, const double* u, FieldView f, double* r,
                            cudaStream_t s) {
  k_apply<<<grid_for(L, L.max_cells), kThreads, 0, s>>>(L, u, r, f, 1);
  return cudaGetLastError();
}

cudaError_t launch_resid_restrict(const LevelView& F, const double* u, FieldView f,
                                  const LevelView& C, double* uhat_dst, double* rho_dst,
                                  cudaStream_t s) {
  k_resid_restrict<<<grid_for(F, F.max_restrict), kThreads, 0, s>>>(F, u, f, C, uhat_dst,
                                                                    rho_dst);
  return cudaGetLastError();
}

cudaError_t launch_coarse_rhs(const LevelView& C, const LevelView& F, const double* u,
                              const double* rho, double* rhs, double* t, cudaStream_t s) {
  k_coarse_rhs<<<grid_for(C, C.max_stored), kThreads, 0, s>>>(C, F, u, rho, rhs, t);
  return cudaGetLastError();
}

cudaError_t launch_transition_rhs(const LevelView& C, const double* t, const double* rho,
                                  double* u, double* rhs, cudaStream_t s) {
  k_transition_rhs<<<grid_for(C, C.max_cells), kThreads, 0, s>>>(C, t, rho, u, rhs);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const LevelView& C, const double* uc, const double* tc,
                           const LevelView& F, double* uf, int add, cudaStream_t s) {
  k_prolong<<<grid_for(F, F.max_prolong), kThreads, 0, s>>>(C, uc, tc, F, uf, add);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const LevelView& L, const double* minv, FieldView f, double* u,
                                cudaStream_t s) {
  const int m = L.n * L.n * L.n;
  const int warps_per_block = 8;
  const int blocks = (m + warps_per_block - 1) / warps_per_block;
  k_coarse_solve<<<blocks, warps_per_block * 32, 0, s>>>(L, minv, f, u);
  return cudaGetLastError();
}

cudaError_t launch_restrict_global(int nf, const double* ff, double* fc, int check,
                                   unsigned int* status, cudaStream_t s) {
  const long long nc = nf / 2;
  const long long cells = nc * nc * nc;
  long long blocks = (cells + kThreads - 1) / kThreads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  k_restrict_global<<<(unsigned)blocks, kThreads, 0, s>>>(nf, ff, fc, check, status);
  return cudaGetLastError();
}

cudaError_t launch_gather_genuine(const LevelView& L, const double* u, double* out,
                                  cudaStream_t s) {
  k_gather_genuine<<<grid_for(L, L.max_genuine), kThreads, 0, s>>>(L, u, out);
  return cudaGetLastError();
}

}  // namespace srfmg
