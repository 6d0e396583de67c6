// Kernels of the 27-point operator (float64), the operator of the paper's
// experiments (Sec. 5.1: "27-point finite volume stencil"):
//   A u = n^2 (w0 u - w1 (6 face neighbours) - w2 (12 edge neighbours)
//              - w3 (8 corner neighbours)),   w0 = 6 w1 + 12 w2 + 8 w3,
// h = 1/n.  Same region conventions as the 7-point kernels (kernels.cu):
// blockIdx.y selects the box, threads stride over the region's cells in
// x-fastest order.  A neighbour outside the domain is its mirror cell with the
// sign flipped once per dimension it lies outside (Sec. 3.3 applied per
// dimension, so edge and corner ghosts of the reflection are exact); a
// neighbour inside the domain but outside the box's compute region is read
// from the box's one-cell shell (frozen SR ghosts, or zero in the smoother's
// residual array).  These kernels read every neighbour through the L1 cache;
// the operator is used for the paper's accuracy experiments, not for the
// 7-point throughput path.
#include "srfmg_internal.cuh"

namespace srfmg {
namespace {

constexpr int kThreads27 = 256;

struct Cell27 {
  int x, y, z;
};

__device__ __forceinline__ long long at27(const BoxDesc& b, int x, int y, int z) {
  return b.base + (long long)(z - b.oz) * b.sz + (long long)(y - b.oy) * b.sy + (x - b.ox);
}

__device__ __forceinline__ Cell27 cell27(int i, const int lo[3], int ex, int ey) {
  Cell27 c;
  c.x = lo[0] + i % ex;
  const int t = i / ex;
  c.y = lo[1] + t % ey;
  c.z = lo[2] + t / ey;
  return c;
}

// sums of the face, edge and corner neighbours of cell (x, y, z) of box B
// on a level grid of nx x ny x nz cells
__device__ __forceinline__ void sums27(const double* __restrict__ a, const BoxDesc& B, int nx,
                                       int ny, int nz, int x, int y, int z, double s[3]) {
  s[0] = s[1] = s[2] = 0.0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    int zz = z + dz;
    const bool oz = zz < 0 || zz >= nz;
    zz = oz ? z : zz;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = y + dy;
      const bool oy = yy < 0 || yy >= ny;
      yy = oy ? y : yy;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int far = (dx != 0) + (dy != 0) + (dz != 0);
        if (far == 0) continue;
        int xx = x + dx;
        const bool ox = xx < 0 || xx >= nx;
        xx = ox ? x : xx;
        const double v = a[at27(B, xx, yy, zz)];
        s[far - 1] += (ox ^ oy ^ oz) ? -v : v;
      }
    }
  }
}

__device__ __forceinline__ bool finite27(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

// r = D^-1 (f - A u) = f h^2/w0 - u + (w1 sf + w2 se + w3 sc)/w0
__global__ void __launch_bounds__(kThreads27) k27_cheb_residual(LevelView L,
                                                                const double* __restrict__ u,
                                                                double* __restrict__ r,
                                                                FieldT<double> f, double cf,
                                                                double cf1, double ce, double cc) {
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell27 q = cell27(i, B.lo, ex, ey);
    const long long c = at27(B, q.x, q.y, q.z);
    double s[3];
    sums27(u, B, L.nx, L.ny, L.nz, q.x, q.y, q.z, s);
    r[c] = f.p[at27(FB, q.x, q.y, q.z)] * cf - u[c] + cf1 * s[0] + ce * s[1] + cc * s[2];
  }
}

// u += a r + bf sf(r) + be se(r) + bc sc(r): the degree-2 Chebyshev
// polynomial x0 + c1 r0 + c2 D^-1 A r0 written with D^-1 A = I - W
__global__ void __launch_bounds__(kThreads27) k27_cheb2_update(LevelView L, double* __restrict__ u,
                                                               const double* __restrict__ r,
                                                               double a, double bf, double be,
                                                               double bc) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[blockIdx.y];
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell27 q = cell27(i, B.lo, ex, ey);
    const long long c = at27(B, q.x, q.y, q.z);
    double s[3];
    sums27(r, B, L.nx, L.ny, L.nz, q.x, q.y, q.z, s);
    u[c] += a * r[c] + bf * s[0] + be * s[1] + bc * s[2];
  }
}

// n^2 (w0 v - w1 sf - w2 se - w3 sc) at (x, y, z)
__device__ __forceinline__ double op27(const double* __restrict__ a, const BoxDesc& B,
                                       const LevelView& L, W27 w, double n2, int x, int y,
                                       int z) {
  double s[3];
  sums27(a, B, L.nx, L.ny, L.nz, x, y, z, s);
  return n2 * (w.w0 * a[at27(B, x, y, z)] - w.w1 * s[0] - w.w2 * s[1] - w.w3 * s[2]);
}

// residual == 0: out = A u;  residual == 1: out = f - A u
__global__ void __launch_bounds__(kThreads27) k27_apply(LevelView L, const double* __restrict__ u,
                                                        double* __restrict__ out,
                                                        FieldT<double> f, int residual, W27 w,
                                                        double n2) {
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = residual ? (f.single ? f.boxes[0] : f.boxes[blockIdx.y]) : B;
  }
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell27 q = cell27(i, B.lo, ex, ey);
    const double au = op27(u, B, L, w, n2, q.x, q.y, q.z);
    out[at27(B, q.x, q.y, q.z)] = residual ? f.p[at27(FB, q.x, q.y, q.z)] - au : au;
  }
}

// per coarse cell of the fine boxes' restriction region: uhat = average of
// the 8 children of u, rho = average of the 8 children of f - A u
__global__ void __launch_bounds__(kThreads27) k27_resid_restrict(LevelView F,
                                                                 const double* __restrict__ u,
                                                                 FieldT<double> f, LevelView C,
                                                                 double* __restrict__ uhat_dst,
                                                                 double* __restrict__ rho_dst,
                                                                 W27 w, double n2) {
  __shared__ BoxDesc B, FB, CB;
  if (threadIdx.x == 0) {
    B = F.boxes[blockIdx.y];
    FB = f.single ? f.boxes[0] : f.boxes[blockIdx.y];
    CB = (C.nbox == 1) ? C.boxes[0] : C.boxes[blockIdx.y];
  }
  __syncthreads();
  const int lo[3] = {B.rlo[0], B.rlo[1], B.rlo[2]};
  const int ex = B.rhi[0] - lo[0], ey = B.rhi[1] - lo[1], ez = B.rhi[2] - lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell27 q = cell27(i, lo, ex, ey);
    double su = 0.0, sr = 0.0;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const int x = 2 * q.x + cx, y = 2 * q.y + cy, z = 2 * q.z + cz;
          su += u[at27(B, x, y, z)];
          sr += f.p[at27(FB, x, y, z)] - op27(u, B, F, w, n2, x, y, z);
        }
    const long long cc = at27(CB, q.x, q.y, q.z);
    uhat_dst[cc] = 0.125 * su;
    rho_dst[cc] = 0.125 * sr;
  }
}

// rhs = rho + A u inside the matching fine box's restriction region, A u on
// the rest of the compute region; t = u on the whole stored box
__global__ void __launch_bounds__(kThreads27) k27_coarse_rhs(LevelView C, LevelView F,
                                                             const double* __restrict__ u,
                                                             const double* __restrict__ rho,
                                                             double* __restrict__ rhs,
                                                             double* __restrict__ t, W27 w,
                                                             double n2) {
  __shared__ BoxDesc B, FBx;
  if (threadIdx.x == 0) {
    B = C.boxes[blockIdx.y];
    FBx = (F.nbox == 1) ? F.boxes[0] : F.boxes[blockIdx.y];
  }
  __syncthreads();
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
    const Cell27 q = cell27(i, lo, ex, ey);
    const bool inside_domain =
        q.x >= 0 && q.x < C.nx && q.y >= 0 && q.y < C.ny && q.z >= 0 && q.z < C.nz;
    if (!inside_domain) continue;
    const long long c = at27(B, q.x, q.y, q.z);
    t[c] = u[c];
    const bool compute = q.x >= B.lo[0] && q.x < B.hi[0] && q.y >= B.lo[1] && q.y < B.hi[1] &&
                         q.z >= B.lo[2] && q.z < B.hi[2];
    if (!compute) continue;
    const bool inF = q.x >= FBx.rlo[0] && q.x < FBx.rhi[0] && q.y >= FBx.rlo[1] &&
                     q.y < FBx.rhi[1] && q.z >= FBx.rlo[2] && q.z < FBx.rhi[2];
    const double au = op27(u, B, C, w, n2, q.x, q.y, q.z);
    rhs[c] = inF ? rho[c] + au : au;
  }
}

// u = t, rhs = rho + A t on the whole (global) transition level
__global__ void __launch_bounds__(kThreads27) k27_transition_rhs(LevelView C,
                                                                 const double* __restrict__ t,
                                                                 const double* __restrict__ rho,
                                                                 double* __restrict__ u,
                                                                 double* __restrict__ rhs, W27 w,
                                                                 double n2) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = C.boxes[0];
  __syncthreads();
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell27 q = cell27(i, B.lo, ex, ey);
    const long long c = at27(B, q.x, q.y, q.z);
    u[c] = t[c];
    rhs[c] = rho[c] + op27(t, B, C, w, n2, q.x, q.y, q.z);
  }
}

// *norm = max |f - A u| (|f| when u is null) over the whole unpadded level,
// as the bits of the non-negative double; *status |= 1 on a value that is not
// finite
__global__ void __launch_bounds__(kThreads27) k27_resid_norm(LevelView L,
                                                             const double* __restrict__ f,
                                                             const double* __restrict__ u,
                                                             unsigned long long* norm,
                                                             unsigned int* status, W27 w,
                                                             double n2) {
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[0];
  __syncthreads();
  const long long ncell = (long long)L.nx * L.ny * L.nz;
  unsigned long long m = 0;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % L.nx);
    const long long t = i / L.nx;
    const int y = (int)(t % L.ny), z = (int)(t / L.ny);
    double r = f[i];
    if (u) r -= op27(u, B, L, w, n2, x, y, z);
    bad |= !finite27(r);
    const unsigned long long a =
        (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(status, 1u);
    atomicMax(norm, m);
  }
}

dim3 grid27(const LevelView& L, int cells) {
  int bx = (cells + kThreads27 - 1) / kThreads27;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)L.nbox, 1);
}

double sq27(int n) { return (double)n * (double)n; }

}  // namespace

cudaError_t launch27_cheb_residual(const LevelView& L, const double* u, double* r,
                                   FieldT<double> f, W27 w, cudaStream_t s) {
  k27_cheb_residual<<<grid27(L, L.max_cells), kThreads27, 0, s>>>(
      L, u, r, f, 1.0 / (w.w0 * sq27(L.n)), w.w1 / w.w0, w.w2 / w.w0, w.w3 / w.w0);
  return cudaGetLastError();
}

cudaError_t launch27_cheb2_update(const LevelView& L, double* u, const double* r, double a,
                                  double c2, W27 w, cudaStream_t s) {
  // W r = (w1 sf + w2 se + w3 sc)/w0 enters with the factor -c2
  k27_cheb2_update<<<grid27(L, L.max_cells), kThreads27, 0, s>>>(
      L, u, r, a, -c2 * w.w1 / w.w0, -c2 * w.w2 / w.w0, -c2 * w.w3 / w.w0);
  return cudaGetLastError();
}

cudaError_t launch27_apply(const LevelView& L, const double* u, double* out, W27 w,
                           cudaStream_t s) {
  FieldT<double> none{nullptr, L.boxes, 0};
  k27_apply<<<grid27(L, L.max_cells), kThreads27, 0, s>>>(L, u, out, none, 0, w, sq27(L.n));
  return cudaGetLastError();
}

cudaError_t launch27_residual(const LevelView& L, const double* u, FieldT<double> f, double* r,
                              W27 w, cudaStream_t s) {
  k27_apply<<<grid27(L, L.max_cells), kThreads27, 0, s>>>(L, u, r, f, 1, w, sq27(L.n));
  return cudaGetLastError();
}

cudaError_t launch27_resid_restrict(const LevelView& F, const double* u, FieldT<double> f,
                                    const LevelView& C, double* uhat_dst, double* rho_dst, W27 w,
                                    cudaStream_t s) {
  k27_resid_restrict<<<grid27(F, F.max_restrict), kThreads27, 0, s>>>(F, u, f, C, uhat_dst,
                                                                      rho_dst, w, sq27(F.n));
  return cudaGetLastError();
}

cudaError_t launch27_coarse_rhs(const LevelView& C, const LevelView& F, const double* u,
                                const double* rho, double* rhs, double* t, W27 w,
                                cudaStream_t s) {
  k27_coarse_rhs<<<grid27(C, C.max_stored), kThreads27, 0, s>>>(C, F, u, rho, rhs, t, w,
                                                                sq27(C.n));
  return cudaGetLastError();
}

cudaError_t launch27_transition_rhs(const LevelView& C, const double* t, const double* rho,
                                    double* u, double* rhs, W27 w, cudaStream_t s) {
  k27_transition_rhs<<<grid27(C, C.max_cells), kThreads27, 0, s>>>(C, t, rho, u, rhs, w,
                                                                   sq27(C.n));
  return cudaGetLastError();
}

cudaError_t launch27_resid_norm(const LevelView& L, const double* f, const double* u,
                                unsigned long long* norm, unsigned int* status, W27 w,
                                cudaStream_t s) {
  long long blocks = ((long long)L.nx * L.ny * L.nz + kThreads27 - 1) / kThreads27;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  if (blocks < 1) blocks = 1;
  k27_resid_norm<<<(unsigned)blocks, kThreads27, 0, s>>>(L, f, u, norm, status, w, sq27(L.n));
  return cudaGetLastError();
}

}  // namespace srfmg
