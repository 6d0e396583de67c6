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
// residual array).  The smoother passes, the residual and the coarse
// right-hand side walk columns in z (below); the transition-level
// right-hand side and the residual norm read every neighbour through the L1
// cache.
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
    const Cell27 q = cell27(i, B.lo, ex, ey);
    const double au = op27(u, B, L, w, n2, q.x, q.y, q.z);
    out[at27(B, q.x, q.y, q.z)] = residual ? f.p[at27(FB, q.x, q.y, q.z)] - au : au;
  }
}

// u = t, rhs = rho + A t on the whole (global) transition level; with r, the
// smoother's first residual D^-1 rho (cr = D^-1)
__global__ void __launch_bounds__(kThreads27) k27_transition_rhs(LevelView C,
                                                                 const double* __restrict__ t,
                                                                 const double* __restrict__ rho,
                                                                 double* __restrict__ u,
                                                                 double* __restrict__ rhs,
                                                                 double* __restrict__ r, W27 w,
                                                                 double n2, double cr) {
  grid_dep_wait();
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
    if (r) r[c] = cr * rho[c];
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
  grid_dep_wait();
  __shared__ BoxDesc B;
  if (threadIdx.x == 0) B = L.boxes[0];
  __syncthreads();
  const long long ncell = (long long)L.nx * L.ny * L.nz;
  unsigned long long m = 0;
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    split3(i, L.nx, L.ny, x, y, z);
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

// ---------------------------------------------------------------------------
// Column (z-marching) forms of the operator's two hot passes.  With, for
// every (x, y) column and plane z, the in-plane quantities
//   c(z) = a(x, y, z),  e(z) = sum of the 4 in-plane face neighbours,
//   k(z) = sum of the 4 in-plane corner neighbours,
// the neighbour classes of cell (x, y, z) are
//   faces   = e(z) + c(z-1) + c(z+1),
//   edges   = k(z) + e(z-1) + e(z+1),
//   corners = k(z-1) + k(z+1),
// so a thread walking a column forms one new plane per cell (6 additions)
// plus 5 additions, instead of 26.  A plane outside the domain is the
// mirror plane negated; in-plane neighbours outside the domain are mirrored
// with one sign flip per outside dimension.  Threads of a block take
// consecutive cells of the box's flattened (x, y) compute plane; blockIdx.x
// enumerates (plane block, z chunk).  As in the 7-point kernels, every
// float64 operation is a fused multiply-add with kernel-parameter constants
// (additions as fma(a, one, b)) and sign flips are integer XORs: on sm_103a
// that form issues faster than DADD, DMUL or a float64 negation.
constexpr int kZ27Threads = 256, kZ27Chunk = 16;

struct Plane27 {
  double c, e, k;
};

struct Col27 {
  long long xm, xp, ym, yp;  // offsets of the in-plane neighbours (mirrored)
  bool fxm, fxp, fym, fyp;   // sign flips
};

__device__ __forceinline__ Col27 column27(const BoxDesc& B, const LevelView& L, int x, int y) {
  Col27 q;
  q.fxm = x == 0;
  q.fxp = x == L.nx - 1;
  q.fym = y == 0;
  q.fyp = y == L.ny - 1;
  q.xm = q.fxm ? 0 : -1;
  q.xp = q.fxp ? 0 : 1;
  q.ym = q.fym ? 0 : -(long long)B.sy;
  q.yp = q.fyp ? 0 : (long long)B.sy;
  return q;
}

// v or -v, the sign bit flipped on the integer pipe (inline PTX, so that the
// compiler cannot turn it into a float64 negation)
__device__ __forceinline__ double sgn27(double v, bool flip) {
  int hi = __double2hiint(v);
  const unsigned m = (unsigned)flip << 31;
  asm("xor.b32 %0, %0, %1;" : "+r"(hi) : "r"(m));
  return __hiloint2double(hi, __double2loint(v));
}

// in-plane quantities of the plane through offset p (the column's cell)
__device__ __forceinline__ Plane27 plane27(const double* __restrict__ a, long long p,
                                           const Col27& q, double one) {
  Plane27 r;
  r.c = a[p];
  r.e = fma(sgn27(a[p + q.xm], q.fxm), one, sgn27(a[p + q.xp], q.fxp));
  r.e = fma(sgn27(a[p + q.ym], q.fym), one, r.e);
  r.e = fma(sgn27(a[p + q.yp], q.fyp), one, r.e);
  r.k = fma(sgn27(a[p + q.xm + q.ym], q.fxm ^ q.fym), one,
            sgn27(a[p + q.xp + q.ym], q.fxp ^ q.fym));
  r.k = fma(sgn27(a[p + q.xm + q.yp], q.fxm ^ q.fyp), one, r.k);
  r.k = fma(sgn27(a[p + q.xp + q.yp], q.fxp ^ q.fyp), one, r.k);
  return r;
}

__device__ __forceinline__ Plane27 neg27(Plane27 p) {
  return Plane27{sgn27(p.c, true), sgn27(p.e, true), sgn27(p.k, true)};
}

__device__ __forceinline__ bool ztile27(const BoxDesc& B, int nplane, int& x, int& y, int& z0,
                                        int& z1) {
  const int tz = blockIdx.x / nplane, pb = blockIdx.x - tz * nplane;
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1];
  const int i = pb * kZ27Threads + threadIdx.x;
  const int iy = i / ex;
  x = B.lo[0] + (i - iy * ex);
  y = B.lo[1] + iy;
  z0 = B.lo[2] + tz * kZ27Chunk;
  z1 = min(z0 + kZ27Chunk, B.hi[2]);
  return iy < ey && z0 < z1;
}

// With nb = cf F + ce E + cc C over the neighbour classes of a_in:
// mode 0: out = f c0 - a_in + nb        (r = D^-1 (f - A u), a_in = u);
// mode 1: out += c0 a_in + nb           (u += a r - c2 W r, a_in = r, out = u);
// mode 2: out = f + c0 a_in + nb        (r = f - A u with c0 = -w0 n^2).
template <int kMode>
__global__ void __launch_bounds__(kZ27Threads) k27_column(LevelView L,
                                                          const double* __restrict__ a_in,
                                                          double* __restrict__ out,
                                                          FieldT<double> f, double c0,
                                                          double cf, double ce, double cc,
                                                          double one, int nplane) {
  grid_dep_wait();
  __shared__ BoxDesc B, FB;
  if (threadIdx.x == 0) {
    B = L.boxes[blockIdx.y];
    FB = (kMode != 1) ? (f.single ? f.boxes[0] : f.boxes[blockIdx.y]) : B;
  }
  __syncthreads();
  int x, y, z0, z1;
  if (!ztile27(B, nplane, x, y, z0, z1)) return;
  const Col27 q = column27(B, L, x, y);
  const long long sz = B.sz;
  long long p = at27(B, x, y, z0);
  long long fp = at27(FB, x, y, z0);
  const long long fsz = FB.sz;
  Plane27 pc = plane27(a_in, p, q, one);
  Plane27 pm = (z0 > 0) ? plane27(a_in, p - sz, q, one) : neg27(pc);
  for (int z = z0; z < z1; ++z) {
    const Plane27 pp = (z < L.nz - 1) ? plane27(a_in, p + sz, q, one) : neg27(pc);
    const double F = fma(pp.c, one, fma(pm.c, one, pc.e));
    const double E = fma(pp.e, one, fma(pm.e, one, pc.k));
    const double C = fma(pm.k, one, pp.k);
    double base;
    if (kMode == 0) {
      base = fma(f.p[fp], c0, sgn27(pc.c, true));
    } else if (kMode == 1) {
      base = fma(c0, pc.c, out[p]);
    } else {
      base = fma(c0, pc.c, f.p[fp]);
    }
    out[p] = fma(cc, C, fma(ce, E, fma(cf, F, base)));
    pm = pc;
    pc = pp;
    p += sz;
    fp += fsz;
  }
}

// The coarse-level right-hand side in column form (15 operations per cell
// instead of 31): rhs = rho + A u inside the restriction region of the
// matching fine box, A u on the rest of the compute region, with A u =
// c0 u + cf F + ce E + cc C over the neighbour classes (c0 = w0 n^2,
// cf = -w1 n^2, ...); t = u and, with r, the smoother's first residual
// D^-1 (rhs - A u), which is D^-1 rho and 0 (cr = D^-1).  t on the box's
// shell is copied by the shell-copy pass that follows on SR levels.
__global__ void __launch_bounds__(kZ27Threads) k27_coarse_rhs_col(
    LevelView C, LevelView F, const double* __restrict__ u, const double* __restrict__ rho,
    double* __restrict__ rhs, double* __restrict__ t, double* __restrict__ r, double c0, double cf,
    double ce, double cc, double cr, double one, double zero, int nplane) {
  grid_dep_wait();
  __shared__ BoxDesc B, FBx;
  if (threadIdx.x == 0) {
    B = C.boxes[blockIdx.y];
    FBx = (F.nbox == 1) ? F.boxes[0] : F.boxes[blockIdx.y];
  }
  __syncthreads();
  int x, y, z0, z1;
  if (!ztile27(B, nplane, x, y, z0, z1)) return;
  const Col27 q = column27(B, C, x, y);
  const long long sz = B.sz;
  long long p = at27(B, x, y, z0);
  const bool in_xy = x >= FBx.rlo[0] && x < FBx.rhi[0] && y >= FBx.rlo[1] && y < FBx.rhi[1];
  Plane27 pc = plane27(u, p, q, one);
  Plane27 pm = (z0 > 0) ? plane27(u, p - sz, q, one) : neg27(pc);
  for (int z = z0; z < z1; ++z) {
    const Plane27 pp = (z < C.nz - 1) ? plane27(u, p + sz, q, one) : neg27(pc);
    const double Fs = fma(pp.c, one, fma(pm.c, one, pc.e));
    const double Es = fma(pp.e, one, fma(pm.e, one, pc.k));
    const double Cs = fma(pm.k, one, pp.k);
    const bool inF = in_xy && z >= FBx.rlo[2] && z < FBx.rhi[2];
    const double rh = inF ? rho[p] : zero;
    t[p] = pc.c;
    rhs[p] = fma(cc, Cs, fma(ce, Es, fma(cf, Fs, fma(c0, pc.c, rh))));
    if (r) r[p] = inF ? cr * rh : zero;
    pm = pc;
    pc = pp;
    p += sz;
  }
}

// uhat = average of the 8 children of u, rho = average of the 8 children of r
// (r = f - A u already formed on the fine compute region)
__global__ void __launch_bounds__(kThreads27) k27_restrict_pair(LevelView F,
                                                                const double* __restrict__ u,
                                                                const double* __restrict__ r,
                                                                LevelView C,
                                                                double* __restrict__ uhat_dst,
                                                                double* __restrict__ rho_dst,
                                                                double one, double eighth,
                                                                double zero) {
  grid_dep_wait();
  __shared__ BoxDesc B, CB;
  if (threadIdx.x == 0) {
    B = F.boxes[blockIdx.y];
    CB = (C.nbox == 1) ? C.boxes[0] : C.boxes[blockIdx.y];
  }
  __syncthreads();
  const int lo[3] = {B.rlo[0], B.rlo[1], B.rlo[2]};
  const int ex = B.rhi[0] - lo[0], ey = B.rhi[1] - lo[1], ez = B.rhi[2] - lo[2];
  const int ncell = ex * ey * ez;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
    const Cell27 q = cell27(i, lo, ex, ey);
    const long long c0 = at27(B, 2 * q.x, 2 * q.y, 2 * q.z);
    const long long sy = B.sy, sz = B.sz;
    // the 8 children summed as fused multiply-adds with a register 1 (the
    // form the float64 pipe issues fastest; each rounds as the addition)
    double su = fma(u[c0], one, u[c0 + 1]), sr = fma(r[c0], one, r[c0 + 1]);
#pragma unroll
    for (int k = 2; k < 8; ++k) {
      const long long c = c0 + (k >> 2) * sz + ((k >> 1) & 1) * sy + (k & 1);
      su = fma(u[c], one, su);
      sr = fma(r[c], one, sr);
    }
    const long long cc = at27(CB, q.x, q.y, q.z);
    uhat_dst[cc] = fma(su, eighth, zero);
    rho_dst[cc] = fma(sr, eighth, zero);
  }
}

int nplane27(const LevelView& L) {
  return (L.max_ex * L.max_ey + kZ27Threads - 1) / kZ27Threads;
}

dim3 zgrid27(const LevelView& L) {
  const int nzc = (L.max_ez + kZ27Chunk - 1) / kZ27Chunk;
  return dim3((unsigned)(nplane27(L) * nzc), (unsigned)L.nbox, 1);
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
  SRFMG_LAUNCH(pdl_launch(k27_column<0>, zgrid27(L), kZ27Threads, 0, s, L, u, r, f,
                          1.0 / (w.w0 * sq27(L.n)), w.w1 / w.w0, w.w2 / w.w0, w.w3 / w.w0, 1.0,
                          nplane27(L)));
  return cudaGetLastError();
}

cudaError_t launch27_cheb2_update(const LevelView& L, double* u, const double* r, double a,
                                  double c2, W27 w, cudaStream_t s) {
  // W r = (w1 sf + w2 se + w3 sc)/w0 enters with the factor -c2
  FieldT<double> none{nullptr, L.boxes, 0};
  SRFMG_LAUNCH(pdl_launch(k27_column<1>, zgrid27(L), kZ27Threads, 0, s, L, r, u, none, a,
                          -c2 * w.w1 / w.w0, -c2 * w.w2 / w.w0, -c2 * w.w3 / w.w0, 1.0,
                          nplane27(L)));
  return cudaGetLastError();
}

cudaError_t launch27_residual_zm(const LevelView& L, const double* u, FieldT<double> f,
                                 double* r, W27 w, cudaStream_t s) {
  const double n2 = sq27(L.n);
  SRFMG_LAUNCH(pdl_launch(k27_column<2>, zgrid27(L), kZ27Threads, 0, s, L, u, r, f, -n2 * w.w0,
                          n2 * w.w1, n2 * w.w2, n2 * w.w3, 1.0, nplane27(L)));
  return cudaGetLastError();
}

cudaError_t launch27_restrict_pair(const LevelView& F, const double* u, const double* r,
                                   const LevelView& C, double* uhat_dst, double* rho_dst,
                                   cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k27_restrict_pair, grid27(F, F.max_restrict), kThreads27, 0, s, F, u, r,
                          C, uhat_dst, rho_dst, 1.0, 0.125, 0.0));
  return cudaGetLastError();
}

cudaError_t launch27_apply(const LevelView& L, const double* u, double* out, W27 w,
                           cudaStream_t s) {
  FieldT<double> none{nullptr, L.boxes, 0};
  SRFMG_LAUNCH(pdl_launch(k27_apply, grid27(L, L.max_cells), kThreads27, 0, s, L, u, out, none, 0,
                          w, sq27(L.n)));
  return cudaGetLastError();
}

cudaError_t launch27_residual(const LevelView& L, const double* u, FieldT<double> f, double* r,
                              W27 w, cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k27_apply, grid27(L, L.max_cells), kThreads27, 0, s, L, u, r, f, 1, w,
                          sq27(L.n)));
  return cudaGetLastError();
}

cudaError_t launch27_coarse_rhs(const LevelView& C, const LevelView& F, const double* u,
                                const double* rho, double* rhs, double* t, double* r, W27 w,
                                cudaStream_t s) {
  const double n2 = sq27(C.n);
  SRFMG_LAUNCH(pdl_launch(k27_coarse_rhs_col, zgrid27(C), kZ27Threads, 0, s, C, F, u, rho, rhs, t,
                          r, w.w0 * n2, -w.w1 * n2, -w.w2 * n2, -w.w3 * n2,
                          1.0 / (w.w0 * n2), 1.0, 0.0, nplane27(C)));
  return cudaGetLastError();
}

cudaError_t launch27_transition_rhs(const LevelView& C, const double* t, const double* rho,
                                    double* u, double* rhs, double* r, W27 w, cudaStream_t s) {
  SRFMG_LAUNCH(pdl_launch(k27_transition_rhs, grid27(C, C.max_cells), kThreads27, 0, s, C, t, rho,
                          u, rhs, r, w, sq27(C.n), 1.0 / (w.w0 * sq27(C.n))));
  return cudaGetLastError();
}

cudaError_t launch27_resid_norm(const LevelView& L, const double* f, const double* u,
                                unsigned long long* norm, unsigned int* status, W27 w,
                                cudaStream_t s) {
  long long blocks = ((long long)L.nx * L.ny * L.nz + kThreads27 - 1) / kThreads27;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  if (blocks < 1) blocks = 1;
  SRFMG_LAUNCH(pdl_launch(k27_resid_norm, (unsigned)blocks, kThreads27, 0, s, L, f, u, norm,
                          status, w, sq27(L.n)));
  return cudaGetLastError();
}

}  // namespace srfmg
