// The global FAS V-cycle (Sec. 3.1, Fig. "FAS multigrid V-cycle") on the
// global levels in one persistent launch (float64, 7-point operator, degree-2
// pre- and post-smoothers).
//
// The global levels are small (the transition level of the benchmark is
// 32^3, its coarsest grid 16^3), and a V-cycle over them is a chain of about
// ten dependent passes of a few microseconds each.  Here all blocks of one
// cooperative launch (co-resident by construction) run the passes in turn,
// each over every cell of its level, separated by a grid barrier:
//   down, per level g > 0:  pre-smoother (the first residual comes from the
//     caller or is formed), residual + restriction onto g-1, coarse
//     right-hand side (with the next first residual above the coarsest);
//   coarsest:  the exact solve (dense inverse or the three separable
//     sine-transform passes);
//   up, per level g > 0:  w - t on g-1, the correction prolongation, the
//     post-smoother (residual, update).
// Every cell takes the operations, in the order, of the separate kernels of
// kernels.cu (k_cheb_residual, k_cheb2_update, k_resid_restrict,
// k_coarse_rhs, k_coarse_solve / k_sep_*, k_diff_zm, k_prolong_zcol), so the
// persistent cycle gives the same bits.
//
// The grid barrier is a counter and a generation in global memory.  Its
// waits are bounded (about a second of %globaltimer; 5 ms when a test forces
// them to run out); on expiry the block sets status bit 2 (SR_ERR_TIMEOUT)
// and goes on, so the launch always ends.
#include <cuda_runtime.h>

#include "srfmg_device.cuh"
#include "srfmg_internal.cuh"

namespace srfmg {
namespace {

using namespace dev;

constexpr unsigned long long kBarrierNs = 1000000000ull;  // about a second
constexpr unsigned long long kForcedNs = 5000000ull;      // a forced timeout: 5 ms

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[0]: blocks arrived at the current barrier (zero at launch); bar[1]:
// generation, advanced by the last block to arrive.  gen: the generation
// this block waits to see change.
__device__ void grid_barrier(unsigned* bar, unsigned& gen, unsigned* status, int force_timeout) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
    if (arrived == gridDim.x + (force_timeout ? 1u : 0u)) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const volatile unsigned* g = bar + 1;
      const unsigned long long t0 = global_ns(), limit = force_timeout ? kForcedNs : kBarrierNs;
      while (*g == gen) {
        if (global_ns() - t0 > limit) {
          atomicOr(status, 2u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  ++gen;
  __syncthreads();
}

__device__ __forceinline__ int gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int gstride() { return gridDim.x * blockDim.x; }

// ---- passes over a whole global level (one box, no shell)

// r = D^-1 (f - A u) = f h^2/6 - u + (sum of neighbours)/6 (k_cheb_residual)
__device__ void p_residual(const LevelView& L, const BoxDesc& B, const double* __restrict__ u,
                           double* __restrict__ r, const double* __restrict__ f, double cf,
                           double sixth) {
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = gtid(); i < ncell; i += gstride()) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double uc = u[c];
    double v[6];
    neighbours<double>(u, c, B, L, q.x, q.y, q.z, uc, v);
    const double fv = f[c];
    r[c] = fma6(sixth, v, fma(fv, cf, negx(uc)));
  }
}

// u += a r + b (sum of the neighbours of r) (k_cheb2_update)
__device__ void p_update(const LevelView& L, const BoxDesc& B, double* __restrict__ u,
                         const double* __restrict__ r, double a, double b) {
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = gtid(); i < ncell; i += gstride()) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double rc = r[c];
    double v[6];
    neighbours<double>(r, c, B, L, q.x, q.y, q.z, rc, v);
    u[c] = fma6(b, v, fma(a, rc, u[c]));
  }
}

// residual of the 8 children restricted with u onto the coarse level
// (k_resid_restrict)
__device__ void p_resid_restrict(const LevelView& F, const BoxDesc& B, const double* __restrict__ u,
                                 const double* __restrict__ f, const BoxDesc& CB,
                                 double* __restrict__ uhat_dst, double* __restrict__ rho_dst,
                                 double cS, double cO, double eighth, Fk<double> k) {
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = B.rlo[d];
    hi[d] = B.rhi[d];
  }
  const int ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
  const int ncell = ex * ey * ez;
  for (int i = gtid(); i < ncell; i += gstride()) {
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
    double fs;
    {
      const long long f0 = c0, fy = sy, fz = sz;  // f has the level's layout
      fs = fma(f[f0], k.one, f[f0 + 1]);
      fs = fma(f[f0 + fy], k.one, fs);
      fs = fma(f[f0 + fy + 1], k.one, fs);
      fs = fma(f[f0 + fz], k.one, fs);
      fs = fma(f[f0 + fz + 1], k.one, fs);
      fs = fma(f[f0 + fz + fy], k.one, fs);
      fs = fma(f[f0 + fz + fy + 1], k.one, fs);
    }
    double S = fma(v[0][0][0], k.one, v[0][0][1]);
    S = fma(v[0][1][0], k.one, S);
    S = fma(v[0][1][1], k.one, S);
    S = fma(v[1][0][0], k.one, S);
    S = fma(v[1][0][1], k.one, S);
    S = fma(v[1][1][0], k.one, S);
    S = fma(v[1][1][1], k.one, S);
    const bool xl = x0 > 0, xr = x0 + 2 < F.nx, yl = y0 > 0, yr = y0 + 2 < F.ny, zl = z0 > 0,
               zr = z0 + 2 < F.nz;
    double O = k.zero;
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

// rhs = rho + A u (the whole coarse level lies under the fine level), t = u,
// and with r the next first residual D^-1 rho (k_coarse_rhs)
__device__ void p_coarse_rhs(const LevelView& C, const BoxDesc& B, const BoxDesc& FBx,
                             const double* __restrict__ u, const double* __restrict__ rho,
                             double* __restrict__ rhs, double* __restrict__ t,
                             double* __restrict__ r, double c6, double cn, double cr,
                             Fk<double> k) {
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = gtid(); i < ncell; i += gstride()) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    const double uc = u[c];
    t[c] = uc;
    const bool inF = q.x >= FBx.rlo[0] && q.x < FBx.rhi[0] && q.y >= FBx.rlo[1] &&
                     q.y < FBx.rhi[1] && q.z >= FBx.rlo[2] && q.z < FBx.rhi[2];
    double v[6];
    neighbours<double>(u, c, B, C, q.x, q.y, q.z, uc, v);
    const double rh = inF ? rho[c] : k.zero;
    rhs[c] = fma6(cn, v, fma(c6, uc, rh));
    if (r) r[c] = cr * rh;
  }
}

// e = u - t on the whole level (k_diff_zm)
__device__ void p_diff(const BoxDesc& B, const double* __restrict__ u, const double* __restrict__ t,
                       double* __restrict__ e, double mone) {
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1], ez = B.hi[2] - B.lo[2];
  const int ncell = ex * ey * ez;
  for (int i = gtid(); i < ncell; i += gstride()) {
    const Cell q = cell_of(i, B.lo, ex, ey);
    const long long c = at(B, q.x, q.y, q.z);
    e[c] = fma(t[c], mone, u[c]);
  }
}

// uf += P ec on the fine level (k_prolong_zcol with add)
__device__ void p_prolong_add(const LevelView& C, const BoxDesc& CB, const double* __restrict__ ec,
                              const BoxDesc& B, double* __restrict__ uf, double three,
                              double w64) {
  const int ex = B.phi[0] - B.plo[0], ey = B.phi[1] - B.plo[1], ez = B.phi[2] - B.plo[2];
  const int ncell = ex * ey * ez;
  for (int i = gtid(); i < ncell; i += gstride()) {
    const Cell q = cell_of(i, B.plo, ex, ey);
    const int X0 = q.x >> 1, Y0 = q.y >> 1;
    const int Xo = (q.x & 1) ? X0 + 1 : X0 - 1, Yo = (q.y & 1) ? Y0 + 1 : Y0 - 1;
    const bool fx = Xo < 0 || Xo >= C.nx, fy = Yo < 0 || Yo >= C.ny;
    const long long dx = fx ? 0 : Xo - X0, dy = fy ? 0 : (long long)(Yo - Y0) * CB.sy;
    auto plane = [&](int Z) -> double {
      const bool fz = Z < 0 || Z >= C.nz;
      const int Zi = fz ? (Z < 0 ? 0 : C.nz - 1) : Z;
      const long long b0 = at(CB, X0, Y0, Zi);
      const double a = fma(three, ec[b0], neg_if(ec[b0 + dx], fx));
      const double b = fma(three, neg_if(ec[b0 + dy], fy), neg_if(ec[b0 + dy + dx], fx ^ fy));
      return neg_if(fma(three, a, b), fz);
    };
    const int Z = q.z >> 1;
    const double pc = plane(Z);
    const double po = (q.z & 1) ? plane(Z + 1) : plane(Z - 1);
    const long long o = at(B, q.x, q.y, q.z);
    uf[o] = fma(w64, fma(three, pc, po), uf[o]);
  }
}

// exact coarsest solve, dense inverse: one warp per row (k_coarse_solve)
__device__ void p_coarse_dense(const LevelView& L, const BoxDesc& B, const double* __restrict__ minv,
                               const double* __restrict__ f, double* __restrict__ u,
                               Fk<double> k) {
  const int nx = L.nx, ny = L.ny, m = nx * ny * L.nz;
  const int lane = threadIdx.x & 31;
  const int nwarps = gstride() >> 5;
  for (int warp = gtid() >> 5; warp < m; warp += nwarps) {
    double s = k.zero;
    for (int j = lane; j < m; j += 32) {
      const int x = j % nx, y = (j / nx) % ny, z = j / (nx * ny);
      s = fma(minv[(long long)warp * m + j], f[at(B, x, y, z)], s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fma(__shfl_xor_sync(0xffffffffu, s, o), k.one, s);
    if (lane == 0) {
      const int x = warp % nx, y = (warp / nx) % ny, z = warp / (nx * ny);
      u[at(B, x, y, z)] = s;
    }
  }
}

// exact coarsest solve, separable transforms: the three passes of
// k_sep_fwd_xy, k_sep_z and k_sep_inv_xy (W lanes per task), barrier-separated
struct SepArgs {
  const double* sep;
  double *g, *q;
  int W;
};

__device__ void p_sep_fwd_xy(const LevelView& L, const BoxDesc& B, const double* __restrict__ f,
                             const SepArgs& S, Fk<double> k) {
  const int nx = L.nx, ny = L.ny, nz = L.nz, W = S.W;
  const double* Px = S.sep;
  const double* Py = S.sep + nx * nx;
  const int tasks = nz * ny;
  // every thread of the grid takes part in each round's shuffles
  const int per_round = gstride() / W;
  for (int base = 0; base < tasks; base += per_round) {
    const int lane = gtid() & (W - 1), task = base + gtid() / W;
    const bool live = task < tasks;
    const int z = live ? task / ny : 0, ky = live ? task - (task / ny) * ny : 0;
    double t = k.zero;
    if (live && lane < nx)
      for (int y = 0; y < ny; ++y) t = fma(Py[ky * ny + y], f[at(B, lane, y, z)], t);
    double o = k.zero;
    for (int x = 0; x < nx; ++x) {
      const double tx = __shfl_sync(0xffffffffu, t, x, W);
      if (lane < nx) o = fma(Px[lane * nx + x], tx, o);
    }
    if (live && lane < nx) S.g[((long long)z * ny + ky) * nx + lane] = o;
  }
}

__device__ void p_sep_z(const LevelView& L, const SepArgs& S, Fk<double> k) {
  const int nx = L.nx, ny = L.ny, nz = L.nz, W = S.W;
  const double* Pz = S.sep + nx * nx + ny * ny;
  const double* il = Pz + nz * nz;
  const long long pl = (long long)ny * nx;
  const int tasks = ny * nx;
  const int per_round = gstride() / W;
  for (int base = 0; base < tasks; base += per_round) {
    const int lane = gtid() & (W - 1), task = base + gtid() / W;
    const bool live = task < tasks;
    const int ky = live ? task / nx : 0, kx = live ? task - (task / nx) * nx : 0;
    const bool on = live && lane < nz;
    const double v = on ? S.g[lane * pl + (long long)ky * nx + kx] : k.zero;
    double h = k.zero;
    for (int z = 0; z < nz; ++z) {
      const double vz = __shfl_sync(0xffffffffu, v, z, W);
      if (lane < nz) h = fma(Pz[lane * nz + z], vz, h);
    }
    if (on) h = fma(h, il[lane * pl + (long long)ky * nx + kx], k.zero);
    double o = k.zero;
    for (int kz = 0; kz < nz; ++kz) {
      const double hz = __shfl_sync(0xffffffffu, h, kz, W);
      if (lane < nz) o = fma(Pz[kz * nz + lane], hz, o);
    }
    if (on) S.q[lane * pl + (long long)ky * nx + kx] = o;
  }
}

__device__ void p_sep_inv_xy(const LevelView& L, const BoxDesc& B, const SepArgs& S,
                             double* __restrict__ u, Fk<double> k) {
  const int nx = L.nx, ny = L.ny, nz = L.nz, W = S.W;
  const double* Px = S.sep;
  const double* Py = S.sep + nx * nx;
  const int tasks = nz * ny;
  const int per_round = gstride() / W;
  for (int base = 0; base < tasks; base += per_round) {
    const int lane = gtid() & (W - 1), task = base + gtid() / W;
    const bool live = task < tasks;
    const int z = live ? task / ny : 0, y = live ? task - (task / ny) * ny : 0;
    double t = k.zero;
    if (live && lane < nx)
      for (int ky = 0; ky < ny; ++ky)
        t = fma(Py[ky * ny + y], S.q[((long long)z * ny + ky) * nx + lane], t);
    double o = k.zero;
    for (int kx = 0; kx < nx; ++kx) {
      const double tk = __shfl_sync(0xffffffffu, t, kx, W);
      if (lane < nx) o = fma(Px[kx * nx + lane], tk, o);
    }
    if (live && lane < nx) u[at(B, lane, y, z)] = o;
  }
}

__global__ void __launch_bounds__(kVcycleThreads) k_vcycle(VcycleArgs a) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  unsigned gen = *(volatile unsigned*)(a.bar + 1);
  const Fk<double> k{a.one, a.zero};
  auto barrier = [&]() { grid_barrier(a.bar, gen, a.status, a.force_timeout); };
  // down-leg
  for (int g = a.top; g >= 1; --g) {
    const VcycleLevel& L = a.lev[g];
    const VcycleLevel& C = a.lev[g - 1];
    const BoxDesc B = L.view.boxes[0];
    const double* rf = (g == a.top) ? a.r_first : L.r;
    if (!rf) {
      p_residual(L.view, B, L.u, L.r, L.f, L.cf, a.sixth);
      barrier();
      rf = L.r;
    }
    p_update(L.view, B, L.u, rf, a.pre_a, a.pre_b);
    barrier();
    const BoxDesc CB = C.view.boxes[0];
    p_resid_restrict(L.view, B, L.u, L.f, CB, C.u, C.rho, L.cS, L.cO, a.eighth, k);
    barrier();
    // the coarse level's first residual comes with its right-hand side,
    // except on the coarsest level (solved exactly)
    p_coarse_rhs(C.view, CB, B, C.u, C.rho, C.rhs, C.t, g - 1 >= 1 ? C.r : nullptr, C.c6, C.cn,
                 C.cr, k);
    barrier();
  }
  // coarsest level: u_0 = A^-1 rhs_0 (the top's f when the cycle starts there)
  {
    const VcycleLevel& L = a.lev[0];
    const BoxDesc B = L.view.boxes[0];
    if (a.minv) {
      p_coarse_dense(L.view, B, a.minv, L.f, L.u, k);
    } else {
      const SepArgs S{a.sep, a.sep_g, a.sep_q, a.sep_w};
      p_sep_fwd_xy(L.view, B, L.f, S, k);
      barrier();
      p_sep_z(L.view, S, k);
      barrier();
      p_sep_inv_xy(L.view, B, S, L.u, k);
    }
    barrier();
  }
  // up-leg
  for (int g = 1; g <= a.top; ++g) {
    const VcycleLevel& L = a.lev[g];
    const VcycleLevel& C = a.lev[g - 1];
    const BoxDesc B = L.view.boxes[0];
    const BoxDesc CB = C.view.boxes[0];
    p_diff(CB, C.u, C.t, C.rho, a.mone);
    barrier();
    p_prolong_add(C.view, CB, C.rho, B, L.u, a.three, a.w64);
    barrier();
    p_residual(L.view, B, L.u, L.r, L.f, L.cf, a.sixth);
    barrier();
    p_update(L.view, B, L.u, L.r, a.post_a, a.post_b);
    if (g < a.top) barrier();
  }
}

}  // namespace

cudaError_t launch_vcycle(const VcycleArgs& a, int blocks, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks, 1, 1);
  cfg.blockDim = dim3(kVcycleThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_vcycle, a);
}

int vcycle_max_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_vcycle, kVcycleThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace srfmg
