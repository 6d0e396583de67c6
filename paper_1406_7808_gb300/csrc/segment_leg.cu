// Segment-resident legs of the SR V-cycle for the float32 inner solver of the
// mixed-precision mode (Sec. 4, Fig. "FAS V-cycle segmental refinement"; the
// paper's point that a segment's levels can live in "near" memory, Sec. 6).
//
// On an SR level j below the stage's top level, the down-leg and the up-leg
// each make several sweeps over every segment's box.  Here one thread-block
// cluster holds one segment's box of level j in shared memory for a whole
// leg, split into z-slabs, one per CTA of the cluster; a stencil that reaches
// a plane of another CTA's slab reads it through distributed shared memory.
//   down leg  (after level j's coarse right-hand side was formed, by the
//     float64-arithmetic kernel at full occupancy): the degree-2
//     pre-smoother; the residual of the 8 children restricted with u onto
//     level j-1.
//   up leg    (after level j-1's correction e_{j-1} = w - t was formed):
//     u += P e_{j-1} on the prolongation range; the degree-2 post-smoother;
//     e_j = u - t for level j+1's correction.
// Global memory is touched once per array and leg: the box planes are
// brought in by bulk asynchronous copies (cp.async.bulk, completing on an
// mbarrier), results are written back once.  Every cell is computed with the
// operations, in the order, of the separate kernels in kernels.cu
// (k_cheb_residual_zm, k_cheb2_update_zm, k_resid_restrict, k_prolong_zcol,
// k_diff_zm), so the fused legs give the same bits.  The right-hand side is
// read from global memory; u and r live in shared memory.
//
// Measured on GB300 the legs are slower than the separate kernels (the
// mixed 512^3 solve: 30 to 32 against 24.2 ms), so the solver runs them only
// when asked (sr_debug_segment_legs): a segment box of 24^3 to 48^3 cells
// split over a cluster leaves slabs of 4 to 13 planes, most cells' stencils
// reach a neighbour's slab, every pass ends in a cluster barrier, and a CTA
// loads its slab before it computes; the streaming kernels keep 2048
// threads per SM busy with no barrier at 3 to 4 TB/s.
//
// Every wait on an mbarrier is bounded (about a second of %globaltimer); on
// expiry the kernel sets status bit 2 (SR_ERR_TIMEOUT) and carries on through
// the same cluster barriers as the other CTAs, so no CTA is left waiting.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "srfmg_device.cuh"
#include "srfmg_internal.cuh"

namespace cg = cooperative_groups;

namespace srfmg {
namespace {

constexpr int kLegThreads = 512;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound on an mbarrier wait

using namespace dev;

// ---- mbarrier and bulk copies (inline PTX)

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned done = 0;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bytes (a multiple of 16, both addresses 16-byte aligned) from global src
// to this CTA's shared dst, completing on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Wait for phase `phase` of bar, for at most kWaitNs; on expiry set status
// bit 2.  Every thread of the CTA calls it.
__device__ void bounded_wait(unsigned long long* bar, unsigned phase, unsigned* status) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase)) {
    if (global_ns() - t0 > kWaitNs) {
      if (threadIdx.x == 0) atomicOr(status, 2u);
      break;
    }
  }
}

// ---- a CTA's slab of the box: stored planes [p0, p1) of the box
// (stored-box z coordinates oz .. oz + e2 - 1), the whole stored (x, y) plane

struct Slab {
  int p0, p1;
  int ox, oy, oz;
  int e0, e1, e2;  // stored extents
  int sy, sz;      // shared-memory strides (e0, e0 e1)
  int rank, C;
};

__device__ __forceinline__ int slab_lo(int oz, int e2, int C, int r) { return oz + (r * e2) / C; }

__device__ __forceinline__ int owner_of(const Slab& s, int z) {
  int r = 0;
  while (r + 1 < s.C && slab_lo(s.oz, s.e2, s.C, r + 1) <= z) ++r;
  return r;
}

// pointer to plane z (stored-box coordinates) of array a (this CTA's copy at
// offset a in shared memory; other planes live at the same offset in the CTA
// that owns them)
__device__ __forceinline__ float* plane(const Slab& s, float* a, int z) {
  if (z >= s.p0 && z < s.p1) return a + (z - s.p0) * s.sz;
  const int r = owner_of(s, z);
  cg::cluster_group cl = cg::this_cluster();
  float* remote = cl.map_shared_rank(a, r);
  return remote + (z - slab_lo(s.oz, s.e2, s.C, r)) * s.sz;
}

__device__ __forceinline__ int sidx(const Slab& s, int x, int y) {
  return (y - s.oy) * s.sy + (x - s.ox);
}

__device__ __forceinline__ void slab_setup(Slab& s, const BoxDesc& B, int C) {
  s.ox = B.ox;
  s.oy = B.oy;
  s.oz = B.oz;
  s.e0 = B.hi[0] - B.lo[0] + 2;
  s.e1 = B.hi[1] - B.lo[1] + 2;
  s.e2 = B.hi[2] - B.lo[2] + 2;
  s.sy = s.e0;
  s.sz = s.e0 * s.e1;
  s.C = C;
  s.rank = (int)cg::this_cluster().block_rank();
  s.p0 = slab_lo(s.oz, s.e2, C, s.rank);
  s.p1 = slab_lo(s.oz, s.e2, C, s.rank + 1);
}

// Load this CTA's planes of `count` arrays (the box's stored planes, one
// contiguous range per array) into shared memory; bounded wait.
__device__ void load_slab(const Slab& s, const BoxDesc& B, const float* const* src, float* const* dst,
                          int count, unsigned long long* bar, unsigned* status, int force_timeout) {
  const unsigned bytes = (unsigned)((s.p1 - s.p0) * s.sz * (int)sizeof(float));
  if (threadIdx.x == 0) {
    // a forced timeout expects one byte more than arrives: the wait runs out
    mbar_expect_tx(bar, bytes * count + (force_timeout ? 16u : 0u));
    for (int a = 0; a < count; ++a)
      bulk_load(dst[a], src[a] + B.base + (long long)(s.p0 - s.oz) * B.sz, bytes, bar);
  }
  bounded_wait(bar, 0, status);
}

}  // namespace

// Shared memory of a leg kernel: two arrays of the CTA's slab (u and the
// smoother's residual r), plus the mbarrier.
size_t leg_smem_bytes(int e0, int e1, int planes) {
  return (size_t)2 * e0 * e1 * planes * sizeof(float) + 16;
}

namespace {

struct LegArrays {
  float* u;
  float* r;
  unsigned long long* bar;
};

__device__ __forceinline__ LegArrays leg_arrays(const Slab& s, int max_planes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = max_planes * s.sz;
  LegArrays a;
  a.u = reinterpret_cast<float*>(smem);
  a.r = a.u + n;
  a.bar = reinterpret_cast<unsigned long long*>(a.r + n);
  return a;
}

// the planes just outside this CTA's slab (in the neighbouring CTAs' shared
// memory), resolved once: p0 - 2, p0 - 1, p1, p1 + 1, or null where the
// stored box ends
struct Halo {
  const float* below2;
  const float* below;
  const float* above;
  const float* above2;
};

__device__ __forceinline__ Halo halo_of(const Slab& s, float* a) {
  Halo h;
  const int zlo = s.oz, zhi = s.oz + s.e2;
  h.below2 = (s.p0 - 2 >= zlo) ? plane(s, a, s.p0 - 2) : nullptr;
  h.below = (s.p0 - 1 >= zlo) ? plane(s, a, s.p0 - 1) : nullptr;
  h.above = (s.p1 < zhi) ? plane(s, a, s.p1) : nullptr;
  h.above2 = (s.p1 + 1 < zhi) ? plane(s, a, s.p1 + 1) : nullptr;
  return h;
}

// plane z of array a for z in [p0 - 2, p1 + 1]
__device__ __forceinline__ const float* near_plane(const Slab& s, const float* a, const Halo& h,
                                                   int z) {
  if (z < s.p0) return z == s.p0 - 1 ? h.below : h.below2;
  if (z >= s.p1) return z == s.p1 ? h.above : h.above2;
  return a + (z - s.p0) * s.sz;
}

// One smoother pass over the compute cells of this slab in z-columns:
// residual (res == 1):  r = rhs h^2/6 - u + (sum of the neighbours of u)/6
//                       (k_cheb_residual_zm);
// update    (res == 0): u += a r + b (sum of the neighbours of r)
//                       (k_cheb2_update_zm).
template <int kRes>
__device__ void column_pass(const Slab& s, const BoxDesc& B, const LevelView& L, float* src,
                            float* dst, const float* __restrict__ rhs, float c0, float c1) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1];
  const int zl = max(B.lo[2], s.p0), zh = min(B.hi[2], s.p1);
  if (zl >= zh) return;
  const Halo h = halo_of(s, src);
  for (int col = threadIdx.x; col < ex * ey; col += blockDim.x) {
    const int yy = col / ex;
    const int x = B.lo[0] + (col - yy * ex), y = B.lo[1] + yy;
    const int o = sidx(s, x, y);
    const bool xl = x > 0, xr = x < nx - 1, yl = y > 0, yr = y < ny - 1;
    float c = src[(zl - s.p0) * s.sz + o];
    float m1 = (zl > 0) ? near_plane(s, src, h, zl - 1)[o] : negx(c);
    long long g = at(B, x, y, zl);
    for (int z = zl; z < zh; ++z, g += B.sz) {
      const float* pc = src + (z - s.p0) * s.sz;
      const float m = negx(c);
      const float p1v = (z < nz - 1) ? near_plane(s, src, h, z + 1)[o] : m;
      float v[6];
      v[0] = xl ? pc[o - 1] : m;
      v[1] = xr ? pc[o + 1] : m;
      v[2] = yl ? pc[o - s.sy] : m;
      v[3] = yr ? pc[o + s.sy] : m;
      v[4] = m1;
      v[5] = p1v;
      float* out = dst + (z - s.p0) * s.sz + o;
      float acc;
      if (kRes) {
        acc = fmaf(rhs[g], c0, m);  // c0 = h^2/6, c1 = 1/6
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fmaf(c1, v[k], acc);
      } else {
        acc = fmaf(c0, c, *out);  // c0 = a, c1 = b; dst is u, src is r
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fmaf(c1, v[k], acc);
      }
      *out = acc;
      m1 = c;
      c = p1v;
    }
  }
}

// Down leg on level j (after the coarse right-hand side of level j was
// formed): the degree-2 pre-smoother, then the residual of the 8 children
// restricted with u onto Cv (level j-1; the global level 0 when j = 1).
__global__ void __launch_bounds__(kLegThreads, 2) k_leg_down(
    LevelView L, LevelView Cv, float* __restrict__ u, const float* __restrict__ rhs,
    float* __restrict__ uhat_dst, float* __restrict__ rho_dst, float cf, float sixth, float ca,
    float cb, float cS, float cO, float eighth, float one, float zero, int C, int max_planes,
    unsigned* status, int force_timeout) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  cg::cluster_group cl = cg::this_cluster();
  const int box = blockIdx.y;
  const BoxDesc B = L.boxes[box];
  const BoxDesc CB = (Cv.nbox == 1) ? Cv.boxes[0] : Cv.boxes[box];
  Slab s;
  slab_setup(s, B, C);
  LegArrays A = leg_arrays(s, max_planes);
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  if (threadIdx.x == 0) mbar_init(A.bar, 1);
  // r starts at zero everywhere: its shell inside the domain reads as zero
  for (int i = threadIdx.x; i < (s.p1 - s.p0) * s.sz; i += blockDim.x) A.r[i] = 0.f;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  {
    const float* src[1] = {u};
    float* dst[1] = {A.u};
    load_slab(s, B, src, dst, 1, A.bar, status, force_timeout);
  }
  cl.sync();  // every CTA's planes of u are in
  column_pass<1>(s, B, L, A.u, A.r, rhs, cf, sixth);
  cl.sync();
  column_pass<0>(s, B, L, A.r, A.u, nullptr, ca, cb);
  cl.sync();
  // u back to global memory (compute cells of the slab)
  {
    const int ex = B.hi[0] - B.lo[0], ey = B.hi[1] - B.lo[1];
    const int zl = max(B.lo[2], s.p0), zh = min(B.hi[2], s.p1);
    for (int col = threadIdx.x; zl < zh && col < ex * ey; col += blockDim.x) {
      const int yy = col / ex;
      const int x = B.lo[0] + (col - yy * ex), y = B.lo[1] + yy;
      const int o = sidx(s, x, y);
      long long g = at(B, x, y, zl);
      for (int z = zl; z < zh; ++z, g += B.sz) u[g] = A.u[(z - s.p0) * s.sz + o];
    }
  }
  // the residual of the 8 children summed through the outer faces of the
  // 2x2x2 block, restricted with u onto level j-1 (coarse cells whose lower
  // fine plane lies in this slab; k_resid_restrict)
  {
    const int lo0 = B.rlo[0], lo1 = B.rlo[1];
    const int cx = B.rhi[0] - B.rlo[0], cy = B.rhi[1] - B.rlo[1];
    const int Zl = max(B.rlo[2], (s.p0 + 1) >> 1), Zh = min(B.rhi[2], (s.p1 + 1) >> 1);
    const Halo hu = halo_of(s, A.u);
    for (int col = threadIdx.x; Zl < Zh && col < cx * cy; col += blockDim.x) {
      const int yy = col / cx;
      const int X = lo0 + (col - yy * cx), Y = lo1 + yy;
      const int x0 = 2 * X, y0 = 2 * Y;
      const int o0 = sidx(s, x0, y0);
      const bool xl = x0 > 0, xr = x0 + 2 < nx, yl = y0 > 0, yr = y0 + 2 < ny;
      for (int Z = Zl; Z < Zh; ++Z) {
        const int z0 = 2 * Z;
        const float* pz[4] = {z0 > 0 ? near_plane(s, A.u, hu, z0 - 1) : nullptr,
                              near_plane(s, A.u, hu, z0), near_plane(s, A.u, hu, z0 + 1),
                              z0 + 2 < nz ? near_plane(s, A.u, hu, z0 + 2) : nullptr};
        float v[2][2][2];
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
          for (int cyy = 0; cyy < 2; ++cyy)
#pragma unroll
            for (int cxx = 0; cxx < 2; ++cxx) v[cz][cyy][cxx] = pz[1 + cz][o0 + cyy * s.sy + cxx];
        const long long f0 = at(B, x0, y0, z0);
        const long long fy = B.sy, fz = B.sz;
        float fs = fmaf(rhs[f0], one, rhs[f0 + 1]);
        fs = fmaf(rhs[f0 + fy], one, fs);
        fs = fmaf(rhs[f0 + fy + 1], one, fs);
        fs = fmaf(rhs[f0 + fz], one, fs);
        fs = fmaf(rhs[f0 + fz + 1], one, fs);
        fs = fmaf(rhs[f0 + fz + fy], one, fs);
        fs = fmaf(rhs[f0 + fz + fy + 1], one, fs);
        float S = fmaf(v[0][0][0], one, v[0][0][1]);
        S = fmaf(v[0][1][0], one, S);
        S = fmaf(v[0][1][1], one, S);
        S = fmaf(v[1][0][0], one, S);
        S = fmaf(v[1][0][1], one, S);
        S = fmaf(v[1][1][0], one, S);
        S = fmaf(v[1][1][1], one, S);
        const bool zlo = z0 > 0, zr = z0 + 2 < nz;
        float O = zero;
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
          for (int cyy = 0; cyy < 2; ++cyy) {
            const float* row = pz[1 + cz] + o0 + cyy * s.sy;
            O = fmaf(xl ? row[-1] : negx(v[cz][cyy][0]), one, O);
            O = fmaf(xr ? row[2] : negx(v[cz][cyy][1]), one, O);
          }
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
          for (int cxx = 0; cxx < 2; ++cxx) {
            const float* colp = pz[1 + cz] + o0 + cxx;
            O = fmaf(yl ? colp[-s.sy] : negx(v[cz][0][cxx]), one, O);
            O = fmaf(yr ? colp[2 * s.sy] : negx(v[cz][1][cxx]), one, O);
          }
#pragma unroll
        for (int cyy = 0; cyy < 2; ++cyy)
#pragma unroll
          for (int cxx = 0; cxx < 2; ++cxx) {
            const int oo = o0 + cyy * s.sy + cxx;
            O = fmaf(zlo ? pz[0][oo] : negx(v[0][cyy][cxx]), one, O);
            O = fmaf(zr ? pz[3][oo] : negx(v[1][cyy][cxx]), one, O);
          }
        const long long cc = at(CB, X, Y, Z);
        rho_dst[cc] = fmaf(cS, S, fmaf(cO, O, fmaf(fs, eighth, zero)));
        uhat_dst[cc] = fmaf(S, eighth, zero);
      }
    }
  }
  cl.sync();  // no CTA leaves while another may still read its slab
}

// Up leg on level j: L = level j, Cv = level j-1 (holding e_{j-1} in ec, the
// global level 0 when j = 1).
__global__ void __launch_bounds__(kLegThreads, 2) k_leg_up(
    LevelView L, LevelView Cv, float* __restrict__ u, const float* __restrict__ t,
    const float* __restrict__ rhs, const float* __restrict__ ec, float* __restrict__ e_out,
    float cf, float sixth, float ca, float cb, float three, float w64, float mone, int C,
    int max_planes, unsigned* status, int force_timeout) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  cg::cluster_group cl = cg::this_cluster();
  const int box = blockIdx.y;
  const BoxDesc B = L.boxes[box];
  const BoxDesc CB = (Cv.nbox == 1) ? Cv.boxes[0] : Cv.boxes[box];
  Slab s;
  slab_setup(s, B, C);
  LegArrays A = leg_arrays(s, max_planes);
  if (threadIdx.x == 0) mbar_init(A.bar, 1);
  for (int i = threadIdx.x; i < (s.p1 - s.p0) * s.sz; i += blockDim.x) A.r[i] = 0.f;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  {
    const float* src[1] = {u};
    float* dst[1] = {A.u};
    load_slab(s, B, src, dst, 1, A.bar, status, force_timeout);
  }
  // u += P e_{j-1} on the prolongation range, in fine z-columns of the slab
  // (k_prolong_zcol: the bilinear (x, y) value of a coarse plane, then the
  // coarse plane of the fine cell and the one on its side)
  const int plo0 = B.plo[0], plo1 = B.plo[1];
  const int pex = B.phi[0] - B.plo[0], pey = B.phi[1] - B.plo[1];
  const int pzl = max(B.plo[2], s.p0), pzh = min(B.phi[2], s.p1);
  for (int col = threadIdx.x; pzl < pzh && col < pex * pey; col += blockDim.x) {
    const int yy = col / pex;
    const int x = plo0 + (col - yy * pex), y = plo1 + yy;
    const int X0 = x >> 1, Y0 = y >> 1;
    const int Xo = (x & 1) ? X0 + 1 : X0 - 1, Yo = (y & 1) ? Y0 + 1 : Y0 - 1;
    const bool fx = Xo < 0 || Xo >= Cv.nx, fy = Yo < 0 || Yo >= Cv.ny;
    const long long dx = fx ? 0 : Xo - X0, dy = fy ? 0 : (long long)(Yo - Y0) * CB.sy;
    auto cplane = [&](int Z) -> float {
      const bool fz = Z < 0 || Z >= Cv.nz;
      const int Zi = fz ? (Z < 0 ? 0 : Cv.nz - 1) : Z;
      const long long b0 = at(CB, X0, Y0, Zi);
      const float a = fmaf(three, ec[b0], neg_if(ec[b0 + dx], fx));
      const float b = fmaf(three, neg_if(ec[b0 + dy], fy), neg_if(ec[b0 + dy + dx], fx ^ fy));
      return neg_if(fmaf(three, a, b), fz);
    };
    const int o = sidx(s, x, y);
    for (int z = pzl; z < pzh; ++z) {
      const int Z = z >> 1;
      const float pc = cplane(Z);
      const float po = (z & 1) ? cplane(Z + 1) : cplane(Z - 1);
      float* pu = A.u + (z - s.p0) * s.sz + o;
      *pu = fmaf(w64, fmaf(three, pc, po), *pu);
    }
  }
  cl.sync();
  column_pass<1>(s, B, L, A.u, A.r, rhs, cf, sixth);
  cl.sync();
  column_pass<0>(s, B, L, A.r, A.u, nullptr, ca, cb);
  __syncthreads();  // this CTA's own planes only from here on
  // u on the prolongation range and e = u - t on the stored cells inside
  // the domain (the same cells) back to global memory (k_diff_zm)
  for (int col = threadIdx.x; pzl < pzh && col < pex * pey; col += blockDim.x) {
    const int yy = col / pex;
    const int x = plo0 + (col - yy * pex), y = plo1 + yy;
    const int o = sidx(s, x, y);
    long long g = at(B, x, y, pzl);
    for (int z = pzl; z < pzh; ++z, g += B.sz) {
      const float uv = A.u[(z - s.p0) * s.sz + o];
      u[g] = uv;
      e_out[g] = fmaf(t[g], mone, uv);
    }
  }
  cl.sync();
}

}  // namespace

namespace {
cudaLaunchConfig_t leg_config(int C, int nbox, size_t smem, cudaStream_t s,
                              cudaLaunchAttribute* attr) {
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, (unsigned)nbox, 1);
  cfg.blockDim = dim3(kLegThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cfg;
}
}  // namespace

cudaError_t launch_leg_down(const LevelView& L, const LevelView& Cv, float* u, const float* rhs,
                            float* uhat_dst, float* rho_dst, double a, double b, int C,
                            int max_planes, size_t smem, unsigned* status, int force_timeout,
                            cudaStream_t s) {
  const double n2 = (double)L.n * L.n;
  cudaLaunchAttribute attr[2];
  const cudaLaunchConfig_t cfg = leg_config(C, L.nbox, smem, s, attr);
  // residual and restriction constants of k_cheb_residual and
  // k_resid_restrict for level j's spacing
  return cudaLaunchKernelEx(&cfg, k_leg_down, L, Cv, u, rhs, uhat_dst, rho_dst,
                            (float)(1.0 / (6.0 * n2)), (float)(1.0 / 6.0), (float)a, (float)b,
                            (float)(-3.0 * n2 / 8.0), (float)(n2 / 8.0), 0.125f, 1.f, 0.f, C,
                            max_planes, status, force_timeout);
}

cudaError_t launch_leg_up(const LevelView& L, const LevelView& Cv, float* u, const float* t,
                          const float* rhs, const float* ec, float* e_out, double a, double b,
                          int C, int max_planes, size_t smem, unsigned* status,
                          int force_timeout, cudaStream_t s) {
  const double n2 = (double)L.n * L.n;
  cudaLaunchAttribute attr[2];
  const cudaLaunchConfig_t cfg = leg_config(C, L.nbox, smem, s, attr);
  return cudaLaunchKernelEx(&cfg, k_leg_up, L, Cv, u, t, rhs, ec, e_out,
                            (float)(1.0 / (6.0 * n2)), (float)(1.0 / 6.0), (float)a, (float)b, 3.f,
                            (float)(1.0 / 64.0), -1.f, C, max_planes, status, force_timeout);
}

int leg_max_clusters(int C, size_t smem) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3(kLegThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_leg_down, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int m = 0;
  if (cudaOccupancyMaxActiveClusters(&m, k_leg_up, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n < m ? n : m;
}

cudaError_t leg_prepare(size_t smem) {
  for (const void* k : {(const void*)k_leg_down, (const void*)k_leg_up}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace srfmg
