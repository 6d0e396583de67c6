// Device helpers shared by the solver's kernel files (kernels.cu,
// segment_leg.cu, persistent.cu): box addressing, sign flips and float
// conversions on the integer pipe, and the fused neighbour sums, so that
// every kernel computing the same cell takes the same operations in the
// same order.
#pragma once

#include "srfmg_internal.cuh"

namespace srfmg {
namespace dev {

// Constants handed to the kernels as parameters so that the compiler cannot
// fold them into immediates: on sm_103a a float64 FMA whose constant operands
// are registers issues faster than DADD, DMUL or an FMA with an immediate.
// Values: one = 1, zero = 0.
template <typename T>
struct Fk {
  T one, zero;
};

template <typename T>
__host__ __device__ inline Fk<T> fk() {
  return Fk<T>{T(1), T(0)};
}

__device__ __forceinline__ long long at(const BoxDesc& b, int x, int y, int z) {
  return b.base + (long long)(z - b.oz) * b.sz + (long long)(y - b.oy) * b.sy + (x - b.ox);
}

// -v, by flipping the sign bit on the integer pipe.  The xor is inline PTX so
// that the compiler cannot turn it back into a floating-point negation (which
// would cost a float64 instruction).
__device__ __forceinline__ double negx(double v) {
  int hi = __double2hiint(v);
  asm("xor.b32 %0, %0, 0x80000000;" : "+r"(hi));
  return __hiloint2double(hi, __double2loint(v));
}
__device__ __forceinline__ float negx(float v) {
  unsigned b = __float_as_uint(v);
  asm("xor.b32 %0, %0, 0x80000000;" : "+r"(b));
  return __uint_as_float(b);
}

// v or -v, selected on the integer pipe
__device__ __forceinline__ double neg_if(double v, bool flip) {
  int hi = __double2hiint(v);
  const unsigned m = (unsigned)flip << 31;
  asm("xor.b32 %0, %0, %1;" : "+r"(hi) : "r"(m));
  return __hiloint2double(hi, __double2loint(v));
}
__device__ __forceinline__ float neg_if(float v, bool flip) {
  unsigned b = __float_as_uint(v);
  const unsigned m = (unsigned)flip << 31;
  asm("xor.b32 %0, %0, %1;" : "+r"(b) : "r"(m));
  return __uint_as_float(b);
}

// float -> double on the integer pipe (the conversion instruction would use
// the float64 pipe): exact for normal floats and zero; float32 subnormals
// (below 1.2e-38) become zero; the solver's values are finite.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned sign = b & 0x80000000u;
  const unsigned hi = e ? (sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)) : sign;
  const unsigned lo = e ? (b << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double x) { return x; }

// double -> float rounded to nearest (ties to even), on the integer pipe
// (the conversion instruction would take a float64-pipe slot, and the
// float64-arithmetic kernels of the mixed mode are bound by that pipe).
// Built from the IEEE 754 binary64 / binary32 formats: keep the leading 24
// significant bits, round on the bits dropped, renormalise on a carry;
// results below the smallest normal float become subnormal floats (rounded
// the same way), results beyond the largest float become infinity, NaN
// stays a (quiet) NaN.
__device__ __forceinline__ float narrow(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long frac = b & 0xfffffffffffffull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (frac ? 0x400000u : 0u));
  if (e < 1023 - 150) return __uint_as_float(sign);  // below half the smallest subnormal
  // significand with its leading one, and the number of low bits to drop:
  // 29 for a normal float result, more for a subnormal one (exponent < -126)
  const unsigned long long sig = frac | (1ull << 52);
  const int fe = e - 1023 + 127;  // biased float exponent of a normal result
  const int drop = fe >= 1 ? 29 : 29 + (1 - fe);
  unsigned long long keep = sig >> drop;
  const unsigned long long rest = sig & ((1ull << drop) - 1), half = 1ull << (drop - 1);
  if (rest > half || (rest == half && (keep & 1ull))) ++keep;
  if (fe >= 1) {
    // keep holds 1.m (24 bits) or, after a carry, 2^24
    int ex = fe;
    if (keep >> 24) {
      keep >>= 1;
      ++ex;
    }
    if (ex >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)ex << 23) | ((unsigned)keep & 0x7fffffu));
  }
  // subnormal result (a carry into bit 23 gives the smallest normal, which
  // the same bit pattern encodes)
  return __uint_as_float(sign | (unsigned)keep);
}

// a float64 result stored in T: unchanged for double, narrow() for float
__device__ __forceinline__ double store_as(double v, double*) { return v; }
__device__ __forceinline__ float store_as(double v, float*) { return narrow(v); }
template <typename T>
__device__ __forceinline__ T stored(double v) {
  return store_as(v, (T*)nullptr);
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

// The six neighbours of stored cell c at (x, y, z), converted to A; a
// neighbour outside the level grid [0, nx) x [0, ny) x [0, nz) is minus the
// centre value (mirror through u = 0 on the face).
template <typename A, typename T>
__device__ __forceinline__ A acc_of(T x) {
  return (A)x;
}
template <>
__device__ __forceinline__ double acc_of<double, float>(float x) {
  return widen(x);
}

template <typename A, typename T>
__device__ __forceinline__ void neighbours(const T* __restrict__ a, long long c, const BoxDesc& b,
                                           const LevelView& L, int x, int y, int z, T centre,
                                           A v[6]) {
  const T m = negx(centre);
  v[0] = acc_of<A>((x > 0) ? a[c - 1] : m);
  v[1] = acc_of<A>((x < L.nx - 1) ? a[c + 1] : m);
  v[2] = acc_of<A>((y > 0) ? a[c - b.sy] : m);
  v[3] = acc_of<A>((y < L.ny - 1) ? a[c + b.sy] : m);
  v[4] = acc_of<A>((z > 0) ? a[c - b.sz] : m);
  v[5] = acc_of<A>((z < L.nz - 1) ? a[c + b.sz] : m);
}

// acc + w * (v0 + ... + v5) as six fused multiply-adds
template <typename A>
__device__ __forceinline__ A fma6(A w, const A v[6], A acc) {
#pragma unroll
  for (int i = 0; i < 6; ++i) acc = fma(w, v[i], acc);
  return acc;
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

}  // namespace dev
}  // namespace srfmg
