// sr_op_smooth_noalloc: the Chebyshev smoother on a whole grid with its
// scratch in a fixed device array instead of memory allocated per call.
//
// Who needs it: callers that cannot allocate device memory at the point they
// smooth -- for example code whose device memory is entirely handed out by
// another allocator, or loops that must not pay cudaMalloc's implicit device
// synchronisation.  They pass their own input and output arrays; everything
// else the smoother needs lives in g_scratch below, which every GPU that
// loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "srfmg.h"
#include "srfmg_internal.cuh"

using namespace srfmg;

namespace {

constexpr int kMaxN = SR_NOALLOC_MAX_N;
constexpr size_t kCells = (size_t)kMaxN * kMaxN * kMaxN;
constexpr size_t kDescBytes = 256;  // one BoxDesc, padded to keep the arrays aligned
constexpr size_t kScratchBytes = kDescBytes + 2 * kCells * sizeof(double);

// [BoxDesc of the grid][r: smoother residual][d: recurrence direction]
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(sizeof(BoxDesc) <= kDescBytes, "descriptor slot too small");

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SR_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SR_OK;
}

__global__ void k_store_desc(BoxDesc b, BoxDesc* dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = b;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int sr_op_smooth_noalloc(int n, int nu, double cheb_lo, double cheb_hi,
                                    const double* f, double* u, void* stream) {
  if (n < 1 || nu < 0 || nu > 16 || !(cheb_lo > 0.0 && cheb_hi > cheb_lo)) return SR_ERR_INVALID;
  if (n > kMaxN) return SR_ERR_UNSUPPORTED_SIZE;
  if (!on_device(f) || !on_device(u)) return SR_ERR_INVALID;
  if (nu == 0) return SR_OK;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  BoxDesc* desc = reinterpret_cast<BoxDesc*>(base);
  double* r = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kDescBytes);
  double* d = r + kCells;

  // the whole n^3 grid as one box without a ghost shell
  BoxDesc b;
  std::memset(&b, 0, sizeof(b));
  for (int k = 0; k < 3; ++k) {
    b.lo[k] = 0; b.hi[k] = n;
    b.plo[k] = 0; b.phi[k] = n;
    b.rlo[k] = 0; b.rhi[k] = n / 2;
    b.glo[k] = 0; b.ghi[k] = n;
  }
  b.sy = n;
  b.sz = (long long)n * n;
  k_store_desc<<<1, 32, 0, s>>>(b, desc);
  if (cudaGetLastError() != cudaSuccess) return SR_ERR_CUDA;
  LevelView L{};
  L.zchunk = kDefaultZChunk;
  L.cpt = kDefaultCellsPerThread;
  L.boxes = desc;
  L.nbox = 1;
  L.n = n;
  L.nx = L.ny = L.nz = n;
  L.max_cells = L.max_stored = L.max_prolong = L.max_genuine = n * n * n;
  L.max_restrict = (n / 2) * (n / 2) * (n / 2);
  L.max_ex = L.max_ey = L.max_ez = n;
  const FieldView fv{f, desc, 1};

  // Chebyshev iteration on D^-1 A over [cheb_lo, cheb_hi] * lambda_max, the
  // coefficients of the allocating path; every scratch cell is written
  // before it is read, so nothing has to be cleared between calls
  const Cheb c = chebyshev(nu, cheb_lo, cheb_hi, kLambdaMax7);
  if (nu == 2) {
    if (launch_cheb_residual(L, u, r, fv, s) != cudaSuccess) return SR_ERR_CUDA;
    if (launch_cheb2_update(L, u, r, c.a, c.b, s) != cudaSuccess) return SR_ERR_CUDA;
    return SR_OK;
  }
  for (int m = 0; m < nu; ++m) {
    const int write_d = (nu > 1 && m < nu - 1) ? 1 : 0;
    if (launch_cheb_residual(L, u, r, fv, s) != cudaSuccess) return SR_ERR_CUDA;
    if (launch_cheb_step(L, u, d, r, c.alpha[m], c.beta[m], write_d, s) != cudaSuccess)
      return SR_ERR_CUDA;
  }
  return SR_OK;
}
