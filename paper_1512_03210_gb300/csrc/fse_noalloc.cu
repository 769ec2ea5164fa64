// fse_noalloc.cu -- float64 mass of a wave function without any device allocation.
//
// Who needs this: code that has to read the mass of a field but holds no
// device allocator of its own -- for instance a monitoring or checkpoint hook
// that runs between steps inside a framework whose caching allocator already
// owns the device memory. There, a cudaMalloc for scratch either fails
// (memory fully reserved by that allocator) or implicitly synchronises the
// device and stalls the framework's streams; and the hook has no plan, so it
// has no workspace to borrow either.
//
// The per-block partial sums therefore live in a file-scope __device__ array
// of fixed size, reserved when the library is loaded and held on every GPU
// that loads it until the process exits. Host code must not pass the array's
// name to a kernel (in host code it is only a stand-in for the symbol): the
// device address is looked up once per device with cudaGetSymbolAddress, on
// the first call made on that device, and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "fse.h"
#include "fse_passes.cuh"

namespace {

constexpr int kMaxBlocks = 4096;              // partials held in the static array (32 KB)
constexpr long long kChunk = 65536;           // points summed by one block
static_assert(FSE_NOALLOC_MAX_POINTS == (long long)kMaxBlocks * kChunk, "header limit");

static __device__ __align__(256) double g_mass_partials[kMaxBlocks];

template <typename C>
__global__ void __launch_bounds__(256) k_mass_chunks(const C* __restrict__ psi, long long n, double* part) {
  __shared__ double red[32];
  const long long base = (long long)blockIdx.x * kChunk;
  const long long end = base + kChunk < n ? base + kChunk : n;
  double acc = 0.0;
  for (long long i = base + threadIdx.x; i < end; i += blockDim.x) {
    const C u = psi[i];
    acc += (double)u.x * u.x + (double)u.y * u.y;
  }
  acc = fse::block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;  // every partial read below is written here
}

__global__ void __launch_bounds__(256) k_mass_total(const double* part, int count, double cell, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  acc = fse::block_sum(acc, red);
  if (threadIdx.x == 0) *out = cell * acc;
}

std::mutex g_mu;
double* g_dev_ptr[64] = {nullptr};

}  // namespace

extern "C" fse_status fse_mass_noalloc(const void* psi, int prec, long long npoints, double cell_volume,
                                       double* mass_out, void* cuda_stream) {
  if (!psi || !mass_out || npoints < 0) return FSE_ERR_INVALID;
  if (prec != FSE_F32 && prec != FSE_F64) return FSE_ERR_INVALID;
  const size_t csize = prec == FSE_F32 ? 8 : 16;
  if (reinterpret_cast<uintptr_t>(psi) % csize != 0 || reinterpret_cast<uintptr_t>(mass_out) % 8 != 0)
    return FSE_ERR_INVALID;
  if (npoints > FSE_NOALLOC_MAX_POINTS) return FSE_ERR_UNSUPPORTED;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FSE_ERR_CUDA;
  if (dev < 0 || dev >= 64) return FSE_ERR_UNSUPPORTED;
  double* part = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
      // once per device, with that device current
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || !p) return FSE_ERR_CUDA;
      g_dev_ptr[dev] = static_cast<double*>(p);
    }
    part = g_dev_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int blocks = npoints == 0 ? 1 : (int)((npoints + kChunk - 1) / kChunk);
  if (prec == FSE_F32)
    k_mass_chunks<float2><<<blocks, 256, 0, st>>>(static_cast<const float2*>(psi), npoints, part);
  else
    k_mass_chunks<double2><<<blocks, 256, 0, st>>>(static_cast<const double2*>(psi), npoints, part);
  if (cudaGetLastError() != cudaSuccess) return FSE_ERR_CUDA;
  k_mass_total<<<1, 256, 0, st>>>(part, blocks, cell_volume, mass_out);
  if (cudaGetLastError() != cudaSuccess) return FSE_ERR_CUDA;
  return FSE_OK;
}
