// Allocation-free Hartree energy: E = 1/2 h^3 sum_r rho(r) V(r) for callers
// that cannot allocate device memory.
//
// The grid reduction needs scratch (one partial sum per CTA and an arrival
// counter). Here that scratch is a file-scope static device array, so the
// entry point calls no cudaMalloc, cudaFree or any allocating routine; every
// GPU that loads the library holds the array until the process exits.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "reduce.cuh"

namespace ps {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 32;                                        // points per thread
constexpr long long kNaPerBlock = (long long)kNaThreads * kNaItems; // 8192 points per CTA
constexpr int kNaMaxBlocks = 65536;                                 // partial-sum slots
constexpr long long kNaMaxPoints = kNaPerBlock * kNaMaxBlocks;      // 536,870,912 points
constexpr int kNaMaxDevices = 64;

// kNaMaxBlocks partial sums, then one slot whose first 4 bytes are the arrival
// counter (512 KiB + 256 B in all).
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxBlocks + 32];

std::mutex g_setup_mu;
double* g_scratch_ptr[kNaMaxDevices] = {};

// Device address of the static array on the current device, looked up once
// per device. In host code the array's name is only a host-side stand-in.
cudaError_t scratch_on_device(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <typename T>
__global__ void __launch_bounds__(kNaThreads)
    energy_noalloc_kernel(const T* __restrict__ rho, const T* __restrict__ V, long long n, double scale,
                          double* scratch, double* E) {
  const long long base = (long long)blockIdx.x * kNaPerBlock + threadIdx.x;
  double acc = 0.0;
#pragma unroll 4
  for (int i = 0; i < kNaItems; ++i) {
    const long long idx = base + (long long)i * kNaThreads;
    if (idx < n) acc += (double)rho[idx] * (double)V[idx];
  }
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNaMaxBlocks);
  energy_finish(acc, scratch, counter, scale, E);
}

}  // namespace
}  // namespace ps

extern "C" int ps_hartree_energy_noalloc(int dtype, long long npoints, double h, const void* rho,
                                         const void* V, double* ehartree_dev, void* stream) {
  using namespace ps;
  set_error("%s", "");
  if (dtype != PS_F32 && dtype != PS_F64) {
    set_error("bad dtype %d", dtype);
    return PS_ERR_ARG;
  }
  if (npoints < 1) {
    set_error("npoints = %lld must be >= 1", npoints);
    return PS_ERR_ARG;
  }
  if (npoints > kNaMaxPoints) {
    set_error("npoints = %lld exceeds the %lld points the static scratch of "
              "ps_hartree_energy_noalloc can reduce", npoints, kNaMaxPoints);
    return PS_ERR_UNSUPPORTED;
  }
  if (!(h > 0.0) || !std::isfinite(h)) {
    set_error("h must be finite and > 0");
    return PS_ERR_ARG;
  }
  if (!rho || !V || !ehartree_dev) {
    set_error("rho, V and ehartree_dev must not be NULL");
    return PS_ERR_ARG;
  }
  const size_t esz = dtype == PS_F32 ? 4 : 8;
  if ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(V)) % esz ||
      reinterpret_cast<uintptr_t>(ehartree_dev) % 8) {
    set_error("pointers must be aligned to their element size");
    return PS_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("cudaGetDevice: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNaMaxDevices) {
    set_error("device %d: ps_hartree_energy_noalloc keeps the scratch address of devices 0 .. %d only", dev,
              kNaMaxDevices - 1);
    return PS_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  if ((e = scratch_on_device(dev, &scratch)) != cudaSuccess) {
    set_error("cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the arrival counter must start at zero (the last CTA also resets it)
  if ((e = cudaMemsetAsync(scratch + kNaMaxBlocks, 0, sizeof(unsigned), s)) != cudaSuccess) {
    set_error("clearing the counter: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  const int blocks = (int)((npoints + kNaPerBlock - 1) / kNaPerBlock);
  const double scale = 0.5 * h * h * h;
  if (dtype == PS_F32)
    energy_noalloc_kernel<float><<<blocks, kNaThreads, 0, s>>>(
        static_cast<const float*>(rho), static_cast<const float*>(V), npoints, scale, scratch, ehartree_dev);
  else
    energy_noalloc_kernel<double><<<blocks, kNaThreads, 0, s>>>(
        static_cast<const double*>(rho), static_cast<const double*>(V), npoints, scale, scratch, ehartree_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    set_error("launch: %s", cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  return PS_OK;
}
